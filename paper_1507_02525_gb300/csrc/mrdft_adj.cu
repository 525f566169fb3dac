// Adjoint MrDFT kernels (sm_103a): x_bar = sum_i (I (x) E_{2^i})^H g_i, the
// conjugate transpose of Eq. 1, taken as the transpose of the level recursion
// of Sec. 3 (Eq. 4) run from the top level down.  For a window at level i with
// accumulated gradient G_i (upstream g_i plus what its parent passed down):
//   even bins: both children receive G_i[2k] at their bin k         (U^T)
//   odd bins : zb = IDFT_h(G_i[2k+1]) (unnormalised), then
//              a_bar[n] += conj(w_{2^i}^n) zb[n], b_bar[n] -= the same (V^T D^H)
//   level 1  : x_bar[2w] += G[0] + G[1], x_bar[2w+1] += G[0] - G[1]   (A^(1)T)
// The inverse DFTs use the forward engine on conjugated data.
//
//   k_adj_window / k_adj_rows + k_adj_cols : levels above the tile, top down;
//     even-bin propagation to the next level in `e_out` (N/2 per signal),
//     time-domain contributions accumulated in `acc` (N per signal);
//     k_adj_cols2 does the cols passes of two consecutive levels at once.
//   k_adj_tile : levels tlog..1 of a tile, adds `acc`, writes x_bar.
// Every gradient-reading kernel has a FUSED variant (mrdft_loss_grad): gy then
// holds Y, the upstream gradient of level i is 2^(1-i) (Y - T) computed on the
// fly, and the block's share of sum_i 2^-i |Y - T|^2 goes to one atomic add.
#include <cuda_runtime.h>

#include "mrdft_fft.cuh"
#include "mrdft_internal.h"

namespace mrdft {

__device__ __forceinline__ float4 ld4s_a(const float2* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4s_a(float2* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float2 conjf2(float2 v) { return make_float2(v.x, -v.y); }

// ===================================================================== tile

struct AdjTileSig {
  int64_t x_base;    // gx / acc offset of the tile's first sample
  int64_t g_base;    // gy offset of the tile's first level-1 bin
  int32_t m;
  int32_t pad;
};
constexpr int kAdjMaxPack = kTile / 32;

// Upstream gradient of a bin pair at p (a float4 inside gy) of level i: g
// itself, or for the fused loss 2^(1-i) (Y - T), with 2^-i |Y - T|^2 added to
// the thread's partial loss.
template <bool FUSED>
__device__ __forceinline__ float4 grad4(const AdjArgs& a, const float4* p, int i, float& lsum) {
  float4 v = __ldcs(p);
  if constexpr (FUSED) {
    const float4 t = __ldcs(reinterpret_cast<const float4*>(a.t) + (p - reinterpret_cast<const float4*>(a.gy)));
    const float sc = ldexpf(1.f, -i);
    const float dx = v.x - t.x, dy = v.y - t.y, dz = v.z - t.z, dw = v.w - t.w;
    lsum = fmaf(sc, dx * dx + dy * dy + dz * dz + dw * dw, lsum);
    const float g = 2.f * sc;
    v = make_float4(g * dx, g * dy, g * dz, g * dw);
  }
  return v;
}
// Adds the block's partial losses to *loss (one atomic per block); every
// thread of the block must call it.
template <bool FUSED>
__device__ __forceinline__ void loss_flush(const AdjArgs& a, float lsum) {
  if constexpr (!FUSED) return;
  if (a.loss == nullptr) return;
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(a.loss, (double)s);
  }
}

// Levels 4..1 of one 16-position chunk (a level-4 window) in registers.
// P = the level-5 parent's even bins for this window, acc = x_bar so far.
template <bool FUSED>
__device__ __forceinline__ void adj_chunk_levels_4_1(const AdjArgs& a, const AdjTileSig& ts, int off,
                                                     float2 (&P)[16], float2 (&acc)[16], float& lsum) {
  const float2* gl = a.gy + ts.g_base + off;
  const int64_t lstride = (int64_t)1 << ts.m;
  static_for<0, 4>([&](auto JJ) MRDFT_INL {
    constexpr int j = 4 - decltype(JJ)::value;  // 4, 3, 2, 1
    constexpr int L = 1 << j, h = L / 2;
    float2 G[16], Pn[8];
    const float4* g4 = reinterpret_cast<const float4*>(gl + (j - 1) * lstride);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 v = grad4<FUSED>(a, g4 + q, j, lsum);
      G[2 * q] = make_float2(v.x, v.y);
      G[2 * q + 1] = make_float2(v.z, v.w);
    }
    static_for<0, 16 / L>([&](auto W) MRDFT_INL {
      constexpr int w = decltype(W)::value;
      // accumulated gradient: upstream plus the parent's even bins (both
      // children of a parent receive the same values)
      static_for<0, L>([&](auto K) MRDFT_INL {
        constexpr int k = decltype(K)::value;
        constexpr int pk = (j == 4) ? k : ((w >> 1) * L + k);
        G[w * L + k] = cadd(G[w * L + k], P[pk]);
      });
      static_for<0, h>([&](auto K) MRDFT_INL {
        constexpr int k = decltype(K)::value;
        Pn[w * h + k] = G[w * L + 2 * k];  // U^T
      });
      if constexpr (j == 1) {
        acc[2 * w] = cadd(acc[2 * w], cadd(G[2 * w], G[2 * w + 1]));
        acc[2 * w + 1] = cadd(acc[2 * w + 1], csub(G[2 * w], G[2 * w + 1]));
      } else {
        float2 zb[h];
        static_for<0, h>([&](auto K) MRDFT_INL {
          constexpr int k = decltype(K)::value;
          zb[k] = G[w * L + 2 * k + 1];
        });
        idft_reg<h>(zb);
        static_for<0, h>([&](auto N) MRDFT_INL {
          constexpr int n = decltype(N)::value;
          const float2 c = cmul_ct<L, (L - n) % L>(zb[n]);  // conj(w_L^n) zb[n]
          acc[w * L + n] = cadd(acc[w * L + n], c);
          acc[w * L + h + n] = csub(acc[w * L + h + n], c);
        });
      }
    });
#pragma unroll
    for (int q = 0; q < 8; ++q) P[q] = Pn[q];
  });
}

template <int TLOG, int NT, bool FUSED>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1) k_adj_tile(const AdjArgs a) {
  constexpr int T = 1 << TLOG;
  static_assert(T == 16 * NT, "tile = 16 samples per thread");
  extern __shared__ __align__(1024) float2 sm[];
  constexpr int TA = pad16_size(T);
  float2* ACC = sm;                          // x_bar accumulator (pad16)
  float2* E[2] = {sm + TA, sm + TA + T / 2}; // even-bin propagation, level i in E[i & 1]
  float2* Z = sm + TA + T;                   // T/2 (staging, then zlay), odd-bin inverse DFT work
  float2* TQ = Z + T / 2;                  // quarter-wave w_{2^TLOG} (padded)
  AdjTileSig* TS = reinterpret_cast<AdjTileSig*>(TQ + twq_size(TLOG));
  const int tid = threadIdx.x;
  const int item = blockIdx.x;
  if (item >= a.nitems) return;
  const TileItem it = reinterpret_cast<const TileItem*>(a.items)[item];
  if (!tile_item_head_ok(it, a.nids, TLOG)) {
    if (tid == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const int tl = it.tlog;
  const int Tn = it.nsig << tl;
  const int tn_log = 31 - __clz(Tn);
  __shared__ int bad;
  if (tid == 0) bad = 0;
  __syncthreads();
  if (tid < it.nsig) {
    SigDesc sd;
    if (tile_sig_ok(a.sigs, a.nsigs, a.sig_ids[it.sig_list + tid], it, sd)) {
      const int64_t t0 = (int64_t)it.tile << tl;
      TS[tid] = AdjTileSig{sd.in_off + t0, sd.out_off + t0, sd.m, 0};
    } else {
      bad = 1;
    }
  }
  load_twq<NT>(TQ, TLOG, a.tw);
  __syncthreads();
  if (bad) {
    if (tid == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  // For a tile of a longer signal (one signal, m > tl) the large levels left
  // contributions in acc and the level-(tl+1) even-bin propagation in e_in.
  const SigDesc sd0 = a.sigs[a.sig_ids[it.sig_list]];
  const bool below = sd0.m > tl;
#pragma unroll 4
  for (int c = tid; c < (Tn >> 1); c += NT) {
    const int e = c << 1;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (below) v = __ldcg(reinterpret_cast<const float4*>(a.acc + 2 * sd0.aux_off + ((int64_t)it.tile << tl) + e));
    st4s_a(ACC + pad16(e), v);
  }

  // ---- levels tl .. 5 through shared memory
  const TwQ tw{TQ, TLOG};
  // the gradient pairs of one level, requested a level ahead: a level's
  // requests are issued before the previous level's FFT and arrive during it
  constexpr int ITER = T / 2 / NT;
  float4 gv[ITER];
  float lsum = 0.f;  // fused loss: this thread's share
  auto load_level = [&](int lv) MRDFT_INL {
#pragma unroll
    for (int q = 0; q < ITER; ++q) {
      const int c = tid + q * NT;
      if (c < (Tn >> 1)) {
        const int e = c << 1;
        const AdjTileSig& ts = TS[e >> tl];
        gv[q] = grad4<FUSED>(a, reinterpret_cast<const float4*>(a.gy + ts.g_base + ((int64_t)(lv - 1) << ts.m) + (e & ((1 << tl) - 1))),
                      lv, lsum);
      }
    }
  };
  load_level(tl);
  // one specialised FFT per level (compile-time lengths), top level first
  static_for<0, TLOG - 4>([&](auto J) MRDFT_INL {
    constexpr int i = TLOG - decltype(J)::value;
    if (i > tl) return;
    constexpr int L = 1 << i, h = L >> 1;
    constexpr int SA = i <= 10 ? 3 : 6;  // staging layout of the odd half
    const float2* Ein = E[(i + 1) & 1];
    float2* Eout = E[i & 1];
    // G_i = g_i + P_i: even half -> Eout, conj(odd half) -> Z.  Pair c (bins
    // e = 2c, e + 1) of window w = e >> i, bin k = e mod 2^i has its half-bin
    // index w h + k / 2 = c, and its parent's even bins at pb(e) = e with bit
    // i deleted; both maps and both layouts are linear over XOR and
    // c = tid + q NT splits into disjoint bit fields, so each index is a
    // per-thread base XOR a constant per q
    auto pbf = [&](int e) MRDFT_INL { return ((e >> (i + 1)) << i) | (e & (L - 1)); };
    const int eb0 = swzf(pbf(tid << 1)), eo0 = swzf(tid), z0 = stg<SA, 0>(tid);
#pragma unroll
    for (int q = 0; q < ITER; ++q) {
      const int c = tid + q * NT;
      if (c >= (Tn >> 1)) continue;
      const int e = c << 1;
      const float4 g = gv[q];
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i == tl) {
        if (below)
          p = __ldcg(reinterpret_cast<const float4*>(a.e_in + sd0.aux_off + ((int64_t)(it.tile >> 1) << tl) +
                                                     (e & (L - 1))));
      } else {
        const int ib = eb0 ^ swzf(pbf((q * NT) << 1));  // pb is even: its pair partner is ib ^ 1
        const float2 pe = Ein[ib], po = Ein[ib ^ 1];
        p = make_float4(pe.x, pe.y, po.x, po.y);
      }
      Eout[eo0 ^ swzf(q * NT)] = make_float2(g.x + p.x, g.y + p.y);
      Z[z0 ^ stg<SA, 0>(q * NT)] = make_float2(g.z + p.z, -(g.w + p.w));
    }
    __syncthreads();
    if constexpr (i > 5) load_level(i - 1);
    const StgGroup<SA, 0> src{Z, 0, i - 1};
    auto sink = [&](int, int b, int n, float2 v) MRDFT_INL {
      const float2 c = cmulc(conjf2(v), twq_l(tw, i, n));  // conj(w^n) zb[n]
      const int base = b << i;
      const int i0 = pad16(base + n), i1 = h >= 32 ? i0 + pad16(h) : pad16(base + h + n);
      ACC[i0] = cadd(ACC[i0], c);
      ACC[i1] = csub(ACC[i1], c);
    };
    cg_fft<i - 1, i - 1, NT, 8, false, kPreNone, 0, true>(Z, i - 1, tn_log - i, tw, src, NoPre{}, sink);
    __syncthreads();
  });

  // ---- levels 4 .. 1 in registers, one 16-position chunk per thread
  const int chunk = tid;
  const int e = chunk << 4;
  if (e < Tn) {
    float2 P[16], acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      acc[q] = ACC[pad16(e + q)];
      P[q] = E[1][swzf(((chunk >> 1) << 4) + q)];  // E_5 of the level-5 parent
    }
    const AdjTileSig& ts = TS[e >> tl];
    const int off = e & ((1 << tl) - 1);
    adj_chunk_levels_4_1<FUSED>(a, ts, off, P, acc, lsum);
    if (it.nsig == 1 && Tn == T) {
      // a whole single-signal tile: each warp stores its 32 rows of x_bar
      // through its own rows of ACC (read above by these lanes only)
      float2* base = a.gx + ts.x_base + ((chunk & ~31) << 4);
      warp_rows16_store(acc, ACC + pad16((tid >> 5) << 9), [&](int r) MRDFT_INL { return base + (r << 4); });
    } else {
      float4* dst = reinterpret_cast<float4*>(a.gx + ts.x_base + off);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        __stcs(dst + q, make_float4(acc[2 * q].x, acc[2 * q].y, acc[2 * q + 1].x, acc[2 * q + 1].y));
    }
  }
  loss_flush<FUSED>(a, lsum);
}

// ============================================================ lone signal

// The adjoint of the forward's lone-signal path: one signal of 2^5..2^12
// samples alone in its plan, one CTA per level.  Level i's share of x_bar is
// the conjugate transpose of its per-window DFTs, an unnormalised inverse DFT
// of length 2^i of every window's upstream gradient (computed as the
// conjugate of the DFT of the conjugate), independent of the other levels;
// each CTA writes its share to the scratch and the CTA that finishes last
// adds the m shares in level order (the same sum on every call).
constexpr int kLevelsThreads = 512;
constexpr size_t adj_levels_smem() { return (size_t)(2 * kTile + twq_size(kTileLog)) * sizeof(float2); }
template <int NT>
__global__ void __launch_bounds__(NT, 1) k_adj_levels(const AdjArgs a) {
  constexpr int T = kTile;
  extern __shared__ __align__(1024) float2 sm[];
  float2* G = sm;           // conj of the level's upstream gradient (swz128)
  float2* Z = sm + T;       // FFT work area
  float2* TQ = sm + 2 * T;  // quarter-wave w_{2^12}
  const int tid = threadIdx.x;
  const int id = a.nids > 0 ? a.sig_ids[0] : -1;
  if (id < 0 || id >= a.nsigs || a.sigs[id].m < 5 || a.sigs[id].m > kTileLog || (int)gridDim.x != a.sigs[id].m) {
    if (tid == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const SigDesc sd = a.sigs[id];
  const int m = sd.m, N = 1 << m;
  const int i = (int)blockIdx.x + 1;
  float2* C = a.scratch + (int64_t)(i - 1) * N;  // this level's share of x_bar
  const float4* gl = reinterpret_cast<const float4*>(a.gy + sd.out_off + ((int64_t)(i - 1) << m));
#pragma unroll 4
  for (int c = tid; c < (N >> 1); c += NT) {
    const float4 g = __ldcs(gl + c);
    st4s_a(G + swz128(2 * c), make_float4(g.x, -g.y, g.z, -g.w));
  }
  load_twq<NT>(TQ, kTileLog, a.tw);
  __syncthreads();
  if (i == 1) {  // H_2 is its own conjugate transpose
    for (int c = tid; c < (N >> 1); c += NT) {
      const float2 g0 = conjf2(G[swz128(2 * c)]), g1 = conjf2(G[swz128(2 * c + 1)]);
      const float2 s0 = cadd(g0, g1), s1 = csub(g0, g1);
      *reinterpret_cast<float4*>(C + 2 * c) = make_float4(s0.x, s0.y, s1.x, s1.y);
    }
  } else {
    const TwQ tw{TQ, kTileLog};
    auto src = [&](int w, int k) MRDFT_INL -> float2 { return G[swz128((w << i) + k)]; };
    auto sink = [&](int, int w, int n, float2 v) MRDFT_INL { C[(w << i) + n] = conjf2(v); };
    cg_fft<1, kTileLog, NT, T / NT, false, kPreNone>(Z, i, m - i, tw, src, NoPre{}, sink);
  }
  // the last CTA to finish adds the shares, level by level
  __threadfence();
  __syncthreads();
  __shared__ int last;
  if (tid == 0) last = atomicAdd(a.ticket, 1) == m - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  float4* gx = reinterpret_cast<float4*>(a.gx + sd.in_off);
  for (int c = tid; c < (N >> 1); c += NT) {
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int l = 0; l < m; ++l) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(a.scratch + (int64_t)l * N) + c);
      s = make_float4(s.x + v.x, s.y + v.y, s.z + v.z, s.w + v.w);
    }
    __stcs(gx + c, s);
  }
  if (tid == 0) *a.ticket = 0;  // ready for the next launch
}

// ===================================================================== tiny

// Signals with N <= 16: conjugate transpose of Eq. 1 term by term.
template <bool FUSED>
__global__ void k_adj_tiny(const AdjArgs a) {
  const int id = (int)blockIdx.x < a.nids ? a.sig_ids[blockIdx.x] : -1;
  if (id < 0 || id >= a.nsigs || a.sigs[id].m < 1 || a.sigs[id].m > 4) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const SigDesc sd = a.sigs[id];
  const int N = 1 << sd.m;
  const int n = threadIdx.x;
  float lsum = 0.f;
  if (n < N) {
    float2 acc = make_float2(0.f, 0.f);
    for (int i = 1; i <= sd.m; ++i) {
      const int L = 1 << i, w = n >> i, nl = n & (L - 1);
      const float sc = ldexpf(1.f, -i);
      for (int k = 0; k < L; ++k) {
        const int64_t idx = sd.out_off + ((int64_t)(i - 1) << sd.m) + (w << i) + k;
        float2 g = a.gy[idx];
        if constexpr (FUSED) {  // fused loss: 2^(1-i) (Y - T); bin n's term counted by thread n
          const float2 d = csub(g, a.t[idx]);
          if (k == nl) lsum = fmaf(sc, d.x * d.x + d.y * d.y, lsum);
          g = make_float2(2.f * sc * d.x, 2.f * sc * d.y);
        }
        acc = cadd(acc, cmulc(g, tw_small(a.tw, i, (nl * k) & (L - 1))));
      }
    }
    a.gx[sd.in_off + n] = acc;
  }
  loss_flush<FUSED>(a, lsum);
}

// =================================================================== window

// Accumulated gradient of a bin pair (2k, 2k+1) of window w at level i:
// upstream g plus the parent's propagated even bins (none at the top level).
template <bool FUSED>
__device__ __forceinline__ float4 adj_G(const AdjArgs& a, const SigDesc& sd, int i, int64_t w, int64_t k2, float& lsum) {
  float4 g = grad4<FUSED>(a, reinterpret_cast<const float4*>(a.gy + sd.out_off + ((int64_t)(i - 1) << sd.m) + (w << i) + k2), i, lsum);
  if (sd.m > i) {
    const float4 p = __ldcg(reinterpret_cast<const float4*>(a.e_in + sd.aux_off + ((w >> 1) << i) + k2));
    g.x += p.x; g.y += p.y; g.z += p.z; g.w += p.w;
  }
  return g;
}

// One window of level i = LB + 1 per CTA: G = g + propagated even bins; even
// half -> e_out; IDFT_h of the odd half; conj(w_{2^i}^n) times it added to
// the accumulator at n and subtracted at h + n (accumulator read per group).
template <int LB, bool FUSED>
__global__ void __launch_bounds__(kWinThreads, 2) k_adj_window(const AdjArgs a) {
  constexpr int NT = kWinThreads;
  constexpr int h = 1 << LB;
  constexpr int i = LB + 1;
  constexpr int PTS = h / NT;
  constexpr int SA = LB == 12 ? 6 : 3, SB = LB == 12 ? 0 : 9;  // staging layout
  extern __shared__ __align__(1024) float2 sm[];
  float2* Z = sm;                               // staging layout, then zlay
  float2* TQ = sm + (1 << kWinMaxLog);          // quarter-wave w_{2^13}
  if ((int)blockIdx.x >= a.nitems) return;
  const LevelItem it = reinterpret_cast<const LevelItem*>(a.items)[blockIdx.x];
  SigDesc sd;
  if (!level_item_ok(a.sigs, a.nsigs, it, i, 1, sd)) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const int64_t w = it.window;
  const bool add = sd.m > i;
  float2* acc = a.acc + 2 * sd.aux_off + (w << i);
  load_twq<NT>(TQ, 13, a.tw);
  const float2 w1 = __ldg(&a.tw.tw13[1]);  // w_{2^14}
  float lsum = 0.f;  // fused loss: this thread's share
#pragma unroll 1
  for (int t0 = 0; t0 < PTS; t0 += 8) {
    float4 g[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) g[t] = adj_G<FUSED>(a, sd, i, w, 2 * (int64_t)(threadIdx.x + (t0 + t) * NT), lsum);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int k = threadIdx.x + (t0 + t) * NT;
      __stcg(a.e_out + sd.aux_off + (w << LB) + k, make_float2(g[t].x, g[t].y));
      Z[stg<SA, SB>(k)] = make_float2(g[t].z, -g[t].w);
    }
  }
  __syncthreads();
  const TwQ tw{TQ, 13};
  const StgGroup<SA, SB> src{Z, 0, 0};
  float2 oa[PTS], ob[PTS];
  auto pre = [&](int slot, int, int n) MRDFT_INL {
    if (add) {
      oa[slot] = __ldcg(acc + n);
      ob[slot] = __ldcg(acc + h + n);
    }
  };
  auto sink = [&](int slot, int, int n, float2 v) MRDFT_INL {
    float2 t;
    if constexpr (i <= 13) {
      t = twq_l(tw, i, n);
    } else {
      t = twq(tw, n >> 1);
      if (n & 1) t = cmul(t, w1);
    }
    const float2 c = cmulc(conjf2(v), t);  // conj(w^n) zb[n]
    if (add) {
      __stcg(acc + n, cadd(oa[slot], c));
      __stcg(acc + h + n, csub(ob[slot], c));
    } else {
      __stcg(acc + n, c);
      __stcg(acc + h + n, make_float2(-c.x, -c.y));
    }
  };
  cg_fft<LB, LB, NT, PTS, false, kPreGroup, 0, true>(Z, LB, 0, tw, src, pre, sink);
  loss_flush<FUSED>(a, lsum);
}

constexpr size_t adj_cols_smem(int E) {
  return (size_t)((1 << E) + twq_size(12) + (1 << (E - 3))) * sizeof(float2);
}
template <int QB>
constexpr int adj_cols_e() { return kPassElemsLog; }
constexpr size_t adj_rows_smem(int E, int CB) {
  return (size_t)((1 << E) + twq_size(CB) + (1 << (E - CB)) * 65 + (1 << (E - 6)) + 16) * sizeof(float2);
}
template <int CB>
constexpr int adj_rows_e() { return rows_elems_log_c(CB, true); }
// threads of a rows CTA of 2^E points
constexpr int adj_rows_nt(int E, int CB) {
  return E < kPassElemsLog ? kColsThreads : (E == kPassElemsLog ? (CB <= 10 ? kColsThreads : kPassThreads) : kPassThreadsWide);
}

// =============================================================== two-pass

// Adjoint of the forward two-pass level (h = Q * C).
// rows: a CTA of 2^E points covers residues k2 in [k0, k0 + KC), KC = 2^E / C:
//   odd-bin gradients at k = Q k1 + k2 -> IDFT_C over k1 -> times
//   conj(w_h^(r k2)) -> scratch U[window][k2][r]; even bins -> e_out.
template <int E, int NT, int CB, bool FUSED>
__global__ void __launch_bounds__(NT, E <= kPassElemsLog ? 2 : 1) k_adj_rows(const AdjArgs a) {
  constexpr int PTS = (1 << E) / NT;
  constexpr int KCB = E - CB, KC = 1 << KCB;
  constexpr int HU = (1 << CB) >> 6;
  constexpr int SH = E - kPassElemsLog;    // CTAs per item: 2^-SH (SH < 0), items per CTA: 2^SH
  // staging layout
  constexpr int SA = (CB <= 10 && KCB == 2) ? 5 : ((CB <= 12 && KCB != 4) ? 6 : 3), SB = (CB <= 10 && KCB == 2) ? 8 : 9;
  extern __shared__ __align__(1024) float2 sm[];
  float2* S = sm;                          // sequence j at j C (staging, then zlay)
  float2* TQ = sm + (1 << E);              // quarter-wave w_C
  float2* TWL = TQ + twq_size(CB);         // [KC][64] (row stride 65): w_h^(k2 t)
  float2* TWH = TWL + KC * 65;             // [KC][C/64] (row stride C/64 + 16/KC): w_h^(k2 64 u)
  int item, blk;
  if constexpr (SH >= 0) {
    item = (int)blockIdx.x << SH;
  } else {
    item = (int)blockIdx.x >> -SH;
  }
  if (item >= a.nitems) return;
  const LevelItem it = reinterpret_cast<const LevelItem*>(a.items)[item];
  if constexpr (SH >= 0) {
    blk = it.block >> SH;
  } else {
    blk = (it.block << -SH) | ((int)blockIdx.x & ((1 << -SH) - 1));
  }
  const int i = a.level;
  const int HB = i - 1, QB = HB - CB;
  SigDesc sd;
  if (!level_item_ok(a.sigs, a.nsigs, it, i, pass_items(i), sd)) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const int64_t w = it.window;
  const int k0 = blk << KCB;
  // gradient pairs (2k, 2k+1): a batch of loads is issued before any store;
  // the twiddle tables are built while the first batch is in flight
  float lsum = 0.f;  // fused loss: this thread's share
  auto load_batch = [&](int t0, float4 (&g)[8]) MRDFT_INL {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = threadIdx.x + (t0 + t) * NT;
      const int64_t k = ((int64_t)(e >> KCB) << QB) + k0 + (e & (KC - 1));
      g[t] = adj_G<FUSED>(a, sd, i, w, 2 * k, lsum);
    }
  };
  auto store_batch = [&](int t0, const float4 (&g)[8]) MRDFT_INL {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = threadIdx.x + (t0 + t) * NT;
      const int j = e & (KC - 1), k1 = e >> KCB;
      const int64_t k = ((int64_t)k1 << QB) + k0 + j;
      __stcg(a.e_out + sd.aux_off + (w << HB) + k, make_float2(g[t].x, g[t].y));
      S[stg<SA, SB>((j << CB) + k1)] = make_float2(g[t].z, -g[t].w);
    }
  };
  {
    float4 g[8];
    load_batch(0, g);
    load_twq<NT>(TQ, CB, a.tw);
    for (int t = threadIdx.x; t < KC * (64 + HU); t += NT) {
      if (t < KC * 64) {
        const int j = t >> 6, u = t & 63;
        TWL[j * 65 + u] = tw_any(a.tw, HB, (int64_t)(k0 + j) * u);
      } else {
        const int t2 = t - KC * 64, j = t2 / HU, u = t2 % HU;
        TWH[j * (HU + 16 / KC) + u] = tw_any(a.tw, HB, (int64_t)(k0 + j) * 64 * u);
      }
    }
    store_batch(0, g);
#pragma unroll 1
    for (int t0 = 8; t0 < PTS; t0 += 8) {
      load_batch(t0, g);
      store_batch(t0, g);
    }
  }
  __syncthreads();
  const TwQ tw{TQ, CB};
  float2* U = a.scratch + sd.aux_off + (w << HB);
  const StgGroup<SA, SB> src{S, 0, CB};
  // the intermediate is read by the cols pass right after: keep it in L2
  const uint64_t keep = l2_evict_last_policy();
  auto sink = [&](int, int b, int r, float2 v) MRDFT_INL {
    const float2 t = cmul(TWL[b * 65 + (r & 63)], TWH[b * (HU + 16 / KC) + (r >> 6)]);
    st_l2_keep(U + ((int64_t)(k0 + b) << CB) + r, cmulc(conjf2(v), t), keep);
  };
  cg_fft<CB, CB, NT, PTS, false, kPreNone, 0, true>(S, CB, KCB, tw, src, NoPre{}, sink);
  loss_flush<FUSED>(a, lsum);
}

// cols: item (sig, window, c) covers chunk offsets r in [r0, r0 + RC),
//   r0 = c RC, RC = 2^13 / Q: U[window][k2][r] -> IDFT_Q over k2 -> zb[r + C q]
//   -> conj(w_{2^i}^n) zb added to acc at n and subtracted at h + n.
template <int NT, int QB, int E>
__global__ void __launch_bounds__(NT, E < kPassElemsLog ? 4 : 2) k_adj_cols(const AdjArgs a) {
  constexpr int PTS = (1 << E) / NT;
  constexpr int SH = kPassElemsLog - E;      // CTAs per item: 2^SH
  constexpr int RCB = E - QB, RC = 1 << RCB;
  extern __shared__ __align__(1024) float2 sm[];
  float2* S = sm;                          // column r position k2 at k2 RC + r (staging, then zlay)
  float2* TQ = sm + (1 << E);              // quarter-wave w_{2^12}
  float2* ZC = TQ + twq_size(12);          // w_{2^i}^(r0 + r), r < RC
  const int item = (int)blockIdx.x >> SH;
  if (item >= a.nitems) return;
  const LevelItem it = reinterpret_cast<const LevelItem*>(a.items)[item];
  const int i = a.level;
  const int HB = i - 1, CB = HB - QB;
  const int64_t h = (int64_t)1 << HB;
  SigDesc sd;
  if (!level_item_ok(a.sigs, a.nsigs, it, i, pass_items(i), sd)) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const int64_t w = it.window;
  const int r0 = ((it.block << SH) | ((int)blockIdx.x & ((1 << SH) - 1))) << RCB;
  const float2* U = a.scratch + sd.aux_off + (w << HB);
  float2* acc = a.acc + 2 * sd.aux_off + (w << i);
  const bool add = sd.m > i;
  // the intermediate in batches of 8 loads; the twiddle tables are built
  // while the first batch is in flight
  auto load_u = [&](int t0, float2 (&u)[8]) MRDFT_INL {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = threadIdx.x + (t0 + t) * NT;
      u[t] = __ldcg(U + ((int64_t)(e >> RCB) << CB) + r0 + (e & (RC - 1)));
    }
  };
  auto stage_u = [&](int t0, const float2 (&u)[8]) MRDFT_INL {
#pragma unroll
    for (int t = 0; t < 8; ++t) S[stg<6, 0>(threadIdx.x + (t0 + t) * NT)] = conjf2(u[t]);  // e = k2 RC + r
  };
  {
    float2 u[8];
    load_u(0, u);
    load_twq<NT>(TQ, 12, a.tw);
    for (int r = threadIdx.x; r < RC; r += NT) ZC[r] = tw_any(a.tw, i, r0 + r);
    stage_u(0, u);
#pragma unroll 1
    for (int t0 = 8; t0 < PTS; t0 += 8) {
      load_u(t0, u);
      stage_u(t0, u);
    }
  }
  __syncthreads();
  // this block's columns of the intermediate are dead: drop them from L2
  if constexpr (RC >= 16)
    for (int l = threadIdx.x; l < (RC / 16) << QB; l += NT)
      discard_l2(U + ((int64_t)(l >> (RCB - 4)) << CB) + r0 + 16 * (l & ((RC / 16) - 1)));
  const TwQ tw{TQ, 12};
  const StgGroup<6, 0> src{S, RCB, 0};
  float2 oa[PTS], ob[PTS];
  // the accumulated gradient at n and h + n, read once per group of 8 outputs
  auto pre = [&](int slot, int b, int q) MRDFT_INL {
    if (add) {
      const int64_t n = ((int64_t)q << CB) + r0 + b;
      oa[slot] = __ldcg(acc + n);
      ob[slot] = __ldcg(acc + h + n);
    }
  };
  auto sink = [&](int slot, int b, int q, float2 v) MRDFT_INL {
    const int64_t n = ((int64_t)q << CB) + r0 + b;
    const float2 c = cmulc(conjf2(v), cmul(ZC[b], twq_l(tw, QB + 1, q)));
    if (add) {
      __stcg(acc + n, cadd(oa[slot], c));
      __stcg(acc + h + n, csub(ob[slot], c));
    } else {
      __stcg(acc + n, c);
      __stcg(acc + h + n, make_float2(-c.x, -c.y));
    }
  };
  cg_fft<QB, QB, NT, PTS, true, kPreHalf, (RCB < 4 ? RCB : 4), true>(S, QB, RCB, tw, src, pre, sink);
}

// Two levels, one update of the accumulated gradient: the cols passes of
// levels i and i + 1 (the same C, Q = 2^QB for level i and 2Q for level
// i + 1), after both rows passes.  A CTA takes chunk offsets
// [r0, r0 + RC) of one level-(i+1) window, whose column strip holds the rows
// q'' < 4Q.  With zb' = IDFT_2Q(U_{i+1}) and zb_c = IDFT_Q(U_i of child c),
// c1[q''] = conj(w_{2^(i+1)}^(r + C q'')) zb'[q''] and
// c0_c[q] = conj(w_{2^i}^(r + C q)) zb_c[q], row q + jQ (j = 0..3) of the
// window receives
//   j = 0: c1[q] + c0_0[q]        j = 1: c1[q + Q] - c0_0[q]
//   j = 2: -c1[q] + c0_1[q]       j = 3: -c1[q + Q] - c0_1[q]
// (the parent's halves a, b and each child's halves), read and written once.
template <int QB, int CB>
__global__ void __launch_bounds__(kColsThreads, 2) k_adj_cols2(const AdjArgs a) {
  constexpr int NT = kColsThreads;
  constexpr int E = kPassElemsLog;
  constexpr int Q = 1 << QB;
  constexpr int RCB = E - QB - 2, RC = 1 << RCB;
  constexpr int PTS = (1 << (E - 1)) / NT;               // FFT points per thread, each level
  constexpr int SA1 = QB == 9 ? 6 : 3;                   // staging layouts
  static_assert(RCB >= 2 && PTS == 8, "column blocks of at least 4, 8 points per thread");
  extern __shared__ __align__(1024) float2 sm[];
  float2* Z1 = sm;                                       // level i+1: k2 RC + b, then c1 at q'' RC + b
  float2* Z0 = sm + (1 << (E - 1));                      // level i: k2 2RC + c RC + b
  float2* TQ = sm + (1 << E);                            // quarter-wave w_{2^12}
  float2* ZC1 = TQ + twq_size(12);                       // w_{2^(i+1)}^(r0 + b)
  float2* ZC0 = ZC1 + RC;                                // w_{2^i}^(r0 + b)
  const int item = (int)blockIdx.x >> 1;
  if (item >= a.nitems) return;
  const LevelItem it = reinterpret_cast<const LevelItem*>(a.items)[item];
  const int i1 = a.level, i = i1 - 1;                    // the pair (i, i + 1)
  SigDesc sd;
  if (!level_item_ok(a.sigs, a.nsigs, it, i1, pass_items(i1), sd)) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const int64_t W = it.window;
  const int r0 = ((it.block << 1) | ((int)blockIdx.x & 1)) << RCB;
  const float2* U1 = a.scratch2 + sd.aux_off + (W << i);
  const float2* U0 = a.scratch + sd.aux_off + ((2 * W) << (i - 1));
  float2* acc = a.acc + 2 * sd.aux_off + (W << i1);
  const bool add = sd.m > i1;
  {
    float2 u1[PTS], u0[PTS];
#pragma unroll
    for (int t = 0; t < PTS; ++t) {
      const int e = threadIdx.x + t * NT;                // e = k2 RC + b, k2 < 2Q
      u1[t] = __ldcg(U1 + ((int64_t)(e >> RCB) << CB) + r0 + (e & (RC - 1)));
      const int s = e & (2 * RC - 1), k2 = e >> (RCB + 1);  // e = k2 2RC + s, s = c RC + b
      u0[t] = __ldcg(U0 + ((int64_t)(s >> RCB) << (i - 1)) + ((int64_t)k2 << CB) + r0 + (s & (RC - 1)));
    }
#pragma unroll
    for (int t = 0; t < PTS; ++t) {
      const int e = threadIdx.x + t * NT;
      Z1[stg<SA1, 0>(e)] = conjf2(u1[t]);
      Z0[stg<3, 0>(e)] = conjf2(u0[t]);
    }
  }
  load_twq<NT>(TQ, 12, a.tw);
  for (int b = threadIdx.x; b < RC; b += NT) {
    ZC1[b] = tw_any(a.tw, i1, r0 + b);
    ZC0[b] = tw_any(a.tw, i, r0 + b);
  }
  __syncthreads();
  // this block's columns of both intermediates are dead: drop them from L2
  if (RC >= 16) {
    constexpr int LPR = RC >= 16 ? RC / 16 : 1;          // 128-byte lines per row
    for (int l = threadIdx.x; l < 4 * Q * LPR; l += NT) {
      const int row = l / LPR, part = l % LPR;           // rows 0..2Q-1: U1; 2Q..4Q-1: U0 of child (row - 2Q) / Q
      const float2* p = row < 2 * Q ? U1 + ((int64_t)row << CB)
                                    : U0 + ((int64_t)((row - 2 * Q) >> QB) << (i - 1)) + ((int64_t)((row - 2 * Q) & (Q - 1)) << CB);
      discard_l2(p + r0 + 16 * part);
    }
  }
  const TwQ tw{TQ, 12};
  // level i + 1: zb' per column, c1 back into Z1 in natural order
  const StgGroup<SA1, 0> src1{Z1, RCB, 0};
  auto sink1 = [&](int, int b, int q, float2 v) MRDFT_INL {
    Z1[(q << RCB) + b] = cmulc(conjf2(v), cmul(ZC1[b], twq_l(tw, QB + 2, q)));
  };
  cg_fft<QB + 1, QB + 1, NT, PTS, true, kPreNone, (RCB < 4 ? RCB : 4), true>(Z1, QB + 1, RCB, tw, src1, NoPre{}, sink1);
  __syncthreads();
  // level i: zb_c per (child, column), combined with c1 into the four rows
  const StgGroup<3, 0> src0{Z0, RCB + 1, 0};
  float2 oa[PTS], ob[PTS];
  auto pre0 = [&](int slot, int s, int q) MRDFT_INL {
    if (add) {
      const int64_t n = ((int64_t)(q + ((s >> RCB) << (QB + 1))) << CB) + r0 + (s & (RC - 1));
      oa[slot] = __ldcg(acc + n);
      ob[slot] = __ldcg(acc + n + ((int64_t)Q << CB));
    }
  };
  auto sink0 = [&](int slot, int s, int q, float2 v) MRDFT_INL {
    const int c = s >> RCB, b = s & (RC - 1);
    const int64_t n = ((int64_t)(q + (c << (QB + 1))) << CB) + r0 + b;
    const float2 c0 = cmulc(conjf2(v), cmul(ZC0[b], twq_l(tw, QB + 1, q)));
    float2 ca = Z1[(q << RCB) + b], cb = Z1[((q + Q) << RCB) + b];
    if (c) {
      ca = make_float2(-ca.x, -ca.y);
      cb = make_float2(-cb.x, -cb.y);
    }
    ca = cadd(ca, c0);
    cb = csub(cb, c0);
    if (add) {
      ca = cadd(oa[slot], ca);
      cb = cadd(ob[slot], cb);
    }
    __stcg(acc + n, ca);
    __stcg(acc + n + ((int64_t)Q << CB), cb);
  };
  cg_fft<QB, QB, NT, PTS, true, kPreHalf, (RCB + 1 < 4 ? RCB + 1 : 4), true>(Z0, QB, RCB + 1, tw, src0, pre0, sink0);
}

constexpr size_t adj_cols2_smem() {
  return (size_t)((1 << kPassElemsLog) + twq_size(12) + 2 * (1 << (kPassElemsLog - 6))) * sizeof(float2);
}

// Launch-time dispatch to the instantiation of a level's FFT sizes.
template <int QB>
void adj_cols_launch(const AdjArgs& a, int grid, cudaStream_t s) {
  constexpr int E = adj_cols_e<QB>();
  constexpr int NT = E < kPassElemsLog ? kPassThreads : kColsThreads;
  k_adj_cols<NT, QB, E><<<grid << (kPassElemsLog - E), NT, adj_cols_smem(E), s>>>(a);
}
template <int E, int CB>
void adj_rows_launch_e(const AdjArgs& a, int grid, cudaStream_t s) {
  constexpr int NT = adj_rows_nt(E, CB);
  // a CTA of 2^E points takes 2^(E-13) items (E >= 13) or half an item
  int g;
  if constexpr (E >= kPassElemsLog) g = grid >> (E - kPassElemsLog);
  else g = grid << (kPassElemsLog - E);
  if (a.t)
    k_adj_rows<E, NT, CB, true><<<g, NT, adj_rows_smem(E, CB), s>>>(a);
  else
    k_adj_rows<E, NT, CB, false><<<g, NT, adj_rows_smem(E, CB), s>>>(a);
}
template <int CB>
void adj_rows_launch(const AdjArgs& a, int grid, cudaStream_t s) {
  if constexpr (CB <= 10) {
    if (a.rows13 || CB < 10) {
      adj_rows_launch_e<kPassElemsLog, CB>(a, grid, s);
      return;
    }
  }
  adj_rows_launch_e<adj_rows_e<CB>(), CB>(a, grid, s);
}
template <int QB>
cudaError_t adj_cols_attr() {
  constexpr int E = adj_cols_e<QB>();
  constexpr int NT = E < kPassElemsLog ? kPassThreads : kColsThreads;
  return cudaFuncSetAttribute(k_adj_cols<NT, QB, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)adj_cols_smem(E));
}
template <int CB, int E = adj_rows_e<CB>()>
cudaError_t adj_rows_attr() {
  constexpr int NT = adj_rows_nt(E, CB);
  cudaError_t e = cudaFuncSetAttribute(k_adj_rows<E, NT, CB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)adj_rows_smem(E, CB));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_rows<E, NT, CB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)adj_rows_smem(E, CB));
  return e;
}

// ================================================================ launchers

static constexpr size_t kAdjTileSmem =
    (size_t)(pad16_size(kTile) + kTile + kTile / 2 + twq_size(kTileLog)) * sizeof(float2) +
    kAdjMaxPack * sizeof(AdjTileSig);
static constexpr size_t kAdjWinSmem = (size_t)((1 << kWinMaxLog) + twq_size(13)) * sizeof(float2);
cudaError_t set_adj_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_adj_tile<kTileLog, kTileThreads, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjTileSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_tile<kTileLog, kTileThreads, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjTileSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_levels<kLevelsThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)adj_levels_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_window<12, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjWinSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_window<12, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjWinSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_window<13, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjWinSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_window<13, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjWinSmem);
  static_for_host<4, 12>([&](auto Q) {
    if (e == cudaSuccess) e = adj_cols_attr<decltype(Q)::value>();
  });
  static_for_host<9, 11>([&](auto C) {
    static_for_host<4, 10>([&](auto Q) {
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_adj_cols2<decltype(Q)::value, decltype(C)::value>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj_cols2_smem());
    });
  });
  static_for_host<10, 15>([&](auto C) {
    if (e == cudaSuccess) e = adj_rows_attr<decltype(C)::value>();
  });
  if (e == cudaSuccess) e = adj_rows_attr<10, kPassElemsLog>();
  if (e == cudaSuccess) e = adj_rows_attr<9, kPassElemsLog>();
  return e;
}

cudaError_t launch_adj_tile(const AdjArgs& a, int grid, cudaStream_t s) {
  if (a.t)
    k_adj_tile<kTileLog, kTileThreads, true><<<grid, kTileThreads, kAdjTileSmem, s>>>(a);
  else
    k_adj_tile<kTileLog, kTileThreads, false><<<grid, kTileThreads, kAdjTileSmem, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_adj_levels(const AdjArgs& a, int m, cudaStream_t s) {
  k_adj_levels<kLevelsThreads><<<m, kLevelsThreads, adj_levels_smem(), s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_adj_tiny(const AdjArgs& a, int nsig_tiny, cudaStream_t s) {
  if (a.t)
    k_adj_tiny<true><<<nsig_tiny, 32, 0, s>>>(a);
  else
    k_adj_tiny<false><<<nsig_tiny, 32, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_adj_window(const AdjArgs& a, int grid, cudaStream_t s) {
  if (a.level == 13)
    a.t ? k_adj_window<12, true><<<grid, kWinThreads, kAdjWinSmem, s>>>(a)
        : k_adj_window<12, false><<<grid, kWinThreads, kAdjWinSmem, s>>>(a);
  else
    a.t ? k_adj_window<13, true><<<grid, kWinThreads, kAdjWinSmem, s>>>(a)
        : k_adj_window<13, false><<<grid, kWinThreads, kAdjWinSmem, s>>>(a);
  return cudaGetLastError();
}
// C = 2^adj_cb of a two-pass level (Q = h / C <= 2^11 keeps cols chunks of >= 4)
static int adj_cb(int cb_min, int i) {
  const int m = cb_min ? cb_min : 10;
  return (i - 1) - 11 > m ? (i - 1) - 11 : m;
}
cudaError_t launch_adj_rows(const AdjArgs& a, int grid, cudaStream_t s) {
  const int CB = adj_cb(a.cb_min, a.level);
  static_for_host<9, 15>([&](auto C) {
    if (CB == decltype(C)::value) adj_rows_launch<decltype(C)::value>(a, grid, s);
  });
  return cudaGetLastError();
}
bool adj_cols2_pairable(int upper_level, int cb_min) {
  const int i = upper_level - 1, CB = adj_cb(cb_min, i), QB = (i - 1) - CB;
  return i >= 15 && adj_cb(cb_min, upper_level) == CB && (CB == 9 || CB == 10) && QB >= 4 && QB <= 9;
}
cudaError_t launch_adj_cols2(const AdjArgs& a, int grid, cudaStream_t s) {
  const int i = a.level - 1, CB = adj_cb(a.cb_min, i), QB = (i - 1) - CB;
  static_for_host<9, 11>([&](auto C) {
    static_for_host<4, 10>([&](auto Q) {
      constexpr int q = decltype(Q)::value, c = decltype(C)::value;
      if (QB == q && CB == c) k_adj_cols2<q, c><<<grid << 1, kColsThreads, adj_cols2_smem(), s>>>(a);
    });
  });
  return cudaGetLastError();
}
cudaError_t launch_adj_cols(const AdjArgs& a, int grid, cudaStream_t s) {
  const int QB = (a.level - 1) - adj_cb(a.cb_min, a.level);
  static_for_host<4, 12>([&](auto Q) {
    if (QB == decltype(Q)::value) adj_cols_launch<decltype(Q)::value>(a, grid, s);
  });
  return cudaGetLastError();
}

}  // namespace mrdft
