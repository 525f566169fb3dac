// Forward MrDFT kernels (sm_103a).
//
// The level recursion of Sec. 3 of Andreatto & Cariow (Eq. 4): for a window
// of length 2^i with halves a, b (h = 2^(i-1)),
//   even bins  Y_i[2k]   = Y_{i-1}^{(a)}[k] + Y_{i-1}^{(b)}[k]        (U, Eq. 2)
//   odd bins   Y_i[2k+1] = DFT_h((a - b) * w_{2^i}^n)[k]            (V, Eq. 3; D; F)
// and level 1 is (x0 + x1, x0 - x1) (A^(1)).  The permutation Gamma is folded
// into the store index (bins are written in natural order).
//
//   k_fwd_tile   levels 1..tlog (tlog <= 12) of a tile in shared memory:
//                levels 1..4 per thread in registers (16 samples per thread),
//                levels 5..12 through the shared-memory FFT engine.
//   k_fwd_tiny   signals of length 2, 4, 8, 16 (Eq. 1 term by term).
//   k_fwd_window one level (13 or 14) of one window per CTA.
//   k_fwd_cols / k_fwd_rows  one level i >= 15 in two passes: DFT_h with
//                h = Q * C split as a length-Q DFT across C-sample chunks
//                (cols) and a length-C DFT per output residue (rows).
//   k_fwd_cols2  the cols passes of two consecutive levels from one read of x.
#include <cuda_runtime.h>

#include <type_traits>

#include "mrdft_fft.cuh"
#include "mrdft_internal.h"

namespace mrdft {

__device__ __forceinline__ float4 ld4s(const float2* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4s(float2* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// x sample (promoted to complex) at flat index e of the input buffer
__device__ __forceinline__ float2 load_x1(const FwdArgs& a, int64_t e) {
  if (a.in_real) return make_float2(__ldg(reinterpret_cast<const float*>(a.x) + e), 0.f);
  return __ldg(reinterpret_cast<const float2*>(a.x) + e);
}
// the same, marked evict-first in L2 (a level reads its x once; keeping it
// out of the way lets the level's intermediate stay in L2 until it is used)
__device__ __forceinline__ float2 load_x1_stream(const FwdArgs& a, int64_t e) {
  if (a.in_real) return make_float2(__ldcs(reinterpret_cast<const float*>(a.x) + e), 0.f);
  return __ldcs(reinterpret_cast<const float2*>(a.x) + e);
}
// two consecutive samples e, e+1 (e even, 16-byte aligned for complex input)
__device__ __forceinline__ float4 load_x2(const FwdArgs& a, int64_t e) {
  if (a.in_real) {
    float2 r = __ldg(reinterpret_cast<const float2*>(reinterpret_cast<const float*>(a.x) + e));
    return make_float4(r.x, 0.f, r.y, 0.f);
  }
  return __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(a.x) + e));
}

// ===================================================================== tile

// Per-item signal table kept in shared memory: for packed items (several
// whole signals of length 2^tlog) each signal has its own input and output
// base; a single-signal item has one entry.
struct TileSig {
  int64_t in_base;   // x offset of the tile's first sample
  int64_t out_base;  // y offset of the tile's first level-1 output
  int32_t m;
  int32_t pad;
};
constexpr int kMaxPack = kTile / 32;  // signals of >= 32 samples per tile
static_assert(sizeof(TileSig) == 24, "TileSig layout");

// Levels 1..4 of one 16-sample chunk (one 128-byte row of the tile), in
// registers: A^(1), then U / V / D / F per level with compile-time twiddles.
// Every level goes to global memory -- with `slice` (a whole single-signal
// tile) through the warp's own shared memory so that the stores coalesce
// (warp_rows16_store), else row by row; level 4 also goes to shared memory
// for level 5.
__device__ __forceinline__ void tile_chunk_levels_1_4(const FwdArgs& a, const float2* X, float2* B4, int chunk,
                                                      const TileSig* TS, int tl, float2* slice) {
  float2 xr[16], yr[16];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 v = ld4s(X + swz128((chunk << 4) + 2 * q));
    xr[2 * q] = make_float2(v.x, v.y);
    xr[2 * q + 1] = make_float2(v.z, v.w);
  }
  const int e = chunk << 4, wrow0 = (chunk & ~31) << 4;  // this row, the warp's first row
  auto store_level = [&](int j) MRDFT_INL {
    if (slice) {
      float2* base = a.y + TS[0].out_base + ((int64_t)(j - 1) << TS[0].m) + wrow0;
      warp_rows16_store(yr, slice, [&](int r) MRDFT_INL { return base + (r << 4); });
    } else {
      const TileSig& t = TS[e >> tl];
      float4* dst = reinterpret_cast<float4*>(a.y + t.out_base + ((int64_t)(j - 1) << t.m) + (e & ((1 << tl) - 1)));
#pragma unroll
      for (int q = 0; q < 8; ++q)
        __stcs(dst + q, make_float4(yr[2 * q].x, yr[2 * q].y, yr[2 * q + 1].x, yr[2 * q + 1].y));
    }
  };
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    yr[2 * w] = cadd(xr[2 * w], xr[2 * w + 1]);
    yr[2 * w + 1] = csub(xr[2 * w], xr[2 * w + 1]);
  }
  store_level(1);
  static_for<2, 5>([&](auto J) MRDFT_INL {
    constexpr int j = decltype(J)::value;
    constexpr int L = 1 << j, h = L / 2;
    static_for<0, 16 / L>([&](auto W) MRDFT_INL {
      constexpr int w = decltype(W)::value;
      float2 ev[h], z[h];
      // U (Eq. 2): even bins are the sum of the children spectra
      static_for<0, h>([&](auto K) MRDFT_INL {
        constexpr int k = decltype(K)::value;
        ev[k] = cadd(yr[w * L + k], yr[w * L + h + k]);
      });
      // V (Eq. 3) and D: twiddled half-difference, then F: DFT_h
      static_for<0, h>([&](auto N) MRDFT_INL {
        constexpr int n = decltype(N)::value;
        z[n] = cmul_ct<L, n>(csub(xr[w * L + n], xr[w * L + h + n]));
      });
      dft_reg<h>(z);
      static_for<0, h>([&](auto K) MRDFT_INL {
        constexpr int k = decltype(K)::value;
        yr[w * L + 2 * k] = ev[k];
        yr[w * L + 2 * k + 1] = z[k];
      });
    });
    store_level(j);
  });
#pragma unroll
  for (int q = 0; q < 8; ++q)
    st4s(B4 + pad16((chunk << 4) + 2 * q), make_float4(yr[2 * q].x, yr[2 * q].y, yr[2 * q + 1].x, yr[2 * q + 1].y));
}

// LEAN: 3 CTAs per SM instead of 2 -- the odd-bin work area aliases the
// level buffer (each thread reads the children of the bins it will store
// before the FFT overwrites them), the twiddles come from a 1 KB two-level
// table (TwS) instead of the quarter-wave one, and registers are capped at 80.
template <bool LEAN>
constexpr size_t tile_smem() {
  return (size_t)(kTile + pad16_size(kTile) + (LEAN ? tws_size(kTileLog) : kTile / 2 + twq_size(kTileLog))) *
             sizeof(float2) +
         kMaxPack * sizeof(TileSig);
}
template <int TLOG, int NT, bool LEAN>
__global__ void __launch_bounds__(NT, LEAN ? 3 : (NT <= 256 ? 2 : 1)) k_fwd_tile(const FwdArgs a) {
  constexpr int T = 1 << TLOG;
  static_assert(T == 16 * NT, "tile = 16 samples per thread");
  extern __shared__ __align__(1024) float2 sm[];
  float2* X = sm;                       // x tile (swz128)
  float2* B = sm + T;                   // current level, updated in place (pad16)
  float2* Z = LEAN ? B : B + pad16_size(T);  // odd-bin DFT work area (zlay)
  float2* TQ = LEAN ? B + pad16_size(T) : B + pad16_size(T) + T / 2;  // twiddle table (LEAN: two-level)
  TileSig* TS = reinterpret_cast<TileSig*>(TQ + (LEAN ? tws_size(TLOG) : twq_size(TLOG)));
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
      TS[tid] = TileSig{sd.in_off + t0, sd.out_off + t0, sd.m, 0};
    } else {
      bad = 1;
    }
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  // ---- stage the tile of x (P^(1): x is read once and reused per level)
  if (!a.in_real) {
    const float2* xg = reinterpret_cast<const float2*>(a.x);
#pragma unroll 4
    for (int c = tid; c < (Tn >> 1); c += NT) {
      const int e = c << 1;
      cp_async16(X + swz128(e), xg + TS[e >> tl].in_base + (e & ((1 << tl) - 1)));
    }
    if constexpr (!LEAN) load_twq<NT>(TQ, TLOG, a.tw);
    else load_tws<NT>(TQ, TLOG, a.tw);
    cp_async_wait_all();
  } else {
    if constexpr (!LEAN) load_twq<NT>(TQ, TLOG, a.tw);
    else load_tws<NT>(TQ, TLOG, a.tw);
#pragma unroll 4
    for (int c = tid; c < (Tn >> 1); c += NT) {
      const int e = c << 1;
      st4s(X + swz128(e), load_x2(a, TS[e >> tl].in_base + (e & ((1 << tl) - 1))));
    }
  }
  __syncthreads();

  // ---- levels 1..4 in registers, one 16-sample chunk per thread; a whole
  // single-signal tile stores them through each warp's own part of B (the
  // rows its level 4 takes there, written after the staged stores)
  {
    const int e = tid << 4;
    float2* slice = (it.nsig == 1 && Tn == T) ? B + pad16((tid >> 5) << 9) : nullptr;
    if (e < Tn) tile_chunk_levels_1_4(a, X, B, tid, TS, tl, slice);
  }
  __syncthreads();

  // ---- levels 5..tlog through the shared-memory FFT engine; B is updated in
  // place: every child read (pre) happens before the barrier in the last pass
  // (LEAN: before the first pass's barrier, since Z is B)
  using TWT = std::conditional_t<LEAN, TwS, TwQ>;
  TWT tw;
  if constexpr (LEAN) tw = TwS{TQ, TQ + tws_pad((1 << (TLOG - 6)) - 1) + 1, TLOG};
  else tw = TwQ{TQ, TLOG};
  const bool single = it.nsig == 1;
  // one specialised FFT per level (compile-time lengths)
  static_for<5, TLOG + 1>([&](auto I) MRDFT_INL {
    constexpr int i = decltype(I)::value;
    if (i > tl) return;
    constexpr int h = 1 << (i - 1);
    const bool keep = i < tl;  // the next level reads this one
    float2* ylev = a.y + TS[0].out_base + ((int64_t)(i - 1) << TS[0].m);  // single-signal tile
    const bool l2keep = i == tl && TS[0].m > tl;  // re-read as children of level tl+1
    float2 ev[8];
    // V (Eq. 3) and D for a first-pass group: n = n0 + r 2^LRB, so
    // w_{2^i}^n = w_{2^i}^n0 w_{2R}^r with the second factor a constant
    if constexpr (LEAN) {
      // the children of this thread's last-pass bins (group G = tid of the
      // last radix-8 pass: window G >> LRB, bins g + 2^LRB kk), read before
      // the first pass writes the work area over them
      constexpr int LRB = (i - 1) - 3;
      if (tid < (Tn >> 4)) {
        const int base = (tid >> LRB) << i, g = tid & ((1 << LRB) - 1);
        // pad16 adds 2 per 32 elements: offsets of whole 32-element blocks
        // (kk 2^LRB with LRB >= 5, and h >= 32) add their padded value
        const int p0 = pad16(base + g);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int k = g + (kk << LRB);
          const int pa = LRB >= 5 ? p0 + pad16(kk << LRB) : pad16(base + k);
          const int pb = h >= 32 ? pa + pad16(h) : pad16(base + h + k);
          ev[kk] = cadd(B[pa], B[pb]);  // U: child sum
        }
      }
    }
    auto src = [&](int b, int n0, int LRB, auto& v, auto RBc) MRDFT_INL {
      constexpr int R = 1 << decltype(RBc)::value;
      const int base = b << i;
      const float2 w0 = twq_l(tw, i, n0);
      // base, n0 < 2^LRB, r 2^LRB < h and h occupy disjoint bits: one swizzle
      // per group, XORs for the rest
      const int s0 = swz128(base + n0);
      constexpr int sh = swz128(h);
      static_for<0, R>([&](auto RR) MRDFT_INL {
        constexpr int r = decltype(RR)::value;
        const int sa = s0 ^ swz128(r << LRB);
        v[r] = cmul_ct<2 * R, r>(cmul(csub(X[sa], X[sa ^ sh]), w0));
      });
    };
    auto pre = [&](int slot, int b, int k) MRDFT_INL {
      if constexpr (!LEAN) {
        const int base = b << i;
        ev[slot] = cadd(B[pad16(base + k)], B[pad16(base + h + k)]);  // U: child sum
      }
    };
    // the last pass gives this thread group G = tid: window tid >> LRB, bins
    // g + slot 2^LRB (g = tid mod 2^LRB), pair index e = eL + slot 2^(LRB+1);
    // pad16 adds whole 32-element blocks once 2^(LRB+1) >= 32
    constexpr int LRBl = (i - 1) - 3;
    const int eL = ((tid >> LRBl) << i) + 2 * (tid & ((1 << LRBl) - 1));
    const int pL = pad16(eL);
    auto sink = [&](int slot, int, int, float2 odd) MRDFT_INL {
      const int e = eL + (slot << (LRBl + 1));
      const float4 v = make_float4(ev[slot].x, ev[slot].y, odd.x, odd.y);
      if (keep) st4s(B + (LRBl >= 4 ? pL + pad16(slot << (LRBl + 1)) : pad16(e)), v);
      float4* dst;
      if (single) {
        dst = reinterpret_cast<float4*>(ylev + e);
      } else {
        const TileSig& ts = TS[e >> tl];
        dst = reinterpret_cast<float4*>(a.y + ts.out_base + ((int64_t)(i - 1) << ts.m) + (e & ((1 << tl) - 1)));
      }
      if (l2keep) __stcg(dst, v);
      else __stcs(dst, v);
    };
    cg_fft<i - 1, i - 1, NT, 8, false, LEAN ? kPreNone : kPreBarrier, 0, true>(Z, i - 1, tn_log - i, tw, src, pre,
                                                                                  sink);
    __syncthreads();
  });
}

// ============================================================ lone signal

// One signal of N = 2^m samples, 2^5 <= N <= 2^12, alone in its plan: one
// CTA per level, level i from x alone.  Both halves of every window come from
// an FFT of length h: the even bins are the DFT of the folded window a + b
// (Eq. 2 unrolled down to x), the odd bins the DFT of (a - b) w^n (Eq. 3, D,
// F), so the m levels run side by side instead of one after another -- the
// in-tile recursion is a chain of a dozen dependent steps, and a signal this
// small is bound by that chain's latency, not by throughput.
constexpr int kLevelsThreads = 512;
constexpr size_t levels_smem() { return (size_t)(2 * kTile + twq_size(kTileLog)) * sizeof(float2); }
template <int NT>
__global__ void __launch_bounds__(NT, 1) k_fwd_levels(const FwdArgs a) {
  constexpr int T = kTile;
  extern __shared__ __align__(1024) float2 sm[];
  float2* X = sm;           // x (swz128)
  float2* Z = sm + T;       // FFT work area
  float2* TQ = sm + 2 * T;  // quarter-wave w_{2^12}
  const int tid = threadIdx.x;
  const int id = a.nids > 0 ? a.sig_ids[0] : -1;
  if (id < 0 || id >= a.nsigs || a.sigs[id].m < 5 || a.sigs[id].m > kTileLog) {
    if (tid == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const SigDesc sd = a.sigs[id];
  const int m = sd.m, N = 1 << m;
  const int i = (int)blockIdx.x + 1;  // the level of this CTA (grid = m)
  if (i > m) return;
#pragma unroll 4
  for (int c = tid; c < (N >> 1); c += NT) st4s(X + swz128(2 * c), load_x2(a, sd.in_off + 2 * c));
  load_twq<NT>(TQ, kTileLog, a.tw);
  __syncthreads();
  float2* ylev = a.y + sd.out_off + ((int64_t)(i - 1) << m);
  if (i == 1) {  // A^(1)
    for (int c = tid; c < (N >> 1); c += NT) {
      const float2 x0 = X[swz128(2 * c)], x1 = X[swz128(2 * c + 1)];
      const float2 s0 = cadd(x0, x1), s1 = csub(x0, x1);
      __stcs(reinterpret_cast<float4*>(ylev) + c, make_float4(s0.x, s0.y, s1.x, s1.y));
    }
    return;
  }
  const TwQ tw{TQ, kTileLog};
  const int h = 1 << (i - 1);
  // sequence s = 2 w + c of window w: c = 0 the folded window, 1 the twiddled
  // half-difference; its bin k is bin 2k + c of the window
  auto src = [&](int s, int n) MRDFT_INL -> float2 {
    const int base = (s >> 1) << i;
    const float2 xa = X[swz128(base + n)], xb = X[swz128(base + h + n)];
    return (s & 1) ? cmul(csub(xa, xb), twq_l(tw, i, n)) : cadd(xa, xb);
  };
  auto sink = [&](int, int s, int k, float2 v) MRDFT_INL { __stcs(ylev + ((s >> 1) << i) + 2 * k + (s & 1), v); };
  cg_fft<1, kTileLog - 1, NT, T / NT, false, kPreNone>(Z, i - 1, m - i + 1, tw, src, NoPre{}, sink);
}

// ===================================================================== tiny

// Signals with N <= 16: Eq. 1 term by term, one thread per output bin.
__global__ void k_fwd_tiny(const FwdArgs a) {
  const int s = blockIdx.x;
  const int id = s < a.nids ? a.sig_ids[s] : -1;
  if (id < 0 || id >= a.nsigs || a.sigs[id].m < 1 || a.sigs[id].m > 4) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const SigDesc sd = a.sigs[id];
  const int N = 1 << sd.m;
  const int t = threadIdx.x;  // output index over m * N
  if (t >= sd.m * N) return;
  const int i = t / N + 1, p = t % N;
  const int L = 1 << i, w = p >> i, k = p & (L - 1);
  float2 acc = make_float2(0.f, 0.f);
  for (int n = 0; n < L; ++n) {
    float2 xv = load_x1(a, sd.in_off + (w << i) + n);
    acc = cadd(acc, cmul(xv, tw_small(a.tw, i, (n * k) & (L - 1))));
  }
  a.y[sd.out_off + t] = acc;
}

// =================================================================== window

// One window of level i = LB + 1 (h = 2^LB odd-bin DFT points) per CTA:
// z from x, DFT_h in shared memory, even bins from the level-(i-1) children
// in y (moved into L2 when the CTA starts, read per group of 8 bins), (even,
// odd) pairs stored at 2k.
template <int LB>
__global__ void __launch_bounds__(kWinThreads, 2) k_fwd_window(const FwdArgs a) {
  constexpr int NT = kWinThreads;
  constexpr int h = 1 << LB;
  constexpr int i = LB + 1;
  constexpr int PTS = h / NT;                   // points per thread per pass
  constexpr int SA = LB == 12 ? 6 : 3, SB = LB == 12 ? 0 : 9;  // staging layout
  extern __shared__ __align__(1024) float2 sm[];
  float2* Z = sm;                               // 2^LB (staging layout, then zlay)
  float2* TQ = sm + (1 << kWinMaxLog);          // quarter-wave w_{2^13}
  if ((int)blockIdx.x >= a.nitems) return;
  const LevelItem it = reinterpret_cast<const LevelItem*>(a.items)[blockIdx.x];
  SigDesc sd;
  if (!level_item_ok(a.sigs, a.nsigs, it, i, 1, sd)) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const int64_t ws = (int64_t)it.window << i;
  const int64_t xs = sd.in_off + ws;
  const float2* yprev = a.y + sd.out_off + ((int64_t)(i - 2) << sd.m) + ws;
  float2* ycur = a.y + sd.out_off + ((int64_t)(i - 1) << sd.m) + ws;
  load_twq<NT>(TQ, 13, a.tw);
  // w_{2^14}^n = w_{2^13}^(n/2) w_{2^14}^(n mod 2)
  const float2 w1 = __ldg(&a.tw.tw13[1]);
  __syncthreads();
  const TwQ tw{TQ, 13};
  // V (Eq. 3) and D: z[n] = (a[n] - b[n]) w_{2^i}^n, loads issued 8 at a time,
  // z staged in the XOR layout that the first FFT pass reads digit-reversed;
  // n = tid + 256 t, so w_{2^i}^n = w_{2^i}^tid w_{2^(i-8)}^t (a constant)
  static_assert(NT == 256, "twiddle split assumes 256 threads");
  float2 wt;
  if constexpr (i <= 13) {
    wt = twq_l(tw, i, threadIdx.x);
  } else {
    wt = twq(tw, threadIdx.x >> 1);
    if (threadIdx.x & 1) wt = cmul(wt, w1);
  }
  static_for<0, PTS / 8>([&](auto T0) MRDFT_INL {
    constexpr int t0 = decltype(T0)::value * 8;
    float2 xa[8], xb[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int n = threadIdx.x + (t0 + t) * NT;
      xa[t] = load_x1_stream(a, xs + n);
      xb[t] = load_x1_stream(a, xs + h + n);
    }
    static_for<0, 8>([&](auto TT) MRDFT_INL {
      constexpr int t = decltype(TT)::value;
      const int n = threadIdx.x + (t0 + t) * NT;
      Z[stg<SA, SB>(n)] = cmul_ct<(1 << (i - 8)), t0 + t>(cmul(csub(xa[t], xb[t]), wt));
    });
  });
  __syncthreads();
  const bool reread = sd.m > i;  // children of the next level: keep in L2
  float2 ea[PTS], eb[PTS];
  const StgGroup<SA, SB> src{Z, 0, 0};
  auto pre = [&](int slot, int, int k) MRDFT_INL {
    ea[slot] = __ldcs(yprev + k);
    eb[slot] = __ldcs(yprev + h + k);
  };
  auto sink = [&](int slot, int, int k, float2 odd) MRDFT_INL {
    const float2 ev = cadd(ea[slot], eb[slot]);
    const float4 v = make_float4(ev.x, ev.y, odd.x, odd.y);
    float4* dst = reinterpret_cast<float4*>(ycur + 2 * k);
    if (reread) __stcg(dst, v);
    else __stcs(dst, v);
  };
  cg_fft<LB, LB, NT, PTS, false, kPreGroup, 0, true>(Z, LB, 0, tw, src, pre, sink);
}

// cols pass: work area 2^E, w_{2^12} table, chunk twiddles (RC <= 2^(E-3))
constexpr size_t cols_smem(int E) { return (size_t)((1 << E) + twq_size(12) + (1 << (E - 3))) * sizeof(float2); }
// cols CTAs of 2^12 points (4 per SM) where Q <= 2^10 keeps chunks of >= 4
template <int QB>
constexpr int cols_e() { return QB <= 10 ? 12 : kPassElemsLog; }
// rows pass: work area, w_C table, twiddle tables KC (64 + 1) + KC (C / 64 + 16 / KC)
// (PF: plus both children of every output bin, 2 x 2^E, from a 16-byte boundary)
__host__ __device__ constexpr int rows_ch_off(int E, int CB) {
  return ((1 << E) + twq_size(CB) + (1 << (E - CB)) * 65 + (1 << (E - 6)) + 16 + 1) & ~1;
}
constexpr size_t rows_smem(int E, int CB, bool PF = false) {
  return (size_t)(rows_ch_off(E, CB) + (PF ? 2 << E : 0)) * sizeof(float2);
}

// =============================================================== two-pass

// Level i with h = 2^(i-1) = Q * C, C = 2^CB (fwd_cb), Q = 2^QB.
// With n = r + C q (r < C, q < Q) and k = Q k1 + k2:
//   DFT_h(z)[Q k1 + k2] = sum_r w_C^(r k1) w_h^(r k2) sum_q z[r + C q] w_Q^(q k2).
// cols: item (sig, window, c) covers chunk offsets r in [r0, r0 + RC),
//   r0 = c RC, RC = 2^13 / Q: z[r + C q] -> DFT_Q over q -> scratch F[window][k2][r].
// rows: a CTA of 2^E points covers residues k2 in [k0, k0 + KC), KC = 2^E / C:
//   F[window][k2][.] times w_h^(r k2) -> DFT_C -> odd bin Q k1 + k2; even bin
//   from the children; (even, odd) pairs stored at 2k.
template <int NT, int QB, int E>
__global__ void __launch_bounds__(NT, E < kPassElemsLog ? 4 : 2) k_fwd_cols(const FwdArgs a) {
  constexpr int PTS = (1 << E) / NT;
  constexpr int SH = kPassElemsLog - E;      // CTAs per item: 2^SH
  constexpr int RCB = E - QB, RC = 1 << RCB;
  extern __shared__ __align__(1024) float2 sm[];
  float2* S = sm;                            // column r position q: q RC + r (staging, then zlay)
  float2* TQ = sm + (1 << E);                // quarter-wave w_{2^12}
  float2* ZC = TQ + twq_size(12);            // w_{2^i}^(r0 + r), r < RC
  const int item = (int)blockIdx.x >> SH;
  if (item >= a.nitems) return;
  const LevelItem it = reinterpret_cast<const LevelItem*>(a.items)[item];
  const int i = a.level;
  const int HB = i - 1, CB = HB - QB;
  SigDesc sd;
  if (!level_item_ok(a.sigs, a.nsigs, it, i, pass_items(i), sd)) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const int64_t xs = sd.in_off + ((int64_t)it.window << i);
  const int r0 = ((it.block << SH) | ((int)blockIdx.x & ((1 << SH) - 1))) << RCB;
  const int64_t h = (int64_t)1 << HB;
  load_twq<NT>(TQ, 12, a.tw);
  for (int r = threadIdx.x; r < RC; r += NT) ZC[r] = tw_any(a.tw, i, r0 + r);
  __syncthreads();
  const TwQ tw{TQ, 12};
  // V (Eq. 3) and D: z[n] = (a[n] - b[n]) w_{2^i}^n, w_{2^i}^(r0 + r + C q) =
  // w_{2^i}^(r0 + r) w_{2Q}^q; the loads of a batch are issued before any use
#pragma unroll 1
  for (int t0 = 0; t0 < PTS; t0 += 8) {
    float2 xa[8], xb[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = threadIdx.x + (t0 + t) * NT;
      const int64_t n = ((int64_t)(e >> RCB) << CB) + r0 + (e & (RC - 1));
      xa[t] = load_x1_stream(a, xs + n);
      xb[t] = load_x1_stream(a, xs + h + n);
    }
    if constexpr (NT >= RC) {
      // every point of this thread has the thread's column r and q = q_tid +
      // (t0 + t) NT / RC, so w_{2Q}^q = w_{2Q}^(q_tid) w_32^(t0 + t) (2Q RC / NT
      // = 32): one lookup per thread, compile-time factors per point
      static_assert((1 << (E + 1)) / NT == 32 && PTS == 16, "w_32 steps over two batches of 8");
      const float2 w0 = cmul(ZC[threadIdx.x & (RC - 1)], twq_l(tw, QB + 1, threadIdx.x >> RCB));
      const float2 wb = t0 ? cmul_mj(w0) : w0;  // w_32^8 = -j
      static_for<0, 8>([&](auto TT) MRDFT_INL {
        constexpr int t = decltype(TT)::value;
        const int e = threadIdx.x + (t0 + t) * NT;
        S[stg<6, 0>(e)] = cmul(csub(xa[t], xb[t]), cmul_ct<32, t>(wb));  // e = q RC + r
      });
    } else {
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int e = threadIdx.x + (t0 + t) * NT;
        const float2 w = cmul(ZC[e & (RC - 1)], twq_l(tw, QB + 1, e >> RCB));
        S[stg<6, 0>(e)] = cmul(csub(xa[t], xb[t]), w);  // e = q RC + r
      }
    }
  }
  __syncthreads();
  float2* F = a.scratch + sd.aux_off + ((int64_t)it.window << HB);
  const StgGroup<6, 0> src{S, RCB, 0};
  // the intermediate is read by the rows pass right after: keep it in L2
  // (f_late: the rows pass comes much later; let it leave L2 first instead)
  const uint64_t keep = a.f_late ? l2_evict_first_policy() : l2_evict_last_policy();
  auto sink = [&](int, int b, int k2, float2 v) MRDFT_INL { st_l2_keep(F + ((int64_t)k2 << CB) + r0 + b, v, keep); };
  cg_fft<QB, QB, NT, PTS, true, kPreNone, (RCB < 4 ? RCB : 4), true>(S, QB, RCB, tw, src, NoPre{}, sink);
}

// Two levels, one read of x: the cols passes of levels i and i + 1 (the same
// C, Q = 2^QB for level i and 2Q for level i + 1).  A CTA takes chunk
// offsets [r0, r0 + RC) of one level-(i+1) window, whose column strip holds the
// rows q'' < 4Q; with x_j = x[r + C (q + j Q)] for j = 0..3,
//   level i + 1 (halves a = rows < 2Q, b = the rest):
//     z'[q] = (x_0 - x_2) w_{2^(i+1)}^(r + C q),  z'[q + Q] = (x_1 - x_3) w_{2^(i+1)}^(r + C (q + Q))
//   level i, child c = 0, 1 (its own halves: rows q and q + Q of the child):
//     z_c[q] = (x_{2c} - x_{2c+1}) w_{2^i}^(r + C q),
// then DFT_2Q of z' and DFT_Q of z_0, z_1 over q, into the two levels'
// intermediates.  The rows passes of both levels follow unchanged.
template <int QB, int CB>
__global__ void __launch_bounds__(kColsThreads, 2) k_fwd_cols2(const FwdArgs a) {
  constexpr int NT = kColsThreads;
  constexpr int E = kPassElemsLog;
  constexpr int Q = 1 << QB;
  constexpr int RCB = E - QB - 2, RC = 1 << RCB;
  constexpr int UNITS = (Q << RCB) / NT;                 // (q, b) units per thread
  constexpr int PTS = (1 << (E - 1)) / NT;               // FFT points per thread, each level
  constexpr int SA1 = QB == 9 ? 6 : 3;                   // staging layouts
  static_assert(RCB >= 2 && UNITS >= 1, "column blocks of at least 4");
  extern __shared__ __align__(1024) float2 sm[];
  float2* Z1 = sm;                                       // level i+1: q' RC + b
  float2* Z0 = sm + (1 << (E - 1));                      // level i: q 2RC + c RC + b
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
  const int64_t xs = sd.in_off + ((int64_t)it.window << i1);
  const int r0 = ((it.block << 1) | ((int)blockIdx.x & 1)) << RCB;
  load_twq<NT>(TQ, 12, a.tw);
  for (int b = threadIdx.x; b < RC; b += NT) {
    ZC1[b] = tw_any(a.tw, i1, r0 + b);
    ZC0[b] = tw_any(a.tw, i, r0 + b);
  }
  __syncthreads();
  const TwQ tw{TQ, 12};
  float2 xv[UNITS][4];
#pragma unroll
  for (int u = 0; u < UNITS; ++u) {
    const int e = threadIdx.x + u * NT;                  // e = q RC + b
    const int64_t n = ((int64_t)(e >> RCB) << CB) + r0 + (e & (RC - 1));
#pragma unroll
    for (int j = 0; j < 4; ++j) xv[u][j] = load_x1_stream(a, xs + n + ((int64_t)(j * Q) << CB));
  }
#pragma unroll
  for (int u = 0; u < UNITS; ++u) {
    const int e = threadIdx.x + u * NT;
    const int q = e >> RCB, b = e & (RC - 1);
    const float2 w1 = cmul(ZC1[b], twq_l(tw, QB + 2, q));     // w_{2^(i+1)}^(r0 + b + C q)
    const float2 w0 = cmul(ZC0[b], twq_l(tw, QB + 1, q));     // w_{2^i}^(r0 + b + C q)
    Z1[stg<SA1, 0>(e)] = cmul(csub(xv[u][0], xv[u][2]), w1);
    Z1[stg<SA1, 0>(e + (Q << RCB))] = cmul_mj(cmul(csub(xv[u][1], xv[u][3]), w1));  // w_{4Q}^Q = -j
    const int e0 = (q << (RCB + 1)) + b;
    Z0[stg<3, 0>(e0)] = cmul(csub(xv[u][0], xv[u][1]), w0);
    Z0[stg<3, 0>(e0 + RC)] = cmul(csub(xv[u][2], xv[u][3]), w0);
  }
  __syncthreads();
  const uint64_t keep = l2_evict_last_policy();
  // level i + 1 (window it.window, h = 2^i): intermediate F1[k2][r]
  float2* F1 = a.scratch2 + sd.aux_off + ((int64_t)it.window << i);
  const StgGroup<SA1, 0> src1{Z1, RCB, 0};
  auto sink1 = [&](int, int b, int k2, float2 v) MRDFT_INL { st_l2_keep(F1 + ((int64_t)k2 << CB) + r0 + b, v, keep); };
  cg_fft<QB + 1, QB + 1, NT, PTS, true, kPreNone, (RCB < 4 ? RCB : 4), true>(Z1, QB + 1, RCB, tw, src1, NoPre{}, sink1);
  // level i (children 2W, 2W + 1, h = 2^(i-1)): sequence s = c RC + b
  float2* F0 = a.scratch + sd.aux_off + ((int64_t)(2 * it.window) << (i - 1));
  const StgGroup<3, 0> src0{Z0, RCB + 1, 0};
  auto sink0 = [&](int, int s, int k2, float2 v) MRDFT_INL {
    const int c = s >> RCB, b = s & (RC - 1);
    st_l2_keep(F0 + ((int64_t)c << (i - 1)) + ((int64_t)k2 << CB) + r0 + b, v, keep);
  };
  cg_fft<QB, QB, NT, PTS, true, kPreNone, (RCB + 1 < 4 ? RCB + 1 : 4), true>(Z0, QB, RCB + 1, tw, src0, NoPre{}, sink0);
}

constexpr size_t cols2_smem() {
  return (size_t)((1 << kPassElemsLog) + twq_size(12) + 2 * (1 << (kPassElemsLog - 5))) * sizeof(float2);
}

// PF: the children of every output bin are copied into shared memory
// (cp.async) when the CTA starts, behind the intermediate, so that their
// latency overlaps the whole FFT instead of stalling the last pass.
template <int E, int NT, int CB, bool PF>
__global__ void __launch_bounds__(NT, PF ? (E < kPassElemsLog ? 2 : 1) : (E < kPassElemsLog ? 4 : (E == kPassElemsLog ? 2 : 1)))
    k_fwd_rows(const FwdArgs a) {
  constexpr int PTS = (1 << E) / NT;
  constexpr int C = 1 << CB;
  constexpr int KCB = E - CB, KC = 1 << KCB;
  constexpr int HU = C >> 6;               // rows of the high twiddle table
  constexpr int SH = E - kPassElemsLog;    // CTAs per item: 2^-SH (SH < 0), items per CTA: 2^SH
  constexpr int SA = CB <= 12 ? 4 : 3, SB = CB <= 12 ? 6 : 9;  // staging layout
  extern __shared__ __align__(1024) float2 sm[];
  float2* S = sm;                          // sequence j position r at r KC + j (staging, then zlay)
  float2* TQ = sm + (1 << E);              // quarter-wave w_C
  float2* TWL = TQ + twq_size(CB);         // [KC][64] (row stride 65): w_h^(k2 t)
  float2* TWH = TWL + KC * 65;             // [KC][C/64] (row stride C/64 + 16/KC): w_h^(k2 64 u)
  float2* CH = sm + rows_ch_off(E, CB);    // PF: child a of bin (k1, j) at k1 KC + j, child b 2^E further
  static_assert(!PF || (KC >= 2 && (1 << E) / 8 >= NT), "children in 16-byte runs; every thread in the last pass");
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
  const int64_t h = (int64_t)1 << HB;
  SigDesc sd;
  if (!level_item_ok(a.sigs, a.nsigs, it, i, pass_items(i), sd)) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const int64_t ws = (int64_t)it.window << i;
  const int k0 = blk << KCB;
  const float2* F = a.scratch + sd.aux_off + ((int64_t)it.window << HB);
  const float2* __restrict__ yprev = a.y + sd.out_off + ((int64_t)(i - 2) << sd.m) + ws;
#pragma unroll 8
  for (int e = threadIdx.x; e < KC * C; e += NT) {
    const int r = e & (C - 1), j = e >> CB;
    cp_async8(S + stg<SA, SB>((r << KCB) + j), F + ((int64_t)(k0 + j) << CB) + r);
  }
  if constexpr (PF) {
    cp_async_commit();
    // U (Eq. 2) inputs: bins k = k1 Q + k0 + j of both children, KC-bin runs
#pragma unroll 8
    for (int t = threadIdx.x; t < C * KC; t += NT) {
      const int half = t >> (CB + KCB - 1), r = t & ((C * KC / 2) - 1);
      const int k1 = r >> (KCB - 1), c = r & (KC / 2 - 1);
      cp_async16(CH + (half << E) + (k1 << KCB) + 2 * c, yprev + half * h + ((int64_t)k1 << QB) + k0 + 2 * c);
    }
    cp_async_commit();
  }
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
  if constexpr (PF) cp_async_wait<1>();  // the intermediate; the children may still be in flight
  else cp_async_wait_all();
  __syncthreads();
  // the intermediate rows are dead now: drop them from L2 without write-back
  for (int l = threadIdx.x; l < KC * C / 16; l += NT) discard_l2(F + ((int64_t)k0 << CB) + 16 * l);
  const TwQ tw{TQ, CB};
  float2* ycur = a.y + sd.out_off + ((int64_t)(i - 1) << sd.m) + ws;
  // w_h^(r k2) = w_h^(k2 (r mod 64)) w_h^(k2 64 (r / 64)); a first-pass group
  // reads r = n0 + 2^LRB j with 2^LRB >= 64, so its low factor is shared
  auto src = [&](int b, int n0, int LRB, auto& v, auto RBc) MRDFT_INL {
    constexpr int R = 1 << decltype(RBc)::value;
    const float2 lo = TWL[b * 65 + (n0 & 63)];
    const int e0 = stg<SA, SB>((n0 << KCB) | b);  // stg is linear over XOR: one layout computation per group
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int n = n0 + (j << LRB);
      v[j] = cmul(S[e0 ^ stg<SA, SB>((j << LRB) << KCB)], cmul(lo, TWH[b * (HU + 16 / KC) + (n >> 6)]));
    }
  };
  const bool reread = sd.m > i;
  auto store = [&](int b, int k1, float2 ev, float2 odd) MRDFT_INL {
    const int64_t k = ((int64_t)k1 << QB) + k0 + b;
    const float4 v = make_float4(ev.x, ev.y, odd.x, odd.y);
    float4* dst = reinterpret_cast<float4*>(ycur + 2 * k);
    if (reread) __stcg(dst, v);
    else __stcs(dst, v);
  };
  static_assert(3 * ((CB + 2) / 3 - 1) >= 6, "first-pass stride below 64");
  if constexpr (PF) {
    // the last pass waits for this thread's children copies before its
    // barrier; after the barrier every thread's copies are visible
    auto pre = [&](int slot, int, int) MRDFT_INL {
      if (slot == 0) cp_async_wait<0>();
    };
    auto sink = [&](int, int b, int k1, float2 odd) MRDFT_INL {
      const int e = (k1 << KCB) + b;
      store(b, k1, cadd(CH[e], CH[(1 << E) + e]), odd);  // U (Eq. 2): child sum
    };
    cg_fft<CB, CB, NT, PTS, true, kPreBarrier, KCB, true>(S, CB, KCB, tw, src, pre, sink);
  } else {
    float2 ea[PTS], eb[PTS];
    // U (Eq. 2): the children of bin k, read once per group of 8 bins
    auto pre = [&](int slot, int b, int k1) MRDFT_INL {
      const int64_t k = ((int64_t)k1 << QB) + k0 + b;
      ea[slot] = __ldcs(yprev + k);
      eb[slot] = __ldcs(yprev + h + k);
    };
    auto sink = [&](int slot, int b, int k1, float2 odd) MRDFT_INL {
      store(b, k1, cadd(ea[slot], eb[slot]), odd);
    };
    cg_fft<CB, CB, NT, PTS, true, kPreHalf, KCB, true>(S, CB, KCB, tw, src, pre, sink);
  }
}

// Launch-time dispatch to the instantiation of a level's FFT sizes.
template <int QB>
void cols_launch(const FwdArgs& a, int grid, cudaStream_t s) {
  constexpr int E = cols_e<QB>();
  constexpr int NT = E < kPassElemsLog ? kPassThreads : kColsThreads;
  k_fwd_cols<NT, QB, E><<<grid << (kPassElemsLog - E), NT, cols_smem(E), s>>>(a);
}
template <int CB>
constexpr int rows_e() { return rows_elems_log_c(CB, false); }
template <int E, bool PF>
constexpr int rows_nt() {
  return PF ? kColsThreads : (E < kPassElemsLog ? kPassThreads : (E == kPassElemsLog ? kColsThreads : kPassThreadsWide));
}
// children-prefetching rows CTAs: 2^12 points (8 residues, 2 CTAs per SM) at
// C = 2^9, 2^13 points (one CTA per SM) above
template <int CB>
constexpr int rows_pf_e() { return CB <= 9 ? 12 : kPassElemsLog; }
template <int CB, int E = rows_e<CB>(), bool PF = false>
void rows_launch_e(const FwdArgs& a, int grid, cudaStream_t s) {
  constexpr int NT = rows_nt<E, PF>();
  // a CTA of 2^E points takes 2^(E-13) items (E >= 13) or half an item
  int g;
  if constexpr (E >= kPassElemsLog) g = grid >> (E - kPassElemsLog);
  else g = grid << (kPassElemsLog - E);
  k_fwd_rows<E, NT, CB, PF><<<g, NT, rows_smem(E, CB, PF), s>>>(a);
}
template <int CB>
void rows_launch(const FwdArgs& a, int grid, cudaStream_t s) {
  if constexpr (CB <= 12) {
    if (a.rows_pf) {
      rows_launch_e<CB, rows_pf_e<CB>(), true>(a, grid, s);
      return;
    }
  }
  if constexpr (CB == 9) {
    if (a.rows12) {  // 2^12-point CTAs of 256 threads: twice as many, up to 4 per SM
      rows_launch_e<CB, 12>(a, grid, s);
      return;
    }
  }
  if constexpr (CB == 12) {
    if (a.rows14) {
      rows_launch_e<CB, 14>(a, grid, s);
      return;
    }
  }
  rows_launch_e<CB>(a, grid, s);
}
template <int QB>
cudaError_t cols_attr() {
  constexpr int E = cols_e<QB>();
  constexpr int NT = E < kPassElemsLog ? kPassThreads : kColsThreads;
  return cudaFuncSetAttribute(k_fwd_cols<NT, QB, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cols_smem(E));
}
template <int CB, int E = rows_e<CB>(), bool PF = false>
cudaError_t rows_attr() {
  return cudaFuncSetAttribute(k_fwd_rows<E, rows_nt<E, PF>(), CB, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)rows_smem(E, CB, PF));
}

// ================================================================ launchers


static constexpr size_t kWinSmem = (size_t)((1 << kWinMaxLog) + twq_size(13)) * sizeof(float2);
static_assert((1 << kWinMaxLog) % kWinThreads == 0, "points per thread");
cudaError_t set_fwd_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_fwd_tile<kTileLog, kTileThreads, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem<false>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fwd_tile<kTileLog, kTileThreads, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tile_smem<true>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fwd_levels<kLevelsThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)levels_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fwd_window<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWinSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fwd_window<13>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWinSmem);
  static_for_host<3, 12>([&](auto Q) {
    if (e == cudaSuccess) e = cols_attr<decltype(Q)::value>();
  });
  static_for_host<9, 15>([&](auto C) {
    if (e == cudaSuccess) e = rows_attr<decltype(C)::value>();
  });
  if (e == cudaSuccess) e = rows_attr<12, 14>();
  if (e == cudaSuccess) e = rows_attr<9, 12>();
  static_for_host<9, 13>([&](auto C) {
    constexpr int c = decltype(C)::value;
    if (e == cudaSuccess) e = rows_attr<c, rows_pf_e<c>(), true>();
  });
  static_for_host<9, 12>([&](auto C) {
    static_for_host<3, 10>([&](auto Q) {
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fwd_cols2<decltype(Q)::value, decltype(C)::value>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cols2_smem());
    });
  });
  return e;
}

cudaError_t launch_fwd_tile(const FwdArgs& a, int grid, cudaStream_t s) {
  if (a.tile_lean)
    k_fwd_tile<kTileLog, kTileThreads, true><<<grid, kTileThreads, tile_smem<true>(), s>>>(a);
  else
    k_fwd_tile<kTileLog, kTileThreads, false><<<grid, kTileThreads, tile_smem<false>(), s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_fwd_levels(const FwdArgs& a, int m, cudaStream_t s) {
  k_fwd_levels<kLevelsThreads><<<m, kLevelsThreads, levels_smem(), s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_fwd_tiny(const FwdArgs& a, int nsig_tiny, cudaStream_t s) {
  k_fwd_tiny<<<nsig_tiny, 64, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_fwd_window(const FwdArgs& a, int grid, cudaStream_t s) {
  if (a.level == 13)
    k_fwd_window<12><<<grid, kWinThreads, kWinSmem, s>>>(a);
  else
    k_fwd_window<13><<<grid, kWinThreads, kWinSmem, s>>>(a);
  return cudaGetLastError();
}
// C = 2^fwd_cb of a two-pass level (Q = h / C <= 2^11 keeps cols chunks of >= 4)
static int fwd_cb(int cb_min, int i) {
  const int m = cb_min ? cb_min : 10;
  return (i - 1) - 11 > m ? (i - 1) - 11 : m;
}
cudaError_t launch_fwd_cols(const FwdArgs& a, int grid, cudaStream_t s) {
  const int QB = (a.level - 1) - fwd_cb(a.cb_min, a.level);
  static_for_host<3, 12>([&](auto Q) {
    if (QB == decltype(Q)::value) cols_launch<decltype(Q)::value>(a, grid, s);
  });
  return cudaGetLastError();
}
bool fwd_cols2_pairable(int upper_level, int cb_min) {
  const int i = upper_level - 1, CB = fwd_cb(cb_min, i), QB = (i - 1) - CB;
  return i >= 15 && fwd_cb(cb_min, upper_level) == CB && CB >= 9 && CB <= 11 && QB >= 3 && QB <= 9;
}
cudaError_t launch_fwd_cols2(const FwdArgs& a, int grid, cudaStream_t s) {
  const int i = a.level - 1, CB = fwd_cb(a.cb_min, i), QB = (i - 1) - CB;
  static_for_host<9, 12>([&](auto C) {
    static_for_host<3, 10>([&](auto Q) {
      constexpr int q = decltype(Q)::value, c = decltype(C)::value;
      if (QB == q && CB == c) k_fwd_cols2<q, c><<<grid << 1, kColsThreads, cols2_smem(), s>>>(a);
    });
  });
  return cudaGetLastError();
}
cudaError_t launch_fwd_rows(const FwdArgs& a, int grid, cudaStream_t s) {
  const int CB = fwd_cb(a.cb_min, a.level);
  static_for_host<9, 15>([&](auto C) {
    if (CB == decltype(C)::value) rows_launch<decltype(C)::value>(a, grid, s);
  });
  return cudaGetLastError();
}

}  // namespace mrdft

// ====================================================== bit-reversed layout
//
// MRDFT_FLAG_BITREV: each window of each level is rewritten in place in the
// order of the paper's Sec. 3 before the permutation Gamma, i.e. position p of
// a window of level i holds bin bitrev_i(p) (the matrix T_{2^i}, an
// involution).  Runs after the natural-order forward.
namespace mrdft {

__device__ __forceinline__ uint32_t brev_bits(uint32_t v, int bits) { return bits ? __brev(v) >> (32 - bits) : 0; }

// Levels i <= 12: a CTA takes one block of 2^B (B = min(m, 12)) outputs of
// one level of one signal -- whole windows -- through shared memory.
// Item: {sig, block, level}.
__global__ void __launch_bounds__(256) k_bitrev_small(const FwdArgs a) {
  __shared__ __align__(16) float2 buf[kTile];
  const LevelItem it = reinterpret_cast<const LevelItem*>(a.items)[blockIdx.x];
  if (it.sig < 0 || it.sig >= a.nsigs) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const SigDesc sd = a.sigs[it.sig];
  const int i = it.block;
  const int B = sd.m < kTileLog ? sd.m : kTileLog;
  if (i < 1 || i > B || it.window < 0 || ((int64_t)it.window << B) >= ((int64_t)1 << sd.m)) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  float2* base = a.y + sd.out_off + ((int64_t)(i - 1) << sd.m) + ((int64_t)it.window << B);
  const int n = 1 << B;
  for (int e = threadIdx.x; e < n; e += blockDim.x) buf[e] = base[e];
  __syncthreads();
  const int mask = (1 << i) - 1;
  for (int e = threadIdx.x; e < n; e += blockDim.x) base[e] = buf[(e & ~mask) | (int)brev_bits(e & mask, i)];
}

// Levels i > 12: window index k = hi (5 bits) | mid (i - 10 bits) | lo (5 bits);
// bitrev(k) = rev(lo) | rev(mid) | rev(hi), so the 32 x 32 tile of a given mid
// maps onto the tile of rev(mid), transposed with both coordinates reversed.
// A CTA takes mid = M of one window (item {sig, window, level}, M =
// blockIdx.y) and swaps tiles M and rev(M) (CTAs with M > rev(M) leave).
__global__ void __launch_bounds__(256) k_bitrev_big(const FwdArgs a) {
  __shared__ float2 ta[32][33], tb[32][33];
  const LevelItem it = reinterpret_cast<const LevelItem*>(a.items)[blockIdx.x];
  if (it.sig < 0 || it.sig >= a.nsigs) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const SigDesc sd = a.sigs[it.sig];
  const int i = it.block;
  if (i <= kTileLog || i > sd.m || it.window < 0 || (int64_t)it.window >= ((int64_t)1 << (sd.m - i)) ||
      (int)blockIdx.y >= (1 << (i - 10))) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadItem);
    return;
  }
  const uint32_t M = blockIdx.y, Mr = brev_bits(M, i - 10);
  if (M > Mr) return;
  float2* base = a.y + sd.out_off + ((int64_t)(i - 1) << sd.m) + ((int64_t)it.window << i);
  auto addr = [&](uint32_t mid, int hi, int lo) { return base + (((int64_t)hi << (i - 5)) | ((int64_t)mid << 5) | lo); };
  const int lo = threadIdx.x & 31, r0 = threadIdx.x >> 5;
  for (int hi = r0; hi < 32; hi += 8) {
    ta[hi][lo] = *addr(M, hi, lo);
    tb[hi][lo] = *addr(Mr, hi, lo);
  }
  __syncthreads();
  // tile Mr position (row R, col c) takes tile M element (hi = rev(c), lo = rev(R)); and vice versa
  for (int R = r0; R < 32; R += 8) {
    const int h = brev_bits(lo, 5), l = brev_bits(R, 5);
    *addr(Mr, R, lo) = ta[h][l];
    if (M != Mr) *addr(M, R, lo) = tb[h][l];
  }
}

cudaError_t launch_bitrev_small(const FwdArgs& a, int grid, cudaStream_t s) {
  k_bitrev_small<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_bitrev_big(const FwdArgs& a, int grid, int level, cudaStream_t s) {
  k_bitrev_big<<<dim3(grid, 1u << (level - 10)), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mrdft
