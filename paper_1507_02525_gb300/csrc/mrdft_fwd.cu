// Forward MrDFT kernels (sm_103a).
//
// The level recursion of Sec. 3 of Andreatto & Cariow (Eq. 4): for a window
// of length 2^i with halves a, b (h = 2^(i-1)),
//   even bins  Y_i[2k]   = Y_{i-1}^{(a)}[k] + Y_{i-1}^{(b)}[k]        (U, Eq. 2)
//   odd bins   Y_i[2k+1] = DFT_h((a - b) * w_{2^i}^n)[k]            (V, Eq. 3; D; F)
// and level 1 is (x0 + x1, x0 - x1) (A^(1)).  The permutation Gamma is folded
// into the store index (bins are written in natural order).
//
//   k_fwd_tile   levels 1..tlog of a 2^tlog-sample tile in shared memory:
//                levels 1..5 per thread in registers (32 samples per thread),
//                levels 6..12 through the shared-memory FFT engine.
//   k_fwd_tiny   signals of length 2, 4, 8, 16 (Eq. 1 term by term).
//   k_fwd_window one level i (2^12 < 2^i <= 2^14) of one window per CTA.
//   k_fwd_cols / k_fwd_rows  one level i > 14 in two passes: DFT_h with
//                h = Q * 4096 split as a length-Q DFT across 4096-sample
//                chunks (cols) and a length-4096 DFT per output residue (rows).
#include <cuda_runtime.h>

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

// Levels 1..4 of one 16-sample chunk (one 128-byte row of the tile), in
// registers: A^(1), then U / V / D / F per level with compile-time twiddles.
// Every level is stored straight to global memory (the thread writes whole
// 128-byte lines); level 4 also goes to shared memory for level 5.
__device__ __forceinline__ void tile_chunk_levels_1_4(const FwdArgs& a, const float2* X, float2* B4,
                                                      int chunk, const TileSig& ts, int off) {
  float2 xr[16], yr[16];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 v = ld4s(X + swz128((chunk << 4) + 2 * q));
    xr[2 * q] = make_float2(v.x, v.y);
    xr[2 * q + 1] = make_float2(v.z, v.w);
  }
  float2* yl = a.y + ts.out_base + off;
  const int64_t lstride = (int64_t)1 << ts.m;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    yr[2 * w] = cadd(xr[2 * w], xr[2 * w + 1]);
    yr[2 * w + 1] = csub(xr[2 * w], xr[2 * w + 1]);
  }
#pragma unroll
  for (int q = 0; q < 8; ++q)
    __stcs(reinterpret_cast<float4*>(yl) + q, make_float4(yr[2 * q].x, yr[2 * q].y, yr[2 * q + 1].x, yr[2 * q + 1].y));
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
    float4* dst = reinterpret_cast<float4*>(yl + (j - 1) * lstride);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      __stcs(dst + q, make_float4(yr[2 * q].x, yr[2 * q].y, yr[2 * q + 1].x, yr[2 * q + 1].y));
  });
#pragma unroll
  for (int q = 0; q < 8; ++q)
    st4s(B4 + swz128((chunk << 4) + 2 * q), make_float4(yr[2 * q].x, yr[2 * q].y, yr[2 * q + 1].x, yr[2 * q + 1].y));
}

template <int TLOG, int NT>
__global__ void __launch_bounds__(NT, 1) k_fwd_tile(const FwdArgs a) {
  constexpr int T = 1 << TLOG;
  static_assert(T == 32 * NT, "tile = 32 samples per thread");
  extern __shared__ __align__(1024) float2 sm[];
  float2* X = sm;
  float2* B[2] = {sm + T, sm + 2 * T};  // level i lives in B[i & 1]
  float2* Z = sm + 3 * T;
  TileSig* TS = reinterpret_cast<TileSig*>(sm + 3 * T + T / 2);
  const int tid = threadIdx.x;

  {
    // one work item per CTA: a persistent loop lets the compiler hoist the
    // per-level address arithmetic out of it and spill
    const int item = blockIdx.x;
    if (item >= a.nitems) return;
    const TileItem it = reinterpret_cast<const TileItem*>(a.items)[item];
    const int tl = it.tlog;
    const int Tn = it.nsig << tl;
    const int tn_log = 31 - __clz(Tn);
    if (tid < it.nsig) {
      const SigDesc sd = a.sigs[a.sig_ids[it.sig_list + tid]];
      const int64_t t0 = (int64_t)it.tile << tl;
      TS[tid] = TileSig{sd.in_off + t0, sd.out_off + t0, sd.m, 0};
    }
    __syncthreads();

    // ---- stage the tile of x (P^(1): x is read once and reused per level)
    for (int c = tid; c < (Tn >> 1); c += NT) {
      const int e = c << 1;
      st4s(X + swz128(e), load_x2(a, TS[e >> tl].in_base + (e & ((1 << tl) - 1))));
    }
    __syncthreads();

    // ---- levels 1..4 in registers, two 16-sample chunks per thread
#pragma unroll 1
    for (int cc = 0; cc < 2; ++cc) {
      const int chunk = 2 * tid + cc;
      const int e = chunk << 4;
      if (e < Tn) tile_chunk_levels_1_4(a, X, B[0], chunk, TS[e >> tl], e & ((1 << tl) - 1));
    }
    __syncthreads();

    // ---- levels 5..tlog through the shared-memory FFT engine
    static_for<5, TLOG + 1>([&](auto I) MRDFT_INL {
      constexpr int i = decltype(I)::value;
      constexpr int L = 1 << i, h = L / 2;
      if (i <= tl) {
        const float2* Bp = B[(i - 1) & 1];
        float2* Bc = B[i & 1];
        const bool keep = i < tl;  // the next level reads this one
        auto src = [&](int b, int n) MRDFT_INL -> float2 {
          const int base = b << i;
          return cmul(csub(X[swz128(base + n)], X[swz128(base + h + n)]), tw_small(a.tw, i, n));
        };
        auto sink = [&](int b, int k, float2 odd) MRDFT_INL {
          const int e = (b << i) + 2 * k;
          const float2 ev = cadd(Bp[swz128((b << i) + k)], Bp[swz128((b << i) + h + k)]);
          const float4 v = make_float4(ev.x, ev.y, odd.x, odd.y);
          if (keep) st4s(Bc + swz128(e), v);
          const TileSig& ts = TS[e >> tl];
          __stcs(reinterpret_cast<float4*>(a.y + ts.out_base + ((int64_t)(i - 1) << ts.m) + (e & ((1 << tl) - 1))), v);
        };
        fft_inplace<i - 1, NT, false>(Z, tn_log - i, a.tw, src, sink);
        __syncthreads();
      }
    });
  }
}

// ===================================================================== tiny

// Signals with N <= 16: Eq. 1 term by term, one thread per output bin.
__global__ void k_fwd_tiny(const FwdArgs a) {
  const int s = blockIdx.x;
  const SigDesc sd = a.sigs[a.sig_ids[s]];
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

// One window of level i (h = 2^(i-1) <= 2^13 points of odd-bin DFT) per item.
template <int LB>
__device__ __forceinline__ void window_level(const FwdArgs& a, const LevelItem& it, float2* Z) {
  constexpr int NT = kWinThreads;
  constexpr int h = 1 << LB;
  const int i = LB + 1;
  const SigDesc sd = a.sigs[it.sig];
  const int64_t ws = (int64_t)it.window << i;
  const int64_t xs = sd.in_off + ws;
  const float2* yprev = a.y + sd.out_off + ((int64_t)(i - 2) << sd.m) + ws;
  float2* ycur = a.y + sd.out_off + ((int64_t)(i - 1) << sd.m) + ws;
  auto src = [&](int, int n) -> float2 {
    return cmul(csub(load_x1(a, xs + n), load_x1(a, xs + h + n)), tw_any(a.tw, i, n));
  };
  auto sink = [&](int, int k, float2 odd) MRDFT_INL {
    const float2 ev = cadd(__ldg(yprev + k), __ldg(yprev + h + k));
    __stcs(reinterpret_cast<float4*>(ycur + 2 * k), make_float4(ev.x, ev.y, odd.x, odd.y));
  };
  fft_inplace<LB, NT, false>(Z, 0, a.tw, src, sink);
}

template <int LB>
__global__ void __launch_bounds__(kWinThreads) k_fwd_window(const FwdArgs a) {
  extern __shared__ __align__(1024) float2 sm[];
  if (blockIdx.x >= a.nitems) return;
  window_level<LB>(a, reinterpret_cast<const LevelItem*>(a.items)[blockIdx.x], sm);
}

// =============================================================== two-pass

// Level i with h = 2^(i-1) = Q * C, C = 2^12, Q = 2^(i-13).
// cols: item (sig, window, block) covers chunk offsets r in [r0, r0 + RC),
//   RC = 2^14 / Q.  z[r + C q] (q < Q) -> DFT_Q over q -> times w_h^(r k2)
//   -> scratch G[window][k2][r].
template <int QB>
__device__ __forceinline__ void cols_level(const FwdArgs& a, const LevelItem& it, float2* S) {
  constexpr int NT = kPassThreads;
  constexpr int CB = kColsLog, C = 1 << CB;
  constexpr int Q = 1 << QB;
  constexpr int RCB = 14 - QB;  // log2 of columns per item
  constexpr int RC = 1 << RCB;
  constexpr int HB = QB + CB;   // log2 h
  const int i = HB + 1;
  const SigDesc sd = a.sigs[it.sig];
  const int64_t ws = (int64_t)it.window << i;
  const int64_t xs = sd.in_off + ws;
  const int r0 = it.block << RCB;
  constexpr int64_t h = (int64_t)1 << HB;
  // load z[r0 + r + C q] into S[r][q]
  for (int e = threadIdx.x; e < RC * Q; e += NT) {
    const int r = e & (RC - 1), q = e >> RCB;
    const int64_t n = (int64_t)q * C + r0 + r;
    const float2 z = cmul(csub(load_x1(a, xs + n), load_x1(a, xs + h + n)), tw_any(a.tw, i, n));
    S[swzf((r << QB) + q)] = z;
  }
  __syncthreads();
  float2* G = a.scratch + sd.aux_off + ((int64_t)it.window << HB);
  auto src = [&](int b, int n) MRDFT_INL -> float2 { return S[swzf((b << QB) + n)]; };
  auto sink = [&](int b, int k2, float2 v) MRDFT_INL {
    const int r = r0 + b;
    __stcg(G + ((int64_t)k2 << CB) + r, cmul(v, tw_any(a.tw, HB, (int64_t)r * k2)));
  };
  if constexpr (QB >= 1) fft_inplace<QB, NT, true>(S, RCB, a.tw, src, sink);
}

template <int QB>
__global__ void __launch_bounds__(kPassThreads) k_fwd_cols(const FwdArgs a) {
  extern __shared__ __align__(1024) float2 sm[];
  if (blockIdx.x >= a.nitems) return;
  cols_level<QB>(a, reinterpret_cast<const LevelItem*>(a.items)[blockIdx.x], sm);
}

// rows: item (sig, window, block) covers residues k2 in [k0, k0 + KC),
//   KC = 2^14 / C = 4.  G[window][k2][0..C) -> DFT_C -> odd bin k = Q k1 + k2,
//   even bin from the children; (even, odd) pairs stored at 2k.
template <int QB>
__device__ __forceinline__ void rows_level(const FwdArgs& a, const LevelItem& it, float2* S) {
  constexpr int NT = kPassThreads;
  constexpr int CB = kColsLog, C = 1 << CB;
  constexpr int KCB = 14 - CB, KC = 1 << KCB;
  constexpr int HB = QB + CB;
  constexpr int64_t h = (int64_t)1 << HB;
  const int i = HB + 1;
  const SigDesc sd = a.sigs[it.sig];
  const int64_t ws = (int64_t)it.window << i;
  const int k0 = it.block << KCB;
  const float2* G = a.scratch + sd.aux_off + ((int64_t)it.window << HB);
  for (int e = threadIdx.x; e < KC * C; e += NT) {
    const int r = e & (C - 1), j = e >> CB;
    S[swzf((j << CB) + r)] = __ldcg(G + ((int64_t)(k0 + j) << CB) + r);
  }
  __syncthreads();
  const float2* yprev = a.y + sd.out_off + ((int64_t)(i - 2) << sd.m) + ws;
  float2* ycur = a.y + sd.out_off + ((int64_t)(i - 1) << sd.m) + ws;
  auto src = [&](int b, int n) MRDFT_INL -> float2 { return S[swzf((b << CB) + n)]; };
  auto sink = [&](int b, int k1, float2 odd) MRDFT_INL {
    const int64_t k = ((int64_t)k1 << QB) + k0 + b;
    const float2 ev = cadd(__ldg(yprev + k), __ldg(yprev + h + k));
    __stcs(reinterpret_cast<float4*>(ycur + 2 * k), make_float4(ev.x, ev.y, odd.x, odd.y));
  };
  fft_inplace<CB, NT, true>(S, KCB, a.tw, src, sink);
}

template <int QB>
__global__ void __launch_bounds__(kPassThreads) k_fwd_rows(const FwdArgs a) {
  extern __shared__ __align__(1024) float2 sm[];
  if (blockIdx.x >= a.nitems) return;
  rows_level<QB>(a, reinterpret_cast<const LevelItem*>(a.items)[blockIdx.x], sm);
}

// ================================================================ launchers

static constexpr size_t kTileSmem = (size_t)(3 * kTile + kTile / 2) * sizeof(float2) + kMaxPack * sizeof(TileSig);
static constexpr size_t kWinSmem = (size_t)(1 << kWinMaxLog) * sizeof(float2);
static constexpr size_t kPassSmem = (size_t)kPassElems * sizeof(float2);

// kernel tables indexed by level
using FwdKernel = void (*)(const FwdArgs);
static FwdKernel win_kernel(int level) {
  switch (level) {
    case 13: return k_fwd_window<12>;
    case 14: return k_fwd_window<13>;
    default: return nullptr;
  }
}
template <int QB>
static void pass_pair(int level, FwdKernel* c, FwdKernel* r) {
  if constexpr (QB <= 13) {
    if (level == QB + kColsLog + 1) {
      *c = k_fwd_cols<QB>;
      *r = k_fwd_rows<QB>;
      return;
    }
    pass_pair<QB + 1>(level, c, r);
  }
}

cudaError_t set_fwd_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_fwd_tile<kTileLog, kTileThreads>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
  for (int lv = 13; lv <= 14 && e == cudaSuccess; ++lv)
    e = cudaFuncSetAttribute(win_kernel(lv), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWinSmem);
  for (int lv = 15; lv <= 26 && e == cudaSuccess; ++lv) {
    FwdKernel c = nullptr, r = nullptr;
    pass_pair<2>(lv, &c, &r);
    e = cudaFuncSetAttribute(c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(r, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmem);
  }
  return e;
}

cudaError_t launch_fwd_tile(const FwdArgs& a, int grid, cudaStream_t s) {
  k_fwd_tile<kTileLog, kTileThreads><<<grid, kTileThreads, kTileSmem, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_fwd_tiny(const FwdArgs& a, int nsig_tiny, cudaStream_t s) {
  k_fwd_tiny<<<nsig_tiny, 64, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_fwd_window(const FwdArgs& a, int grid, cudaStream_t s) {
  FwdKernel k = win_kernel(a.level);
  if (!k) return cudaErrorInvalidValue;
  k<<<grid, kWinThreads, kWinSmem, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_fwd_cols(const FwdArgs& a, int grid, cudaStream_t s) {
  FwdKernel c = nullptr, r = nullptr;
  pass_pair<2>(a.level, &c, &r);
  if (!c) return cudaErrorInvalidValue;
  c<<<grid, kPassThreads, kPassSmem, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_fwd_rows(const FwdArgs& a, int grid, cudaStream_t s) {
  FwdKernel c = nullptr, r = nullptr;
  pass_pair<2>(a.level, &c, &r);
  if (!r) return cudaErrorInvalidValue;
  r<<<grid, kPassThreads, kPassSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mrdft
