// Shared-memory FFT engine used by every MrDFT kernel for the odd-bin DFTs
// (the F^(i) / R^(i) step of Sec. 3 of Andreatto & Cariow, there a radix-2
// decimation-in-frequency FFT with bit-reversed output).  Here the same DFT
// is taken in radix-16 passes (remainder radix last), in place, over `nseq`
// independent sequences of length L = 2^LB held in one shared buffer; the
// bit-reversed order is undone by the thread mapping of the last pass, so the
// sink receives bins in natural order with consecutive lanes on consecutive
// bins.
#pragma once
#include "mrdft_common.cuh"

namespace mrdft {

// reverse D hexadecimal digits of v
template <int D>
__device__ __forceinline__ int drev16(int v) {
  if constexpr (D <= 1) return v;
  else if constexpr (D == 2) return ((v & 15) << 4) | (v >> 4);
  else if constexpr (D == 3) return ((v & 15) << 8) | (v & 0xF0) | (v >> 8);
  else return ((v & 15) << 12) | ((v & 0xF0) << 4) | ((v >> 4) & 0xF0) | (v >> 12);
}

// In-place forward DFT of nseq = 2^nseq_log sequences of length 2^LB.
//   Z      : work buffer, element p of sequence b at Z[swzf(b * L + p)]
//   src    : float2 src(int b, int n) -- input sample n of sequence b (first pass)
//   sink   : void sink(int b, int k, float2 v) -- bin k (natural order) of b
//   SEQ_FAST: consecutive threads walk sequences first (for sinks that store
//            one bin of many sequences contiguously), else bins first.
// All NT threads of the block must call it; it synchronises between passes
// but not before the first or after the last.
template <int LB, int NT, bool SEQ_FAST, class Src, class Sink>
__device__ __forceinline__ void fft_inplace(float2* __restrict__ Z, int nseq_log,
                                            const Twiddles& T, Src&& src, Sink&& sink) {
  constexpr int L = 1 << LB;
  constexpr int P = (LB + 3) / 4;
  const int tid = threadIdx.x;
  static_for<0, P>([&](auto PP) MRDFT_INL {
    constexpr int p = decltype(PP)::value;
    constexpr int rb = (p < LB / 4) ? 4 : (LB % 4);
    constexpr int R = 1 << rb;
    constexpr int MB = LB - 4 * p;  // log2 of the sub-problem length at this pass
    constexpr int M = 1 << MB;
    constexpr int MR = M / R;
    constexpr int GPT = 16 / R;     // groups per thread per round (16 points)
    constexpr int LR_LOG = LB - rb; // log2(L / R)
    constexpr bool FIRST = (p == 0), LAST = (p == P - 1);
    const int ngroups = 1 << (nseq_log + LR_LOG);
#pragma unroll 1
    for (int base = 0; base < ngroups; base += NT * GPT) {
      float2 v[GPT][R];
      int gb[GPT], gr[GPT];
#pragma unroll
      for (int j = 0; j < GPT; ++j) {
        const int g = base + tid + j * NT;
        int b, r;
        if constexpr (SEQ_FAST) {
          b = g & ((1 << nseq_log) - 1);
          r = g >> nseq_log;
        } else {
          b = g >> LR_LOG;
          r = g & ((1 << LR_LOG) - 1);
        }
        gb[j] = b;
        gr[j] = r;
        if (g < ngroups) {
          // sub-problem u, offset n2 inside it
          int u, n2;
          if constexpr (LAST && P > 1) {
            u = drev16<P - 1>(r);
            n2 = 0;
          } else {
            u = r / MR;
            n2 = r % MR;
          }
          const int pos0 = u * M + n2;
#pragma unroll
          for (int n1 = 0; n1 < R; ++n1) {
            const int pos = pos0 + n1 * MR;
            if constexpr (FIRST) v[j][n1] = src(b, pos);
            else v[j][n1] = Z[swzf((b << LB) + pos)];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < GPT; ++j) {
        const int g = base + tid + j * NT;
        if (g >= ngroups) continue;
        dft_reg<R>(v[j]);
        if constexpr (!LAST) {
          const int n2 = gr[j] % MR;
          if (n2 != 0) {
#pragma unroll
            for (int k1 = 1; k1 < R; ++k1) v[j][k1] = cmul(v[j][k1], tw_small(T, MB, n2 * k1));
          }
          const int u = gr[j] / MR;
          const int pos0 = u * M + n2;
#pragma unroll
          for (int k1 = 0; k1 < R; ++k1) Z[swzf((gb[j] << LB) + pos0 + k1 * MR)] = v[j][k1];
        } else {
          // bins: k = l + (L / R) * k1 with l = r (digit-reversed sub-problem)
#pragma unroll
          for (int k1 = 0; k1 < R; ++k1) sink(gb[j], gr[j] + k1 * (L / R), v[j][k1]);
        }
      }
    }
    if constexpr (!LAST) __syncthreads();
  });
}

}  // namespace mrdft
