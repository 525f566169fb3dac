// Shared-memory FFT engine used by every MrDFT kernel for the odd-bin DFTs
// (the F^(i) / R^(i) step of Sec. 3 of Andreatto & Cariow, there a radix-2
// decimation-in-frequency FFT with bit-reversed output).
//
// Here the same DFT runs as a constant-geometry decimation-in-time FFT (the
// transpose of a constant-geometry DIF factorisation): the input is read in
// digit-reversed order by the first pass, and every pass then reads 2^RB
// consecutive elements per group and writes them at a fixed stride L / 2^RB,
// so the last pass emits bins in natural order with consecutive lanes on
// consecutive bins.  All radices are 8 except the first pass (2, 4 or 8).
//
// Shared layout (no padding): element a of the work buffer lives at
// zlay<ZS>(a), an XOR permutation inside every aligned block of 16 elements
// chosen so that every pass's reads (8 consecutive elements per lane) and
// writes (lane-consecutive elements) are free of bank conflicts; ZS = log2 of
// the number of interleaved sequences for position-major storage (capped at
// 4), 0 for sequence-major storage (16-byte chunks permuted, read four
// chunks at a time).  The first pass reads its input through src();
// callers that stage the input in shared memory use an XOR layout stg<A,B>()
// there, picked per FFT shape so that the digit-reversed read of the first
// pass is conflict-free; the first pass then rewrites the buffer in place.
// Sequences are stored sequence-major (b * L + pos) or, SEQ_MINOR,
// position-major (pos * nseq + b, consecutive lanes on consecutive sequences).
#pragma once
#include "mrdft_common.cuh"

namespace mrdft {

// Work-buffer layouts.  Sequence-major storage (ZS = 0) permutes 16-byte
// chunks: element a of row a >> 4 (16 elements, 128 bytes) keeps its half
// a & 1 of chunk (a >> 1) & 7, and the chunk moves to chunk ^ (row & 7).  A
// pass's group of 8 consecutive elements then stays in 4 whole chunks, read
// with four 16-byte loads (every quarter-warp touches 8 distinct chunks), and
// lane-consecutive 8-byte stores stay conflict-free.  Position-major storage
// of 2^ZS interleaved sequences (ZS >= 1) XORs the low element bits.
template <int ZS>
__device__ __forceinline__ int zlay(int a) {
  if constexpr (ZS >= 4) return a;
  else if constexpr (ZS == 0) return a ^ (((a >> 4) & 7) << 1);
  else return a ^ (((a >> (3 + ZS)) & ((1 << (4 - ZS)) - 1)) << ZS);
}
// staging layout: the low 4 index bits XOR bits A.. (and B.., B > 0)
template <int A, int B>
__device__ __forceinline__ int stg(int e) {
  if constexpr (B == 0) return e ^ ((e >> A) & 15);
  else return e ^ (((e >> A) ^ (e >> B)) & 15);
}
// two pad elements per 32 (level buffers: lane-consecutive 8-byte reads and
// window-strided accesses stay conflict-free, and every pair (2k, 2k+1) stays
// adjacent and 16-byte aligned, so a bin pair moves as one 16-byte access)
__device__ __forceinline__ int pad16(int a) { return a + ((a >> 5) << 1); }
__host__ __device__ constexpr int pad16_size(int n) { return n + n / 16; }

// Twiddles w_{2^TB}^e from a quarter-wave table q[r] = w_{2^TB}^r, r < 2^(TB-2)
// (FP64 values rounded once), using w^(r + s 2^(TB-2)) = (-j)^s w^r.  The
// table is stored padded (entry r at r + r/16 + r/256) so that lanes reading
// exponents with a power-of-two stride hit distinct banks.
struct TwQ {
  const float2* q;
  int TB;
};
__device__ __forceinline__ int twq_pad(int r) { return r + (r >> 4) + (r >> 8); }
__host__ __device__ constexpr int twq_size(int TB) {
  return (1 << (TB - 2)) + (TB >= 6 ? 1 << (TB - 6) : 0) + (TB >= 10 ? 1 << (TB - 10) : 0) + 1;
}
__device__ __forceinline__ float2 twq(const TwQ& t, int e) {
  const int qb = t.TB - 2;
  const float2 w = t.q[twq_pad(e & ((1 << qb) - 1))];
  // times (-j)^s for the quadrant s, branch-free: swap re/im for odd s, then
  // sign flips (re for s = 2, 3; im for s = 1, 2)
  const int s = (e >> qb) & 3;
  const float a = (s & 1) ? w.y : w.x;
  const float b = (s & 1) ? w.x : w.y;
  const unsigned sre = (unsigned)(s & 2) << 30;
  const unsigned sim = (unsigned)((s ^ (s >> 1)) & 1) << 31;
  return make_float2(__uint_as_float(__float_as_uint(a) ^ sre), __uint_as_float(__float_as_uint(b) ^ sim));
}
// w_{2^l}^e for l <= TB
__device__ __forceinline__ float2 twq_l(const TwQ& t, int l, int e) { return twq(t, e << (t.TB - l)); }

// The same twiddles read straight from the global table w_{2^14}^e (through
// L1), for kernels that keep no per-CTA copy in shared memory.
struct TwG {
  const float2* t14;
  int TB;
};
__device__ __forceinline__ float2 twq(const TwG& t, int e) {
  return __ldg(&t.t14[(e << (kTwLog - t.TB)) & ((1 << kTwLog) - 1)]);
}
__device__ __forceinline__ float2 twq_l(const TwG& t, int l, int e) { return twq(t, e << (t.TB - l)); }

// A two-level table in shared memory: w_{2^TB}^e = hi[e >> 6] lo[e & 63]
// (hi[j] = w^(64 j), lo[k] = w^k, both FP64 values rounded once; one extra
// rounding in the product), 2^(TB-6) + 64 entries -- 1 KB for TB = 12 instead
// of the quarter-wave table's 8.7 KB.  Entries are padded (k + k / 16) so that
// lanes reading exponents with a power-of-two stride hit distinct banks.
struct TwS {
  const float2* hi;
  const float2* lo;
  int TB;
};
__host__ __device__ constexpr int tws_size(int TB) { return (1 << (TB - 6)) + ((1 << (TB - 6)) >> 4) + 64 + 4; }
__device__ __forceinline__ int tws_pad(int k) { return k + (k >> 4); }
__device__ __forceinline__ float2 twq(const TwS& t, int e) {
  e &= (1 << t.TB) - 1;
  return cmul(t.hi[tws_pad(e >> 6)], t.lo[tws_pad(e & 63)]);
}
__device__ __forceinline__ float2 twq_l(const TwS& t, int l, int e) { return twq(t, e << (t.TB - l)); }

// w^(k * step), k = 0 .. R-1, from one table entry (w^step) and products of
// it (at most four extra roundings, far inside the FP32 error budget): one
// lookup instead of log2(R) keeps the table-index and quadrant arithmetic off
// the critical path of every butterfly group.
__device__ __forceinline__ float2 csq(float2 a) { return make_float2(fmaf(a.x, a.x, -a.y * a.y), 2.f * a.x * a.y); }
template <int R, class TW>
__device__ __forceinline__ void twiddle_set(const TW& tw, int step, float2 (&w)[R]) {
  w[0] = make_float2(1.f, 0.f);
  if constexpr (R >= 2) w[1] = twq(tw, step);
  if constexpr (R >= 4) {
    w[2] = csq(w[1]);
    w[3] = cmul(w[1], w[2]);
  }
  if constexpr (R >= 8) {
    w[4] = csq(w[2]);
    w[5] = cmul(w[4], w[1]);
    w[6] = csq(w[3]);
    w[7] = cmul(w[4], w[3]);
  }
}

// reverse the d low octal digits of v
__device__ __forceinline__ int drev8(int v, int d) {
  int r = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (i < d) r |= ((v >> (3 * i)) & 7) << (3 * (d - 1 - i));
  return r;
}

// First-pass group source over input staged in the stg<A, B> layout at index
// (n << ns) | (b << bs) (n and b in disjoint bit fields): the R inputs
// n0 + r 2^LRB of a group share one layout computation and take an XOR each
// (stg is linear over XOR, and r 2^LRB lies above n0 < 2^LRB).
template <int A, int B>
struct StgGroup {
  const float2* S;
  int ns, bs;
  template <class V, class RBc>
  __device__ __forceinline__ void operator()(int b, int n0, int LRB, V& v, RBc) const {
    constexpr int R = 1 << RBc::value;
    const int e0 = stg<A, B>((n0 << ns) | (b << bs));
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = S[e0 ^ stg<A, B>((r << LRB) << ns)];
  }
};

// One pass of the constant-geometry DIT FFT.
//   LB: log2 sequence length; nseq_log: log2 number of sequences;
//   RB: log2 radix of this pass; SH: 3 * (DIF pass index) -- the twiddle of
//   input r of group g is w_M^((g >> SH) r) with M = L >> SH; P: pass count.
//   FIRST: inputs come from src(b, n) in natural index n (the digit reversal
//   is folded into the index); LAST: outputs go to sink(slot, b, k, v) with
//   bin k natural; PRE: pre(slot, b, k) runs for every output bin --
//   kPreBarrier: before the barrier that separates every read of this pass
//   from the sink's writes (the caller may read what the sink overwrites);
//   kPreGroup: after each group's DFT, for the group's R bins, before their
//   sinks (global reads issued in one batch per group, few registers held);
//   kPreHalf: the same in batches of R/2 bins (fewer registers still).
// Every thread loads all its groups before the pass's barrier, so the pass is
// in place; PTS bounds the points per thread (NT * PTS >= points per pass).
constexpr int kPreNone = 0, kPreBarrier = 1, kPreGroup = 2, kPreHalf = 3;

template <int RB, int NT, int PTS, bool SEQ_MINOR, bool FIRST, bool LAST, int PRE, int ZS, bool GSRC, class TW,
          class Src, class Pre, class Sink>
__device__ __forceinline__ void cg_pass(float2* __restrict__ Z, int LB, int nseq_log, int SH, int P, const TW& tw,
                                        Src&& src, Pre&& pre, Sink&& sink) {
  constexpr int R = 1 << RB;
  constexpr int GMAX = (PTS >> RB) > 0 ? (PTS >> RB) : 1;  // groups per thread
  const int LRB = LB - RB;                      // log2(L / R): groups per sequence
  const int ngroups = 1 << (nseq_log + LRB);
  const int tid = threadIdx.x;
  float2 v[GMAX][R];
#pragma unroll
  for (int j = 0; j < GMAX; ++j) {
    const int G = tid + j * NT;
    if (G < ngroups) {
      int b, g;
      if constexpr (SEQ_MINOR) {
        b = G & ((1 << nseq_log) - 1);
        g = G >> nseq_log;
      } else {
        b = G >> LRB;
        g = G & ((1 << LRB) - 1);
      }
      if constexpr (FIRST) {
        // position R g + r holds natural index drev8(g) + (L / R) r
        const int n0 = drev8(g, P - 1);
        if constexpr (GSRC) {
          src(b, n0, LRB, v[j], IC<RB>{});  // all R inputs n0 + (L / R) r at once
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) v[j][r] = src(b, n0 + (r << LRB));
        }
      } else {
        const int a0 = SEQ_MINOR ? (((g << RB) << nseq_log) + b) : ((b << LB) + (g << RB));
        // zlay is linear over XOR and the element offsets occupy bits a0
        // leaves clear: one layout computation per group
        const int z0 = zlay<ZS>(a0);
        if constexpr (!SEQ_MINOR && ZS == 0 && R == 8) {
          // 8 consecutive elements = chunks c0 .. c0 + 3 of row a0 >> 4 (c0 = 0 or 4)
          const float2* rowp = Z + ((a0 >> 4) << 4);
          const int x = (a0 >> 4) & 7, c0 = (a0 >> 1) & 7;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 t = *reinterpret_cast<const float4*>(rowp + (((c0 + q) ^ x) << 1));
            v[j][2 * q] = make_float2(t.x, t.y);
            v[j][2 * q + 1] = make_float2(t.z, t.w);
          }
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) v[j][r] = Z[z0 ^ zlay<ZS>(SEQ_MINOR ? (r << nseq_log) : r)];
        }
      }
      const int tg = g >> SH;
      if (tg != 0) {
        float2 w[R];
        twiddle_set<R>(tw, tg << (tw.TB - (LB - SH)), w);  // w_M^(tg r)
#pragma unroll
        for (int r = 1; r < R; ++r) v[j][r] = cmul(v[j][r], w[r]);
      }
      if constexpr (LAST && PRE == kPreBarrier) {
#pragma unroll
        for (int k = 0; k < R; ++k) pre(j * R + k, b, g + (k << LRB));
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < GMAX; ++j) {
    const int G = tid + j * NT;
    if (G >= ngroups) continue;
    int b, g;
    if constexpr (SEQ_MINOR) {
      b = G & ((1 << nseq_log) - 1);
      g = G >> nseq_log;
    } else {
      b = G >> LRB;
      g = G & ((1 << LRB) - 1);
    }
    dft_reg<R>(v[j]);
    if constexpr (LAST) {
      if constexpr (PRE == kPreHalf && R >= 2) {
#pragma unroll
        for (int k0 = 0; k0 < R; k0 += R / 2) {
#pragma unroll
          for (int k = k0; k < k0 + R / 2; ++k) pre(j * R + k, b, g + (k << LRB));
#pragma unroll
          for (int k = k0; k < k0 + R / 2; ++k) sink(j * R + k, b, g + (k << LRB), v[j][k]);
        }
      } else {
        if constexpr (PRE == kPreGroup || PRE == kPreHalf) {
#pragma unroll
          for (int k = 0; k < R; ++k) pre(j * R + k, b, g + (k << LRB));
        }
#pragma unroll
        for (int k = 0; k < R; ++k) sink(j * R + k, b, g + (k << LRB), v[j][k]);
      }
    } else {
      const int a0 = SEQ_MINOR ? ((g << nseq_log) + b) : ((b << LB) + g);
      const int z0 = zlay<ZS>(a0);  // as for the loads: offsets k 2^LRB lie above g's bits
#pragma unroll
      for (int k = 0; k < R; ++k) Z[z0 ^ zlay<ZS>(SEQ_MINOR ? ((k << LRB) << nseq_log) : (k << LRB))] = v[j][k];
    }
  }
}

// Full forward DFT of 2^nseq_log sequences of runtime length 2^LB
// (LBMIN <= LB <= LBMAX, LB >= 1).  Starts with a barrier-free read of src,
// ends after the sink; synchronises internally.  The caller synchronises
// before reusing Z or reading what the sink wrote.
//   src(b, n) -> float2, or with GSRC src(b, n0, LRB, float2 (&v)[R], IC<RB>)
//   filling the R first-pass inputs n0 + (r << LRB) of a group at once;
//   pre(slot, b, k) (PRE != kPreNone);  sink(slot, b, k, v).
template <int LBMIN, int LBMAX, int NT, int PTS, bool SEQ_MINOR, int PRE, int ZS = 0, bool GSRC = false,
          class TW, class Src, class Pre, class Sink>
__device__ __forceinline__ void cg_fft(float2* __restrict__ Z, int LB, int nseq_log, const TW& tw, Src&& src,
                                       Pre&& pre, Sink&& sink) {
  const int P = (LB + 2) / 3;
  const int r0 = LB - 3 * (P - 1);  // radix bits of the first (remainder) pass
  if (P == 1) {
    static_for<1, 4>([&](auto RR) MRDFT_INL {
      constexpr int rb = decltype(RR)::value;
      if constexpr (rb >= LBMIN && rb <= LBMAX)
        if (r0 == rb)
          cg_pass<rb, NT, PTS, SEQ_MINOR, true, true, PRE, ZS, GSRC>(Z, LB, nseq_log, LB, 1, tw, src, pre, sink);
    });
    return;
  }
  if constexpr (LBMAX >= 4) {
    static_for<1, 4>([&](auto RR) MRDFT_INL {
      constexpr int rb = decltype(RR)::value;
      if (r0 == rb)
        cg_pass<rb, NT, PTS, SEQ_MINOR, true, false, kPreNone, ZS, GSRC>(Z, LB, nseq_log, 3 * (P - 1), P, tw, src, pre, sink);
    });
#pragma unroll 1
    for (int p = P - 2; p >= 1; --p) {
      __syncthreads();
      cg_pass<3, NT, PTS, SEQ_MINOR, false, false, kPreNone, ZS, false>(Z, LB, nseq_log, 3 * p, P, tw, src, pre, sink);
    }
    __syncthreads();
    cg_pass<3, NT, PTS, SEQ_MINOR, false, true, PRE, ZS, false>(Z, LB, nseq_log, 0, P, tw, src, pre, sink);
  }
}

// Fill a quarter-wave table of w_{2^TB} in shared memory from the global
// FP64-rounded-once table w_{2^14}^e (TB <= 14).
template <int NT>
__device__ __forceinline__ void load_twq(float2* q, int TB, const Twiddles& T) {
  const int n = 1 << (TB - 2);
  for (int r = threadIdx.x; r < n; r += NT) q[twq_pad(r)] = __ldg(&T.tw13[r << (kTwLog - TB)]);
}

// Fill a two-level table (TwS) of w_{2^TB} at q: hi first, then lo.
template <int NT>
__device__ __forceinline__ TwS load_tws(float2* q, int TB, const Twiddles& T) {
  const int nh = 1 << (TB - 6);
  float2* hi = q;
  float2* lo = q + tws_pad(nh - 1) + 1;
  for (int r = threadIdx.x; r < nh + 64; r += NT) {
    if (r < nh) hi[tws_pad(r)] = __ldg(&T.tw13[(r << 6) << (kTwLog - TB)]);
    else lo[tws_pad(r - nh)] = __ldg(&T.tw13[(r - nh) << (kTwLog - TB)]);
  }
  return TwS{hi, lo, TB};
}

// no-op pre-sink
struct NoPre {
  __device__ __forceinline__ void operator()(int, int, int) const {}
};

}  // namespace mrdft
