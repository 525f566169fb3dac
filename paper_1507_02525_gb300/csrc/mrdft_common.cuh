// Device-side building blocks of the MrDFT library (sm_103a).
//
// Complex values are float2 (re, im), FP32, interleaved -- the complex64
// layout of the C ABI.  Forward transforms use the sign exp(-j 2 pi n k / L)
// of the DEF matrix E_{2^i} (Sec. 2 of Andreatto & Cariow); nothing is
// normalised.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

// Forces inlining of the small lambdas (static_for bodies, FFT sources and
// sinks) so the register arrays they touch never go to local memory.
#define MRDFT_INL __attribute__((always_inline))

namespace mrdft {

// ------------------------------------------------------------ complex math
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// a * (-j)
__device__ __forceinline__ float2 cmul_mj(float2 a) { return make_float2(a.y, -a.x); }
// a * (+j)
__device__ __forceinline__ float2 cmul_pj(float2 a) { return make_float2(-a.y, a.x); }

// ------------------------------------------------- compile-time twiddles
// cos(2 pi q / 64) for q = 0..16 as FP64 literals; every compile-time twiddle
// below is one of these (or its negation), rounded once to FP32.
__host__ __device__ constexpr double kcos64(int q) {
  return q == 0 ? 1.0 : q == 1 ? 0.99518472667219688624 : q == 2 ? 0.98078528040323044913
       : q == 3 ? 0.95694033573220886494 : q == 4 ? 0.92387953251128675613
       : q == 5 ? 0.88192126434835502971 : q == 6 ? 0.83146961230254523708
       : q == 7 ? 0.77301045336273696081 : q == 8 ? 0.70710678118654752440
       : q == 9 ? 0.63439328416364549822 : q == 10 ? 0.55557023301960222474
       : q == 11 ? 0.47139673682599764856 : q == 12 ? 0.38268343236508977173
       : q == 13 ? 0.29028467725446236764 : q == 14 ? 0.19509032201612826785
       : q == 15 ? 0.09801714032956060199 : 0.0;
}

// w_L^E = exp(-j 2 pi E / L) for L | 64, as compile-time constants.
template <int L, int E>
struct CTw {
  static constexpr int q = (E * (64 / L)) & 63;
  static constexpr int quad = q >> 4, r = q & 15;
  static constexpr double c = kcos64(r), s = kcos64(16 - r);
  static constexpr float re = (float)(quad == 0 ? c : quad == 1 ? -s : quad == 2 ? -c : s);
  static constexpr float im = (float)(quad == 0 ? -s : quad == 1 ? -c : quad == 2 ? s : c);
};

// a * w_L^E with the trivial twiddles (1, -j, -1, +j) reduced to swaps/negations
template <int L, int E>
__device__ __forceinline__ float2 cmul_ct(float2 a) {
  constexpr int q = CTw<L, E>::q;
  if constexpr (q == 0) return a;
  else if constexpr (q == 16) return cmul_mj(a);
  else if constexpr (q == 32) return make_float2(-a.x, -a.y);
  else if constexpr (q == 48) return cmul_pj(a);
  else return cmul(a, make_float2(CTw<L, E>::re, CTw<L, E>::im));
}

template <int V>
struct IC { static constexpr int value = V; };

template <int B, int E, int S = 1, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(IC<B>{});
    static_for<B + S, E, S>(f);
  }
}

// host-side compile-time loop (launch dispatch over template instantiations)
template <int B, int E, typename F>
inline void static_for_host(F&& f) {
  if constexpr (B < E) {
    f(IC<B>{});
    static_for_host<B + 1, E>(f);
  }
}

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }
__host__ __device__ constexpr int bitrevc(int v, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((v >> b) & 1) << (bits - 1 - b);
  return r;
}

template <int R, int LEN>
__device__ __forceinline__ void dif_stage(float2 (&v)[R]) {
  constexpr int half = LEN / 2;
  static_for<0, R, LEN>([&](auto S) MRDFT_INL {
    static_for<0, half>([&](auto J) MRDFT_INL {
      constexpr int s = decltype(S)::value, j = decltype(J)::value;
      float2 a = v[s + j], b = v[s + j + half];
      v[s + j] = cadd(a, b);
      v[s + j + half] = cmul_ct<LEN, j>(csub(a, b));
    });
  });
  if constexpr (LEN > 2) dif_stage<R, LEN / 2>(v);
}

// In-register DFT of length R (power of two, 1 <= R <= 64), natural order in
// and out: radix-2 decimation in frequency with compile-time twiddles, then a
// compile-time bit reversal (register renaming only).
template <int R>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
  if constexpr (R >= 2) {
    dif_stage<R, R>(v);
    float2 t[R];
    static_for<0, R>([&](auto K) MRDFT_INL {
      constexpr int k = decltype(K)::value;
      t[k] = v[bitrevc(k, ilog2c(R))];
    });
    static_for<0, R>([&](auto K) MRDFT_INL { v[decltype(K)::value] = t[decltype(K)::value]; });
  }
}

// Unnormalised inverse (sign +j): conj(DFT(conj(v))).
template <int R>
__device__ __forceinline__ void idft_reg(float2 (&v)[R]) {
#pragma unroll
  for (int k = 0; k < R; ++k) v[k].y = -v[k].y;
  dft_reg<R>(v);
#pragma unroll
  for (int k = 0; k < R; ++k) v[k].y = -v[k].y;
}

// ------------------------------------------------------ shared-memory maps
// Level / input tile buffers: rows of 16 complex (128 B); the 16-byte chunk c
// (two complex) of row r lives at chunk c ^ ((r ^ r>>3 ^ r>>6) & 7), so that
// lanes walking rows with any power-of-two stride up to 64 rows, or walking
// consecutive elements, hit distinct banks.  Index in float2 units; pairs
// (2q, 2q+1) stay adjacent, so 16-byte vector accesses remain valid.
__host__ __device__ __forceinline__ constexpr int swz128(int e) {
  const int r = e >> 4;
  return (r << 4) | ((((e >> 1) & 7) ^ ((r ^ (r >> 3) ^ (r >> 6)) & 7)) << 1) | (e & 1);
}
// swz128 is linear over XOR: for indices whose set bits do not overlap,
// swz128(a + b) = swz128(a) ^ swz128(b), so offsets known at compile time
// cost one XOR.
// FFT work buffers: XOR the low 4 index bits with bits 4..7 and 8..11 so that
// power-of-two strides up to 2^12 spread over all banks (8-byte elements).
__device__ __forceinline__ int swzf(int e) { return e ^ (((e >> 4) ^ (e >> 8)) & 15); }

// ------------------------------------------------------------ twiddle tables
// Device tables written once by the plan from FP64 host values rounded once:
//   tw13[e] = w_{2^14}^e, e < 2^14   (every FFT of length <= 2^14 and the
//                                       level twiddles w_{2^i}^n, i <= 14)
//   twlo[e] = w_{2^28}^e, e < 2^14 and twhi[e] = w_{2^28}^{e * 2^14},
//   e < 2^14: w_{2^28}^e = twhi[e >> 14] * twlo[e & 16383] for larger levels
//   (the product of two once-rounded values: one extra FP32 rounding).
struct Twiddles {
  const float2* tw13;
  const float2* twlo;
  const float2* twhi;
};
constexpr int kTwLog = 14;
constexpr int kTwBigLog = 28;
constexpr int kTwSplit = 14;

// w_{2^l}^e, l <= 13
__device__ __forceinline__ float2 tw_small(const Twiddles& T, int l, int e) {
  return __ldg(&T.tw13[(e << (kTwLog - l)) & ((1 << kTwLog) - 1)]);
}
// w_{2^l}^e for l <= 28: one table entry for l <= 13, else a product of two
__device__ __forceinline__ float2 tw_any(const Twiddles& T, int l, int64_t e) {
  if (l <= kTwLog) return tw_small(T, l, (int)(e & ((1 << l) - 1)));
  uint32_t q = (uint32_t)((e << (kTwBigLog - l)) & ((1 << kTwBigLog) - 1));
  return cmul(__ldg(&T.twhi[q >> kTwSplit]), __ldg(&T.twlo[q & ((1 << kTwSplit) - 1)]));
}

// ------------------------------------------------------------ async copies
// 16-byte global -> shared copy that bypasses registers (cp.async, L2 only).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
// 8-byte variant (goes through L1; destination only 8-byte aligned)
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N committed groups of this thread are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// L2 policies that keep lines resident ahead of normal and evict-first data
// (evict_last), or let them go first (evict_first), and an 8-byte store that
// carries one.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void st_l2_keep(float2* p, float2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;\n" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol)
               : "memory");
}

// Rows of 16 complex values (128 bytes), one row per thread of a warp,
// moved between registers and global memory so that every global access
// instruction covers 512 contiguous bytes instead of 16 bytes in each of 32
// lines: the warp's 32 rows pass through its own 4 KB of shared memory
// (`slice`, 16-byte aligned), 16-byte chunks XOR-swizzled by row, which is
// conflict-free both ways.  Chunk c = lane + 32 t of the transfer is chunk
// c & 7 of row c >> 3 of the warp.  Every lane of the warp calls.
//   store: row_ptr(r) = global address of row r (r < 32), 16-byte aligned
//   load:  chunk(r, q) = the float4 q (< 8) of row r, read from global memory
template <class RowPtr>
__device__ __forceinline__ void warp_rows16_store(const float2 (&v)[16], float2* slice, RowPtr&& row_ptr) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    *reinterpret_cast<float4*>(slice + (lane << 4) + ((q ^ (lane & 7)) << 1)) =
        make_float4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y);
  __syncwarp();
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int c = lane + 32 * t, r = c >> 3;
    __stcs(reinterpret_cast<float4*>(row_ptr(r)) + (c & 7),
           *reinterpret_cast<const float4*>(slice + (r << 4) + (((c & 7) ^ (r & 7)) << 1)));
  }
  __syncwarp();
}
template <class Chunk>
__device__ __forceinline__ void warp_rows16_load(float2 (&v)[16], float2* slice, Chunk&& chunk) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int c = lane + 32 * t, r = c >> 3;
    *reinterpret_cast<float4*>(slice + (r << 4) + (((c & 7) ^ (r & 7)) << 1)) = chunk(r, c & 7);
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 x = *reinterpret_cast<const float4*>(slice + (lane << 4) + ((q ^ (lane & 7)) << 1));
    v[2 * q] = make_float2(x.x, x.y);
    v[2 * q + 1] = make_float2(x.z, x.w);
  }
  __syncwarp();
}

// Invalidate one 128-byte L2 line without writing it back (dead scratch).
// p must be 128-byte aligned.
__device__ __forceinline__ void discard_l2(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(p) : "memory");
}

// ------------------------------------------------------------ status word
enum : int { kStatusOk = 0, kStatusTimeout = 5, kStatusBadItem = 6 };
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

}  // namespace mrdft
