/*
 * FP64 CPU oracle for the multiresolution discrete Fourier transform (MrDFT).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, table or helper with the CUDA
 * library; the two are compared, never combined.
 *
 * Paper: B. Andreatto, A. Cariow, "An algorithm for fast computation of the
 * multiresolution discrete Fourier transform", arXiv:1507.02525.
 *
 * Definition (Sec. 2, Eq. 1, with the DEF matrix E_{2^i} of Sec. 2):
 *   for a signal x of length N = 2^m, level i = 1..m, window w = 0..N/2^i-1,
 *   bin k = 0..2^i-1:
 *       Y^(i)[w*2^i + k] = sum_{n=0}^{2^i-1} x[w*2^i + n] * exp(-j*2*pi*n*k/2^i).
 *   The printed identity factor I_{2^{m-1}} in Eq. 1 is read as I_{2^{m-i}}
 *   (N/2^i windows per level), the only reading that makes each level N x N.
 *   Output layout: levels ascending, windows ascending, bins in natural order
 *   (after the permutation Gamma of Sec. 3).  Complex numbers are interleaved
 *   (re, im) doubles.
 *
 * Adjoint: the conjugate transpose of Eq. 1, x_bar = sum_i (I (x) E_{2^i})^H g_i,
 * an unnormalised inverse DFT per window, summed over levels.
 *
 * Functions:
 *   mro_forward_direct   - Eq. 1 evaluated term by term (O(N * 2^i) per level).
 *   mro_forward_fft      - the same result through a per-window iterative
 *                          radix-2 FFT (textbook decimation in time), which is
 *                          NOT the paper's level recursion.
 *   mro_forward_level_fft- one level of the above (for full-size checks).
 *   mro_bin              - one output bin, by the direct sum (sampled checks).
 *   mro_adjoint_direct / mro_adjoint_fft - the adjoint, dense / per-window FFT.
 *   mro_rationalized     - the paper's rationalised algorithm, Eq. 4, executed
 *                          in its printed order (P, A, D, F per iteration, then
 *                          Gamma) with every complex multiplication and addition
 *                          counted, for the operation counts of Eqs. 6 and 7.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MRO_TWO_PI 6.283185307179586476925286766559

static int g_threads = 0; /* 0 = OpenMP default */

int mro_set_num_threads(int n) {
  g_threads = n;
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#endif
  return 0;
}

int mro_num_threads(void) {
#ifdef _OPENMP
  return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
  return 1;
#endif
}

/* exp(-j 2 pi q / L) for integer q, evaluated in FP64. */
static void mro_root(int64_t q, int64_t L, double *re, double *im) {
  double a = -MRO_TWO_PI * (double)(q % L) / (double)L;
  *re = cos(a);
  *im = sin(a);
}

/* Table of exp(-j 2 pi q / L), q < L; caller frees. */
static double *mro_root_table(int64_t L) {
  double *t = (double *)malloc(sizeof(double) * 2 * (size_t)L);
  if (!t) return NULL;
  for (int64_t q = 0; q < L; ++q) mro_root(q, L, &t[2 * q], &t[2 * q + 1]);
  return t;
}

/* ---------------------------------------------------------------- direct */

/* Eq. 1, level i only: y gets N complex values. */
static int mro_level_direct(const double *x, int m, int i, double *y) {
  const int64_t N = (int64_t)1 << m, L = (int64_t)1 << i;
  double *w = mro_root_table(L);
  if (!w) return 1;
#pragma omp parallel for schedule(static)
  for (int64_t win = 0; win < N / L; ++win) {
    const double *xw = x + 2 * win * L;
    double *yw = y + 2 * win * L;
    for (int64_t k = 0; k < L; ++k) {
      double sr = 0.0, si = 0.0;
      for (int64_t n = 0; n < L; ++n) {
        int64_t q = (n * k) & (L - 1); /* n*k mod 2^i */
        double wr = w[2 * q], wi = w[2 * q + 1];
        double xr = xw[2 * n], xi = xw[2 * n + 1];
        sr += xr * wr - xi * wi;
        si += xr * wi + xi * wr;
      }
      yw[2 * k] = sr;
      yw[2 * k + 1] = si;
    }
  }
  free(w);
  return 0;
}

int mro_forward_direct(const double *x, int m, double *y) {
  if (m < 1 || m > 30) return 1;
  const int64_t N = (int64_t)1 << m;
  for (int i = 1; i <= m; ++i)
    if (mro_level_direct(x, m, i, y + 2 * (int64_t)(i - 1) * N)) return 2;
  return 0;
}

/* One output bin by the direct sum; level i (1-based), position p in [0,N). */
int mro_bin(const double *x, int m, int i, int64_t p, double *out) {
  if (m < 1 || m > 30 || i < 1 || i > m) return 1;
  const int64_t L = (int64_t)1 << i;
  const int64_t win = p / L, k = p % L;
  const double *xw = x + 2 * win * L;
  double sr = 0.0, si = 0.0;
  for (int64_t n = 0; n < L; ++n) {
    double wr, wi;
    mro_root((n * k) & (L - 1), L, &wr, &wi);
    sr += xw[2 * n] * wr - xw[2 * n + 1] * wi;
    si += xw[2 * n] * wi + xw[2 * n + 1] * wr;
  }
  out[0] = sr;
  out[1] = si;
  return 0;
}

/* ------------------------------------------------------------------- FFT */

static int64_t mro_bitrev(int64_t v, int bits) {
  int64_t r = 0;
  for (int b = 0; b < bits; ++b) r |= ((v >> b) & 1) << (bits - 1 - b);
  return r;
}

/* In-place iterative radix-2 decimation-in-time FFT of length L = 2^bits on
 * one window (after a bit-reversal copy), with sign -1 (forward) or +1
 * (unnormalised inverse).  roots[q] = exp(-j 2 pi q / L). */
static void mro_fft_window(const double *in, double *out, int bits,
                           const double *roots, int inverse) {
  const int64_t L = (int64_t)1 << bits;
  for (int64_t n = 0; n < L; ++n) {
    int64_t r = mro_bitrev(n, bits);
    out[2 * r] = in[2 * n];
    out[2 * r + 1] = in[2 * n + 1];
  }
  for (int64_t len = 2; len <= L; len <<= 1) {
    const int64_t half = len >> 1, step = L / len;
    for (int64_t s = 0; s < L; s += len) {
      for (int64_t j = 0; j < half; ++j) {
        double wr = roots[2 * j * step];
        double wi = roots[2 * j * step + 1];
        if (inverse) wi = -wi;
        double *u = out + 2 * (s + j), *v = out + 2 * (s + j + half);
        double tr = v[0] * wr - v[1] * wi;
        double ti = v[0] * wi + v[1] * wr;
        v[0] = u[0] - tr;
        v[1] = u[1] - ti;
        u[0] += tr;
        u[1] += ti;
      }
    }
  }
}

int mro_forward_level_fft(const double *x, int m, int i, double *y) {
  if (m < 1 || m > 30 || i < 1 || i > m) return 1;
  const int64_t N = (int64_t)1 << m, L = (int64_t)1 << i;
  double *w = mro_root_table(L);
  if (!w) return 2;
#pragma omp parallel for schedule(static)
  for (int64_t win = 0; win < N / L; ++win)
    mro_fft_window(x + 2 * win * L, y + 2 * win * L, i, w, 0);
  free(w);
  return 0;
}

int mro_forward_fft(const double *x, int m, double *y) {
  if (m < 1 || m > 30) return 1;
  const int64_t N = (int64_t)1 << m;
  for (int i = 1; i <= m; ++i)
    if (mro_forward_level_fft(x, m, i, y + 2 * (int64_t)(i - 1) * N)) return 2;
  return 0;
}

/* --------------------------------------------------------------- adjoint */

int mro_adjoint_direct(const double *gy, int m, double *gx) {
  if (m < 1 || m > 30) return 1;
  const int64_t N = (int64_t)1 << m;
  memset(gx, 0, sizeof(double) * 2 * (size_t)N);
  for (int i = 1; i <= m; ++i) {
    const int64_t L = (int64_t)1 << i;
    const double *g = gy + 2 * (int64_t)(i - 1) * N;
    double *w = mro_root_table(L);
    if (!w) return 2;
#pragma omp parallel for schedule(static)
    for (int64_t win = 0; win < N / L; ++win) {
      for (int64_t n = 0; n < L; ++n) {
        double sr = 0.0, si = 0.0;
        for (int64_t k = 0; k < L; ++k) {
          int64_t q = (n * k) & (L - 1);
          double wr = w[2 * q], wi = -w[2 * q + 1]; /* conj */
          double gr = g[2 * (win * L + k)], gi = g[2 * (win * L + k) + 1];
          sr += gr * wr - gi * wi;
          si += gr * wi + gi * wr;
        }
        gx[2 * (win * L + n)] += sr;
        gx[2 * (win * L + n) + 1] += si;
      }
    }
    free(w);
  }
  return 0;
}

int mro_adjoint_fft(const double *gy, int m, double *gx) {
  if (m < 1 || m > 30) return 1;
  const int64_t N = (int64_t)1 << m;
  memset(gx, 0, sizeof(double) * 2 * (size_t)N);
  double *tmp = (double *)malloc(sizeof(double) * 2 * (size_t)N);
  if (!tmp) return 2;
  for (int i = 1; i <= m; ++i) {
    const int64_t L = (int64_t)1 << i;
    const double *g = gy + 2 * (int64_t)(i - 1) * N;
    double *w = mro_root_table(L);
    if (!w) { free(tmp); return 2; }
#pragma omp parallel for schedule(static)
    for (int64_t win = 0; win < N / L; ++win)
      mro_fft_window(g + 2 * win * L, tmp + 2 * win * L, i, w, 1);
    free(w);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < 2 * N; ++n) gx[n] += tmp[n];
  }
  free(tmp);
  return 0;
}

/* --------------------------------------------- rationalised, Eq. 4, counted */

/*
 * Executes the paper's procedure of Sec. 3 (Eq. 4) one iteration at a time and
 * counts operations.  The state is kept as the level blocks the matrices act
 * on; no matrix is formed.
 *
 *   P^(1): m copies of X (the x copy that each later iteration consumes).
 *   A^(1) = (I (x) H_2): pairs (x0 + x1, x0 - x1) -> level 1 (internal order).
 *   D^(1), F^(1): identities; D~^(1) = I_1 (+) w_2^0 is one trivial
 *         multiplication per pair and is counted as such (Eq. 6 at i = 1).
 *   Iteration i >= 2, per window of 2^i (h = 2^(i-1)):
 *     P^(i): duplicates the level-(i-1) block next to the i-th x copy.
 *     A^(i) = [U | V]: U (Eq. 2) puts the element-wise sum of the two child
 *            blocks (level i-1, internal order) in the upper half; V (Eq. 3)
 *            puts a - b of the time-domain halves of the x copy in the lower
 *            half.
 *     D^(i): lower half n-th element times w_{2^i}^n, n < h.
 *     F^(i): lower half through R = (W^(i-1) S^(i-1)) ... (W^(1) S^(1)) with
 *            S^(j) = I_{2^(j-1)} (x) (H_2 (x) I_{2^(i-j-1)}) and
 *            W^(j) = I_{2^(j-1)} (x) [I_{2^(i-j-1)} (+) diag(w_{2^(i-j)}^0..)].
 *   Gamma: per window, T_{2^i} with t_{k, rev(k)} = 1 ("binary inversion" read
 *          as bit reversal over i bits) brings bins to natural order.
 *
 * counts (if non-NULL) receives 3*m int64: for each level i (index i-1),
 *   [0] complex multiplications including trivial twiddles (Eq. 6),
 *   [1] multiplications by a twiddle other than 1 and -j (Eq. 7),
 *   [2] complex additions/subtractions.
 * y (if non-NULL) receives the natural-order result, 2*m*N doubles.
 * compute = 0 walks the same loops and counts without doing arithmetic.
 */
int mro_rationalized(const double *x, int m, double *y, int64_t *counts,
                     int compute) {
  if (m < 1 || m > 30) return 1;
  const int64_t N = (int64_t)1 << m;
  double *prev = NULL, *cur = NULL, *root = NULL;
  if (compute) {
    prev = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    cur = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    root = mro_root_table(N > 1 ? N : 2);
    if (!prev || !cur || !root) { free(prev); free(cur); free(root); return 2; }
  }
  if (counts) memset(counts, 0, sizeof(int64_t) * 3 * (size_t)m);

  /* twiddle w_{2^l}^e as an index into the root table of length N */
#define TW_RE(l, e) root[2 * (((int64_t)(e) << (m - (l))) & (N - 1))]
#define TW_IM(l, e) root[2 * (((int64_t)(e) << (m - (l))) & (N - 1)) + 1]
  /* trivial twiddle: w_L^0 = 1 or w_L^{L/4} = -j */
#define TRIVIAL(L, e) ((e) == 0 || ((L) >= 4 && (e) == (L) / 4))

  for (int i = 1; i <= m; ++i) {
    const int64_t L = (int64_t)1 << i, h = L >> 1;
    int64_t mul = 0, mul_nt = 0, add = 0;
    for (int64_t win = 0; win < N / L; ++win) {
      const int64_t s = win * L;
      if (i == 1) {
        /* A^(1) = H_2 on the x copy, then D~^(1) = I_1 (+) w_2^0 */
        if (compute) {
          double a0 = x[2 * s], a1 = x[2 * s + 1];
          double b0 = x[2 * s + 2], b1 = x[2 * s + 3];
          cur[2 * s] = a0 + b0;
          cur[2 * s + 1] = a1 + b1;
          cur[2 * s + 2] = a0 - b0; /* times w_2^0 = 1 */
          cur[2 * s + 3] = a1 - b1;
        }
        add += 2;
        mul += 1; /* trivial (w_2^0) */
        continue;
      }
      /* A^(i): U (Eq. 2) on the duplicated level-(i-1) block */
      for (int64_t n = 0; n < h; ++n) {
        if (compute) {
          cur[2 * (s + n)] = prev[2 * (s + n)] + prev[2 * (s + h + n)];
          cur[2 * (s + n) + 1] = prev[2 * (s + n) + 1] + prev[2 * (s + h + n) + 1];
        }
        add += 1;
      }
      /* A^(i): V (Eq. 3) on the x copy, lower half: a - b */
      for (int64_t n = 0; n < h; ++n) {
        if (compute) {
          cur[2 * (s + h + n)] = x[2 * (s + n)] - x[2 * (s + h + n)];
          cur[2 * (s + h + n) + 1] = x[2 * (s + n) + 1] - x[2 * (s + h + n) + 1];
        }
        add += 1;
      }
      /* D^(i): lower half times w_{2^i}^n */
      for (int64_t n = 0; n < h; ++n) {
        if (compute) {
          double vr = cur[2 * (s + h + n)], vi = cur[2 * (s + h + n) + 1];
          double wr = TW_RE(i, n), wi = TW_IM(i, n);
          cur[2 * (s + h + n)] = vr * wr - vi * wi;
          cur[2 * (s + h + n) + 1] = vr * wi + vi * wr;
        }
        mul += 1;
        if (!TRIVIAL(L, n)) mul_nt += 1;
      }
      /* F^(i): R^(i) = prod_{j = i-1 .. 1} W^(j) S^(j), applied S^(1) first */
      double *v = compute ? cur + 2 * (s + h) : NULL;
      for (int j = 1; j <= i - 1; ++j) {
        const int64_t blk = (int64_t)1 << (i - j);     /* H_2 (x) I_{blk/2} */
        const int64_t half = blk >> 1;
        for (int64_t b = 0; b < ((int64_t)1 << (j - 1)); ++b) {
          const int64_t o = b * blk;
          /* S^(j): H_2 (x) I_half on this block */
          for (int64_t n = 0; n < half; ++n) {
            if (compute) {
              double ur = v[2 * (o + n)], ui = v[2 * (o + n) + 1];
              double wr = v[2 * (o + half + n)], wi = v[2 * (o + half + n) + 1];
              v[2 * (o + n)] = ur + wr;
              v[2 * (o + n) + 1] = ui + wi;
              v[2 * (o + half + n)] = ur - wr;
              v[2 * (o + half + n) + 1] = ui - wi;
            }
            add += 2;
          }
          /* W^(j): I_half (+) diag(w_blk^0 .. w_blk^{half-1}) */
          for (int64_t n = 0; n < half; ++n) {
            if (compute) {
              double ur = v[2 * (o + half + n)], ui = v[2 * (o + half + n) + 1];
              double wr = TW_RE(i - j, n), wi = TW_IM(i - j, n);
              v[2 * (o + half + n)] = ur * wr - ui * wi;
              v[2 * (o + half + n) + 1] = ur * wi + ui * wr;
            }
            mul += 1;
            if (!TRIVIAL(blk, n)) mul_nt += 1;
          }
        }
      }
    }
    if (counts) {
      counts[3 * (i - 1) + 0] = mul;
      counts[3 * (i - 1) + 1] = mul_nt;
      counts[3 * (i - 1) + 2] = add;
    }
    if (compute) {
      /* Gamma: natural order out; the internal order stays for iteration i+1 */
      double *yl = y ? y + 2 * (int64_t)(i - 1) * N : NULL;
      if (yl) {
        for (int64_t win = 0; win < N / L; ++win)
          for (int64_t k = 0; k < L; ++k) {
            int64_t p = win * L + mro_bitrev(k, i);
            yl[2 * (win * L + k)] = cur[2 * p];
            yl[2 * (win * L + k) + 1] = cur[2 * p + 1];
          }
      }
      double *t = prev; prev = cur; cur = t;
    }
  }
#undef TW_RE
#undef TW_IM
#undef TRIVIAL
  free(prev);
  free(cur);
  free(root);
  return 0;
}
