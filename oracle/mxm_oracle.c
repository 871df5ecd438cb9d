/*
 * mxm_oracle.c -- CPU oracle for the mod2am dense product and its
 * FP64-accurate Ozaki-split emulation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the package smoke check and the CPU-baseline leg of the benchmark load it.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * Build: gcc -std=c11 -O2 -fno-fast-math -ffp-contract=off [-fopenmp]
 * (-ffp-contract=off matters: every a*b+c below is two roundings, never an
 * FMA, except where fma() is written out on purpose in Dot2.)
 *
 * Storage: every matrix is dense row-major, element (i,j) of an r x c matrix
 * at X[i*c + j]; A is m x k, B is k x n, C is m x n (Sec. 3.1 states the
 * square n x n case; general m,k,n is the reading used throughout).
 *
 * Contents
 *   oracle_gemm_naive   c_ij = sum_l a_il b_lj, three nested loops, l in order
 *                       (Sec. 3.1: the naive three-loop C version, arbb_mxm0);
 *                       rows shared out by an OpenMP parallel-for on the
 *                       outermost loop, as in the paper's OpenMP baseline.
 *   oracle_gemm_outer   rank-1 update order of arbb_mxm2a (Sec. 3.1):
 *                       c = a_col(0) b_row(0); c += a_col(l) b_row(l).
 *   oracle_gemm_dot2    each c_ij by Dot2 (Ogita, Rump, Oishi, "Accurate sum
 *                       and dot product", SIAM J. Sci. Comput. 26(6), 2005,
 *                       Algorithm 5.3): as accurate as twice-FP64 evaluation.
 *   oracle_gemm_abs     |A|.|B|, the scale of the elementwise error bound.
 *   oracle_ozaki_*      the Ozaki split (Ozaki, Ogita, Oishi, Rump, Numer.
 *                       Algorithms 59, 2012; integer-slice form of Ootomo,
 *                       Ozaki, Yokota, IJHPCA 2024) in the steps:
 *                       scale, split, exact slice products, recombination.
 *                       oracle_ozaki_*_rn8: the same with balanced 8-bit
 *                       digits, the value rounded once to nearest.
 *   oracle_gemm_f32     FP32 naive loop (comparison mode).
 *   oracle_round_bf16   double -> bfloat16, round to nearest even.
 *   oracle_spmv         mod2as (Sec. 3.2): y = A x, A in the 3-array CSR
 *                       form, every row summed in storage order (the
 *                       OMP2 loop of Sec. 3.2), rows shared out by OpenMP.
 *   oracle_spmv_dot2    the same rows by Dot2 (accuracy reference).
 *   oracle_spmv_abs     |A|.|x|, the scale of the error bound.
 *   oracle_cg           conjugate gradients (Sec. 3.4, Fig. 6) for an SPD
 *                       matrix in the same CSR form, steps in the paper's
 *                       order, dot products summed in index order.
 *   oracle_dft          mod2f (Sec. 3.3): the DFT of Eq. 1 term by term.
 *   oracle_fft_dif      the radix-2 decimation-in-frequency recursion of
 *                       Eqs. 2-3, level by level, bit-reversed read-out.
 */
#define _USE_MATH_DEFINES
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_NONFINITE 4
#define ORACLE_INVALID 1

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads the OpenMP loops use from now on (n >= 1); returns the count in
   effect.  Lets a caller time the same loop on one core and on all. */
int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Plain definition: c_ij = sum_{l=0}^{k-1} a_il * b_lj  (Sec. 3.1).   */
/* ------------------------------------------------------------------ */
void oracle_gemm_naive(const double* A, const double* B, double* C,
                       int64_t m, int64_t k, int64_t n) {
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < m; ++i) {
    for (int64_t j = 0; j < n; ++j) {
      double s = 0.0;
      for (int64_t l = 0; l < k; ++l) s += A[i * k + l] * B[l * n + j];
      C[i * n + j] = s;
    }
  }
}

/* arbb_mxm2a (Sec. 3.1): c starts as the first rank-1 product
 * a.col(0) * b.row(0), then every further l adds a.col(l) * b.row(l).
 * Per element this is the same left-to-right sum as the naive loop.    */
void oracle_gemm_outer(const double* A, const double* B, double* C,
                       int64_t m, int64_t k, int64_t n) {
  if (k == 0) {
    for (int64_t t = 0; t < m * n; ++t) C[t] = 0.0;
    return;
  }
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) C[i * n + j] = A[i * k + 0] * B[0 * n + j];
  for (int64_t l = 1; l < k; ++l)
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) C[i * n + j] += A[i * k + l] * B[l * n + j];
}

/* Error-free transformations (Ogita, Rump, Oishi 2005, Sec. 2-3). */
static void two_sum(double a, double b, double* x, double* y) {
  double s = a + b;
  double z = s - a;
  *x = s;
  *y = (a - (s - z)) + (b - z);
}

static void two_product(double a, double b, double* x, double* y) {
  double p = a * b;
  *x = p;
  *y = fma(a, b, -p);
}

/* Dot2 of row i of A with column j of B. */
static double dot2_entry(const double* A, const double* B, int64_t k, int64_t n,
                         int64_t i, int64_t j) {
  if (k == 0) return 0.0;
  double p, s;
  two_product(A[i * k + 0], B[0 * n + j], &p, &s);
  for (int64_t l = 1; l < k; ++l) {
    double h, r, q;
    two_product(A[i * k + l], B[l * n + j], &h, &r);
    two_sum(p, h, &p, &q);
    s = s + (q + r);
  }
  return p + s;
}

void oracle_gemm_dot2(const double* A, const double* B, double* C,
                      int64_t m, int64_t k, int64_t n) {
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) C[i * n + j] = dot2_entry(A, B, k, n, i, j);
}

/* (|A|.|B|)_ij, naive order. */
void oracle_gemm_abs(const double* A, const double* B, double* C,
                     int64_t m, int64_t k, int64_t n) {
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < m; ++i) {
    for (int64_t j = 0; j < n; ++j) {
      double s = 0.0;
      for (int64_t l = 0; l < k; ++l) s += fabs(A[i * k + l]) * fabs(B[l * n + j]);
      C[i * n + j] = s;
    }
  }
}

/* Selected entries (ii[t], jj[t]) only: used to check full-size results on
 * a sample.  out_dot2 and out_abs may each be NULL.                    */
void oracle_entries_dot2_abs(const double* A, const double* B, int64_t m,
                             int64_t k, int64_t n, int64_t count,
                             const int64_t* ii, const int64_t* jj,
                             double* out_dot2, double* out_abs) {
  (void)m;
  int64_t t;
#pragma omp parallel for schedule(dynamic, 16)
  for (t = 0; t < count; ++t) {
    int64_t i = ii[t], j = jj[t];
    if (out_dot2) out_dot2[t] = dot2_entry(A, B, k, n, i, j);
    if (out_abs) {
      double s = 0.0;
      for (int64_t l = 0; l < k; ++l) s += fabs(A[i * k + l]) * fabs(B[l * n + j]);
      out_abs[t] = s;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Ozaki split, step by step.                                          */
/*                                                                     */
/* Step 1, scale: every row i of A gets the exponent e_i with          */
/*   max_l |a_il| = mu * 2^{e_i},  mu in [1/2, 1)   (frexp),            */
/* so that every a_il * 2^{-e_i} lies in (-1, 1); an all-zero row gets  */
/* e_i = 0.  Columns j of B get f_j the same way.                       */
/* Step 2, split: with r_0 = x * 2^{-e} and slice width beta bits,      */
/*   t_s = r_{s-1} * 2^beta,  d_s = trunc(t_s),  r_s = t_s - d_s,       */
/* for s = 1..S, so x = 2^e (sum_s d_s 2^{-beta s} + r_S 2^{-beta S})   */
/* with integer digits |d_s| <= 2^beta - 1 (127 for beta = 7: int8).     */
/* Step 3, exact products: for every diagonal g = s + t in 2..S+1,       */
/*   D_g(i,j) = sum_{s+t=g} sum_l d^A_s(i,l) d^B_t(l,j),  in int64.      */
/* Step 4, recombine in FP64, smallest weight first:                    */
/*   acc = 0; for g = S+1 down to 2: acc = acc + D_g * 2^{-beta g};     */
/*   c_ij = acc * 2^{e_i + f_j}.                                        */
/* ------------------------------------------------------------------ */

/* frexp exponent of |x|, 0 for x == 0 (x finite). */
static int oracle_exponent(double x) {
  int e = 0;
  if (x == 0.0) return 0;
  (void)frexp(x, &e);
  return e;
}

static int is_finite(double x) { return isfinite(x) ? 1 : 0; }

/* Step 1 for the rows of an r x c matrix (by_col = 0) or for its
 * columns (by_col = 1).  Returns ORACLE_NONFINITE if any entry is not
 * finite (exps then unspecified).                                      */
int oracle_ozaki_exponents(const double* X, int64_t rows, int64_t cols,
                           int by_col, int32_t* exps) {
  int bad = 0;
  if (!by_col) {
    for (int64_t i = 0; i < rows; ++i) {
      double mx = 0.0;
      for (int64_t l = 0; l < cols; ++l) {
        double v = X[i * cols + l];
        if (!is_finite(v)) bad = 1;
        if (fabs(v) > mx) mx = fabs(v);
      }
      exps[i] = oracle_exponent(mx);
    }
  } else {
    for (int64_t j = 0; j < cols; ++j) {
      double mx = 0.0;
      for (int64_t l = 0; l < rows; ++l) {
        double v = X[l * cols + j];
        if (!is_finite(v)) bad = 1;
        if (fabs(v) > mx) mx = fabs(v);
      }
      exps[j] = oracle_exponent(mx);
    }
  }
  return bad ? ORACLE_NONFINITE : ORACLE_OK;
}

/* Step 2 for one value. */
static void split_value(double x, int e, int beta, int S, int16_t* d, int64_t stride) {
  double r = ldexp(x, -e);
  for (int s = 0; s < S; ++s) {
    double t = ldexp(r, beta);
    double q = trunc(t);
    r = t - q;
    d[s * stride] = (int16_t)q;
  }
}

/* Step 2 with balanced 8-bit digits, the round-to-nearest variant of the
 * split (the original Ozaki splitting rounds to nearest too).  The scale
 * exponent is one more (e' = e + 1, so |x| 2^-e' < 1/2); the value is
 * rounded once, to the nearest integer with ties to even,
 *   V = round(x 2^(8S - e')),   |V| <= 2^(8S - 1), exact in int64 (S <= 7),
 * and written in base 256 from the least significant digit up: each lower
 * digit is V mod 256 taken in [-128, 127] and V becomes (V - d) / 256; the
 * top digit is what remains, in [-128, 128].  So sum_s d_s 2^(8(S-s)) = V,
 * every digit product is at most 2^14 in magnitude, and x is approximated
 * to within 2^(e' - 8S - 1).  Digit s goes to d[(s - 1) stride].        */
static void split_value_rn8(double x, int e1, int S, int16_t* d, int64_t stride) {
  int64_t V = (int64_t)nearbyint(ldexp(x, 8 * S - e1));
  for (int s = S; s >= 2; --s) {
    int64_t r = V % 256;
    if (r < 0) r += 256;
    const int64_t dig = r >= 128 ? r - 256 : r;
    d[(s - 1) * stride] = (int16_t)dig;
    V = (V - dig) / 256;
  }
  d[0] = (int16_t)V;
}

/* Steps 1 and 2 for a whole matrix.  digits is [S][rows][cols] int16.
 * rn8: balanced 8-bit digits (beta is then 8) with exps = e + 1.      */
static int ozaki_split_any(const double* X, int64_t rows, int64_t cols, int by_col, int beta,
                           int S, int rn8, int32_t* exps, int16_t* digits) {
  if (beta < 1 || beta > 8 || S < 1 || (rn8 && (beta != 8 || S > 7))) return ORACLE_INVALID;
  int st = oracle_ozaki_exponents(X, rows, cols, by_col, exps);
  if (st != ORACLE_OK) return st;
  const int64_t cnt = by_col ? cols : rows;
  if (rn8)
    for (int64_t i = 0; i < cnt; ++i) exps[i] += 1;
  const int64_t plane = rows * cols;
  for (int64_t i = 0; i < rows; ++i)
    for (int64_t l = 0; l < cols; ++l) {
      int e = by_col ? exps[l] : exps[i];
      if (rn8)
        split_value_rn8(X[i * cols + l], e, S, digits + i * cols + l, plane);
      else
        split_value(X[i * cols + l], e, beta, S, digits + i * cols + l, plane);
    }
  return ORACLE_OK;
}

int oracle_ozaki_split(const double* X, int64_t rows, int64_t cols, int by_col,
                       int beta, int S, int32_t* exps, int16_t* digits) {
  return ozaki_split_any(X, rows, cols, by_col, beta, S, 0, exps, digits);
}

int oracle_ozaki_split_rn8(const double* X, int64_t rows, int64_t cols, int by_col, int S,
                           int32_t* exps, int16_t* digits) {
  return ozaki_split_any(X, rows, cols, by_col, 8, S, 1, exps, digits);
}

/* Steps 3 and 4 for one entry.  dA is [S][m][k]; dBt holds the digits of
 * B with each column stored contiguously, [S][n][k] (a storage choice:
 * the integer sums are exact, so it does not change any value).        */
static double ozaki_entry(const int16_t* dA, const int16_t* dBt, int64_t m,
                          int64_t k, int64_t n, int S, int beta, int32_t e_i,
                          int32_t f_j, int64_t i, int64_t j) {
  const int64_t planeA = m * k, planeB = n * k;
  double acc = 0.0;
  for (int g = S + 1; g >= 2; --g) {
    int64_t Dg = 0;
    for (int s = 1; s <= g - 1; ++s) {
      int t = g - s;
      const int16_t* a = dA + (int64_t)(s - 1) * planeA + i * k;
      const int16_t* b = dBt + (int64_t)(t - 1) * planeB + j * k;
      for (int64_t l = 0; l < k; ++l) Dg += (int64_t)a[l] * (int64_t)b[l];
    }
    acc = acc + ldexp((double)Dg, -beta * g);
  }
  return ldexp(acc, e_i + f_j);
}

/* Full emulated product C = A.B with S slices of beta bits (rn8: the
 * balanced 8-bit digits; steps 3 and 4 are the same). */
static int ozaki_gemm_any(const double* A, const double* B, double* C, int64_t m, int64_t k,
                          int64_t n, int S, int beta, int rn8) {
  if (beta < 1 || beta > 8 || S < 1 || S > 16) return ORACLE_INVALID;
  size_t szA = (size_t)(S * m * k > 0 ? S * m * k : 1);
  size_t szB = (size_t)(S * k * n > 0 ? S * k * n : 1);
  int32_t* e = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t* f = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int16_t* dA = (int16_t*)malloc(sizeof(int16_t) * szA);
  int16_t* dB = (int16_t*)malloc(sizeof(int16_t) * szB);
  int16_t* dBt = (int16_t*)malloc(sizeof(int16_t) * szB);
  int st = ORACLE_OK;
  if (!e || !f || !dA || !dB || !dBt) { st = ORACLE_INVALID; goto done; }
  st = ozaki_split_any(A, m, k, 0, beta, S, rn8, e, dA);
  if (st == ORACLE_OK) st = ozaki_split_any(B, k, n, 1, beta, S, rn8, f, dB);
  if (st != ORACLE_OK) goto done;
  for (int s = 0; s < S; ++s)
    for (int64_t l = 0; l < k; ++l)
      for (int64_t j = 0; j < n; ++j)
        dBt[(int64_t)s * n * k + j * k + l] = dB[(int64_t)s * k * n + l * n + j];
  {
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
    for (i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j)
        C[i * n + j] = ozaki_entry(dA, dBt, m, k, n, S, beta, e[i], f[j], i, j);
  }
done:
  free(e); free(f); free(dA); free(dB); free(dBt);
  return st;
}

int oracle_ozaki_gemm(const double* A, const double* B, double* C, int64_t m, int64_t k,
                      int64_t n, int S, int beta) {
  return ozaki_gemm_any(A, B, C, m, k, n, S, beta, 0);
}

int oracle_ozaki_gemm_rn8(const double* A, const double* B, double* C, int64_t m, int64_t k,
                          int64_t n, int S) {
  return ozaki_gemm_any(A, B, C, m, k, n, S, 8, 1);
}

/* Selected entries of the emulated product; splits only the rows and
 * columns the sample touches.                                          */
static int ozaki_entries_any(const double* A, const double* B, int64_t m, int64_t k, int64_t n,
                             int S, int beta, int rn8, int64_t count, const int64_t* ii,
                             const int64_t* jj, double* out) {
  (void)m;
  if (beta < 1 || beta > 8 || S < 1 || S > 16 || (rn8 && (beta != 8 || S > 7)))
    return ORACLE_INVALID;
  int bad = 0;
  int64_t t;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
  for (t = 0; t < count; ++t) {
    int64_t i = ii[t], j = jj[t];
    int16_t* da = (int16_t*)malloc(sizeof(int16_t) * (size_t)(S * k > 0 ? S * k : 1));
    int16_t* db = (int16_t*)malloc(sizeof(int16_t) * (size_t)(S * k > 0 ? S * k : 1));
    double ma = 0.0, mb = 0.0;
    for (int64_t l = 0; l < k; ++l) {
      double a = A[i * k + l], b = B[l * n + j];
      if (!is_finite(a) || !is_finite(b)) bad = 1;
      if (fabs(a) > ma) ma = fabs(a);
      if (fabs(b) > mb) mb = fabs(b);
    }
    /* the column exponent needs the whole column of B; the row exponent
     * the whole row of A: both were just scanned.                      */
    int ei = oracle_exponent(ma) + rn8, fj = oracle_exponent(mb) + rn8;
    for (int64_t l = 0; l < k; ++l) {
      if (rn8) {
        split_value_rn8(A[i * k + l], ei, S, da + l, k);
        split_value_rn8(B[l * n + j], fj, S, db + l, k);
      } else {
        split_value(A[i * k + l], ei, beta, S, da + l, k);
        split_value(B[l * n + j], fj, beta, S, db + l, k);
      }
    }
    double acc = 0.0;
    for (int g = S + 1; g >= 2; --g) {
      int64_t Dg = 0;
      for (int s = 1; s <= g - 1; ++s) {
        const int16_t* a = da + (int64_t)(s - 1) * k;
        const int16_t* b = db + (int64_t)(g - s - 1) * k;
        for (int64_t l = 0; l < k; ++l) Dg += (int64_t)a[l] * (int64_t)b[l];
      }
      acc = acc + ldexp((double)Dg, -beta * g);
    }
    out[t] = ldexp(acc, ei + fj);
    free(da); free(db);
  }
  return bad ? ORACLE_NONFINITE : ORACLE_OK;
}

int oracle_ozaki_entries(const double* A, const double* B, int64_t m, int64_t k, int64_t n,
                         int S, int beta, int64_t count, const int64_t* ii, const int64_t* jj,
                         double* out) {
  return ozaki_entries_any(A, B, m, k, n, S, beta, 0, count, ii, jj, out);
}

int oracle_ozaki_entries_rn8(const double* A, const double* B, int64_t m, int64_t k, int64_t n,
                             int S, int64_t count, const int64_t* ii, const int64_t* jj,
                             double* out) {
  return ozaki_entries_any(A, B, m, k, n, S, 8, 1, count, ii, jj, out);
}

/* ------------------------------------------------------------------ */
/* Comparison modes.                                                   */
/* ------------------------------------------------------------------ */
/* FP32 inputs, FP32 naive accumulation. */
void oracle_gemm_f32(const float* A, const float* B, float* C, int64_t m,
                     int64_t k, int64_t n) {
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      float s = 0.0f;
      for (int64_t l = 0; l < k; ++l) s += A[i * k + l] * B[l * n + j];
      C[i * n + j] = s;
    }
}

/* double -> bfloat16 (1 sign, 8 exponent, 7 fraction bits), round to
 * nearest, ties to even, by exact arithmetic on the value: bf16 spacing
 * in [2^q, 2^{q+1}) is 2^{q-7}; below 2^-126 the spacing is 2^-133.
 * Returns the 16-bit pattern.                                          */
static uint16_t round_bf16_one(double x) {
  uint64_t bits;
  memcpy(&bits, &x, sizeof bits);
  uint16_t sign = (uint16_t)((bits >> 48) & 0x8000u);
  if (isnan(x)) return (uint16_t)(sign | 0x7FC0u);
  double ax = fabs(x);
  if (isinf(x)) return (uint16_t)(sign | 0x7F80u);
  if (ax == 0.0) return sign;
  int q;
  (void)frexp(ax, &q);          /* ax in [2^{q-1}, 2^q) */
  int lsb_exp = (q - 1) - 7;    /* spacing of the bf16 grid at ax */
  if (lsb_exp < -133) lsb_exp = -133;
  double scaled = ldexp(ax, -lsb_exp); /* exact: in [0, 2^8) */
  double lo = floor(scaled);
  double frac = scaled - lo;
  double r = lo;
  if (frac > 0.5 || (frac == 0.5 && fmod(lo, 2.0) != 0.0)) r = lo + 1.0;
  double v = ldexp(r, lsb_exp);
  if (v >= ldexp(1.0, 128)) return (uint16_t)(sign | 0x7F80u);
  /* encode v exactly */
  float fv = (float)v; /* exact: v has <= 8 significant bits, in float range */
  uint32_t fb;
  memcpy(&fb, &fv, sizeof fb);
  return (uint16_t)(sign | (uint16_t)((fb >> 16) & 0x7FFFu));
}

void oracle_round_bf16(const double* x, uint16_t* out, int64_t count) {
  for (int64_t t = 0; t < count; ++t) out[t] = round_bf16_one(x[t]);
}

/* ------------------------------------------------------------------ */
/* mod2as (Sec. 3.2): y = A x for an nrows x ncols matrix in the 3-array */
/* CSR form of the paper: matvals[j] is the j-th non-zero, indx[j] its   */
/* column, rowp[i] the position of the first non-zero of row i, and      */
/* rowp[nrows] = nnz.  Every row is summed (the ArBB kernel maps over    */
/* all nrows rows; the OpenMP listings' "i < nrows - 1" would skip the   */
/* last one), and y is overwritten (the ArBB reduce starts from 0).      */
/* A structure that is not monotone or indexes outside the arrays is     */
/* rejected with ORACLE_INVALID before anything is read through it.      */
static int csr_valid(const int32_t* indx, const int32_t* rowp, int64_t nrows, int64_t ncols,
                     int64_t nnz) {
  if (nrows < 0 || ncols < 0 || nnz < 0) return 0;
  if (rowp[0] != 0 || rowp[nrows] != nnz) return 0;
  for (int64_t i = 0; i < nrows; ++i)
    if (rowp[i] > rowp[i + 1]) return 0;
  for (int64_t j = 0; j < nnz; ++j)
    if (indx[j] < 0 || indx[j] >= ncols) return 0;
  return 1;
}

int oracle_spmv(const double* vals, const int32_t* indx, const int32_t* rowp, const double* x,
                double* y, int64_t nrows, int64_t ncols, int64_t nnz) {
  if (!csr_valid(indx, rowp, nrows, ncols, nnz)) return ORACLE_INVALID;
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < nrows; ++i) {
    double t = 0.0;
    for (int64_t j = rowp[i]; j < rowp[i + 1]; ++j) t = t + vals[j] * x[indx[j]];
    y[i] = t;
  }
  return ORACLE_OK;
}

int oracle_spmv_dot2(const double* vals, const int32_t* indx, const int32_t* rowp,
                     const double* x, double* y, int64_t nrows, int64_t ncols, int64_t nnz) {
  if (!csr_valid(indx, rowp, nrows, ncols, nnz)) return ORACLE_INVALID;
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < nrows; ++i) {
    double p = 0.0, s = 0.0;
    for (int64_t j = rowp[i]; j < rowp[i + 1]; ++j) {
      double h, r, q;
      two_product(vals[j], x[indx[j]], &h, &r);
      two_sum(p, h, &p, &q);
      s = s + (q + r);
    }
    y[i] = p + s;
  }
  return ORACLE_OK;
}

int oracle_spmv_abs(const double* vals, const int32_t* indx, const int32_t* rowp,
                    const double* x, double* y, int64_t nrows, int64_t ncols, int64_t nnz) {
  if (!csr_valid(indx, rowp, nrows, ncols, nnz)) return ORACLE_INVALID;
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < nrows; ++i) {
    double t = 0.0;
    for (int64_t j = rowp[i]; j < rowp[i + 1]; ++j) t = t + fabs(vals[j]) * fabs(x[indx[j]]);
    y[i] = t;
  }
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* Conjugate gradients (Sec. 3.4, Fig. 6 and the ArBB loop beside it)    */
/* for A x = b, A symmetric positive definite in the CSR form above      */
/* (n x n).  x0 = 0, so r0 = b and p0 = b; r2 = (b, b).  While           */
/* r2 > stop and fewer than max_iters steps were taken:                  */
/*   q = A p (every row in storage order, as oracle_spmv);               */
/*   alpha = r2 / (p, q);  r2_old = r2;  r = r - alpha q;                */
/*   r2 = (r, r);  beta = r2 / r2_old;  x = x + alpha p;  p = r + beta p. */
/* Dot products are summed in index order.  The paper does not say what  */
/* happens when (p, A p) <= 0 (A not positive definite along p): here    */
/* the step is not taken, the loop ends and ORACLE_BREAKDOWN is returned. */
/* iters receives the number of steps taken, r2_final the last r2, and   */
/* r2_hist (if not NULL, max_iters entries) the r2 after every step.     */
#define ORACLE_BREAKDOWN 9

int oracle_cg(const double* vals, const int32_t* indx, const int32_t* rowp, const double* b,
              double* x, int64_t n, int64_t nnz, double stop, int64_t max_iters, int64_t* iters,
              double* r2_final, double* r2_hist) {
  if (!csr_valid(indx, rowp, n, n, nnz)) return ORACLE_INVALID;
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!r || !p || !q) {
    free(r);
    free(p);
    free(q);
    return ORACLE_INVALID;
  }
  double r2 = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    x[i] = 0.0;
    r[i] = b[i];
    p[i] = b[i];
    r2 = r2 + b[i] * b[i];
  }
  int status = ORACLE_OK;
  int64_t k = 0;
  while (r2 > stop && k < max_iters) {
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
      double t = 0.0;
      for (int64_t j = rowp[i]; j < rowp[i + 1]; ++j) t = t + vals[j] * p[indx[j]];
      q[i] = t;
    }
    double pq = 0.0;
    for (i = 0; i < n; ++i) pq = pq + p[i] * q[i];
    if (!(pq > 0.0)) {
      status = ORACLE_BREAKDOWN;
      break;
    }
    const double alpha = r2 / pq;
    const double r2_old = r2;
    for (i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
    r2 = 0.0;
    for (i = 0; i < n; ++i) r2 = r2 + r[i] * r[i];
    const double beta = r2 / r2_old;
    for (i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
    for (i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    if (r2_hist) r2_hist[k] = r2;
    ++k;
  }
  *iters = k;
  *r2_final = r2;
  free(r);
  free(p);
  free(q);
  return status;
}

/* ------------------------------------------------------------------ */
/* mod2f (Sec. 3.3): the 1-D complex DFT of Eq. 1,                       */
/*   F(k) = sum_{n=0}^{N-1} f(n) exp(-2 pi i k n / N),                   */
/* for complex FP64 data stored interleaved (re, im) per point.          */
/* Twiddle W_N^m = exp(-2 pi i m / N) = cos(2 pi m / N) - i sin(2 pi m / */
/* N), with m reduced mod N first (so the angle is in [0, 2 pi)).        */
/* Complex products (a + bi)(c + di) = (ac - bd) + (ad + bc) i, each     */
/* product and sum rounded separately.                                   */
static void twiddle(int64_t m, int64_t N, double* c, double* s) {
  const double ang = 2.0 * M_PI * (double)(m % N) / (double)N;
  *c = cos(ang);
  *s = -sin(ang);
}

/* The definition (Eq. 1) term by term, n in order: O(N^2). */
void oracle_dft(const double* f, double* F, int64_t N) {
  int64_t k;
#pragma omp parallel for schedule(static)
  for (k = 0; k < N; ++k) {
    double re = 0.0, im = 0.0;
    for (int64_t n = 0; n < N; ++n) {
      double c, s;
      twiddle((k * n) % N, N, &c, &s);
      const double a = f[2 * n], b = f[2 * n + 1];
      re = re + (a * c - b * s);
      im = im + (a * s + b * c);
    }
    F[2 * k] = re;
    F[2 * k + 1] = im;
  }
}

/* Radix-2 decimation in frequency (Eqs. 2-3), applied level by level:  */
/* a block of length L (a sub-transform) becomes its f_e (first half)   */
/* and f_o (second half),                                               */
/*   f_e(n) = f(n) + f(n + L/2),                                        */
/*   f_o(n) = (f(n) - f(n + L/2)) W_L^n,       0 <= n < L/2,            */
/* and both halves are transformed further.  After the last level the   */
/* value at position p is F(bitrev(p)) (Eq. 2: the even frequencies come */
/* from the first half, the odd from the second), so the result is read */
/* out through the bit reversal.  N must be a power of two.             */
int oracle_fft_dif(const double* f, double* F, int64_t N) {
  if (N < 1 || (N & (N - 1)) != 0) return ORACLE_INVALID;
  double* w = (double*)malloc(sizeof(double) * 2 * (size_t)N);
  if (!w) return ORACLE_INVALID;
  memcpy(w, f, sizeof(double) * 2 * (size_t)N);
  for (int64_t L = N; L >= 2; L /= 2) {
    const int64_t h = L / 2;
    for (int64_t blk = 0; blk < N; blk += L) {
      for (int64_t n = 0; n < h; ++n) {
        double* x0 = w + 2 * (blk + n);
        double* x1 = w + 2 * (blk + n + h);
        const double ar = x0[0], ai = x0[1], br = x1[0], bi = x1[1];
        double c, s;
        twiddle(n, L, &c, &s);
        const double dr = ar - br, di = ai - bi;
        x0[0] = ar + br;
        x0[1] = ai + bi;
        x1[0] = dr * c - di * s;
        x1[1] = dr * s + di * c;
      }
    }
  }
  int bits = 0;
  while (((int64_t)1 << bits) < N) ++bits;
  for (int64_t p = 0; p < N; ++p) {
    int64_t r = 0;
    for (int b = 0; b < bits; ++b) r |= ((p >> b) & 1) << (bits - 1 - b);
    F[2 * r] = w[2 * p];
    F[2 * r + 1] = w[2 * p + 1];
  }
  free(w);
  return ORACLE_OK;
}
