/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the sketch  A_hat = S * A  and
 * for sketch-and-precondition (SAP) least squares.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the test-suite, the package's smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * What it computes (paper: "Fast multiplication of random dense matrices with
 * sparse matrices", arXiv 2310.15419):
 *   - Eq. (1) ("goal"): A_hat = S A, A an m x n sparse matrix in CSC, S a d x m
 *     matrix with iid entries from N(0,1), U(-1,1) or {+1,-1} (Sec. 1.1).
 *   - S is never stored: every entry is a pure function of (seed, stream, i, j)
 *     through a counter-based generator (Sec. 4.2 "Counter Based RNG" and the
 *     threading-independent reproducibility policy of Sec. 4.3).  The
 *     generator is Philox4x32-10 of Salmon et al. (SC'11, the Random123 family
 *     the paper names in Sec. 4.2).
 *   - Distribution transforms of Sec. 3.3 (int -> uniform; Gaussian is the
 *     expensive one), in the exact forms chosen below.
 *   - Alg. 3 (variant kji, regenerate S[:, j] for every nonzero) and Alg. 4
 *     (variant jki, generate S[:, j] once per nonempty row), both with one
 *     block covering all of d and n (Alg. 1 with b_d = d, b_n = n).
 *   - Sec. 5.3: SAP least squares -- Householder QR of A_hat, LSQR (Paige &
 *     Saunders 1982) on the preconditioned operator A R^{-1}, and the error
 *     metric Error(x) = ||A^T (A x - b)||_2 / (||A||_F ||A x - b||_2).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   counter layout   ctr = (i_blk, j, stream, 0), key = (seed lo32, seed hi32)
 *   +-1              i_blk = i >> 7; bit b = i & 127 of the 128-bit output
 *                    (word b >> 5, bit b & 31); S = bit ? -1 : +1
 *   U(-1,1)          i_blk = i >> 2; w = word (i & 3); u = w >> 8 read as a
 *                    signed 24-bit integer; S = (2u + 1) * 2^-24
 *                    (symmetric, open interval, exact in FP32; the paper's
 *                    int32 / 2^31 form can round to +-1 in FP32)
 *   N(0,1)           i_blk = i >> 2; Box-Muller on the word pairs (0,1) and
 *                    (2,3): u1 = ((w_even >> 8) + 1) * 2^-24 in (0,1],
 *                    u2 = (w_odd >> 8) * 2^-24 in [0,1),
 *                    r = sqrt(-2 ln u1); even i -> r cos(2 pi u2),
 *                    odd i -> r sin(2 pi u2)
 *
 * Every floating-point result here is FP64.
 */
#define _GNU_SOURCE
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PM1 0
#define ORACLE_UNIFORM 1
#define ORACLE_NORMAL 2

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).                        */
/* One round: two 32x32->64 multiplies of counter words 0 and 2 by the       */
/* round multipliers, the high halves xor-ed with the other counter words    */
/* and the key, then the key is bumped by the Weyl constants.  Ten rounds.   */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The 128-bit block that holds S(i, j): counter (i_blk, j, stream, 0). */
static void philox_block(uint64_t seed, uint32_t stream, uint32_t i_blk,
                         uint32_t j, uint32_t out[4]) {
  uint32_t ctr[4] = {i_blk, j, stream, 0u};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  oracle_philox4x32_10(ctr, key, out);
}

/* w >> 8 read as a two's-complement 24-bit integer, without relying on
 * implementation-defined signed shifts. */
static int64_t top24_signed(uint32_t w) {
  int64_t u = (int64_t)(w >> 8);
  if (u >= (1 << 23)) u -= (1 << 24);
  return u;
}

/* Sec. 3.3: uniform (-1,1) from the integer stream, exact form (2u+1) 2^-24. */
double oracle_uniform_from_word(uint32_t w) {
  return (double)(2 * top24_signed(w) + 1) * ldexp(1.0, -24);
}

/* Box-Muller pair from two words; sel = 0 -> cosine branch, 1 -> sine. */
double oracle_normal_from_words(uint32_t w_radius, uint32_t w_angle, int sel) {
  double u1 = (double)((w_radius >> 8) + 1u) * ldexp(1.0, -24); /* (0, 1] */
  double u2 = (double)(w_angle >> 8) * ldexp(1.0, -24);         /* [0, 1) */
  double r = sqrt(-2.0 * log(u1));
  const double two_pi = 6.283185307179586476925286766559;
  double t = two_pi * u2;
  return sel ? r * sin(t) : r * cos(t);
}

/* S(i, j), literally: one Philox block per entry. */
double oracle_S_entry(int dist, uint64_t seed, uint32_t stream, int64_t i,
                      int64_t j) {
  uint32_t x[4];
  if (dist == ORACLE_PM1) {
    philox_block(seed, stream, (uint32_t)(i >> 7), (uint32_t)j, x);
    int b = (int)(i & 127);
    uint32_t bit = (x[b >> 5] >> (b & 31)) & 1u;
    return bit ? -1.0 : 1.0;
  }
  philox_block(seed, stream, (uint32_t)(i >> 2), (uint32_t)j, x);
  int q = (int)(i & 3);
  if (dist == ORACLE_UNIFORM) return oracle_uniform_from_word(x[q]);
  /* ORACLE_NORMAL */
  int pair = q >> 1;
  return oracle_normal_from_words(x[2 * pair], x[2 * pair + 1], q & 1);
}

/* Column S(0:d, j).  Same values as oracle_S_entry; one Philox block per
 * group of entries that share it. */
void oracle_S_column(int dist, uint64_t seed, uint32_t stream, int64_t d,
                     int64_t j, double* out) {
  uint32_t x[4];
  if (dist == ORACLE_PM1) {
    for (int64_t i0 = 0; i0 < d; i0 += 128) {
      philox_block(seed, stream, (uint32_t)(i0 >> 7), (uint32_t)j, x);
      for (int b = 0; b < 128 && i0 + b < d; ++b)
        out[i0 + b] = ((x[b >> 5] >> (b & 31)) & 1u) ? -1.0 : 1.0;
    }
    return;
  }
  for (int64_t i0 = 0; i0 < d; i0 += 4) {
    philox_block(seed, stream, (uint32_t)(i0 >> 2), (uint32_t)j, x);
    for (int q = 0; q < 4 && i0 + q < d; ++q) {
      if (dist == ORACLE_UNIFORM)
        out[i0 + q] = oracle_uniform_from_word(x[q]);
      else
        out[i0 + q] =
            oracle_normal_from_words(x[2 * (q >> 1)], x[2 * (q >> 1) + 1], q & 1);
    }
  }
}

/* Dense S (d x m, column-major, ld = d): only for brute-force checks. */
void oracle_S_dense(int dist, uint64_t seed, uint32_t stream, int64_t d,
                    int64_t m, double* S) {
  for (int64_t j = 0; j < m; ++j) oracle_S_column(dist, seed, stream, d, j, S + j * d);
}

/* ------------------------------------------------------------------------ */
/* Sketch A_hat = S A.                                                       */
/* ------------------------------------------------------------------------ */

/* Alg. 3 (variant kji with RNG), one block covering all of d and n:
 * for each column k, for each nonzero (j, a) of column k, regenerate
 * v = S(:, j) and add a * v into A_hat(:, k).  Generates d * nnz numbers
 * (Sec. 3.2).  A_hat is d x n column-major FP64, overwritten (Alg. 1 starts
 * from A_hat = 0).  Returns the number of S entries generated. */
int64_t oracle_sketch_kji(int64_t m, int64_t n, int64_t d, int dist,
                          uint64_t seed, uint32_t stream, const int32_t* colptr,
                          const int32_t* rowidx, const double* values,
                          double* Ahat) {
  (void)m;
  double* v = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
  int64_t generated = 0;
  memset(Ahat, 0, sizeof(double) * (size_t)(d * n));
  for (int64_t k = 0; k < n; ++k) {
    double* col = Ahat + k * d;
    for (int64_t p = colptr[k]; p < colptr[k + 1]; ++p) {
      int64_t j = rowidx[p];
      double a = values[p];
      oracle_S_column(dist, seed, stream, d, j, v);
      generated += d;
      for (int64_t i = 0; i < d; ++i) col[i] += a * v[i];
    }
  }
  free(v);
  return generated;
}

/* Alg. 4 (variant jki with RNG), one vertical block covering all n columns:
 * transpose A to CSR (the blocked-CSR structure of Sec. 3.2 with one block),
 * then for each nonempty row j generate v = S(:, j) once and add A(j, k) * v
 * into A_hat(:, k) for every nonzero of the row.  Generates d * (number of
 * nonempty rows) numbers.  Returns that count (or -1 on allocation failure).
 * If row_lo/row_hi select a row range [row_lo, row_hi), only rows in it
 * contribute (used to time a bounded sample of a workload). */
int64_t oracle_sketch_jki_rows(int64_t m, int64_t n, int64_t d, int dist,
                               uint64_t seed, uint32_t stream,
                               const int32_t* colptr, const int32_t* rowidx,
                               const double* values, double* Ahat,
                               int64_t row_lo, int64_t row_hi) {
  int64_t nnz = colptr[n];
  int64_t* rowptr = (int64_t*)calloc((size_t)(m + 1), sizeof(int64_t));
  int64_t* cursor = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
  int64_t* csr_col = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  double* csr_val = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  double* v = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
  if (!rowptr || !cursor || !csr_col || !csr_val || !v) {
    free(rowptr); free(cursor); free(csr_col); free(csr_val); free(v);
    return -1;
  }
  for (int64_t p = 0; p < nnz; ++p) rowptr[rowidx[p] + 1]++;
  for (int64_t j = 0; j < m; ++j) rowptr[j + 1] += rowptr[j];
  memcpy(cursor, rowptr, sizeof(int64_t) * (size_t)(m + 1));
  for (int64_t k = 0; k < n; ++k)
    for (int64_t p = colptr[k]; p < colptr[k + 1]; ++p) {
      int64_t q = cursor[rowidx[p]]++;
      csr_col[q] = k;
      csr_val[q] = values[p];
    }
  memset(Ahat, 0, sizeof(double) * (size_t)(d * n));
  int64_t generated = 0;
  if (row_lo < 0) row_lo = 0;
  if (row_hi > m || row_hi < 0) row_hi = m;
  for (int64_t j = row_lo; j < row_hi; ++j) {
    if (rowptr[j] == rowptr[j + 1]) continue; /* zero row: S(:, j) not needed */
    oracle_S_column(dist, seed, stream, d, j, v);
    generated += d;
    for (int64_t q = rowptr[j]; q < rowptr[j + 1]; ++q) {
      double a = csr_val[q];
      double* col = Ahat + csr_col[q] * d;
      for (int64_t i = 0; i < d; ++i) col[i] += a * v[i];
    }
  }
  free(rowptr); free(cursor); free(csr_col); free(csr_val); free(v);
  return generated;
}

/* Entries S(i0:i1, j) into out[0 .. i1-i0): the same values as
 * oracle_S_column, computed only for the rows asked for (the blocks that
 * hold them). */
static void S_rows(int dist, uint64_t seed, uint32_t stream, int64_t i0, int64_t i1,
                   int64_t j, double* out) {
  uint32_t x[4];
  const int64_t per = (dist == ORACLE_PM1) ? 128 : 4;
  for (int64_t b0 = (i0 / per) * per; b0 < i1; b0 += per) {
    philox_block(seed, stream, (uint32_t)(b0 / per), (uint32_t)j, x);
    for (int64_t i = (b0 > i0 ? b0 : i0); i < b0 + per && i < i1; ++i) {
      const int q = (int)(i - b0);
      double v;
      if (dist == ORACLE_PM1)
        v = ((x[q >> 5] >> (q & 31)) & 1u) ? -1.0 : 1.0;
      else if (dist == ORACLE_UNIFORM)
        v = oracle_uniform_from_word(x[q]);
      else
        v = oracle_normal_from_words(x[2 * (q >> 1)], x[2 * (q >> 1) + 1], q & 1);
      out[i - i0] = v;
    }
  }
}

/* Alg. 4 (variant jki) on all host cores: the same CSR transpose and row
 * order as oracle_sketch_jki_rows, with the rows of A_hat (rows of S) split
 * into `threads` contiguous slices on Philox block boundaries.  A thread
 * walks every nonempty row j in order, generates only its slice of S(:, j)
 * and adds it into its slice of A_hat, so every element of A_hat receives
 * exactly the serial oracle's additions in the serial oracle's order: the
 * result is bit-identical to oracle_sketch_jki_rows, with no reduction.
 * The total RNG work is the serial oracle's too (each block is generated by
 * the one thread whose slice holds it).  threads <= 0: OpenMP's default.
 * Returns the entries generated, or -1 on allocation failure. */
int64_t oracle_sketch_jki_omp(int64_t m, int64_t n, int64_t d, int dist,
                              uint64_t seed, uint32_t stream,
                              const int32_t* colptr, const int32_t* rowidx,
                              const double* values, double* Ahat,
                              int64_t row_lo, int64_t row_hi, int threads) {
  int64_t nnz = colptr[n];
  int64_t* rowptr = (int64_t*)calloc((size_t)(m + 1), sizeof(int64_t));
  int64_t* cursor = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
  int64_t* csr_col = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  double* csr_val = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!rowptr || !cursor || !csr_col || !csr_val) {
    free(rowptr); free(cursor); free(csr_col); free(csr_val);
    return -1;
  }
  for (int64_t p = 0; p < nnz; ++p) rowptr[rowidx[p] + 1]++;
  for (int64_t j = 0; j < m; ++j) rowptr[j + 1] += rowptr[j];
  memcpy(cursor, rowptr, sizeof(int64_t) * (size_t)(m + 1));
  for (int64_t k = 0; k < n; ++k)
    for (int64_t p = colptr[k]; p < colptr[k + 1]; ++p) {
      int64_t q = cursor[rowidx[p]]++;
      csr_col[q] = k;
      csr_val[q] = values[p];
    }
  memset(Ahat, 0, sizeof(double) * (size_t)(d * n));
  if (row_lo < 0) row_lo = 0;
  if (row_hi > m || row_hi < 0) row_hi = m;
  int64_t nonempty = 0;
  for (int64_t j = row_lo; j < row_hi; ++j) nonempty += rowptr[j] != rowptr[j + 1];
  const int64_t per = (dist == ORACLE_PM1) ? 128 : 4;
  const int64_t blocks = (d + per - 1) / per;
  int T = threads > 0 ? threads : omp_get_max_threads();
  if (T > blocks) T = (int)blocks;
  if (T < 1) T = 1;
  int failed = 0;
#pragma omp parallel for num_threads(T) schedule(static, 1) reduction(|| : failed)
  for (int t = 0; t < T; ++t) {
    const int64_t i0 = per * (blocks * t / T);
    const int64_t i1t = per * (blocks * (t + 1) / T);
    const int64_t i1 = i1t < d ? i1t : d;
    if (i1 <= i0) continue;
    double* v = (double*)malloc(sizeof(double) * (size_t)(i1 - i0));
    if (!v) {
      failed = 1;
      continue;
    }
    for (int64_t j = row_lo; j < row_hi; ++j) {
      if (rowptr[j] == rowptr[j + 1]) continue;
      S_rows(dist, seed, stream, i0, i1, j, v);
      for (int64_t q = rowptr[j]; q < rowptr[j + 1]; ++q) {
        double a = csr_val[q];
        double* col = Ahat + csr_col[q] * d;
        for (int64_t i = i0; i < i1; ++i) col[i] += a * v[i - i0];
      }
    }
    free(v);
  }
  free(rowptr); free(cursor); free(csr_col); free(csr_val);
  return failed ? -1 : nonempty * d;
}

/* Threads an OpenMP region of this library would use by default. */
int oracle_max_threads(void) { return omp_get_max_threads(); }

/* ------------------------------------------------------------------------ */
/* Householder QR of a dense d x n matrix (column-major, d >= n), FP64.      */
/* Sec. 5.3: the decomposition of the sketch that gives the preconditioner.  */
/* Convention: for column x, alpha = -sign(x_0) ||x||, v = x - alpha e_1,    */
/* H = I - 2 v v^T / (v^T v); R(k,k) = alpha; when x(1:) is already zero the */
/* reflector is the identity and R(k,k) = x_0.  Writes R (n x n, col-major  */
/* upper triangle; the strict lower triangle is set to 0).  Returns 0, or -1 */
/* if a column is exactly zero (rank deficient; R(k,k) = 0 is still stored). */
/* ------------------------------------------------------------------------ */
int oracle_householder_qr(int64_t d, int64_t n, const double* A, double* R) {
  double* W = (double*)malloc(sizeof(double) * (size_t)(d * n));
  double* v = (double*)malloc(sizeof(double) * (size_t)d);
  if (!W || !v) { free(W); free(v); return -2; }
  memcpy(W, A, sizeof(double) * (size_t)(d * n));
  int status = 0;
  for (int64_t k = 0; k < n; ++k) {
    double* x = W + k * d + k; /* rows k..d-1 of column k */
    int64_t len = d - k;
    double tail2 = 0.0; /* squared norm of the part below the diagonal */
    for (int64_t t = 1; t < len; ++t) tail2 += x[t] * x[t];
    if (tail2 == 0.0) {
      /* nothing to eliminate: H = I, R(k,k) = x_0 (a zero column is rank
       * deficient and leaves R(k,k) = 0) */
      if (x[0] == 0.0) status = -1;
      continue;
    }
    double norm = sqrt(x[0] * x[0] + tail2);
    double alpha = (x[0] >= 0.0) ? -norm : norm;
    for (int64_t t = 0; t < len; ++t) v[t] = x[t];
    v[0] -= alpha;
    double vtv = 0.0;
    for (int64_t t = 0; t < len; ++t) vtv += v[t] * v[t];
    /* apply H to columns k..n-1 */
    for (int64_t c = k; c < n; ++c) {
      double* y = W + c * d + k;
      double dot = 0.0;
      for (int64_t t = 0; t < len; ++t) dot += v[t] * y[t];
      double f = 2.0 * dot / vtv;
      for (int64_t t = 0; t < len; ++t) y[t] -= f * v[t];
    }
    x[0] = alpha;
  }
  for (int64_t c = 0; c < n; ++c)
    for (int64_t r = 0; r < n; ++r) R[c * n + r] = (r <= c) ? W[c * d + r] : 0.0;
  free(W); free(v);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Sparse products (CSC, FP64 values).                                       */
/* ------------------------------------------------------------------------ */
/* y (m) = A x (n) */
static void csc_matvec(int64_t m, int64_t n, const int32_t* colptr,
                       const int32_t* rowidx, const double* values,
                       const double* x, double* y) {
  for (int64_t j = 0; j < m; ++j) y[j] = 0.0;
  for (int64_t k = 0; k < n; ++k)
    for (int64_t p = colptr[k]; p < colptr[k + 1]; ++p)
      y[rowidx[p]] += values[p] * x[k];
}
/* z (n) = A^T y (m) */
static void csc_rmatvec(int64_t n, const int32_t* colptr, const int32_t* rowidx,
                        const double* values, const double* y, double* z) {
  for (int64_t k = 0; k < n; ++k) {
    double s = 0.0;
    for (int64_t p = colptr[k]; p < colptr[k + 1]; ++p) s += values[p] * y[rowidx[p]];
    z[k] = s;
  }
}
static double vnorm(int64_t len, const double* x) {
  double s = 0.0;
  for (int64_t t = 0; t < len; ++t) s += x[t] * x[t];
  return sqrt(s);
}
/* R upper triangular (n x n column-major).  Solve R z = y in place. */
static void trsv_upper(int64_t n, const double* R, double* y) {
  for (int64_t r = n - 1; r >= 0; --r) {
    double s = y[r];
    for (int64_t c = r + 1; c < n; ++c) s -= R[c * n + r] * y[c];
    y[r] = s / R[r * n + r];
  }
}
/* Solve R^T z = y in place. */
static void trsv_upper_t(int64_t n, const double* R, double* y) {
  for (int64_t r = 0; r < n; ++r) {
    double s = y[r];
    for (int64_t c = 0; c < r; ++c) s -= R[r * n + c] * y[c];
    y[r] = s / R[r * n + r];
  }
}

/* Sec. 5.3 error metric: ||A^T (A x - b)|| / (||A||_F ||A x - b||). */
double oracle_ls_error(int64_t m, int64_t n, const int32_t* colptr,
                       const int32_t* rowidx, const double* values,
                       const double* b, const double* x) {
  double* r = (double*)malloc(sizeof(double) * (size_t)m);
  double* g = (double*)malloc(sizeof(double) * (size_t)n);
  csc_matvec(m, n, colptr, rowidx, values, x, r);
  for (int64_t j = 0; j < m; ++j) r[j] -= b[j];
  csc_rmatvec(n, colptr, rowidx, values, r, g);
  double fro2 = 0.0;
  for (int64_t p = 0; p < colptr[n]; ++p) fro2 += values[p] * values[p];
  double num = vnorm(n, g), rn = vnorm(m, r);
  free(r); free(g);
  if (rn == 0.0) return 0.0;
  return num / (sqrt(fro2) * rn);
}

/* ------------------------------------------------------------------------ */
/* Preconditioners M of Sec. 5.3's LSQR on min || A M y - b || (x = M y):     */
/*   PC_TRI   M = R^{-1}, R upper triangular n x n (SAP-QR)                  */
/*   PC_DENSE M = P, a dense n x k matrix (SAP-SVD: P = V_k Sigma_k^{-1})    */
/*   PC_DIAG  M = diag(D) (LSQR-D: D_ii = 1 / ||A_i||)                       */
/*   PC_NONE  M = I                                                          */
/* ------------------------------------------------------------------------ */
enum { PC_NONE = 0, PC_TRI = 1, PC_DENSE = 2, PC_DIAG = 3 };
typedef struct {
  int kind;
  int64_t k;        /* columns of A M (unknowns of the preconditioned system) */
  const double* R;  /* PC_TRI: n x n column-major, upper triangle used */
  const double* P;  /* PC_DENSE: n x k column-major */
  const double* D;  /* PC_DIAG: n */
} precond;

/* out (n) = M y (y has k entries) */
static void pc_apply(const precond* pc, int64_t n, const double* y, double* out) {
  if (pc->kind == PC_DENSE) {
    for (int64_t i = 0; i < n; ++i) out[i] = 0.0;
    for (int64_t j = 0; j < pc->k; ++j)
      for (int64_t i = 0; i < n; ++i) out[i] += pc->P[j * n + i] * y[j];
    return;
  }
  for (int64_t i = 0; i < n; ++i) out[i] = y[i];
  if (pc->kind == PC_TRI) trsv_upper(n, pc->R, out);
  if (pc->kind == PC_DIAG)
    for (int64_t i = 0; i < n; ++i) out[i] *= pc->D[i];
}

/* out (k) = M^T z (z has n entries) */
static void pc_apply_t(const precond* pc, int64_t n, const double* z, double* out) {
  if (pc->kind == PC_DENSE) {
    for (int64_t j = 0; j < pc->k; ++j) {
      double s = 0.0;
      for (int64_t i = 0; i < n; ++i) s += pc->P[j * n + i] * z[i];
      out[j] = s;
    }
    return;
  }
  for (int64_t i = 0; i < n; ++i) out[i] = z[i];
  if (pc->kind == PC_TRI) trsv_upper_t(n, pc->R, out);
  if (pc->kind == PC_DIAG)
    for (int64_t i = 0; i < n; ++i) out[i] *= pc->D[i];
}

/* ------------------------------------------------------------------------ */
/* LSQR (Paige & Saunders, ACM TOMS 1982) on min || A M y - b ||, then       */
/* x = M y.  Sec. 5.3.                                                       */
/* Stopping rule (the solver's own estimates for the preconditioned system): */
/*   test1 = ||r|| / ||b||                         <= tol + tol*||M||*||y||/||b|| */
/*   test2 = ||M^T r|| / (||M||_F ||r||)           <= tol                     */
/* info[0] = iterations, info[1] = istop (1 = test1, 2 = test2, 0 = maxit),  */
/* info[2] = final test2 estimate, info[3] = ||A M||_F estimate.            */
/* ------------------------------------------------------------------------ */
static int lsqr_core(int64_t m, int64_t n, const int32_t* colptr,
                     const int32_t* rowidx, const double* values, const double* b,
                     const precond* pc, double tol, int64_t maxit, double* x,
                     double* info) {
  const int64_t k = pc->k;
  const int64_t kk = k > 0 ? k : 1;
  double* u = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  double* Mv = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  double* v = (double*)malloc(sizeof(double) * (size_t)kk);
  double* w = (double*)malloc(sizeof(double) * (size_t)kk);
  double* y = (double*)malloc(sizeof(double) * (size_t)kk);
  double* t = (double*)malloc(sizeof(double) * (size_t)(n > kk ? n : kk));
  double* t2 = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!u || !Mv || !v || !w || !y || !t || !t2) {
    free(u); free(Mv); free(v); free(w); free(y); free(t); free(t2);
    return -2;
  }
  for (int64_t q = 0; q < k; ++q) y[q] = 0.0;
  for (int64_t j = 0; j < m; ++j) u[j] = b[j];
  double bnorm = vnorm(m, u);
  double beta = bnorm, alpha = 0.0;
  int istop = 0;
  int64_t it = 0;
  double anorm2 = 0.0, test2 = 0.0;
  if (beta > 0.0) {
    for (int64_t j = 0; j < m; ++j) u[j] /= beta;
    csc_rmatvec(n, colptr, rowidx, values, u, t2); /* v = M^T A^T u */
    pc_apply_t(pc, n, t2, v);
    alpha = vnorm(k, v);
  }
  if (alpha > 0.0)
    for (int64_t q = 0; q < k; ++q) v[q] /= alpha;
  for (int64_t q = 0; q < k; ++q) w[q] = v[q];
  double phibar = beta, rhobar = alpha;
  if (alpha == 0.0 || beta == 0.0) istop = 1; /* x = 0 is already exact */
  while (!istop && it < maxit) {
    ++it;
    /* Golub-Kahan bidiagonalisation: beta u = A M v - alpha u */
    pc_apply(pc, n, v, t);
    csc_matvec(m, n, colptr, rowidx, values, t, Mv);
    for (int64_t j = 0; j < m; ++j) u[j] = Mv[j] - alpha * u[j];
    beta = vnorm(m, u);
    if (beta > 0.0)
      for (int64_t j = 0; j < m; ++j) u[j] /= beta;
    anorm2 += alpha * alpha + beta * beta;
    /* alpha v = M^T A^T u - beta v */
    csc_rmatvec(n, colptr, rowidx, values, u, t2);
    pc_apply_t(pc, n, t2, t);
    for (int64_t q = 0; q < k; ++q) v[q] = t[q] - beta * v[q];
    alpha = vnorm(k, v);
    if (alpha > 0.0)
      for (int64_t q = 0; q < k; ++q) v[q] /= alpha;
    /* plane rotation eliminating the subdiagonal beta */
    double rho = sqrt(rhobar * rhobar + beta * beta);
    double c = rhobar / rho, s = beta / rho;
    double theta = s * alpha;
    rhobar = -c * alpha;
    double phi = c * phibar;
    phibar = s * phibar;
    /* solution and search-direction updates */
    for (int64_t q = 0; q < k; ++q) {
      y[q] += (phi / rho) * w[q];
      w[q] = v[q] - (theta / rho) * w[q];
    }
    /* the solver's estimates for the preconditioned system */
    double rnorm = phibar;
    double arnorm = phibar * alpha * fabs(c);
    double anorm = sqrt(anorm2);
    double ynorm = vnorm(k, y);
    double test1 = rnorm / bnorm;
    test2 = (rnorm > 0.0) ? arnorm / (anorm * rnorm) : 0.0;
    double rtol = tol + tol * anorm * ynorm / bnorm;
    if (test2 <= tol) istop = 2;
    if (test1 <= rtol) istop = 1;
  }
  pc_apply(pc, n, y, x); /* x = M y */
  free(u); free(Mv); free(v); free(w); free(y); free(t); free(t2);
  info[0] = (double)it;
  info[1] = (double)istop;
  info[2] = test2;
  info[3] = sqrt(anorm2);
  return istop ? 0 : 1;
}

/* LSQR with M = R^{-1} (R upper triangular, column-major n x n), or M = I
 * when R is NULL.  Returns 0 (converged), 1 (maxit) or -2 (allocation). */
int oracle_lsqr(int64_t m, int64_t n, const int32_t* colptr,
                const int32_t* rowidx, const double* values, const double* b,
                const double* R, double tol, int64_t maxit, double* x,
                double* info) {
  precond pc = {R ? PC_TRI : PC_NONE, n, R, NULL, NULL};
  return lsqr_core(m, n, colptr, rowidx, values, b, &pc, tol, maxit, x, info);
}

/* Full SAP-QR pipeline (Sec. 5.3): A_hat = S A (Alg. 4 order, FP64),
 * Householder QR of A_hat -> R, LSQR on A R^{-1}, x = R^{-1} y.
 * info as for oracle_lsqr, plus info[4] = Error(x). */
int oracle_sap_qr_solve(int64_t m, int64_t n, int64_t d, int dist,
                        uint64_t seed, uint32_t stream, const int32_t* colptr,
                        const int32_t* rowidx, const double* values,
                        const double* b, double tol, int64_t maxit, double* x,
                        double* info) {
  double* Ahat = (double*)malloc(sizeof(double) * (size_t)(d * n));
  double* R = (double*)malloc(sizeof(double) * (size_t)(n * n));
  if (!Ahat || !R) { free(Ahat); free(R); return -2; }
  oracle_sketch_jki_rows(m, n, d, dist, seed, stream, colptr, rowidx, values,
                         Ahat, 0, m);
  int qs = oracle_householder_qr(d, n, Ahat, R);
  int ls = (qs == 0) ? oracle_lsqr(m, n, colptr, rowidx, values, b, R, tol,
                                   maxit, x, info)
                     : -1;
  if (qs == 0) info[4] = oracle_ls_error(m, n, colptr, rowidx, values, b, x);
  free(Ahat); free(R);
  return ls;
}

/* ------------------------------------------------------------------------ */
/* One-sided (Hestenes) Jacobi SVD of a dense d x n matrix (column-major,    */
/* d >= n), FP64.  Sec. 5.3's SVD of the sketch.  Sweeps over all column     */
/* pairs (p < q) in order; a pair whose columns are not orthogonal to        */
/* working precision (|a_p . a_q| > 1e-15 sqrt(||a_p||^2 ||a_q||^2)) is      */
/* rotated by the 2 x 2 symmetric Schur rotation of its Gram matrix          */
/* (Golub & Van Loan, Alg. 8.4.1), which makes the two columns orthogonal;   */
/* V accumulates the rotations.  At convergence A V = U diag(sigma) with     */
/* sigma_j = ||column j||.  sigma (n) is returned in decreasing order with   */
/* the columns of V (n x n, column-major) permuted to match.  Returns the    */
/* number of sweeps, -1 if 80 sweeps did not converge, -2 on allocation      */
/* failure.                                                                  */
/* ------------------------------------------------------------------------ */
int oracle_jacobi_svd(int64_t d, int64_t n, const double* A, double* sigma, double* V) {
  double* W = (double*)malloc(sizeof(double) * (size_t)(d * n));
  double* Vw = (double*)malloc(sizeof(double) * (size_t)(n * n));
  if (!W || !Vw) { free(W); free(Vw); return -2; }
  memcpy(W, A, sizeof(double) * (size_t)(d * n));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) Vw[j * n + i] = (i == j) ? 1.0 : 0.0;
  int sweeps = 0, converged = 0;
  while (!converged && sweeps < 80) {
    ++sweeps;
    int64_t rotations = 0;
    for (int64_t p = 0; p + 1 < n; ++p)
      for (int64_t q = p + 1; q < n; ++q) {
        double* ap = W + p * d;
        double* aq = W + q * d;
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int64_t i = 0; i < d; ++i) {
          alpha += ap[i] * ap[i];
          beta += aq[i] * aq[i];
          gamma += ap[i] * aq[i];
        }
        if (gamma == 0.0 || fabs(gamma) <= 1e-15 * sqrt(alpha * beta)) continue;
        ++rotations;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int64_t i = 0; i < d; ++i) {
          double x0 = ap[i], x1 = aq[i];
          ap[i] = c * x0 - s * x1;
          aq[i] = s * x0 + c * x1;
        }
        double* vp = Vw + p * n;
        double* vq = Vw + q * n;
        for (int64_t i = 0; i < n; ++i) {
          double x0 = vp[i], x1 = vq[i];
          vp[i] = c * x0 - s * x1;
          vq[i] = s * x0 + c * x1;
        }
      }
    if (rotations == 0) converged = 1;
  }
  /* sigma_j = ||column j||, then sort decreasing (selection sort) */
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  double* sv = (double*)malloc(sizeof(double) * (size_t)n);
  if (!order || !sv) { free(W); free(Vw); free(order); free(sv); return -2; }
  for (int64_t j = 0; j < n; ++j) {
    sv[j] = vnorm(d, W + j * d);
    order[j] = j;
  }
  for (int64_t a = 0; a < n; ++a) {
    int64_t best = a;
    for (int64_t c = a + 1; c < n; ++c)
      if (sv[order[c]] > sv[order[best]]) best = c;
    int64_t tmp = order[a]; order[a] = order[best]; order[best] = tmp;
  }
  for (int64_t a = 0; a < n; ++a) {
    sigma[a] = sv[order[a]];
    memcpy(V + a * n, Vw + order[a] * n, sizeof(double) * (size_t)n);
  }
  free(W); free(Vw); free(order); free(sv);
  return converged ? sweeps : -1;
}

/* SAP-SVD (Sec. 5.3): A_hat = S A (Alg. 4 order, FP64), A_hat = U Sigma V^T
 * by the Jacobi SVD above, singular values below sigma_max / 10^12 dropped
 * (k kept), LSQR on A P with P = V_k Sigma_k^{-1} (n x k), x = P y.
 * info as for oracle_lsqr, plus info[4] = Error(x), info[5] = k,
 * info[6] = Jacobi sweeps.  Returns 0, 1 (maxit), -1 (SVD did not
 * converge) or -2 (allocation). */
int oracle_sap_svd_solve(int64_t m, int64_t n, int64_t d, int dist,
                         uint64_t seed, uint32_t stream, const int32_t* colptr,
                         const int32_t* rowidx, const double* values,
                         const double* b, double tol, int64_t maxit, double* x,
                         double* info) {
  double* Ahat = (double*)malloc(sizeof(double) * (size_t)(d * n));
  double* sigma = (double*)malloc(sizeof(double) * (size_t)n);
  double* V = (double*)malloc(sizeof(double) * (size_t)(n * n));
  if (!Ahat || !sigma || !V) { free(Ahat); free(sigma); free(V); return -2; }
  oracle_sketch_jki_rows(m, n, d, dist, seed, stream, colptr, rowidx, values, Ahat, 0, m);
  int sweeps = oracle_jacobi_svd(d, n, Ahat, sigma, V);
  free(Ahat);
  if (sweeps < 0) { free(sigma); free(V); return sweeps == -2 ? -2 : -1; }
  int64_t k = 0;
  while (k < n && sigma[k] > 0.0 && sigma[k] >= sigma[0] / 1e12) ++k;
  /* P = V_k Sigma_k^{-1}: column j of V divided by sigma_j */
  for (int64_t j = 0; j < k; ++j)
    for (int64_t i = 0; i < n; ++i) V[j * n + i] /= sigma[j];
  precond pc = {PC_DENSE, k, NULL, V, NULL};
  int ls = lsqr_core(m, n, colptr, rowidx, values, b, &pc, tol, maxit, x, info);
  if (ls >= 0) {
    info[4] = oracle_ls_error(m, n, colptr, rowidx, values, b, x);
    info[5] = (double)k;
    info[6] = (double)sweeps;
  }
  free(sigma); free(V);
  return ls;
}

/* LSQR-D (Sec. 5.3's first comparator): LSQR with the diagonal
 * preconditioner D_ii = 1 / ||A_i||_2 (A_i the i-th column), except that
 * D_ii = 1 when ||A_i||_2 <= eps sqrt(n) max_i ||A_i||_2 (eps = 2^-52, the
 * FP64 machine epsilon); x = D y.  info as for oracle_lsqr, plus info[4] =
 * Error(x).  Returns 0, 1 (maxit) or -2 (allocation). */
int oracle_lsqr_d_solve(int64_t m, int64_t n, const int32_t* colptr,
                        const int32_t* rowidx, const double* values,
                        const double* b, double tol, int64_t maxit, double* x,
                        double* info) {
  double* D = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!D) return -2;
  double nmax = 0.0;
  for (int64_t k = 0; k < n; ++k) {
    double s = 0.0;
    for (int64_t p = colptr[k]; p < colptr[k + 1]; ++p) s += values[p] * values[p];
    D[k] = sqrt(s);
    if (D[k] > nmax) nmax = D[k];
  }
  const double eps = ldexp(1.0, -52);
  for (int64_t k = 0; k < n; ++k)
    D[k] = (D[k] <= eps * sqrt((double)n) * nmax) ? 1.0 : 1.0 / D[k];
  precond pc = {PC_DIAG, n, NULL, NULL, D};
  int ls = lsqr_core(m, n, colptr, rowidx, values, b, &pc, tol, maxit, x, info);
  if (ls >= 0) info[4] = oracle_ls_error(m, n, colptr, rowidx, values, b, x);
  free(D);
  return ls;
}
