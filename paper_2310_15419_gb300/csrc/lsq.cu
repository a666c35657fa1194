// lsq.cu -- sketch-and-precondition least squares (Sec. 5.3) on the GPU.
//
//   1. A_hat = S A (FP32, the sketch kernels; d = the handle's d, normally 2n)
//   2. Householder QR of A_hat in FP64 -> R  (LAPACK-style reflectors
//      H = I - tau v v^T, v_0 = 1, R(k,k) = -sign(x_0) ||x||, H = I when the
//      part below the diagonal is already zero)
//   3. R^{-1} explicitly (FP64), stored row-major together with R^{-T} so the
//      two matrix-vector products of every iteration read contiguous rows
//   4. LSQR (Paige & Saunders 1982) on M = A R^{-1} with FP64 vectors, norms
//      and recurrences; every reduction runs in a fixed order (deterministic)
//   5. x = R^{-1} y and Error(x) = ||A^T(Ax-b)|| / (||A||_F ||Ax-b||) in FP64
//
// LSQR iterations run as CUDA graphs of kIterPerGraph iterations; every
// kernel returns at once when the device-side `done` flag is set, and the
// host reads the flag after each replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "handle.h"
#include "internal.h"

namespace sk {

namespace {

constexpr int kIterPerGraph = 8;

// LSQR state that one iteration reads and the next writes lives in two slots
// indexed by the parity of the iteration inside a captured graph, so that no
// kernel reads a slot it writes.
struct Slot {
  double alpha, rhobar, phibar, anorm2;  // alpha_k, rhobar_k, phibar_k, ||B_k||_F^2
  double cabs;    // |c| of the last plane rotation
  double f_next;  // alpha_k / beta_k for the next rows pass
  int iters, pad;
};

struct Scalars {
  double beta, inv_beta, bnorm, tol;
  double usq;   // ||u_raw||^2 after the rows pass
  double zsq;   // the part of usq from rows of A with no nonzero
  double ynorm2;
  double afro2, err_num2, err_res2;
  Slot slot[2];
  int maxit, done, istop, latest;  // latest: slot of the last finished iteration
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in a fixed order; every thread gets the result.
template <int NT>
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < NT / 32 ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// float -> double, exactly, with integer operations for zeros and normal
// numbers (IEEE 754 binary32 -> binary64: rebias the exponent by 1023 - 127,
// widen the significand by 29 bits); subnormals, infinities and NaNs take
// the conversion instruction.
__device__ __forceinline__ double f64_of(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) {
    if ((b << 1) == 0u)
      return __longlong_as_double(static_cast<long long>(static_cast<uint64_t>(b) << 32));
    return static_cast<double>(f);
  }
  const uint64_t bits = (static_cast<uint64_t>(b & 0x80000000u) << 32) |
                        (static_cast<uint64_t>(e + 896u) << 52) |
                        (static_cast<uint64_t>(b & 0x7fffffu) << 29);
  return __longlong_as_double(static_cast<long long>(bits));
}

// Block-wide fixed-order sum for kernels of NT threads (warp 0 gets it):
// every thread stores its value, then lane l of warp 0 adds entries l,
// l + 32, ... and the warp adds across lanes.  That is NT/32 + 5 FP64
// instructions for the block instead of five per warp.  red holds NT
// doubles.
template <int NT>
__device__ __forceinline__ double block_sum0(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  double p = 0.0;
  if (threadIdx.x < 32) {
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int q = 0; q < NT / 32; q += 2) {
      a0 += red[threadIdx.x + 32 * q];
      if (q + 1 < NT / 32) a1 += red[threadIdx.x + 32 * (q + 1)];
    }
    p = warp_sum(a0 + a1);
  }
  __syncthreads();
  return p;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor finishes; it reads only
// data the predecessor does not write before pdl_wait(), which returns once
// the predecessor has completed and its writes are visible.  Each kernel
// lets its successor launch only after its own wait, so everything older
// than the predecessor is complete when the successor starts.  Without the
// launch attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename VT>
__device__ __forceinline__ double val_at(const VT* v, int64_t i) {
  return f64_of(to_f32(v[i]));
}

// ---------------------------------------------------------------------------
// QR
// ---------------------------------------------------------------------------
__global__ void k_to_double(int64_t total, const float* __restrict__ a,
                            double* __restrict__ w) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       i < total; i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    w[i] = static_cast<double>(a[i]);
}

constexpr int kQrThreads = 128;
constexpr int kQrRegs = 8;  // column entries a thread keeps in registers
constexpr int kQrCols = 4;  // columns an update block carries at once

// Householder QR of W (d x n, column-major) with LAPACK's reflectors
// H_k = I - tau_k v_k v_k^T, v_k(k) = 1, R(k,k) = beta = -sign(alpha) ||x||
// (H = I, tau = 0, when the part below the diagonal is already zero).  Below
// the diagonal column k keeps v_k unscaled: v_k(r) = vs[k] * W(r,k), r > k,
// with vs[k] = 1 / (alpha - beta); consumers fold vs[k] into their scalars.
//
// Step k is one launch of min(n - k - 1, #SMs) blocks, so each block has an
// SM to itself.  Block 0 carries the critical path: it applies H_k to
// column k + 1 and forms reflector k + 1 (a dot product, an update fused
// with the squared norm, two block sums and one sqrt / two divides in
// thread 0).  The other blocks apply H_k to columns k + 2 .. n - 1, up to
// kQrCols at a time, one warp reducing each column's dot product.

// Column c = k + 1: apply H_k (k >= 0), then form reflector c.
__device__ void qr_form(double* __restrict__ W, int64_t d, int k, double* __restrict__ tau,
                        double* __restrict__ vs, double* red, double* bc) {
  const int tid = threadIdx.x;
  const int c = k + 1;
  double* y = W + static_cast<int64_t>(c) * d;
  const int64_t r0 = c;  // rows r0.. are touched (row k separately)
  const int64_t rtail = r0 + static_cast<int64_t>(kQrThreads) * kQrRegs;
  const double t = k >= 0 ? tau[k] : 0.0;
  const double* w = W + static_cast<int64_t>(k >= 0 ? k : 0) * d;
  double yr[kQrRegs], wr[kQrRegs];
#pragma unroll
  for (int q = 0; q < kQrRegs; ++q) {
    const int64_t r = r0 + tid + kQrThreads * q;
    yr[q] = r < d ? y[r] : 0.0;
    wr[q] = (t != 0.0 && r < d) ? w[r] : 0.0;
  }
  double nrm = 0.0;
  if (t != 0.0) {
    const double sk = vs[k];
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int q = 0; q < kQrRegs; q += 2) {
      s0 = fma(wr[q], yr[q], s0);
      s1 = fma(wr[q + 1], yr[q + 1], s1);
    }
    for (int64_t r = rtail + tid; r < d; r += kQrThreads) s0 = fma(w[r], y[r], s0);
    const double sum = block_sum0<kQrThreads>(s0 + s1, red);
    if (tid == 0) {
      const double yk = y[k];
      const double f = t * fma(sk, sum, yk);
      y[k] = yk - f;
      bc[0] = f * sk;
    }
    __syncthreads();
    const double g = bc[0];
#pragma unroll
    for (int q = 0; q < kQrRegs; ++q) {
      const int64_t r = r0 + tid + kQrThreads * q;
      yr[q] = fma(-g, wr[q], yr[q]);
      if (r > c) nrm = fma(yr[q], yr[q], nrm);
    }
    for (int64_t r = rtail + tid; r < d; r += kQrThreads) {
      const double v = fma(-g, w[r], y[r]);
      y[r] = v;
      nrm = fma(v, v, nrm);
    }
  } else {
#pragma unroll
    for (int q = 0; q < kQrRegs; ++q) {
      const int64_t r = r0 + tid + kQrThreads * q;
      if (r > c) nrm = fma(yr[q], yr[q], nrm);
    }
    for (int64_t r = rtail + tid; r < d; r += kQrThreads) nrm = fma(y[r], y[r], nrm);
  }
  const double sigma = block_sum0<kQrThreads>(nrm, red);
  if (tid == 0) {
    if (sigma == 0.0) {
      tau[c] = 0.0;
      vs[c] = 1.0;
    } else {
      const double alpha = yr[0];  // row c
      const double norm = sqrt(fma(alpha, alpha, sigma));
      const double beta = alpha >= 0.0 ? -norm : norm;
      vs[c] = 1.0 / (alpha - beta);
      tau[c] = (beta - alpha) / beta;
      yr[0] = beta;
    }
  }
  if (t != 0.0 || tid == 0) {
#pragma unroll
    for (int q = 0; q < kQrRegs; ++q) {
      const int64_t r = r0 + tid + kQrThreads * q;
      if (r < d) y[r] = yr[q];
    }
  }
}

// Apply H_k to up to kQrCols columns cols[0..nc) (rows k..d-1).
__device__ void qr_apply(double* __restrict__ W, int64_t d, int k, const int* cols, int nc,
                         const double* __restrict__ wr, double t, double sk, double* red,
                         double* bc) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = k + 1;
  const int64_t rtail = r0 + static_cast<int64_t>(kQrThreads) * kQrRegs;
  const double* w = W + static_cast<int64_t>(k) * d;
  double yr[kQrCols][kQrRegs];
#pragma unroll
  for (int j = 0; j < kQrCols; ++j) {
    const double* y = W + static_cast<int64_t>(j < nc ? cols[j] : cols[0]) * d;
#pragma unroll
    for (int q = 0; q < kQrRegs; ++q) {
      const int64_t r = r0 + tid + kQrThreads * q;
      yr[j][q] = (j < nc && r < d) ? y[r] : 0.0;
    }
  }
#pragma unroll
  for (int j = 0; j < kQrCols; ++j) {
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int q = 0; q < kQrRegs; q += 2) {
      s0 = fma(wr[q], yr[j][q], s0);
      s1 = fma(wr[q + 1], yr[j][q + 1], s1);
    }
    if (j < nc) {
      const double* y = W + static_cast<int64_t>(cols[j]) * d;
      for (int64_t r = rtail + tid; r < d; r += kQrThreads) s0 = fma(w[r], y[r], s0);
    }
    red[j * kQrThreads + tid] = s0 + s1;
  }
  __syncthreads();
  // warp j sums column j in a fixed order
  if (warp < nc) {
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int q = 0; q < kQrThreads / 32; q += 2) {
      a0 += red[warp * kQrThreads + lane + 32 * q];
      a1 += red[warp * kQrThreads + lane + 32 * (q + 1)];
    }
    const double sum = warp_sum(a0 + a1);
    if (lane == 0) {
      double* y = W + static_cast<int64_t>(cols[warp]) * d;
      const double yk = y[k];
      const double f = t * fma(sk, sum, yk);
      y[k] = yk - f;
      bc[warp] = f * sk;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kQrCols; ++j) {
    if (j < nc) {
      const double g = bc[j];
      double* y = W + static_cast<int64_t>(cols[j]) * d;
#pragma unroll
      for (int q = 0; q < kQrRegs; ++q) {
        const int64_t r = r0 + tid + kQrThreads * q;
        if (r < d) y[r] = fma(-g, wr[q], yr[j][q]);
      }
      for (int64_t r = rtail + tid; r < d; r += kQrThreads) y[r] = fma(-g, w[r], y[r]);
    }
  }
  __syncthreads();  // red and bc are reused by the next group of columns
}

__global__ void __launch_bounds__(kQrThreads)
    k_qr_first(double* W, int64_t d, double* tau, double* vs) {
  __shared__ double red[kQrThreads];
  __shared__ double bc[kQrCols];
  qr_form(W, d, -1, tau, vs, red, bc);
}

// Step k (see above).  Launched with programmatic stream serialization:
// every read depends on the previous step.
__global__ void __launch_bounds__(kQrThreads)
    k_qr_step(double* W, int64_t d, int n, int k, double* tau, double* vs) {
  __shared__ double red[kQrThreads * kQrCols];
  __shared__ double bc[kQrCols];
  pdl_wait();
  pdl_launch();
  if (blockIdx.x == 0) {
    qr_form(W, d, k, tau, vs, red, bc);
    return;
  }
  const double t = tau[k];
  if (t == 0.0) return;
  const double sk = vs[k];
  const double* w = W + static_cast<int64_t>(k) * d;
  double wr[kQrRegs];
#pragma unroll
  for (int q = 0; q < kQrRegs; ++q) {
    const int64_t r = k + 1 + threadIdx.x + kQrThreads * q;
    wr[q] = r < d ? w[r] : 0.0;
  }
  const int nb = gridDim.x - 1;
  for (int c0 = k + 2 + static_cast<int>(blockIdx.x) - 1; c0 < n; c0 += nb * kQrCols) {
    int cols[kQrCols];
    int nc = 0;
#pragma unroll
    for (int j = 0; j < kQrCols; ++j) {
      const int c = c0 + nb * j;
      cols[j] = c < n ? c : c0;
      nc += c < n;
    }
    qr_apply(W, d, k, cols, nc, wr, t, sk, red, bc);
  }
}

// Blocks of step k: one for column k + 1, the rest for columns k + 2 ..
unsigned qr_step_blocks(int64_t n, int k) {
  return static_cast<unsigned>(
      1 + std::min<int64_t>(std::max<int64_t>(n - k - 2, 0), num_sms() - 1));
}

// Rrow = R (upper n x n of W) row-major, rdiag = 1 / diag(R); flags a zero
// diagonal.
__global__ void k_extract_r(const double* __restrict__ W, int64_t d, int n,
                            double* __restrict__ Rrow, double* __restrict__ rdiag,
                            int* status) {
  const int64_t total = static_cast<int64_t>(n) * n;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       t < total; t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(t / n), c = static_cast<int>(t % n);
    const double v = c >= i ? W[static_cast<int64_t>(c) * d + i] : 0.0;
    Rrow[t] = v;
    if (c == i) {
      rdiag[i] = v != 0.0 ? 1.0 / v : 0.0;
      if (v == 0.0) atomicOr(status, 4);
    }
  }
}

// X = R^{-1} by back substitution, one block per column j of X (longest
// first), in the column (axpy) form: with s = e_j, for c = j, j-1, ..., 0:
//   X[c][j] = s[c] / R[c][c];   s[0..c-1] -= R[0..c-1][c] * X[c][j].
// s lives in shared memory (n doubles); R is read column-major from the QR
// workspace W, the next column while the current one is applied; rdiag =
// 1 / diag(R).  Thread t owns rows t + blockDim.x q, q < NR.  Writes Xrow
// (row-major X) and XTrow (row-major X^T).
template <int NR>
__global__ void k_trtri(const double* __restrict__ W, int64_t d, int n,
                        const double* __restrict__ rdiag, double* __restrict__ Xrow,
                        double* __restrict__ XTrow) {
  extern __shared__ double sx[];
  const int T = blockDim.x, tid = threadIdx.x;
  const int j = n - 1 - static_cast<int>(blockIdx.x);
  for (int r = tid; r <= j; r += T) sx[r] = r == j ? 1.0 : 0.0;
  double rc[NR], rn[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    const int r = tid + T * q;
    rc[q] = r < j ? W[static_cast<int64_t>(j) * d + r] : 0.0;
  }
  __syncthreads();
  for (int c = j; c >= 0; --c) {
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const int r = tid + T * q;
      rn[q] = r < c - 1 ? W[static_cast<int64_t>(c - 1) * d + r] : 0.0;
    }
    const double xc = sx[c] * rdiag[c];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const int r = tid + T * q;
      if (r < c) sx[r] = fma(-rc[q], xc, sx[r]);
    }
    __syncthreads();
    if (tid == 0) sx[c] = xc;
#pragma unroll
    for (int q = 0; q < NR; ++q) rc[q] = rn[q];
  }
  __syncthreads();
  for (int r = tid; r < n; r += T) {
    const double x = r <= j ? sx[r] : 0.0;
    Xrow[static_cast<int64_t>(r) * n + j] = x;
    XTrow[static_cast<int64_t>(j) * n + r] = x;
  }
}

// Launch of k_trtri: NR = 4 rows per thread up to n = 4096, else 8.
cudaError_t launch_trtri(const double* W, int64_t d, int n, const double* rdiag,
                         double* Xrow, double* XTrow, cudaStream_t s) {
  const size_t smem = sizeof(double) * static_cast<size_t>(n);
  if (n <= 4096) {
    int T = 128;
    while (T * 4 < n) T *= 2;
    const cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(k_trtri<4>), smem);
    if (e != cudaSuccess) return e;
    k_trtri<4><<<n, T, smem, s>>>(W, d, n, rdiag, Xrow, XTrow);
  } else {
    const cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(k_trtri<8>), smem);
    if (e != cudaSuccess) return e;
    k_trtri<8><<<n, 1024, smem, s>>>(W, d, n, rdiag, Xrow, XTrow);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// LSQR kernels
//
// On this GPU a warp-wide FP64 instruction occupies its SM partition's FP64
// pipe for about 80 cycles whatever the number of active lanes, and a
// dependent FP64 add, sqrt or divide costs about 67, 720 and 460 cycles.  So
// the kernels below keep FP64 scalar chains in one thread per block, reduce
// per thread before reducing across lanes, convert float values to double
// with integer operations, and let the scalar chain of one step overlap the
// vector work of the next.  One iteration is four kernels:
//   rows:  u_raw <- A t - (alpha/beta) u_raw and per-block sums of u_raw^2
//   cols:  t2 <- A^T u_raw (unscaled)
//   vraw:  beta <- ||u_raw|| (every block, same fixed order) while the warps
//          form rows of R^{-T} t2; vraw = R^{-T} t2 / beta - beta v and
//          per-block sums of vraw^2
//   step:  alpha <- ||vraw||, the plane rotation, v = vraw/alpha,
//          y += (phi/rho) w, w = v - (theta/rho) w, t = R^{-1} v for the next
//          rows pass; the last block to finish forms the stopping tests.
// Each kernel returns at once when `done` is set.
// ---------------------------------------------------------------------------
constexpr int kRows = 256;  // threads per block of the rows pass
constexpr int kTriWarps = 4;  // rows of R^{-1} / R^{-T} per block

// The first 256 entries of a warp's row [lo, hi): lane l holds
// row[lo + l + 32 q], q < 8 (0 beyond hi).
__device__ __forceinline__ void row_chunk(const double* __restrict__ row, int64_t lo,
                                          int64_t hi, int lane, double r[8]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t c = lo + lane + 32 * q;
    r[q] = c < hi ? row[c] : 0.0;
  }
}

// sum_{c in [lo, hi)} row[c] x[c] across one warp (every lane gets it), with
// the first 256 row entries already in r0 (row_chunk).  Each later round
// issues all sixteen loads of a lane before the first multiply, so a row
// costs one memory latency per 256 entries.
__device__ __forceinline__ double warp_row_dot_pre(const double* __restrict__ row,
                                                   const double* __restrict__ x,
                                                   int64_t lo, int64_t hi, int lane,
                                                   const double r0[8]) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  {
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t c = lo + lane + 32 * q;
      v[q] = c < hi ? x[c] : 0.0;
    }
    a0 = fma(r0[0], v[0], a0); a1 = fma(r0[1], v[1], a1);
    a2 = fma(r0[2], v[2], a2); a3 = fma(r0[3], v[3], a3);
    a0 = fma(r0[4], v[4], a0); a1 = fma(r0[5], v[5], a1);
    a2 = fma(r0[6], v[6], a2); a3 = fma(r0[7], v[7], a3);
  }
  for (int64_t c0 = lo + lane + 256; c0 < hi; c0 += 256) {
    double r[8], v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t c = c0 + 32 * q;
      r[q] = c < hi ? row[c] : 0.0;
      v[q] = c < hi ? x[c] : 0.0;
    }
    a0 = fma(r[0], v[0], a0); a1 = fma(r[1], v[1], a1);
    a2 = fma(r[2], v[2], a2); a3 = fma(r[3], v[3], a3);
    a0 = fma(r[4], v[4], a0); a1 = fma(r[5], v[5], a1);
    a2 = fma(r[6], v[6], a2); a3 = fma(r[7], v[7], a3);
  }
  return warp_sum((a0 + a1) + (a2 + a3));
}

__device__ __forceinline__ double warp_row_dot(const double* __restrict__ row,
                                               const double* __restrict__ x,
                                               int64_t lo, int64_t hi, int lane) {
  double r0[8];
  row_chunk(row, lo, hi, lane, r0);
  return warp_row_dot_pre(row, x, lo, hi, lane, r0);
}

// Fixed-order sum of part[0..np) by one warp (every lane gets it); loads in
// rounds of eight per lane.
__device__ __forceinline__ double warp_sum_parts(const double* __restrict__ part,
                                                 int np, int lane) {
  double a0 = 0.0, a1 = 0.0;
  for (int g0 = lane; g0 < np; g0 += 256) {
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = g0 + 32 * q < np ? part[g0 + 32 * q] : 0.0;
    a0 += (v[0] + v[2]) + (v[4] + v[6]);
    a1 += (v[1] + v[3]) + (v[5] + v[7]);
  }
  return warp_sum(a0 + a1);
}

// The preconditioner M of LSQR on A M (x = M y), kept as two row-major n x n
// matrices, M and M^T:
//   kPcTri   M = R^{-1} (SAP-QR): M upper triangular, M^T lower triangular
//   kPcDense M = V_k Sigma_k^{-1} padded with zero columns (SAP-SVD): full
//   kPcDiag  M = diag(D) (LSQR-D): only the diagonal is read
constexpr int kPcTri = 0, kPcDense = 1, kPcDiag = 2;

// Columns [lo, hi) of row i that can be nonzero, for M (lower = 0) or M^T
// (lower = 1).
__device__ __forceinline__ void pc_range(int pk, int lower, int64_t i, int n, int64_t& lo,
                                         int64_t& hi) {
  if (pk == kPcDense) {
    lo = 0;
    hi = n;
  } else if (pk == kPcDiag) {
    lo = i;
    hi = i + 1;
  } else {
    lo = lower ? 0 : i;
    hi = lower ? i + 1 : n;
  }
}

// out[i] = sum_c Mrow[i][c] x[c] over the columns pc_range allows.  One warp
// per row.  Used for x = M y.
__global__ void k_gemv_tri(const double* __restrict__ Mrow, int n,
                           const double* __restrict__ x, double* __restrict__ out,
                           int lower, int pk) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5);
       i < n; i += warps) {
    int64_t lo, hi;
    pc_range(pk, lower, i, n, lo, hi);
    const double s = warp_row_dot(Mrow + i * n, x, lo, hi, lane);
    if (lane == 0) out[i] = s;
  }
}

// Rows pass over the CSR whose rows are ordered by decreasing length (row p
// of it is row perm[p] of A; rows [0, *mnz) have nonzeros).  u_raw is double
// buffered: the pass reads uin and writes uout.
// init: uout[p] = b[perm[p]] for every row; partial = sums of uout^2 over
// the rows with nonzeros, partial_z over the others.
// Otherwise, for p < *mnz: uout[p] = sum_e val t[col] - f uin[p] with
// f = alpha_k / beta_k; partial as above.  Rows without nonzeros follow
// u_raw <- -f u_raw, which only scales their sum of squares; the columns
// pass applies that factor to it instead of touching them.
__global__ void __launch_bounds__(kRows, 8)
    k_lsqr_rows(int32_t m, const int32_t* __restrict__ mnz_ptr,
                const int32_t* __restrict__ rowptr, const int32_t* __restrict__ ccol,
                const float* __restrict__ cval, const double* __restrict__ t,
                const double* __restrict__ uin, double* __restrict__ uout,
                const double* __restrict__ b, const int32_t* __restrict__ perm,
                double* __restrict__ partial, double* __restrict__ partial_z,
                const Scalars* __restrict__ sc, int par, int init) {
  __shared__ double red[kRows];
  const int32_t mnz = *mnz_ptr;
  pdl_wait();
  pdl_launch();
  if (sc->done) return;
  const double f = init ? 0.0 : sc->slot[par].f_next;
  const int64_t rows = init ? m : mnz;
  double s2 = 0.0, sz = 0.0;
  for (int64_t p = blockIdx.x * static_cast<int64_t>(kRows) + threadIdx.x; p < rows;
       p += static_cast<int64_t>(gridDim.x) * kRows) {
    if (init) {
      const double nu = b[perm[p]];
      uout[p] = nu;
      if (p < mnz)
        s2 = fma(nu, nu, s2);
      else
        sz = fma(nu, nu, sz);
    } else {
      const int32_t lo = rowptr[p], hi = rowptr[p + 1];
      const double up = uin[p];
      double acc = 0.0;
      for (int32_t e = lo; e < hi; ++e) acc = fma(f64_of(cval[e]), t[ccol[e]], acc);
      const double nu = fma(-f, up, acc);
      uout[p] = nu;
      s2 = fma(nu, nu, s2);
    }
  }
  s2 = block_sum0<kRows>(s2, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s2;
  if (init) {
    sz = block_sum0<kRows>(sz, red);
    if (threadIdx.x == 0) partial_z[blockIdx.x] = sz;
  }
}

// Paige & Saunders' stopping rules for the iterate in slot S, without
// divisions or square roots:  istop 1 when ||r|| <= tol ||b|| + tol ||A||
// ||y|| (compatible system), istop 2 when ||M^T r|| <= tol ||M|| ||r||
// (least-squares solution), with ||r|| = phibar, ||M^T r|| = phibar alpha |c|
// and ||M||^2 estimated by anorm2.  Returns istop, or -1 at maxit.
__device__ __forceinline__ int lsqr_test(const Slot& S, double bnorm, double tol, double y2,
                                         int maxit) {
  if (S.iters == 0) return (S.alpha == 0.0 || bnorm == 0.0) ? 1 : 0;
  const double rnorm = S.phibar;
  const double arnorm = rnorm * S.alpha * S.cabs;
  const double tol2 = tol * tol;
  int istop = 0;
  if (rnorm == 0.0 || arnorm * arnorm <= tol2 * S.anorm2 * (rnorm * rnorm)) istop = 2;
  const double lhs = rnorm - tol * bnorm;
  if (lhs <= 0.0 || lhs * lhs <= tol2 * S.anorm2 * y2) istop = 1;
  if (istop == 0 && S.iters >= maxit) return -1;
  return istop;
}

// Records the outcome of lsqr_test (one thread).
__device__ __forceinline__ bool lsqr_record(Scalars* sc, int istop, double y2) {
  if (istop == 0) return false;
  sc->istop = istop > 0 ? istop : 0;
  sc->ynorm2 = y2;
  sc->done = 1;
  return true;
}

// Columns pass: out[k] = sum_{e in column k} val[e] u[row[e]] (unscaled), one
// block of 32*W threads per column k < n, fixed-order reduction.  With
// lsqr = 1 the grid has one more block, which first applies the stopping
// test to the previous iteration (slot par, sums of y^2 in party; not at
// start-up) and sets `done`, else completes ||u_raw||^2 = sum partial2 + z,
// with z = sum partial_z (init) or f^2 times the previous z (rows without
// nonzeros).
template <typename VT, int W>
__global__ void __launch_bounds__(32 * W)
    k_cols(int32_t n, const int32_t* __restrict__ colptr,
           const int32_t* __restrict__ rowidx, const VT* __restrict__ vals,
           const double* __restrict__ u, double* __restrict__ out, Scalars* sc, int lsqr,
           const double* __restrict__ partial2, const double* __restrict__ partial_z,
           int np2, const double* __restrict__ party, int npy, int par, int init) {
  __shared__ double red[32 * W];
  __shared__ int stop;
  const int k = blockIdx.x;
  if (k == n) {  // the scalar block
    // the test reads only what the step kernel before the rows pass wrote
    if (!init && !sc->done) {
      double a = 0.0;
      for (int g0 = threadIdx.x; g0 < npy; g0 += 4 * 32 * W) {
        double v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int g = g0 + 32 * W * q;
          v[q] = g < npy ? party[g] : 0.0;
        }
        a += (v[0] + v[1]) + (v[2] + v[3]);
      }
      const double y2 = block_sum0<32 * W>(a, red);
      if (threadIdx.x == 0) {
        const int istop = lsqr_test(sc->slot[par], sc->bnorm, sc->tol, y2, sc->maxit);
        stop = lsqr_record(sc, istop, y2);
      }
      __syncthreads();
      if (stop) {
        pdl_launch();
        return;
      }
    }
    pdl_wait();
    pdl_launch();
    if (sc->done) return;
    // fixed-order sums of the rows pass's partials, eight loads per thread
    // in flight per round
    double a = 0.0, z = 0.0;
    for (int g0 = threadIdx.x; g0 < np2; g0 += 8 * 32 * W) {
      double v[8], vz[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int g = g0 + 32 * W * q;
        v[q] = g < np2 ? partial2[g] : 0.0;
        vz[q] = (init && g < np2) ? partial_z[g] : 0.0;
      }
      a += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
      if (init) z += ((vz[0] + vz[1]) + (vz[2] + vz[3])) + ((vz[4] + vz[5]) + (vz[6] + vz[7]));
    }
    a = block_sum0<32 * W>(a, red);
    if (init) z = block_sum0<32 * W>(z, red);
    if (threadIdx.x == 0) {
      if (!init) {
        const double f = sc->slot[par].f_next;
        z = f * f * sc->zsq;
      }
      sc->zsq = z;
      sc->usq = a + z;
    }
    return;
  }
  const int32_t lo = colptr[k], hi = colptr[k + 1];
  double a0 = 0.0, a1 = 0.0;
  bool first = true;
  for (int32_t e0 = lo + threadIdx.x; e0 < hi || first; e0 += 256 * W) {
    int32_t row[8];
    double val[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int32_t e = e0 + 32 * W * q;
      row[q] = e < hi ? rowidx[e] : -1;
      val[q] = e < hi ? val_at(vals, e) : 0.0;
    }
    if (first) {  // the indices and values are the caller's: load them first
      first = false;
      pdl_wait();
      pdl_launch();
      if (lsqr) {  // the scalar block of this grid may set `done` meanwhile
        if (threadIdx.x == 0) stop = sc->done;
        __syncthreads();
        if (stop) return;
      }
    }
    double uu[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) uu[q] = row[q] >= 0 ? u[row[q]] : 0.0;
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      a0 = fma(val[q], uu[q], a0);
      a1 = fma(val[q + 1], uu[q + 1], a1);
    }
  }
  const double s = block_sum0<32 * W>(a0 + a1, red);
  if (threadIdx.x == 0) out[k] = s;
}

// The stopping test alone (one warp), for the last iteration of a captured
// graph.
__global__ void k_lsqr_test(const double* __restrict__ party, int npy, Scalars* sc, int par) {
  pdl_wait();
  pdl_launch();
  if (sc->done) return;
  const double y2 = warp_sum_parts(party, npy, threadIdx.x & 31);
  if (threadIdx.x == 0)
    lsqr_record(sc, lsqr_test(sc->slot[par], sc->bnorm, sc->tol, y2, sc->maxit), y2);
}

// vraw = R^{-T} t2 / beta - beta v  (init: without the beta v term), one warp
// per row of the row-major lower-triangular R^{-T}.  Every block forms
// 1/beta = rsqrt(usq) and beta while its warps form their dot products;
// block 0 publishes them.  partial4[block] = sum of vraw^2 over its rows.
__global__ void __launch_bounds__(32 * kTriWarps)
    k_lsqr_vraw(int n, const double* __restrict__ RinvT, const double* __restrict__ t2,
                const double* __restrict__ v, double* __restrict__ vraw,
                double* __restrict__ partial4, Scalars* sc, int init, int pk) {
  __shared__ double sh[2 + kTriWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kTriWarps + warp;
  const bool has = i < n;
  int64_t lo = 0, hi = 0;
  if (has) pc_range(pk, 1, i, n, lo, hi);
  double r0[8];  // M^T and v are not written by the columns pass
  row_chunk(RinvT + (has ? i : 0) * n, lo, hi, lane, r0);
  const double vi = (!init && has && lane == 0) ? v[i] : 0.0;
  pdl_wait();
  pdl_launch();
  if (sc->done) return;
  if (threadIdx.x == 0) {
    const double usq = sc->usq;
    const double ib = usq > 0.0 ? rsqrt(usq) : 0.0;
    sh[0] = usq * ib;
    sh[1] = ib;
  }
  const double dot = has ? warp_row_dot_pre(RinvT + i * n, t2, lo, hi, lane, r0) : 0.0;
  __syncthreads();
  const double beta = sh[0], ib = sh[1];
  if (lane == 0) {
    double vr2 = 0.0;
    if (i < n) {
      const double vr = fma(-beta, vi, ib * dot);
      vraw[i] = vr;
      vr2 = vr * vr;
    }
    sh[2 + warp] = vr2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double p = 0.0;
#pragma unroll
    for (int w = 0; w < kTriWarps; ++w) p += sh[2 + w];
    partial4[blockIdx.x] = p;
    if (blockIdx.x == 0) {
      sc->beta = beta;
      sc->inv_beta = ib;
    }
  }
}

// One LSQR step after vraw: alpha = ||vraw|| (every block, same fixed
// order), the plane rotation, v = vraw / alpha, y += (phi/rho) w,
// w = v - (theta/rho) w, and t = R^{-1} v for the next rows pass (one warp
// per row of the row-major upper-triangular R^{-1}; element i of v, w, y
// belongs to the warp of row i).  Reads slot par, block 0 writes slot
// par ^ 1; party[block] = sum of y^2 over its rows.  init: start-up
// (v = w = vraw / alpha, y = 0, rhobar = alpha, phibar = beta).
__global__ void __launch_bounds__(32 * kTriWarps)
    k_lsqr_step(int n, const double* __restrict__ Rinv, const double* __restrict__ vraw,
                double* __restrict__ v, double* __restrict__ w, double* __restrict__ y,
                double* __restrict__ t, const double* __restrict__ partial4, int np4,
                double* __restrict__ party, Scalars* sc, int par, int init, int pk) {
  __shared__ double sh[8 + kTriWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kTriWarps + warp;
  const bool has = i < n;
  int64_t lo = 0, hi = 0;
  if (has) pc_range(pk, 0, i, n, lo, hi);
  // M, w, y and slot par are not written by the vraw kernel
  double r0[8];
  row_chunk(Rinv + (has ? i : 0) * n, lo, hi, lane, r0);
  double wi = 0.0, yi = 0.0;
  if (lane == 0 && has && !init) {
    wi = w[i];
    yi = y[i];
  }
  Slot S{};
  if (threadIdx.x == 0 && !init) S = sc->slot[par];
  pdl_wait();
  pdl_launch();
  if (sc->done) return;
  const double vri = (lane == 0 && has) ? vraw[i] : 0.0;
  if (warp == 0) {
    const double s = warp_sum_parts(partial4, np4, lane);
    if (lane == 0) {
      const double ia = s > 0.0 ? rsqrt(s) : 0.0;
      const double alpha = s * ia;
      const double beta = sc->beta;
      Slot o{};
      o.alpha = alpha;
      o.f_next = alpha * sc->inv_beta;
      double f_y = 0.0, f_w = 0.0;
      if (init) {
        o.rhobar = alpha;
        o.phibar = beta;
      } else {
        const double rb = S.rhobar, pb = S.phibar;
        const double irho = rsqrt(fma(rb, rb, beta * beta));
        const double c = rb * irho, sn = beta * irho;
        f_y = c * pb * irho;
        f_w = sn * alpha * irho;
        o.rhobar = -c * alpha;
        o.phibar = sn * pb;
        o.cabs = fabs(c);
        o.anorm2 = S.anorm2 + S.alpha * S.alpha + beta * beta;
        o.iters = S.iters + 1;
      }
      if (blockIdx.x == 0) {
        sc->slot[par ^ 1] = o;
        sc->latest = par ^ 1;
        if (init) sc->bnorm = beta;
      }
      sh[0] = ia;
      sh[1] = f_y;
      sh[2] = f_w;
    }
  }
  const double dot = has ? warp_row_dot_pre(Rinv + i * n, vraw, lo, hi, lane, r0) : 0.0;
  __syncthreads();
  const double ia = sh[0];
  if (lane == 0) {
    double y2 = 0.0;
    if (i < n) {
      t[i] = ia * dot;
      const double vi = ia * vri;
      v[i] = vi;
      if (init) {
        w[i] = vi;
        y[i] = 0.0;
      } else {
        const double yn = fma(sh[1], wi, yi);
        y[i] = yn;
        w[i] = fma(-sh[2], wi, vi);
        y2 = yn * yn;
      }
    }
    sh[8 + warp] = y2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double p = 0.0;
#pragma unroll
    for (int q = 0; q < kTriWarps; ++q) p += sh[8 + q];
    party[blockIdx.x] = p;
  }
}

// Error check: r = A x - b over the length-ordered CSR (row p is row perm[p]
// of A) and per-block sums of r^2.
__global__ void __launch_bounds__(kRows)
    k_residual(int32_t m, const int32_t* __restrict__ rowptr,
               const int32_t* __restrict__ ccol, const float* __restrict__ cval,
               const double* __restrict__ x, const double* __restrict__ b,
               const int32_t* __restrict__ perm, double* __restrict__ r,
               double* __restrict__ partial) {
  __shared__ double red[kRows / 32];
  double s2 = 0.0;
  for (int64_t j = blockIdx.x * static_cast<int64_t>(kRows) + threadIdx.x; j < m;
       j += static_cast<int64_t>(gridDim.x) * kRows) {
    double s = 0.0;
    const int32_t hi = rowptr[j + 1];
    for (int32_t e = rowptr[j]; e < hi; ++e) s = fma(f64_of(cval[e]), x[ccol[e]], s);
    const double rj = s - b[perm[j]];
    r[j] = rj;
    s2 = fma(rj, rj, s2);
  }
  s2 = warp_sum(s2);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = s2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double p = 0.0;
#pragma unroll
    for (int w = 0; w < kRows / 32; ++w) p += red[w];
    partial[blockIdx.x] = p;
  }
}

template <typename VT>
__global__ void k_fro2(int64_t nnz, const VT* __restrict__ vals,
                       double* __restrict__ partial) {
  __shared__ double red[33];
  double s = 0.0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       e < nnz; e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double v = val_at(vals, e);
    s = fma(v, v, s);
  }
  s = block_sum<256>(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Error(x) pieces: ||A||_F^2, ||A x - b||^2 and ||A^T (A x - b)||^2, each a
// fixed-order sum by one warp.
__global__ void k_finish_error(const double* __restrict__ pfro, int nfro,
                               const double* __restrict__ pres, int nres,
                               const double* __restrict__ g, int n, Scalars* sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    const double s = warp_sum_parts(pfro, nfro, lane);
    if (lane == 0) sc->afro2 = s;
  } else if (warp == 1) {
    const double s = warp_sum_parts(pres, nres, lane);
    if (lane == 0) sc->err_res2 = s;
  } else if (warp == 2) {
    double a0 = 0.0;
    for (int i = lane; i < n; i += 32) a0 = fma(g[i], g[i], a0);
    const double s = warp_sum(a0);
    if (lane == 0) sc->err_num2 = s;
  }
}

// Deterministic CSR: each row's nonzeros placed in column order (the scatter
// that built the CSR used atomics).  One warp per row; an entry's rank is the
// number of entries of the row with a smaller column.
__global__ void k_sort_rows(int32_t m, const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ ccol,
                            const float* __restrict__ cval,
                            int32_t* __restrict__ ocol, float* __restrict__ oval) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5);
       j < m; j += warps) {
    const int32_t lo = rowptr[j], hi = rowptr[j + 1];
    for (int32_t e = lo + lane; e - lane < hi; e += 32) {
      const int32_t my = e < hi ? ccol[e] : 0;
      int32_t rank = 0;
      for (int32_t f = lo; f < hi; ++f) rank += ccol[f] < my;
      if (e < hi) {
        ocol[lo + rank] = my;
        oval[lo + rank] = cval[e];
      }
    }
  }
}

// Continue LSQR with a 10x tighter internal tolerance (the true Error(x)
// missed the requested one).  flip: the last iteration's state is in slot 1
// and buffer 1 of u_raw; move it to slot 0 / buffer 0, where a captured
// graph starts.
__global__ void k_tighten(Scalars* sc, int flip, int64_t m, const double* __restrict__ u1,
                          double* __restrict__ u0) {
  if (flip) {
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < m;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x)
      u0[p] = u1[p];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->tol *= 0.1;
    sc->done = 0;
    sc->istop = 0;
    if (flip) {
      sc->slot[0] = sc->slot[1];
      sc->latest = 0;
    }
  }
}

// ---- rows of A by decreasing nonzero count ------------------------------
// A stable counting sort on the row lengths (lengths >= kLenBuckets - 1
// share the first bucket), so that the 32 rows of a warp in the rows pass
// have (nearly) the same length and rows without nonzeros come last.
constexpr int kLenBuckets = 64;
constexpr int kSortBlock = 1024;

__device__ __forceinline__ int len_bucket(int32_t len) {
  return kLenBuckets - 1 - min(len, kLenBuckets - 1);
}

// hist[b * nblk + blk] = rows of block blk (kSortBlock consecutive rows) in
// bucket b.
__global__ void __launch_bounds__(kSortBlock)
    k_len_hist(int32_t m, const int32_t* __restrict__ rowptr, int32_t* __restrict__ hist,
               int nblk) {
  __shared__ int32_t cnt[kLenBuckets];
  if (threadIdx.x < kLenBuckets) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t j = blockIdx.x * static_cast<int64_t>(kSortBlock) + threadIdx.x;
  if (j < m) atomicAdd(&cnt[len_bucket(rowptr[j + 1] - rowptr[j])], 1);
  __syncthreads();
  if (threadIdx.x < kLenBuckets) hist[threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// perm[pos] = j, inv[j] = pos with pos = off[b * nblk + blk] + (rows of the
// same bucket before j in its block).
__global__ void __launch_bounds__(kSortBlock)
    k_len_place(int32_t m, const int32_t* __restrict__ rowptr,
                const int32_t* __restrict__ off, int nblk, int32_t* __restrict__ perm,
                int32_t* __restrict__ inv) {
  __shared__ int32_t wcnt[kSortBlock / 32][kLenBuckets];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < (kSortBlock / 32) * kLenBuckets; q += kSortBlock)
    (&wcnt[0][0])[q] = 0;
  __syncthreads();
  const int64_t j = blockIdx.x * static_cast<int64_t>(kSortBlock) + threadIdx.x;
  const bool ok = j < m;
  const int b = ok ? len_bucket(rowptr[j + 1] - rowptr[j]) : kLenBuckets;
  const unsigned same = __match_any_sync(0xffffffffu, b);
  const int rank = __popc(same & ((1u << lane) - 1u));
  if (ok && rank == 0) wcnt[warp][b] = __popc(same);
  __syncthreads();
  if (threadIdx.x < kLenBuckets) {
    int32_t run = 0;
    for (int w = 0; w < kSortBlock / 32; ++w) {
      const int32_t c = wcnt[w][threadIdx.x];
      wcnt[w][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
  if (ok) {
    const int32_t pos = off[b * nblk + blockIdx.x] + wcnt[warp][b] + rank;
    perm[pos] = static_cast<int32_t>(j);
    inv[j] = pos;
  }
}

// lenp[p] = length of row perm[p]; lenp[m] = 0 (so its exclusive scan ends
// with nnz).
__global__ void k_perm_len(int32_t m, const int32_t* __restrict__ rowptr,
                           const int32_t* __restrict__ perm, int32_t* __restrict__ lenp) {
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p <= m;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x)
    lenp[p] = p < m ? rowptr[perm[p] + 1] - rowptr[perm[p]] : 0;
}

// Row p of the ordered CSR = row perm[p] of the column-sorted CSR.
__global__ void k_perm_copy(int32_t m, const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ scol, const float* __restrict__ sval,
                            const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ rowptr_p, int32_t* __restrict__ ccol_p,
                            float* __restrict__ cval_p) {
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < m;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t src = rowptr[perm[p]], len = rowptr[perm[p] + 1] - src;
    const int32_t dst = rowptr_p[p];
    for (int32_t k = 0; k < len; ++k) {
      ccol_p[dst + k] = scol[src + k];
      cval_p[dst + k] = sval[src + k];
    }
  }
}

// rowidx_p[e] = position of row rowidx[e] in the ordered CSR.
__global__ void k_map_rows(int64_t nnz, const int32_t* __restrict__ rowidx,
                           const int32_t* __restrict__ inv, int32_t* __restrict__ rowidx_p) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    rowidx_p[e] = inv[rowidx[e]];
}

size_t al(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

// ---------------------------------------------------------------------------
// SAP-SVD (Sec. 5.3): the SVD of the sketch from its R (A_hat = Q R, so A_hat
// and R have the same singular values and right singular vectors), by the
// one-sided (Hestenes) Jacobi method in FP64: rotate pairs of columns of R
// until all are orthogonal; then R V = U Sigma with sigma_j the column norms
// and V the accumulated rotations.  A sweep visits every pair once in
// n' - 1 rounds of n'/2 disjoint pairs (n' = n rounded up to even, the
// round-robin "circle" order); one kernel per round, one block per pair.
// ---------------------------------------------------------------------------
constexpr int kJacobiThreads = 256;

// Rc = R column-major (n x n) from the QR workspace W (d x n, R in its upper
// triangle), V = I.
__global__ void k_svd_init(const double* __restrict__ W, int64_t d, int n,
                           double* __restrict__ Rc, double* __restrict__ V) {
  const int64_t total = static_cast<int64_t>(n) * n;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = t / n, r = t % n;
    Rc[t] = r <= c ? W[c * d + r] : 0.0;
    V[t] = r == c ? 1.0 : 0.0;
  }
}

// Pair `p` of round `r` of the circle order on n2 (even) slots: slot 0 stays,
// slots 1 .. n2 - 1 turn by one position per round.
__device__ __forceinline__ void jacobi_pair(int n2, int r, int p, int& a, int& b) {
  const int m1 = n2 - 1;
  if (p == 0) {
    a = 0;
    b = 1 + r % m1;
  } else {
    a = 1 + (r + p) % m1;
    b = 1 + (r + m1 - p) % m1;
  }
  if (a > b) {
    const int t = a;
    a = b;
    b = t;
  }
}

// One round: block p rotates its pair of columns of Rc (and V) when they are
// not orthogonal to working precision (|a.b| > 1e-15 sqrt(|a|^2 |b|^2)), by
// the 2 x 2 symmetric Schur rotation of their Gram matrix; counts rotations.
__global__ void __launch_bounds__(kJacobiThreads)
    k_jacobi_round(int n, int n2, int r, double* __restrict__ Rc, double* __restrict__ V,
                   unsigned long long* __restrict__ rotations) {
  __shared__ double red[3][kJacobiThreads / 32];
  __shared__ double cs[2];
  int a, b;
  jacobi_pair(n2, r, blockIdx.x, a, b);
  if (b >= n) return;  // the padding slot of an odd n
  double* ca = Rc + static_cast<int64_t>(a) * n;
  double* cb = Rc + static_cast<int64_t>(b) * n;
  double al = 0.0, be = 0.0, ga = 0.0;
  for (int i = threadIdx.x; i < n; i += kJacobiThreads) {
    const double x = ca[i], y = cb[i];
    al = fma(x, x, al);
    be = fma(y, y, be);
    ga = fma(x, y, ga);
  }
  al = warp_sum(al);
  be = warp_sum(be);
  ga = warp_sum(ga);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = al;
    red[1][warp] = be;
    red[2][warp] = ga;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double A = 0.0, B = 0.0, G = 0.0;
    for (int w = 0; w < kJacobiThreads / 32; ++w) {
      A += red[0][w];
      B += red[1][w];
      G += red[2][w];
    }
    double c = 1.0, sn = 0.0;
    if (G != 0.0 && fabs(G) > 1e-15 * sqrt(A * B)) {
      const double zeta = (B - A) / (2.0 * G);
      const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      c = 1.0 / sqrt(1.0 + t * t);
      sn = c * t;
      atomicAdd(rotations, 1ULL);
    }
    cs[0] = c;
    cs[1] = sn;
  }
  __syncthreads();
  const double c = cs[0], sn = cs[1];
  if (sn == 0.0) return;
  double* va = V + static_cast<int64_t>(a) * n;
  double* vb = V + static_cast<int64_t>(b) * n;
  for (int i = threadIdx.x; i < n; i += kJacobiThreads) {
    const double x = ca[i], y = cb[i];
    ca[i] = c * x - sn * y;
    cb[i] = sn * x + c * y;
    const double p = va[i], q = vb[i];
    va[i] = c * p - sn * q;
    vb[i] = sn * p + c * q;
  }
}

// sigma_j = ||column j of Rc|| (one warp per column); then (one block) the
// cutoff sigma_max / 1e12 and the rank: keep[j] = 1 / sigma_j for kept j,
// else 0; rank[0] = number kept.
__global__ void k_svd_sigma(const double* __restrict__ Rc, int n, double* __restrict__ sig) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5);
       j < n; j += warps) {
    double a = 0.0;
    for (int i = lane; i < n; i += 32) {
      const double x = Rc[j * n + i];
      a = fma(x, x, a);
    }
    a = warp_sum(a);
    if (lane == 0) sig[j] = sqrt(a);
  }
}

__global__ void __launch_bounds__(1024)
    k_svd_cutoff(int n, const double* __restrict__ sig, double* __restrict__ keep,
                 int* __restrict__ rank) {
  __shared__ double red[32];
  __shared__ int cnt[32];
  double mx = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) mx = fmax(mx, sig[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (blockDim.x + 31) / 32; ++w) m = fmax(m, red[w]);
    red[0] = m;
  }
  __syncthreads();
  const double smax = red[0];
  int k = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const bool kept = sig[j] > 0.0 && sig[j] >= smax / 1e12;
    keep[j] = kept ? 1.0 / sig[j] : 0.0;
    k += kept;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  __syncthreads();
  if (lane == 0) cnt[warp] = k;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (blockDim.x + 31) / 32; ++w) t += cnt[w];
    rank[0] = t;
  }
}

// P = V diag(keep) (row-major n x n: P[i][j] = V[j][i] keep[j], V
// column-major) and P^T (row-major).
__global__ void k_svd_precond(const double* __restrict__ V, const double* __restrict__ keep,
                              int n, double* __restrict__ P, double* __restrict__ PT) {
  const int64_t total = static_cast<int64_t>(n) * n;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = t / n, j = t % n;
    P[t] = V[j * n + i] * keep[j];   // row i, column j
    PT[t] = V[i * n + j] * keep[i];  // row i of P^T = column i of P
  }
}

// ---------------------------------------------------------------------------
// LSQR-D (Sec. 5.3's diagonal preconditioner): colnorm[k] = ||A_k||_2 in FP64
// (one warp per column), then D_k = 1 / ||A_k|| or 1 when ||A_k|| <= eps
// sqrt(n) max ||A_k|| (eps = 2^-52), written on the diagonals of the two
// row-major preconditioner matrices (the diagonal kind reads nothing else).
// ---------------------------------------------------------------------------
template <typename VT>
__global__ void k_colnorm(int32_t n, int64_t nnz, const int32_t* __restrict__ colptr,
                          const VT* __restrict__ vals, double* __restrict__ norm) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5);
       k < n; k += warps) {
    const int2 range = column_range(colptr, k, nnz, nullptr);
    double a = 0.0;
    for (int32_t e = range.x + lane; e < range.y; e += 32) {
      const double v = static_cast<double>(to_f32(vals[e]));
      a = fma(v, v, a);
    }
    a = warp_sum(a);
    if (lane == 0) norm[k] = sqrt(a);
  }
}

__global__ void __launch_bounds__(1024)
    k_diag_precond(int n, const double* __restrict__ norm, double* __restrict__ P,
                   double* __restrict__ PT) {
  __shared__ double red[32];
  double mx = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) mx = fmax(mx, norm[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (blockDim.x + 31) / 32; ++w) m = fmax(m, red[w]);
    red[0] = m;
  }
  __syncthreads();
  const double thr = 0x1p-52 * sqrt(static_cast<double>(n)) * red[0];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double dj = norm[j] <= thr ? 1.0 : 1.0 / norm[j];
    P[static_cast<int64_t>(j) * n + j] = dj;
    PT[static_cast<int64_t>(j) * n + j] = dj;
  }
}

struct LsqState {
  void* ws = nullptr;
  size_t ws_bytes = 0;
  Scalars* host = nullptr;       // pinned mirror of the scalars
  cudaStream_t ls = nullptr;     // internal stream (capturable)
  cudaEvent_t ev[6] = {};
  cudaGraphExec_t graph = nullptr;
  const void* graph_key[10] = {};  // what the captured iterations read/write
  cudaGraphExec_t qr_graph = nullptr;  // the QR's n launches, per shape
  int64_t qr_key[3] = {-1, -1, -1};     // (d, n, workspace address) of qr_graph
  int64_t qr_seen[3] = {-1, -1, -1};    // shape of the previous solve
  cudaGraphExec_t jacobi_graph = nullptr;  // one Jacobi sweep, per shape
  const void* jacobi_key[4] = {};  // the rounds' arrays and n
  int svd_sweeps = 0;                    // sweeps of the last SAP-SVD solve
};

void destroy_lsq_state(sketch_t h) {
  if (!h->lsq) return;
  LsqState* st = h->lsq;
  if (st->ls) cudaStreamSynchronize(st->ls);
  if (st->graph) cudaGraphExecDestroy(st->graph);
  if (st->qr_graph) cudaGraphExecDestroy(st->qr_graph);
  if (st->jacobi_graph) cudaGraphExecDestroy(st->jacobi_graph);
  for (auto& e : st->ev)
    if (e) cudaEventDestroy(e);
  if (st->ls) cudaStreamDestroy(st->ls);
  if (st->ws) cudaFree(st->ws);
  if (st->host) cudaFreeHost(st->host);
  delete st;
  h->lsq = nullptr;
}

}  // namespace sk

using namespace sk;

namespace {

struct LsqLayout {
  float* Ahat;
  double *W, *tau, *vs, *Rrow, *rdiag, *Rinv, *RinvT, *t, *t2, *v, *vraw, *w, *y;
  double* u[2];  // u_raw, double buffered by iteration parity
  double *p2, *p4, *py, *pfro, *pres;  // per-block partial sums
  double* r;  // A x - b for the error check (kept apart from LSQR's u)
  Scalars* sc;
  int32_t* scol;  // column-sorted CSR rows
  float* sval;
  // rows ordered by decreasing length: perm[p] = row of A at position p,
  // inv its inverse, the ordered CSR's rowptr, the CSC's rows mapped to
  // positions, the counting sort's histogram and offsets, scan scratch
  int32_t *perm, *inv, *lenp, *rowptr_p, *rowidx_p, *hist, *hoff;
  double* pz;  // per-block sums of b^2 over rows without nonzeros
  char* scan_tmp;
  void* csr_ws;
  int* status;
  // SAP-SVD: R column-major, V, sigma, 1/sigma of the kept values, rank and
  // the rotation counter (sized only for that method); LSQR-D: column norms
  double *Rc, *Vj, *sig, *keep, *colnorm;
  int* rank;
  unsigned long long* rotations;
  size_t bytes;
};

constexpr int kFroBlocks = 512;

int rows_blocks(int64_t m) {
  return static_cast<int>(
      std::max<int64_t>(1, std::min<int64_t>((m + kRows - 1) / kRows, 8LL * num_sms())));
}

int tri_blocks(int64_t n) { return static_cast<int>((n + kTriWarps - 1) / kTriWarps); }

LsqLayout layout(void* base, int64_t m, int64_t n, int64_t d, int64_t nnz, int method = 0) {
  LsqLayout L{};
  char* p = static_cast<char*>(base);
  auto take = [&](size_t b) {
    char* r = p;
    p += al(b);
    return r;
  };
  L.Ahat = reinterpret_cast<float*>(take(sizeof(float) * d * n));
  L.W = reinterpret_cast<double*>(take(sizeof(double) * d * n));
  L.tau = reinterpret_cast<double*>(take(sizeof(double) * n));
  L.vs = reinterpret_cast<double*>(take(sizeof(double) * n));
  L.Rrow = reinterpret_cast<double*>(take(sizeof(double) * n * n));
  L.rdiag = reinterpret_cast<double*>(take(sizeof(double) * n));
  L.Rinv = reinterpret_cast<double*>(take(sizeof(double) * n * n));
  L.RinvT = reinterpret_cast<double*>(take(sizeof(double) * n * n));
  L.u[0] = reinterpret_cast<double*>(take(sizeof(double) * m));
  L.u[1] = reinterpret_cast<double*>(take(sizeof(double) * m));
  L.r = reinterpret_cast<double*>(take(sizeof(double) * m));
  L.t = reinterpret_cast<double*>(take(sizeof(double) * n));
  L.t2 = reinterpret_cast<double*>(take(sizeof(double) * n));
  L.v = reinterpret_cast<double*>(take(sizeof(double) * n));
  L.vraw = reinterpret_cast<double*>(take(sizeof(double) * n));
  L.w = reinterpret_cast<double*>(take(sizeof(double) * n));
  L.y = reinterpret_cast<double*>(take(sizeof(double) * n));
  L.p2 = reinterpret_cast<double*>(take(sizeof(double) * rows_blocks(m)));
  L.pres = reinterpret_cast<double*>(take(sizeof(double) * rows_blocks(m)));
  L.p4 = reinterpret_cast<double*>(take(sizeof(double) * tri_blocks(n)));
  L.py = reinterpret_cast<double*>(take(sizeof(double) * tri_blocks(n)));
  L.pfro = reinterpret_cast<double*>(take(sizeof(double) * kFroBlocks));
  L.sc = reinterpret_cast<Scalars*>(take(sizeof(Scalars)));
  L.status = reinterpret_cast<int*>(take(256));
  L.scol = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (nnz > 0 ? nnz : 1)));
  L.sval = reinterpret_cast<float*>(take(sizeof(float) * (nnz > 0 ? nnz : 1)));
  const int64_t nblk = (m + kSortBlock - 1) / kSortBlock;
  L.perm = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * m));
  L.inv = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * m));
  L.lenp = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (m + 1)));
  L.rowptr_p = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (m + 1)));
  L.rowidx_p = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (nnz > 0 ? nnz : 1)));
  L.hist = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * kLenBuckets * nblk));
  L.hoff = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * kLenBuckets * nblk));
  L.pz = reinterpret_cast<double*>(take(sizeof(double) * rows_blocks(m)));
  L.scan_tmp = take(static_cast<size_t>(
      scan_bytes_for(std::max<int64_t>(m + 1, kLenBuckets * nblk))));
  L.csr_ws = take(csr_workspace_bytes(m, nnz));
  const int64_t nsvd = method == 1 ? n : 0;
  L.Rc = reinterpret_cast<double*>(take(sizeof(double) * nsvd * nsvd));
  L.Vj = reinterpret_cast<double*>(take(sizeof(double) * nsvd * nsvd));
  L.sig = reinterpret_cast<double*>(take(sizeof(double) * n));
  L.keep = reinterpret_cast<double*>(take(sizeof(double) * n));
  L.colnorm = reinterpret_cast<double*>(take(sizeof(double) * n));
  L.rank = reinterpret_cast<int*>(take(256));
  L.rotations = reinterpret_cast<unsigned long long*>(take(256));
  L.bytes = static_cast<size_t>(p - static_cast<char*>(base));
  return L;
}

// The CSC of A with its rows mapped to positions of the ordered CSR.
struct CscView {
  int32_t n;
  int64_t nnz;
  const int32_t* colptr;
  const int32_t* rowidx;
  const void* values;
  int32_t dtype;
};

// Launch with programmatic stream serialization (pdl = 1): the kernel may
// start while the previous kernel on the stream finishes (see pdl_wait).
template <typename... KArgs, typename... Args>
void launch(void (*kern)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, int pdl,
            Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Columns pass launch.  lsqr = 1 adds the scalar block (stopping test and
// ||u_raw||^2) of an LSQR iteration.
struct ColsArgs {
  int lsqr = 0;
  const double *p2 = nullptr, *pz = nullptr, *py = nullptr;
  int np2 = 0, npy = 0, par = 0, init = 0, pdl = 0;
};

template <typename VT>
void launch_cols(const CscView& A, const double* u, double* out, Scalars* sc,
                 const ColsArgs& c, cudaStream_t s) {
  // warps per column from the mean column length: about 8 entries per
  // thread, one round of loads (any choice is correct; 16 warps measured
  // slower on a 2000-entry column)
  const int64_t avg = A.nnz / std::max<int64_t>(1, A.n);
  int W = 1;
  while (W < 8 && avg > 256LL * W) W *= 2;
  const unsigned g = static_cast<unsigned>(A.n + (c.lsqr ? 1 : 0));
  const VT* vals = static_cast<const VT*>(A.values);
#define SK_COLS(WW)                                                                     \
  launch(k_cols<VT, WW>, g, 32 * WW, s, c.pdl, A.n, A.colptr, A.rowidx, vals, u, out, sc, \
         c.lsqr, c.p2, c.pz, c.np2, c.py, c.npy, c.par, c.init)
  switch (W) {
    case 1: SK_COLS(1); break;
    case 2: SK_COLS(2); break;
    case 4: SK_COLS(4); break;
    default: SK_COLS(8); break;
  }
#undef SK_COLS
}

void cols(const CscView& A, const double* u, double* out, Scalars* sc, const ColsArgs& c,
          cudaStream_t s) {
  if (A.dtype == SKETCH_F32)
    launch_cols<float>(A, u, out, sc, c, s);
  else
    launch_cols<__nv_bfloat16>(A, u, out, sc, c, s);
}

unsigned gemv_blocks(int64_t n) {
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, 32LL * num_sms())));
}

// LSQR start-up (init = 1, par = 1) or iteration j of a graph (par = j & 1):
// four kernels.  The rows pass reads u_raw[par] and writes u_raw[par ^ 1];
// the step reads slot par and writes slot par ^ 1.
void lsqr_kernels(const LsqLayout& L, const CscView& A, const CsrView& csr,
                  const int32_t* mnz, const double* b, int32_t m, int par, int init,
                  int pdl, int pk, cudaStream_t s) {
  const int n = A.n;
  const int g2 = rows_blocks(m), gt = tri_blocks(n);
  launch(k_lsqr_rows, g2, kRows, s, pdl, m, mnz, csr.rowptr, csr.ccol, csr.cval, L.t, L.u[par],
         L.u[par ^ 1], b, L.perm, L.p2, L.pz, L.sc, par, init);
  ColsArgs c;
  c.lsqr = 1;
  c.p2 = L.p2;
  c.pz = L.pz;
  c.np2 = g2;
  c.py = L.py;
  c.npy = gt;
  c.par = par;
  c.init = init;
  c.pdl = pdl;
  cols(A, L.u[par ^ 1], L.t2, L.sc, c, s);
  launch(k_lsqr_vraw, gt, 32 * kTriWarps, s, pdl, n, L.RinvT, L.t2, L.v, L.vraw, L.p4, L.sc,
         init, pk);
  launch(k_lsqr_step, gt, 32 * kTriWarps, s, pdl, n, L.Rinv, L.vraw, L.v, L.w, L.y, L.t, L.p4,
         gt, L.py, L.sc, par, init, pk);
}

}  // namespace

namespace sk {
size_t lsq_workspace_bytes(int64_t m, int64_t n, int64_t d, int64_t nnz) {
  return layout(nullptr, m, n, d, nnz).bytes + 256;
}
}  // namespace sk

namespace {

// The solve of sketch_lsq_solve / sketch_lsq_solve_method.  method:
// SKETCH_LSQ_SAP_QR (preconditioner R^{-1}), SKETCH_LSQ_SAP_SVD (V_k
// Sigma_k^{-1} from the Jacobi SVD of R) or SKETCH_LSQ_LSQR_D (diagonal, no
// sketch).
int lsq_solve(sketch_t h, const sketch_csc* A, const double* b, double* x, double tol,
              int32_t maxit, int method, sketch_lsq_info* info, sketch_stream_t stream) {
  if (!h) return fail(nullptr, SKETCH_ERR_ARG, "handle is null");
  int rc = check_csc_args(h, A);
  if (rc != SKETCH_OK) return rc;
  if (!b || !x) return fail(h, SKETCH_ERR_ARG, "b or x is null");
  if (!(tol > 0.0)) return fail(h, SKETCH_ERR_ARG, "tol must be > 0");
  if (maxit < 1) return fail(h, SKETCH_ERR_ARG, "maxit must be >= 1");
  if (method < SKETCH_LSQ_SAP_QR || method > SKETCH_LSQ_LSQR_D)
    return fail(h, SKETCH_ERR_ARG, "unknown least-squares method");
  const bool sketched = method != SKETCH_LSQ_LSQR_D;
  if (sketched && h->d < h->n) return fail(h, SKETCH_ERR_ARG, "sketch size d must be >= n");
  if (h->n > 8192) return fail(h, SKETCH_ERR_UNSUPPORTED, "n > 8192");
  if (method == SKETCH_LSQ_SAP_SVD && h->n > 4096)
    return fail(h, SKETCH_ERR_UNSUPPORTED, "SAP-SVD takes n <= 4096");
  const int pk = method == SKETCH_LSQ_SAP_QR ? kPcTri
                 : method == SKETCH_LSQ_SAP_SVD ? kPcDense : kPcDiag;
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  const int64_t m = A->m, n = A->n, d = h->d, nnz = A->nnz;
  if (!h->lsq) h->lsq = new (std::nothrow) LsqState();
  if (!h->lsq) return fail(h, SKETCH_ERR_OOM, "host allocation failed");
  LsqState& st = *h->lsq;
  if (!st.ls) {
    if (cudaStreamCreateWithFlags(&st.ls, cudaStreamNonBlocking) != cudaSuccess)
      return fail(h, SKETCH_ERR_CUDA, "cudaStreamCreate failed");
    for (auto& e : st.ev) cudaEventCreate(&e);
  }
  const size_t need = layout(nullptr, m, n, d, nnz, method).bytes + 256;
  if (st.ws_bytes < need) {
    cudaStreamSynchronize(st.ls);
    if (st.ws) cudaFree(st.ws);
    if (st.graph) {
      cudaGraphExecDestroy(st.graph);
      st.graph = nullptr;
    }
    if (st.qr_graph) {
      cudaGraphExecDestroy(st.qr_graph);
      st.qr_graph = nullptr;
    }
    if (st.jacobi_graph) {
      cudaGraphExecDestroy(st.jacobi_graph);
      st.jacobi_graph = nullptr;
    }
    st.ws = nullptr;
    st.ws_bytes = 0;
    if (cudaMalloc(&st.ws, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, SKETCH_ERR_OOM, "cudaMalloc(lsq workspace) failed");
    }
    st.ws_bytes = need;
  }
  if (!st.host && cudaMallocHost(&st.host, sizeof(Scalars)) != cudaSuccess) {
    st.host = nullptr;
    return fail(h, SKETCH_ERR_OOM, "cudaMallocHost failed");
  }
  const LsqLayout L = layout(st.ws, m, n, d, nnz, method);
  cudaStream_t s = st.ls;
  cudaEventRecord(st.ev[4], user);  // the solve starts after the caller's work
  cudaStreamWaitEvent(s, st.ev[4], 0);
  cudaEventRecord(st.ev[0], s);

  // ---- 0. a malformed CSC is refused before any kernel walks its columns ---
  {
    int bad = 0;
    cudaError_t ve = cudaMemsetAsync(L.status, 0, sizeof(int), s);
    if (ve == cudaSuccess)
      ve = launch_validate(static_cast<int32_t>(m), static_cast<int32_t>(n), nnz, A->colptr,
                           A->rowidx, L.status, s);
    if (ve == cudaSuccess)
      ve = cudaMemcpyAsync(&bad, L.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (ve == cudaSuccess) ve = cudaStreamSynchronize(s);
    if (ve != cudaSuccess) return cuda_fail(h, ve, "CSC check (lsq)");
    h->launches += 1;
    if (bad) return fail(h, SKETCH_ERR_CSC, "malformed CSC (colptr or row indices)");
  }

  // ---- 1. sketch (not for LSQR-D) -------------------------------------------
  if (sketched &&
      (rc = sketch_apply(h, A, L.Ahat, reinterpret_cast<sketch_stream_t>(s))) != SKETCH_OK)
    return rc;
  cudaError_t e = cudaSuccess;
  cudaEventRecord(st.ev[1], s);

  // ---- 2. FP64 Householder QR of the sketch, 3. R^{-1} ----------------------
  cudaMemsetAsync(L.status, 0, sizeof(int), s);
  const int pdl = h->dependent_launch ? 1 : 0;
  const int64_t dn = d * n;
  const unsigned gb = static_cast<unsigned>(std::max<int64_t>(1, 16LL * num_sms()));
  if (sketched) {
    // the QR is n dependent launches.  When a shape repeats (same d, n and
    // workspace as the previous solve) they are captured once as a graph
    // and replayed; a one-off shape launches them directly.
    const int64_t qk[3] = {d, n, static_cast<int64_t>(reinterpret_cast<intptr_t>(st.ws))};
    auto enqueue_qr = [&]() {
      k_to_double<<<gb, 256, 0, s>>>(dn, L.Ahat, L.W);
      k_qr_first<<<1, kQrThreads, 0, s>>>(L.W, d, L.tau, L.vs);
      for (int k = 0; k + 1 < n; ++k)
        launch(k_qr_step, qr_step_blocks(n, k), kQrThreads, s, pdl, L.W, d,
               static_cast<int>(n), k, L.tau, L.vs);
      k_extract_r<<<gb, 256, 0, s>>>(L.W, d, static_cast<int>(n), L.Rrow, L.rdiag, L.status);
      launch_trtri(L.W, d, static_cast<int>(n), L.rdiag, L.Rinv, L.RinvT, s);
    };
    const bool repeat = std::memcmp(qk, st.qr_seen, sizeof(qk)) == 0;
    std::memcpy(st.qr_seen, qk, sizeof(qk));
    if (st.qr_graph && std::memcmp(qk, st.qr_key, sizeof(qk)) != 0) {
      cudaGraphExecDestroy(st.qr_graph);
      st.qr_graph = nullptr;
    }
    if (!st.qr_graph && repeat) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(h, e, "begin QR capture");
      enqueue_qr();
      e = cudaStreamEndCapture(s, &g);
      if (e != cudaSuccess) return cuda_fail(h, e, "end QR capture");
      e = cudaGraphInstantiate(&st.qr_graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        st.qr_graph = nullptr;
        return cuda_fail(h, e, "QR graph instantiate");
      }
      std::memcpy(st.qr_key, qk, sizeof(qk));
    }
    if (st.qr_graph) {
      e = cudaGraphLaunch(st.qr_graph, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "QR graph launch");
    } else {
      enqueue_qr();
    }
  }
  if (sketched) h->launches += 4 + (n - 1);
  int rank = static_cast<int>(n);
  if (method == SKETCH_LSQ_SAP_SVD) {
    // one-sided Jacobi on R: sweeps of n' - 1 rounds (a graph per sweep, per
    // shape), until a sweep rotates nothing or 40 sweeps have run
    const int n32 = static_cast<int>(n), n2 = n32 + (n32 & 1);
    k_svd_init<<<gb, 256, 0, s>>>(L.W, d, n32, L.Rc, L.Vj);
    h->launches += 1;
    const void* jkey[4] = {L.Rc, L.Vj, L.rotations,
                           reinterpret_cast<const void*>(static_cast<intptr_t>(n))};
    if (st.jacobi_graph && std::memcmp(jkey, st.jacobi_key, sizeof(jkey)) != 0) {
      cudaGraphExecDestroy(st.jacobi_graph);
      st.jacobi_graph = nullptr;
    }
    if (!st.jacobi_graph) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(h, e, "begin Jacobi capture");
      for (int r = 0; r < n2 - 1; ++r)
        k_jacobi_round<<<n2 / 2, kJacobiThreads, 0, s>>>(n32, n2, r, L.Rc, L.Vj, L.rotations);
      e = cudaStreamEndCapture(s, &g);
      if (e != cudaSuccess) return cuda_fail(h, e, "end Jacobi capture");
      e = cudaGraphInstantiate(&st.jacobi_graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        st.jacobi_graph = nullptr;
        return cuda_fail(h, e, "Jacobi graph instantiate");
      }
      std::memcpy(st.jacobi_key, jkey, sizeof(jkey));
    }
    unsigned long long rot = 1;
    int sweeps = 0;
    for (; sweeps < 40 && rot != 0; ++sweeps) {
      cudaMemsetAsync(L.rotations, 0, sizeof(unsigned long long), s);
      e = cudaGraphLaunch(st.jacobi_graph, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "Jacobi sweep");
      h->launches += n2 - 1;
      cudaMemcpyAsync(&rot, L.rotations, sizeof(rot), cudaMemcpyDeviceToHost, s);
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(h, e, "Jacobi sweep");
    }
    st.svd_sweeps = sweeps;
    k_svd_sigma<<<gemv_blocks(n), 256, 0, s>>>(L.Rc, n32, L.sig);
    k_svd_cutoff<<<1, 1024, 0, s>>>(n32, L.sig, L.keep, L.rank);
    k_svd_precond<<<gb, 256, 0, s>>>(L.Vj, L.keep, n32, L.Rinv, L.RinvT);
    h->launches += 3;
    e = cudaMemcpyAsync(&rank, L.rank, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "SVD rank");
  } else if (method == SKETCH_LSQ_LSQR_D) {
    if (A->dtype == SKETCH_F32)
      k_colnorm<float><<<gemv_blocks(n), 256, 0, s>>>(
          static_cast<int32_t>(n), nnz, A->colptr, static_cast<const float*>(A->values),
          L.colnorm);
    else
      k_colnorm<__nv_bfloat16><<<gemv_blocks(n), 256, 0, s>>>(
          static_cast<int32_t>(n), nnz, A->colptr,
          static_cast<const __nv_bfloat16*>(A->values), L.colnorm);
    k_diag_precond<<<1, 1024, 0, s>>>(static_cast<int>(n), L.colnorm, L.Rinv, L.RinvT);
    h->launches += 2;
  }
  cudaEventRecord(st.ev[2], s);

  // ---- 4. LSQR on A R^{-1} ---------------------------------------------------
  CsrView csr{};
  int nl = 0;
  e = build_csr(static_cast<int32_t>(m), static_cast<int32_t>(n), nnz, A->colptr,
                A->rowidx, A->values, A->dtype, L.csr_ws, &csr, L.status, s, &nl);
  if (e != cudaSuccess) return cuda_fail(h, e, "csr build (lsq)");
  k_sort_rows<<<gb, 256, 0, s>>>(static_cast<int32_t>(m), csr.rowptr, csr.ccol, csr.cval,
                                 L.scol, L.sval);
  // rows by decreasing length; the ordered CSR reuses the unsorted arrays
  {
    const int32_t m32 = static_cast<int32_t>(m);
    const int nblk = static_cast<int>((m + kSortBlock - 1) / kSortBlock);
    k_len_hist<<<nblk, kSortBlock, 0, s>>>(m32, csr.rowptr, L.hist, nblk);
    e = scan_i32(L.hist, L.hoff, static_cast<int64_t>(kLenBuckets) * nblk, L.scan_tmp, s, &nl);
    if (e != cudaSuccess) return cuda_fail(h, e, "row order scan");
    k_len_place<<<nblk, kSortBlock, 0, s>>>(m32, csr.rowptr, L.hoff, nblk, L.perm, L.inv);
    k_perm_len<<<gb, 256, 0, s>>>(m32, csr.rowptr, L.perm, L.lenp);
    e = scan_i32(L.lenp, L.rowptr_p, m + 1, L.scan_tmp, s, &nl);
    if (e != cudaSuccess) return cuda_fail(h, e, "row order scan");
    k_perm_copy<<<gb, 256, 0, s>>>(m32, csr.rowptr, L.scol, L.sval, L.perm, L.rowptr_p,
                                   csr.ccol, csr.cval);
    k_map_rows<<<gb, 256, 0, s>>>(nnz, A->rowidx, L.inv, L.rowidx_p);
    csr.rowptr = L.rowptr_p;
  }
  const int32_t* mnz = L.hoff + static_cast<int64_t>(kLenBuckets - 1) *
                                    ((m + kSortBlock - 1) / kSortBlock);
  const CscView csc{static_cast<int32_t>(n), nnz, A->colptr, L.rowidx_p, A->values, A->dtype};
  h->launches += nl + 7;
  Scalars init{};
  init.tol = tol;
  init.maxit = maxit;
  *st.host = init;
  cudaMemcpyAsync(L.sc, st.host, sizeof(Scalars), cudaMemcpyHostToDevice, s);
  // u = b, beta = ||b||, v = R^{-T} A^T u / (beta alpha), w = v, y = 0
  lsqr_kernels(L, csc, csr, mnz, b, static_cast<int32_t>(m), 1, 1, pdl, pk, s);
  h->launches += 4;
  // iterations: a cached graph of kIterPerGraph iterations, replayed until
  // the device sets `done`.  The key holds every value the captured launches
  // take: A's arrays, the workspace and the shape that lays it out (nnz
  // places the ordered CSR and everything after it), and the value type.
  const void* key[10] = {A->colptr, A->rowidx, A->values, st.ws,
                         reinterpret_cast<const void*>(n), reinterpret_cast<const void*>(m),
                         reinterpret_cast<const void*>(static_cast<intptr_t>(pk)),
                         reinterpret_cast<const void*>(d),
                         reinterpret_cast<const void*>(static_cast<intptr_t>(nnz)),
                         reinterpret_cast<const void*>(static_cast<intptr_t>(A->dtype))};
  if (st.graph && std::memcmp(key, st.graph_key, sizeof(key)) != 0) {
    cudaGraphExecDestroy(st.graph);
    st.graph = nullptr;
  }
  if (!st.graph) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "begin capture");
    static_assert(kIterPerGraph % 2 == 0, "a graph starts and ends on slot 0");
    for (int it = 0; it < kIterPerGraph; ++it)
      lsqr_kernels(L, csc, csr, mnz, nullptr, static_cast<int32_t>(m), it & 1, 0, pdl, pk, s);
    launch(k_lsqr_test, 1, 32, s, pdl, L.py, tri_blocks(n), L.sc, 0);
    e = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
    e = cudaGraphInstantiate(&st.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      st.graph = nullptr;
      return cuda_fail(h, e, "graph instantiate");
    }
    std::memcpy(st.graph_key, key, sizeof(key));
  }
  // LSQR stops on its own estimate for the preconditioned system; the
  // paper's Error(x) for A itself can land above it, so verify and, if
  // needed, continue from the same state with a tighter internal tolerance.
  int qr_status = 0;
  int launched = 0;
  double prev_err = 1e300;
  for (int round = 0; round < 6; ++round) {
    for (;; launched += kIterPerGraph) {
      e = cudaGraphLaunch(st.graph, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
      h->launches += 4 * kIterPerGraph + 1;
      cudaMemcpyAsync(st.host, L.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s);
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(h, e, "lsqr iterations");
      if (st.host->done || launched >= maxit) break;
    }
    // x = M y
    k_gemv_tri<<<gemv_blocks(n), 256, 0, s>>>(L.Rinv, static_cast<int>(n), L.y, x, 0, pk);
    cudaEventRecord(st.ev[3], s);
    // ---- 5. Error(x) = ||A^T (A x - b)|| / (||A||_F ||A x - b||) in FP64 ----
    const int g2 = rows_blocks(m);
    k_residual<<<g2, kRows, 0, s>>>(static_cast<int32_t>(m), csr.rowptr, csr.ccol, csr.cval,
                                    x, b, L.perm, L.r, L.pres);
    cols(csc, L.r, L.t2, L.sc, ColsArgs{}, s);
    if (A->dtype == SKETCH_F32)
      k_fro2<float><<<kFroBlocks, 256, 0, s>>>(nnz, static_cast<const float*>(A->values), L.pfro);
    else
      k_fro2<__nv_bfloat16><<<kFroBlocks, 256, 0, s>>>(
          nnz, static_cast<const __nv_bfloat16*>(A->values), L.pfro);
    k_finish_error<<<1, 96, 0, s>>>(L.pfro, kFroBlocks, L.pres, g2, L.t2,
                                    static_cast<int>(n), L.sc);
    h->launches += 5;
    cudaMemcpyAsync(st.host, L.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&qr_status, L.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "lsq error check");
    const Scalars& c = *st.host;
    const double den = std::sqrt(c.afro2) * std::sqrt(c.err_res2);
    const double err = den > 0.0 ? std::sqrt(c.err_num2) / den : 0.0;
    // The FP64 floor of the metric: r = A x - b carries the rounding of b,
    // about eps ||b||, and A^T moves that by at most ||A||_2 eps ||b|| <=
    // ||A||_F eps ||b||, so Error(x) cannot be resolved below about
    // eps ||b|| / ||r||.  Within 2x of that, more LSQR rounds are wasted.
    const double rnorm = std::sqrt(c.err_res2);
    const double floor_est = rnorm > 0.0 ? 0x1p-52 * c.bnorm / rnorm : 0.0;
    // stop when the metric is met, LSQR ran out of iterations, the metric
    // is at its FP64 floor, or another round gained less than 2x
    if (err <= tol || c.istop == 0 || qr_status != 0 ||
        c.slot[c.latest & 1].iters >= maxit || err <= 2.0 * floor_est ||
        err > 0.5 * prev_err)
      break;
    prev_err = err;
    k_tighten<<<gb, 256, 0, s>>>(L.sc, c.latest == 1, m, L.u[1], L.u[0]);
    h->launches += 1;
  }
  cudaEventRecord(st.ev[5], s);
  cudaStreamWaitEvent(user, st.ev[5], 0);  // the caller's stream sees x
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "lsq solve");
  const Scalars& sc = *st.host;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    const Slot& S = sc.slot[sc.latest & 1];
    info->iters = S.iters;
    info->istop = sc.istop;
    const double arnorm = S.phibar * S.alpha * S.cabs;
    const double anorm = std::sqrt(S.anorm2);
    info->test2 = S.phibar > 0.0 && anorm > 0.0 ? arnorm / (anorm * S.phibar) : 0.0;
    const double den = std::sqrt(sc.afro2) * std::sqrt(sc.err_res2);
    info->error = den > 0.0 ? std::sqrt(sc.err_num2) / den : 0.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, st.ev[0], st.ev[1]);
    info->ms_sketch = ms;
    cudaEventElapsedTime(&ms, st.ev[1], st.ev[2]);
    info->ms_qr = ms;
    cudaEventElapsedTime(&ms, st.ev[2], st.ev[3]);
    info->ms_lsqr = ms;
    info->rank = rank;
  }
  // a zero diagonal of R is an error of SAP-QR only (SAP-SVD drops the
  // small singular values instead)
  if ((qr_status & 4) && method == SKETCH_LSQ_SAP_QR)
    return fail(h, SKETCH_ERR_CSC, "R has a zero diagonal entry (rank-deficient A)");
  if (qr_status & (kStatusBadRow | kStatusBadColptr))
    return fail(h, SKETCH_ERR_CSC, "a kernel met an out-of-range index");
  const int status = sc.istop ? SKETCH_OK : SKETCH_ERR_NO_CONVERGENCE;
  if (info) info->status = status;
  if (status != SKETCH_OK) fail(h, status, "LSQR reached maxit");
  return status;
}

}  // namespace

extern "C" int sketch_lsq_solve(sketch_t h, const sketch_csc* A, const double* b, double* x,
                                double tol, int32_t maxit, sketch_lsq_info* info,
                                sketch_stream_t stream) {
  return lsq_solve(h, A, b, x, tol, maxit, SKETCH_LSQ_SAP_QR, info, stream);
}

extern "C" int sketch_lsq_solve_method(sketch_t h, const sketch_csc* A, const double* b,
                                       double* x, double tol, int32_t maxit, int32_t method,
                                       sketch_lsq_info* info, sketch_stream_t stream) {
  return lsq_solve(h, A, b, x, tol, maxit, method, info, stream);
}

extern "C" int sketch_debug_qr(int64_t d, int64_t n, const double* A, double* R,
                               double* Rinv, sketch_stream_t stream) {
  if (d < 1 || n < 1 || d < n || n > 8192 || !A || !R || !Rinv)
    return fail(nullptr, SKETCH_ERR_ARG, "bad arguments");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double *W = nullptr, *tau = nullptr, *RT = nullptr, *rdiag = nullptr;
  int* status = nullptr;
  if (cudaMalloc(&W, sizeof(double) * d * n) != cudaSuccess ||
      cudaMalloc(&tau, sizeof(double) * 2 * n) != cudaSuccess ||
      cudaMalloc(&RT, sizeof(double) * n * n) != cudaSuccess ||
      cudaMalloc(&rdiag, sizeof(double) * n) != cudaSuccess ||
      cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
    cudaFree(W); cudaFree(tau); cudaFree(RT); cudaFree(rdiag); cudaFree(status);
    cudaGetLastError();
    return fail(nullptr, SKETCH_ERR_OOM, "cudaMalloc failed");
  }
  cudaMemcpyAsync(W, A, sizeof(double) * d * n, cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(status, 0, sizeof(int), s);
  double* vs = tau + n;
  k_qr_first<<<1, kQrThreads, 0, s>>>(W, d, tau, vs);
  for (int k = 0; k + 1 < n; ++k)
    launch(k_qr_step, qr_step_blocks(n, k), kQrThreads, s, 1, W, d, static_cast<int>(n), k,
           tau, vs);
  const unsigned gb = static_cast<unsigned>(std::max<int64_t>(1, 16LL * num_sms()));
  k_extract_r<<<gb, 256, 0, s>>>(W, d, static_cast<int>(n), R, rdiag, status);
  launch_trtri(W, d, static_cast<int>(n), rdiag, Rinv, RT, s);
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(W); cudaFree(tau); cudaFree(RT); cudaFree(rdiag); cudaFree(status);
  return e == cudaSuccess ? SKETCH_OK : cuda_fail(nullptr, e, "debug_qr");
}
