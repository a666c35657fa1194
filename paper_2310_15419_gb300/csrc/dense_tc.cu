// dense_tc.cu -- densified panels on the tensor cores (+-1 S only).
//
// Rows of A with many nonzeros form a dense panel A_D (K rows x n).  Their
// part of the sketch, S(:, D) A_D, is a real dense contraction (the large-
// density case of Sec. 3.1), so it runs as a BF16 MMA with FP32 accumulation:
//   * +-1 entries of S are exact in BF16;
//   * each FP32 value of A is split exactly into three BF16 terms
//     a = a1 + a2 + a3 (8 + 8 + 8 significant bits), so the panel is
//     A3 = [A1; A2; A3] (3K x n) against S3 = [S_D, S_D, S_D] and no input
//     rounding happens -- only the FP32 accumulation rounds;
//   * S_D's signs come straight from Philox bits: one block per (128 rows of
//     S, dense row), expanded to BF16 +-1 in registers (no S in memory).
// The sparse kernels run on the rest of A (a compacted CSC without the
// panel's rows), so A_hat = S A_rest + S_D A_D with the MMA adding into A_hat
// afterwards.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace sk {

namespace {

constexpr int kBM = 128;   // rows of S (A_hat) per CTA
constexpr int kBN = 128;   // columns of A per CTA
constexpr int kBK = 32;    // contraction step
constexpr int kLdB = 40;   // padded row length of the B tile (bf16)
constexpr int kTcThreads = 256;

__device__ __forceinline__ uint16_t bf16_bits(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// flag[j] = 1 for rows with at least `tau` nonzeros (counts from k_row_count)
__global__ void k_dense_flags(int32_t m, const int32_t* __restrict__ cnt, int32_t tau,
                              int32_t* __restrict__ flag) {
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j <= m;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x)
    flag[j] = (j < m && cnt[j] >= tau) ? 1 : 0;
}

// didx[j] = dense index of row j or -1; rows[k] = k-th dense row id.
__global__ void k_dense_index(int32_t m, const int32_t* __restrict__ flag,
                              const int32_t* __restrict__ pos, int32_t* __restrict__ didx,
                              int32_t* __restrict__ rows) {
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < m;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (flag[j]) {
      didx[j] = pos[j];
      rows[pos[j]] = static_cast<int32_t>(j);
    } else {
      didx[j] = -1;
    }
  }
}

// A3[k * K3 + t * Kp + didx[j]] = t-th BF16 term of A(j, k) for dense rows.
template <typename VT>
__global__ void k_dense_scatter(int32_t n, int32_t m, int32_t Kp,
                                const int32_t* __restrict__ colptr,
                                const int32_t* __restrict__ rowidx,
                                const VT* __restrict__ vals,
                                const int32_t* __restrict__ didx,
                                uint16_t* __restrict__ A3) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  const int64_t K3 = 3LL * Kp;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5);
       k < n; k += warps) {
    for (int32_t e = colptr[k] + lane; e < colptr[k + 1]; e += 32) {
      const int32_t j = rowidx[e];
      if (static_cast<uint32_t>(j) >= static_cast<uint32_t>(m)) continue;
      const int32_t q = didx[j];
      if (q < 0) continue;
      const float a = to_f32(vals[e]);
      const float a1 = __bfloat162float(__float2bfloat16_rn(a));
      const float r1 = a - a1;  // exact
      const float a2 = __bfloat162float(__float2bfloat16_rn(r1));
      const float a3 = r1 - a2;  // exact, fits BF16
      uint16_t* col = A3 + k * K3;
      col[q] = bf16_bits(a1);
      col[Kp + q] = bf16_bits(a2);
      col[2 * Kp + q] = bf16_bits(a3);
    }
  }
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4],
                                               const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// +-1 in BF16 for sign bits b0 (low half) and b1 (high half): 0 -> +1, 1 -> -1
__device__ __forceinline__ uint32_t pm1_pair(uint32_t b0, uint32_t b1) {
  return (0x3F80u | (b0 << 15)) | ((0x3F80u | (b1 << 15)) << 16);
}

// A_hat(rows d0.., cols n0..) += S3 A3 for a 128 x 128 tile; 8 warps as
// 4 (rows) x 2 (cols), each warp 32 x 64 = 2 x 8 fragments of 16 x 8.
// The contraction runs over the dense rows in steps of 32; each step's S
// signs (one Philox block per dense row) and the warps' +-1 A fragments are
// built once and serve the three BF16 terms of A.  The A3 tiles (128
// columns x 32 values of one term) stream through two shared buffers
// filled by cp.async one tile ahead of the MMAs.
__device__ __forceinline__ void tc_load_tile(uint16_t (*dst)[kLdB], const uint16_t* A3,
                                             int32_t n, int32_t n0, int64_t K3, int64_t koff) {
  for (int t = threadIdx.x; t < kBN * 4; t += kTcThreads) {
    const int c = t >> 2, part = t & 3;  // part: 8 values (16 bytes)
    const int col = n0 + c;
    const uint16_t* src = col < n ? A3 + col * K3 + koff + 8 * part : A3;
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(&dst[c][8 * part]));
    const int bytes = col < n ? 16 : 0;  // zero fill past the last column
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(kTcThreads)
    k_tc_gemm(int32_t d, int32_t n, int32_t Kp, const int32_t* __restrict__ rows,
              const int32_t* __restrict__ Kdev, const uint16_t* __restrict__ A3,
              float* __restrict__ Ahat, uint32_t k0, uint32_t k1, uint32_t stream_id,
              int accumulate) {
  __shared__ uint32_t sbits[kBK][4];                           // S signs, 128 rows
  __shared__ __align__(16) uint16_t btile[2][kBN][kLdB];       // A3 tiles, K fastest
  const int K = *Kdev;
  const int d0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = warp & 3, wn = warp >> 2;  // warp tile: rows wm*32, cols wn*64
  const int gid = lane >> 2, tig = lane & 3;
  const int64_t K3 = 3LL * Kp;
  const int steps = Kp / kBK;  // 32 dense rows per step, three terms each
  float acc[2][8][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

  // tile l = 3 * step + term holds A3 values [term * Kp + 32 step, +32)
  auto koff = [&](int l) { return static_cast<int64_t>(l % 3) * Kp + (l / 3) * kBK; };
  tc_load_tile(btile[0], A3, n, n0, K3, koff(0));
  for (int st = 0; st < steps; ++st) {
    // --- S signs for the 32 dense rows of this step --------------------------
    if (threadIdx.x < kBK) {
      const int q = st * kBK + threadIdx.x;
      const int32_t j = q < K ? rows[q] : 0;  // padding rows multiply zeros
      const uint4 x = philox_block(static_cast<uint32_t>(d0 >> 7), static_cast<uint32_t>(j),
                                   stream_id, k0, k1);
      sbits[threadIdx.x][0] = x.x;
      sbits[threadIdx.x][1] = x.y;
      sbits[threadIdx.x][2] = x.z;
      sbits[threadIdx.x][3] = x.w;
    }
    __syncthreads();
    // A fragments (S, 16 x 16 row-major) for both k halves, from sign bits
    uint32_t af[2][2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int fm = 0; fm < 2; ++fm) {
        const int r0 = wm * 32 + fm * 16 + gid, r1 = r0 + 8;
        const int c0 = 16 * h + 2 * tig, c8 = c0 + 8;
        auto bit = [&](int r, int c) { return (sbits[c][r >> 5] >> (r & 31)) & 1u; };
        af[h][fm][0] = pm1_pair(bit(r0, c0), bit(r0, c0 + 1));
        af[h][fm][1] = pm1_pair(bit(r1, c0), bit(r1, c0 + 1));
        af[h][fm][2] = pm1_pair(bit(r0, c8), bit(r0, c8 + 1));
        af[h][fm][3] = pm1_pair(bit(r1, c8), bit(r1, c8 + 1));
      }
#pragma unroll
    for (int term = 0; term < 3; ++term) {
      const int l = 3 * st + term;
      // the next tile streams in while this one is multiplied
      if (l + 1 < 3 * steps) {
        tc_load_tile(btile[(l + 1) & 1], A3, n, n0, K3, koff(l + 1));
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      __syncthreads();
      uint16_t (*bt)[kLdB] = btile[l & 1];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int ks = 16 * h;
#pragma unroll
        for (int fn = 0; fn < 8; ++fn) {
          const int cn = wn * 64 + fn * 8 + gid;
          uint32_t bf[2];
          bf[0] = *reinterpret_cast<const uint32_t*>(&bt[cn][ks + 2 * tig]);
          bf[1] = *reinterpret_cast<const uint32_t*>(&bt[cn][ks + 2 * tig + 8]);
          mma_bf16_16816(acc[0][fn], af[h][0], bf);
          mma_bf16_16816(acc[1][fn], af[h][1], bf);
        }
      }
      __syncthreads();  // the buffer is refilled two tiles later
    }
  }
  // --- add into (accumulate) or store to A_hat (column-major, ld = d) ------
#pragma unroll
  for (int fm = 0; fm < 2; ++fm)
#pragma unroll
    for (int fn = 0; fn < 8; ++fn) {
      const int r0 = d0 + wm * 32 + fm * 16 + gid;
      const int c0 = n0 + wn * 64 + fn * 8 + 2 * tig;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = r0 + 8 * h;
#pragma unroll
        for (int w = 0; w < 2; ++w) {
          const int c = c0 + w;
          if (r < d && c < n) {
            float* o = Ahat + static_cast<int64_t>(c) * d + r;
            *o = accumulate ? *o + acc[fm][fn][2 * h + w] : acc[fm][fn][2 * h + w];
          }
        }
      }
    }
}

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

namespace {
struct DenseLayout {
  int32_t *cnt, *flag, *pos, *didx, *Kdev;
  uint16_t* A3;
  char* scan_tmp;
  int32_t *rcnt, *rcolptr, *rrowidx;  // the rest of A (CSC)
  void* rvalues;
  size_t bytes;
};
DenseLayout dense_layout(void* ws, int64_t m, int64_t n, int64_t kmax, int64_t nnz) {
  DenseLayout L{};
  char* p = static_cast<char*>(ws);
  auto take = [&](size_t b) {
    char* r = p;
    p += al256(b);
    return r;
  };
  L.cnt = reinterpret_cast<int32_t*>(take((m + 1) * sizeof(int32_t)));
  L.flag = reinterpret_cast<int32_t*>(take((m + 1) * sizeof(int32_t)));
  L.pos = reinterpret_cast<int32_t*>(take((m + 1) * sizeof(int32_t)));
  L.didx = reinterpret_cast<int32_t*>(take((m + 1) * sizeof(int32_t)));
  L.Kdev = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 64));
  const int64_t Kp = (kmax + kBK - 1) / kBK * kBK;
  L.A3 = reinterpret_cast<uint16_t*>(take(static_cast<size_t>(n) * 3 * Kp * 2));
  L.scan_tmp = take(static_cast<size_t>(scan_bytes_for(std::max(m, n) + 1)));
  L.rcnt = reinterpret_cast<int32_t*>(take((n + 1) * sizeof(int32_t)));
  L.rcolptr = reinterpret_cast<int32_t*>(take((n + 1) * sizeof(int32_t)));
  L.rrowidx = reinterpret_cast<int32_t*>(take(std::max<int64_t>(1, nnz) * sizeof(int32_t)));
  L.rvalues = take(std::max<int64_t>(1, nnz) * sizeof(float));
  L.bytes = static_cast<size_t>(p - static_cast<char*>(ws));
  return L;
}

// Entries of column k that stay in the sparse part: rows outside the panel
// (and out-of-range rows, which the sparse kernels then flag).
__device__ __forceinline__ bool rest_keeps(int32_t j, int32_t m, const int32_t* didx) {
  return static_cast<uint32_t>(j) >= static_cast<uint32_t>(m) || didx[j] < 0;
}

// rcnt[k] = entries of column k outside the panel; rcnt[n] = 0.
__global__ void k_rest_count(int32_t n, int32_t m, const int32_t* __restrict__ colptr,
                             const int32_t* __restrict__ rowidx,
                             const int32_t* __restrict__ didx, int32_t* __restrict__ rcnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5);
       k <= n; k += warps) {
    int32_t c = 0;
    if (k < n)
      for (int32_t e = colptr[k] + lane; e < colptr[k + 1]; e += 32)
        c += rest_keeps(rowidx[e], m, didx);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) rcnt[k] = c;
  }
}

// The kept entries of column k, in their order, at rcolptr[k].. (one warp
// per column, ballot compaction).
template <typename VT>
__global__ void k_rest_copy(int32_t n, int32_t m, const int32_t* __restrict__ colptr,
                            const int32_t* __restrict__ rowidx, const VT* __restrict__ vals,
                            const int32_t* __restrict__ didx,
                            const int32_t* __restrict__ rcolptr,
                            int32_t* __restrict__ rrowidx, VT* __restrict__ rvals) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5);
       k < n; k += warps) {
    int32_t out = rcolptr[k];
    const int32_t hi = colptr[k + 1];
    for (int32_t e0 = colptr[k]; e0 < hi; e0 += 32) {
      const int32_t e = e0 + lane;
      int32_t j = 0;
      bool keep = false;
      if (e < hi) {
        j = rowidx[e];
        keep = rest_keeps(j, m, didx);
      }
      const unsigned mask = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int32_t pos = out + __popc(mask & below);
        rrowidx[pos] = j;
        rvals[pos] = vals[e];
      }
      out += __popc(mask);
    }
  }
}
}  // namespace

size_t dense_workspace_bytes(int64_t m, int64_t n, int64_t kmax, int64_t nnz) {
  return dense_layout(nullptr, m, n, kmax, nnz).bytes;
}

// Phase 1: choose the dense rows (at least tau nonzeros).  Writes didx,
// rows and K to the workspace, and the offsets of the rest of A; the caller
// reads K (the panel height) and rest_colptr[n] (the rest's nonzeros).
cudaError_t select_dense_rows(const DenseArgs& a, void* ws, DenseView* out, cudaStream_t s,
                              int* launches) {
  const DenseLayout L = dense_layout(ws, a.m, a.n, a.kmax, a.nnz);
  int32_t* rows = L.cnt;  // the counts are dead once the flags exist
  const int sms = num_sms();
  auto grid_for = [&](int64_t work) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 32LL * sms)));
  };
  cudaError_t e = cudaMemsetAsync(L.cnt, 0, (a.m + 1) * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  if ((e = row_counts(a.nnz, a.m, a.rowidx, L.cnt, a.status, s)) != cudaSuccess) return e;
  ++*launches;
  k_dense_flags<<<grid_for(a.m + 1), 256, 0, s>>>(a.m, L.cnt, a.tau, L.flag);
  ++*launches;
  if ((e = scan_i32(L.flag, L.pos, a.m + 1, L.scan_tmp, s, launches)) != cudaSuccess) return e;
  k_dense_index<<<grid_for(a.m), 256, 0, s>>>(a.m, L.flag, L.pos, L.didx, rows);
  ++*launches;
  if ((e = cudaMemcpyAsync(L.Kdev, L.pos + a.m, sizeof(int32_t), cudaMemcpyDeviceToDevice, s)) !=
      cudaSuccess)
    return e;
  out->didx = L.didx;
  out->rows = rows;
  out->Kdev = L.Kdev;
  out->A3 = L.A3;
  out->Kp = 0;
  out->rest_colptr = L.rcolptr;
  out->rest_rowidx = L.rrowidx;
  out->rest_values = L.rvalues;
  out->rest_cnt = L.rcnt;
  out->scan_tmp = L.scan_tmp;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the rest of A: per-column counts and offsets (rest_colptr[n] = its nnz)
  const int64_t wblocks = std::max<int64_t>(1, std::min<int64_t>((a.n + 8) / 8, 32LL * sms));
  k_rest_count<<<static_cast<unsigned>(wblocks), 256, 0, s>>>(a.n, a.m, a.colptr, a.rowidx,
                                                              L.didx, L.rcnt);
  ++*launches;
  return scan_i32(L.rcnt, L.rcolptr, a.n + 1, L.scan_tmp, s, launches);
}

// Phase 2: the panel's BF16 terms for K dense rows (K <= kmax).
cudaError_t build_dense_panel(const DenseArgs& a, int32_t K, DenseView* v, cudaStream_t s,
                              int* launches) {
  const int64_t Kp = (static_cast<int64_t>(K) + kBK - 1) / kBK * kBK;
  v->Kp = static_cast<int32_t>(Kp);
  uint16_t* A3 = const_cast<uint16_t*>(v->A3);
  cudaError_t e = cudaMemsetAsync(A3, 0, static_cast<size_t>(a.n) * 3 * Kp * 2, s);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((a.n + 7) / 8, 32LL * num_sms()));
  if (a.dtype == 0)
    k_dense_scatter<float><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
        a.n, a.m, static_cast<int32_t>(Kp), a.colptr, a.rowidx,
        static_cast<const float*>(a.values), v->didx, A3);
  else
    k_dense_scatter<__nv_bfloat16><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
        a.n, a.m, static_cast<int32_t>(Kp), a.colptr, a.rowidx,
        static_cast<const __nv_bfloat16*>(a.values), v->didx, A3);
  ++*launches;
  return cudaGetLastError();
}

// Phase 3: the rest of A (entries outside the panel's rows) compacted into
// its own CSC at the offsets phase 1 computed.
cudaError_t build_dense_rest(const DenseArgs& a, const DenseView& v, cudaStream_t s,
                             int* launches) {
  const int64_t wblocks = std::max<int64_t>(1, std::min<int64_t>((a.n + 8) / 8, 32LL * num_sms()));
  if (a.dtype == 0)
    k_rest_copy<float><<<static_cast<unsigned>(wblocks), 256, 0, s>>>(
        a.n, a.m, a.colptr, a.rowidx, static_cast<const float*>(a.values), v.didx,
        v.rest_colptr, const_cast<int32_t*>(v.rest_rowidx),
        static_cast<float*>(const_cast<void*>(v.rest_values)));
  else
    k_rest_copy<__nv_bfloat16><<<static_cast<unsigned>(wblocks), 256, 0, s>>>(
        a.n, a.m, a.colptr, a.rowidx, static_cast<const __nv_bfloat16*>(a.values), v.didx,
        v.rest_colptr, const_cast<int32_t*>(v.rest_rowidx),
        static_cast<__nv_bfloat16*>(const_cast<void*>(v.rest_values)));
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const DenseArgs& a, const DenseView& v, float* Ahat,
                           int accumulate, cudaStream_t s, int* launches) {
  const dim3 grid((a.d + kBM - 1) / kBM, (a.n + kBN - 1) / kBN);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  k_tc_gemm<<<grid, kTcThreads, 0, s>>>(a.d, a.n, v.Kp, v.rows, v.Kdev, v.A3, Ahat, a.k0,
                                        a.k1, a.stream_id, accumulate);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace sk
