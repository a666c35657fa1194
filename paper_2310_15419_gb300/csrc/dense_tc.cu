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
//     S, dense row), expanded to a BF16 +-1 tile in shared memory (no S in
//     global memory);
//   * the MMA is tcgen05 (5th-generation tensor cores) with the accumulator
//     in tensor memory.
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
__global__ void k_dense_scatter(int32_t n, int32_t m, int32_t Kp, int64_t nnz,
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
    const int2 range = column_range(colptr, k, nnz, nullptr);
    for (int32_t e = range.x + lane; e < range.y; e += 32) {
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

// +-1 in BF16 for sign bits b0 (low half) and b1 (high half): 0 -> +1, 1 -> -1
__device__ __forceinline__ uint32_t pm1_pair(uint32_t b0, uint32_t b1) {
  return (0x3F80u | (b0 << 15)) | ((0x3F80u | (b1 << 15)) << 16);
}

// ---------------------------------------------------------------------------
// A_hat(rows d0.., cols n0..) (+)= S3 A3 for a 128 x 128 tile on the
// 5th-generation tensor cores (tcgen05).  One thread issues
// `tcgen05.mma.cta_group::1.kind::f16` (M = N = 128, K = 16, BF16 in, FP32
// accumulate) with both operands in shared memory and the 128 x 128
// accumulator in tensor memory (128 columns, allocated per CTA).  Operand
// tiles (128 rows x 32 k, BF16) use the K-major layout without swizzle:
// 8-row x 16-byte core matrices, the next one along K 128 bytes on, along
// M/N 512 bytes on.  One iteration per 32 dense rows: the A tile (+-1 S,
// built once from Philox sign bits) and the three B tiles (the BF16 terms of
// A3, by cp.async one iteration ahead) form a stage; six MMAs (3 terms x 2 k
// halves) and one tcgen05.commit per iteration; a stage is reused once that
// commit has arrived on its mbarrier.  Every wait has an iteration limit: on
// expiry the CTA records kStatusTimeout, frees its tensor memory and stops.
// (N = 256 per CTA measured slower on Abnormal_A: 0.80 against 0.75 ms.)
constexpr uint32_t kUmmaLbo = 128, kUmmaSbo = 512;
constexpr int kUmmaTile = 8192;  // bytes of one 128 x 32 BF16 operand tile
// instruction descriptor: F32 accumulator, BF16 A and B, both K-major,
// N = 128 (N >> 3 at bit 17), M = 128 (M >> 4 at bit 24)
constexpr uint32_t kUmmaIdesc =
    (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
constexpr int kUmmaStages = 2;  // stage = A tile + the three B terms of a step
constexpr int kUmmaStageBytes = 4 * kUmmaTile;
// two stages + alignment; at most three CTAs share an SM, so 3 x 128
// tensor-memory columns never exceed the 512 there and tcgen05.alloc never
// waits for another CTA
constexpr size_t kUmmaSmem = kUmmaStages * kUmmaStageBytes + 1024;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N)
// byte offsets in 16-byte units, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) |
         (static_cast<uint64_t>((kUmmaLbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((kUmmaSbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// wait for the phase of parity `parity` of an mbarrier; false after `limit`
// polls
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit = 1 << 22) {
  for (int i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_umma(int32_t d, int32_t n, int32_t Kp, const int32_t* __restrict__ rows,
              const int32_t* __restrict__ Kdev, const uint16_t* __restrict__ A3,
              float* __restrict__ Ahat, uint32_t k0, uint32_t k1, uint32_t stream_id,
              int accumulate, int* status) {
  extern __shared__ uint8_t sm_raw[];
  __shared__ uint32_t sbits[kBK][4];
  // one mbarrier per stage, plus one that only the drain commit of the
  // failure path arrives on
  __shared__ __align__(8) uint64_t mbar[kUmmaStages + 1];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  uint8_t* base = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int d0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
  const int K = *Kdev;
  const int64_t K3 = 3LL * Kp;
  const int steps = Kp / kBK;
  auto tileA = [&](int stg) { return base + stg * kUmmaStageBytes; };
  auto tileB = [&](int stg, int term) { return base + stg * kUmmaStageBytes + (1 + term) * kUmmaTile; };
  // the three B tiles of step st: terms of A3, dense rows 32 st .. + 31
  auto load_B = [&](int st) {
    for (int c = tid; c < 3 * kBN * 4; c += kTcThreads) {
      const int term = c / (kBN * 4), cc = c % (kBN * 4);
      const int nn = cc >> 2, part = cc & 3;
      const int col = n0 + nn;
      const int64_t koff = static_cast<int64_t>(term) * Kp + kBK * st;
      const uint16_t* src = col < n ? A3 + col * K3 + koff + 8 * part : A3;
      const uint32_t dst = smem_u32(tileB(st % kUmmaStages, term) + (nn >> 3) * kUmmaSbo +
                                    part * kUmmaLbo + (nn & 7) * 16);
      const int bytes = col < n ? 16 : 0;  // zero fill past the last column
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                   "r"(bytes)
                   : "memory");
    }
  };
  if (tid == 0) {
    failed = 0;
    for (int q = 0; q <= kUmmaStages; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[q])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
                     smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  load_B(0);
  asm volatile("cp.async.commit_group;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  for (int st = 0; st < steps; ++st) {
    const int sb = st % kUmmaStages;
    // prefetch step st + 1 into the stage MMA(st - 1) read
    if (st + 1 < steps && st >= 1 && tid == 0 &&
        !mbar_wait(smem_u32(&mbar[(st - 1) % kUmmaStages]), ((st - 1) / kUmmaStages) & 1))
      failed = 1;
    if (tid < kBK) {  // S signs for the 32 dense rows of this step
      const int q = st * kBK + tid;
      const int32_t j = q < K ? rows[q] : 0;  // padding rows multiply zeros
      const uint4 x = philox_block(static_cast<uint32_t>(d0 >> 7), static_cast<uint32_t>(j),
                                   stream_id, k0, k1);
      sbits[tid][0] = x.x;
      sbits[tid][1] = x.y;
      sbits[tid][2] = x.z;
      sbits[tid][3] = x.w;
    }
    __syncthreads();
    if (failed) break;
    if (st + 1 < steps) load_B(st + 1);
    asm volatile("cp.async.commit_group;" ::: "memory");
    // A tile of step st: +-1 S (BF16), row r of the tile, k = dense row of
    // the step (its stage was last read by MMA(st - 2), which the wait of
    // iteration st - 1 covered)
    {
      uint8_t* smA = tileA(sb);
      const int r = tid & 127;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kc = 2 * (tid >> 7) + h;
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int ka = 8 * kc + 2 * u;
          const uint32_t b0 = (sbits[ka][r >> 5] >> (r & 31)) & 1u;
          const uint32_t b1 = (sbits[ka + 1][r >> 5] >> (r & 31)) & 1u;
          w[u] = pm1_pair(b0, b1);
        }
        *reinterpret_cast<uint4*>(smA + (r >> 3) * kUmmaSbo + kc * kUmmaLbo + (r & 7) * 16) =
            make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    // this step's B tiles have landed (at most one newer group)
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    // generic-proxy writes (st.shared, cp.async) -> visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int term = 0; term < 3; ++term)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint64_t ad = umma_desc(smem_u32(tileA(sb)) + 256 * h);
          const uint64_t bd = umma_desc(smem_u32(tileB(sb, term)) + 256 * h);
          const uint32_t acc = (st > 0 || term > 0 || h > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(kUmmaIdesc), "r"(acc)
              : "memory");
        }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar[sb]))
          : "memory");
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  // the last commit completes after every MMA before it
  if (!failed && tid == 0 &&
      !mbar_wait(smem_u32(&mbar[(steps - 1) % kUmmaStages]), ((steps - 1) / kUmmaStages) & 1))
    failed = 1;
  // After a timeout, MMAs issued earlier may still be running and writing
  // tensor memory: one more commit (it arrives once every MMA this thread
  // issued has completed) drains them before the memory is freed.  If even
  // that wait runs out, kStatusTimeout still goes to the host, and the
  // tensor-memory columns are freed with work possibly in flight (the error
  // documentation tells the caller to treat the context as unreliable).
  if (failed && tid == 0) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&mbar[kUmmaStages]))
        : "memory");
    mbar_wait(smem_u32(&mbar[kUmmaStages]), 0);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!failed) {
    // warp w: lanes (rows of S) 32 (w & 3) .. + 31, columns 64 (w >> 2) .. + 63
    const int rq = warp & 3;
    const int r = d0 + 32 * rq + lane;
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      const int c0 = 64 * (warp >> 2) + 32 * cc;
      uint32_t v[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
          "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, "
          "%26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
            "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
            "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
            "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
            "=r"(v[30]), "=r"(v[31])
          : "r"(tmem + (static_cast<uint32_t>(32 * rq) << 16) + static_cast<uint32_t>(c0)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (r < d) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = n0 + c0 + j;
          if (c < n) {
            float* o = Ahat + static_cast<int64_t>(c) * d + r;
            const float x = __uint_as_float(v[j]);
            *o = accumulate ? *o + x : x;
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(status, kStatusTimeout);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

// The timeout path of mbar_wait on purpose: a fresh mbarrier whose phase
// nothing completes; the bounded wait gives up and records kStatusTimeout.
__global__ void k_debug_wait_timeout(int* status, int limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(smem_u32(&bar), 0, limit)) atomicOr(status, kStatusTimeout);
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

// rcnt[k] = entries of column k outside the panel; rcnt[n] = 0.  A malformed
// colptr is recorded in *status (its column ranges are clamped to [0, nnz]).
__global__ void k_rest_count(int32_t n, int32_t m, int64_t nnz,
                             const int32_t* __restrict__ colptr,
                             const int32_t* __restrict__ rowidx,
                             const int32_t* __restrict__ didx, int32_t* __restrict__ rcnt,
                             int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5);
       k <= n; k += warps) {
    int32_t c = 0;
    if (k < n) {
      const int2 range = column_range(colptr, k, nnz, lane == 0 ? status : nullptr);
      for (int32_t e = range.x + lane; e < range.y; e += 32)
        c += rest_keeps(rowidx[e], m, didx);
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) rcnt[k] = c;
  }
}

// The kept entries of column k, in their order, at rcolptr[k].. (one warp
// per column, ballot compaction).
// (Write positions stay below nnz: overlapping column ranges of a malformed
// colptr could otherwise count more kept entries than A holds.)
template <typename VT>
__global__ void k_rest_copy(int32_t n, int32_t m, int64_t nnz,
                            const int32_t* __restrict__ colptr,
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
    const int2 range = column_range(colptr, k, nnz, nullptr);
    const int32_t hi = range.y;
    for (int32_t e0 = range.x; e0 < hi; e0 += 32) {
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
        if (static_cast<uint32_t>(pos) < static_cast<uint64_t>(nnz)) {
          rrowidx[pos] = j;
          rvals[pos] = vals[e];
        }
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
  k_rest_count<<<static_cast<unsigned>(wblocks), 256, 0, s>>>(a.n, a.m, a.nnz, a.colptr,
                                                              a.rowidx, L.didx, L.rcnt,
                                                              a.status);
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
        a.n, a.m, static_cast<int32_t>(Kp), a.nnz, a.colptr, a.rowidx,
        static_cast<const float*>(a.values), v->didx, A3);
  else
    k_dense_scatter<__nv_bfloat16><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
        a.n, a.m, static_cast<int32_t>(Kp), a.nnz, a.colptr, a.rowidx,
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
        a.n, a.m, a.nnz, a.colptr, a.rowidx, static_cast<const float*>(a.values), v.didx,
        v.rest_colptr, const_cast<int32_t*>(v.rest_rowidx),
        static_cast<float*>(const_cast<void*>(v.rest_values)));
  else
    k_rest_copy<__nv_bfloat16><<<static_cast<unsigned>(wblocks), 256, 0, s>>>(
        a.n, a.m, a.nnz, a.colptr, a.rowidx, static_cast<const __nv_bfloat16*>(a.values), v.didx,
        v.rest_colptr, const_cast<int32_t*>(v.rest_rowidx),
        static_cast<__nv_bfloat16*>(const_cast<void*>(v.rest_values)));
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_debug_wait_timeout(int* status, cudaStream_t s) {
  k_debug_wait_timeout<<<1, 32, 0, s>>>(status, 1 << 14);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const DenseArgs& a, const DenseView& v, float* Ahat,
                           int accumulate, cudaStream_t s, int* launches) {
  const dim3 grid((a.d + kBM - 1) / kBM, (a.n + kBN - 1) / kBN);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_tc_umma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kUmmaSmem));
  if (e != cudaSuccess) return e;
  k_tc_umma<<<grid, kTcThreads, kUmmaSmem, s>>>(a.d, a.n, v.Kp, v.rows, v.Kdev, v.A3, Ahat,
                                                a.k0, a.k1, a.stream_id, accumulate, a.status);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace sk
