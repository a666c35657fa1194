// sketch_kernels.cu -- the sketch A_hat = S A on sm_103a.
//
//  REGEN  (Alg. 3, variant kji, "regenerate per nonzero"): output-stationary.
//         A work item is (column k of A) x (tile of 128*Q rows of S).  The
//         item's accumulators live in registers; every nonzero (j, a) of the
//         column regenerates the S entries of the tile for row j.  For +-1
//         one Philox block gives 128 signs, so a warp computes one block per
//         nonzero (lane t for nonzero t of a batch of 32) and shares the
//         words through shared memory.  Deterministic.
//
//  PANEL  (Alg. 4, variant jki, "generate once per row"): a CTA owns a tile
//         of 32 rows of S, a block of columns and a contiguous range of rows
//         of A.  Its slice of A_hat lives in shared memory.  Each nonempty
//         row j of A generates S(tile, j) once and scatters it into all of
//         the row's nonzeros.  Row ranges give partial sums that an ordered
//         reduction adds up (Sec. 2.1's unblocked inner dimension is split
//         here only to fill the GPU and to bound FP32 summation length).
//
//  CSR    the per-row structure PANEL needs (the paper's blocked CSR with a
//         single vertical block, Sec. 3.2), built on the device: row counts,
//         exclusive scan, scatter.
#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "common.cuh"
#include "internal.h"

namespace sk {

// ---------------------------------------------------------------------------
// REGEN
// ---------------------------------------------------------------------------
constexpr int kRegenWarps = 8;

// sum += x with Kahan compensation c (no reassociation: plain FP32 ops)
__device__ __forceinline__ void kahan_add(float& sum, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(sum, y);
  c = __fsub_rn(__fsub_rn(t, sum), y);
  sum = t;
}

// One warp accumulates column nonzeros [lo, hi) against rows d0 .. d0+128Q-1
// of S; lane L owns rows d0 + 128 q + 4 L + r.  On return outer[q][r] holds
// the column's contribution to those rows.  `stage` is the warp's slice of
// the shared staging buffer (+-1 only).  Returns the S entries generated.
template <int DIST, int Q, typename VT>
__device__ __forceinline__ unsigned long long regen_accumulate(
    int32_t lo, int32_t hi, int32_t m, int32_t d0, int rows_valid,
    const int32_t* __restrict__ rowidx, const VT* __restrict__ vals,
    uint32_t k0, uint32_t k1, uint32_t stream_id, int* status,
    uint32_t (*stage)[4 * Q + 4], float (&outer)[Q][4]) {
  const int lane = threadIdx.x & 31;
  // Two-level sums: a batch of 32 nonzeros accumulates in `inner`, batch
  // sums are added to `outer` with Kahan compensation (`comp`), so the FP32
  // error stays near one rounding per batch however long the column is.
  float comp[Q][4];
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int r = 0; r < 4; ++r) outer[q][r] = comp[q][r] = 0.f;
  float t_outer = 0.f, t_comp = 0.f;  // +-1 only: sum of the column's values
  unsigned long long generated = 0;
  // bit masks of this lane's four rows inside its Philox word (+-1)
  uint32_t mask[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) mask[r] = 1u << (4 * (lane & 7) + r);

  for (int32_t base = lo; base < hi; base += 32) {
    const int cnt = min(32, hi - base);
    int32_t j = 0;
    float a = 0.f;
    if (lane < cnt) {
      j = rowidx[base + lane];
      a = to_f32(vals[base + lane]);
      if (static_cast<uint32_t>(j) >= static_cast<uint32_t>(m)) {
        atomicOr(status, kStatusBadRow);
        j = 0;
        a = 0.f;
      }
    }
    generated += static_cast<unsigned long long>(cnt) * rows_valid;
    float inner[Q][4];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) inner[q][r] = 0.f;

    if constexpr (DIST == kPM1) {
      // lane t: Philox blocks of nonzero t for the Q 128-row blocks
      if (lane < cnt) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const uint4 x = philox_block(static_cast<uint32_t>((d0 >> 7) + q),
                                       static_cast<uint32_t>(j), stream_id, k0, k1);
          *reinterpret_cast<uint4*>(&stage[lane][4 * q]) = x;
        }
      }
      __syncwarp();
      float t_inner = 0.f;
      const int wsel = lane >> 3;
      for (int t = 0; t < cnt; ++t) {
        const float at = __shfl_sync(0xffffffffu, a, t);
        t_inner += at;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const uint32_t w = stage[t][4 * q + wsel];
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (w & mask[r]) inner[q][r] += at;
        }
      }
      __syncwarp();
      kahan_add(t_outer, t_comp, t_inner);
    } else {
      for (int t = 0; t < cnt; ++t) {
        const int32_t jt = __shfl_sync(0xffffffffu, j, t);
        const float at = __shfl_sync(0xffffffffu, a, t);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const uint4 x = philox_block(static_cast<uint32_t>((d0 >> 2) + 32 * q + lane),
                                       static_cast<uint32_t>(jt), stream_id, k0, k1);
          const float4 sv = four_entries<DIST>(x);
          inner[q][0] = fmaf(at, sv.x, inner[q][0]);
          inner[q][1] = fmaf(at, sv.y, inner[q][1]);
          inner[q][2] = fmaf(at, sv.z, inner[q][2]);
          inner[q][3] = fmaf(at, sv.w, inner[q][3]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) kahan_add(outer[q][r], comp[q][r], inner[q][r]);
  }
  if constexpr (DIST == kPM1) {
    // sum over +1 rows minus sum over -1 rows = T - 2 P
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) outer[q][r] = t_outer - 2.f * outer[q][r];
  }
  return generated;
}

template <int DIST, int Q, typename VT>
__global__ void __launch_bounds__(kRegenWarps * 32, 2)
    k_regen(int32_t m, int32_t n, int32_t d, int32_t split, int64_t nnz,
            const int32_t* __restrict__ colptr,
            const int32_t* __restrict__ rowidx, const VT* __restrict__ vals,
            float* __restrict__ Ahat, uint32_t k0, uint32_t k1,
            uint32_t stream_id, int* status,
            unsigned long long* gen_count) {
  constexpr int TD = 128 * Q;          // rows of S per item
  constexpr int SW = 4 * Q + 4;        // staged words per nonzero (+pad)
  __shared__ float red[kRegenWarps][TD];
  __shared__ __align__(16) uint32_t stage[kRegenWarps][DIST == kPM1 ? 32 : 1][SW];

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int items_per_cta = kRegenWarps / split;
  const int sub = warp % split;
  const int dtiles = (d + TD - 1) / TD;
  const int64_t item =
      static_cast<int64_t>(blockIdx.x) * items_per_cta + warp / split;
  const bool valid = item < static_cast<int64_t>(n) * dtiles;
  const int32_t k = valid ? static_cast<int32_t>(item / dtiles) : 0;
  const int32_t d0 = valid ? static_cast<int32_t>(item % dtiles) * TD : 0;

  float outer[Q][4];
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int r = 0; r < 4; ++r) outer[q][r] = 0.f;
  unsigned long long generated = 0;

  if (valid) {
    const int2 range = column_range(colptr, k, nnz, status);
    const int32_t p0 = range.x;
    const int32_t len = range.y - range.x;
    const int32_t chunk = (len + split - 1) / split;
    const int32_t lo = p0 + min(len, sub * chunk);
    const int32_t hi = p0 + min(len, (sub + 1) * chunk);
    generated = regen_accumulate<DIST, Q, VT>(lo, hi, m, d0, min(TD, d - d0), rowidx,
                                             vals, k0, k1, stream_id, status,
                                             stage[warp], outer);
  }

  if (split == 1) {
    if (valid) {
#pragma unroll
      for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int32_t i = d0 + 128 * q + 4 * lane + r;
          if (i < d) Ahat[static_cast<int64_t>(k) * d + i] = outer[q][r];
        }
    }
  } else {
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) red[warp][128 * q + 4 * lane + r] = outer[q][r];
    __syncthreads();
    if (valid && sub == 0) {
#pragma unroll
      for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int c = 128 * q + 4 * lane + r;
          float sum = red[warp][c];
          for (int u = 1; u < split; ++u) sum += red[warp + u][c];
          const int32_t i = d0 + c;
          if (i < d) Ahat[static_cast<int64_t>(k) * d + i] = sum;
        }
    }
  }
  if (gen_count && valid) {
    // every lane holds the same warp-uniform count; lane 0 reports it
    if (lane == 0) atomicAdd(gen_count, generated);
  }
}

// ---------------------------------------------------------------------------
// Batched REGEN: many uneven sketches in one persistent launch.  Items
// (instance, column, tile of 128*Q rows of S) sit in a device work list
// sorted by decreasing nonzero count; each warp claims the next item from a
// counter (bounded: the loop ends when the counter passes the list), so the
// launch is fair to uneven instances and can be replayed from a CUDA graph
// once the counter is reset.
// ---------------------------------------------------------------------------
template <int DIST, int Q>
__global__ void __launch_bounds__(kRegenWarps * 32, 2)
    k_regen_batched(const BatchInstance* __restrict__ inst,
                    const BatchItem* __restrict__ items, int64_t n_items,
                    unsigned long long* __restrict__ counter, int* status) {
  constexpr int TD = 128 * Q;
  constexpr int SW = 4 * Q + 4;
  __shared__ __align__(16) uint32_t stage[kRegenWarps][DIST == kPM1 ? 32 : 1][SW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(counter, 1ULL);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= static_cast<unsigned long long>(n_items)) break;
    const BatchItem w = items[it];
    const BatchInstance& I = inst[w.instance];
    const int32_t d0 = w.tile * TD;
    const int32_t lo = I.colptr[w.column], hi = max(lo, I.colptr[w.column + 1]);
    float outer[Q][4];
    if (I.dtype == 0)
      regen_accumulate<DIST, Q, float>(lo, hi, I.m, d0, min(TD, I.d - d0), I.rowidx,
                                       static_cast<const float*>(I.values), I.k0, I.k1,
                                       I.stream_id, status, stage[warp], outer);
    else
      regen_accumulate<DIST, Q, __nv_bfloat16>(
          lo, hi, I.m, d0, min(TD, I.d - d0), I.rowidx,
          static_cast<const __nv_bfloat16*>(I.values), I.k0, I.k1, I.stream_id, status,
          stage[warp], outer);
    float* col = I.Ahat + static_cast<int64_t>(w.column) * I.d;
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int32_t i = d0 + 128 * q + 4 * lane + r;
        if (i < I.d) col[i] = outer[q][r];
      }
  }
}

cudaError_t launch_regen_batched(int dist, int q_tiles, const BatchInstance* inst,
                                 const BatchItem* items, int64_t n_items,
                                 unsigned long long* counter, int* status,
                                 int blocks, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const dim3 grid(blocks), block(kRegenWarps * 32);
#define SK_BATCH_CASE(DD, QQ)                                                  \
  if (dist == DD && q_tiles == QQ) {                                           \
    k_regen_batched<DD, QQ><<<grid, block, 0, s>>>(inst, items, n_items,      \
                                                   counter, status);          \
    return cudaGetLastError();                                                 \
  }
  SK_BATCH_CASE(kPM1, 1) SK_BATCH_CASE(kPM1, 2) SK_BATCH_CASE(kPM1, 4)
  SK_BATCH_CASE(kUniform, 1) SK_BATCH_CASE(kUniform, 2) SK_BATCH_CASE(kUniform, 4)
  SK_BATCH_CASE(kNormal, 1) SK_BATCH_CASE(kNormal, 2) SK_BATCH_CASE(kNormal, 4)
#undef SK_BATCH_CASE
  return cudaErrorInvalidValue;
}

int batched_blocks_per_sm(int dist, int q_tiles) {
  int nb = 0;
#define SK_OCC(DD, QQ)                                                          \
  if (dist == DD && q_tiles == QQ)                                              \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_regen_batched<DD, QQ>, \
                                                  kRegenWarps * 32, 0);
  SK_OCC(kPM1, 1) SK_OCC(kPM1, 2) SK_OCC(kPM1, 4)
  SK_OCC(kUniform, 1) SK_OCC(kUniform, 2) SK_OCC(kUniform, 4)
  SK_OCC(kNormal, 1) SK_OCC(kNormal, 2) SK_OCC(kNormal, 4)
#undef SK_OCC
  return nb > 0 ? nb : 1;
}

template <int DIST, typename VT>
static cudaError_t launch_regen_q(const RegenArgs& a, cudaStream_t s) {
  const int TD = 128 * a.q_tiles;
  const int64_t dtiles = (a.d + TD - 1) / TD;
  const int64_t items = static_cast<int64_t>(a.n) * dtiles;
  const int items_per_cta = kRegenWarps / a.split;
  const int64_t blocks = (items + items_per_cta - 1) / items_per_cta;
  if (blocks == 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const dim3 grid(static_cast<unsigned>(blocks)), block(kRegenWarps * 32);
  const VT* v = static_cast<const VT*>(a.values);
#define SK_REGEN_CASE(QQ)                                                   \
  case QQ:                                                                  \
    k_regen<DIST, QQ, VT><<<grid, block, 0, s>>>(                           \
        a.m, a.n, a.d, a.split, a.nnz, a.colptr, a.rowidx, v, a.Ahat, a.k0, a.k1, \
        a.stream_id, a.status, a.gen_count);                                \
    break;
  switch (a.q_tiles) {
    SK_REGEN_CASE(1)
    SK_REGEN_CASE(2)
    SK_REGEN_CASE(3)
    SK_REGEN_CASE(4)
    default:
      return cudaErrorInvalidValue;
  }
#undef SK_REGEN_CASE
  return cudaGetLastError();
}

cudaError_t launch_regen(const RegenArgs& a, cudaStream_t s) {
  if (a.split != 1 && a.split != 2 && a.split != 4 && a.split != 8)
    return cudaErrorInvalidValue;
  if (a.dtype == 0) {
    switch (a.dist) {
      case kPM1: return launch_regen_q<kPM1, float>(a, s);
      case kUniform: return launch_regen_q<kUniform, float>(a, s);
      case kNormal: return launch_regen_q<kNormal, float>(a, s);
    }
  } else {
    switch (a.dist) {
      case kPM1: return launch_regen_q<kPM1, __nv_bfloat16>(a, s);
      case kUniform: return launch_regen_q<kUniform, __nv_bfloat16>(a, s);
      case kNormal: return launch_regen_q<kNormal, __nv_bfloat16>(a, s);
    }
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// CSR build (row counts -> exclusive scan -> scatter)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void k_row_count(int64_t nnz, int32_t m,
                            const int32_t* __restrict__ rowidx,
                            int32_t* __restrict__ cnt, int* status) {
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       p < nnz; p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t j = rowidx[p];
    if (static_cast<uint32_t>(j) < static_cast<uint32_t>(m))
      atomicAdd(&cnt[j], 1);
    else
      atomicOr(status, kStatusBadRow);
  }
}

// Block-level exclusive scan of kScanTile ints; writes the tile total.
__global__ void __launch_bounds__(kScanThreads)
    k_scan_tiles(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                 int64_t len, int32_t* __restrict__ tile_sums) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile +
                       static_cast<int64_t>(threadIdx.x) * kScanItems;
  int32_t v[kScanItems];
  int32_t run = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    v[t] = (base + t < len) ? in[base + t] : 0;
    run += v[t];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int32_t w = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = w;  // inclusive
  }
  __syncthreads();
  int32_t excl = incl - run + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    if (base + t < len) out[base + t] = excl;
    excl += v[t];
  }
  if (threadIdx.x == kScanThreads - 1 && tile_sums)
    tile_sums[blockIdx.x] = warp_tot[kScanThreads / 32 - 1];
}

__global__ void k_scan_add(int32_t* __restrict__ out, int64_t len,
                           const int32_t* __restrict__ tile_offsets) {
  const int64_t tile = blockIdx.x;
  const int32_t off = tile_offsets[tile];
  const int64_t base = tile * kScanTile;
  for (int t = threadIdx.x; t < kScanTile; t += blockDim.x)
    if (base + t < len) out[base + t] += off;
}

static int64_t scan_levels_bytes(int64_t len) {
  int64_t bytes = 0;
  while (len > 1) {
    const int64_t tiles = (len + kScanTile - 1) / kScanTile;
    bytes += tiles * 2 * static_cast<int64_t>(sizeof(int32_t)) + 256;
    len = tiles;
  }
  return bytes;
}

// Exclusive scan of `len` ints (in may equal out).  `tmp` needs
// scan_levels_bytes(len) bytes.
static cudaError_t exclusive_scan(const int32_t* in, int32_t* out, int64_t len,
                                  char* tmp, cudaStream_t s, int* launches) {
  const int64_t tiles = (len + kScanTile - 1) / kScanTile;
  if (tiles <= 0) return cudaSuccess;
  int32_t* sums = reinterpret_cast<int32_t*>(tmp);
  int32_t* sums_scanned = sums + tiles;
  k_scan_tiles<<<static_cast<unsigned>(tiles), kScanThreads, 0, s>>>(
      in, out, len, tiles > 1 ? sums : nullptr);
  ++*launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || tiles == 1) return e;
  char* next = tmp + ((tiles * 2 * sizeof(int32_t) + 255) / 256) * 256;
  e = exclusive_scan(sums, sums_scanned, tiles, next, s, launches);
  if (e != cudaSuccess) return e;
  k_scan_add<<<static_cast<unsigned>(tiles), 256, 0, s>>>(out, len,
                                                          sums_scanned);
  ++*launches;
  return cudaGetLastError();
}

// Each column's nonzeros go to their rows' next free slots.  A slot past the
// row's end (only possible when colptr's column ranges overlap) is not
// written; the malformed colptr is recorded instead.
template <typename VT>
__global__ void k_csr_scatter(int32_t n, int32_t m, int64_t nnz,
                              const int32_t* __restrict__ colptr,
                              const int32_t* __restrict__ rowidx,
                              const VT* __restrict__ vals,
                              const int32_t* __restrict__ rowptr,
                              int32_t* __restrict__ cursor,
                              int32_t* __restrict__ ccol,
                              float* __restrict__ cval, int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) +
                   (threadIdx.x >> 5);
       k < n; k += warps) {
    const int2 range = column_range(colptr, k, nnz, status);
    for (int32_t p = range.x + lane; p < range.y; p += 32) {
      const int32_t j = rowidx[p];
      if (static_cast<uint32_t>(j) >= static_cast<uint32_t>(m)) continue;
      const int32_t pos = rowptr[j] + atomicAdd(&cursor[j], 1);
      if (pos >= rowptr[j + 1]) {
        atomicOr(status, kStatusBadColptr);
        continue;
      }
      ccol[pos] = static_cast<int32_t>(k);
      cval[pos] = to_f32(vals[p]);
    }
  }
}

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

size_t csr_workspace_bytes(int64_t m, int64_t nnz) {
  return align256((m + 1) * sizeof(int32_t)) * 2 +       // cnt/cursor, rowptr
         align256(nnz * sizeof(int32_t)) +               // ccol
         align256(nnz * sizeof(float)) +                 // cval
         align256(static_cast<size_t>(scan_levels_bytes(m + 1)));
}

cudaError_t build_csr(int32_t m, int32_t n, int64_t nnz, const int32_t* colptr,
                      const int32_t* rowidx, const void* values, int32_t dtype,
                      void* ws, CsrView* out, int* status, cudaStream_t s,
                      int* launches) {
  char* p = static_cast<char*>(ws);
  int32_t* cnt = reinterpret_cast<int32_t*>(p);
  p += align256((m + 1) * sizeof(int32_t));
  int32_t* rowptr = reinterpret_cast<int32_t*>(p);
  p += align256((m + 1) * sizeof(int32_t));
  int32_t* ccol = reinterpret_cast<int32_t*>(p);
  p += align256(nnz * sizeof(int32_t));
  float* cval = reinterpret_cast<float*>(p);
  p += align256(nnz * sizeof(float));
  char* scan_tmp = p;

  cudaError_t e = cudaMemsetAsync(cnt, 0, (m + 1) * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  const int sms = num_sms();
  if (nnz > 0) {
    const int64_t blocks = std::min<int64_t>((nnz + 255) / 256, 32LL * sms);
    k_row_count<<<static_cast<unsigned>(blocks), 256, 0, s>>>(nnz, m, rowidx,
                                                              cnt, status);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = exclusive_scan(cnt, rowptr, m + 1, scan_tmp, s, launches)) !=
      cudaSuccess)
    return e;
  if (nnz > 0) {
    if ((e = cudaMemsetAsync(cnt, 0, (m + 1) * sizeof(int32_t), s)) !=
        cudaSuccess)
      return e;
    const int64_t blocks = std::min<int64_t>((n + 7) / 8, 32LL * sms);
    if (dtype == 0)
      k_csr_scatter<float><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
          n, m, nnz, colptr, rowidx, static_cast<const float*>(values), rowptr, cnt,
          ccol, cval, status);
    else
      k_csr_scatter<__nv_bfloat16><<<static_cast<unsigned>(blocks), 256, 0,
                                     s>>>(
          n, m, nnz, colptr, rowidx, static_cast<const __nv_bfloat16*>(values),
          rowptr, cnt, ccol, cval, status);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  out->rowptr = rowptr;
  out->ccol = ccol;
  out->cval = cval;
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// PANEL
// ---------------------------------------------------------------------------
constexpr int kPanelWarps = 16;
constexpr int kPanelRows = 32;  // rows of S per CTA
constexpr int kBatchRows = 8;   // rows of A a warp takes at a time

size_t panel_smem_bytes(int32_t n_block, bool compensated) {
  return static_cast<size_t>(n_block) * kPanelRows * sizeof(float) * (compensated ? 2 : 1) +
         kPanelWarps * kBatchRows * 32 * sizeof(float);
}

// old + x as the atomic add stored it (round to nearest even), and the exact
// rounding error of that addition (Knuth's TwoSum), so that
// old + x = fl(old + x) + err holds exactly.
__device__ __forceinline__ float two_sum_err(float old, float x) {
  const float s = __fadd_rn(old, x);
  const float bb = __fsub_rn(s, old);
  return __fadd_rn(__fsub_rn(old, __fsub_rn(s, bb)), __fsub_rn(x, bb));
}

// COMP = true: every shared-memory atomic add also adds its own rounding
// error (two_sum_err of the value it replaced and the addend) into a second
// array, and the output is sum + compensation.  A column's whole nonzero list
// can then be summed in one row group (no partial buffers) and still keep
// the error near one rounding of the result, however long the column is.
template <int DIST, bool COMP>
__global__ void __launch_bounds__(kPanelWarps * 32, 1)
    k_panel(int32_t m, int32_t n, int32_t d, int32_t nb, int32_t G,
            const int32_t* __restrict__ rowptr,
            const int32_t* __restrict__ ccol, const float* __restrict__ cval,
            float* __restrict__ partial, uint32_t k0, uint32_t k1,
            uint32_t stream_id, unsigned long long* gen_count) {
  extern __shared__ __align__(16) float smem[];
  const int tile = blockIdx.x;
  const int32_t kb0 = blockIdx.y * nb;
  const int g = blockIdx.z;
  const int32_t nbw = min(nb, n - kb0);
  float* acc = smem;                                // [nbw][32]
  float* comp = smem + static_cast<size_t>(nb) * kPanelRows;  // [nbw][32] (COMP)
  float* stage_all = smem + static_cast<size_t>(nb) * kPanelRows * (COMP ? 2 : 1);
  for (int t = threadIdx.x; t < nbw * kPanelRows; t += blockDim.x) {
    acc[t] = 0.f;
    if constexpr (COMP) comp[t] = 0.f;
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* stage = stage_all + warp * (kBatchRows * 32);
  const int32_t r0 = static_cast<int32_t>(static_cast<int64_t>(m) * g / G);
  const int32_t r1 = static_cast<int32_t>(static_cast<int64_t>(m) * (g + 1) / G);
  const int rows_valid = min(kPanelRows, d - tile * kPanelRows);
  unsigned long long generated = 0;

  for (int32_t jb = r0 + kBatchRows * warp; jb < r1;
       jb += kBatchRows * kPanelWarps) {
    // --- row pointers of the batch: one load, lanes 0..kBatchRows ---------
    const int32_t rp = rowptr[min(jb + min(lane, kBatchRows), r1)];
    const int32_t p_beg = __shfl_sync(0xffffffffu, rp, 0);
    const int32_t p_end = __shfl_sync(0xffffffffu, rp, kBatchRows);
    if (p_beg == p_end) continue;  // the whole batch is empty
    // --- first chunk of the batch's nonzeros (contiguous in the CSR) ------
    int32_t chunk = p_beg;
    int32_t kk = -1;
    float aa = 0.f;
    if (chunk + lane < p_end) {
      kk = ccol[chunk + lane] - kb0;
      aa = cval[chunk + lane];
    }
    // --- generate S(tile, j) once for every nonempty row of the batch -----
#pragma unroll
    for (int h = 0; h < kBatchRows / 4; ++h) {
      const int r = 4 * h + (lane >> 3), q = lane & 7;
      const int32_t lo = __shfl_sync(0xffffffffu, rp, r);
      const int32_t hi = __shfl_sync(0xffffffffu, rp, r + 1);
      const bool nonempty = hi > lo;  // rows past r1 have lo == hi
      const uint32_t j = static_cast<uint32_t>(jb + r);
      if constexpr (DIST == kPM1) {
        // block (tile >> 2, j) holds this tile's 32 signs in word (tile & 3)
        if (q == 0 && nonempty) {
          const uint4 x = philox_block(static_cast<uint32_t>(tile >> 2), j,
                                       stream_id, k0, k1);
          const int wsel = tile & 3;
          const uint32_t w = wsel == 0 ? x.x : wsel == 1 ? x.y : wsel == 2 ? x.z : x.w;
          reinterpret_cast<uint32_t*>(stage)[r * 32] = w;
        }
      } else {
        if (nonempty) {
          const uint4 x = philox_block(static_cast<uint32_t>(tile * 8 + q), j,
                                       stream_id, k0, k1);
          *reinterpret_cast<float4*>(&stage[r * 32 + 4 * q]) = four_entries<DIST>(x);
        }
      }
      if (q == 0 && nonempty) generated += rows_valid;
    }
    __syncwarp();
    float sv[kBatchRows];
#pragma unroll
    for (int rr = 0; rr < kBatchRows; ++rr) {
      if constexpr (DIST == kPM1) {
        const uint32_t w = reinterpret_cast<const uint32_t*>(stage)[rr * 32];
        sv[rr] = ((w >> lane) & 1u) ? -1.f : 1.f;
      } else {
        sv[rr] = stage[rr * 32 + lane];
      }
    }
    __syncwarp();
    // --- scatter each row's S column into its nonzeros --------------------
#pragma unroll
    for (int rr = 0; rr < kBatchRows; ++rr) {
      const int32_t lo = __shfl_sync(0xffffffffu, rp, rr);
      const int32_t hi = __shfl_sync(0xffffffffu, rp, rr + 1);
      for (int32_t e = lo; e < hi; ++e) {
        if (e - chunk >= 32) {  // warp-uniform: next chunk of nonzeros
          chunk += 32;
          kk = -1;
          aa = 0.f;
          if (chunk + lane < p_end) {
            kk = ccol[chunk + lane] - kb0;
            aa = cval[chunk + lane];
          }
        }
        const int32_t kt = __shfl_sync(0xffffffffu, kk, e - chunk);
        const float at = __shfl_sync(0xffffffffu, aa, e - chunk);
        if (static_cast<uint32_t>(kt) < static_cast<uint32_t>(nbw)) {
          const float x = at * sv[rr];
          const float old = atomicAdd(&acc[kt * kPanelRows + lane], x);
          if constexpr (COMP) atomicAdd(&comp[kt * kPanelRows + lane], two_sum_err(old, x));
        }
      }
    }
  }
  __syncthreads();
  float* out = partial + (static_cast<int64_t>(g) * n + kb0) * d +
               static_cast<int64_t>(tile) * kPanelRows;
  for (int t = threadIdx.x; t < nbw * kPanelRows; t += blockDim.x) {
    const int kk2 = t >> 5, i = t & 31;
    if (i < rows_valid) {
      float v = acc[t];
      if constexpr (COMP) v += comp[t];
      out[static_cast<int64_t>(kk2) * d + i] = v;
    }
  }
  if (gen_count) {
    // lanes 0, 8, 16, 24 counted different rows: sum over the warp
    unsigned long long tot = generated;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0 && tot) atomicAdd(gen_count, tot);
  }
}

// A_hat = sum over g of partial[g] in the fixed order g = 0, 1, ...
__global__ void k_reduce_partials(int64_t total, int32_t G,
                                  const float* __restrict__ partial,
                                  float* __restrict__ Ahat) {
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       idx < total; idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float s = partial[idx];
    for (int g = 1; g < G; ++g) s += partial[static_cast<int64_t>(g) * total + idx];
    Ahat[idx] = s;
  }
}

cudaError_t launch_panel(const PanelArgs& a, cudaStream_t s, int* launches) {
  if (a.n_block <= 0 || a.row_groups <= 0) return cudaErrorInvalidValue;
  const size_t smem = panel_smem_bytes(a.n_block, a.compensated != 0);
  const int tiles = (a.d + kPanelRows - 1) / kPanelRows;
  const int cblocks = (a.n + a.n_block - 1) / a.n_block;
  if (cblocks > 65535 || a.row_groups > 65535) return cudaErrorInvalidValue;
  const dim3 grid(tiles, cblocks, a.row_groups), block(kPanelWarps * 32);
  cudaError_t e;
  // a single row group writes straight into A_hat
  float* dst = a.row_groups == 1 ? a.Ahat : a.partial;
#define SK_PANEL_CASE(DD, CC)                                                \
  if (a.dist == DD && (a.compensated != 0) == CC) {                          \
    e = raise_smem_limit(reinterpret_cast<const void*>(k_panel<DD, CC>), smem); \
    if (e != cudaSuccess) return e;                                          \
    k_panel<DD, CC><<<grid, block, smem, s>>>(                               \
        a.m, a.n, a.d, a.n_block, a.row_groups, a.csr.rowptr, a.csr.ccol,    \
        a.csr.cval, dst, a.k0, a.k1, a.stream_id, a.gen_count);              \
    ++*launches;                                                             \
    launched = true;                                                         \
  }
  bool launched = false;
  SK_PANEL_CASE(kPM1, false) SK_PANEL_CASE(kUniform, false) SK_PANEL_CASE(kNormal, false)
  SK_PANEL_CASE(kPM1, true) SK_PANEL_CASE(kUniform, true) SK_PANEL_CASE(kNormal, true)
#undef SK_PANEL_CASE
  if (!launched) return cudaErrorInvalidValue;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.row_groups > 1) {
    const int64_t total = static_cast<int64_t>(a.n) * a.d;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 16LL * num_sms());
    k_reduce_partials<<<static_cast<unsigned>(blocks), 256, 0, s>>>(
        total, a.row_groups, a.partial, a.Ahat);
    ++*launches;
    e = cudaGetLastError();
  }
  return e;
}


// ---------------------------------------------------------------------------
// TILE: the three-level blocking of Sec. 3.1 (S_sub d1 x m1, A_sub m1 x n1).
// A CTA owns a tile of 32 rows of S (d1 = 32) and a range of row panels of A
// (m1 = R rows each) for a block of columns (n1 = warps * CPW).  Per panel it
// generates S(tile, panel) ONCE into shared memory -- d1 * m1 entries, the
// minimum -- then every warp sweeps its columns in CSC order, reading S from
// shared memory, with its running sums in registers or in tensor memory.  No
// atomics; each output is written once per row group, so results are
// deterministic.
// ---------------------------------------------------------------------------
// TILE's S source besides the three distributions: S read from memory, as
// written by k_generate_S (the "pre-generated S" of Fig. percent_peak).
constexpr int kFromMemory = 3;
// Warps per CTA: 16 with register sums (64 columns each), 32 with
// tensor-memory sums (32 columns each); n1 = 1024 columns either way.
__host__ __device__ constexpr int tile_warps(bool tacc) { return tacc ? 32 : 16; }
// Staged nonzeros per warp and panel (a panel that holds more for a warp's
// columns sweeps the rest from global memory): 512, or 256 for the warps of
// half as many columns.
__host__ __device__ constexpr int tile_warp_buf(bool tacc) { return tacc ? 256 : 512; }

// Panel-major copy of A for TILE: nonzeros sorted by (panel, column, row),
// each stored as (row within its panel, value bits).  For panel p and column
// k the nonzeros are packed[off[p * (n + 1) + k] .. off[p * (n + 1) + k + 1]),
// so a warp's contiguous column range is one contiguous range of memory.

// pp[p * n + k] = first position of column k whose row is >= p * R
// (p = 0..P): a binary search over the column's sorted rows.
__global__ void k_panel_pointers(int32_t n, int32_t P, int32_t R, int64_t nnz,
                                 const int32_t* __restrict__ colptr,
                                 const int32_t* __restrict__ rowidx,
                                 int32_t* __restrict__ pp, int* status) {
  const int64_t total = static_cast<int64_t>(P + 1) * n;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       t < total; t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t p = static_cast<int32_t>(t / n), k = static_cast<int32_t>(t % n);
    const int2 range = column_range(colptr, k, nnz, p == 0 ? status : nullptr);
    int32_t lo = range.x, hi = range.y;
    const int64_t key = static_cast<int64_t>(p) * R;
    while (lo < hi) {
      const int32_t mid = lo + ((hi - lo) >> 1);
      if (rowidx[mid] < key) lo = mid + 1; else hi = mid;
    }
    pp[t] = lo;
  }
}

// cnt[p * (n + 1) + k] = pp[p + 1][k] - pp[p][k]; slot (p, n) and the final
// cell are 0, so an exclusive scan gives the panel-major offsets.
__global__ void k_panel_counts(int32_t n, int32_t P, const int32_t* __restrict__ pp,
                               int32_t* __restrict__ cnt) {
  const int64_t cells = static_cast<int64_t>(P) * (n + 1) + 1;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       t < cells; t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t p = t / (n + 1), k = t % (n + 1);
    // negative only for rows not sorted within a column (malformed input)
    cnt[t] = (p < P && k < n) ? max(0, pp[(p + 1) * n + k] - pp[p * n + k]) : 0;
  }
}

// One thread per (panel, column) segment copies it to its panel-major slot
// as (32 * row within the panel, value bits): the row pre-scaled to its
// offset in the [R][32] S tile.  A row outside the panel (unsorted
// or out-of-range input) becomes (0, 0.0) and is flagged.
template <typename VT>
__global__ void k_panel_copy(int32_t n, int32_t P, int32_t R, int32_t m, int64_t nnz,
                             const int32_t* __restrict__ rowidx,
                             const VT* __restrict__ vals,
                             const int32_t* __restrict__ pp,
                             const int32_t* __restrict__ off,
                             int2* __restrict__ packed, int* status) {
  const int64_t total = static_cast<int64_t>(P) * n;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       t < total; t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t p = t / n, k = t % n;
    const int32_t lo = pp[t], hi = pp[t + n];
    int32_t dst = off[p * (n + 1) + k];
    const int32_t j0 = static_cast<int32_t>(p * R);
    for (int32_t e = lo; e < hi; ++e, ++dst) {
      if (dst >= nnz) {  // only for rows not sorted within a column
        atomicOr(status, kStatusBadRow);
        break;
      }
      const int32_t jl = rowidx[e] - j0;
      if (static_cast<uint32_t>(jl) < static_cast<uint32_t>(R) && j0 + jl < m) {
        packed[dst] = make_int2(jl * 32, __float_as_int(to_f32(vals[e])));
      } else {
        atomicOr(status, kStatusBadRow);
        packed[dst] = make_int2(0, 0);
      }
    }
  }
}

// Tensor-memory accumulators for TILE (tcgen05.ld / tcgen05.st, shape
// 32x32b: thread t of a warp reads or writes lane 32 * (warp % 4) + t, four
// consecutive 32-bit columns).  The waits take the loaded registers as
// operands so no use of them is scheduled before the data has landed.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld4(uint32_t (&r)[4]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, float4 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
               "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)),
               "r"(__float_as_uint(v.z)), "r"(__float_as_uint(v.w))
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Tensor-memory sums (TACC = true) run as one wave of C CTAs per column
// block that walk the G row groups ("phases") in order; in every phase CTA c
// takes the same share c / C of the phase's units u = tile * Pp + panel
// (tile-major, Pp panels), so all CTAs sweep the same panels of A at about
// the same time (shared in L2) and every share costs the same (a tile's
// units of one phase are the same panels).  A share meets at most
// ceil(tiles / C) + 1 tiles, from tile c * tiles / C or the next on.  After a
// tile's units of a phase the CTA adds its tensor-memory sums into that
// tile's slot (a 32 x n block in global memory, L2-resident), so each tile
// gets the register path's additions: running sums over a row group, then
// the row groups in order.  A tile one CTA owns entirely goes straight to
// A_hat after the last phase; the other tiles' slots are added in CTA order
// by k_reduce_segments.

// CTA c of C owns all of tile x in every phase.
__host__ __device__ __forceinline__ bool tile_whole(int64_t x, int64_t c, int64_t tiles,
                                                    int64_t C) {
  return c * tiles <= x * C && (c + 1) * tiles >= (x + 1) * C;
}

// TACC = false: 16 warps; the CTA's 32 x (16 * CPW) accumulators live in
// registers (64 per thread at CPW = 64), so one CTA fills an SM's register
// file with 4 warps per scheduler.  Grid (tiles, column blocks, G): the CTA
// takes row group blockIdx.z of tile blockIdx.x; with G > 1 each group
// writes a full partial copy of A_hat for k_reduce_partials.
// TACC = true (CPW = 32 only): 32 warps, and the 32 x 1024 accumulators live
// in tensor memory, 256 columns per CTA (warp w: lanes 32 (w % 4) ..,
// columns 32 (w / 4) ..), each quad's float4 read, added to and written back
// after its sweep; at <= 64 registers per thread the SM runs 8 warps per
// scheduler with the same panel height.  Grid (C, column blocks): see above;
// `slots` holds kslots blocks of n x 32 floats per CTA and `sflags` marks
// the ones k_reduce_segments adds.
template <int DIST, int CPW, bool TACC>
__global__ void __launch_bounds__(tile_warps(TACC) * 32, 1)
    k_tile(int32_t m, int32_t n, int32_t d, int32_t R, int32_t P, int32_t G,
           const int2* __restrict__ packed, const int32_t* __restrict__ off, int32_t nnz,
           float* __restrict__ out, float* __restrict__ slots, int32_t kslots,
           int32_t* __restrict__ sflags, const __grid_constant__ PhiloxKeys keys,
           uint32_t stream_id, unsigned long long* gen_count,
           const float* __restrict__ S_mem, int64_t ld_s) {
  static_assert(CPW % 4 == 0, "columns per warp come in quads");
  static_assert(!TACC || CPW == 32, "tensor-memory accumulators take 32 columns per warp");
  constexpr int kWarps = tile_warps(TACC);
  constexpr uint32_t kTmemCols = (kWarps / 4) * CPW;  // kWarps / 4 warps per lane quarter
  constexpr int wbuf = tile_warp_buf(TACC);
  // shared memory: S tile [R][32] floats, per-warp nonzero buffers (wbuf
  // entries + a zero entry), per-warp column offsets, the tensor-memory base
  extern __shared__ __align__(16) float smem[];
  float* S_tile = smem;
  int2* ent_all = reinterpret_cast<int2*>(smem + static_cast<size_t>(R) * 32);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // lane = (column group cg, rows 4*i4 .. 4*i4+3 of the tile): the warp works
  // on four columns at a time, eight lanes (32 rows of S) per column
  const int cg = lane >> 3, i4 = lane & 7;
  int2* ent = ent_all + warp * (wbuf + 1);
  if (lane == 0) ent[wbuf] = make_int2(0, 0);  // the zero entry
  // this warp's column offsets for the current panel (CPW + 1 values)
  int32_t* offs_all = reinterpret_cast<int32_t*>(ent_all + kWarps * (wbuf + 1));
  int32_t* offs = offs_all + warp * (CPW + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(offs_all + kWarps * (CPW + 4));
  // this warp's columns: kw0 .. kw0 + ncol - 1 (contiguous)
  const int32_t kw0 = blockIdx.y * (kWarps * CPW) + warp * CPW;
  const int32_t ncol = max(0, min(CPW, n - kw0));
  const int tiles = (d + 31) / 32;
  // tensor-memory sums: C CTAs per column block; share c starts in tile x0
  const int32_t C = TACC ? static_cast<int32_t>(gridDim.x) : 1;
  const int32_t c = blockIdx.x;
  const int32_t x0 = TACC ? static_cast<int32_t>(static_cast<int64_t>(c) * tiles / C) : c;
  const float* S_lane = S_tile + 4 * i4;
  constexpr int OFFR = (CPW + 32) / 32;  // registers holding CPW + 1 offsets
  constexpr int NQ = CPW / 4;

  float4 acc[TACC ? 1 : NQ];
  uint32_t tacc = 0;  // this warp's first accumulator column in tensor memory
  if constexpr (TACC) {
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       static_cast<uint32_t>(__cvta_generic_to_shared(tmem_slot))),
                   "r"(kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tacc = *tmem_slot + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
           static_cast<uint32_t>(CPW * (warp >> 2));
  } else {
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // this warp's column offsets of panel p (CPW + 1 values over OFFR
  // registers); the next unit's are loaded while the current one is swept
  int32_t offv[OFFR];
  auto load_offsets = [&](int32_t p, bool valid) {
    const int32_t* offp = off + static_cast<int64_t>(p) * (n + 1) + kw0;
#pragma unroll
    for (int u = 0; u < OFFR; ++u) {
      const int cc = lane + 32 * u;
      // at most nnz (malformed input can push the scanned offsets past it)
      offv[u] = (ncol > 0 && cc <= ncol && valid) ? min(offp[cc], nnz) : 0;
    }
  };
  // TACC: a share meets a run of tiles in every phase, starting at x0 or
  // x0 + 1, so the slots holding sums of earlier phases are those of the
  // tiles xlo .. xhi
  int xlo = 0x7fffffff, xhi = -1;
  // the sums of tile x over this phase's units: register sums to their row
  // group's copy (or A_hat); tensor-memory sums added into the tile's slot,
  // or, for a tile this CTA owns, into A_hat after the last phase
  auto flush = [&](int x, bool last_phase) {
    const int rows_valid = min(32, d - x * 32);
    const int k = x - x0;
    const bool has = TACC && xlo <= x && x <= xhi;
    const bool to_out = !TACC || (last_phase && tile_whole(x, c, tiles, C));
    float* o_base = out + (TACC ? 0 : static_cast<int64_t>(blockIdx.z) * n * d) + x * 32;
    float* s_base = TACC ? slots + (static_cast<int64_t>(c) * kslots + k) * n * 32 : nullptr;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int col = kw0 + 4 * q + cg;
      if (4 * q < ncol) {  // warp-uniform
        float4 r;
        if constexpr (TACC) {
          uint32_t t[4];
          tmem_ld4(tacc + 4 * q, t);
          tmem_wait_ld4(t);
          r = make_float4(__uint_as_float(t[0]), __uint_as_float(t[1]), __uint_as_float(t[2]),
                          __uint_as_float(t[3]));
        } else {
          r = acc[q];
        }
        if (col < n) {
          float4* sp = TACC ? reinterpret_cast<float4*>(s_base + static_cast<int64_t>(col) * 32 +
                                                       4 * i4)
                            : nullptr;
          if (has) {  // earlier phases first: the row groups' order
            const float4 e = *sp;
            r = make_float4(e.x + r.x, e.y + r.y, e.z + r.z, e.w + r.w);
          }
          if (to_out) {
            float* o = o_base + static_cast<int64_t>(col) * d + 4 * i4;
            if (4 * i4 + 0 < rows_valid) o[0] = r.x;
            if (4 * i4 + 1 < rows_valid) o[1] = r.y;
            if (4 * i4 + 2 < rows_valid) o[2] = r.z;
            if (4 * i4 + 3 < rows_valid) o[3] = r.w;
          } else {
            *sp = r;
          }
        }
      }
    }
  };
  // TACC: a tile's sums start at zero in every phase
  auto zero_sums = [&]() {
    if constexpr (TACC) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) tmem_st4(tacc + 4 * q, make_float4(0.f, 0.f, 0.f, 0.f));
      tmem_wait_st();
    }
  };
  int64_t gen_rows = 0;  // S entries generated (thread 0's count)
  const int nphase = TACC ? G : 1;
  for (int ph = 0; ph < nphase; ++ph) {
    // the phase's panels [pa, pa + Pp) and this CTA's units [s0, s1) of them
    const int32_t g = TACC ? ph : static_cast<int32_t>(blockIdx.z);
    const int32_t pa = static_cast<int32_t>(static_cast<int64_t>(P) * g / G);
    const int32_t Pp = static_cast<int32_t>(static_cast<int64_t>(P) * (g + 1) / G) - pa;
    int32_t s0 = 0, s1 = Pp;
    if constexpr (TACC) {
      // the rounding offset turns with the phase, so the shares one unit
      // larger than the others are not always the same CTAs'
      const int64_t T = static_cast<int64_t>(tiles) * Pp;
      const int64_t rho = static_cast<int64_t>(ph) * C / G;
      s0 = static_cast<int32_t>((T * c + rho) / C);
      s1 = static_cast<int32_t>((T * (c + 1) + rho) / C);
    }
    if (s0 >= s1) continue;
    load_offsets(pa + (TACC ? s0 % Pp : s0), true);
    int xcur = TACC ? -1 : static_cast<int>(blockIdx.x);
    for (int32_t u = s0; u < s1; ++u) {
      const int x = TACC ? u / Pp : static_cast<int>(blockIdx.x);  // the row tile of S
      const int32_t p = pa + (TACC ? u - x * Pp : u);                // the panel of A
      if constexpr (TACC) {
        if (x != xcur) {
          if (xcur >= 0) flush(xcur, ph == nphase - 1);
          zero_sums();
          xcur = x;
        }
      }
      const int rows_valid = min(32, d - x * 32);
      const int32_t j0 = p * R;
      const int32_t rows = min(R, m - j0);
      if constexpr (TACC) gen_rows += static_cast<int64_t>(rows) * rows_valid;
      // ---- this warp's nonzeros (one contiguous range) copied global ->
      //      shared asynchronously; the copies land while the S tile is
      //      generated
      int32_t e_lo = 0;
      if (ncol > 0) {
        e_lo = __shfl_sync(0xffffffffu, offv[0], 0);
        int32_t o_end = offv[0];  // offv[ncol >> 5] without a dynamic index
#pragma unroll
        for (int v = 1; v < OFFR; ++v)
          if ((ncol >> 5) == v) o_end = offv[v];
        const int32_t e_hi = __shfl_sync(0xffffffffu, o_end, ncol & 31);
        const int32_t cnt = min(e_hi - e_lo, wbuf);
        for (int32_t t = lane; t < cnt; t += 32) {
          const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(ent + t));
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst),
                       "l"(packed + e_lo + t)
                       : "memory");
        }
#pragma unroll
        for (int v = 0; v < OFFR; ++v) {
          const int c = lane + 32 * v;
          if (c <= ncol) offs[c] = offv[v];
        }
      }
      // ---- S(tile, j0 .. j0 + rows) once into shared memory ---------------
      for (int idx = threadIdx.x; idx < rows * 8; idx += kWarps * 32) {
        const int jl = idx >> 3, q = idx & 7;
        const uint32_t j = static_cast<uint32_t>(j0 + jl);
        if constexpr (DIST == kFromMemory) {
          // S read from memory: 16 bytes (rows 4q .. 4q+3 of the tile) by
          // cp.async; rows past d are zero-filled (src-size below 16)
          const int valid = min(4, max(0, rows_valid - 4 * q));
          const float* src = valid > 0 ? S_mem + static_cast<int64_t>(j) * ld_s + x * 32 + 4 * q
                                       : S_mem;
          const unsigned dst =
              static_cast<unsigned>(__cvta_generic_to_shared(&S_tile[jl * 32 + 4 * q]));
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                       "r"(4 * valid)
                       : "memory");
        } else {
          float4 v;
          if constexpr (DIST == kPM1) {
            const uint4 xb = philox_block(static_cast<uint32_t>(x >> 2), j, stream_id, keys);
            const int wsel = x & 3;
            const uint32_t w =
                (wsel == 0 ? xb.x : wsel == 1 ? xb.y : wsel == 2 ? xb.z : xb.w) >> (4 * q);
            v = make_float4((w & 1u) ? -1.f : 1.f, (w & 2u) ? -1.f : 1.f,
                            (w & 4u) ? -1.f : 1.f, (w & 8u) ? -1.f : 1.f);
          } else {
            v = four_entries<DIST>(
                philox_block(static_cast<uint32_t>(x * 8 + q), j, stream_id, keys));
          }
          *reinterpret_cast<float4*>(&S_tile[jl * 32 + 4 * q]) = v;
        }
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      // used by the next unit; lands during the sweep
      load_offsets(pa + (TACC ? (u + 1) % Pp : u + 1), u + 1 < s1);
      // ---- sweep: four columns per step, one per group of eight lanes ------
      const int32_t buf_end = e_lo + wbuf;
      // register sums need the quad index at compile time; tensor-memory sums
      // do not, and a rolled loop keeps them within 64 registers
      constexpr int kQuadUnroll = TACC ? 1 : NQ;
#pragma unroll kQuadUnroll
      for (int q = 0; q < NQ; ++q) {
        if (4 * q < ncol) {  // warp-uniform
          const int c = 4 * q + cg;  // this lane's column slot (differs by group)
          const int32_t lo = offs[c], hi = offs[c + 1];
          const int32_t cnt = c < ncol ? hi - lo : 0;
          const int32_t steps = __reduce_max_sync(0xffffffffu, cnt);
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (__all_sync(0xffffffffu, c >= ncol || hi <= buf_end)) {
            // fast path: every entry is staged; lanes past their column's end
            // read the zero entry at ent[wbuf] (no branch per step).
            // Two steps per iteration with separate accumulators: both
            // entries, then both S loads, then the FMAs (more loads in flight)
            const int2* ep = ent + (lo - e_lo);
            const int2* zero = ent + wbuf;
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            int32_t t = 0;
            for (; t + 1 < steps; t += 2) {
              const int2 ja = *(t < cnt ? ep + t : zero);
              const int2 jb = *(t + 1 < cnt ? ep + t + 1 : zero);
              const float4 sa = *reinterpret_cast<const float4*>(S_lane + ja.x);
              const float4 sb = *reinterpret_cast<const float4*>(S_lane + jb.x);
              const float a = __int_as_float(ja.y), b = __int_as_float(jb.y);
              v.x = fmaf(a, sa.x, v.x);
              v.y = fmaf(a, sa.y, v.y);
              v.z = fmaf(a, sa.z, v.z);
              v.w = fmaf(a, sa.w, v.w);
              w.x = fmaf(b, sb.x, w.x);
              w.y = fmaf(b, sb.y, w.y);
              w.z = fmaf(b, sb.z, w.z);
              w.w = fmaf(b, sb.w, w.w);
            }
            if (t < steps) {
              const int2 ja = *(t < cnt ? ep + t : zero);
              const float4 sa = *reinterpret_cast<const float4*>(S_lane + ja.x);
              const float a = __int_as_float(ja.y);
              v.x = fmaf(a, sa.x, v.x);
              v.y = fmaf(a, sa.y, v.y);
              v.z = fmaf(a, sa.z, v.z);
              v.w = fmaf(a, sa.w, v.w);
            }
            v.x += w.x;
            v.y += w.y;
            v.z += w.z;
            v.w += w.w;
          } else {
            // entries read from global memory; the same split of the sum
            // (even steps into v, odd steps into w) as the fast path, so the
            // bits do not depend on how much of the panel was staged
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int32_t t = 0; t < steps; t += 2) {
              if (t < cnt) {
                const int2 ja = packed[lo + t];
                const float a = __int_as_float(ja.y);
                const float4 sv = *reinterpret_cast<const float4*>(S_lane + ja.x);
                v.x = fmaf(a, sv.x, v.x);
                v.y = fmaf(a, sv.y, v.y);
                v.z = fmaf(a, sv.z, v.z);
                v.w = fmaf(a, sv.w, v.w);
              }
              if (t + 1 < cnt) {
                const int2 jb = packed[lo + t + 1];
                const float b = __int_as_float(jb.y);
                const float4 sv = *reinterpret_cast<const float4*>(S_lane + jb.x);
                w.x = fmaf(b, sv.x, w.x);
                w.y = fmaf(b, sv.y, w.y);
                w.z = fmaf(b, sv.z, w.z);
                w.w = fmaf(b, sv.w, w.w);
              }
            }
            v.x += w.x;
            v.y += w.y;
            v.z += w.z;
            v.w += w.w;
          }
          if constexpr (TACC) {
            uint32_t prev[4];  // the quad's running sums
            tmem_ld4(tacc + 4 * q, prev);
            tmem_wait_ld4(prev);
            tmem_st4(tacc + 4 * q,
                     make_float4(__uint_as_float(prev[0]) + v.x, __uint_as_float(prev[1]) + v.y,
                                 __uint_as_float(prev[2]) + v.z, __uint_as_float(prev[3]) + v.w));
          } else {
            acc[q].x += v.x;
            acc[q].y += v.y;
            acc[q].z += v.z;
            acc[q].w += v.w;
          }
        }
      }
      // TACC: this panel's stores complete before the next panel reads them
      if constexpr (TACC) tmem_wait_st();
      __syncthreads();
    }
    flush(xcur, ph == nphase - 1);
    xlo = min(xlo, TACC ? s0 / Pp : xcur);
    xhi = max(xhi, xcur);
    if constexpr (!TACC)  // one tile: the rows of panels [pa, pa + Pp)
      gen_rows = (min(static_cast<int64_t>(pa + Pp) * R, static_cast<int64_t>(m)) -
                  static_cast<int64_t>(pa) * R) *
                 min(32, d - static_cast<int>(blockIdx.x) * 32);
  }
  if constexpr (TACC) {
    // the slots k_reduce_segments adds: tiles met but not owned
    if (blockIdx.y == 0)
      for (int k = threadIdx.x; k < kslots; k += blockDim.x)
        sflags[static_cast<int64_t>(c) * kslots + k] =
            (xlo <= x0 + k && x0 + k <= xhi && !tile_whole(x0 + k, c, tiles, C)) ? 1 : 0;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tmem_slot),
                   "r"(kTmemCols)
                   : "memory");
  }
  if (gen_count && threadIdx.x == 0 && gen_rows > 0)
    atomicAdd(gen_count, static_cast<unsigned long long>(gen_rows));
}

// Tensor-memory TILE: the tiles of A_hat that several CTAs met, as the sum
// of their slots in CTA order (C CTAs; share c starts in tile
// c * tiles / C, its slot k holds tile c * tiles / C + k and is flagged in
// sflags when it is to be added).  Block (tile x, 128-column chunk); warp w,
// lane = row of the tile.  A tile one CTA owns was written by that CTA.
__global__ void __launch_bounds__(256)
    k_reduce_segments(int32_t n, int32_t d, int32_t C, int32_t kslots,
                      const int32_t* __restrict__ sflags, const float* __restrict__ slots,
                      float* __restrict__ Ahat) {
  const int64_t tiles = (d + 31) / 32, x = blockIdx.x;
  const int64_t cw = x * C / tiles;
  if (tile_whole(x, cw, tiles, C)) return;
  // the CTAs whose shares can meet tile x
  const int64_t c_lo = max(int64_t(0), cw - 1);
  const int64_t c_hi = min(int64_t(C) - 1, ((x + 1) * C + tiles - 1) / tiles);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t row = x * 32 + lane;
  if (row >= d) return;
  const int col_end = min(n, static_cast<int>(blockIdx.y + 1) * 128);
  for (int col = blockIdx.y * 128 + warp; col < col_end; col += 8) {
    float acc_s = 0.f;
    bool first = true;
    for (int64_t c = c_lo; c <= c_hi; ++c) {
      const int64_t k = x - c * tiles / C;
      if (k < 0 || k >= kslots || !sflags[c * kslots + k]) continue;
      const float v = slots[((c * kslots + k) * n + col) * 32 + lane];
      acc_s = first ? v : acc_s + v;
      first = false;
    }
    Ahat[static_cast<int64_t>(col) * d + row] = acc_s;
  }
}

// Slots per CTA of the tensor-memory TILE (C CTAs per column block): the
// tiles one share can meet.
int32_t tile_kslots(int32_t d, int32_t C) {
  const int32_t tiles = (d + 31) / 32;
  return (tiles + C - 1) / C + 1;
}

// CTAs per column block of the tensor-memory TILE: one wave on the GPU.
int32_t tile_ctas(int32_t n) {
  const int32_t cblocks = (n + 1023) / 1024;
  return std::max(1, num_sms() / std::max(1, cblocks));
}

size_t tile_workspace_bytes(int64_t m, int64_t n, int64_t d, int64_t nnz,
                            int32_t R, int32_t G, int32_t tacc) {
  const int64_t P = (m + R - 1) / R;
  const int64_t cells = P * (n + 1) + 1;
  size_t b = align256(nnz * sizeof(int2)) + align256((P + 1) * n * sizeof(int32_t)) +
             2 * align256(cells * sizeof(int32_t)) +
             align256(static_cast<size_t>(scan_levels_bytes(cells)));
  if (tacc) {  // the CTAs' slots and their flags
    const int32_t C = tile_ctas(static_cast<int32_t>(n));
    const size_t nslots = static_cast<size_t>(C) * tile_kslots(static_cast<int32_t>(d), C);
    b += align256(nslots * n * 32 * sizeof(float)) + align256(nslots * sizeof(int32_t));
  } else if (G > 1) {
    b += align256(static_cast<size_t>(G) * n * d * sizeof(float));
  }
  return b;
}

size_t tile_smem_bytes(int32_t R, int32_t tacc) {
  return static_cast<size_t>(R) * 32 * sizeof(float) +
         tile_warps(tacc != 0) * (tile_warp_buf(tacc != 0) + 1) * sizeof(int2) +
         tile_warps(tacc != 0) * ((tacc ? 32 : 64) + 4) * sizeof(int32_t) +  // offsets
         16;                                         // tensor-memory base address
}

cudaError_t launch_tile(const TileArgs& a, void* ws, cudaStream_t s, int* launches) {
  if (a.R < 8 || a.G < 1 || a.cpw < 1) return cudaErrorInvalidValue;
  const int64_t P = (static_cast<int64_t>(a.m) + a.R - 1) / a.R;
  const int64_t cells = P * (a.n + 1) + 1;
  char* p = static_cast<char*>(ws);
  int2* packed = reinterpret_cast<int2*>(p);
  p += align256(a.nnz * sizeof(int2));
  int32_t* pp = reinterpret_cast<int32_t*>(p);
  p += align256((P + 1) * a.n * sizeof(int32_t));
  int32_t* cnt = reinterpret_cast<int32_t*>(p);
  p += align256(cells * sizeof(int32_t));
  int32_t* off = reinterpret_cast<int32_t*>(p);
  p += align256(cells * sizeof(int32_t));
  char* scan_tmp = p;
  p += align256(static_cast<size_t>(scan_levels_bytes(cells)));
  float* partial = reinterpret_cast<float*>(p);  // row groups' copies, or the CTAs' slots
  const int32_t C = a.tacc ? tile_ctas(a.n) : 1;  // tensor-memory sums: CTAs per column block
  const int32_t kslots = a.tacc ? tile_kslots(a.d, C) : 0;
  int32_t* sflags = reinterpret_cast<int32_t*>(
      p + (a.tacc ? align256(static_cast<size_t>(C) * kslots * a.n * 32 * sizeof(float)) : 0));
  const int sms = num_sms();
  cudaError_t e;
  if (!a.prepared) {  // the panel-major copy of A, its panel pointers and offsets
    auto grid_for = [&](int64_t work) {
      return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 32LL * sms)));
    };
    k_panel_pointers<<<grid_for((P + 1) * a.n), 256, 0, s>>>(
        a.n, static_cast<int32_t>(P), a.R, a.nnz, a.colptr, a.rowidx, pp, a.status);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_panel_counts<<<grid_for(cells), 256, 0, s>>>(a.n, static_cast<int32_t>(P), pp, cnt);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan(cnt, off, cells, scan_tmp, s, launches)) != cudaSuccess) return e;
    if (a.dtype == 0)
      k_panel_copy<float><<<grid_for(P * a.n), 256, 0, s>>>(
          a.n, static_cast<int32_t>(P), a.R, a.m, a.nnz, a.rowidx,
          static_cast<const float*>(a.values), pp, off, packed, a.status);
    else
      k_panel_copy<__nv_bfloat16><<<grid_for(P * a.n), 256, 0, s>>>(
          a.n, static_cast<int32_t>(P), a.R, a.m, a.nnz, a.rowidx,
          static_cast<const __nv_bfloat16*>(a.values), pp, off, packed, a.status);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int cols_per_cta = tile_warps(a.tacc != 0) * a.cpw;
  const int tiles = (a.d + 31) / 32;
  const int cblocks = (a.n + cols_per_cta - 1) / cols_per_cta;
  if (cblocks > 65535 || a.G > 65535) return cudaErrorInvalidValue;
  if (static_cast<int64_t>(tiles) * P >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
  // tensor-memory sums: C CTAs per column block walking G phases; register
  // sums: G row groups of each row tile
  const dim3 grid = a.tacc ? dim3(C, cblocks, 1) : dim3(tiles, cblocks, a.G);
  const dim3 block(tile_warps(a.tacc != 0) * 32);
  const size_t smem = tile_smem_bytes(a.R, a.tacc);
  const PhiloxKeys keys = philox_keys(a.k0, a.k1);
  float* dst = (a.tacc || a.G == 1) ? a.Ahat : partial;
  if (a.tacc && a.cpw != 32) return cudaErrorInvalidValue;
  if (a.dist == kFromMemory &&
      (!a.tacc || !a.S_mem || a.ld_s < a.d || a.ld_s % 4 != 0 ||
       reinterpret_cast<uintptr_t>(a.S_mem) % 16 != 0))
    return cudaErrorInvalidValue;
#define SK_TILE_CASE(DD, CC, TT)                                                 \
  if (a.dist == DD && a.cpw == CC && (a.tacc != 0) == TT) {                      \
    e = raise_smem_limit(reinterpret_cast<const void*>(k_tile<DD, CC, TT>), smem); \
    if (e != cudaSuccess) return e;                                              \
    k_tile<DD, CC, TT><<<grid, block, smem, s>>>(a.m, a.n, a.d, a.R,             \
                                                 static_cast<int32_t>(P), a.G,   \
                                                 packed, off,                    \
                                                 static_cast<int32_t>(a.nnz), dst, \
                                                 partial, kslots, sflags, keys,  \
                                                 a.stream_id, a.gen_count,       \
                                                 a.S_mem, a.ld_s);               \
    ++*launches;                                                                 \
    launched = true;                                                             \
  }
  bool launched = false;
  SK_TILE_CASE(kPM1, 4, false) SK_TILE_CASE(kPM1, 16, false) SK_TILE_CASE(kPM1, 64, false)
  SK_TILE_CASE(kUniform, 4, false) SK_TILE_CASE(kUniform, 16, false)
  SK_TILE_CASE(kUniform, 64, false)
  SK_TILE_CASE(kNormal, 4, false) SK_TILE_CASE(kNormal, 16, false)
  SK_TILE_CASE(kNormal, 64, false)
  SK_TILE_CASE(kPM1, 32, true) SK_TILE_CASE(kUniform, 32, true) SK_TILE_CASE(kNormal, 32, true)
  SK_TILE_CASE(kFromMemory, 32, true)
#undef SK_TILE_CASE
  if (!launched) return cudaErrorInvalidValue;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.tacc) {
    if (C > 1) {  // the tiles that several CTAs met
      const dim3 rgrid(tiles, (a.n + 127) / 128);
      k_reduce_segments<<<rgrid, 256, 0, s>>>(a.n, a.d, C, kslots, sflags, partial, a.Ahat);
      ++*launches;
      e = cudaGetLastError();
    }
  } else if (a.G > 1) {
    const int64_t total = static_cast<int64_t>(a.n) * a.d;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 16LL * sms);
    k_reduce_partials<<<static_cast<unsigned>(blocks), 256, 0, s>>>(total, a.G,
                                                                    partial, a.Ahat);
    ++*launches;
    e = cudaGetLastError();
  }
  return e;
}

// ---------------------------------------------------------------------------
// Validation and test hooks
// ---------------------------------------------------------------------------
__global__ void k_validate(int32_t m, int32_t n, int64_t nnz,
                           const int32_t* __restrict__ colptr,
                           const int32_t* __restrict__ rowidx, int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) +
                   (threadIdx.x >> 5);
       k < n; k += warps) {
    const int32_t p0 = colptr[k], p1 = colptr[k + 1];
    if (k == 0 && p0 != 0 && lane == 0) atomicOr(status, kStatusBadColptr);
    if (k == n - 1 && p1 != nnz && lane == 0) atomicOr(status, kStatusBadColptr);
    if (p1 < p0 || p0 < 0 || p1 > nnz) {
      if (lane == 0) atomicOr(status, kStatusBadColptr);
      continue;
    }
    for (int32_t p = p0 + lane; p < p1; p += 32) {
      const int32_t j = rowidx[p];
      if (static_cast<uint32_t>(j) >= static_cast<uint32_t>(m) ||
          (p > p0 && rowidx[p - 1] >= j))
        atomicOr(status, kStatusBadRow);
    }
  }
}

cudaError_t launch_validate(int32_t m, int32_t n, int64_t nnz,
                            const int32_t* colptr, const int32_t* rowidx,
                            int* status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 7) / 8, 32LL * num_sms());
  k_validate<<<static_cast<unsigned>(blocks), 256, 0, s>>>(m, n, nnz, colptr,
                                                           rowidx, status);
  return cudaGetLastError();
}

// Both forms of the generator (running key, precomputed round keys) on the
// same counters: slots [0, count) and [count, 2 count) of `out`.
__global__ void k_debug_philox(const uint32_t* __restrict__ ctr, uint32_t k0,
                               uint32_t k1, const __grid_constant__ PhiloxKeys keys,
                               uint32_t* __restrict__ out, int64_t count) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       t < count; t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint4 c = make_uint4(ctr[4 * t], ctr[4 * t + 1], ctr[4 * t + 2],
                               ctr[4 * t + 3]);
    const uint4 x = philox4x32_10(c, k0, k1);
    const uint4 y = philox4x32_10(c, keys);
    reinterpret_cast<uint4*>(out)[t] = x;
    reinterpret_cast<uint4*>(out)[count + t] = y;
  }
}

cudaError_t launch_debug_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1,
                                uint32_t* out, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
  k_debug_philox<<<static_cast<unsigned>(blocks), 256, 0, s>>>(
      ctr, k0, k1, philox_keys(k0, k1), out, count);
  return cudaGetLastError();
}

__global__ void k_debug_normal_pair(const uint32_t* __restrict__ words,
                                    float* __restrict__ out, int64_t count) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       t < count; t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float2 z = normal_pair(words[2 * t], words[2 * t + 1]);
    out[2 * t] = z.x;
    out[2 * t + 1] = z.y;
  }
}

cudaError_t launch_debug_normal_pair(const uint32_t* words, float* out, int64_t count,
                                     cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
  k_debug_normal_pair<<<static_cast<unsigned>(blocks), 256, 0, s>>>(words, out, count);
  return cudaGetLastError();
}

// S itself: S_mem[j * ld_s + i] = S(i, j) for i < d, j < m, the entries the
// sketch kernels regenerate.  One item = four rows of a column: one
// generator block (U, N: its four entries; +-1: four of its 128 signs).
template <int DIST>
__global__ void k_generate_S(const __grid_constant__ PhiloxKeys keys, uint32_t stream_id,
                             int32_t d, int32_t m, float* __restrict__ S_mem, int64_t ld_s) {
  const int32_t g4 = (d + 3) / 4;
  const int64_t items = static_cast<int64_t>(m) * g4;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < items;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t j = static_cast<uint32_t>(t / g4);
    const int32_t g = static_cast<int32_t>(t % g4);
    float4 v;
    if constexpr (DIST == kPM1) {
      const uint4 x = philox_block(static_cast<uint32_t>(g >> 5), j, stream_id, keys);
      const int b = (4 * g) & 127;  // rows 4g .. 4g+3 are bits b .. b+3 of the block
      const uint32_t w = ((b < 32) ? x.x : (b < 64) ? x.y : (b < 96) ? x.z : x.w) >> (b & 31);
      v = make_float4((w & 1u) ? -1.f : 1.f, (w & 2u) ? -1.f : 1.f, (w & 4u) ? -1.f : 1.f,
                      (w & 8u) ? -1.f : 1.f);
    } else {
      v = four_entries<DIST>(philox_block(static_cast<uint32_t>(g), j, stream_id, keys));
    }
    float* o = S_mem + static_cast<int64_t>(j) * ld_s + 4 * g;
    if (4 * g + 4 <= d) {
      *reinterpret_cast<float4*>(o) = v;  // ld_s % 4 == 0 and S_mem 16-byte aligned
    } else {
      o[0] = v.x;
      if (4 * g + 1 < d) o[1] = v.y;
      if (4 * g + 2 < d) o[2] = v.z;
    }
  }
}

cudaError_t launch_generate_S(int dist, uint32_t k0, uint32_t k1, uint32_t stream_id,
                              int32_t d, int32_t m, float* S_mem, int64_t ld_s,
                              cudaStream_t s) {
  if (d <= 0 || m <= 0) return cudaSuccess;
  if (!S_mem || ld_s < d || ld_s % 4 != 0 || reinterpret_cast<uintptr_t>(S_mem) % 16 != 0)
    return cudaErrorInvalidValue;
  const int64_t items = static_cast<int64_t>(m) * ((d + 3) / 4);
  const unsigned blocks =
      static_cast<unsigned>(std::min<int64_t>((items + 255) / 256, 32LL * num_sms()));
  const PhiloxKeys keys = philox_keys(k0, k1);
  switch (dist) {
    case kPM1:
      k_generate_S<kPM1><<<blocks, 256, 0, s>>>(keys, stream_id, d, m, S_mem, ld_s);
      break;
    case kUniform:
      k_generate_S<kUniform><<<blocks, 256, 0, s>>>(keys, stream_id, d, m, S_mem, ld_s);
      break;
    case kNormal:
      k_generate_S<kNormal><<<blocks, 256, 0, s>>>(keys, stream_id, d, m, S_mem, ld_s);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

__global__ void k_debug_S(int dist, uint32_t k0, uint32_t k1,
                          uint32_t stream_id, const int64_t* __restrict__ ii,
                          const int64_t* __restrict__ jj,
                          float* __restrict__ out, int64_t count) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       t < count; t += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[t] = S_entry(dist, k0, k1, stream_id, ii[t], jj[t]);
}

cudaError_t launch_debug_S(int dist, uint32_t k0, uint32_t k1,
                           uint32_t stream_id, const int64_t* i,
                           const int64_t* j, float* out, int64_t count,
                           cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
  k_debug_S<<<static_cast<unsigned>(blocks), 256, 0, s>>>(dist, k0, k1,
                                                          stream_id, i, j, out,
                                                          count);
  return cudaGetLastError();
}

template <int DIST>
__global__ void k_bench_generator(const __grid_constant__ PhiloxKeys keys, int64_t threads,
                                  int64_t blocks_per_thread,
                                  float* __restrict__ sink) {
  const int64_t tid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (tid >= threads) return;
  // every entry is consumed by two three-input xors per block (the
  // cheapest use that still forces each value to be computed), so the rate
  // is the generator's own and not that of an add chain
  // Two independent blocks per iteration (counters b and b + half) give
  // each thread two dependency chains to interleave.
  uint32_t bits = 0;
  const int64_t half = (blocks_per_thread + 1) / 2;
  for (int64_t b = 0; b < half; ++b) {
    const bool second = b + half < blocks_per_thread;
    const uint4 x = philox_block(static_cast<uint32_t>(b), static_cast<uint32_t>(tid), 0u, keys);
    const uint4 y = philox_block(static_cast<uint32_t>(b + half), static_cast<uint32_t>(tid), 0u,
                                 keys);
    if constexpr (DIST == kPM1) {
      bits ^= x.x ^ x.y ^ x.z ^ x.w;
      if (second) bits ^= y.x ^ y.y ^ y.z ^ y.w;
    } else {
      const float4 v = four_entries<DIST>(x);
      const float4 u = four_entries<DIST>(y);
      bits ^= __float_as_uint(v.x) ^ __float_as_uint(v.y) ^ __float_as_uint(v.z) ^
              __float_as_uint(v.w);
      if (second)
        bits ^= __float_as_uint(u.x) ^ __float_as_uint(u.y) ^ __float_as_uint(u.z) ^
                __float_as_uint(u.w);
    }
  }
  sink[tid] = __uint_as_float(bits & 0x007fffffu);
}

cudaError_t launch_bench_generator(int dist, uint32_t k0, uint32_t k1,
                                   int64_t threads, int64_t blocks_per_thread,
                                   float* sink, cudaStream_t s) {
  if (threads <= 0) return cudaSuccess;
  const int64_t blocks = (threads + 255) / 256;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  const PhiloxKeys keys = philox_keys(k0, k1);
  switch (dist) {
    case kPM1:
      k_bench_generator<kPM1><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
          keys, threads, blocks_per_thread, sink);
      break;
    case kUniform:
      k_bench_generator<kUniform><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
          keys, threads, blocks_per_thread, sink);
      break;
    case kNormal:
      k_bench_generator<kNormal><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
          keys, threads, blocks_per_thread, sink);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// FP32 FMA throughput probe: every thread runs eight independent FMA chains
// (x <- x * a + c), so the rate is the FMA pipe's and not a chain's latency.
__global__ void k_bench_fma(int64_t threads, int64_t iters, float a, float* __restrict__ sink) {
  const int64_t tid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (tid >= threads) return;
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = static_cast<float>(tid & 1023) * 1e-3f + static_cast<float>(i);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, 0.5f);
  }
  float t = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) t += x[i];
  sink[tid] = t;
}

cudaError_t launch_bench_fma(int64_t threads, int64_t iters, float* sink, cudaStream_t s) {
  if (threads <= 0) return cudaSuccess;
  const int64_t blocks = (threads + 255) / 256;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_bench_fma<<<static_cast<unsigned>(blocks), 256, 0, s>>>(threads, iters, 0.999f, sink);
  return cudaGetLastError();
}

// Pattern features of A for the plan tuner, from row counts cnt[0..m):
// f[0] = nonempty rows, f[1] = the longest row, f[2] = nonzeros in rows of
// at least 32 entries, f[3] = the longest column (from colptr, clamped).
// ---------------------------------------------------------------------------
// Content hash of A, to recognise a matrix seen before: entry e of array a
// (0 colptr, 1 rowidx, 2 values) with 32-bit word w gives the key
// (e << 32 | w) ^ seed_a, mixed by the splitmix64 finalizer (Steele, Lea,
// Flood, OOPSLA 2014; constants of Vigna's public version), and the mixed
// keys are XOR-reduced, which makes the result independent of the order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void k_content_hash(int32_t n, int64_t nnz, const int32_t* __restrict__ colptr,
                               const int32_t* __restrict__ rowidx,
                               const void* __restrict__ values, int32_t value_bytes,
                               unsigned long long* out) {
  unsigned long long h = 0;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  for (int64_t e = t0; e <= n; e += stride)
    h ^= mix64(((static_cast<unsigned long long>(e) << 32) |
                static_cast<uint32_t>(colptr[e])) ^ 0x243F6A8885A308D3ULL);
  for (int64_t e = t0; e < nnz; e += stride) {
    const uint32_t w = value_bytes == 2
                           ? static_cast<const uint16_t*>(values)[e]
                           : static_cast<const uint32_t*>(values)[e];
    h ^= mix64(((static_cast<unsigned long long>(e) << 32) |
                static_cast<uint32_t>(rowidx[e])) ^ 0x13198A2E03707344ULL);
    h ^= mix64(((static_cast<unsigned long long>(e) << 32) | w) ^ 0xA4093822299F31D0ULL);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h ^= __shfl_xor_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31) == 0 && h) atomicXor(out, h);
}

cudaError_t content_hash(int32_t n, int64_t nnz, const int32_t* colptr,
                         const int32_t* rowidx, const void* values, int32_t value_bytes,
                         unsigned long long* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int64_t work = std::max<int64_t>(nnz, static_cast<int64_t>(n) + 1);
  const unsigned blocks = static_cast<unsigned>(
      std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 8LL * num_sms())));
  k_content_hash<<<blocks, 256, 0, s>>>(n, nnz, colptr, rowidx, values, value_bytes, out);
  return cudaGetLastError();
}

__global__ void k_pattern_features(int32_t m, int32_t n, int64_t nnz,
                                   const int32_t* __restrict__ cnt,
                                   const int32_t* __restrict__ colptr,
                                   unsigned long long* __restrict__ f) {
  unsigned long long ne = 0, heavy = 0, mx = 0, mc = 0;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < m;
       j += stride) {
    const unsigned long long c = static_cast<unsigned long long>(max(cnt[j], 0));
    ne += c > 0;
    heavy += c >= 32 ? c : 0;
    mx = c > mx ? c : mx;
  }
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += stride) {
    const int2 r = column_range(colptr, k, nnz, nullptr);
    const unsigned long long c = static_cast<unsigned long long>(r.y - r.x);
    mc = c > mc ? c : mc;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ne += __shfl_xor_sync(0xffffffffu, ne, o);
    heavy += __shfl_xor_sync(0xffffffffu, heavy, o);
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, mx, o);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, mc, o);
    mx = a > mx ? a : mx;
    mc = b > mc ? b : mc;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&f[0], ne);
    atomicMax(&f[1], mx);
    atomicAdd(&f[2], heavy);
    atomicMax(&f[3], mc);
  }
}

cudaError_t pattern_features(int32_t m, int32_t n, int64_t nnz, const int32_t* colptr,
                             const int32_t* rowidx, int32_t* cnt, unsigned long long* f,
                             int* status, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(cnt, 0, static_cast<size_t>(m) * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(f, 0, 4 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = row_counts(nnz, m, rowidx, cnt, status, s);
  if (e != cudaSuccess) return e;
  const int64_t work = std::max<int64_t>(m, n);
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 8LL * num_sms()));
  k_pattern_features<<<static_cast<unsigned>(blocks), 256, 0, s>>>(m, n, nnz, cnt, colptr, f);
  return cudaGetLastError();
}

int64_t scan_bytes_for(int64_t len) { return scan_levels_bytes(len); }

cudaError_t scan_i32(const int32_t* in, int32_t* out, int64_t len, char* tmp,
                     cudaStream_t s, int* launches) {
  return exclusive_scan(in, out, len, tmp, s, launches);
}

cudaError_t row_counts(int64_t nnz, int32_t m, const int32_t* rowidx, int32_t* cnt,
                       int* status, cudaStream_t s) {
  if (nnz <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((nnz + 255) / 256, 32LL * num_sms());
  k_row_count<<<static_cast<unsigned>(blocks), 256, 0, s>>>(nnz, m, rowidx, cnt, status);
  return cudaGetLastError();
}

int num_sms() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached = v > 0 ? v : 1;
  }
  return cached;
}

cudaError_t raise_smem_limit(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> limit;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[kernel];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(bytes));
  if (e == cudaSuccess) cur = bytes;
  return e;
}

}  // namespace sk
