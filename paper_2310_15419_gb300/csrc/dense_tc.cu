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
//     in tensor memory, in one persistent kernel (k_tc_panel);
//   * optionally FP8: E4M3 +-1 S against two E4M3 terms of A, each column
//     first scaled by a power of two (undone exactly on the output).
// The sparse kernels run on the rest of A (a compacted CSC without the
// panel's rows), so A_hat = S A_rest + S_D A_D with the MMA adding into A_hat
// afterwards.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace sk {

namespace {

constexpr int kBK = 32;    // contraction step (dense rows per step)

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

// Column of entry e of a CSC: the k with colptr[k] <= e < colptr[k + 1]
// (binary search; entries outside every column range give -1).
__device__ __forceinline__ int32_t column_of(const int32_t* __restrict__ colptr, int32_t n,
                                             int64_t e) {
  int32_t lo = 0, hi = n;  // colptr[lo] <= e < colptr[hi] if e is in range
  if (e < colptr[0] || e >= colptr[n]) return -1;
  while (hi - lo > 1) {
    const int32_t mid = lo + ((hi - lo) >> 1);
    if (colptr[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

// The t-th BF16 term of A(j, k) for dense rows j (q = didx[j]), one thread
// per entry (its column by binary search), so the build runs at memory speed
// however long the columns are.  Layout of A3, for column tiles of
// 2^lg columns (128, or 256 for short panels): each step's three B tiles
// contiguous in the operand layout the MMA reads -- tile k >> lg, step
// q >> 5, term t, k-chunk (q >> 3) & 3, column k within the tile, 8
// consecutive q -- one bulk copy per step.
__device__ __forceinline__ int64_t a3_offset(int32_t k, int32_t q, int t, int64_t Kp, int lg) {
  const int64_t steps = Kp >> 5;
  const int64_t tile_step = (static_cast<int64_t>(k >> lg) * steps + (q >> 5)) * 3 + t;
  return ((tile_step * 4 + ((q >> 3) & 3)) * (int64_t(1) << lg) + (k & ((1 << lg) - 1))) * 8 +
         (q & 7);
}

// FP8 panels: colinv[k] = 2^(x - 8) for the largest |A(j, k)| over the
// panel's rows, f 2^x with f in [0.5, 1) (so A(j, k) / colinv[k] <= 256 <
// 448, the E4M3 maximum); 1 for a column without panel entries.  cmax holds
// the bits of the largest magnitude (non-negative floats order as integers).
template <typename VT>
__global__ void k_panel_colmax(int32_t n, int32_t m, int64_t nnz,
                               const int32_t* __restrict__ colptr,
                               const int32_t* __restrict__ rowidx, const VT* __restrict__ vals,
                               const int32_t* __restrict__ didx, uint32_t* __restrict__ cmax) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t j = rowidx[e];
    if (static_cast<uint32_t>(j) >= static_cast<uint32_t>(m) || didx[j] < 0) continue;
    const int32_t k = column_of(colptr, n, e);
    if (k < 0) continue;
    atomicMax(&cmax[k], __float_as_uint(fabsf(to_f32(vals[e]))));
  }
}

__global__ void k_panel_colscale(int32_t n, const uint32_t* __restrict__ cmax,
                                 float* __restrict__ colinv) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float mx = __uint_as_float(cmax[k]);
    int x = 0;
    frexpf(mx, &x);
    colinv[k] = mx > 0.0f ? ldexpf(1.0f, x - 8) : 1.0f;
  }
}

// The FP8 panel in the same tiled layout: for tile k >> lg and step q >> 5
// a block of two terms x two 16-byte k-chunks x 2^lg columns; term t of
// A(j, k) / colinv[k] (E4M3, round to nearest): t = 0 the value, t = 1 its
// remainder.
__device__ __forceinline__ int64_t a3_offset_fp8(int32_t k, int32_t q, int t, int64_t Kp,
                                                 int lg) {
  const int64_t steps = Kp >> 5;
  const int64_t tile_step = (static_cast<int64_t>(k >> lg) * steps + (q >> 5)) * 2 + t;
  return ((tile_step * 2 + ((q >> 4) & 1)) * (int64_t(1) << lg) + (k & ((1 << lg) - 1))) * 16 +
         (q & 15);
}

template <typename VT>
__global__ void k_dense_scatter_fp8(int32_t n, int32_t m, int32_t Kp, int lg, int64_t nnz,
                                    const int32_t* __restrict__ colptr,
                                    const int32_t* __restrict__ rowidx,
                                    const VT* __restrict__ vals,
                                    const int32_t* __restrict__ didx,
                                    const float* __restrict__ colinv,
                                    uint8_t* __restrict__ A8) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t j = rowidx[e];
    if (static_cast<uint32_t>(j) >= static_cast<uint32_t>(m)) continue;
    const int32_t q = didx[j];
    if (q < 0) continue;
    const int32_t k = column_of(colptr, n, e);
    if (k < 0) continue;
    const float a = to_f32(vals[e]) / colinv[k];  // exact: a power of two
    const __nv_fp8_e4m3 t1(a);
    const __nv_fp8_e4m3 t2(a - static_cast<float>(t1));
    A8[a3_offset_fp8(k, q, 0, Kp, lg)] = t1.__x;
    A8[a3_offset_fp8(k, q, 1, Kp, lg)] = t2.__x;
  }
}

template <typename VT>
__global__ void k_dense_scatter(int32_t n, int32_t m, int32_t Kp, int lg, int64_t nnz,
                                const int32_t* __restrict__ colptr,
                                const int32_t* __restrict__ rowidx,
                                const VT* __restrict__ vals,
                                const int32_t* __restrict__ didx,
                                uint16_t* __restrict__ A3) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t j = rowidx[e];
    if (static_cast<uint32_t>(j) >= static_cast<uint32_t>(m)) continue;
    const int32_t q = didx[j];
    if (q < 0) continue;
    const int32_t k = column_of(colptr, n, e);
    if (k < 0) continue;
    const float a = to_f32(vals[e]);
    const float a1 = __bfloat162float(__float2bfloat16_rn(a));
    const float r1 = a - a1;  // exact
    const float a2 = __bfloat162float(__float2bfloat16_rn(r1));
    const float a3 = r1 - a2;  // exact, fits BF16
    A3[a3_offset(k, q, 0, Kp, lg)] = bf16_bits(a1);
    A3[a3_offset(k, q, 1, Kp, lg)] = bf16_bits(a2);
    A3[a3_offset(k, q, 2, Kp, lg)] = bf16_bits(a3);
  }
}


__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Wait for the phase of parity `parity` of an mbarrier; false once
// `limit_ns` nanoseconds (by the global timer) have passed.  Each poll lets
// the hardware suspend the thread until the phase completes or a few
// microseconds pass, so waiting warps take few issue slots from the
// working ones.
constexpr uint32_t kSuspendNs = 10000;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          uint64_t limit_ns = kWaitLimitNs) {
  uint64_t t0 = 0;
  for (bool first = true;; first = false) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(kSuspendNs)
        : "memory");
    if (ok) return true;
    const uint64_t t = global_ns();
    if (first)
      t0 = t;
    else if (t - t0 > limit_ns)
      return false;
  }
}

// ---------------------------------------------------------------------------
// k_tc_panel: the same product, persistent, warp specialised and pipelined.
// One CTA per SM walks a list of units, a unit being a 128 x 128 tile of
// A_hat (rows of S x columns of A) and one of `splits` slices of the dense
// rows (split-K; the slices' partial tiles are added in a fixed order
// afterwards).  Steps of 32 dense rows are counted over the CTA's units.
// Two rings of shared-memory stages: one S tile per builder, and for long
// panels kPanBStages B blocks.  Two ways to feed the B operand (the terms of
// A3):
//   streaming (long panels): each step's B block (all terms, one contiguous
//     block of the tiled A3) is bulk-copied (TMA) into the B ring; CTA b
//     takes units b, b + G, ... (G CTAs), so the CTAs running at once share
//     B blocks in L2;
//   resident (short panels, all steps' B of a column tile within
//     kPanResBytes): a column tile's whole B stays in shared memory while the
//     CTA works through a contiguous run of units with that column tile (the
//     row tiles vary fastest), so A3 is read about once per CTA.
// Roles (512 threads):
//   warp 0 (one thread): the bulk copies;
//   warps 1 and 2 (one thread each): the MMAs, in groups of kPanGroup steps
//     of a unit: thread g takes the groups G with G % 2 == g and owns
//     tensor-memory accumulator g (so each accumulator's MMAs keep one order
//     and the result its bits).  Per step six BF16 MMAs (3 terms x 2 k
//     halves, M = N = 128, K = 16) or two FP8 ones; commits free the stages
//     and, after a group, hand the accumulator to the promoters.  A thread
//     issuing tcgen05.mma runs in step with the tensor pipe, so any wait or
//     commit on one thread would idle the pipe; two threads hide each
//     other's;
//   warps 4-11 (the builders): builder w fills S stage w, for whichever MMA
//     thread takes the step (a full barrier per stage and MMA thread); lane k
//     computes the Philox block of the step's dense row k (the signs of all
//     128 rows of S).  BF16: the tile is
//     MN-major, so lane k writes its own column (16 B per 8 rows, each pair
//     of signs spread into two BF16 +-1 by one multiply).  E4M3: the tile is
//     K-major; four five-stage shuffle transposes give lane L the signs of
//     rows L, 32 + L, 64 + L and 96 + L.  The dense-row id of the builder's
//     next step is loaded a step ahead;
//   warps 12-15 (the promoters): each finished accumulator (kPanGroup steps,
//     up to 24 MMAs: the tensor core's truncating accumulation stays near
//     4e-7 relative) is added with round-to-nearest FP32 additions into
//     running sums in tensor memory and freed; a unit's last one is added in
//     registers and stored to A_hat (or the slice's partial copy).
// Every mbarrier wait has a time limit; on a timeout the CTA records
// kStatusTimeout, drains the MMAs it issued and frees its tensor memory.
// ---------------------------------------------------------------------------
constexpr int kPanBStages = 4;
constexpr int kPanThreads = 512;
constexpr uint32_t kPanLbo = 2048;       // K-direction core-matrix stride
constexpr uint32_t kPanSbo = 128;        // M/N-direction 8-row-group stride
constexpr int kPanTileBytes = 8192;      // one 128 x 32 BF16 operand tile
constexpr int kPanResBytes = 160 * 1024; // resident: all steps' B of a column tile
constexpr uint32_t kPanSums = 256;       // tensor-memory column of the running sums
constexpr int kPanGroup = 4;             // steps accumulated by the tensor core between promotions
// Short panels (at most one group of steps) take 128 x 256 units: the whole
// unit stays in one accumulator, so two 256-column accumulators fill the
// tensor memory with no promotion sums needed, and an N = 256 MMA costs what
// an N = 128 one does.
__host__ __device__ constexpr bool pan_wide(int64_t Kp) { return Kp / kBK <= kPanGroup; }

// The unit grid of one launch.
struct PanelGrid {
  int32_t d, n, steps, sps, tiles_d, tiles_n;
  int64_t units;
  int32_t resident;
};

struct PanUnit {
  int32_t x, y, z, st0, ns;
};

// Unit u (< 2^31, checked on the host) in 32-bit arithmetic: every role
// decodes each of its units, so a 64-bit division would cost more than a
// step of S.
__device__ __forceinline__ PanUnit pan_unit(const PanelGrid& g, int64_t u64) {
  PanUnit t;
  const uint32_t u = static_cast<uint32_t>(u64);
  const uint32_t r = u / static_cast<uint32_t>(g.tiles_d);
  t.x = static_cast<int32_t>(u - r * static_cast<uint32_t>(g.tiles_d));
  const uint32_t z = r / static_cast<uint32_t>(g.tiles_n);
  t.y = static_cast<int32_t>(r - z * static_cast<uint32_t>(g.tiles_n));
  t.z = static_cast<int32_t>(z);
  t.st0 = t.z * g.sps;
  t.ns = max(0, min(g.steps, t.st0 + g.sps) - t.st0);
  return t;
}

// This CTA's units: a contiguous run (resident B) or every G-th one.
__device__ __forceinline__ void pan_range(const PanelGrid& g, int64_t& lo, int64_t& hi,
                                          int64_t& stride) {
  const int64_t G = gridDim.x, b = blockIdx.x;
  if (g.resident) {
    lo = b * g.units / G;
    hi = (b + 1) * g.units / G;
    stride = 1;
  } else {
    lo = b;
    hi = g.units;
    stride = G;
  }
}

// The CTA's steps in order, each with its index s among them (which places
// it in the stage rings: stage s % stages, round s / stages) and its group
// (a unit's steps in groups of kPanGroup; MMA thread g & 1 takes group g).
// Every role walks the same sequence.
struct PanWalk {
  int64_t u, hi, stride;
  PanUnit t;
  int i;  // step within the unit
  int P;  // groups before this unit
  int s;  // steps before this one
  bool valid;
};
__device__ __forceinline__ void walk_settle(const PanelGrid& g, PanWalk& w) {
  while (w.u < w.hi && w.i >= w.t.ns) {
    w.P += (w.t.ns + kPanGroup - 1) / kPanGroup;
    w.u += w.stride;
    w.i = 0;
    if (w.u < w.hi) w.t = pan_unit(g, w.u);
  }
  w.valid = w.u < w.hi;
}
__device__ __forceinline__ void walk_init(const PanelGrid& g, PanWalk& w, int64_t lo,
                                          int64_t hi, int64_t stride) {
  w.u = lo;
  w.hi = hi;
  w.stride = stride;
  w.i = 0;
  w.P = 0;
  w.s = 0;
  w.t = PanUnit{0, 0, 0, 0, 0};
  if (lo < hi) w.t = pan_unit(g, lo);
  walk_settle(g, w);
}
__device__ __forceinline__ int walk_group(const PanWalk& w) { return w.P + w.i / kPanGroup; }
__device__ __forceinline__ int walk_thread(const PanWalk& w) { return walk_group(w) & 1; }
__device__ __forceinline__ void walk_next(const PanelGrid& g, PanWalk& w) {
  ++w.s;
  ++w.i;
  walk_settle(g, w);
}

// Shared-memory matrix descriptor (no swizzle): `lbo` the K-direction stride
// between 8-element core-matrix chunks (the rows of an operand tile times
// 16 B), kPanSbo between 8-row groups.
__device__ __forceinline__ uint64_t pan_desc(uint32_t saddr, uint32_t lbo = kPanLbo) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((kPanSbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
          bar),
      "r"(bytes)
      : "memory");
}
// Bulk copy (TMA, untiled) of `bytes` contiguous bytes into shared memory,
// completing them on the mbarrier (both addresses 16-byte aligned, bytes a
// multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
      "[%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

#define SK_TMEM_X32_REGS(v)                                                              \
  "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),     \
      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),         \
      "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),      \
      "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),      \
      "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),      \
      "=r"(v[31])
#define SK_TMEM_X32_ARGS(v)                                                              \
  "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), \
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),  \
      "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), \
      "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), \
      "r"(v[29]), "r"(v[30]), "r"(v[31])
#define SK_X32_LIST                                                                       \
  "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, " \
  "%19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}"

__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 " SK_X32_LIST ", [%32];"
               : SK_TMEM_X32_REGS(v)
               : "r"(taddr));
}
// Wait for the loads in flight; the registers are operands so no use of
// them is scheduled before the data has landed.
__device__ __forceinline__ void tmem_wait_ld32(uint32_t (&a)[32], uint32_t (&b)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]),
                 "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]),
                 "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]), "+r"(a[16]), "+r"(a[17]),
                 "+r"(a[18]), "+r"(a[19]), "+r"(a[20]), "+r"(a[21]), "+r"(a[22]), "+r"(a[23]),
                 "+r"(a[24]), "+r"(a[25]), "+r"(a[26]), "+r"(a[27]), "+r"(a[28]), "+r"(a[29]),
                 "+r"(a[30]), "+r"(a[31])
               :
               : "memory");
  asm volatile(""
               : "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]),
                 "+r"(b[6]), "+r"(b[7]), "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]),
                 "+r"(b[12]), "+r"(b[13]), "+r"(b[14]), "+r"(b[15]), "+r"(b[16]), "+r"(b[17]),
                 "+r"(b[18]), "+r"(b[19]), "+r"(b[20]), "+r"(b[21]), "+r"(b[22]), "+r"(b[23]),
                 "+r"(b[24]), "+r"(b[25]), "+r"(b[26]), "+r"(b[27]), "+r"(b[28]), "+r"(b[29]),
                 "+r"(b[30]), "+r"(b[31])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
               "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, "
               "%18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(
                   taddr),
               SK_TMEM_X32_ARGS(v)
               : "memory");
}

// FP8 = true: E4M3 operands (kind::f8f6f4, K = 32 per MMA): the S tile is
// 128 rows x 32 bytes, the A panel two terms of 4 KB per step (one 8 KB
// block), two MMAs per step, and the output is multiplied by the column
// scale colinv.  Same layout rules: 16-byte core-matrix rows, k-chunks
// 2048 B apart.
// Instruction descriptor of kind::f8f6f4: F32 accumulator, E4M3 A and B
// (format code 0), both K-major, N = kN, M = 128.
__host__ __device__ constexpr uint32_t idesc_fp8(uint32_t kN) {
  return (1u << 4) | ((kN >> 3) << 17) | ((128u >> 4) << 24);
}
// Instruction descriptor of kind::f16: F32 accumulator, BF16 A and B, A (the
// S tile) MN-major (bit 15), B K-major, N = kN (N >> 3 at bit 17), M = 128
// (M >> 4 at bit 24).  The MN-major no-swizzle S tile: 8 (rows of S) x 8
// (dense rows) core matrices of 8 x 16 B, dense row k's 8 values 16 B, the
// next group of 8 rows of S 128 B on (the SBO field), the next group of 8
// dense rows 2048 B on (the LBO field).
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t kN) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((kN >> 3) << 17) | ((128u >> 4) << 24);
}

// Per mode: columns per unit, S stages (= builder warps), promoter warps.
// Wide units (short panels): 256 columns, 4 builders, 8 promoters (two per
// tensor-memory lane quarter, 128 columns each); else 128, 8 and 4.
__host__ __device__ constexpr int pan_cols(bool wide) { return wide ? 256 : 128; }
__host__ __device__ constexpr int pan_sstages(bool wide) { return wide ? 4 : 8; }
__host__ __device__ constexpr int pan_promoters(bool wide) { return wide ? 8 : 4; }

// Shared memory of one CTA: the S ring, then the B ring (streaming) or one
// column tile's B for every step (resident).
__host__ __device__ constexpr int pan_term_bytes(bool fp8, bool wide) {
  return (fp8 ? 32 : 64) * pan_cols(wide);
}
__host__ __device__ constexpr int pan_step_bytes(bool fp8, bool wide) {
  return (fp8 ? 2 : 3) * pan_term_bytes(fp8, wide);
}
size_t pan_smem_bytes(bool fp8, bool wide, bool resident, int steps) {
  const size_t b = resident ? static_cast<size_t>(steps) * pan_step_bytes(fp8, wide)
                            : static_cast<size_t>(kPanBStages) * pan_step_bytes(fp8, wide);
  return static_cast<size_t>(pan_sstages(wide)) * kPanTileBytes + b + 1024;
}

// +-1 S words from sign bits (bit set = -1): BF16, the two signs in bits 0
// and 1 of t go to bits 15 and 31 over 0x3F80 (+1) halves; E4M3, the four
// signs in bits 0..3 go to bit 7 of each byte over 0x38 (+1) bytes.  The
// multiplies place every other product bit away from the kept ones, so no
// carry reaches them.
__device__ __forceinline__ uint32_t pm1_bf16x2(uint32_t t) {
  return (((t & 3u) * 0x40008000u) & 0x80008000u) | 0x3F803F80u;
}
__device__ __forceinline__ uint32_t pm1_e4m3x4(uint32_t t) {
  return (((t & 15u) * 0x10204080u) & 0x80808080u) | 0x38383838u;
}

template <bool FP8, bool WIDE>
__global__ void __launch_bounds__(kPanThreads, 1)
    k_tc_panel(const PanelGrid g, const int32_t* __restrict__ rows,
               const int32_t* __restrict__ Kdev, const uint8_t* __restrict__ A3,
               const float* __restrict__ colinv, float* __restrict__ out,
               int64_t split_stride, int accumulate, uint32_t k0, uint32_t k1,
               uint32_t stream_id, int* status) {
  constexpr int kN = pan_cols(WIDE);               // columns of A per unit
  constexpr int kSSt = pan_sstages(WIDE);          // S stages = builder warps
  constexpr int kProm = pan_promoters(WIDE);       // promoter warps: the last kProm
  constexpr int kTermBytes = pan_term_bytes(FP8, WIDE);
  constexpr uint32_t kTx = pan_step_bytes(FP8, WIDE);
  constexpr uint32_t kBLbo = 16u * kN;             // B tile: K-direction chunk stride
  constexpr uint32_t kIdesc = FP8 ? idesc_fp8(kN) : idesc_bf16(kN);
  static_assert(4 + kSSt <= 16 - kProm, "builders and promoters overlap");
  extern __shared__ uint8_t sm_raw[];
  // A stage's consumers alternate between the two MMA threads, so each stage
  // has one "full" barrier per MMA thread: the thread is its only waiter and
  // takes its phases in order (one parity bit per stage tracks them), which
  // a single barrier shared by both threads could not guarantee (a thread
  // could wait two phases ahead and take an old phase for the one it needs).
  // The "empty" barriers have one waiter, the filler, which frees rounds in
  // order: a stage's round r + 1 is filled only after round r is released.
  __shared__ __align__(8) uint64_t sfull[kSSt][2], sempty[kSSt],
      bfull[kPanBStages][2], bempty[kPanBStages], acc_full[2], acc_empty[2], rfull, rempty,
      drain_bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int failed;  // set by any role whose bounded wait gave up
  uint8_t* base = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int d = g.d, n = g.n;
  const bool res = g.resident != 0;
  int64_t lo, hi, stride;
  pan_range(g, lo, hi, stride);
  // S stage sg; term t of the B operand of step i of a unit (resident) or of
  // the step in B stage bs (streaming)
  auto tileS = [&](int sg) { return base + sg * kPanTileBytes; };
  uint8_t* const bbase = base + kSSt * kPanTileBytes;
  auto tileB = [&](int bs, int i, int t) {
    return bbase + (res ? i : bs) * kTx + t * kTermBytes;
  };
  if (tid == 0) {
    failed = 0;
    for (int q = 0; q < kSSt; ++q) {
      for (int th = 0; th < 2; ++th) mbar_init(smem_u32(&sfull[q][th]), 1);  // the builder warp
      mbar_init(smem_u32(&sempty[q]), 1);  // the MMA commit
    }
    for (int q = 0; q < kPanBStages; ++q) {
      for (int th = 0; th < 2; ++th)
        mbar_init(smem_u32(&bfull[q][th]), 1);  // the bulk copy with its bytes
      mbar_init(smem_u32(&bempty[q]), 1);  // the MMA commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);   // the MMA commit of a two-step accumulator
      mbar_init(smem_u32(&acc_empty[b]), kProm);  // one arrival per promoting warp
    }
    mbar_init(smem_u32(&rfull), 1);   // resident B: the copies' bytes
    mbar_init(smem_u32(&rempty), 2);  // resident B: both MMA threads' commits after its last use
    for (int b = 0; b < 2; ++b) mbar_init(smem_u32(&drain_bar[b]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {  // bulk copies of the B operand
      if (res) {
        int loads = 0, yprev = -1;
        for (int64_t u = lo; u < hi && !failed; u += stride) {
          const PanUnit t = pan_unit(g, u);
          if (t.y == yprev) continue;
          // the previous column tile's B is overwritten once its MMAs are done
          if (loads > 0 && !mbar_wait(smem_u32(&rempty), (loads - 1) & 1)) {
            failed = 1;
            break;
          }
          mbar_arrive_tx(smem_u32(&rfull), static_cast<uint32_t>(g.steps) * kTx);
          for (int i = 0; i < g.steps; ++i)
            bulk_load(smem_u32(tileB(0, i, 0)),
                      A3 + (static_cast<int64_t>(t.y) * g.steps + i) * kTx, kTx,
                      smem_u32(&rfull));
          ++loads;
          yprev = t.y;
        }
      } else {
        // each step's B block into the B ring, signalled to its MMA thread
        PanWalk w;
        walk_init(g, w, lo, hi, stride);
        for (; w.valid && !failed; walk_next(g, w)) {
          const int bs = w.s % kPanBStages, round = w.s / kPanBStages;
          if (round > 0 && !mbar_wait(smem_u32(&bempty[bs]), (round - 1) & 1)) {
            failed = 1;
            break;
          }
          const uint32_t full = smem_u32(&bfull[bs][walk_thread(w)]);
          mbar_arrive_tx(full, kTx);
          // the step's B tiles (all terms) are one contiguous block of A3
          bulk_load(smem_u32(tileB(bs, 0, 0)),
                    A3 + (static_cast<int64_t>(w.t.y) * g.steps + w.t.st0 + w.i) * kTx, kTx,
                    full);
        }
      }
    }
  } else if (warp == 1 || warp == 2) {
    if (lane == 0) {  // MMA issuers: thread `me` takes the groups G with G % 2 == me
      const int me = warp - 1;
      bool ok = true;
      int loads = 0, yprev = -1;
      uint32_t spar = 0, bpar = 0;  // parity of the next phase of sfull[.][me], bfull[.][me]
      int64_t ucur = -1;
      PanWalk w;
      walk_init(g, w, lo, hi, stride);
      for (; w.valid; walk_next(g, w)) {
        if (w.u != ucur) {  // a new unit
          ucur = w.u;
          if (failed) {
            ok = false;
            break;
          }
          if (res && w.t.y != yprev) {
            // free the previous column tile's B once this thread's MMAs on
            // it finish (both threads commit), then wait for this one's
            if (loads > 0)
              asm volatile(
                  "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
                  "[%0];" ::"r"(smem_u32(&rempty))
                  : "memory");
            if (!mbar_wait(smem_u32(&rfull), loads & 1)) {
              ok = false;
              break;
            }
            ++loads;
            yprev = w.t.y;
          }
        }
        const int Pi = walk_group(w);  // the step's group
        if ((Pi & 1) != me) continue;
        const int i = w.i, sg = w.s % kSSt, bs = w.s % kPanBStages;
        if ((i % kPanGroup == 0 && Pi >= 2 &&
             !mbar_wait(smem_u32(&acc_empty[me]), ((Pi >> 1) - 1) & 1)) ||
            !mbar_wait(smem_u32(&sfull[sg][me]), (spar >> sg) & 1u) ||
            (!res && !mbar_wait(smem_u32(&bfull[bs][me]), (bpar >> bs) & 1u))) {
          ok = false;
          break;
        }
        spar ^= 1u << sg;
        if (!res) bpar ^= 1u << bs;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_addr = tmem + static_cast<uint32_t>(kN * me);
        if constexpr (FP8) {
#pragma unroll
          for (int tt = 0; tt < 2; ++tt) {  // K = 32: the whole step
            const uint64_t ad = pan_desc(smem_u32(tileS(sg)));
            const uint64_t bd = pan_desc(smem_u32(tileB(bs, i, tt)), kBLbo);
            const uint32_t acc = (i % kPanGroup || tt > 0) ? 1u : 0u;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                    acc_addr),
                "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                : "memory");
          }
        } else {
#pragma unroll
          for (int tt = 0; tt < 3; ++tt)
#pragma unroll
            for (int kh = 0; kh < 2; ++kh) {
              const uint64_t ad = pan_desc(smem_u32(tileS(sg)) + kh * 2 * kPanLbo);
              const uint64_t bd = pan_desc(smem_u32(tileB(bs, i, tt)) + kh * 2 * kBLbo, kBLbo);
              const uint32_t acc = (i % kPanGroup || tt > 0 || kh > 0) ? 1u : 0u;
              asm volatile(
                  "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                      acc_addr),
                  "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                  : "memory");
            }
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&sempty[sg]))
            : "memory");
        if (!res)
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
              "[%0];" ::"r"(smem_u32(&bempty[bs]))
              : "memory");
        if (i % kPanGroup == kPanGroup - 1 || i == w.t.ns - 1)
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
              "[%0];" ::"r"(smem_u32(&acc_full[me]))
              : "memory");
      }
      if (!ok) {  // drain the MMAs this thread issued before the memory is freed
        failed = 1;
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&drain_bar[me]))
            : "memory");
        mbar_wait(smem_u32(&drain_bar[me]), 0);
      }
    }
  } else if (warp >= 4 && warp < 4 + kSSt) {  // S-tile builders
    // builder bw fills S stage bw: the steps s with s % kSSt == bw, in order
    const int bw = warp - 4;
    const int K = *Kdev;
    PanWalk w;
    walk_init(g, w, lo, hi, stride);
    auto next_mine = [&]() {
      while (w.valid && w.s % kSSt != bw) walk_next(g, w);
      return w.valid;
    };
    auto row_id = [&]() {  // this lane's dense row of the current step (0 past K)
      const int q = (w.t.st0 + w.i) * kBK + lane;
      return q < K ? rows[q] : 0;  // padding rows multiply zeros
    };
    bool have = next_mine();
    int32_t jn = have ? row_id() : 0;
    while (have) {
      const int round = w.s / kSSt, d0 = w.t.x * 128, th = walk_thread(w);
      const int32_t j = jn;
      walk_next(g, w);
      have = next_mine();        // this builder's next step
      if (have) jn = row_id();   // in flight while this step is built
      int ok = 1;
      if (lane == 0 && round > 0 && !mbar_wait(smem_u32(&sempty[bw]), (round - 1) & 1)) ok = 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) failed = 1;
      if (failed) break;
      // lane k: the Philox block of dense row k, the signs of all 128 rows
      const uint4 x = philox_block(static_cast<uint32_t>(d0 >> 7), static_cast<uint32_t>(j),
                                   stream_id, k0, k1);
      if constexpr (FP8) {
        // K-major E4M3 tile: four shuffle transposes give lane L the signs
        // of rows L, 32 + L, 64 + L, 96 + L over the step's dense rows
#pragma unroll
        for (int wq = 0; wq < 4; ++wq) {
          uint32_t v = wq == 0 ? x.x : wq == 1 ? x.y : wq == 2 ? x.z : x.w;
#pragma unroll
          for (int sh = 16; sh > 0; sh >>= 1) {
            const uint32_t m = sh == 16 ? 0x0000FFFFu : sh == 8 ? 0x00FF00FFu
                             : sh == 4 ? 0x0F0F0F0Fu : sh == 2 ? 0x33333333u : 0x55555555u;
            const uint32_t o = __shfl_xor_sync(0xffffffffu, v, sh);
            v = (lane & sh) ? ((v & ~m) | ((o >> sh) & m)) : ((v & m) | ((o & m) << sh));
          }
          uint8_t* dstS = tileS(bw) + (32 * wq + lane) * 16;
#pragma unroll
          for (int c = 0; c < 2; ++c)  // k-chunk c: dense rows 16c .. 16c + 15
            *reinterpret_cast<uint4*>(dstS + c * kPanLbo) =
                make_uint4(pm1_e4m3x4(v >> (16 * c)), pm1_e4m3x4(v >> (16 * c + 4)),
                           pm1_e4m3x4(v >> (16 * c + 8)), pm1_e4m3x4(v >> (16 * c + 12)));
        }
      } else {
        // MN-major BF16 tile: lane k writes column k (its dense row), 16 B
        // (8 rows of S) per group of 8 rows, straight from its own block
        uint8_t* col = tileS(bw) + (lane >> 3) * kPanLbo + (lane & 7) * 16;
#pragma unroll
        for (int mg = 0; mg < 16; ++mg) {
          const uint32_t w = (mg >> 2) == 0 ? x.x : (mg >> 2) == 1 ? x.y : (mg >> 2) == 2 ? x.z : x.w;
          const uint32_t s8 = w >> (8 * (mg & 3));  // the signs of rows 8 mg .. 8 mg + 7
          *reinterpret_cast<uint4*>(col + mg * kPanSbo) =
              make_uint4(pm1_bf16x2(s8), pm1_bf16x2(s8 >> 2), pm1_bf16x2(s8 >> 4),
                         pm1_bf16x2(s8 >> 6));
        }
      }
      // generic-proxy writes -> visible to the tensor core, then one arrival
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sfull[bw][th]));
    }
  } else if (warp >= 16 - kProm) {  // promoters: lanes 32 (warp & 3) .., a column half
    const int rq = warp & 3;
    const int c_lo = 4 * ((warp - (16 - kProm)) >> 2);  // first 32-column chunk
    const uint32_t lanes = static_cast<uint32_t>(32 * rq) << 16;
    bool ok = true;
    int P = 0;
    for (int64_t u = lo; u < hi && ok; u += stride) {
      const PanUnit t = pan_unit(g, u);
      const int ngroups = (t.ns + kPanGroup - 1) / kPanGroup;
      const int r = t.x * 128 + 32 * rq + lane, n0 = t.y * kN;
      float* dst = out + t.z * split_stride;
      if (ngroups == 0) {  // an empty slice contributes zeros
        if (!accumulate && r < d)
          for (int c = n0 + 32 * c_lo; c < min(n, n0 + 32 * c_lo + 128); ++c)
            dst[static_cast<int64_t>(c) * d + r] = 0.f;
        continue;
      }
      for (int p = 0; p < ngroups; ++p, ++P) {
        const int b = P & 1;
        int got = 1;
        if (lane == 0) got = mbar_wait(smem_u32(&acc_full[b]), (P >> 1) & 1) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got || failed) {
          ok = false;
          failed = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const bool last = p == ngroups - 1;
        // (wide units are one group each, so they never touch the sums)
#pragma unroll 1
        for (int cc = c_lo; cc < c_lo + 4; ++cc) {
          uint32_t v[32], sm[32];
          // both loads in flight before one wait
          tmem_ld32_nowait(tmem + lanes + static_cast<uint32_t>(kN * b + 32 * cc), v);
          if (!WIDE && p > 0)
            tmem_ld32_nowait(tmem + lanes + kPanSums + static_cast<uint32_t>(32 * cc), sm);
          tmem_wait_ld32(v, sm);
          if (!WIDE && p > 0) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj)
              v[jj] = __float_as_uint(__fadd_rn(__uint_as_float(sm[jj]), __uint_as_float(v[jj])));
          }
          if (!WIDE && !last) {
            tmem_st32(tmem + lanes + kPanSums + static_cast<uint32_t>(32 * cc), v);
            continue;
          }
          // the unit's sums: to A_hat or the slice's copy
          const int c0 = n0 + 32 * cc;
          if constexpr (FP8) {  // lane l holds the scale of column c0 + l (2^k: exact)
            const float sc = c0 + lane < n ? colinv[c0 + lane] : 1.0f;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj)
              v[jj] = __float_as_uint(__uint_as_float(v[jj]) * __shfl_sync(0xffffffffu, sc, jj));
          }
          float* o = dst + static_cast<int64_t>(c0) * d + r;
          if (r < d && c0 + 32 <= n && !accumulate) {  // a full chunk: plain stores
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) o[static_cast<int64_t>(jj) * d] = __uint_as_float(v[jj]);
          } else if (r < d) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              if (c0 + jj < n) {
                float* oj = o + static_cast<int64_t>(jj) * d;
                const float x = __uint_as_float(v[jj]);
                *oj = accumulate ? *oj + x : x;
              }
            }
          }
        }
        if (!last) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&acc_empty[b]));
      }
    }
  }
  __syncthreads();
  if (tid == 0 && failed) atomicOr(status, kStatusTimeout);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// A_hat (+)= the splits' partial tiles, added in the fixed order 0, 1, ...
__global__ void k_panel_reduce(int64_t total, int splits, const float* __restrict__ partial,
                               float* __restrict__ Ahat, int accumulate) {
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float v = partial[idx];
    for (int z = 1; z < splits; ++z) v += partial[static_cast<int64_t>(z) * total + idx];
    Ahat[idx] = accumulate ? Ahat[idx] + v : v;
  }
}

// The timeout path of mbar_wait on purpose: a fresh mbarrier whose phase
// nothing completes; the bounded wait gives up and records kStatusTimeout.
__global__ void k_debug_wait_timeout(int* status, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(smem_u32(&bar), 0, limit_ns)) atomicOr(status, kStatusTimeout);
  }
}

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

namespace {
struct DenseLayout {
  int32_t *cnt, *flag, *pos, *didx, *Kdev;
  uint16_t* A3;
  char* scan_tmp;
  int32_t *rpos, *rcolptr, *rrowidx;  // the rest of A (CSC); rpos: nnz + 1 positions
  float* partial;                      // split-K partial copies of A_hat (panel kernel)
  float* colinv;                       // FP8: the per-column scale undone on output
  uint32_t* cmax;                      // FP8: largest panel magnitude per column (bits)
  int32_t max_splits;
  void* rvalues;
  size_t bytes;
};
// Split-K copies of A_hat the pipelined panel kernel may use: up to 64, and
// at most 1 GiB of them (none when the panel cannot reach a useful length).
int64_t panel_max_splits(int64_t n, int64_t d, int64_t kmax) {
  const int64_t Kp = (kmax + kBK - 1) / kBK * kBK;
  if (Kp < kBK) return 0;
  const int64_t one = n * d * static_cast<int64_t>(sizeof(float));
  return std::min<int64_t>(64, (int64_t(1) << 30) / std::max<int64_t>(one, 1));
}

DenseLayout dense_layout(void* ws, int64_t m, int64_t n, int64_t d, int64_t kmax,
                         int64_t nnz) {
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
  // n padded to the widest column tile (256)
  L.A3 = reinterpret_cast<uint16_t*>(take(static_cast<size_t>((n + 255) / 256 * 256) * 3 * Kp * 2));
  L.scan_tmp = take(static_cast<size_t>(scan_bytes_for(std::max(std::max(m, n), nnz) + 1)));
  L.rpos = reinterpret_cast<int32_t*>(take((std::max<int64_t>(1, nnz) + 1) * sizeof(int32_t)));
  L.rcolptr = reinterpret_cast<int32_t*>(take((n + 1) * sizeof(int32_t)));
  L.rrowidx = reinterpret_cast<int32_t*>(take(std::max<int64_t>(1, nnz) * sizeof(int32_t)));
  L.rvalues = take(std::max<int64_t>(1, nnz) * sizeof(float));
  L.colinv = reinterpret_cast<float*>(take(std::max<int64_t>(1, n) * sizeof(float)));
  L.cmax = reinterpret_cast<uint32_t*>(take(std::max<int64_t>(1, n) * sizeof(uint32_t)));
  L.max_splits = static_cast<int32_t>(panel_max_splits(n, d, kmax));
  L.partial = reinterpret_cast<float*>(
      take(static_cast<size_t>(L.max_splits > 1 ? L.max_splits : 0) * n * d * sizeof(float)));
  L.bytes = static_cast<size_t>(p - static_cast<char*>(ws));
  return L;
}

// Entries of column k that stay in the sparse part: rows outside the panel
// (and out-of-range rows, which the sparse kernels then flag).
__device__ __forceinline__ bool rest_keeps(int32_t j, int32_t m, const int32_t* didx) {
  return static_cast<uint32_t>(j) >= static_cast<uint32_t>(m) || didx[j] < 0;
}

// The rest of A (entries outside the panel's rows) as a stream compaction
// over all entries: rpos[e] = 1 for kept entries (rows outside the panel,
// and out-of-range rows, which the sparse kernels then flag), 0 otherwise,
// and rpos[nnz] = 0; an exclusive scan turns the flags into output
// positions.  One thread per entry throughout.
__global__ void k_rest_flags(int64_t nnz, int32_t m, const int32_t* __restrict__ rowidx,
                             const int32_t* __restrict__ didx, int32_t* __restrict__ rpos) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e <= nnz;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    rpos[e] = e < nnz ? (rest_keeps(rowidx[e], m, didx) ? 1 : 0) : 0;
}

// rest_colptr[k] = kept entries before column k's first entry (column
// ranges clamped to [0, nnz]; a malformed colptr is recorded in *status).
__global__ void k_rest_colptr(int32_t n, int64_t nnz, const int32_t* __restrict__ colptr,
                              const int32_t* __restrict__ rpos, int32_t* __restrict__ rcolptr,
                              int* status) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k <= n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t p = colptr[k];
    const int64_t c = p < 0 ? 0 : (p > nnz ? nnz : p);
    if (c != p || (k < n && colptr[k + 1] < p)) atomicOr(status, kStatusBadColptr);
    rcolptr[k] = rpos[c];
  }
}

// Kept entry e goes to position rpos[e] (positions stay below nnz).
template <typename VT>
__global__ void k_rest_scatter(int64_t nnz, int32_t m, const int32_t* __restrict__ rowidx,
                               const VT* __restrict__ vals, const int32_t* __restrict__ didx,
                               const int32_t* __restrict__ rpos, int32_t* __restrict__ rrowidx,
                               VT* __restrict__ rvals) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t j = rowidx[e];
    if (!rest_keeps(j, m, didx)) continue;
    const int32_t pos = rpos[e];
    if (static_cast<uint64_t>(pos) < static_cast<uint64_t>(nnz)) {
      rrowidx[pos] = j;
      rvals[pos] = vals[e];
    }
  }
}
}  // namespace

size_t dense_workspace_bytes(int64_t m, int64_t n, int64_t d, int64_t kmax, int64_t nnz) {
  return dense_layout(nullptr, m, n, d, kmax, nnz).bytes;
}

// Phase 1: choose the dense rows (at least tau nonzeros).  Writes didx,
// rows and K to the workspace, and the offsets of the rest of A; the caller
// reads K (the panel height) and rest_colptr[n] (the rest's nonzeros).
void dense_view(const DenseArgs& a, void* ws, DenseView* out) {
  const DenseLayout L = dense_layout(ws, a.m, a.n, a.d, a.kmax, a.nnz);
  out->didx = L.didx;
  out->rows = L.cnt;  // the panel's row ids reuse the counts' space
  out->Kdev = L.Kdev;
  out->A3 = L.A3;
  out->Kp = 0;
  out->rest_colptr = L.rcolptr;
  out->rest_rowidx = L.rrowidx;
  out->rest_values = L.rvalues;
  out->rest_pos = L.rpos;
  out->partial = L.partial;
  out->colscale = L.colinv;
  out->cmax = L.cmax;
  out->max_splits = L.max_splits;
  out->scan_tmp = L.scan_tmp;
}

cudaError_t select_dense_rows(const DenseArgs& a, void* ws, DenseView* out, cudaStream_t s,
                              int* launches) {
  const DenseLayout L = dense_layout(ws, a.m, a.n, a.d, a.kmax, a.nnz);
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
  dense_view(a, ws, out);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the rest of A: each kept entry's output position (an exclusive scan of
  // keep flags over all entries) and the column offsets (rest_colptr[n] =
  // its nnz)
  k_rest_flags<<<grid_for(a.nnz + 1), 256, 0, s>>>(a.nnz, a.m, a.rowidx, L.didx, L.rpos);
  ++*launches;
  if ((e = scan_i32(L.rpos, L.rpos, a.nnz + 1, L.scan_tmp, s, launches)) != cudaSuccess)
    return e;
  k_rest_colptr<<<grid_for(a.n + 1), 256, 0, s>>>(a.n, a.nnz, a.colptr, L.rpos, L.rcolptr,
                                                  a.status);
  ++*launches;
  return cudaGetLastError();
}

// Phase 2: the panel's BF16 terms for K dense rows (K <= kmax).
cudaError_t build_dense_panel(const DenseArgs& a, int32_t K, DenseView* v, cudaStream_t s,
                              int* launches) {
  const int64_t Kp = (static_cast<int64_t>(K) + kBK - 1) / kBK * kBK;
  v->Kp = static_cast<int32_t>(Kp);
  uint16_t* A3 = const_cast<uint16_t*>(v->A3);
  if (a.fp8) {
    // E4M3 panel: per-column scales from the panel's largest magnitudes,
    // then the two terms in the tiled layout (n padded to the tile width,
    // 2 bytes per entry)
    if (Kp < kBK) return cudaErrorNotSupported;
    const int lg = pan_wide(Kp) ? 8 : 7;
    const unsigned gb = static_cast<unsigned>(
        std::max<int64_t>(1, std::min<int64_t>((a.nnz + 255) / 256, 32LL * num_sms())));
    const unsigned gn = static_cast<unsigned>(
        std::max<int64_t>(1, std::min<int64_t>((a.n + 255) / 256, 32LL * num_sms())));
    cudaError_t e = cudaMemsetAsync(v->cmax, 0, static_cast<size_t>(a.n) * sizeof(uint32_t), s);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(A3, 0, static_cast<size_t>(((a.n + (1 << lg) - 1) >> lg) << lg) * Kp * 2, s);
    if (e != cudaSuccess) return e;
    if (a.dtype == 0)
      k_panel_colmax<float><<<gb, 256, 0, s>>>(a.n, a.m, a.nnz, a.colptr, a.rowidx,
                                               static_cast<const float*>(a.values), v->didx,
                                               v->cmax);
    else
      k_panel_colmax<__nv_bfloat16><<<gb, 256, 0, s>>>(
          a.n, a.m, a.nnz, a.colptr, a.rowidx, static_cast<const __nv_bfloat16*>(a.values),
          v->didx, v->cmax);
    k_panel_colscale<<<gn, 256, 0, s>>>(a.n, v->cmax, v->colscale);
    uint8_t* A8 = reinterpret_cast<uint8_t*>(A3);
    if (a.dtype == 0)
      k_dense_scatter_fp8<float><<<gb, 256, 0, s>>>(
          a.n, a.m, static_cast<int32_t>(Kp), lg, a.nnz, a.colptr, a.rowidx,
          static_cast<const float*>(a.values), v->didx, v->colscale, A8);
    else
      k_dense_scatter_fp8<__nv_bfloat16><<<gb, 256, 0, s>>>(
          a.n, a.m, static_cast<int32_t>(Kp), lg, a.nnz, a.colptr, a.rowidx,
          static_cast<const __nv_bfloat16*>(a.values), v->didx, v->colscale, A8);
    *launches += 3;
    return cudaGetLastError();
  }
  const int lg = pan_wide(Kp) ? 8 : 7;
  cudaError_t e =
      cudaMemsetAsync(A3, 0, static_cast<size_t>(((a.n + (1 << lg) - 1) >> lg) << lg) * 3 * Kp * 2, s);
  if (e != cudaSuccess) return e;
  const int64_t blocks =
      std::max<int64_t>(1, std::min<int64_t>((a.nnz + 255) / 256, 32LL * num_sms()));
  if (a.dtype == 0)
    k_dense_scatter<float><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
        a.n, a.m, static_cast<int32_t>(Kp), lg, a.nnz, a.colptr, a.rowidx,
        static_cast<const float*>(a.values), v->didx, A3);
  else
    k_dense_scatter<__nv_bfloat16><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
        a.n, a.m, static_cast<int32_t>(Kp), lg, a.nnz, a.colptr, a.rowidx,
        static_cast<const __nv_bfloat16*>(a.values), v->didx, A3);
  ++*launches;
  return cudaGetLastError();
}

// Phase 3: the rest of A (entries outside the panel's rows) compacted into
// its own CSC at the offsets phase 1 computed.
cudaError_t build_dense_rest(const DenseArgs& a, const DenseView& v, cudaStream_t s,
                             int* launches) {
  const int64_t blocks =
      std::max<int64_t>(1, std::min<int64_t>((a.nnz + 255) / 256, 32LL * num_sms()));
  if (a.dtype == 0)
    k_rest_scatter<float><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
        a.nnz, a.m, a.rowidx, static_cast<const float*>(a.values), v.didx, v.rest_pos,
        const_cast<int32_t*>(v.rest_rowidx), static_cast<float*>(const_cast<void*>(v.rest_values)));
  else
    k_rest_scatter<__nv_bfloat16><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
        a.nnz, a.m, a.rowidx, static_cast<const __nv_bfloat16*>(a.values), v.didx, v.rest_pos,
        const_cast<int32_t*>(v.rest_rowidx),
        static_cast<__nv_bfloat16*>(const_cast<void*>(v.rest_values)));
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_debug_wait_timeout(int* status, cudaStream_t s) {
  k_debug_wait_timeout<<<1, 32, 0, s>>>(status, 2000000ull);  // 2 ms
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const DenseArgs& a, const DenseView& v, float* Ahat,
                           int accumulate, cudaStream_t s, int* launches) {
  if (v.Kp < kBK) return cudaErrorInvalidValue;
  const bool fp8 = a.fp8 != 0;
  const int64_t sms = num_sms();
  PanelGrid g{};
  g.d = a.d;
  g.n = a.n;
  g.steps = v.Kp / kBK;
  // a panel of at most one group: 128 x 256 units (the layout build_dense_panel chose)
  const bool wide = pan_wide(v.Kp);
  const int kN = pan_cols(wide);
  g.tiles_d = (a.d + 127) / 128;
  g.tiles_n = (a.n + kN - 1) / kN;
  const int64_t tiles = static_cast<int64_t>(g.tiles_d) * g.tiles_n;
  int64_t splits = 1;
  if (wide || static_cast<int64_t>(g.steps) * pan_step_bytes(fp8, false) <= kPanResBytes) {
    g.resident = 1;  // a short panel: each column tile's B stays in shared memory
  } else {
    // split-K by a small cost model in units of one step of one CTA
    // (about 0.3 us): the busiest CTA's steps plus two a unit, plus each
    // partial copy of A_hat written and read back at HBM speed
    const double copy_steps = 2.0 * 4.0 * a.n * static_cast<double>(a.d) / 6.7e12 / 0.3e-6;
    const int64_t smax = std::max<int64_t>(1, std::min<int64_t>(v.max_splits, g.steps));
    double best = 1e300;
    for (int64_t sp = 1; sp <= smax; ++sp) {
      const int64_t sps = (g.steps + sp - 1) / sp;
      if ((g.steps + sps - 1) / sps != sp) continue;  // no empty slice
      const int64_t U = tiles * sp, G = std::min<int64_t>(U, sms);
      const double cost = static_cast<double>((U + G - 1) / G) * static_cast<double>(sps + 2) +
                          (sp > 1 ? static_cast<double>(sp) * copy_steps : 0.0);
      if (cost < best) {
        best = cost;
        splits = sp;
      }
    }
  }
  g.sps = static_cast<int32_t>((g.steps + splits - 1) / splits);
  g.units = tiles * splits;
  if (g.units >= (int64_t(1) << 31)) return cudaErrorInvalidValue;  // 32-bit unit ids
  const unsigned grid = static_cast<unsigned>(std::min<int64_t>(g.units, sms));
  const size_t smem = pan_smem_bytes(fp8, wide, g.resident != 0, g.steps);
  auto kern = fp8 ? (wide ? k_tc_panel<true, true> : k_tc_panel<true, false>)
                  : (wide ? k_tc_panel<false, true> : k_tc_panel<false, false>);
  cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  const int64_t total = static_cast<int64_t>(a.n) * a.d;
  float* out = splits > 1 ? v.partial : Ahat;
  kern<<<grid, kPanThreads, smem, s>>>(
      g, v.rows, v.Kdev, reinterpret_cast<const uint8_t*>(v.A3), v.colscale, out,
      splits > 1 ? total : 0, splits > 1 ? 0 : accumulate, a.k0, a.k1, a.stream_id, a.status);
  ++*launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (splits > 1) {
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 16LL * sms);
    k_panel_reduce<<<static_cast<unsigned>(blocks), 256, 0, s>>>(
        total, static_cast<int>(splits), v.partial, Ahat, accumulate);
    ++*launches;
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace sk
