// internal.h -- host-side launchers shared between the translation units of
// libsketch.so.  Not part of the public ABI (see include/sketch.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <string>

namespace sk {

struct RegenArgs {
  int32_t m, n, d;
  int32_t dtype;  // 0 = f32, 1 = bf16
  int64_t nnz;
  const int32_t* colptr;
  const int32_t* rowidx;
  const void* values;
  float* Ahat;
  uint32_t k0, k1, stream_id;
  int32_t dist;
  int32_t q_tiles;  // 1..4
  int32_t split;    // 1, 2, 4, 8
  int* status;
  unsigned long long* gen_count;  // may be null
};
cudaError_t launch_regen(const RegenArgs& a, cudaStream_t s);

// One instance of a batched sketch (device-resident descriptor).
struct BatchInstance {
  const int32_t* colptr;
  const int32_t* rowidx;
  const void* values;
  float* Ahat;
  int32_t m, n, d, dtype;
  uint32_t k0, k1, stream_id, pad;
};
// One work item: column `column` of instance `instance`, rows of S
// [tile * 128 * Q, (tile + 1) * 128 * Q).
struct BatchItem {
  int32_t instance, column, tile, pad;
};
cudaError_t launch_regen_batched(int dist, int q_tiles, const BatchInstance* inst,
                                 const BatchItem* items, int64_t n_items,
                                 unsigned long long* counter, int* status,
                                 int blocks, cudaStream_t s);
int batched_blocks_per_sm(int dist, int q_tiles);

// CSR copy of A (the single-vertical-block "blocked CSR" of Sec. 3.2) built
// on the device.  Workspace sizes in bytes for m rows and nnz nonzeros.
size_t csr_workspace_bytes(int64_t m, int64_t nnz);
struct CsrView {
  int32_t* rowptr;  // m + 1
  int32_t* ccol;    // nnz
  float* cval;      // nnz
};
cudaError_t build_csr(int32_t m, int32_t n, int64_t nnz, const int32_t* colptr,
                      const int32_t* rowidx, const void* values, int32_t dtype,
                      void* ws, CsrView* out, int* status, cudaStream_t s,
                      int* launches);

struct PanelArgs {
  int32_t m, n, d;
  CsrView csr;
  float* partial;  // row_groups * n * d floats
  float* Ahat;
  uint32_t k0, k1, stream_id;
  int32_t dist;
  int32_t n_block;
  int32_t row_groups;
  int32_t compensated;  // 1: compensated shared-memory sums (k_panel COMP)
  unsigned long long* gen_count;
};
size_t panel_smem_bytes(int32_t n_block, bool compensated);
cudaError_t launch_panel(const PanelArgs& a, cudaStream_t s, int* launches);

struct TileArgs {
  int32_t m, n, d;
  int64_t nnz;
  int32_t dtype;
  const int32_t* colptr;
  const int32_t* rowidx;
  const void* values;
  float* Ahat;
  uint32_t k0, k1, stream_id;
  int32_t dist;
  int32_t R;    // rows of A per panel (m1)
  int32_t G;    // row ranges of the panels: register sums, one CTA per (tile,
                // range) writing a partial copy; tensor-memory sums, the phases
                // one wave of CTAs walks in order
  int32_t cpw;  // columns per warp: 4, 16 or 64; 32 with tacc (n1 = warps * cpw)
  int32_t tacc;  // 1: accumulators in tensor memory (32 warps of cpw 32)
  // dist 3: S read from S_mem (d x m, column j at S_mem + j * ld_s; ld_s a
  // multiple of 4 and >= d, S_mem 16-byte aligned) instead of generated
  const float* S_mem = nullptr;
  int64_t ld_s = 0;
  int* status;
  unsigned long long* gen_count;
  // 1: the panel-major copy, panel pointers and offsets already sit in the
  // workspace from an earlier call on the same A (same content hash) and plan
  int32_t prepared = 0;
};
size_t tile_workspace_bytes(int64_t m, int64_t n, int64_t d, int64_t nnz,
                            int32_t R, int32_t G, int32_t tacc);
size_t tile_smem_bytes(int32_t R, int32_t tacc);
cudaError_t launch_tile(const TileArgs& a, void* ws, cudaStream_t s,
                        int* launches);

cudaError_t launch_validate(int32_t m, int32_t n, int64_t nnz,
                            const int32_t* colptr, const int32_t* rowidx,
                            int* status, cudaStream_t s);
cudaError_t launch_debug_normal_pair(const uint32_t* words, float* out, int64_t count,
                                     cudaStream_t s);
cudaError_t launch_debug_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1,
                                uint32_t* out, int64_t count, cudaStream_t s);
// S_mem[j * ld_s + i] = S(i, j), i < d, j < m (ld_s >= d, a multiple of 4;
// S_mem 16-byte aligned).
cudaError_t launch_generate_S(int dist, uint32_t k0, uint32_t k1, uint32_t stream_id,
                              int32_t d, int32_t m, float* S_mem, int64_t ld_s,
                              cudaStream_t s);
cudaError_t launch_debug_S(int dist, uint32_t k0, uint32_t k1,
                           uint32_t stream_id, const int64_t* i,
                           const int64_t* j, float* out, int64_t count,
                           cudaStream_t s);

cudaError_t launch_bench_fma(int64_t threads, int64_t iters, float* sink, cudaStream_t s);
cudaError_t launch_bench_generator(int dist, uint32_t k0, uint32_t k1,
                                   int64_t threads, int64_t blocks_per_thread,
                                   float* sink, cudaStream_t s);

// Tensor-core densified panels (dense_tc.cu).
struct DenseArgs {
  int32_t m, n, d;
  int64_t nnz;
  int32_t dtype;
  const int32_t* colptr;
  const int32_t* rowidx;
  const void* values;
  int32_t tau;   // rows with at least tau nonzeros go to the panel
  int32_t fp8;   // 1: E4M3 operands (two terms of A, per-column scales)
  int64_t kmax;  // capacity: nnz / tau bounds the number of such rows
  uint32_t k0, k1, stream_id;
  int* status;
};
struct DenseView {
  const int32_t* didx;  // m: dense index of a row, or -1
  const int32_t* rows;  // K: dense row ids
  const int32_t* Kdev;  // device copy of K
  const uint16_t* A3;   // n x 3Kp BF16 terms (column-major, K fastest)
  int32_t Kp;
  // A without the panel's rows, in CSC (same dtype; rows stay sorted per
  // column); rest_nnz is an upper bound (A's nnz), the exact count lives in
  // rest_colptr[n]
  const int32_t* rest_colptr;
  const int32_t* rest_rowidx;
  const void* rest_values;
  const int32_t* rest_pos;  // output position of each kept entry (scan of keep flags)
  float* partial;           // split-K partial copies of A_hat (pipelined panel kernel)
  float* colscale;          // FP8: 2^e per column of A, undone on output
  uint32_t* cmax;           // FP8: workspace, largest panel magnitude per column
  int32_t max_splits;       // how many of them the workspace holds (0: none)
  char* scan_tmp;     // workspace: scan scratch
};
size_t dense_workspace_bytes(int64_t m, int64_t n, int64_t d, int64_t kmax, int64_t nnz);
// The workspace pointers of a panel (no launches): what select_dense_rows
// fills in, for a panel already built in `ws` by an earlier call.
void dense_view(const DenseArgs& a, void* ws, DenseView* out);
cudaError_t select_dense_rows(const DenseArgs& a, void* ws, DenseView* out, cudaStream_t s,
                              int* launches);
cudaError_t build_dense_panel(const DenseArgs& a, int32_t K, DenseView* v, cudaStream_t s,
                              int* launches);
cudaError_t build_dense_rest(const DenseArgs& a, const DenseView& v, cudaStream_t s,
                             int* launches);
cudaError_t launch_debug_wait_timeout(int* status, cudaStream_t s);
cudaError_t launch_tc_gemm(const DenseArgs& a, const DenseView& v, float* Ahat,
                           int accumulate, cudaStream_t s, int* launches);

// Shared building blocks (sketch_kernels.cu).
int64_t scan_bytes_for(int64_t len);
cudaError_t scan_i32(const int32_t* in, int32_t* out, int64_t len, char* tmp,
                     cudaStream_t s, int* launches);
cudaError_t row_counts(int64_t nnz, int32_t m, const int32_t* rowidx, int32_t* cnt,
                       int* status, cudaStream_t s);

// A 64-bit content hash of A (colptr, rowidx and the value words), XOR of one
// mixed key per array entry, so it does not depend on the order the entries
// are visited in: written to *out (zeroed here first).
cudaError_t content_hash(int32_t n, int64_t nnz, const int32_t* colptr,
                         const int32_t* rowidx, const void* values, int32_t value_bytes,
                         unsigned long long* out, cudaStream_t s);

// Pattern features of A for the plan tuner (see k_pattern_features): f[0]
// nonempty rows, f[1] longest row, f[2] nonzeros in rows of >= 32 entries,
// f[3] longest column.  cnt: m ints of scratch.
cudaError_t pattern_features(int32_t m, int32_t n, int64_t nnz, const int32_t* colptr,
                             const int32_t* rowidx, int32_t* cnt, unsigned long long* f,
                             int* status, cudaStream_t s);

int num_sms();
// Raise a kernel's dynamic shared-memory limit to at least `bytes`; never
// lowers it.  The attribute belongs to the kernel, not to a thread, so
// launches from several host threads (the solve server's slots) must not
// set it down under one another; each size is set once.
cudaError_t raise_smem_limit(const void* kernel, size_t bytes);

}  // namespace sk
