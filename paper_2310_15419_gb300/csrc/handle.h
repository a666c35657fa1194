// handle.h -- the state behind a sketch_t and the helpers the C ABI files
// share.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>

#include "../../include/sketch.h"

namespace sk {
struct LsqState;  // lsq.cu
}

struct sketch_s {
  int64_t m = 0, n = 0, d = 0;
  int32_t dist = 0;
  uint64_t seed = 0;
  uint32_t k0 = 0, k1 = 0;       // Philox key = (seed lo32, seed hi32)
  uint32_t stream_id = 0;        // Philox counter word 2
  bool has_forced = false;
  sketch_plan forced{};
  std::map<uint64_t, sketch_plan> plans;  // tuned plans per shape
  std::string last_error;
  void* ws = nullptr;            // device workspace (CSR copy, partial sums)
  size_t ws_bytes = 0;
  void* d_small = nullptr;       // 256 B: status word at 0, entry count at 64
  bool counting = false;
  bool autotune = true;
  int64_t launches = 0;          // kernels launched so far
  bool capturing = false;        // the caller's stream is being captured
  // least-squares kernels start while their predecessor finishes
  // (programmatic dependent launch); off for handles whose solves share the
  // GPU with other streams, where early-started blocks would hold SMs
  bool dependent_launch = true;
  sk::LsqState* lsq = nullptr;   // least-squares workspace (lazy)
  // Derived data of the last A run through the workspace -- a tensor-core
  // plan's panel and the rest of A, TILE's panel-major copy -- reused while
  // A's content hash, its arrays, the shape, the plan and the workspace match
  struct Prepared {
    bool valid = false;
    uint64_t hash = 0;
    const void* arrays[3] = {};
    int64_t m = 0, n = 0, nnz = 0, d = 0;
    int32_t dtype = 0;
    sketch_plan plan{};
    void* ws = nullptr;
    int32_t K = 0, rest_nnz = 0;  // the panel's rows and the rest's nonzeros
  } prep;
};

namespace sk {
int fail(sketch_t h, int code, const std::string& msg);
int cuda_fail(sketch_t h, cudaError_t e, const char* where);
int ensure_small(sketch_t h);
int ensure_workspace(sketch_t h, size_t bytes);
int32_t default_row_groups(const sketch_s* h, const sketch_csc* A,
                           int32_t n_block);
sketch_plan heuristic_plan(const sketch_s* h, const sketch_csc* A);
size_t plan_workspace_bytes(const sketch_s* h, const sketch_csc* A,
                            const sketch_plan& p);
int check_plan(sketch_t h, const sketch_plan& p);
int run_plan(sketch_t h, const sketch_csc* A, float* Ahat,
             const sketch_plan& p, void* ws, cudaStream_t s);
int choose_plan(sketch_t h, const sketch_csc* A, float* Ahat, cudaStream_t s,
                sketch_plan* out);
int check_csc_args(sketch_t h, const sketch_csc* A);
uint64_t shape_key(const sketch_s* h, const sketch_csc* A);
size_t lsq_workspace_bytes(int64_t m, int64_t n, int64_t d, int64_t nnz);
void destroy_lsq_state(sketch_t h);
}  // namespace sk
