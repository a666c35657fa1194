// sketch_capi.cu -- the C ABI (include/sketch.h): handles, device workspace,
// the launch planner / autotuner, and the sketch entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/sketch.h"
#include "common.cuh"
#include "handle.h"
#include "internal.h"

using namespace sk;

namespace sk {

static thread_local std::string g_global_error;

int fail(sketch_t h, int code, const std::string& msg) {
  if (h)
    h->last_error = msg;
  else
    g_global_error = msg;
  return code;
}

int cuda_fail(sketch_t h, cudaError_t e, const char* where) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  return fail(h, SKETCH_ERR_CUDA, buf);
}

int ensure_small(sketch_t h) {
  if (h->d_small) return SKETCH_OK;
  cudaError_t e = cudaMalloc(&h->d_small, 256);
  if (e != cudaSuccess) {
    h->d_small = nullptr;
    return fail(h, SKETCH_ERR_OOM, "cudaMalloc(status words) failed");
  }
  e = cudaMemset(h->d_small, 0, 256);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemset(status words)");
  return SKETCH_OK;
}

int ensure_workspace(sketch_t h, size_t bytes) {
  if (bytes <= h->ws_bytes) return SKETCH_OK;
  // growing the workspace is not allowed while the caller captures a graph
  if (h->capturing)
    return fail(h, SKETCH_ERR_OOM,
                "workspace too small during stream capture; "
                "call sketch_apply once before capturing");
  if (h->ws) {
    cudaDeviceSynchronize();
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  const size_t want = bytes + bytes / 8;
  h->prep.valid = false;  // a new allocation may reuse the old address
  cudaError_t e = cudaMalloc(&h->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->ws = nullptr;
    return fail(h, SKETCH_ERR_OOM, "cudaMalloc(workspace) failed");
  }
  h->ws_bytes = want;
  return SKETCH_OK;
}

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// TILE plan for a panel height R: columns per warp covering n (up to 1024
// per CTA).  Register sums: row groups that fill the GPU and keep each
// column's partial sums to ~512 terms.  Tensor-memory sums: one wave of CTAs
// walks the row groups in order, so the groups only bound the chains (~512
// terms) and the slice of A shared in L2 (at least 8 groups).
sketch_plan tile_plan(const sketch_s* h, const sketch_csc* A, int32_t R, int32_t tile_acc) {
  sketch_plan p{};
  p.mode = SKETCH_MODE_TILE;
  p.panel_rows = R;
  p.cols_per_warp = A->n <= 64 ? 4 : A->n <= 256 ? 16 : 64;
  if (tile_acc && p.cols_per_warp == 64) {  // 32 warps of 32 columns
    p.tile_acc = 1;
    p.cols_per_warp = 32;
  }
  const int64_t n1 = (p.tile_acc ? 32 : 16) * p.cols_per_warp;
  const int64_t tiles = (h->d + 31) / 32;
  const int64_t cblocks = (A->n + n1 - 1) / n1;
  const int64_t P = (A->m + R - 1) / R;
  const double avg_col = A->n > 0 ? double(A->nnz) / double(A->n) : 0.0;
  if (p.tile_acc) {
    const int64_t g = std::max<int64_t>(8, static_cast<int64_t>(std::ceil(avg_col / 512.0)));
    p.row_groups = static_cast<int32_t>(std::max<int64_t>(1, std::min<int64_t>({g, P, 4096})));
    return p;
  }
  const int per_sm = 1;
  int64_t g_fill = (2LL * per_sm * num_sms() + tiles * cblocks - 1) / (tiles * cblocks);
  int64_t g_acc = static_cast<int64_t>(std::ceil(avg_col / 512.0));
  int64_t g = std::max<int64_t>({1, g_fill, g_acc});
  g = std::min<int64_t>({g, P, 4096});
  // One CTA per SM: among g .. 2g row groups take the one whose last wave
  // of CTAs is fullest (g = 20 on 94 row tiles leaves the 13th wave 37%
  // full; g = 21 fills it), the smallest on ties
  const int64_t slots = static_cast<int64_t>(per_sm) * num_sms();
  int64_t best_g = g;
  double best_fill = 0.0;
  for (int64_t c = g; c <= std::min<int64_t>({2 * g, P, 4096}); ++c) {
    const int64_t units = tiles * cblocks * c;
    const double fill = double(units) / double(((units + slots - 1) / slots) * slots);
    if (fill > best_fill + 1e-9) {
      best_fill = fill;
      best_g = c;
    }
  }
  p.row_groups = static_cast<int32_t>(std::max<int64_t>(1, best_g));
  return p;
}

// Heuristic plan (used when tuning is off or not possible).
sketch_plan heuristic_plan(const sketch_s* h, const sketch_csc* A) {
  sketch_plan p{};
  const double avg_col = A->n > 0 ? double(A->nnz) / double(A->n) : 0.0;
  const int q = static_cast<int>(std::min<int64_t>(4, (h->d + 127) / 128));
  if (h->dist == SKETCH_PM1 || A->nnz < 4 * A->n) {
    p.mode = SKETCH_MODE_REGEN;
    p.q_tiles = std::max(1, q);
    p.split = avg_col >= 4096 ? 8 : avg_col >= 1024 ? 4 : avg_col >= 256 ? 2 : 1;
  } else {
    p = A->n > 256 ? tile_plan(h, A, 1248, 1) : tile_plan(h, A, 1024, 0);
  }
  return p;
}

// Row groups for PANEL: enough CTAs to fill the GPU twice over, and at most
// ~512 nonzeros of a column per group so FP32 partial sums stay short.
int32_t default_row_groups(const sketch_s* h, const sketch_csc* A,
                           int32_t n_block) {
  const int64_t tiles = (h->d + 31) / 32;
  const int64_t cblocks = (A->n + n_block - 1) / n_block;
  const double avg_col = A->n > 0 ? double(A->nnz) / double(A->n) : 0.0;
  int64_t g_fill = (2LL * num_sms() + tiles * cblocks - 1) / (tiles * cblocks);
  int64_t g_acc = static_cast<int64_t>(std::ceil(avg_col / 512.0));
  int64_t g = std::max<int64_t>({1, g_fill, g_acc});
  g = std::min<int64_t>(g, std::max<int64_t>(1, A->m / 64));
  g = std::min<int64_t>(g, 4096);
  return static_cast<int32_t>(g);
}

static int64_t dense_capacity(const sketch_csc* A, const sketch_plan& p) {
  // every dense row holds at least tau nonzeros, so at most nnz / tau rows
  return std::max<int64_t>(1, std::min<int64_t>(A->m, A->nnz / std::max(1, p.tc_min_row_nnz)));
}

static size_t sparse_workspace_bytes(const sketch_s* h, const sketch_csc* A,
                                     const sketch_plan& p);

size_t plan_workspace_bytes(const sketch_s* h, const sketch_csc* A,
                            const sketch_plan& p) {
  size_t b = sparse_workspace_bytes(h, A, p);
  if (p.tc_min_row_nnz > 0)
    b = align256(b) + dense_workspace_bytes(A->m, A->n, h->d, dense_capacity(A, p), A->nnz);
  return b;
}

static size_t sparse_workspace_bytes(const sketch_s* h, const sketch_csc* A,
                                     const sketch_plan& p) {
  if (p.mode == SKETCH_MODE_TILE)
    return tile_workspace_bytes(A->m, A->n, h->d, A->nnz, p.panel_rows, p.row_groups,
                                p.tile_acc);
  if (p.mode != SKETCH_MODE_PANEL) return 0;
  size_t b = align256(csr_workspace_bytes(A->m, A->nnz));
  if (p.row_groups > 1)
    b += align256(static_cast<size_t>(p.row_groups) * A->n * h->d * sizeof(float));
  return b;
}

int check_plan(sketch_t h, const sketch_plan& p) {
  if (p.tc_min_row_nnz < 0) return fail(h, SKETCH_ERR_ARG, "tc_min_row_nnz < 0");
  if (p.tc_min_row_nnz > 0 && h->dist != SKETCH_PM1)
    return fail(h, SKETCH_ERR_UNSUPPORTED,
                "tensor-core panels need +-1 S (exact in BF16)");
  if (p.tc_min_row_nnz > 0 && p.mode == SKETCH_MODE_PANEL)
    return fail(h, SKETCH_ERR_UNSUPPORTED, "tensor-core panels pair with REGEN or TILE");
  if (p.tc_fp8 != 0 && p.tc_fp8 != 1) return fail(h, SKETCH_ERR_ARG, "tc_fp8 must be 0 or 1");
  if (p.tc_fp8 && p.tc_min_row_nnz <= 0)
    return fail(h, SKETCH_ERR_ARG, "tc_fp8 needs tensor-core panels (tc_min_row_nnz > 0)");
  if (p.mode == SKETCH_MODE_REGEN) {
    if (p.q_tiles < 1 || p.q_tiles > 4)
      return fail(h, SKETCH_ERR_ARG, "q_tiles must be 1..4");
    if (p.split != 1 && p.split != 2 && p.split != 4 && p.split != 8)
      return fail(h, SKETCH_ERR_ARG, "split must be 1, 2, 4 or 8");
  } else if (p.mode == SKETCH_MODE_PANEL) {
    if (p.n_block < 1 || p.n_block > 1536)
      return fail(h, SKETCH_ERR_ARG, "n_block must be 1..1536");
    if (p.row_groups < 1 || p.row_groups > 65535)
      return fail(h, SKETCH_ERR_ARG, "row_groups must be 1..65535");
  } else if (p.mode == SKETCH_MODE_TILE) {
    if (p.tile_acc != 0 && p.tile_acc != 1)
      return fail(h, SKETCH_ERR_ARG, "tile_acc must be 0 or 1");
    // the S tile (panel_rows x 32 floats) and the staged entries share the
    // 227 KB of dynamic shared memory a CTA can have: up to 1248 rows
    if (p.panel_rows < 8 || p.panel_rows > 1248 ||
        tile_smem_bytes(p.panel_rows, p.tile_acc) > 232448 - 1024)
      return fail(h, SKETCH_ERR_ARG, "panel_rows must be 8..1248");
    if (p.tile_acc == 0 && p.cols_per_warp != 4 && p.cols_per_warp != 16 &&
        p.cols_per_warp != 64)
      return fail(h, SKETCH_ERR_ARG, "cols_per_warp must be 4, 16 or 64");
    if (p.tile_acc == 1 && p.cols_per_warp != 32)
      return fail(h, SKETCH_ERR_ARG, "tile_acc = 1 needs cols_per_warp = 32");
    if (p.row_groups < 1 || p.row_groups > 65535)
      return fail(h, SKETCH_ERR_ARG, "row_groups must be 1..65535");
  } else if (p.mode != SKETCH_MODE_AUTO) {
    return fail(h, SKETCH_ERR_ARG, "unknown mode");
  }
  return SKETCH_OK;
}

int run_sparse(sketch_t h, const sketch_csc* A, float* Ahat, const sketch_plan& p,
               void* ws, cudaStream_t s, int* status, unsigned long long* gen,
               bool prepared);

static int run_plan_body(sketch_t h, const sketch_csc* A, float* Ahat,
                         const sketch_plan& p, void* ws, cudaStream_t s, bool prepared,
                         int32_t* K_out, int32_t* rest_out);

static bool same_plan(const sketch_plan& a, const sketch_plan& b) {
  return a.mode == b.mode && a.q_tiles == b.q_tiles && a.split == b.split &&
         a.n_block == b.n_block && a.row_groups == b.row_groups &&
         a.panel_rows == b.panel_rows && a.cols_per_warp == b.cols_per_warp &&
         a.tc_min_row_nnz == b.tc_min_row_nnz && a.tile_acc == b.tile_acc &&
         a.tc_fp8 == b.tc_fp8;
}

// Run one plan.  `ws` must hold plan_workspace_bytes.  Plans that derive
// data from A before the sketch (a tensor-core panel, TILE's panel-major
// copy) first hash A's content on the device; when the hash, A's arrays, the
// shape, the plan and the workspace match the previous such call and no
// error has been flagged since, the derived data still in the workspace is
// reused and only the sketch kernels run.  Under stream capture (no host
// read possible) the data is always rebuilt.
int run_plan(sketch_t h, const sketch_csc* A, float* Ahat,
             const sketch_plan& p, void* ws, cudaStream_t s) {
  const bool cacheable = !h->capturing && ws == h->ws && A->n > 0 && A->nnz > 0 &&
                         h->d > 0 && (p.tc_min_row_nnz > 0 || p.mode == SKETCH_MODE_TILE);
  bool hit = false;
  uint64_t hash = 0;
  if (cacheable) {
    auto* dh = reinterpret_cast<unsigned long long*>(static_cast<char*>(h->d_small) + 128);
    int st = 0;
    cudaError_t e = content_hash(static_cast<int32_t>(A->n), A->nnz, A->colptr, A->rowidx,
                                 A->values, A->dtype == SKETCH_BF16 ? 2 : 4, dh, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hash, dh, sizeof(hash), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, h->d_small, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "content hash");
    h->launches += 1;
    const auto& c = h->prep;
    hit = c.valid && st == 0 && c.hash == hash && c.ws == ws && c.m == A->m && c.n == A->n &&
          c.nnz == A->nnz && c.d == h->d && c.dtype == A->dtype &&
          c.arrays[0] == A->colptr && c.arrays[1] == A->rowidx && c.arrays[2] == A->values &&
          same_plan(c.plan, p);
  }
  h->prep.valid = false;  // the workspace is (re)written below
  int32_t K = hit ? h->prep.K : 0, rest_nnz = hit ? h->prep.rest_nnz : 0;
  const int rc = run_plan_body(h, A, Ahat, p, ws, s, hit, &K, &rest_nnz);
  if (rc == SKETCH_OK && cacheable) {
    auto& c = h->prep;
    c.valid = true;
    c.hash = hash;
    c.arrays[0] = A->colptr;
    c.arrays[1] = A->rowidx;
    c.arrays[2] = A->values;
    c.m = A->m;
    c.n = A->n;
    c.nnz = A->nnz;
    c.d = h->d;
    c.dtype = A->dtype;
    c.plan = p;
    c.ws = ws;
    c.K = K;
    c.rest_nnz = rest_nnz;
  }
  return rc;
}

static int run_plan_body(sketch_t h, const sketch_csc* A, float* Ahat,
                         const sketch_plan& p, void* ws, cudaStream_t s, bool prepared,
                         int32_t* K_out, int32_t* rest_out) {
  int* status = reinterpret_cast<int*>(h->d_small);
  unsigned long long* gen =
      h->counting ? reinterpret_cast<unsigned long long*>(
                        static_cast<char*>(h->d_small) + 64)
                  : nullptr;
  if (gen) {
    cudaError_t e = cudaMemsetAsync(gen, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync(count)");
  }
  if (A->n == 0 || h->d == 0) return SKETCH_OK;
  if (A->nnz == 0) {
    cudaError_t e = cudaMemsetAsync(Ahat, 0, sizeof(float) * A->n * h->d, s);
    return e == cudaSuccess ? SKETCH_OK : cuda_fail(h, e, "cudaMemsetAsync");
  }
  // tensor-core densified panel: pick its rows first (the sparse kernels
  // then leave them out); the panel's product is added at the end
  DenseArgs da{};
  DenseView dv{};
  int32_t K = prepared ? *K_out : 0, rest_nnz = prepared ? *rest_out : 0;
  if (p.tc_min_row_nnz > 0) {
    if (h->capturing)
      return fail(h, SKETCH_ERR_UNSUPPORTED, "a tensor-core plan cannot be captured");
    da.m = static_cast<int32_t>(A->m);
    da.n = static_cast<int32_t>(A->n);
    da.d = static_cast<int32_t>(h->d);
    da.nnz = A->nnz;
    da.dtype = A->dtype;
    da.colptr = A->colptr;
    da.rowidx = A->rowidx;
    da.values = A->values;
    da.tau = p.tc_min_row_nnz;
    da.fp8 = p.tc_fp8;
    da.kmax = dense_capacity(A, p);
    da.k0 = h->k0;
    da.k1 = h->k1;
    da.stream_id = h->stream_id;
    da.status = status;
    void* dws = static_cast<char*>(ws) + align256(sparse_workspace_bytes(h, A, p));
    int nl = 0;
    if (prepared) {  // the panel and the rest of A from the previous call
      dense_view(da, dws, &dv);
      dv.Kp = (K + 31) / 32 * 32;
    }
    if (!prepared) {
      cudaError_t e = select_dense_rows(da, dws, &dv, s, &nl);
      h->launches += nl;
      if (e != cudaSuccess) return cuda_fail(h, e, "dense row selection");
      e = cudaMemcpyAsync(&K, dv.Kdev, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&rest_nnz, dv.rest_colptr + A->n, sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(h, e, "dense row count");
      // overlapping column ranges of a malformed colptr (flagged on the
      // device) can count more kept entries than A holds
      if (rest_nnz < 0 || rest_nnz > A->nnz) rest_nnz = static_cast<int32_t>(A->nnz);
      if (K > 0) {
        nl = 0;
        e = build_dense_panel(da, K, &dv, s, &nl);
        if (e == cudaSuccess && rest_nnz > 0) e = build_dense_rest(da, dv, s, &nl);
        h->launches += nl;
        if (e != cudaSuccess) return cuda_fail(h, e, "dense panel");
      }
      *K_out = K;
      *rest_out = rest_nnz;
    }
  }
  // the sparse kernels see A without the panel's rows; with nothing left
  // the panel's product is stored into A_hat directly
  sketch_csc rest = *A;
  int rc_sparse = SKETCH_OK;
  const bool rest_empty = K > 0 && rest_nnz == 0;
  if (!rest_empty) {
    if (K > 0) {
      rest.colptr = dv.rest_colptr;
      rest.rowidx = dv.rest_rowidx;
      rest.values = dv.rest_values;
      rest.nnz = rest_nnz;
    }
    rc_sparse = run_sparse(h, &rest, Ahat, p, ws, s, status, gen, prepared);
  }
  if (rc_sparse != SKETCH_OK || K == 0) return rc_sparse;
  int nl = 0;
  cudaError_t e = launch_tc_gemm(da, dv, Ahat, rest_empty ? 0 : 1, s, &nl);
  h->launches += nl;
  return e == cudaSuccess ? SKETCH_OK : cuda_fail(h, e, "tensor-core panel");
}

int run_sparse(sketch_t h, const sketch_csc* A, float* Ahat, const sketch_plan& p,
               void* ws, cudaStream_t s, int* status, unsigned long long* gen,
               bool prepared) {
  if (p.mode == SKETCH_MODE_REGEN) {
    RegenArgs a{};
    a.m = static_cast<int32_t>(A->m);
    a.n = static_cast<int32_t>(A->n);
    a.d = static_cast<int32_t>(h->d);
    a.dtype = A->dtype;
    a.nnz = A->nnz;
    a.colptr = A->colptr;
    a.rowidx = A->rowidx;
    a.values = A->values;
    a.Ahat = Ahat;
    a.k0 = h->k0;
    a.k1 = h->k1;
    a.stream_id = h->stream_id;
    a.dist = h->dist;
    a.q_tiles = p.q_tiles;
    a.split = p.split;
    a.status = status;
    a.gen_count = gen;
    cudaError_t e = launch_regen(a, s);
    h->launches += 1;
    return e == cudaSuccess ? SKETCH_OK : cuda_fail(h, e, "regen kernel");
  }
  if (p.mode == SKETCH_MODE_TILE) {
    TileArgs a{};
    a.m = static_cast<int32_t>(A->m);
    a.n = static_cast<int32_t>(A->n);
    a.d = static_cast<int32_t>(h->d);
    a.nnz = A->nnz;
    a.dtype = A->dtype;
    a.colptr = A->colptr;
    a.rowidx = A->rowidx;
    a.values = A->values;
    a.Ahat = Ahat;
    a.k0 = h->k0;
    a.k1 = h->k1;
    a.stream_id = h->stream_id;
    a.dist = h->dist;
    a.R = p.panel_rows;
    // register sums: at most one row group per panel; tensor-memory sums:
    // the shares the workspace was sized for (an empty share does nothing)
    a.G = std::min<int32_t>(p.row_groups,
                            static_cast<int32_t>((A->m + p.panel_rows - 1) / p.panel_rows));
    a.cpw = p.cols_per_warp;
    a.tacc = p.tile_acc;
    a.status = status;
    a.gen_count = gen;
    a.prepared = prepared ? 1 : 0;
    int nl = 0;
    cudaError_t e = launch_tile(a, ws, s, &nl);
    h->launches += nl;
    return e == cudaSuccess ? SKETCH_OK : cuda_fail(h, e, "tile kernel");
  }
  // PANEL
  CsrView csr{};
  int nl = 0;
  cudaError_t e = build_csr(static_cast<int32_t>(A->m), static_cast<int32_t>(A->n),
                            A->nnz, A->colptr, A->rowidx, A->values, A->dtype, ws,
                            &csr, status, s, &nl);
  if (e != cudaSuccess) return cuda_fail(h, e, "csr build");
  PanelArgs a{};
  a.m = static_cast<int32_t>(A->m);
  a.n = static_cast<int32_t>(A->n);
  a.d = static_cast<int32_t>(h->d);
  a.csr = csr;
  a.partial = reinterpret_cast<float*>(
      static_cast<char*>(ws) + align256(csr_workspace_bytes(A->m, A->nnz)));
  a.Ahat = Ahat;
  a.k0 = h->k0;
  a.k1 = h->k1;
  a.stream_id = h->stream_id;
  a.dist = h->dist;
  a.n_block = p.n_block;
  a.row_groups = p.row_groups;
  a.gen_count = gen;
  e = launch_panel(a, s, &nl);
  h->launches += nl;
  return e == cudaSuccess ? SKETCH_OK : cuda_fail(h, e, "panel kernel");
}

// Candidate plans for the tuner.
static std::vector<sketch_plan> candidates(const sketch_s* h, const sketch_csc* A) {
  std::vector<sketch_plan> c;
  const int qmax = static_cast<int>(std::min<int64_t>(4, (h->d + 127) / 128));
  for (int q : {qmax, std::max(1, qmax / 2)}) {
    for (int sp : {1, 2, 4, 8}) {
      sketch_plan p{};
      p.mode = SKETCH_MODE_REGEN;
      p.q_tiles = q;
      p.split = sp;
      bool dup = false;
      for (auto& o : c)
        if (o.mode == p.mode && o.q_tiles == p.q_tiles && o.split == p.split) dup = true;
      if (!dup) c.push_back(p);
    }
  }
  // TILE panel heights (the S tile takes R * 128 bytes of shared memory):
  // register sums at 1024 and 512 rows, and for n > 256 the tensor-memory
  // sums (32 warps per CTA) at 1248 and 1024
  for (auto [R, tacc] : {std::pair<int32_t, int32_t>{1024, 0}, {512, 0}, {1248, 1}, {1024, 1}}) {
    sketch_plan p = tile_plan(h, A, R, tacc);
    if (p.tile_acc != tacc) continue;
    if (tile_workspace_bytes(A->m, A->n, h->d, A->nnz, R, p.row_groups, p.tile_acc) <=
        (size_t(8) << 30))
      c.push_back(p);
  }
  // +-1 S: densified panels on the tensor cores for rows holding at least
  // half, a fifth, a tenth or a sixteenth of the columns, or 32 nonzeros
  // (REGEN for the rest): the heavy rows of a skewed matrix (Sec. 3.1's
  // large-density case).  With no such row a candidate costs its base plan
  // plus the row count, so it only wins when there are dense-enough rows.
  if (h->dist == SKETCH_PM1 && A->n >= 64) {
    const double avg_col = A->n > 0 ? double(A->nnz) / double(A->n) : 0.0;
    std::vector<int32_t> taus;
    for (int64_t t : {A->n / 2, A->n / 5, A->n / 10, A->n / 16, int64_t(32)})
      if (t >= 16 && std::find(taus.begin(), taus.end(), static_cast<int32_t>(t)) == taus.end())
        taus.push_back(static_cast<int32_t>(t));
    for (int32_t tau : taus) {
      sketch_plan p{};
      p.mode = SKETCH_MODE_REGEN;
      p.q_tiles = qmax;
      p.split = avg_col >= 4096 ? 8 : avg_col >= 1024 ? 4 : avg_col >= 256 ? 2 : 1;
      p.tc_min_row_nnz = tau;
      c.push_back(p);
    }
  }
  // PANEL (shared-memory atomics, order-dependent at the last bit) is not a
  // candidate: every plan the tuner picks is deterministic.
  return c;
}

// The in-memory plan cache key: the shape and the addresses of A's arrays,
// so two matrices of one shape but different patterns tune separately (a
// caller that rewrites A in place with another pattern resets the cache
// with sketch_set_autotune).
uint64_t shape_key(const sketch_s* h, const sketch_csc* A) {
  uint64_t k = 1469598103934665603ULL;
  auto mix = [&](uint64_t v) { k = (k ^ v) * 1099511628211ULL; };
  mix(A->m); mix(A->n); mix(A->nnz); mix(h->d); mix(h->dist); mix(A->dtype);
  mix(reinterpret_cast<uintptr_t>(A->colptr));
  mix(reinterpret_cast<uintptr_t>(A->rowidx));
  mix(reinterpret_cast<uintptr_t>(A->values));
  return k;
}

// Pattern features measured on the device when a plan is tuned.
struct Features {
  int64_t nonempty = 0, max_row = 0, heavy_nnz = 0, max_col = 0;
};

static bool measure_features(sketch_t h, const sketch_csc* A, cudaStream_t s, Features* f) {
  int32_t* cnt = nullptr;
  unsigned long long* dev = nullptr;
  if (cudaMalloc(&cnt, sizeof(int32_t) * std::max<int64_t>(1, A->m)) != cudaSuccess ||
      cudaMalloc(&dev, 4 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(cnt);
    cudaGetLastError();
    return false;
  }
  unsigned long long host[4] = {};
  cudaError_t e = pattern_features(static_cast<int32_t>(A->m), static_cast<int32_t>(A->n),
                                   A->nnz, A->colptr, A->rowidx, cnt, dev,
                                   reinterpret_cast<int*>(h->d_small), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, dev, sizeof(host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(cnt);
  cudaFree(dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  h->launches += 3;
  f->nonempty = static_cast<int64_t>(host[0]);
  f->max_row = static_cast<int64_t>(host[1]);
  f->heavy_nnz = static_cast<int64_t>(host[2]);
  f->max_col = static_cast<int64_t>(host[3]);
  return true;
}

// The persisted plan cache key: shape plus quantised pattern features
// (nonempty-row share and heavy-row share in 1/32 steps, longest row and
// column in powers of two), valid across processes.
static uint64_t feature_key(const sketch_s* h, const sketch_csc* A, const Features& f) {
  uint64_t k = 0x9E3779B97F4A7C15ULL;
  auto mix = [&](uint64_t v) { k = (k ^ v) * 1099511628211ULL; };
  auto lg = [](int64_t v) { int b = 0; while (v > 1) { v >>= 1; ++b; } return b; };
  mix(A->m); mix(A->n); mix(A->nnz); mix(h->d); mix(h->dist); mix(A->dtype);
  mix(static_cast<uint64_t>(32 * f.nonempty / std::max<int64_t>(1, A->m)));
  mix(static_cast<uint64_t>(32 * f.heavy_nnz / std::max<int64_t>(1, A->nnz)));
  mix(static_cast<uint64_t>(lg(f.max_row)));
  mix(static_cast<uint64_t>(lg(f.max_col)));
  mix(5);  // version of the plan set (5: tensor-memory TILE phases)
  return k;
}

// Persisted plans (the file named by SKETCH_PLAN_CACHE, one plan per line:
// key in hex, then the ten plan fields), loaded once per process.
static std::mutex g_cache_mu;
static std::map<uint64_t, sketch_plan> g_cache;
static bool g_cache_loaded = false;

static const char* cache_path() {
  const char* p = std::getenv("SKETCH_PLAN_CACHE");
  return (p && p[0]) ? p : nullptr;
}

static bool cache_lookup(uint64_t key, sketch_plan* out) {
  const char* path = cache_path();
  if (!path) return false;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  if (!g_cache_loaded) {
    g_cache_loaded = true;
    if (FILE* f = std::fopen(path, "r")) {
      unsigned long long k = 0;
      sketch_plan p{};
      while (std::fscanf(f, "%llx %d %d %d %d %d %d %d %d %d %d", &k, &p.mode, &p.q_tiles,
                         &p.split, &p.n_block, &p.row_groups, &p.panel_rows, &p.cols_per_warp,
                         &p.tc_min_row_nnz, &p.tile_acc, &p.tc_fp8) == 11)
        g_cache[k] = p;
      std::fclose(f);
    }
  }
  auto it = g_cache.find(key);
  if (it == g_cache.end()) return false;
  *out = it->second;
  return true;
}

static void cache_store(uint64_t key, const sketch_plan& p) {
  const char* path = cache_path();
  if (!path) return;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  g_cache[key] = p;
  if (FILE* f = std::fopen(path, "a")) {
    std::fprintf(f, "%llx %d %d %d %d %d %d %d %d %d %d\n",
                 static_cast<unsigned long long>(key), p.mode, p.q_tiles, p.split, p.n_block,
                 p.row_groups, p.panel_rows, p.cols_per_warp, p.tc_min_row_nnz, p.tile_acc,
                 p.tc_fp8);
    std::fclose(f);
  }
}

// A cost model in the spirit of Sec. 3.1, used to order and prune the
// tuner's candidates (every kept candidate is still timed): generation at
// the generator rate of the distribution for the S entries a plan draws --
// d * nnz for Alg. 3 (REGEN), d * nonempty rows for the generate-once TILE
// -- plus d * nnz multiply-adds at the rate each kernel family reaches.
static double model_seconds(const sketch_s* h, const sketch_csc* A, const Features& f,
                            const sketch_plan& p) {
  const double gen = h->dist == SKETCH_PM1 ? 5.5e13 : h->dist == SKETCH_UNIFORM ? 1.5e12 : 6.2e11;
  const double d = static_cast<double>(h->d);
  const double nnz = static_cast<double>(A->nnz);
  double dense_share = 0.0;
  if (p.tc_min_row_nnz > 0)
    dense_share = f.max_row >= p.tc_min_row_nnz
                      ? std::min(1.0, static_cast<double>(f.heavy_nnz) / std::max(1.0, nnz))
                      : 0.0;
  const double sparse = nnz * (1.0 - dense_share);
  if (p.mode == SKETCH_MODE_TILE)
    return d * static_cast<double>(f.nonempty) / gen + d * sparse / 3.5e12;
  // REGEN: each nonzero regenerates its S column (+-1: 128 signs a block)
  const double regen = h->dist == SKETCH_PM1 ? 9.6e12 : gen;
  return d * sparse / regen + (dense_share > 0.0 ? d * nnz * dense_share / 4e13 : 0.0);
}

int choose_plan(sketch_t h, const sketch_csc* A, float* Ahat, cudaStream_t s,
                sketch_plan* out) {
  if (h->has_forced) {
    *out = h->forced;
    return SKETCH_OK;
  }
  const uint64_t key = shape_key(h, A);
  auto it = h->plans.find(key);
  if (it != h->plans.end()) {
    *out = it->second;
    // a tuned tensor-core panel needs a host read of its height, which a
    // captured stream cannot do: under capture the same plan runs without
    // the panel (same sketch, CUDA cores only)
    if (h->capturing) out->tc_min_row_nnz = 0;
    return SKETCH_OK;
  }
  const char* env = std::getenv("SKETCH_TUNE");
  const bool tune = h->autotune && !(env && env[0] == '0') && !h->capturing &&
                    Ahat != nullptr;
  if (!tune) {  // the heuristic is cheap: planned on every call, not cached
    *out = heuristic_plan(h, A);
    return SKETCH_OK;
  }
  // Pattern features (one device pass), then the persisted cache.
  Features feat{};
  const bool have_feat = measure_features(h, A, s, &feat);
  const uint64_t fkey = have_feat ? feature_key(h, A, feat) : 0;
  sketch_plan cached{};
  if (have_feat && cache_lookup(fkey, &cached) && check_plan(h, cached) == SKETCH_OK) {
    h->plans[key] = cached;
    *out = cached;
    return SKETCH_OK;
  }
  // Empirical tuning, seeded by the cost model: candidates whose predicted
  // time is more than four times the best prediction are dropped, panel
  // candidates whose threshold no row reaches are dropped, and the rest run
  // once on the real input (warm-up: workspace, caches), then twice timed,
  // keeping the faster run; the fastest candidate wins.
  auto cands = candidates(h, A);
  if (have_feat) {
    std::vector<std::pair<double, sketch_plan>> ranked;
    for (const auto& p : cands) {
      if (p.tc_min_row_nnz > 0 && feat.max_row < p.tc_min_row_nnz) continue;
      ranked.emplace_back(model_seconds(h, A, feat, p), p);
    }
    std::stable_sort(ranked.begin(), ranked.end(),
                     [](const auto& a, const auto& b) { return a.first < b.first; });
    cands.clear();
    for (const auto& r : ranked)
      if (r.first <= 4.0 * ranked.front().first) cands.push_back(r.second);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  sketch_plan best_p = heuristic_plan(h, A);
  const bool saved_counting = h->counting;
  h->counting = false;
  for (const auto& p : cands) {
    int rc = ensure_workspace(h, plan_workspace_bytes(h, A, p));
    if (rc != SKETCH_OK) {
      h->last_error.clear();
      continue;
    }
    if (run_plan(h, A, Ahat, p, h->ws, s) != SKETCH_OK) {
      cudaGetLastError();
      h->last_error.clear();
      continue;
    }
    float ms = 1e30f;
    for (int rep = 0; rep < 2 && rc == SKETCH_OK; ++rep) {
      cudaEventRecord(e0, s);
      rc = run_plan(h, A, Ahat, p, h->ws, s);
      cudaEventRecord(e1, s);
      float t = 1e30f;
      if (cudaEventSynchronize(e1) != cudaSuccess || rc != SKETCH_OK) {
        cudaGetLastError();
        rc = SKETCH_ERR_CUDA;
        break;
      }
      cudaEventElapsedTime(&t, e0, e1);
      ms = std::min(ms, t);
    }
    if (rc != SKETCH_OK) {
      h->last_error.clear();
      continue;
    }
    if (ms < best) {
      best = ms;
      best_p = p;
    }
  }
  h->counting = saved_counting;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->plans[key] = best_p;
  if (have_feat && best < 1e29f) cache_store(fkey, best_p);
  *out = best_p;
  return SKETCH_OK;
}

int check_csc_args(sketch_t h, const sketch_csc* A) {
  if (!A) return fail(h, SKETCH_ERR_ARG, "A is null");
  if (A->m != h->m || A->n != h->n)
    return fail(h, SKETCH_ERR_ARG, "A's shape differs from the handle's (m, n)");
  if (A->nnz < 0) return fail(h, SKETCH_ERR_ARG, "nnz < 0");
  if (A->nnz >= (int64_t(1) << 31))
    return fail(h, SKETCH_ERR_UNSUPPORTED, "nnz >= 2^31 (int32 indices)");
  if (A->dtype != SKETCH_F32 && A->dtype != SKETCH_BF16)
    return fail(h, SKETCH_ERR_ARG, "dtype must be SKETCH_F32 or SKETCH_BF16");
  if (!A->colptr) return fail(h, SKETCH_ERR_ARG, "colptr is null");
  if (A->nnz > 0 && (!A->rowidx || !A->values))
    return fail(h, SKETCH_ERR_ARG, "rowidx or values is null");
  return SKETCH_OK;
}

}  // namespace sk

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int sketch_create(int64_t m, int64_t n, int64_t d, int32_t dist, uint64_t seed,
                  sketch_t* out) {
  if (!out) return fail(nullptr, SKETCH_ERR_ARG, "out is null");
  *out = nullptr;
  if (m < 1 || n < 1 || d < 1 || m >= (int64_t(1) << 31) ||
      n >= (int64_t(1) << 31) || d >= (int64_t(1) << 31))
    return fail(nullptr, SKETCH_ERR_ARG, "need 1 <= m, n, d < 2^31");
  if (dist != SKETCH_PM1 && dist != SKETCH_UNIFORM && dist != SKETCH_NORMAL)
    return fail(nullptr, SKETCH_ERR_ARG, "unknown distribution");
  if (static_cast<int64_t>(n) * d >= (int64_t(1) << 40))
    return fail(nullptr, SKETCH_ERR_UNSUPPORTED, "d * n too large");
  sketch_s* h = new (std::nothrow) sketch_s();
  if (!h) return fail(nullptr, SKETCH_ERR_OOM, "host allocation failed");
  h->m = m;
  h->n = n;
  h->d = d;
  h->dist = dist;
  h->seed = seed;
  h->k0 = static_cast<uint32_t>(seed & 0xffffffffu);
  h->k1 = static_cast<uint32_t>(seed >> 32);
  *out = h;
  return SKETCH_OK;
}

int sketch_destroy(sketch_t h) {
  if (!h) return SKETCH_ERR_ARG;
  if (h->ws || h->d_small) cudaDeviceSynchronize();
  if (h->ws) cudaFree(h->ws);
  if (h->d_small) cudaFree(h->d_small);
  destroy_lsq_state(h);
  delete h;
  return SKETCH_OK;
}

int sketch_reshape(sketch_t h, int64_t m, int64_t n, int64_t d) {
  if (!h) return fail(nullptr, SKETCH_ERR_ARG, "handle is null");
  if (m < 1 || n < 1 || d < 1 || m >= (int64_t(1) << 31) ||
      n >= (int64_t(1) << 31) || d >= (int64_t(1) << 31))
    return fail(h, SKETCH_ERR_ARG, "need 1 <= m, n, d < 2^31");
  if (n * d >= (int64_t(1) << 40)) return fail(h, SKETCH_ERR_UNSUPPORTED, "d * n too large");
  h->m = m;
  h->n = n;
  h->d = d;
  return SKETCH_OK;
}

int sketch_set_autotune(sketch_t h, int32_t enable) {
  if (!h) return SKETCH_ERR_ARG;
  h->autotune = enable != 0;
  h->plans.clear();  // the next apply plans (and, when on, tunes) afresh
  return SKETCH_OK;
}

int sketch_set_stream_id(sketch_t h, uint32_t stream_id) {
  if (!h) return SKETCH_ERR_ARG;
  h->stream_id = stream_id;
  return SKETCH_OK;
}

int sketch_set_plan(sketch_t h, const sketch_plan* plan) {
  if (!h || !plan) return fail(h, SKETCH_ERR_ARG, "null argument");
  int rc = check_plan(h, *plan);
  if (rc != SKETCH_OK) return rc;
  if (plan->mode == SKETCH_MODE_AUTO) {
    h->has_forced = false;
  } else {
    h->forced = *plan;
    h->has_forced = true;
  }
  return SKETCH_OK;
}

int sketch_get_plan(sketch_t h, const sketch_csc* A, sketch_plan* out,
                    sketch_stream_t stream) {
  if (!h || !out) return fail(h, SKETCH_ERR_ARG, "null argument");
  int rc = check_csc_args(h, A);
  if (rc != SKETCH_OK) return rc;
  if (h->has_forced) {
    *out = h->forced;
    return SKETCH_OK;
  }
  auto it = h->plans.find(sk::shape_key(h, A));
  if (it != h->plans.end()) {
    *out = it->second;
    return SKETCH_OK;
  }
  (void)stream;
  *out = heuristic_plan(h, A);
  return SKETCH_OK;
}

int sketch_apply(sketch_t h, const sketch_csc* A, float* Ahat,
                 sketch_stream_t stream) {
  if (!h) return fail(nullptr, SKETCH_ERR_ARG, "handle is null");
  if (!Ahat) return fail(h, SKETCH_ERR_ARG, "Ahat is null");
  int rc = check_csc_args(h, A);
  if (rc != SKETCH_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusNone;
  }
  h->capturing = (cs != cudaStreamCaptureStatusNone);
  if ((rc = ensure_small(h)) != SKETCH_OK) return rc;
  sketch_plan p{};
  if ((rc = choose_plan(h, A, Ahat, s, &p)) != SKETCH_OK) return rc;
  if ((rc = ensure_workspace(h, plan_workspace_bytes(h, A, p))) != SKETCH_OK)
    return rc;
  return run_plan(h, A, Ahat, p, h->ws, s);
}

static int check_S_mem(sketch_t h, const float* S, int64_t ld_s) {
  if (!S) return fail(h, SKETCH_ERR_ARG, "S is null");
  if (ld_s < h->d || ld_s % 4 != 0)
    return fail(h, SKETCH_ERR_ARG, "ld_s must be >= d and a multiple of 4");
  if (reinterpret_cast<uintptr_t>(S) % 16 != 0)
    return fail(h, SKETCH_ERR_ARG, "S must be 16-byte aligned");
  return SKETCH_OK;
}

int sketch_generate_S(sketch_t h, float* S, int64_t ld_s, sketch_stream_t stream) {
  if (!h) return fail(nullptr, SKETCH_ERR_ARG, "handle is null");
  int rc = check_S_mem(h, S, ld_s);
  if (rc != SKETCH_OK) return rc;
  cudaError_t e = launch_generate_S(h->dist, h->k0, h->k1, h->stream_id,
                                    static_cast<int32_t>(h->d), static_cast<int32_t>(h->m), S,
                                    ld_s, reinterpret_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) h->launches += 1;
  return e == cudaSuccess ? SKETCH_OK : cuda_fail(h, e, "generate_S");
}

int sketch_apply_pregen(sketch_t h, const sketch_csc* A, const float* S, int64_t ld_s,
                        float* Ahat, sketch_stream_t stream) {
  if (!h) return fail(nullptr, SKETCH_ERR_ARG, "handle is null");
  if (!Ahat) return fail(h, SKETCH_ERR_ARG, "Ahat is null");
  int rc = check_csc_args(h, A);
  if (rc != SKETCH_OK) return rc;
  if ((rc = check_S_mem(h, S, ld_s)) != SKETCH_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if ((rc = ensure_small(h)) != SKETCH_OK) return rc;
  if (A->n == 0) return SKETCH_OK;
  if (A->nnz == 0) {
    cudaError_t e = cudaMemsetAsync(Ahat, 0, sizeof(float) * A->n * h->d, s);
    return e == cudaSuccess ? SKETCH_OK : cuda_fail(h, e, "cudaMemsetAsync");
  }
  // a forced TILE plan with tensor-memory sums sets R and the row groups;
  // otherwise panels of 1248 rows
  sketch_plan p{};
  if (h->has_forced && h->forced.mode == SKETCH_MODE_TILE && h->forced.tile_acc == 1) {
    p = h->forced;
  } else {
    p = tile_plan(h, A, 1248, 1);
    p.tile_acc = 1;
    p.cols_per_warp = 32;
  }
  if ((rc = ensure_workspace(h, plan_workspace_bytes(h, A, p))) != SKETCH_OK) return rc;
  TileArgs a{};
  a.m = static_cast<int32_t>(A->m);
  a.n = static_cast<int32_t>(A->n);
  a.d = static_cast<int32_t>(h->d);
  a.nnz = A->nnz;
  a.dtype = A->dtype;
  a.colptr = A->colptr;
  a.rowidx = A->rowidx;
  a.values = A->values;
  a.Ahat = Ahat;
  a.k0 = h->k0;
  a.k1 = h->k1;
  a.stream_id = h->stream_id;
  a.dist = 3;  // S from memory
  a.R = p.panel_rows;
  a.G = std::min<int32_t>(p.row_groups,
                          static_cast<int32_t>((A->m + p.panel_rows - 1) / p.panel_rows));
  a.cpw = 32;
  a.tacc = 1;
  a.status = reinterpret_cast<int*>(h->d_small);
  a.gen_count = nullptr;
  a.S_mem = S;
  a.ld_s = ld_s;
  int nl = 0;
  h->prep.valid = false;  // the panel-major copy below replaces any prepared data
  cudaError_t e = launch_tile(a, h->ws, s, &nl);
  h->launches += nl;
  return e == cudaSuccess ? SKETCH_OK : cuda_fail(h, e, "tile kernel (S from memory)");
}

const char* sketch_last_error(sketch_t h) {
  return h ? h->last_error.c_str() : sk::g_global_error.c_str();
}

int sketch_device_status(sketch_t h, sketch_stream_t stream) {
  if (!h) return SKETCH_ERR_ARG;
  if (!h->d_small) return SKETCH_OK;
  int v = 0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&v, h->d_small, sizeof(int),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "status read");
  if (v) {
    cudaMemsetAsync(h->d_small, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    if (v & kStatusTimeout)
      return fail(h, SKETCH_ERR_TIMEOUT, "a kernel's bounded wait gave up");
    return fail(h, SKETCH_ERR_CSC, "a kernel met an out-of-range index");
  }
  return SKETCH_OK;
}

int sketch_validate_csc(const sketch_csc* A, sketch_stream_t stream) {
  if (!A || !A->colptr || A->m < 1 || A->n < 1 || A->nnz < 0)
    return fail(nullptr, SKETCH_ERR_ARG, "bad CSC descriptor");
  if (A->nnz > 0 && !A->rowidx) return fail(nullptr, SKETCH_ERR_ARG, "rowidx null");
  if (A->nnz >= (int64_t(1) << 31) || A->m >= (int64_t(1) << 31) ||
      A->n >= (int64_t(1) << 31))
    return fail(nullptr, SKETCH_ERR_UNSUPPORTED, "sizes exceed int32");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* d_status = nullptr;
  cudaError_t e = cudaMalloc(&d_status, sizeof(int));
  if (e != cudaSuccess) return fail(nullptr, SKETCH_ERR_OOM, "cudaMalloc");
  cudaMemsetAsync(d_status, 0, sizeof(int), s);
  e = launch_validate(static_cast<int32_t>(A->m), static_cast<int32_t>(A->n),
                      A->nnz, A->colptr, A->rowidx, d_status, s);
  int v = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&v, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_status);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "validate");
  return v ? fail(nullptr, SKETCH_ERR_CSC, "malformed CSC") : SKETCH_OK;
}

int sketch_debug_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out,
                        int64_t count, sketch_stream_t stream) {
  if (count < 0 || (count > 0 && (!ctr || !out)))
    return fail(nullptr, SKETCH_ERR_ARG, "bad arguments");
  cudaError_t e = launch_debug_philox(
      ctr, static_cast<uint32_t>(seed & 0xffffffffu),
      static_cast<uint32_t>(seed >> 32), out, count,
      reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SKETCH_OK : cuda_fail(nullptr, e, "debug_philox");
}

int sketch_debug_normal_pair(const uint32_t* words, float* out, int64_t count,
                             sketch_stream_t stream) {
  if (count < 0 || (count > 0 && (!words || !out)))
    return fail(nullptr, SKETCH_ERR_ARG, "bad arguments");
  cudaError_t e = launch_debug_normal_pair(words, out, count,
                                           reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SKETCH_OK : cuda_fail(nullptr, e, "debug_normal_pair");
}

int sketch_debug_wait_timeout(sketch_t h, sketch_stream_t stream) {
  if (!h) return fail(nullptr, SKETCH_ERR_ARG, "handle is null");
  int rc = ensure_small(h);
  if (rc != SKETCH_OK) return rc;
  cudaError_t e = launch_debug_wait_timeout(reinterpret_cast<int*>(h->d_small),
                                            reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SKETCH_OK : cuda_fail(h, e, "debug_wait_timeout");
}

int sketch_debug_S(int32_t dist, uint64_t seed, uint32_t stream_id,
                   const int64_t* i, const int64_t* j, float* out,
                   int64_t count, sketch_stream_t stream) {
  if (dist < 0 || dist > 2 || count < 0 || (count > 0 && (!i || !j || !out)))
    return fail(nullptr, SKETCH_ERR_ARG, "bad arguments");
  cudaError_t e = launch_debug_S(dist, static_cast<uint32_t>(seed & 0xffffffffu),
                                 static_cast<uint32_t>(seed >> 32), stream_id,
                                 i, j, out, count,
                                 reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SKETCH_OK : cuda_fail(nullptr, e, "debug_S");
}

int sketch_bench_generator(int32_t dist, uint64_t seed, int64_t threads,
                           int64_t blocks_per_thread, float* sink,
                           sketch_stream_t stream) {
  if (dist < 0 || dist > 2 || threads < 0 || blocks_per_thread < 0 ||
      (threads > 0 && !sink))
    return fail(nullptr, SKETCH_ERR_ARG, "bad arguments");
  cudaError_t e = launch_bench_generator(
      dist, static_cast<uint32_t>(seed & 0xffffffffu),
      static_cast<uint32_t>(seed >> 32), threads, blocks_per_thread, sink,
      reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SKETCH_OK : cuda_fail(nullptr, e, "bench_generator");
}

int sketch_debug_candidates(sketch_t h, const sketch_csc* A, sketch_plan* out,
                            int32_t max_plans, int32_t* count) {
  if (!h || !count || (max_plans > 0 && !out)) return fail(h, SKETCH_ERR_ARG, "null argument");
  int rc = check_csc_args(h, A);
  if (rc != SKETCH_OK) return rc;
  const std::vector<sketch_plan> c = candidates(h, A);
  *count = static_cast<int32_t>(c.size());
  for (int32_t t = 0; t < max_plans && t < static_cast<int32_t>(c.size()); ++t) out[t] = c[t];
  return SKETCH_OK;
}

int sketch_bench_fma(int64_t threads, int64_t iters, float* sink, sketch_stream_t stream) {
  if (threads < 0 || iters < 0 || (threads > 0 && !sink))
    return fail(nullptr, SKETCH_ERR_ARG, "bad arguments");
  cudaError_t e = launch_bench_fma(threads, iters, sink, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SKETCH_OK : cuda_fail(nullptr, e, "bench_fma");
}

int sketch_set_counting(sketch_t h, int32_t enable) {
  if (!h) return SKETCH_ERR_ARG;
  h->counting = enable != 0;
  return SKETCH_OK;
}

int64_t sketch_launch_count(sketch_t h) { return h ? h->launches : -1; }

int64_t sketch_generated_entries(sketch_t h, sketch_stream_t stream) {
  if (!h || !h->d_small) return 0;
  unsigned long long v = 0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&v, static_cast<char*>(h->d_small) + 64, sizeof(v),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return -1;
  return static_cast<int64_t>(v);
}

}  // extern "C"
