// batch.cu -- many uneven sketches in one persistent launch (C ABI).
//
// sketch_batch_create builds, once, a device work list of (instance, column,
// tile of S rows) items over all instances, sorted by decreasing nonzero
// count so that the longest items start first, and tunes the tile height on
// the real batch.  sketch_batch_apply is one counter reset plus one
// persistent kernel launch, so it can be captured in a CUDA graph and
// replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "handle.h"
#include "internal.h"

struct sketch_batch_s {
  int32_t count = 0, dist = 0, q_tiles = 4, blocks = 1;
  sk::BatchInstance* d_inst = nullptr;
  sk::BatchItem* d_items = nullptr;
  int64_t n_items = 0;
  void* d_small = nullptr;  // counter at 0, status at 64
  int64_t launches = 0;
  std::string last_error;
};

namespace {

int bfail(sketch_batch_t b, int code, const std::string& msg) {
  if (b) b->last_error = msg;
  return sk::fail(nullptr, code, msg);
}

void free_batch(sketch_batch_t b) {
  if (!b) return;
  cudaFree(b->d_inst);
  cudaFree(b->d_items);
  cudaFree(b->d_small);
  delete b;
}

// Items for tile height 128 * q, longest columns first.
std::vector<sk::BatchItem> make_items(const std::vector<std::vector<int32_t>>& colptrs,
                                      const std::vector<sk::BatchInstance>& inst, int q) {
  struct Keyed {
    int32_t len;
    sk::BatchItem it;
  };
  std::vector<Keyed> v;
  const int TD = 128 * q;
  for (size_t i = 0; i < inst.size(); ++i) {
    const int tiles = (inst[i].d + TD - 1) / TD;
    for (int32_t k = 0; k < inst[i].n; ++k) {
      const int32_t len = colptrs[i][k + 1] - colptrs[i][k];
      // empty columns keep their items so their tiles are written (zeros)
      for (int t = 0; t < tiles; ++t)
        v.push_back({len, {static_cast<int32_t>(i), k, t, 0}});
    }
  }
  std::stable_sort(v.begin(), v.end(), [](const Keyed& a, const Keyed& b) {
    return a.len > b.len;
  });
  std::vector<sk::BatchItem> out(v.size());
  for (size_t t = 0; t < v.size(); ++t) out[t] = v[t].it;
  return out;
}

}  // namespace

extern "C" {

int sketch_batch_create(int32_t count, const sketch_t* handles,
                        const sketch_csc* As, float* const* Ahats,
                        sketch_stream_t stream, sketch_batch_t* out) {
  if (!out) return sk::fail(nullptr, SKETCH_ERR_ARG, "out is null");
  *out = nullptr;
  if (count < 1 || !handles || !As || !Ahats)
    return sk::fail(nullptr, SKETCH_ERR_ARG, "bad batch arguments");
  const int32_t dist = handles[0] ? handles[0]->dist : -1;
  std::vector<sk::BatchInstance> inst(count);
  std::vector<std::vector<int32_t>> colptrs(count);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int32_t i = 0; i < count; ++i) {
    sketch_t h = handles[i];
    if (!h) return sk::fail(nullptr, SKETCH_ERR_ARG, "null handle in batch");
    if (h->dist != dist)
      return sk::fail(nullptr, SKETCH_ERR_UNSUPPORTED,
                      "all instances of a batch need the same distribution");
    int rc = sk::check_csc_args(h, &As[i]);
    if (rc != SKETCH_OK) return sk::fail(nullptr, rc, h->last_error);
    if (!Ahats[i]) return sk::fail(nullptr, SKETCH_ERR_ARG, "null A_hat in batch");
    colptrs[i].resize(As[i].n + 1);
    if (cudaMemcpyAsync(colptrs[i].data(), As[i].colptr, sizeof(int32_t) * (As[i].n + 1),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return sk::fail(nullptr, SKETCH_ERR_CUDA, "reading colptr");
    inst[i] = {As[i].colptr, As[i].rowidx, As[i].values, Ahats[i],
               static_cast<int32_t>(As[i].m), static_cast<int32_t>(As[i].n),
               static_cast<int32_t>(h->d), As[i].dtype, h->k0, h->k1, h->stream_id, 0};
  }
  if (cudaStreamSynchronize(s) != cudaSuccess)
    return sk::fail(nullptr, SKETCH_ERR_CUDA, "reading colptr");
  // the work list and the persistent kernel walk these column ranges: they
  // must start at 0, never decrease and end at nnz
  for (int32_t i = 0; i < count; ++i) {
    const std::vector<int32_t>& cp = colptrs[i];
    bool ok = cp[0] == 0 && cp[As[i].n] == As[i].nnz;
    for (int64_t k = 0; ok && k < As[i].n; ++k) ok = cp[k] <= cp[k + 1];
    if (!ok) return sk::fail(nullptr, SKETCH_ERR_CSC, "malformed colptr in batch instance");
  }

  sketch_batch_t b = new (std::nothrow) sketch_batch_s();
  if (!b) return sk::fail(nullptr, SKETCH_ERR_OOM, "host allocation failed");
  b->count = count;
  b->dist = dist;
  if (cudaMalloc(&b->d_inst, sizeof(sk::BatchInstance) * count) != cudaSuccess ||
      cudaMalloc(&b->d_small, 256) != cudaSuccess) {
    free_batch(b);
    return sk::fail(nullptr, SKETCH_ERR_OOM, "cudaMalloc failed");
  }
  cudaMemcpy(b->d_inst, inst.data(), sizeof(sk::BatchInstance) * count,
             cudaMemcpyHostToDevice);
  cudaMemset(b->d_small, 0, 256);
  auto* counter = static_cast<unsigned long long*>(b->d_small);
  int* status = reinterpret_cast<int*>(static_cast<char*>(b->d_small) + 64);

  // tune the tile height on the real batch: time one launch per candidate
  int best_q = 4;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int dmax = 0;
  for (auto& x : inst) dmax = std::max(dmax, x.d);
  std::vector<int> qs = {4, 2, 1};
  for (int q : qs) {
    if (q > 1 && 128 * (q / 2) >= dmax) continue;  // tiles larger than any d
    std::vector<sk::BatchItem> items = make_items(colptrs, inst, q);
    sk::BatchItem* d_items = nullptr;
    if (cudaMalloc(&d_items, sizeof(sk::BatchItem) * std::max<size_t>(1, items.size())) !=
        cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaMemcpy(d_items, items.data(), sizeof(sk::BatchItem) * items.size(),
               cudaMemcpyHostToDevice);
    const int blocks = sk::num_sms() * sk::batched_blocks_per_sm(dist, q);
    float ms = 1e30f;
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {
      cudaEventRecord(e0, s);
      ok = sk::launch_regen_batched(dist, q, b->d_inst, d_items,
                                    static_cast<int64_t>(items.size()), counter, status,
                                    blocks, s) == cudaSuccess;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
      if (ok) cudaEventElapsedTime(&ms, e0, e1);
    }
    if (ok && ms < best_ms) {
      best_ms = ms;
      best_q = q;
      cudaFree(b->d_items);
      b->d_items = d_items;
      b->n_items = static_cast<int64_t>(items.size());
      b->blocks = blocks;
    } else {
      cudaFree(d_items);
    }
    cudaGetLastError();
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!b->d_items) {
    free_batch(b);
    return sk::fail(nullptr, SKETCH_ERR_CUDA, "no batched plan could run");
  }
  b->q_tiles = best_q;
  cudaMemset(status, 0, sizeof(int));
  *out = b;
  return SKETCH_OK;
}

int sketch_batch_apply(sketch_batch_t b, sketch_stream_t stream) {
  if (!b) return sk::fail(nullptr, SKETCH_ERR_ARG, "batch is null");
  auto* counter = static_cast<unsigned long long*>(b->d_small);
  int* status = reinterpret_cast<int*>(static_cast<char*>(b->d_small) + 64);
  cudaError_t e = sk::launch_regen_batched(b->dist, b->q_tiles, b->d_inst, b->d_items,
                                           b->n_items, counter, status, b->blocks,
                                           reinterpret_cast<cudaStream_t>(stream));
  b->launches += 1;
  if (e != cudaSuccess) return bfail(b, SKETCH_ERR_CUDA, cudaGetErrorString(e));
  return SKETCH_OK;
}

int sketch_batch_info(sketch_batch_t b, int32_t* q_tiles, int64_t* n_items,
                      int64_t* launches) {
  if (!b) return SKETCH_ERR_ARG;
  if (q_tiles) *q_tiles = b->q_tiles;
  if (n_items) *n_items = b->n_items;
  if (launches) *launches = b->launches;
  return SKETCH_OK;
}

int sketch_batch_status(sketch_batch_t b, sketch_stream_t stream) {
  if (!b) return SKETCH_ERR_ARG;
  int v = 0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* status = reinterpret_cast<int*>(static_cast<char*>(b->d_small) + 64);
  if (cudaMemcpyAsync(&v, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SKETCH_ERR_CUDA;
  return v ? SKETCH_ERR_CSC : SKETCH_OK;
}

int sketch_batch_destroy(sketch_batch_t b) {
  if (!b) return SKETCH_ERR_ARG;
  cudaDeviceSynchronize();
  free_batch(b);
  return SKETCH_OK;
}

}  // extern "C"
