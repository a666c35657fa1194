// server.cpp -- continuous-batching server for sketch-and-precondition
// least-squares requests (Sec. 5.3), host-side C++.
//
// Worker threads (the "slots") each own a CUDA stream and one long-lived
// sketch handle that is reshaped per request, so its workspaces are reused.
// A request is admitted in arrival order as soon as a slot is free and its
// device footprint fits in the memory budget alongside the running requests;
// admitted requests then overlap on the GPU (separate streams).  Per-request
// device buffers use stream-ordered allocation (cudaMallocAsync), which does
// not synchronise the device.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/sketch.h"
#include "handle.h"

namespace {

struct Request {
  int64_t id = 0;
  sketch_csc A{};  // host pointers
  const double* b = nullptr;
  double* x = nullptr;
  int64_t d = 0;
  int64_t footprint = 0;
  sketch_server_result res{};
};

}  // namespace

struct sketch_server_s {
  int32_t slots = 1;
  int64_t budget = 0;
  int32_t dist = 0;
  uint64_t seed = 0;
  double gamma = 2.0, tol = 1e-10;
  int32_t maxit = 1000;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::deque<Request*> done;
  int64_t in_use = 0, next_id = 0, outstanding = 0;
  bool stopping = false;
  std::vector<std::thread> workers;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

int64_t footprint(const sketch_csc& A, int64_t d) {
  const int64_t vb = A.dtype == SKETCH_BF16 ? 2 : 4;
  const int64_t a = A.nnz * (4 + vb) + (A.n + 1) * 4;
  const int64_t vec = 8 * (A.m + A.n);
  return a + vec + static_cast<int64_t>(sk::lsq_workspace_bytes(A.m, A.n, d, A.nnz)) +
         A.nnz * 16 + 4 * d * A.n;  // sketch workspace (TILE copy, partials)
}

void worker(sketch_server_s* srv) {
  cudaSetDevice(srv->device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  sketch_t h = nullptr;
  sketch_create(1, 1, 1, srv->dist, srv->seed, &h);
  if (h) {
    sketch_set_autotune(h, 0);
    h->dependent_launch = false;  // requests overlap on separate streams
  }
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lock(srv->mu);
      srv->cv_work.wait(lock, [&] {
        if (srv->pending.empty()) return srv->stopping;
        return srv->in_use + srv->pending.front()->footprint <= srv->budget ||
               srv->in_use == 0;
      });
      if (srv->pending.empty()) break;  // stopping and nothing left
      r = srv->pending.front();
      srv->pending.pop_front();
      srv->in_use += r->footprint;
    }
    r->res.t_start = srv->now();
    int rc = h ? SKETCH_OK : SKETCH_ERR_OOM;
    const sketch_csc& A = r->A;
    const int64_t vb = A.dtype == SKETCH_BF16 ? 2 : 4;
    int32_t *colptr = nullptr, *rowidx = nullptr;
    void* vals = nullptr;
    double *b = nullptr, *x = nullptr;
    if (rc == SKETCH_OK &&
        (cudaMallocAsync(reinterpret_cast<void**>(&colptr), 4 * (A.n + 1), s) != cudaSuccess ||
         cudaMallocAsync(reinterpret_cast<void**>(&rowidx), 4 * std::max<int64_t>(1, A.nnz), s) != cudaSuccess ||
         cudaMallocAsync(&vals, vb * std::max<int64_t>(1, A.nnz), s) != cudaSuccess ||
         cudaMallocAsync(reinterpret_cast<void**>(&b), 8 * A.m, s) != cudaSuccess ||
         cudaMallocAsync(reinterpret_cast<void**>(&x), 8 * A.n, s) != cudaSuccess)) {
      cudaGetLastError();
      rc = SKETCH_ERR_OOM;
    }
    if (rc == SKETCH_OK) {
      cudaMemcpyAsync(colptr, A.colptr, 4 * (A.n + 1), cudaMemcpyHostToDevice, s);
      if (A.nnz > 0) {
        cudaMemcpyAsync(rowidx, A.rowidx, 4 * A.nnz, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(vals, A.values, vb * A.nnz, cudaMemcpyHostToDevice, s);
      }
      cudaMemcpyAsync(b, r->b, 8 * A.m, cudaMemcpyHostToDevice, s);
      sketch_csc dA{A.m, A.n, A.nnz, colptr, rowidx, vals, A.dtype};
      rc = sketch_reshape(h, A.m, A.n, r->d);
      sketch_lsq_info info{};
      if (rc == SKETCH_OK)
        rc = sketch_lsq_solve(h, &dA, b, x, srv->tol, srv->maxit, &info,
                              reinterpret_cast<sketch_stream_t>(s));
      if (rc == SKETCH_OK || rc == SKETCH_ERR_NO_CONVERGENCE)
        cudaMemcpyAsync(r->x, x, 8 * A.n, cudaMemcpyDeviceToHost, s);
      r->res.iters = info.iters;
      r->res.error = info.error;
    }
    cudaFreeAsync(colptr, s);
    cudaFreeAsync(rowidx, s);
    cudaFreeAsync(vals, s);
    cudaFreeAsync(b, s);
    cudaFreeAsync(x, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == SKETCH_OK) rc = SKETCH_ERR_CUDA;
    r->res.status = rc;
    r->res.t_done = srv->now();
    {
      std::lock_guard<std::mutex> lock(srv->mu);
      srv->in_use -= r->footprint;
      srv->done.push_back(r);
      --srv->outstanding;
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();  // memory was freed
  }
  if (h) sketch_destroy(h);
  cudaStreamDestroy(s);
}

}  // namespace

extern "C" {

int sketch_server_create(int32_t slots, int64_t mem_budget_bytes, int32_t dist,
                         uint64_t seed, double d_over_n, double tol,
                         int32_t maxit, sketch_server_t* out) {
  if (!out) return sk::fail(nullptr, SKETCH_ERR_ARG, "out is null");
  *out = nullptr;
  if (slots < 1 || slots > 256 || mem_budget_bytes <= 0 || d_over_n < 1.0 ||
      !(tol > 0.0) || maxit < 1 || dist < 0 || dist > 2)
    return sk::fail(nullptr, SKETCH_ERR_ARG, "bad server arguments");
  sketch_server_s* srv = new (std::nothrow) sketch_server_s();
  if (!srv) return sk::fail(nullptr, SKETCH_ERR_OOM, "host allocation failed");
  srv->slots = slots;
  srv->budget = mem_budget_bytes;
  srv->dist = dist;
  srv->seed = seed;
  srv->gamma = d_over_n;
  srv->tol = tol;
  srv->maxit = maxit;
  cudaGetDevice(&srv->device);
  srv->t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < slots; ++i) srv->workers.emplace_back(worker, srv);
  *out = srv;
  return SKETCH_OK;
}

int sketch_server_submit(sketch_server_t srv, const sketch_csc* A,
                         const double* b, double* x, int64_t* id) {
  if (!srv || !A || !b || !x || !A->colptr || A->m < 1 || A->n < 1 || A->m < A->n ||
      A->nnz < 0 || (A->nnz > 0 && (!A->rowidx || !A->values)) ||
      (A->dtype != SKETCH_F32 && A->dtype != SKETCH_BF16))
    return sk::fail(nullptr, SKETCH_ERR_ARG, "bad request");
  Request* r = new (std::nothrow) Request();
  if (!r) return sk::fail(nullptr, SKETCH_ERR_OOM, "host allocation failed");
  r->A = *A;
  r->b = b;
  r->x = x;
  r->d = static_cast<int64_t>(std::ceil(srv->gamma * static_cast<double>(A->n)));
  r->footprint = footprint(*A, r->d);
  r->res.t_submit = srv->now();
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    if (srv->stopping) {
      delete r;
      return sk::fail(nullptr, SKETCH_ERR_ARG, "server is stopping");
    }
    r->id = r->res.id = srv->next_id++;
    if (id) *id = r->id;
    ++srv->outstanding;
    if (r->footprint > srv->budget) {  // can never be admitted
      r->res.status = SKETCH_ERR_OOM;
      r->res.t_start = r->res.t_done = srv->now();
      srv->done.push_back(r);
      --srv->outstanding;
      srv->cv_done.notify_all();
      return SKETCH_OK;
    }
    srv->pending.push_back(r);
  }
  srv->cv_work.notify_one();
  return SKETCH_OK;
}

int sketch_server_poll(sketch_server_t srv, sketch_server_result* out,
                       int32_t max_results, int32_t* n_out, int32_t wait_ms) {
  if (!srv || !n_out || (max_results > 0 && !out)) return SKETCH_ERR_ARG;
  std::unique_lock<std::mutex> lock(srv->mu);
  if (srv->done.empty() && wait_ms > 0)
    srv->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms),
                          [&] { return !srv->done.empty(); });
  int32_t k = 0;
  while (k < max_results && !srv->done.empty()) {
    Request* r = srv->done.front();
    srv->done.pop_front();
    out[k++] = r->res;
    delete r;
  }
  *n_out = k;
  return SKETCH_OK;
}

int sketch_server_drain(sketch_server_t srv) {
  if (!srv) return SKETCH_ERR_ARG;
  std::unique_lock<std::mutex> lock(srv->mu);
  srv->cv_done.wait(lock, [&] { return srv->outstanding == 0; });
  return SKETCH_OK;
}

double sketch_server_now(sketch_server_t srv) { return srv ? srv->now() : 0.0; }

int sketch_server_destroy(sketch_server_t srv) {
  if (!srv) return SKETCH_ERR_ARG;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->stopping = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  for (Request* r : srv->done) delete r;
  delete srv;
  return SKETCH_OK;
}

}  // extern "C"
