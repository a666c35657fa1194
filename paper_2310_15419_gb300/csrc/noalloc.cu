// noalloc.cu -- sketch_apply_noalloc: the PANEL sketch (one row group, so it
// writes A_hat directly) with its scratch in a fixed device array instead of
// a cudaMalloc'd workspace.  Its shared-memory sums are compensated (every
// atomic add also adds its own rounding error into a second array), so a
// column summed in one piece -- up to the whole row limit -- stays within
// about one rounding of the exact result.  The atomics leave the order of the
// additions to the hardware, so the last bit of a float result can differ
// between calls; +-1 S with integer-valued A is exact in any order.
//
// Why it exists: some callers cannot let a library allocate device memory
// while they run -- e.g. a process whose device memory is entirely handed out
// by another allocator (a framework's caching pool that reserved the HBM up
// front), or a latency-critical loop in which cudaMalloc/cudaFree would
// synchronise the device.  This entry point performs no device or host
// allocation of its own: the scratch (the device CSR copy of A and the
// status word) lives in `g_noalloc_scratch` below, which every GPU that loads
// the library holds until the process exits.
//
// Limits: A may have at most kNoAllocMaxRows rows and kNoAllocMaxNnz
// nonzeros; larger inputs are rejected with SKETCH_ERR_UNSUPPORTED.
//
// Sharing: all calls in the process share the one array per device and it
// keeps the previous call's contents; the kernels clear what must start at
// zero.  Calls whose work overlaps on the GPU (e.g. on two streams at once)
// race on the array and must be serialised by the caller.
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress (the array's name is only a host-side stand-in in host
// code).  Make that first call before any stream capture begins.
#include <cuda_runtime.h>

#include <mutex>

#include "handle.h"
#include "internal.h"

namespace sk {
namespace {

constexpr int64_t kNoAllocMaxRows = int64_t(1) << 18;  // 262,144 rows of A
constexpr int64_t kNoAllocMaxNnz = int64_t(1) << 20;   // 1,048,576 nonzeros
constexpr size_t kStatusBytes = 256;
// Upper bound of csr_workspace_bytes(kNoAllocMaxRows, kNoAllocMaxNnz):
// two (m+1)-int arrays, two nnz-sized arrays, scan temporaries (checked at
// set-up against the real formula).
constexpr size_t kCsrBytes = 2 * (((kNoAllocMaxRows + 1) * 4 + 255) / 256 * 256) +
                             2 * ((kNoAllocMaxNnz * 4 + 255) / 256 * 256) +
                             64 * 1024;
constexpr size_t kNoAllocBytes = kStatusBytes + kCsrBytes;  // ~10.1 MiB

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (set up once).
int scratch_for_current_device(sketch_t h, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return fail(h, SKETCH_ERR_UNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    if (csr_workspace_bytes(kNoAllocMaxRows, kNoAllocMaxNnz) > kCsrBytes)
      return fail(h, SKETCH_ERR_UNSUPPORTED, "static scratch too small");
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return cuda_fail(h, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return SKETCH_OK;
}

}  // namespace
}  // namespace sk

using namespace sk;

extern "C" int sketch_apply_noalloc(sketch_t h, const sketch_csc* A,
                                    float* Ahat, sketch_stream_t stream) {
  if (!h) return fail(nullptr, SKETCH_ERR_ARG, "handle is null");
  if (!Ahat) return fail(h, SKETCH_ERR_ARG, "Ahat is null");
  int rc = check_csc_args(h, A);
  if (rc != SKETCH_OK) return rc;
  if (A->m > kNoAllocMaxRows || A->nnz > kNoAllocMaxNnz)
    return fail(h, SKETCH_ERR_UNSUPPORTED,
                "sketch_apply_noalloc: A exceeds 262,144 rows or 1,048,576 "
                "nonzeros (the fixed scratch size)");
  void* base = nullptr;
  if ((rc = scratch_for_current_device(h, &base)) != SKETCH_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* status = static_cast<int*>(base);
  void* csr_ws = static_cast<unsigned char*>(base) + kStatusBytes;
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync(status)");
  if (A->nnz == 0) {
    e = cudaMemsetAsync(Ahat, 0, sizeof(float) * A->n * h->d, s);
    return e == cudaSuccess ? SKETCH_OK : cuda_fail(h, e, "cudaMemsetAsync");
  }
  int launches = 0;
  CsrView csr{};
  e = build_csr(static_cast<int32_t>(A->m), static_cast<int32_t>(A->n), A->nnz,
                A->colptr, A->rowidx, A->values, A->dtype, csr_ws, &csr,
                status, s, &launches);
  if (e != cudaSuccess) return cuda_fail(h, e, "csr build (no-alloc)");
  PanelArgs a{};
  a.m = static_cast<int32_t>(A->m);
  a.n = static_cast<int32_t>(A->n);
  a.d = static_cast<int32_t>(h->d);
  a.csr = csr;
  a.partial = nullptr;  // one row group: the kernel writes A_hat directly
  a.Ahat = Ahat;
  a.k0 = h->k0;
  a.k1 = h->k1;
  a.stream_id = h->stream_id;
  a.dist = h->dist;
  // two shared-memory arrays (sums, compensation) of 32 x n_block floats
  a.n_block = static_cast<int32_t>(A->n < 768 ? A->n : 768);
  a.row_groups = 1;
  a.compensated = 1;
  a.gen_count = nullptr;
  e = launch_panel(a, s, &launches);
  h->launches += launches;
  return e == cudaSuccess ? SKETCH_OK : cuda_fail(h, e, "panel kernel (no-alloc)");
}
