// lsq.cu -- sketch-and-precondition least squares (Sec. 5.4).
#include "handle.h"

namespace sk {
struct LsqState {};
void destroy_lsq_state(sketch_t h) {
  delete h->lsq;
  h->lsq = nullptr;
}
}  // namespace sk

extern "C" int sketch_lsq_solve(sketch_t h, const sketch_csc* A,
                                const double* b, double* x, double tol,
                                int32_t maxit, sketch_lsq_info* info,
                                sketch_stream_t stream) {
  (void)A; (void)b; (void)x; (void)tol; (void)maxit; (void)info; (void)stream;
  return sk::fail(h, SKETCH_ERR_UNSUPPORTED, "not built yet");
}
