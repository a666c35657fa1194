/*
 * sketch.h -- C ABI of the GB300 (sm_103a) sketching library.
 *
 * The library computes the sketch  A_hat = S A  of arXiv 2310.15419
 * ("Fast multiplication of random dense matrices with sparse matrices"),
 * Eq. (1): A is a tall m x n sparse matrix in CSC (Sec. 1.1 takes CSC as the
 * default format) and S is a d x m matrix with iid entries from {+1,-1},
 * U(-1,1) or N(0,1) (Sec. 1.1) that is never stored: every entry is
 * regenerated on the GPU from a counter-based generator (Sec. 4.2,
 * Philox4x32-10) keyed by (seed, stream, i, j), so S is the same under any
 * tiling, launch shape or kernel choice (the reproducibility policy of
 * Sec. 4.3).  On top of the sketch it provides the sketch-and-precondition
 * least-squares solver of Sec. 5.3 (Householder QR of A_hat in FP64, LSQR on
 * A R^{-1} with FP64 vector arithmetic), a batched launch for many uneven
 * sketches, and a continuous-batching solve server.
 *
 * Definition of S(i, j), 0 <= i < d, 0 <= j < m (key = (seed lo32, seed hi32)):
 *   +-1      x = Philox4x32-10(ctr = (i >> 7, j, stream, 0)); b = i & 127;
 *            S = bit (b & 31) of x[b >> 5] ? -1 : +1
 *   U(-1,1)  x = Philox(ctr = (i >> 2, j, stream, 0)); u = x[i & 3] >> 8 as a
 *            signed 24-bit integer; S = (2u + 1) 2^-24   (exact in FP32)
 *   N(0,1)   x = Philox(ctr = (i >> 2, j, stream, 0)); p = (i & 3) >> 1;
 *            u1 = ((x[2p] >> 8) + 1) 2^-24, u2 = (x[2p+1] >> 8) 2^-24;
 *            S = sqrt(-2 ln u1) * (i odd ? sin : cos)(2 pi u2)  (Box-Muller)
 *
 * Conventions for every call:
 *   - 0-based indices, int32 colptr / rowidx (nnz < 2^31), rows strictly
 *     increasing inside each column.
 *   - Matrix pointers are DEVICE pointers owned by the caller unless a
 *     function says otherwise; dense outputs are column-major.
 *   - A_hat is d x n, column-major, leading dimension d, FP32.  It is
 *     overwritten (the paper's Alg. 1 starts from A_hat = 0).
 *   - Calls taking a stream are asynchronous on that stream (NULL = the
 *     legacy default stream) unless documented as synchronous.
 *   - Errors are returned as negative SKETCH_ERR_* codes, never thrown or
 *     aborted; sketch_last_error() gives a message for the last failure of a
 *     handle.  Out-of-range row indices met inside a kernel are skipped and
 *     recorded in a device status word (sketch_device_status).
 *   - The handle owns its workspace (device scratch, plan cache).  A handle
 *     must not be used from two host threads at once.
 */
#ifndef SKETCH_H_
#define SKETCH_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sketch_s* sketch_t;
/* Same type as cudaStream_t; declared here so this header needs no CUDA
 * header.  NULL selects the legacy default stream. */
typedef struct CUstream_st* sketch_stream_t;

enum sketch_status {
  SKETCH_OK = 0,
  SKETCH_ERR_ARG = -1,             /* bad argument (null, size, enum)        */
  SKETCH_ERR_OOM = -2,             /* device or host allocation failed       */
  SKETCH_ERR_CSC = -3,             /* malformed CSC (validator / kernels)    */
  SKETCH_ERR_CUDA = -4,            /* a CUDA runtime call failed             */
  SKETCH_ERR_TIMEOUT = -5,         /* a bounded device wait gave up          */
  SKETCH_ERR_NO_CONVERGENCE = -6,  /* LSQR reached its iteration limit       */
  SKETCH_ERR_UNSUPPORTED = -7      /* size or option outside what is built   */
};

enum sketch_dist { SKETCH_PM1 = 0, SKETCH_UNIFORM = 1, SKETCH_NORMAL = 2 };
enum sketch_dtype { SKETCH_F32 = 0, SKETCH_BF16 = 1 };

/* Kernel families (Sec. 2.2): REGEN = variant kji (Alg. 3), every nonzero
 * regenerates its column of S; PANEL = variant jki (Alg. 4), each nonempty
 * row of A generates its column of S once per tile and scatters it into the
 * row's nonzeros; TILE = the three-level blocking of Sec. 3.1's model
 * (S_sub d1 x m1 generated once, reused by every column of A_sub m1 x n1),
 * swept in CSC order.  AUTO lets the tuner choose per shape. */
enum sketch_mode {
  SKETCH_MODE_AUTO = 0,
  SKETCH_MODE_REGEN = 1,
  SKETCH_MODE_PANEL = 2,
  SKETCH_MODE_TILE = 3
};

/* A sparse m x n matrix in CSC.  All pointers are device pointers owned by
 * the caller; they must stay valid until the work using them completes. */
typedef struct {
  int64_t m, n, nnz;
  const int32_t* colptr;  /* n + 1 entries, colptr[0] = 0, colptr[n] = nnz */
  const int32_t* rowidx;  /* nnz entries, strictly increasing per column   */
  const void* values;     /* nnz entries of type `dtype`                    */
  int32_t dtype;          /* SKETCH_F32 or SKETCH_BF16                      */
} sketch_csc;

/* Launch plan (Alg. 1's block sizes mapped onto the GPU).  REGEN: each work
 * item is one column of A times a tile of 128*q_tiles rows of S; `split`
 * warps share a column's nonzeros.  PANEL: a CTA owns 32 rows of S,
 * `n_block` columns and one of `row_groups` contiguous row ranges of A.
 * TILE: S is cut into tiles of 32 rows (d1) and A into panels of
 * `panel_rows` rows (m1) and blocks of n1 columns; a CTA generates each
 * (tile, panel) block of S once and sweeps the panel's nonzeros in its
 * columns, and the panels form `row_groups` contiguous ranges.
 * tile_acc = 0: 16 warps, n1 = 16*cols_per_warp, running sums in registers;
 * a CTA takes one range of one tile, and the ranges' partial copies of A_hat
 * are added in order.  tile_acc = 1: 32 warps, cols_per_warp = 32,
 * n1 = 1024, running sums in tensor memory; one wave of CTAs (one per SM,
 * over the column blocks) walks the ranges in order, each CTA taking the
 * same share of every range's (tile, panel) blocks and adding its sums per
 * range into a scratch copy of its tiles; tiles that several CTAs share are
 * added in CTA order.  The additions per tile are those of tile_acc = 0
 * (sums within a range, then ranges in order), so where every CTA owns
 * whole tiles the two give the same bits. */
typedef struct {
  int32_t mode;          /* sketch_mode                                   */
  int32_t q_tiles;       /* REGEN: 1..4 blocks of 128 rows of S per warp  */
  int32_t split;         /* REGEN: 1, 2, 4 or 8 warps per column           */
  int32_t n_block;       /* PANEL: columns per CTA (<= 1536)               */
  int32_t row_groups;    /* PANEL, TILE: number of row ranges of A         */
  int32_t panel_rows;    /* TILE: rows of A per panel, 8..1248 (m1)        */
  int32_t cols_per_warp; /* TILE: 4, 16 or 64 (32 with tile_acc = 1)       */
  int32_t tc_min_row_nnz;/* +-1 only: rows of A with at least this many     */
                         /* nonzeros form a dense panel multiplied on the   */
                         /* tensor cores (BF16 S, A split exactly into three */
                         /* BF16 terms, FP32 accumulate); 0 = off.  Such a  */
                         /* plan reads the panel height back to the host    */
                         /* once per call (not capturable in a graph).      */
  int32_t tile_acc;      /* TILE: 0 = register, 1 = tensor-memory sums     */
  int32_t tc_fp8;        /* tensor-core panels in FP8 (1) instead of BF16   */
                         /* (0): +-1 S in E4M3 (exact) times A split into  */
                         /* two E4M3 terms after a power-of-two scale per  */
                         /* column (undone exactly on output), FP32        */
                         /* accumulate; about 2^-8 relative error per      */
                         /* value of A (integer values up to 16 in         */
                         /* magnitude stay exact), so it suits the         */
                         /* preconditioner sketch of sketch_lsq_solve      */
                         /* (Sec. 5.3) rather than the 1e-6 sketch.  The   */
                         /* tuner never picks it; a forced plan does.      */
} sketch_plan;

/* Create a sketch handle for A (m x n) and S (d x m) with the distribution
 * `dist` and the 64-bit `seed`.  Requires 1 <= d, n, m; d, n, m < 2^31.
 * Section: Sec. 1.1 (problem), Sec. 4.2 (counter-based generator).
 * Errors: SKETCH_ERR_ARG, SKETCH_ERR_OOM.  No device memory is touched. */
int sketch_create(int64_t m, int64_t n, int64_t d, int32_t dist, uint64_t seed,
                  sketch_t* out);

/* Release the handle and its device workspace (synchronises the device). */
int sketch_destroy(sketch_t h);

/* Change the handle's problem shape (m, n, d) and keep its seed,
 * distribution, stream id, options and device workspaces (which grow on
 * demand), so a long-lived handle serves a stream of differently shaped
 * problems without reallocating.  Same limits as sketch_create. */
int sketch_reshape(sketch_t h, int64_t m, int64_t n, int64_t d);

/* Autotuning on (1, default) or off (0).  Off, the planner uses its
 * heuristic plan (deterministic, no timing runs); a server does this so every
 * request of a given shape runs the same kernels alone or in a mix.  Either
 * way the handle's plan cache is cleared.
 * Tuning (the first apply of a matrix): one device pass measures A's pattern
 * (nonempty rows, longest row and column, nonzeros in rows of >= 32
 * entries); a cost model after Sec. 3.1 (S entries drawn: d * nnz for
 * Alg. 3, d * nonempty rows generate-once; multiply-adds d * nnz) orders the
 * candidate plans and drops those predicted four times slower than the best
 * prediction; the rest are timed on A and the fastest is kept, keyed by the
 * shape and the addresses of A's arrays (a caller that rewrites A in place
 * with another pattern calls this function to re-plan).  With the
 * environment variable SKETCH_PLAN_CACHE naming a file, tuned plans are also
 * appended there keyed by shape and quantised pattern features, and a later
 * process (or handle) with a matching entry uses it without timing. */
int sketch_set_autotune(sketch_t h, int32_t enable);

/* Third Philox counter word ("stream", default 0).  Instances of a batch use
 * their index, so one seed yields independent S per instance. */
int sketch_set_stream_id(sketch_t h, uint32_t stream_id);

/* Force a plan (mode != AUTO) or return to autotuning (mode == AUTO).
 * Errors: SKETCH_ERR_ARG for out-of-range fields. */
int sketch_set_plan(sketch_t h, const sketch_plan* plan);

/* The plan that sketch_apply would use for A (runs the tuner if needed;
 * synchronous when it tunes).  */
int sketch_get_plan(sketch_t h, const sketch_csc* A, sketch_plan* out,
                    sketch_stream_t stream);

/* A_hat (device, d x n, ld = d, FP32) = S A.  Eq. (1); kernels follow Alg. 3
 * (REGEN) or Alg. 4 (PANEL) with Alg. 1's outer blocking mapped to the CTA
 * grid.  Asynchronous on `stream`, except that plans deriving data from A (a
 * tensor-core panel, TILE's panel-major copy) first read a 64-bit content
 * hash of A back to the host: when it, A's array addresses, the shape, the
 * plan and the workspace equal those of the handle's previous such call and
 * no error has been flagged since, the derived data still in the workspace
 * is reused (A changed in place is recognised by its hash and rebuilt).  The
 * first call for a new shape may tune (synchronously) and may grow the
 * handle's device workspace.
 * Errors: SKETCH_ERR_ARG (null pointers, A->m/n differ from the handle,
 * dtype), SKETCH_ERR_UNSUPPORTED (nnz >= 2^31), SKETCH_ERR_OOM,
 * SKETCH_ERR_CUDA. */
int sketch_apply(sketch_t h, const sketch_csc* A, float* Ahat,
                 sketch_stream_t stream);

/* A_hat = S A like sketch_apply, but without allocating anything: for
 * callers that cannot have a library allocate device memory while they run
 * (for instance when another allocator owns the device's memory, or in a
 * latency-critical loop where cudaMalloc / cudaFree would synchronise the
 * device).  The paper has no counterpart; this is a deployment variant.
 * It always runs the PANEL kernel with a single row group (A_hat written
 * directly), and its scratch -- the device CSR copy of A -- is a fixed
 * array of about 10 MiB inside the library that every GPU loading the
 * library keeps until the process exits.  Each column is summed in one
 * piece with compensated shared-memory atomics (the sum plus the exact
 * rounding error of every addition), which keeps the 1e-6 relative error
 * bound at the row limit; the hardware picks the order of the additions, so
 * float results may differ in the last bit from call to call (+-1 S with
 * integer-valued A is exact).
 *   Limits: A->m <= 262,144 and A->nnz <= 1,048,576, otherwise
 *   SKETCH_ERR_UNSUPPORTED.
 *   Sharing: every call uses the same array and finds the previous call's
 *   contents in it (cleared where needed); calls whose work overlaps on the
 *   GPU race and must be serialised by the caller.
 *   Set-up: the first call on a device looks up the array's address; make
 *   that call before any stream capture begins.
 *   Out-of-range row indices are skipped but not reported.
 * Asynchronous on `stream`.  Errors as for sketch_apply. */
int sketch_apply_noalloc(sketch_t h, const sketch_csc* A, float* Ahat,
                         sketch_stream_t stream);

/* The "pre-generated S" method of Sec. 3.3 (Fig. percent_peak): S stored in
 * device memory instead of regenerated.  sketch_generate_S writes
 * S[j * ld_s + i] = S(i, j) for i < d, j < m -- exactly the entries the
 * sketch kernels regenerate, for the handle's distribution, seed and stream
 * id.  S is a caller-owned device buffer of ld_s * m floats; ld_s >= d, a
 * multiple of 4; S 16-byte aligned.  Asynchronous.
 * Errors: SKETCH_ERR_ARG (null S, ld_s, alignment), SKETCH_ERR_CUDA. */
int sketch_generate_S(sketch_t h, float* S, int64_t ld_s, sketch_stream_t stream);

/* A_hat = S A with S read from such a buffer: the TILE kernel with
 * tensor-memory sums, each 32-row x panel_rows tile of S copied from memory
 * (cp.async, 16 bytes a thread) where the other paths generate it.  Same
 * additions as the generated path, so the same bits.  Uses a forced TILE plan
 * with tile_acc = 1 if one is set, else panels of 1248 rows.  Same
 * requirements on S and ld_s as sketch_generate_S; same errors as
 * sketch_apply.  Asynchronous. */
int sketch_apply_pregen(sketch_t h, const sketch_csc* A, const float* S, int64_t ld_s,
                        float* Ahat, sketch_stream_t stream);

/* Message for the last error returned on this handle ("" if none). */
const char* sketch_last_error(sketch_t h);

/* Read and clear the device status word of the handle (synchronous):
 * 0, SKETCH_ERR_TIMEOUT if a kernel's bounded wait on the tensor cores gave
 * up (its output is then incomplete), or SKETCH_ERR_CSC if a kernel met a
 * row index outside [0, m) or a malformed colptr (decreasing, negative or past
 * nnz; the kernels clamp every column range to [0, nnz] and never read or
 * write outside A's arrays or their workspace, but A_hat is then not
 * meaningful).  A timeout of a tensor-core plan drains the MMAs that CTA
 * issued before it frees its tensor memory; if that drain also times out,
 * the tensor cores did not finish work in time and the caller should treat
 * the CUDA context as unreliable (destroy the handle, restart the process). */
int sketch_device_status(sketch_t h, sketch_stream_t stream);

/* Full CSC check on the device (synchronous): colptr[0] = 0, colptr
 * nondecreasing, colptr[n] = nnz, rows in [0, m) and strictly increasing in
 * each column (so no duplicates).  Returns SKETCH_OK or SKETCH_ERR_CSC. */
int sketch_validate_csc(const sketch_csc* A, sketch_stream_t stream);

/* ---- many uneven sketches in one persistent launch ---------------------- */
typedef struct sketch_batch_s* sketch_batch_t;

/* Prepare a batch: instance i computes Ahats[i] = S_i As[i] with handle
 * handles[i] (its own m, n, d and Philox stream id; all handles must share
 * one distribution).  Builds a device work list of (instance, column, tile of
 * 128*q rows of S) items sorted by decreasing nonzero count, and picks q by
 * timing each candidate once on the real batch (so it runs the batch, on
 * `stream`, synchronously).  Alg. 3's per-column work (Sec. 2.2) with
 * Alg. 1's outer blocking spread over instances.  Pointers in As / Ahats are
 * device pointers that must stay valid for the life of the batch.
 * Errors: SKETCH_ERR_ARG, SKETCH_ERR_UNSUPPORTED (mixed distributions),
 * SKETCH_ERR_CSC (a colptr that does not start at 0, decreases or does not
 * end at nnz), SKETCH_ERR_OOM, SKETCH_ERR_CUDA. */
int sketch_batch_create(int32_t count, const sketch_t* handles,
                        const sketch_csc* As, float* const* Ahats,
                        sketch_stream_t stream, sketch_batch_t* out);

/* Run the whole batch: one counter reset and one persistent kernel launch on
 * `stream` (asynchronous, no allocation, so it can be captured in a CUDA
 * graph and replayed). */
int sketch_batch_apply(sketch_batch_t b, sketch_stream_t stream);

/* Tile height chosen (q: 128*q rows of S per item), number of work items and
 * launches so far. */
int sketch_batch_info(sketch_batch_t b, int32_t* q_tiles, int64_t* n_items,
                      int64_t* launches);

/* Read and clear-free check of the batch's device status word (synchronous):
 * SKETCH_OK or SKETCH_ERR_CSC. */
int sketch_batch_status(sketch_batch_t b, sketch_stream_t stream);

int sketch_batch_destroy(sketch_batch_t b);

/* ---- least squares (Sec. 5.3, sketch-and-precondition with QR) -------- */
/* Least-squares methods of Sec. 5.3: SAP with a QR of the sketch
 * (preconditioner R^{-1}), SAP with an SVD of the sketch (singular values
 * below sigma_max(S A) / 10^12 dropped; preconditioner V_k Sigma_k^{-1}, for
 * problems with singular values near zero), and the paper's comparator
 * LSQR-D (no sketch; D_ii = 1 / ||A_i||_2, or 1 when ||A_i||_2 <= eps
 * sqrt(n) max_i ||A_i||_2 with eps = 2^-52). */
enum sketch_lsq_method {
  SKETCH_LSQ_SAP_QR = 0,
  SKETCH_LSQ_SAP_SVD = 1,
  SKETCH_LSQ_LSQR_D = 2
};

typedef struct {
  int32_t iters;        /* LSQR iterations                                 */
  int32_t status;       /* SKETCH_OK or SKETCH_ERR_NO_CONVERGENCE          */
  int32_t istop;        /* 1: ||r|| test, 2: ||M^T r|| test, 0: max iters  */
  int32_t rank;         /* columns of the preconditioner: the singular     */
                        /* values kept (SAP-SVD), else n                   */
  double error;         /* Error(x) = ||A^T(Ax-b)|| / (||A||_F ||Ax-b||)   */
  double test2;         /* LSQR's own estimate for the preconditioned system*/
  double ms_sketch, ms_qr, ms_lsqr;  /* stage times (CUDA events)          */
} sketch_lsq_info;

/* Solve min ||A x - b||_2 (m >= n): A_hat = S A with this handle's S
 * (d = the handle's d, normally 2n), FP64 Householder QR of A_hat -> R,
 * LSQR on A R^{-1} with FP64 residual and norm updates until LSQR's own
 * estimate for the preconditioned system falls below `tol` (the stopping
 * rule of Sec. 5.3), then x = R^{-1} y and Error(x) = ||A^T(Ax-b)|| /
 * (||A||_F ||Ax-b||) in FP64.  If Error(x) is still above `tol`, LSQR
 * continues from the same state with a 10x tighter internal tolerance, for
 * as long as each round at least halves Error(x) (up to 6 rounds); the
 * achieved Error(x) is returned in info->error either way (it can sit at
 * the FP64 floor of the metric for badly scaled, nearly consistent data).
 * b (m) and x (n) are FP64 device pointers.  Synchronous: returns when x
 * and *info are final.  A is checked on the device first (the checks of
 * sketch_validate_csc); a malformed A returns SKETCH_ERR_CSC before any other
 * kernel runs.  Errors: SKETCH_ERR_ARG (d < n, tol <= 0),
 * SKETCH_ERR_NO_CONVERGENCE (maxit reached; x holds the last iterate),
 * SKETCH_ERR_CSC (malformed A, or a zero column makes R singular),
 * SKETCH_ERR_OOM, SKETCH_ERR_CUDA. */
int sketch_lsq_solve(sketch_t h, const sketch_csc* A, const double* b,
                     double* x, double tol, int32_t maxit,
                     sketch_lsq_info* info, sketch_stream_t stream);

/* sketch_lsq_solve with a choice of method (sketch_lsq_method), Sec. 5.3.
 *   SKETCH_LSQ_SAP_QR: exactly sketch_lsq_solve.
 *   SKETCH_LSQ_SAP_SVD: the same sketch and QR, then the SVD of R (= the
 *     SVD of the sketch up to the left factor) by one-sided Jacobi in FP64
 *     (sweeps of round-robin column-pair rotations until a sweep rotates
 *     nothing, at most 40); singular values below sigma_max / 10^12 are
 *     dropped (info->rank = the number kept) and LSQR runs on A V_k
 *     Sigma_k^{-1}, so a rank-deficient A gives its minimum-norm
 *     least-squares solution instead of SKETCH_ERR_CSC.  n <= 4096; extra
 *     workspace 2 n^2 doubles.
 *   SKETCH_LSQ_LSQR_D: no sketch; LSQR on A D with the diagonal D above
 *     (ms_sketch = 0, ms_qr = the column norms).
 * Same arguments, synchronisation and errors as sketch_lsq_solve, plus
 * SKETCH_ERR_ARG for an unknown method and SKETCH_ERR_UNSUPPORTED for
 * SAP-SVD with n > 4096. */
int sketch_lsq_solve_method(sketch_t h, const sketch_csc* A, const double* b,
                            double* x, double tol, int32_t maxit, int32_t method,
                            sketch_lsq_info* info, sketch_stream_t stream);

/* ---- continuous-batching solve server ---------------------------------- */
typedef struct sketch_server_s* sketch_server_t;

typedef struct {
  int64_t id;        /* from sketch_server_submit                          */
  int32_t status;    /* sketch_lsq_solve's status, or SKETCH_ERR_OOM when   */
                     /* the request can never fit the memory budget         */
  int32_t iters;     /* LSQR iterations                                      */
  double error;      /* Error(x) of Sec. 5.3                                 */
  double t_submit, t_start, t_done;  /* seconds on the server's clock       */
} sketch_server_result;

/* Start a server for SAP-QR least-squares requests (Sec. 5.3): `slots`
 * worker threads, each with its own CUDA stream and a reusable sketch handle
 * (autotuning off, so a request runs the same kernels alone or in a mix).
 * A request is admitted, oldest first, as soon as a slot is free and its
 * device footprint (A, b, x, the sketch, QR and LSQR workspaces) fits in
 * `mem_budget_bytes` together with the requests already running; admitted
 * requests overlap on the GPU.  d = ceil(d_over_n * n); S is keyed by
 * (seed, stream id 0, i, j) for every request.  Errors: SKETCH_ERR_ARG,
 * SKETCH_ERR_OOM. */
int sketch_server_create(int32_t slots, int64_t mem_budget_bytes, int32_t dist,
                         uint64_t seed, double d_over_n, double tol,
                         int32_t maxit, sketch_server_t* out);

/* Queue one request.  A's arrays, b (m) and x (n) are HOST pointers that the
 * caller keeps valid until the request is returned by sketch_server_poll;
 * x receives the solution.  Returns at once with the request id. */
int sketch_server_submit(sketch_server_t srv, const sketch_csc* A,
                         const double* b, double* x, int64_t* id);

/* Move up to `max_results` completed requests into `out` (oldest first);
 * waits up to `wait_ms` milliseconds for at least one.  *n_out = number
 * returned. */
int sketch_server_poll(sketch_server_t srv, sketch_server_result* out,
                       int32_t max_results, int32_t* n_out, int32_t wait_ms);

/* Block until every submitted request has completed (they stay pollable). */
int sketch_server_drain(sketch_server_t srv);

/* Seconds since the server started (the clock of the result timestamps). */
double sketch_server_now(sketch_server_t srv);

/* Stop accepting, finish queued requests, join the workers, free all. */
int sketch_server_destroy(sketch_server_t srv);

/* ---- test hooks: the generator and S itself --------------------------- */
/* out[4t..4t+3] = Philox4x32-10(ctr[4t..4t+3], key = seed) for t < count,
 * computed with the key advanced round by round; out[4(count+t)..] holds
 * the same blocks from the ten precomputed round keys (the form the TILE
 * kernel and the generator benchmark use).  ctr (4 count words) and out
 * (8 count words) are device pointers.  Sec. 4.2.  Asynchronous. */
int sketch_debug_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out,
                        int64_t count, sketch_stream_t stream);

/* The N(0,1) transform alone: (out[2t], out[2t+1]) = Box-Muller of the word
 * pair (words[2t] radius word, words[2t+1] angle word): u1 = ((w >> 8) + 1)
 * 2^-24, u2 = (w >> 8) 2^-24, r = sqrt(-2 ln u1), (r cos 2 pi u2,
 * r sin 2 pi u2) (Sec. 4.2).  words and out are device pointers.
 * Asynchronous. */
int sketch_debug_normal_pair(const uint32_t* words, float* out, int64_t count,
                             sketch_stream_t stream);

/* The timeout path of the kernels' bounded waits, on purpose: a kernel
 * waits on an mbarrier phase that nothing completes, gives up after its
 * time limit (2 ms here; 2 s in the real kernels) and records the timeout in the
 * handle's device status word, so that sketch_device_status then returns
 * SKETCH_ERR_TIMEOUT; the context stays usable.  Asynchronous. */
int sketch_debug_wait_timeout(sketch_t h, sketch_stream_t stream);

/* out[t] = S(i[t], j[t]) (FP32) for distribution `dist`, key `seed`, counter
 * word 2 = `stream_id`.  i, j, out are device pointers.  Asynchronous. */
int sketch_debug_S(int32_t dist, uint64_t seed, uint32_t stream_id,
                   const int64_t* i, const int64_t* j, float* out,
                   int64_t count, sketch_stream_t stream);

/* Generator throughput probe: `threads` threads each evaluate
 * `blocks_per_thread` Philox blocks at distinct counters and apply the
 * distribution's transform (4 entries per block for U and N, 128 signs for
 * +-1), folding the entries' bits together with xors (no floating-point
 * work beyond the transform) into one word per thread written to sink
 * (device, `threads` floats) so nothing is optimised away.  Asynchronous.
 * Entries generated = threads * blocks_per_thread * (dist == +-1 ? 128 : 4).
 * Used to measure the RNG leg of the ALU roofline (Sec. 3.1's cost h of
 * generating one entry). */
int sketch_bench_generator(int32_t dist, uint64_t seed, int64_t threads,
                           int64_t blocks_per_thread, float* sink,
                           sketch_stream_t stream);

/* The tuner's candidate plans for A on this handle (the plans sketch_apply
 * times when it tunes), so a test can time each one itself: up to
 * `max_plans` are written to `out` (host), *count = how many there are.
 * No device work.  Errors: SKETCH_ERR_ARG. */
int sketch_debug_candidates(sketch_t h, const sketch_csc* A, sketch_plan* out,
                            int32_t max_plans, int32_t* count);

/* FP32 FMA throughput probe: `threads` threads each run `iters` rounds of
 * eight independent FMAs (x = x * a + c) and write one float to sink
 * (device, `threads` floats).  FMAs executed = threads * iters * 8.  Used to
 * show that the FMA leg of the ALU roofline (d * nnz FMAs at 128 FP32 lanes
 * per SM per clock, Sec. 3.1's cost of one multiply-add) is reachable on
 * this part.  Asynchronous. */
int sketch_bench_fma(int64_t threads, int64_t iters, float* sink, sketch_stream_t stream);

/* Householder QR of a dense d x n FP64 matrix A (device, column-major,
 * d >= n) with the kernels sketch_lsq_solve uses (Sec. 5.3): writes R
 * (n x n, ROW-major, upper triangular; R(k,k) = -sign(x_0)||x||, or x_0 when
 * the column below the diagonal is already zero) and R^{-1} (n x n,
 * row-major).  Synchronous; allocates temporary device memory. */
int sketch_debug_qr(int64_t d, int64_t n, const double* A, double* R,
                    double* Rinv, sketch_stream_t stream);

/* Number of S entries the last sketch_apply on this handle generated
 * (counted on the device when counting is enabled; synchronous read).
 * Alg. 3 generates d * nnz entries and Alg. 4 d per nonempty row and
 * column block (Sec. 3.2). */
int sketch_set_counting(sketch_t h, int32_t enable);
int64_t sketch_generated_entries(sketch_t h, sketch_stream_t stream);

/* Cumulative number of kernels this handle has launched (host counter; no
 * device access).  Lets a benchmark state how many of the library's own
 * kernels ran inside a timed region. */
int64_t sketch_launch_count(sketch_t h);

#ifdef __cplusplus
}
#endif
#endif /* SKETCH_H_ */
