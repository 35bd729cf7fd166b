/*
 * fj.h - C ABI of the GB300 Friedkin-Johnsen solver library (libfj.so).
 *
 * The library evaluates the opinion-dynamics quantities of Xu, Bao and Zhang,
 * "Fast Evaluation for Relevant Quantities of Opinion Dynamics" (WWW 2021):
 *
 *   graph    G = (V, E, w), undirected, weights w_e > 0            (Sec. 2.1)
 *   L        = D - A = B^T W B, the weighted Laplacian              (Sec. 2.1)
 *   z        = (I + L)^-1 s, the FJ equilibrium opinions     (Eq. FJmodel02)
 *   C_I      = sum_i (z_i - s_i)^2          internal conflict  (Sec. 3.2)
 *   D        = sum_{(i,j) in E} w_ij (z_i - z_j)^2 disagreement (Sec. 3.2)
 *   P        = sum_i (z_i - mean(z))^2      polarization       (Sec. 3.2)
 *   C        = sum_i z_i^2                  controversy        (Sec. 3.2)
 *   I_dc     = D + C                        disagreement-controversy index
 *
 * Algorithm 1 (APPROXIM) reduces the quantities to two Laplacian solves and
 * five squared l2 norms (Lemma PropA).  This library computes the same five
 * numbers from ONE centred solve q = (I + L)^-1 s_bar, s_bar = s - mean(s) 1:
 * because Omega 1 = 1 (Sec. 2.2), z = q + mean(s) 1 exactly, and
 *   P = ||q||^2, C = ||q + mean(s) 1||^2, C_I = ||s_bar - q||^2,
 *   D = ||W^1/2 B q||^2, I_dc = D + C.
 * The solve is Jacobi-preconditioned conjugate gradients on the GPU, with
 * float32 inner iterations refined by double-float residuals (or all
 * float64).  Each right-hand side is first scaled by an exact power of two so
 * that max |s_bar| lies in [1, 2); z and the quantities are scaled back, so
 * results hold at every finite opinion scale.
 * The paper's accuracy parameter delta (Algorithm 1, first step) is replaced
 * by a relative-residual target ||s_bar - (I + L) q||_2 <= tol ||s_bar||_2.
 *
 * Conventions for every call:
 *   - Return value: FJ_OK (0) on success, FJ_PENDING (1) from fj_poll while a
 *     request runs, a negative FJ_ERR_* code otherwise.  After an error,
 *     fj_last_error() gives a message for the calling thread.
 *   - Pointers named "host or device" are read according to the FJ_*_PTRS
 *     flag passed with them.  Device pointers must belong to the context's
 *     device.  Inputs are copied or consumed before the call returns (except
 *     where a call says otherwise); the caller keeps ownership of its buffers.
 *   - All GPU work of a context runs on the context's stream (fj_set_stream).
 *     fj_solve / fj_quantities return only after their results are written.
 *   - A context must not be used from two threads at once; distinct contexts
 *     are independent.
 */
#ifndef FJ_H
#define FJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t fj_status;

enum {
  FJ_OK = 0,
  FJ_PENDING = 1,              /* fj_poll: request not finished yet          */
  FJ_ERR_ARG = -1,             /* null pointer, n <= 0, bad size/flag        */
  FJ_ERR_GRAPH = -2,           /* node id out of range, weight <= 0/NaN/Inf  */
  FJ_ERR_OOM = -3,             /* device allocation failed                   */
  FJ_ERR_ADMIT = -4,           /* request larger than the serving budget     */
  FJ_ERR_NOT_CONVERGED = -5,   /* iteration caps reached before tol          */
  FJ_ERR_NUMERIC = -6,         /* NaN or Inf met in the iteration            */
  FJ_ERR_TIMEOUT = -7,         /* a bounded device-side wait gave up         */
  FJ_ERR_CUDA = -8,            /* a CUDA runtime call failed                 */
  FJ_ERR_TICKET = -9           /* unknown or already collected ticket        */
};

/* Where a call's pointers live. */
#define FJ_HOST_PTRS 0u
#define FJ_DEVICE_PTRS 1u
/* Upload flag: a pair listed more than once is a set of parallel edges whose
 * weights add (default: such an edge list is rejected with FJ_ERR_GRAPH). */
#define FJ_MERGE_DUPLICATES 2u
/* Solve option (fj_opts.flags, fj_solve_ex / fj_solve / fj_quantities only):
 * Algorithm 1 as printed, with two solves per opinion vector,
 * z~ = (I + L)^-1 s and q = (I + L)^-1 s_bar, and the quantities
 * C_I = ||L z~||^2, D = ||W^1/2 B q||^2, P = ||q||^2, C = ||z~||^2,
 * I_dc = D + C.  z is z~.  The default (one centred solve, z = q + mu 1)
 * gives the same values in exact arithmetic at half the work. */
#define FJ_TWO_SOLVES 4u
/* Solve option (fj_opts.flags; every solve call and fj_submit, not with
 * FJ_TWO_SOLVES or FJ_PREC_FP32): opts.tol bounds the relative error of each
 * of the five quantities against the exact solution, instead of the
 * relative residual.  The bound is certified at each float64 residual
 * evaluation from eps = ||s_bar - (I+L) q|| alone: (I+L) has no eigenvalue
 * below 1, so the error e of the iterate has ||e|| <= eps and
 * e^T L e <= eps^2; each of C_I, D, P, C is a squared norm of a vector that
 * moves with the iterate by e, its centred part or W^1/2 B e, so it is off by
 * at most eps (2 sqrt(x) + eps) where x is its value at the iterate, and
 * I_dc = D + C by the sum of two such terms.  The solve stops once every
 * such bound, relative to x minus the bound, is at most 0.9 tol (the rest
 * kept as margin for rounding); a quantity equal to zero bounds nothing.
 * In the mixed mode the first inner solve aims at 3% of opts.inner_tol
 * (3e-7 by default, about the accuracy a float32 iteration attains; tol / 10
 * if larger), the next at half the residual that would meet the bound.
 * info->rel_residual still reports the relative residual reached. */
#define FJ_QUANTITY_TOL 8u

/* Arithmetic of the solve (fj_opts.precision). */
enum {
  FJ_PREC_MIXED = 0, /* float32 PCG inner iterations, refinement residuals,
                        iterate and quantity sums in double-float (two
                        float32, ~48-bit significand): results to `tol` like
                        FP64 (default)                                       */
  FJ_PREC_FP64 = 1,  /* float64 throughout (inner iterations, residuals,
                        iterate, sums): the plain reference solve            */
  FJ_PREC_FP32 = 2   /* float32 PCG only; double-float used only for the
                        final residual and the quantity sums                 */
};

typedef struct fj_ctx fj_ctx;     /* device, stream, workspace               */
typedef struct fj_graph fj_graph; /* device-resident CSR of I + L            */

typedef struct fj_opts {
  double tol;         /* target ||s_bar - (I+L) q|| / ||s_bar|| (1e-10)      */
  double inner_tol;   /* residual reduction per float32 inner solve (1e-5)   */
  int32_t precision;  /* FJ_PREC_* (FJ_PREC_MIXED)                           */
  int32_t max_iter;   /* cap on inner iterations over the whole solve (20000)*/
  int32_t max_refine; /* cap on float64 refinement steps (12)                */
  uint32_t flags;     /* FJ_HOST_PTRS or FJ_DEVICE_PTRS for s, z; for
                         fj_submit_edges also FJ_MERGE_DUPLICATES; for
                         fj_solve_ex also FJ_TWO_SOLVES                     */
} fj_opts;

typedef struct fj_info {
  int32_t iterations;  /* inner PCG iterations (all refinement steps)        */
  int32_t refinements; /* float64 residual evaluations                       */
  double rel_residual; /* final ||s_bar-(I+L)q||/||s_bar||, max over columns */
  double device_ms;    /* device time of the solve kernels                   */
  int32_t status;      /* same as the return value of the call               */
  int32_t columns;     /* k                                                  */
  int32_t blocks;      /* thread blocks of the solve's grid (largest launch)  */
  uint32_t warnings;   /* FJ_WARN_* bits (conditions that are not errors)    */
  double t_begin_ms;   /* served requests (fj_poll): device time, in ms since
                          the serving worker started, when the request was
                          admitted (its first GPU work) ...                  */
  double t_end_ms;     /* ... and when its last GPU work ended; 0 otherwise  */
  int32_t batched;     /* served requests: 1 if it ran in a packed batch      */
  int32_t reserved;
} fj_info;

/* fj_info.warnings: some s_i lies outside [0, 1], the range Sec. 2.2
 * assumes.  The solve and the quantities are computed all the same. */
#define FJ_WARN_OPINION_RANGE 1u

/* The five quantities of one opinion vector (Sec. 3.2 definitions). */
typedef struct fj_quant {
  double C_I;  /* internal conflict        */
  double D;    /* disagreement             */
  double P;    /* polarization             */
  double C;    /* controversy              */
  double I_dc; /* disagreement-controversy */
} fj_quant;

/* Fills *opts with the defaults listed in fj_opts. */
void fj_default_opts(fj_opts* opts);

/* Thread-local text of the last error raised on this thread ("" if none). */
const char* fj_last_error(void);

/* Number of CUDA kernels the library has launched in this process, over all
 * contexts (a counter for measuring how much device work a call issues). */
int64_t fj_kernel_launches(void);

/* Library version string. */
const char* fj_version(void);

/* Creates a context on CUDA device `device` with its own non-blocking stream.
 * The context owns a workspace that grows to the largest solve it has run.
 * Errors: FJ_ERR_ARG (bad device / null out), FJ_ERR_CUDA. */
fj_status fj_create(int device, fj_ctx** out);

/* Waits for the context's stream, frees its workspace and the context.
 * Graphs created on it must be freed first (fj_graph_free); requests still
 * queued by fj_submit are cancelled. */
fj_status fj_destroy(fj_ctx* ctx);

/* Runs the context's later GPU work on `stream` (a cudaStream_t of the
 * context's device; NULL restores the context's own stream). */
fj_status fj_set_stream(fj_ctx* ctx, void* stream);

/* Caps the number of thread blocks of the persistent solve kernel (0, the
 * default, uses every block that can be co-resident on the device).  Lets
 * several contexts run solves side by side on one GPU.
 * Errors: FJ_ERR_ARG (NULL ctx or negative cap). */
fj_status fj_set_max_blocks(fj_ctx* ctx, int32_t max_blocks);

/* Runs later solves of this context on a grid of exactly `blocks` thread
 * blocks (at most the co-resident count, and at most the fj_set_max_blocks
 * cap if one is set) instead of sizing it by the work; 0, the default,
 * restores the sizing (or fj_tune's choice).  fj_info.blocks reports the
 * grid a solve ran on.  Errors: FJ_ERR_ARG (NULL ctx or negative count). */
fj_status fj_set_grid(fj_ctx* ctx, int32_t blocks);

/* Builds the device CSR of I + L for an undirected weighted graph given as an
 * edge list (Sec. 2.1: A, d_i = sum_j w_ij, L = D - A).
 *   n        number of nodes (1 <= n <= 2^31 - 2)
 *   m        number of listed undirected edges (>= 0); each edge once
 *   src,dst  int32[m] endpoints in [0, n) (host or device, see flags)
 *   w        float32[m] weights > 0 and finite, or NULL for unit weights
 *   flags    FJ_HOST_PTRS or FJ_DEVICE_PTRS, optionally | FJ_MERGE_DUPLICATES
 * Self-loops are dropped (b_e = 0 adds nothing to L).  The graph of Sec. 2.1
 * is simple: a pair {u, v} listed more than once (in either orientation) is
 * rejected, unless FJ_MERGE_DUPLICATES is given, in which case the repeats
 * are parallel edges whose weights add, as in L = sum_e w_e b_e b_e^T.  The
 * graph need not be connected.  2 * m (minus self-loops) must stay below
 * 2^31.  The graph lives in device memory until fj_graph_free.
 * Errors: FJ_ERR_ARG, FJ_ERR_GRAPH (bad id or weight, or a repeated pair
 * without FJ_MERGE_DUPLICATES; nothing allocated remains), FJ_ERR_OOM,
 * FJ_ERR_CUDA. */
fj_status fj_graph_upload(fj_ctx* ctx, int64_t n, int64_t m,
                          const int32_t* src, const int32_t* dst,
                          const float* w, uint32_t flags, fj_graph** out);

/* Gives existing edges new weights (the FJ model on a changed graph,
 * Sec. 3.1), in place: no re-sort, no new layout.  Update i sets the weight
 * of the pair {src[i], dst[i]} (ids of g, in either orientation) to w[i];
 * a pair listed several times at upload (FJ_MERGE_DUPLICATES) has its first
 * listing changed.  The Jacobi preconditioner is recomputed as the upload
 * computes it, so the graph is the same bits as a fresh upload of the
 * changed edge list (in the same order).  A graph uploaded without weights
 * gets a weight array (all ones) first.  A pair should appear at most once
 * per call (otherwise which of its weights is kept is unspecified).  Warm
 * starts (fj_solve_warm from the previous z) then re-solve cheaply.
 *   count      number of updates (>= 0)
 *   src, dst   int32[count] endpoints; w: float32[count] new weights > 0
 *   flags      FJ_HOST_PTRS or FJ_DEVICE_PTRS for src, dst, w
 * Errors: FJ_ERR_ARG, FJ_ERR_GRAPH (an id out of range, a self-loop, a
 * weight not finite and > 0, or a pair that is not an edge; the graph is
 * unchanged), FJ_ERR_OOM, FJ_ERR_CUDA. */
fj_status fj_graph_update_weights(fj_ctx* ctx, fj_graph* g, int64_t count,
                                  const int32_t* src, const int32_t* dst,
                                  const float* w, uint32_t flags);

/* Frees a graph made by fj_graph_upload on this context. */
fj_status fj_graph_free(fj_ctx* ctx, fj_graph* g);

/* The subgraph induced on the largest connected component of g (the
 * paper's experiments run on each network's largest connected component,
 * Sec. 5).  Its nodes are those of the component in increasing order of
 * their id in g; fj_graph_node_ids gives that map.  Of components of equal
 * size, the one holding the smallest id wins.  Weights carry over.  *out
 * lives until fj_graph_free.
 * Errors: FJ_ERR_ARG, FJ_ERR_OOM, FJ_ERR_NOT_CONVERGED (the components did not
 * settle within the round cap), FJ_ERR_CUDA. */
fj_status fj_graph_lcc(fj_ctx* ctx, const fj_graph* g, fj_graph** out);

/* ids[i] (HOST int32[n], n from fj_graph_stats) = the id in the parent graph
 * of node i of a graph made by fj_graph_lcc, or i for an uploaded graph.
 * Errors: FJ_ERR_ARG, FJ_ERR_CUDA. */
fj_status fj_graph_node_ids(fj_ctx* ctx, const fj_graph* g, int32_t* ids);

/* Size of a graph: nodes, stored off-diagonal CSR entries (2 x non-loop
 * edges), and whether it carries a weight array (0 = unit weights). */
fj_status fj_graph_stats(const fj_graph* g, int64_t* n, int64_t* nnz,
                         int32_t* weighted);

/* Solves (I + L) z = s for k opinion vectors (Eq. FJmodel02) and optionally
 * returns z and the five quantities of each column.
 *   s     float64[n*k], column-major (column c at s + c*n), host or device
 *   z     float64[n*k] output, same layout and location as s, or NULL
 *   quant fj_quant[k] output in HOST memory, or NULL
 *   opts  options (NULL: defaults); opts->flags says where s and z live
 *   info  optional host output
 * Any finite s is accepted (the paper assumes s in [0,1]; the algebra does
 * not need it); values outside [0, 1] set FJ_WARN_OPINION_RANGE in
 * info->warnings.  Errors: FJ_ERR_ARG, FJ_ERR_OOM, FJ_ERR_NOT_CONVERGED (z and
 * quant still hold the last iterate), FJ_ERR_NUMERIC, FJ_ERR_TIMEOUT,
 * FJ_ERR_CUDA. */
fj_status fj_solve_ex(fj_ctx* ctx, const fj_graph* g, int32_t k,
                      const double* s, double* z, fj_quant* quant,
                      const fj_opts* opts, fj_info* info);

/* fj_solve_ex started from an initial guess z0 instead of 0 (for example the
 * z of an earlier solve, after s or a few weights changed).  The iteration
 * starts at q = z0 - mu 1 with one float64 residual evaluation; the stopping
 * rule, the results and their accuracy are those of fj_solve_ex, only the
 * number of iterations depends on how close z0 is.
 *   z0   float64[n*k], same layout and location as s (not modified)
 * Errors: as fj_solve_ex; FJ_ERR_ARG for a NULL z0. */
fj_status fj_solve_warm(fj_ctx* ctx, const fj_graph* g, int32_t k,
                        const double* s, const double* z0, double* z,
                        fj_quant* quant, const fj_opts* opts, fj_info* info);

/* fj_solve_ex with quant = NULL: the equilibrium z = (I + L)^-1 s. */
fj_status fj_solve(fj_ctx* ctx, const fj_graph* g, int32_t k, const double* s,
                   double* z, const fj_opts* opts, fj_info* info);

/* fj_solve_ex with z = NULL: Algorithm 1's five outputs for each column of s
 * (out: fj_quant[k] in host memory). */
fj_status fj_quantities(fj_ctx* ctx, const fj_graph* g, int32_t k,
                        const double* s, fj_quant* out, const fj_opts* opts,
                        fj_info* info);

/* Grid autotuner.  A solve is one persistent launch per group of at most
 * 32 columns, so the launch shape left to choose per graph is its grid.  The
 * default sizing takes about 16 CSR entries or nodes per thread, up to every
 * co-resident block.  That suits large graphs; on small ones more blocks
 * can win (more loads in flight, more float64 units), or fewer (each of the
 * iteration's grid barriers costs more with more blocks).  fj_tune times
 * solves of the k columns of s (solve kernels only, median of `repeats`
 * after one warm-up) with the default sizing and with grids of exactly
 * 2*SMs, SMs, SMs/2, ..., 1 blocks, keeps the fastest, and runs later
 * fj_solve_ex / fj_solve_warm / fj_solve / fj_quantities calls on g with the
 * same k and the same precision class (float64 or not) on it, unless the
 * context's fj_set_grid asks for another grid; the fj_set_max_blocks cap
 * still applies.  A later fj_tune on g replaces the choice; fj_graph_free
 * forgets it.  The grid changes only the order of the floating-point sums,
 * so results stay within the solve's tolerance and are bit-reproducible for
 * a fixed grid.
 *   s        float64[n*k] opinions as for fj_solve_ex (host or device)
 *   opts     solve options (NULL: defaults); FJ_TWO_SOLVES is rejected
 *   repeats  timed solves per grid, 1 to 64
 *   out      host output: the grids timed and their median device times
 * Errors: FJ_ERR_ARG, and any error of the solves it runs. */
#define FJ_TUNE_MAX 16
typedef struct fj_tune_result {
  int32_t best;                /* fastest grid in blocks; 0 = default     */
  int32_t count;               /* grids timed                             */
  int32_t blocks[FJ_TUNE_MAX]; /* the grids timed, 0 = default sizing     */
  double ms[FJ_TUNE_MAX];      /* median device milliseconds of each      */
} fj_tune_result;
fj_status fj_tune(fj_ctx* ctx, const fj_graph* g, int32_t k, const double* s,
                  const fj_opts* opts, int32_t repeats, fj_tune_result* out);

/* Many independent problems, each its own graph and opinion vectors, in
 * shared persistent launches: every problem is cut into parts of 32/16/8/4/
 * 2/1 columns as in fj_solve_ex, and parts of equal width are packed, up to
 * FJ_PACK_MAX per launch and up to the blocks the device holds at once, into
 * one cooperative launch.  Each part runs on its own block range (sized by
 * its work as fj_solve_ex sizes a grid) with its own grid barrier, reduction
 * slots, workspace and stopping test, so its results are the same bits as
 * fj_solve_ex gives for that part on that many blocks (fj_set_grid); small
 * graphs no longer pay a whole-device launch each.  Launches run one after
 * another on the context's stream.
 *   count   number of problems, 1 <= count <= FJ_BATCH_MAX
 *   graphs  const fj_graph*[count] of this context's device (may repeat)
 *   k       int32[count], 1 <= k[i] <= 1024
 *   s       const double*[count]; s[i]: float64[n_i * k_i] column-major,
 *           host or device per opts->flags
 *   z       double*[count] or NULL, entries NULL or outputs shaped like s[i]
 *   quant   fj_quant*[count] or NULL, entries NULL or HOST fj_quant[k_i]
 *   opts    options shared by all problems (NULL: defaults); FJ_TWO_SOLVES
 *           is rejected
 *   info    fj_info[count] or NULL: per problem; blocks = its largest part's
 *           block range, device_ms = the whole call's device time
 * Returns FJ_OK, FJ_ERR_ARG / FJ_ERR_OOM / FJ_ERR_CUDA for the call, or the
 * first problem's solve error (each problem's own in info[i].status). */
#define FJ_PACK_MAX 24
#define FJ_BATCH_MAX 4096
fj_status fj_solve_batch(fj_ctx* ctx, int32_t count,
                         const fj_graph* const* graphs, const int32_t* k,
                         const double* const* s, double* const* z,
                         fj_quant* const* quant, const fj_opts* opts,
                         fj_info* info);

/* Layout of a graph on the device (the SpMV's row split): rows of more than
 * sell_max entries are "long" and cut into chunks of at most chunk_len
 * entries, each walked by a whole warp; shorter rows are stored as sliced
 * ELL (32-row slices, one lane per row).  The defaults (512, 64) suit the
 * power-law graphs measured here; fj_tune_layout picks per workload. */
typedef struct fj_layout {
  int32_t chunk_len; /* 32 .. 65536 entries (default 512)                    */
  int32_t sell_max;  /* 8 .. 64 entries (default 64)                         */
} fj_layout;

/* Later uploads on this context use this layout (NULL: the defaults).
 * Errors: FJ_ERR_ARG (NULL ctx, values out of range). */
fj_status fj_set_layout(fj_ctx* ctx, const fj_layout* layout);

/* The layout a graph was built with. */
fj_status fj_graph_layout(const fj_graph* g, fj_layout* out);

/* Layout autotuner: uploads the edge list (as fj_graph_upload, with
 * upload_flags) once per candidate layout - chunk lengths 256 to 4096 and
 * sliced-ELL limits 32 and 64, the default first - and times solves of the k
 * columns of s on each (solve kernels only, median of `repeats` after one
 * warm-up).  The fastest becomes the context's layout for later uploads
 * (fj_set_layout); out lists every candidate and its time.  The layout
 * changes only the order of floating-point sums, so results stay within the
 * solve's tolerance.  Errors: FJ_ERR_ARG, and any error of the uploads and
 * solves it runs. */
#define FJ_LAYOUT_TUNE_MAX 16
typedef struct fj_layout_tune_result {
  fj_layout best;
  int32_t count;                          /* candidates timed              */
  fj_layout tried[FJ_LAYOUT_TUNE_MAX];
  double ms[FJ_LAYOUT_TUNE_MAX];          /* median device milliseconds    */
} fj_layout_tune_result;
fj_status fj_tune_layout(fj_ctx* ctx, int64_t n, int64_t m, const int32_t* src,
                         const int32_t* dst, const float* w,
                         uint32_t upload_flags, int32_t k, const double* s,
                         const fj_opts* opts, int32_t repeats,
                         fj_layout_tune_result* out);

/* ---------------------------------------------------------------------
 * Serving: continuous batching of solve requests (one worker thread per
 * context, started by the first call below).  A request is queued on submit;
 * it is admitted as soon as an in-flight slot is free and the device memory
 * it needs fits the serving budget, and then runs side by side with the
 * other admitted requests (small ones packed together, see fj_serve_pack).
 * Admission follows arrival order, except that a request that does not fit
 * the budget yet is passed over by later requests that do, at most 32 times;
 * after that nothing behind it is admitted until it fits.  Finished requests
 * release their memory and slot at once, so queued requests start while
 * others still run.  These calls may come from several threads.
 */

/* Sets the serving limits: at most max_inflight requests on the GPU at once
 * (default 16; 0 keeps the current value), a device-memory budget for
 * admitted requests (default half the free memory when serving starts; <= 0
 * keeps the current value) and a cap on the thread blocks of each request's
 * solve (0, the default: the device's co-resident solve blocks divided by
 * max_inflight, so that the in-flight requests run side by side, and a
 * quarter of them for a graph of more than 131072 nodes; < 0 keeps the
 * current value).
 * Errors: FJ_ERR_ARG, FJ_ERR_CUDA. */
fj_status fj_serve_config(fj_ctx* ctx, int32_t max_inflight,
                          int64_t mem_budget_bytes,
                          int32_t max_blocks_per_request);

/* Requests whose graph has at most max_nodes nodes (default 0: none) are
 * solved in packed batches: once their graphs are resident, the
 * waiting small requests are solved together, their parts of equal column
 * count packed into shared persistent launches as in fj_solve_batch, each
 * part on its own block range of at most the per-request block cap.  Larger
 * requests run their own persistent solve.  A request's results depend only
 * on its own size and the cap, so they are the same bits packed or not.
 * Packing is off by default: on GB300 the requests' own launches, each on
 * its slot's stream right after its graph build, served both a mixed stream
 * (n in [1e3, 1e6]) and a stream of small graphs (n in [1e3, 1e4]) faster
 * than packed batches, which hold every request until their slowest part
 * ends.  Many small graphs already at hand are best given to fj_solve_batch.
 * Errors: FJ_ERR_ARG, FJ_ERR_CUDA. */
fj_status fj_serve_pack(fj_ctx* ctx, int64_t max_nodes);

/* Queues the solve of k opinion vectors on a resident graph (which must stay
 * alive until the request is collected).  s: HOST float64[n*k], column-major,
 * copied before the call returns.  *ticket identifies the request for
 * fj_poll.  Errors: FJ_ERR_ARG (1 <= k <= 1024), FJ_ERR_ADMIT (the request
 * needs more device memory than the whole serving budget). */
fj_status fj_submit(fj_ctx* ctx, const fj_graph* g, int32_t k,
                    const double* s, const fj_opts* opts, uint64_t* ticket);

/* Queues a request that brings its own graph: an edge list as for
 * fj_graph_upload (HOST pointers, copied before the call returns).  The graph
 * is built on the device when the request is admitted and freed when it
 * finishes; a bad node id or weight, or a repeated pair unless opts->flags
 * has FJ_MERGE_DUPLICATES, is reported by fj_poll (FJ_ERR_GRAPH). */
fj_status fj_submit_edges(fj_ctx* ctx, int64_t n, int64_t m,
                          const int32_t* src, const int32_t* dst,
                          const float* w, int32_t k, const double* s,
                          const fj_opts* opts, uint64_t* ticket);

/* Collects a request.  Waits up to timeout_us microseconds (0: do not wait,
 * < 0: wait until done).  Returns FJ_PENDING while the request runs;
 * otherwise the request's status (FJ_OK or a solve error) with out[0..k-1]
 * (HOST) and *info filled (info->device_ms: milliseconds from admission to
 * completion), and the ticket is consumed.  Errors: FJ_ERR_TICKET (unknown
 * or already collected ticket). */
fj_status fj_poll(fj_ctx* ctx, uint64_t ticket, int32_t timeout_us,
                  fj_quant* out, fj_info* info);

/* ---------------------------------------------------------------------
 * Allocation-free solve.  The paper has no counterpart: this entry point
 * serves callers that must not allocate device memory while solving - code
 * inside a latency-critical loop, where cudaMalloc/cudaFree could stall the
 * whole device, and programs whose device memory belongs to another
 * allocator.  It runs the same solver as fj_solve_ex but takes every scratch
 * buffer from one array of FJ_FIXED_SCRATCH_BYTES bytes that is compiled into
 * the library; each device that loads the library's solver code keeps that
 * array until the process exits.  The call allocates nothing.
 *   g       graph from fj_graph_upload (its device becomes current)
 *   stream  cudaStream_t of that device to run on (NULL: the default stream)
 *   k       number of opinion vectors, 1 <= k <= 32
 *   s       DEVICE float64[n*k], column-major; z: DEVICE float64[n*k] or NULL
 *   quant   fj_quant[k] output in HOST memory, or NULL; info: optional
 * The first call on each device looks up the array's device address.  All
 * calls on a device share the one array and leave the last call's contents
 * in it (the solver clears what it needs zeroed): calls whose GPU work
 * overlaps in time race on it, so run them one after another (same stream,
 * or synchronized).  The call blocks until its results are on the host (it
 * ends with device-to-host copies and a stream synchronization), so it
 * cannot be called while its stream is being captured into a CUDA graph.
 * Errors: FJ_ERR_ARG (NULL pointer, k out of range, s or z not device memory
 * of the graph's device, or a solve whose scratch exceeds
 * FJ_FIXED_SCRATCH_BYTES; fj_solve_ex has no such limit), and the solve
 * errors of fj_solve_ex. */
#define FJ_FIXED_SCRATCH_BYTES (64u << 20)
fj_status fj_solve_fixed(const fj_graph* g, void* stream, int32_t k,
                         const double* s, double* z, fj_quant* quant,
                         const fj_opts* opts, fj_info* info);

/* ---------------------------------------------------------------------
 * Failure-detection test hook.  The paper has no counterpart.  Every grid
 * barrier of a solve waits at most a bounded time (4 s by default), after
 * which the solve is abandoned with FJ_ERR_TIMEOUT and the context stays
 * usable.  This call sets that limit for later solves in this process
 * (wait_ns <= 0 restores the default; otherwise 1e5 <= wait_ns <= 6e10) and,
 * for tests of the timeout path, makes block 0 of later multi-block solves
 * skip its arrival at grid barrier number `withhold` (1 = the first; 0, the
 * default, never), so that the other blocks' wait runs out.  Not for
 * production use.  Errors: FJ_ERR_ARG. */
fj_status fj_debug_barrier(int64_t wait_ns, int32_t withhold);

#ifdef __cplusplus
}
#endif
#endif /* FJ_H */
