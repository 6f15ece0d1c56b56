/*
 * gencd.h -- C ABI of libgencd, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of GenCD from Scherrer, Halappanavar, Tewari and
 * Haglin, "Scaling Up Coordinate Descent Algorithms for Large l1
 * Regularization Problems".
 *
 * Problem (Section 1, Eq. 1):
 *     min_w (1/n) sum_i l(y_i, (Xw)_i) + lambda ||w||_1
 * with squared loss l(y,t) = (y - t)^2 / 2 (Lasso) or logistic loss
 * l(y,t) = log(1 + exp(-y t)), X an n x k sparse matrix.
 *
 * One GenCD iteration (Algorithm 1) is Select -> Propose -> Accept -> Update:
 *   Propose (Algorithm 4): g_j = <l'(y, z), X_j> / n, the step of Eq. 7,
 *           delta_j = -psi(w_j; (g_j - lambda)/beta_j, (g_j + lambda)/beta_j),
 *           and the proxy of Eq. 9,
 *           phi_j = beta_j/2 delta_j^2 + g_j delta_j + lambda(|w_j+delta_j| - |w_j|);
 *   Accept  (Table 2): Shotgun and Coloring accept all proposals, Thread-Greedy
 *           the best proxy per partition, Greedy the single best;
 *   Update  (Algorithm 3): w_j += delta_j, z += delta_j X_j, and the loss
 *           derivative u = l'(y, z) on the touched rows (Section 2.4).
 *
 * Conventions for every entry point:
 *  - Return value: GENCD_OK (0), GENCD_NOT_CONVERGED (1, results valid) or a
 *    negative error code.  On error, gencd_last_error() returns a message
 *    (thread-local, valid until the next call on the same thread).  No C++
 *    exception crosses this boundary.
 *  - `memory` selects where a caller buffer lives: GENCD_HOST (pageable or
 *    pinned host memory) or GENCD_DEVICE (memory of the problem's GPU).
 *  - All GPU work runs on the CUDA stream given to gencd_create.  Calls that
 *    return values to the host synchronise that stream before returning.
 *  - Indices are 0-based.  Limits: n, k < 2^31, nnz < 2^31 - 64.
 *  - A problem handle must not be used from two threads at once.
 */
#ifndef GENCD_H
#define GENCD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GENCD_OK 0
#define GENCD_NOT_CONVERGED 1 /* max_iter or timeout reached; w is valid      */
#define GENCD_EINVAL (-1)     /* bad argument or malformed CSC input          */
#define GENCD_ENOMEM (-2)     /* device or pinned host allocation failed      */
#define GENCD_ECUDA (-3)      /* a CUDA runtime call failed                   */
#define GENCD_ETIMEOUT (-4)   /* a bounded device wait gave up                */
#define GENCD_EDIVERGED (-5)  /* objective or KKT value became non-finite     */
#define GENCD_ESTATE (-6)     /* call not valid in the problem's state        */

typedef enum { GENCD_LOSS_SQUARED = 0, GENCD_LOSS_LOGISTIC = 1 } gencd_loss;

/* Table 2 of the paper. */
typedef enum {
  GENCD_SHOTGUN = 0,       /* Select: random subset of P columns; Accept: all   */
  GENCD_THREAD_GREEDY = 1, /* Select: all; Accept: best proxy per partition     */
  GENCD_GREEDY = 2,        /* Select: all; Accept: the single best proxy        */
  GENCD_COLORING = 3,      /* Select: random colour class; Accept: all          */
  GENCD_TOP_GREEDY = 4,    /* Select: all; Accept: the `blocks` lowest proxies
                              of all columns, wherever they fall (Section 7's
                              extension of Thread-Greedy)                       */
  GENCD_SHOTGUN_BLOCKS = 5 /* Section 7's block Shotgun: `blocks` contiguous
                              column blocks (0 => 16, at most 1024), each with
                              its own P*_b (gencd_block_pstar); Select: the
                              next P*_b columns of every block's per-epoch
                              permutation (block b's stream seeded with
                              seed + b); Accept: all                            */
} gencd_variant;

/* Storage and arithmetic of the hot path.  F64: X, u and the sums in FP64.
 * F32: X and u in FP32, sums in FP32 (z, w, objective in FP64; Thread-Greedy
 * ranks columns with FP32 proxies and applies the winner's FP64 step).
 * BF16: as F32, with the values of X rounded to bfloat16 (round to nearest
 * even) at create and streamed as bfloat16 by the propose over all columns.
 * BINARY: as F32, index only: all non-zeros of a column must share one value
 * s_j (GENCD_EINVAL otherwise); the propose over all columns streams row
 * indices only and scales each column's sum of u by s_j.  Neither storage
 * mode is in the paper; its data sets are binary or tf-idf (Section 5). */
typedef enum { GENCD_F64 = 0, GENCD_F32 = 1, GENCD_BF16 = 2, GENCD_BINARY = 3 } gencd_precision;
typedef enum { GENCD_HOST = 0, GENCD_DEVICE = 1 } gencd_memory;

typedef struct gencd_problem gencd_problem; /* opaque, owned by the library */

typedef struct {
  int32_t variant;     /* gencd_variant                                         */
  int32_t blocks;      /* Thread-Greedy partitions B (contiguous column chunks
                          [floor(b k/B), floor((b+1) k/B))); 0 => min(k, 1024)  */
  int64_t P;           /* Shotgun subset size; 0 => P* = floor(k / (2 rho)),
                          rho = spectral radius of D^-1/2 X^T X D^-1/2 (Sec 4.1) */
  uint64_t seed;       /* seed of the selection stream (SplitMix64)             */
  int64_t max_iter;    /* iteration cap of gencd_solve                          */
  double tol_kkt;      /* gencd_solve stops when the KKT violation <= tol_kkt   */
  int32_t check_every; /* iterations between convergence checks                 */
  int32_t beta_mode;   /* 0: beta_j = beta * ||X_j||^2 / n (default);
                          1: the literal beta of Eq. 7 (1 squared, 1/4 logistic) */
  double timeout_s;    /* wall-clock cap of gencd_solve in seconds; 0 = none    */
  int32_t improve_steps; /* "Improve delta_j" (Algorithm 3, Section 4.1): up to
                            this many Eq. 7 steps refine each accepted increment
                            on its own coordinate from the iteration-start state
                            (Thread-Greedy, Greedy, Shotgun; 0 = off, at most
                            100000)                                              */
  int32_t reserved;
  double tol_gap;      /* > 0: gencd_solve also stops when the duality gap of a
                          full evaluation (gencd_duality_gap) is at most
                          tol_gap * |P(w)|, which bounds the relative objective
                          error (P(w) - P*) / P(w); every convergence check is
                          then a full evaluation.  0 = off (default)            */
} gencd_params;

typedef struct {
  int32_t status;        /* return code of the call                           */
  int32_t reserved;
  int64_t iters;         /* GenCD iterations run by the call                  */
  int64_t updates;       /* accepted proposals applied (Algorithm 3)          */
  int64_t nnz_processed; /* sum over proposals and updates of column nnz      */
  double objective;      /* P(w) of Eq. 1 after the call (FP64)               */
  double kkt;            /* max_j KKT violation after the call (FP64):
                            max(|g_j| - lambda, 0) if w_j = 0,
                            |g_j + lambda sign(w_j)| otherwise                 */
  double seconds;        /* host wall time of the call                        */
} gencd_result;

/*
 * Creates a problem from X in CSC form (Table 1; X is traversed by columns,
 * Section 1) and labels y.
 *   col_ptr  int64[k+1], non-decreasing, col_ptr[0] = 0, col_ptr[k] = nnz
 *   row_idx  int32[nnz], strictly increasing within each column, in [0, n)
 *   val      nnz values, double (val_dtype 0) or float (val_dtype 1)
 *   y        double[n]; for logistic loss every y_i must be -1 or +1
 *   loss     gencd_loss;  precision  gencd_precision (storage of X and u and
 *            the precision of the sums X_j^T u; see gencd_precision)
 *   memory   where col_ptr/row_idx/val/y live; the library copies them into
 *            its own device buffers, so the caller may free them on return
 *   stream   cudaStream_t (may be NULL for the legacy default stream)
 * Initial state: w = 0, z = 0, lambda = 0, default parameters, iteration 0.
 * Errors: GENCD_EINVAL for malformed input (the message names the first bad
 * index), GENCD_ENOMEM, GENCD_ECUDA.  *out is NULL on error.
 */
int gencd_create(gencd_problem** out, int64_t n, int64_t k, int64_t nnz, const int64_t* col_ptr,
                 const int32_t* row_idx, const void* val, int32_t val_dtype, const double* y,
                 int32_t loss, int32_t precision, int32_t memory, void* stream);

/* Frees every device and host buffer of the problem.  NULL is ignored. */
void gencd_destroy(gencd_problem* p);

/* Sets the l1 weight lambda >= 0 of Eq. 1 (state w, z is kept). */
int gencd_set_lambda(gencd_problem* p, double lambda);

/* Changes the loss (gencd_loss) of the problem; for logistic loss every y_i
 * must be -1 or +1 (GENCD_EINVAL otherwise, and the loss is unchanged).  The
 * state w, z and lambda are kept; u, beta_j and lambda_max follow the new
 * loss. */
int gencd_set_loss(gencd_problem* p, int32_t loss);

/* lambda_max = max_j |g_j(w = 0)|, the smallest lambda for which w = 0 is
 * optimal.  Computed on the GPU at create time. */
int gencd_lambda_max(gencd_problem* p, double* lambda_max);

/* Fills *out with the default parameters (Thread-Greedy, B = 0 (auto),
 * P = 0 (auto), seed 0, max_iter 100000, tol_kkt 1e-8, check_every 10,
 * beta_mode 0, no timeout, tol_gap 0). */
int gencd_default_params(gencd_params* out);

/* Validates and stores the iteration parameters. */
int gencd_set_params(gencd_problem* p, const gencd_params* params);
int gencd_get_params(gencd_problem* p, gencd_params* params);

/*
 * Runs GenCD iterations (Algorithm 1) until the KKT violation is at most
 * tol_kkt, max_iter iterations or the timeout.  Convergence is checked every
 * check_every iterations (Thread-Greedy and Greedy read the KKT value their
 * Propose step computes and confirm convergence with one full pass; Shotgun
 * and Coloring make a full pass over X at each check).  Returns GENCD_OK,
 * GENCD_NOT_CONVERGED, GENCD_EDIVERGED (objective non-finite, or above 1e6
 * times its value at the start of the call) or an error.
 * Accept backoff (Thread-Greedy and the global top-|J'| Accept with B > 1;
 * not in the paper, which gives them no convergence guarantee): when the
 * objective is not finite or above its value at the start of the call, the
 * solve restarts from the w it started with and, G growing 4x per restart,
 * Thread-Greedy keeps of every G consecutive partitions only the best
 * accepted proxy while top-|J'| accepts the max(1, B/G) lowest proxies.
 * G = B is Greedy, whose steps always lower the objective.  A solve that
 * converges never restarts.  A solve that cycles below its start value
 * (checks covering 500 iterations in a row with neither a new lowest
 * objective, by 1e-12 of itself, nor a KKT violation 1% below the lowest
 * since the start or the last restart, while the violation is at least
 * 1e-3 lambda) doubles G without a restart.  G returns to 1 at gencd_set_params; gencd_iterate
 * applies the current G.
 * `out` (nullable) receives the statistics of the call.
 */
int gencd_solve(gencd_problem* p, gencd_result* out);

/*
 * Enqueues exactly `iters` GenCD iterations of the configured variant with no
 * convergence test between them, then synchronises and fills `out` (nullable)
 * with the objective and the KKT violation of the final state.  When `out` is
 * NULL the call returns without synchronising (the work stays queued on the
 * stream) and evaluates no objective.
 */
int gencd_iterate(gencd_problem* p, int64_t iters, gencd_result* out);

/*
 * Work counters accumulated since the last gencd_stats_reset (or since the
 * last gencd_solve / gencd_iterate call made with a non-NULL result):
 * iterations, accepted updates and non-zeros processed; objective and kkt
 * hold the values last computed on the device (Thread-Greedy and Greedy
 * iterations compute both for their start state).  Synchronises the stream.
 */
int gencd_stats(gencd_problem* p, gencd_result* out);
int gencd_stats_reset(gencd_problem* p);

/* Iteration counter t that drives Select (Shotgun chunk, Coloring colour). */
int gencd_set_iteration(gencd_problem* p, int64_t t);
int gencd_get_iteration(gencd_problem* p, int64_t* t);

/* Copies w (double[k]) out to, or in from, a caller buffer.  gencd_set_w
 * recomputes z = Xw (from a row-major copy of X built on first use) and u. */
int gencd_get_w(gencd_problem* p, double* w, int64_t k, int32_t memory);
int gencd_set_w(gencd_problem* p, const double* w, int64_t k, int32_t memory);
/* Copies z = Xw (double[n], maintained incrementally by Algorithm 3). */
int gencd_get_z(gencd_problem* p, double* z, int64_t n, int32_t memory);

/* Objective P(w) of Eq. 1 and the KKT violation at the current state. */
int gencd_objective(gencd_problem* p, double* objective, double* kkt);

/*
 * Duality gap at the current state (not in the paper, which states no
 * stopping rule; a certificate of the objective error).  With
 * u = l'(y, Xw) in FP64, g = X^T u / n and s = min(1, lambda / max_j |g_j|),
 * s u is a feasible point of the Fenchel dual of Eq. 1,
 *     D(v) = -(1/n) sum_i l*(y_i, v_i)  subject to  ||X^T v|| / n <= lambda,
 * with l*(y, v) = sup_t (v t - l(y, t)) the conjugate of the loss (squared:
 * v y + v^2 / 2; logistic: p log p + (1 - p) log(1 - p), p = -y v), so
 * gap = P(w) - D(s u) >= P(w) - P* by weak duality, and it is 0 at the
 * optimum.  The sums g are those of the problem's arithmetic: in the FP32
 * storage modes the dual point's feasibility, hence the bound, holds to the
 * FP32 rounding of g.  Any output pointer may be NULL.
 */
int gencd_duality_gap(gencd_problem* p, double* gap, double* primal, double* dual);

/*
 * Parity hook for Algorithm 4: for the m columns J[0..m) (int32, in [0, k),
 * repeats allowed) computes delta (Eq. 7) and phi (Eq. 9) at the current
 * state without changing it.  J, delta and phi (double[m]) live in `memory`.
 */
int gencd_propose_at(gencd_problem* p, const int32_t* J, int64_t m, double* delta, double* phi,
                     int32_t memory);

/*
 * Streaming propose over all k columns (the Thread-Greedy / Greedy Propose
 * step, Table 2): writes delta and phi (double[k]) for every column at the
 * current state; *kkt (nullable) receives the KKT violation.
 */
int gencd_propose_all(gencd_problem* p, double* delta, double* phi, int32_t memory, double* kkt);

/* Spectral radius of D^-1/2 X^T X D^-1/2 by power iteration from the all-ones
 * vector (at most 100 iterations, relative change 1e-6), and Shotgun's
 * P* = max(1, floor(k / (2 rho))) (Section 4.1). */
int gencd_spectral_radius(gencd_problem* p, double* rho, int64_t* pstar, int32_t* iters);

/* Block Shotgun's subset sizes (Section 7): for the B contiguous column
 * blocks [floor(b k / B), floor((b+1) k / B)), rho_b is the spectral radius
 * of the block's D^-1/2 X_b^T X_b D^-1/2 (power iteration as
 * gencd_spectral_radius, from the block's all-ones vector) and
 * P*_b = max(1, floor(k_b / (2 rho_b))).  pstar int64[B] and rho double[B]
 * (nullable) are host buffers; 1 <= B <= min(k, 1024). */
int gencd_block_pstar(gencd_problem* p, int32_t B, int64_t* pstar, double* rho);

/*
 * Partial distance-2 colouring of the columns (Section 4.1: columns that
 * share a row get different colours), computed on the GPU.  The result equals
 * greedy first-fit in column order.  *ncolors receives the colour count.
 */
int gencd_color(gencd_problem* p, int32_t* ncolors);
/*
 * Balanced distance-2 colouring on the host (preprocessing, no GPU work):
 * the paper notes that the fewest colours need not give the most parallelism
 * and that balanced colour classes are preferable (Section 7).  Columns in
 * index order; column j takes, among the colours no lower-index column
 * sharing a row with it uses, the one with the fewest columns so far that is
 * still below `cap` (ties: the lower colour), or a new colour.  cap <= 0:
 * ceil(k / C), C the first-fit colour count of gencd_color.  col_ptr
 * int64[k+1] and row_idx int32[nnz] are host arrays (validated as by
 * gencd_create); colors int32[k] receives the colours, *ncolors their count.
 * Install them with gencd_set_colors to run the Coloring variant on them.
 */
int gencd_color_balanced_csc(int64_t n, int64_t k, const int64_t* col_ptr, const int32_t* row_idx, int64_t cap,
                             int32_t* colors, int32_t* ncolors);
/* Copies the colours (int32[k]) out, or installs caller colours (validated:
 * columns sharing a row must differ; colours in [0, k)). */
int gencd_get_colors(gencd_problem* p, int32_t* colors, int64_t k, int32_t memory);
int gencd_set_colors(gencd_problem* p, const int32_t* colors, int64_t k, int32_t memory);

/*
 * Selection permutation of 0..m-1 for `epoch` (computed on the GPU): the sort
 * of (key_i >> 32, i) where key_i is output i of the SplitMix64 stream seeded
 * with output `epoch` of the stream seeded with `seed`.  perm is int32[m] on
 * the host.  Uses the problem's stream and scratch memory.
 */
int gencd_permutation(gencd_problem* p, uint64_t seed, int64_t epoch, int64_t m, int32_t* perm);

/* Kernel launch counts and, when profiling is enabled, summed device time
 * (ms, CUDA events on the problem's stream) and number of timed invocations
 * per kernel family: 0 streaming propose (the whole family: 9 + 10, or 12,
 * and 11 with index-only storage), 1 finalize, 2 accept, 3 update,
 * 4 refresh, 5 list propose, 6 Coloring iteration, 7 objective,
 * 8 setup/selection, 9 light-column pass, 10 row-slab pass, 11 the heavy
 * columns' g_j times their value (index-only storage), 12 row-slab and
 * light-column passes in one kernel.  ms / calls is the mean duration of one
 * invocation; ms, launches, calls may be NULL. */
int gencd_profile_enable(gencd_problem* p, int32_t enable);
int gencd_profile_read(gencd_problem* p, int32_t kernel, double* ms, int64_t* launches, int64_t* calls);
int gencd_profile_reset(gencd_problem* p);

/*
 * Schedule of the streaming propose over all columns, chosen at create by the
 * library's autotuner (not in the paper): the row-slab pass over the heavy
 * columns and the light-column pass run as two kernels (*split = 0) or as one
 * kernel whose first *split of 32 warps per SM start on the row slabs and the
 * rest on a shared pool of light tiles.  ms[0..nms) receives the autotuner's
 * mean time per invocation (ms) of the two kernels, then of the splits 20,
 * 24, 28 and 31 (-1 where a form was not timed: FP64 arithmetic, or no light
 * or no heavy columns).  split and ms may be NULL.
 */
int gencd_propose_schedule(gencd_problem* p, int32_t* split, double* ms, int32_t nms);
/* Sets that schedule (every form computes the same sums): 0 the two kernels,
 * 20, 24, 28 or 31 the fused kernel with that many slab warps, -1 runs the
 * autotuner again.  GENCD_EINVAL for another value, or a fused split on a
 * problem whose propose has one form only. */
int gencd_set_propose_schedule(gencd_problem* p, int32_t split);

/*
 * gencd_propose_all_noalloc -- the streaming Propose over all k columns
 * (same quantities as gencd_propose_all) for callers that cannot allocate
 * device memory: a thread that must not block on cudaMalloc/cudaFree, a
 * process whose framework already holds all device memory in its own pool, or
 * code enqueueing work on a stream that another thread is capturing.  The
 * paper has no counterpart; this is a deployment entry point.
 *
 * It allocates nothing: no problem handle, no cudaMalloc/cudaFree, no
 * allocating library call.  Its scratch is a fixed device array of 9.44 MB
 * (9,437,192 bytes; every GPU that loads this library holds it until the
 * process exits), which
 * bounds the input: k <= 524,288 columns and nnz <= 33,554,432 non-zeros;
 * larger inputs, a non-finite or negative lambda return GENCD_EINVAL.  The
 * first call on each device looks up the scratch's device address
 * (cudaGetSymbolAddress); make that first call before capturing any stream.  All calls on a device share the scratch and
 * each clears what it accumulates into, so calls that overlap on the GPU
 * (no stream ordering between them) race.
 *
 * Inputs (device memory of the current device, not re-validated: they must
 * satisfy the CSC rules of gencd_create): col_ptr int64[k+1], row_idx
 * int32[nnz], val double[nnz], y double[n], z = Xw double[n], w double[k];
 * loss, lambda >= 0, beta_mode as in gencd_params.  u = l'(y, z) is evaluated
 * on the fly.  Outputs (device): delta, phi double[k], kkt double[1].
 * Work is enqueued on `stream`; the call returns without synchronising.
 */
int gencd_propose_all_noalloc(int64_t n, int64_t k, int64_t nnz, const int64_t* col_ptr, const int32_t* row_idx,
                              const double* val, const double* y, const double* z, const double* w, int32_t loss,
                              double lambda, int32_t beta_mode, double* delta, double* phi, double* kkt,
                              void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* gencd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
