/*
 * gencd_batch.h -- many GenCD solves over one shared X on one GPU.
 *
 * A regularisation path solves Eq. 1 for a decreasing sequence of lambda
 * values, each solve started from the previous solution (the decreasing-lambda
 * schedule that Section 3 mentions from Bradley et al.), and cross-validation
 * repeats the path on row subsets of X.  All these solves share X.  A batch
 * keeps S solve "slots" resident on the device and advances every active slot
 * by one Thread-Greedy iteration (Algorithm 1, Table 2) per step:
 *   Propose  G = X^T U for all slots at once (U = the slots' loss derivatives
 *            l'(y, z_s), n x S): X is streamed once per step for all slots;
 *            then delta and phi of Eq. 7 / Eq. 9 per (column, slot);
 *   Accept   per slot, the best phi < 0 of each of the B column partitions;
 *   Update   w_s += delta, z_s += delta X_j, u_s on the touched rows.
 *
 * Training sets.  A row-fold array assigns each row to one of F folds.  A
 * slot trains on all rows (held_out = -1) or on the rows outside one fold
 * (held_out = f): its objective is (1/n_s) sum over its rows of l(y_i, z_i)
 * + lambda_s ||w_s||_1, with n_s its row count, and beta_j uses the column
 * norms over its rows.  This is the problem of gencd_create on the subset.
 *
 * Arithmetic is that of GENCD_F32 (include/gencd.h): X and u in FP32, sums in
 * FP32, columns ranked by FP32 Eq. 7 / Eq. 9 and the winner's step recomputed
 * in FP64 with the FP64 w; z, w and objectives in FP64.  Slots never mix: a
 * slot's iterates depend only on its own state, whatever the other slots do
 * (sums reach it in a rounding order that can differ from run to run).
 *
 * Conventions (status codes, `memory`, the stream, thread safety) are those
 * of include/gencd.h.  Every call runs on the stream given at create.
 */
#ifndef GENCD_BATCH_H
#define GENCD_BATCH_H

#include <stdint.h>

#include "gencd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gencd_batch gencd_batch; /* opaque, owned by the library */

/*
 * Creates a batch over X (CSC, the same arrays and validation as
 * gencd_create; values are stored in FP32) with labels y.
 *   fold     uint8[n] fold of each row, each < nfolds; NULL when nfolds is 0
 *            (then only held_out = -1 is valid)
 *   nfolds   0..31
 *   slots    1..256 solve slots (rounded up to 8, 16 or a multiple of 32; the
 *            propose pass streams X once per step for all of them)
 *   memory   where col_ptr/row_idx/val/y/fold live (copied; free on return)
 * All slots start inactive.  Parameters start at gencd_default_params().
 * Errors: GENCD_EINVAL (malformed input, message names the first bad index),
 * GENCD_ENOMEM, GENCD_ECUDA.  *out is NULL on error.
 */
int gencd_batch_create(gencd_batch** out, int64_t n, int64_t k, int64_t nnz, const int64_t* col_ptr,
                       const int32_t* row_idx, const void* val, int32_t val_dtype, const double* y,
                       int32_t loss, const uint8_t* fold, int32_t nfolds, int32_t slots, int32_t memory,
                       void* stream);

/* Frees every buffer of the batch.  NULL is ignored. */
void gencd_batch_destroy(gencd_batch* b);

/* Number of slots the batch holds (8, 16 or a multiple of 32). */
int gencd_batch_slots(gencd_batch* b, int32_t* slots);

/*
 * Schedule of the batched step, chosen by the batch's autotuner (not in the
 * paper).  The X^T U pass runs with lanes over entries and 8 slots per lane
 * (spmm_kind 0) or with lanes over slots (1; S a multiple of 32): at create,
 * each form is timed over three passes and the faster is kept.  The update
 * runs one warp per (partition, slot) (update_kind 0) or one warp per
 * (partition, 32 slots), the slots that accepted the same column adding
 * into each z row side by side (1): the first call that runs at least four
 * steps times them alternately and keeps the faster (-1 until then).
 * ms[0..nms): the mean times (ms) of X^T U kinds 0 and 1, then of a whole
 * step with update kinds 0 and 1 (-1 where not timed).  Any pointer may be
 * NULL when nms is 0.
 */
int gencd_batch_schedule(gencd_batch* b, int32_t* spmm_kind, int32_t* update_kind, double* ms, int32_t nms);
/* Sets the schedule (each kind 0 or 1, or -1: autotune it again); every
 * schedule computes the same step.  GENCD_EINVAL for spmm_kind 1 with 8 or
 * 16 slots. */
int gencd_batch_set_schedule(gencd_batch* b, int32_t spmm_kind, int32_t update_kind);

/* lambda_max of the training set of held_out (-1: all rows): the smallest
 * lambda for which w = 0 is optimal, max_j |g_j(0)| (computed at create). */
int gencd_batch_lambda_max(gencd_batch* b, int32_t held_out, double* lambda_max);

/* Iteration parameters (include/gencd.h): variant THREAD_GREEDY or GREEDY,
 * blocks (B partitions, 0 = min(k, 1024)), tol_kkt, tol_gap, check_every and
 * max_iter (per solve, gencd_batch_path), beta_mode.  P, seed and timeout_s
 * are ignored.  GENCD_EINVAL for another variant or a value out of range.
 * tol_gap > 0: gencd_batch_path also ends a solve when its duality gap
 * (include/gencd.h, gencd_duality_gap; the dual point's scale from the FP32
 * sums) is at most tol_gap * |P(w)|, checked when the solve's objective is
 * evaluated (every 8 checks). */
int gencd_batch_set_params(gencd_batch* b, const gencd_params* params);

/*
 * Activates `slot` for the training set of held_out (-1 or a fold) and lambda,
 * with w = the double[k] array `w` in `memory` (NULL: w = 0).  z = Xw and u
 * are recomputed for the slot.
 */
int gencd_batch_set_slot(gencd_batch* b, int32_t slot, int32_t held_out, double lambda, const double* w,
                         int32_t memory);
/* Activates dst with src's current w and z (a warm start) for the training
 * set of held_out and lambda; u is recomputed for dst.  src must be active. */
int gencd_batch_copy_slot(gencd_batch* b, int32_t dst, int32_t src, int32_t held_out, double lambda);
/* Deactivates a slot (its w is kept until the slot is set again). */
int gencd_batch_clear_slot(gencd_batch* b, int32_t slot);
/* Copies the slot's w (double[k]) to `w` in `memory`. */
int gencd_batch_get_w(gencd_batch* b, int32_t slot, double* w, int64_t k, int32_t memory);

/*
 * Enqueues `iters` Thread-Greedy iterations of every active slot (no
 * convergence test).  When `sync` is non-zero the call waits for them.
 */
int gencd_batch_iterate(gencd_batch* b, int64_t iters, int32_t sync);

/*
 * Objective (Eq. 1 on the slot's training set, FP64) and KKT violation (FP32
 * sums, as include/gencd.h defines it) of every slot at its current state;
 * objective and kkt are double[slots] on the host, NaN for inactive slots.
 */
int gencd_batch_objective(gencd_batch* b, double* objective, double* kkt);

/*
 * Parity hook: delta (Eq. 7) and phi (Eq. 9) of every column for every slot
 * at the current state, double[slots * k] slot-major in `memory` (inactive
 * slots: 0).  The state does not change.
 */
int gencd_batch_propose(gencd_batch* b, double* delta, double* phi, int32_t memory);

/*
 * A regularisation path: nchains chains of nlambda solves.  Chain c trains on
 * held_out[c] and solves lambda[c * nlambda + t] for t = 0, 1, ... in order;
 * solve t + 1 starts from solve t's w (warm != 0) or from w = 0.  A solve
 * ends when its KKT violation is at most tol_kkt (GENCD_OK), after max_iter
 * iterations (GENCD_NOT_CONVERGED) or when its KKT value is not finite
 * (GENCD_EDIVERGED).  With handoff > 0, solve t + 1 may start as soon as solve
 * t's KKT violation is at most handoff, from solve t's iterate at that time,
 * while solve t runs on: chains then fill more slots at once.  Every solve
 * still runs to its own tolerance.
 *
 * Accept backoff.  Thread-Greedy has no convergence guarantee (the paper's
 * closing discussion): on correlated columns the B simultaneous updates can
 * oscillate or diverge.  A solve accepts, of every G consecutive partitions,
 * only the best proxy (G = 1 is Thread-Greedy, G = B is Greedy, which lowers
 * the objective at every step).  The rules are gencd_solve's: when a
 * solve's FP64 objective (evaluated every 8 checks) is not finite or above
 * its value at the solve's start, or its KKT violation is not finite, it
 * restarts from its start with 4G; checks covering 500 iterations in a row
 * with neither a new lowest objective (by 1e-12 of itself) nor a KKT
 * violation 1% below the lowest since the (re)start double G while the
 * violation is at least 1e-3 lambda.  A chain's next solve starts at half
 * the G its predecessor reached, or at G = 1 after a solve of the chain that
 * did not converge.
 */
typedef struct {
  int32_t nchains;         /* chains (e.g. cross-validation folds)            */
  int32_t nlambda;         /* solves per chain                                */
  const int32_t* held_out; /* int32[nchains]: fold held out (-1: all rows)    */
  const double* lambda;    /* double[nchains * nlambda], chain-major          */
  double handoff;          /* KKT level at which the next solve may start; 0 */
  int32_t warm;            /* 1: warm starts, 0: every solve from w = 0      */
  int32_t reserved;
  double tol_rel;          /* > 0: solve q stops at KKT <= tol_rel * lambda_q
                              (instead of the absolute tol_kkt); handoff is
                              then relative to lambda too (as it is when the
                              parameters' tol_gap is set)                     */
} gencd_path;

typedef struct {
  int32_t status;   /* GENCD_OK, GENCD_NOT_CONVERGED or GENCD_EDIVERGED     */
  int32_t slot;     /* slot that ran the solve                              */
  int64_t iters;    /* Thread-Greedy iterations of this solve               */
  double objective; /* P(w) of Eq. 1 on the chain's training set (FP64)     */
  double kkt;       /* KKT violation at the start of the solve's last iteration */
  double t_start;   /* seconds from the start of the call                   */
  double t_end;
  int32_t group;    /* partitions per accept group at the end (see below)   */
  int32_t reserved;
} gencd_path_solve;

/*
 * Runs a path on the batch's slots (the slots' previous contents are lost).
 * solves: gencd_path_solve[nchains * nlambda] (host), chain-major.
 * w: NULL, or double[nchains * nlambda * k] (host) receiving each solve's w.
 * out (nullable): iterations = batched steps, updates, nnz_processed and
 * seconds of the whole call; objective and kkt are 0.
 * Returns GENCD_OK when every solve converged, GENCD_NOT_CONVERGED when one
 * did not (see its status), or an error.
 */
int gencd_batch_path(gencd_batch* b, const gencd_path* path, gencd_path_solve* solves, double* w,
                     gencd_result* out);

#ifdef __cplusplus
}
#endif

#endif /* GENCD_BATCH_H */
