/*
 * gencd_oracle.h -- plain FP64 CPU oracle for GenCD (Scherrer, Halappanavar,
 * Tewari, Haglin: "Scaling Up Coordinate Descent Algorithms for Large l1
 * Regularization Problems").
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * helper with the CUDA library; the two only consume the same input arrays.
 *
 * Problem (Eq. 1):  min_w (1/n) sum_i l(y_i, (Xw)_i) + lambda ||w||_1,
 * X given as CSC: col_ptr int64[k+1], row_idx int32[nnz], val double[nnz].
 *
 * Every function is single-threaded, deterministic, and sums in CSC order.
 */
#ifndef GENCD_ORACLE_H
#define GENCD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_SQUARED = 0, ORACLE_LOGISTIC = 1 };
enum {
  ORACLE_SHOTGUN = 0,       /* Table 2: random subset, accept all            */
  ORACLE_THREAD_GREEDY = 1, /* Table 2: all, best proxy per partition        */
  ORACLE_GREEDY = 2,        /* Table 2: all, single best proxy               */
  ORACLE_COLORING = 3,      /* Table 2: random colour, accept all            */
  ORACLE_CCD = 4,           /* Section 2.1: cyclic singleton                 */
  ORACLE_TOP_GREEDY = 5,    /* Section 7 (R12): all, the best B proxies      */
  ORACLE_SHOTGUN_BLOCKS = 6 /* Section 7 (R14): Shotgun with P*_b per block  */
};

typedef struct {
  int64_t n, k;
  const int64_t* col_ptr;
  const int32_t* row_idx;
  const double* val;
  const double* y;
  int32_t loss;      /* ORACLE_SQUARED / ORACLE_LOGISTIC                    */
  int32_t beta_mode; /* 0: beta_j = beta * c_j ; 1: literal beta (Eq. 7)    */
  double lambda;
} oracle_problem;

typedef struct {
  int32_t variant;       /* ORACLE_* variant                                 */
  int32_t B;             /* Thread-Greedy partitions; top-greedy: |J'| (>= 1) */
  int64_t P;             /* Shotgun subset size (>= 1)                       */
  uint64_t seed;         /* selection stream seed                            */
  const int32_t* colors; /* Coloring: colour of each column, 0..ncolors-1    */
  int32_t ncolors;
  int32_t improve_steps; /* R11: "Improve delta_j" steps per accepted proposal (0: off) */
  const int64_t* block_P; /* R14: subset size of each of the B column blocks   */
} oracle_params;

/* Section 1 losses and their derivative in the fitted value t. */
double oracle_loss(int32_t loss, double y, double t);
double oracle_dloss(int32_t loss, double y, double t);
/* Section 3.2: curvature bound beta (1 squared, 1/4 logistic). */
double oracle_beta(int32_t loss);

/* z = Xw (Table 1 "fitted value"). */
void oracle_fitted(const oracle_problem* pr, const double* w, double* z);
/* c_j = ||X_j||^2 / n (diagonal of the Hessian factor of Section 3). */
void oracle_col_scale(const oracle_problem* pr, double* c);
/* g_j = (1/n) X_j^T l'(y, z) for all j (gradient of F, Section 3). */
void oracle_gradient(const oracle_problem* pr, const double* z, double* g);
/* P(w) = (1/n) sum_i l(y_i, z_i) + lambda ||w||_1 with z = Xw (Eq. 1, 3). */
double oracle_objective(const oracle_problem* pr, const double* w);
double oracle_objective_z(const oracle_problem* pr, const double* w, const double* z);
/* Largest KKT violation of (w, z = Xw). */
double oracle_kkt(const oracle_problem* pr, const double* w, const double* z);
/* lambda_max = max_j |g_j(0)|: the smallest lambda with w = 0 optimal. */
double oracle_lambda_max(const oracle_problem* pr);

/* Convex conjugate of the loss in its second argument,
 * l*(y, v) = sup_t (v t - l(y, t)):  squared  v y + v^2 / 2;  logistic
 * p log p + (1 - p) log(1 - p) with p = -y v, finite for p in [0, 1]
 * (0 log 0 = 0; HUGE_VAL outside). */
double oracle_conjugate(int32_t loss, double y, double v);
/* Duality gap of (w, z = Xw) for Eq. 1 (Fenchel duality; the paper states
 * no stopping rule, this is a certificate of P(w) - P*):  P(w) - D(s u) with
 * u = l'(y, z), g = X^T u / n, s = min(1, lambda / max_j |g_j|) (s = 1 when
 * g = 0), D(nu) = -(1/n) sum_i l*(y_i, nu_i).  s u is dual feasible
 * (||X^T s u|| / n <= lambda), so by weak duality the gap is >= P(w) - P*, and
 * it is 0 at the optimum. */
double oracle_duality_gap(const oracle_problem* pr, const double* w, const double* z);

/* Eq. 7 step and Eq. 9 proxy for one coordinate. */
void oracle_step(double g, double w_j, double lambda, double beta_j, double* delta, double* phi);
/* Algorithm 4 over the columns J[0..m) at the state (w, z). */
void oracle_propose(const oracle_problem* pr, const double* w, const double* z,
                    const int32_t* J, int64_t m, double* delta, double* phi);

/* SplitMix64 (Steele, Lea, Flood 2014): output number i (i >= 0) of the
 * stream whose state starts at s. */
/* Values of X as a storage mode holds them (R10): mode 0 FP64 (copy), 1 FP32,
 * 2 bfloat16 from the FP32 value, 3 index-only binary (FP32; every column's
 * values must be equal).  out[q] is the stored value of entry q, as a double.
 * Returns -1, or the lowest column whose values differ (mode 3), or -2 for a
 * value outside the bfloat16 range (mode 2). */
int64_t oracle_stored_values(int32_t mode, int64_t k, const int64_t* col_ptr, const double* val,
                             double* out);

/* R11, "Improve delta_j" (Algorithm 3, Section 4.1): starting from the
 * proposal d of column j, repeat the Eq. 7 step on coordinate j at w_j + d
 * with g_j evaluated at z + d X_j (every other coordinate held at the state
 * (w, z)), at most `steps` times or until a step is 0.  Returns the improved
 * increment. */
double oracle_improve(const oracle_problem* pr, const double* w, const double* z, int64_t j, double d,
                      int32_t steps);

uint64_t oracle_splitmix64(uint64_t s, uint64_t i);
/* Selection permutation of 0..m-1 for one epoch. */
void oracle_permutation(uint64_t seed, int64_t epoch, int64_t m, int32_t* perm);

/* Largest eigenvalue of D^-1/2 X^T X D^-1/2 (D = diag X^T X) by power
 * iteration from the all-ones vector. */
double oracle_spectral_radius(const oracle_problem* pr, int32_t max_iter, double rel_tol,
                              int32_t* iters_out);
/* Shotgun's P* = max(1, floor(k / (2 rho))) (Section 4.1). */
int64_t oracle_pstar(int64_t k, double rho);

/* R14: P*_b of each of B contiguous column blocks (block b = columns
 * floor(b k / B) .. floor((b+1) k / B) - 1): oracle_pstar of the block's own
 * spectral radius (power iteration as oracle_spectral_radius). */
void oracle_block_pstar(const oracle_problem* pr, int32_t B, int32_t max_iter, double rel_tol, int64_t* Pb);

/* Greedy first-fit partial distance-2 colouring of the columns in index
 * order.  Returns the number of colours. */
int32_t oracle_color(const oracle_problem* pr, int32_t* colors);
/* R13: balanced distance-2 colouring (Section 7 asks for balanced colour
 * classes rather than the fewest colours).  Columns in index order; column j
 * takes, among the colours not used by lower-index columns sharing a row with
 * it, the one with the fewest columns so far that is still below `cap`
 * (ties: the lower colour), or a new colour when none is.  cap <= 0 means
 * ceil(k / C), C the first-fit colour count (R8).  Returns the colour count. */
int32_t oracle_color_balanced(const oracle_problem* pr, int64_t cap, int32_t* colors);

/* Runs GenCD iterations t0 .. t0+iters-1 (Algorithm 1) from (w, z), updating
 * both in place.  obj_trace (nullable) receives P(w) after every iteration.
 * stats (nullable, 3 entries): accepted updates, nnz processed, iterations.
 * Returns 0, or -1 on invalid parameters. */
int oracle_run(const oracle_problem* pr, const oracle_params* pa, int64_t t0, int64_t iters,
               double* w, double* z, double* obj_trace, int64_t* stats);

/* Runs windows of check_every iterations until oracle_kkt <= tol_kkt or
 * max_iter iterations.  Returns the number of iterations run; *kkt_out gets
 * the last KKT value. */
int64_t oracle_solve(const oracle_problem* pr, const oracle_params* pa, double tol_kkt,
                     int64_t max_iter, int64_t check_every, double* w, double* z,
                     double* kkt_out, int64_t* stats);

#ifdef __cplusplus
}
#endif
#endif
