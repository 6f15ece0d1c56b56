/*
 * gencd_oracle.c -- plain FP64 CPU oracle for GenCD.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this code.  It shares nothing with the CUDA
 * library.  Loops are written in the order of the paper's algorithms, with no
 * blocking or reordering, so that each function can be checked against the
 * cited passage by eye.
 *
 * Readings of the paper used here (each is listed with its reason in the
 * design notes of the repository):
 *  R1  l' and l'' are derivatives in the fitted value t (the second argument);
 *      Section 3 says "first variable", but the gradient of F needs d/dt.
 *  R2  beta_mode 0 uses the per-column bound beta_j = beta * c_j with
 *      c_j = ||X_j||^2 / n, which is a valid upper bound for Eq. 5-6 for any
 *      column scaling and equals H_jj for squared loss (so Eq. 7 == Eq. 4);
 *      beta_mode 1 uses the literal beta of Eq. 7.  A column with
 *      beta_j == 0 (no non-zeros) does not enter F; its step is the exact
 *      minimiser of lambda |w_j + delta|, i.e. delta = -w_j.
 *  R3  The proxy of Eq. 9 is a change of the surrogate (<= 0); the best
 *      proposal is the most negative proxy; a partition whose best proxy is
 *      not < 0 accepts nothing.  Ties go to the lower column index.
 *  R4  Thread-Greedy selects all columns (Table 2) and splits them into B
 *      contiguous chunks, chunk b = [floor(b k / B), floor((b+1) k / B)),
 *      like an OpenMP static schedule (Section 4.2).  Greedy is B = 1.
 *  R5  Every proposal of an iteration is computed from the iteration-start
 *      state (Jacobi); accepted updates are then applied in ascending j.
 *  R6  Random selection: a per-epoch permutation of 0..m-1, the sort of
 *      (key_i >> 32, i) ascending where key_i is SplitMix64 output i of the
 *      stream seeded with SplitMix64 output `epoch` of the stream seeded with
 *      `seed`.  Shotgun takes consecutive chunks of P columns of it (the last
 *      chunk of an epoch may be shorter); Coloring takes one colour per
 *      iteration in the order of a permutation of the colours.
 *  R7  rho is the largest eigenvalue of D^-1/2 X^T X D^-1/2 (unit diagonal,
 *      as Shotgun's bound assumes), found by power iteration.
 *  R8  The colouring is greedy first-fit over the columns in index order.
 *  R9  KKT violation: max(|g_j| - lambda, 0) if w_j == 0, else
 *      |g_j + lambda sign(w_j)|.
 *  R14 Block Shotgun (Section 7: partition the columns into blocks and
 *      compute a P*_b per block): B contiguous column blocks; P*_b is P* of
 *      the block's own normalised Gram matrix; an iteration takes, from
 *      every block, the next P*_b columns of that block's per-epoch
 *      permutation (block b's stream seeded with seed + b, so one block is
 *      Shotgun at P*) and accepts them all.
 *  R13 Balanced colouring (Section 7: fewer colours need not mean more
 *      parallelism; a balanced distribution is preferable): greedy in column
 *      order, each column taking the least-used admissible colour below a
 *      size cap (default ceil(k / C_first-fit)), a new colour if none.
 *  R12 Thread-Greedy with a global top-|J'| Accept (Section 7 leaves it as
 *      an extension): every column is proposed, as for Thread-Greedy, and
 *      the B proposals with the lowest proxies are accepted (only proxies
 *      < 0; equal proxies go to the lower column), whichever partition they
 *      fall in.  B = 1 is Greedy.
 *  R11 "Improve delta_j" (Algorithm 3; Section 4.1 adds "500 steps using the
 *      quadratic approximation" per accepted proposal, without further
 *      detail): the Eq. 7 step is repeated on coordinate j alone, each time
 *      from w_j + d with g_j recomputed at z + d X_j, until the step is 0 or
 *      the step budget ends; every accepted proposal is improved from the
 *      iteration-start state (R5) before any update is applied.  This is a
 *      majorise-minimise iteration on the one-coordinate problem, so it
 *      reaches that coordinate's exact minimiser; for the squared loss with
 *      beta_mode 0 the first step already is (Eq. 4).
 *  R10 Storage modes (not in the paper): a mode replaces each value of X by
 *      the value it stores, and the method then runs on that X.  FP32 rounds
 *      to nearest even; bfloat16 keeps the sign, the 8 exponent bits and the
 *      top 7 mantissa bits of the FP32 value, rounded to nearest even;
 *      binary stores one FP32 value per column.
 */
#include "gencd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- Section 1: the two losses --------------------------------------- */

/* l(y, t): squared 1/2 (y - t)^2; logistic log(1 + exp(-y t)), written as
 * m + log1p(exp(-m)) for m = -y t > 0 so that exp cannot overflow. */
double oracle_loss(int32_t loss, double y, double t) {
  if (loss == ORACLE_SQUARED) {
    double r = y - t;
    return 0.5 * r * r;
  }
  double m = -y * t;
  if (m > 0.0) return m + log1p(exp(-m));
  return log1p(exp(m));
}

/* dl/dt (R1): squared t - y; logistic -y / (1 + exp(y t)). */
double oracle_dloss(int32_t loss, double y, double t) {
  if (loss == ORACLE_SQUARED) return t - y;
  double m = y * t;
  if (m > 0.0) {
    double e = exp(-m);
    return -y * e / (1.0 + e);
  }
  return -y / (1.0 + exp(m));
}

/* Section 3.2: sup_t l''(y, t) is 1 for squared loss and 1/4 for logistic. */
double oracle_beta(int32_t loss) { return loss == ORACLE_SQUARED ? 1.0 : 0.25; }

/* ---- Table 1 arrays and Section 3 quantities -------------------------- */

void oracle_fitted(const oracle_problem* pr, const double* w, double* z) {
  for (int64_t i = 0; i < pr->n; ++i) z[i] = 0.0;
  for (int64_t j = 0; j < pr->k; ++j) {
    if (w[j] == 0.0) continue;
    for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p)
      z[pr->row_idx[p]] += pr->val[p] * w[j];
  }
}

void oracle_col_scale(const oracle_problem* pr, double* c) {
  for (int64_t j = 0; j < pr->k; ++j) {
    double s = 0.0;
    for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) s += pr->val[p] * pr->val[p];
    c[j] = s / (double)pr->n;
  }
}

/* g_j = <l'(y, z), X_j> / n  (Algorithm 4, first line). */
static double column_gradient(const oracle_problem* pr, const double* z, int64_t j) {
  double s = 0.0;
  for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) {
    int32_t i = pr->row_idx[p];
    s += pr->val[p] * oracle_dloss(pr->loss, pr->y[i], z[i]);
  }
  return s / (double)pr->n;
}

void oracle_gradient(const oracle_problem* pr, const double* z, double* g) {
  for (int64_t j = 0; j < pr->k; ++j) g[j] = column_gradient(pr, z, j);
}

double oracle_objective_z(const oracle_problem* pr, const double* w, const double* z) {
  double f = 0.0;
  for (int64_t i = 0; i < pr->n; ++i) f += oracle_loss(pr->loss, pr->y[i], z[i]);
  double l1 = 0.0;
  for (int64_t j = 0; j < pr->k; ++j) l1 += fabs(w[j]);
  return (pr->n > 0 ? f / (double)pr->n : 0.0) + pr->lambda * l1;
}

double oracle_objective(const oracle_problem* pr, const double* w) {
  double* z = (double*)malloc(sizeof(double) * (size_t)(pr->n > 0 ? pr->n : 1));
  oracle_fitted(pr, w, z);
  double v = oracle_objective_z(pr, w, z);
  free(z);
  return v;
}

static double kkt_violation(double g, double w_j, double lambda) {
  if (w_j == 0.0) {
    double v = fabs(g) - lambda;
    return v > 0.0 ? v : 0.0;
  }
  return fabs(g + lambda * (w_j > 0.0 ? 1.0 : -1.0));
}

double oracle_kkt(const oracle_problem* pr, const double* w, const double* z) {
  double worst = 0.0;
  for (int64_t j = 0; j < pr->k; ++j) {
    double v = kkt_violation(column_gradient(pr, z, j), w[j], pr->lambda);
    if (v > worst) worst = v;
  }
  return worst;
}

double oracle_lambda_max(const oracle_problem* pr) {
  double* z = (double*)calloc((size_t)(pr->n > 0 ? pr->n : 1), sizeof(double));
  double m = 0.0;
  for (int64_t j = 0; j < pr->k; ++j) {
    double g = fabs(column_gradient(pr, z, j));
    if (g > m) m = g;
  }
  free(z);
  return m;
}

/* ---- a certificate of P(w) - P*: the Fenchel duality gap of Eq. 1 -------- */

/* l*(y, v) = sup_t (v t - l(y, t)).  Squared: the sup is at t = y + v.
 * Logistic: with s = y t and p = -y v the sup of -p s - log(1 + e^-s) is at
 * e^-s / (1 + e^-s) = p, which gives p log p + (1 - p) log(1 - p). */
double oracle_conjugate(int32_t loss, double y, double v) {
  if (loss == ORACLE_SQUARED) return v * y + 0.5 * v * v;
  double p = -y * v;
  if (p < 0.0 || p > 1.0) return HUGE_VAL;
  double a = p > 0.0 ? p * log(p) : 0.0;
  double b = p < 1.0 ? (1.0 - p) * log1p(-p) : 0.0;
  return a + b;
}

double oracle_duality_gap(const oracle_problem* pr, const double* w, const double* z) {
  double gmax = 0.0;
  for (int64_t j = 0; j < pr->k; ++j) {
    double g = fabs(column_gradient(pr, z, j));
    if (g > gmax) gmax = g;
  }
  double s = gmax > pr->lambda ? pr->lambda / gmax : 1.0;
  double dual = 0.0;
  for (int64_t i = 0; i < pr->n; ++i)
    dual -= oracle_conjugate(pr->loss, pr->y[i], s * oracle_dloss(pr->loss, pr->y[i], z[i]));
  if (pr->n > 0) dual /= (double)pr->n;
  return oracle_objective_z(pr, w, z) - dual;
}

/* ---- Section 3.2-3.3: the step of Eq. 7 and the proxy of Eq. 9 ---------- */

/* |w + d| - |w| of Eq. 9.  When w + d keeps the sign of w the difference is
 * exactly sign(w) d; evaluating it that way avoids the cancellation of two
 * nearly equal magnitudes, which otherwise rounds a tiny negative proxy up to
 * zero near the optimum and stalls the greedy accept rules. */
static double abs_change(double w, double d) {
  double x = w + d;
  if (w > 0.0 && x >= 0.0) return d;
  if (w < 0.0 && x <= 0.0) return -d;
  return fabs(x) - fabs(w);
}

/* psi(x; a, b): clip x into [a, b] (Section 3.1). */
static double psi(double x, double a, double b) {
  if (x < a) return a;
  if (x > b) return b;
  return x;
}

void oracle_step(double g, double w_j, double lambda, double beta_j, double* delta, double* phi) {
  if (beta_j > 0.0) {
    double d = -psi(w_j, (g - lambda) / beta_j, (g + lambda) / beta_j);        /* Eq. 7 */
    *delta = d;
    *phi = 0.5 * beta_j * d * d + g * d + lambda * abs_change(w_j, d);          /* Eq. 9 */
  } else { /* R2: F does not depend on w_j */
    *delta = -w_j;
    *phi = -lambda * fabs(w_j);
  }
}

static double beta_of(const oracle_problem* pr, int64_t j) {
  double b = oracle_beta(pr->loss);
  if (pr->beta_mode == 1) return b;
  double s = 0.0;
  for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) s += pr->val[p] * pr->val[p];
  return b * s / (double)pr->n;
}

void oracle_propose(const oracle_problem* pr, const double* w, const double* z, const int32_t* J,
                    int64_t m, double* delta, double* phi) {
  for (int64_t t = 0; t < m; ++t) {
    int64_t j = J[t];
    double g = column_gradient(pr, z, j);
    oracle_step(g, w[j], pr->lambda, beta_of(pr, j), &delta[t], &phi[t]);
  }
}

/* R11: g_j at z + d X_j, only column j's rows moved */
static double column_gradient_moved(const oracle_problem* pr, const double* z, int64_t j, double d) {
  double s = 0.0;
  for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) {
    int32_t i = pr->row_idx[p];
    s += pr->val[p] * oracle_dloss(pr->loss, pr->y[i], z[i] + d * pr->val[p]);
  }
  return s / (double)pr->n;
}

double oracle_improve(const oracle_problem* pr, const double* w, const double* z, int64_t j, double d,
                      int32_t steps) {
  double beta_j = beta_of(pr, j);
  if (!(beta_j > 0.0)) return d; /* R2: the step already is the exact minimiser */
  for (int32_t s = 0; s < steps; ++s) {
    double g = column_gradient_moved(pr, z, j, d);
    double step, phi;
    oracle_step(g, w[j] + d, pr->lambda, beta_j, &step, &phi);
    if (step == 0.0) break;
    d += step;
  }
  return d;
}

/* ---- R6: selection randomness ------------------------------------------ */

uint64_t oracle_splitmix64(uint64_t s, uint64_t i) {
  uint64_t x = s + (i + 1) * 0x9e3779b97f4a7c15ULL;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}

typedef struct {
  uint32_t key;
  int32_t idx;
} keyed;

static int cmp_keyed(const void* a, const void* b) {
  const keyed* x = (const keyed*)a;
  const keyed* y = (const keyed*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->idx > y->idx) - (x->idx < y->idx);
}

void oracle_permutation(uint64_t seed, int64_t epoch, int64_t m, int32_t* perm) {
  uint64_t s = oracle_splitmix64(seed, (uint64_t)epoch);
  keyed* a = (keyed*)malloc(sizeof(keyed) * (size_t)(m > 0 ? m : 1));
  for (int64_t i = 0; i < m; ++i) {
    a[i].key = (uint32_t)(oracle_splitmix64(s, (uint64_t)i) >> 32);
    a[i].idx = (int32_t)i;
  }
  qsort(a, (size_t)m, sizeof(keyed), cmp_keyed);
  for (int64_t i = 0; i < m; ++i) perm[i] = a[i].idx;
  free(a);
}

/* ---- R7: spectral radius for Shotgun's P* ------------------------------ */

double oracle_spectral_radius(const oracle_problem* pr, int32_t max_iter, double rel_tol,
                              int32_t* iters_out) {
  int64_t n = pr->n, k = pr->k;
  double* d = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
  double* v = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
  double* t = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t j = 0; j < k; ++j) {
    double s = 0.0;
    for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) s += pr->val[p] * pr->val[p];
    d[j] = s > 0.0 ? 1.0 / sqrt(s) : 0.0; /* D^-1/2, zero for empty columns */
    v[j] = 1.0 / sqrt((double)k);
  }
  double rho = 0.0;
  int32_t it = 0;
  for (it = 1; it <= max_iter; ++it) {
    /* r = X D^-1/2 v */
    for (int64_t i = 0; i < n; ++i) r[i] = 0.0;
    for (int64_t j = 0; j < k; ++j)
      for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p)
        r[pr->row_idx[p]] += pr->val[p] * d[j] * v[j];
    /* t = D^-1/2 X^T r */
    double norm2 = 0.0;
    for (int64_t j = 0; j < k; ++j) {
      double s = 0.0;
      for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) s += pr->val[p] * r[pr->row_idx[p]];
      t[j] = d[j] * s;
      norm2 += t[j] * t[j];
    }
    double rho_new = sqrt(norm2); /* ||M v|| with ||v|| = 1 */
    if (rho_new == 0.0) {
      rho = 0.0;
      break;
    }
    for (int64_t j = 0; j < k; ++j) v[j] = t[j] / rho_new;
    int done = fabs(rho_new - rho) <= rel_tol * rho_new;
    rho = rho_new;
    if (done) break;
  }
  if (iters_out) *iters_out = it > max_iter ? max_iter : it;
  free(d);
  free(v);
  free(t);
  free(r);
  return rho;
}

int64_t oracle_pstar(int64_t k, double rho) {
  if (!(rho > 0.0)) return k > 0 ? k : 1;
  double p = floor((double)k / (2.0 * rho));
  if (p < 1.0) return 1;
  if (p > (double)k) return k;
  return (int64_t)p;
}

void oracle_block_pstar(const oracle_problem* pr, int32_t B, int32_t max_iter, double rel_tol, int64_t* Pb) {
  for (int32_t b = 0; b < B; ++b) {
    int64_t lo = pr->k * b / B, hi = pr->k * (b + 1) / B;
    oracle_problem view = *pr; /* the block's columns; offsets stay absolute */
    view.col_ptr = pr->col_ptr + lo;
    view.k = hi - lo;
    Pb[b] = hi > lo ? oracle_pstar(hi - lo, oracle_spectral_radius(&view, max_iter, rel_tol, NULL)) : 0;
  }
}

/* ---- R8: greedy first-fit partial distance-2 colouring ------------------ */

int32_t oracle_color(const oracle_problem* pr, int32_t* colors) {
  int64_t n = pr->n, k = pr->k, nnz = pr->col_ptr[k];
  /* rows of X as lists of columns (the bipartite graph seen from the rows) */
  int64_t* rp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t* rc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t p = 0; p < nnz; ++p) rp[pr->row_idx[p] + 1] += 1;
  for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  for (int64_t i = 0; i < n; ++i) fill[i] = rp[i];
  for (int64_t j = 0; j < k; ++j)
    for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) rc[fill[pr->row_idx[p]]++] = (int32_t)j;
  /* mark[c] == j + 1 means colour c is used by a lower-index neighbour of j */
  int64_t* mark = (int64_t*)calloc((size_t)k + 1, sizeof(int64_t));
  int32_t ncolors = 0;
  for (int64_t j = 0; j < k; ++j) {
    for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) {
      int32_t i = pr->row_idx[p];
      for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
        int32_t c = rc[q];
        if (c < j) mark[colors[c]] = j + 1;
      }
    }
    int32_t col = 0;
    while (mark[col] == j + 1) ++col;
    colors[j] = col;
    if (col + 1 > ncolors) ncolors = col + 1;
  }
  free(rp);
  free(rc);
  free(fill);
  free(mark);
  return ncolors;
}

int32_t oracle_color_balanced(const oracle_problem* pr, int64_t cap, int32_t* colors) {
  int64_t n = pr->n, k = pr->k, nnz = pr->col_ptr[k];
  if (k == 0) return 0;
  if (cap <= 0) {
    int32_t c0 = oracle_color(pr, colors);
    cap = (k + c0 - 1) / c0;
  }
  int64_t* rp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t* rc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t p = 0; p < nnz; ++p) rp[pr->row_idx[p] + 1] += 1;
  for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  for (int64_t i = 0; i < n; ++i) fill[i] = rp[i];
  for (int64_t j = 0; j < k; ++j)
    for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) rc[fill[pr->row_idx[p]]++] = (int32_t)j;
  int64_t* mark = (int64_t*)calloc((size_t)k + 1, sizeof(int64_t));
  int64_t* size = (int64_t*)calloc((size_t)k + 1, sizeof(int64_t));
  int32_t ncolors = 0;
  for (int64_t j = 0; j < k; ++j) {
    for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) {
      int32_t i = pr->row_idx[p];
      for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
        if (rc[q] < j) mark[colors[rc[q]]] = j + 1;
    }
    int32_t best = -1;
    for (int32_t c = 0; c < ncolors; ++c)
      if (mark[c] != j + 1 && size[c] < cap && (best < 0 || size[c] < size[best])) best = c;
    if (best < 0) best = ncolors++;
    colors[j] = best;
    size[best] += 1;
  }
  free(rp);
  free(rc);
  free(fill);
  free(mark);
  free(size);
  return ncolors;
}

/* ---- Algorithm 1: GenCD iterations -------------------------------------- */

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* R12: positions ordered by proxy, equal proxies by position (= column) */
static const double* qsort_ctx_phi = NULL; /* the oracle is single-threaded */
static int cmp_by_phi(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  double px = qsort_ctx_phi[x], py = qsort_ctx_phi[y];
  if (px < py) return -1;
  if (px > py) return 1;
  return (x > y) - (x < y);
}
static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* Update (Algorithm 3) for one accepted proposal: w_j += delta, z += delta X_j. */
static void apply_update(const oracle_problem* pr, int64_t j, double delta, double* w, double* z) {
  w[j] += delta;
  for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) z[pr->row_idx[p]] += delta * pr->val[p];
}

static int64_t col_len(const oracle_problem* pr, int64_t j) { return pr->col_ptr[j + 1] - pr->col_ptr[j]; }

int oracle_run(const oracle_problem* pr, const oracle_params* pa, int64_t t0, int64_t iters, double* w,
               double* z, double* obj_trace, int64_t* stats) {
  int64_t k = pr->k;
  if (k <= 0) return -1;
  int v = pa->variant;
  if (v == ORACLE_SHOTGUN && (pa->P < 1)) return -1;
  if ((v == ORACLE_THREAD_GREEDY || v == ORACLE_TOP_GREEDY) && pa->B < 1) return -1;
  if (v == ORACLE_SHOTGUN_BLOCKS && (pa->B < 1 || pa->block_P == NULL)) return -1;
  if (v == ORACLE_COLORING && (pa->colors == NULL || pa->ncolors < 1)) return -1;

  int32_t* J = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  double* delta = (double*)malloc(sizeof(double) * (size_t)k);
  double* phi = (double*)malloc(sizeof(double) * (size_t)k);
  int64_t* acc = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
  int64_t perm_epoch = -1;
  int64_t n_updates = 0, n_nnz = 0;

  for (int64_t t = t0; t < t0 + iters; ++t) {
    /* Select (Section 2.1, Table 2) */
    int64_t m = 0;
    if (v == ORACLE_CCD) {
      J[m++] = (int32_t)(t % k);
    } else if (v == ORACLE_SHOTGUN) {
      int64_t P = pa->P < k ? pa->P : k;
      int64_t per_epoch = (k + P - 1) / P;
      int64_t e = t / per_epoch, q = t % per_epoch;
      if (e != perm_epoch) {
        oracle_permutation(pa->seed, e, k, perm);
        perm_epoch = e;
      }
      for (int64_t a = q * P; a < k && a < (q + 1) * P; ++a) J[m++] = perm[a];
      qsort(J, (size_t)m, sizeof(int32_t), cmp_i32); /* R5: ascending application */
    } else if (v == ORACLE_SHOTGUN_BLOCKS) { /* R14: P*_b columns from every block */
      for (int32_t b = 0; b < pa->B; ++b) {
        int64_t lo = k * b / pa->B, hi = k * (b + 1) / pa->B, kb = hi - lo;
        if (kb == 0) continue;
        int64_t P = pa->block_P[b] < 1 ? 1 : (pa->block_P[b] < kb ? pa->block_P[b] : kb);
        int64_t per_epoch = (kb + P - 1) / P;
        int64_t e = t / per_epoch, q = t % per_epoch;
        oracle_permutation(pa->seed + (uint64_t)b, e, kb, perm);
        for (int64_t a = q * P; a < kb && a < (q + 1) * P; ++a) J[m++] = (int32_t)(lo + perm[a]);
      }
      qsort(J, (size_t)m, sizeof(int32_t), cmp_i32); /* R5: ascending application */
    } else if (v == ORACLE_COLORING) {
      int64_t C = pa->ncolors;
      int64_t e = t / C, q = t % C;
      if (e != perm_epoch) {
        oracle_permutation(pa->seed, e, C, perm);
        perm_epoch = e;
      }
      int32_t colour = perm[q];
      for (int64_t j = 0; j < k; ++j)
        if (pa->colors[j] == colour) J[m++] = (int32_t)j;
    } else { /* Thread-Greedy, Greedy and top-greedy select all columns */
      for (int64_t j = 0; j < k; ++j) J[m++] = (int32_t)j;
    }

    /* Propose (Algorithm 4) from the iteration-start state (R5) */
    oracle_propose(pr, w, z, J, m, delta, phi);
    for (int64_t a = 0; a < m; ++a) n_nnz += col_len(pr, J[a]);

    /* Accept (Section 2.3): the positions a of the accepted proposals */
    int64_t na = 0;
    if (v == ORACLE_THREAD_GREEDY || v == ORACLE_GREEDY) {
      int64_t B = v == ORACLE_GREEDY ? 1 : pa->B;
      for (int64_t b = 0; b < B; ++b) {
        int64_t lo = (b * m) / B, hi = ((b + 1) * m) / B;
        int64_t best = -1;
        for (int64_t a = lo; a < hi; ++a)
          if (best < 0 || phi[a] < phi[best]) best = a; /* strict: ties keep the lower j */
        if (best >= 0 && phi[best] < 0.0) acc[na++] = best;
      }
    } else if (v == ORACLE_TOP_GREEDY) { /* R12: the B lowest proxies < 0 */
      for (int64_t a = 0; a < m; ++a)
        if (phi[a] < 0.0) acc[na++] = a;
      qsort_ctx_phi = phi;
      qsort(acc, (size_t)na, sizeof(int64_t), cmp_by_phi);
      if (na > pa->B) na = pa->B;
      qsort(acc, (size_t)na, sizeof(int64_t), cmp_i64); /* R5: ascending application */
    } else { /* Shotgun, Coloring, CCD accept every proposal */
      for (int64_t a = 0; a < m; ++a) acc[na++] = a;
    }
    /* Update (Algorithm 3): improve every accepted increment from the
     * iteration-start state (R11), then apply them in ascending j (R5) */
    if (pa->improve_steps > 0)
      for (int64_t r = 0; r < na; ++r)
        delta[acc[r]] = oracle_improve(pr, w, z, J[acc[r]], delta[acc[r]], pa->improve_steps);
    for (int64_t r = 0; r < na; ++r) {
      apply_update(pr, J[acc[r]], delta[acc[r]], w, z);
      n_updates += 1;
      n_nnz += col_len(pr, J[acc[r]]);
    }
    if (obj_trace) obj_trace[t - t0] = oracle_objective_z(pr, w, z);
  }
  if (stats) {
    stats[0] += n_updates;
    stats[1] += n_nnz;
    stats[2] += iters;
  }
  free(J);
  free(perm);
  free(delta);
  free(phi);
  free(acc);
  return 0;
}

int64_t oracle_solve(const oracle_problem* pr, const oracle_params* pa, double tol_kkt, int64_t max_iter,
                     int64_t check_every, double* w, double* z, double* kkt_out, int64_t* stats) {
  int64_t t = 0;
  double kkt = oracle_kkt(pr, w, z);
  if (check_every < 1) check_every = 1;
  while (kkt > tol_kkt && t < max_iter) {
    int64_t step = check_every < max_iter - t ? check_every : max_iter - t;
    if (oracle_run(pr, pa, t, step, w, z, NULL, stats) != 0) break;
    t += step;
    kkt = oracle_kkt(pr, w, z);
    if (!isfinite(kkt)) break;
  }
  if (kkt_out) *kkt_out = kkt;
  return t;
}

/* R10: stored values.  bfloat16 rounding: with u the FP32 bit pattern, the
 * discarded low 16 bits are compared with half of the kept last place; adding
 * 0x7fff plus the kept last bit rounds up exactly when they exceed half, or
 * equal half with an odd kept part (ties to even). */
int64_t oracle_stored_values(int32_t mode, int64_t k, const int64_t* col_ptr, const double* val,
                             double* out) {
  const int64_t nnz = col_ptr[k];
  for (int64_t q = 0; q < nnz; ++q) {
    if (mode == 0) {
      out[q] = val[q];
      continue;
    }
    float f = (float)val[q];
    if (mode == 2) {
      uint32_t u;
      memcpy(&u, &f, 4);
      u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
      memcpy(&f, &u, 4);
      if (!isfinite(f)) return -2;
    }
    out[q] = (double)f;
  }
  if (mode == 3)
    for (int64_t j = 0; j < k; ++j)
      for (int64_t q = col_ptr[j] + 1; q < col_ptr[j + 1]; ++q)
        if (out[q] != out[col_ptr[j]]) return j;
  return -1;
}
