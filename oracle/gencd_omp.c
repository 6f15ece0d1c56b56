/*
 * gencd_omp.c -- Thread-Greedy and Greedy (Table 2) in the shared-memory
 * design of Section 4.2, with OpenMP: the timed multi-core CPU baseline.
 *
 * TEST INFRASTRUCTURE.  Only the benchmark's CPU-baseline leg, its reference
 * arm and the tests load this code; it shares nothing with the CUDA library.
 * The deterministic single-threaded oracle (gencd_oracle.c, whose step and
 * loss derivative this file calls) stays the parity reference.
 *
 * Section 4.2's design, as this file follows it:
 *  - the work of a loop is divided among the threads by a static schedule;
 *  - Thread-Greedy: every partition (a contiguous chunk of columns, as the
 *    oracle's R4 defines them) proposes for all of its columns from the
 *    iteration-start state and keeps its best proxy; with B partitions and T
 *    threads each thread owns B / T partitions;
 *  - the accepted updates are applied in parallel, with atomic additions to
 *    the shared fitted values z;
 *  - Greedy: each thread finds the best proposal of its own columns and the
 *    threads' candidates are merged in a critical section.
 * The loss derivative u = l'(y, z) is kept per row and refreshed on the rows
 * an iteration touched.  With one thread the iterates equal the oracle's bit
 * for bit; with more, the atomic additions to z happen in a varying order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

#include "gencd_oracle.h"

struct omp_solver {
  const oracle_problem* pr;
  int32_t threads;
  double* w;
  double* z;
  double* u;     /* l'(y_i, z_i) */
  double* beta;  /* beta_j of Eq. 7 (R2), computed once */
  int64_t* acc_j;
  double* acc_d;
  int64_t acc_cap;
};

typedef struct omp_solver omp_solver;

int32_t omp_solver_max_threads(void) { return (int32_t)omp_get_max_threads(); }

omp_solver* omp_solver_create(const oracle_problem* pr, const double* w, const double* z, int32_t threads) {
  omp_solver* s = (omp_solver*)calloc(1, sizeof(omp_solver));
  if (!s) return NULL;
  const int64_t n = pr->n, k = pr->k;
  s->pr = pr;
  s->threads = threads > 0 ? threads : omp_get_max_threads();
  s->w = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
  s->z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  s->u = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  s->beta = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
  if (!s->w || !s->z || !s->u || !s->beta) {
    free(s->w), free(s->z), free(s->u), free(s->beta), free(s);
    return NULL;
  }
  memcpy(s->w, w, sizeof(double) * (size_t)k);
  memcpy(s->z, z, sizeof(double) * (size_t)n);
  const double b = oracle_beta(pr->loss);
#pragma omp parallel for schedule(static) num_threads(s->threads)
  for (int64_t i = 0; i < n; ++i) s->u[i] = oracle_dloss(pr->loss, pr->y[i], s->z[i]);
#pragma omp parallel for schedule(static) num_threads(s->threads)
  for (int64_t j = 0; j < k; ++j) {
    double ss = 0.0;
    for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) ss += pr->val[p] * pr->val[p];
    s->beta[j] = pr->beta_mode == 1 ? b : b * ss / (double)pr->n;
  }
  return s;
}

void omp_solver_destroy(omp_solver* s) {
  if (!s) return;
  free(s->w), free(s->z), free(s->u), free(s->beta), free(s->acc_j), free(s->acc_d), free(s);
}

void omp_solver_get(const omp_solver* s, double* w, double* z) {
  if (w) memcpy(w, s->w, sizeof(double) * (size_t)s->pr->k);
  if (z) memcpy(z, s->z, sizeof(double) * (size_t)s->pr->n);
}

/* g_j = <u, X_j> / n in CSC order (Algorithm 4), then Eq. 7 and Eq. 9 */
static void propose_one(const omp_solver* s, int64_t j, double* d, double* f) {
  const oracle_problem* pr = s->pr;
  double acc = 0.0;
  for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) acc += pr->val[p] * s->u[pr->row_idx[p]];
  oracle_step(acc / (double)pr->n, s->w[j], pr->lambda, s->beta[j], d, f);
}

/* Runs `iters` iterations of Thread-Greedy with B partitions (greedy = 0) or
 * of Greedy (greedy = 1).  stats (nullable, 3 entries) accumulates accepted
 * updates, non-zeros processed and iterations.  Returns 0, or -1 on invalid
 * parameters or allocation failure. */
int omp_solver_iterate(omp_solver* s, int32_t B, int32_t greedy, int64_t iters, int64_t* stats) {
  const oracle_problem* pr = s->pr;
  const int64_t k = pr->k;
  if (k < 1 || iters < 0 || (!greedy && B < 1)) return -1;
  const int64_t parts = greedy ? 1 : (B < k ? B : k);
  if (s->acc_cap < parts) {
    free(s->acc_j), free(s->acc_d);
    s->acc_j = (int64_t*)malloc(sizeof(int64_t) * (size_t)parts);
    s->acc_d = (double*)malloc(sizeof(double) * (size_t)parts);
    if (!s->acc_j || !s->acc_d) return -1;
    s->acc_cap = parts;
  }
  int64_t* acc_j = s->acc_j;
  double* acc_d = s->acc_d;
  double* w = s->w;
  double* z = s->z;
  double* u = s->u;
  int64_t upd = 0, nnz = 0;
  for (int64_t t = 0; t < iters; ++t) {
    /* Select all columns; Propose and Accept */
    if (greedy) {
      int64_t gbest = -1;
      double gphi = 0.0, gd = 0.0;
#pragma omp parallel num_threads(s->threads)
      {
        int64_t best = -1;
        double bphi = 0.0, bd = 0.0;
#pragma omp for schedule(static) nowait
        for (int64_t j = 0; j < k; ++j) {
          double d, f;
          propose_one(s, j, &d, &f);
          if (best < 0 || f < bphi) best = j, bphi = f, bd = d; /* strict: ties keep the lower j */
        }
#pragma omp critical
        {
          if (best >= 0 && (gbest < 0 || bphi < gphi || (bphi == gphi && best < gbest)))
            gbest = best, gphi = bphi, gd = bd;
        }
      }
      acc_j[0] = (gbest >= 0 && gphi < 0.0) ? gbest : -1;
      acc_d[0] = gd;
    } else {
#pragma omp parallel for schedule(static) num_threads(s->threads)
      for (int64_t b = 0; b < parts; ++b) {
        const int64_t lo = (b * k) / parts, hi = ((b + 1) * k) / parts;
        int64_t best = -1;
        double bphi = 0.0, bd = 0.0;
        for (int64_t j = lo; j < hi; ++j) {
          double d, f;
          propose_one(s, j, &d, &f);
          if (best < 0 || f < bphi) best = j, bphi = f, bd = d;
        }
        acc_j[b] = (best >= 0 && bphi < 0.0) ? best : -1;
        acc_d[b] = bd;
      }
    }
    nnz += pr->col_ptr[k];
    /* Update (Algorithm 3): w_j += delta, z += delta X_j with atomic adds */
    int64_t t_upd = 0, t_nnz = 0;
#pragma omp parallel for schedule(static) num_threads(s->threads) reduction(+ : t_upd, t_nnz)
    for (int64_t b = 0; b < parts; ++b) {
      const int64_t j = acc_j[b];
      if (j < 0) continue;
      const double d = acc_d[b];
      w[j] += d;
      for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) {
        const double x = d * pr->val[p];
#pragma omp atomic
        z[pr->row_idx[p]] += x;
      }
      t_upd += 1;
      t_nnz += pr->col_ptr[j + 1] - pr->col_ptr[j];
    }
    /* u = l'(y, z) on the touched rows */
#pragma omp parallel for schedule(static) num_threads(s->threads)
    for (int64_t b = 0; b < parts; ++b) {
      const int64_t j = acc_j[b];
      if (j < 0) continue;
      for (int64_t p = pr->col_ptr[j]; p < pr->col_ptr[j + 1]; ++p) {
        const int32_t i = pr->row_idx[p];
#pragma omp atomic write
        u[i] = oracle_dloss(pr->loss, pr->y[i], z[i]);
      }
    }
    upd += t_upd;
    nnz += t_nnz;
  }
  if (stats) {
    stats[0] += upd;
    stats[1] += nnz;
    stats[2] += iters;
  }
  return 0;
}
