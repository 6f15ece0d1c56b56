/*
 * gencd_omp.h -- Thread-Greedy and Greedy in the OpenMP design of Section 4.2
 * (static schedule, atomic additions to z, a critical section for Greedy):
 * the timed multi-core CPU baseline.  TEST INFRASTRUCTURE, like the oracle it
 * links with; see gencd_omp.c.
 */
#ifndef GENCD_OMP_H
#define GENCD_OMP_H

#include <stdint.h>

#include "gencd_oracle.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct omp_solver omp_solver;

/* Threads OpenMP would use by default (the host's cores unless limited). */
int32_t omp_solver_max_threads(void);
/* A solver state (copies of w and z = Xw, u = l'(y, z), beta_j) for `pr`,
 * run with `threads` threads (<= 0: the default).  NULL on failure. */
omp_solver* omp_solver_create(const oracle_problem* pr, const double* w, const double* z, int32_t threads);
/* `iters` iterations of Thread-Greedy with B partitions (greedy = 0) or of
 * Greedy (greedy = 1); stats (nullable): += accepted updates, non-zeros
 * processed, iterations.  Returns 0 or -1. */
int omp_solver_iterate(omp_solver* s, int32_t B, int32_t greedy, int64_t iters, int64_t* stats);
/* Copies the current w (double[k]) and z (double[n]); either may be NULL. */
void omp_solver_get(const omp_solver* s, double* w, double* z);
void omp_solver_destroy(omp_solver* s);

#ifdef __cplusplus
}
#endif
#endif
