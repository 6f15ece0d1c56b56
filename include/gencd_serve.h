/*
 * gencd_serve.h -- a serving loop for independent l1 solves on one GPU.
 *
 * Requests are separate problems (their own X, y, loss and lambda) that
 * arrive over time.  gencd_serve keeps up to `workers` requests in flight in
 * slots: it admits each arrived request, in arrival order, as soon as a slot
 * is free and the HBM it needs fits the budget, solves it to its KKT
 * tolerance (gencd_solve's loop: Algorithm 1 with the configured variant and
 * its accept backoff) and returns its memory for the next.  Device memory
 * comes from one memory pool reserved at the start of the call, so no
 * request allocates or frees device memory itself (cudaMalloc / cudaFree
 * would stall the device for the others).  Every slot owns a CUDA stream; one
 * host thread creates the admitted requests' problems and another advances
 * every running solve whenever its last enqueued iterations have completed,
 * so the kernels of all requests in flight overlap on the device.  A
 * request's result does not depend on which others run beside it (its
 * arithmetic is its own; sums reach it in a rounding order that can vary from
 * run to run).
 *
 * Conventions (status codes, thread-local error message) are those of
 * include/gencd.h.  The paper has no serving loop; this is a deployment entry
 * point around its method.
 */
#ifndef GENCD_SERVE_H
#define GENCD_SERVE_H

#include <stdint.h>

#include "gencd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int64_t n, k, nnz;        /* X is n x k with nnz non-zeros (CSC, as gencd_create) */
  const int64_t* col_ptr;   /* host arrays, valid until gencd_serve returns         */
  const int32_t* row_idx;
  const void* val;          /* double (val_dtype 0) or float (val_dtype 1)          */
  int32_t val_dtype;
  int32_t loss;             /* gencd_loss                                           */
  const double* y;
  double lambda_frac;       /* lambda = lambda_frac * lambda_max of this problem    */
  double arrival;           /* seconds after the call starts; non-decreasing        */
} gencd_request;

typedef struct {
  int32_t workers;      /* slots: requests in flight at most (one stream each), 1..64  */
  int32_t precision;    /* gencd_precision of every request                             */
  double hbm_fraction;  /* share of the device's free memory at the start that the
                           memory pool reserves and the requests in flight may hold
                           (0 < f <= 1); a request whose estimate exceeds the whole
                           budget runs alone                                          */
  gencd_params params;  /* iteration parameters of every solve                         */
  double tol_rel;       /* > 0: request q stops at KKT <= tol_rel * lambda_q instead of
                           params.tol_kkt                                              */
} gencd_serve_params;

typedef struct {
  int32_t status;   /* gencd_solve's status (or the error of gencd_create)  */
  int32_t worker;   /* slot that ran the request                             */
  int64_t iters;    /* GenCD iterations                                      */
  double lambda;    /* lambda_frac * lambda_max                              */
  double objective; /* P(w) of Eq. 1 (FP64)                                  */
  double kkt;       /* KKT violation of the returned w                       */
  double arrival;   /* seconds from the start of the call                    */
  double start;     /* admission                                             */
  double end;       /* result ready; latency = end - arrival                 */
  int64_t bytes;    /* HBM estimate the request was admitted with            */
} gencd_response;

/*
 * Runs the request stream to the end and returns GENCD_OK (every request
 * has a response; see each status) or an error that stopped the loop.
 * out: gencd_response[nreq].  w_out: NULL, or nreq pointers (each NULL or a
 * host double[k] of its request) that receive each solution.  Requests are
 * admitted in arrival order (first come, first served).
 * Errors: GENCD_EINVAL (bad parameters, arrivals out of order), GENCD_ECUDA.
 */
int gencd_serve(const gencd_request* requests, int64_t nreq, const gencd_serve_params* params, gencd_response* out,
                double* const* w_out);

/*
 * The same admission policy without a GPU, for capacity planning: request q
 * holds a slot for service_s[q] seconds (no GPU work, the X arrays are not
 * read), the budget is hbm_fraction * budget_bytes and each request's HBM
 * estimate is computed as gencd_serve does.  Fills worker, arrival, start,
 * end and bytes of every response (status GENCD_OK).
 */
int gencd_serve_dry_run(const gencd_request* requests, int64_t nreq, const gencd_serve_params* params,
                        double budget_bytes, const double* service_s, gencd_response* out);

#ifdef __cplusplus
}
#endif

#endif /* GENCD_SERVE_H */
