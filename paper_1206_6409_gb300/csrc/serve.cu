// serve.cu -- the serving loop of include/gencd_serve.h: worker threads, one
// CUDA stream each, take arrived requests in arrival order when the HBM
// budget admits them, solve each with the library's own calls and record its
// timings.  Host code only: every step of a solve runs in the library's
// kernels on the worker's stream.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gencd_internal.cuh"
#include "gencd_serve.h"

namespace gencd {

namespace {

using Clock = std::chrono::steady_clock;

struct Server {
  const gencd_request* req = nullptr;
  int64_t nreq = 0;
  gencd_serve_params sp{};
  gencd_response* out = nullptr;
  double* const* w_out = nullptr;
  int device = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  int64_t next = 0;       // next request to admit (arrival order)
  double budget = 0.0;    // bytes the requests in flight may hold
  double held = 0.0;      // estimates of the requests in flight
  int running = 0;
  int err = GENCD_OK;
  std::string err_msg;
  const double* service = nullptr;  // dry run: seconds each request holds its worker (no GPU work)

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

// Device bytes of one problem: the CSC, the streaming plan (at most one more
// copy of the entries), a row-major copy (built when a solve needs z = Xw
// from scratch), per-row and per-column state, and a fixed allowance.
double footprint(const gencd_request& r, int precision) {
  const double vsz = precision == GENCD_F64 ? 8.0 : 4.0;
  return (double)r.nnz * (4.0 + vsz) * 3.0 + (double)r.n * 48.0 + (double)r.k * 96.0 + 64.0 * (1 << 20);
}

void solve_one(Server* S, int wid, int64_t q, cudaStream_t st) {
  const gencd_request& r = S->req[q];
  gencd_response& o = S->out[q];
  gencd_problem* p = nullptr;
  int rc = gencd_create(&p, r.n, r.k, r.nnz, r.col_ptr, r.row_idx, r.val, r.val_dtype, r.y, r.loss,
                        S->sp.precision, GENCD_HOST, st);
  o.worker = wid;
  if (rc == GENCD_OK) {
    double lmax = 0.0;
    gencd_lambda_max(p, &lmax);
    o.lambda = r.lambda_frac * lmax;
    rc = gencd_set_lambda(p, o.lambda);
    if (rc == GENCD_OK) rc = gencd_set_params(p, &S->sp.params);
    gencd_result res;
    std::memset(&res, 0, sizeof(res));
    if (rc == GENCD_OK) {
      rc = gencd_solve(p, &res);
      o.iters = res.iters;
      o.objective = res.objective;
      o.kkt = res.kkt;
    }
    if (rc >= 0 && S->w_out && S->w_out[q]) {
      const int rw = gencd_get_w(p, S->w_out[q], r.k, GENCD_HOST);
      if (rw < 0) rc = rw;
    }
  }
  if (p) gencd_destroy(p);
  o.status = rc;
  o.end = S->now();
}

void dry_one(Server* S, int wid, int64_t q) {
  std::this_thread::sleep_for(std::chrono::duration<double>(S->service[q]));
  S->out[q].worker = wid;
  S->out[q].status = GENCD_OK;
  S->out[q].end = S->now();
}

void worker(Server* S, int wid) {
  cudaStream_t st = nullptr;
  if (!S->service) cudaSetDevice(S->device);
  if (!S->service && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    std::lock_guard<std::mutex> g(S->mu);
    S->err = GENCD_ECUDA;
    S->err_msg = "worker stream creation failed";
    S->cv.notify_all();
    return;
  }
  for (;;) {
    int64_t q = -1;
    double need = 0.0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->err != GENCD_OK || S->next >= S->nreq) break;
        const gencd_request& r = S->req[S->next];
        const double wait = r.arrival - S->now();
        if (wait > 0.0) {  // not arrived yet
          S->cv.wait_for(lk, std::chrono::duration<double>(std::min(wait, 0.05)));
          continue;
        }
        need = footprint(r, S->sp.precision);
        if (S->running == 0 || S->held + need <= S->budget) {  // admitted
          q = S->next++;
          S->held += need;
          S->running += 1;
          S->out[q].arrival = r.arrival;
          S->out[q].start = S->now();
          S->out[q].bytes = (int64_t)need;
          break;
        }
        S->cv.wait_for(lk, std::chrono::milliseconds(20));  // a finishing request frees budget
      }
    }
    if (q < 0) break;
    if (S->service)
      dry_one(S, wid, q);
    else
      solve_one(S, wid, q, st);
    {
      std::lock_guard<std::mutex> g(S->mu);
      S->held -= need;
      S->running -= 1;
    }
    S->cv.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

int check_stream(const gencd_request* requests, int64_t nreq, const gencd_serve_params* params, gencd_response* out) {
  if (nreq < 0 || (nreq > 0 && (!requests || !out)) || !params) {
    set_error("bad requests / params / out");
    return GENCD_EINVAL;
  }
  if (params->workers < 1 || params->workers > 64 || !(params->hbm_fraction > 0.0) || params->hbm_fraction > 1.0 ||
      (params->precision < GENCD_F64 || params->precision > GENCD_BINARY)) {
    set_error("serve parameters out of range");
    return GENCD_EINVAL;
  }
  for (int64_t q = 0; q < nreq; ++q) {
    if (!std::isfinite(requests[q].arrival) || requests[q].arrival < 0.0 ||
        (q > 0 && requests[q].arrival < requests[q - 1].arrival)) {
      set_error("request " + std::to_string(q) + ": arrival times must be finite, >= 0 and non-decreasing");
      return GENCD_EINVAL;
    }
    if (!(requests[q].lambda_frac >= 0.0) || !std::isfinite(requests[q].lambda_frac)) {
      set_error("request " + std::to_string(q) + ": lambda_frac must be finite and >= 0");
      return GENCD_EINVAL;
    }
  }
  return GENCD_OK;
}

// runs the workers to the end of the stream; S is filled but for t0
int run_workers(Server& S, int workers) {
  S.t0 = Clock::now();
  std::vector<std::thread> th;
  try {
    th.reserve((size_t)workers);
    for (int w = 0; w < workers; ++w) th.emplace_back(worker, &S, w);
  } catch (const std::exception& e) {  // no exception crosses the C ABI: stop the workers already started
    {
      std::lock_guard<std::mutex> g(S.mu);
      if (S.err == GENCD_OK) {
        S.err = GENCD_ENOMEM;
        S.err_msg = std::string("worker thread creation failed: ") + e.what();
      }
    }
    S.cv.notify_all();
  }
  for (auto& t : th) t.join();
  if (S.err != GENCD_OK) {
    set_error(S.err_msg);
    return S.err;
  }
  return GENCD_OK;
}

}  // namespace

}  // namespace gencd

using namespace gencd;

extern "C" int gencd_serve(const gencd_request* requests, int64_t nreq, const gencd_serve_params* params,
                           gencd_response* out, double* const* w_out) {
  GENCD_TRY(check_stream(requests, nreq, params, out));
  std::memset(out, 0, sizeof(gencd_response) * (size_t)nreq);
  Server S;
  S.req = requests;
  S.nreq = nreq;
  S.sp = *params;
  S.out = out;
  S.w_out = w_out;
  if (cudaGetDevice(&S.device) != cudaSuccess) {
    set_error("no CUDA device");
    return GENCD_ECUDA;
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    set_error("cudaMemGetInfo failed");
    return GENCD_ECUDA;
  }
  S.budget = (double)free_b * params->hbm_fraction;
  return run_workers(S, params->workers);
}

extern "C" int gencd_serve_dry_run(const gencd_request* requests, int64_t nreq, const gencd_serve_params* params,
                                   double budget_bytes, const double* service_s, gencd_response* out) {
  GENCD_TRY(check_stream(requests, nreq, params, out));
  if (!(budget_bytes > 0.0) || (nreq > 0 && !service_s)) {
    set_error("budget_bytes must be > 0 and service_s given");
    return GENCD_EINVAL;
  }
  for (int64_t q = 0; q < nreq; ++q)
    if (!(service_s[q] >= 0.0) || !std::isfinite(service_s[q])) {
      set_error("service_s[" + std::to_string(q) + "] must be finite and >= 0");
      return GENCD_EINVAL;
    }
  std::memset(out, 0, sizeof(gencd_response) * (size_t)nreq);
  Server S;
  S.req = requests;
  S.nreq = nreq;
  S.sp = *params;
  S.out = out;
  S.budget = budget_bytes * params->hbm_fraction;
  S.service = service_s;
  return run_workers(S, params->workers);
}
