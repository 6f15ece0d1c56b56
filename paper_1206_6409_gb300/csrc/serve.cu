// serve.cu -- the serving loop of include/gencd_serve.h: requests admitted
// into slots as memory frees, their solves advanced together on the device.
//
// Runtime (host code only: every step of a solve runs in the library's
// kernels on its slot's stream):
//  - memory: one stream-ordered memory pool reserved at start (the budget);
//    a request's problem takes all of its device buffers from it and returns
//    them when it is done, so no request calls cudaMalloc or cudaFree (which
//    would stall the device for every other request);
//  - slots: each slot owns a CUDA stream and a pinned block for its solve's
//    scalars;
//  - a loader thread admits the next arrived request (first come, first
//    served) when a slot is free and its HBM estimate fits the budget, creates
//    its problem on the slot's stream (copies, validation, setup) and starts
//    its solve;
//  - the calling thread is the stepper: it polls every running slot's last
//    enqueued work (an event), and when it has completed takes the solve's
//    next decision and enqueues its next iterations (gencd_solve's loop, one
//    step at a time: solve_advance), so the kernels of all requests in
//    flight overlap on the device while no host thread waits on one solve.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gencd_internal.cuh"
#include "gencd_serve.h"

namespace gencd {

namespace {

using Clock = std::chrono::steady_clock;

enum SlotState { kFree = 0, kLoading = 1, kRunning = 2 };

struct Slot {
  int state = kFree;
  cudaStream_t st = nullptr;
  double* hpin = nullptr;  // kScalars pinned doubles lent to the slot's problem
  gencd_problem* p = nullptr;
  SolveRun S;
  int64_t q = -1;
  double need = 0.0;
  double deadline = 0.0;  // dry run: when the request releases the slot
};

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
  int inflight = 0;       // slots loading or running
  int err = GENCD_OK;
  std::string err_msg;
  std::vector<Slot> slots;
  std::deque<int> started;  // slots the loader has started (handed to the stepper)
  cudaMemPool_t pool = nullptr;
  double* pinned = nullptr;
  const double* service = nullptr;  // dry run: seconds each request holds its slot (no GPU work)

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

// Device bytes of one problem: the CSC, the streaming plan (at most one more
// copy of the entries with its masks), a row-major copy and the scratch of
// its sort (built when a solve restarts from its start state or needs z =
// Xw), per-row state (y, z, u), per-column state (w, c, beta_j, sums, steps,
// proxies, lists, the Thread-Greedy backoff's start point, the top-|J'|
// Accept's sort buffers) and a fixed allowance for small buffers.
double footprint(const gencd_request& r, int precision, const gencd_params& params) {
  const double vsz = precision == GENCD_F64 ? 8.0 : 4.0;
  const double nnz = (double)r.nnz, n = (double)r.n, k = (double)r.k;
  double b = nnz * (4.0 + vsz)               // CSC
             + nnz * (4.0 + vsz + 0.25)      // streaming plan
             + nnz * (4.0 + vsz) + 8.0 * n   // row-major copy
             + nnz * 24.0                    // its sort scratch
             + n * (16.0 + vsz)              // y, z, u
             + k * 128.0                     // per-column state and lists
             + 64.0 * (1 << 20);
  if (params.variant == GENCD_THREAD_GREEDY || params.variant == GENCD_TOP_GREEDY) b += 8.0 * k;  // backoff start
  if (params.variant == GENCD_TOP_GREEDY) b += 28.0 * k;  // sort keys, indices and scratch
  return b;
}

void respond(Server* S, Slot& sl, int status, const gencd_result* res) {
  gencd_response& o = S->out[sl.q];
  o.status = status;
  if (res) {
    o.iters = res->iters;
    o.objective = res->objective;
    o.kkt = res->kkt;
  }
  o.end = S->now();
}

// releases a slot (its problem destroyed: buffers back to the pool in stream order)
void release(Server* S, int i) {
  Slot& sl = S->slots[(size_t)i];
  if (sl.p) {
    gencd_destroy(sl.p);
    sl.p = nullptr;
  }
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->held -= sl.need;
    S->inflight -= 1;
    sl.state = kFree;
    sl.q = -1;
  }
  S->cv.notify_all();
}

// creates request q's problem in slot i and starts its solve; false when the
// request failed (its response is written and the slot released)
bool load(Server* S, int i) {
  Slot& sl = S->slots[(size_t)i];
  const gencd_request& r = S->req[sl.q];
  gencd_response& o = S->out[sl.q];
  if (S->service) {  // dry run
    sl.deadline = S->now() + S->service[sl.q];
    return true;
  }
  gencd_problem* p = nullptr;
  int rc = create_problem(&p, r.n, r.k, r.nnz, r.col_ptr, r.row_idx, r.val, r.val_dtype, r.y, r.loss,
                          S->sp.precision, GENCD_HOST, sl.st, S->pool, sl.hpin);
  if (rc == GENCD_OK) {
    sl.p = p;
    double lmax = 0.0;
    gencd_lambda_max(p, &lmax);
    o.lambda = r.lambda_frac * lmax;
    rc = gencd_set_lambda(p, o.lambda);
    gencd_params a = S->sp.params;
    if (S->sp.tol_rel > 0.0) a.tol_kkt = S->sp.tol_rel * o.lambda;  // a tolerance relative to the request's lambda
    if (rc == GENCD_OK) rc = gencd_set_params(p, &a);
    if (rc == GENCD_OK) rc = solve_begin(p, &sl.S);
  }
  if (rc != GENCD_OK) {
    respond(S, sl, rc, nullptr);
    release(S, i);
    return false;
  }
  return true;
}

// admits requests into free slots in arrival order and loads them
void loader(Server* S) {
  if (!S->service && cudaSetDevice(S->device) != cudaSuccess) {
    cudaGetLastError();
    std::lock_guard<std::mutex> g(S->mu);
    if (S->err == GENCD_OK) {
      S->err = GENCD_ECUDA;
      S->err_msg = "the loader thread could not select the device";
    }
    S->cv.notify_all();
    return;
  }
  for (;;) {
    int i = -1;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->err != GENCD_OK || S->next >= S->nreq) return;
        const gencd_request& r = S->req[S->next];
        const double wait = r.arrival - S->now();
        if (wait > 0.0) {  // not arrived yet
          S->cv.wait_for(lk, std::chrono::duration<double>(std::min(wait, 0.01)));
          continue;
        }
        const double need = footprint(r, S->sp.precision, S->sp.params);
        int free_slot = -1;
        for (size_t s = 0; s < S->slots.size(); ++s)
          if (S->slots[s].state == kFree) {
            free_slot = (int)s;
            break;
          }
        // a slot is free and the estimate fits (a request above the whole
        // budget runs alone)
        if (free_slot >= 0 && (S->inflight == 0 || S->held + need <= S->budget)) {
          i = free_slot;
          Slot& sl = S->slots[(size_t)i];
          sl.state = kLoading;
          sl.q = S->next++;
          sl.need = need;
          S->held += need;
          S->inflight += 1;
          gencd_response& o = S->out[sl.q];
          o.arrival = r.arrival;
          o.start = S->now();
          o.bytes = (int64_t)need;
          o.worker = i;
          break;
        }
        S->cv.wait_for(lk, std::chrono::milliseconds(2));  // a finishing request frees a slot or budget
      }
    }
    if (load(S, i)) {
      std::lock_guard<std::mutex> g(S->mu);
      S->slots[(size_t)i].state = kRunning;
      S->started.push_back(i);
    }
  }
}

// advances every running slot whose last work has completed; returns when the
// stream is served or an error stopped it
void stepper(Server* S) {
  std::vector<int> running;
  for (;;) {
    {
      std::lock_guard<std::mutex> g(S->mu);
      while (!S->started.empty()) {
        running.push_back(S->started.front());
        S->started.pop_front();
      }
      if (S->err != GENCD_OK) return;
      if (running.empty() && S->inflight == 0 && S->next >= S->nreq) return;
    }
    bool progressed = false;
    for (size_t t = 0; t < running.size();) {
      const int i = running[t];
      Slot& sl = S->slots[(size_t)i];
      int r = 1;
      gencd_result res;
      std::memset(&res, 0, sizeof(res));
      if (S->service) {
        if (S->now() >= sl.deadline) r = 0, sl.S.status = GENCD_OK;
      } else {
        const cudaError_t e = cudaEventQuery(sl.p->ev_scalars);
        if (e == cudaErrorNotReady) {
          ++t;
          continue;
        }
        r = e == cudaSuccess ? solve_advance(sl.p, &sl.S) : GENCD_ECUDA;
        if (e != cudaSuccess) cudaGetLastError();
      }
      progressed = true;
      if (r == 1) {  // more work enqueued
        ++t;
        continue;
      }
      int status = r < 0 ? r : sl.S.status;
      if (!S->service && r == 0) {
        solve_result(sl.p, &sl.S, &res);
        if (S->w_out && S->w_out[sl.q]) {
          const int rw = gencd_get_w(sl.p, S->w_out[sl.q], S->req[sl.q].k, GENCD_HOST);
          if (rw < 0) status = rw;
        }
      }
      respond(S, sl, status, S->service ? nullptr : &res);
      release(S, i);
      running[t] = running.back();
      running.pop_back();
    }
    if (!progressed) {  // nothing completed: wait a little for the device or an admission
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait_for(lk, std::chrono::microseconds(100));
    }
  }
}

int check_stream(const gencd_request* requests, int64_t nreq, const gencd_serve_params* params, gencd_response* out) {
  if (nreq < 0 || (nreq > 0 && (!requests || !out)) || !params) {
    set_error("bad requests / params / out");
    return GENCD_EINVAL;
  }
  if (params->workers < 1 || params->workers > 64 || !(params->hbm_fraction > 0.0) || params->hbm_fraction > 1.0 ||
      (params->precision < GENCD_F64 || params->precision > GENCD_BINARY) || !(params->tol_rel >= 0.0)) {
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

// runs the loader and the stepper to the end of the stream
int run(Server& S) {
  S.t0 = Clock::now();
  std::thread th;
  try {
    th = std::thread(loader, &S);
  } catch (const std::exception& e) {  // no exception crosses the C ABI
    set_error(std::string("loader thread creation failed: ") + e.what());
    return GENCD_ENOMEM;
  }
  stepper(&S);
  if (S.err != GENCD_OK) S.cv.notify_all();
  th.join();
  // a request the loader started after the stepper stopped on an error
  for (size_t i = 0; i < S.slots.size(); ++i)
    if (S.slots[i].p) {
      gencd_destroy(S.slots[i].p);
      S.slots[i].p = nullptr;
    }
  if (S.err != GENCD_OK) {
    set_error(S.err_msg);
    return S.err;
  }
  return GENCD_OK;
}

// slots, their streams and pinned scalars, and the memory pool with the
// budget reserved (allocated once and returned to the pool, which keeps it)
int setup(Server& S, int slots) {
  S.slots.resize((size_t)slots);
  if (S.service) return GENCD_OK;
  GENCD_CUDA_TRY(cudaMallocHost((void**)&S.pinned, sizeof(double) * kScalars * (size_t)slots));
  for (int i = 0; i < slots; ++i) {
    GENCD_CUDA_TRY(cudaStreamCreateWithFlags(&S.slots[(size_t)i].st, cudaStreamNonBlocking));
    S.slots[(size_t)i].hpin = S.pinned + kScalars * i;
  }
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = S.device;
  GENCD_CUDA_TRY(cudaMemPoolCreate(&S.pool, &props));
  uint64_t keep = (uint64_t)S.budget;
  GENCD_CUDA_TRY(cudaMemPoolSetAttribute(S.pool, cudaMemPoolAttrReleaseThreshold, &keep));
  void* reserve = nullptr;
  cudaStream_t st = S.slots[0].st;
  GENCD_CUDA_TRY(cudaMallocFromPoolAsync(&reserve, (size_t)S.budget, S.pool, st));
  GENCD_CUDA_TRY(cudaFreeAsync(reserve, st));
  GENCD_CUDA_TRY(cudaStreamSynchronize(st));
  return GENCD_OK;
}

void teardown(Server& S) {
  for (auto& sl : S.slots)
    if (sl.st) {
      cudaStreamSynchronize(sl.st);
      cudaStreamDestroy(sl.st);
    }
  if (S.pool) cudaMemPoolDestroy(S.pool);
  if (S.pinned) cudaFreeHost(S.pinned);
  cudaGetLastError();
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
  int rc = setup(S, params->workers);
  if (rc == GENCD_OK) rc = run(S);
  teardown(S);
  return rc;
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
  GENCD_TRY(setup(S, params->workers));
  return run(S);
}
