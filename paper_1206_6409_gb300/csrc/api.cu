// api.cu -- the C ABI of libgencd: problem lifecycle, the GenCD iteration
// loop (Algorithm 1) for each variant of Table 2, and the parity hooks.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "device_math.cuh"
#include "gencd_internal.cuh"

namespace gencd {

static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
const char* last_error() { return g_err.c_str(); }

static int fail(int code, const std::string& m) {
  set_error(m);
  return code;
}

// ---- profiling -------------------------------------------------------------
static void prof_flush(gencd_problem* p) {
  if (p->prof.used == 0) return;
  cudaStreamSynchronize(p->stream);
  for (size_t q = 0; q < p->prof.pending_id.size(); ++q) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->prof.pool[2 * q], p->prof.pool[2 * q + 1]) == cudaSuccess)
      p->prof.ms[p->prof.pending_id[q]] += ms;
  }
  cudaGetLastError();
  p->prof.pending_id.clear();
  p->prof.used = 0;
}

void prof_begin(gencd_problem* p, int id, cudaEvent_t* stop, int launches) {
  p->prof.launches[id] += launches;
  p->prof.calls[id] += 1;
  *stop = nullptr;
  if (!p->prof.enabled || p->prof.pool.empty()) return;
  if (p->prof.used + 2 > p->prof.pool.size()) prof_flush(p);
  cudaEvent_t a = p->prof.pool[p->prof.used];
  *stop = p->prof.pool[p->prof.used + 1];
  p->prof.used += 2;
  p->prof.pending_id.push_back(id);
  cudaEventRecord(a, p->stream);
}

void prof_end(gencd_problem* p, cudaEvent_t stop) {
  if (stop) cudaEventRecord(stop, p->stream);
}

// ---- small kernels used only here -------------------------------------------
template <typename S, typename D>
__global__ void k_convert(const S* __restrict__ in, int64_t m, D* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) out[i] = (D)in[i];
}

__global__ void k_inv_beta(const double* __restrict__ c, int64_t k, double beta, int beta_mode,
                           double* __restrict__ bj, double* __restrict__ ib, float* __restrict__ bj32,
                           float* __restrict__ ib32) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    const double b = beta_mode ? beta : beta * c[j];
    bj[j] = b;
    ib[j] = b > 0.0 ? 1.0 / b : 0.0;
    if (bj32) {
      bj32[j] = (float)b;
      ib32[j] = b > 0.0 ? (float)(1.0 / b) : 0.0f;
    }
  }
}

__global__ void k_mirror_w(const double* __restrict__ w, int64_t k, float* __restrict__ w32) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) w32[j] = w_mirror(w[j]);
}

int launch_mirror_w(gencd_problem* p) {
  if (!p->w32) return GENCD_OK;
  k_mirror_w<<<grid_for(p->k, kThreads, p->num_sms * 8), kThreads, 0, p->stream>>>(p->w, p->k, p->w32);
  p->prof.launches[K_SETUP] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

int launch_inv_beta(gencd_problem* p) {
  if (p->ib_mode == p->params.beta_mode) return GENCD_OK;
  const double beta = p->loss == GENCD_LOSS_SQUARED ? 1.0 : 0.25;
  k_inv_beta<<<grid_for(p->k, kThreads, p->num_sms * 8), kThreads, 0, p->stream>>>(
      p->c, p->k, beta, p->params.beta_mode, p->bj, p->ib, p->bj32, p->ib32);
  p->prof.launches[K_SETUP] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  p->ib_mode = p->params.beta_mode;
  return GENCD_OK;
}

// D^-1/2 and the start vector of the power iteration on the columns
// [lo, hi): v_j = 1 / sqrt(hi - lo) there, 0 elsewhere
__global__ void k_dinv(const double* __restrict__ c, int64_t k, double n, int64_t lo, int64_t hi,
                       double* __restrict__ dinv, double* __restrict__ v) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const double v0 = 1.0 / sqrt((double)(hi - lo));
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    const double s = c[j] * n;  // ||X_j||^2
    dinv[j] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    v[j] = (j >= lo && j < hi) ? v0 : 0.0;
  }
}

// t_j = dinv_j * gacc_j on the columns [lo, hi), 0 elsewhere (gacc reset to
// 0); red[block] = sum of t_j^2
__global__ void __launch_bounds__(kThreads)
    k_power_finish(double* __restrict__ gacc, const double* __restrict__ dinv, int64_t k, int64_t lo, int64_t hi,
                   double* __restrict__ t, double* __restrict__ red) {
  __shared__ double sm[kThreads / 32];
  double s = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    const double x = (j >= lo && j < hi) ? dinv[j] * gacc[j] : 0.0;
    gacc[j] = 0.0;
    t[j] = x;
    s = fma(x, x, s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) b += sm[q];
    red[blockIdx.x] = b;
  }
}

__global__ void k_sum_partials(const double* __restrict__ red, int nb, double* __restrict__ out) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) s += red[b];
  s = warp_sum(s);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_div(const double* __restrict__ t, int64_t k, double r, double* __restrict__ v) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) v[j] = t[j] / r;
}

__global__ void k_check_colors(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                               const int32_t* __restrict__ color, int64_t n, int64_t k,
                               unsigned long long* __restrict__ bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    for (int64_t a = row_ptr[i]; a < row_ptr[i + 1]; ++a) {
      const int32_t ca = color[col_idx[a]];
      if (ca < 0 || ca >= k) atomicMin(bad, (unsigned long long)i);
      for (int64_t b = a + 1; b < row_ptr[i + 1]; ++b)
        if (color[col_idx[b]] == ca) atomicMin(bad, (unsigned long long)i);
    }
  }
}

__global__ void k_max_i32(const int32_t* __restrict__ a, int64_t m, unsigned long long* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int32_t mx = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) mx = a[i] > mx ? a[i] : mx;
  atomicMax(out, (unsigned long long)mx);
}

// ---- helpers -----------------------------------------------------------------
static cudaMemcpyKind kind_in(int32_t memory) {
  return memory == GENCD_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
static cudaMemcpyKind kind_out(int32_t memory) {
  return memory == GENCD_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

int dev_alloc_bytes(gencd_problem* p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  const cudaError_t e = p->pool ? cudaMallocFromPoolAsync(ptr, bytes, p->pool, p->stream) : cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(GENCD_ENOMEM, std::string(p->pool ? "allocation from the memory pool" : "cudaMalloc") + " of " +
                                  std::to_string(bytes) + " bytes failed");
  }
  return GENCD_OK;
}

void dev_free(gencd_problem* p, void* ptr) {
  if (!ptr) return;
  if (p->pool)
    cudaFreeAsync(ptr, p->stream);
  else
    cudaFree(ptr);
}

int ensure_slots(gencd_problem* p, int64_t count) {
  if (count <= p->slot_cap) return GENCD_OK;
  GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
  dev_free(p, p->slot_m);
  dev_free(p, p->slot_d);
  dev_free(p, p->slot_j);
  p->slot_m = nullptr;
  p->slot_d = nullptr;
  p->slot_j = nullptr;
  p->slot_cap = 0;
  GENCD_TRY(dev_alloc(p, &p->slot_m, count));
  GENCD_TRY(dev_alloc(p, &p->slot_d, count));
  GENCD_TRY(dev_alloc(p, &p->slot_j, count));
  p->slot_cap = count;
  return GENCD_OK;
}

static int reset_counters(gencd_problem* p) {
  GENCD_CUDA_TRY(cudaMemsetAsync(p->dscal + 4, 0, 2 * sizeof(double), p->stream));
  p->stat_iters = 0;
  p->stat_host_nnz = 0;
  return GENCD_OK;
}

static int effective_B(const gencd_problem* p) {
  if (p->params.variant == GENCD_GREEDY) return 1;
  int64_t B = p->params.blocks > 0 ? p->params.blocks : 1024;
  if (B > p->k) B = p->k;
  return (int)B;
}

// KKT violation (dscal[0]) and objective (dscal[1]) of the current state
// KKT violation (dscal[0]), objective (dscal[1]) and, with gap, the duality
// gap (dscal[9]) of the current state (the gap's conjugates cost FP64
// transcendentals on every row: only where a gap is asked for)
static int enqueue_evaluate(gencd_problem* p, bool gap = false) {
  GENCD_CUDA_TRY(cudaMemsetAsync(p->dscal, 0, sizeof(double), p->stream));
  GENCD_CUDA_TRY(cudaMemsetAsync(p->dscal + 7, 0, sizeof(double), p->stream));
  GENCD_TRY(launch_propose_all(p, p->u, p->precision == GENCD_F64));
  GENCD_TRY(launch_finalize(p, p->lambda, false));
  GENCD_TRY(launch_objective(p, gap));
  return GENCD_OK;
}

static int read_scalars(gencd_problem* p) {
  GENCD_CUDA_TRY(cudaMemcpyAsync(p->hpin, p->dscal, kScalars * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return GENCD_OK;
}

// the device scalars to hpin without waiting; ev_scalars marks their arrival
static int read_scalars_async(gencd_problem* p) {
  GENCD_CUDA_TRY(cudaMemcpyAsync(p->hpin, p->dscal, kScalars * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  GENCD_CUDA_TRY(cudaEventRecord(p->ev_scalars, p->stream));
  return GENCD_OK;
}

static int compute_pstar(gencd_problem* p, int32_t* iters_out);
static int compute_block_pstar(gencd_problem* p, int32_t B);
__global__ void k_block_select(int64_t t, int32_t B, const int64_t* __restrict__ blo, const int64_t* __restrict__ bP,
                               const int32_t* __restrict__ perm, int32_t* __restrict__ J);

static int ensure_selection(gencd_problem* p, int64_t epoch, int64_t m) {
  if (p->perm_epoch == epoch && p->perm_m == m) return GENCD_OK;
  GENCD_TRY(make_permutation(p, p->params.seed, epoch, m, p->perm));
  p->perm_epoch = epoch;
  p->perm_m = m;
  return GENCD_OK;
}

// Global top-|J'| Accept (Section 7): the B columns with the lowest proxies
// below 0 (ties: the lower column).  Keys are the proxies' candidate
// magnitudes, inverted so that ascending order is best first (non-candidates
// last); two stable 32-bit radix passes (low half, then high half) order all
// k columns by the 64-bit key with the column index breaking ties.
__global__ void k_top_keys(const double* __restrict__ phi, int64_t k, uint32_t* __restrict__ hi,
                           uint32_t* __restrict__ lo, uint32_t* __restrict__ idx) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    const uint64_t m = candidate_mag(phi[j]);
    const uint64_t key = m ? ~m : ~0ull;
    hi[j] = (uint32_t)(key >> 32);
    lo[j] = (uint32_t)key;
    idx[j] = (uint32_t)j;
  }
}

__global__ void k_top_gather(const uint32_t* __restrict__ hi, const uint32_t* __restrict__ idx, int64_t k,
                             uint32_t* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < k; e += stride) out[e] = hi[idx[e]];
}

__global__ void k_top_take(const uint32_t* __restrict__ order, const double* __restrict__ phi,
                           const double* __restrict__ delta, int64_t B, int32_t* __restrict__ list_j,
                           double* __restrict__ list_d) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < B; e += stride) {
    const uint32_t j = order[e];
    const bool ok = candidate_mag(phi[j]) != 0ull;
    list_j[e] = ok ? (int32_t)j : -1;
    list_d[e] = ok ? delta[j] : 0.0;
  }
}

static int launch_top_accept(gencd_problem* p, int64_t B) {
  const int64_t k = p->k;
  // keys, indices, their alternates, the high halves and the radix scratch:
  // sized once, so the Accept allocates nothing per iteration
  if (!p->top_buf) GENCD_TRY(dev_alloc(p, &p->top_buf, 6 * (size_t)k + radix_tmp_words(k)));
  uint32_t *lo = p->top_buf, *idx = lo + k, *lo_alt = lo + 2 * k, *idx_alt = lo + 3 * k, *hi = lo + 4 * k,
           *hi_g = lo + 5 * k, *rtmp = lo + 6 * k;
  const int g = grid_for(k, kThreads, p->num_sms * 8);
  k_top_keys<<<g, kThreads, 0, p->stream>>>(p->phi, k, hi, lo, idx);
  GENCD_CUDA_TRY(cudaGetLastError());
  bool alt1 = false, alt2 = false;
  GENCD_TRY(radix_sort_with_tmp(p, lo, idx, k, 32, lo_alt, idx_alt, rtmp, &alt1));  // by the low half
  uint32_t* idx1 = alt1 ? idx_alt : idx;
  k_top_gather<<<g, kThreads, 0, p->stream>>>(hi, idx1, k, hi_g);
  uint32_t *free_k = alt1 ? lo : lo_alt, *free_v = alt1 ? idx : idx_alt;  // the pair the first pass left free
  GENCD_TRY(radix_sort_with_tmp(p, hi_g, idx1, k, 32, free_k, free_v, rtmp, &alt2));  // then by the high half,
                                                                                   // stably
  const uint32_t* order = alt2 ? free_v : idx1;
  k_top_take<<<grid_for(B, kThreads, p->num_sms * 8), kThreads, 0, p->stream>>>(order, p->phi, p->delta, B,
                                                                                p->list_j, p->list_d);
  p->prof.launches[K_ACCEPT] += 3;
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

// one GenCD iteration (Algorithm 1) of the configured variant, enqueued
static int enqueue_iteration(gencd_problem* p, int64_t* host_nnz, bool want_kkt) {
  const int v = p->params.variant;
  if (v == GENCD_THREAD_GREEDY || v == GENCD_GREEDY) {
    const int B = effective_B(p);
    GENCD_CUDA_TRY(cudaMemsetAsync(p->dscal, 0, sizeof(double), p->stream));  // KKT maximum
    GENCD_TRY(launch_propose_all(p, p->u, p->precision == GENCD_F64));  // Propose, all columns
    GENCD_TRY(launch_finalize_accept(p, B, want_kkt));  // step, proxy (+ KKT of the start state); Accept
    GENCD_TRY(launch_merge_accept(p, B));               // accept backoff (groups of partitions), if any
    GENCD_TRY(launch_improve_list(p, p->list_j, p->list_d, B));  // Improve delta_j (Algorithm 3), if asked
    GENCD_TRY(launch_update_list(p, p->list_j, p->list_d, B, true));     // Update (atomic z)
    GENCD_TRY(launch_refresh_list(p, p->list_j, p->list_d, B, true));
    *host_nnz += p->nnz;
    p->stat_host_nnz += p->nnz;
  } else if (v == GENCD_TOP_GREEDY) {
    // |J'|; the accept backoff of a solve divides it by the accept group
    const int64_t B = std::max<int64_t>(1, effective_B(p) / p->accept_group);
    GENCD_CUDA_TRY(cudaMemsetAsync(p->dscal, 0, sizeof(double), p->stream));  // KKT maximum
    GENCD_TRY(launch_propose_all(p, p->u, p->precision == GENCD_F64));  // Propose, all columns
    GENCD_TRY(launch_finalize(p, p->lambda, true));    // delta, phi of every column (+ KKT of the start state)
    GENCD_TRY(launch_top_accept(p, B));                 // Accept: the B lowest proxies
    GENCD_TRY(launch_improve_list(p, p->list_j, p->list_d, B));
    GENCD_TRY(launch_update_list(p, p->list_j, p->list_d, B, true));  // Update (atomic z)
    GENCD_TRY(launch_refresh_list(p, p->list_j, p->list_d, B, true));
    *host_nnz += p->nnz;
    p->stat_host_nnz += p->nnz;
  } else if (v == GENCD_SHOTGUN) {
    if (p->pstar == 0 && p->params.P == 0) GENCD_TRY(compute_pstar(p, nullptr));
    int64_t P = p->params.P > 0 ? p->params.P : p->pstar;
    if (P > p->k) P = p->k;
    const int64_t per_epoch = (p->k + P - 1) / P;
    const int64_t e = p->t / per_epoch, q = p->t % per_epoch;
    GENCD_TRY(ensure_selection(p, e, p->k));                             // Select, random subset
    const int64_t lo = q * P, m = (lo + P <= p->k ? P : p->k - lo);
    const int32_t* J = p->perm + lo;
    GENCD_TRY(launch_propose_list(p, J, m, p->list_d, p->phi));          // Propose (Jacobi)
    GENCD_TRY(launch_improve_list(p, J, p->list_d, m));                  // Improve delta_j, if asked
    GENCD_TRY(launch_update_list(p, J, p->list_d, m, false));            // Accept all, Update
    GENCD_TRY(launch_refresh_list(p, J, p->list_d, m, false));
  } else if (v == GENCD_SHOTGUN_BLOCKS) {
    const int32_t B = (int32_t)std::min<int64_t>(p->params.blocks > 0 ? p->params.blocks : 16, p->k);
    GENCD_TRY(compute_block_pstar(p, B));
    int64_t m = 0;
    for (int32_t b = 0; b < B; ++b) {  // Select: each block's next P*_b columns (block b's stream: seed + b)
      const int64_t lo = p->hblock_lo[b], kb = p->hblock_lo[b + 1] - lo;
      if (kb == 0) continue;
      const int64_t P = std::min<int64_t>(std::max<int64_t>(p->hblock_P[b], 1), kb);
      const int64_t per_epoch = (kb + P - 1) / P, e = p->t / per_epoch, q = p->t % per_epoch;
      if (p->hblock_epoch[b] != e) {
        GENCD_TRY(make_permutation(p, p->params.seed + (uint64_t)b, e, kb, p->perm + lo));
        p->hblock_epoch[b] = e;
      }
      m += std::min<int64_t>(P, kb - q * P);
    }
    p->perm_epoch = -1;  // perm now holds the blocks' permutations
    k_block_select<<<1, kThreads, 0, p->stream>>>(p->t, B, p->block_lo, p->block_P, p->perm, p->list_j);
    p->prof.launches[K_SETUP] += 1;
    GENCD_CUDA_TRY(cudaGetLastError());
    GENCD_TRY(launch_propose_list(p, p->list_j, m, p->list_d, p->phi));  // Propose (Jacobi)
    GENCD_TRY(launch_improve_list(p, p->list_j, p->list_d, m));         // Improve delta_j, if asked
    GENCD_TRY(launch_update_list(p, p->list_j, p->list_d, m, false));   // Accept all, Update
    GENCD_TRY(launch_refresh_list(p, p->list_j, p->list_d, m, false));
  } else if (v == GENCD_COLORING) {
    if (!p->color) GENCD_TRY(run_coloring(p));
    const int64_t C = p->ncolors;
    const int64_t e = p->t / C, q = p->t % C;
    GENCD_TRY(ensure_selection(p, e, C));                                // Select, random colour
    GENCD_TRY(launch_coloring_iter(p, q));                               // Propose + Update fused
  } else {
    return fail(GENCD_EINVAL, "unknown variant");
  }
  p->t += 1;
  p->stat_iters += 1;
  return GENCD_OK;
}

// Spectral radius of D^-1/2 X_b^T X_b D^-1/2 for the columns b = [lo, hi)
// (all columns: Shotgun's rho; one block: block Shotgun's rho_b) by power
// iteration from the block's all-ones vector, at most 100 iterations or a
// relative change below 1e-6 (Section 4.1)
static int power_radius(gencd_problem* p, int64_t lo, int64_t hi, double* rho_out, int32_t* iters_out) {
  GENCD_TRY(build_csr(p));
  const int64_t k = p->k;
  double *dinv = nullptr, *v = nullptr, *s = nullptr, *t = nullptr, *r = nullptr;
  int rc = GENCD_OK;
  if ((rc = dev_alloc(p, &dinv, k)) || (rc = dev_alloc(p, &v, k)) || (rc = dev_alloc(p, &s, k)) || (rc = dev_alloc(p, &t, k)) ||
      (rc = dev_alloc(p, &r, p->n))) {
    dev_free(p, dinv);
    dev_free(p, v);
    dev_free(p, s);
    dev_free(p, t);
    dev_free(p, r);
    return rc;
  }
  const int g = p->num_sms * 8;
  k_dinv<<<grid_for(k, kThreads, g), kThreads, 0, p->stream>>>(p->c, k, (double)p->n, lo, hi, dinv, v);
  double rho = 0.0;
  int it = 0;
  const int nb = grid_for(k, kThreads, kRedBlocks);
  for (it = 1; it <= 100 && rc == GENCD_OK; ++it) {
    if ((rc = launch_power_step(p, v, dinv, r, s)) != GENCD_OK) break;
    k_power_finish<<<nb, kThreads, 0, p->stream>>>(p->gacc, dinv, k, lo, hi, t, p->red);
    k_sum_partials<<<1, 32, 0, p->stream>>>(p->red, nb, p->dscal + 6);
    p->prof.launches[K_SETUP] += 2;
    if ((rc = read_scalars(p)) != GENCD_OK) break;
    const double rho_new = std::sqrt(p->hpin[6]);
    if (rho_new == 0.0) {
      rho = 0.0;
      break;
    }
    k_div<<<grid_for(k, kThreads, g), kThreads, 0, p->stream>>>(t, k, rho_new, v);
    const bool done = std::fabs(rho_new - rho) <= 1e-6 * rho_new;
    rho = rho_new;
    if (done) break;
  }
  if (it > 100) it = 100;
  dev_free(p, dinv);
  dev_free(p, v);
  dev_free(p, s);
  dev_free(p, t);
  dev_free(p, r);
  if (rc != GENCD_OK) return rc;
  *rho_out = rho;
  if (iters_out) *iters_out = it;
  return GENCD_OK;
}

// P* = max(1, floor(m / (2 rho))), at most m (Section 4.1)
static int64_t pstar_of(int64_t m, double rho) {
  double ps = rho > 0.0 ? std::floor((double)m / (2.0 * rho)) : (double)m;
  if (ps < 1.0) ps = 1.0;
  if (ps > (double)m) ps = (double)m;
  return (int64_t)ps;
}

static int compute_pstar(gencd_problem* p, int32_t* iters_out) {
  double rho = 0.0;
  GENCD_TRY(power_radius(p, 0, p->k, &rho, iters_out));
  p->rho = rho;
  p->pstar = pstar_of(p->k, rho);
  return GENCD_OK;
}

// Block Shotgun (Section 7): B contiguous column blocks [floor(b k / B),
// floor((b+1) k / B)) and each block's P*_b from its own spectral radius
static int compute_block_pstar(gencd_problem* p, int32_t B) {
  if (p->block_B == B && !p->hblock_P.empty()) return GENCD_OK;
  std::vector<int64_t> lo(B + 1), P(B);
  std::vector<double> rho(B);
  for (int32_t b = 0; b <= B; ++b) lo[b] = p->k * b / B;
  for (int32_t b = 0; b < B; ++b) {
    rho[b] = 0.0;
    if (lo[b + 1] > lo[b]) GENCD_TRY(power_radius(p, lo[b], lo[b + 1], &rho[b], nullptr));
    P[b] = lo[b + 1] > lo[b] ? pstar_of(lo[b + 1] - lo[b], rho[b]) : 0;
  }
  dev_free(p, p->block_lo);
  dev_free(p, p->block_P);
  p->block_lo = nullptr;
  p->block_P = nullptr;
  p->block_B = 0;
  GENCD_TRY(dev_alloc(p, &p->block_lo, B + 1));
  GENCD_TRY(dev_alloc(p, &p->block_P, B));
  GENCD_CUDA_TRY(cudaMemcpyAsync(p->block_lo, lo.data(), sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice,
                                 p->stream));
  GENCD_CUDA_TRY(cudaMemcpyAsync(p->block_P, P.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice, p->stream));
  GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
  p->hblock_lo = lo;
  p->hblock_P = P;
  p->hblock_rho = rho;
  p->hblock_epoch.assign(B, -1);
  p->block_B = B;
  return GENCD_OK;
}

// Select of block Shotgun for iteration t: from every block b the next
// m_b = min(P_b, k_b - q P_b) columns of its epoch permutation (q = t mod
// ceil(k_b / P_b)), laid end to end in block order.  One CTA; the blocks'
// offsets by a prefix sum in shared memory (B <= kMaxShotgunBlocks).
__global__ void __launch_bounds__(kThreads)
    k_block_select(int64_t t, int32_t B, const int64_t* __restrict__ blo, const int64_t* __restrict__ bP,
                   const int32_t* __restrict__ perm, int32_t* __restrict__ J) {
  __shared__ int64_t off[kMaxShotgunBlocks + 1];
  __shared__ int64_t start[kMaxShotgunBlocks];
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const int64_t kb = blo[b + 1] - blo[b];
    int64_t m = 0, q0 = 0;
    if (kb > 0) {
      const int64_t P = bP[b] < 1 ? 1 : (bP[b] < kb ? bP[b] : kb);
      const int64_t per_epoch = (kb + P - 1) / P;
      q0 = (t % per_epoch) * P;
      m = kb - q0 < P ? kb - q0 : P;
    }
    off[b + 1] = m;
    start[b] = q0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    off[0] = 0;
    for (int b = 0; b < B; ++b) off[b + 1] += off[b];
  }
  __syncthreads();
  for (int b = 0; b < B; ++b) {
    const int64_t lo = blo[b], m = off[b + 1] - off[b];
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) J[off[b] + i] = (int32_t)(lo + perm[lo + start[b] + i]);
  }
}

static void free_problem(gencd_problem* p) {
  if (!p) return;
  void* bufs[] = {p->col_ptr, p->row_idx, p->val, p->y, p->z, p->u, p->w, p->c, p->ib, p->tile_col, p->gacc,
                  p->delta, p->phi, p->list_j, p->list_d, p->list_m, p->w_start, p->top_buf, p->dscal, p->red, p->perm,
                  p->sort_tmp,
                  p->row_ptr, p->col_idx, p->csr_val, p->color, p->color_ptr, p->cols_by_color,
                  p->slot_m, p->slot_d, p->slot_j, p->list_off, p->scan_tmp, p->bj, p->w32, p->bj32, p->ib32,
                  p->part_lo, p->col_val, p->block_lo, p->block_P};
  if (p->stream) cudaStreamSynchronize(p->stream);
  free_propose_plan(p);
  if (p->gnat && p->gnat != p->gacc) dev_free(p, p->gnat);
  for (void* b : bufs)
    if (b) dev_free(p, b);
  if (p->hpin && p->own_hpin) cudaFreeHost(p->hpin);
  if (p->ev_scalars) cudaEventDestroy(p->ev_scalars);
  for (cudaEvent_t e : p->prof.pool) cudaEventDestroy(e);
  cudaGetLastError();
  delete p;
}

// bfloat16 storage: the FP32 values rounded to bfloat16 (nearest even), in
// place; *bad = 0 when a value leaves the bfloat16 range
__global__ void k_round_bf16(float* __restrict__ v, int64_t m, unsigned long long* __restrict__ bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const float r = __bfloat162float(__float2bfloat16_rn(v[i]));
    if (!isfinite(r)) atomicMin(bad, 0ull);
    v[i] = r;
  }
}

// index-only storage: s_j = the value of column j's non-zeros (0 for an empty
// column); *bad = the lowest column whose non-zeros differ
__global__ void k_column_values(const int64_t* __restrict__ col_ptr, const float* __restrict__ val, int64_t k,
                                float* __restrict__ col_val, unsigned long long* __restrict__ bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    const int64_t s = col_ptr[j], e = col_ptr[j + 1];
    const float v0 = s < e ? val[s] : 0.0f;
    col_val[j] = v0;
    for (int64_t t = s + 1; t < e; ++t)
      if (val[t] != v0) {
        atomicMin(bad, (unsigned long long)j);
        break;
      }
  }
}

// Converts the FP32 values to the storage mode's (bfloat16 rounding, or the
// per-column values of binary storage).  *bad: -1 if the values fit the mode,
// else the first offending column (binary) or 0 (a value beyond bfloat16).
static int store_values(gencd_problem* p, int64_t* bad_out) {
  *bad_out = -1;
  if (p->vmode == kValPlain) return GENCD_OK;
  if (p->vmode == kValNone) GENCD_TRY(dev_alloc(p, &p->col_val, p->k));
  unsigned long long* bad = nullptr;
  GENCD_TRY(dev_alloc(p, &bad, 1));
  unsigned long long h = ~0ull;
  int rc = GENCD_OK;
  if (cudaMemcpyAsync(bad, &h, 8, cudaMemcpyHostToDevice, p->stream) != cudaSuccess) rc = GENCD_ECUDA;
  if (rc == GENCD_OK) {
    if (p->vmode == kValBf16)
      k_round_bf16<<<grid_for(p->nnz, kThreads, p->num_sms * 8), kThreads, 0, p->stream>>>((float*)p->val, p->nnz,
                                                                                          bad);
    else
      k_column_values<<<grid_for(p->k, kThreads, p->num_sms * 8), kThreads, 0, p->stream>>>(
          p->col_ptr, (const float*)p->val, p->k, p->col_val, bad);
    if (cudaMemcpyAsync(&h, bad, 8, cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess)
      rc = fail(GENCD_ECUDA, std::string("storage conversion: ") + cudaGetErrorString(cudaGetLastError()));
  }
  dev_free(p, bad);
  p->prof.launches[K_SETUP] += 1;
  if (rc == GENCD_OK && h != ~0ull) *bad_out = (int64_t)h;
  return rc;
}

static int create_impl(gencd_problem* p, const int64_t* col_ptr, const int32_t* row_idx, const void* val,
                       int32_t val_dtype, const double* y, int32_t memory) {
  const int64_t n = p->n, k = p->k, nnz = p->nnz;
  GENCD_CUDA_TRY(cudaGetDevice(&p->device));
  GENCD_CUDA_TRY(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
  p->items = p->precision == GENCD_F64 ? kItemsF64 : kItemsF32;
  p->nnz_pad = ((nnz + kPadNnz - 1) / kPadNnz) * kPadNnz + kPadNnz;
  const int64_t tile = 32LL * p->items;
  p->ntiles = (nnz + tile - 1) / tile;
  const size_t vsz = p->precision == GENCD_F64 ? 8 : 4;

  GENCD_TRY(dev_alloc(p, &p->col_ptr, k + 1));
  GENCD_TRY(dev_alloc(p, &p->row_idx, p->nnz_pad));
  GENCD_TRY(dev_alloc(p, (char**)&p->val, vsz * p->nnz_pad));
  GENCD_TRY(dev_alloc(p, &p->y, n));
  GENCD_TRY(dev_alloc(p, &p->z, n));
  GENCD_TRY(dev_alloc(p, (char**)&p->u, vsz * (n + 1)));  // u[n] = 0: the row that padding entries may gather
  GENCD_TRY(dev_alloc(p, &p->w, k));
  GENCD_TRY(dev_alloc(p, &p->c, k));
  GENCD_TRY(dev_alloc(p, &p->ib, k));
  GENCD_TRY(dev_alloc(p, &p->bj, k));
  if (p->precision == GENCD_F32) {
    GENCD_TRY(dev_alloc(p, &p->w32, k));
    GENCD_TRY(dev_alloc(p, &p->bj32, k));
    GENCD_TRY(dev_alloc(p, &p->ib32, k));
  }
  GENCD_TRY(dev_alloc(p, &p->tile_col, p->ntiles + 1));
  GENCD_TRY(dev_alloc(p, &p->gacc, k));
  if (p->precision == GENCD_F64) {
    p->gnat = p->gacc;
  } else {
    float* gf = nullptr;
    GENCD_TRY(dev_alloc(p, &gf, k));
    p->gnat = gf;
  }
  GENCD_TRY(dev_alloc(p, &p->delta, k));
  GENCD_TRY(dev_alloc(p, &p->phi, k));
  GENCD_TRY(dev_alloc(p, &p->list_j, k));
  GENCD_TRY(dev_alloc(p, &p->list_d, k));
  GENCD_TRY(dev_alloc(p, &p->list_m, k));
  GENCD_TRY(dev_alloc(p, &p->perm, k));
  GENCD_TRY(dev_alloc(p, &p->list_off, k + 2));
  GENCD_TRY(dev_alloc(p, &p->scan_tmp, scan_tmp_words(k + 2)));
  GENCD_TRY(dev_alloc(p, &p->dscal, kScalars));
  GENCD_TRY(dev_alloc(p, &p->red, 3 * kRedBlocks));
  GENCD_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_scalars, cudaEventDisableTiming));
  if (!p->hpin && cudaMallocHost((void**)&p->hpin, kScalars * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(GENCD_ENOMEM, "pinned host allocation failed");
  }
  cudaStream_t st = p->stream;
  GENCD_CUDA_TRY(cudaMemsetAsync(p->row_idx, 0, sizeof(int32_t) * p->nnz_pad, st));
  GENCD_CUDA_TRY(cudaMemsetAsync(p->val, 0, vsz * p->nnz_pad, st));
  GENCD_CUDA_TRY(cudaMemcpyAsync(p->col_ptr, col_ptr, sizeof(int64_t) * (k + 1), kind_in(memory), st));
  if (nnz > 0) {
    GENCD_CUDA_TRY(cudaMemcpyAsync(p->row_idx, row_idx, sizeof(int32_t) * nnz, kind_in(memory), st));
    const size_t in_sz = val_dtype == 0 ? 8 : 4;
    if (in_sz == vsz) {
      GENCD_CUDA_TRY(cudaMemcpyAsync(p->val, val, vsz * nnz, kind_in(memory), st));
    } else {
      void* tmp = nullptr;
      GENCD_TRY(dev_alloc_bytes(p, &tmp, in_sz * nnz));
      GENCD_CUDA_TRY(cudaMemcpyAsync(tmp, val, in_sz * nnz, kind_in(memory), st));
      const int g = grid_for(nnz, kThreads, p->num_sms * 8);
      if (val_dtype == 0)
        k_convert<double, float><<<g, kThreads, 0, st>>>((const double*)tmp, nnz, (float*)p->val);
      else
        k_convert<float, double><<<g, kThreads, 0, st>>>((const float*)tmp, nnz, (double*)p->val);
      GENCD_CUDA_TRY(cudaGetLastError());
      dev_free(p, tmp);
    }
  }
  GENCD_CUDA_TRY(cudaMemcpyAsync(p->y, y, sizeof(double) * n, kind_in(memory), st));

  int64_t bad_col = -1, bad_row = -1;
  int stage = 0;
  GENCD_TRY(validate_input(p, &bad_col, &bad_row, &stage));
  if (bad_col >= 0)
    return fail(GENCD_EINVAL, stage == 0 ? "col_ptr is not a valid CSC pointer array at column " +
                                               std::to_string(bad_col)
                                         : "column " + std::to_string(bad_col) +
                                               " has unsorted, duplicate or out-of-range rows or a "
                                               "non-finite value");
  if (bad_row >= 0)
    return fail(GENCD_EINVAL, "label y[" + std::to_string(bad_row) + "] is not finite" +
                                  (p->loss == GENCD_LOSS_LOGISTIC ? " or not -1/+1 (logistic loss)" : ""));

  int64_t bad_store = -1;  // bfloat16 rounding, or binary storage's one value per column
  GENCD_TRY(store_values(p, &bad_store));
  if (bad_store >= 0)
    return fail(GENCD_EINVAL, p->vmode == kValBf16 ? std::string("a value of X is beyond the bfloat16 range")
                                                    : "column " + std::to_string(bad_store) +
                                                          " has non-zeros of different values (binary storage "
                                                          "holds one value per column)");
  GENCD_CUDA_TRY(cudaMemsetAsync(p->z, 0, sizeof(double) * n, st));
  GENCD_CUDA_TRY(cudaMemsetAsync(p->u, 0, vsz * (n + 1), st));
  GENCD_CUDA_TRY(cudaMemsetAsync(p->w, 0, sizeof(double) * k, st));
  if (p->w32) GENCD_CUDA_TRY(cudaMemsetAsync(p->w32, 0, sizeof(float) * k, st));
  GENCD_CUDA_TRY(cudaMemsetAsync(p->gacc, 0, sizeof(double) * k, st));
  if (p->gnat != p->gacc) GENCD_CUDA_TRY(cudaMemsetAsync(p->gnat, 0, sizeof(float) * k, st));
  GENCD_CUDA_TRY(cudaMemsetAsync(p->dscal, 0, kScalars * sizeof(double), st));
  GENCD_TRY(launch_tile_map(p));
  GENCD_TRY(launch_col_scale(p));
  GENCD_TRY(build_propose_plan(p));
  GENCD_TRY(launch_fill_u(p));
  gencd_default_params(&p->params);
  GENCD_TRY(launch_inv_beta(p));
  // lambda_max = KKT violation of w = 0 at lambda = 0
  GENCD_TRY(launch_propose_all(p, p->u, p->precision == GENCD_F64));
  GENCD_TRY(launch_finalize(p, 0.0, false));
  GENCD_TRY(read_scalars(p));
  p->lambda_max = p->hpin[0];
  return GENCD_OK;
}

// ---- a solve, step by step ----------------------------------------------
// gencd_solve's loop as a state machine, so that a caller can keep many
// solves in flight: solve_begin enqueues the first evaluation; whenever the
// work enqueued last has completed (ev_scalars), solve_advance decides from
// the scalars it copied back (hpin) and enqueues the next work (returns 1) or
// finishes (returns 0, status in S->status).

static void fill_result(gencd_problem* p, gencd_result* out, int status, int64_t iters, int64_t host_nnz,
                        double secs) {
  if (!out) return;
  std::memset(out, 0, sizeof(*out));
  out->status = status;
  out->iters = iters;
  int64_t upd, nz;
  std::memcpy(&upd, p->hpin + 4, 8);
  std::memcpy(&nz, p->hpin + 5, 8);
  out->updates = upd;
  out->nnz_processed = nz + host_nnz;
  out->objective = p->hpin[1];
  out->kkt = p->hpin[0];
  out->seconds = secs;
}

void solve_result(gencd_problem* p, const SolveRun* S, gencd_result* out) {
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - S->t0).count();
  fill_result(p, out, S->status, S->iters, S->host_nnz, secs);
}

constexpr int64_t kStallIters = 500;   // iterations without progress taken as a stall (50 checks of 10)
constexpr double kStallGain = 1e-2;    // a new lowest KKT value is 1% below the previous one
constexpr double kObjGain = 1e-12;     // a new lowest objective is this far (relative) below the previous one
constexpr double kStallKkt = 1e-3;     // stalls count while the KKT value is at least this times lambda

static int solve_evaluate(gencd_problem* p, SolveRun* S) {
  GENCD_TRY(enqueue_evaluate(p, p->params.tol_gap > 0.0));
  GENCD_TRY(read_scalars_async(p));
  S->host_nnz += p->nnz;
  p->stat_host_nnz += p->nnz;
  S->evaluated = true;
  return GENCD_OK;
}

int solve_begin(gencd_problem* p, SolveRun* S) {
  *S = SolveRun();
  S->t0 = std::chrono::steady_clock::now();
  const gencd_params& a = p->params;
  // Thread-Greedy and Greedy compute the KKT violation of each iteration's
  // start state inside the iteration; their checks read it and only run a
  // full evaluation to confirm convergence.  Shotgun and Coloring evaluate.
  const bool tg = a.variant == GENCD_THREAD_GREEDY || a.variant == GENCD_GREEDY;
  S->fused = tg || a.variant == GENCD_TOP_GREEDY;
  // Accept backoff (neither Thread-Greedy nor the global top-|J'| Accept has
  // a convergence guarantee): an objective that is not finite or above its
  // value at the start restarts the solve from its start with 4x larger
  // accept groups.  Thread-Greedy applies only the best proxy of every G
  // partitions; top-|J'| accepts the |J'|/G lowest proxies.  G = B is Greedy.
  S->B = S->fused ? effective_B(p) : 1;
  S->backoff = S->fused && S->B > 1;
  GENCD_TRY(reset_counters(p));
  if (S->backoff) {
    if (!p->w_start) GENCD_TRY(dev_alloc(p, &p->w_start, p->k));
    GENCD_CUDA_TRY(cudaMemcpyAsync(p->w_start, p->w, sizeof(double) * p->k, cudaMemcpyDeviceToDevice, p->stream));
  }
  return solve_evaluate(p, S);
}

static int solve_finish(gencd_problem* p, SolveRun* S) {
  if (!S->evaluated && S->status != GENCD_EDIVERGED) {  // report the values of the returned state
    GENCD_TRY(solve_evaluate(p, S));
    S->finishing = true;
    return 1;
  }
  return 0;
}

int solve_advance(gencd_problem* p, SolveRun* S) {
  const gencd_params& a = p->params;
  if (!S->started) {
    S->obj_start = p->hpin[1];
    S->started = true;
  }
  if (S->finishing) return 0;
  const double kkt = p->hpin[0], obj = p->hpin[1];
  const bool blown = !std::isfinite(kkt) || !std::isfinite(obj) || obj > 1e6 * (std::fabs(S->obj_start) + 1e-300);
  // divergence: the objective is not finite or above its value at the start
  const bool above = !(obj <= S->obj_start * (1.0 + 1e-6) + 1e-300);
  if (S->backoff && p->accept_group < S->B && S->iters < a.max_iter && (blown || above)) {
    p->accept_group = std::min<int64_t>(S->B, 4 * p->accept_group);  // restart from the start state
    S->best_kkt = S->best_obj = HUGE_VAL;
    S->stall = 0;
    GENCD_CUDA_TRY(cudaMemcpyAsync(p->w, p->w_start, sizeof(double) * p->k, cudaMemcpyDeviceToDevice, p->stream));
    GENCD_TRY(launch_mirror_w(p));
    GENCD_TRY(build_csr(p));
    GENCD_TRY(launch_csr_spmv(p, p->w, p->z));
    GENCD_TRY(launch_fill_u(p));
    GENCD_TRY(solve_evaluate(p, S));
    return 1;
  }
  if (blown) {
    S->status = GENCD_EDIVERGED;
    set_error("objective is not finite or grew beyond 1e6 times its starting value");
    return solve_finish(p, S);
  }
  // converged: the KKT violation, or (tol_gap > 0) the relative duality gap
  // of a full evaluation, within tolerance
  const bool gap_ok = a.tol_gap > 0.0 && S->evaluated && p->hpin[9] <= a.tol_gap * std::fabs(obj);
  if (kkt <= a.tol_kkt || gap_ok) {
    if (S->evaluated) {
      S->status = GENCD_OK;
      return 0;
    }
    GENCD_TRY(solve_evaluate(p, S));  // confirm on the current state
    return 1;
  }
  if (S->iters >= a.max_iter) return solve_finish(p, S);
  // A stall (Thread-Greedy cycling below its start): checks covering
  // kStallIters iterations in a row that set neither a new lowest objective
  // (by kObjGain of itself) nor a KKT value kStallGain below the lowest so
  // far double G (no restart), if the KKT value is still above kStallKkt *
  // lambda.  The
  // lowest values are kept from the solve's (re)start, so the phases of a
  // cycle do not pass for progress, and a solve whose objective keeps falling
  // is never touched.  Near the optimum both values stop improving at the
  // rounding level of the FP32 sums, where fewer updates would not help.
  if (S->backoff && p->accept_group < S->B) {
    bool progress = false;
    if (obj < S->best_obj * (1.0 - kObjGain)) {  // P >= 0 for both losses
      S->best_obj = obj;
      progress = true;
    }
    if (kkt < S->best_kkt * (1.0 - kStallGain)) {
      S->best_kkt = kkt;
      progress = true;
    }
    if (progress) {
      S->stall = 0;
    } else if (++S->stall >= std::max<int64_t>(1, (kStallIters + a.check_every - 1) / a.check_every)) {
      if (kkt >= kStallKkt * p->lambda) p->accept_group = std::min<int64_t>(S->B, 2 * p->accept_group);
      S->stall = 0;
    }
  }
  const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - S->t0).count();
  if (a.timeout_s > 0.0 && el >= a.timeout_s) return solve_finish(p, S);
  const int64_t step = std::min<int64_t>(a.check_every, a.max_iter - S->iters);
  for (int64_t i = 0; i < step; ++i) GENCD_TRY(enqueue_iteration(p, &S->host_nnz, i + 1 == step));
  S->iters += step;
  if (S->fused && !(a.tol_gap > 0.0)) {
    GENCD_TRY(launch_objective(p, false));  // divergence watch on the current state
    GENCD_TRY(read_scalars_async(p));
    S->evaluated = false;
  } else {
    GENCD_TRY(solve_evaluate(p, S));  // the convergence check streams X once
  }
  return 1;
}

}  // namespace gencd

using namespace gencd;

#define GENCD_CHECK_HANDLE(p)                                      \
  do {                                                             \
    if (!(p)) return fail(GENCD_EINVAL, "problem handle is NULL"); \
  } while (0)

extern "C" {

const char* gencd_last_error(void) { return last_error(); }

int gencd_default_params(gencd_params* out) {
  if (!out) return fail(GENCD_EINVAL, "params is NULL");
  std::memset(out, 0, sizeof(*out));
  out->variant = GENCD_THREAD_GREEDY;
  out->blocks = 0;
  out->P = 0;
  out->seed = 0;
  out->max_iter = 100000;
  out->tol_kkt = 1e-8;
  out->check_every = 10;
  out->beta_mode = 0;
  out->timeout_s = 0.0;
  return GENCD_OK;
}

int gencd_create(gencd_problem** out, int64_t n, int64_t k, int64_t nnz, const int64_t* col_ptr,
                 const int32_t* row_idx, const void* val, int32_t val_dtype, const double* y, int32_t loss,
                 int32_t precision, int32_t memory, void* stream) {
  return create_problem(out, n, k, nnz, col_ptr, row_idx, val, val_dtype, y, loss, precision, memory,
                        (cudaStream_t)stream, nullptr, nullptr);
}

}  // extern "C"

namespace gencd {

int create_problem(gencd_problem** out, int64_t n, int64_t k, int64_t nnz, const int64_t* col_ptr,
                   const int32_t* row_idx, const void* val, int32_t val_dtype, const double* y, int32_t loss,
                   int32_t precision, int32_t memory, cudaStream_t stream, cudaMemPool_t pool, double* hpin) {
  set_error("");
  if (!out) return fail(GENCD_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || k < 1 || nnz < 0) return fail(GENCD_EINVAL, "need n >= 1, k >= 1, nnz >= 0");
  if (n >= (int64_t(1) << 31) || k >= (int64_t(1) << 31) || nnz >= (int64_t(1) << 31) - 2 * kPadNnz)
    return fail(GENCD_EINVAL, "n, k and nnz must be below 2^31");
  if (!col_ptr || !y || (nnz > 0 && (!row_idx || !val)))
    return fail(GENCD_EINVAL, "a required input pointer is NULL");
  if (val_dtype != 0 && val_dtype != 1) return fail(GENCD_EINVAL, "val_dtype must be 0 (double) or 1 (float)");
  if (loss != GENCD_LOSS_SQUARED && loss != GENCD_LOSS_LOGISTIC) return fail(GENCD_EINVAL, "unknown loss");
  if (precision != GENCD_F64 && precision != GENCD_F32 && precision != GENCD_BF16 && precision != GENCD_BINARY)
    return fail(GENCD_EINVAL, "unknown precision");
  if (memory != GENCD_HOST && memory != GENCD_DEVICE) return fail(GENCD_EINVAL, "unknown memory kind");
  gencd_problem* p = new (std::nothrow) gencd_problem();
  if (!p) return fail(GENCD_ENOMEM, "host allocation failed");
  p->n = n;
  p->k = k;
  p->nnz = nnz;
  p->loss = loss;
  p->user_precision = precision;
  p->precision = precision == GENCD_F64 ? GENCD_F64 : GENCD_F32;  // BF16 and BINARY compute in FP32
  p->vmode = precision == GENCD_BF16 ? kValBf16 : precision == GENCD_BINARY ? kValNone : kValPlain;
  p->stream = stream;
  p->pool = pool;
  if (hpin) {
    p->hpin = hpin;
    p->own_hpin = false;
  }
  int rc = create_impl(p, col_ptr, row_idx, val, val_dtype, y, memory);
  if (rc != GENCD_OK) {
    std::string keep = last_error();
    free_problem(p);
    set_error(keep);
    return rc;
  }
  *out = p;
  return GENCD_OK;
}

}  // namespace gencd

extern "C" {

void gencd_destroy(gencd_problem* p) { free_problem(p); }

int gencd_set_lambda(gencd_problem* p, double lambda) {
  GENCD_CHECK_HANDLE(p);
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(GENCD_EINVAL, "lambda must be finite and >= 0");
  p->lambda = lambda;
  return GENCD_OK;
}

int gencd_set_loss(gencd_problem* p, int32_t loss) {
  GENCD_CHECK_HANDLE(p);
  if (loss != GENCD_LOSS_SQUARED && loss != GENCD_LOSS_LOGISTIC) return fail(GENCD_EINVAL, "unknown loss");
  if (loss == p->loss) return GENCD_OK;
  const int32_t old = p->loss;
  p->loss = loss;
  if (loss == GENCD_LOSS_LOGISTIC) {  // labels must be -1 / +1
    int64_t bad_col = -1, bad_row = -1;
    int stage = 0;
    const int rc = validate_input(p, &bad_col, &bad_row, &stage);
    if (rc != GENCD_OK || bad_row >= 0) {
      p->loss = old;
      return rc != GENCD_OK ? rc
                            : fail(GENCD_EINVAL, "label y[" + std::to_string(bad_row) +
                                                     "] is not -1/+1 (logistic loss)");
    }
  }
  // l'(y, 0) is -y (squared) and -y/2 (logistic): lambda_max scales by exactly 2
  p->lambda_max = loss == GENCD_LOSS_LOGISTIC ? 0.5 * p->lambda_max : 2.0 * p->lambda_max;
  p->ib_mode = -1;  // beta_j depends on the loss
  GENCD_TRY(launch_inv_beta(p));
  GENCD_TRY(launch_fill_u(p));
  p->accept_group = 1;
  GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return GENCD_OK;
}

int gencd_lambda_max(gencd_problem* p, double* lambda_max) {
  GENCD_CHECK_HANDLE(p);
  if (!lambda_max) return fail(GENCD_EINVAL, "lambda_max is NULL");
  *lambda_max = p->lambda_max;
  return GENCD_OK;
}

int gencd_set_params(gencd_problem* p, const gencd_params* a) {
  GENCD_CHECK_HANDLE(p);
  if (!a) return fail(GENCD_EINVAL, "params is NULL");
  if (a->variant < 0 || a->variant > 5) return fail(GENCD_EINVAL, "unknown variant");
  if (a->variant == GENCD_SHOTGUN_BLOCKS && a->blocks > kMaxShotgunBlocks)
    return fail(GENCD_EINVAL, "block Shotgun takes at most " + std::to_string(kMaxShotgunBlocks) + " blocks");
  if (a->blocks < 0 || a->P < 0 || a->max_iter < 0 || !(a->tol_kkt >= 0.0) || !(a->tol_gap >= 0.0) ||
      a->check_every < 1 ||
      (a->beta_mode != 0 && a->beta_mode != 1) || !(a->timeout_s >= 0.0) || a->improve_steps < 0 ||
      a->improve_steps > 100000)
    return fail(GENCD_EINVAL, "parameter out of range");
  const bool reseed = a->seed != p->params.seed;
  p->params = *a;
  p->accept_group = 1;
  if (reseed) {
    p->perm_epoch = -1;
    std::fill(p->hblock_epoch.begin(), p->hblock_epoch.end(), int64_t(-1));
  }
  GENCD_TRY(launch_inv_beta(p));
  return GENCD_OK;
}

int gencd_get_params(gencd_problem* p, gencd_params* a) {
  GENCD_CHECK_HANDLE(p);
  if (!a) return fail(GENCD_EINVAL, "params is NULL");
  *a = p->params;
  return GENCD_OK;
}

int gencd_set_iteration(gencd_problem* p, int64_t t) {
  GENCD_CHECK_HANDLE(p);
  if (t < 0) return fail(GENCD_EINVAL, "iteration must be >= 0");
  p->t = t;
  return GENCD_OK;
}

int gencd_get_iteration(gencd_problem* p, int64_t* t) {
  GENCD_CHECK_HANDLE(p);
  if (!t) return fail(GENCD_EINVAL, "t is NULL");
  *t = p->t;
  return GENCD_OK;
}


int gencd_iterate(gencd_problem* p, int64_t iters, gencd_result* out) {
  GENCD_CHECK_HANDLE(p);
  if (iters < 0) return fail(GENCD_EINVAL, "iters must be >= 0");
  auto t0 = std::chrono::steady_clock::now();
  if (out) GENCD_TRY(reset_counters(p));
  int64_t host_nnz = 0;
  // the KKT violation of the start state is reduced in every check_every-th
  // iteration (a5 of the hot path) and in the last one
  for (int64_t i = 0; i < iters; ++i)
    GENCD_TRY(enqueue_iteration(p, &host_nnz, i + 1 == iters || (p->t + 1) % p->params.check_every == 0));
  if (!out) {
    GENCD_CUDA_TRY(cudaGetLastError());
    return GENCD_OK;
  }
  GENCD_TRY(enqueue_evaluate(p));
  GENCD_TRY(read_scalars(p));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  fill_result(p, out, GENCD_OK, iters, host_nnz, secs);
  return GENCD_OK;
}

int gencd_solve(gencd_problem* p, gencd_result* out) {
  GENCD_CHECK_HANDLE(p);
  SolveRun S;
  GENCD_TRY(solve_begin(p, &S));
  for (;;) {
    GENCD_CUDA_TRY(cudaEventSynchronize(p->ev_scalars));
    const int r = solve_advance(p, &S);
    if (r < 0) return r;
    if (r == 0) break;
  }
  solve_result(p, &S, out);
  return S.status;
}

int gencd_stats(gencd_problem* p, gencd_result* out) {
  GENCD_CHECK_HANDLE(p);
  if (!out) return fail(GENCD_EINVAL, "out is NULL");
  GENCD_TRY(read_scalars(p));
  fill_result(p, out, GENCD_OK, p->stat_iters, p->stat_host_nnz, 0.0);
  return GENCD_OK;
}

int gencd_stats_reset(gencd_problem* p) {
  GENCD_CHECK_HANDLE(p);
  GENCD_TRY(reset_counters(p));
  return GENCD_OK;
}

int gencd_get_w(gencd_problem* p, double* w, int64_t k, int32_t memory) {
  GENCD_CHECK_HANDLE(p);
  if (!w || k != p->k) return fail(GENCD_EINVAL, "w must hold exactly k doubles");
  GENCD_CUDA_TRY(cudaMemcpyAsync(w, p->w, sizeof(double) * k, kind_out(memory), p->stream));
  GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return GENCD_OK;
}

int gencd_get_z(gencd_problem* p, double* z, int64_t n, int32_t memory) {
  GENCD_CHECK_HANDLE(p);
  if (!z || n != p->n) return fail(GENCD_EINVAL, "z must hold exactly n doubles");
  GENCD_CUDA_TRY(cudaMemcpyAsync(z, p->z, sizeof(double) * n, kind_out(memory), p->stream));
  GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return GENCD_OK;
}

int gencd_set_w(gencd_problem* p, const double* w, int64_t k, int32_t memory) {
  GENCD_CHECK_HANDLE(p);
  if (!w || k != p->k) return fail(GENCD_EINVAL, "w must hold exactly k doubles");
  if (memory == GENCD_HOST) {
    for (int64_t j = 0; j < k; ++j)
      if (!std::isfinite(w[j])) return fail(GENCD_EINVAL, "w[" + std::to_string(j) + "] is not finite");
  }
  GENCD_CUDA_TRY(cudaMemcpyAsync(p->w, w, sizeof(double) * k, kind_in(memory), p->stream));
  GENCD_TRY(launch_mirror_w(p));
  GENCD_TRY(build_csr(p));
  GENCD_TRY(launch_csr_spmv(p, p->w, p->z));
  GENCD_TRY(launch_fill_u(p));
  GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return GENCD_OK;
}

int gencd_duality_gap(gencd_problem* p, double* gap, double* primal, double* dual) {
  GENCD_CHECK_HANDLE(p);
  GENCD_TRY(enqueue_evaluate(p, true));
  GENCD_TRY(read_scalars(p));
  if (gap) *gap = p->hpin[9];
  if (primal) *primal = p->hpin[1];
  if (dual) *dual = p->hpin[1] - p->hpin[9];
  return GENCD_OK;
}

int gencd_objective(gencd_problem* p, double* objective, double* kkt) {
  GENCD_CHECK_HANDLE(p);
  GENCD_TRY(enqueue_evaluate(p));
  GENCD_TRY(read_scalars(p));
  if (objective) *objective = p->hpin[1];
  if (kkt) *kkt = p->hpin[0];
  return GENCD_OK;
}

int gencd_propose_at(gencd_problem* p, const int32_t* J, int64_t m, double* delta, double* phi,
                     int32_t memory) {
  GENCD_CHECK_HANDLE(p);
  if (m < 0 || (m > 0 && (!J || !delta || !phi))) return fail(GENCD_EINVAL, "bad J / outputs");
  if (m == 0) return GENCD_OK;
  std::vector<int32_t> hj((size_t)m);
  GENCD_CUDA_TRY(cudaMemcpy(hj.data(), J, sizeof(int32_t) * m,
                            memory == GENCD_DEVICE ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
  for (int64_t e = 0; e < m; ++e)
    if (hj[e] < 0 || hj[e] >= p->k) return fail(GENCD_EINVAL, "J[" + std::to_string(e) + "] out of range");
  int32_t* dj = nullptr;
  double *dd = nullptr, *df = nullptr;
  int rc = GENCD_OK;
  if ((rc = dev_alloc(p, &dj, m)) || (rc = dev_alloc(p, &dd, m)) || (rc = dev_alloc(p, &df, m))) {
    dev_free(p, dj);
    dev_free(p, dd);
    dev_free(p, df);
    return rc;
  }
  if (cudaMemcpyAsync(dj, hj.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, p->stream) != cudaSuccess)
    rc = fail(GENCD_ECUDA, "copy of J failed");
  if (rc == GENCD_OK) rc = launch_propose_list(p, dj, m, dd, df);
  if (rc == GENCD_OK && (cudaMemcpyAsync(delta, dd, sizeof(double) * m, kind_out(memory), p->stream) != cudaSuccess ||
                         cudaMemcpyAsync(phi, df, sizeof(double) * m, kind_out(memory), p->stream) != cudaSuccess ||
                         cudaStreamSynchronize(p->stream) != cudaSuccess))
    rc = fail(GENCD_ECUDA, std::string("propose_at: ") + cudaGetErrorString(cudaGetLastError()));
  dev_free(p, dj);
  dev_free(p, dd);
  dev_free(p, df);
  return rc;
}

int gencd_propose_all(gencd_problem* p, double* delta, double* phi, int32_t memory, double* kkt) {
  GENCD_CHECK_HANDLE(p);
  GENCD_CUDA_TRY(cudaMemsetAsync(p->dscal, 0, sizeof(double), p->stream));
  GENCD_TRY(launch_propose_all(p, p->u, p->precision == GENCD_F64));
  GENCD_TRY(launch_finalize(p, p->lambda, true));
  if (delta) GENCD_CUDA_TRY(cudaMemcpyAsync(delta, p->delta, sizeof(double) * p->k, kind_out(memory), p->stream));
  if (phi) GENCD_CUDA_TRY(cudaMemcpyAsync(phi, p->phi, sizeof(double) * p->k, kind_out(memory), p->stream));
  GENCD_TRY(read_scalars(p));
  if (kkt) *kkt = p->hpin[0];
  return GENCD_OK;
}

int gencd_spectral_radius(gencd_problem* p, double* rho, int64_t* pstar, int32_t* iters) {
  GENCD_CHECK_HANDLE(p);
  int32_t it = 0;
  GENCD_TRY(compute_pstar(p, &it));
  if (rho) *rho = p->rho;
  if (pstar) *pstar = p->pstar;
  if (iters) *iters = it;
  return GENCD_OK;
}

int gencd_block_pstar(gencd_problem* p, int32_t B, int64_t* pstar, double* rho) {
  GENCD_CHECK_HANDLE(p);
  if (B < 1 || B > kMaxShotgunBlocks || B > p->k)
    return fail(GENCD_EINVAL, "B must be in [1, min(k, " + std::to_string(kMaxShotgunBlocks) + ")]");
  GENCD_TRY(compute_block_pstar(p, B));
  for (int32_t b = 0; b < B; ++b) {
    if (pstar) pstar[b] = p->hblock_P[b];
    if (rho) rho[b] = p->hblock_rho[b];
  }
  return GENCD_OK;
}

int gencd_color(gencd_problem* p, int32_t* ncolors) {
  GENCD_CHECK_HANDLE(p);
  GENCD_TRY(run_coloring(p));
  if (ncolors) *ncolors = p->ncolors;
  return GENCD_OK;
}

int gencd_get_colors(gencd_problem* p, int32_t* colors, int64_t k, int32_t memory) {
  GENCD_CHECK_HANDLE(p);
  if (!colors || k != p->k) return fail(GENCD_EINVAL, "colors must hold exactly k ints");
  if (!p->color) return fail(GENCD_ESTATE, "no colouring yet: call gencd_color or gencd_set_colors");
  GENCD_CUDA_TRY(cudaMemcpyAsync(colors, p->color, sizeof(int32_t) * k, kind_out(memory), p->stream));
  GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return GENCD_OK;
}

int gencd_set_colors(gencd_problem* p, const int32_t* colors, int64_t k, int32_t memory) {
  GENCD_CHECK_HANDLE(p);
  if (!colors || k != p->k) return fail(GENCD_EINVAL, "colors must hold exactly k ints");
  GENCD_TRY(build_csr(p));
  if (!p->color) GENCD_TRY(dev_alloc(p, &p->color, k));
  GENCD_CUDA_TRY(cudaMemcpyAsync(p->color, colors, sizeof(int32_t) * k, kind_in(memory), p->stream));
  unsigned long long* chk = nullptr;
  GENCD_TRY(dev_alloc(p, &chk, 2));
  GENCD_CUDA_TRY(cudaMemsetAsync(chk, 0xff, sizeof(unsigned long long), p->stream));
  GENCD_CUDA_TRY(cudaMemsetAsync(chk + 1, 0, sizeof(unsigned long long), p->stream));
  const int g = p->num_sms * 8;
  k_check_colors<<<grid_for(p->n, kThreads, g), kThreads, 0, p->stream>>>(p->row_ptr, p->col_idx, p->color,
                                                                          p->n, k, chk);
  k_max_i32<<<grid_for(k, kThreads, g), kThreads, 0, p->stream>>>(p->color, k, chk + 1);
  unsigned long long h[2];
  GENCD_CUDA_TRY(cudaMemcpyAsync(h, chk, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
  GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
  dev_free(p, chk);
  int32_t mn = 0;
  {
    std::vector<int32_t> hc((size_t)k);
    GENCD_CUDA_TRY(cudaMemcpy(hc.data(), p->color, sizeof(int32_t) * k, cudaMemcpyDeviceToHost));
    for (int32_t c : hc) mn = c < mn ? c : mn;
  }
  if (mn < 0 || h[1] >= (unsigned long long)k) {
    dev_free(p, p->color);
    p->color = nullptr;
    return fail(GENCD_EINVAL, "colours must lie in [0, k)");
  }
  if (h[0] != ~0ull) {
    dev_free(p, p->color);
    p->color = nullptr;
    return fail(GENCD_EINVAL, "two columns sharing row " + std::to_string(h[0]) + " have the same colour");
  }
  p->ncolors = (int32_t)h[1] + 1;
  return build_color_classes(p);
}

int gencd_permutation(gencd_problem* p, uint64_t seed, int64_t epoch, int64_t m, int32_t* perm) {
  GENCD_CHECK_HANDLE(p);
  if (m < 0 || epoch < 0 || (m > 0 && !perm)) return fail(GENCD_EINVAL, "bad permutation arguments");
  if (m == 0) return GENCD_OK;
  int32_t* d = nullptr;
  GENCD_TRY(dev_alloc(p, &d, m));
  int rc = make_permutation(p, seed, epoch, m, d);
  if (rc == GENCD_OK &&
      (cudaMemcpyAsync(perm, d, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
       cudaStreamSynchronize(p->stream) != cudaSuccess))
    rc = fail(GENCD_ECUDA, "permutation copy failed");
  dev_free(p, d);
  return rc;
}

int gencd_profile_enable(gencd_problem* p, int32_t enable) {
  GENCD_CHECK_HANDLE(p);
  if (!enable) prof_flush(p);
  if (enable && p->prof.pool.empty()) {  // event pairs, created on first use
    for (int i = 0; i < 2 * 4096; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) break;
      p->prof.pool.push_back(e);
    }
    cudaGetLastError();
  }
  p->prof.enabled = enable != 0;
  return GENCD_OK;
}

int gencd_profile_read(gencd_problem* p, int32_t kernel, double* ms, int64_t* launches, int64_t* calls) {
  GENCD_CHECK_HANDLE(p);
  if (kernel < 0 || kernel >= K_NUM) return fail(GENCD_EINVAL, "unknown kernel family");
  prof_flush(p);
  if (ms) *ms = p->prof.ms[kernel];
  if (launches) *launches = p->prof.launches[kernel];
  if (calls) *calls = p->prof.calls[kernel];
  return GENCD_OK;
}

int gencd_set_propose_schedule(gencd_problem* p, int32_t split) {
  GENCD_CHECK_HANDLE(p);
  if (split == -1) return tune_propose_plan(p);
  const bool fusable = p->plan.built && p->plan.light_counter != nullptr;
  if (split != 0 && !(fusable && (split == 20 || split == 24 || split == 28 || split == 31)))
    return fail(GENCD_EINVAL, fusable ? "split must be -1, 0, 20, 24, 28 or 31"
                                      : "this problem's streaming propose has one form only (split 0 or -1)");
  p->plan.fused_split = split;
  return GENCD_OK;
}

int gencd_propose_schedule(gencd_problem* p, int32_t* split, double* ms, int32_t nms) {
  GENCD_CHECK_HANDLE(p);
  if (nms < 0 || (nms > 0 && !ms)) return fail(GENCD_EINVAL, "ms must hold nms >= 0 values");
  if (split) *split = p->plan.fused_split;
  const bool timed = p->plan.built && p->plan.light_counter != nullptr;
  for (int32_t i = 0; i < nms; ++i) ms[i] = (timed && i < 5) ? p->plan.tuned_ms[i] : -1.0;
  return GENCD_OK;
}

int gencd_profile_reset(gencd_problem* p) {
  GENCD_CHECK_HANDLE(p);
  prof_flush(p);
  for (int i = 0; i < K_NUM; ++i) {
    p->prof.ms[i] = 0.0;
    p->prof.launches[i] = 0;
    p->prof.calls[i] = 0;
  }
  return GENCD_OK;
}

}  // extern "C"
