// kernels_update.cu -- the Update step of GenCD (Algorithm 3) on sm_103a.
//
//  * k_update_flat: z += delta_j X_j for accepted columns that may share rows
//    (Shotgun, Thread-Greedy, Greedy), FP64 atomic adds into z (the paper's
//    OpenMP `atomic`, Section 4.2), work spread evenly over the non-zeros of
//    all accepted columns; k_apply_w does w_j += delta_j.
//  * k_refresh_flat: u_i = l'(y_i, z_i) on the rows of the accepted columns,
//    launched after every atomic add of the iteration has landed.
//  * k_coloring_iter: one Coloring iteration fused into a single pass: the
//    columns of one colour class share no row (Section 4.1), so each warp
//    proposes its column and then writes z and u of its own rows with plain
//    stores -- no atomics, no second pass.
//  * k_fill_u, k_csr_spmv: u from z for all rows, and z = Xw by rows.
#include "device_math.cuh"
#include "gencd_internal.cuh"

namespace gencd {

template <typename U>
__global__ void __launch_bounds__(kThreads)
    k_fill_u(const double* __restrict__ y, const double* __restrict__ z, int64_t n, int loss,
             U* __restrict__ u) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    u[i] = u_value<U>(loss, y[i], z[i]);
}

// The applied columns of a list (J[e] >= 0 and D[e] != 0) are laid end to end
// in a virtual range [0, off[m]) (off = exclusive prefix of their lengths), and
// threads take equal runs of that range: a 50,000-nnz column is spread over
// the whole GPU instead of one CTA.
__global__ void k_list_len(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ J,
                           const double* __restrict__ D, int64_t m, uint32_t* __restrict__ len) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e <= m; e += stride) {
    uint32_t l = 0;
    if (e < m) {
      const int32_t j = J[e];
      if (j >= 0 && D[e] != 0.0) l = (uint32_t)(col_ptr[j + 1] - col_ptr[j]);
    }
    len[e] = l;
  }
}

// w_j += delta_j for the applied entries (distinct columns), and the counters
__global__ void k_apply_w(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ J,
                          const double* __restrict__ D, int64_t m, double* __restrict__ w, float* __restrict__ w32,
                          unsigned long long* __restrict__ counters) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long upd = 0, work = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const int32_t j = J[e];
    const double d = D[e];
    if (j < 0 || d == 0.0) continue;
    const double wn = w[j] + d;
    w[j] = wn;
    if (w32) w32[j] = w_mirror(wn);
    upd += 1;
    work += (unsigned long long)(col_ptr[j + 1] - col_ptr[j]);
  }
  upd = warp_sum(upd);
  work = warp_sum(work);
  if ((threadIdx.x & 31) == 0 && upd) {
    atomicAdd(counters + 0, upd);
    atomicAdd(counters + 1, work);
  }
}

// One CTA for lists of at most kListPlanMax entries: lengths of the applied
// entries, their exclusive prefix (off[0..m]), w_j += delta_j and the counters
// -- k_list_len, the scan and k_apply_w in one launch.

__global__ void __launch_bounds__(kListPlanThreads)
    k_list_plan(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ J, const double* __restrict__ D,
                int64_t m, double* __restrict__ w, float* __restrict__ w32, uint32_t* __restrict__ off,
                unsigned long long* __restrict__ counters) {
  __shared__ uint32_t s_warp[kListPlanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  uint32_t len[kListPlanPer];
  uint32_t mine = 0, upd = 0;
#pragma unroll
  for (int q = 0; q < kListPlanPer; ++q) {
    const int64_t e = (int64_t)tid * kListPlanPer + q;
    len[q] = 0;
    if (e < m) {
      const int32_t j = J[e];
      const double d = D[e];
      if (j >= 0 && d != 0.0) {
        len[q] = (uint32_t)(col_ptr[j + 1] - col_ptr[j]);
        const double wn = w[j] + d;  // the entries name distinct columns
        w[j] = wn;
        if (w32) w32[j] = w_mirror(wn);
        ++upd;
      }
    }
    mine += len[q];
  }
  // block-wide exclusive prefix of the per-thread sums
  uint32_t incl = mine;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t v = s_warp[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v += y;
    }
    s_warp[lane] = v;  // inclusive over warps
  }
  __syncthreads();
  uint32_t run = (wid > 0 ? s_warp[wid - 1] : 0u) + incl - mine;
#pragma unroll
  for (int q = 0; q < kListPlanPer; ++q) {
    const int64_t e = (int64_t)tid * kListPlanPer + q;
    if (e < m) off[e] = run;
    run += len[q];
  }
  const uint32_t total = s_warp[kListPlanThreads / 32 - 1];
  if (tid == 0) off[m] = total;
  const unsigned long long u_all = warp_sum((unsigned long long)upd);
  if (lane == 0 && u_all) atomicAdd(counters + 0, u_all);
  if (tid == 0 && total) atomicAdd(counters + 1, (unsigned long long)total);
}

// last entry e in [0, m) with off[e] <= q
__device__ __forceinline__ int64_t entry_of(const uint32_t* __restrict__ off, int64_t m, uint32_t q) {
  int64_t lo = 0, hi = m - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= q)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

constexpr int kFlatRun = 4;  // consecutive virtual positions per thread

// z_i += delta_j X_ij over the applied columns (atomic: columns may share rows)
template <typename V>
__global__ void __launch_bounds__(kThreads)
    k_update_flat(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                  const V* __restrict__ val, const int32_t* __restrict__ J, const double* __restrict__ D,
                  const uint32_t* __restrict__ off, int64_t m, double* __restrict__ z) {
  const uint32_t total = off[m];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * kFlatRun;
  for (int64_t q0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kFlatRun; q0 < total; q0 += stride) {
    int64_t e = entry_of(off, m, (uint32_t)q0);
    for (int r = 0; r < kFlatRun; ++r) {
      const uint32_t q = (uint32_t)(q0 + r);
      if (q >= total) break;
      while (q >= off[e + 1]) ++e;
      const int32_t j = J[e];
      const int64_t p = col_ptr[j] + (q - off[e]);
      atomicAdd(z + row_idx[p], D[e] * (double)val[p]);
    }
  }
}

// u_i = l'(y_i, z_i) on the rows of the applied columns, or on all rows when
// the iteration touched at least n entries (one dense pass is cheaper then)
template <typename U>
__global__ void __launch_bounds__(kThreads)
    k_refresh_flat(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                   const int32_t* __restrict__ J, const uint32_t* __restrict__ off, int64_t m,
                   const double* __restrict__ y, const double* __restrict__ z, int64_t n, int loss,
                   U* __restrict__ u) {
  const uint32_t total = off[m];
  if ((int64_t)total >= n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
      u[i] = u_value<U>(loss, y[i], z[i]);
    return;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * kFlatRun;
  for (int64_t q0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kFlatRun; q0 < total; q0 += stride) {
    int64_t e = entry_of(off, m, (uint32_t)q0);
    for (int r = 0; r < kFlatRun; ++r) {
      const uint32_t q = (uint32_t)(q0 + r);
      if (q >= total) break;
      while (q >= off[e + 1]) ++e;
      const int64_t p = col_ptr[J[e]] + (q - off[e]);
      const int32_t i = row_idx[p];
      u[i] = u_value<U>(loss, y[i], z[i]);
    }
  }
}

template <typename V, typename U>
__global__ void __launch_bounds__(kThreads)
    k_coloring_iter(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                    const V* __restrict__ val, U* __restrict__ u, double* __restrict__ w,
                    float* __restrict__ w32, const double* __restrict__ bjs, const double* __restrict__ ib,
                    double* __restrict__ z,
                    const double* __restrict__ y, const int32_t* __restrict__ perm, int64_t q,
                    const int32_t* __restrict__ color_ptr, const int32_t* __restrict__ cols_by_color,
                    double n, double lam, int loss,
                    unsigned long long* __restrict__ counters) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t colour = perm[q];
  const int32_t lo = color_ptr[colour], hi = color_ptr[colour + 1];
  unsigned long long upd = 0, work = 0;
  for (int64_t e = lo + warp; e < hi; e += nwarps) {
    const int32_t j = cols_by_color[e];
    const int64_t s = col_ptr[j], t = col_ptr[j + 1];
    V acc = V(0);
    for (int64_t p = s + lane; p < t; p += 32) acc = fma(val[p], (V)u[row_idx[p]], acc);
    const double g = warp_sum((double)acc) / n;
    const double wj = w[j];
    double d, f;
    eq7_step(g, wj, lam, bjs[j], ib[j], d, f);  // identical on every lane
    work += (unsigned long long)(t - s);
    if (d != 0.0) {
      // every lane has read its u values above (warp_sum synchronised them)
      for (int64_t p = s + lane; p < t; p += 32) {
        const int32_t i = row_idx[p];
        const double zi = z[i] + d * (double)val[p];
        z[i] = zi;
        u[i] = u_value<U>(loss, y[i], zi);
      }
      if (lane == 0) {
        w[j] = wj + d;
        if (w32) w32[j] = w_mirror(wj + d);
      }
      upd += 1;
      work += (unsigned long long)(t - s);
    }
  }
  if (lane == 0 && (upd | work)) {
    atomicAdd(counters + 0, upd);
    atomicAdd(counters + 1, work);
  }
}

template <typename V>
__global__ void __launch_bounds__(kThreads)
    k_csr_spmv(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
               const V* __restrict__ csr_val, const double* __restrict__ x, int64_t n,
               double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    double acc = 0.0;
    for (int64_t q = row_ptr[i] + lane; q < row_ptr[i + 1]; q += 32)
      acc = fma((double)csr_val[q], x[col_idx[q]], acc);
    acc = warp_sum(acc);
    if (lane == 0) out[i] = acc;
  }
}

// ---------------------------------------------------------------------------
// launchers

// Improve delta_j (Algorithm 3; Section 4.1: further steps of the quadratic
// approximation per accepted increment): one warp per accepted column j
// repeats the Eq. 7 step on coordinate j from w_j + d, with g_j at
// z + d X_j (the iteration-start z: every accepted increment is improved
// before any is applied), until a step is 0 or `steps` steps.  FP64 in both
// storage modes.
template <typename V>
__global__ void k_improve_list(const int32_t* __restrict__ J, double* __restrict__ D, int64_t m,
                               const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                               const V* __restrict__ val, const double* __restrict__ y, const double* __restrict__ z,
                               const double* __restrict__ w, const double* __restrict__ bjs,
                               const double* __restrict__ ibs, int loss, double lam, double inv_n, int steps) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < m; e += nw) {
    const int32_t j = J[e];
    if (j < 0) continue;
    const double bj = bjs[j];
    if (!(bj > 0.0)) continue;  // a column without entries: its step is already exact
    const double wj = w[j], ibj = ibs[j];
    const int64_t a = col_ptr[j], b = col_ptr[j + 1];
    double d = D[e];
    for (int s = 0; s < steps; ++s) {  // warp-uniform: g is the same in every lane
      double acc = 0.0;
      for (int64_t t = a + lane; t < b; t += 32) {
        const double x = (double)val[t];
        const int32_t i = row_idx[t];
        acc += x * loss_deriv(loss, y[i], z[i] + d * x);
      }
      const double g = warp_sum(acc) * inv_n;
      double step, phi;
      eq7_step(g, wj + d, lam, bj, ibj, step, phi);
      if (step == 0.0) break;
      d += step;
    }
    if (lane == 0) D[e] = d;
  }
}

int launch_improve_list(gencd_problem* p, const int32_t* J, double* D, int64_t m) {
  const int steps = p->params.improve_steps;
  if (steps <= 0 || m <= 0) return GENCD_OK;
  const int grid = grid_for(m * 32, kThreads, p->num_sms * 8);
  const double inv_n = 1.0 / (double)p->n;
  if (p->precision == GENCD_F64)
    k_improve_list<double><<<grid, kThreads, 0, p->stream>>>(J, D, m, p->col_ptr, p->row_idx, (const double*)p->val,
                                                             p->y, p->z, p->w, p->bj, p->ib, p->loss, p->lambda,
                                                             inv_n, steps);
  else
    k_improve_list<float><<<grid, kThreads, 0, p->stream>>>(J, D, m, p->col_ptr, p->row_idx, (const float*)p->val,
                                                            p->y, p->z, p->w, p->bj, p->ib, p->loss, p->lambda, inv_n,
                                                            steps);
  p->prof.launches[K_UPDATE] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

int launch_fill_u(gencd_problem* p) {
  if (p->n == 0) return GENCD_OK;
  const int grid = grid_for(p->n, kThreads, p->num_sms * 8);
  if (p->precision == GENCD_F64)
    k_fill_u<double><<<grid, kThreads, 0, p->stream>>>(p->y, p->z, p->n, p->loss, (double*)p->u);
  else
    k_fill_u<float><<<grid, kThreads, 0, p->stream>>>(p->y, p->z, p->n, p->loss, (float*)p->u);
  p->prof.launches[K_SETUP] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

// Update (Algorithm 3) for the list (J, d): w, then z (atomic), then u.
int launch_update_list(gencd_problem* p, const int32_t* J, const double* d, int64_t m, bool) {
  if (m <= 0) return GENCD_OK;
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(p->dscal + 4);
  const int g = p->num_sms * 8;
  cudaEvent_t ev = nullptr;
  const bool one_cta = m <= kListPlanMax;
  prof_begin(p, K_UPDATE, &ev, one_cta ? 2 : 3);  // plan kernel(s) and the scatter (+ the scan)
  if (one_cta) {
    k_list_plan<<<1, kListPlanThreads, 0, p->stream>>>(p->col_ptr, J, d, m, p->w, p->w32, p->list_off, ctr);
  } else {
    k_list_len<<<grid_for(m + 1, kThreads, g), kThreads, 0, p->stream>>>(p->col_ptr, J, d, m, p->list_off);
    GENCD_TRY(exclusive_scan(p, p->list_off, p->list_off, m + 1, p->scan_tmp));
    k_apply_w<<<grid_for(m, kThreads, g), kThreads, 0, p->stream>>>(p->col_ptr, J, d, m, p->w, p->w32, ctr);
  }
  if (p->precision == GENCD_F64)
    k_update_flat<double><<<g, kThreads, 0, p->stream>>>(p->col_ptr, p->row_idx, (const double*)p->val, J, d,
                                                         p->list_off, m, p->z);
  else
    k_update_flat<float><<<g, kThreads, 0, p->stream>>>(p->col_ptr, p->row_idx, (const float*)p->val, J, d,
                                                        p->list_off, m, p->z);
  prof_end(p, ev);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

// needs the prefix list_off left by launch_update_list for the same list
int launch_refresh_list(gencd_problem* p, const int32_t* J, const double*, int64_t m, bool) {
  if (m <= 0) return GENCD_OK;
  const int g = p->num_sms * 8;
  cudaEvent_t ev = nullptr;
  prof_begin(p, K_REFRESH, &ev);
  if (p->precision == GENCD_F64)
    k_refresh_flat<double><<<g, kThreads, 0, p->stream>>>(p->col_ptr, p->row_idx, J, p->list_off, m, p->y, p->z,
                                                           p->n, p->loss, (double*)p->u);
  else
    k_refresh_flat<float><<<g, kThreads, 0, p->stream>>>(p->col_ptr, p->row_idx, J, p->list_off, m, p->y, p->z,
                                                          p->n, p->loss, (float*)p->u);
  prof_end(p, ev);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

int launch_coloring_iter(gencd_problem* p, int64_t q) {
  const int64_t warps = p->max_class > 0 ? p->max_class : 1;
  const int grid = grid_for(warps * 32, kThreads, p->num_sms * 8);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(p->dscal + 4);
  cudaEvent_t ev = nullptr;
  prof_begin(p, K_COLOR_ITER, &ev);
  if (p->precision == GENCD_F64)
    k_coloring_iter<double, double><<<grid, kThreads, 0, p->stream>>>(
        p->col_ptr, p->row_idx, (const double*)p->val, (double*)p->u, p->w, p->w32, p->bj, p->ib, p->z, p->y, p->perm, q,
        p->color_ptr, p->cols_by_color, (double)p->n, p->lambda, p->loss, ctr);
  else
    k_coloring_iter<float, float><<<grid, kThreads, 0, p->stream>>>(
        p->col_ptr, p->row_idx, (const float*)p->val, (float*)p->u, p->w, p->w32, p->bj, p->ib, p->z, p->y, p->perm, q,
        p->color_ptr, p->cols_by_color, (double)p->n, p->lambda, p->loss, ctr);
  prof_end(p, ev);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

int launch_csr_spmv(gencd_problem* p, const double* x, double* out) {
  if (p->n == 0) return GENCD_OK;
  const int grid = grid_for(p->n * 32, kThreads, p->num_sms * 8);
  if (p->precision == GENCD_F64)
    k_csr_spmv<double><<<grid, kThreads, 0, p->stream>>>(p->row_ptr, p->col_idx, (const double*)p->csr_val,
                                                         x, p->n, out);
  else
    k_csr_spmv<float><<<grid, kThreads, 0, p->stream>>>(p->row_ptr, p->col_idx, (const float*)p->csr_val,
                                                        x, p->n, out);
  p->prof.launches[K_SETUP] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

}  // namespace gencd
