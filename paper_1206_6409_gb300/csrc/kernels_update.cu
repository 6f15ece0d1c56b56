// kernels_update.cu -- the Update step of GenCD (Algorithm 3) on sm_103a.
//
//  * k_update_list: w_j += delta_j and z += delta_j X_j for accepted columns
//    that may share rows (Shotgun, Thread-Greedy, Greedy): one CTA per column,
//    FP64 atomic adds into z (the paper's OpenMP `atomic`, Section 4.2).
//  * k_refresh_list: u_i = l'(y_i, z_i) on the rows of the accepted columns,
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

template <typename V>
__global__ void __launch_bounds__(kThreads)
    k_update_list(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                  const V* __restrict__ val, const int32_t* __restrict__ J,
                  const double* __restrict__ D, int64_t m, double* __restrict__ w,
                  double* __restrict__ z, unsigned long long* __restrict__ counters) {
  for (int64_t e = blockIdx.x; e < m; e += gridDim.x) {
    const int32_t j = J[e];
    const double d = D[e];
    if (j < 0 || d == 0.0) continue;  // rejected (Thread-Greedy) or a null step
    const int64_t s = col_ptr[j], t = col_ptr[j + 1];
    if (threadIdx.x == 0) {
      w[j] += d;
      atomicAdd(counters + 0, 1ull);
      atomicAdd(counters + 1, (unsigned long long)(t - s));
      atomicAdd(counters + 3, (unsigned long long)(t - s));  // touched this iteration
    }
    for (int64_t p = s + threadIdx.x; p < t; p += blockDim.x) atomicAdd(z + row_idx[p], d * (double)val[p]);
  }
}

// When the updates of the iteration touched at least n non-zeros, one dense
// pass over all rows is cheaper than revisiting every touched entry (each
// costs a gather and an exp); both leave u = l'(y, z) on every touched row.
template <typename U>
__global__ void __launch_bounds__(kThreads)
    k_refresh_list(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                   const int32_t* __restrict__ J, const double* __restrict__ D, int64_t m,
                   const double* __restrict__ y, const double* __restrict__ z, int64_t n, int loss,
                   U* __restrict__ u, const unsigned long long* __restrict__ touched) {
  if (*touched >= (unsigned long long)n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
      u[i] = u_value<U>(loss, y[i], z[i]);
    return;
  }
  for (int64_t e = blockIdx.x; e < m; e += gridDim.x) {
    const int32_t j = J[e];
    if (j < 0 || D[e] == 0.0) continue;
    const int64_t s = col_ptr[j], t = col_ptr[j + 1];
    for (int64_t p = s + threadIdx.x; p < t; p += blockDim.x) {
      const int32_t i = row_idx[p];
      u[i] = u_value<U>(loss, y[i], z[i]);
    }
  }
}

template <typename V, typename U>
__global__ void __launch_bounds__(kThreads)
    k_coloring_iter(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                    const V* __restrict__ val, U* __restrict__ u, double* __restrict__ w,
                    const double* __restrict__ c, double* __restrict__ z,
                    const double* __restrict__ y, const int32_t* __restrict__ perm, int64_t q,
                    const int32_t* __restrict__ color_ptr, const int32_t* __restrict__ cols_by_color,
                    double n, double lam, double beta, int beta_mode, int loss,
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
    const double bj = beta_mode ? beta : beta * c[j];
    double d, f;
    eq7_step(g, wj, lam, bj, d, f);  // identical on every lane
    work += (unsigned long long)(t - s);
    if (d != 0.0) {
      // every lane has read its u values above (warp_sum synchronised them)
      for (int64_t p = s + lane; p < t; p += 32) {
        const int32_t i = row_idx[p];
        const double zi = z[i] + d * (double)val[p];
        z[i] = zi;
        u[i] = u_value<U>(loss, y[i], zi);
      }
      if (lane == 0) w[j] = wj + d;
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

int launch_update_list(gencd_problem* p, const int32_t* J, const double* d, int64_t m, bool) {
  if (m <= 0) return GENCD_OK;
  const int grid = (int)(m < (int64_t)p->num_sms * 16 ? m : (int64_t)p->num_sms * 16);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(p->dscal + 4);
  cudaEvent_t ev = nullptr;
  prof_begin(p, K_UPDATE, &ev);
  if (p->precision == GENCD_F64)
    k_update_list<double><<<grid, kThreads, 0, p->stream>>>(p->col_ptr, p->row_idx, (const double*)p->val,
                                                            J, d, m, p->w, p->z, ctr);
  else
    k_update_list<float><<<grid, kThreads, 0, p->stream>>>(p->col_ptr, p->row_idx, (const float*)p->val,
                                                           J, d, m, p->w, p->z, ctr);
  prof_end(p, ev);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

int launch_refresh_list(gencd_problem* p, const int32_t* J, const double* d, int64_t m, bool) {
  if (m <= 0) return GENCD_OK;
  const int grid = p->num_sms * 16;
  const unsigned long long* touched = reinterpret_cast<const unsigned long long*>(p->dscal + 7);
  cudaEvent_t ev = nullptr;
  prof_begin(p, K_REFRESH, &ev);
  if (p->precision == GENCD_F64)
    k_refresh_list<double><<<grid, kThreads, 0, p->stream>>>(p->col_ptr, p->row_idx, J, d, m, p->y, p->z,
                                                             p->n, p->loss, (double*)p->u, touched);
  else
    k_refresh_list<float><<<grid, kThreads, 0, p->stream>>>(p->col_ptr, p->row_idx, J, d, m, p->y, p->z,
                                                            p->n, p->loss, (float*)p->u, touched);
  prof_end(p, ev);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

int launch_coloring_iter(gencd_problem* p, int64_t q) {
  const double beta = p->loss == GENCD_LOSS_SQUARED ? 1.0 : 0.25;
  const int64_t warps = p->max_class > 0 ? p->max_class : 1;
  const int grid = grid_for(warps * 32, kThreads, p->num_sms * 8);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(p->dscal + 4);
  cudaEvent_t ev = nullptr;
  prof_begin(p, K_COLOR_ITER, &ev);
  if (p->precision == GENCD_F64)
    k_coloring_iter<double, double><<<grid, kThreads, 0, p->stream>>>(
        p->col_ptr, p->row_idx, (const double*)p->val, (double*)p->u, p->w, p->c, p->z, p->y, p->perm, q,
        p->color_ptr, p->cols_by_color, (double)p->n, p->lambda, beta, p->params.beta_mode, p->loss, ctr);
  else
    k_coloring_iter<float, float><<<grid, kThreads, 0, p->stream>>>(
        p->col_ptr, p->row_idx, (const float*)p->val, (float*)p->u, p->w, p->c, p->z, p->y, p->perm, q,
        p->color_ptr, p->cols_by_color, (double)p->n, p->lambda, beta, p->params.beta_mode, p->loss, ctr);
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
