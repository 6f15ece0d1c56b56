// kernels_setup.cu -- one-time preparation and Select support on sm_103a.
//
//  * input validation, column scales c_j = ||X_j||^2 / n, the tile map of the
//    streaming propose;
//  * a stable LSD radix sort of (uint32 key, uint32 value) pairs, 8 bits per
//    pass: per-tile digit histograms, an exclusive scan, and a stable scatter
//    that ranks equal digits with __match_any_sync;
//  * Select's per-epoch permutation (SplitMix64 keys, radix sort);
//  * the row-major copy of X (radix sort of the non-zeros by row, stable, so
//    columns stay ascending within a row);
//  * the partial distance-2 colouring (Section 4.1) by Jones-Plassmann rounds
//    with priority = lower column index, which reproduces greedy first-fit in
//    column order exactly: a column is coloured once every lower-index column
//    that shares a row with it is coloured, with the smallest colour none of
//    them uses;
//  * the pieces of the power iteration for rho (Section 4.1).
#include <algorithm>
#include <vector>

#include "device_math.cuh"
#include "gencd_internal.cuh"

namespace gencd {

// ---------------------------------------------------------------------------
// validation: err[0] <- smallest bad column, err[1] <- smallest bad row (y)
__global__ void k_validate_colptr(const int64_t* __restrict__ col_ptr, int64_t k, int64_t nnz,
                                  unsigned long long* __restrict__ err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    const int64_t s = col_ptr[j], t = col_ptr[j + 1];
    bool bad = s < 0 || t < s || t > nnz || (j == 0 && s != 0) || (j == k - 1 && t != nnz);
    if (bad) atomicMin(err, (unsigned long long)j);
  }
}

// bit p of starts is set when nnz position p begins a non-empty column
__global__ void k_mark_starts(const int64_t* __restrict__ col_ptr, int64_t k, uint32_t* __restrict__ starts) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    const int64_t s = col_ptr[j];
    if (col_ptr[j + 1] > s) atomicOr(starts + (s >> 5), 1u << (s & 31));
  }
}

// one thread per non-zero: row in range, rows strictly increasing inside a
// column, finite value; a failure records the column (found by bisection)
template <typename V>
__global__ void k_validate_rows(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                                const V* __restrict__ val, const uint32_t* __restrict__ starts, int64_t k,
                                int64_t n, int64_t nnz, unsigned long long* __restrict__ err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
    const int32_t r = row_idx[p];
    const bool start = (starts[p >> 5] >> (p & 31)) & 1u;
    bool bad = r < 0 || r >= n || !isfinite((double)val[p]) || (!start && r <= row_idx[p - 1]);
    if (bad) {
      int64_t lo = 0, hi = k - 1;  // the column holding p: last c with col_ptr[c] <= p
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (col_ptr[mid] <= p)
          lo = mid;
        else
          hi = mid - 1;
      }
      atomicMin(err, (unsigned long long)lo);
    }
  }
}

__global__ void k_validate_y(const double* __restrict__ y, int64_t n, int logistic,
                             unsigned long long* __restrict__ err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double v = y[i];
    bool bad = !isfinite(v) || (logistic && v != 1.0 && v != -1.0);
    if (bad) atomicMin(err, (unsigned long long)i);
  }
}

// tile_col[t] = column holding nnz position t * tile; tile_col[ntiles] = k - 1
__global__ void k_tile_map(const int64_t* __restrict__ col_ptr, int64_t k, int64_t tile, int64_t ntiles,
                           int32_t* __restrict__ tile_col) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    const int64_t s = col_ptr[j], e = col_ptr[j + 1];
    if (e <= s) continue;
    for (int64_t t = (s + tile - 1) / tile; t * tile < e; ++t) tile_col[t] = (int32_t)j;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tile_col[ntiles] = (int32_t)(k - 1);
}

// ---------------------------------------------------------------------------
// exclusive scan of uint32 (totals < 2^32)
constexpr int kScanItems = 8;
constexpr int kScanBlock = kThreads * kScanItems;  // 2048 entries per CTA

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_tot[kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  uint32_t wpre = 0, all = 0;
  for (int q = 0; q < kThreads / 32; ++q) {
    if (q < wid) wpre += warp_tot[q];
    all += warp_tot[q];
  }
  __syncthreads();
  *total = all;
  return wpre + x - v;
}

__global__ void __launch_bounds__(kThreads)
    k_scan_sums(const uint32_t* __restrict__ in, int64_t m, uint32_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < m) s += in[base + i];
  uint32_t tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// in and out may be the same array: every thread reads its entries before the
// block-wide scan and writes them after it
__global__ void __launch_bounds__(kThreads)
    k_scan_apply(const uint32_t* in, int64_t m, const uint32_t* __restrict__ offs, uint32_t* out) {
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
  uint32_t x[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    x[i] = base + i < m ? in[base + i] : 0u;
    s += x[i];
  }
  uint32_t tot;
  uint32_t pre = block_exclusive_scan(s, &tot) + (offs ? offs[blockIdx.x] : 0u);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < m) out[base + i] = pre;
    pre += x[i];
  }
}

// out = exclusive_scan(in); tmp needs scan_tmp_words(m) uint32 words
int64_t scan_tmp_words(int64_t m) {
  int64_t w = 0;
  while (m > kScanBlock) {
    m = (m + kScanBlock - 1) / kScanBlock;
    w += 2 * m;
  }
  return w + 2;
}

int exclusive_scan(gencd_problem* p, const uint32_t* in, uint32_t* out, int64_t m, uint32_t* tmp) {
  if (m <= 0) return GENCD_OK;
  const int64_t nb = (m + kScanBlock - 1) / kScanBlock;
  if (nb == 1) {
    k_scan_apply<<<1, kThreads, 0, p->stream>>>(in, m, nullptr, out);
    p->prof.launches[K_SETUP] += 1;
  } else {
    uint32_t* sums = tmp;
    uint32_t* sums_scanned = tmp + nb;
    k_scan_sums<<<(unsigned)nb, kThreads, 0, p->stream>>>(in, m, sums);
    GENCD_TRY(exclusive_scan(p, sums, sums_scanned, nb, tmp + 2 * nb));
    k_scan_apply<<<(unsigned)nb, kThreads, 0, p->stream>>>(in, m, sums_scanned, out);
    p->prof.launches[K_SETUP] += 2;
  }
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8 bits per pass
constexpr int kRsItems = 16;
constexpr int kRsTile = kThreads * kRsItems;  // 4096 pairs per CTA

__global__ void __launch_bounds__(kThreads)
    k_radix_hist(const uint32_t* __restrict__ keys, int64_t m, int shift, uint32_t* __restrict__ counts,
                 int64_t nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  for (int i = threadIdx.x; i < kRsTile; i += kThreads) {
    const int64_t idx = base + i;
    if (idx < m) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads)
    k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, int64_t m, int shift,
                    const uint32_t* __restrict__ offsets, int64_t nblocks, uint32_t* __restrict__ kout,
                    uint32_t* __restrict__ vout) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t wcnt[kThreads / 32][256];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  run[threadIdx.x] = offsets[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  for (int w = 0; w < kThreads / 32; ++w) wcnt[w][threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int round = 0; round < kRsItems; ++round) {
    const int64_t idx = base + (int64_t)round * kThreads + threadIdx.x;
    const bool valid = idx < m;
    const uint32_t key = valid ? kin[idx] : 0u;
    const uint32_t d = (key >> shift) & 255u;
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? d : 256u + lane);
    const uint32_t rank = __popc(peers & lt);
    if (valid && rank == 0) wcnt[wid][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pre = run[d] + rank;
      for (int w = 0; w < wid; ++w) pre += wcnt[w][d];
      kout[pre] = key;
      vout[pre] = vin[idx];
    }
    __syncthreads();
    uint32_t tot = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
      tot += wcnt[w][threadIdx.x];
      wcnt[w][threadIdx.x] = 0;
    }
    run[threadIdx.x] += tot;
    __syncthreads();
  }
}

int ensure_sort_tmp(gencd_problem* p, size_t bytes) {
  if (bytes <= p->sort_tmp_bytes) return GENCD_OK;
  if (p->sort_tmp) {
    GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
    dev_free(p, p->sort_tmp);
    p->sort_tmp = nullptr;
    p->sort_tmp_bytes = 0;
  }
  GENCD_TRY(dev_alloc_bytes(p, &p->sort_tmp, bytes));
  p->sort_tmp_bytes = bytes;
  return GENCD_OK;
}

// scratch layout for sorting m pairs: counts (256 * nblocks) + offsets + scan tmp
size_t radix_tmp_words(int64_t m) {
  const int64_t nb = (m + kRsTile - 1) / kRsTile;
  const int64_t nc = 256 * (nb > 0 ? nb : 1);
  return (size_t)(2 * nc + scan_tmp_words(nc));
}

// Sorts (keys, vals) by the low `bits` bits of the keys, stably.  Ping-pongs
// with (keys_alt, vals_alt); *result_in_alt tells where the result is.
// Needs radix_tmp_words(m) words of scratch at tmp (provided by the caller).
int radix_sort_with_tmp(gencd_problem* p, uint32_t* keys, uint32_t* vals, int64_t m, int bits,
                        uint32_t* keys_alt, uint32_t* vals_alt, uint32_t* tmp, bool* result_in_alt) {
  *result_in_alt = false;
  if (m <= 1 || bits <= 0) return GENCD_OK;
  const int64_t nb = (m + kRsTile - 1) / kRsTile;
  const int64_t nc = 256 * nb;
  uint32_t* counts = tmp;
  uint32_t* offs = tmp + nc;
  uint32_t* stmp = tmp + 2 * nc;
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  bool alt = false;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<<<(unsigned)nb, kThreads, 0, p->stream>>>(ki, m, shift, counts, nb);
    GENCD_TRY(exclusive_scan(p, counts, offs, nc, stmp));
    k_radix_scatter<<<(unsigned)nb, kThreads, 0, p->stream>>>(ki, vi, m, shift, offs, nb, ko, vo);
    p->prof.launches[K_SETUP] += 2;
    GENCD_CUDA_TRY(cudaGetLastError());
    std::swap(ki, ko);
    std::swap(vi, vo);
    alt = !alt;
  }
  *result_in_alt = alt;
  return GENCD_OK;
}

// ---------------------------------------------------------------------------
// Select: permutation of 0..m-1 for one epoch
__global__ void k_perm_keys(uint64_t s, int64_t m, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    keys[i] = (uint32_t)(splitmix64_at(s, (uint64_t)i) >> 32);
    vals[i] = (uint32_t)i;
  }
}

int make_permutation(gencd_problem* p, uint64_t seed, int64_t epoch, int64_t m, int32_t* out) {
  if (m <= 0) return GENCD_OK;
  const size_t words = 4 * (size_t)m + radix_tmp_words(m);
  GENCD_TRY(ensure_sort_tmp(p, words * 4));
  uint32_t* buf = (uint32_t*)p->sort_tmp;
  uint32_t *keys = buf, *vals = buf + m, *ka = buf + 2 * m, *va = buf + 3 * m, *tmp = buf + 4 * m;
  const uint64_t s = splitmix64_at(seed, (uint64_t)epoch);
  k_perm_keys<<<grid_for(m, kThreads, p->num_sms * 8), kThreads, 0, p->stream>>>(s, m, keys, vals);
  p->prof.launches[K_SETUP] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  bool in_alt = false;
  GENCD_TRY(radix_sort_with_tmp(p, keys, vals, m, 32, ka, va, tmp, &in_alt));
  GENCD_CUDA_TRY(cudaMemcpyAsync(out, in_alt ? va : vals, (size_t)m * 4, cudaMemcpyDeviceToDevice, p->stream));
  return GENCD_OK;
}

// ---------------------------------------------------------------------------
// row-major copy of X
__global__ void k_expand_cols(const int64_t* __restrict__ col_ptr, int64_t k, uint32_t* __restrict__ colof) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = warp; j < k; j += nwarps)
    for (int64_t p = col_ptr[j] + lane; p < col_ptr[j + 1]; p += 32) colof[p] = (uint32_t)j;
}

__global__ void k_rows_iota(const int32_t* __restrict__ row_idx, int64_t nnz, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += stride) {
    keys[q] = (uint32_t)row_idx[q];
    vals[q] = (uint32_t)q;
  }
}

template <typename V>
__global__ void k_csr_gather(const uint32_t* __restrict__ order, const uint32_t* __restrict__ colof,
                             const V* __restrict__ val, int64_t nnz, int32_t* __restrict__ col_idx,
                             V* __restrict__ csr_val) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += stride) {
    const uint32_t src = order[q];
    col_idx[q] = (int32_t)colof[src];
    csr_val[q] = val[src];
  }
}

// ptr[i] = first position q with sorted[q] >= i, for i in [0, count]
__global__ void k_lower_bounds(const uint32_t* __restrict__ sorted, int64_t m, int64_t count,
                               int64_t* __restrict__ ptr64, int32_t* __restrict__ ptr32) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= count; i += stride) {
    int64_t lo = 0, hi = m;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)sorted[mid] < i)
        lo = mid + 1;
      else
        hi = mid;
    }
    if (ptr64) ptr64[i] = lo;
    if (ptr32) ptr32[i] = (int32_t)lo;
  }
}

int bits_for_max(int64_t maxval) {
  int b = 1;
  while (b < 32 && (int64_t(1) << b) <= maxval) ++b;
  return b;
}

int lower_bounds_u32_to_i64(gencd_problem* p, const uint32_t* sorted, int64_t m, int64_t count, int64_t* out) {
  k_lower_bounds<<<grid_for(count + 1, kThreads, p->num_sms * 8), kThreads, 0, p->stream>>>(sorted, m, count, out,
                                                                                            nullptr);
  p->prof.launches[K_SETUP] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

__global__ void k_iota_u32(uint32_t* __restrict__ a, int64_t m) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) a[i] = (uint32_t)i;
}

int iota_u32(gencd_problem* p, uint32_t* a, int64_t m) {
  k_iota_u32<<<grid_for(m, kThreads, p->num_sms * 8), kThreads, 0, p->stream>>>(a, m);
  p->prof.launches[K_SETUP] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

int fail_plan(const char* msg) {
  set_error(msg);
  return GENCD_EINVAL;
}

int build_csr(gencd_problem* p) {
  if (p->row_ptr) return GENCD_OK;
  const int64_t nnz = p->nnz;
  const size_t vsz = p->precision == GENCD_F64 ? 8 : 4;
  GENCD_TRY(dev_alloc_bytes(p, (void**)&p->row_ptr, sizeof(int64_t) * (size_t)(p->n + 1)));
  GENCD_TRY(dev_alloc_bytes(p, (void**)&p->col_idx, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1)));
  GENCD_TRY(dev_alloc_bytes(p, (void**)&p->csr_val, vsz * (size_t)(nnz > 0 ? nnz : 1)));
  if (nnz == 0) {
    GENCD_CUDA_TRY(cudaMemsetAsync(p->row_ptr, 0, sizeof(int64_t) * (size_t)(p->n + 1), p->stream));
    return GENCD_OK;
  }
  const size_t words = 5 * (size_t)nnz + radix_tmp_words(nnz);
  GENCD_TRY(ensure_sort_tmp(p, words * 4));
  uint32_t* buf = (uint32_t*)p->sort_tmp;
  uint32_t *keys = buf, *vals = buf + nnz, *ka = buf + 2 * nnz, *va = buf + 3 * nnz, *colof = buf + 4 * nnz,
           *tmp = buf + 5 * nnz;
  const int g = p->num_sms * 8;
  k_expand_cols<<<grid_for(p->k * 32, kThreads, g), kThreads, 0, p->stream>>>(p->col_ptr, p->k, colof);
  k_rows_iota<<<grid_for(nnz, kThreads, g), kThreads, 0, p->stream>>>(p->row_idx, nnz, keys, vals);
  p->prof.launches[K_SETUP] += 2;
  GENCD_CUDA_TRY(cudaGetLastError());
  bool in_alt = false;
  GENCD_TRY(radix_sort_with_tmp(p, keys, vals, nnz, bits_for_max(p->n - 1), ka, va, tmp, &in_alt));
  const uint32_t* sk = in_alt ? ka : keys;
  const uint32_t* sv = in_alt ? va : vals;
  if (p->precision == GENCD_F64)
    k_csr_gather<double><<<grid_for(nnz, kThreads, g), kThreads, 0, p->stream>>>(
        sv, colof, (const double*)p->val, nnz, p->col_idx, (double*)p->csr_val);
  else
    k_csr_gather<float><<<grid_for(nnz, kThreads, g), kThreads, 0, p->stream>>>(
        sv, colof, (const float*)p->val, nnz, p->col_idx, (float*)p->csr_val);
  k_lower_bounds<<<grid_for(p->n + 1, kThreads, g), kThreads, 0, p->stream>>>(sk, nnz, p->n, p->row_ptr,
                                                                               nullptr);
  p->prof.launches[K_SETUP] += 2;
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

// ---------------------------------------------------------------------------
// Jones-Plassmann colouring with index priority (== first-fit in index order)
constexpr int kColourWindow = 1024;  // colours examined per scan of the neighbourhood

__global__ void __launch_bounds__(kThreads)
    k_jp_round(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
               const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
               const int32_t* __restrict__ work_in, int64_t m_in, int32_t* __restrict__ work_out,
               unsigned long long* __restrict__ m_out, int32_t* color,
               unsigned long long* __restrict__ max_colour) {
  __shared__ uint32_t bitmap[kThreads / 32][kColourWindow / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < m_in; e += nwarps) {
    const int32_t j = work_in[e];
    const int64_t s = col_ptr[j], t = col_ptr[j + 1];
    // ready iff every lower-index neighbour is coloured
    bool waiting = false;
    for (int64_t p = s + lane; p < t && !waiting; p += 32) {
      const int32_t i = row_idx[p];
      for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
        const int32_t cn = col_idx[q];
        if (cn >= j) break;  // columns ascend within a row
        if (__ldcg(color + cn) < 0) {
          waiting = true;
          break;
        }
      }
    }
    if (__any_sync(0xffffffffu, waiting)) {
      if (lane == 0) {
        const unsigned long long slot = atomicAdd(m_out, 1ull);
        work_out[slot] = j;
      }
      continue;
    }
    // smallest colour not used by a lower-index neighbour
    int32_t chosen = -1;
    for (int32_t base = 0; chosen < 0; base += kColourWindow) {
      bitmap[wid][lane] = 0u;
      __syncwarp();
      for (int64_t p = s + lane; p < t; p += 32) {
        const int32_t i = row_idx[p];
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
          const int32_t cn = col_idx[q];
          if (cn >= j) break;
          const int32_t cc = __ldcg(color + cn) - base;
          if (cc >= 0 && cc < kColourWindow) atomicOr(&bitmap[wid][cc >> 5], 1u << (cc & 31));
        }
      }
      __syncwarp();
      const uint32_t freebits = ~bitmap[wid][lane];
      const unsigned has = __ballot_sync(0xffffffffu, freebits != 0u);
      if (has) {
        const int first = __ffs(has) - 1;
        const uint32_t fb = __shfl_sync(0xffffffffu, freebits, first);
        chosen = base + first * 32 + (__ffs(fb) - 1);
      }
      __syncwarp();
    }
    if (lane == 0) {
      color[j] = chosen;
      atomicMax(max_colour, (unsigned long long)chosen);
    }
  }
}

__global__ void k_iota_i32(int32_t* __restrict__ a, int64_t m) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) a[i] = (int32_t)i;
}

__global__ void k_color_keys(const int32_t* __restrict__ color, int64_t k, uint32_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    keys[j] = (uint32_t)color[j];
    vals[j] = (uint32_t)j;
  }
}

int build_color_classes(gencd_problem* p) {
  const int64_t k = p->k;
  const size_t words = 4 * (size_t)k + radix_tmp_words(k);
  GENCD_TRY(ensure_sort_tmp(p, words * 4));
  uint32_t* buf = (uint32_t*)p->sort_tmp;
  uint32_t *keys = buf, *vals = buf + k, *ka = buf + 2 * k, *va = buf + 3 * k, *tmp = buf + 4 * k;
  const int g = p->num_sms * 8;
  k_color_keys<<<grid_for(k, kThreads, g), kThreads, 0, p->stream>>>(p->color, k, keys, vals);
  GENCD_CUDA_TRY(cudaGetLastError());
  bool in_alt = false;
  GENCD_TRY(radix_sort_with_tmp(p, keys, vals, k, bits_for_max(p->ncolors - 1), ka, va, tmp, &in_alt));
  if (p->color_ptr) dev_free(p, p->color_ptr);
  p->color_ptr = nullptr;
  GENCD_TRY(dev_alloc_bytes(p, (void**)&p->color_ptr, sizeof(int32_t) * (size_t)(p->ncolors + 1)));
  if (!p->cols_by_color) GENCD_TRY(dev_alloc_bytes(p, (void**)&p->cols_by_color, sizeof(int32_t) * (size_t)k));
  GENCD_CUDA_TRY(cudaMemcpyAsync(p->cols_by_color, in_alt ? va : vals, (size_t)k * 4, cudaMemcpyDeviceToDevice,
                                 p->stream));
  k_lower_bounds<<<grid_for(p->ncolors + 1, kThreads, g), kThreads, 0, p->stream>>>(
      in_alt ? ka : keys, k, p->ncolors, nullptr, p->color_ptr);
  p->prof.launches[K_SETUP] += 2;
  GENCD_CUDA_TRY(cudaGetLastError());
  std::vector<int32_t> h((size_t)p->ncolors + 1);
  GENCD_CUDA_TRY(cudaMemcpyAsync(h.data(), p->color_ptr, h.size() * 4, cudaMemcpyDeviceToHost, p->stream));
  GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
  int32_t mx = 0;
  for (int32_t c = 0; c < p->ncolors; ++c) mx = std::max(mx, h[c + 1] - h[c]);
  p->max_class = mx;
  p->perm_epoch = -1;  // the colour permutation must be redrawn
  return GENCD_OK;
}

int run_coloring(gencd_problem* p) {
  GENCD_TRY(build_csr(p));
  const int64_t k = p->k;
  if (!p->color) GENCD_TRY(dev_alloc_bytes(p, (void**)&p->color, sizeof(int32_t) * (size_t)k));
  GENCD_CUDA_TRY(cudaMemsetAsync(p->color, 0xff, sizeof(int32_t) * (size_t)k, p->stream));  // -1
  int32_t *wa = nullptr, *wb = nullptr;
  unsigned long long* ctr = nullptr;  // [0] next worklist size, [1] max colour
  GENCD_TRY(dev_alloc_bytes(p, (void**)&wa, sizeof(int32_t) * (size_t)k));
  GENCD_TRY(dev_alloc_bytes(p, (void**)&wb, sizeof(int32_t) * (size_t)k));
  GENCD_TRY(dev_alloc_bytes(p, (void**)&ctr, 2 * sizeof(unsigned long long)));
  GENCD_CUDA_TRY(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), p->stream));
  const int g = p->num_sms * 8;
  k_iota_i32<<<grid_for(k, kThreads, g), kThreads, 0, p->stream>>>(wa, k);
  int64_t m = k;
  int rc = GENCD_OK;
  // every round colours at least the lowest-index waiting column, so k rounds suffice
  for (int64_t round = 0; m > 0 && round <= k; ++round) {
    if (cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), p->stream) != cudaSuccess) {
      rc = GENCD_ECUDA;
      break;
    }
    k_jp_round<<<grid_for(m * 32, kThreads, g), kThreads, 0, p->stream>>>(
        p->col_ptr, p->row_idx, p->row_ptr, p->col_idx, wa, m, wb, ctr, p->color, ctr + 1);
    p->prof.launches[K_SETUP] += 1;
    unsigned long long next = 0;
    if (cudaMemcpyAsync(&next, ctr, sizeof(next), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess) {
      set_error(std::string("colouring round failed: ") + cudaGetErrorString(cudaGetLastError()));
      rc = GENCD_ECUDA;
      break;
    }
    m = (int64_t)next;
    std::swap(wa, wb);
  }
  unsigned long long mc = 0;
  if (rc == GENCD_OK) {
    if (cudaMemcpy(&mc, ctr + 1, sizeof(mc), cudaMemcpyDeviceToHost) != cudaSuccess) rc = GENCD_ECUDA;
    if (m > 0 && rc == GENCD_OK) {
      set_error("colouring did not finish");
      rc = GENCD_ETIMEOUT;
    }
  }
  dev_free(p, wa);
  dev_free(p, wb);
  dev_free(p, ctr);
  if (rc != GENCD_OK) return rc;
  p->ncolors = k > 0 ? (int32_t)mc + 1 : 0;
  return build_color_classes(p);
}

// ---------------------------------------------------------------------------
// power iteration pieces: s = dinv .* v ; r = X s ; gacc = X^T r
__global__ void k_scale_vec(const double* __restrict__ a, const double* __restrict__ b, int64_t m,
                            double* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) out[i] = a[i] * b[i];
}

int launch_power_step(gencd_problem* p, const double* v, const double* dinv, double* r, double* s) {
  const int g = p->num_sms * 8;
  k_scale_vec<<<grid_for(p->k, kThreads, g), kThreads, 0, p->stream>>>(v, dinv, p->k, s);
  p->prof.launches[K_SETUP] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  GENCD_TRY(launch_csr_spmv(p, s, r));
  return launch_propose_all(p, r, true);
}

__global__ void k_scale_from_acc(double* __restrict__ gacc, int64_t k, double inv_n, double* __restrict__ c) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    c[j] = gacc[j] * inv_n;
    gacc[j] = 0.0;
  }
}

// c_j = ||X_j||^2 / n with the load-balanced streaming pass (needs the tile map)
int launch_col_scale(gencd_problem* p) {
  GENCD_TRY(launch_col_sumsq(p));
  k_scale_from_acc<<<grid_for(p->k, kThreads, p->num_sms * 8), kThreads, 0, p->stream>>>(
      p->gacc, p->k, 1.0 / (double)p->n, p->c);
  p->prof.launches[K_SETUP] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

int launch_tile_map_of(gencd_problem* p, const int64_t* col_ptr, int64_t k, int64_t ntiles, int32_t* tile_col,
                       int64_t tile) {
  k_tile_map<<<grid_for(k, kThreads, p->num_sms * 8), kThreads, 0, p->stream>>>(col_ptr, k, tile, ntiles, tile_col);
  p->prof.launches[K_SETUP] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

int launch_tile_map(gencd_problem* p) {
  return launch_tile_map_of(p, p->col_ptr, p->k, p->ntiles, p->tile_col, 32LL * p->items);
}

// validation entry used by the API: returns first bad column / row or -1
int validate_input(gencd_problem* p, int64_t* bad_col, int64_t* bad_row, int* stage) {
  unsigned long long* err = nullptr;
  GENCD_TRY(dev_alloc_bytes(p, (void**)&err, 3 * sizeof(unsigned long long)));
  GENCD_CUDA_TRY(cudaMemsetAsync(err, 0xff, 3 * sizeof(unsigned long long), p->stream));
  const int g = p->num_sms * 8;
  k_validate_colptr<<<grid_for(p->k, kThreads, g), kThreads, 0, p->stream>>>(p->col_ptr, p->k, p->nnz, err);
  unsigned long long h[3] = {0, 0, 0};
  GENCD_CUDA_TRY(cudaMemcpyAsync(h, err, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
  GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
  *stage = 0;
  if (h[0] != ~0ull) {
    *bad_col = (int64_t)h[0];
    dev_free(p, err);
    return GENCD_OK;
  }
  *stage = 1;
  uint32_t* starts = nullptr;
  const int64_t words = (p->nnz + 31) / 32 + 1;
  GENCD_TRY(dev_alloc_bytes(p, (void**)&starts, words * sizeof(uint32_t)));
  GENCD_CUDA_TRY(cudaMemsetAsync(starts, 0, words * sizeof(uint32_t), p->stream));
  k_mark_starts<<<grid_for(p->k, kThreads, g), kThreads, 0, p->stream>>>(p->col_ptr, p->k, starts);
  if (p->precision == GENCD_F64)
    k_validate_rows<double><<<grid_for(p->nnz, kThreads, g), kThreads, 0, p->stream>>>(
        p->col_ptr, p->row_idx, (const double*)p->val, starts, p->k, p->n, p->nnz, err);
  else
    k_validate_rows<float><<<grid_for(p->nnz, kThreads, g), kThreads, 0, p->stream>>>(
        p->col_ptr, p->row_idx, (const float*)p->val, starts, p->k, p->n, p->nnz, err);
  dev_free(p, starts);
  k_validate_y<<<grid_for(p->n, kThreads, g), kThreads, 0, p->stream>>>(p->y, p->n,
                                                                        p->loss == GENCD_LOSS_LOGISTIC, err + 1);
  p->prof.launches[K_SETUP] += 4;
  GENCD_CUDA_TRY(cudaMemcpyAsync(h, err, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
  GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
  dev_free(p, err);
  *bad_col = h[0] == ~0ull ? -1 : (int64_t)h[0];
  *bad_row = h[1] == ~0ull ? -1 : (int64_t)h[1];
  return GENCD_OK;
}

}  // namespace gencd
