// noalloc.cu -- gencd_propose_all_noalloc: the streaming Propose over all
// columns for callers that cannot allocate device memory.
//
// Who needs it: a host thread that must not synchronise the device (cudaMalloc
// and cudaFree can wait for the GPU to go idle), a process whose framework
// has already reserved all device memory in its own pool, or code that
// enqueues work while another thread captures the stream into a graph.  Such
// a caller passes the inputs and outputs; the call creates no problem handle
// and allocates nothing.  Its scratch (per-column sums and the tile map) is a
// file-scope device array of fixed size that every GPU loading this library
// holds until the process exits.
//
// The scratch is shared by every call on a device and keeps the last call's
// contents: each call clears the part it accumulates into before using it,
// and two calls that overlap on the GPU (different streams, no ordering
// between them) race on it.
#include <mutex>
#include <string>

#include "device_math.cuh"
#include "gencd_internal.cuh"

namespace gencd {

constexpr int64_t kNoAllocMaxCols = int64_t(1) << 19;  // columns (k)
constexpr int kNoAllocItems = 4;                        // nnz per lane
constexpr int64_t kNoAllocTile = 32 * kNoAllocItems;
constexpr int64_t kNoAllocMaxNnz = int64_t(1) << 25;   // non-zeros
constexpr int64_t kNoAllocMaxTiles = kNoAllocMaxNnz / kNoAllocTile;

// layout: [0, K) column sums X_j^T u, [K, 2K) sums of X_ij^2, then the tile map
// (int32, max tiles + 1 entries); 2 K + (max tiles + 2) / 2 = 1,179,649 doubles
// = 9,437,192 bytes (9.44 MB, 9.0 MiB)
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxCols + (kNoAllocMaxTiles + 2) / 2];

__global__ void k_na_clear(double* __restrict__ sums, int64_t k, double* __restrict__ kkt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < 2 * k; j += stride) sums[j] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *kkt = 0.0;
}

__global__ void k_na_tile_map(const int64_t* __restrict__ col_ptr, int64_t k, int64_t ntiles,
                              int32_t* __restrict__ tile_col) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    const int64_t s = col_ptr[j], e = col_ptr[j + 1];
    for (int64_t t = (s + kNoAllocTile - 1) / kNoAllocTile; t * kNoAllocTile < e; ++t) tile_col[t] = (int32_t)j;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tile_col[ntiles] = (int32_t)(k - 1);
}

__device__ __forceinline__ void na_emit(double* __restrict__ sums, int64_t k, int32_t c, double su, double sq,
                                        bool whole) {
  if (whole) {
    sums[c] = su;
    sums[k + c] = sq;
  } else {
    atomicAdd(sums + c, su);
    atomicAdd(sums + k + c, sq);
  }
}

// Lane-segmented pass over the non-zeros: u_i = l'(y_i, z_i) is evaluated on
// the fly (no u array), and the sums of squares give beta_j without a
// separate pass.  Scalar loads: the caller's arrays need no padding.
__global__ void __launch_bounds__(kThreads)
    k_na_stream(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                const double* __restrict__ val, const double* __restrict__ y, const double* __restrict__ z, int loss,
                const int32_t* __restrict__ tile_col, int64_t nnz, int64_t ntiles, int64_t k,
                double* __restrict__ sums) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = warp; t < ntiles; t += nwarps) {
    const int64_t a = t * kNoAllocTile + (int64_t)lane * kNoAllocItems;
    if (a >= nnz) continue;
    const int64_t b = a + kNoAllocItems < nnz ? a + kNoAllocItems : nnz;
    int32_t lo = tile_col[t], hi = tile_col[t + 1];
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (col_ptr[mid] <= a)
        lo = mid;
      else
        hi = mid - 1;
    }
    int32_t c = lo;
    int64_t cend = col_ptr[c + 1];
    bool whole = col_ptr[c] >= a;
    double su = 0.0, sq = 0.0;
    for (int64_t p = a; p < b; ++p) {
      while (p >= cend) {
        na_emit(sums, k, c, su, sq, whole);
        ++c;
        cend = col_ptr[c + 1];
        su = sq = 0.0;
        whole = true;
      }
      const int32_t i = row_idx[p];
      const double v = val[p];
      su = fma(v, loss_deriv(loss, y[i], z[i]), su);
      sq = fma(v, v, sq);
    }
    na_emit(sums, k, c, su, sq, whole && cend <= b);
  }
}

__global__ void __launch_bounds__(kThreads)
    k_na_finalize(const double* __restrict__ sums, const double* __restrict__ w, int64_t k, double n, double lam,
                  double beta, int beta_mode, double* __restrict__ delta, double* __restrict__ phi,
                  double* __restrict__ kkt) {
  double vmax = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    const double g = sums[j] / n;
    const double bj = beta_mode ? beta : beta * (sums[k + j] / n);
    double d, f;
    eq7_step(g, w[j], lam, bj, bj > 0.0 ? 1.0 / bj : 0.0, d, f);
    delta[j] = d;
    phi[j] = f;
    const double v = kkt_violation(g, w[j], lam);
    vmax = (v > vmax || v != v) ? v : vmax;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double x = __shfl_xor_sync(0xffffffffu, vmax, o);
    vmax = (x > vmax || x != x) ? x : vmax;
  }
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(kkt, vmax);
}

// device address of the scratch array, looked up once per device with that
// device current (the host symbol is not a device address)
static std::mutex g_na_mutex;
static double* g_na_ptr[64] = {nullptr};

static int noalloc_scratch(double** out) {
  int dev = 0;
  GENCD_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail_plan("device index out of range for the no-allocation scratch table");
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* ptr = nullptr;
    GENCD_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_na_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = g_na_ptr[dev];
  return GENCD_OK;
}

}  // namespace gencd

using namespace gencd;

extern "C" int gencd_propose_all_noalloc(int64_t n, int64_t k, int64_t nnz, const int64_t* col_ptr,
                                         const int32_t* row_idx, const double* val, const double* y,
                                         const double* z, const double* w, int32_t loss, double lambda,
                                         int32_t beta_mode, double* delta, double* phi, double* kkt,
                                         void* stream) {
  set_error("");
  if (n < 1 || k < 1 || nnz < 0) return fail_plan("need n >= 1, k >= 1, nnz >= 0");
  if (k > kNoAllocMaxCols || nnz > kNoAllocMaxNnz)
    return fail_plan(("gencd_propose_all_noalloc handles at most " + std::to_string(kNoAllocMaxCols) +
                      " columns and " + std::to_string(kNoAllocMaxNnz) + " non-zeros (its scratch is a fixed "
                      "device array); use a problem handle for larger inputs")
                         .c_str());
  if (!col_ptr || !y || !z || !w || !delta || !phi || !kkt || (nnz > 0 && (!row_idx || !val)))
    return fail_plan("a required pointer is NULL");
  if (loss != GENCD_LOSS_SQUARED && loss != GENCD_LOSS_LOGISTIC) return fail_plan("unknown loss");
  if (!(lambda >= 0.0) || !std::isfinite(lambda) || (beta_mode != 0 && beta_mode != 1))
    return fail_plan("lambda must be finite and >= 0, beta_mode 0 or 1");
  double* scratch = nullptr;
  GENCD_TRY(noalloc_scratch(&scratch));
  double* sums = scratch;
  int32_t* tile_col = reinterpret_cast<int32_t*>(scratch + 2 * kNoAllocMaxCols);
  cudaStream_t st = (cudaStream_t)stream;
  int sms = 0, dev = 0;
  GENCD_CUDA_TRY(cudaGetDevice(&dev));
  GENCD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int g = sms * 8;
  const int64_t ntiles = (nnz + kNoAllocTile - 1) / kNoAllocTile;
  k_na_clear<<<grid_for(2 * k, kThreads, g), kThreads, 0, st>>>(sums, k, kkt);
  if (ntiles > 0) {
    k_na_tile_map<<<grid_for(k, kThreads, g), kThreads, 0, st>>>(col_ptr, k, ntiles, tile_col);
    k_na_stream<<<grid_for(ntiles * 32, kThreads, g), kThreads, 0, st>>>(col_ptr, row_idx, val, y, z, loss, tile_col,
                                                                         nnz, ntiles, k, sums);
  }
  const double beta = loss == GENCD_LOSS_SQUARED ? 1.0 : 0.25;
  k_na_finalize<<<grid_for(k, kThreads, g), kThreads, 0, st>>>(sums, w, k, (double)n, lambda, beta, beta_mode, delta,
                                                               phi, kkt);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}
