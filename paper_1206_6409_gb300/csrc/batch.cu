// batch.cu -- many GenCD solves over one shared X: the batched Thread-Greedy
// step (Algorithm 1 with Table 2's Thread-Greedy Accept, one step for every
// active slot) and the host runtime that runs regularisation paths on it.
//
// Layout (S = slots, a multiple of 32):
//   U  float [n][S]   u_is = l'(y_i, z_is) on the slot's training rows, else 0
//   z  double[n][S]   fitted values
//   G  float [k][S]   column sums X_j^T u_s (unscaled)
//   w  double[k][S], w32 float[k][S] (zero exactly when w is)
// so that one row of U or z, and one row of G or w, is one contiguous vector
// of S values: a warp reads 32 slots of it in one 128-byte transaction.
//
// Kernels of one step:
//   k_b_prep    zero the G rows that k_b_spmm accumulates atomically, and the
//               per-slot KKT maxima
//   k_b_spmm    G = X^T U: warps own equal ranges of 32-entry tiles of the CSC
//               (load balanced for any column length); per entry a warp
//               gathers the entry's U row (S floats, coalesced) and lanes add
//               x * u into per-slot accumulators; a start bit per entry marks
//               column starts; whole columns are stored, the first and last
//               column of a warp's range are added atomically
//   k_b_accept  one CTA per partition b: Eq. 7 / Eq. 9 in FP32 for every
//               (column, slot), the best proxy per slot, the winner's step
//               recomputed in FP64, the KKT violation per slot
//   k_b_update  one warp per accepted (partition, slot): w += delta and
//               z_s += delta X_j (FP64 atomics: partitions may share rows)
//   k_b_refresh the same traversal: u_s on the touched rows
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "device_math.cuh"
#include "gencd_batch.h"
#include "gencd_internal.cuh"

namespace gencd {

constexpr int kBatchMaxSlots = 256;
constexpr int kBatchMaxFolds = 31;
constexpr int kSpmmThreads = 256;
constexpr int kAcceptThreads = 512;  // per partition: slots x column strides
constexpr int kObjChecks = 8;        // convergence checks between objective evaluations of a path solve
constexpr int kStallIters = 500;     // iterations without progress taken as a stall (as gencd_solve)
constexpr double kStallGain = 1e-2;  // a new lowest KKT value is 1% below the previous one
constexpr double kObjGain = 1e-12;   // a new lowest objective is this far (relative) below the previous one
constexpr double kStallKkt = 1e-3;   // stalls count while the KKT value is at least this times lambda

static int bfail(int code, const std::string& m) {
  set_error(m);
  return code;
}

template <typename T>
static int balloc(T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void**)ptr, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return bfail(GENCD_ENOMEM, "cudaMalloc of " + std::to_string(sizeof(T) * count) + " bytes failed");
  }
  return GENCD_OK;
}

// ---------------------------------------------------------------------------
// setup kernels

// start bit of every non-empty column's first entry; flag of non-empty columns
__global__ void k_b_starts(const int64_t* __restrict__ col_ptr, int64_t k, uint32_t* __restrict__ tstart,
                           uint32_t* __restrict__ flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    const int64_t s = col_ptr[j], e = col_ptr[j + 1];
    flag[j] = e > s ? 1u : 0u;
    if (e > s) atomicOr(tstart + (s >> 5), 1u << (s & 31));
  }
}

__global__ void k_b_compact(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos, int64_t k,
                            int32_t* __restrict__ nzcols) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride)
    if (flag[j]) nzcols[pos[j]] = (int32_t)j;
}

// tile_cc[t] = compact index of the column holding entry 32 t
__global__ void k_b_tile_cc(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ nzcols, int64_t nc,
                            int32_t* __restrict__ tile_cc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += stride) {
    const int32_t j = nzcols[c];
    const int64_t s = col_ptr[j], e = col_ptr[j + 1];
    for (int64_t t = (s + 31) >> 5; (t << 5) < e; ++t) tile_cc[t] = (int32_t)c;
  }
}

// the columns a warp's range adds atomically: its first and its last column
__global__ void k_b_bounds(const int32_t* __restrict__ tile_cc, const uint32_t* __restrict__ tstart,
                           const int32_t* __restrict__ nzcols, int64_t ntiles, int64_t W, int32_t* __restrict__ bnd) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < W; w += stride) {
    const int64_t t0 = ntiles * w / W, t1 = ntiles * (w + 1) / W;
    if (t0 >= t1) {
      bnd[2 * w] = bnd[2 * w + 1] = -1;
      continue;
    }
    bnd[2 * w] = nzcols[tile_cc[t0]];
    bnd[2 * w + 1] = nzcols[tile_cc[t1 - 1] + __popc(tstart[t1 - 1] & ~1u)];
  }
}

// rows per fold; *bad = first row whose fold is out of range
__global__ void k_b_fold_counts(const uint8_t* __restrict__ fold, int64_t n, int nfolds,
                                unsigned long long* __restrict__ counts, unsigned long long* __restrict__ bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int f = fold[i];
    if (f >= nfolds)
      atomicMin(bad, (unsigned long long)i);
    else
      atomicAdd(counts + f, 1ull);
  }
}

// Column sums of squares over each training set: sq[f][j] = sum over rows
// outside fold f of X_ij^2 (f < F) and sq[F][j] over all rows.  The sums
// per fold are formed first and the training sums add the other folds', so
// a column with no rows in a training set gets exactly 0.
__global__ void k_b_colsq(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row,
                          const float* __restrict__ val, const uint8_t* __restrict__ fold, int64_t k, int nfolds,
                          double* __restrict__ sq) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    double per[kBatchMaxFolds + 1];
    for (int f = 0; f <= nfolds; ++f) per[f] = 0.0;
    for (int64_t t = col_ptr[j]; t < col_ptr[j + 1]; ++t) {
      const double x = (double)val[t];
      per[nfolds > 0 ? fold[row[t]] : 0] += x * x;
    }
    double all = 0.0;
    for (int f = 0; f < (nfolds > 0 ? nfolds : 1); ++f) all += per[f];
    for (int f = 0; f < nfolds; ++f) {
      double tr = 0.0;
      for (int g = 0; g < nfolds; ++g)
        if (g != f) tr += per[g];
      sq[(int64_t)f * k + j] = tr;
    }
    sq[(int64_t)nfolds * k + j] = all;
  }
}

// beta_j and 1/beta_j of every training set (Eq. 7; beta_mode as gencd_params)
__global__ void k_b_beta(const double* __restrict__ sq, int64_t m, int64_t k, const double* __restrict__ inv_n,
                         double beta, int beta_mode, double* __restrict__ bj, double* __restrict__ ib,
                         float* __restrict__ bj32, float* __restrict__ ib32) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += stride) {
    const double c = sq[q] * inv_n[q / k];
    const double b = c > 0.0 ? (beta_mode ? beta : beta * c) : 0.0;
    const double i = b > 0.0 ? 1.0 / b : 0.0;
    bj[q] = b;
    ib[q] = i;
    bj32[q] = (float)b;
    ib32[q] = (float)i;
  }
}

// U0[i][f] = l'(y_i, 0) on training set f's rows (f <= F), for lambda_max
__global__ void k_b_u0(const double* __restrict__ y, const uint8_t* __restrict__ fold, int64_t n, int nfolds, int loss,
                       float* __restrict__ U0) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * 32; q += stride) {
    const int64_t i = q >> 5;
    const int f = (int)(q & 31);
    float v = 0.0f;
    if (f <= nfolds && (f == nfolds || fold[i] != f)) v = u_value<float>(loss, y[i], 0.0);
    U0[q] = v;
  }
}

// bits[f] = max_j |G0[j][f]| (non-negative floats order like their bits)
__global__ void k_b_absmax(const float* __restrict__ G0, int64_t k, int nsets, unsigned int* __restrict__ bits) {
  const int lane = threadIdx.x & 31;
  float m = 0.0f;
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < k; j += stride)
    m = fmaxf(m, fabsf(G0[j * 32 + lane]));
  if (lane < nsets) atomicMax(bits + lane, __float_as_uint(m));
}

// ---------------------------------------------------------------------------
// the step

// zero the G rows added atomically by k_b_spmm, and the per-slot KKT maxima
__global__ void k_b_prep(const int32_t* __restrict__ bnd, int64_t nb, int Sp, float* __restrict__ G,
                         unsigned int* __restrict__ kkt_bits) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t total = nb * Sp;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
    const int32_t j = bnd[q / Sp];
    if (j >= 0) G[(int64_t)j * Sp + (q % Sp)] = 0.0f;
  }
  if (kkt_bits && blockIdx.x == 0)
    for (int s = threadIdx.x; s < 2 * Sp; s += blockDim.x) kkt_bits[s] = 0u;  // KKT and max |g| per slot
}

template <int NC>
__device__ __forceinline__ void b_flush(float* __restrict__ G, const int32_t* __restrict__ nzcols, int32_t cc,
                                        const float (&acc)[NC], bool atomic, int lane) {
  float* g = G + (int64_t)__ldg(nzcols + cc) * (32 * NC) + lane;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (atomic)
      atomicAdd(g + 32 * c, acc[c]);
    else
      g[32 * c] = acc[c];
  }
}

// G = X^T U for S = 32 NC slots.  Warp w owns tiles [T w / W, T (w+1) / W)
// of 32 entries; GRP entries' U rows are loaded together (GRP * NC loads in
// flight per lane), and the next tile's rows and values are loaded while the
// current tile is summed.
template <int NC, int GRP>
__global__ void __launch_bounds__(kSpmmThreads)
    k_b_spmm(const int32_t* __restrict__ row, const float* __restrict__ val, const uint32_t* __restrict__ tstart,
             const int32_t* __restrict__ tile_cc, const int32_t* __restrict__ nzcols, const float* __restrict__ U,
             float* __restrict__ G, int64_t ntiles, int64_t W) {
  constexpr int Sp = 32 * NC;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= W) return;
  const int64_t t0 = ntiles * w / W, t1 = ntiles * (w + 1) / W;
  if (t0 >= t1) return;
  int32_t cc = __ldg(tile_cc + t0);
  bool first = true;
  float acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0f;
  int32_t rn = __ldcs(row + t0 * 32 + lane);
  float xn = __ldcs(val + t0 * 32 + lane);
  uint32_t mn = __ldg(tstart + t0) & ~1u;  // the range's first entry closes nothing
  for (int64_t t = t0; t < t1; ++t) {
    const int32_t rl = rn;
    const float xl = xn;
    const uint32_t m = mn;
    if (t + 1 < t1) {
      rn = __ldcs(row + (t + 1) * 32 + lane);
      xn = __ldcs(val + (t + 1) * 32 + lane);
      mn = __ldg(tstart + t + 1);
    }
#pragma unroll
    for (int g = 0; g < 32; g += GRP) {
      int32_t r[GRP];
      float x[GRP], uu[GRP][NC];
#pragma unroll
      for (int q = 0; q < GRP; ++q) {
        r[q] = __shfl_sync(FULL, rl, g + q);
        x[q] = __shfl_sync(FULL, xl, g + q);
      }
#pragma unroll
      for (int q = 0; q < GRP; ++q)
#pragma unroll
        for (int c = 0; c < NC; ++c) uu[q][c] = __ldg(U + (int64_t)r[q] * Sp + 32 * c + lane);
#pragma unroll
      for (int q = 0; q < GRP; ++q) {
        if ((m >> (g + q)) & 1u) {  // warp-uniform: entry g + q starts the next column
          b_flush<NC>(G, nzcols, cc, acc, first, lane);
          first = false;
          ++cc;
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[c] = 0.0f;
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fmaf(x[q], uu[q][c], acc[c]);
      }
    }
  }
  b_flush<NC>(G, nzcols, cc, acc, true, lane);
}

// per-slot parameters, one array of S values each
struct SlotArgs {
  const int32_t* set;  // training set (0..F; F = all rows), -1 inactive
  const int32_t* group;  // partitions merged per accept group (1: plain Thread-Greedy)
  const double* lam;
  const float* lam32;
  const double* invn;  // 1 / n_s
  const float* invn32;
};

// Thread-Greedy Accept for every slot of partition b = blockIdx.x.  Thread
// (s, r) scans columns lo + r, lo + r + R, ... of the partition for slot s.
// MODE 1: accept (acc_j = column or -1, acc_d = FP64 step) and KKT; MODE 0:
// KKT only.
template <int MODE>
__global__ void __launch_bounds__(kAcceptThreads)
    k_b_accept(const float* __restrict__ G, const float* __restrict__ w32, const double* __restrict__ w,
               const float* __restrict__ bj32, const float* __restrict__ ib32, const double* __restrict__ bjs,
               const double* __restrict__ ibs, int64_t k, SlotArgs sa, const int64_t* __restrict__ part_lo, int Sp,
               int R, int32_t* __restrict__ acc_j, double* __restrict__ acc_d, double* __restrict__ acc_phi,
               unsigned int* __restrict__ kkt_bits) {
  __shared__ uint32_t s_mag[kAcceptThreads];
  __shared__ int32_t s_col[kAcceptThreads];
  __shared__ float s_v[kAcceptThreads];
  const int b = blockIdx.x;
  const int s = threadIdx.x % Sp, r = threadIdx.x / Sp;
  const bool live = r < R;
  const int set = live ? sa.set[s] : -1;
  uint32_t best = 0u;
  int32_t bcol = INT_MAX;
  float vmax = 0.0f, gmax = 0.0f;
  if (set >= 0) {
    const int64_t lo = part_lo[b], hi = part_lo[b + 1];
    const float lam = sa.lam32[s], invn = sa.invn32[s];
    const float* bjv = bj32 + (int64_t)set * k;
    const float* ibv = ib32 + (int64_t)set * k;
    for (int64_t j = lo + r; j < hi; j += R) {
      const float g = __ldg(G + j * Sp + s) * invn;
      const float wj = __ldg(w32 + j * Sp + s);
      float d, phi;
      eq7_step_f32(g, wj, lam, __ldg(bjv + j), __ldg(ibv + j), d, phi);
      const uint32_t m = candidate_mag32(phi);
      if (m > best) {  // columns ascend per thread: ties keep the lower column
        best = m;
        bcol = (int32_t)j;
      }
      vmax = fmaxf(vmax, kkt_violation_f32(g, wj, lam));
      gmax = fmaxf(gmax, fabsf(g));
    }
  }
  s_mag[threadIdx.x] = best;
  s_col[threadIdx.x] = bcol;
  s_v[threadIdx.x] = vmax;
  __syncthreads();
  float gm = 0.0f;  // max |g| over the partition (reusing s_v)
  if (live) {
    for (int q = 1; q < R; ++q) vmax = fmaxf(vmax, s_v[q * Sp + s]);
  }
  __syncthreads();
  s_v[threadIdx.x] = gmax;
  __syncthreads();
  if (r != 0 || s >= Sp) return;
  gm = gmax;
  for (int q = 1; q < R; ++q) {
    const int o = q * Sp + s;
    if (s_mag[o] > best || (s_mag[o] == best && s_col[o] < bcol)) {
      best = s_mag[o];
      bcol = s_col[o];
    }
    gm = fmaxf(gm, s_v[o]);
  }
  const int64_t slot = (int64_t)b * Sp + s;
  if (set < 0) {
    if (MODE == 1) {
      acc_j[slot] = -1;
      acc_phi[slot] = 0.0;
    }
    return;
  }
  if (vmax > 0.0f) atomicMax(kkt_bits + s, __float_as_uint(vmax));
  if (gm > 0.0f) atomicMax(kkt_bits + Sp + s, __float_as_uint(gm));
  if (MODE == 1) {
    int32_t oj = -1;
    double od = 0.0, of = 0.0;
    if (best > 0u) {  // the FP32 winner's step and proxy in FP64
      const int64_t q = (int64_t)set * k + bcol;
      const double g = (double)G[(int64_t)bcol * Sp + s] * sa.invn[s];
      double d, phi;
      eq7_step(g, w[(int64_t)bcol * Sp + s], sa.lam[s], bjs[q], ibs[q], d, phi);
      if (phi < 0.0) {
        oj = bcol;
        od = d;
        of = phi;
      }
    }
    acc_j[slot] = oj;
    acc_d[slot] = od;
    acc_phi[slot] = of;
  }
}

// Accept backoff: a slot whose group size G > 1 keeps, of every G
// consecutive partitions, only the one whose accepted proxy is lowest (ties:
// the lower partition).  G = B is Greedy.
__global__ void k_b_merge(int32_t* __restrict__ acc_j, const double* __restrict__ acc_phi, int B, int Sp,
                          const int32_t* __restrict__ group) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B * Sp) return;
  const int b = q / Sp, s = q % Sp;
  const int G = group[s];
  if (G <= 1 || b % G != 0) return;
  const int end = min(B, b + G);
  int win = -1;
  double best = 0.0;
  for (int c = b; c < end; ++c) {
    const double f = acc_phi[c * Sp + s];
    if (acc_j[c * Sp + s] >= 0 && (win < 0 || f < best)) {
      win = c;
      best = f;
    }
  }
  for (int c = b; c < end; ++c)
    if (c != win) acc_j[c * Sp + s] = -1;
}

// w += delta and z_s += delta X_j for every accepted (partition, slot)
__global__ void k_b_update(const int32_t* __restrict__ acc_j, const double* __restrict__ acc_d, int npairs, int Sp,
                           const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row,
                           const float* __restrict__ val, double* __restrict__ w, float* __restrict__ w32,
                           double* __restrict__ z, unsigned long long* __restrict__ ctr) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < npairs; q += nw) {
    const int32_t j = acc_j[q];
    if (j < 0) continue;
    const int s = q % Sp;
    const double d = acc_d[q];
    const int64_t a = col_ptr[j], e = col_ptr[j + 1];
    if (lane == 0) {
      const int64_t o = (int64_t)j * Sp + s;
      const double nwj = w[o] + d;
      w[o] = nwj;
      w32[o] = w_mirror(nwj);
      atomicAdd(ctr, (unsigned long long)(e - a));
      atomicAdd(ctr + 1, 1ull);
    }
    for (int64_t t = a + lane; t < e; t += 32) atomicAdd(z + (int64_t)row[t] * Sp + s, d * (double)val[t]);
  }
}

// The same update with the slots that accepted the same column grouped: one
// warp per (partition, 32-slot chunk), lane = slot.  A column accepted by at
// least kGroupMin slots of the chunk is walked once, entry by entry, and the
// slots add into the entry's z row side by side (their S values are
// contiguous, so the atomics of one entry share a few L2 lines); a column
// accepted by fewer slots is walked by the lanes, one slot after another.
constexpr int kGroupMin = 4;

__global__ void k_b_update_grouped(const int32_t* __restrict__ acc_j, const double* __restrict__ acc_d, int B,
                                   int Sp, const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row,
                                   const float* __restrict__ val, double* __restrict__ w, float* __restrict__ w32,
                                   double* __restrict__ z, unsigned long long* __restrict__ ctr) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int per = (Sp + 31) / 32;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < (int64_t)B * per; q += nw) {
    const int b = (int)(q / per), c = (int)(q % per);
    const int s = 32 * c + lane;
    const bool in = s < Sp;
    const int32_t j = in ? acc_j[(int64_t)b * Sp + s] : -1;
    const double d = in ? acc_d[(int64_t)b * Sp + s] : 0.0;
    int64_t a = 0, e = 0;
    if (j >= 0) {
      a = col_ptr[j];
      e = col_ptr[j + 1];
      const int64_t o = (int64_t)j * Sp + s;
      const double nwj = w[o] + d;
      w[o] = nwj;
      w32[o] = w_mirror(nwj);
      atomicAdd(ctr, (unsigned long long)(e - a));
      atomicAdd(ctr + 1, 1ull);
    }
    unsigned pending = __ballot_sync(FULL, j >= 0);
    while (pending) {  // warp-uniform: one accepted column at a time
      const int leader = __ffs(pending) - 1;
      const int32_t jl = __shfl_sync(FULL, j, leader);
      const unsigned mask = __ballot_sync(FULL, j == jl) & pending;
      pending &= ~mask;
      const int64_t al = __shfl_sync(FULL, a, leader), el = __shfl_sync(FULL, e, leader);
      if (__popc(mask) >= kGroupMin) {
        for (int64_t t0 = al; t0 < el; t0 += 32) {
          const int64_t t = t0 + lane;
          const int32_t r = t < el ? row[t] : 0;
          const float v = t < el ? val[t] : 0.0f;
          const int cnt = (int)(el - t0 < 32 ? el - t0 : 32);
          for (int i = 0; i < cnt; ++i) {
            const int32_t ri = __shfl_sync(FULL, r, i);
            const float vi = __shfl_sync(FULL, v, i);
            if ((mask >> lane) & 1u) atomicAdd(z + (int64_t)ri * Sp + s, d * (double)vi);
          }
        }
      } else {
        unsigned m = mask;
        while (m) {
          const int l = __ffs(m) - 1;
          m &= m - 1;
          const double dl = __shfl_sync(FULL, d, l);
          const int sl = 32 * c + l;
          for (int64_t t = al + lane; t < el; t += 32) atomicAdd(z + (int64_t)row[t] * Sp + sl, dl * (double)val[t]);
        }
      }
    }
  }
}

__device__ __forceinline__ bool b_train(const uint8_t* __restrict__ fold, int64_t i, int set, int nfolds) {
  return set == nfolds || fold[i] != set;
}

// u_s on the rows of every accepted (partition, slot)'s column
__global__ void k_b_refresh(const int32_t* __restrict__ acc_j, int npairs, int Sp, const int64_t* __restrict__ col_ptr,
                            const int32_t* __restrict__ row, const double* __restrict__ y,
                            const uint8_t* __restrict__ fold, int nfolds, int loss, const int32_t* __restrict__ sset,
                            const double* __restrict__ z, float* __restrict__ U) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < npairs; q += nw) {
    const int32_t j = acc_j[q];
    if (j < 0) continue;
    const int s = q % Sp;
    const int set = sset[s];
    for (int64_t t = col_ptr[j] + lane; t < col_ptr[j + 1]; t += 32) {
      const int64_t i = row[t];
      const int64_t o = i * Sp + s;
      U[o] = b_train(fold, i, set, nfolds) ? u_value<float>(loss, y[i], z[o]) : 0.0f;
    }
  }
}

// u_s on every row of every slot (thread (s, row), block Sp x rows): the
// dense form of k_b_refresh, cheaper when the accepted columns touch more
// (row, slot) entries than there are rows times slots
__global__ void k_b_refresh_all(const double* __restrict__ y, const uint8_t* __restrict__ fold, int nfolds, int loss,
                                const int32_t* __restrict__ sset, const double* __restrict__ z, int64_t n, int Sp,
                                float* __restrict__ U) {
  const int s = threadIdx.x;
  const int set = sset[s];
  const int64_t stride = (int64_t)gridDim.x * blockDim.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < n; i += stride) {
    const int64_t o = i * Sp + s;
    const bool train = set >= 0 && (set == nfolds || fold[i] != set);
    U[o] = train ? u_value<float>(loss, y[i], z[o]) : 0.0f;
  }
}

// G[:, 8c .. 8c+8) = X^T U[:, 8c .. 8c+8) for chunk c = blockIdx.y, lanes over
// entries: a warp takes 256-entry tiles, a lane 8 consecutive entries, and
// each lane keeps the 8 slots' sums of its current column in registers (one
// 32-byte U row per entry, loaded as two 16-byte vectors).  Start bits (one
// byte per 8 entries) mark column starts; a lane stores the columns that
// start and end inside it, and the column continuing from the left (cont) or
// leaving to the right (tail) is combined across the warp by a segmented
// suffix sum, so only a tile's first and last column are added atomically.
// G must be zero before the launch.
__device__ __forceinline__ void b_row8(const float* __restrict__ p, float (&u)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  u[0] = a.x, u[1] = a.y, u[2] = a.z, u[3] = a.w, u[4] = b.x, u[5] = b.y, u[6] = b.z, u[7] = b.w;
}

__device__ __forceinline__ void b_store8(float* __restrict__ p, const float (&v)[8]) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}

__device__ __forceinline__ void b_add8(float* __restrict__ p, const float (&v)[8]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) atomicAdd(p + q, v[q]);
}

__global__ void __launch_bounds__(kThreads, 2)
    k_b_spmm_runs8(const int32_t* __restrict__ row, const float* __restrict__ val, const uint8_t* __restrict__ smask,
                   const int32_t* __restrict__ tile_cc, const int32_t* __restrict__ nzcols,
                   const float* __restrict__ U, int S, float* __restrict__ G, int64_t nnz, int64_t ntiles) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const float* __restrict__ Uc = U + 8 * blockIdx.y;
  float* __restrict__ Gc = G + 8 * blockIdx.y;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntiles; t += nwarps) {
    const int64_t a = t * 256 + (int64_t)lane * 8;
    const bool active = a < nnz;
    int32_t r[8];
    float x[8];
    uint32_t m = 0;
    if (active) {  // rows and values are padded: a lane's 8 entries are in bounds
      const int4 r0 = __ldcs(reinterpret_cast<const int4*>(row + a));
      const int4 r1 = __ldcs(reinterpret_cast<const int4*>(row + a) + 1);
      const float4 x0 = __ldcs(reinterpret_cast<const float4*>(val + a));
      const float4 x1 = __ldcs(reinterpret_cast<const float4*>(val + a) + 1);
      r[0] = r0.x, r[1] = r0.y, r[2] = r0.z, r[3] = r0.w, r[4] = r1.x, r[5] = r1.y, r[6] = r1.z, r[7] = r1.w;
      x[0] = x0.x, x[1] = x0.y, x[2] = x0.z, x[3] = x0.w, x[4] = x1.x, x[5] = x1.y, x[6] = x1.z, x[7] = x1.w;
      m = smask[a >> 3];
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) r[i] = 0, x[i] = 0.0f;
    }
    const uint32_t lc0 = (uint32_t)__ldg(tile_cc + t * 8);
    // compact column of this lane's first entry: the tile's first column plus
    // the column starts before it (lane 0's entry 0 is the tile's own start)
    const uint32_t cnt = __popc(lane == 0 ? (m & 0xfeu) : m);
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t yv = __shfl_up_sync(FULL, incl, d);
      if (lane >= d) incl += yv;
    }
    const uint32_t q = lc0 + (incl - cnt) + (lane > 0 ? (m & 1u) : 0u);
    float acc[8], first[8], cont[8], tail[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) acc[s] = first[s] = cont[s] = tail[s] = 0.0f;
    bool has_tail = false;
    if (active) {
      const uint32_t inner = m & 0xfeu;
      const int bf = inner ? __ffs(inner) - 1 : 8;
      uint32_t qi = q;
#pragma unroll
      for (int h = 0; h < 8; h += 4) {
        float u[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i) b_row8(Uc + (int64_t)r[h + i] * S, u[i]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if ((inner >> (h + i)) & 1u) {
            if (h + i == bf) {
#pragma unroll
              for (int s = 0; s < 8; ++s) first[s] = acc[s];
            } else {  // a whole column inside the lane
              b_store8(Gc + (int64_t)__ldg(nzcols + qi) * S, acc);
            }
#pragma unroll
            for (int s = 0; s < 8; ++s) acc[s] = 0.0f;
            ++qi;
          }
#pragma unroll
          for (int s = 0; s < 8; ++s) acc[s] = fmaf(x[h + i], u[i][s], acc[s]);
        }
      }
      if (inner) {
        if (m & 1u)  // started at entry 0 and ended inside
          b_store8(Gc + (int64_t)__ldg(nzcols + q) * S, first);
        else
#pragma unroll
          for (int s = 0; s < 8; ++s) cont[s] = first[s];
#pragma unroll
        for (int s = 0; s < 8; ++s) tail[s] = acc[s];
        has_tail = true;
      } else if (m & 1u) {
#pragma unroll
        for (int s = 0; s < 8; ++s) tail[s] = acc[s];
        has_tail = true;
      } else {
#pragma unroll
        for (int s = 0; s < 8; ++s) cont[s] = acc[s];
      }
    }
    const bool stop = !active || m != 0u;
    const bool lead = lane == 0 && active && !(m & 1u);
    if (__ballot_sync(FULL, stop) == 0u) {  // the whole tile lies inside column lc0
#pragma unroll
      for (int s = 0; s < 8; ++s) cont[s] = warp_sum(cont[s]);
      if (lane == 0) b_add8(Gc + (int64_t)__ldg(nzcols + lc0) * S, cont);
    } else {
      // segmented suffix sum of cont over the lanes up to the next stop
      bool e = stop;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const bool en = __shfl_down_sync(FULL, (int)e, d) != 0;
        float tn[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) tn[s] = __shfl_down_sync(FULL, cont[s], d);
        if (!e && lane + d < 32) {
#pragma unroll
          for (int s = 0; s < 8; ++s) cont[s] += tn[s];
          e = en;
        }
      }
      const bool e1 = __shfl_down_sync(FULL, (int)e, 1) != 0;
      float t1[8];
#pragma unroll
      for (int s = 0; s < 8; ++s) t1[s] = __shfl_down_sync(FULL, cont[s], 1);
      if (lead) b_add8(Gc + (int64_t)__ldg(nzcols + lc0) * S, cont);  // column from the previous tile
      if (has_tail) {
        const uint32_t ql = q + __popc(m & 0xfeu);
#pragma unroll
        for (int s = 0; s < 8; ++s) tail[s] += lane < 31 ? t1[s] : 0.0f;
        float* g = Gc + (int64_t)__ldg(nzcols + ql) * S;
        if (lane < 31 && e1)
          b_store8(g, tail);  // the column ends inside this tile
        else
          b_add8(g, tail);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// slot state and evaluation

// w column s from src (double[k]; NULL: zeros)
__global__ void k_b_set_w(const double* __restrict__ src, int64_t k, int Sp, int s, double* __restrict__ w,
                          float* __restrict__ w32) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    const double v = src ? src[j] : 0.0;
    w[j * Sp + s] = v;
    w32[j * Sp + s] = w_mirror(v);
  }
}

__global__ void k_b_get_w(const double* __restrict__ w, int64_t k, int Sp, int s, double* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) out[j] = w[j * Sp + s];
}

template <typename T>
__global__ void k_b_copy_col(T* __restrict__ a, int64_t m, int Sp, int from, int to) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += stride) a[q * Sp + to] = a[q * Sp + from];
}

__global__ void k_b_zero_col(double* __restrict__ z, int64_t n, int Sp, int s) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) z[i * Sp + s] = 0.0;
}

// z_s += w_js X_j for every column with w_js != 0 (one warp per column)
__global__ void k_b_scatter_z(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row,
                              const float* __restrict__ val, const double* __restrict__ w, int64_t k, int Sp, int s,
                              double* __restrict__ z) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < k; j += nw) {
    const double wj = w[j * Sp + s];
    if (wj == 0.0) continue;
    for (int64_t t = col_ptr[j] + lane; t < col_ptr[j + 1]; t += 32)
      atomicAdd(z + (int64_t)row[t] * Sp + s, wj * (double)val[t]);
  }
}

// u_s on every row
__global__ void k_b_fill_col(const double* __restrict__ y, const uint8_t* __restrict__ fold, int nfolds, int set,
                             int loss, const double* __restrict__ z, int64_t n, int Sp, int s, float* __restrict__ U) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t o = i * Sp + s;
    U[o] = (set >= 0 && b_train(fold, i, set, nfolds)) ? u_value<float>(loss, y[i], z[o]) : 0.0f;
  }
}

// acc[q] += loss sum over slot list[q]'s training rows; acc[m + q] += ||w_s||_1
// (block: 32 x 8 threads, threadIdx.x = list position)
// dual_scale (nullable): per listed slot, s = lambda_s / max(lambda_s,
// max_j |g_js|); then acc[2m + q] += the slot's sum over its training rows of
// l*(y_i, s u_is) (u from the FP64 fitted values): the duality gap's dual
// point (reading on the duality gap)
__global__ void k_b_objective(const double* __restrict__ y, const double* __restrict__ z,
                              const uint8_t* __restrict__ fold, int nfolds, int loss, int64_t n,
                              const double* __restrict__ w, int64_t k, int Sp, const int32_t* __restrict__ list,
                              const int32_t* __restrict__ list_set, int m, const double* __restrict__ dual_scale,
                              double* __restrict__ acc) {
  __shared__ double red[3][8][33];
  const int q = threadIdx.x;
  double sl = 0.0, s1 = 0.0, sc = 0.0;
  if (q < m) {
    const int s = list[q], set = list_set[q];
    const double sc_s = dual_scale ? dual_scale[q] : 0.0;
    const int64_t stride = (int64_t)gridDim.x * 8;
    for (int64_t i = (int64_t)blockIdx.x * 8 + threadIdx.y; i < n; i += stride)
      if (b_train(fold, i, set, nfolds)) {
        const double zi = z[i * Sp + s];
        sl += loss_value(loss, y[i], zi);
        if (dual_scale) sc += loss_conjugate(loss, y[i], sc_s * loss_deriv(loss, y[i], zi));
      }
    for (int64_t j = (int64_t)blockIdx.x * 8 + threadIdx.y; j < k; j += stride) s1 += fabs(w[j * Sp + s]);
  }
  red[0][threadIdx.y][q] = sl;
  red[1][threadIdx.y][q] = s1;
  red[2][threadIdx.y][q] = sc;
  __syncthreads();
  if (threadIdx.y == 0 && q < m) {
    for (int r = 1; r < 8; ++r) {
      sl += red[0][r][q];
      s1 += red[1][r][q];
      sc += red[2][r][q];
    }
    atomicAdd(acc + q, sl);
    atomicAdd(acc + m + q, s1);
    if (dual_scale) atomicAdd(acc + 2 * m + q, sc);
  }
}

// parity hook: FP64 Eq. 7 / Eq. 9 of every (column, slot), slot-major output
__global__ void k_b_propose(const float* __restrict__ G, const double* __restrict__ w, const double* __restrict__ bjs,
                            const double* __restrict__ ibs, int64_t k, SlotArgs sa, int Sp, double* __restrict__ delta,
                            double* __restrict__ phi) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < k * Sp; q += stride) {
    const int64_t j = q / Sp;
    const int s = (int)(q % Sp);
    const int set = sa.set[s];
    double d = 0.0, f = 0.0;
    if (set >= 0) {
      const double g = (double)G[q] * sa.invn[s];
      eq7_step(g, w[q], sa.lam[s], bjs[(int64_t)set * k + j], ibs[(int64_t)set * k + j], d, f);
    }
    delta[(int64_t)s * k + j] = d;
    phi[(int64_t)s * k + j] = f;
  }
}

}  // namespace gencd

using namespace gencd;

// ---------------------------------------------------------------------------
// the batch object

struct gencd_batch {
  gencd_problem* X = nullptr;  // X in FP32 (CSC, validation), y
  int64_t n = 0, k = 0, nnz = 0;
  int loss = 1;
  int S = 32, NC = 1;  // slots = 32 NC
  int nfolds = 0;
  cudaStream_t st = nullptr;
  gencd_params params{};
  int B = 1;

  uint8_t* fold = nullptr;
  std::vector<int64_t> set_rows;  // rows of training set f (f = nfolds: all rows)
  std::vector<double> lam_max;    // per training set
  double* inv_n = nullptr;        // per training set
  double* sq = nullptr;           // [(F+1)][k] column sums of squares
  double *bj = nullptr, *ib = nullptr;
  float *bj32 = nullptr, *ib32 = nullptr;

  // SpMM tiles
  int64_t ntiles = 0, W = 0;
  int spmm_grid = 0;
  uint32_t* tstart = nullptr;
  int32_t* tile_cc = nullptr;
  int32_t* nzcols = nullptr;
  int32_t* bnd = nullptr;

  // state
  double *w = nullptr, *z = nullptr;
  float *w32 = nullptr, *U = nullptr, *G = nullptr;
  int32_t* acc_j = nullptr;
  double* acc_d = nullptr;
  double* acc_phi = nullptr;
  int64_t* part_lo = nullptr;
  unsigned int* kkt_bits = nullptr;
  unsigned long long* ctr = nullptr;  // accepted non-zeros, updates
  double* obj_acc = nullptr;
  int32_t* obj_list = nullptr;
  double* tmp_k = nullptr;  // k doubles (w in/out)

  // per-slot parameters (device) and their host copy
  int32_t* d_set = nullptr;
  int32_t* d_group = nullptr;
  double *d_lam = nullptr, *d_invn = nullptr;
  float *d_lam32 = nullptr, *d_invn32 = nullptr;
  std::vector<int32_t> h_set, h_group;
  std::vector<double> h_lam;

  // schedule of the step, chosen by the autotuner (or set): the X^T U pass
  // as lanes over slots (1, k_b_spmm; S a multiple of 32) or lanes over
  // entries with 8 slots per lane (0, k_b_spmm_runs8), and the update per
  // (partition, slot) (0) or grouped by column (1); tuned_ms: mean ms of the
  // candidates (X^T U: kinds 0, 1; a whole step: update kinds 0, 1), -1 if
  // not timed
  int spmm_kind = 0, update_kind = 0;
  bool spmm_forced = false, update_forced = false, update_tuned = false;
  double tuned_ms[4] = {-1.0, -1.0, -1.0, -1.0};

  // captured steps
  bool dense_refresh = false;  // refresh u over all rows after each step
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0, graph_B = 0;
  int64_t steps = 0;  // batched steps enqueued
};

namespace gencd {

static SlotArgs slot_args(const gencd_batch* b) {
  return SlotArgs{b->d_set, b->d_group, b->d_lam, b->d_lam32, b->d_invn, b->d_invn32};
}

static int upload_slots(gencd_batch* b) {
  const int S = b->S;
  std::vector<float> l32(S), i32(S);
  std::vector<double> inv(S);
  for (int s = 0; s < S; ++s) {
    const int set = b->h_set[s];
    inv[s] = set >= 0 && b->set_rows[set] > 0 ? 1.0 / (double)b->set_rows[set] : 0.0;
    l32[s] = (float)b->h_lam[s];
    i32[s] = (float)inv[s];
  }
  // pageable sources: each copy has read its source when the call returns
  GENCD_CUDA_TRY(cudaMemcpyAsync(b->d_set, b->h_set.data(), 4 * S, cudaMemcpyHostToDevice, b->st));
  GENCD_CUDA_TRY(cudaMemcpyAsync(b->d_group, b->h_group.data(), 4 * S, cudaMemcpyHostToDevice, b->st));
  GENCD_CUDA_TRY(cudaMemcpyAsync(b->d_lam, b->h_lam.data(), 8 * S, cudaMemcpyHostToDevice, b->st));
  GENCD_CUDA_TRY(cudaMemcpyAsync(b->d_invn, inv.data(), 8 * S, cudaMemcpyHostToDevice, b->st));
  GENCD_CUDA_TRY(cudaMemcpyAsync(b->d_lam32, l32.data(), 4 * S, cudaMemcpyHostToDevice, b->st));
  GENCD_CUDA_TRY(cudaMemcpyAsync(b->d_invn32, i32.data(), 4 * S, cudaMemcpyHostToDevice, b->st));
  return GENCD_OK;
}

template <int NC>
static int launch_spmm_nc(gencd_batch* b, const float* U, float* G) {
  constexpr int GRP = NC <= 2 ? 8 : 4;
  k_b_spmm<NC, GRP><<<b->spmm_grid, kSpmmThreads, 0, b->st>>>(b->X->row_idx, (const float*)b->X->val, b->tstart,
                                                              b->tile_cc, b->nzcols, U, G, b->ntiles, b->W);
  return GENCD_OK;
}

// kind 1: lanes over slots, NC = S / 32 slot chunks of lanes; kind 0: lanes
// over entries and 8 slots per lane, one launch row per 8-slot chunk (G
// zeroed first)
static int launch_spmm(gencd_batch* b, int kind, const float* U, float* G) {
  const int NC = b->NC;
  if (kind == 0 || NC == 0) {
    GENCD_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(float) * (size_t)b->k * b->S, b->st));
    const int64_t t256 = (b->nnz + 255) / 256;
    if (t256 == 0) return GENCD_OK;
    const dim3 grid(grid_for(t256 * 32, kThreads, b->X->num_sms * 2), b->S / 8);
    k_b_spmm_runs8<<<grid, kThreads, 0, b->st>>>(b->X->row_idx, (const float*)b->X->val,
                                                  reinterpret_cast<const uint8_t*>(b->tstart), b->tile_cc, b->nzcols,
                                                  U, b->S, G, b->nnz, t256);
    return GENCD_OK;
  }
  switch (NC) {
    case 1: return launch_spmm_nc<1>(b, U, G);
    case 2: return launch_spmm_nc<2>(b, U, G);
    case 3: return launch_spmm_nc<3>(b, U, G);
    case 4: return launch_spmm_nc<4>(b, U, G);
    case 5: return launch_spmm_nc<5>(b, U, G);
    case 6: return launch_spmm_nc<6>(b, U, G);
    case 7: return launch_spmm_nc<7>(b, U, G);
    case 8: return launch_spmm_nc<8>(b, U, G);
  }
  return bfail(GENCD_EINVAL, "slot count out of range");
}

template <int NC>
static int spmm_occupancy(int* blocks) {
  constexpr int GRP = NC <= 2 ? 8 : 4;
  GENCD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_b_spmm<NC, GRP>, kSpmmThreads, 0));
  return GENCD_OK;
}

static int spmm_blocks_per_sm(int NC, int* blocks) {
  if (NC == 0) {
    *blocks = 2;
    return GENCD_OK;
  }
  switch (NC) {
    case 1: return spmm_occupancy<1>(blocks);
    case 2: return spmm_occupancy<2>(blocks);
    case 3: return spmm_occupancy<3>(blocks);
    case 4: return spmm_occupancy<4>(blocks);
    case 5: return spmm_occupancy<5>(blocks);
    case 6: return spmm_occupancy<6>(blocks);
    case 7: return spmm_occupancy<7>(blocks);
    case 8: return spmm_occupancy<8>(blocks);
  }
  return bfail(GENCD_EINVAL, "slot count out of range");
}

static int accept_R(const gencd_batch* b) { return std::max(1, kAcceptThreads / b->S); }

// G = X^T U and the per-slot KKT maxima (MODE 0), or a whole step (MODE 1)
static int enqueue_propose(gencd_batch* b, bool accept) {
  const int g = b->X->num_sms * 8;
  // the lanes-over-entries pass zeroes all of G itself
  const int64_t nb = (b->NC == 0 || b->spmm_kind == 0) ? 0 : 2 * b->W;
  k_b_prep<<<grid_for(std::max<int64_t>(1, nb * b->S), kThreads, g), kThreads, 0, b->st>>>(b->bnd, nb, b->S, b->G,
                                                                                          b->kkt_bits);
  GENCD_TRY(launch_spmm(b, b->spmm_kind, b->U, b->G));
  const int R = accept_R(b);
  if (accept)
    k_b_accept<1><<<b->B, b->S * R, 0, b->st>>>(b->G, b->w32, b->w, b->bj32, b->ib32, b->bj, b->ib, b->k,
                                                 slot_args(b), b->part_lo, b->S, R, b->acc_j, b->acc_d,
                                                 b->acc_phi, b->kkt_bits);
  else
    k_b_accept<0><<<b->B, b->S * R, 0, b->st>>>(b->G, b->w32, b->w, b->bj32, b->ib32, b->bj, b->ib, b->k,
                                                 slot_args(b), b->part_lo, b->S, R, nullptr, nullptr, nullptr,
                                                 b->kkt_bits);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

static int launch_refresh_all(gencd_batch* b) {
  const int rows = std::max(1, 256 / b->S);
  const int g = grid_for(b->n, rows, b->X->num_sms * 16);
  k_b_refresh_all<<<g, dim3(b->S, rows), 0, b->st>>>(b->X->y, b->fold, b->nfolds, b->loss, b->d_set, b->z, b->n,
                                                     b->S, b->U);
  return GENCD_OK;
}

static int enqueue_step(gencd_batch* b) {
  GENCD_TRY(enqueue_propose(b, true));
  const int npairs = b->B * b->S;
  if (b->B > 1)
    k_b_merge<<<(npairs + kThreads - 1) / kThreads, kThreads, 0, b->st>>>(b->acc_j, b->acc_phi, b->B, b->S,
                                                                         b->d_group);
  const int g = grid_for((int64_t)npairs * 32, kThreads, b->X->num_sms * 8);
  if (b->update_kind == 1) {
    const int per = (b->S + 31) / 32;
    k_b_update_grouped<<<grid_for((int64_t)b->B * per * 32, kThreads, b->X->num_sms * 8), kThreads, 0, b->st>>>(
        b->acc_j, b->acc_d, b->B, b->S, b->X->col_ptr, b->X->row_idx, (const float*)b->X->val, b->w, b->w32, b->z,
        b->ctr);
  } else {
    k_b_update<<<g, kThreads, 0, b->st>>>(b->acc_j, b->acc_d, npairs, b->S, b->X->col_ptr, b->X->row_idx,
                                          (const float*)b->X->val, b->w, b->w32, b->z, b->ctr);
  }
  if (b->dense_refresh)
    GENCD_TRY(launch_refresh_all(b));
  else
    k_b_refresh<<<g, kThreads, 0, b->st>>>(b->acc_j, npairs, b->S, b->X->col_ptr, b->X->row_idx, b->X->y, b->fold,
                                           b->nfolds, b->loss, b->d_set, b->z, b->U);
  GENCD_CUDA_TRY(cudaGetLastError());
  b->steps += 1;
  return GENCD_OK;
}

static void drop_graph(gencd_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_iters = 0;
}

// `iters` steps as one CUDA graph (captured once per (iters, B)); streams that
// cannot be captured (the legacy default stream) launch the kernels directly
// Autotuner of the update: the first time at least 4 steps run, they run
// one by one with the update per (partition, slot) and grouped by column
// alternately, each timed with CUDA events; the faster form is kept.  Every
// step is a correct step either way.
static int tune_update(gencd_batch* b, int* done) {
  *done = 0;
  if (b->update_tuned || b->update_forced) return GENCD_OK;
  cudaEvent_t e[5];
  for (int i = 0; i < 5; ++i)
    if (cudaEventCreate(&e[i]) != cudaSuccess) {
      for (int q = 0; q < i; ++q) cudaEventDestroy(e[q]);
      return bfail(GENCD_ECUDA, "cudaEventCreate failed");
    }
  int rc = GENCD_OK;
  cudaEventRecord(e[0], b->st);
  for (int i = 0; i < 4 && rc == GENCD_OK; ++i) {
    b->update_kind = i & 1;
    rc = enqueue_step(b);
    cudaEventRecord(e[i + 1], b->st);
  }
  if (rc == GENCD_OK && cudaEventSynchronize(e[4]) != cudaSuccess) rc = bfail(GENCD_ECUDA, "tuning steps failed");
  float ms[4] = {0.f, 0.f, 0.f, 0.f};
  for (int i = 0; rc == GENCD_OK && i < 4; ++i) cudaEventElapsedTime(&ms[i], e[i], e[i + 1]);
  for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]);
  if (rc != GENCD_OK) return rc;
  b->tuned_ms[2] = 0.5 * (ms[0] + ms[2]);
  b->tuned_ms[3] = 0.5 * (ms[1] + ms[3]);
  b->update_kind = b->tuned_ms[3] < b->tuned_ms[2] ? 1 : 0;
  b->update_tuned = true;
  drop_graph(b);
  *done = 4;
  return GENCD_OK;
}

static int run_steps(gencd_batch* b, int iters) {
  if (iters <= 0) return GENCD_OK;
  if (iters >= 4) {
    int done = 0;
    GENCD_TRY(tune_update(b, &done));
    iters -= done;
    if (iters <= 0) return GENCD_OK;
  }
  if (b->st != nullptr && (b->graph_iters != iters || b->graph_B != b->B)) {
    drop_graph(b);
    cudaGraph_t gr = nullptr;
    GENCD_CUDA_TRY(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    int rc = GENCD_OK;
    const int64_t steps0 = b->steps;
    for (int i = 0; i < iters && rc == GENCD_OK; ++i) rc = enqueue_step(b);
    b->steps = steps0;
    const cudaError_t e = cudaStreamEndCapture(b->st, &gr);
    if (rc != GENCD_OK) {
      if (gr) cudaGraphDestroy(gr);
      return rc;
    }
    if (e != cudaSuccess) return bfail(GENCD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    const cudaError_t e2 = cudaGraphInstantiate(&b->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e2 != cudaSuccess) {
      b->graph = nullptr;
      return bfail(GENCD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
    }
    b->graph_iters = iters;
    b->graph_B = b->B;
  }
  if (b->graph) {
    GENCD_CUDA_TRY(cudaGraphLaunch(b->graph, b->st));
    b->steps += iters;
    return GENCD_OK;
  }
  for (int i = 0; i < iters; ++i) GENCD_TRY(enqueue_step(b));
  return GENCD_OK;
}

static int check_slot(const gencd_batch* b, int32_t slot) {
  if (!b) return bfail(GENCD_EINVAL, "batch handle is NULL");
  if (slot < 0 || slot >= b->S) return bfail(GENCD_EINVAL, "slot " + std::to_string(slot) + " out of range");
  return GENCD_OK;
}

static int set_of(const gencd_batch* b, int32_t held_out, int* set) {
  if (held_out < -1 || held_out >= b->nfolds)
    return bfail(GENCD_EINVAL, "held_out " + std::to_string(held_out) + " is not -1 or a fold");
  *set = held_out < 0 ? b->nfolds : held_out;
  return GENCD_OK;
}

// z_s = X w_s and u_s for slot s (w_s already in place)
static int slot_recompute(gencd_batch* b, int s) {
  const int g = b->X->num_sms * 8;
  k_b_zero_col<<<grid_for(b->n, kThreads, g), kThreads, 0, b->st>>>(b->z, b->n, b->S, s);
  k_b_scatter_z<<<grid_for(b->k * 32, kThreads, g), kThreads, 0, b->st>>>(
      b->X->col_ptr, b->X->row_idx, (const float*)b->X->val, b->w, b->k, b->S, s, b->z);
  k_b_fill_col<<<grid_for(b->n, kThreads, g), kThreads, 0, b->st>>>(b->X->y, b->fold, b->nfolds, b->h_set[s], b->loss,
                                                                    b->z, b->n, b->S, s, b->U);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

static int slot_set(gencd_batch* b, int s, int set, double lambda, const double* w_dev, int group = 1) {
  b->h_set[s] = set;
  b->h_lam[s] = lambda;
  b->h_group[s] = group;
  GENCD_TRY(upload_slots(b));
  k_b_set_w<<<grid_for(b->k, kThreads, b->X->num_sms * 8), kThreads, 0, b->st>>>(w_dev, b->k, b->S, s, b->w, b->w32);
  return slot_recompute(b, s);
}

static int slot_copy(gencd_batch* b, int dst, int src, int set, double lambda, int group = 1) {
  const int g = b->X->num_sms * 8;
  b->h_set[dst] = set;
  b->h_lam[dst] = lambda;
  b->h_group[dst] = group;
  GENCD_TRY(upload_slots(b));
  k_b_copy_col<double><<<grid_for(b->k, kThreads, g), kThreads, 0, b->st>>>(b->w, b->k, b->S, src, dst);
  k_b_copy_col<float><<<grid_for(b->k, kThreads, g), kThreads, 0, b->st>>>(b->w32, b->k, b->S, src, dst);
  k_b_copy_col<double><<<grid_for(b->n, kThreads, g), kThreads, 0, b->st>>>(b->z, b->n, b->S, src, dst);
  k_b_fill_col<<<grid_for(b->n, kThreads, g), kThreads, 0, b->st>>>(b->X->y, b->fold, b->nfolds, set, b->loss, b->z,
                                                                    b->n, b->S, dst, b->U);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

static int slot_clear(gencd_batch* b, int s) {
  b->h_set[s] = -1;
  b->h_lam[s] = 0.0;
  b->h_group[s] = 1;
  GENCD_TRY(upload_slots(b));
  k_b_fill_col<<<grid_for(b->n, kThreads, b->X->num_sms * 8), kThreads, 0, b->st>>>(
      b->X->y, b->fold, b->nfolds, -1, b->loss, b->z, b->n, b->S, s, b->U);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

// objectives of the listed slots (FP64), synchronising; gap (nullable): their
// duality gaps, which need the max |g_js| of the slots' current state (a
// propose pass over the current state must have run since the last step)
static int slot_objectives(gencd_batch* b, const std::vector<int32_t>& slots, std::vector<double>* obj,
                           std::vector<double>* gap = nullptr) {
  obj->assign(slots.size(), 0.0);
  if (gap) gap->assign(slots.size(), 0.0);
  std::vector<unsigned int> gbits;
  if (gap) {
    gbits.resize(b->S);
    GENCD_CUDA_TRY(cudaMemcpyAsync(gbits.data(), b->kkt_bits + b->S, 4 * b->S, cudaMemcpyDeviceToHost, b->st));
    GENCD_CUDA_TRY(cudaStreamSynchronize(b->st));
  }
  for (size_t q0 = 0; q0 < slots.size(); q0 += 32) {
    const int m = (int)std::min<size_t>(32, slots.size() - q0);
    std::vector<int32_t> lst(64);
    for (int q = 0; q < m; ++q) {
      lst[q] = slots[q0 + q];
      lst[32 + q] = b->h_set[slots[q0 + q]];
    }
    GENCD_CUDA_TRY(cudaMemcpyAsync(b->obj_list, lst.data(), 4 * 64, cudaMemcpyHostToDevice, b->st));
    GENCD_CUDA_TRY(cudaMemsetAsync(b->obj_acc, 0, sizeof(double) * 96, b->st));
    std::vector<double> scale(32, 0.0);
    if (gap) {  // s = lambda / max(lambda, max_j |g_j|): the dual point s u is feasible
      for (int q = 0; q < m; ++q) {
        const int s = slots[q0 + q];
        float gm;
        std::memcpy(&gm, &gbits[s], 4);
        const double lam = b->h_lam[s];
        scale[q] = (double)gm > lam ? lam / (double)gm : 1.0;
      }
      GENCD_CUDA_TRY(cudaMemcpyAsync(b->obj_acc + 96, scale.data(), sizeof(double) * 32, cudaMemcpyHostToDevice,
                                     b->st));
    }
    const int64_t work = std::max(b->n, b->k);
    const int grid = (int)std::min<int64_t>((work + 7) / 8, (int64_t)b->X->num_sms * 8);
    k_b_objective<<<grid, dim3(32, 8), 0, b->st>>>(b->X->y, b->z, b->fold, b->nfolds, b->loss, b->n, b->w, b->k, b->S,
                                                  b->obj_list, b->obj_list + 32, m, gap ? b->obj_acc + 96 : nullptr,
                                                  b->obj_acc);
    GENCD_CUDA_TRY(cudaGetLastError());
    double h[96];
    GENCD_CUDA_TRY(cudaMemcpyAsync(h, b->obj_acc, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, b->st));
    GENCD_CUDA_TRY(cudaStreamSynchronize(b->st));
    for (int q = 0; q < m; ++q) {
      const int s = slots[q0 + q], set = b->h_set[s];
      const double rows = (double)b->set_rows[set];  // an empty training set has no loss term
      const double P = (rows > 0.0 ? h[q] / rows : 0.0) + b->h_lam[s] * h[m + q];
      (*obj)[q0 + q] = P;
      if (gap) (*gap)[q0 + q] = P + (rows > 0.0 ? h[2 * m + q] / rows : 0.0);
    }
  }
  return GENCD_OK;
}

static int read_kkt(gencd_batch* b, std::vector<double>* kkt) {
  std::vector<unsigned int> bits(b->S);
  GENCD_CUDA_TRY(cudaMemcpyAsync(bits.data(), b->kkt_bits, 4 * b->S, cudaMemcpyDeviceToHost, b->st));
  GENCD_CUDA_TRY(cudaStreamSynchronize(b->st));
  kkt->resize(b->S);
  for (int s = 0; s < b->S; ++s) {
    float f;
    std::memcpy(&f, &bits[s], 4);
    (*kkt)[s] = (double)f;
  }
  return GENCD_OK;
}

static int set_partitions(gencd_batch* b) {
  int B = b->params.variant == GENCD_GREEDY ? 1 : b->params.blocks;
  if (B <= 0) B = 1024;
  if ((int64_t)B > b->k) B = (int)std::max<int64_t>(1, b->k);
  std::vector<int64_t> lo(B + 1);
  for (int q = 0; q <= B; ++q) lo[q] = b->k * q / B;
  cudaFree(b->part_lo);
  b->part_lo = nullptr;
  cudaFree(b->acc_j);
  b->acc_j = nullptr;
  cudaFree(b->acc_d);
  b->acc_d = nullptr;
  cudaFree(b->acc_phi);
  b->acc_phi = nullptr;
  GENCD_TRY(balloc(&b->part_lo, B + 1));
  GENCD_TRY(balloc(&b->acc_phi, (size_t)B * b->S));
  GENCD_TRY(balloc(&b->acc_j, (size_t)B * b->S));
  GENCD_TRY(balloc(&b->acc_d, (size_t)B * b->S));
  GENCD_CUDA_TRY(cudaMemcpyAsync(b->part_lo, lo.data(), 8 * (B + 1), cudaMemcpyHostToDevice, b->st));
  GENCD_CUDA_TRY(cudaStreamSynchronize(b->st));
  b->B = B;
  // dense refresh when the accepted columns (heavier than the mean column,
  // taken as 4x) touch at least n (row, slot) entries per slot
  b->dense_refresh = (double)B * 4.0 * (double)b->nnz / (double)std::max<int64_t>(1, b->k) >= (double)b->n;
  drop_graph(b);
  return GENCD_OK;
}

static int set_betas(gencd_batch* b) {
  const int64_t m = (int64_t)(b->nfolds + 1) * b->k;
  const double beta = b->loss == GENCD_LOSS_SQUARED ? 1.0 : 0.25;
  k_b_beta<<<grid_for(m, kThreads, b->X->num_sms * 8), kThreads, 0, b->st>>>(
      b->sq, m, b->k, b->inv_n, beta, b->params.beta_mode, b->bj, b->ib, b->bj32, b->ib32);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

static void free_batch(gencd_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  drop_graph(b);
  void* bufs[] = {b->fold, b->inv_n, b->sq, b->bj, b->ib, b->bj32, b->ib32, b->tstart, b->tile_cc, b->nzcols,
                  b->bnd, b->w, b->z, b->w32, b->U, b->G, b->acc_j, b->acc_d, b->acc_phi, b->part_lo, b->kkt_bits,
                  b->ctr, b->obj_acc, b->obj_list, b->tmp_k, b->d_set, b->d_group, b->d_lam, b->d_invn,
                  b->d_lam32, b->d_invn32};
  for (void* q : bufs) cudaFree(q);
  cudaGetLastError();
  if (b->X) gencd_destroy(b->X);
  delete b;
}

// Autotuner of the X^T U pass: with S a multiple of 32 both forms apply;
// each is timed over three launches on the current U and the faster kept.
static int tune_spmm(gencd_batch* b) {
  if (b->spmm_forced) return GENCD_OK;
  if (b->NC == 0) {
    b->spmm_kind = 0;
    return GENCD_OK;
  }
  cudaEvent_t e0, e1;
  GENCD_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return bfail(GENCD_ECUDA, "cudaEventCreate failed");
  }
  int rc = GENCD_OK;
  for (int kind = 0; kind < 2 && rc == GENCD_OK; ++kind) {
    b->spmm_kind = kind;
    rc = enqueue_propose(b, false);  // warm-up
    cudaEventRecord(e0, b->st);
    for (int r = 0; r < 3 && rc == GENCD_OK; ++r) rc = enqueue_propose(b, false);
    cudaEventRecord(e1, b->st);
    float ms = 0.f;
    if (rc == GENCD_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
      b->tuned_ms[kind] = ms / 3.0;
    else if (rc == GENCD_OK)
      rc = bfail(GENCD_ECUDA, "timing the X^T U pass failed");
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GENCD_OK) return rc;
  b->spmm_kind = b->tuned_ms[1] <= b->tuned_ms[0] ? 1 : 0;
  drop_graph(b);
  return GENCD_OK;
}

static int create_batch(gencd_batch* b, const uint8_t* fold, int32_t memory) {
  const int64_t n = b->n, k = b->k, nnz = b->nnz;
  const int F = b->nfolds, S = b->S;
  cudaStream_t st = b->st;
  const int g = b->X->num_sms * 8;
  // folds and training-set sizes
  GENCD_TRY(balloc(&b->fold, n > 0 ? n : 1));
  b->set_rows.assign(F + 1, n);
  if (F > 0) {
    GENCD_CUDA_TRY(cudaMemcpyAsync(b->fold, fold, n, memory == GENCD_DEVICE ? cudaMemcpyDeviceToDevice
                                                                             : cudaMemcpyHostToDevice, st));
    unsigned long long* cnt = nullptr;
    GENCD_TRY(balloc(&cnt, 33));
    std::vector<unsigned long long> h(33, 0ull);
    h[32] = ~0ull;
    int rc = GENCD_OK;
    if (cudaMemcpyAsync(cnt, h.data(), 8 * 33, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = GENCD_ECUDA;
    if (rc == GENCD_OK) {
      k_b_fold_counts<<<grid_for(n, kThreads, g), kThreads, 0, st>>>(b->fold, n, F, cnt, cnt + 32);
      if (cudaMemcpyAsync(h.data(), cnt, 8 * 33, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        rc = bfail(GENCD_ECUDA, "fold counts failed");
    }
    cudaFree(cnt);
    if (rc != GENCD_OK) return rc;
    if (h[32] != ~0ull)
      return bfail(GENCD_EINVAL, "fold[" + std::to_string(h[32]) + "] is not below nfolds");
    for (int f = 0; f < F; ++f) b->set_rows[f] = n - (int64_t)h[f];
  } else {
    GENCD_CUDA_TRY(cudaMemsetAsync(b->fold, 0, n > 0 ? n : 1, st));
  }
  std::vector<double> inv(F + 1);
  for (int f = 0; f <= F; ++f) inv[f] = b->set_rows[f] > 0 ? 1.0 / (double)b->set_rows[f] : 0.0;
  GENCD_TRY(balloc(&b->inv_n, F + 1));
  GENCD_CUDA_TRY(cudaMemcpyAsync(b->inv_n, inv.data(), 8 * (F + 1), cudaMemcpyHostToDevice, st));

  // per training set: column sums of squares, beta_j, 1/beta_j
  const int64_t m = (int64_t)(F + 1) * k;
  GENCD_TRY(balloc(&b->sq, m));
  GENCD_TRY(balloc(&b->bj, m));
  GENCD_TRY(balloc(&b->ib, m));
  GENCD_TRY(balloc(&b->bj32, m));
  GENCD_TRY(balloc(&b->ib32, m));
  k_b_colsq<<<grid_for(k, 128, g * 2), 128, 0, st>>>(b->X->col_ptr, b->X->row_idx, (const float*)b->X->val, b->fold,
                                                      k, F, b->sq);
  GENCD_CUDA_TRY(cudaGetLastError());
  GENCD_TRY(set_betas(b));

  // SpMM tiles: start bits, compact non-empty columns, tile -> column
  b->ntiles = (nnz + 31) / 32;
  GENCD_TRY(balloc(&b->tstart, b->ntiles + 1));
  GENCD_TRY(balloc(&b->tile_cc, b->ntiles + 1));
  GENCD_TRY(balloc(&b->nzcols, k + 1));
  GENCD_CUDA_TRY(cudaMemsetAsync(b->tstart, 0, 4 * (b->ntiles + 1), st));
  {
    uint32_t *flag = nullptr, *pos = nullptr, *tmp = nullptr;
    int rc = balloc(&flag, k + 1);
    if (rc == GENCD_OK) rc = balloc(&pos, k + 1);
    if (rc == GENCD_OK) rc = balloc(&tmp, scan_tmp_words(k + 1));
    if (rc == GENCD_OK) {
      k_b_starts<<<grid_for(k, kThreads, g), kThreads, 0, st>>>(b->X->col_ptr, k, b->tstart, flag);
      if (cudaMemsetAsync(flag + k, 0, 4, st) != cudaSuccess) rc = GENCD_ECUDA;
    }
    if (rc == GENCD_OK) rc = exclusive_scan(b->X, flag, pos, k + 1, tmp);
    uint32_t nc = 0;
    if (rc == GENCD_OK) {
      k_b_compact<<<grid_for(k, kThreads, g), kThreads, 0, st>>>(flag, pos, k, b->nzcols);
      if (cudaMemcpyAsync(&nc, pos + k, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        rc = bfail(GENCD_ECUDA, "column compaction failed");
    }
    if (rc == GENCD_OK && nc > 0)
      k_b_tile_cc<<<grid_for(nc, kThreads, g), kThreads, 0, st>>>(b->X->col_ptr, b->nzcols, nc, b->tile_cc);
    cudaFree(flag);
    cudaFree(pos);
    cudaFree(tmp);
    if (rc != GENCD_OK) return rc;
  }
  int per_sm = 1;
  GENCD_TRY(spmm_blocks_per_sm(b->NC, &per_sm));
  b->spmm_grid = std::max(1, per_sm) * b->X->num_sms;
  b->W = std::min<int64_t>((int64_t)b->spmm_grid * (kSpmmThreads / 32), std::max<int64_t>(1, b->ntiles));
  b->spmm_grid = (int)((b->W + kSpmmThreads / 32 - 1) / (kSpmmThreads / 32));
  GENCD_TRY(balloc(&b->bnd, 2 * b->W));
  if (b->ntiles > 0) {
    k_b_bounds<<<grid_for(b->W, kThreads, g), kThreads, 0, st>>>(b->tile_cc, b->tstart, b->nzcols, b->ntiles, b->W,
                                                                  b->bnd);
  } else {
    GENCD_CUDA_TRY(cudaMemsetAsync(b->bnd, 0xff, 8 * b->W, st));
  }
  GENCD_CUDA_TRY(cudaGetLastError());

  // state
  GENCD_TRY(balloc(&b->w, (size_t)k * S));
  GENCD_TRY(balloc(&b->w32, (size_t)k * S));
  GENCD_TRY(balloc(&b->G, (size_t)k * S));
  GENCD_TRY(balloc(&b->z, (size_t)n * S));
  GENCD_TRY(balloc(&b->U, (size_t)n * S));
  GENCD_CUDA_TRY(cudaMemsetAsync(b->w, 0, 8 * (size_t)k * S, st));
  GENCD_CUDA_TRY(cudaMemsetAsync(b->w32, 0, 4 * (size_t)k * S, st));
  GENCD_CUDA_TRY(cudaMemsetAsync(b->G, 0, 4 * (size_t)k * S, st));
  GENCD_CUDA_TRY(cudaMemsetAsync(b->z, 0, 8 * (size_t)n * S, st));
  GENCD_CUDA_TRY(cudaMemsetAsync(b->U, 0, 4 * (size_t)n * S, st));
  GENCD_TRY(balloc(&b->kkt_bits, 2 * S));  // KKT and max |g| per slot
  GENCD_TRY(balloc(&b->ctr, 2));
  GENCD_CUDA_TRY(cudaMemsetAsync(b->ctr, 0, 16, st));
  GENCD_TRY(balloc(&b->obj_acc, 128));
  GENCD_TRY(balloc(&b->obj_list, 64));
  GENCD_TRY(balloc(&b->tmp_k, k));
  GENCD_TRY(balloc(&b->d_set, S));
  GENCD_TRY(balloc(&b->d_group, S));
  GENCD_TRY(balloc(&b->d_lam, S));
  GENCD_TRY(balloc(&b->d_invn, S));
  GENCD_TRY(balloc(&b->d_lam32, S));
  GENCD_TRY(balloc(&b->d_invn32, S));
  b->h_set.assign(S, -1);
  b->h_group.assign(S, 1);
  b->h_lam.assign(S, 0.0);
  GENCD_TRY(upload_slots(b));
  gencd_default_params(&b->params);
  GENCD_TRY(set_partitions(b));

  // lambda_max of every training set: max_j |X_j^T u(z = 0)| / n_f
  b->lam_max.assign(F + 1, 0.0);
  if (b->ntiles > 0) {
    float *U0 = nullptr, *G0 = nullptr;
    unsigned int* bits = nullptr;
    int rc = balloc(&U0, (size_t)n * 32);
    if (rc == GENCD_OK) rc = balloc(&G0, (size_t)k * 32);
    if (rc == GENCD_OK) rc = balloc(&bits, 32);
    std::vector<unsigned int> hb(32, 0u);
    if (rc == GENCD_OK) {
      k_b_u0<<<grid_for(n * 32, kThreads, g), kThreads, 0, st>>>(b->X->y, b->fold, n, F, b->loss, U0);
      cudaMemsetAsync(G0, 0, 4 * (size_t)k * 32, st);
      cudaMemsetAsync(bits, 0, 4 * 32, st);
      k_b_prep<<<grid_for(2 * b->W * 32, kThreads, g), kThreads, 0, st>>>(b->bnd, 2 * b->W, 32, G0, nullptr);
      rc = launch_spmm_nc<1>(b, U0, G0);  // 32 columns of U0: the training sets
    }
    if (rc == GENCD_OK) {
      k_b_absmax<<<grid_for(k * 32, kThreads, g), kThreads, 0, st>>>(G0, k, F + 1, bits);
      if (cudaMemcpyAsync(hb.data(), bits, 4 * 32, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        rc = bfail(GENCD_ECUDA, std::string("lambda_max: ") + cudaGetErrorString(cudaGetLastError()));
    }
    cudaFree(U0);
    cudaFree(G0);
    cudaFree(bits);
    if (rc != GENCD_OK) return rc;
    for (int f = 0; f <= F; ++f) {
      float v;
      std::memcpy(&v, &hb[f], 4);
      b->lam_max[f] = (double)v * inv[f];
    }
  }
  GENCD_TRY(tune_spmm(b));
  GENCD_CUDA_TRY(cudaStreamSynchronize(st));
  return GENCD_OK;
}

}  // namespace gencd

extern "C" {

static int batch_create(gencd_batch** out, int64_t n, int64_t k, int64_t nnz, const int64_t* col_ptr,
                        const int32_t* row_idx, const void* val, int32_t val_dtype, const double* y, int32_t loss,
                        const uint8_t* fold, int32_t nfolds, int32_t slots, int32_t memory, void* stream);

int gencd_batch_create(gencd_batch** out, int64_t n, int64_t k, int64_t nnz, const int64_t* col_ptr,
                       const int32_t* row_idx, const void* val, int32_t val_dtype, const double* y, int32_t loss,
                       const uint8_t* fold, int32_t nfolds, int32_t slots, int32_t memory, void* stream) {
  try {  // no exception crosses the C ABI
    return batch_create(out, n, k, nnz, col_ptr, row_idx, val, val_dtype, y, loss, fold, nfolds, slots, memory,
                        stream);
  } catch (const std::exception& e) {
    return bfail(GENCD_ENOMEM, std::string("host allocation failed: ") + e.what());
  }
}

static int batch_create(gencd_batch** out, int64_t n, int64_t k, int64_t nnz, const int64_t* col_ptr,
                        const int32_t* row_idx, const void* val, int32_t val_dtype, const double* y, int32_t loss,
                        const uint8_t* fold, int32_t nfolds, int32_t slots, int32_t memory, void* stream) {
  if (!out) return bfail(GENCD_EINVAL, "out is NULL");
  *out = nullptr;
  if (nfolds < 0 || nfolds > kBatchMaxFolds) return bfail(GENCD_EINVAL, "nfolds must be in [0, 31]");
  if (nfolds > 0 && !fold) return bfail(GENCD_EINVAL, "fold is NULL with nfolds > 0");
  if (slots < 1 || slots > kBatchMaxSlots) return bfail(GENCD_EINVAL, "slots must be in [1, 256]");
  gencd_batch* b = new (std::nothrow) gencd_batch();
  if (!b) return bfail(GENCD_ENOMEM, "host allocation failed");
  int rc = gencd_create(&b->X, n, k, nnz, col_ptr, row_idx, val, val_dtype, y, loss, GENCD_F32, memory, stream);
  if (rc != GENCD_OK) {
    delete b;
    return rc;
  }
  b->n = n;
  b->k = k;
  b->nnz = nnz;
  b->loss = loss;
  b->nfolds = nfolds;
  if (slots <= 16) {  // one or two 32-byte segments of U per entry
    b->NC = 0;
    b->S = slots <= 8 ? 8 : 16;
  } else {
    b->NC = (slots + 31) / 32;
    b->S = 32 * b->NC;
  }
  b->st = (cudaStream_t)stream;
  rc = create_batch(b, fold, memory);
  if (rc != GENCD_OK) {
    std::string keep = last_error();
    free_batch(b);
    set_error(keep);
    return rc;
  }
  *out = b;
  return GENCD_OK;
}

void gencd_batch_destroy(gencd_batch* b) { free_batch(b); }

int gencd_batch_schedule(gencd_batch* b, int32_t* spmm_kind, int32_t* update_kind, double* ms, int32_t nms) {
  if (!b) return bfail(GENCD_EINVAL, "batch handle is NULL");
  if (nms < 0 || (nms > 0 && !ms)) return bfail(GENCD_EINVAL, "ms must hold nms >= 0 values");
  if (spmm_kind) *spmm_kind = b->spmm_kind;
  if (update_kind) *update_kind = b->update_tuned || b->update_forced ? b->update_kind : -1;
  for (int32_t i = 0; i < nms; ++i) ms[i] = i < 4 ? b->tuned_ms[i] : -1.0;
  return GENCD_OK;
}

int gencd_batch_set_schedule(gencd_batch* b, int32_t spmm_kind, int32_t update_kind) {
  if (!b) return bfail(GENCD_EINVAL, "batch handle is NULL");
  if (spmm_kind < -1 || spmm_kind > 1 || update_kind < -1 || update_kind > 1)
    return bfail(GENCD_EINVAL, "schedule kinds are -1 (autotune), 0 or 1");
  if (spmm_kind == 1 && b->NC == 0) return bfail(GENCD_EINVAL, "lanes over slots need a multiple of 32 slots");
  b->spmm_forced = spmm_kind >= 0;
  if (spmm_kind >= 0) {
    b->spmm_kind = spmm_kind;
  } else {
    GENCD_TRY(tune_spmm(b));
  }
  b->update_forced = update_kind >= 0;
  if (update_kind >= 0) b->update_kind = update_kind;
  else b->update_tuned = false;
  drop_graph(b);
  return GENCD_OK;
}

int gencd_batch_slots(gencd_batch* b, int32_t* slots) {
  if (!b || !slots) return bfail(GENCD_EINVAL, "NULL argument");
  *slots = b->S;
  return GENCD_OK;
}

int gencd_batch_lambda_max(gencd_batch* b, int32_t held_out, double* lambda_max) {
  if (!b || !lambda_max) return bfail(GENCD_EINVAL, "NULL argument");
  int set;
  GENCD_TRY(set_of(b, held_out, &set));
  *lambda_max = b->lam_max[set];
  return GENCD_OK;
}

int gencd_batch_set_params(gencd_batch* b, const gencd_params* a) {
  if (!b || !a) return bfail(GENCD_EINVAL, "NULL argument");
  if (a->variant != GENCD_THREAD_GREEDY && a->variant != GENCD_GREEDY)
    return bfail(GENCD_EINVAL, "the batch runs Thread-Greedy or Greedy");
  if (a->blocks < 0 || a->max_iter < 0 || !(a->tol_kkt >= 0.0) || !(a->tol_gap >= 0.0) || a->check_every < 1 ||
      (a->beta_mode != 0 && a->beta_mode != 1))
    return bfail(GENCD_EINVAL, "parameter out of range");
  const bool betas = a->beta_mode != b->params.beta_mode;
  b->params = *a;
  GENCD_TRY(set_partitions(b));
  if (betas) GENCD_TRY(set_betas(b));
  return GENCD_OK;
}

int gencd_batch_set_slot(gencd_batch* b, int32_t slot, int32_t held_out, double lambda, const double* w,
                         int32_t memory) {
  GENCD_TRY(check_slot(b, slot));
  int set;
  GENCD_TRY(set_of(b, held_out, &set));
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return bfail(GENCD_EINVAL, "lambda must be finite and >= 0");
  const double* src = nullptr;
  if (w) {
    if (memory == GENCD_HOST) {
      for (int64_t j = 0; j < b->k; ++j)
        if (!std::isfinite(w[j])) return bfail(GENCD_EINVAL, "w[" + std::to_string(j) + "] is not finite");
      GENCD_CUDA_TRY(cudaMemcpyAsync(b->tmp_k, w, 8 * b->k, cudaMemcpyHostToDevice, b->st));
      src = b->tmp_k;
    } else {
      src = w;
    }
  }
  GENCD_TRY(slot_set(b, slot, set, lambda, src));
  GENCD_CUDA_TRY(cudaStreamSynchronize(b->st));
  return GENCD_OK;
}

int gencd_batch_copy_slot(gencd_batch* b, int32_t dst, int32_t src, int32_t held_out, double lambda) {
  GENCD_TRY(check_slot(b, dst));
  GENCD_TRY(check_slot(b, src));
  if (b->h_set[src] < 0) return bfail(GENCD_ESTATE, "source slot is not active");
  int set;
  GENCD_TRY(set_of(b, held_out, &set));
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return bfail(GENCD_EINVAL, "lambda must be finite and >= 0");
  if (dst == src) {
    b->h_set[dst] = set;
    b->h_lam[dst] = lambda;
    GENCD_TRY(upload_slots(b));
    k_b_fill_col<<<grid_for(b->n, kThreads, b->X->num_sms * 8), kThreads, 0, b->st>>>(
        b->X->y, b->fold, b->nfolds, set, b->loss, b->z, b->n, b->S, dst, b->U);
  } else {
    GENCD_TRY(slot_copy(b, dst, src, set, lambda));
  }
  GENCD_CUDA_TRY(cudaStreamSynchronize(b->st));
  return GENCD_OK;
}

int gencd_batch_clear_slot(gencd_batch* b, int32_t slot) {
  GENCD_TRY(check_slot(b, slot));
  GENCD_TRY(slot_clear(b, slot));
  GENCD_CUDA_TRY(cudaStreamSynchronize(b->st));
  return GENCD_OK;
}

int gencd_batch_get_w(gencd_batch* b, int32_t slot, double* w, int64_t k, int32_t memory) {
  GENCD_TRY(check_slot(b, slot));
  if (!w || k != b->k) return bfail(GENCD_EINVAL, "w must hold exactly k doubles");
  k_b_get_w<<<grid_for(b->k, kThreads, b->X->num_sms * 8), kThreads, 0, b->st>>>(b->w, b->k, b->S, slot, b->tmp_k);
  GENCD_CUDA_TRY(cudaMemcpyAsync(w, b->tmp_k, 8 * b->k,
                                 memory == GENCD_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->st));
  GENCD_CUDA_TRY(cudaStreamSynchronize(b->st));
  return GENCD_OK;
}

int gencd_batch_iterate(gencd_batch* b, int64_t iters, int32_t sync) {
  if (!b) return bfail(GENCD_EINVAL, "batch handle is NULL");
  if (iters < 0) return bfail(GENCD_EINVAL, "iters must be >= 0");
  for (int64_t i = 0; i < iters; ++i) GENCD_TRY(enqueue_step(b));
  if (sync) GENCD_CUDA_TRY(cudaStreamSynchronize(b->st));
  return GENCD_OK;
}

int gencd_batch_objective(gencd_batch* b, double* objective, double* kkt) {
  if (!b) return bfail(GENCD_EINVAL, "batch handle is NULL");
  GENCD_TRY(enqueue_propose(b, false));
  std::vector<double> kv;
  GENCD_TRY(read_kkt(b, &kv));
  std::vector<int32_t> act;
  for (int s = 0; s < b->S; ++s)
    if (b->h_set[s] >= 0) act.push_back(s);
  std::vector<double> ob;
  GENCD_TRY(slot_objectives(b, act, &ob));
  const double nan = std::nan("");
  for (int s = 0; s < b->S; ++s) {
    if (objective) objective[s] = nan;
    if (kkt) kkt[s] = b->h_set[s] >= 0 ? kv[s] : nan;
  }
  if (objective)
    for (size_t q = 0; q < act.size(); ++q) objective[act[q]] = ob[q];
  return GENCD_OK;
}

int gencd_batch_propose(gencd_batch* b, double* delta, double* phi, int32_t memory) {
  if (!b || !delta || !phi) return bfail(GENCD_EINVAL, "NULL argument");
  GENCD_TRY(enqueue_propose(b, false));
  const size_t m = (size_t)b->S * b->k;
  double *dd = nullptr, *df = nullptr;
  int rc = balloc(&dd, m);
  if (rc == GENCD_OK) rc = balloc(&df, m);
  if (rc == GENCD_OK) {
    k_b_propose<<<grid_for((int64_t)m, kThreads, b->X->num_sms * 8), kThreads, 0, b->st>>>(
        b->G, b->w, b->bj, b->ib, b->k, slot_args(b), b->S, dd, df);
    const cudaMemcpyKind kind = memory == GENCD_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (cudaMemcpyAsync(delta, dd, 8 * m, kind, b->st) != cudaSuccess ||
        cudaMemcpyAsync(phi, df, 8 * m, kind, b->st) != cudaSuccess || cudaStreamSynchronize(b->st) != cudaSuccess)
      rc = bfail(GENCD_ECUDA, std::string("batch propose: ") + cudaGetErrorString(cudaGetLastError()));
  }
  cudaFree(dd);
  cudaFree(df);
  return rc;
}

static int batch_path(gencd_batch* b, const gencd_path* path, gencd_path_solve* solves, double* w_out,
                      gencd_result* out);

int gencd_batch_path(gencd_batch* b, const gencd_path* path, gencd_path_solve* solves, double* w_out,
                     gencd_result* out) {
  try {  // no exception crosses the C ABI
    return batch_path(b, path, solves, w_out, out);
  } catch (const std::exception& e) {
    return bfail(GENCD_ENOMEM, std::string("host allocation failed: ") + e.what());
  }
}

static int batch_path(gencd_batch* b, const gencd_path* path, gencd_path_solve* solves, double* w_out,
                      gencd_result* out) {
  if (!b || !path || !solves) return bfail(GENCD_EINVAL, "NULL argument");
  const int C = path->nchains, L = path->nlambda;
  if (C < 1 || L < 1 || !path->held_out || !path->lambda || !(path->handoff >= 0.0) || !(path->tol_rel >= 0.0))
    return bfail(GENCD_EINVAL, "malformed path");
  std::vector<int> cset(C);
  for (int c = 0; c < C; ++c) GENCD_TRY(set_of(b, path->held_out[c], &cset[c]));
  for (int64_t q = 0; q < (int64_t)C * L; ++q)
    if (!(path->lambda[q] >= 0.0) || !std::isfinite(path->lambda[q]))
      return bfail(GENCD_EINVAL, "lambda[" + std::to_string(q) + "] must be finite and >= 0");
  const auto t0 = std::chrono::steady_clock::now();
  auto secs = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
  const int S = b->S;
  const int m = std::max(1, b->params.check_every);
  const int stall_checks = std::max(1, (kStallIters + m - 1) / m);
  const int64_t max_iter = b->params.max_iter;
  const double tol = b->params.tol_kkt;
  // per chain: the last finished solve's w (warm starts from a retired solve);
  // per slot: the w its solve started from (restarts after a divergence)
  double *w_last = nullptr, *w_start = nullptr;
  GENCD_TRY(balloc(&w_last, (size_t)C * b->k));
  if (balloc(&w_start, (size_t)S * b->k) != GENCD_OK) {
    cudaFree(w_last);
    return GENCD_ENOMEM;
  }
  std::vector<int> next(C, 0), ready(C, 1), pred_slot(C, -1), slot_solve(S, -1), last_q(C, -1);
  // a chain's next solve starts at half the accept group its live solves
  // reached, unless one of them started before the chain's last solve that
  // did not converge (fails[c]; slot_epoch: the count at the slot's start):
  // after such a solve the chain starts again from G = 1
  std::vector<int> chain_group(C, 1), obj_wait(S, 0), stall(S, 0), fails(C, 0), slot_epoch(S, 0);
  std::vector<int64_t> slot_iters(S, 0);
  std::vector<double> best_v(S, HUGE_VAL), best_p(S, HUGE_VAL), p_start(S, HUGE_VAL);
  const int g_sm = b->X->num_sms * 8;
  for (int64_t q = 0; q < (int64_t)C * L; ++q) {
    std::memset(&solves[q], 0, sizeof(gencd_path_solve));
    solves[q].status = GENCD_NOT_CONVERGED;
    solves[q].slot = -1;
  }
  int rc = GENCD_OK;
  for (int s = 0; s < S && rc == GENCD_OK; ++s) rc = slot_clear(b, s);
  GENCD_CUDA_TRY(cudaMemsetAsync(b->ctr, 0, 16, b->st));
  const int64_t steps0 = b->steps;
  int done = 0, all_ok = 1;
  std::vector<double> kv;
  std::vector<int32_t> started;
  while (rc == GENCD_OK && done < C * L) {
    // start ready solves in free slots, chains in turn
    for (int c = 0, free_s = 0; c < C && rc == GENCD_OK; ++c) {
      if (!ready[c] || next[c] >= L) continue;
      while (free_s < S && slot_solve[free_s] >= 0) ++free_s;
      if (free_s >= S) break;
      const int t = next[c], q = c * L + t, s = free_s;
      const double lam = path->lambda[q];
      if (t == 0 || !path->warm)
        rc = slot_set(b, s, cset[c], lam, nullptr, chain_group[c]);
      else if (pred_slot[c] >= 0)
        rc = slot_copy(b, s, pred_slot[c], cset[c], lam, chain_group[c]);
      else
        rc = slot_set(b, s, cset[c], lam, w_last + (size_t)c * b->k, chain_group[c]);
      if (rc == GENCD_OK)
        k_b_get_w<<<grid_for(b->k, kThreads, g_sm), kThreads, 0, b->st>>>(b->w, b->k, S, s,
                                                                           w_start + (size_t)s * b->k);
      slot_solve[s] = q;
      slot_epoch[s] = fails[c];
      slot_iters[s] = 0;
      obj_wait[s] = 0;
      stall[s] = 0;
      best_v[s] = HUGE_VAL;
      best_p[s] = HUGE_VAL;
      solves[q].slot = s;
      solves[q].t_start = secs();
      next[c] += 1;
      ready[c] = 0;
      started.push_back(s);
    }
    if (rc != GENCD_OK) break;
    if (!started.empty()) {  // the objective each new solve starts from (the backoff's reference)
      std::vector<double> p0;
      rc = slot_objectives(b, started, &p0);
      for (size_t r = 0; r < started.size() && rc == GENCD_OK; ++r) p_start[started[r]] = p0[r];
      started.clear();
      if (rc != GENCD_OK) break;
    }
    rc = run_steps(b, m);
    if (rc == GENCD_OK) rc = read_kkt(b, &kv);
    if (rc != GENCD_OK) break;
    // Accept backoff (Thread-Greedy has no convergence guarantee), the rules
    // of gencd_solve: an objective (evaluated every kObjChecks checks) that is
    // not finite or above the solve's start value, or a KKT value that is not
    // finite, restarts the solve from its start with 4x the accept group;
    // checks covering kStallIters iterations in a row that set neither a KKT
    // value kStallGain below the lowest since the (re)start nor (at an
    // objective evaluation) a new lowest objective double the group, while
    // the KKT value is above kStallKkt * lambda, and the solve goes on.
    // G = B is Greedy.
    std::vector<int32_t> retire, restart, watch;
    bool regroup = false;
    for (int s = 0; s < S; ++s) {
      const int q = slot_solve[s];
      if (q < 0) continue;
      const int c = q / L;
      slot_iters[s] += m;
      const double v = kv[s];
      const double lam_q = path->lambda[q];
      const double tol_q = path->tol_rel > 0.0 ? path->tol_rel * lam_q : tol;
      const bool rel = path->tol_rel > 0.0 || b->params.tol_gap > 0.0;  // handoff relative to lambda
      const double hand_q = rel ? path->handoff * lam_q : path->handoff;
      solves[q].iters = slot_iters[s];
      solves[q].kkt = v;
      if (v <= tol_q) {
        solves[q].status = GENCD_OK;
        retire.push_back(s);
      } else if (!std::isfinite(v)) {
        if (b->h_group[s] < b->B && slot_iters[s] < max_iter) {
          b->h_group[s] = std::min(b->B, 4 * b->h_group[s]);
          restart.push_back(s);
        } else {
          solves[q].status = GENCD_EDIVERGED;
          retire.push_back(s);
        }
      } else if (slot_iters[s] >= max_iter) {
        solves[q].status = GENCD_NOT_CONVERGED;
        retire.push_back(s);
      } else {
        if (v < best_v[s] * (1.0 - kStallGain)) {
          best_v[s] = v;
          stall[s] = 0;
        } else {
          stall[s] += 1;
        }
        if (++obj_wait[s] >= kObjChecks) watch.push_back(s);
        if (hand_q > 0.0 && v <= hand_q && next[c] == (q % L) + 1 && !ready[c]) {
          ready[c] = 1;  // the successor may start from this iterate
          pred_slot[c] = s;
        }
      }
    }
    if (!watch.empty()) {
      // with tol_gap, the watched slots' duality gaps: a propose pass over the
      // current state gives max_j |g_j| (the step's own pass saw its start)
      const bool gaps = b->params.tol_gap > 0.0;
      std::vector<double> pw, pg;
      if (gaps) rc = enqueue_propose(b, false);
      if (rc == GENCD_OK) rc = slot_objectives(b, watch, &pw, gaps ? &pg : nullptr);
      for (size_t r = 0; r < watch.size() && rc == GENCD_OK; ++r) {
        const int s = watch[r];
        obj_wait[s] = 0;
        const double P = pw[r];
        if (gaps && pg[r] <= b->params.tol_gap * std::fabs(P)) {  // certified within tol_gap of its optimum
          solves[slot_solve[s]].status = GENCD_OK;
          retire.push_back(s);
          continue;
        }
        if (!std::isfinite(P) || !(P <= p_start[s] * (1.0 + 1e-6) + 1e-300)) {  // above its start: restart
          if (b->h_group[s] < b->B && slot_iters[s] < max_iter) {
            b->h_group[s] = std::min(b->B, 4 * b->h_group[s]);
            restart.push_back(s);
          } else if (!std::isfinite(P)) {
            solves[slot_solve[s]].status = GENCD_EDIVERGED;
            retire.push_back(s);
          }
          continue;
        }
        if (P < best_p[s] * (1.0 - kObjGain)) {  // P >= 0 for both losses
          best_p[s] = P;
          stall[s] = 0;
        } else if (stall[s] >= stall_checks) {  // neither value improved for kStallIters iterations
          if (b->h_group[s] < b->B && kv[s] >= kStallKkt * b->h_lam[s]) {
            b->h_group[s] = std::min(b->B, 2 * b->h_group[s]);
            regroup = true;
          }
          stall[s] = 0;
        }
      }
    }
    for (size_t r = 0; r < restart.size() && rc == GENCD_OK; ++r) {
      const int s = restart[r];
      rc = slot_set(b, s, b->h_set[s], b->h_lam[s], w_start + (size_t)s * b->k, b->h_group[s]);
      best_v[s] = HUGE_VAL;
      best_p[s] = HUGE_VAL;
      obj_wait[s] = 0;
      stall[s] = 0;
    }
    for (int s = 0; s < S; ++s) {
      if (slot_solve[s] < 0) continue;
      const int c = slot_solve[s] / L;
      if (slot_epoch[s] == fails[c]) chain_group[c] = std::max(1, b->h_group[s] / 2);
    }
    if (regroup) rc = upload_slots(b);
    if (rc != GENCD_OK || retire.empty()) continue;
    std::vector<double> ob;
    rc = slot_objectives(b, retire, &ob);
    for (size_t r = 0; r < retire.size() && rc == GENCD_OK; ++r) {
      const int s = retire[r], q = slot_solve[s], c = q / L;
      solves[q].objective = ob[r];
      solves[q].t_end = secs();
      solves[q].group = b->h_group[s];
      if (solves[q].status != GENCD_OK) {
        all_ok = 0;
        fails[c] += 1;
        chain_group[c] = 1;
      }
      // the chain's latest finished lambda is the warm start of the solves still to come
      double* dst = q > last_q[c] ? w_last + (size_t)c * b->k : b->tmp_k;
      if (q > last_q[c]) last_q[c] = q;
      k_b_get_w<<<grid_for(b->k, kThreads, b->X->num_sms * 8), kThreads, 0, b->st>>>(b->w, b->k, S, s, dst);
      if (w_out && (cudaMemcpyAsync(w_out + (size_t)q * b->k, dst, 8 * b->k, cudaMemcpyDeviceToHost, b->st) !=
                        cudaSuccess ||
                    cudaStreamSynchronize(b->st) != cudaSuccess))
        rc = bfail(GENCD_ECUDA, "copy of w failed");
      if (rc == GENCD_OK) rc = slot_clear(b, s);
      slot_solve[s] = -1;
      if (pred_slot[c] == s) pred_slot[c] = -1;
      if (next[c] == (q % L) + 1) ready[c] = 1;  // the successor starts from the final w
      done += 1;
    }
    if (rc == GENCD_OK && cudaStreamSynchronize(b->st) != cudaSuccess)
      rc = bfail(GENCD_ECUDA, std::string("path: ") + cudaGetErrorString(cudaGetLastError()));
  }
  unsigned long long hc[2] = {0ull, 0ull};
  if (rc == GENCD_OK) {
    if (cudaMemcpyAsync(hc, b->ctr, 16, cudaMemcpyDeviceToHost, b->st) != cudaSuccess ||
        cudaStreamSynchronize(b->st) != cudaSuccess)
      rc = bfail(GENCD_ECUDA, "counters");
  }
  cudaFree(w_last);
  cudaFree(w_start);
  if (rc != GENCD_OK) return rc;
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->status = all_ok ? GENCD_OK : GENCD_NOT_CONVERGED;
    out->iters = b->steps - steps0;
    out->updates = (int64_t)hc[1];
    int64_t prop = 0;
    for (int64_t q = 0; q < (int64_t)C * L; ++q) prop += solves[q].iters;
    out->nnz_processed = prop * b->nnz + (int64_t)hc[0];
    out->seconds = secs();
  }
  return all_ok ? GENCD_OK : GENCD_NOT_CONVERGED;
}

}  // extern "C"
