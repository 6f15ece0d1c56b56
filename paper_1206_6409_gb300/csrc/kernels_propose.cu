// kernels_propose.cu -- the Propose and Accept steps of GenCD on sm_103a.
//
//  * k_propose_all: Algorithm 4's inner product g_j = <u, X_j> for every
//    column, streamed over the CSC arrays in nnz order.  Each warp owns a tile
//    of 32*ITEMS consecutive non-zeros, each lane ITEMS of them, loaded with
//    128-bit streaming loads; u is gathered through the read-only path.  A lane
//    sums its non-zeros column by column in registers (one FMA per non-zero);
//    a column that lies inside one lane is stored, a column cut by a lane or
//    tile boundary is added atomically into gacc (FP64).  Work per warp is
//    constant whatever the column lengths (1 ... 50,000 non-zeros).
//  * k_finalize: g_j = gacc_j / n, the Eq. 7 step, the Eq. 9 proxy and the
//    KKT violation per column; resets gacc for the next launch.
//  * k_accept: Thread-Greedy / Greedy accept (Table 2), one CTA per partition,
//    argmin of phi with ties to the lower column; accepted iff phi < 0.
//  * k_propose_list: Algorithm 4 over a selected list J (Shotgun, parity hook),
//    one warp per column with a shuffle reduction.
//  * k_objective_*: P(w) of Eq. 1 in FP64 with a fixed-order two-pass sum.
#include <float.h>

#include "device_math.cuh"
#include "gencd_internal.cuh"

namespace gencd {

// ---------------------------------------------------------------------------
// 128-bit streaming loads of ITEMS consecutive entries (16-byte aligned).
template <int ITEMS>
__device__ __forceinline__ void load_idx(const int32_t* __restrict__ p, int32_t (&r)[ITEMS]) {
#pragma unroll
  for (int q = 0; q < ITEMS / 4; ++q) {
    int4 v = __ldcs(reinterpret_cast<const int4*>(p) + q);
    r[4 * q + 0] = v.x;
    r[4 * q + 1] = v.y;
    r[4 * q + 2] = v.z;
    r[4 * q + 3] = v.w;
  }
}

template <int ITEMS>
__device__ __forceinline__ void load_val(const double* __restrict__ p, double (&v)[ITEMS]) {
#pragma unroll
  for (int q = 0; q < ITEMS / 2; ++q) {
    double2 x = __ldcs(reinterpret_cast<const double2*>(p) + q);
    v[2 * q + 0] = x.x;
    v[2 * q + 1] = x.y;
  }
}

template <int ITEMS>
__device__ __forceinline__ void load_val(const float* __restrict__ p, float (&v)[ITEMS]) {
#pragma unroll
  for (int q = 0; q < ITEMS / 4; ++q) {
    float4 x = __ldcs(reinterpret_cast<const float4*>(p) + q);
    v[4 * q + 0] = x.x;
    v[4 * q + 1] = x.y;
    v[4 * q + 2] = x.z;
    v[4 * q + 3] = x.w;
  }
}

template <typename G>
__device__ __forceinline__ void emit_partial(G* __restrict__ gacc, int32_t c, G s, bool whole) {
  if (whole)
    gacc[c] = s;  // the only writer of this column
  else
    atomicAdd(gacc + c, s);
}

// SQ: sum X_ij^2 instead of X_ij u_i (the column scales c_j, at setup).
// G: type of the sums in gacc (float in FP32 mode, so that no FP64 unit work
// or conversion is on this path; double otherwise).
template <typename V, typename U, int ITEMS, typename G, bool SQ = false>
__global__ void __launch_bounds__(kThreads)
    k_propose_all(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                  const V* __restrict__ val, const U* __restrict__ u,
                  const int32_t* __restrict__ tile_col, int64_t nnz, int64_t ntiles,
                  const int32_t* __restrict__ cmap, G* __restrict__ gacc) {
  constexpr int TILE = 32 * ITEMS;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = warp; t < ntiles; t += nwarps) {
    const int64_t a = t * TILE + (int64_t)lane * ITEMS;
    if (a >= nnz) continue;
    int32_t r[ITEMS];
    V v[ITEMS];
    load_idx<ITEMS>(row_idx + a, r);  // arrays are padded: always in bounds
    load_val<ITEMS>(val + a, v);
    const int64_t b = a + ITEMS < nnz ? a + ITEMS : nnz;
    const int nvalid = (int)(b - a);
    U uu[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (SQ)
        uu[i] = (U)v[i];
      else
        uu[i] = i < nvalid ? __ldg(u + r[i]) : U(0);
    }

    // column holding position a: the largest c in [tile_col[t], tile_col[t+1]]
    // with col_ptr[c] <= a (empty columns share their start with the next one)
    int32_t lo = __ldg(tile_col + t), hi = __ldg(tile_col + t + 1);
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (__ldg(col_ptr + mid) <= a)
        lo = mid;
      else
        hi = mid - 1;
    }
    int32_t c = lo;
    int64_t cend = __ldg(col_ptr + c + 1);
    bool whole = __ldg(col_ptr + c) >= a;
    V acc = V(0);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (i < nvalid) {
        const int64_t p = a + i;
        while (p >= cend) {  // column c ended before p (c + 1 <= k - 1 since p < nnz)
          emit_partial<G>(gacc, cmap ? cmap[c] : c, (G)acc, whole);
          ++c;
          cend = __ldg(col_ptr + c + 1);
          acc = V(0);
          whole = true;
        }
        acc = fma(v[i], (V)uu[i], acc);
      }
    }
    emit_partial<G>(gacc, cmap ? cmap[c] : c, (G)acc, whole && cend <= b);
  }
}


// Per-column part of Propose: Eq. 7 step, Eq. 9 proxy and KKT violation from
// g_j.  A column with w_j = 0 and |g_j| <= lambda does not move (delta = 0,
// phi = 0, KKT 0).  That test runs on the raw sum: |gacc_j| <= lambda n, both
// sides non-negative doubles, whose order is the order of their bit patterns,
// so the idle bulk of a sparse solution costs integer compares only.
__device__ __forceinline__ bool column_is_idle(double gacc, double wj, uint64_t lam_n_bits) {
  const uint64_t wb = (uint64_t)__double_as_longlong(wj) << 1;            // drop the sign
  const uint64_t gb = (uint64_t)__double_as_longlong(gacc) & 0x7fffffffffffffffull;
  return wb == 0 && gb <= lam_n_bits;
}


__device__ __forceinline__ bool cand_better(uint64_t ma, int32_t ja, uint64_t mb, int32_t jb) {
  return ma > mb || (ma == mb && ma != 0 && ja < jb);
}

// block reduction of the best candidate (mag, j, delta) over NT threads;
// valid in thread 0
template <int NT = kThreads>
__device__ __forceinline__ void block_best(uint64_t& m, int32_t& j, double& d) {
  __shared__ uint64_t s_m[NT / 32];
  __shared__ double s_d[NT / 32];
  __shared__ int32_t s_j[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t xm = __shfl_xor_sync(0xffffffffu, m, o);
    const int32_t xj = __shfl_xor_sync(0xffffffffu, j, o);
    const double xd = __shfl_xor_sync(0xffffffffu, d, o);
    if (cand_better(xm, xj, m, j)) {
      m = xm;
      j = xj;
      d = xd;
    }
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
    s_m[wid] = m;
    s_j[wid] = j;
    s_d[wid] = d;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 1; q < NT / 32; ++q)
      if (cand_better(s_m[q], s_j[q], m, j)) {
        m = s_m[q];
        j = s_j[q];
        d = s_d[q];
      }
}

// NaN-propagating max of non-negative doubles on their bit patterns
__device__ __forceinline__ void max_bits(uint64_t& acc, double v) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  acc = b > acc ? b : acc;
}

__device__ __forceinline__ void block_max_bits_to(double* out, uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t x = __shfl_xor_sync(0xffffffffu, v, o);
    v = x > v ? x : v;
  }
  if ((threadIdx.x & 31) == 0 && v) atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)v);
}

// partition of column j: the b with floor(b k / B) <= j < floor((b+1) k / B)
__device__ __forceinline__ int64_t partition_of(int64_t j, int64_t k, int64_t B) {
  return ((j + 1) * B - 1) / k;
}

// Eq. 7 step and Eq. 9 proxy of an active column from its raw sum
__device__ __forceinline__ void active_step(double ga, double inv_n, double wj, double lam, double bj, double ibj,
                                            double& g, double& d, double& phi) {
  g = ga * inv_n;
  eq7_step(g, wj, lam, bj, ibj, d, phi);
}

// A column with w_j = 0 whose raw sum satisfies |gacc_j| <= lambda n does not
// move; tested on bit patterns (both sides non-negative), no FP64 unit work.
__device__ __forceinline__ bool idle_raw(double ga, double wj, uint64_t lnb64, uint32_t) {
  return column_is_idle(ga, wj, lnb64);
}
__device__ __forceinline__ bool idle_raw(float ga, double wj, uint64_t, uint32_t lnb32) {
  const uint64_t wb = (uint64_t)__double_as_longlong(wj) << 1;
  return wb == 0 && ((uint32_t)__float_as_int(ga) & 0x7fffffffu) <= lnb32;
}

constexpr int kColsPerThread = 4;
constexpr int kRoundCols = kColsPerThread * kThreads;  // columns a CTA scans per round

// One round of the per-column pass: every thread loads 4 columns (loads in
// flight together), zeroes their sums, tests them with integer compares, and
// queues the active ones in shared memory; after a barrier the queue is
// processed packed (one active column per thread), so FP64 work is
// proportional to the number of active columns, not to the warps that hold
// one.  Returns the queue length; the queue holds (j, raw sum, w_j).
template <typename G>
__device__ __forceinline__ int scan_round(G* __restrict__ gacc, const double* __restrict__ w, int64_t base,
                                          int64_t hi, uint64_t lnb64, uint32_t lnb32, int* s_n, int64_t* s_j,
                                          double* s_g, double* s_w, double* delta, double* phi) {
  G ga[kColsPerThread];
  double wv[kColsPerThread];
#pragma unroll
  for (int q = 0; q < kColsPerThread; ++q) {
    const int64_t j = base + q * kThreads + threadIdx.x;
    ga[q] = j < hi ? gacc[j] : G(0);
    wv[q] = j < hi ? w[j] : 0.0;
  }
#pragma unroll
  for (int q = 0; q < kColsPerThread; ++q) {
    const int64_t j = base + q * kThreads + threadIdx.x;
    if (j >= hi) continue;
    gacc[j] = G(0);
    if (!idle_raw(ga[q], wv[q], lnb64, lnb32)) {
      const int slot = atomicAdd(s_n, 1);
      s_j[slot] = j;
      s_g[slot] = (double)ga[q];
      s_w[slot] = wv[q];
    } else if (delta) {
      delta[j] = 0.0;
      phi[j] = 0.0;
    }
  }
  __syncthreads();
  return *s_n;
}

// Per-column step, proxy and KKT for every column (the parity hook
// gencd_propose_all and the convergence checks); same arithmetic as the
// fused Thread-Greedy kernel.
template <typename G>
__global__ void __launch_bounds__(kThreads)
    k_finalize(G* __restrict__ gacc, const double* __restrict__ w, const double* __restrict__ bjs,
               const double* __restrict__ ib, int64_t k, double inv_n, double lam, uint64_t lnb64, uint32_t lnb32,
               double* __restrict__ delta, double* __restrict__ phi, double* __restrict__ kkt_out,
               int write_steps) {
  __shared__ int s_n;
  __shared__ int64_t s_j[kRoundCols];
  __shared__ double s_g[kRoundCols], s_w[kRoundCols];
  uint64_t vmax = 0, gmax = 0;
  for (int64_t base = (int64_t)blockIdx.x * kRoundCols; base < k; base += (int64_t)gridDim.x * kRoundCols) {
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    const int na = scan_round(gacc, w, base, k, lnb64, lnb32, &s_n, s_j, s_g, s_w, write_steps ? delta : nullptr, phi);
    for (int e = threadIdx.x; e < na; e += kThreads) {
      const int64_t j = s_j[e];
      double g, d, f;
      active_step(s_g[e], inv_n, s_w[e], lam, bjs[j], ib[j], g, d, f);
      max_bits(vmax, kkt_violation(g, s_w[e], lam));
      max_bits(gmax, fabs(g));
      if (write_steps) {
        delta[j] = d;
        phi[j] = f;
      }
    }
    __syncthreads();  // the queue is reused
  }
  block_max_bits_to(kkt_out, vmax);
  block_max_bits_to(kkt_out + 7, gmax);  // max |g_j| over the active columns (idle ones have |g_j| <= lambda)
}

// Thread-Greedy with many partitions: one CTA per partition computes the
// step and proxy of its columns and accepts the best proxy (Table 2, "greedy
// per thread"), so delta and phi never reach memory.  want_kkt: also reduce
// the KKT violation (convergence checks only).  Idle columns (phi = 0) are
// never accepted and are not queued.
template <typename G>
__global__ void __launch_bounds__(kThreads)
    k_finalize_accept(G* __restrict__ gacc, const double* __restrict__ w, const double* __restrict__ bjs,
                      const double* __restrict__ ib, int64_t k, double inv_n, double lam, uint64_t lnb64,
                      uint32_t lnb32, int64_t B, int want_kkt, int32_t* __restrict__ list_j,
                      double* __restrict__ list_d, uint64_t* __restrict__ list_m, double* __restrict__ kkt_out) {
  __shared__ int s_n;
  __shared__ int64_t s_j[kRoundCols];
  __shared__ double s_g[kRoundCols], s_w[kRoundCols];
  __shared__ int64_t s_lo, s_hi;
  uint64_t vmax = 0;
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    // 64-bit divisions run on the FP64 unit, which is small on this GPU:
    // one thread computes the partition bounds
    if (threadIdx.x == 0) {
      s_lo = b * k / B;
      s_hi = (b + 1) * k / B;
    }
    __syncthreads();
    const int64_t lo = s_lo, hi = s_hi;
    uint64_t bm = 0;
    int32_t bj = INT32_MAX;
    double bd = 0.0;
    for (int64_t base = lo; base < hi; base += kRoundCols) {  // uniform across the CTA
      if (threadIdx.x == 0) s_n = 0;
      __syncthreads();
      const int na = scan_round(gacc, w, base, hi, lnb64, lnb32, &s_n, s_j, s_g, s_w, (double*)nullptr,
                                (double*)nullptr);
      for (int e = threadIdx.x; e < na; e += kThreads) {
        const int64_t j = s_j[e];
        double g, d, f;
        active_step(s_g[e], inv_n, s_w[e], lam, bjs[j], ib[j], g, d, f);
        if (want_kkt) max_bits(vmax, kkt_violation(g, s_w[e], lam));
        const uint64_t m = candidate_mag(f);
        if (cand_better(m, (int32_t)j, bm, bj)) {
          bm = m;
          bj = (int32_t)j;
          bd = d;
        }
      }
      __syncthreads();
    }
    block_best(bm, bj, bd);
    if (threadIdx.x == 0) {
      list_j[b] = bm ? bj : -1;
      list_d[b] = bm ? bd : 0.0;
      list_m[b] = bm;
    }
  }
  if (want_kkt) block_max_bits_to(kkt_out, vmax);
}

// ---------------------------------------------------------------------------
// FP32 mode: the per-column pass ranks the columns with Eq. 7 / Eq. 9 in FP32
// (FP32 sums, the float copies of w, beta_j and 1/beta_j); only the accepted
// column's step is recomputed in FP64 (eq7_step with the FP64 w), and it is
// accepted when that proxy is negative.  GB300 runs FP64 at a small fraction
// of its FP32 rate, so the per-column work stays on the FP32 pipe.


// one round of 4 columns per thread of NT: load, zero the sums, integer idle
// test, queue the active columns (j, raw sum) in shared memory
template <int NT>
__device__ __forceinline__ int scan_round_f32(float* __restrict__ gacc, const float* __restrict__ w32, int64_t base,
                                              int64_t hi, uint32_t lnb32, int* s_n, int32_t* s_j, float* s_g) {
  float ga[kColsPerThread], wv[kColsPerThread];
#pragma unroll
  for (int q = 0; q < kColsPerThread; ++q) {
    const int64_t j = base + q * NT + threadIdx.x;
    ga[q] = j < hi ? gacc[j] : 0.0f;
    wv[q] = j < hi ? w32[j] : 0.0f;
  }
#pragma unroll
  for (int q = 0; q < kColsPerThread; ++q) {
    const int64_t j = base + q * NT + threadIdx.x;
    if (j >= hi) continue;
    gacc[j] = 0.0f;
    const bool idle = (__float_as_uint(wv[q]) << 1) == 0 && (__float_as_uint(ga[q]) & 0x7fffffffu) <= lnb32;
    if (!idle) {
      const int slot = atomicAdd(s_n, 1);
      s_j[slot] = (int32_t)j;
      s_g[slot] = ga[q];
    }
  }
  __syncthreads();
  return *s_n;
}

// FP64 step and proxy of the ranked winner (raw sum ga): the accepted delta,
// or no acceptance (false) when that proxy is not negative
__device__ __forceinline__ bool accept_fp64(double ga, int32_t j, double inv_n, double lam,
                                            const double* __restrict__ w, const double* __restrict__ bjs,
                                            const double* __restrict__ ib, double& d) {
  double f;
  eq7_step(ga * inv_n, w[j], lam, bjs[j], ib[j], d, f);
  return candidate_mag(f) != 0;
}

__device__ __forceinline__ uint64_t kkt_bits_f32(uint32_t vmax32) {
  return (uint64_t)__double_as_longlong((double)__uint_as_float(vmax32));
}

constexpr int kFinThreads = 256;  // small CTAs: every partition of config 2 (3,906 columns, 4 rounds) resident at once

__global__ void __launch_bounds__(kFinThreads)
    k_finalize_accept_f32(float* __restrict__ gacc, const float* __restrict__ w32, const float* __restrict__ bj32,
                          const float* __restrict__ ib32, const double* __restrict__ w,
                          const double* __restrict__ bjs, const double* __restrict__ ib, int64_t k, float inv_nf,
                          float lamf, double inv_n, double lam, uint32_t lnb32, int64_t B,
                          const int64_t* __restrict__ part_lo, int want_kkt, int32_t* __restrict__ list_j,
                          double* __restrict__ list_d, uint64_t* __restrict__ list_m, double* __restrict__ kkt_out) {
  constexpr int ROUND = kColsPerThread * kFinThreads;
  __shared__ int s_n;
  __shared__ int32_t s_j[ROUND];
  __shared__ float s_g[ROUND];
  uint32_t vmax = 0;
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    const int64_t lo = part_lo[b], hi = part_lo[b + 1];  // precomputed: no 64-bit division here
    uint64_t bm = 0;
    int32_t bj = INT32_MAX;
    float bga = 0.0f;
    for (int64_t base = lo; base < hi; base += ROUND) {  // uniform across the CTA
      if (threadIdx.x == 0) s_n = 0;
      __syncthreads();
      const int na = scan_round_f32<kFinThreads>(gacc, w32, base, hi, lnb32, &s_n, s_j, s_g);
      for (int e = threadIdx.x; e < na; e += kFinThreads) {
        const int32_t j = s_j[e];
        const float g = s_g[e] * inv_nf, wj = w32[j];
        float d, f;
        eq7_step_f32(g, wj, lamf, bj32[j], ib32[j], d, f);
        if (want_kkt) {
          const uint32_t v = __float_as_uint(kkt_violation_f32(g, wj, lamf));
          vmax = v > vmax ? v : vmax;
        }
        const uint64_t m = candidate_mag32(f);
        if (cand_better(m, j, bm, bj)) {
          bm = m;
          bj = j;
          bga = s_g[e];
        }
      }
      __syncthreads();
    }
    double dga = (double)bga;
    block_best<kFinThreads>(bm, bj, dga);
    if (threadIdx.x == 0) {
      double d = 0.0;
      const bool ok = bm && accept_fp64(dga, bj, inv_n, lam, w, bjs, ib, d);
      list_j[b] = ok ? bj : -1;
      list_d[b] = ok ? d : 0.0;
      list_m[b] = ok ? bm : 0ull;
    }
    __syncthreads();  // s_n and the queue are reused by the next partition
  }
  if (want_kkt) block_max_bits_to(kkt_out, kkt_bits_f32(vmax));
}

// few partitions, stage 1 in FP32 (see k_finalize_chunks); slot_d carries the
// winner's raw sum, and k_accept_slots computes its FP64 step
__global__ void __launch_bounds__(kThreads)
    k_finalize_chunks_f32(float* __restrict__ gacc, const float* __restrict__ w32, const float* __restrict__ bj32,
                          const float* __restrict__ ib32, int64_t k, float inv_nf, float lamf, uint32_t lnb32,
                          int64_t B, int64_t S, int64_t nchunks, int want_kkt, uint64_t* __restrict__ slot_m,
                          int32_t* __restrict__ slot_j, double* __restrict__ slot_d, double* __restrict__ kkt_out) {
  __shared__ int64_t s_b[3];
  uint32_t vmax = 0;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t lo = ch * S, hi = lo + S < k ? lo + S : k;
    if (threadIdx.x == 0) {  // one thread does the 64-bit divisions
      s_b[0] = partition_of(lo, k, B);
      s_b[1] = partition_of(hi - 1, k, B);
      s_b[2] = (s_b[0] + 1) * k / B;  // first column after partition b0
    }
    __syncthreads();
    const int64_t b0 = s_b[0], b1 = s_b[1], end0 = s_b[2];
    uint64_t m0 = 0, m1 = 0;
    int32_t j0 = INT32_MAX, j1 = INT32_MAX;
    float g0 = 0.0f, g1 = 0.0f;
    for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
      const float ga = gacc[j];
      gacc[j] = 0.0f;
      const float wj = w32[j];
      if ((__float_as_uint(wj) << 1) == 0 && (__float_as_uint(ga) & 0x7fffffffu) <= lnb32) continue;
      const float g = ga * inv_nf;
      float d, f;
      eq7_step_f32(g, wj, lamf, bj32[j], ib32[j], d, f);
      if (want_kkt) {
        const uint32_t v = __float_as_uint(kkt_violation_f32(g, wj, lamf));
        vmax = v > vmax ? v : vmax;
      }
      const uint64_t m = candidate_mag32(f);
      if (j < end0) {
        if (cand_better(m, (int32_t)j, m0, j0)) {
          m0 = m;
          j0 = (int32_t)j;
          g0 = ga;
        }
      } else if (cand_better(m, (int32_t)j, m1, j1)) {
        m1 = m;
        j1 = (int32_t)j;
        g1 = ga;
      }
    }
    double d0 = (double)g0, d1 = (double)g1;
    block_best(m0, j0, d0);
    block_best(m1, j1, d1);
    if (threadIdx.x == 0) {
      slot_m[ch + b0] = m0;
      slot_j[ch + b0] = j0;
      slot_d[ch + b0] = d0;
      if (b1 != b0) {
        slot_m[ch + b1] = m1;
        slot_j[ch + b1] = j1;
        slot_d[ch + b1] = d1;
      }
    }
    __syncthreads();
  }
  if (want_kkt) block_max_bits_to(kkt_out, kkt_bits_f32(vmax));
}

// Thread-Greedy with few partitions (Greedy: B = 1), stage 1: one CTA per
// chunk of S <= floor(k / B) columns, which meets at most two partitions;
// the best candidate of (chunk c, partition b) goes to slot c + b.
template <typename G>
__global__ void __launch_bounds__(kThreads)
    k_finalize_chunks(G* __restrict__ gacc, const double* __restrict__ w, const double* __restrict__ bjs,
                      const double* __restrict__ ib, int64_t k, double inv_n, double lam, uint64_t lnb64,
                      uint32_t lnb32,
                      int64_t B, int64_t S, int64_t nchunks, int want_kkt, uint64_t* __restrict__ slot_m,
                      int32_t* __restrict__ slot_j, double* __restrict__ slot_d, double* __restrict__ kkt_out) {
  __shared__ int64_t s_b[3];
  uint64_t vmax = 0;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t lo = ch * S, hi = lo + S < k ? lo + S : k;
    if (threadIdx.x == 0) {  // one thread does the 64-bit divisions (FP64 unit)
      s_b[0] = partition_of(lo, k, B);
      s_b[1] = partition_of(hi - 1, k, B);
      s_b[2] = (s_b[0] + 1) * k / B;  // first column after partition b0
    }
    __syncthreads();
    const int64_t b0 = s_b[0], b1 = s_b[1], end0 = s_b[2];
    uint64_t m0 = 0, m1 = 0;
    int32_t j0 = INT32_MAX, j1 = INT32_MAX;
    double d0 = 0.0, d1 = 0.0;
    for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
      const G ga = gacc[j];
      gacc[j] = G(0);
      const double wj = w[j];
      if (idle_raw(ga, wj, lnb64, lnb32)) continue;
      double g, d, f;
      active_step((double)ga, inv_n, wj, lam, bjs[j], ib[j], g, d, f);
      if (want_kkt) max_bits(vmax, kkt_violation(g, wj, lam));
      const uint64_t m = candidate_mag(f);
      if (j < end0) {  // partition b0
        if (cand_better(m, (int32_t)j, m0, j0)) {
          m0 = m;
          j0 = (int32_t)j;
          d0 = d;
        }
      } else if (cand_better(m, (int32_t)j, m1, j1)) {
        m1 = m;
        j1 = (int32_t)j;
        d1 = d;
      }
    }
    block_best(m0, j0, d0);
    block_best(m1, j1, d1);
    if (threadIdx.x == 0) {
      slot_m[ch + b0] = m0;
      slot_j[ch + b0] = j0;
      slot_d[ch + b0] = d0;
      if (b1 != b0) {
        slot_m[ch + b1] = m1;
        slot_j[ch + b1] = j1;
        slot_d[ch + b1] = d1;
      }
    }
    __syncthreads();
  }
  if (want_kkt) block_max_bits_to(kkt_out, vmax);
}

// stage 2: partition b reduces its slots c + b for the chunks c it meets
// (FP32 mode: slot_d holds raw sums and the winner's step is computed here
// in FP64 from w, bjs, ib; FP64 mode: w is null and slot_d holds the steps)
__global__ void __launch_bounds__(kThreads)
    k_accept_slots(const uint64_t* __restrict__ slot_m, const int32_t* __restrict__ slot_j,
                   const double* __restrict__ slot_d, int64_t k, int64_t B, int64_t S,
                   int32_t* __restrict__ list_j, double* __restrict__ list_d, uint64_t* __restrict__ list_m,
                   const double* __restrict__ w, const double* __restrict__ bjs, const double* __restrict__ ib,
                   double inv_n, double lam) {
  __shared__ int64_t s_c[2];
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    if (threadIdx.x == 0) {  // one thread does the 64-bit divisions (FP64 unit)
      s_c[0] = (b * k / B) / S;
      s_c[1] = ((b + 1) * k / B - 1) / S;
    }
    __syncthreads();
    const int64_t c0 = s_c[0], c1 = s_c[1];
    uint64_t bm = 0;
    int32_t bj = INT32_MAX;
    double bd = 0.0;
    for (int64_t ch = c0 + threadIdx.x; ch <= c1; ch += blockDim.x) {
      const uint64_t m = slot_m[ch + b];
      const int32_t j = slot_j[ch + b];
      if (cand_better(m, j, bm, bj)) {
        bm = m;
        bj = j;
        bd = slot_d[ch + b];
      }
    }
    block_best(bm, bj, bd);
    if (threadIdx.x == 0) {
      bool ok = bm != 0;
      if (ok && w) ok = accept_fp64(bd, bj, inv_n, lam, w, bjs, ib, bd);
      list_j[b] = ok ? bj : -1;
      list_d[b] = ok ? bd : 0.0;
      list_m[b] = ok ? bm : 0ull;
    }
    __syncthreads();
  }
}

template <typename V, typename U>
__global__ void __launch_bounds__(kThreads)
    k_propose_list(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                   const V* __restrict__ val, const U* __restrict__ u, const double* __restrict__ w,
                   const double* __restrict__ bjs, const double* __restrict__ ib, const int32_t* __restrict__ J,
                   int64_t m, double n, double lam, double* __restrict__ delta,
                   double* __restrict__ phi, unsigned long long* __restrict__ counters) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < m; e += nwarps) {
    const int32_t j = J[e];
    const int64_t s = col_ptr[j], t = col_ptr[j + 1];
    V acc = V(0);
    for (int64_t p = s + lane; p < t; p += 32) acc = fma(val[p], (V)__ldg(u + row_idx[p]), acc);
    const double g = warp_sum((double)acc) / n;
    if (lane == 0) {
      double d, f;
      eq7_step(g, w[j], lam, bjs[j], ib[j], d, f);
      delta[e] = d;
      phi[e] = f;
      if (counters) atomicAdd(counters + 1, (unsigned long long)(t - s));
    }
  }
}


template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sm) {
  v = warp_sum(v);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sm[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < NT / 32; ++q) s += sm[q];
  return s;
}

// Per-block partial sums of the loss and of |w_j|; with gap, also of the
// conjugates l*(y_i, s u_i) of the dual point s u (u_i = l'(y_i, z_i) in
// FP64, s = lambda / max(lambda, max_j |g_j|) from the finalize that ran
// before: dscal[7]), so that ||X^T s u|| / n <= lambda.
__global__ void __launch_bounds__(kThreads)
    k_objective_partial(const double* __restrict__ y, const double* __restrict__ z, int64_t n,
                        const double* __restrict__ w, int64_t k, int loss, double lam, int gap,
                        const double* __restrict__ dscal, double* __restrict__ red) {
  __shared__ double sm[kThreads / 32];
  double sl = 0.0, sw = 0.0, sc = 0.0;
  double scale = 1.0;
  if (gap) {
    const double gm = dscal[7];
    scale = gm > lam ? lam / gm : 1.0;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t i = i0; i < n; i += stride) {
    sl += loss_value(loss, y[i], z[i]);
    if (gap) sc += loss_conjugate(loss, y[i], scale * loss_deriv(loss, y[i], z[i]));
  }
  for (int64_t j = i0; j < k; j += stride) sw += fabs(w[j]);
  sl = block_sum<kThreads>(sl, sm);
  sw = block_sum<kThreads>(sw, sm);
  if (gap) sc = block_sum<kThreads>(sc, sm);
  if (threadIdx.x == 0) {
    red[blockIdx.x] = sl;
    red[kRedBlocks + blockIdx.x] = sw;
    if (gap) red[2 * kRedBlocks + blockIdx.x] = sc;
  }
}

// fixed-order reduction of the per-block partials: lane l sums blocks
// l, l+32, ...; then a fixed butterfly.  gap: D = -(1/n) sum of conjugates
// and dscal[9] = P(w) - D
__global__ void k_objective_final(const double* __restrict__ red, int nblocks, double n, double lam, int gap,
                                  double* __restrict__ dscal) {
  const int lane = threadIdx.x & 31;
  double sl = 0.0, sw = 0.0, sc = 0.0;
  for (int b = lane; b < nblocks; b += 32) {
    sl += red[b];
    sw += red[kRedBlocks + b];
    if (gap) sc += red[2 * kRedBlocks + b];
  }
  sl = warp_sum(sl);
  sw = warp_sum(sw);
  if (gap) sc = warp_sum(sc);
  if (threadIdx.x == 0) {
    const double P = (n > 0 ? sl / n : 0.0) + lam * sw;
    dscal[1] = P;
    dscal[2] = sl;
    dscal[3] = sw;
    if (gap) {
      dscal[8] = sc;
      dscal[9] = P + (n > 0 ? sc / n : 0.0);
    }
  }
}

// ---------------------------------------------------------------------------
// launchers

static int blocks_per_sm_cap(gencd_problem* p, int per_sm) { return p->num_sms * per_sm; }

// Lane-segmented streaming pass over the whole CSC: out[col] += X_col^T u
// (the path without a row-slab plan, and the setup passes).  With u
// in the storage precision the sums go to the native accumulator (float in
// FP32 mode), otherwise (power iteration in FP32 mode) to the FP64 gacc.
int launch_propose_csc(gencd_problem* p, const CscView& a, const void* u_vec, bool u_is_double) {
  if (a.ntiles == 0) return GENCD_OK;
  const int grid = grid_for(a.ntiles * 32, kThreads, blocks_per_sm_cap(p, 8));
  if (p->precision == GENCD_F64) {
    k_propose_all<double, double, kItemsF64, double><<<grid, kThreads, 0, p->stream>>>(
        a.col_ptr, a.row_idx, (const double*)a.val, (const double*)u_vec, a.tile_col, a.nnz, a.ntiles, a.cmap,
        p->gacc);
  } else if (u_is_double) {
    k_propose_all<float, double, kItemsF32, double><<<grid, kThreads, 0, p->stream>>>(
        a.col_ptr, a.row_idx, (const float*)a.val, (const double*)u_vec, a.tile_col, a.nnz, a.ntiles, a.cmap,
        p->gacc);
  } else {
    k_propose_all<float, float, kItemsF32, float><<<grid, kThreads, 0, p->stream>>>(
        a.col_ptr, a.row_idx, (const float*)a.val, (const float*)u_vec, a.tile_col, a.nnz, a.ntiles, a.cmap,
        (float*)p->gnat);
  }
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

// native accumulator <- X^T u for every column: the row-slab plan (heavy
// columns, u from shared memory) plus the light columns, or the plain CSC
// pass when no plan was built.  Non-native u (power iteration in FP32 mode)
// always takes the plain pass into the FP64 gacc.
int launch_propose_all(gencd_problem* p, const void* u_vec, bool u_is_double) {
  cudaEvent_t ev = nullptr;
  prof_begin(p, K_PROPOSE_ALL, &ev, 0);  // the whole family; its kernels count their launches
  const bool native = u_is_double == (p->precision == GENCD_F64);
  if (p->plan.built && native) {
    GENCD_TRY(launch_propose_plan(p, u_vec));
  } else {
    CscView a{p->col_ptr, p->row_idx, p->val, p->tile_col, p->nnz, p->ntiles, nullptr};
    cudaEvent_t e2 = nullptr;
    prof_begin(p, K_PROPOSE_LIGHT, &e2);
    GENCD_TRY(launch_propose_csc(p, a, u_vec, u_is_double));
    prof_end(p, e2);
  }
  prof_end(p, ev);
  return GENCD_OK;
}

int launch_col_sumsq(gencd_problem* p) {
  if (p->ntiles == 0) return GENCD_OK;
  const int grid = grid_for(p->ntiles * 32, kThreads, blocks_per_sm_cap(p, 8));
  if (p->precision == GENCD_F64)
    k_propose_all<double, double, kItemsF64, double, true><<<grid, kThreads, 0, p->stream>>>(
        p->col_ptr, p->row_idx, (const double*)p->val, nullptr, p->tile_col, p->nnz, p->ntiles, nullptr,
        p->gacc);
  else
    k_propose_all<float, double, kItemsF32, double, true><<<grid, kThreads, 0, p->stream>>>(
        p->col_ptr, p->row_idx, (const float*)p->val, nullptr, p->tile_col, p->nnz, p->ntiles, nullptr,
        p->gacc);
  p->prof.launches[K_SETUP] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

static void lambda_bits(gencd_problem* p, double lambda, uint64_t* b64, uint32_t* b32) {
  const double ln = lambda * (double)p->n;
  *b64 = (uint64_t)__builtin_bit_cast(int64_t, ln);
  *b32 = (uint32_t)__builtin_bit_cast(int32_t, (float)ln);
}

int launch_finalize(gencd_problem* p, double lambda, bool write_steps) {
  const int grid = grid_for(p->k, kThreads, blocks_per_sm_cap(p, 8));
  uint64_t b64;
  uint32_t b32;
  lambda_bits(p, lambda, &b64, &b32);
  const double inv_n = 1.0 / (double)p->n;
  cudaEvent_t ev = nullptr;
  prof_begin(p, K_FINALIZE, &ev);
  if (p->precision == GENCD_F64)
    k_finalize<double><<<grid, kThreads, 0, p->stream>>>((double*)p->gnat, p->w, p->bj, p->ib, p->k, inv_n, lambda,
                                                         b64, b32, p->delta, p->phi, p->dscal + 0, write_steps ? 1 : 0);
  else
    k_finalize<float><<<grid, kThreads, 0, p->stream>>>((float*)p->gnat, p->w, p->bj, p->ib, p->k, inv_n, lambda,
                                                        b64, b32, p->delta, p->phi, p->dscal + 0, write_steps ? 1 : 0);
  prof_end(p, ev);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

__global__ void k_part_bounds(int64_t k, int64_t B, int64_t* __restrict__ lo) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= B; b += stride) lo[b] = b * k / B;
}

// part_lo[b] = floor(b k / B), b = 0..B (Thread-Greedy partitions, reading 4)
static int ensure_part_bounds(gencd_problem* p, int64_t B) {
  if (p->part_B == B && p->part_lo) return GENCD_OK;
  if (p->part_cap < B + 1) {
    GENCD_CUDA_TRY(cudaStreamSynchronize(p->stream));
    dev_free(p, p->part_lo);
    p->part_lo = nullptr;
    p->part_cap = 0;
    GENCD_TRY(dev_alloc(p, &p->part_lo, (size_t)(B + 1)));
    p->part_cap = B + 1;
  }
  k_part_bounds<<<grid_for(B + 1, kThreads, p->num_sms * 8), kThreads, 0, p->stream>>>(p->k, B, p->part_lo);
  p->prof.launches[K_SETUP] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  p->part_B = B;
  return GENCD_OK;
}

int launch_finalize_accept(gencd_problem* p, int64_t B, bool want_kkt) {
  const double inv_n = 1.0 / (double)p->n;
  uint64_t b64;
  uint32_t b32;
  lambda_bits(p, p->lambda, &b64, &b32);
  const bool f64 = p->precision == GENCD_F64;
  cudaEvent_t ev = nullptr;
  prof_begin(p, K_FINALIZE, &ev);
  if (B >= 2LL * p->num_sms) {
    const int grid = (int)(B < (int64_t)p->num_sms * 16 ? B : (int64_t)p->num_sms * 16);
    if (f64)
      k_finalize_accept<double><<<grid, kThreads, 0, p->stream>>>((double*)p->gnat, p->w, p->bj, p->ib, p->k, inv_n,
                                                                  p->lambda, b64, b32, B, want_kkt ? 1 : 0, p->list_j,
                                                                  p->list_d, p->list_m, p->dscal + 0);
    else {
      GENCD_TRY(ensure_part_bounds(p, B));
      k_finalize_accept_f32<<<grid, kFinThreads, 0, p->stream>>>(
          (float*)p->gnat, p->w32, p->bj32, p->ib32, p->w, p->bj, p->ib, p->k, (float)inv_n, (float)p->lambda, inv_n,
          p->lambda, b32, B, p->part_lo, want_kkt ? 1 : 0, p->list_j, p->list_d, p->list_m, p->dscal + 0);
    }
  } else {
    int64_t S = p->k / B;  // >= 1 since B <= k; a chunk meets at most two partitions
    if (S > 4096) S = 4096;
    const int64_t nchunks = (p->k + S - 1) / S;
    GENCD_TRY(ensure_slots(p, nchunks + B));
    const int grid = grid_for(nchunks * kThreads, kThreads, blocks_per_sm_cap(p, 8));
    if (f64)
      k_finalize_chunks<double><<<grid, kThreads, 0, p->stream>>>((double*)p->gnat, p->w, p->bj, p->ib, p->k, inv_n,
                                                                  p->lambda, b64, b32, B, S, nchunks, want_kkt ? 1 : 0,
                                                                  p->slot_m, p->slot_j, p->slot_d, p->dscal + 0);
    else
      k_finalize_chunks_f32<<<grid, kThreads, 0, p->stream>>>((float*)p->gnat, p->w32, p->bj32, p->ib32, p->k,
                                                              (float)inv_n, (float)p->lambda, b32, B, S, nchunks,
                                                              want_kkt ? 1 : 0, p->slot_m, p->slot_j, p->slot_d,
                                                              p->dscal + 0);
    const int g2 = (int)(B < (int64_t)p->num_sms * 16 ? B : (int64_t)p->num_sms * 16);
    k_accept_slots<<<g2, kThreads, 0, p->stream>>>(p->slot_m, p->slot_j, p->slot_d, p->k, B, S, p->list_j,
                                                   p->list_d, p->list_m, f64 ? nullptr : p->w, p->bj, p->ib, inv_n,
                                                   p->lambda);
    p->prof.launches[K_ACCEPT] += 1;
  }
  prof_end(p, ev);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

// Accept backoff for Thread-Greedy: of every G consecutive partitions only
// the accepted column with the best proxy (largest candidate magnitude, ties
// to the lower partition) is kept.
__global__ void k_merge_accept(int32_t* __restrict__ list_j, const uint64_t* __restrict__ list_m, int64_t B, int64_t G) {
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * G;
  if (b >= B) return;
  const int64_t end = b + G < B ? b + G : B;
  int64_t win = -1;
  uint64_t best = 0;
  for (int64_t c = b; c < end; ++c)
    if (list_j[c] >= 0 && (win < 0 || list_m[c] > best)) {
      win = c;
      best = list_m[c];
    }
  for (int64_t c = b; c < end; ++c)
    if (c != win) list_j[c] = -1;
}

int launch_merge_accept(gencd_problem* p, int64_t B) {
  const int64_t G = p->accept_group;
  if (G <= 1 || B <= 1) return GENCD_OK;
  const int64_t groups = (B + G - 1) / G;
  k_merge_accept<<<grid_for(groups, kThreads, (int)((groups + kThreads - 1) / kThreads) + 1), kThreads, 0,
                   p->stream>>>(p->list_j, p->list_m, B, G);
  p->prof.launches[K_ACCEPT] += 1;
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

int launch_propose_list(gencd_problem* p, const int32_t* J, int64_t m, double* delta, double* phi) {
  if (m <= 0) return GENCD_OK;
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(p->dscal + 4);
  const int grid = grid_for(m * 32, kThreads, blocks_per_sm_cap(p, 8));
  cudaEvent_t ev = nullptr;
  prof_begin(p, K_PROPOSE_LIST, &ev);
  if (p->precision == GENCD_F64)
    k_propose_list<double, double><<<grid, kThreads, 0, p->stream>>>(
        p->col_ptr, p->row_idx, (const double*)p->val, (const double*)p->u, p->w, p->bj, p->ib, J, m,
        (double)p->n, p->lambda, delta, phi, ctr);
  else
    k_propose_list<float, float><<<grid, kThreads, 0, p->stream>>>(
        p->col_ptr, p->row_idx, (const float*)p->val, (const float*)p->u, p->w, p->bj, p->ib, J, m,
        (double)p->n, p->lambda, delta, phi, ctr);
  prof_end(p, ev);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

int launch_objective(gencd_problem* p, bool gap) {
  const int64_t work = p->n > p->k ? p->n : p->k;
  const int grid = grid_for(work, kThreads, kRedBlocks);
  cudaEvent_t ev = nullptr;
  prof_begin(p, K_OBJECTIVE, &ev);
  k_objective_partial<<<grid, kThreads, 0, p->stream>>>(p->y, p->z, p->n, p->w, p->k, p->loss, p->lambda,
                                                        gap ? 1 : 0, p->dscal, p->red);
  k_objective_final<<<1, 32, 0, p->stream>>>(p->red, grid, (double)p->n, p->lambda, gap ? 1 : 0, p->dscal);
  prof_end(p, ev);
  p->prof.launches[K_OBJECTIVE] += 1;  // two launches per objective
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

}  // namespace gencd
