// propose_plan.cu -- row-slab layout of the streaming propose (g = X^T u over
// all columns) on sm_103a.
//
// Gathering u_i at random rows costs one 32-byte L2 sector per 4- or 8-byte
// value, which makes a plain CSC pass L2-bound long before HBM is saturated.
// Here the rows are cut into slabs of at most 192 KB of u.  A persistent CTA
// (one per SM, 1024 threads) copies the u slab of its work into shared memory
// once and gathers from there.  Only columns with at least heavy_min
// non-zeros use this layout (their entries are regrouped slab by slab, with
// 16-bit in-slab rows); every (slab, column) "pair" produces one partial sum,
// added atomically into the column's g_j.  Columns with fewer non-zeros would
// produce about one partial per non-zero, so they keep a compact CSC copy and
// the lane-segmented pass with gathers from L2.
//
// Within a slab the kernel works like the CSC pass: a warp owns a tile of
// 256 consecutive entries, a lane 8 of them (128-bit loads of rows and
// values), a lane sums its entries pair by pair in registers and adds each
// run's sum into g_j (an atomic add that returns nothing: other slabs and
// tiles add to the same column); a run cut by lane boundaries is combined by
// a segmented warp suffix sum first, and a full tile inside one pair is
// reduced by the warp.  Sums are kept in the storage precision (FP32 atomics
// in FP32 mode), so the order of a heavy column's additions, and with it the
// last bits of g_j, can differ between launches.
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "device_math.cuh"
#include "gencd_internal.cuh"

namespace gencd {

constexpr int kSlabBytes = 192 * 1024;
constexpr int kSlabThreadsF32 = 1024;  // 32 warps, the next tile's loads in flight
constexpr int kSlabThreadsF64 = 1024;  // 32 warps, loads issued tile by tile
constexpr int kSlabItemsF32 = 8;   // entries per lane and tile step
constexpr int kSlabItemsF64 = 8;
constexpr int kSlabPad = 16;       // slab entry ranges are padded to this
constexpr int kSlabZeroSlot = 4;   // shared u slots past the slab (16 B); the first holds 0

// ---------------------------------------------------------------------------
// the kernel

template <typename V, int N>
__device__ __forceinline__ void load_vals(const V* __restrict__ p, V (&v)[N]) {
  constexpr int PER = 16 / (int)sizeof(V);  // values per 128-bit load
#pragma unroll
  for (int q = 0; q < N / PER; ++q) {
    if (sizeof(V) == 4) {
      const float4 x = __ldcs(reinterpret_cast<const float4*>(p) + q);
      v[4 * q] = (V)x.x, v[4 * q + 1] = (V)x.y, v[4 * q + 2] = (V)x.z, v[4 * q + 3] = (V)x.w;
    } else {
      const double2 x = __ldcs(reinterpret_cast<const double2*>(p) + q);
      v[2 * q] = (V)x.x, v[2 * q + 1] = (V)x.y;
    }
  }
}

template <typename V>
__device__ __forceinline__ void load8(const V* __restrict__ p, V (&v)[8]) {
  load_vals<V, 8>(p, v);
}

template <typename G>
__device__ __forceinline__ void emit_pair(G* __restrict__ out, uint32_t slot, G s, bool whole) {
  if (whole)
    out[slot] = s;
  else
    atomicAdd(out + slot, s);
}

// Values of a lane's entries as stored by the plan (SV): float or double,
// bfloat16 (kept packed, two per register, widened on use), or none at all
// (NoVal: index-only columns, every value 1; the column scale is applied to
// the column's sum outside the streaming loop).
struct NoVal {};

// a heavy column's run sum into g_j: other slabs and tiles add to the same
// column, so always atomically (index-only storage: the sum of u over the
// column's rows; k_scale_heavy applies the column's value afterwards)
template <typename G>
__device__ __forceinline__ void add_col(G* __restrict__ gacc, uint32_t j, G v) {
  atomicAdd(gacc + j, v);
}

template <typename SV, int N>
struct ValRegs;

template <int N>
struct ValRegs<float, N> {
  float v[N];
  __device__ __forceinline__ void load(const float* __restrict__ p) { load_vals<float, N>(p, v); }
  __device__ __forceinline__ float get(int i) const { return v[i]; }
};

template <int N>
struct ValRegs<double, N> {
  double v[N];
  __device__ __forceinline__ void load(const double* __restrict__ p) { load_vals<double, N>(p, v); }
  __device__ __forceinline__ double get(int i) const { return v[i]; }
};

template <int N>
struct ValRegs<__nv_bfloat16, N> {
  uint32_t w[N / 2];  // value 2q in the low half of w[q], 2q + 1 in the high half
  __device__ __forceinline__ void load(const __nv_bfloat16* __restrict__ p) {
#pragma unroll
    for (int q = 0; q < N / 8; ++q) {
      const uint4 x = __ldcs(reinterpret_cast<const uint4*>(p) + q);
      w[4 * q] = x.x, w[4 * q + 1] = x.y, w[4 * q + 2] = x.z, w[4 * q + 3] = x.w;
    }
  }
  __device__ __forceinline__ float get(int i) const {  // bfloat16 -> float: the upper 16 bits
    const uint32_t x = w[i >> 1];
    return __uint_as_float((i & 1) ? (x & 0xffff0000u) : (x << 16));
  }
};

template <int N>
struct ValRegs<NoVal, N> {
  __device__ __forceinline__ void load(const NoVal*) {}
  __device__ __forceinline__ float get(int) const { return 1.0f; }
};

// the entries of one lane: ITEMS in-slab rows (128-bit loads of 8) and values
template <typename SV, int ITEMS>
struct LaneLoad {
  uint4 rr[ITEMS / 8];
  ValRegs<SV, ITEMS> val;
};

template <typename SV, int ITEMS>
__device__ __forceinline__ void load_lane(const uint16_t* __restrict__ s_row, const SV* __restrict__ s_val,
                                          uint32_t a, LaneLoad<SV, ITEMS>& L) {
#pragma unroll
  for (int h = 0; h < ITEMS / 8; ++h) L.rr[h] = __ldcs(reinterpret_cast<const uint4*>(s_row + a) + h);
  L.val.load(s_val + a);
}

// start bits of a lane's ITEMS entries (one byte per 8 entries, little-endian)
template <int ITEMS>
__device__ __forceinline__ uint32_t lane_mask(const uint8_t* __restrict__ pmask, uint32_t a) {
  if (ITEMS == 16) return reinterpret_cast<const uint16_t*>(pmask)[a >> 4];
  return pmask[a >> 3];
}

// Segmented suffix sum over the lanes: T_L = x_L + x_{L+1} + ... + x_M where M
// is the first lane >= L with stop set (all lanes to 31 when there is none);
// ended_L reports whether such an M exists.  Five shuffle steps.
template <typename V>
__device__ __forceinline__ V lane_suffix_sum(V x, bool stop, int lane, bool& ended) {
  V t = x;
  bool e = stop;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const V tn = __shfl_down_sync(0xffffffffu, t, d);
    const bool en = __shfl_down_sync(0xffffffffu, (int)e, d) != 0;
    if (!e && lane + d < 32) {
      t += tn;
      e = en;
    }
  }
  ended = e;
  return t;
}

// Pairs are numbered in entry order; pmask holds one byte per 8 entries whose
// bit i says "entry 8g + i starts a pair", and tile_pair[t] is the pair of the
// tile's first entry.  A lane finds the pair of its first entry from a warp
// prefix count of the start bits, so no pair table is searched.  Per lane:
// runs that start and end inside the lane are stored; the run that continues
// from the left (cont) and the run that leaves to the right (tail) are
// combined across the warp by a segmented suffix sum, so only the tile's first
// and last pairs take atomic adds.
// one tile's loads for one lane: ITEMS rows and values, the start bits, and
// the pair of the tile's first entry
template <typename SV, int ITEMS>
struct TileStage {
  LaneLoad<SV, ITEMS> L;
  uint32_t m, q0;
};

template <typename SV, int ITEMS>
__device__ __forceinline__ void load_stage(const uint16_t* __restrict__ s_row, const SV* __restrict__ s_val,
                                           const uint8_t* __restrict__ pmask,
                                           const uint32_t* __restrict__ tile_pair, int t, int t1, uint32_t base,
                                           int tb, uint32_t slab_end, int lane, TileStage<SV, ITEMS>& S) {
  S.m = 0;
  if (t < t1) {
    S.q0 = __ldg(tile_pair + t);
    const uint32_t a = base + (uint32_t)(t - tb) * (32 * ITEMS) + lane * ITEMS;
    if (a < slab_end) {
      load_lane<SV, ITEMS>(s_row, s_val, a, S.L);
      S.m = lane_mask<ITEMS>(pmask, a);
    }
  }
}

// Barrier of the warps that share a CTA's u slab: the whole CTA (BAR_THREADS
// = 0), or the first BAR_THREADS threads on named barrier 1 when other warps
// of the CTA do other work (the fused pass below).
template <int BAR_THREADS>
__device__ __forceinline__ void slab_barrier() {
  if (BAR_THREADS == 0)
    __syncthreads();
  else
    asm volatile("bar.sync 1, %0;" ::"n"(BAR_THREADS) : "memory");
}

// The row-slab pass of one CTA's contiguous run of tiles [t0, t_end), by the
// warps warp = 0 .. nw - 1 of the slab group (ITEMS entries per lane, a tile
// is 32 * ITEMS entries; DEPTH tiles of loads in flight per warp beyond the
// one being processed).
template <typename V, typename U, typename G, int DEPTH, int ITEMS, typename SV, int BAR_THREADS>
__device__ __forceinline__ void slab_pass(const uint16_t* __restrict__ s_row, const SV* __restrict__ s_val,
                                          const uint8_t* __restrict__ pmask, const uint32_t* __restrict__ pair_col,
                                          const uint32_t* __restrict__ tile_start,
                                          const uint32_t* __restrict__ tile_end,
                                          const uint32_t* __restrict__ tile_pair,
                                          const int32_t* __restrict__ tile_slab,
                                          const int32_t* __restrict__ slab_tile_begin, int t0, const int t_end,
                                          const U* __restrict__ u, int64_t n, int32_t slab_rows,
                                          G* __restrict__ gacc, U* s_u, const int warp, const int nw,
                                          const int gtid, const int gthreads) {
  constexpr int TILE = 32 * ITEMS;
  constexpr uint32_t NOT_FIRST = ((1u << ITEMS) - 1u) & ~1u;  // start bits after a lane's first entry
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  if (gtid == 0) s_u[slab_rows] = U(0);  // the row of padding entries (index-only storage)
  while (t0 < t_end) {
    const int r = tile_slab[t0];
    const int tb = slab_tile_begin[r], tnext = slab_tile_begin[r + 1];
    const int t1 = min(t_end, tnext);
    const uint32_t base = tile_start[tb], slab_end = tile_end[tnext - 1];  // the slab's entries
    const int64_t row0 = (int64_t)r * slab_rows;
    const int rows = (int)min((int64_t)slab_rows, n - row0);
    slab_barrier<BAR_THREADS>();  // the previous slab is no longer read
    {  // 16-byte loads, four in flight per thread, when u + row0 is 16-byte aligned
      const bool al = (reinterpret_cast<uintptr_t>(u + row0) & 15u) == 0;
      const int nvec = al ? (int)(((int64_t)rows * (int64_t)sizeof(U)) / 16) : 0;
      const uint4* src = reinterpret_cast<const uint4*>(u + row0);
      uint4* dst = reinterpret_cast<uint4*>(s_u);
#pragma unroll 4
      for (int i = gtid; i < nvec; i += gthreads) dst[i] = __ldcg(src + i);
      for (int i = (int)((int64_t)nvec * 16 / (int64_t)sizeof(U)) + gtid; i < rows; i += gthreads) s_u[i] = u[row0 + i];
    }
    slab_barrier<BAR_THREADS>();
    TileStage<SV, ITEMS> stg[DEPTH > 0 ? DEPTH : 1];
    int t = t0 + warp;
#pragma unroll
    for (int d = 0; d < DEPTH; ++d)
      load_stage<SV, ITEMS>(s_row, s_val, pmask, tile_pair, t + d * nw, t1, base, tb, slab_end, lane, stg[d]);
    for (; t < t1; t += nw) {  // warp-uniform loop
      TileStage<SV, ITEMS> cur;
      if (DEPTH > 0) {
        cur = stg[0];
#pragma unroll
        for (int d = 0; d + 1 < DEPTH; ++d) stg[d] = stg[d + 1];
        load_stage<SV, ITEMS>(s_row, s_val, pmask, tile_pair, t + DEPTH * nw, t1, base, tb, slab_end, lane,
                              stg[DEPTH - 1]);
      } else {
        load_stage<SV, ITEMS>(s_row, s_val, pmask, tile_pair, t, t1, base, tb, slab_end, lane, cur);
      }
      const uint32_t ts = base + (uint32_t)(t - tb) * TILE;
      const uint32_t te = slab_end - ts < (uint32_t)TILE ? slab_end : ts + TILE;
      const uint32_t q0 = cur.q0;
      uint32_t m = cur.m;
      const uint32_t a = ts + lane * ITEMS;
      const bool active = a < te;  // slab ends are multiples of ITEMS
      if (!active) m = 0;
      // pair of the lane's first entry: q0 + start bits in (ts, a] of the tile
      const uint32_t cnt = __popc(lane == 0 ? (m & NOT_FIRST) : m);
      uint32_t incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += y;
      }
      uint32_t q = q0 + (incl - cnt) + (lane > 0 ? (m & 1u) : 0u);
      // columns of the pairs this lane may emit, loaded early: the tile's
      // first pair (lane 0) and the pair of the lane's last run
      const bool lead = lane == 0 && active && !(m & 1u);
      const uint32_t col0 = lead ? __ldg(pair_col + q0) : 0u;
      const uint32_t col_last = (active && m != 0u) ? __ldg(pair_col + q + __popc(m & NOT_FIRST)) : 0u;
      V cont = V(0), tail = V(0);
      bool has_tail = false;
      if (active) {
        U uu[ITEMS];
#pragma unroll
        for (int h = 0; h < ITEMS / 8; ++h) {
          const uint32_t w4[4] = {cur.L.rr[h].x, cur.L.rr[h].y, cur.L.rr[h].z, cur.L.rr[h].w};
#pragma unroll
          for (int k2 = 0; k2 < 4; ++k2) {
            uu[8 * h + 2 * k2] = s_u[w4[k2] & 0xffffu];
            uu[8 * h + 2 * k2 + 1] = s_u[w4[k2] >> 16];
          }
        }
        // one FMA chain over the lane's entries; at each start bit after
        // entry 0 the running sum closes a run: the first run (continuing
        // from the left, or a whole run when it began at entry 0) or a run
        // between two start bits (whole: stored); the last run stays in acc
        const uint32_t inner = m & NOT_FIRST;
        const int bf = inner ? __ffs(inner) - 1 : ITEMS;  // first start bit after entry 0
        V acc = V(0), first = V(0);
        uint32_t qi = q;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
          if ((inner >> i) & 1u) {
            if (i == bf)
              first = acc;
            else
              add_col<G>(gacc, __ldg(pair_col + qi), (G)acc);  // started and ended inside the lane
            acc = V(0);
            ++qi;
          }
          acc = fma((V)cur.L.val.get(i), (V)uu[i], acc);
        }
        if (inner) {
          if (m & 1u)
            add_col<G>(gacc, __ldg(pair_col + q), (G)first);  // started at entry 0, ended inside
          else
            cont = first;  // continues from the left
          tail = acc;  // the last run started inside the lane
          has_tail = true;
        } else if (m & 1u) {  // one run, starting at the lane's first entry
          tail = acc;
          has_tail = true;
        } else {
          cont = acc;
        }
      }
      const bool stop = !active || m != 0u;
      if (__ballot_sync(FULL, stop) == 0u) {
        // the whole tile lies inside pair q0
        const V sum = warp_sum(cont);
        if (lane == 0) add_col<G>(gacc, col0, (G)sum);
      } else {
        bool ended;
        const V tsum = lane_suffix_sum(cont, stop, lane, ended);
        const V t1s = __shfl_down_sync(FULL, tsum, 1);
        if (lead) add_col<G>(gacc, col0, (G)tsum);  // pair from the previous tile
        if (has_tail) add_col<G>(gacc, col_last, (G)(tail + (lane < 31 ? t1s : V(0))));
      }
    }
    t0 = t1;
  }
}

// THREADS per CTA (one CTA per SM); see slab_pass
template <typename V, typename U, typename G, int THREADS, int DEPTH, int ITEMS, typename SV>
__global__ void __launch_bounds__(THREADS, 1)
    k_propose_slabs(const uint16_t* __restrict__ s_row, const SV* __restrict__ s_val,
                    const uint8_t* __restrict__ pmask, const uint32_t* __restrict__ pair_col,
                    const uint32_t* __restrict__ tile_start,
                    const uint32_t* __restrict__ tile_end, const uint32_t* __restrict__ tile_pair,
                    const int32_t* __restrict__ tile_slab, const int32_t* __restrict__ slab_tile_begin,
                    const int32_t* __restrict__ cta_tile_begin, const U* __restrict__ u, int64_t n,
                    int32_t slab_rows, G* __restrict__ gacc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  U* s_u = reinterpret_cast<U*>(smem_raw);
  slab_pass<V, U, G, DEPTH, ITEMS, SV, 0>(s_row, s_val, pmask, pair_col, tile_start, tile_end, tile_pair, tile_slab,
                                          slab_tile_begin, cta_tile_begin[blockIdx.x],
                                          cta_tile_begin[blockIdx.x + 1], u, n, slab_rows, gacc, s_u,
                                          threadIdx.x >> 5, blockDim.x >> 5, threadIdx.x, blockDim.x);
}

// ---------------------------------------------------------------------------
// the light columns: a compact CSC copy streamed in 256-entry tiles, u gathered
// from L2.  Column starts are marked like pair starts above (one byte per 8
// entries), tile_lc[t] is the light column of the tile's first entry, and the
// same per-lane runs / segmented suffix sum assign every partial sum to its
// column without a search; results go to out[light_cols[lc]].
constexpr int kLightItems = 8;
constexpr int kLightTile = 32 * kLightItems;

__device__ __forceinline__ void load_rows8(const int32_t* __restrict__ p, int32_t (&r)[8]) {
  const int4 a = __ldcs(reinterpret_cast<const int4*>(p));
  const int4 b = __ldcs(reinterpret_cast<const int4*>(p) + 1);
  r[0] = a.x, r[1] = a.y, r[2] = a.z, r[3] = a.w, r[4] = b.x, r[5] = b.y, r[6] = b.z, r[7] = b.w;
}

// one lane's loads of a light tile: 8 rows, 8 values (as stored), the start
// bits, and the light column of the tile's first entry
template <typename SV>
struct LightStage {
  int32_t r[8];
  ValRegs<SV, 8> val;
  uint32_t m, lc0;
};

template <typename SV>
__device__ __forceinline__ void load_light_stage(const int32_t* __restrict__ row, const SV* __restrict__ val,
                                                 const uint8_t* __restrict__ lmask,
                                                 const int32_t* __restrict__ tile_lc, int64_t t, int64_t ntiles,
                                                 int64_t nnz, int lane, LightStage<SV>& S) {
  S.m = 0;
  if (t < ntiles) {
    S.lc0 = (uint32_t)__ldg(tile_lc + t);
    const int64_t a = t * kLightTile + (int64_t)lane * kLightItems;
    if (a < nnz) {  // the arrays are padded: a lane's 8 entries are in bounds
      load_rows8(row + a, S.r);
      S.val.load(val + a);
      S.m = lmask[a >> 3];
    }
  }
}

// One light tile's sums from its loads `cur` (lscale: index-only columns,
// each column's sum scaled by its value); results go to out[light_cols[lc]].
template <typename V, typename U, typename G, typename SV>
__device__ __forceinline__ void light_tile(const LightStage<SV>& cur, int64_t t, int64_t nnz,
                                           const int32_t* __restrict__ light_cols,
                                           const float* __restrict__ lscale, const U* __restrict__ u,
                                           G* __restrict__ out, int lane) {
  const unsigned FULL = 0xffffffffu;
  constexpr bool kScaled = std::is_same<SV, NoVal>::value;
  const int64_t a = t * kLightTile + (int64_t)lane * kLightItems;
  const bool active = a < nnz;
  const uint32_t m = cur.m, lc0 = cur.lc0;
  const int32_t* r = cur.r;
  const uint32_t cnt = __popc(lane == 0 ? (m & 0xfeu) : m);
  uint32_t incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += y;
  }
  uint32_t q = lc0 + (incl - cnt) + (lane > 0 ? (m & 1u) : 0u);
  // columns this lane may write (and their scales), loaded early
  const bool lead = lane == 0 && active && !(m & 1u);
  const uint32_t ql = q + __popc(m & 0xfeu);
  const int32_t j0 = lead ? __ldg(light_cols + lc0) : 0;
  const int32_t jl = (active && m != 0u) ? __ldg(light_cols + ql) : 0;
  V s0 = V(1), sl = V(1);
  if (kScaled) {
    s0 = lead ? (V)__ldg(lscale + lc0) : V(1);
    sl = (active && m != 0u) ? (V)__ldg(lscale + ql) : V(1);
  }
  V cont = V(0), tail = V(0);
  bool has_tail = false;
  if (active) {
    U uu[8];
#pragma unroll
    // gathers of u through L2 without allocating in L1 (no reuse to keep)
    for (int i = 0; i < 8; ++i) uu[i] = __ldcg(u + r[i]);  // padding rows are 0, values 0
    // first run, last run and the whole columns between (see k_propose_slabs)
    const uint32_t inner = m & 0xfeu;
    const int bf = inner ? __ffs(inner) - 1 : 8;
    V acc = V(0), first = V(0);
    uint32_t qi = q;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if ((inner >> i) & 1u) {
        if (i == bf) {
          first = acc;
        } else {  // a whole column inside the lane
          const V sc = kScaled ? (V)__ldg(lscale + qi) : V(1);
          out[__ldg(light_cols + qi)] = (G)(acc * sc);
        }
        acc = V(0);
        ++qi;
      }
      acc = fma((V)cur.val.get(i), (V)uu[i], acc);
    }
    if (inner) {
      if (m & 1u) {  // started at entry 0, ended inside
        const V sc = kScaled ? (V)__ldg(lscale + q) : V(1);
        out[__ldg(light_cols + q)] = (G)(first * sc);
      } else {
        cont = first;
      }
      tail = acc;
      has_tail = true;
    } else if (m & 1u) {
      tail = acc;
      has_tail = true;
    } else {
      cont = acc;
    }
  }
  const bool stop = !active || m != 0u;
  if (__ballot_sync(FULL, stop) == 0u) {
    const V sum = warp_sum(cont);  // the whole tile is inside column lc0
    if (lane == 0) atomicAdd(out + j0, (G)(sum * s0));
  } else {
    bool ended;
    const V tsum = lane_suffix_sum(cont, stop, lane, ended);
    const V t1s = __shfl_down_sync(FULL, tsum, 1);
    const bool e1 = __shfl_down_sync(FULL, (int)ended, 1) != 0;
    if (lead) atomicAdd(out + j0, (G)(tsum * s0));  // column from the previous tile
    if (has_tail) {
      const V sum = tail + (lane < 31 ? t1s : V(0));
      emit_pair<G>(out, (uint32_t)jl, (G)(sum * sl), lane < 31 && e1);
    }
  }
}

template <typename V, typename U, typename G, typename SV>
__global__ void __launch_bounds__(kThreads, 3)
    k_propose_light_runs(const int32_t* __restrict__ row, const SV* __restrict__ val,
                         const uint8_t* __restrict__ lmask, const int32_t* __restrict__ tile_lc,
                         const int32_t* __restrict__ light_cols, const float* __restrict__ lscale,
                         const U* __restrict__ u, int64_t nnz, int64_t ntiles, G* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  constexpr bool kPrefetch = sizeof(V) == 4;  // FP64 stages are too large to double in registers
  LightStage<SV> nxt;
  if (kPrefetch) load_light_stage<SV>(row, val, lmask, tile_lc, warp, ntiles, nnz, lane, nxt);
  for (int64_t t = warp; t < ntiles; t += nwarps) {  // warp-uniform
    LightStage<SV> cur;
    if (kPrefetch) {
      cur = nxt;
      load_light_stage<SV>(row, val, lmask, tile_lc, t + nwarps, ntiles, nnz, lane, nxt);  // next tile in flight
    } else {
      load_light_stage<SV>(row, val, lmask, tile_lc, t, ntiles, nnz, lane, cur);
    }
    light_tile<V, U, G, SV>(cur, t, nnz, light_cols, lscale, u, out, lane);
  }
}

// The light tiles as a shared pool: warps take kLightChunk tiles at a time
// from a global counter (reset to 0 by k_pairs_to_gacc after every launch),
// the next tile's loads in flight while one is summed.
constexpr int kLightChunk = 4;

template <typename V, typename U, typename G, typename SV>
__device__ __forceinline__ void light_pool(const int32_t* __restrict__ row, const SV* __restrict__ val,
                                           const uint8_t* __restrict__ lmask, const int32_t* __restrict__ tile_lc,
                                           const int32_t* __restrict__ light_cols,
                                           const float* __restrict__ lscale, const U* __restrict__ u, int64_t nnz,
                                           int64_t ntiles, G* __restrict__ out, unsigned int* counter) {
  const int lane = threadIdx.x & 31;
  auto grab = [&](int64_t& t, int64_t& t_end) {
    unsigned int b = 0;
    if (lane == 0) b = atomicAdd(counter, (unsigned int)kLightChunk);
    b = __shfl_sync(0xffffffffu, b, 0);
    t = (int64_t)b;
    t_end = t + kLightChunk < ntiles ? t + kLightChunk : ntiles;
  };
  int64_t t, t_end;
  grab(t, t_end);
  if (t >= ntiles) return;
  LightStage<SV> nxt;
  load_light_stage<SV>(row, val, lmask, tile_lc, t, ntiles, nnz, lane, nxt);
  for (;;) {  // warp-uniform
    const LightStage<SV> cur = nxt;
    const int64_t tc = t;
    if (++t >= t_end) grab(t, t_end);
    const bool more = t < ntiles;
    if (more) load_light_stage<SV>(row, val, lmask, tile_lc, t, ntiles, nnz, lane, nxt);  // next tile in flight
    light_tile<V, U, G, SV>(cur, tc, nnz, light_cols, lscale, u, out, lane);
    if (!more) break;
  }
}

// Both streaming passes in one persistent kernel, one CTA per SM: warps
// 0 .. SLAB_WARPS - 1 run the CTA's row-slab tiles (u slab in shared memory,
// synchronised on named barrier 1), the other warps take light tiles from
// the pool, and the slab warps join the pool when their tiles are done.  The
// slab pass waits on memory latency and the light pass on L1 gathers, so
// running them side by side on every SM overlaps the two.
template <typename V, typename U, typename G, int THREADS, int SLAB_WARPS, int DEPTH, int ITEMS, typename SV>
__global__ void __launch_bounds__(THREADS, 1)
    k_propose_fused(const uint16_t* __restrict__ s_row, const SV* __restrict__ s_val,
                    const uint8_t* __restrict__ pmask, const uint32_t* __restrict__ pair_col,
                    const uint32_t* __restrict__ tile_start, const uint32_t* __restrict__ tile_end,
                    const uint32_t* __restrict__ tile_pair, const int32_t* __restrict__ tile_slab,
                    const int32_t* __restrict__ slab_tile_begin, const int32_t* __restrict__ cta_tile_begin,
                    const int32_t* __restrict__ lrow, const SV* __restrict__ lval,
                    const uint8_t* __restrict__ lmask, const int32_t* __restrict__ tile_lc,
                    const int32_t* __restrict__ light_cols, const float* __restrict__ lscale, int64_t lnnz,
                    int64_t lntiles, unsigned int* counter, const U* __restrict__ u, int64_t n, int32_t slab_rows,
                    G* __restrict__ gacc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  U* s_u = reinterpret_cast<U*>(smem_raw);
  const int warp = threadIdx.x >> 5;
  if (warp < SLAB_WARPS)
    slab_pass<V, U, G, DEPTH, ITEMS, SV, 32 * SLAB_WARPS>(
        s_row, s_val, pmask, pair_col, tile_start, tile_end, tile_pair, tile_slab, slab_tile_begin,
        cta_tile_begin[blockIdx.x], cta_tile_begin[blockIdx.x + 1], u, n, slab_rows, gacc, s_u, warp, SLAB_WARPS,
        threadIdx.x, 32 * SLAB_WARPS);
  light_pool<V, U, G, SV>(lrow, lval, lmask, tile_lc, light_cols, lscale, u, lnnz, lntiles, gacc, counter);
  // the last warp out resets the pool for the next launch: every warp has
  // taken its last tiles when it gets here (counter[1] counts the exits)
  if ((threadIdx.x & 31) == 0) {
    const unsigned int warps = gridDim.x * (THREADS / 32);
    __threadfence();  // this warp's takes from the pool are performed before its exit counts
    if (atomicAdd(counter + 1, 1u) == warps - 1) {
      counter[0] = 0u;
      counter[1] = 0u;
    }
  }
}

// index-only storage: g_j of every heavy column times the column's value
// (the row-slab pass adds the sums of u over the column's rows)
template <typename G>
__global__ void k_scale_heavy(const int32_t* __restrict__ heavy_cols, int64_t nheavy,
                              const float* __restrict__ col_val, G* __restrict__ gacc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nheavy; h += stride) {
    const int32_t j = heavy_cols[h];
    gacc[j] *= (G)col_val[j];
  }
}

template <typename G, typename SV>
static int scale_heavy(gencd_problem* p) {
  ProposePlan& P = p->plan;
  if (!std::is_same<SV, NoVal>::value || P.nheavy == 0) return GENCD_OK;
  cudaEvent_t e = nullptr;
  prof_begin(p, K_SCALE_HEAVY, &e);
  k_scale_heavy<G><<<grid_for(P.nheavy, kThreads, p->num_sms * 8), kThreads, 0, p->stream>>>(
      P.heavy_cols, P.nheavy, p->col_val, (G*)p->gnat);
  prof_end(p, e);
  GENCD_CUDA_TRY(cudaGetLastError());
  return GENCD_OK;
}

// the two streaming passes for one value storage SV (V compute type, U type
// of u, G accumulator)
constexpr int kFusedThreads = 1024;
// candidate splits of the fused kernel's 32 warps: warps that start on the
// row slabs (the rest start on the light pool); the plan's autotuner times
// each, and the two separate kernels, on the problem at hand
constexpr int kFusedSplits[] = {20, 24, 28, 31};
constexpr int kNumFusedSplits = 4;

template <typename V, typename U, typename G, typename SV, int DEPTH, int ITEMS, int SW>
static void launch_fused(gencd_problem* p, const void* u_vec, size_t smem) {
  ProposePlan& P = p->plan;
  k_propose_fused<V, U, G, kFusedThreads, SW, DEPTH, ITEMS, SV><<<P.grid, kFusedThreads, smem, p->stream>>>(
      P.s_row, (const SV*)P.s_val, P.pmask, P.pair_col, P.tile_start, P.tile_end, P.tile_pair, P.tile_slab,
      P.slab_tile_begin, P.cta_tile_begin, P.light_row, (const SV*)P.light_val, P.lmask, P.light_tile_lc,
      P.light_cols, P.light_scale, P.light_nnz, P.light_ntiles, P.light_counter, (const U*)u_vec, p->n,
      P.slab_rows, (G*)p->gnat);
}

template <typename V, typename U, typename G, typename SV, int THREADS, int DEPTH, int ITEMS>
static int launch_plan_passes(gencd_problem* p, const void* u_vec) {
  ProposePlan& P = p->plan;
  if (P.fused_split > 0) {  // both passes in one kernel
    const size_t smem = (size_t)(P.slab_rows + kSlabZeroSlot) * sizeof(U);
    cudaEvent_t e1 = nullptr;
    prof_begin(p, K_PROPOSE_FUSED, &e1);
    switch (P.fused_split) {
      case 20: launch_fused<V, U, G, SV, DEPTH, ITEMS, 20>(p, u_vec, smem); break;
      case 24: launch_fused<V, U, G, SV, DEPTH, ITEMS, 24>(p, u_vec, smem); break;
      case 28: launch_fused<V, U, G, SV, DEPTH, ITEMS, 28>(p, u_vec, smem); break;
      default: launch_fused<V, U, G, SV, DEPTH, ITEMS, 31>(p, u_vec, smem); break;
    }
    prof_end(p, e1);
    GENCD_CUDA_TRY(cudaGetLastError());
    return scale_heavy<G, SV>(p);
  }
  if (P.nlight > 0) {
    cudaEvent_t e = nullptr;
    prof_begin(p, K_PROPOSE_LIGHT, &e);
    const int grid = grid_for(P.light_ntiles * 32, kThreads, p->num_sms * 3);  // resident CTAs: persistent warps
    k_propose_light_runs<V, U, G, SV><<<grid, kThreads, 0, p->stream>>>(
        P.light_row, (const SV*)P.light_val, P.lmask, P.light_tile_lc, P.light_cols, P.light_scale,
        (const U*)u_vec, P.light_nnz, P.light_ntiles, (G*)p->gnat);
    prof_end(p, e);
    GENCD_CUDA_TRY(cudaGetLastError());
  }
  if (P.nheavy > 0) {
    const size_t smem = (size_t)(P.slab_rows + kSlabZeroSlot) * sizeof(U);
    cudaEvent_t e1 = nullptr;
    prof_begin(p, K_PROPOSE_SLABS, &e1);
    k_propose_slabs<V, U, G, THREADS, DEPTH, ITEMS, SV><<<P.grid, THREADS, smem, p->stream>>>(
        P.s_row, (const SV*)P.s_val, P.pmask, P.pair_col, P.tile_start, P.tile_end, P.tile_pair, P.tile_slab,
        P.slab_tile_begin, P.cta_tile_begin, (const U*)u_vec, p->n, P.slab_rows, (G*)p->gnat);
    prof_end(p, e1);
    GENCD_CUDA_TRY(cudaGetLastError());
  }
  return scale_heavy<G, SV>(p);
}

template <typename V, typename U, typename G, typename SV, int THREADS, int DEPTH, int ITEMS>
static int set_slab_smem(const ProposePlan& P) {
  const int smem = (int)((size_t)(P.slab_rows + kSlabZeroSlot) * sizeof(U));
  GENCD_CUDA_TRY(cudaFuncSetAttribute(k_propose_slabs<V, U, G, THREADS, DEPTH, ITEMS, SV>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  if (P.light_counter) {
    GENCD_CUDA_TRY(cudaFuncSetAttribute(k_propose_fused<V, U, G, kFusedThreads, 31, DEPTH, ITEMS, SV>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    GENCD_CUDA_TRY(cudaFuncSetAttribute(k_propose_fused<V, U, G, kFusedThreads, 20, DEPTH, ITEMS, SV>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    GENCD_CUDA_TRY(cudaFuncSetAttribute(k_propose_fused<V, U, G, kFusedThreads, 24, DEPTH, ITEMS, SV>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    GENCD_CUDA_TRY(cudaFuncSetAttribute(k_propose_fused<V, U, G, kFusedThreads, 28, DEPTH, ITEMS, SV>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  }
  return GENCD_OK;
}

#define GENCD_PLAN_F64 double, double, double, double, kSlabThreadsF64, 0, kSlabItemsF64
#define GENCD_PLAN_F32(SV) float, float, float, SV, kSlabThreadsF32, 1, kSlabItemsF32

int launch_propose_plan(gencd_problem* p, const void* u_vec) {
  if (p->precision == GENCD_F64) return launch_plan_passes<GENCD_PLAN_F64>(p, u_vec);
  if (p->vmode == kValBf16) return launch_plan_passes<GENCD_PLAN_F32(__nv_bfloat16)>(p, u_vec);
  if (p->vmode == kValNone) return launch_plan_passes<GENCD_PLAN_F32(NoVal)>(p, u_vec);
  return launch_plan_passes<GENCD_PLAN_F32(float)>(p, u_vec);
}

// ---------------------------------------------------------------------------
// building the plan (once per problem)

__global__ void k_plan_classify(const int64_t* __restrict__ col_ptr, int64_t k, int64_t hmin,
                                uint32_t* __restrict__ hid, uint32_t* __restrict__ lid,
                                uint32_t* __restrict__ hoff, uint32_t* __restrict__ loff) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= k; j += stride) {
    uint32_t len = j < k ? (uint32_t)(col_ptr[j + 1] - col_ptr[j]) : 0u;
    const bool heavy = len > 0 && (int64_t)len >= hmin;
    const bool light = len > 0 && !heavy;
    hid[j] = heavy;
    lid[j] = light;
    hoff[j] = heavy ? len : 0u;
    loff[j] = light ? len : 0u;
  }
}

__global__ void k_plan_columns(const int64_t* __restrict__ col_ptr, int64_t k, int64_t hmin,
                               const uint32_t* __restrict__ hid, const uint32_t* __restrict__ lid,
                               const uint32_t* __restrict__ loff, int32_t* __restrict__ heavy_cols,
                               int32_t* __restrict__ light_cols, int64_t* __restrict__ light_col_ptr) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += stride) {
    const int64_t len = col_ptr[j + 1] - col_ptr[j];
    if (len <= 0) continue;
    if (len >= hmin) {
      heavy_cols[hid[j]] = (int32_t)j;
    } else {
      light_cols[lid[j]] = (int32_t)j;
      light_col_ptr[lid[j]] = loff[j];
    }
  }
}

template <typename V>
__global__ void k_plan_copy_light(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                                  const V* __restrict__ val, int64_t k, int64_t hmin,
                                  const uint32_t* __restrict__ loff, int32_t* __restrict__ lrow,
                                  V* __restrict__ lval) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = warp; j < k; j += nwarps) {
    const int64_t s = col_ptr[j], len = col_ptr[j + 1] - s;
    if (len <= 0 || len >= hmin) continue;
    for (int64_t t = lane; t < len; t += 32) {
      lrow[loff[j] + t] = row_idx[s + t];
      lval[loff[j] + t] = val[s + t];
    }
  }
}

// value storage of the plan: bfloat16 copies (the values are bfloat16-exact)
__global__ void k_plan_to_bf16(const float* __restrict__ src, int64_t m, __nv_bfloat16* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
    dst[i] = __float2bfloat16_rn(src[i]);
}

template <typename T>
__global__ void k_plan_fill(T* __restrict__ a, int64_t m, T v) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) a[i] = v;
}

// index-only storage: scale[c] = col_val[cols[c]]
__global__ void k_plan_gather_scales(const int32_t* __restrict__ cols, int64_t m, const float* __restrict__ col_val,
                                     float* __restrict__ scale) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < m; c += stride) scale[c] = col_val[cols[c]];
}

// bit p % 32 of word p / 32 (= bit p % 8 of byte p / 8) for the first entry p of
// every light column
__global__ void k_plan_light_starts(const int64_t* __restrict__ light_col_ptr, int64_t nlight,
                                    uint32_t* __restrict__ words) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nlight; c += stride) {
    const int64_t p = light_col_ptr[c];
    atomicOr(words + (p >> 5), 1u << (p & 31));
  }
}

// heavy entry e (column-major order): key = slab, plus its row, value, heavy id
template <typename V>
__global__ void k_plan_heavy_entries(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                                     const V* __restrict__ val, int64_t k, int64_t hmin,
                                     const uint32_t* __restrict__ hid, const uint32_t* __restrict__ hoff,
                                     int32_t slab_rows, uint32_t* __restrict__ keys, uint32_t* __restrict__ order,
                                     uint32_t* __restrict__ hrow, uint32_t* __restrict__ hh, V* __restrict__ hval) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = warp; j < k; j += nwarps) {
    const int64_t s = col_ptr[j], len = col_ptr[j + 1] - s;
    if (len <= 0 || len < hmin) continue;
    for (int64_t t = lane; t < len; t += 32) {
      const uint32_t e = hoff[j] + (uint32_t)t;
      const int32_t r = row_idx[s + t];
      keys[e] = (uint32_t)(r / slab_rows);
      order[e] = e;
      hrow[e] = (uint32_t)r;
      hh[e] = hid[j];
      hval[e] = val[s + t];
    }
  }
}

// entries in slab order -> padded slab arrays, and the flag "a pair starts here"
template <typename V>
__global__ void k_plan_fill_slabs(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ se, int64_t E,
                                  const int64_t* __restrict__ slab_begin, const int64_t* __restrict__ pad_off,
                                  int32_t slab_rows, const uint32_t* __restrict__ hrow,
                                  const uint32_t* __restrict__ hh, const V* __restrict__ hval,
                                  uint16_t* __restrict__ s_row, V* __restrict__ s_val,
                                  uint32_t* __restrict__ newpair, uint32_t* __restrict__ pmask_words) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E; i += stride) {
    const uint32_t r = sk[i], e = se[i];
    const int64_t ip = pad_off[r] + (i - slab_begin[r]);
    s_row[ip] = (uint16_t)(hrow[e] - r * (uint32_t)slab_rows);
    s_val[ip] = hval[e];
    const bool starts = i == slab_begin[r] || hh[e] != hh[se[i - 1]];
    newpair[i] = starts ? 1u : 0u;
    // bit ip % 32 of word ip / 32 = bit ip % 8 of byte ip / 8 (little-endian)
    if (starts) atomicOr(pmask_words + (ip >> 5), 1u << (ip & 31));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) newpair[E] = 0u;
}

__global__ void k_plan_fill_pairs(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ se, int64_t E,
                                  const int64_t* __restrict__ slab_begin, const int64_t* __restrict__ pad_off,
                                  const uint32_t* __restrict__ hh, const uint32_t* __restrict__ pidx,
                                  uint32_t* __restrict__ pair_start, uint32_t* __restrict__ pair_h) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E; i += stride) {
    if (pidx[i + 1] == pidx[i]) continue;
    const uint32_t q = pidx[i], r = sk[i];
    pair_start[q] = (uint32_t)(pad_off[r] + (i - slab_begin[r]));
    pair_h[q] = hh[se[i]];
  }
}

__global__ void k_plan_pair_cols(const uint32_t* __restrict__ pair_h, int64_t npairs,
                                 const int32_t* __restrict__ heavy_cols, uint32_t* __restrict__ pair_col) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < npairs; q += stride)
    pair_col[q] = (uint32_t)heavy_cols[pair_h[q]];
}

__global__ void k_plan_tiles(const int32_t* __restrict__ slab_tile_begin, const int64_t* __restrict__ pad_off,
                             int32_t R, int64_t T, int64_t tile, const uint32_t* __restrict__ pair_start,
                             int64_t npairs,
                             uint32_t* __restrict__ tile_start, uint32_t* __restrict__ tile_end,
                             uint32_t* __restrict__ tile_pair, int32_t* __restrict__ tile_slab) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += stride) {
    int32_t lo = 0, hi = R - 1;  // slab: last r with slab_tile_begin[r] <= t
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (slab_tile_begin[mid] <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    const int32_t r = lo;
    const int64_t s = pad_off[r] + (t - slab_tile_begin[r]) * tile;
    const int64_t e = s + tile < pad_off[r + 1] ? s + tile : pad_off[r + 1];
    tile_start[t] = (uint32_t)s;
    tile_end[t] = (uint32_t)e;
    tile_slab[t] = r;
    int64_t a = 0, b = npairs - 1;  // pair of the tile's first entry: last q with pair_start[q] <= s
    while (a < b) {
      const int64_t mid = (a + b + 1) >> 1;
      if ((int64_t)pair_start[mid] <= s)
        a = mid;
      else
        b = mid - 1;
    }
    tile_pair[t] = (uint32_t)a;
  }
}

void free_propose_plan(gencd_problem* p) {
  ProposePlan& P = p->plan;
  void* bufs[] = {P.light_cols, P.light_col_ptr, P.light_row, P.light_val, P.light_tile_lc, P.lmask, P.light_scale,
                  P.heavy_cols,
                  P.s_row, P.s_val, P.pmask, P.pair_col, P.tile_start,
                  P.tile_end, P.tile_pair, P.tile_slab, P.slab_tile_begin, P.cta_tile_begin, P.light_counter};
  for (void* b : bufs)
    if (b) dev_free(p, b);
  P = ProposePlan();
}

template <typename T>
static int palloc(gencd_problem* p, T** ptr, int64_t count) {
  return dev_alloc(p, ptr, (size_t)(count > 0 ? count : 1));
}

// scratch that is freed when the build returns
struct Scratch {
  gencd_problem* p;
  std::vector<void*> bufs;
  explicit Scratch(gencd_problem* q) : p(q) {}
  template <typename T>
  int get(T** ptr, int64_t count) {
    int rc = palloc(p, ptr, count);
    if (rc == GENCD_OK) bufs.push_back(*ptr);
    return rc;
  }
  ~Scratch() {
    for (void* b : bufs) dev_free(p, b);
  }
};

static int build_plan_impl(gencd_problem* p, Scratch& S) {
  ProposePlan& P = p->plan;
  const int64_t k = p->k, n = p->n;
  const bool f64 = p->precision == GENCD_F64;
  const size_t vsz = f64 ? 8 : 4;
  const int g = p->num_sms * 8;
  cudaStream_t st = p->stream;
  P.slab_rows = (int32_t)(kSlabBytes / (f64 ? 8 : 4));
  P.nslabs = (int32_t)((n + P.slab_rows - 1) / P.slab_rows);
  // one slab: every non-empty column reads u from shared memory; otherwise a
  // column takes this layout once it averages >= 2 entries per slab in FP32
  // arithmetic (the fused pass and the warp reduction of the partials make
  // that pay: fewer entries left to the light pass's gathers of u from L2,
  // one L1 wavefront each) and >= 8 in FP64 (two separate passes)
  P.heavy_min = P.nslabs == 1 ? 1 : (f64 ? 8LL : 2LL) * P.nslabs;

  // classify, number and offset the columns
  uint32_t *hid, *lid, *hoff, *loff, *tmp;
  GENCD_TRY(S.get(&hid, k + 1));
  GENCD_TRY(S.get(&lid, k + 1));
  GENCD_TRY(S.get(&hoff, k + 1));
  GENCD_TRY(S.get(&loff, k + 1));
  GENCD_TRY(S.get(&tmp, scan_tmp_words(k + 1)));
  k_plan_classify<<<grid_for(k + 1, kThreads, g), kThreads, 0, st>>>(p->col_ptr, k, P.heavy_min, hid, lid, hoff,
                                                                      loff);
  GENCD_TRY(exclusive_scan(p, hid, hid, k + 1, tmp));
  GENCD_TRY(exclusive_scan(p, lid, lid, k + 1, tmp));
  GENCD_TRY(exclusive_scan(p, hoff, hoff, k + 1, tmp));
  GENCD_TRY(exclusive_scan(p, loff, loff, k + 1, tmp));
  uint32_t tot[4];
  GENCD_CUDA_TRY(cudaMemcpyAsync(&tot[0], hid + k, 4, cudaMemcpyDeviceToHost, st));
  GENCD_CUDA_TRY(cudaMemcpyAsync(&tot[1], lid + k, 4, cudaMemcpyDeviceToHost, st));
  GENCD_CUDA_TRY(cudaMemcpyAsync(&tot[2], hoff + k, 4, cudaMemcpyDeviceToHost, st));
  GENCD_CUDA_TRY(cudaMemcpyAsync(&tot[3], loff + k, 4, cudaMemcpyDeviceToHost, st));
  GENCD_CUDA_TRY(cudaStreamSynchronize(st));
  P.nheavy = tot[0];
  P.nlight = tot[1];
  const int64_t E = tot[2];
  P.light_nnz = tot[3];

  GENCD_TRY(palloc(p, &P.heavy_cols, P.nheavy));
  GENCD_TRY(palloc(p, &P.light_cols, P.nlight));
  GENCD_TRY(palloc(p, &P.light_col_ptr, P.nlight + 1));
  k_plan_columns<<<grid_for(k, kThreads, g), kThreads, 0, st>>>(p->col_ptr, k, P.heavy_min, hid, lid, loff,
                                                                 P.heavy_cols, P.light_cols, P.light_col_ptr);
  GENCD_CUDA_TRY(cudaGetLastError());

  // light columns: compact CSC copy and its tile map
  if (P.nlight > 0) {
    const int64_t lpad = ((P.light_nnz + kPadNnz - 1) / kPadNnz) * kPadNnz + kPadNnz;
    GENCD_TRY(palloc(p, &P.light_row, lpad));
    GENCD_TRY(palloc(p, (char**)&P.light_val, lpad * (int64_t)vsz));
    GENCD_CUDA_TRY(cudaMemsetAsync(P.light_row, 0, sizeof(int32_t) * lpad, st));
    GENCD_CUDA_TRY(cudaMemsetAsync(P.light_val, 0, vsz * lpad, st));
    if (p->vmode == kValNone) {  // padding has no value to zero it: it gathers u[n] = 0 instead
      k_plan_fill<int32_t><<<grid_for(lpad, kThreads, g), kThreads, 0, st>>>(P.light_row, lpad, (int32_t)n);
      GENCD_CUDA_TRY(cudaGetLastError());
    }
    const int64_t ln = P.light_nnz;
    GENCD_CUDA_TRY(cudaMemcpyAsync(P.light_col_ptr + P.nlight, &ln, 8, cudaMemcpyHostToDevice, st));
    if (f64)
      k_plan_copy_light<double><<<grid_for(k * 32, kThreads, g), kThreads, 0, st>>>(
          p->col_ptr, p->row_idx, (const double*)p->val, k, P.heavy_min, loff, P.light_row, (double*)P.light_val);
    else
      k_plan_copy_light<float><<<grid_for(k * 32, kThreads, g), kThreads, 0, st>>>(
          p->col_ptr, p->row_idx, (const float*)p->val, k, P.heavy_min, loff, P.light_row, (float*)P.light_val);
    GENCD_CUDA_TRY(cudaGetLastError());
    if (!f64 && p->vmode != kValPlain) {  // bfloat16 copy, or no values and a scale per column
      if (p->vmode == kValBf16) {
        __nv_bfloat16* b16 = nullptr;
        GENCD_TRY(palloc(p, &b16, lpad));
        k_plan_to_bf16<<<grid_for(lpad, kThreads, g), kThreads, 0, st>>>((const float*)P.light_val, lpad, b16);
        GENCD_CUDA_TRY(cudaStreamSynchronize(st));
        dev_free(p, P.light_val);
        P.light_val = b16;
      } else {
        GENCD_CUDA_TRY(cudaStreamSynchronize(st));
        dev_free(p, P.light_val);
        P.light_val = nullptr;
        GENCD_TRY(palloc(p, &P.light_scale, P.nlight));
        k_plan_gather_scales<<<grid_for(P.nlight, kThreads, g), kThreads, 0, st>>>(P.light_cols, P.nlight, p->col_val,
                                                                                    P.light_scale);
      }
      GENCD_CUDA_TRY(cudaGetLastError());
    }
    P.light_ntiles = (P.light_nnz + kLightTile - 1) / kLightTile;
    GENCD_TRY(palloc(p, &P.light_tile_lc, P.light_ntiles + 1));
    GENCD_TRY(launch_tile_map_of(p, P.light_col_ptr, P.nlight, P.light_ntiles, P.light_tile_lc, kLightTile));
    const int64_t lwords = (lpad + 31) / 32;  // start bits, one byte per 8 entries
    GENCD_TRY(palloc(p, (uint32_t**)&P.lmask, lwords));
    GENCD_CUDA_TRY(cudaMemsetAsync(P.lmask, 0, 4 * (size_t)lwords, st));
    k_plan_light_starts<<<grid_for(P.nlight, kThreads, g), kThreads, 0, st>>>(P.light_col_ptr, P.nlight,
                                                                              (uint32_t*)P.lmask);
    GENCD_CUDA_TRY(cudaGetLastError());
  }
  if (P.nheavy == 0) return GENCD_OK;

  // heavy entries grouped by slab (stable: column-major order kept inside a slab)
  uint32_t *keys, *order, *ka, *va, *hrow, *hh, *stmp;
  char* hval;
  GENCD_TRY(S.get(&keys, E));
  GENCD_TRY(S.get(&order, E));
  GENCD_TRY(S.get(&ka, E));
  GENCD_TRY(S.get(&va, E));
  GENCD_TRY(S.get(&hrow, E));
  GENCD_TRY(S.get(&hh, E));
  GENCD_TRY(S.get(&hval, E * (int64_t)vsz));
  GENCD_TRY(S.get(&stmp, (int64_t)radix_tmp_words(E)));
  if (f64)
    k_plan_heavy_entries<double><<<grid_for(k * 32, kThreads, g), kThreads, 0, st>>>(
        p->col_ptr, p->row_idx, (const double*)p->val, k, P.heavy_min, hid, hoff, P.slab_rows, keys, order, hrow,
        hh, (double*)hval);
  else
    k_plan_heavy_entries<float><<<grid_for(k * 32, kThreads, g), kThreads, 0, st>>>(
        p->col_ptr, p->row_idx, (const float*)p->val, k, P.heavy_min, hid, hoff, P.slab_rows, keys, order, hrow,
        hh, (float*)hval);
  GENCD_CUDA_TRY(cudaGetLastError());
  bool in_alt = false;
  GENCD_TRY(radix_sort_with_tmp(p, keys, order, E, bits_for_max(P.nslabs - 1), ka, va, stmp, &in_alt));
  const uint32_t* sk = in_alt ? ka : keys;
  const uint32_t* se = in_alt ? va : order;

  // slab offsets (unpadded from the sorted keys; padded to 8 entries on the host)
  const int R = P.nslabs;
  int64_t *slab_begin, *pad_off;
  GENCD_TRY(S.get(&slab_begin, R + 1));
  GENCD_TRY(S.get(&pad_off, R + 1));
  GENCD_TRY(lower_bounds_u32_to_i64(p, sk, E, R, slab_begin));
  std::vector<int64_t> hb(R + 1), hp(R + 1);
  GENCD_CUDA_TRY(cudaMemcpyAsync(hb.data(), slab_begin, 8 * (R + 1), cudaMemcpyDeviceToHost, st));
  GENCD_CUDA_TRY(cudaStreamSynchronize(st));
  hp[0] = 0;
  for (int r = 0; r < R; ++r) hp[r + 1] = hp[r] + ((hb[r + 1] - hb[r] + kSlabPad - 1) / kSlabPad) * kSlabPad;
  P.entries = hp[R];
  if (P.entries >= (int64_t(1) << 32)) return fail_plan("heavy entries exceed 2^32");
  GENCD_CUDA_TRY(cudaMemcpyAsync(pad_off, hp.data(), 8 * (R + 1), cudaMemcpyHostToDevice, st));

  GENCD_TRY(palloc(p, &P.s_row, P.entries + 8));
  GENCD_TRY(palloc(p, (char**)&P.s_val, (P.entries + 8) * (int64_t)vsz));
  GENCD_CUDA_TRY(cudaMemsetAsync(P.s_row, 0, 2 * (P.entries + 8), st));
  GENCD_CUDA_TRY(cudaMemsetAsync(P.s_val, 0, vsz * (P.entries + 8), st));
  if (p->vmode == kValNone) {  // padding reads the zero slot past the slab
    k_plan_fill<uint16_t><<<grid_for(P.entries + 8, kThreads, g), kThreads, 0, st>>>(P.s_row, P.entries + 8,
                                                                                     (uint16_t)P.slab_rows);
    GENCD_CUDA_TRY(cudaGetLastError());
  }
  // start bits: one byte per 8 entries, written as 32-bit words (entries + 8 bits, rounded up to words)
  const int64_t mask_words = (P.entries + 8 + 31) / 32;
  GENCD_TRY(palloc(p, (uint32_t**)&P.pmask, mask_words));
  GENCD_CUDA_TRY(cudaMemsetAsync(P.pmask, 0, 4 * (size_t)mask_words, st));
  uint32_t* pidx;
  GENCD_TRY(S.get(&pidx, E + 1));
  if (f64)
    k_plan_fill_slabs<double><<<grid_for(E, kThreads, g), kThreads, 0, st>>>(
        sk, se, E, slab_begin, pad_off, P.slab_rows, hrow, hh, (const double*)hval, P.s_row, (double*)P.s_val,
        pidx, (uint32_t*)P.pmask);
  else
    k_plan_fill_slabs<float><<<grid_for(E, kThreads, g), kThreads, 0, st>>>(
        sk, se, E, slab_begin, pad_off, P.slab_rows, hrow, hh, (const float*)hval, P.s_row, (float*)P.s_val, pidx,
        (uint32_t*)P.pmask);
  GENCD_CUDA_TRY(cudaGetLastError());
  if (!f64 && p->vmode != kValPlain) {  // bfloat16 copy, or no values and a scale per column
    if (p->vmode == kValBf16) {
      __nv_bfloat16* b16 = nullptr;
      GENCD_TRY(palloc(p, &b16, P.entries + 8));
      k_plan_to_bf16<<<grid_for(P.entries + 8, kThreads, g), kThreads, 0, st>>>((const float*)P.s_val, P.entries + 8,
                                                                                b16);
      GENCD_CUDA_TRY(cudaStreamSynchronize(st));
      dev_free(p, P.s_val);
      P.s_val = b16;
    } else {
      GENCD_CUDA_TRY(cudaStreamSynchronize(st));
      dev_free(p, P.s_val);
      P.s_val = nullptr;  // k_scale_heavy applies col_val[j] after the pass
    }
    GENCD_CUDA_TRY(cudaGetLastError());
  }
  uint32_t* ptmp;
  GENCD_TRY(S.get(&ptmp, scan_tmp_words(E + 1)));
  GENCD_TRY(exclusive_scan(p, pidx, pidx, E + 1, ptmp));
  uint32_t np32 = 0;
  GENCD_CUDA_TRY(cudaMemcpyAsync(&np32, pidx + E, 4, cudaMemcpyDeviceToHost, st));
  GENCD_CUDA_TRY(cudaStreamSynchronize(st));
  P.npairs = np32;

  // pairs: first entry and column
  uint32_t *pair_start, *pair_h;
  GENCD_TRY(S.get(&pair_start, P.npairs + 1));
  GENCD_TRY(S.get(&pair_h, P.npairs));
  k_plan_fill_pairs<<<grid_for(E, kThreads, g), kThreads, 0, st>>>(sk, se, E, slab_begin, pad_off, hh, pidx,
                                                                    pair_start, pair_h);
  const uint32_t ent32 = (uint32_t)P.entries;
  GENCD_CUDA_TRY(cudaMemcpyAsync(pair_start + P.npairs, &ent32, 4, cudaMemcpyHostToDevice, st));
  GENCD_TRY(palloc(p, &P.pair_col, P.npairs));
  k_plan_pair_cols<<<grid_for(P.npairs, kThreads, g), kThreads, 0, st>>>(pair_h, P.npairs, P.heavy_cols,
                                                                          P.pair_col);
  GENCD_CUDA_TRY(cudaGetLastError());

  // tiles inside each slab, and contiguous runs of tiles per CTA
  std::vector<int32_t> tb(R + 1);
  tb[0] = 0;
  const int64_t tile = 32LL * (f64 ? kSlabItemsF64 : kSlabItemsF32);  // the kernel's tile
  for (int r = 0; r < R; ++r) tb[r + 1] = tb[r] + (int32_t)((hp[r + 1] - hp[r] + tile - 1) / tile);
  P.ntiles = tb[R];
  GENCD_TRY(palloc(p, &P.slab_tile_begin, R + 1));
  GENCD_TRY(palloc(p, &P.tile_start, P.ntiles));
  GENCD_TRY(palloc(p, &P.tile_end, P.ntiles));
  GENCD_TRY(palloc(p, &P.tile_pair, P.ntiles));
  GENCD_TRY(palloc(p, &P.tile_slab, P.ntiles));
  GENCD_CUDA_TRY(cudaMemcpyAsync(P.slab_tile_begin, tb.data(), 4 * (R + 1), cudaMemcpyHostToDevice, st));
  k_plan_tiles<<<grid_for(P.ntiles, kThreads, g), kThreads, 0, st>>>(P.slab_tile_begin, pad_off, R, P.ntiles, tile,
                                                                      pair_start, P.npairs, P.tile_start,
                                                                      P.tile_end, P.tile_pair, P.tile_slab);
  GENCD_CUDA_TRY(cudaGetLastError());
  P.grid = p->num_sms;
  // both passes may run in one kernel when there are light and heavy columns
  // (FP32 arithmetic: FP64 stages do not fit the fused kernel's registers);
  // the autotuner below decides
  P.fused_split = 0;
  if (!f64 && P.nlight > 0 && P.nheavy > 0) {
    GENCD_TRY(palloc(p, &P.light_counter, 2));  // tiles taken, warps finished
    GENCD_CUDA_TRY(cudaMemsetAsync(P.light_counter, 0, 2 * sizeof(unsigned int), st));
  }
  std::vector<int32_t> ctb(P.grid + 1);
  for (int b = 0; b <= P.grid; ++b) ctb[b] = (int32_t)((int64_t)b * P.ntiles / P.grid);
  GENCD_TRY(palloc(p, &P.cta_tile_begin, P.grid + 1));
  GENCD_CUDA_TRY(cudaMemcpyAsync(P.cta_tile_begin, ctb.data(), 4 * (P.grid + 1), cudaMemcpyHostToDevice, st));
  if (f64)
    GENCD_TRY(set_slab_smem<GENCD_PLAN_F64>(P));
  else if (p->vmode == kValBf16)
    GENCD_TRY(set_slab_smem<GENCD_PLAN_F32(__nv_bfloat16)>(P));
  else if (p->vmode == kValNone)
    GENCD_TRY(set_slab_smem<GENCD_PLAN_F32(NoVal)>(P));
  else
    GENCD_TRY(set_slab_smem<GENCD_PLAN_F32(float)>(P));
  GENCD_CUDA_TRY(cudaStreamSynchronize(st));  // scratch is freed on return
  p->prof.launches[K_SETUP] += 10;
  return GENCD_OK;
}

int build_propose_plan(gencd_problem* p) {
  free_propose_plan(p);
  int rc;
  {
    Scratch S(p);
    rc = build_plan_impl(p, S);
    if (rc != GENCD_OK) cudaStreamSynchronize(p->stream);
  }
  if (rc != GENCD_OK) {
    free_propose_plan(p);
    return rc;
  }
  p->plan.built = true;
  return tune_propose_plan(p);
}

// Autotuner of the streaming propose: times the separate light and slab
// kernels and every split of the fused kernel on this problem (three
// launches each, CUDA events, u as it stands) and keeps the fastest.  All
// candidates compute the same sums; the scratch they leave is cleared.
int tune_propose_plan(gencd_problem* p) {
  ProposePlan& P = p->plan;
  P.tuned_ms[0] = -1.0;
  if (!P.built || !P.light_counter) return GENCD_OK;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  GENCD_CUDA_TRY(cudaEventCreate(&ev[0]));
  if (cudaEventCreate(&ev[1]) != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    return fail_plan("cudaEventCreate failed");
  }
  const bool prof = p->prof.enabled;
  p->prof.enabled = false;
  int rc = GENCD_OK;
  float best_ms = 0.f;
  int best = 0;
  for (int c = 0; c <= kNumFusedSplits && rc == GENCD_OK; ++c) {
    P.fused_split = c == 0 ? 0 : kFusedSplits[c - 1];
    if ((rc = launch_propose_plan(p, p->u)) != GENCD_OK) break;  // warm-up
    cudaEventRecord(ev[0], p->stream);
    for (int r = 0; r < 3 && rc == GENCD_OK; ++r) rc = launch_propose_plan(p, p->u);
    cudaEventRecord(ev[1], p->stream);
    if (rc != GENCD_OK || cudaEventSynchronize(ev[1]) != cudaSuccess) {
      rc = rc != GENCD_OK ? rc : fail_plan("autotuning the streaming propose failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    P.tuned_ms[c] = ms / 3.0;
    if (c == 0 || ms < best_ms) best_ms = ms, best = P.fused_split;
  }
  p->prof.enabled = prof;
  P.fused_split = best;
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (rc != GENCD_OK) return rc;
  // the candidates' sums are scratch: the hot path expects them zero
  const size_t gsz = p->precision == GENCD_F64 ? sizeof(double) : sizeof(float);
  GENCD_CUDA_TRY(cudaMemsetAsync(p->gnat, 0, gsz * (size_t)p->k, p->stream));
  return GENCD_OK;
}

}  // namespace gencd
