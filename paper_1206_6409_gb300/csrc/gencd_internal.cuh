// gencd_internal.cuh -- internal declarations of the GB300 GenCD library.
//
// Device layout of one problem (all arrays owned by the library):
//   CSC   col_ptr int64[k+1], row_idx int32[nnz_pad], val V[nnz_pad]
//         (nnz_pad = nnz rounded up to 64; the pad holds row 0 / value 0)
//   rows  y f64[n], z f64[n], u U[n]           (u_i = l'(y_i, z_i))
//   cols  w f64[k], c f64[k] (c_j = ||X_j||^2 / n)
//   TG    gacc f64[k] (zero between launches), delta f64[k], phi f64[k]
//   tiles tile_col int32[ntiles+1]: column holding nnz position t * TILE
//   CSR   (built on first use) row_ptr int64[n+1], col_idx int32[nnz], csr_val V[nnz]
// V = U = double in FP64 mode, float in FP32 mode.  z, w, the objective and
// the KKT test stay in FP64 in both modes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/gencd.h"

namespace gencd {

// ---------------------------------------------------------------------------
// error plumbing
void set_error(const std::string& msg);
const char* last_error();

#define GENCD_CUDA_TRY(expr)                                                                  \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      ::gencd::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));                \
      return GENCD_ECUDA;                                                                     \
    }                                                                                         \
  } while (0)

#define GENCD_TRY(expr)        \
  do {                         \
    int rc_ = (expr);          \
    if (rc_ < 0) return rc_;   \
  } while (0)

// ---------------------------------------------------------------------------
// tuning constants
constexpr int kItemsF64 = 4;   // nnz per lane in the streaming propose (FP64 mode)
constexpr int kItemsF32 = 8;   // nnz per lane in the streaming propose (FP32 mode)
constexpr int kPadNnz = 64;    // CSC arrays are padded to a multiple of this
constexpr int kThreads = 256;  // default CTA size
// value storage of the streaming plan in FP32 arithmetic (gencd_problem::vmode)
constexpr int kValPlain = 0;  // the storage precision's values
constexpr int kValBf16 = 1;   // bfloat16 (GENCD_BF16)
constexpr int kValNone = 2;   // index only, one value per column (GENCD_BINARY)
// the single-CTA plan of an update list (lengths, prefix, w) takes lists of at
// most kListPlanMax entries
constexpr int kListPlanThreads = 1024;
constexpr int kListPlanPer = 4;
constexpr int64_t kListPlanMax = (int64_t)kListPlanThreads * kListPlanPer;
constexpr int32_t kMaxShotgunBlocks = 1024;  // column blocks of block Shotgun (one selection CTA)
constexpr int kScalars = 16;  // device scalars of a problem (dscal / hpin)

// kernel ids for launch counting / profiling
enum KernelId {
  K_PROPOSE_ALL = 0,  // streaming partial sums of X^T u over all columns
  K_FINALIZE,         // g, delta, phi, KKT per column
  K_ACCEPT,           // Thread-Greedy / Greedy argmin per partition
  K_UPDATE,           // atomic scatter into z
  K_REFRESH,          // u refresh on touched rows
  K_PROPOSE_LIST,     // propose over a selected list J
  K_COLOR_ITER,       // fused Coloring iteration
  K_OBJECTIVE,        // objective reduction
  K_SETUP,            // one-time and selection kernels
  K_PROPOSE_LIGHT,    // streaming propose: lane-segmented pass over the light columns
  K_PROPOSE_SLABS,    // streaming propose: row-slab pass over the heavy columns
  K_SCALE_HEAVY,      // streaming propose, index-only storage: heavy columns' g_j times their value
  K_PROPOSE_FUSED,    // streaming propose: row-slab and light passes in one kernel
  K_NUM
};

struct Profiler {
  bool enabled = false;
  std::vector<cudaEvent_t> pool;       // pairs (start, stop)
  std::vector<int> pending_id;         // kernel id of each recorded pair
  size_t used = 0;
  double ms[K_NUM] = {0};
  int64_t launches[K_NUM] = {0};       // kernel launches, counted whether or not profiling is on
  int64_t calls[K_NUM] = {0};          // timed invocations (one event pair each)
};

// A CSC matrix as the streaming propose sees it (cmap: column map, may be null)
struct CscView {
  const int64_t* col_ptr;
  const int32_t* row_idx;
  const void* val;
  const int32_t* tile_col;
  int64_t nnz;
  int64_t ntiles;
  const int32_t* cmap;
};

// Row-slab plan of the streaming propose.  Rows are cut into slabs of
// slab_rows rows, small enough that a slab of u fits in shared memory.
// Heavy columns (>= heavy_min non-zeros) are stored slab by slab: for each
// slab, the entries of every heavy column with rows in it (a "pair"), row as
// a 16-bit offset inside the slab.  Each pair yields one partial sum, added
// atomically into the column's g_j (zero before the pass).  Light columns keep
// a compact CSC copy for the lane-segmented pass.
struct ProposePlan {
  bool built = false;
  int32_t slab_rows = 0, nslabs = 0;
  int64_t heavy_min = 0;
  // light columns
  int64_t nlight = 0, light_nnz = 0, light_ntiles = 0;
  int32_t* light_cols = nullptr;
  int64_t* light_col_ptr = nullptr;
  int32_t* light_row = nullptr;
  void* light_val = nullptr;
  int32_t* light_tile_lc = nullptr;  // light column of each 256-entry tile's first entry
  float* light_scale = nullptr;      // index-only storage: the value of light column lc
  uint8_t* lmask = nullptr;          // per 8 light entries: bit i = entry 8g + i starts a column
  // heavy columns
  int64_t nheavy = 0, entries = 0, npairs = 0, ntiles = 0;
  int32_t* heavy_cols = nullptr;   // original column of heavy id h
  uint16_t* s_row = nullptr;       // slab-local row of each entry
  void* s_val = nullptr;           // value of each entry (padding: 0)
  uint8_t* pmask = nullptr;        // per 8 entries: bit i = entry 8g + i starts a pair (pairs in entry order)
  uint32_t* pair_col = nullptr;    // the column j of each pair (its run sums go to g_j)
  uint32_t* tile_start = nullptr;  // tiles of 32*ITEMS entries inside one slab
  uint32_t* tile_end = nullptr;
  uint32_t* tile_pair = nullptr;   // pair holding the tile's first entry
  int32_t* tile_slab = nullptr;
  int32_t* slab_tile_begin = nullptr;  // nslabs + 1
  int32_t* cta_tile_begin = nullptr;   // grid + 1
  int grid = 0;
  // both passes in one kernel (k_propose_fused) when fused_split > 0 (the
  // number of warps that start on the row slabs; 0: two kernels), chosen by
  // the plan's autotuner (tuned_ms: mean ms of the separate kernels, then of
  // each split); light tiles are taken from a pool: light_counter[0] counts
  // the tiles taken, light_counter[1] the warps finished, and the last warp
  // of a launch resets both
  int fused_split = 0;
  double tuned_ms[8] = {-1.0};
  unsigned int* light_counter = nullptr;
};

// ---------------------------------------------------------------------------
}  // namespace gencd

struct gencd_problem {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  // device memory: stream-ordered from this pool when set (problems of the
  // serving loop, which must not synchronise the device), else cudaMalloc
  cudaMemPool_t pool = nullptr;
  bool own_hpin = true;               // hpin allocated by the problem (else lent by its owner)
  cudaEvent_t ev_scalars = nullptr;   // recorded after each copy of dscal to hpin
  int64_t n = 0, k = 0, nnz = 0, nnz_pad = 0;
  int32_t loss = GENCD_LOSS_LOGISTIC;
  int32_t precision = GENCD_F64;  // arithmetic: GENCD_F64 or GENCD_F32 (BF16 and BINARY compute in FP32)
  int32_t vmode = gencd::kValPlain;     // value storage of the streaming plan
  int32_t user_precision = GENCD_F64;
  float* col_val = nullptr;       // index-only storage: the value s_j shared by column j's non-zeros
  double lambda = 0.0;
  double lambda_max = 0.0;
  gencd_params params{};
  int64_t t = 0;  // GenCD iteration counter (drives Select)
  int64_t stat_iters = 0;     // iterations since the last counter reset
  int64_t stat_host_nnz = 0;  // non-zeros streamed by full passes since the reset

  // CSC + rows + cols
  int64_t* col_ptr = nullptr;
  int32_t* row_idx = nullptr;
  void* val = nullptr;
  double* y = nullptr;
  double* z = nullptr;
  void* u = nullptr;
  double* w = nullptr;
  double* c = nullptr;
  double* ib = nullptr;     // 1 / beta_j (0 for a column without non-zeros)
  double* bj = nullptr;     // beta_j of the current beta_mode
  int32_t ib_mode = -1;     // beta_mode that ib was computed for

  // streaming propose over all columns
  int items = 4;
  int64_t ntiles = 0;
  int32_t* tile_col = nullptr;
  double* gacc = nullptr;   // FP64 sums (setup passes, power iteration)
  void* gnat = nullptr;     // sums of the hot path in the storage precision (== gacc in FP64 mode)
  double* delta = nullptr;
  double* phi = nullptr;

  // accepted / selected lists (capacity k)
  int32_t* list_j = nullptr;
  uint64_t* list_m = nullptr;   // candidate magnitude of each partition's accepted column (accept backoff)
  uint32_t* top_buf = nullptr;  // global top-|J'| Accept: sort keys and indices (6 k words)
  double* w_start = nullptr;    // w at the start of a solve (restarts of the accept backoff)
  int64_t accept_group = 1;     // Thread-Greedy partitions merged per accept group (1: none)
  double* list_d = nullptr;
  uint32_t* list_off = nullptr;  // exclusive prefix of the listed columns' nnz (k + 2)
  uint32_t* scan_tmp = nullptr;  // scratch of the prefix sum

  // Thread-Greedy partition bounds floor(b k / B), b = 0..part_B
  int64_t* part_lo = nullptr;
  int64_t part_B = 0, part_cap = 0;

  // accept candidates of (chunk, partition) pairs when partitions are few
  uint64_t* slot_m = nullptr;
  double* slot_d = nullptr;
  int32_t* slot_j = nullptr;
  int64_t slot_cap = 0;

  // FP32 mode: float copies of w, beta_j and 1/beta_j for the per-column
  // selection pass (w32[j] is 0 exactly when w[j] is); null in FP64 mode
  float* w32 = nullptr;
  float* bj32 = nullptr;
  float* ib32 = nullptr;

  // device scalars (kScalars doubles, mirrored to hpin): [0] kkt bits,
  // [1] objective, [2] loss sum, [3] l1 sum, [4] updates (int64), [5] nnz
  // processed (int64), [6] scratch, [7] max_j |g_j| of the last full
  // evaluation (bits; idle columns count as lambda), [8] the duality gap's
  // sum of conjugates, [9] the duality gap P(w) - D
  double* dscal = nullptr;
  double* red = nullptr;  // per-block partial sums (2 * kRedBlocks)
  double* hpin = nullptr; // pinned host mirror of dscal

  // selection
  int32_t* perm = nullptr;  // current epoch permutation (k, or C for Coloring)
  int64_t perm_epoch = -1;
  int64_t perm_m = 0;

  // radix sort scratch (grown on demand)
  void* sort_tmp = nullptr;
  size_t sort_tmp_bytes = 0;

  // CSR (lazy)
  int64_t* row_ptr = nullptr;
  int32_t* col_idx = nullptr;
  void* csr_val = nullptr;

  // colouring
  int32_t* color = nullptr;
  int32_t ncolors = 0;
  int32_t* color_ptr = nullptr;      // device, ncolors+1
  int32_t* cols_by_color = nullptr;  // device, k
  int32_t max_class = 0;

  // Shotgun
  double rho = 0.0;
  int64_t pstar = 0;

  // block Shotgun (Section 7): block_B contiguous column blocks, their
  // bounds (B + 1) and P*_b on the device and the host, rho_b, and the epoch
  // whose permutation each block's part of perm holds
  int32_t block_B = 0;
  int64_t* block_lo = nullptr;
  int64_t* block_P = nullptr;
  std::vector<int64_t> hblock_lo, hblock_P, hblock_epoch;
  std::vector<double> hblock_rho;

  gencd::Profiler prof;
  gencd::ProposePlan plan;
};

namespace gencd {

constexpr int kRedBlocks = 1024;

// ---- launchers (defined next to their kernels) ------------------------------
// kernels_propose.cu
int launch_propose_all(gencd_problem* p, const void* u_vec, bool u_is_double);
int launch_propose_csc(gencd_problem* p, const CscView& a, const void* u_vec, bool u_is_double);
// propose_plan.cu
int build_propose_plan(gencd_problem* p);
int launch_propose_plan(gencd_problem* p, const void* u_vec);
int tune_propose_plan(gencd_problem* p);  // picks the fastest form of the streaming propose
void free_propose_plan(gencd_problem* p);
int launch_finalize(gencd_problem* p, double lambda, bool write_steps);
int launch_finalize_accept(gencd_problem* p, int64_t B, bool want_kkt);  // Thread-Greedy / Greedy
int launch_merge_accept(gencd_problem* p, int64_t B);  // keep the best of every accept_group partitions
// Improve delta_j (Algorithm 3): refine the accepted steps D[e] of columns
// J[e] >= 0 in place (params.improve_steps Eq. 7 steps each; 0: nothing)
int launch_improve_list(gencd_problem* p, const int32_t* J, double* D, int64_t m);
int ensure_slots(gencd_problem* p, int64_t count);
// exclusive prefix sum of m uint32 (in place allowed); tmp holds scan_tmp_words(m)
int exclusive_scan(gencd_problem* p, const uint32_t* in, uint32_t* out, int64_t m, uint32_t* tmp);
int64_t scan_tmp_words(int64_t m);
size_t radix_tmp_words(int64_t m);
int radix_sort_with_tmp(gencd_problem* p, uint32_t* keys, uint32_t* vals, int64_t m, int bits,
                        uint32_t* keys_alt, uint32_t* vals_alt, uint32_t* tmp, bool* result_in_alt);
int bits_for_max(int64_t maxval);
int lower_bounds_u32_to_i64(gencd_problem* p, const uint32_t* sorted, int64_t m, int64_t count, int64_t* out);
int iota_u32(gencd_problem* p, uint32_t* a, int64_t m);
int fail_plan(const char* msg);
// tile_col[t] = column holding entry t * tile (columns without entries hold none)
int launch_tile_map_of(gencd_problem* p, const int64_t* col_ptr, int64_t k, int64_t ntiles, int32_t* tile_col,
                       int64_t tile);
int launch_propose_list(gencd_problem* p, const int32_t* J, int64_t m, double* delta, double* phi);
int launch_objective(gencd_problem* p, bool gap);  // P(w); with gap also the duality gap (after a finalize)
int launch_col_sumsq(gencd_problem* p);  // gacc_j = sum_i X_ij^2
int launch_inv_beta(gencd_problem* p);   // ib_j = 1 / beta_j for the current beta_mode
int launch_mirror_w(gencd_problem* p);   // w32 from w (FP32 mode)

// kernels_update.cu
int launch_fill_u(gencd_problem* p);
int launch_update_list(gencd_problem* p, const int32_t* J, const double* d, int64_t m, bool skip_neg);
int launch_refresh_list(gencd_problem* p, const int32_t* J, const double* d, int64_t m, bool skip_neg);
int launch_coloring_iter(gencd_problem* p, int64_t q);
int launch_csr_spmv(gencd_problem* p, const double* x, double* out);  // out = X x (FP64)

// kernels_setup.cu
int launch_col_scale(gencd_problem* p);
int launch_tile_map(gencd_problem* p);
int make_permutation(gencd_problem* p, uint64_t seed, int64_t epoch, int64_t m, int32_t* out);
int build_csr(gencd_problem* p);
int run_coloring(gencd_problem* p);
int build_color_classes(gencd_problem* p);
int launch_power_step(gencd_problem* p, const double* v, const double* dinv, double* r, double* s);
int validate_input(gencd_problem* p, int64_t* bad_col, int64_t* bad_row, int* stage);

// gencd_create with the problem's device memory taken from `pool`
// (stream-ordered on `stream`; NULL: cudaMalloc) and, when hpin is not NULL,
// its pinned scalars lent by the caller (kScalars doubles, kept until destroy)
int create_problem(gencd_problem** out, int64_t n, int64_t k, int64_t nnz, const int64_t* col_ptr,
                   const int32_t* row_idx, const void* val, int32_t val_dtype, const double* y, int32_t loss,
                   int32_t precision, int32_t memory, cudaStream_t stream, cudaMemPool_t pool, double* hpin);

// a solve driven step by step (api.cu; gencd_solve and the serving loop)
struct SolveRun {
  std::chrono::steady_clock::time_point t0;
  int64_t host_nnz = 0, iters = 0;
  double obj_start = 0.0;
  bool started = false;    // obj_start is known
  bool evaluated = true;   // hpin holds a full evaluation of the current state
  bool finishing = false;  // the final evaluation is in flight
  int status = GENCD_NOT_CONVERGED;
  int64_t B = 1;
  bool backoff = false, fused = false;
  // stall watch of the accept backoff: the lowest KKT value and objective
  // since the solve's (re)start, and the checks since either last improved
  double best_kkt = HUGE_VAL, best_obj = HUGE_VAL;
  int stall = 0;
};
int solve_begin(gencd_problem* p, SolveRun* S);
int solve_advance(gencd_problem* p, SolveRun* S);  // 1: more work enqueued, 0: done, < 0: error
void solve_result(gencd_problem* p, const SolveRun* S, gencd_result* out);

// profiling helpers (api.cu)
void prof_begin(gencd_problem* p, int id, cudaEvent_t* stop_out, int launches = 1);
void prof_end(gencd_problem* p, cudaEvent_t stop);

// grow a device allocation
int ensure_sort_tmp(gencd_problem* p, size_t bytes);

// Device memory of a problem: from its pool (stream-ordered on its stream)
// when it has one, else cudaMalloc / cudaFree.  dev_alloc returns
// GENCD_ENOMEM with a message on failure and leaves *ptr null.
int dev_alloc_bytes(gencd_problem* p, void** ptr, size_t bytes);
void dev_free(gencd_problem* p, void* ptr);
template <typename T>
inline int dev_alloc(gencd_problem* p, T** ptr, size_t count) {
  return dev_alloc_bytes(p, reinterpret_cast<void**>(ptr), sizeof(T) * (count > 0 ? count : 1));
}

inline int grid_for(int64_t work, int threads, int max_blocks) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

}  // namespace gencd
