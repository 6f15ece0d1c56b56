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
  K_NUM
};

struct Profiler {
  bool enabled = false;
  std::vector<cudaEvent_t> pool;       // pairs (start, stop)
  std::vector<int> pending_id;         // kernel id of each recorded pair
  size_t used = 0;
  double ms[K_NUM] = {0};
  int64_t launches[K_NUM] = {0};       // counted whether or not profiling is on
};

// ---------------------------------------------------------------------------
}  // namespace gencd

struct gencd_problem {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  int64_t n = 0, k = 0, nnz = 0, nnz_pad = 0;
  int32_t loss = GENCD_LOSS_LOGISTIC;
  int32_t precision = GENCD_F64;
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

  // streaming propose over all columns
  int items = 4;
  int64_t ntiles = 0;
  int32_t* tile_col = nullptr;
  double* gacc = nullptr;
  double* delta = nullptr;
  double* phi = nullptr;

  // accepted / selected lists (capacity k)
  int32_t* list_j = nullptr;
  double* list_d = nullptr;
  uint32_t* list_off = nullptr;  // exclusive prefix of the listed columns' nnz (k + 2)
  uint32_t* scan_tmp = nullptr;  // scratch of the prefix sum

  // accept candidates of (chunk, partition) pairs when partitions are few
  double* slot_f = nullptr;
  double* slot_d = nullptr;
  int32_t* slot_j = nullptr;
  int64_t slot_cap = 0;

  // device scalars: [0] kkt bits, [1] objective, [2] loss sum, [3] l1 sum,
  // [4] updates (int64), [5] nnz processed (int64), [6] scratch
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

  gencd::Profiler prof;
};

namespace gencd {

constexpr int kRedBlocks = 1024;

// ---- launchers (defined next to their kernels) ------------------------------
// kernels_propose.cu
int launch_propose_all(gencd_problem* p, const void* u_vec, bool u_is_double);
int launch_finalize(gencd_problem* p, double lambda, bool write_steps);
int launch_finalize_accept(gencd_problem* p, int64_t B);  // Thread-Greedy / Greedy
int ensure_slots(gencd_problem* p, int64_t count);
// exclusive prefix sum of m uint32 (in place allowed); tmp holds scan_tmp_words(m)
int exclusive_scan(gencd_problem* p, const uint32_t* in, uint32_t* out, int64_t m, uint32_t* tmp);
int64_t scan_tmp_words(int64_t m);
int launch_propose_list(gencd_problem* p, const int32_t* J, int64_t m, double* delta, double* phi);
int launch_objective(gencd_problem* p);
int launch_col_sumsq(gencd_problem* p);  // gacc_j = sum_i X_ij^2

// kernels_update.cu
int launch_fill_u(gencd_problem* p);
int launch_update_list(gencd_problem* p, const int32_t* J, const double* d, int64_t m, bool skip_neg);
int launch_refresh_list(gencd_problem* p, const int32_t* J, const double* d, int64_t m, bool skip_neg);
int launch_coloring_iter(gencd_problem* p, int64_t q);
int launch_csr_spmv(gencd_problem* p, const double* x, double* out);  // out = X x (FP64)

// kernels_setup.cu
int launch_col_scale(gencd_problem* p);
int launch_tile_map(gencd_problem* p);
int radix_sort_pairs(gencd_problem* p, uint32_t* keys, uint32_t* vals, int64_t m, int bits,
                     uint32_t* keys_alt, uint32_t* vals_alt, bool* result_in_alt);
int make_permutation(gencd_problem* p, uint64_t seed, int64_t epoch, int64_t m, int32_t* out);
int build_csr(gencd_problem* p);
int run_coloring(gencd_problem* p);
int build_color_classes(gencd_problem* p);
int launch_power_step(gencd_problem* p, const double* v, const double* dinv, double* r, double* s);
int validate_input(gencd_problem* p, int64_t* bad_col, int64_t* bad_row, int* stage);

// profiling helpers (api.cu)
void prof_begin(gencd_problem* p, int id, cudaEvent_t* stop_out);
void prof_end(gencd_problem* p, cudaEvent_t stop);

// grow a device allocation
int ensure_sort_tmp(gencd_problem* p, size_t bytes);

inline int grid_for(int64_t work, int threads, int max_blocks) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

}  // namespace gencd
