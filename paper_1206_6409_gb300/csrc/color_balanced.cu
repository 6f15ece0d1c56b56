// color_balanced.cu -- balanced distance-2 colouring of X's columns (host
// preprocessing, like the paper's own colouring step).  The paper closes by
// noting that the fewest colours need not give the most parallelism and that
// a balanced distribution of colour-class sizes is preferable (Section 7).
// Rule: columns in index order; column j takes, among the colours that no
// lower-index column sharing a row with it uses, the one with the fewest
// columns so far that is still below a size cap (ties: the lower colour), or
// a new colour.  The default cap is ceil(k / C), C the first-fit colour count
// (the colouring gencd_color computes).  The result installs with
// gencd_set_colors and runs through the Coloring variant on the GPU.
#include <algorithm>
#include <map>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "gencd_internal.cuh"

namespace {

int cfail(int code, const std::string& m) {
  gencd::set_error(m);
  return code;
}

// rows of X as column lists
void row_lists(int64_t n, int64_t k, const int64_t* col_ptr, const int32_t* row_idx, std::vector<int64_t>& rp,
               std::vector<int32_t>& rc) {
  const int64_t nnz = col_ptr[k];
  rp.assign((size_t)n + 1, 0);
  rc.resize((size_t)nnz);
  for (int64_t t = 0; t < nnz; ++t) rp[(size_t)row_idx[t] + 1] += 1;
  for (int64_t i = 0; i < n; ++i) rp[(size_t)i + 1] += rp[(size_t)i];
  std::vector<int64_t> at(rp.begin(), rp.end() - 1);
  for (int64_t j = 0; j < k; ++j)
    for (int64_t t = col_ptr[j]; t < col_ptr[j + 1]; ++t) rc[(size_t)at[(size_t)row_idx[t]]++] = (int32_t)j;
}

// stamps, for column j, the colours of its lower-index neighbours
void stamp_neighbours(int64_t j, const int64_t* col_ptr, const int32_t* row_idx, const std::vector<int64_t>& rp,
                      const std::vector<int32_t>& rc, const std::vector<int32_t>& colors,
                      std::vector<int64_t>& stamp) {
  for (int64_t t = col_ptr[j]; t < col_ptr[j + 1]; ++t) {
    const int32_t i = row_idx[t];
    for (int64_t q = rp[(size_t)i]; q < rp[(size_t)i + 1]; ++q) {
      const int32_t c = rc[(size_t)q];
      if (c >= j) break;  // a row's columns are in increasing order
      stamp[(size_t)colors[(size_t)c]] = j + 1;
    }
  }
}

int color_balanced(int64_t n, int64_t k, const int64_t* col_ptr, const int32_t* row_idx, int64_t cap,
                   int32_t* out, int32_t* ncolors_out) {
  std::vector<int64_t> rp;
  std::vector<int32_t> rc;
  row_lists(n, k, col_ptr, row_idx, rp, rc);
  std::vector<int32_t> colors((size_t)k, 0);
  std::vector<int64_t> stamp((size_t)k + 1, 0);
  if (cap <= 0) {  // first-fit colour count
    int32_t c0 = 0;
    for (int64_t j = 0; j < k; ++j) {
      stamp_neighbours(j, col_ptr, row_idx, rp, rc, colors, stamp);
      int32_t c = 0;
      while (stamp[(size_t)c] == j + 1) ++c;
      colors[(size_t)j] = c;
      c0 = std::max(c0, c + 1);
    }
    cap = (k + c0 - 1) / std::max<int32_t>(1, c0);
    std::fill(stamp.begin(), stamp.end(), 0);
  }
  // colours grouped by their class size; each group ordered by colour
  std::map<int64_t, std::set<int32_t>> by_size;
  std::vector<int64_t> size;
  for (int64_t j = 0; j < k; ++j) {
    stamp_neighbours(j, col_ptr, row_idx, rp, rc, colors, stamp);
    int32_t pick = -1;
    for (auto it = by_size.begin(); it != by_size.end() && it->first < cap && pick < 0; ++it)
      for (int32_t c : it->second)
        if (stamp[(size_t)c] != j + 1) {
          pick = c;
          break;
        }
    if (pick < 0) {
      pick = (int32_t)size.size();
      size.push_back(0);
    } else {
      auto it = by_size.find(size[(size_t)pick]);
      it->second.erase(pick);
      if (it->second.empty()) by_size.erase(it);
    }
    size[(size_t)pick] += 1;
    by_size[size[(size_t)pick]].insert(pick);
    colors[(size_t)j] = pick;
  }
  std::copy(colors.begin(), colors.end(), out);
  *ncolors_out = (int32_t)size.size();
  return GENCD_OK;
}

}  // namespace

extern "C" int gencd_color_balanced_csc(int64_t n, int64_t k, const int64_t* col_ptr, const int32_t* row_idx,
                                        int64_t cap, int32_t* colors, int32_t* ncolors) {
  if (n < 0 || k < 0 || !col_ptr || !colors || !ncolors || (k > 0 && col_ptr[k] > 0 && !row_idx))
    return cfail(GENCD_EINVAL, "bad arguments");
  if (col_ptr[0] != 0) return cfail(GENCD_EINVAL, "col_ptr[0] must be 0");
  for (int64_t j = 0; j < k; ++j) {
    if (col_ptr[j + 1] < col_ptr[j]) return cfail(GENCD_EINVAL, "col_ptr decreases at column " + std::to_string(j));
    for (int64_t t = col_ptr[j]; t < col_ptr[j + 1]; ++t)
      if (row_idx[t] < 0 || row_idx[t] >= n || (t > col_ptr[j] && row_idx[t] <= row_idx[t - 1]))
        return cfail(GENCD_EINVAL, "column " + std::to_string(j) + " has unsorted, duplicate or out-of-range rows");
  }
  try {  // no exception crosses the C ABI
    return color_balanced(n, k, col_ptr, row_idx, cap, colors, ncolors);
  } catch (const std::exception& e) {
    return cfail(GENCD_ENOMEM, std::string("host allocation failed: ") + e.what());
  }
}
