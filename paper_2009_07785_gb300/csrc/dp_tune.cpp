// Autotuners (C ABI in include/domprop.h).  dp_autotune, for the
// single-instance path, times
// a few propagation rounds of the caller's problem for every candidate row
// split length ("chunk": rows longer than it are split across threads and
// combined in a second pass, the paper's long-row bin, Sec. 3.2) and block
// shape (warps per block of the round kernel), and reports the fastest.  It
// uses only the library's own entry points: each distinct layout is loaded
// once, each shape set with dp_matrix_set_launch, and timed with the
// host-driven loop's CUDA-event kernel times.  dp_autotune_nodes does the
// same for the batched-node path over a sample of node bound vectors.
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/domprop.h"
#include "dp_trace.h"

extern "C" int dp_autotune(dp_ctx *ctx, int32_t m, int32_t n, int64_t nnz,
                           const int64_t *row_ptr, const int32_t *col_idx, const double *val,
                           const double *lb, const double *ub, const uint8_t *vartype,
                           const double *lhs, const double *rhs, const dp_params *params,
                           int32_t rounds, dp_tune_entry *entries, int32_t max_entries,
                           int32_t *count, dp_tune_entry *best) {
  dp::TraceRange trace_range("dp_autotune");
  if (!ctx || !best || max_entries < 0 || (max_entries > 0 && !entries) ||
      (m > 0 && !row_ptr))
    return DP_ERR_INVALID_ARG;
  dp_params p;
  if (params) p = *params; else dp_params_default(&p);
  if (rounds > 0) p.max_rounds = rounds;  // else: to the fixed point (or the cap)
  // distinct layouts only: every chunk at least as long as the longest row
  // gives the layout of the shortest such chunk
  int64_t maxlen = 0;
  for (int32_t i = 0; i < m; ++i)
    if (row_ptr[i + 1] - row_ptr[i] > maxlen) maxlen = row_ptr[i + 1] - row_ptr[i];
  const int32_t chunks[] = {64, 128, 256, 512, 1024};
  const int32_t shapes[] = {4, 8};
  std::vector<double> out_lb((size_t)(n > 0 ? n : 1)), out_ub((size_t)(n > 0 ? n : 1));
  int32_t k = 0;
  bool have = false;
  bool covered = false;
  for (int32_t chunk : chunks) {
    if (covered) break;
    if (chunk >= maxlen) covered = true;
    dp_matrix *mat = nullptr;
    int rc = dp_matrix_load_sides(ctx, m, n, nnz, row_ptr, col_idx, val, chunk, lhs, rhs, &mat);
    if (rc == DP_ERR_INVALID_ARG || rc == DP_ERR_BAD_CSR) {
      // device sides cannot order rows: load without them
      rc = dp_matrix_load(ctx, m, n, nnz, row_ptr, col_idx, val, chunk, &mat);
    }
    if (rc) return rc;
    dp_matrix_set_compression(mat, 0, nullptr);  // the binary64 values (the default layout)
    for (int32_t w : shapes) {
      rc = dp_matrix_set_launch(mat, w);
      if (rc) break;
      int32_t inf = 0, rr = 0;
      float ms[5];
      int32_t launches[5];
      double best_us = -1.0;
      for (int rep = 0; rep < 4 && rc >= 0; ++rep) {  // first call warms up
        rc = dp_propagate_hostloop(ctx, mat, lb, ub, vartype, lhs, rhs, &p, out_lb.data(),
                                   out_ub.data(), &inf, &rr, ms, launches);
        if (rc < 0 || rep == 0) continue;
        double tot = 0.0;
        for (int q = 0; q < 5; ++q) tot += ms[q];
        const double us = tot * 1e3 / (rr > 0 ? rr : 1);
        if (best_us < 0 || us < best_us) best_us = us;
      }
      if (rc < 0) break;
      rc = DP_OK;
      dp_tune_entry e;
      std::memset(&e, 0, sizeof(e));
      e.chunk = chunk;
      e.round_warps = w;
      e.us_per_round = (float)best_us;
      if (k < max_entries) entries[k] = e;
      ++k;
      if (!have || e.us_per_round < best->us_per_round) {
        *best = e;
        have = true;
      }
    }
    dp_matrix_free(mat);
    if (rc < 0) return rc;
  }
  if (count) *count = k;
  return have ? DP_OK : DP_ERR_INVALID_ARG;
}

extern "C" int dp_autotune_nodes(dp_ctx *ctx, int32_t m, int32_t n, int64_t nnz,
                                 const int64_t *row_ptr, const int32_t *col_idx,
                                 const double *val, int32_t nodes, const double *lb,
                                 const double *ub, const uint8_t *vartype, const double *lhs,
                                 const double *rhs, const dp_params *params,
                                 dp_tune_entry *entries, int32_t max_entries, int32_t *count,
                                 dp_tune_entry *best) {
  dp::TraceRange trace_range("dp_autotune_nodes");
  if (!ctx || !best || nodes < 1 || max_entries < 0 || (max_entries > 0 && !entries) ||
      (m > 0 && !row_ptr))
    return DP_ERR_INVALID_ARG;
  int64_t maxlen = 0;
  for (int32_t i = 0; i < m; ++i)
    if (row_ptr[i + 1] - row_ptr[i] > maxlen) maxlen = row_ptr[i + 1] - row_ptr[i];
  const int32_t chunks[] = {32, 64, 128, 256, 512};
  const size_t cells = (size_t)nodes * (size_t)(n > 0 ? n : 1);
  std::vector<double> out_lb(cells), out_ub(cells);
  std::vector<int32_t> inf((size_t)nodes), rr((size_t)nodes);
  int32_t k = 0;
  bool have = false, covered = false;
  for (int32_t chunk : chunks) {
    if (covered) break;
    if (chunk >= maxlen) covered = true;
    dp_matrix *mat = nullptr;
    int rc = dp_matrix_load_sides(ctx, m, n, nnz, row_ptr, col_idx, val, chunk, lhs, rhs, &mat);
    if (rc == DP_ERR_INVALID_ARG || rc == DP_ERR_BAD_CSR)
      rc = dp_matrix_load(ctx, m, n, nnz, row_ptr, col_idx, val, chunk, &mat);
    if (rc) return rc;
    double best_us = -1.0;
    for (int rep = 0; rep < 4 && rc >= 0; ++rep) {  // first call warms up
      float ms[6];
      int32_t launches[6];
      rc = dp_propagate_nodes_hostloop(ctx, mat, nodes, lb, ub, vartype, lhs, rhs, params,
                                       out_lb.data(), out_ub.data(), inf.data(), rr.data(),
                                       nullptr, ms, launches);
      if (rc < 0 || rep == 0) continue;
      double tot = 0.0;
      for (int q = 0; q < 6; ++q) tot += ms[q];
      const double us = tot * 1e3 / (launches[0] > 0 ? launches[0] : 1);
      if (best_us < 0 || us < best_us) best_us = us;
    }
    dp_matrix_free(mat);
    if (rc < 0) return rc;
    dp_tune_entry e;
    std::memset(&e, 0, sizeof(e));
    e.chunk = chunk;
    e.us_per_round = (float)best_us;
    if (k < max_entries) entries[k] = e;
    ++k;
    if (!have || e.us_per_round < best->us_per_round) {
      *best = e;
      have = true;
    }
  }
  if (count) *count = k;
  return have ? DP_OK : DP_ERR_INVALID_ARG;
}
