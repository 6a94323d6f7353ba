// Host-side launchers of the device kernels (dp_kernels.cu) and the host
// layout builder (dp_layout.cpp), used by the C ABI in dp_capi.cu.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "dp_internal.h"

namespace dp {

cudaError_t launch_prologue(const DevMatrix &M, const DevState &S, uint8_t *vt_ws,
                            int32_t m, int32_t n, const double *lb, const double *ub,
                            const uint8_t *vartype, const double *lhs,
                            const double *rhs, double eps_int, double tau_rel,
                            double thr, int num_sms, cudaStream_t st);

cudaError_t launch_epilogue(const DevState &S, int32_t n, double *lb_out,
                            double *ub_out, int num_sms, cudaStream_t st);

cudaError_t launch_round_body(const DevMatrix &M, const DevState &S,
                              const uint8_t *vt_ws,
                              cudaGraphConditionalHandle handle, int num_sms,
                              cudaStream_t st);

cudaError_t launch_round_kernels(const DevMatrix &M, const DevState &S,
                                 const uint8_t *vt_ws,
                                 cudaGraphConditionalHandle handle,
                                 int use_cond, int num_sms, cudaStream_t st,
                                 cudaEvent_t *ev);

// One launch of the round's memory access pattern without its arithmetic
// (k_floor; sliced layout only) on `st`.
cudaError_t launch_access_floor(const DevMatrix &M, const DevState &S, unsigned *sink,
                                cudaStream_t st);

// The whole round loop as one cooperative (persistent) launch on `st`
// (single problems only).
cudaError_t launch_persistent(const DevMatrix &M, const DevState &S, const uint8_t *vt_ws,
                              int num_sms, cudaStream_t st);

// Batched branch-and-bound nodes (dp_batch.cu).  The prologue normalises
// `count` node-major bound vectors (lb[node*n + j]) into the node-minor
// state; the epilogue writes them back node-major.
cudaError_t launch_batch_prologue(const DevMatrix &M, const BatchState &S, int32_t count,
                                  const double *lb, const double *ub, const uint8_t *vartype,
                                  const double *lhs, const double *rhs, double eps_int,
                                  double tau_rel, double eps_feas, double thr, int num_sms,
                                  cudaStream_t st);
cudaError_t launch_batch_epilogue(const DevMatrix &M, const BatchState &S, int32_t count,
                                  double *lb_out, double *ub_out, int num_sms,
                                  cudaStream_t st);
// One batched round; in a graph body (use_cond = 1) the last kernel sets
// the WHILE condition.  With `ev` (12 events) each of the six stages (mark,
// mark_split, act, combine, cand_split, finish) is bracketed by a pair.
// The batch's round loop as one cooperative kernel (all rounds; no graph).
cudaError_t launch_batch_persistent(const DevMatrix &M, const BatchState &S, int num_sms,
                                    cudaStream_t st);
cudaError_t launch_batch_round(const DevMatrix &M, const BatchState &S,
                               cudaGraphConditionalHandle handle, int use_cond,
                               int num_sms, cudaStream_t st, cudaEvent_t *ev);

// Serving slots (dp_batch.cu): a batch whose nodes are independent requests.
// launch_slots_init writes the sides and types and leaves every slot empty;
// launch_slots_admit resets the per-node state of `count` slots (device
// array `slots`) and fills their bounds from `stage` (slot i: lb at
// stage + 2*i*n, ub at stage + (2*i+1)*n, validated by the host);
// launch_slots_extract copies the bounds of `count` slots to `out` in the
// same layout.
cudaError_t launch_slots_init(const DevMatrix &M, const BatchState &S, int32_t Bp,
                              const uint8_t *vartype, const double *lhs, const double *rhs,
                              double thr, int num_sms, cudaStream_t st);
cudaError_t launch_slots_admit(const DevMatrix &M, const BatchState &S, int32_t Bp,
                               const int32_t *slots, int32_t count, const double *stage,
                               double eps_int, double tau_rel, double eps_feas, double thr,
                               int num_sms, cudaStream_t st);
cudaError_t launch_slots_extract(const DevMatrix &M, const BatchState &S, int32_t Bp,
                                 const int32_t *slots, int32_t count, double *out,
                                 int num_sms, cudaStream_t st);

// Merge-path layout (dp_merge.cu): the activity pass over the segments,
// the combination of split rows and the per-row pass that runs Step 2 and
// queues the nonzeros that survive the screen (with the warp-level re-read
// of long rows).  With `ev`, the three are bracketed by ev[0..1], ev[2..3]
// and ev[4..5].
cudaError_t launch_merge_front(const DevMatrix &M, const DevState &S, int num_sms,
                               cudaStream_t st, cudaEvent_t *ev);
// Per call (after the sides are written): the activities each warp of the
// activity pass needs.
cudaError_t launch_merge_prologue(const DevMatrix &M, const DevState &S, cudaStream_t st);

// Host image of the device layout described in dp_internal.h.
struct HostLayout {
  int32_t m = 0, n = 0;
  int64_t nnz = 0;
  int32_t nslices = 0, nslices_split = 0, nsplit_rows = 0;
  int32_t layout = kLayoutEll;
  int32_t mp_ipt = 0, mp_nseg = 0, mp_nlong = 0;
  std::vector<int32_t> mp_ptr, mp_srow;
  std::vector<int4> mp_piece;
  std::vector<double> val;
  std::vector<int8_t> val8;  // empty unless every coefficient is an integer in [-127, 127]
  std::vector<int32_t> col;
  std::vector<int64_t> slice_off;
  std::vector<int32_t> slice_len;
  std::vector<int32_t> chunk_row, chunk_len, chunk_sidx;
  std::vector<int32_t> split_row, split_cbeg, split_cidx;
};

// Validates a host CSR matrix and builds its layout; lhs_hint/rhs_hint
// (host, may be NULL) only order rows of equal length by the finiteness of
// their sides.  Returns DP_OK, DP_ERR_INVALID_ARG, DP_ERR_BAD_CSR or
// DP_ERR_OOM.
int build_layout(int32_t m, int32_t n, int64_t nnz, const int64_t *row_ptr,
                 const int32_t *col_idx, const double *val, int32_t chunk,
                 const double *lhs_hint, const double *rhs_hint, HostLayout &out);

// The same for the merge-path layout with `ipt` items per segment
// (4..4096).
int build_merge_layout(int32_t m, int32_t n, int64_t nnz, const int64_t *row_ptr,
                       const int32_t *col_idx, const double *val, int32_t ipt,
                       const double *lhs_hint, const double *rhs_hint, HostLayout &out);

}  // namespace dp
