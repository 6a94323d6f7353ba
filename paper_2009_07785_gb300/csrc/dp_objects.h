// Host-side objects behind the opaque handles of the C ABI, shared by the
// library's host sources (dp_capi.cu, dp_server.cpp).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "dp_internal.h"

struct dp_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  dp::Ctrl *h_ctrl = nullptr;  // pinned mirror of the device control block
  int live_matrices = 0;
  long long wait_limit = dp::kDefaultWaitLimit;  // grid-barrier wait of the persistent loop
};

struct dp_matrix {
  dp_ctx *ctx = nullptr;
  dp::DevMatrix M{};
  dp::DevState S{};
  int64_t padded = 0;
  std::vector<void *> allocs;
  uint8_t *vt_ws = nullptr;
  // staging for host inputs / outputs
  double *st_lb = nullptr, *st_ub = nullptr, *st_lhs = nullptr, *st_rhs = nullptr;
  uint8_t *st_vt = nullptr;
  double *out_lb = nullptr, *out_ub = nullptr;
  // the round loop
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // batched nodes (allocated on the first dp_propagate_nodes call)
  struct BatchWs *batch = nullptr;
  const int8_t *val8 = nullptr;  // int8 copy of the values (small integers only)
  // problem sets (dp_matrix_load_set): first row / variable of each problem
  int32_t ninst = 0;
  std::vector<int32_t> row_off, var_off;
  int32_t *h_inst = nullptr;  // pinned [3*ninst]: infeasible, rounds, status
};

// Workspace of dp_propagate_nodes for up to Bp_cap nodes per launch.
struct BatchWs {
  int32_t Bp_cap = 0;
  std::vector<void *> allocs;
  dp::BatchState S{};
  dp::BCtrl *h_ctrl = nullptr;  // pinned
  int32_t *h_nodes = nullptr;   // pinned [3*Bp_cap]: infeasible, rounds, status
  // staging of host inputs / outputs, allocated when first needed
  double *st_lb = nullptr, *st_ub = nullptr, *out_lb = nullptr, *out_ub = nullptr;
  double *st_lhs = nullptr, *st_rhs = nullptr;
  uint8_t *st_vt = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace dp {

// Allocates the device state of a batch of Bp nodes (a multiple of 32, at
// most 32*kMaxGroups) over matrix M; every allocation is appended to
// `allocs`, which the caller frees.  Returns DP_OK, DP_ERR_OOM or DP_ERR_CUDA.
int alloc_batch_state(const DevMatrix &M, int32_t Bp, std::vector<void *> &allocs,
                      BatchState &S);
// Device bytes alloc_batch_state takes for Bp nodes.
size_t batch_state_bytes(const DevMatrix &M, int32_t Bp);
// True for device (or managed) memory.
bool is_device_ptr(const void *p);

}  // namespace dp
