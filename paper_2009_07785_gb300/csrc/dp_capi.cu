// C ABI of libdomprop.so (declared in include/domprop.h).
//
// One dp_propagate call: inputs are copied (host) or read in place (device)
// by a prologue kernel that normalises them into the matrix's workspace;
// then a CUDA graph runs the propagation rounds of Alg. 2 (arXiv 2009.07785)
// under a WHILE conditional node whose condition the last kernel of each
// round sets on the device (the role of the paper's gpu_loop, Sec. 3.7,
// without a one-thread driver kernel); an epilogue decodes the bounds; the
// stream is synchronised once.
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "dp_internal.h"
#include "dp_launch.h"
#include "dp_objects.h"
#include "../../include/domprop.h"
#include "dp_trace.h"

namespace dp {
namespace {
std::atomic<int32_t> g_fail_countdown{0};  // the k-th allocation from now fails (0: none)
std::atomic<int64_t> g_live_allocs{0};
}  // namespace

cudaError_t dev_malloc(void **p, size_t bytes) {
  int32_t k = g_fail_countdown.load();
  while (k > 0 && !g_fail_countdown.compare_exchange_weak(k, k - 1)) {
  }
  if (k == 1) {  // this allocation is the one asked to fail
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_live_allocs.fetch_add(1);
  return e;
}

void dev_free(void *p) {
  if (!p) return;
  cudaFree(p);
  g_live_allocs.fetch_sub(1);
}

void arm_alloc_failure(int32_t k) { g_fail_countdown.store(k); }
int64_t live_allocs() { return g_live_allocs.load(); }
}  // namespace dp

namespace {

#define CUDA_TRY(x)                          \
  do {                                       \
    cudaError_t e_ = (x);                    \
    if (e_ != cudaSuccess) return DP_ERR_CUDA; \
  } while (0)

template <typename T>
int dev_alloc(dp_matrix *mat, T **p, size_t count) {
  void *q = nullptr;
  size_t bytes = sizeof(T) * (count > 0 ? count : 1);
  cudaError_t e = dp::dev_malloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DP_ERR_OOM : DP_ERR_CUDA;
  }
  mat->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return DP_OK;
}

template <typename T>
int upload(dp_matrix *mat, const std::vector<T> &v, const T **out, cudaStream_t st) {
  T *d = nullptr;
  int rc = dev_alloc(mat, &d, v.size());
  if (rc) return rc;
  if (!v.empty()) CUDA_TRY(cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  *out = d;
  return DP_OK;
}

using dp::is_device_ptr;

// Makes a round-loop graph: one WHILE node whose body is the kernels that
// `body(handle, stream)` launches; the condition starts at 1 on every launch
// and the last kernel of the body sets it on the device.
template <typename Body>
int build_loop_graph(Body body, cudaGraph_t *graph_out, cudaGraphExec_t *exec_out) {
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    cudaGraphDestroy(g);
    return DP_ERR_CUDA;
  }
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) {
    cudaGraphDestroy(g);
    return DP_ERR_CUDA;
  }
  cudaGraph_t bodyg = np.conditional.phGraph_out[0];
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGraphDestroy(g);
    return DP_ERR_CUDA;
  }
  cudaError_t e = cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t le = body(h, cs);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    if (le != cudaSuccess) e = le;
  }
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return DP_ERR_CUDA;
  }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return DP_ERR_CUDA;
  }
  *graph_out = g;
  *exec_out = ex;
  return DP_OK;
}

// The variables' records are gathered once per nonzero and round while the
// matrix streams past them; the round graph's kernels ask L2 to keep the
// records resident (an access-policy window with the persisting property,
// within the L2 set-aside of this context) so that the stream does not
// evict them.  Best effort: a device or driver that refuses leaves the
// ordinary policy in place.
void l2_keep_records(const dp_matrix *mat, cudaStream_t cs) {
  const size_t bytes = sizeof(dp::VarRec) * (size_t)(mat->M.n > 0 ? mat->M.n : 1);
  int max_persist = 0, max_window = 0;
  const int dev = mat->ctx->device;
  if (cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev) !=
          cudaSuccess ||
      max_persist <= 0 || max_window <= 0) {
    cudaGetLastError();
    return;
  }
  size_t cur = 0;
  cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
  const size_t want = bytes < (size_t)max_persist ? bytes : (size_t)max_persist;
  if (cur < want && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
  cudaStreamAttrValue v = {};
  v.accessPolicyWindow.base_ptr = mat->S.rec;
  v.accessPolicyWindow.num_bytes = bytes < (size_t)max_window ? bytes : (size_t)max_window;
  const double ratio = (double)cur / (double)v.accessPolicyWindow.num_bytes;
  v.accessPolicyWindow.hitRatio = (float)(ratio < 1.0 ? ratio : 1.0);
  v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
  v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
  if (cudaStreamSetAttribute(cs, cudaStreamAttributeAccessPolicyWindow, &v) != cudaSuccess)
    cudaGetLastError();
}

int build_graph(dp_matrix *mat) {
  const int sms = mat->ctx->num_sms;
  return build_loop_graph(
      [mat, sms](cudaGraphConditionalHandle h, cudaStream_t cs) {
        l2_keep_records(mat, cs);
        return dp::launch_round_body(mat->M, mat->S, mat->vt_ws, h, sms, cs);
      },
      &mat->graph, &mat->exec);
}

}  // namespace

extern "C" {

int dp_params_default(dp_params *out) {
  if (!out) return DP_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->max_rounds = 100;
  out->eps_int = 1e-6;
  out->tau_rel = 1e-6;
  out->eps_feas = 1e-6;
  out->inf_threshold = 1e20;
  return DP_OK;
}

const char *dp_strerror(int code) {
  switch (code) {
    case DP_OK: return "ok";
    case DP_CAP_HIT: return "round cap hit (bounds valid)";
    case DP_ERR_INVALID_ARG: return "invalid argument";
    case DP_ERR_BAD_CSR: return "malformed CSR matrix or invalid coefficient";
    case DP_ERR_NAN_INPUT: return "NaN or contradictory infinity in bounds or sides";
    case DP_ERR_OOM: return "out of memory";
    case DP_ERR_CUDA: return "CUDA runtime error";
    case DP_ERR_TIMEOUT: return "bounded device wait timed out";
    default: return "unknown status";
  }
}

int dp_ctx_set_wait_limit(dp_ctx *ctx, int64_t sleeps) {
  if (!ctx || sleeps < 0) return DP_ERR_INVALID_ARG;
  ctx->wait_limit = sleeps == 0 ? dp::kDefaultWaitLimit : (long long)sleeps;
  return DP_OK;
}

int dp_debug_fail_alloc(int32_t k) {
  if (k < 0) return DP_ERR_INVALID_ARG;
  dp::arm_alloc_failure(k);
  return DP_OK;
}

int64_t dp_debug_live_allocs(void) { return dp::live_allocs(); }

int dp_create(dp_ctx **out, int device, void *cuda_stream) {
  if (!out) return DP_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return DP_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return DP_ERR_INVALID_ARG;
  CUDA_TRY(cudaSetDevice(device));
  dp_ctx *ctx = new (std::nothrow) dp_ctx();
  if (!ctx) return DP_ERR_OOM;
  ctx->device = device;
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete ctx;
    return DP_ERR_CUDA;
  }
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return DP_ERR_CUDA;
    }
    ctx->own_stream = true;
  }
  if (cudaMallocHost(&ctx->h_ctrl, sizeof(dp::Ctrl)) != cudaSuccess) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return DP_ERR_OOM;
  }
  *out = ctx;
  return DP_OK;
}

void dp_destroy(dp_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->h_ctrl) cudaFreeHost(ctx->h_ctrl);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

namespace {
void free_batch(BatchWs *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (void *p : b->allocs) dp::dev_free(p);
  if (b->h_ctrl) cudaFreeHost(b->h_ctrl);
  if (b->h_nodes) cudaFreeHost(b->h_nodes);
  delete b;
}
}  // namespace

void dp_matrix_free(dp_matrix *mat) {
  if (!mat) return;
  cudaSetDevice(mat->ctx->device);
  cudaStreamSynchronize(mat->ctx->stream);
  free_batch(mat->batch);
  if (mat->h_inst) cudaFreeHost(mat->h_inst);
  if (mat->exec) cudaGraphExecDestroy(mat->exec);
  if (mat->graph) cudaGraphDestroy(mat->graph);
  for (void *p : mat->allocs) dp::dev_free(p);
  mat->ctx->live_matrices--;
  delete mat;
}

int dp_matrix_load(dp_ctx *ctx, int32_t m, int32_t n, int64_t nnz,
                   const int64_t *row_ptr, const int32_t *col_idx,
                   const double *val, int32_t chunk, dp_matrix **out) {
  dp::TraceRange trace_range("dp_matrix_load");
  return dp_matrix_load_sides(ctx, m, n, nnz, row_ptr, col_idx, val, chunk, nullptr, nullptr,
                              out);
}

}  // extern "C"

namespace {

// Loads a matrix; with row_off/var_off (count+1 offsets each) it is the
// block-diagonal union of `count` independent problems; with merge_ipt > 0
// it gets the merge-path layout with that many items per segment.
int load_impl(dp_ctx *ctx, int32_t m, int32_t n, int64_t nnz, const int64_t *row_ptr,
              const int32_t *col_idx, const double *val, int32_t chunk, const double *lhs,
              const double *rhs, const std::vector<int32_t> *row_off,
              const std::vector<int32_t> *var_off, dp_matrix **out, int32_t merge_ipt = 0) {
  if (!ctx || !out) return DP_ERR_INVALID_ARG;
  *out = nullptr;
  if ((lhs == nullptr) != (rhs == nullptr)) return DP_ERR_INVALID_ARG;
  dp::HostLayout H;
  int rc = merge_ipt > 0
               ? dp::build_merge_layout(m, n, nnz, row_ptr, col_idx, val, merge_ipt, lhs, rhs, H)
               : dp::build_layout(m, n, nnz, row_ptr, col_idx, val, chunk, lhs, rhs, H);
  if (rc) return rc;
  CUDA_TRY(cudaSetDevice(ctx->device));
  dp_matrix *mat = new (std::nothrow) dp_matrix();
  if (!mat) return DP_ERR_OOM;
  mat->ctx = ctx;
  ctx->live_matrices++;
  cudaStream_t st = ctx->stream;
  dp::DevMatrix &M = mat->M;
  M.m = m;
  M.n = n;
  M.nnz = nnz;
  M.nslices = H.nslices;
  M.nslices_split = H.nslices_split;
  M.nsplit_rows = H.nsplit_rows;
  M.round_warps = 8;
  M.layout = H.layout;
  M.mp_ipt = H.mp_ipt;
  M.mp_nseg = H.mp_nseg;
  M.mp_nlong = H.mp_nlong;
  M.mp_npiece = (int32_t)H.mp_piece.size();
  mat->padded = (int64_t)H.val.size();
#define TRY(x)                 \
  do {                         \
    int r_ = (x);              \
    if (r_) {                  \
      dp_matrix_free(mat);     \
      return r_;               \
    }                          \
  } while (0)
  TRY(upload(mat, H.val, &M.val, st));
  if (!H.val8.empty()) {
    TRY(upload(mat, H.val8, &mat->val8, st));
    M.val8 = nullptr;  // off by default: measured slower on GB300 (see the header)
  }
  TRY(upload(mat, H.col, &M.col, st));
  TRY(upload(mat, H.slice_off, &M.slice_off, st));
  TRY(upload(mat, H.slice_len, &M.slice_len, st));
  TRY(upload(mat, H.chunk_row, &M.chunk_row, st));
  TRY(upload(mat, H.chunk_len, &M.chunk_len, st));
  TRY(upload(mat, H.chunk_sidx, &M.chunk_sidx, st));
  TRY(upload(mat, H.split_row, &M.split_row, st));
  TRY(upload(mat, H.split_cbeg, &M.split_cbeg, st));
  TRY(upload(mat, H.split_cidx, &M.split_cidx, st));
  TRY(upload(mat, H.mp_ptr, &M.mp_ptr, st));
  TRY(upload(mat, H.mp_srow, &M.mp_srow, st));
  TRY(upload(mat, H.mp_piece, &M.mp_piece, st));
  dp::DevState &S = mat->S;
  TRY(dev_alloc(mat, &S.rec, (size_t)n));
  TRY(dev_alloc(mat, &S.keys, 2 * (size_t)n));
  TRY(dev_alloc(mat, &S.lhs, (size_t)m));
  TRY(dev_alloc(mat, &S.rhs, (size_t)m));
  if (H.layout == dp::kLayoutMerge) {
    // pieces: head and carry of every segment; activities of every row
    TRY(dev_alloc(mat, &S.part, 2 * (size_t)H.mp_nseg));
    TRY(dev_alloc(mat, &S.rowact, (size_t)m));
    TRY(dev_alloc(mat, &S.mp_need, ((size_t)H.mp_nseg + 31) / 32));
    TRY(dev_alloc(mat, &S.rowtot, (size_t)H.mp_nlong));
  } else {
    TRY(dev_alloc(mat, &S.part, (size_t)H.nslices_split * dp::kSliceW));
    TRY(dev_alloc(mat, &S.rowtot, (size_t)H.nsplit_rows));
  }
  // candidate queue: at most one entry per slot and round, so it never
  // overflows; row sums are stored per chunk slot
  TRY(dev_alloc(mat, &S.queue, (size_t)mat->padded));
  TRY(dev_alloc(mat, &S.rowsum, (size_t)H.nslices * dp::kSliceW));
  TRY(dev_alloc(mat, &S.side, (size_t)H.nslices * dp::kSliceW));
  TRY(dev_alloc(mat, &S.ctrl, 1));
  TRY(dev_alloc(mat, &S.dirty, ((size_t)n + 31) / 32));  // dirty bitmap
  TRY(dev_alloc(mat, &S.bar, 2));
  TRY(dev_alloc(mat, &mat->vt_ws, (size_t)n));
  TRY(dev_alloc(mat, &mat->st_lb, (size_t)n));
  TRY(dev_alloc(mat, &mat->st_ub, (size_t)n));
  TRY(dev_alloc(mat, &mat->st_vt, (size_t)n));
  TRY(dev_alloc(mat, &mat->st_lhs, (size_t)m));
  TRY(dev_alloc(mat, &mat->st_rhs, (size_t)m));
  TRY(dev_alloc(mat, &mat->out_lb, (size_t)n));
  TRY(dev_alloc(mat, &mat->out_ub, (size_t)n));
  if (row_off) {
    // problem of every chunk slot (by its row) and of every variable
    const int32_t count = (int32_t)row_off->size() - 1;
    std::vector<int32_t> slot_inst(H.chunk_row.size(), -1), var_inst((size_t)n, 0);
    for (size_t c = 0; c < H.chunk_row.size(); ++c) {
      const int32_t r = H.chunk_row[c];
      if (r >= 0)
        slot_inst[c] = (int32_t)(std::upper_bound(row_off->begin(), row_off->end(), r) -
                                 row_off->begin()) - 1;
    }
    for (int32_t k = 0; k < count; ++k)
      for (int32_t j = (*var_off)[k]; j < (*var_off)[k + 1]; ++j) var_inst[(size_t)j] = k;
    TRY(upload(mat, slot_inst, &S.I.slot_inst, st));
    TRY(upload(mat, var_inst, &S.I.var_inst, st));
    TRY(dev_alloc(mat, &S.I.changed, (size_t)count));
    TRY(dev_alloc(mat, &S.I.infeasible, (size_t)count));
    TRY(dev_alloc(mat, &S.I.done, (size_t)count));
    TRY(dev_alloc(mat, &S.I.rounds, (size_t)count));
    TRY(dev_alloc(mat, &S.I.status, (size_t)count));
    S.I.ninst = count;
    mat->ninst = count;
    mat->row_off = *row_off;
    mat->var_off = *var_off;
    if (cudaMallocHost(&mat->h_inst, sizeof(int32_t) * 3 * (size_t)count) != cudaSuccess) {
      cudaGetLastError();
      dp_matrix_free(mat);
      return DP_ERR_OOM;
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    dp_matrix_free(mat);
    return DP_ERR_CUDA;
  }
  TRY(build_graph(mat));
#undef TRY
  *out = mat;
  return DP_OK;
}

}  // namespace

extern "C" {

int dp_matrix_load_sides(dp_ctx *ctx, int32_t m, int32_t n, int64_t nnz,
                         const int64_t *row_ptr, const int32_t *col_idx, const double *val,
                         int32_t chunk, const double *lhs, const double *rhs,
                         dp_matrix **out) {
  dp::TraceRange trace_range("dp_matrix_load_sides");
  return load_impl(ctx, m, n, nnz, row_ptr, col_idx, val, chunk, lhs, rhs, nullptr, nullptr,
                   out);
}

int dp_matrix_load_merge(dp_ctx *ctx, int32_t m, int32_t n, int64_t nnz,
                         const int64_t *row_ptr, const int32_t *col_idx, const double *val,
                         int32_t items_per_thread, const double *lhs, const double *rhs,
                         dp_matrix **out) {
  dp::TraceRange trace_range("dp_matrix_load_merge");
  if (items_per_thread < 4 || items_per_thread > 4096) {
    if (out) *out = nullptr;
    return DP_ERR_INVALID_ARG;
  }
  return load_impl(ctx, m, n, nnz, row_ptr, col_idx, val, 0, lhs, rhs, nullptr, nullptr, out,
                   items_per_thread);
}

int dp_matrix_load_set(dp_ctx *ctx, int32_t count, const int32_t *m, const int32_t *n,
                       const int64_t *const *row_ptr, const int32_t *const *col_idx,
                       const double *const *val, int32_t chunk, const double *const *lhs,
                       const double *const *rhs, dp_matrix **out) {
  dp::TraceRange trace_range("dp_matrix_load_set");
  if (!ctx || !out || count <= 0 || !m || !n || !row_ptr || !col_idx || !val)
    return DP_ERR_INVALID_ARG;
  *out = nullptr;
  if ((lhs == nullptr) != (rhs == nullptr)) return DP_ERR_INVALID_ARG;
  std::vector<int32_t> row_off(1, 0), var_off(1, 0);
  int64_t mt = 0, nt = 0, nzt = 0;
  for (int32_t k = 0; k < count; ++k) {
    if (m[k] < 0 || n[k] < 0 || (m[k] > 0 && !row_ptr[k])) return DP_ERR_INVALID_ARG;
    mt += m[k];
    nt += n[k];
    if (m[k] > 0) nzt += row_ptr[k][m[k]];
    if (mt >= (int64_t(1) << 31) || nt >= (int64_t(1) << 31) || nzt >= (int64_t(1) << 31))
      return DP_ERR_INVALID_ARG;
    row_off.push_back((int32_t)mt);
    var_off.push_back((int32_t)nt);
  }
  std::vector<int64_t> rp;
  std::vector<int32_t> col;
  std::vector<double> vv, sl, sr;
  try {
    rp.reserve((size_t)mt + 1);
    col.reserve((size_t)nzt);
    vv.reserve((size_t)nzt);
    rp.push_back(0);
    for (int32_t k = 0; k < count; ++k) {
      const int64_t base = rp.back();
      for (int32_t i = 0; i < m[k]; ++i) rp.push_back(base + row_ptr[k][i + 1]);
      const int64_t nz = m[k] > 0 ? row_ptr[k][m[k]] : 0;
      if (m[k] > 0 && row_ptr[k][0] != 0) return DP_ERR_BAD_CSR;
      if (nz > 0 && (!col_idx[k] || !val[k])) return DP_ERR_INVALID_ARG;
      for (int64_t q = 0; q < nz; ++q) {
        const int32_t c = col_idx[k][q];
        if (c < 0 || c >= n[k]) return DP_ERR_BAD_CSR;
        col.push_back(c + var_off[(size_t)k]);
        vv.push_back(val[k][q]);
      }
      if (lhs) {
        for (int32_t i = 0; i < m[k]; ++i) {
          sl.push_back(lhs[k][i]);
          sr.push_back(rhs[k][i]);
        }
      }
    }
  } catch (const std::bad_alloc &) {
    return DP_ERR_OOM;
  }
  return load_impl(ctx, (int32_t)mt, (int32_t)nt, nzt, rp.data(), col.data(), vv.data(), chunk,
                   lhs ? sl.data() : nullptr, lhs ? sr.data() : nullptr, &row_off, &var_off,
                   out);
}

int dp_matrix_set_launch(dp_matrix *mat, int32_t round_warps) {
  if (!mat || (round_warps != 4 && round_warps != 8)) return DP_ERR_INVALID_ARG;
  if (mat->M.round_warps == round_warps) return DP_OK;
  CUDA_TRY(cudaSetDevice(mat->ctx->device));
  CUDA_TRY(cudaStreamSynchronize(mat->ctx->stream));
  if (mat->exec) cudaGraphExecDestroy(mat->exec);
  if (mat->graph) cudaGraphDestroy(mat->graph);
  mat->exec = nullptr;
  mat->graph = nullptr;
  mat->M.round_warps = round_warps;
  return build_graph(mat);
}

int dp_matrix_set_compression(dp_matrix *mat, int32_t on, int32_t *active) {
  if (!mat) return DP_ERR_INVALID_ARG;
  const int8_t *want = (on && mat->val8) ? mat->val8 : nullptr;
  if (want != mat->M.val8) {
    CUDA_TRY(cudaSetDevice(mat->ctx->device));
    CUDA_TRY(cudaStreamSynchronize(mat->ctx->stream));
    if (mat->exec) cudaGraphExecDestroy(mat->exec);
    if (mat->graph) cudaGraphDestroy(mat->graph);
    mat->exec = nullptr;
    mat->graph = nullptr;
    mat->M.val8 = want;
    int rc = build_graph(mat);
    if (rc) return rc;
  }
  if (active) *active = mat->M.val8 ? 1 : 0;
  return DP_OK;
}

int dp_matrix_set_offsets(const dp_matrix *set, int32_t *count, int32_t *row_off,
                          int32_t *var_off) {
  if (!set) return DP_ERR_INVALID_ARG;
  if (count) *count = set->ninst;
  for (int32_t k = 0; k <= set->ninst && set->ninst > 0; ++k) {
    if (row_off) row_off[k] = set->row_off[(size_t)k];
    if (var_off) var_off[k] = set->var_off[(size_t)k];
  }
  return DP_OK;
}

int dp_matrix_info(const dp_matrix *mat, int32_t *m, int32_t *n, int64_t *nnz,
                   int64_t *padded_slots, int32_t *split_rows) {
  if (!mat) return DP_ERR_INVALID_ARG;
  if (m) *m = mat->M.m;
  if (n) *n = mat->M.n;
  if (nnz) *nnz = mat->M.nnz;
  if (padded_slots) *padded_slots = mat->padded;
  if (split_rows) *split_rows = mat->M.nsplit_rows;
  return DP_OK;
}

int dp_matrix_access_floor(dp_ctx *ctx, const dp_matrix *mat, int32_t reps, float *us) {
  dp::TraceRange trace_range("dp_matrix_access_floor");
  if (!ctx || !mat || !us || reps < 1 || mat->ctx != ctx) return DP_ERR_INVALID_ARG;
  if (mat->M.layout != dp::kLayoutEll) return DP_ERR_INVALID_ARG;
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  unsigned *sink = reinterpret_cast<unsigned *>(&mat->S.ctrl->pad);  // an unused word
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return DP_ERR_CUDA;
  }
  float best = -1.0f;
  int rc = DP_OK;
  for (int r = 0; r <= reps && rc == DP_OK; ++r) {  // the first launch warms up
    if (cudaEventRecord(e0, st) != cudaSuccess ||
        dp::launch_access_floor(mat->M, mat->S, sink, st) != cudaSuccess ||
        cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      cudaGetLastError();
      rc = DP_ERR_CUDA;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && (best < 0.0f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == DP_OK) *us = best * 1000.0f;
  return rc;
}

}  // extern "C"

namespace {

// Stages inputs, writes the control block and runs the prologue.
int begin_call(dp_ctx *ctx, dp_matrix *mat, const double *lb, const double *ub,
               const uint8_t *vartype, const double *lhs, const double *rhs,
               const dp_params &p) {
  const int32_t m = mat->M.m, n = mat->M.n;
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  // inputs: device pointers are read in place, host pointers staged
  const double *d_lb = lb, *d_ub = ub, *d_lhs = lhs, *d_rhs = rhs;
  const uint8_t *d_vt = vartype;
  if (n > 0) {
    if (!is_device_ptr(lb)) { CUDA_TRY(cudaMemcpyAsync(mat->st_lb, lb, 8 * (size_t)n, cudaMemcpyDefault, st)); d_lb = mat->st_lb; }
    if (!is_device_ptr(ub)) { CUDA_TRY(cudaMemcpyAsync(mat->st_ub, ub, 8 * (size_t)n, cudaMemcpyDefault, st)); d_ub = mat->st_ub; }
    if (!is_device_ptr(vartype)) { CUDA_TRY(cudaMemcpyAsync(mat->st_vt, vartype, (size_t)n, cudaMemcpyDefault, st)); d_vt = mat->st_vt; }
  }
  if (m > 0) {
    if (!is_device_ptr(lhs)) { CUDA_TRY(cudaMemcpyAsync(mat->st_lhs, lhs, 8 * (size_t)m, cudaMemcpyDefault, st)); d_lhs = mat->st_lhs; }
    if (!is_device_ptr(rhs)) { CUDA_TRY(cudaMemcpyAsync(mat->st_rhs, rhs, 8 * (size_t)m, cudaMemcpyDefault, st)); d_rhs = mat->st_rhs; }
  }
  dp::Ctrl *hc = ctx->h_ctrl;
  std::memset(hc, 0, sizeof(*hc));
  hc->max_rounds = p.max_rounds;
  hc->eps_int = p.eps_int;
  hc->tau_rel = p.tau_rel;
  hc->eps_feas = p.eps_feas;
  hc->inf_thr = p.inf_threshold;
  hc->wait_limit = ctx->wait_limit;
  CUDA_TRY(cudaMemcpyAsync(mat->S.ctrl, hc, sizeof(*hc), cudaMemcpyHostToDevice, st));
  CUDA_TRY(dp::launch_prologue(mat->M, mat->S, mat->vt_ws, m, n, d_lb, d_ub, d_vt, d_lhs, d_rhs,
                               p.eps_int, p.tau_rel, p.inf_threshold, ctx->num_sms, st));
  return DP_OK;
}

// Decodes the bounds into the outputs, reads the control block back and
// synchronises the stream once.
int end_call(dp_ctx *ctx, dp_matrix *mat, const dp_params &p, double *lb_out,
             double *ub_out, int32_t *infeasible, int32_t *rounds) {
  const int32_t n = mat->M.n;
  cudaStream_t st = ctx->stream;
  dp::Ctrl *hc = ctx->h_ctrl;
  if (n > 0) {
    const bool dl = is_device_ptr(lb_out), du = is_device_ptr(ub_out);
    double *o_lb = dl ? lb_out : mat->out_lb;
    double *o_ub = du ? ub_out : mat->out_ub;
    CUDA_TRY(dp::launch_epilogue(mat->S, n, o_lb, o_ub, ctx->num_sms, st));
    if (!dl) CUDA_TRY(cudaMemcpyAsync(lb_out, o_lb, 8 * (size_t)n, cudaMemcpyDefault, st));
    if (!du) CUDA_TRY(cudaMemcpyAsync(ub_out, o_ub, 8 * (size_t)n, cudaMemcpyDefault, st));
  }
  CUDA_TRY(cudaMemcpyAsync(hc, mat->S.ctrl, sizeof(*hc), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (hc->err) return hc->err;
  *infeasible = hc->infeasible ? 1 : 0;
  *rounds = hc->round;
  if (!hc->infeasible && hc->last_changed && hc->round >= p.max_rounds && p.max_rounds > 0)
    return DP_CAP_HIT;
  return DP_OK;
}

int check_call(dp_ctx *ctx, const dp_matrix *mat, const double *lb, const double *ub,
               const uint8_t *vartype, const double *lhs, const double *rhs,
               const dp_params *params, double *lb_out, double *ub_out,
               int32_t *infeasible, int32_t *rounds, dp_params *p) {
  if (!ctx || !mat || !infeasible || !rounds) return DP_ERR_INVALID_ARG;
  if (mat->ctx != ctx) return DP_ERR_INVALID_ARG;
  const int32_t m = mat->M.m, n = mat->M.n;
  if (n > 0 && (!lb || !ub || !vartype || !lb_out || !ub_out)) return DP_ERR_INVALID_ARG;
  if (m > 0 && (!lhs || !rhs)) return DP_ERR_INVALID_ARG;
  if (params) *p = *params; else dp_params_default(p);
  if (p->max_rounds < 0 || !(p->eps_int >= 0) || !(p->tau_rel >= 0) || !(p->eps_feas >= 0) ||
      !(p->inf_threshold > 0))
    return DP_ERR_INVALID_ARG;
  return DP_OK;
}

}  // namespace

extern "C" {

int dp_propagate(dp_ctx *ctx, const dp_matrix *cmat, const double *lb,
                 const double *ub, const uint8_t *vartype, const double *lhs,
                 const double *rhs, const dp_params *params, double *lb_out,
                 double *ub_out, int32_t *infeasible, int32_t *rounds) {
  dp::TraceRange trace_range("dp_propagate");
  dp_params p;
  int rc = check_call(ctx, cmat, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out,
                      infeasible, rounds, &p);
  if (rc) return rc;
  dp_matrix *mat = const_cast<dp_matrix *>(cmat);
  rc = begin_call(ctx, mat, lb, ub, vartype, lhs, rhs, p);
  if (rc) return rc;
  if (p.max_rounds > 0) CUDA_TRY(cudaGraphLaunch(mat->exec, ctx->stream));
  return end_call(ctx, mat, p, lb_out, ub_out, infeasible, rounds);
}

int dp_propagate_persistent(dp_ctx *ctx, const dp_matrix *cmat, const double *lb,
                            const double *ub, const uint8_t *vartype, const double *lhs,
                            const double *rhs, const dp_params *params, double *lb_out,
                            double *ub_out, int32_t *infeasible, int32_t *rounds) {
  dp::TraceRange trace_range("dp_propagate_persistent");
  dp_params p;
  int rc = check_call(ctx, cmat, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out,
                      infeasible, rounds, &p);
  if (rc) return rc;
  if (cmat->ninst > 0 || cmat->M.layout != dp::kLayoutEll) return DP_ERR_INVALID_ARG;
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device) != cudaSuccess ||
      !coop)
    return DP_ERR_CUDA;
  dp_matrix *mat = const_cast<dp_matrix *>(cmat);
  rc = begin_call(ctx, mat, lb, ub, vartype, lhs, rhs, p);
  if (rc) return rc;
  if (p.max_rounds > 0)
    CUDA_TRY(dp::launch_persistent(mat->M, mat->S, mat->vt_ws, ctx->num_sms, ctx->stream));
  return end_call(ctx, mat, p, lb_out, ub_out, infeasible, rounds);
}

}  // extern "C"

namespace {

// One dp_propagate_set call: the round loop as the captured graph or as one
// persistent cooperative kernel.
int set_call(dp_ctx *ctx, const dp_matrix *cset, const double *lb, const double *ub,
             const uint8_t *vartype, const double *lhs, const double *rhs,
             const dp_params *params, double *lb_out, double *ub_out, int32_t *infeasible,
             int32_t *rounds, int32_t *status, bool persistent) {
  if (!cset || cset->ninst <= 0 || !infeasible || !rounds) return DP_ERR_INVALID_ARG;
  dp_params p;
  int32_t dummy_inf = 0, dummy_rounds = 0;
  int rc = check_call(ctx, cset, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out, &dummy_inf,
                      &dummy_rounds, &p);
  if (rc) return rc;
  if (persistent) {
    if (cset->M.layout != dp::kLayoutEll) return DP_ERR_INVALID_ARG;
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device) !=
            cudaSuccess ||
        !coop)
      return DP_ERR_CUDA;
  }
  dp_matrix *set = const_cast<dp_matrix *>(cset);
  rc = begin_call(ctx, set, lb, ub, vartype, lhs, rhs, p);
  if (rc) return rc;
  cudaStream_t st = ctx->stream;
  const dp::InstState &I = set->S.I;
  const size_t cb = sizeof(int32_t) * (size_t)I.ninst;
  CUDA_TRY(cudaMemsetAsync(I.changed, 0, cb, st));
  CUDA_TRY(cudaMemsetAsync(I.infeasible, 0, cb, st));
  CUDA_TRY(cudaMemsetAsync(I.done, 0, cb, st));
  CUDA_TRY(cudaMemsetAsync(I.rounds, 0, cb, st));
  CUDA_TRY(cudaMemsetAsync(I.status, 0, cb, st));
  if (p.max_rounds > 0) {
    if (persistent)
      CUDA_TRY(dp::launch_persistent(set->M, set->S, set->vt_ws, ctx->num_sms, st));
    else
      CUDA_TRY(cudaGraphLaunch(set->exec, st));
  }
  int32_t *h = set->h_inst;
  CUDA_TRY(cudaMemcpyAsync(h, I.infeasible, cb, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(h + I.ninst, I.rounds, cb, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(h + 2 * I.ninst, I.status, cb, cudaMemcpyDeviceToHost, st));
  rc = end_call(ctx, set, p, lb_out, ub_out, &dummy_inf, &dummy_rounds);
  if (rc < 0) return rc;
  bool cap = false;
  for (int32_t k = 0; k < I.ninst; ++k) {
    infeasible[k] = h[k] ? 1 : 0;
    rounds[k] = h[I.ninst + k];
    if (status) status[k] = h[2 * I.ninst + k];
    cap |= h[2 * I.ninst + k] != 0;
  }
  return cap ? DP_CAP_HIT : DP_OK;
}

}  // namespace

extern "C" {

int dp_propagate_set(dp_ctx *ctx, const dp_matrix *cset, const double *lb, const double *ub,
                     const uint8_t *vartype, const double *lhs, const double *rhs,
                     const dp_params *params, double *lb_out, double *ub_out,
                     int32_t *infeasible, int32_t *rounds, int32_t *status) {
  dp::TraceRange trace_range("dp_propagate_set");
  return set_call(ctx, cset, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out, infeasible,
                  rounds, status, false);
}

int dp_propagate_set_persistent(dp_ctx *ctx, const dp_matrix *cset, const double *lb,
                                const double *ub, const uint8_t *vartype, const double *lhs,
                                const double *rhs, const dp_params *params, double *lb_out,
                                double *ub_out, int32_t *infeasible, int32_t *rounds,
                                int32_t *status) {
  dp::TraceRange trace_range("dp_propagate_set_persistent");
  return set_call(ctx, cset, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out, infeasible,
                  rounds, status, true);
}

int dp_propagate_hostloop(dp_ctx *ctx, const dp_matrix *cmat, const double *lb,
                          const double *ub, const uint8_t *vartype,
                          const double *lhs, const double *rhs,
                          const dp_params *params, double *lb_out,
                          double *ub_out, int32_t *infeasible, int32_t *rounds,
                          float *kernel_ms, int32_t *kernel_launches) {
  dp::TraceRange trace_range("dp_propagate_hostloop");
  dp_params p;
  int rc = check_call(ctx, cmat, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out,
                      infeasible, rounds, &p);
  if (rc) return rc;
  dp_matrix *mat = const_cast<dp_matrix *>(cmat);
  rc = begin_call(ctx, mat, lb, ub, vartype, lhs, rhs, p);
  if (rc) return rc;
  cudaStream_t st = ctx->stream;
  const bool timed = kernel_ms != nullptr;
  constexpr int kK = 5;             // kernels of a round, in the documented order
  const int ev_of[kK] = {0, 2, 4, 8, 6};  // event pair of each (see launch_round_kernels)
  cudaEvent_t ev[10] = {};
  if (timed) {
    for (int i = 0; i < kK; ++i) kernel_ms[i] = 0.0f;
    for (int i = 0; i < 10; ++i)
      if (cudaEventCreate(&ev[i]) != cudaSuccess) {
        for (int q = 0; q < i; ++q) cudaEventDestroy(ev[q]);
        return DP_ERR_CUDA;
      }
  }
  if (kernel_launches)
    for (int i = 0; i < kK; ++i) kernel_launches[i] = 0;
  dp::Ctrl *hc = ctx->h_ctrl;
  int status = DP_OK;
  for (int32_t r = 0; r < p.max_rounds; ++r) {
    cudaError_t e = dp::launch_round_kernels(mat->M, mat->S, mat->vt_ws, 0, 0, ctx->num_sms, st,
                                             timed ? ev : nullptr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc, mat->S.ctrl, sizeof(*hc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { status = DP_ERR_CUDA; break; }
    const bool split = mat->M.nsplit_rows > 0;
    const bool launched[kK] = {true, split, split, true, true};
    for (int k = 0; k < kK; ++k) {
      if (!launched[k]) continue;
      if (kernel_launches) kernel_launches[k] += 1;
      float t;
      if (timed && cudaEventElapsedTime(&t, ev[ev_of[k]], ev[ev_of[k] + 1]) == cudaSuccess)
        kernel_ms[k] += t;
    }
    if (hc->err || !hc->last_changed || hc->infeasible) break;
  }
  if (timed)
    for (int i = 0; i < 10; ++i) cudaEventDestroy(ev[i]);
  if (status) return status;
  return end_call(ctx, mat, p, lb_out, ub_out, infeasible, rounds);
}

}  // extern "C"

// ------------------------------------------------------ batched B&B nodes --

namespace dp {

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

namespace {
template <typename T>
int track_alloc(std::vector<void *> &allocs, T **p, size_t count, size_t *bytes) {
  const size_t nb = sizeof(T) * (count > 0 ? count : 1);
  if (bytes) {
    *bytes += (nb + 255) & ~(size_t)255;
    *p = nullptr;
    return DP_OK;
  }
  void *q = nullptr;
  cudaError_t e = dev_malloc(&q, nb);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DP_ERR_OOM : DP_ERR_CUDA;
  }
  allocs.push_back(q);
  *p = static_cast<T *>(q);
  return DP_OK;
}

// Allocates (or, with `bytes`, only sizes) the state of a batch.
int batch_state(const DevMatrix &M, int32_t Bp, std::vector<void *> &allocs, BatchState &S,
                size_t *bytes) {
  const size_t n = (size_t)M.n, m = (size_t)M.m;
  const size_t G = (size_t)Bp / 32, Gs = (G + 3) & ~(size_t)3;
  const size_t nslots = (size_t)M.nslices * kSliceW;
  const size_t split_slots = (size_t)M.nslices_split * kSliceW;
  const size_t srows = (size_t)M.nsplit_rows;
  int rc;
#define ATRY(x) \
  if ((rc = (x)) != DP_OK) return rc
  ATRY(track_alloc(allocs, &S.cur, n * Bp, bytes));
  ATRY(track_alloc(allocs, &S.wid, n * Bp, bytes));
  ATRY(track_alloc(allocs, &S.nkey, 2 * n * Bp, bytes));
  ATRY(track_alloc(allocs, &S.chg[0], n * Gs, bytes));
  ATRY(track_alloc(allocs, &S.chg[1], n * Gs, bytes));
  ATRY(track_alloc(allocs, &S.cmask, nslots * Gs, bytes));
  ATRY(track_alloc(allocs, &S.items, G * nslots, bytes));
  ATRY(track_alloc(allocs, &S.part, split_slots * Bp, bytes));
  ATRY(track_alloc(allocs, &S.rowtot, srows * Bp, bytes));
  ATRY(track_alloc(allocs, &S.srow_act, srows * Gs, bytes));
  ATRY(track_alloc(allocs, &S.inf_bits, (size_t)kMaxGroups, bytes));
  ATRY(track_alloc(allocs, &S.chg_bits, (size_t)kMaxGroups, bytes));
  ATRY(track_alloc(allocs, &S.node_rounds, (size_t)Bp, bytes));
  ATRY(track_alloc(allocs, &S.node_status, (size_t)Bp, bytes));
  ATRY(track_alloc(allocs, &S.node_done, (size_t)Bp, bytes));
  ATRY(track_alloc(allocs, &S.alive, (size_t)kMaxGroups, bytes));
  ATRY(track_alloc(allocs, &S.fresh, (size_t)kMaxGroups, bytes));
  ATRY(track_alloc(allocs, &S.lhs, m, bytes));
  ATRY(track_alloc(allocs, &S.rhs, m, bytes));
  ATRY(track_alloc(allocs, &S.vt, n, bytes));
  ATRY(track_alloc(allocs, &S.ctrl, 1, bytes));
#undef ATRY
  S.nslots = (int64_t)nslots;
  return DP_OK;
}
}  // namespace

int alloc_batch_state(const DevMatrix &M, int32_t Bp, std::vector<void *> &allocs,
                      BatchState &S) {
  return batch_state(M, Bp, allocs, S, nullptr);
}

size_t batch_state_bytes(const DevMatrix &M, int32_t Bp) {
  std::vector<void *> none;
  BatchState S{};
  size_t bytes = 0;
  batch_state(M, Bp, none, S, &bytes);
  return bytes;
}

}  // namespace dp

namespace {

template <typename T>
int batch_alloc(BatchWs *b, T **p, size_t count) {
  void *q = nullptr;
  cudaError_t e = dp::dev_malloc(&q, sizeof(T) * (count > 0 ? count : 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DP_ERR_OOM : DP_ERR_CUDA;
  }
  b->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return DP_OK;
}

// Largest node count of one launch for this matrix: a multiple of 32, at
// most 32*kMaxGroups, and small enough that entry indices (j*Bp + node,
// 32-bit) and list counts (2*n*Bp dirty entries, G*slots work items) fit in
// a signed 32-bit integer.
int32_t batch_slab(const dp_matrix *mat) {
  const int64_t n = mat->M.n > 0 ? mat->M.n : 1;
  const int64_t slots = (int64_t)mat->M.nslices * dp::kSliceW > 0
                            ? (int64_t)mat->M.nslices * dp::kSliceW : 1;
  int64_t bp = 32 * dp::kMaxGroups;
  const int64_t lim = (int64_t(1) << 30) - 1;
  while (bp >= 32 && (n * bp > lim || slots * (bp / 32) > lim)) bp -= 32;
  return (int32_t)bp;
}

// Makes (or reuses) the workspace for Bp nodes per launch.
int ensure_batch(dp_matrix *mat, int32_t Bp) {
  if (mat->batch && mat->batch->Bp_cap >= Bp) return DP_OK;
  if (mat->batch) {
    cudaStreamSynchronize(mat->ctx->stream);
    free_batch(mat->batch);
    mat->batch = nullptr;
  }
  BatchWs *b = new (std::nothrow) BatchWs();
  if (!b) return DP_ERR_OOM;
  dp::BatchState &S = b->S;
  int rc = DP_OK;
#define BTRY(x)                 \
  do {                          \
    if ((rc = (x)) != DP_OK) {  \
      free_batch(b);            \
      return rc;                \
    }                           \
  } while (0)
  BTRY(dp::alloc_batch_state(mat->M, Bp, b->allocs, S));
  if (cudaMallocHost(&b->h_ctrl, sizeof(dp::BCtrl)) != cudaSuccess ||
      cudaMallocHost(&b->h_nodes, sizeof(int32_t) * 3 * (size_t)Bp) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return DP_ERR_OOM;
  }
  b->Bp_cap = Bp;
  const int sms = mat->ctx->num_sms;
  const dp::DevMatrix Mc = mat->M;
  const dp::BatchState Sc = b->S;
  BTRY(build_loop_graph(
      [Mc, Sc, sms](cudaGraphConditionalHandle h, cudaStream_t cs) {
        return dp::launch_batch_round(Mc, Sc, h, 1, sms, cs, nullptr);
      },
      &b->graph, &b->exec));
#undef BTRY
  mat->batch = b;
  return DP_OK;
}

// Device copy of a host input (staged), or the device pointer itself.
// The staging buffer holds `cap` elements (allocated on first use).
template <typename T>
int stage_in(BatchWs *b, T **slot, const T *src, size_t count, size_t cap, cudaStream_t st,
             const T **out) {
  if (count == 0 || is_device_ptr(src)) {
    *out = src;
    return DP_OK;
  }
  if (!*slot) {
    int rc = batch_alloc(b, slot, cap);
    if (rc) return rc;
  }
  CUDA_TRY(cudaMemcpyAsync(*slot, src, sizeof(T) * count, cudaMemcpyHostToDevice, st));
  *out = *slot;
  return DP_OK;
}

constexpr int kBatchStages = 6;  // mark, mark_split, act, combine, cand_split, finish

int batch_hostloop(dp_matrix *mat, BatchWs *b, int32_t max_rounds, float *kernel_ms,
                   int32_t *kernel_launches) {
  dp_ctx *ctx = mat->ctx;
  cudaStream_t st = ctx->stream;
  cudaEvent_t ev[2 * kBatchStages] = {};
  const bool timed = kernel_ms != nullptr;
  if (timed)
    for (int i = 0; i < 2 * kBatchStages; ++i)
      if (cudaEventCreate(&ev[i]) != cudaSuccess) {
        for (int q = 0; q < i; ++q) cudaEventDestroy(ev[q]);
        return DP_ERR_CUDA;
      }
  const bool split = mat->M.nsplit_rows > 0;
  const bool launched[kBatchStages] = {true, split, true, split, split, true};
  int status = DP_OK;
  for (int32_t r = 0; r < max_rounds; ++r) {
    cudaError_t e = dp::launch_batch_round(mat->M, b->S, 0, 0, ctx->num_sms, st,
                                           timed ? ev : nullptr);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->h_ctrl, b->S.ctrl, sizeof(dp::BCtrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      status = DP_ERR_CUDA;
      break;
    }
    for (int k = 0; k < kBatchStages; ++k) {
      if (!launched[k]) continue;
      if (kernel_launches) kernel_launches[k] += 1;
      float t;
      if (timed && cudaEventElapsedTime(&t, ev[2 * k], ev[2 * k + 1]) == cudaSuccess)
        kernel_ms[k] += t;
    }
    if (b->h_ctrl->err || !b->h_ctrl->any_alive) break;
  }
  if (timed)
    for (int i = 0; i < 2 * kBatchStages; ++i) cudaEventDestroy(ev[i]);
  return status;
}

// How a dp_propagate_nodes call runs its rounds: the captured graph (a
// WHILE loop of the round kernels), the host (one synchronisation per round,
// so that each stage can be timed with CUDA events), or one persistent
// cooperative kernel.  The results are the same.
enum NodesMode { kNodesGraph, kNodesHostloop, kNodesPersistent };

int nodes_call(dp_ctx *ctx, const dp_matrix *cmat, int32_t count, const double *lb,
               const double *ub, const uint8_t *vartype, const double *lhs, const double *rhs,
               const dp_params *params, double *lb_out, double *ub_out, int32_t *infeasible,
               int32_t *rounds, int32_t *status, NodesMode mode, float *kernel_ms,
               int32_t *kernel_launches) {
  if (!ctx || !cmat || count < 0) return DP_ERR_INVALID_ARG;
  if (cmat->ctx != ctx || cmat->M.layout != dp::kLayoutEll) return DP_ERR_INVALID_ARG;
  if (count == 0) return DP_OK;
  if (!infeasible || !rounds) return DP_ERR_INVALID_ARG;
  dp_matrix *mat = const_cast<dp_matrix *>(cmat);
  const int32_t m = mat->M.m, n = mat->M.n;
  if (n > 0 && (!lb || !ub || !vartype || !lb_out || !ub_out)) return DP_ERR_INVALID_ARG;
  if (m > 0 && (!lhs || !rhs)) return DP_ERR_INVALID_ARG;
  dp_params p;
  if (params) p = *params; else dp_params_default(&p);
  if (p.max_rounds < 0 || !(p.eps_int >= 0) || !(p.tau_rel >= 0) || !(p.eps_feas >= 0) ||
      !(p.inf_threshold > 0))
    return DP_ERR_INVALID_ARG;
  const int32_t slab = batch_slab(mat);
  if (slab < 32) return DP_ERR_INVALID_ARG;
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  {
    const int32_t want = count < slab ? (count + 31) / 32 * 32 : slab;
    int rc = ensure_batch(mat, want);
    if (rc) return rc;
  }
  BatchWs *b = mat->batch;
  const int32_t per = count < b->Bp_cap ? count : b->Bp_cap;
  const uint8_t *d_vt = nullptr;
  const double *d_lhs = nullptr, *d_rhs = nullptr;
  int rc;
  if ((rc = stage_in(b, &b->st_vt, vartype, (size_t)n, (size_t)n, st, &d_vt))) return rc;
  if ((rc = stage_in(b, &b->st_lhs, lhs, (size_t)m, (size_t)m, st, &d_lhs))) return rc;
  if ((rc = stage_in(b, &b->st_rhs, rhs, (size_t)m, (size_t)m, st, &d_rhs))) return rc;
  const bool host_out = n > 0 && !(is_device_ptr(lb_out) && is_device_ptr(ub_out));
  const size_t cap = (size_t)b->Bp_cap * (size_t)n;
  if (host_out && !b->out_lb) {
    if ((rc = batch_alloc(b, &b->out_lb, cap))) return rc;
    if ((rc = batch_alloc(b, &b->out_ub, cap))) return rc;
  }
  bool any_cap = false;
  for (int32_t s0 = 0; s0 < count; s0 += per) {
    dp::TraceRange batch_range("node batch launch");
    const int32_t cnt = count - s0 < per ? count - s0 : per;
    const int32_t Bp = (cnt + 31) / 32 * 32;
    const size_t off = (size_t)s0 * (size_t)n, len = (size_t)cnt * (size_t)n;
    const double *d_lb = nullptr, *d_ub = nullptr;
    if ((rc = stage_in(b, &b->st_lb, n > 0 ? lb + off : lb, len, cap, st, &d_lb))) return rc;
    if ((rc = stage_in(b, &b->st_ub, n > 0 ? ub + off : ub, len, cap, st, &d_ub))) return rc;
    dp::BCtrl *hc = b->h_ctrl;
    std::memset(hc, 0, sizeof(*hc));
    hc->max_rounds = p.max_rounds;
    hc->B = cnt;
    hc->Bp = Bp;
    hc->G = Bp / 32;
    hc->any_alive = 1;
    hc->eps_int = p.eps_int;
    hc->tau_rel = p.tau_rel;
    hc->eps_feas = p.eps_feas;
    hc->inf_thr = p.inf_threshold;
    hc->wait_limit = ctx->wait_limit;
    const size_t Gs = (size_t)((Bp / 32 + 3) & ~3);
    CUDA_TRY(cudaMemcpyAsync(b->S.ctrl, hc, sizeof(*hc), cudaMemcpyHostToDevice, st));
    if (n > 0) {
      CUDA_TRY(cudaMemsetAsync(b->S.chg[0], 0, sizeof(uint32_t) * Gs * n, st));
      CUDA_TRY(cudaMemsetAsync(b->S.chg[1], 0, sizeof(uint32_t) * Gs * n, st));
    }
    CUDA_TRY(dp::launch_batch_prologue(mat->M, b->S, cnt, d_lb, d_ub, d_vt, d_lhs, d_rhs,
                                       p.eps_int, p.tau_rel, p.eps_feas, p.inf_threshold,
                                       ctx->num_sms, st));
    if (p.max_rounds > 0 && mode == kNodesGraph) CUDA_TRY(cudaGraphLaunch(b->exec, st));
    if (p.max_rounds > 0 && mode == kNodesPersistent)
      CUDA_TRY(dp::launch_batch_persistent(mat->M, b->S, ctx->num_sms, st));
    if (p.max_rounds > 0 && mode == kNodesHostloop) {
      int r2 = batch_hostloop(mat, b, p.max_rounds, kernel_ms, kernel_launches);
      if (r2) return r2;
    }
    if (n > 0) {
      double *o_lb = host_out ? b->out_lb : lb_out + off;
      double *o_ub = host_out ? b->out_ub : ub_out + off;
      CUDA_TRY(dp::launch_batch_epilogue(mat->M, b->S, cnt, o_lb, o_ub, ctx->num_sms, st));
      if (host_out) {
        CUDA_TRY(cudaMemcpyAsync(lb_out + off, o_lb, 8 * len, cudaMemcpyDefault, st));
        CUDA_TRY(cudaMemcpyAsync(ub_out + off, o_ub, 8 * len, cudaMemcpyDefault, st));
      }
    }
    int32_t *hn = b->h_nodes;
    CUDA_TRY(cudaMemcpyAsync(hn, b->S.inf_bits, 4 * (size_t)dp::kMaxGroups, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hn + Bp, b->S.node_rounds, 4 * (size_t)cnt, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hn + 2 * Bp, b->S.node_status, 4 * (size_t)cnt, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hc, b->S.ctrl, sizeof(*hc), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (hc->err) return hc->err;
    for (int32_t i = 0; i < cnt; ++i) {
      infeasible[s0 + i] = (int32_t)(((uint32_t)hn[i >> 5] >> (i & 31)) & 1u);
      rounds[s0 + i] = hn[Bp + i];
      if (status) status[s0 + i] = hn[2 * Bp + i];
      any_cap |= hn[2 * Bp + i] != 0;
    }
  }
  return any_cap ? DP_CAP_HIT : DP_OK;
}

}  // namespace

extern "C" int dp_propagate_nodes(dp_ctx *ctx, const dp_matrix *mat, int32_t count,
                                  const double *lb, const double *ub, const uint8_t *vartype,
                                  const double *lhs, const double *rhs,
                                  const dp_params *params, double *lb_out, double *ub_out,
                                  int32_t *infeasible, int32_t *rounds, int32_t *status) {
  dp::TraceRange trace_range("dp_propagate_nodes");
  return nodes_call(ctx, mat, count, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out,
                    infeasible, rounds, status, kNodesGraph, nullptr, nullptr);
}

extern "C" int dp_propagate_nodes_persistent(dp_ctx *ctx, const dp_matrix *mat, int32_t count,
                                             const double *lb, const double *ub,
                                             const uint8_t *vartype, const double *lhs,
                                             const double *rhs, const dp_params *params,
                                             double *lb_out, double *ub_out,
                                             int32_t *infeasible, int32_t *rounds,
                                             int32_t *status) {
  dp::TraceRange trace_range("dp_propagate_nodes_persistent");
  if (!ctx) return DP_ERR_INVALID_ARG;
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device) != cudaSuccess ||
      !coop)
    return DP_ERR_CUDA;
  return nodes_call(ctx, mat, count, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out,
                    infeasible, rounds, status, kNodesPersistent, nullptr, nullptr);
}

extern "C" int dp_propagate_nodes_hostloop(dp_ctx *ctx, const dp_matrix *mat, int32_t count,
                                           const double *lb, const double *ub,
                                           const uint8_t *vartype, const double *lhs,
                                           const double *rhs, const dp_params *params,
                                           double *lb_out, double *ub_out,
                                           int32_t *infeasible, int32_t *rounds,
                                           int32_t *status, float *kernel_ms,
                                           int32_t *kernel_launches) {
  dp::TraceRange trace_range("dp_propagate_nodes_hostloop");
  if (kernel_ms)
    for (int k = 0; k < kBatchStages; ++k) kernel_ms[k] = 0.0f;
  if (kernel_launches)
    for (int k = 0; k < kBatchStages; ++k) kernel_launches[k] = 0;
  return nodes_call(ctx, mat, count, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out,
                    infeasible, rounds, status, kNodesHostloop, kernel_ms, kernel_launches);
}
