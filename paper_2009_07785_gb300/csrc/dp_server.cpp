// Request serving with continuous batching (C ABI in include/domprop.h).
//
// A server keeps matrices resident and answers propagation requests: a
// request is one node bound vector of a resident matrix, propagated exactly
// as dp_propagate would propagate it alone (Alg. 2, round-synchronous).
//
// Each resident matrix is a lane: a batch of `slots` node slots (the batched
// kernels of dp_batch.cu), its own CUDA stream, and a one-round CUDA graph
// (the round's kernels plus a copy of the per-node flags to pinned host
// memory).  A worker thread drives every lane round by round.  Between two
// rounds of a lane it reads out the nodes that finished (no change,
// infeasible, or the round cap), frees their slots, and admits waiting
// requests into free slots; an admitted node starts with every row active
// and counts its own rounds, so requests that arrive while others are on
// the GPU join the running batch at the next round boundary.  Lanes run on
// separate streams, so the rounds of different matrices overlap on the
// device.  A lane's device workspace is allocated when it first has work
// and only while the server's memory budget allows (admission by device
// memory); idle lanes give their workspace back when another lane needs it.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "dp_internal.h"
#include "dp_launch.h"
#include "dp_objects.h"
#include "../../include/domprop.h"
#include "dp_trace.h"

namespace {

double now_us() {
  return std::chrono::duration<double, std::micro>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t tag = 0;
  int32_t matrix = 0;
  const double *lb = nullptr, *ub = nullptr;  // caller memory
  double *lb_out = nullptr, *ub_out = nullptr;
  double arrival_us = 0.0;
};

struct Finished {  // a request whose bounds are being copied out
  Request req;
  int32_t stage = 0;  // index in the lane's output staging
  int32_t infeasible = 0, rounds = 0, status = 0;
};

struct Lane {
  const dp_matrix *mat = nullptr;
  int32_t m = 0, n = 0;
  int32_t id = 0;
  // sides and types (device copies owned by the lane)
  double *d_lhs = nullptr, *d_rhs = nullptr;
  uint8_t *d_vt = nullptr;
  // workspace (allocated on demand)
  bool has_ws = false;
  size_t ws_bytes = 0;
  std::vector<void *> dev_allocs;
  std::vector<void *> host_allocs;
  dp::BatchState S{};
  cudaStream_t stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev_round = nullptr, ev_extract = nullptr;
  int32_t *d_admit = nullptr, *h_admit = nullptr;      // slot lists
  int32_t *d_extract = nullptr, *h_extract = nullptr;
  double *d_in = nullptr, *h_in = nullptr;             // [slots * 2n] staged requests
  double *d_out = nullptr, *h_out = nullptr;           // [slots * 2n] finished bounds
  int32_t *h_flags = nullptr;  // done[Bp], rounds[Bp], status[Bp], inf_bits[kMaxGroups]
  // scheduling state (worker thread only)
  bool round_in_flight = false, extract_in_flight = false;
  std::vector<int8_t> occupied;     // per slot: holds a request
  std::vector<int8_t> propagating;  // per slot: its node had not finished at the last look
  std::vector<Request> slot_req;
  std::deque<Request> pending;
  std::vector<Finished> extracting;
  double last_used_us = 0.0;
};

}  // namespace

struct dp_server {
  dp_ctx *ctx = nullptr;
  dp_server_config cfg{};
  int32_t Bp = 64;
  int64_t budget = 0;
  int64_t used = 0;  // device bytes of lane workspaces
  std::vector<Lane *> lanes;
  // shared with client threads
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> inbox;
  std::deque<dp_completion> done;
  bool stop = false;
  int64_t in_system = 0;  // submitted and not yet completed
  dp_server_stats stats{};
  int32_t error = 0;      // sticky CUDA error seen by the worker
  std::thread worker;
};

namespace {

#define SRV_TRY(x)                                 \
  do {                                             \
    cudaError_t e_ = (x);                          \
    if (e_ != cudaSuccess) {                       \
      cudaGetLastError();                          \
      return DP_ERR_CUDA;                          \
    }                                              \
  } while (0)

void free_workspace(Lane &L) {
  if (L.exec) cudaGraphExecDestroy(L.exec);
  if (L.graph) cudaGraphDestroy(L.graph);
  if (L.ev_round) cudaEventDestroy(L.ev_round);
  if (L.ev_extract) cudaEventDestroy(L.ev_extract);
  if (L.stream) cudaStreamDestroy(L.stream);
  for (void *p : L.dev_allocs) dp::dev_free(p);
  for (void *p : L.host_allocs) cudaFreeHost(p);
  L.dev_allocs.clear();
  L.host_allocs.clear();
  L.exec = nullptr;
  L.graph = nullptr;
  L.ev_round = L.ev_extract = nullptr;
  L.stream = nullptr;
  L.has_ws = false;
}

size_t lane_bytes(const Lane &L, int32_t Bp) {
  return dp::batch_state_bytes(L.mat->M, Bp) + 2 * (size_t)Bp * 2 * (size_t)L.n * sizeof(double) +
         2 * (size_t)Bp * sizeof(int32_t) + 4096;
}

template <typename T>
int lane_dev(Lane &L, T **p, size_t count) {
  void *q = nullptr;
  if (dp::dev_malloc(&q, sizeof(T) * (count > 0 ? count : 1)) != cudaSuccess) {
    cudaGetLastError();
    return DP_ERR_OOM;
  }
  L.dev_allocs.push_back(q);
  *p = static_cast<T *>(q);
  return DP_OK;
}

template <typename T>
int lane_host(Lane &L, T **p, size_t count) {
  void *q = nullptr;
  if (cudaMallocHost(&q, sizeof(T) * (count > 0 ? count : 1)) != cudaSuccess) {
    cudaGetLastError();
    return DP_ERR_OOM;
  }
  L.host_allocs.push_back(q);
  *p = static_cast<T *>(q);
  return DP_OK;
}

// Allocates a lane's workspace, writes its sides/types and empty slots, and
// captures its one-round graph.
int make_workspace(dp_server *s, Lane &L) {
  const int32_t Bp = s->Bp;
  const size_t n = (size_t)L.n;
  int rc;
#define WTRY(x)            \
  if ((rc = (x)) != DP_OK) \
  return rc
  WTRY(dp::alloc_batch_state(L.mat->M, Bp, L.dev_allocs, L.S));
  WTRY(lane_dev(L, &L.d_admit, (size_t)Bp));
  WTRY(lane_dev(L, &L.d_extract, (size_t)Bp));
  WTRY(lane_dev(L, &L.d_in, (size_t)Bp * 2 * n));
  WTRY(lane_dev(L, &L.d_out, (size_t)Bp * 2 * n));
  WTRY(lane_host(L, &L.h_admit, (size_t)Bp));
  WTRY(lane_host(L, &L.h_extract, (size_t)Bp));
  WTRY(lane_host(L, &L.h_in, (size_t)Bp * 2 * n));
  WTRY(lane_host(L, &L.h_out, (size_t)Bp * 2 * n));
  WTRY(lane_host(L, &L.h_flags, 3 * (size_t)Bp + dp::kMaxGroups));
#undef WTRY
  SRV_TRY(cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking));
  SRV_TRY(cudaEventCreateWithFlags(&L.ev_round, cudaEventDisableTiming));
  SRV_TRY(cudaEventCreateWithFlags(&L.ev_extract, cudaEventDisableTiming));
  // control block, empty change masks, sides and types, empty slots
  dp::BCtrl c;
  std::memset(&c, 0, sizeof(c));
  c.max_rounds = s->cfg.params.max_rounds;
  c.B = Bp;
  c.Bp = Bp;
  c.G = Bp / 32;
  c.any_alive = 1;
  c.eps_int = s->cfg.params.eps_int;
  c.tau_rel = s->cfg.params.tau_rel;
  c.eps_feas = s->cfg.params.eps_feas;
  c.inf_thr = s->cfg.params.inf_threshold;
  const size_t Gs = (size_t)((Bp / 32 + 3) & ~3);
  SRV_TRY(cudaMemcpyAsync(L.S.ctrl, &c, sizeof(c), cudaMemcpyHostToDevice, L.stream));
  if (n > 0) {
    SRV_TRY(cudaMemsetAsync(L.S.chg[0], 0, sizeof(uint32_t) * Gs * n, L.stream));
    SRV_TRY(cudaMemsetAsync(L.S.chg[1], 0, sizeof(uint32_t) * Gs * n, L.stream));
  }
  SRV_TRY(dp::launch_slots_init(L.mat->M, L.S, Bp, L.d_vt, L.d_lhs, L.d_rhs,
                                s->cfg.params.inf_threshold, s->ctx->num_sms, L.stream));
  SRV_TRY(cudaStreamSynchronize(L.stream));
  // the one-round graph: kernels, then the per-node flags to the host
  cudaStream_t cs = nullptr;
  SRV_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t le = dp::launch_batch_round(L.mat->M, L.S, 0, 0, s->ctx->num_sms, cs, nullptr);
    if (le == cudaSuccess)
      le = cudaMemcpyAsync(L.h_flags, L.S.node_done, 4 * (size_t)Bp, cudaMemcpyDeviceToHost, cs);
    if (le == cudaSuccess)
      le = cudaMemcpyAsync(L.h_flags + Bp, L.S.node_rounds, 4 * (size_t)Bp, cudaMemcpyDeviceToHost,
                           cs);
    if (le == cudaSuccess)
      le = cudaMemcpyAsync(L.h_flags + 2 * Bp, L.S.node_status, 4 * (size_t)Bp,
                           cudaMemcpyDeviceToHost, cs);
    if (le == cudaSuccess)
      le = cudaMemcpyAsync(L.h_flags + 3 * Bp, L.S.inf_bits, 4 * (size_t)dp::kMaxGroups,
                           cudaMemcpyDeviceToHost, cs);
    e = cudaStreamEndCapture(cs, &L.graph);
    if (le != cudaSuccess) e = le;
  }
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DP_ERR_CUDA;
  }
  SRV_TRY(cudaGraphInstantiate(&L.exec, L.graph, 0));
  std::memset(L.h_flags, 0, sizeof(int32_t) * (3 * (size_t)Bp + dp::kMaxGroups));
  L.occupied.assign((size_t)Bp, 0);
  L.propagating.assign((size_t)Bp, 0);
  L.slot_req.assign((size_t)Bp, Request());
  L.round_in_flight = L.extract_in_flight = false;
  L.has_ws = true;
  return DP_OK;
}

bool lane_idle(const Lane &L) {
  if (L.round_in_flight || L.extract_in_flight || !L.pending.empty() || !L.extracting.empty())
    return false;
  for (int8_t o : L.occupied)
    if (o) return false;
  return true;
}

// Makes room for a lane's workspace under the budget (frees the least
// recently used idle lanes) and allocates it.  False if it cannot yet.
bool acquire_workspace(dp_server *s, Lane &L) {
  const int64_t need = (int64_t)lane_bytes(L, s->Bp);
  std::vector<Lane *> lanes;
  {
    std::lock_guard<std::mutex> g(s->mu);
    lanes = s->lanes;
  }
  while (s->used + need > s->budget) {
    Lane *victim = nullptr;
    for (Lane *o : lanes)
      if (o != &L && o->has_ws && lane_idle(*o) &&
          (!victim || o->last_used_us < victim->last_used_us))
        victim = o;
    if (!victim) return false;
    free_workspace(*victim);
    std::lock_guard<std::mutex> g(s->mu);
    s->used -= (int64_t)victim->ws_bytes;
    victim->ws_bytes = 0;
    s->stats.evictions++;
  }
  int rc = make_workspace(s, L);
  if (rc != DP_OK) {
    free_workspace(L);
    if (rc != DP_ERR_OOM) s->error = rc;
    return false;
  }
  std::lock_guard<std::mutex> g(s->mu);
  L.ws_bytes = (size_t)need;
  s->used += need;
  s->stats.workspaces_allocated++;
  return true;
}

void post(dp_server *s, const Finished &f, int32_t matrix) {
  dp_completion c;
  std::memset(&c, 0, sizeof(c));
  c.tag = f.req.tag;
  c.status = f.status ? DP_CAP_HIT : DP_OK;
  c.infeasible = f.infeasible;
  c.rounds = f.rounds;
  c.matrix = matrix;
  c.arrival_us = f.req.arrival_us;
  c.done_us = now_us();
  std::lock_guard<std::mutex> g(s->mu);
  s->done.push_back(c);
  s->in_system--;
  s->stats.completed++;
  s->cv_done.notify_all();
}

// One scheduling step of a lane; returns whether anything happened.
bool service(dp_server *s, Lane &L) {
  bool did = false;
  const int32_t Bp = s->Bp;
  const size_t n = (size_t)L.n;
  // 1. finished bounds arrived in pinned memory: hand them to the callers
  if (L.extract_in_flight && cudaEventQuery(L.ev_extract) == cudaSuccess) {
    for (const Finished &f : L.extracting) {
      if (n > 0) {
        std::memcpy(f.req.lb_out, L.h_out + 2 * (size_t)f.stage * n, n * sizeof(double));
        std::memcpy(f.req.ub_out, L.h_out + (2 * (size_t)f.stage + 1) * n, n * sizeof(double));
      }
      post(s, f, L.id);
    }
    L.extracting.clear();
    L.extract_in_flight = false;
    did = true;
  }
  // 2. a round ended: read out the nodes that finished
  if (L.round_in_flight) {
    if (cudaEventQuery(L.ev_round) != cudaSuccess) return did;
    L.round_in_flight = false;
    for (int32_t k = 0; k < Bp; ++k)
      if (L.propagating[k] && L.h_flags[k]) L.propagating[k] = 0;
    did = true;
  }
  if (!L.has_ws) {
    if (L.pending.empty()) return did;
    if (!acquire_workspace(s, L)) return did;
  }
  if (!L.extract_in_flight) {
    int32_t cnt = 0;
    for (int32_t k = 0; k < Bp; ++k) {
      if (!L.occupied[k] || L.propagating[k]) continue;
      Finished f;
      f.req = L.slot_req[k];
      f.stage = cnt;
      f.infeasible = (int32_t)(((uint32_t)L.h_flags[3 * Bp + (k >> 5)] >> (k & 31)) & 1u);
      f.rounds = L.h_flags[Bp + k];
      f.status = L.h_flags[2 * Bp + k];
      L.extracting.push_back(f);
      L.h_extract[cnt++] = k;
      L.occupied[k] = 0;
    }
    if (cnt > 0) {
      cudaError_t e = cudaMemcpyAsync(L.d_extract, L.h_extract, 4 * (size_t)cnt,
                                      cudaMemcpyHostToDevice, L.stream);
      if (e == cudaSuccess)
        e = dp::launch_slots_extract(L.mat->M, L.S, Bp, L.d_extract, cnt, L.d_out,
                                     s->ctx->num_sms, L.stream);
      if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(L.h_out, L.d_out, 2 * (size_t)cnt * n * sizeof(double),
                            cudaMemcpyDeviceToHost, L.stream);
      if (e == cudaSuccess) e = cudaEventRecord(L.ev_extract, L.stream);
      if (e != cudaSuccess) s->error = DP_ERR_CUDA;
      L.extract_in_flight = true;
      did = true;
    }
  }
  // 3. admit waiting requests into free slots, then run the next round
  int32_t cnt = 0;
  for (int32_t k = 0; k < Bp && !L.pending.empty(); ++k) {
    if (L.occupied[k]) continue;
    Request r = L.pending.front();
    L.pending.pop_front();
    if (n > 0) {
      std::memcpy(L.h_in + 2 * (size_t)cnt * n, r.lb, n * sizeof(double));
      std::memcpy(L.h_in + (2 * (size_t)cnt + 1) * n, r.ub, n * sizeof(double));
    }
    L.h_admit[cnt++] = k;
    L.occupied[k] = 1;
    L.propagating[k] = 1;
    L.slot_req[k] = r;
  }
  if (cnt > 0) {
    cudaError_t e = cudaMemcpyAsync(L.d_admit, L.h_admit, 4 * (size_t)cnt,
                                    cudaMemcpyHostToDevice, L.stream);
    if (e == cudaSuccess && n > 0)
      e = cudaMemcpyAsync(L.d_in, L.h_in, 2 * (size_t)cnt * n * sizeof(double),
                          cudaMemcpyHostToDevice, L.stream);
    if (e == cudaSuccess)
      e = dp::launch_slots_admit(L.mat->M, L.S, Bp, L.d_admit, cnt, L.d_in,
                                 s->cfg.params.eps_int, s->cfg.params.tau_rel,
                                 s->cfg.params.eps_feas, s->cfg.params.inf_threshold,
                                 s->ctx->num_sms, L.stream);
    if (e != cudaSuccess) s->error = DP_ERR_CUDA;
    std::lock_guard<std::mutex> g(s->mu);
    s->stats.admissions += cnt;
    did = true;
  }
  int32_t active = 0;
  for (int32_t k = 0; k < Bp; ++k) active += L.propagating[k];
  if (active > 0) {
    // the host copy of the admission staging must not be overwritten before
    // the copy above has run: rounds and admissions alternate, and the next
    // admission waits for this round's event
    cudaError_t e = cudaGraphLaunch(L.exec, L.stream);
    if (e == cudaSuccess) e = cudaEventRecord(L.ev_round, L.stream);
    if (e != cudaSuccess) s->error = DP_ERR_CUDA;
    L.round_in_flight = true;
    L.last_used_us = now_us();
    std::lock_guard<std::mutex> g(s->mu);
    s->stats.rounds++;
    s->stats.slot_rounds += active;
    if (active > s->stats.max_active_slots) s->stats.max_active_slots = active;
    did = true;
  }
  return did;
}

void worker_main(dp_server *s) {
  cudaSetDevice(s->ctx->device);
  std::vector<Lane *> lanes;
  for (;;) {
    bool stopping;
    {
      std::unique_lock<std::mutex> g(s->mu);
      lanes = s->lanes;  // matrices may be added meanwhile
      while (!s->inbox.empty()) {
        Request r = s->inbox.front();
        s->inbox.pop_front();
        s->lanes[(size_t)r.matrix]->pending.push_back(r);
      }
      stopping = s->stop && (s->in_system == 0 || s->error);
    }
    if (stopping) break;
    bool did = false, busy = false;
    for (Lane *L : lanes) {
      did |= service(s, *L);
      busy |= L->round_in_flight || L->extract_in_flight;
    }
    if (!did) {
      if (busy) {
        std::this_thread::yield();  // device work in flight: poll its events
      } else {
        std::unique_lock<std::mutex> g(s->mu);
        if (s->inbox.empty() && !(s->stop && s->in_system == 0))
          s->cv_work.wait_for(g, std::chrono::microseconds(200));
      }
    }
  }
}

bool finite_request(const double *lb, const double *ub, int32_t n, double thr) {
  for (int32_t j = 0; j < n; ++j) {
    const double L = lb[j], U = ub[j];
    if (std::isnan(L) || std::isnan(U) || L >= thr || U <= -thr) return false;
  }
  return true;
}

}  // namespace

extern "C" {

int dp_server_create(dp_ctx *ctx, const dp_server_config *cfg, dp_server **out) {
  if (!ctx || !out) return DP_ERR_INVALID_ARG;
  *out = nullptr;
  dp_server_config c;
  std::memset(&c, 0, sizeof(c));
  if (cfg) c = *cfg;
  if (!cfg) dp_params_default(&c.params);
  if (c.slots == 0) c.slots = 64;
  if (c.slots < 32 || c.slots > 32 * dp::kMaxGroups || c.slots % 32) return DP_ERR_INVALID_ARG;
  const dp_params &p = c.params;
  if (p.max_rounds < 1 || !(p.eps_int >= 0) || !(p.tau_rel >= 0) || !(p.eps_feas >= 0) ||
      !(p.inf_threshold > 0))
    return DP_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DP_ERR_CUDA;
  if (c.mem_budget <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return DP_ERR_CUDA;
    c.mem_budget = (int64_t)(fr / 2);
  }
  dp_server *s = new (std::nothrow) dp_server();
  if (!s) return DP_ERR_OOM;
  s->ctx = ctx;
  s->cfg = c;
  s->Bp = c.slots;
  s->budget = c.mem_budget;
  try {
    s->worker = std::thread(worker_main, s);
  } catch (...) {
    delete s;
    return DP_ERR_OOM;
  }
  *out = s;
  return DP_OK;
}

int dp_server_add_matrix(dp_server *s, const dp_matrix *mat, const uint8_t *vartype,
                         const double *lhs, const double *rhs, int32_t *matrix_id) {
  dp::TraceRange trace_range("dp_server_add_matrix");
  if (!s || !mat || !matrix_id || mat->ctx != s->ctx) return DP_ERR_INVALID_ARG;
  if (mat->M.layout != dp::kLayoutEll) return DP_ERR_INVALID_ARG;
  const int32_t m = mat->M.m, n = mat->M.n;
  if ((n > 0 && !vartype) || (m > 0 && (!lhs || !rhs))) return DP_ERR_INVALID_ARG;
  if ((int64_t)n * s->Bp >= (int64_t(1) << 30) ||
      (int64_t)mat->M.nslices * dp::kSliceW * (s->Bp / 32) >= (int64_t(1) << 30))
    return DP_ERR_INVALID_ARG;
  const double thr = s->cfg.params.inf_threshold;
  if (m > 0 && !dp::is_device_ptr(lhs) && !dp::is_device_ptr(rhs))
    for (int32_t i = 0; i < m; ++i)
      if (std::isnan(lhs[i]) || std::isnan(rhs[i]) || lhs[i] >= thr || rhs[i] <= -thr)
        return DP_ERR_NAN_INPUT;
  Lane *L = new (std::nothrow) Lane();
  if (!L) return DP_ERR_OOM;
  L->mat = mat;
  L->m = m;
  L->n = n;
  if (cudaSetDevice(s->ctx->device) != cudaSuccess ||
      dp::dev_malloc((void **)&L->d_lhs, 8 * (size_t)(m > 0 ? m : 1)) != cudaSuccess ||
      dp::dev_malloc((void **)&L->d_rhs, 8 * (size_t)(m > 0 ? m : 1)) != cudaSuccess ||
      dp::dev_malloc((void **)&L->d_vt, (size_t)(n > 0 ? n : 1)) != cudaSuccess ||
      (m > 0 && cudaMemcpy(L->d_lhs, lhs, 8 * (size_t)m, cudaMemcpyDefault) != cudaSuccess) ||
      (m > 0 && cudaMemcpy(L->d_rhs, rhs, 8 * (size_t)m, cudaMemcpyDefault) != cudaSuccess) ||
      (n > 0 && cudaMemcpy(L->d_vt, vartype, (size_t)n, cudaMemcpyDefault) != cudaSuccess)) {
    cudaGetLastError();
    dp::dev_free(L->d_lhs);
    dp::dev_free(L->d_rhs);
    dp::dev_free(L->d_vt);
    delete L;
    return DP_ERR_CUDA;
  }
  std::lock_guard<std::mutex> g(s->mu);
  L->id = (int32_t)s->lanes.size();
  s->lanes.push_back(L);
  *matrix_id = L->id;
  return DP_OK;
}

int dp_server_submit(dp_server *s, int32_t matrix_id, const double *lb, const double *ub,
                     double *lb_out, double *ub_out, uint64_t tag, double arrival_us) {
  dp::TraceRange trace_range("dp_server_submit");
  if (!s) return DP_ERR_INVALID_ARG;
  Request r;
  const Lane *L = nullptr;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop || matrix_id < 0 || matrix_id >= (int32_t)s->lanes.size())
      return DP_ERR_INVALID_ARG;
    if (s->error) return s->error;
    L = s->lanes[(size_t)matrix_id];
  }
  if (L->n > 0 && (!lb || !ub || !lb_out || !ub_out)) return DP_ERR_INVALID_ARG;
  if (L->n > 0 && (dp::is_device_ptr(lb) || dp::is_device_ptr(ub) || dp::is_device_ptr(lb_out) ||
                   dp::is_device_ptr(ub_out)))
    return DP_ERR_INVALID_ARG;
  if (!finite_request(lb, ub, L->n, s->cfg.params.inf_threshold)) return DP_ERR_NAN_INPUT;
  r.tag = tag;
  r.matrix = matrix_id;
  r.lb = lb;
  r.ub = ub;
  r.lb_out = lb_out;
  r.ub_out = ub_out;
  r.arrival_us = arrival_us > 0.0 ? arrival_us : now_us();
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->inbox.push_back(r);
    s->in_system++;
    s->stats.submitted++;
  }
  s->cv_work.notify_one();
  return DP_OK;
}

int dp_server_poll(dp_server *s, dp_completion *out, int32_t max, int32_t *count,
                   int32_t wait_us) {
  dp::TraceRange trace_range("dp_server_poll");
  if (!s || !count || max < 0 || (max > 0 && !out)) return DP_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> g(s->mu);
  if (s->done.empty() && wait_us > 0 && !s->error)
    s->cv_done.wait_for(g, std::chrono::microseconds(wait_us),
                        [s] { return !s->done.empty() || s->error; });
  int32_t k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *count = k;
  return s->error ? s->error : DP_OK;
}

int dp_server_stats_get(dp_server *s, dp_server_stats *out) {
  if (!s || !out) return DP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  *out = s->stats;
  out->device_bytes = s->used;
  out->in_system = s->in_system;
  return DP_OK;
}

double dp_server_clock_us(void) { return now_us(); }

int dp_server_destroy(dp_server *s) {
  if (!s) return DP_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->ctx->device);
  int rc = s->error;
  for (Lane *L : s->lanes) {
    if (L->stream) cudaStreamSynchronize(L->stream);
    free_workspace(*L);
    dp::dev_free(L->d_lhs);
    dp::dev_free(L->d_rhs);
    dp::dev_free(L->d_vt);
    delete L;
  }
  delete s;
  return rc;
}

}  // extern "C"
