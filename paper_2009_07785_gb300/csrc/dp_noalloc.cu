// Allocation-free propagation entry point (dp_propagate_noalloc).
//
// Who needs it: callers that must not call cudaMalloc/cudaFree themselves or
// through a library -- for example a solver embedded in a process whose
// device memory belongs to a pool allocator (PyTorch's caching allocator, a
// MIP solver's own arena), where a stray cudaMalloc fragments or exhausts the
// pool, or a latency-sensitive pipeline where cudaMalloc/cudaFree would
// synchronise the device.  dp_matrix_load allocates the matrix's device
// layout and workspace; this entry point instead works directly on a CSR
// matrix and problem the caller already holds in device memory, and keeps
// its only scratch (the next-state bound keys and a control block) in one
// file-scope __device__ array of fixed size.
//
// The scratch array is shared by every call in the process on a given
// device and keeps the previous call's contents; each call re-initialises
// what it uses.  Calls whose GPU work overlaps (two streams, two host
// threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstring>

#include "../../include/domprop.h"
#include "dp_trace.h"

namespace {

// next-state keys (2 per variable) followed by the control block
constexpr size_t kNoallocCtrlWords = 32;  // int64 words reserved for the control block
constexpr size_t kNoallocWords = 2 * (size_t)DP_NOALLOC_MAX_VARS + kNoallocCtrlWords;

__device__ __align__(256) long long g_noalloc_scratch[kNoallocWords];

// control block layout inside the scratch array (int32 view)
struct NoallocCtrl {
  int32_t err, changed, infeasible, pad;
};

constexpr int kMaxDevices = 64;
// Device address of the array, per device.  Host threads that call the entry
// point on different devices may fill their entries concurrently; the lookup
// is idempotent, so an atomic store per entry is all the synchronisation it
// needs.
std::atomic<long long *> g_scratch_addr[kMaxDevices] = {};

__device__ __forceinline__ bool is_inf_d(double x) {
  return ((unsigned long long)__double_as_longlong(x) << 1) == 0xFFE0000000000000ull;
}
__device__ __forceinline__ bool is_finite_d(double x) {
  return ((__double2hiint(x) >> 20) & 0x7FF) != 0x7FF;
}
__device__ __forceinline__ bool is_nan_d(double x) {
  return ((unsigned long long)__double_as_longlong(x) << 1) > 0xFFE0000000000000ull;
}
__device__ __forceinline__ long long okey(double x) {
  long long b = __double_as_longlong(x);
  return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ double okey_val(long long k) {
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7FFFFFFFFFFFFFFFll));
}
__device__ __forceinline__ double side_norm(double v, double thr) {
  const double pinf = __longlong_as_double(0x7FF0000000000000ll);
  if (v >= thr) return pinf;
  if (v <= -thr) return -pinf;
  return v;
}

// Checks the caller's CSR (so that no later kernel can read out of range)
// and normalises the bounds into the outputs (the round state) and keys.
__global__ void k_na_prologue(int32_t m, int32_t n, const int64_t *row_ptr,
                              const int32_t *col, const double *val, int64_t nnz,
                              const double *lb, const double *ub, const uint8_t *vt,
                              const double *lhs, const double *rhs, double eps_int, double thr,
                              double *lo, double *hi, long long *keys, NoallocCtrl *ctrl) {
  const double pinf = __longlong_as_double(0x7FF0000000000000ll);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz; i += stride) {
    double a = val[i];
    if (col[i] < 0 || col[i] >= n || !is_finite_d(a) || a == 0.0) atomicExch(&ctrl->err, DP_ERR_BAD_CSR);
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= m; i += stride) {
    if (i == 0 && row_ptr[0] != 0) atomicExch(&ctrl->err, DP_ERR_BAD_CSR);
    if (i == m && row_ptr[m] != nnz) atomicExch(&ctrl->err, DP_ERR_BAD_CSR);
    if (i < m && row_ptr[i + 1] < row_ptr[i]) atomicExch(&ctrl->err, DP_ERR_BAD_CSR);
    if (i < m) {
      double l = lhs[i], r = rhs[i];
      if (is_nan_d(l) || is_nan_d(r) || l >= thr || r <= -thr) atomicExch(&ctrl->err, DP_ERR_NAN_INPUT);
    }
  }
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += stride) {
    double L = lb[j], U = ub[j];
    if (is_nan_d(L) || is_nan_d(U) || L >= thr || U <= -thr) {
      atomicExch(&ctrl->err, DP_ERR_NAN_INPUT);
      L = U = 0.0;
    }
    if (L <= -thr) L = -pinf;
    if (U >= thr) U = pinf;
    if (vt[j]) {
      if (is_finite_d(L)) L = ceil(L - eps_int);
      if (is_finite_d(U)) U = floor(U + eps_int);
    }
    lo[j] = L;
    hi[j] = U;
    keys[2 * j] = okey(L);
    keys[2 * j + 1] = okey(U);
  }
}

// One round, one thread per row: the activity chain in CSR order, Step 2,
// every nonzero's candidates (Eq. 3a/3b in residual form, Eq. 5a/5b, the
// exactly-one-infinity rule), integer rounding and filtered atomics into the
// next-state keys.  State is read from lo/hi (start of the round).
__global__ void k_na_round(int32_t m, const int64_t *row_ptr, const int32_t *col,
                           const double *val, const double *lhs_in, const double *rhs_in,
                           const uint8_t *vt, const double *lo, const double *hi,
                           long long *keys, NoallocCtrl *ctrl, double eps_int, double tau,
                           double eps_feas, double thr) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double lhs = side_norm(lhs_in[i], thr), rhs = side_norm(rhs_in[i], thr);
  const int64_t b = row_ptr[i], e = row_ptr[i + 1];
  double minfin = 0.0, maxfin = 0.0;
  int mininf = 0, maxinf = 0;
  for (int64_t k = b; k < e; ++k) {
    const double a = val[k];
    const int32_t j = col[k];
    const double bmin = a > 0.0 ? lo[j] : hi[j];
    const double bmax = a > 0.0 ? hi[j] : lo[j];
    if (is_inf_d(bmin)) ++mininf; else minfin = fma(a, bmin, minfin);
    if (is_inf_d(bmax)) ++maxinf; else maxfin = fma(a, bmax, maxfin);
  }
  if (mininf == 0 && is_finite_d(rhs) && minfin > rhs + eps_feas * fmax(1.0, fabs(rhs)))
    atomicExch(&ctrl->infeasible, 1);
  if (maxinf == 0 && is_finite_d(lhs) && maxfin < lhs - eps_feas * fmax(1.0, fabs(lhs)))
    atomicExch(&ctrl->infeasible, 1);
  for (int64_t k = b; k < e; ++k) {
    const double a = val[k];
    const int32_t j = col[k];
    const double L = lo[j], U = hi[j];
    const double bmin = a > 0.0 ? L : U;
    const double bmax = a > 0.0 ? U : L;
    double resmin, resmax;
    if (mininf == 0) resmin = fma(-a, bmin, minfin);
    else if (mininf == 1 && is_inf_d(bmin)) resmin = minfin;
    else resmin = -__longlong_as_double(0x7FF0000000000000ll);
    if (maxinf == 0) resmax = fma(-a, bmax, maxfin);
    else if (maxinf == 1 && is_inf_d(bmax)) resmax = maxfin;
    else resmax = __longlong_as_double(0x7FF0000000000000ll);
    bool hl = false, hu = false;
    double lc = 0.0, uc = 0.0;
    if (is_finite_d(rhs) && is_finite_d(resmin)) {
      double c = (rhs - resmin) / a;
      if (a > 0.0) { uc = c; hu = true; } else { lc = c; hl = true; }
    }
    if (is_finite_d(lhs) && is_finite_d(resmax)) {
      double c = (lhs - resmax) / a;
      if (a > 0.0) { lc = c; hl = true; } else { uc = c; hu = true; }
    }
    const bool isint = vt[j] != 0;
    if (hl) {
      if (isint) lc = ceil(lc - eps_int);
      if (!(fabs(lc) < thr)) hl = false;
    }
    if (hu) {
      if (isint) uc = floor(uc + eps_int);
      if (!(fabs(uc) < thr)) hu = false;
    }
    if (hl) {
      bool acc = is_inf_d(L) || (isint ? lc > L : lc > L + tau * fmax(1.0, fabs(L)));
      if (acc) {
        atomicMax(&keys[2 * (int64_t)j], okey(lc));
        ctrl->changed = 1;
      }
    }
    if (hu) {
      bool acc = is_inf_d(U) || (isint ? uc < U : uc < U - tau * fmax(1.0, fabs(U)));
      if (acc) {
        atomicMin(&keys[2 * (int64_t)j + 1], okey(uc));
        ctrl->changed = 1;
      }
    }
  }
}

// Ends a round: the keys become the state; crossing bounds are infeasible.
__global__ void k_na_finish(int32_t n, const uint8_t *vt, const long long *keys, double *lo,
                            double *hi, NoallocCtrl *ctrl, double eps_feas) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double L = okey_val(keys[2 * j]), U = okey_val(keys[2 * j + 1]);
  const bool cross = vt[j] ? (L > U) : (L > U + eps_feas * fmax(1.0, fabs(U)));
  if (cross) atomicExch(&ctrl->infeasible, 1);
  lo[j] = L;
  hi[j] = U;
}

// Device memory that `device` can read without peer access: memory allocated
// on that device, or managed memory.  A pointer to another GPU's memory is
// refused (reading it would need peer access the library never enables).
bool on_device(const void *p, int device) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == device;
}

// Device address of the scratch array on `device` (which must be current);
// looked up once per device.
long long *scratch_on(int device) {
  if (device < 0 || device >= kMaxDevices) return nullptr;
  long long *addr = g_scratch_addr[device].load(std::memory_order_acquire);
  if (!addr) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    addr = static_cast<long long *>(p);
    g_scratch_addr[device].store(addr, std::memory_order_release);
  }
  return addr;
}

// Makes `device` current for its lifetime and gives the caller's current
// device back on every return path.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
    ok = cudaSetDevice(device) == cudaSuccess;
    if (!ok) cudaGetLastError();
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int grid(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return (int)b;
}

}  // namespace

extern "C" int dp_propagate_noalloc(int device, void *cuda_stream, int32_t m, int32_t n,
                                    int64_t nnz, const int64_t *row_ptr,
                                    const int32_t *col_idx, const double *val,
                                    const double *lb, const double *ub,
                                    const uint8_t *vartype, const double *lhs,
                                    const double *rhs, const dp_params *params,
                                    double *lb_out, double *ub_out, int32_t *infeasible,
                                    int32_t *rounds) {
  dp::TraceRange trace_range("dp_propagate_noalloc");
  if (!infeasible || !rounds || m < 0 || n < 0 || nnz < 0) return DP_ERR_INVALID_ARG;
  if (n > DP_NOALLOC_MAX_VARS) return DP_ERR_INVALID_ARG;
  dp_params p;
  if (params) {
    p = *params;
  } else {
    std::memset(&p, 0, sizeof(p));
    p.max_rounds = 100;
    p.eps_int = 1e-6;
    p.tau_rel = 1e-6;
    p.eps_feas = 1e-6;
    p.inf_threshold = 1e20;
  }
  if (p.max_rounds < 0 || !(p.eps_int >= 0) || !(p.tau_rel >= 0) || !(p.eps_feas >= 0) ||
      !(p.inf_threshold > 0))
    return DP_ERR_INVALID_ARG;
  DeviceGuard guard(device);
  if (!guard.ok) return DP_ERR_INVALID_ARG;
  auto dev_ok = [device](const void *q) { return on_device(q, device); };
  if (!dev_ok(row_ptr) || (nnz > 0 && (!dev_ok(col_idx) || !dev_ok(val))))
    return DP_ERR_INVALID_ARG;
  if (n > 0 && (!dev_ok(lb) || !dev_ok(ub) || !dev_ok(vartype) || !dev_ok(lb_out) ||
                !dev_ok(ub_out)))
    return DP_ERR_INVALID_ARG;
  if (m > 0 && (!dev_ok(lhs) || !dev_ok(rhs))) return DP_ERR_INVALID_ARG;
  long long *scratch = scratch_on(device);
  if (!scratch) return DP_ERR_CUDA;
  long long *keys = scratch;
  NoallocCtrl *ctrl = reinterpret_cast<NoallocCtrl *>(scratch + 2 * (size_t)DP_NOALLOC_MAX_VARS);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  NoallocCtrl h;
  std::memset(&h, 0, sizeof(h));
  // the control block starts at zero on every call
  if (cudaMemsetAsync(ctrl, 0, sizeof(NoallocCtrl), st) != cudaSuccess) return DP_ERR_CUDA;
  int64_t work = nnz > (int64_t)n ? nnz : (int64_t)n;
  if ((int64_t)m + 1 > work) work = (int64_t)m + 1;
  k_na_prologue<<<grid(work, 256), 256, 0, st>>>(m, n, row_ptr, col_idx, val, nnz, lb, ub,
                                                 vartype, lhs, rhs, p.eps_int, p.inf_threshold,
                                                 lb_out, ub_out, keys, ctrl);
  if (cudaGetLastError() != cudaSuccess) return DP_ERR_CUDA;
  if (cudaMemcpyAsync(&h, ctrl, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return DP_ERR_CUDA;
  if (h.err) return h.err;

  int32_t r = 0;
  bool changed = false;
  for (; r < p.max_rounds;) {
    if (cudaMemsetAsync(ctrl, 0, sizeof(NoallocCtrl), st) != cudaSuccess) return DP_ERR_CUDA;
    if (m > 0)
      k_na_round<<<(int)((m + 127) / 128), 128, 0, st>>>(m, row_ptr, col_idx, val, lhs, rhs,
                                                          vartype, lb_out, ub_out, keys, ctrl,
                                                          p.eps_int, p.tau_rel, p.eps_feas,
                                                          p.inf_threshold);
    if (n > 0)
      k_na_finish<<<(int)((n + 255) / 256), 256, 0, st>>>(n, vartype, keys, lb_out, ub_out, ctrl,
                                                          p.eps_feas);
    if (cudaGetLastError() != cudaSuccess) return DP_ERR_CUDA;
    if (cudaMemcpyAsync(&h, ctrl, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return DP_ERR_CUDA;
    ++r;
    changed = h.changed != 0;
    if (h.infeasible || !changed) break;
  }
  *rounds = r;
  *infeasible = h.infeasible ? 1 : 0;
  if (!h.infeasible && changed && r >= p.max_rounds && p.max_rounds > 0) return DP_CAP_HIT;
  return DP_OK;
}
