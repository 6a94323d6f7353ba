// Device kernels of one propagation round (Alg. 2 of arXiv 2009.07785 with
// round-synchronous semantics) for sm_103a, plus the per-call prologue and
// epilogue.  All arithmetic that decides a bound is binary64; binary32 is
// used only in a conservative screen that proves some rows cannot tighten
// anything (their binary64 work is then skipped, with identical results).
//
// Round structure (all launched from a CUDA graph whose WHILE node repeats
// the round until k_finish clears the condition -- no host round trip):
//   k_round      one warp per slice, one lane per chunk: activities of every
//                chunk (Def. 1, Eq. 2a/2b, Sec. 3.4 infinity counts); for
//                whole rows also Step 2, the screen, and the candidates
//                (Eq. 3a/3b via Eq. 5a/5b) with filtered atomics (Sec. 3.5)
//   k_combine    one warp per split row: sums the chunk partials in a fixed
//                order, Step 2 and screen for the row
//   k_cand_split one lane per chunk of an active split row: candidates
//   k_finish     one thread per variable: decode the next state, crossing
//                test (Sec. 1.1, remark after Step 3), write the records the
//                next round gathers; the last block decides whether to loop
#include <cuda_runtime.h>
#include <cstdint>
#include <cfloat>

#include "dp_internal.h"
#include "dp_launch.h"
#include "../../include/domprop.h"

namespace dp {

// ---------------------------------------------------------------- helpers --

__device__ __forceinline__ bool d_isinf(double x) {
  return ((unsigned long long)__double_as_longlong(x) << 1) == 0xFFE0000000000000ull;
}
__device__ __forceinline__ bool d_isfinite(double x) {
  return ((__double2hiint(x) >> 20) & 0x7FF) != 0x7FF;
}
__device__ __forceinline__ bool d_isnan(double x) {
  return ((unsigned long long)__double_as_longlong(x) << 1) > 0xFFE0000000000000ull;
}
__device__ __forceinline__ bool d_is_neginf(double x) {
  return (unsigned long long)__double_as_longlong(x) == 0xFFF0000000000000ull;
}
__device__ __forceinline__ bool d_is_posinf(double x) {
  return (unsigned long long)__double_as_longlong(x) == 0x7FF0000000000000ull;
}
__device__ __forceinline__ double d_abs(double x) {
  return __longlong_as_double(__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll);
}
// coefficient sign without an FP64 comparison (coefficients are nonzero)
__device__ __forceinline__ bool d_pos(double a) { return __double2hiint(a) >= 0; }

// Order-preserving map between binary64 values and signed 64-bit keys, so
// that integer atomicMax/atomicMin implement max/min of doubles.
__device__ __forceinline__ long long key_of(double x) {
  long long b = __double_as_longlong(x);
  return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ double val_of_key(long long k) {
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7FFFFFFFFFFFFFFFll));
}

// A binary32 value >= x, from the bit pattern (IEEE 754 field layout), with
// no FP64-pipe conversion.  Truncates the significand toward zero and steps
// one unit up when bits were dropped from a positive value.
__device__ __forceinline__ float f32_up(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  unsigned mh = hi & 0x7FFFFFFFu;
  bool neg = (hi >> 31) != 0;
  unsigned e = mh >> 20;
  if (e == 0x7FFu) return __uint_as_float((hi & 0x80000000u) | 0x7F800000u);
  if (e >= 1151u) return neg ? -FLT_MAX : __uint_as_float(0x7F800000u);
  if (e < 897u) {
    if (neg) return -0.0f;
    return (mh | lo) ? FLT_MIN : 0.0f;
  }
  unsigned t = ((mh << 3) | (lo >> 29)) - (896u << 23);
  bool exact = (lo & 0x1FFFFFFFu) == 0u;
  if (!neg) return __uint_as_float(exact ? t : t + 1u);
  return -__uint_as_float(t);
}
__device__ __forceinline__ float f32_dn(double x) { return -f32_up(-x); }

// Upper bound on |a| as binary32 for |a| in [2^-126, 2^127); rows holding a
// coefficient outside [2^-120, 2^120] are flagged on the host and never use
// this value.
__device__ __forceinline__ float absup_fast(double a) {
  unsigned long long b = (unsigned long long)__double_as_longlong(a);
  unsigned mh = (unsigned)(b >> 32) & 0x7FFFFFFFu, lo = (unsigned)b;
  return __uint_as_float((((mh << 3) | (lo >> 29)) - (896u << 23)) + 1u);
}

// Upper bound on max(0, (U-L) + 2^-40 (|L|+|U|)) in binary32 (+inf if
// unbounded).  The 2^-40 term absorbs the rounding of the binary64 candidate
// formulas, so that the screen below stays sound even with tau_rel =
// eps_int = 0.  Clamping at 0 keeps |a|_up * W an upper bound when the
// bounds cross within the feasibility tolerance (U < L).
__device__ __forceinline__ float width_up(double L, double U) {
  float w = __fsub_ru(f32_up(U), f32_dn(L));
  float mg = __fmul_ru(0x1p-40f, __fadd_ru(f32_up(d_abs(L)), f32_up(d_abs(U))));
  return fmaxf(__fadd_ru(w, mg), 0.0f);
}

__device__ __forceinline__ void ld_rec(const VarRec *p, double &L, double &U,
                                       float &W, uint32_t &flags) {
  double d2, d3;
  asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
      : "=d"(L), "=d"(U), "=d"(d2), "=d"(d3)
      : "l"(p));
  long long w = __double_as_longlong(d2);
  W = __int_as_float((int)(w & 0xFFFFFFFFll));
  flags = (uint32_t)((unsigned long long)w >> 32);
}

__device__ __forceinline__ void st_rec(VarRec *p, double L, double U, float W,
                                       uint32_t flags) {
  long long w = (long long)(((unsigned long long)flags << 32) |
                            (unsigned long long)__float_as_uint(W));
  double d2 = __longlong_as_double(w);
  double d3 = 0.0;
  asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(L),
               "d"(U), "d"(d2), "d"(d3)
               : "memory");
}

__device__ __forceinline__ void set_flag(int32_t *f) {
  atomicExch(f, 1);
  __threadfence();
}

// ------------------------------------------------------- per-row decisions --

// Everything the candidate step needs to know about one row.
struct RowView {
  double minfin, maxfin, lhs, rhs;
  int32_t mininf, maxinf;
  float thr_r, thr_l;  // screen thresholds (see row_sides)
  bool act;            // some nonzero may produce an accepted candidate
};

// Step 2 of Sec. 1.1 for both sides of a row, and the binary32 screen.
//
// Screen (sound, never changes a result): for a > 0 the upper-bound
// candidate of x_j from the right-hand side is L_j + s/a with slack
// s = rhs - minact, and it can only be applied if s < a (U_j - L_j); the
// three other sign/side cases reduce to the same test s < |a| (U_j - L_j)
// with s the slack of that side.  With W_j >= (U_j-L_j) + 2^-40 (|L_j|+|U_j|)
// and t = an upper bound on |a| W_j, a side whose slack satisfies
//    s (1 - 2^-20) - 2^-40 (|side| + |activity|) >= t
// provably yields no accepted candidate for that nonzero, whatever the
// rounding of the binary64 formulas.  thr is a binary32 lower bound on the
// left-hand side; T is the row maximum of t.
__device__ __forceinline__ void row_sides(RowView &rv, float T, double eps_feas,
                                          int32_t *infeasible_flag) {
  bool infeas = false;
  bool act_r = false, act_l = false;
  rv.thr_r = __uint_as_float(0x7F800000u);
  rv.thr_l = __uint_as_float(0x7F800000u);
  if (d_isfinite(rv.rhs) && rv.mininf <= 1) {
    if (rv.mininf == 1) {
      act_r = true;  // only the nonzero with the infinite contribution
    } else {
      double s = rv.rhs - rv.minfin;
      if (s < 0.0) {
        double thr = rv.rhs + eps_feas * fmax(1.0, fabs(rv.rhs));
        if (rv.minfin > thr) infeas = true;
      }
      float sd = f32_dn(s);
      float mg = __fmul_ru(0x1p-40f, __fadd_ru(f32_up(d_abs(rv.rhs)), f32_up(d_abs(rv.minfin))));
      rv.thr_r = __fsub_rd(__fmul_rd(sd, 1.0f - 0x1p-20f), mg);
      act_r = T > rv.thr_r;
    }
  }
  if (d_isfinite(rv.lhs) && rv.maxinf <= 1) {
    if (rv.maxinf == 1) {
      act_l = true;
    } else {
      double s = rv.maxfin - rv.lhs;
      if (s < 0.0) {
        double thr = rv.lhs - eps_feas * fmax(1.0, fabs(rv.lhs));
        if (rv.maxfin < thr) infeas = true;
      }
      float sd = f32_dn(s);
      float mg = __fmul_ru(0x1p-40f, __fadd_ru(f32_up(d_abs(rv.lhs)), f32_up(d_abs(rv.maxfin))));
      rv.thr_l = __fsub_rd(__fmul_rd(sd, 1.0f - 0x1p-20f), mg);
      act_l = T > rv.thr_l;
    }
  }
  if (infeas) set_flag(infeasible_flag);
  rv.act = act_r || act_l;
}

// Bound candidates of one nonzero (Eq. 3a/3b in the residual form of
// Eq. 5a/5b, with the exactly-one-infinity rule of Sec. 3.4), integer
// rounding (Step 3), and the filtered atomic update (Sec. 3.5).  Candidates
// are compared with the bounds at the start of the round (L, U) and applied
// to the next state with order-preserving 64-bit atomics.
__device__ __forceinline__ void nnz_candidates(double a, int32_t j, double L,
                                               double U, float W,
                                               uint32_t flags, bool exact,
                                               const RowView &rv,
                                               const Ctrl &prm,
                                               long long *keys,
                                               int32_t *changed) {
  bool pos = d_pos(a);
  double bmin = pos ? L : U;
  double bmax = pos ? U : L;
  float t = exact ? __uint_as_float(0x7F800000u) : __fmul_ru(absup_fast(a), W);
  bool try_r = d_isfinite(rv.rhs) &&
               ((rv.mininf == 0 && t > rv.thr_r) || (rv.mininf == 1 && d_isinf(bmin)));
  bool try_l = d_isfinite(rv.lhs) &&
               ((rv.maxinf == 0 && t > rv.thr_l) || (rv.maxinf == 1 && d_isinf(bmax)));
  if (!try_r && !try_l) return;
  double lc = 0.0, uc = 0.0;
  bool hl = false, hu = false;
  if (try_r) {
    double res = (rv.mininf == 0) ? fma(-a, bmin, rv.minfin) : rv.minfin;
    if (d_isfinite(res)) {
      double c = (rv.rhs - res) / a;
      if (pos) { uc = c; hu = true; } else { lc = c; hl = true; }
    }
  }
  if (try_l) {
    double res = (rv.maxinf == 0) ? fma(-a, bmax, rv.maxfin) : rv.maxfin;
    if (d_isfinite(res)) {
      double c = (rv.lhs - res) / a;
      if (pos) { lc = c; hl = true; } else { uc = c; hu = true; }
    }
  }
  bool isint = (flags & 1u) != 0u;
  if (hl) {
    if (isint) lc = ceil(lc - prm.eps_int);
    if (!(fabs(lc) < prm.inf_thr)) hl = false;
  }
  if (hu) {
    if (isint) uc = floor(uc + prm.eps_int);
    if (!(fabs(uc) < prm.inf_thr)) hu = false;
  }
  if (hl) {
    bool acc;
    if (d_is_neginf(L)) acc = true;
    else if (isint) acc = lc > L;
    else acc = lc > L + prm.tau_rel * fmax(1.0, fabs(L));
    if (acc) {
      atomicMax(&keys[2 * (int64_t)j], key_of(lc));
      *changed = 1;
    }
  }
  if (hu) {
    bool acc;
    if (d_is_posinf(U)) acc = true;
    else if (isint) acc = uc < U;
    else acc = uc < U - prm.tau_rel * fmax(1.0, fabs(U));
    if (acc) {
      atomicMin(&keys[2 * (int64_t)j + 1], key_of(uc));
      *changed = 1;
    }
  }
}

// ------------------------------------------------------------- k_round --

constexpr int kRoundWarps = 8;

__global__ void __launch_bounds__(kRoundWarps * 32)
k_round(DevMatrix M, DevState S) {
  const Ctrl *ctrl = S.ctrl;
  if (ctrl->err) return;
  const int slice = blockIdx.x * kRoundWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (slice >= M.nslices) return;
  const int64_t c = (int64_t)slice * kSliceW + lane;
  const int32_t lenf = M.chunk_len[c];
  const int32_t len = lenf & kLenMask;
  const int32_t row = M.chunk_row[c];
  const int64_t base = M.slice_off[slice] + lane;
  const double *vp = M.val + base;
  const int32_t *cp = M.col + base;

  // ---- activities of the chunk (Def. 1, Eq. 2a/2b; Sec. 3.4) ----
  double minfin = 0.0, maxfin = 0.0;
  int32_t mininf = 0, maxinf = 0;
  float T = 0.0f;
  int k = 0;
  for (; k + 4 <= len; k += 4) {
    double a[4];
    int32_t j[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = __ldcs(vp + (int64_t)(k + u) * kSliceW);
      j[u] = __ldcs(cp + (int64_t)(k + u) * kSliceW);
    }
    double L[4], U[4];
    float W[4];
    uint32_t fl[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) ld_rec(S.rec + j[u], L[u], U[u], W[u], fl[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      bool pos = d_pos(a[u]);
      double bmin = pos ? L[u] : U[u];
      double bmax = pos ? U[u] : L[u];
      bool imin = d_isinf(bmin), imax = d_isinf(bmax);
      mininf += imin;
      maxinf += imax;
      minfin = fma(a[u], imin ? 0.0 : bmin, minfin);
      maxfin = fma(a[u], imax ? 0.0 : bmax, maxfin);
      T = fmaxf(T, __fmul_ru(absup_fast(a[u]), W[u]));
    }
  }
  for (; k < len; ++k) {
    double a = __ldcs(vp + (int64_t)k * kSliceW);
    int32_t j = __ldcs(cp + (int64_t)k * kSliceW);
    double L, U;
    float W;
    uint32_t fl;
    ld_rec(S.rec + j, L, U, W, fl);
    bool pos = d_pos(a);
    double bmin = pos ? L : U;
    double bmax = pos ? U : L;
    bool imin = d_isinf(bmin), imax = d_isinf(bmax);
    mininf += imin;
    maxinf += imax;
    minfin = fma(a, imin ? 0.0 : bmin, minfin);
    maxfin = fma(a, imax ? 0.0 : bmax, maxfin);
    T = fmaxf(T, __fmul_ru(absup_fast(a), W));
  }
  if (row < 0) return;  // padding lane
  const bool exact = (lenf & kExactFlag) != 0;
  if (exact) T = __uint_as_float(0x7F800000u);

  if (c < (int64_t)M.nslices_split * kSliceW) {
    // chunk of a split row: hand the partial sums to k_combine
    Partial p;
    p.minfin = minfin;
    p.maxfin = maxfin;
    p.mininf = mininf;
    p.maxinf = maxinf;
    p.T = T;
    p.exact = exact ? 1 : 0;
    S.part[c] = p;
    return;
  }

  // ---- whole row: Step 2, screen, candidates ----
  RowView rv;
  rv.minfin = minfin;
  rv.maxfin = maxfin;
  rv.mininf = mininf;
  rv.maxinf = maxinf;
  rv.lhs = S.lhs[row];
  rv.rhs = S.rhs[row];
  Ctrl prm = *ctrl;
  row_sides(rv, T, prm.eps_feas, &S.ctrl->infeasible);
  if (!rv.act) return;
  for (int q = 0; q < len; ++q) {
    double a = vp[(int64_t)q * kSliceW];
    int32_t j = cp[(int64_t)q * kSliceW];
    double L, U;
    float W;
    uint32_t fl;
    ld_rec(S.rec + j, L, U, W, fl);
    nnz_candidates(a, j, L, U, W, fl, exact, rv, prm, S.keys, &S.ctrl->changed);
  }
}

// ------------------------------------------------------------ k_combine --

constexpr int kCombineWarps = 8;

__global__ void __launch_bounds__(kCombineWarps * 32)
k_combine(DevMatrix M, DevState S) {
  const Ctrl *ctrl = S.ctrl;
  if (ctrl->err) return;
  const int w = blockIdx.x * kCombineWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= M.nsplit_rows) return;
  const int32_t cb = M.split_cbeg[w], ce = M.split_cbeg[w + 1];
  double mnf = 0.0, mxf = 0.0;
  int32_t mni = 0, mxi = 0, ex = 0;
  float T = 0.0f;
  for (int32_t c = cb + lane; c < ce; c += kSliceW) {
    Partial p = S.part[c];
    mnf += p.minfin;
    mxf += p.maxfin;
    mni += p.mininf;
    mxi += p.maxinf;
    T = fmaxf(T, p.T);
    ex |= p.exact;
  }
  // butterfly reduction: a fixed pattern, so the sum is reproducible and
  // identical in every lane (binary64 addition is commutative)
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mnf += __shfl_xor_sync(0xFFFFFFFFu, mnf, off);
    mxf += __shfl_xor_sync(0xFFFFFFFFu, mxf, off);
    mni += __shfl_xor_sync(0xFFFFFFFFu, mni, off);
    mxi += __shfl_xor_sync(0xFFFFFFFFu, mxi, off);
    T = fmaxf(T, __shfl_xor_sync(0xFFFFFFFFu, T, off));
    ex |= __shfl_xor_sync(0xFFFFFFFFu, ex, off);
  }
  if (lane != 0) return;
  const int32_t row = M.split_row[w];
  RowView rv;
  rv.minfin = mnf;
  rv.maxfin = mxf;
  rv.mininf = mni;
  rv.maxinf = mxi;
  rv.lhs = S.lhs[row];
  rv.rhs = S.rhs[row];
  if (ex) T = __uint_as_float(0x7F800000u);
  row_sides(rv, T, ctrl->eps_feas, &S.ctrl->infeasible);
  RowTot rt;
  rt.minfin = mnf;
  rt.maxfin = mxf;
  rt.mininf = mni;
  rt.maxinf = mxi;
  rt.thr_r = rv.thr_r;
  rt.thr_l = rv.thr_l;
  rt.active = rv.act ? 1 : 0;
  rt.row = row;
  S.rowtot[w] = rt;
}

// --------------------------------------------------------- k_cand_split --

__global__ void __launch_bounds__(kRoundWarps * 32)
k_cand_split(DevMatrix M, DevState S) {
  const Ctrl *ctrl = S.ctrl;
  if (ctrl->err) return;
  const int slice = blockIdx.x * kRoundWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (slice >= M.nslices_split) return;
  const int64_t c = (int64_t)slice * kSliceW + lane;
  const int32_t sidx = M.chunk_sidx[c];
  if (sidx < 0) return;
  const RowTot rt = S.rowtot[sidx];
  if (!rt.active) return;
  const int32_t lenf = M.chunk_len[c];
  const int32_t len = lenf & kLenMask;
  const bool exact = (lenf & kExactFlag) != 0;
  const int64_t base = M.slice_off[slice] + lane;
  RowView rv;
  rv.minfin = rt.minfin;
  rv.maxfin = rt.maxfin;
  rv.mininf = rt.mininf;
  rv.maxinf = rt.maxinf;
  rv.thr_r = rt.thr_r;
  rv.thr_l = rt.thr_l;
  rv.lhs = S.lhs[rt.row];
  rv.rhs = S.rhs[rt.row];
  rv.act = true;
  Ctrl prm = *ctrl;
  for (int q = 0; q < len; ++q) {
    double a = M.val[base + (int64_t)q * kSliceW];
    int32_t j = M.col[base + (int64_t)q * kSliceW];
    double L, U;
    float W;
    uint32_t fl;
    ld_rec(S.rec + j, L, U, W, fl);
    nnz_candidates(a, j, L, U, W, fl, exact, rv, prm, S.keys, &S.ctrl->changed);
  }
}

// ------------------------------------------------------------- k_finish --

constexpr int kFinishThreads = 256;

// Ends a round: the next state becomes the current one.  The last block to
// arrive (threadfence-reduction pattern; nobody waits) counts the round and
// sets the WHILE condition of the enclosing graph node.
__global__ void __launch_bounds__(kFinishThreads)
k_finish(DevState S, const uint8_t *vartype, int32_t n,
         cudaGraphConditionalHandle handle) {
  Ctrl *ctrl = S.ctrl;
  const int32_t err = ctrl->err;
  const double eps_feas = ctrl->eps_feas;
  if (!err) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
      longlong2 kk = reinterpret_cast<const longlong2 *>(S.keys)[j];
      double L = val_of_key(kk.x), U = val_of_key(kk.y);
      uint32_t vt = vartype[j] ? 1u : 0u;
      if (kk.x > kk.y) {  // L > U in key order: test the crossing exactly
        bool cross = vt ? (L > U) : (L > U + eps_feas * fmax(1.0, fabs(U)));
        if (cross) set_flag(&ctrl->infeasible);
      }
      st_rec(S.rec + j, L, U, width_up(L, U), vt);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned prev = atomicAdd(&ctrl->blocks_done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      volatile Ctrl *vc = ctrl;
      int32_t r = vc->round + 1;
      vc->round = r;
      int32_t ch = vc->changed;
      int32_t cont = (ch && !vc->infeasible && !vc->err && r < vc->max_rounds) ? 1 : 0;
      vc->last_changed = ch;
      vc->changed = 0;
      vc->blocks_done = 0;
      __threadfence();
      cudaGraphSetConditional(handle, (unsigned)cont);
    }
  }
}

// ------------------------------------------------------ prologue/epilogue --

// Normalises one call's inputs into the workspace: |v| >= inf_threshold
// becomes +-inf; integer bounds are rounded (ceil(lb - eps_int),
// floor(ub + eps_int)); NaN and contradictory infinities set ctrl->err.
__global__ void k_prologue(DevState S, uint8_t *vt_ws, int32_t m, int32_t n,
                           const double *lb, const double *ub,
                           const uint8_t *vartype, const double *lhs,
                           const double *rhs, double eps_int, double thr) {
  int64_t total = (int64_t)(n > m ? n : m);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      double L = lb[i], U = ub[i];
      uint8_t vt = vartype[i] ? 1 : 0;
      bool bad = d_isnan(L) || d_isnan(U) || L >= thr || U <= -thr;
      if (bad) {
        atomicExch(&S.ctrl->err, DP_ERR_NAN_INPUT);
        L = 0.0;
        U = 0.0;
      }
      if (L <= -thr) L = -__longlong_as_double(0x7FF0000000000000ll);
      if (U >= thr) U = __longlong_as_double(0x7FF0000000000000ll);
      if (vt) {
        if (d_isfinite(L)) L = ceil(L - eps_int);
        if (d_isfinite(U)) U = floor(U + eps_int);
      }
      reinterpret_cast<longlong2 *>(S.keys)[i] = make_longlong2(key_of(L), key_of(U));
      st_rec(S.rec + i, L, U, width_up(L, U), vt);
      vt_ws[i] = vt;
    }
    if (i < m) {
      double l = lhs[i], r = rhs[i];
      bool bad = d_isnan(l) || d_isnan(r) || l >= thr || r <= -thr;
      if (bad) {
        atomicExch(&S.ctrl->err, DP_ERR_NAN_INPUT);
        l = 0.0;
        r = 0.0;
      }
      if (l <= -thr) l = -__longlong_as_double(0x7FF0000000000000ll);
      if (r >= thr) r = __longlong_as_double(0x7FF0000000000000ll);
      S.lhs[i] = l;
      S.rhs[i] = r;
    }
  }
}

__global__ void k_epilogue(DevState S, int32_t n, double *lb_out,
                           double *ub_out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    longlong2 kk = reinterpret_cast<const longlong2 *>(S.keys)[j];
    lb_out[j] = val_of_key(kk.x);
    ub_out[j] = val_of_key(kk.y);
  }
}

// ------------------------------------------------------------ launchers --

static int grid_for(int64_t work, int threads, int max_blocks) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

cudaError_t launch_prologue(const DevState &S, uint8_t *vt_ws, int32_t m,
                            int32_t n, const double *lb, const double *ub,
                            const uint8_t *vartype, const double *lhs,
                            const double *rhs, double eps_int, double thr,
                            int num_sms, cudaStream_t st) {
  int64_t total = n > m ? n : m;
  k_prologue<<<grid_for(total, 256, num_sms * 16), 256, 0, st>>>(
      S, vt_ws, m, n, lb, ub, vartype, lhs, rhs, eps_int, thr);
  return cudaGetLastError();
}

cudaError_t launch_epilogue(const DevState &S, int32_t n, double *lb_out,
                            double *ub_out, int num_sms, cudaStream_t st) {
  k_epilogue<<<grid_for(n, 256, num_sms * 16), 256, 0, st>>>(S, n, lb_out, ub_out);
  return cudaGetLastError();
}

// Launches one round's kernels on `st` (called while `st` captures the body
// of the graph's WHILE node).
cudaError_t launch_round_body(const DevMatrix &M, const DevState &S,
                              const uint8_t *vt_ws,
                              cudaGraphConditionalHandle handle, int num_sms,
                              cudaStream_t st) {
  int nb = (M.nslices + kRoundWarps - 1) / kRoundWarps;
  if (nb < 1) nb = 1;
  k_round<<<nb, kRoundWarps * 32, 0, st>>>(M, S);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (M.nsplit_rows > 0) {
    int nbc = (M.nsplit_rows + kCombineWarps - 1) / kCombineWarps;
    k_combine<<<nbc, kCombineWarps * 32, 0, st>>>(M, S);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int nbs = (M.nslices_split + kRoundWarps - 1) / kRoundWarps;
    k_cand_split<<<nbs, kRoundWarps * 32, 0, st>>>(M, S);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  int nbf = grid_for(M.n, kFinishThreads, num_sms * 8);
  k_finish<<<nbf, kFinishThreads, 0, st>>>(S, vt_ws, M.n, handle);
  return cudaGetLastError();
}

}  // namespace dp
