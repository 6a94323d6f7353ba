// Device kernels of one propagation round (Alg. 2 of arXiv 2009.07785 with
// round-synchronous semantics) for sm_103a, plus the per-call prologue and
// epilogue.  All arithmetic that decides a bound is binary64; binary32 is
// used only in a conservative screen that proves that a nonzero cannot yield
// an accepted candidate (its binary64 candidate work is then skipped; the
// result is identical).
//
// Round structure (launched from a CUDA graph whose WHILE node repeats the
// round until k_finish clears the condition -- no host round trip):
//   k_round      one warp per slice, one lane per chunk: activities of every
//                chunk (Def. 1, Eq. 2a/2b, Sec. 3.4 infinity counts); for
//                whole rows also Step 2 and the binary32 screen, which
//                queues the nonzeros whose candidates may be accepted
//   k_combine    split rows of few pieces one per lane, rows of many pieces
//                one per warp: sums the chunk partials in a fixed order,
//                Step 2 and screen for the row
//   k_cand_split one lane per chunk of an active split row: queueing
//   k_cand_queue one thread per queued nonzero: the candidates (Eq. 3a/3b
//                via Eq. 5a/5b) with filtered atomics (Sec. 3.5); marks the
//                variables it updates in a dirty bitmap
//   k_finish     one warp per 8 bitmap words, per marked variable (the
//                warp together): decode the next state, crossing test
//                (Sec. 1.1, remark after Step 3), write the record the next
//                round gathers; the last block decides whether to loop
// (The merge-path layout replaces the first three by the kernels of
// dp_merge.cu.)
//
// GB300 has little binary64 throughput (about 0.5 T lane-ops/s, the same for
// any number of active lanes in a warp), so binary64 work is kept lane-dense:
// the activity sums run one chunk per lane over length-sorted slices, and
// candidate formulas run 32 at a time from a per-warp work list.
#include <cuda_runtime.h>
#include <cstdint>
#include <cfloat>
#include <type_traits>

#include "dp_device.cuh"
#include "dp_internal.h"
#include "dp_round.cuh"
#include "dp_launch.h"
#include "../../include/domprop.h"

namespace dp {

// Bound candidates of one nonzero from the sides that survived the screen
// (side_candidate), applied to the next state with order-preserving 64-bit
// atomics.  Candidates are compared with the bounds at the start of the
// round (L, U).  A variable that receives a candidate is marked in the
// round's dirty bitmap; the atomics return nothing, so none of them waits
// for its answer.
__device__ __forceinline__ void nnz_candidates(double a, int32_t j, double L, double U,
                                               uint32_t flags, unsigned sides,
                                               const RowView &rv, const Ctrl &prm,
                                               long long *keys, uint32_t *dirty,
                                               int32_t *changed) {
  const bool isint = (flags & 1u) != 0u;
  bool any = false;
  auto apply = [&](const SideCand &c) {
    if (!c.apply) return;
    if (c.upper) atomicMin(&keys[2 * (int64_t)j + 1], key_of(c.v));
    else atomicMax(&keys[2 * (int64_t)j], key_of(c.v));
    any = true;
  };
  apply(side_candidate(a, L, U, isint, (sides & 1u) != 0u, rv, prm.eps_int, prm.tau_rel,
                       prm.inf_thr));
  if (sides == 3u)  // both sides: the left-hand one too
    apply(side_candidate(a, L, U, isint, false, rv, prm.eps_int, prm.tau_rel, prm.inf_thr));
  if (any) {
    atomicOr(&dirty[j >> 5], 1u << (j & 31));
    *changed = 1;
  }
}

// ---------------------------------------------------------- k_cand_queue --

// One queued nonzero's operands: the entry, its row's sums and sides, its
// coefficient and column, and the start-of-round record of its variable.
struct QueuedNnz {
  CandEntry E;
  RowSum rs;
  double2 sd;
  double a;
  int32_t j;
  double L, U;
  float WU, WL;
  uint32_t fl;
};

// Evaluates kN queued nonzeros per thread (entries e0 + u*stride, u < kN,
// those below cnt): every load of one dependence level is issued for all
// of them before the next level, so kN chains are in flight at once.
template <bool kMulti, int kN, bool kCo = false>
__device__ __forceinline__ void cand_entries(const DevMatrix &M, const DevState &S,
                                             const Ctrl &prm, int64_t e0, int64_t stride,
                                             int32_t cnt) {
  QueuedNnz q[kN];
  bool ok[kN];
#pragma unroll
  for (int u = 0; u < kN; ++u) {
    ok[u] = e0 + u * stride < cnt;
    if (ok[u]) q[u].E = S.queue[e0 + u * stride];
  }
#pragma unroll
  for (int u = 0; u < kN; ++u) {
    if (!ok[u]) continue;
    const uint32_t c = q[u].E.cs >> 2;
    q[u].rs = S.rowsum[c];
    q[u].sd = S.side[c];
    q[u].a = ld_coef(M, q[u].E.off);
    q[u].j = M.col[q[u].E.off];
  }
#pragma unroll
  for (int u = 0; u < kN; ++u)
    if (ok[u]) ld_rec_t<kCo>(S.rec + q[u].j, q[u].L, q[u].U, q[u].WU, q[u].WL, q[u].fl);
#pragma unroll
  for (int u = 0; u < kN; ++u) {
    if (!ok[u]) continue;
    const uint32_t c = q[u].E.cs >> 2;
    RowView rv;
    rv.minfin = q[u].rs.minfin;
    rv.maxfin = q[u].rs.maxfin;
    rv.mininf = q[u].rs.mininf;
    rv.maxinf = q[u].rs.maxinf;
    rv.lhs = q[u].sd.x;
    rv.rhs = q[u].sd.y;
    rv.thr_r = rv.thr_l = f_inf();
    rv.exact = 0;
    rv.act = 1;
    int32_t *changed = kMulti ? &S.I.changed[S.I.slot_inst[c]] : &S.ctrl->changed;
    nnz_candidates(q[u].a, q[u].j, q[u].L, q[u].U, q[u].fl, q[u].E.cs & 3u, rv, prm, S.keys,
                   S.dirty, changed);
  }
}

// Evaluates the queued nonzeros, one per thread and step (grid-stride; the
// grid is sized to the blocks that fit on the GPU at once).
template <bool kMulti>
__global__ void __launch_bounds__(256) k_cand_queue(DevMatrix M, DevState S) {
  const Ctrl *ctrl = S.ctrl;
  if (ctrl->err) return;
  const int32_t cnt = ctrl->qcount;
  const Ctrl prm = *ctrl;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += stride)
    cand_entries<kMulti, 1>(M, S, prm, e, stride, cnt);
}

// ------------------------------------------------------------- k_round --

// Warps per block of k_round / k_cand_split: a launch shape the autotuner
// chooses (4 or 8); the register budget per thread stays the same (32
// resident warps per SM for a single problem, 24 for problem sets).
constexpr int kRoundWarpsPerSM = 32;
constexpr int kGroup = 2;         // slots per group in the activity loop
// the problem-set variant (more live state per lane) and the persistent
// kernel measured faster with fewer resident warps and longer groups
constexpr int kRoundWarpsPerSMMulti = 24;
constexpr int kGroupWide = 4;

// One slice of the round (warp-level: the 32 lanes are its 32 chunks).
// kVal8: the coefficients come from the int8 copy (converted when used, so
// that the prefetched loads stay in flight).  kCo: records are loaded
// through L2 (the persistent loop).
template <bool kMulti, bool kVal8, int kG = kGroup, bool kCo = false>
__device__ __forceinline__ void round_slice(const DevMatrix &M, const DevState &S, int slice) {
  const Ctrl *ctrl = S.ctrl;
  const int lane = threadIdx.x & 31;
  const int64_t c = (int64_t)slice * kSliceW + lane;
  const int32_t lenf = M.chunk_len[c];
  int32_t len = lenf & kLenMask;
  int32_t row = M.chunk_row[c];
  int32_t *inf_flag = &S.ctrl->infeasible;
  if (kMulti && row >= 0) {  // a stopped problem's rows do nothing
    const int32_t inst = S.I.slot_inst[c];
    if (S.I.done[inst]) {
      row = -1;
      len = 0;
    } else {
      inf_flag = &S.I.infeasible[inst];
    }
  }
  const int64_t sbase = M.slice_off[slice];
  const int32_t *scp = M.col + sbase;
  const int64_t vo = sbase + lane;
  const int32_t *cp = scp + lane;

  // A side's activity is needed only by rows whose side is finite (Step 2
  // and the candidates of that side); a warp skips the activity no lane
  // needs (warp-uniform: rows are ordered by side pattern when the sides
  // are known at load time).
  const double2 sd = (row >= 0) ? S.side[c] : make_double2(0.0, 0.0);  // slot order
  const bool need_min = __any_sync(kFull, row >= 0 && d_isfinite(sd.y));
  const bool need_max = __any_sync(kFull, row >= 0 && d_isfinite(sd.x));

  // ---- activities of the chunk (Def. 1, Eq. 2a/2b; Sec. 3.4) ----
  double minfin = 0.0, maxfin = 0.0;
  int32_t mininf = 0, maxinf = 0;
  Top2 t = top2_init();
  // groups of kG slots: all loads and gathers of a group are issued
  // before any is consumed, and the next group's values and columns are
  // fetched while this group's gathers are in flight; the last group's
  // missing slots are skipped (uniformly within a length-sorted slice)
  using Raw = typename std::conditional<kVal8, int, double>::type;
  auto raw = [&](int64_t off) -> Raw {
    if constexpr (kVal8) return (int)__ldcs(M.val8 + off);
    else return __ldcs(M.val + off);
  };
  auto coef = [](Raw r) -> double {
    if constexpr (kVal8) return small_int_to_double(r);
    else return r;
  };
  Raw an[kG];
  int32_t jn[kG];
#pragma unroll
  for (int u = 0; u < kG; ++u) {
    an[u] = (Raw)1;
    jn[u] = 0;
    if (u < len) {
      an[u] = raw(vo + (int64_t)u * kSliceW);
      jn[u] = __ldcs(cp + (int64_t)u * kSliceW);
    }
  }
  for (int k = 0; k < len; k += kG) {
    Raw a[kG];
    double L[kG], U[kG];
    float WU[kG], WL[kG];
    uint32_t fl[kG];
#pragma unroll
    for (int u = 0; u < kG; ++u) {
      a[u] = an[u];
      L[u] = U[u] = 0.0;
      WU[u] = WL[u] = 0.0f;
      if (k + u < len) ld_rec_t<kCo>(S.rec + jn[u], L[u], U[u], WU[u], WL[u], fl[u]);
    }
    if (k + kG < len) {
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        an[u] = (Raw)1;
        jn[u] = 0;
        if (k + kG + u < len) {
          an[u] = raw(vo + (int64_t)(k + kG + u) * kSliceW);
          jn[u] = __ldcs(cp + (int64_t)(k + kG + u) * kSliceW);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kG; ++u) {
      if (k + u < len) {
        const double av = coef(a[u]);
        bool pos = d_pos(av);
        float au = absup_fast(av), ad = absdn_fast(av);
        if (need_min) {
          double bmin = pos ? L[u] : U[u];
          bool imin = d_isinf(bmin);
          mininf += imin;
          if (imin) t.kinf_min = k + u;
          minfin = fma(av, imin ? 0.0 : bmin, minfin);
          top2_add(screen_prod(au, ad, pos ? WU[u] : WL[u]), k + u, t.r1, t.r2, t.kr);
        }
        if (need_max) {
          double bmax = pos ? U[u] : L[u];
          bool imax = d_isinf(bmax);
          maxinf += imax;
          if (imax) t.kinf_max = k + u;
          maxfin = fma(av, imax ? 0.0 : bmax, maxfin);
          top2_add(screen_prod(au, ad, pos ? WL[u] : WU[u]), k + u, t.l1, t.l2, t.kl);
        }
      }
    }
  }
  const bool exact = (lenf & kExactFlag) != 0;
  if (exact) t.r1 = t.r2 = t.l1 = t.l2 = f_inf();

  if (slice < M.nslices_split) {  // warp-uniform: split chunks only
    if (row >= 0) {
      Partial p;
      p.minfin = minfin;
      p.maxfin = maxfin;
      p.mininf = mininf;
      p.maxinf = maxinf;
      p.t = t;
      p.exact = exact ? 1 : 0;
      p.pad = 0;
      S.part[c] = p;
    }
    return;
  }

  // ---- whole rows: Step 2, screen, candidates ----
  RowView rv;
  rv.minfin = minfin;
  rv.maxfin = maxfin;
  rv.mininf = mininf;
  rv.maxinf = maxinf;
  rv.exact = exact ? 1 : 0;
  rv.act = 0;
  rv.thr_r = rv.thr_l = f_inf();
  if (row >= 0) {
    rv.lhs = sd.x;
    rv.rhs = sd.y;
    row_sides(rv, t.r1, t.l1, ctrl->eps_feas, inf_flag);
  } else {
    rv.lhs = rv.rhs = 0.0;
  }
  warp_enqueue<kSliceW, kCo>(rv, t, mininf, maxinf, len, c, sbase + lane, M, M.col, S);
}

template <bool kMulti, int kRoundWarps, bool kVal8>
__global__ void __launch_bounds__(kRoundWarps * 32,
                                  (kMulti ? kRoundWarpsPerSMMulti : kRoundWarpsPerSM) / kRoundWarps)
k_round(DevMatrix M, DevState S) {
  if (S.ctrl->err) return;
  const int slice = blockIdx.x * kRoundWarps + (threadIdx.x >> 5);
  if (slice >= M.nslices) return;  // warp-uniform
  round_slice<kMulti, kVal8, kMulti ? kGroupWide : kGroup>(M, S, slice);
}

// ------------------------------------------------------------- k_floor --
//
// The memory access pattern of k_round's activity pass alone, on the same
// layout and in the same launch shape: every slot's value and column
// streamed, every nonzero's 32-byte record gathered, no arithmetic beyond an
// integer fold that keeps the loads alive.  Its time is the floor that the
// round kernel's memory traffic sets on this matrix (a measurement, not part
// of propagation).
template <int kRoundWarps>
__global__ void __launch_bounds__(kRoundWarps * 32, kRoundWarpsPerSM / kRoundWarps)
k_floor(DevMatrix M, DevState S, unsigned *sink) {
  const int slice = blockIdx.x * kRoundWarps + (threadIdx.x >> 5);
  if (slice >= M.nslices) return;
  const int lane = threadIdx.x & 31;
  const int64_t c = (int64_t)slice * kSliceW + lane;
  const int32_t len = M.chunk_len[c] & kLenMask;
  const int64_t vo = M.slice_off[slice] + lane;
  unsigned acc = 0u;
  for (int k = 0; k < len; k += kGroup) {
    double a[kGroup];
    int32_t j[kGroup];
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      a[u] = 0.0;
      j[u] = 0;
      if (k + u < len) {
        a[u] = __ldcs(M.val + vo + (int64_t)(k + u) * kSliceW);
        j[u] = __ldcs(M.col + vo + (int64_t)(k + u) * kSliceW);
      }
    }
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      if (k + u < len) {
        double L, U;
        float WU, WL;
        uint32_t fl;
        ld_rec(S.rec + j[u], L, U, WU, WL, fl);
        acc ^= (unsigned)__double_as_longlong(L) ^ (unsigned)__double_as_longlong(a[u]) ^
               __float_as_uint(WU) ^ fl;
      }
    }
  }
  if (acc == 0x9E3779B9u) *sink = acc;  // practically never: keeps the loads
}

cudaError_t launch_access_floor(const DevMatrix &M, const DevState &S, unsigned *sink,
                                cudaStream_t st) {
  if (M.layout != kLayoutEll) return cudaErrorInvalidValue;
  const int w = M.round_warps == 4 ? 4 : 8;
  int nb = (M.nslices + w - 1) / w;
  if (nb < 1) nb = 1;
  if (w == 4) k_floor<4><<<nb, 4 * 32, 0, st>>>(M, S, sink);
  else k_floor<8><<<nb, 8 * 32, 0, st>>>(M, S, sink);
  return cudaGetLastError();
}

// ------------------------------------------------------------ k_combine --

constexpr int kCombineWarps = 8;
constexpr int kCombineShort = 4;  // rows with at most this many pieces: their own lane

// Running sums of a split row's pieces.
struct RowAcc {
  double mnf, mxf;
  int32_t mni, mxi, ex;
  float Tr, Tl;
};

__device__ __forceinline__ void acc_init(RowAcc &a) {
  a.mnf = a.mxf = 0.0;
  a.mni = a.mxi = a.ex = 0;
  a.Tr = a.Tl = -f_inf();
}

__device__ __forceinline__ void acc_add(RowAcc &a, const Partial &p) {
  a.mnf += p.minfin;
  a.mxf += p.maxfin;
  a.mni += p.mininf;
  a.mxi += p.maxinf;
  a.Tr = fmaxf(a.Tr, p.t.r1);
  a.Tl = fmaxf(a.Tl, p.t.l1);
  a.ex |= p.exact;
}

// Step 2 and the screen thresholds of split row w from its sums (thread-level).
__device__ __forceinline__ void combine_commit(const DevMatrix &M, const DevState &S, int64_t w,
                                               RowAcc &a, int32_t *inf_flag) {
  const int32_t row = M.split_row[w];
  RowView rv;
  rv.minfin = a.mnf;
  rv.maxfin = a.mxf;
  rv.mininf = a.mni;
  rv.maxinf = a.mxi;
  rv.lhs = S.lhs[row];
  rv.rhs = S.rhs[row];
  rv.exact = a.ex;
  if (a.ex) a.Tr = a.Tl = f_inf();
  row_sides(rv, a.Tr, a.Tl, S.ctrl->eps_feas, inf_flag);
  RowTot rt;
  rt.minfin = a.mnf;
  rt.maxfin = a.mxf;
  rt.mininf = a.mni;
  rt.maxinf = a.mxi;
  rt.thr_r = rv.thr_r;
  rt.thr_l = rv.thr_l;
  rt.active = rv.act;
  rt.row = row;
  S.rowtot[w] = rt;
}

// Warp w of the split-row pass (warp-level, all 32 lanes): rows [32w,
// 32w + 32) of at most kCombineShort pieces are summed each by its own lane
// in piece order; row w, if it has more pieces, by the whole warp, lanes
// strided over its pieces and then a fixed butterfly (reproducible, and the
// same in every lane).  Which of the two sums a row depends only on its
// piece count, and every row is summed once.
template <bool kMulti>
__device__ __forceinline__ void combine_rows(const DevMatrix &M, const DevState &S, int64_t w) {
  const int lane = threadIdx.x & 31;
  auto flag_of = [&](int32_t first_piece) -> int32_t * {
    return kMulti ? &S.I.infeasible[S.I.slot_inst[M.split_cidx[first_piece]]]
                  : &S.ctrl->infeasible;
  };
  auto stopped = [&](int32_t first_piece) {  // a stopped problem: no candidates
    return kMulti && S.I.done[S.I.slot_inst[M.split_cidx[first_piece]]];
  };
  // short rows, one per lane
  const int64_t r = w * 32 + lane;
  if (r < M.nsplit_rows) {
    const int32_t cb = M.split_cbeg[r], ce = M.split_cbeg[r + 1];
    if (ce - cb <= kCombineShort) {
      if (stopped(cb)) {
        S.rowtot[r].active = 0;
      } else {
        RowAcc a;
        acc_init(a);
        Partial p[kCombineShort];
#pragma unroll
        for (int u = 0; u < kCombineShort; ++u)
          if (cb + u < ce) p[u] = S.part[M.split_cidx[cb + u]];
#pragma unroll
        for (int u = 0; u < kCombineShort; ++u)
          if (cb + u < ce) acc_add(a, p[u]);
        combine_commit(M, S, r, a, flag_of(cb));
      }
    }
  }
  // row w if it has many pieces (warp-uniform)
  const int32_t b = M.split_cbeg[w], e = M.split_cbeg[w + 1];
  if (e - b <= kCombineShort) return;
  if (stopped(b)) {
    if (lane == 0) S.rowtot[w].active = 0;
    return;
  }
  RowAcc a;
  acc_init(a);
  // each lane sums its pieces in order; the loads of four pieces are issued
  // before they are consumed
  int32_t q = b + lane;
  for (; q + 3 * kSliceW < e; q += 4 * kSliceW) {
    int32_t ci[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) ci[u] = M.split_cidx[q + u * kSliceW];
    Partial p[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) p[u] = S.part[ci[u]];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc_add(a, p[u]);
  }
  for (; q < e; q += kSliceW) acc_add(a, S.part[M.split_cidx[q]]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a.mnf += __shfl_xor_sync(kFull, a.mnf, off);
    a.mxf += __shfl_xor_sync(kFull, a.mxf, off);
    a.mni += __shfl_xor_sync(kFull, a.mni, off);
    a.mxi += __shfl_xor_sync(kFull, a.mxi, off);
    a.Tr = fmaxf(a.Tr, __shfl_xor_sync(kFull, a.Tr, off));
    a.Tl = fmaxf(a.Tl, __shfl_xor_sync(kFull, a.Tl, off));
    a.ex |= __shfl_xor_sync(kFull, a.ex, off);
  }
  if (lane == 0) combine_commit(M, S, w, a, flag_of(b));
}

template <bool kMulti>
__global__ void __launch_bounds__(kCombineWarps * 32)
k_combine(DevMatrix M, DevState S) {
  if (S.ctrl->err) return;
  const int64_t w = blockIdx.x * (int64_t)kCombineWarps + (threadIdx.x >> 5);
  if (w >= M.nsplit_rows) return;  // warp-uniform
  combine_rows<kMulti>(M, S, w);
}

// --------------------------------------------------------- k_cand_split --

// Candidates of the active split rows' chunks of one slice (warp-level).
template <bool kCo = false>
__device__ __forceinline__ void cand_split_slice(const DevMatrix &M, const DevState &S,
                                                 int slice) {
  const int lane = threadIdx.x & 31;
  const int64_t c = (int64_t)slice * kSliceW + lane;
  const int32_t sidx = M.chunk_sidx[c];
  RowView rv;
  rv.act = 0;
  rv.exact = 0;
  rv.mininf = rv.maxinf = 0;
  rv.minfin = rv.maxfin = rv.lhs = rv.rhs = 0.0;
  rv.thr_r = rv.thr_l = f_inf();
  Top2 t = top2_init();
  int32_t len = 0, cmin = 0, cmax = 0;
  if (sidx >= 0) {
    const RowTot rt = S.rowtot[sidx];
    if (rt.active) {
      const Partial p = S.part[c];
      const int32_t lenf = M.chunk_len[c];
      len = lenf & kLenMask;
      rv.minfin = rt.minfin;
      rv.maxfin = rt.maxfin;
      rv.mininf = rt.mininf;
      rv.maxinf = rt.maxinf;
      rv.thr_r = rt.thr_r;
      rv.thr_l = rt.thr_l;
      rv.lhs = S.lhs[rt.row];
      rv.rhs = S.rhs[rt.row];
      rv.exact = (lenf & kExactFlag) ? 1 : 0;
      rv.act = 1;
      t = p.t;
      cmin = p.mininf;
      cmax = p.maxinf;
    }
  }
  const int64_t sbase = M.slice_off[slice];
  warp_enqueue<kSliceW, kCo>(rv, t, cmin, cmax, len, c, sbase + lane, M, M.col, S);
}

template <int kRoundWarps>
__global__ void __launch_bounds__(kRoundWarps * 32)
k_cand_split(DevMatrix M, DevState S) {
  if (S.ctrl->err) return;
  const int slice = blockIdx.x * kRoundWarps + (threadIdx.x >> 5);
  if (slice >= M.nslices_split) return;  // warp-uniform
  cand_split_slice(M, S, slice);
}

// ------------------------------------------------------------- k_finish --

constexpr int kFinishThreads = 256;

// Ends a round: the next state becomes the current one.  The last block to
// arrive (threadfence-reduction pattern; nobody waits) counts the round and
// sets the WHILE condition of the enclosing graph node.
// Commits one variable's next state (thread-level): the keys become the
// record the next round gathers; crossing bounds flag infeasibility.
template <bool kMulti>
__device__ __forceinline__ void finish_var(const DevState &S, const uint8_t *vartype, int64_t j,
                                           double eps_feas, float tau_dn, float eps_dn) {
  int32_t *inf_flag = &S.ctrl->infeasible;
  if (kMulti) {
    const int32_t inst = S.I.var_inst[j];
    if (S.I.done[inst]) return;  // a stopped problem keeps its bounds
    inf_flag = &S.I.infeasible[inst];
  }
  longlong2 kk = reinterpret_cast<const longlong2 *>(S.keys)[j];
  double L = val_of_key(kk.x), U = val_of_key(kk.y);
  uint32_t vt = vartype[j] ? 1u : 0u;
  if (kk.x > kk.y) {  // L > U in key order: test the crossing exactly
    bool cross = vt ? (L > U) : (L > U + eps_feas * d_max1abs(U));
    if (cross) set_flag(inf_flag);
  }
  write_var(S.rec + j, L, U, vt, tau_dn, eps_dn);
}

constexpr int kFinishWords = 8;  // bitmap words per warp and step of k_finish

// Commits the variables marked in words [w0, w0 + kFinishWords) of the
// dirty bitmap and clears those words (warp-level, all 32 lanes): lanes
// read one word each, then the warp commits the 32 variables of every
// nonzero word together.
template <bool kMulti>
__device__ __forceinline__ void finish_words(const DevState &S, const uint8_t *vartype,
                                             int64_t w0, int64_t nwords, double eps_feas,
                                             float tau_dn, float eps_dn) {
  const int lane = threadIdx.x & 31;
  const int64_t w = w0 + lane;
  uint32_t bits = 0u;
  if (lane < kFinishWords && w < nwords) {
    bits = S.dirty[w];
    if (bits) S.dirty[w] = 0u;
  }
  unsigned todo = __ballot_sync(kFull, bits != 0u);
  while (todo) {
    const int src = __ffs(todo) - 1;
    todo &= todo - 1u;
    const uint32_t b = __shfl_sync(kFull, bits, src);
    if ((b >> lane) & 1u)
      finish_var<kMulti>(S, vartype, (w0 + src) * 32 + lane, eps_feas, tau_dn, eps_dn);
  }
}

// Ends a round (one block, all threads; after every variable is committed):
// counts the round, resets the round's counters and returns whether to
// continue.  For a problem set each problem counts its rounds and stops on
// its own (no change, infeasible, or the cap); the loop runs while any
// problem is live.
template <bool kMulti>
__device__ __forceinline__ int decide_round(const DevState &S) {
  volatile Ctrl *vc = S.ctrl;
  const int32_t r = vc->round + 1;
  int32_t cont;
  if (kMulti) {
    volatile int32_t *ch = S.I.changed, *inf = S.I.infeasible, *dn = S.I.done;
    int live = 0;
    for (int i = threadIdx.x; i < S.I.ninst; i += blockDim.x) {
      if (dn[i]) continue;
      const int32_t ri = S.I.rounds[i] + 1;
      S.I.rounds[i] = ri;
      int32_t d = 0;
      if (inf[i]) d = 1;
      else if (!ch[i]) d = 1;
      else if (ri >= vc->max_rounds) {
        d = 1;
        S.I.status[i] = 1;
      }
      dn[i] = d;
      ch[i] = 0;
      live |= !d;
    }
    live = __syncthreads_or(live);
    cont = (live && !vc->err && r < vc->max_rounds) ? 1 : 0;
    if (threadIdx.x == 0) vc->last_changed = live;
  } else {
    const int32_t chg = vc->changed;
    cont = (chg && !vc->infeasible && !vc->err && r < vc->max_rounds) ? 1 : 0;
    __syncthreads();
    if (threadIdx.x == 0) vc->last_changed = chg;
  }
  if (threadIdx.x == 0) {
    vc->round = r;
    vc->changed = 0;
    vc->qcount = 0;
    vc->cont = cont;
    __threadfence();
  }
  return cont;
}

// Ends a round: every variable's next state becomes the current one.  The
// last block to arrive (threadfence-reduction pattern; nobody waits) decides
// whether to loop and sets the WHILE condition of the enclosing graph node.
template <bool kMulti>
__global__ void __launch_bounds__(kFinishThreads)
k_finish(DevState S, const uint8_t *vartype, int32_t n, cudaGraphConditionalHandle handle,
         int use_cond) {
  Ctrl *ctrl = S.ctrl;
  const int32_t err = ctrl->err;
  const double eps_feas = ctrl->eps_feas;
  const float tau_dn = f32_dn(ctrl->tau_rel), eps_dn = f32_dn(ctrl->eps_int);
  if (!err) {  // only variables whose next state changed (the dirty bitmap)
    const int64_t nwords = ((int64_t)n + 31) >> 5;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w0 = warp * kFinishWords; w0 < nwords; w0 += nwarps * kFinishWords)
      finish_words<kMulti>(S, vartype, w0, nwords, eps_feas, tau_dn, eps_dn);
  }
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned prev = atomicAdd(&ctrl->blocks_done, 1u);
    s_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int cont = decide_round<kMulti>(S);
  if (threadIdx.x == 0) {
    ctrl->blocks_done = 0;
    __threadfence();
    if (use_cond) cudaGraphSetConditional(handle, (unsigned)cont);
  }
}

// ------------------------------------------------------- persistent loop --
//
// The whole round loop as one cooperative launch (every block resident):
// the round's phases are separated by grid barriers instead of kernel
// boundaries, and the loop condition is read by every block after the last
// barrier of a round -- the paper's device-driven loop (Sec. 3.7) as a
// single persistent kernel, measured against the graph's WHILE node.

constexpr int kPersistThreads = 256;
// Grid-wide barrier (sense by generation count).  Bounded: a block that
// waits more than `limit` sleeps of 64 ns records DP_ERR_TIMEOUT and leaves;
// every block returns false once an error is recorded.  Cannot deadlock
// under a cooperative launch, which guarantees that all blocks are resident.
__device__ __forceinline__ bool grid_sync(const DevState &S, long long limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = S.bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(S.bar, 1u) == gridDim.x - 1) {
      S.bar[0] = 0u;  // every block has arrived; none leaves before gen moves
      __threadfence();
      atomicAdd(S.bar + 1, 1u);
    } else {
      long long it = 0;
      while (*gen == g) {
        if (++it > limit) {
          atomicExch(&S.ctrl->err, DP_ERR_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ((volatile Ctrl *)S.ctrl)->err == 0;
}

// Two resident blocks per SM: the union of all phases needs more registers
// than three blocks allow (spills), and fewer resident warps hide less latency.
// kMulti: a problem set (per-problem termination, as the graph's kernels).
template <bool kMulti>
__global__ void __launch_bounds__(kPersistThreads, 2)
k_persistent(DevMatrix M, DevState S, const uint8_t *vartype) {
  if (((volatile Ctrl *)S.ctrl)->err) return;  // set before the launch: uniform
  const Ctrl prm = *S.ctrl;  // parameters (constant during the run)
  const long long lim = prm.wait_limit;
  const float tau_dn = f32_dn(prm.tau_rel), eps_dn = f32_dn(prm.eps_int);
  const int wpb = kPersistThreads / 32;
  const int gw = blockIdx.x * wpb + (threadIdx.x >> 5), nw = gridDim.x * wpb;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  for (;;) {
    if (M.val8)
      for (int sl = gw; sl < M.nslices; sl += nw)
        round_slice<kMulti, true, kGroupWide, true>(M, S, sl);
    else
      for (int sl = gw; sl < M.nslices; sl += nw)
        round_slice<kMulti, false, kGroupWide, true>(M, S, sl);
    if (!grid_sync(S, lim)) return;
    if (M.nsplit_rows > 0) {
      for (int w = gw; w < M.nsplit_rows; w += nw) combine_rows<kMulti>(M, S, w);
      if (!grid_sync(S, lim)) return;
      for (int sl = gw; sl < M.nslices_split; sl += nw) cand_split_slice<true>(M, S, sl);
      if (!grid_sync(S, lim)) return;
    }
    const int32_t cnt = ((volatile Ctrl *)S.ctrl)->qcount;
    for (int64_t e = gt; e < cnt; e += nt) cand_entries<kMulti, 1, true>(M, S, prm, e, nt, cnt);
    if (!grid_sync(S, lim)) return;
    for (int64_t w0 = (gt >> 5) * kFinishWords; w0 < ((int64_t)M.n + 31) >> 5;
         w0 += (nt >> 5) * kFinishWords)
      finish_words<kMulti>(S, vartype, w0, ((int64_t)M.n + 31) >> 5, prm.eps_feas, tau_dn, eps_dn);
    if (!grid_sync(S, lim)) return;
    if (blockIdx.x == 0) decide_round<kMulti>(S);
    if (!grid_sync(S, lim)) return;
    if (!((volatile Ctrl *)S.ctrl)->cont) return;
  }
}

// ------------------------------------------------------ prologue/epilogue --

// Normalises one call's inputs into the workspace: |v| >= inf_threshold
// becomes +-inf; integer bounds are rounded (ceil(lb - eps_int),
// floor(ub + eps_int)); NaN and contradictory infinities set ctrl->err.
__global__ void k_prologue(DevState S, uint8_t *vt_ws, int32_t m, int32_t n,
                           const double *lb, const double *ub, const uint8_t *vartype,
                           const double *lhs, const double *rhs, double eps_int,
                           double tau_rel, double thr) {
  const float tau_dn = f32_dn(tau_rel), eps_dn = f32_dn(eps_int);
  const double pinf = __longlong_as_double(0x7FF0000000000000ll);
  int64_t total = (int64_t)(n > m ? n : m);
  const int lane = threadIdx.x & 31;
  // warp-uniform loop (the block size and the stride are multiples of 32)
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); i0 < total;
       i0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = i0 + lane;
    bool cross = false;
    if (i < n) {
      double L = lb[i], U = ub[i];
      uint8_t vt = vartype[i] ? 1 : 0;
      bool bad = d_isnan(L) || d_isnan(U) || L >= thr || U <= -thr;
      if (bad) {
        atomicExch(&S.ctrl->err, DP_ERR_NAN_INPUT);
        L = 0.0;
        U = 0.0;
      }
      if (L <= -thr) L = -pinf;
      if (U >= thr) U = pinf;
      if (vt) {
        if (d_isfinite(L)) L = ceil(L - eps_int);
        if (d_isfinite(U)) U = floor(U + eps_int);
      }
      reinterpret_cast<longlong2 *>(S.keys)[i] = make_longlong2(key_of(L), key_of(U));
      write_var(S.rec + i, L, U, vt, tau_dn, eps_dn);
      vt_ws[i] = vt;
      cross = key_of(L) > key_of(U);
    }
    // A round commits only the variables marked in the dirty bitmap; bounds
    // that cross on input are marked for round 1, whose commit tests them.
    // Writing whole words also clears what an aborted call left behind.
    const unsigned cw = __ballot_sync(kFull, cross);
    if (i0 < n && lane == 0) S.dirty[i0 >> 5] = cw;
    if (i < m) {
      double l = lhs[i], r = rhs[i];
      bool bad = d_isnan(l) || d_isnan(r) || l >= thr || r <= -thr;
      if (bad) {
        atomicExch(&S.ctrl->err, DP_ERR_NAN_INPUT);
        l = 0.0;
        r = 0.0;
      }
      if (l <= -thr) l = -pinf;
      if (r >= thr) r = pinf;
      S.lhs[i] = l;
      S.rhs[i] = r;
    }
  }
}

// Copies the normalised sides of each chunk's row into slot order, so that
// the round kernel reads them coalesced.
__global__ void k_prologue_sides(DevMatrix M, DevState S, const double *lhs, const double *rhs,
                                 double thr) {
  const double pinf = __longlong_as_double(0x7FF0000000000000ll);
  const int64_t nslots = (int64_t)M.nslices * kSliceW;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nslots;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int32_t row = M.chunk_row[c];
    double l = 0.0, r = 0.0;
    if (row >= 0) {
      l = lhs[row];
      r = rhs[row];
      if (l <= -thr) l = -pinf;
      if (r >= thr) r = pinf;
    }
    S.side[c] = make_double2(l, r);
  }
}

__global__ void k_epilogue(DevState S, int32_t n, double *lb_out, double *ub_out) {
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

cudaError_t launch_prologue(const DevMatrix &M, const DevState &S, uint8_t *vt_ws, int32_t m,
                            int32_t n, const double *lb, const double *ub,
                            const uint8_t *vartype, const double *lhs, const double *rhs,
                            double eps_int, double tau_rel, double thr, int num_sms,
                            cudaStream_t st) {
  int64_t total = n > m ? n : m;
  k_prologue<<<grid_for(total, 256, num_sms * 16), 256, 0, st>>>(
      S, vt_ws, m, n, lb, ub, vartype, lhs, rhs, eps_int, tau_rel, thr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (m > 0) {
    k_prologue_sides<<<grid_for((int64_t)M.nslices * kSliceW, 256, num_sms * 16), 256, 0, st>>>(
        M, S, lhs, rhs, thr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && M.layout == kLayoutMerge) e = launch_merge_prologue(M, S, st);
  return e;
}

cudaError_t launch_epilogue(const DevState &S, int32_t n, double *lb_out, double *ub_out,
                            int num_sms, cudaStream_t st) {
  k_epilogue<<<grid_for(n, 256, num_sms * 16), 256, 0, st>>>(S, n, lb_out, ub_out);
  return cudaGetLastError();
}

// The sliced-ELL part of a round: activities, split rows, Step 2 and the
// screen (events ev[0..5] as in launch_round_kernels).
template <bool kMulti, int kRoundWarps>
cudaError_t launch_ell_front(const DevMatrix &M, const DevState &S, cudaStream_t st,
                             cudaEvent_t *ev) {
  cudaError_t e;
  int nb = (M.nslices + kRoundWarps - 1) / kRoundWarps;
  if (nb < 1) nb = 1;
  if (ev) cudaEventRecord(ev[0], st);
  if (M.val8)
    k_round<kMulti, kRoundWarps, true><<<nb, kRoundWarps * 32, 0, st>>>(M, S);
  else
    k_round<kMulti, kRoundWarps, false><<<nb, kRoundWarps * 32, 0, st>>>(M, S);
  if (ev) cudaEventRecord(ev[1], st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (M.nsplit_rows > 0) {
    int nbc = (M.nsplit_rows + kCombineWarps - 1) / kCombineWarps;  // a warp per row
    if (ev) cudaEventRecord(ev[2], st);
    k_combine<kMulti><<<nbc, kCombineWarps * 32, 0, st>>>(M, S);
    if (ev) cudaEventRecord(ev[3], st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int nbs = (M.nslices_split + kRoundWarps - 1) / kRoundWarps;
    if (ev) cudaEventRecord(ev[4], st);
    k_cand_split<kRoundWarps><<<nbs, kRoundWarps * 32, 0, st>>>(M, S);
    if (ev) cudaEventRecord(ev[5], st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <bool kMulti, int kRoundWarps>
cudaError_t launch_round_t(const DevMatrix &M, const DevState &S, const uint8_t *vt_ws,
                           cudaGraphConditionalHandle handle, int use_cond, int num_sms,
                           cudaStream_t st, cudaEvent_t *ev) {
  cudaError_t e = M.layout == kLayoutMerge ? launch_merge_front(M, S, num_sms, st, ev)
                                           : launch_ell_front<kMulti, kRoundWarps>(M, S, st, ev);
  if (e != cudaSuccess) return e;
  // the queue kernel's grid: the blocks that are resident at once (a
  // larger grid-stride grid would run its last blocks as a second wave)
  static int queue_blocks_per_sm = 0;
  if (queue_blocks_per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cand_queue<kMulti>, 256, 0) !=
            cudaSuccess ||
        b < 1)
      b = 4;
    queue_blocks_per_sm = b;
  }
  if (ev) cudaEventRecord(ev[8], st);
  k_cand_queue<kMulti><<<num_sms * queue_blocks_per_sm, 256, 0, st>>>(M, S);
  if (ev) cudaEventRecord(ev[9], st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // one warp per kFinishWords bitmap words
  int nbf = grid_for(((int64_t)M.n + 31) / 32 * 32 / kFinishWords, kFinishThreads, num_sms * 6);
  if (ev) cudaEventRecord(ev[6], st);
  k_finish<kMulti><<<nbf, kFinishThreads, 0, st>>>(S, vt_ws, M.n, handle, use_cond);
  if (ev) cudaEventRecord(ev[7], st);
  return cudaGetLastError();
}

// Launches one round's kernels on `st`.  In the graph body (use_cond = 1)
// k_finish sets the WHILE condition; in the host-driven loop it does not.
// With `ev` (10 events) each kernel is bracketed by a pair of events.  A
// problem set (S.I.ninst > 0) runs the per-problem variants.
cudaError_t launch_round_kernels(const DevMatrix &M, const DevState &S, const uint8_t *vt_ws,
                                 cudaGraphConditionalHandle handle, int use_cond, int num_sms,
                                 cudaStream_t st, cudaEvent_t *ev) {
  const bool w4 = M.round_warps == 4;
  if (S.I.ninst > 0)
    return w4 ? launch_round_t<true, 4>(M, S, vt_ws, handle, use_cond, num_sms, st, ev)
              : launch_round_t<true, 8>(M, S, vt_ws, handle, use_cond, num_sms, st, ev);
  return w4 ? launch_round_t<false, 4>(M, S, vt_ws, handle, use_cond, num_sms, st, ev)
            : launch_round_t<false, 8>(M, S, vt_ws, handle, use_cond, num_sms, st, ev);
}

cudaError_t launch_persistent(const DevMatrix &M, const DevState &S, const uint8_t *vt_ws,
                              int num_sms, cudaStream_t st) {
  const void *kern = S.I.ninst > 0 ? (const void *)k_persistent<true>
                                    : (const void *)k_persistent<false>;
  int per_sm = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPersistThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  if ((e = cudaMemsetAsync(S.bar, 0, 2 * sizeof(unsigned), st)) != cudaSuccess) return e;
  DevMatrix m = M;
  DevState s = S;
  const uint8_t *vt = vt_ws;
  void *args[] = {&m, &s, &vt};
  return cudaLaunchCooperativeKernel(kern, dim3(num_sms * per_sm), dim3(kPersistThreads), args,
                                     0, st);
}

cudaError_t launch_round_body(const DevMatrix &M, const DevState &S, const uint8_t *vt_ws,
                              cudaGraphConditionalHandle handle, int num_sms,
                              cudaStream_t st) {
  return launch_round_kernels(M, S, vt_ws, handle, 1, num_sms, st, nullptr);
}

}  // namespace dp
