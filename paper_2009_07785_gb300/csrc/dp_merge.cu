// Merge-path round kernels (layout kLayoutMerge, described in dp_internal.h):
// an alternative load balancing of the activity computation (Def. 1,
// Eq. 2a/2b with the infinity counts of Sec. 3.4) to the length-sorted
// slices of dp_kernels.cu.  Per round:
//   k_mp_act   one thread per segment of ipt items of the merged sequence
//              of row ends and nonzeros: sums its rows' nonzeros in CSR
//              order and tracks the binary32 screen's top-2 per side; a row
//              that ends in the segment and began in it is complete
//              (written to rowact), the first row's piece when that row
//              began earlier is the segment's head, the piece of a row still
//              open at the end is its carry
//   k_mp_fix   one thread per split row (one warp for rows of many
//              pieces): adds the row's pieces in segment order
//   k_mp_rows  one lane per row: Step 2 and the screen; queues the
//              nonzeros that survive it for k_cand_queue (dp_kernels.cu),
//              which computes their candidates exactly as for the other
//              layout, and k_finish commits the round
//   k_mp_long  one warp per piece of a long row whose screen needs every
//              nonzero re-read (the lane-level re-read would serialise it)
// A row inside one segment is summed in exactly the order of the oracle;
// a split row in segment order of its pieces (within the parity tolerance).
#include <cuda_runtime.h>
#include <cstdint>

#include "dp_device.cuh"
#include "dp_internal.h"
#include "dp_launch.h"
#include "dp_round.cuh"

namespace dp {
namespace {

constexpr int kMpGroup = 4;        // nonzeros of a thread whose loads are in flight together
constexpr int kMpWarpsPerSM = 24;  // occupancy target of the activity pass
constexpr int kMpFixShort = 8;     // split rows with at most this many pieces: one lane

__device__ __forceinline__ void part_clear(Partial &p) {
  p.minfin = p.maxfin = 0.0;
  p.mininf = p.maxinf = 0;
  p.t = top2_init();
  p.exact = 0;
  p.pad = 0;
}

// Activities each warp of the activity pass needs (bit 0: minimum, for rows
// with a finite right-hand side; bit 1: maximum, for a finite left-hand
// side): every row a segment touches -- the rows that end in it and the one
// open at its end -- counts for the segment's warp.
__global__ void k_mp_need(DevMatrix M, DevState S) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((t & ~(int64_t)31) >= M.mp_nseg) return;  // warp-uniform
  unsigned bits = 0u;
  if (t < M.mp_nseg) {
    const int32_t r0 = M.mp_srow[t], r1 = M.mp_srow[t + 1];
    for (int32_t p = r0; p <= r1 && p < M.m; ++p) {
      const double2 sd = S.side[p];
      if (d_isfinite(sd.y)) bits |= 1u;
      if (d_isfinite(sd.x)) bits |= 2u;
    }
  }
  bits = __reduce_or_sync(kFull, bits);
  if ((threadIdx.x & 31) == 0) S.mp_need[t >> 5] = bits;
}

template <int kWarps>
__global__ void __launch_bounds__(kWarps * 32, kMpWarpsPerSM / kWarps)
k_mp_act(DevMatrix M, DevState S) {
  if (S.ctrl->err) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((t & ~(int64_t)31) >= M.mp_nseg) return;  // warp-uniform
  // a side's activity is skipped by warps none of whose rows need it
  const unsigned need = S.mp_need[t >> 5];
  const bool need_min = (need & 1u) != 0u, need_max = (need & 2u) != 0u;
  const bool valid = t < M.mp_nseg;
  const int64_t total = (int64_t)M.m + M.nnz;
  const int64_t d0 = t * M.mp_ipt;
  const int64_t d1 = valid ? (d0 + M.mp_ipt < total ? d0 + M.mp_ipt : total) : d0;
  const int32_t *ptr = M.mp_ptr;
  // merge coordinates: rows [p, p_end) end in this segment; its nonzeros
  // are [k, k_end)
  int32_t p = valid ? M.mp_srow[t] : M.m;
  const int32_t p_end = valid ? M.mp_srow[t + 1] : M.m;
  const int32_t k0 = (int32_t)(d0 - p);
  const int32_t k_end = valid ? (int32_t)(d1 - p_end) : k0;
  int32_t rbeg = p < M.m ? ptr[p] : (int32_t)M.nnz;
  int32_t rend = p < M.m ? ptr[p + 1] : rbeg;
  int32_t rnext = p + 1 < M.m ? ptr[p + 2] : rend;  // next row's end, fetched ahead
  bool head = p < M.m && (int64_t)p + rbeg < d0;    // the first row began earlier

  double minfin = 0.0, maxfin = 0.0;
  int32_t mininf = 0, maxinf = 0;
  Top2 tt = top2_init();
  auto store = [&](Partial *dst) {
    Partial o;
    o.minfin = minfin;
    o.maxfin = maxfin;
    o.mininf = mininf;
    o.maxinf = maxinf;
    o.t = tt;
    o.exact = 0;
    o.pad = 0;
    *dst = o;
  };
  auto row_end = [&]() {  // row p ends: its sums (or its head piece) are final
    store(head ? S.part + 2 * t : S.rowact + p);
    minfin = maxfin = 0.0;
    mininf = maxinf = 0;
    tt = top2_init();
    head = false;
    ++p;
    rbeg = rend;
    rend = rnext;
    if (p + 1 < M.m) rnext = ptr[p + 2];
  };

  const int32_t nz = k_end - k0;
  for (int32_t g = 0; g < nz; g += kMpGroup) {
    double a[kMpGroup], L[kMpGroup], U[kMpGroup];
    float WU[kMpGroup], WL[kMpGroup];
    uint32_t fl[kMpGroup];
    int32_t j[kMpGroup];
#pragma unroll
    for (int u = 0; u < kMpGroup; ++u) {
      a[u] = 1.0;
      j[u] = 0;
      if (g + u < nz) {
        a[u] = __ldg(M.val + k0 + g + u);
        j[u] = __ldg(M.col + k0 + g + u);
      }
    }
#pragma unroll
    for (int u = 0; u < kMpGroup; ++u) {
      L[u] = U[u] = 0.0;
      WU[u] = WL[u] = 0.0f;
      if (g + u < nz) ld_rec(S.rec + j[u], L[u], U[u], WU[u], WL[u], fl[u]);
    }
#pragma unroll
    for (int u = 0; u < kMpGroup; ++u) {
      if (g + u < nz) {
        const int32_t kk = k0 + g + u;
        while (kk >= rend && p < M.m) row_end();  // rows (empty ones too) ending before kk
        const int32_t kr = kk - rbeg;  // position within the row
        const double av = a[u];
        const bool pos = d_pos(av);
        const float au = absup_fast(av), ad = absdn_fast(av);
        if (need_min) {
          const double bmin = pos ? L[u] : U[u];
          const bool imin = d_isinf(bmin);
          mininf += imin;
          if (imin) tt.kinf_min = kr;
          minfin = fma(av, imin ? 0.0 : bmin, minfin);
          top2_add(screen_prod(au, ad, pos ? WU[u] : WL[u]), kr, tt.r1, tt.r2, tt.kr);
        }
        if (need_max) {
          const double bmax = pos ? U[u] : L[u];
          const bool imax = d_isinf(bmax);
          maxinf += imax;
          if (imax) tt.kinf_max = kr;
          maxfin = fma(av, imax ? 0.0 : bmax, maxfin);
          top2_add(screen_prod(au, ad, pos ? WL[u] : WU[u]), kr, tt.l1, tt.l2, tt.kl);
        }
      }
    }
  }
  while (p < p_end) row_end();  // rows ending after the segment's last nonzero
  // a row still open at the end (begun here or earlier) leaves a carry
  if (valid && p < M.m && k_end > rbeg) store(S.part + 2 * t + 1);
}

// Adds piece q after the pieces already in acc (segment order).  The top-2
// of the screen values merge exactly: the largest of the union and the
// largest of the rest.
__device__ __forceinline__ void piece_add(Partial &acc, const Partial &q) {
  acc.minfin += q.minfin;
  acc.maxfin += q.maxfin;
  if (q.mininf > 0) acc.t.kinf_min = q.t.kinf_min;
  if (q.maxinf > 0) acc.t.kinf_max = q.t.kinf_max;
  acc.mininf += q.mininf;
  acc.maxinf += q.maxinf;
  if (q.t.r1 > acc.t.r1) {
    acc.t.r2 = fmaxf(acc.t.r1, fmaxf(acc.t.r2, q.t.r2));
    acc.t.r1 = q.t.r1;
    acc.t.kr = q.t.kr;
  } else {
    acc.t.r2 = fmaxf(acc.t.r2, fmaxf(q.t.r1, q.t.r2));
  }
  if (q.t.l1 > acc.t.l1) {
    acc.t.l2 = fmaxf(acc.t.l1, fmaxf(acc.t.l2, q.t.l2));
    acc.t.l1 = q.t.l1;
    acc.t.kl = q.t.kl;
  } else {
    acc.t.l2 = fmaxf(acc.t.l2, fmaxf(q.t.l1, q.t.l2));
  }
}

// The same merge for two lanes of a butterfly: symmetric, so both lanes of
// a pair get the same result (ties between two largest values keep the
// smaller position; a tie also makes the second largest equal the largest,
// so the position is then never used alone).
__device__ __forceinline__ void top_merge_sym(float &a1, float &a2, int32_t &ak, float b1,
                                              float b2, int32_t bk) {
  const float hi = fmaxf(a1, b1), lo = fminf(a1, b1);
  const int32_t k = a1 > b1 ? ak : (b1 > a1 ? bk : min(ak, bk));
  a2 = fmaxf(lo, fmaxf(a2, b2));
  a1 = hi;
  ak = k;
}

// Adds the pieces [q0, q1) of split_cidx in order into acc, one piece per
// step, loads of four pieces in flight (lane-strided when stride = 32).
__device__ __forceinline__ void add_pieces(Partial &acc, const DevMatrix &M, const DevState &S,
                                           int32_t q0, int32_t q1, int32_t stride) {
  int32_t q = q0;
  for (; q + 3 * stride < q1; q += 4 * stride) {
    Partial p[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) p[u] = S.part[M.split_cidx[q + u * stride]];
#pragma unroll
    for (int u = 0; u < 4; ++u) piece_add(acc, p[u]);
  }
  for (; q < q1; q += stride) piece_add(acc, S.part[M.split_cidx[q]]);
}

__global__ void __launch_bounds__(256) k_mp_fix(DevMatrix M, DevState S) {
  if (S.ctrl->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((w & ~(int64_t)31) >= M.nsplit_rows) return;  // warp-uniform
  const bool mine = w < M.nsplit_rows;
  const int32_t cb = mine ? M.split_cbeg[w] : 0, ce = mine ? M.split_cbeg[w + 1] : 0;
  const bool lone = mine && ce - cb <= kMpFixShort;
  if (lone) {  // most split rows: two or three pieces, one lane
    Partial acc;
    part_clear(acc);
    add_pieces(acc, M, S, cb, ce, 1);
    S.rowact[M.split_row[w]] = acc;
  }
  // rows of many pieces (long rows over many segments): the whole warp,
  // lanes strided over the pieces, then a fixed butterfly (reproducible,
  // and the same in every lane)
  unsigned todo = __ballot_sync(kFull, mine && !lone);
  while (todo) {
    const int src = __ffs(todo) - 1;
    todo &= todo - 1u;
    const int32_t b = __shfl_sync(kFull, cb, src), e = __shfl_sync(kFull, ce, src);
    const int64_t ws = __shfl_sync(kFull, w, src);
    Partial acc;
    part_clear(acc);
    add_pieces(acc, M, S, b + lane, e, kSliceW);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc.minfin += __shfl_xor_sync(kFull, acc.minfin, off);
      acc.maxfin += __shfl_xor_sync(kFull, acc.maxfin, off);
      // position of an infinite contribution: the larger of the two when
      // both lanes hold one (symmetric); unique when the row has exactly one
      const int32_t cn = __shfl_xor_sync(kFull, acc.mininf, off);
      const int32_t kn = __shfl_xor_sync(kFull, acc.t.kinf_min, off);
      const int32_t cx = __shfl_xor_sync(kFull, acc.maxinf, off);
      const int32_t kx = __shfl_xor_sync(kFull, acc.t.kinf_max, off);
      if (cn > 0 && (acc.mininf == 0 || kn > acc.t.kinf_min)) acc.t.kinf_min = kn;
      if (cx > 0 && (acc.maxinf == 0 || kx > acc.t.kinf_max)) acc.t.kinf_max = kx;
      acc.mininf += cn;
      acc.maxinf += cx;
      const float r1 = __shfl_xor_sync(kFull, acc.t.r1, off), r2 = __shfl_xor_sync(kFull, acc.t.r2, off);
      const int32_t kr = __shfl_xor_sync(kFull, acc.t.kr, off);
      const float l1 = __shfl_xor_sync(kFull, acc.t.l1, off), l2 = __shfl_xor_sync(kFull, acc.t.l2, off);
      const int32_t kl = __shfl_xor_sync(kFull, acc.t.kl, off);
      top_merge_sym(acc.t.r1, acc.t.r2, acc.t.kr, r1, r2, kr);
      top_merge_sym(acc.t.l1, acc.t.l2, acc.t.kl, l1, l2, kl);
    }
    if (lane == 0) S.rowact[M.split_row[ws]] = acc;
  }
}

// Step 2 and the screen of one row per lane; queues the survivors.
__global__ void __launch_bounds__(256) k_mp_rows(DevMatrix M, DevState S) {
  const Ctrl *ctrl = S.ctrl;
  if (ctrl->err) return;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((p & ~(int64_t)31) >= M.m) return;  // warp-uniform
  RowView rv;
  rv.minfin = rv.maxfin = rv.lhs = rv.rhs = 0.0;
  rv.mininf = rv.maxinf = 0;
  rv.thr_r = rv.thr_l = f_inf();
  rv.exact = 0;
  rv.act = 0;
  Top2 t = top2_init();
  int32_t len = 0;
  int64_t elem0 = 0;
  if (p < M.m) {
    const Partial a = S.rowact[p];
    const double2 sd = S.side[p];
    const int32_t lenf = M.chunk_len[p];
    len = lenf & kLenMask;
    rv.minfin = a.minfin;
    rv.maxfin = a.maxfin;
    rv.mininf = a.mininf;
    rv.maxinf = a.maxinf;
    rv.lhs = sd.x;
    rv.rhs = sd.y;
    rv.exact = (lenf & kExactFlag) ? 1 : 0;
    t = a.t;
    if (rv.exact) t.r1 = t.r2 = t.l1 = t.l2 = f_inf();
    row_sides(rv, t.r1, t.l1, ctrl->eps_feas, &S.ctrl->infeasible);
    elem0 = M.mp_ptr[p];
  }
  // a long row's full re-read is left to k_mp_long (its verdict goes to
  // rowtot, and its sums to rowsum for the queue entries)
  const int32_t lidx = p < M.m ? M.chunk_sidx[p] : -1;
  const bool full = warp_enqueue<1>(rv, t, rv.mininf, rv.maxinf, lidx >= 0 ? 0 : len, p, elem0,
                                    M, M.col, S);
  if (lidx >= 0) {
    RowTot rt;
    rt.minfin = rv.minfin;
    rt.maxfin = rv.maxfin;
    rt.mininf = rv.mininf;
    rt.maxinf = rv.maxinf;
    rt.thr_r = rv.thr_r;
    rt.thr_l = rv.thr_l;
    rt.active = full ? 1 : 0;
    rt.row = (int32_t)p;
    S.rowtot[lidx] = rt;
    if (full) {
      RowSum rs;
      rs.minfin = rv.minfin;
      rs.maxfin = rv.maxfin;
      rs.mininf = rv.mininf;
      rs.maxinf = rv.maxinf;
      S.rowsum[p] = rs;
    }
  }
}

// The screen of one piece of a long row that needs its full re-read
// (warp-level, coalesced): queues each nonzero with a surviving side.
__global__ void __launch_bounds__(256) k_mp_long(DevMatrix M, DevState S) {
  if (S.ctrl->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= M.mp_npiece) return;  // warp-uniform
  const int4 pc = M.mp_piece[w];
  const RowTot rt = S.rowtot[pc.y];
  if (!rt.active) return;  // warp-uniform
  const double2 sd = S.side[pc.x];
  RowView rv;
  rv.minfin = rt.minfin;
  rv.maxfin = rt.maxfin;
  rv.mininf = rt.mininf;
  rv.maxinf = rt.maxinf;
  rv.thr_r = rt.thr_r;
  rv.thr_l = rt.thr_l;
  rv.lhs = sd.x;
  rv.rhs = sd.y;
  rv.exact = (M.chunk_len[pc.x] & kExactFlag) ? 1 : 0;
  rv.act = 1;
  for (int32_t k0 = 0; k0 < pc.w; k0 += kSliceW) {
    const int32_t k = k0 + lane;
    unsigned sides = 0u;
    if (k < pc.w) {
      const int64_t off = (int64_t)pc.z + k;
      double L, U;
      float WU, WL;
      uint32_t fl;
      const double a = ld_coef(M, off);
      ld_rec(S.rec + M.col[off], L, U, WU, WL, fl);
      sides = nnz_sides(a, L, U, WU, WL, rv);
    }
    warp_push(sides != 0u, (int64_t)pc.z + k, pc.x, sides, S);
  }
}

template <int kWarps>
cudaError_t launch_act(const DevMatrix &M, const DevState &S, cudaStream_t st) {
  const int64_t threads = kWarps * 32;
  const int nb = (int)((M.mp_nseg + threads - 1) / threads);
  if (nb > 0) k_mp_act<kWarps><<<nb, kWarps * 32, 0, st>>>(M, S);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_merge_prologue(const DevMatrix &M, const DevState &S, cudaStream_t st) {
  const int nb = (int)(((int64_t)M.mp_nseg + 255) / 256);
  if (nb > 0) k_mp_need<<<nb, 256, 0, st>>>(M, S);
  return cudaGetLastError();
}

cudaError_t launch_merge_front(const DevMatrix &M, const DevState &S, int num_sms,
                               cudaStream_t st, cudaEvent_t *ev) {
  (void)num_sms;
  cudaError_t e;
  if (ev) cudaEventRecord(ev[0], st);
  e = M.round_warps == 4 ? launch_act<4>(M, S, st) : launch_act<8>(M, S, st);
  if (ev) cudaEventRecord(ev[1], st);
  if (e != cudaSuccess) return e;
  if (M.nsplit_rows > 0) {
    if (ev) cudaEventRecord(ev[2], st);
    k_mp_fix<<<(M.nsplit_rows + 255) / 256, 256, 0, st>>>(M, S);
    if (ev) cudaEventRecord(ev[3], st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (M.m > 0) {
    if (ev) cudaEventRecord(ev[4], st);
    k_mp_rows<<<(M.m + 255) / 256, 256, 0, st>>>(M, S);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (M.mp_npiece > 0) {
      k_mp_long<<<(int)(((int64_t)M.mp_npiece * 32 + 255) / 256), 256, 0, st>>>(M, S);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[5], st);
  }
  return cudaSuccess;
}

}  // namespace dp
