// Round helpers shared by the sliced-ELL kernels (dp_kernels.cu) and the
// merge-path kernels (dp_merge.cu): the per-side top-2 of the binary32
// screen values and the queueing of the nonzeros that survive the screen.
#pragma once
#include "dp_device.cuh"

namespace dp {

__device__ __forceinline__ void top2_add(float t, int k, float &t1, float &t2, int32_t &k1) {
  if (t > t1) {
    t2 = t1;
    t1 = t;
    k1 = k;
  } else if (t > t2) {
    t2 = t;
  }
}

__device__ __forceinline__ Top2 top2_init() {
  Top2 t;
  t.r1 = t.r2 = t.l1 = t.l2 = -f_inf();
  t.kr = t.kl = 0;
  t.kinf_min = t.kinf_max = 0;
  return t;
}

// Reserves c (0..7) consecutive queue entries per lane with one atomic per
// warp (all 32 lanes call): the lanes' offsets come from three ballots of
// the bits of c, not from a shuffle scan.  Returns the lane's first entry
// (meaningless when c = 0).
__device__ __forceinline__ int warp_reserve(int c, int32_t *counter) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const unsigned b0 = __ballot_sync(kFull, c & 1), b1 = __ballot_sync(kFull, c & 2),
                 b2 = __ballot_sync(kFull, c & 4);
  const int total = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
  if (total == 0) return 0;
  int base = 0;
  if (lane == 0) base = atomicAdd(counter, total);
  base = __shfl_sync(kFull, base, 0);
  return base + __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt);
}

// Queues nonzeros of the lanes' chunks whose candidates survive the screen.
// Entries go to a global queue (warp-aggregated slots) and are evaluated by
// k_cand_queue, one per thread, so the binary64 candidate formulas run
// lane-dense across the whole GPU however few survivors a warp has.  When
// the second-largest screen value of a side is below the threshold, only the
// chunk's largest can survive and it is queued directly (no re-read);
// otherwise the lane re-reads its chunk (values and columns from L2, records
// through the same gather), four slots at a time.  Element k of a lane's
// chunk sits at elem0 + k * kStride of val/col (slot-major slices: the
// lane's slot in the slice, stride 32; CSR rows: the row's offset, stride
// 1).  All 32 lanes must call this (warp collectives).  Returns whether the
// lane's chunk needed the full re-read (done here for its first mylen
// slots).  kCo: records are loaded through L2 (the persistent loop, which
// rewrites them between its phases).
template <int kStride, bool kCo = false>
__device__ __forceinline__ bool warp_enqueue(const RowView &mine, const Top2 &t, int chunk_mininf,
                                             int chunk_maxinf, int32_t mylen, int64_t chunk_slot,
                                             int64_t elem0, const DevMatrix &M,
                                             const int32_t *col, const DevState &S) {
  const bool act = mine.act != 0;
  if (__ballot_sync(kFull, act) == 0u) return false;

  bool wrote_sums = false;
  auto sums = [&]() {  // the row's sums, once, before its first queued entry
    if (wrote_sums) return;
    RowSum rs;
    rs.minfin = mine.minfin;
    rs.maxfin = mine.maxfin;
    rs.mininf = mine.mininf;
    rs.maxinf = mine.maxinf;
    S.rowsum[chunk_slot] = rs;
    wrote_sums = true;
  };
  auto entry = [&](int k, unsigned sides) {
    CandEntry e;
    e.off = (uint32_t)(elem0 + (int64_t)k * kStride);
    e.cs = ((uint32_t)chunk_slot << 2) | sides;
    return e;
  };

  // Survivors can be named without re-reading the chunk unless a side has
  // two screen values above its threshold (or the row skips the screen).
  // With exactly one infinite contribution to a side's activity, only that
  // nonzero gets a finite residual on that side (Sec. 3.4); its slot was
  // recorded by the activity pass.
  const bool full = act && (mine.exact || (mine.mininf == 0 && t.r2 > mine.thr_r) ||
                            (mine.maxinf == 0 && t.l2 > mine.thr_l));
  bool h1 = false, h2 = false;
  int k1 = 0, k2 = 0;
  if (act && !full) {
    const bool fr = d_isfinite(mine.rhs), fl = d_isfinite(mine.lhs);
    if (fr && mine.mininf == 0 && t.r1 > mine.thr_r) { h1 = true; k1 = t.kr; }
    if (fr && mine.mininf == 1 && chunk_mininf > 0) { h1 = true; k1 = t.kinf_min; }
    if (fl && mine.maxinf == 0 && t.l1 > mine.thr_l) { h2 = true; k2 = t.kl; }
    if (fl && mine.maxinf == 1 && chunk_maxinf > 0) { h2 = true; k2 = t.kinf_max; }
  }
  const bool merge = h1 && h2 && k1 == k2;
  {
    const bool q2 = h2 && !merge;
    int pos = warp_reserve((h1 ? 1 : 0) + (q2 ? 1 : 0), &S.ctrl->qcount);
    if (h1 || q2) sums();
    if (h1) S.queue[pos++] = entry(k1, merge ? 3u : 1u);
    if (q2) S.queue[pos] = entry(k2, 2u);
  }

  // full re-read of the chunk, four slots at a time
  const int len = full ? mylen : 0;
  int maxlen = len;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) maxlen = max(maxlen, __shfl_xor_sync(kFull, maxlen, o));
  const int64_t vo = elem0;
  const int32_t *cp = col + elem0;
  // software-pipelined: the next group's values and columns are fetched
  // while this group's records are gathered
  double an[4];
  int32_t jn[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      an[u] = 1.0;
      jn[u] = 0;
      if (k0 + u < len) {
        an[u] = ld_coef(M, vo + (int64_t)(k0 + u) * kStride);
        jn[u] = cp[(int64_t)(k0 + u) * kStride];
      }
    }
  };
  if (maxlen > 0) fetch(0);
  for (int k = 0; k < maxlen; k += 4) {
    double a[4], L[4], U[4];
    float WU[4], WL[4];
    uint32_t fl[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = an[u];
      L[u] = U[u] = 0.0;
      WU[u] = WL[u] = 0.0f;
      if (k + u < len) ld_rec_t<kCo>(S.rec + jn[u], L[u], U[u], WU[u], WL[u], fl[u]);
    }
    if (k + 4 < maxlen) fetch(k + 4);
    unsigned sd[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      sd[u] = k + u < len ? nnz_sides(a[u], L[u], U[u], WU[u], WL[u], mine) : 0u;
    // one reservation for the group's survivors of all lanes
    int c = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) c += sd[u] != 0u;
    int pos = warp_reserve(c, &S.ctrl->qcount);
    if (c > 0) sums();
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (sd[u] != 0u) S.queue[pos++] = entry(k + u, sd[u]);
  }
  return full;
}

// Appends one queue entry per lane with h set (warp-aggregated; all 32
// lanes call): element offset `off` of a row whose sums are at rowsum[slot].
__device__ __forceinline__ void warp_push(bool h, int64_t off, int64_t slot, unsigned sides,
                                          const DevState &S) {
  const unsigned pm = __ballot_sync(kFull, h);
  if (pm == 0u) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(pm) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(&S.ctrl->qcount, __popc(pm));
  base = __shfl_sync(kFull, base, leader);
  if (!h) return;
  CandEntry e;
  e.off = (uint32_t)off;
  e.cs = ((uint32_t)slot << 2) | sides;
  S.queue[base + __popc(pm & ((1u << lane) - 1u))] = e;
}

}  // namespace dp
