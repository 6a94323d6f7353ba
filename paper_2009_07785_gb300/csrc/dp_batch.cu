// Batched propagation of branch-and-bound nodes: many bound vectors over
// one matrix in one graph-driven round loop (or, k_bpersistent, in one
// persistent cooperative kernel running the same phases).  The paper propagates one
// problem per call and notes (Sec. 5) that after branching a solver
// propagates from an already propagated state with a few bound changes;
// a throughput device is fed by running many such nodes at once.
//
// Every node follows exactly the round-synchronous algorithm of the single
// instance path (Alg. 2 with Jacobi rounds): the same activities (Def. 1,
// Eq. 2a/2b, with the infinity counts of Sec. 3.4), the same candidates
// (Eq. 3a/3b in the residual form of Eq. 5a/5b), the same integer rounding
// and acceptance threshold, and its own termination and round count.
//
// Layout.  Bounds are node-minor (entry e = j*Bp + node).  The 32 lanes of
// a warp are the 32 nodes of one node group; a warp walks one chunk of the
// sliced-ELL matrix with warp-uniform loads of its values and columns and
// one coalesced 512-byte load of the 32 nodes' bounds per nonzero.  The
// side pattern of a row is warp-uniform, so a row with one infinite side
// computes only the activity its finite side needs.
//
// Marking (the constraint marking of Alg. 1, Sec. 2.1).  In round r > 1 a
// row is processed for a node only if a bound of one of its variables
// changed for that node in round r-1.  Skipping the other rows is exact:
// their activities, hence their candidates, are those of round r-1, which
// were then applied or rejected against bounds that have not moved since.
//
// Round kernels (graph body):
//   k_bmark        thread per chunk (warp per split-row chunk): the nodes
//                  that must process it (OR of the change masks of its
//                  variables); work lists per group
//   k_bmark_split  block per split row: all chunks of a split row get the
//                  row's mask
//   k_bact         warp per work item: activities; for whole rows also
//                  Step 2, the binary32 screen and the candidates with
//                  filtered 64-bit atomics
//   k_bcombine     block per (split row, group): sums chunk partials in a
//                  fixed order, Step 2 and screen thresholds
//   k_bcand_split  warp per (split chunk, group): candidates of split rows
//   k_bfinish      warp per 32 change-mask words, lane per node: commit,
//                  crossing test; the last block ends nodes and sets the
//                  condition
#include <cuda_runtime.h>
#include <cstdint>
#include <cfloat>

#include "dp_device.cuh"
#include "dp_internal.h"
#include "dp_launch.h"
#include "../../include/domprop.h"

namespace dp {

namespace {

constexpr int kThreads = 256;
constexpr int kActWarps = 8;

struct BParams {
  int32_t Bp, G, Gs, round, max_rounds, err;
  double eps_int, tau_rel, eps_feas, inf_thr;
  float tau_dn, eps_dn;
};

__device__ __forceinline__ BParams load_params(const BCtrl *c) {
  BParams P;
  P.Bp = c->Bp;
  P.G = c->G;
  P.Gs = (c->G + 3) & ~3;
  P.round = c->round;
  P.max_rounds = c->max_rounds;
  P.err = c->err;
  P.eps_int = c->eps_int;
  P.tau_rel = c->tau_rel;
  P.eps_feas = c->eps_feas;
  P.inf_thr = c->inf_thr;
  P.tau_dn = f32_dn(c->tau_rel);
  P.eps_dn = f32_dn(c->eps_int);
  return P;
}

// Bounds {L, U} of one (variable, node) entry and their screen widths.
// A round kernel of the graph never sees them change (read-only path); the
// persistent loop (kCo) rewrites them between its phases, so it loads them
// through L2, which is coherent across the grid.
template <bool kCo>
__device__ __forceinline__ double2 ld_bounds(const double2 *p) {
  if (kCo) return __ldcg(p);
  double2 v;
  asm("ld.global.nc.v2.f64 {%0,%1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}
template <bool kCo>
__device__ __forceinline__ float2 ld_widths(const float2 *p) {
  if (kCo) return __ldcg(p);
  float2 v;
  asm("ld.global.nc.v2.f32 {%0,%1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
// Bounds and widths of one entry, as every kernel that changes them writes
// them (the widths are those of the binary32 screen, see screen_widths).
__device__ __forceinline__ void put_entry(const BatchState &S, int64_t e, double L, double U,
                                          bool isint, float tau_dn, float eps_dn) {
  float WU, WL;
  screen_widths(L, U, isint, tau_dn, eps_dn, WU, WL);
  S.cur[e] = make_double2(L, U);
  S.wid[e] = make_float2(WU, WL);
}

__device__ __forceinline__ uint4 or4(uint4 a, uint4 b) {
  return make_uint4(a.x | b.x, a.y | b.y, a.z | b.z, a.w | b.w);
}
__device__ __forceinline__ uint32_t word4(const uint4 &v, int u) {
  return u == 0 ? v.x : (u == 1 ? v.y : (u == 2 ? v.z : v.w));
}

// Appends `e` for every lane with h set (warp-aggregated); all 32 lanes call.
template <typename T>
__device__ __forceinline__ void warp_append(bool h, T e, T *list, int32_t *count) {
  const unsigned m = __ballot_sync(kFull, h);
  if (m == 0u) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(kFull, base, leader);
  if (h) list[base + __popc(m & ((1u << lane) - 1u))] = e;
}

// Sets, in bits[g], the bits of the lanes (nodes g*32 + lane) with h set.
// The word only gains bits, so reading it first (possibly stale) saves the
// atomic in the common case that the bits are already there.  All 32 lanes
// call.
__device__ __forceinline__ void note_nodes(uint32_t *bits, int g, bool h) {
  const unsigned m = __ballot_sync(kFull, h);
  if (m == 0u) return;
  if ((threadIdx.x & 31) == 0 && (bits[g] & m) != m) atomicOr(&bits[g], m);
}

// Activity of one chunk for this lane's node (Def. 1 / Eq. 2a, 2b; an
// infinite contribution is counted, not summed, Sec. 3.4), plus the
// largest binary32 screen value of each needed side.  The sums are one
// FMA chain per side in the chunk's CSR order.
struct BAct {
  double minfin, maxfin;
  int32_t mininf, maxinf;
  float tr, tl;
};

__device__ __forceinline__ void act_add(double a, double2 b, float2 w, bool need_min,
                                        bool need_max, bool screen, BAct &r) {
  const bool pos = d_pos(a);
  const double bmin = pos ? b.x : b.y;
  const double bmax = pos ? b.y : b.x;
  if (need_min) {
    const bool i = d_isinf(bmin);
    r.mininf += i ? 1 : 0;
    r.minfin = fma(a, i ? 0.0 : bmin, r.minfin);
  }
  if (need_max) {
    const bool i = d_isinf(bmax);
    r.maxinf += i ? 1 : 0;
    r.maxfin = fma(a, i ? 0.0 : bmax, r.maxfin);
  }
  if (screen) {
    const float au = absup_fast(a), ad = absdn_fast(a);
    if (need_min) r.tr = fmaxf(r.tr, screen_prod(au, ad, pos ? w.x : w.y));
    if (need_max) r.tl = fmaxf(r.tl, screen_prod(au, ad, pos ? w.y : w.x));
  }
}

template <bool kCo>
__device__ __forceinline__ BAct chunk_activity(const DevMatrix &M, const BatchState &S,
                                               int64_t base, int len, int node, bool need_min,
                                               bool need_max, bool screen, const BParams &P) {
  BAct r;
  r.minfin = r.maxfin = 0.0;
  r.mininf = r.maxinf = 0;
  r.tr = r.tl = -f_inf();
  const double *vp = M.val + base;
  const int32_t *cp = M.col + base;
  const double2 *bp = S.cur + node;
  const float2 *wp = S.wid + node;
  int k = 0;
  // software-pipelined: the next group's columns are fetched while this
  // group's bounds are gathered; its values load beside the gathers
  int32_t jn[4];
  if (len >= 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) jn[u] = __ldg(cp + (int64_t)u * kSliceW);
  }
  for (; k + 4 <= len; k += 4) {
    int32_t j[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) j[u] = jn[u];
    if (k + 8 <= len) {
#pragma unroll
      for (int u = 0; u < 4; ++u) jn[u] = __ldg(cp + (int64_t)(k + 4 + u) * kSliceW);
    }
    double2 b[4];
    float2 w[4];
    double a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      b[u] = ld_bounds<kCo>(bp + (int64_t)j[u] * P.Bp);
      w[u] = screen ? ld_widths<kCo>(wp + (int64_t)j[u] * P.Bp) : make_float2(0.0f, 0.0f);
      a[u] = __ldg(vp + (int64_t)(k + u) * kSliceW);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) act_add(a[u], b[u], w[u], need_min, need_max, screen, r);
  }
  for (; k < len; ++k) {
    const double a = __ldg(vp + (int64_t)k * kSliceW);
    const int32_t j = __ldg(cp + (int64_t)k * kSliceW);
    const double2 b = ld_bounds<kCo>(bp + (int64_t)j * P.Bp);
    const float2 w = screen ? ld_widths<kCo>(wp + (int64_t)j * P.Bp) : make_float2(0.0f, 0.0f);
    act_add(a, b, w, need_min, need_max, screen, r);
  }
  if (!screen) r.tr = r.tl = f_inf();
  return r;
}

// Candidates of one nonzero for one node from the sides that survived the
// screen (side_candidate), applied with order-preserving 64-bit atomics to
// the node's next state kp = {lower key, upper key}; nothing waits for the
// atomics.  Returns whether a candidate was applied (it improves the
// round's starting bound, so the entry changes this round).
__device__ __forceinline__ bool bnnz_candidates(double a, bool isint, double L, double U,
                                                unsigned sides, const RowView &rv,
                                                const BParams &P, long long *kp) {
  bool applied = false;
  auto apply = [&](const SideCand &c) {
    if (!c.apply) return;
    const long long nk = key_of(c.v);
    if (c.upper) atomicMin(&kp[1], nk);
    else atomicMax(&kp[0], nk);
    applied = true;
  };
  apply(side_candidate(a, L, U, isint, (sides & 1u) != 0u, rv, P.eps_int, P.tau_rel,
                       P.inf_thr));
  if (sides == 3u)
    apply(side_candidate(a, L, U, isint, false, rv, P.eps_int, P.tau_rel, P.inf_thr));
  return applied;
}

// Nonzero-node pairs that survived the screen wait in a per-warp buffer and
// are evaluated 32 at a time, one pair per lane, so that the binary64
// candidate formulas (two divisions) run lane-dense whatever the pattern of
// survivors across the 32 nodes of a warp.  Each entry carries its own
// context, so a batch may mix pairs of several rows.
constexpr int kPairCap = 64;

struct PairBuf {
  uint32_t off[kPairCap];   // element offset of the nonzero in val/col
  uint32_t info[kPairCap];  // node << 4 | maxinf==0 << 3 | mininf==0 << 2 | sides
  int32_t row[kPairCap];
  double minfin[kPairCap], maxfin[kPairCap];
};

struct PairQueue {
  PairBuf *buf;  // this warp's shared-memory buffer
  int n;         // buffered pairs (warp-uniform)
};

// Evaluates pairs [from, from + count) of the buffer, count <= 32, and
// marks the entries they change in the round's change mask chg_next (one
// atomic per mask word among the lanes).  All 32 lanes call.
template <bool kCo>
__device__ __forceinline__ void eval_pairs(PairQueue &pq, int from, int count,
                                           const DevMatrix &M, const BatchState &S,
                                           const BParams &P, uint32_t *chg_next) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  unsigned long long widx = ~0ull;
  uint32_t bit = 0u;
  if (lane < count) {
    const int q = from + lane;
    const PairBuf &B = *pq.buf;
    const uint32_t off = B.off[q], info = B.info[q];
    const int32_t row = B.row[q];
    const uint32_t node = info >> 4;
    RowView rv;
    rv.minfin = B.minfin[q];
    rv.maxfin = B.maxfin[q];
    rv.mininf = (info & 4u) ? 0 : 1;
    rv.maxinf = (info & 8u) ? 0 : 1;
    rv.lhs = S.lhs[row];
    rv.rhs = S.rhs[row];
    const double a = __ldg(M.val + off);
    const int32_t j = __ldg(M.col + off);
    const int64_t e = (int64_t)j * P.Bp + node;
    const double2 b = ld_bounds<kCo>(S.cur + e);
    const bool isint = __ldg(S.vt + j) != 0;
    if (bnnz_candidates(a, isint, b.x, b.y, info & 3u, rv, P, S.nkey + 2 * e)) {
      widx = (unsigned long long)j * P.Gs + (node >> 5);
      bit = 1u << (node & 31);
    }
  }
  const unsigned peers = __match_any_sync(kFull, widx);
  const uint32_t bits = __reduce_or_sync(peers, bit);
  if (bit != 0u && lane == __ffs(peers) - 1) atomicOr(&chg_next[widx], bits);
  __syncwarp();
}

// Candidates of one chunk for this lane's node; `on` = the node processes
// the chunk and its row may yield an accepted candidate.  The screen is
// recomputed from the bounds (binary32 and integer work, which overlaps
// with the loads), so binary64 candidate work runs only for nonzeros that
// can tighten.  Four nonzeros are screened per step, their loads in flight
// together; the survivors then enter the pair buffer in CSR order.  All 32
// lanes call.
template <bool kCo>
__device__ __forceinline__ void chunk_candidates(const DevMatrix &M, const BatchState &S,
                                                 int64_t base, int len, int node, bool on,
                                                 int32_t row, const RowView &rv,
                                                 const BParams &P, PairQueue &pq,
                                                 uint32_t *chg_next) {
  const int lane = threadIdx.x & 31;
  const double *vp = M.val + base;
  const int32_t *cp = M.col + base;
  const uint32_t ctx = ((uint32_t)node << 4) | (rv.maxinf == 0 ? 8u : 0u) |
                       (rv.mininf == 0 ? 4u : 0u);
  const double2 *bp = S.cur + node;
  const float2 *wp = S.wid + node;
  for (int k0 = 0; k0 < len; k0 += 4) {
    const int nk = min(4, len - k0);
    // bits 2u, 2u+1: the surviving sides of nonzero k0 + u
    unsigned sides4 = 0u;
    if (on) {
      double a[4];
      int32_t j[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = k0 + (u < nk ? u : 0);
        a[u] = __ldg(vp + (int64_t)k * kSliceW);
        j[u] = __ldg(cp + (int64_t)k * kSliceW);
      }
      double2 b[4];
      float2 w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        b[u] = ld_bounds<kCo>(bp + (int64_t)j[u] * P.Bp);
        w[u] = ld_widths<kCo>(wp + (int64_t)j[u] * P.Bp);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (u < nk) sides4 |= nnz_sides(a[u], b[u].x, b[u].y, w[u].x, w[u].y, rv) << (2 * u);
    }
    if (__ballot_sync(kFull, sides4 != 0u) == 0u) continue;
#pragma unroll 1
    for (int u = 0; u < nk; ++u) {
      const unsigned sides = (sides4 >> (2 * u)) & 3u;
      const unsigned m = __ballot_sync(kFull, sides != 0u);
      if (m == 0u) continue;
      if (sides) {
        const int q = pq.n + __popc(m & ((1u << lane) - 1u));
        PairBuf &B = *pq.buf;
        B.off[q] = (uint32_t)(base + (int64_t)(k0 + u) * kSliceW);
        B.info[q] = ctx | sides;
        B.row[q] = row;
        B.minfin[q] = rv.minfin;
        B.maxfin[q] = rv.maxfin;
      }
      pq.n += __popc(m);
      if (pq.n >= 32) {
        pq.n -= 32;
        eval_pairs<kCo>(pq, pq.n, 32, M, S, P, chg_next);
      }
    }
  }
}

// Evaluates what is left in the pair buffer (end of a warp's work).
template <bool kCo>
__device__ __forceinline__ void drain_pairs(PairQueue &pq, const DevMatrix &M,
                                            const BatchState &S, const BParams &P,
                                            uint32_t *chg_next) {
  if (pq.n > 0) eval_pairs<kCo>(pq, 0, pq.n, M, S, P, chg_next);
  pq.n = 0;
}

// ------------------------------------------------------------- k_bmark --

// The nodes of one node-group quad [gq, gq + 4) that must process a chunk
// (the OR of its variables' change masks, every node in its first round),
// restricted to live nodes.  `len` nonzeros from `base`, lane-strided by
// `step` from `k0` (a thread walks all of them with k0 = 0, step = 1).
__device__ __forceinline__ uint4 chunk_mask(const DevMatrix &M, const BatchState &S,
                                            const BParams &P, const uint32_t *chg, int64_t base,
                                            int len, int k0, int step, int gq) {
  uint4 m = make_uint4(0u, 0u, 0u, 0u);
  int k = k0;
  // four elements' loads in flight at a time
  for (; k + 3 * step < len; k += 4 * step) {
    int32_t j[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) j[u] = M.col[base + (int64_t)(k + u * step) * kSliceW];
    uint4 w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      w[u] = *reinterpret_cast<const uint4 *>(chg + (int64_t)j[u] * P.Gs + gq);
#pragma unroll
    for (int u = 0; u < 4; ++u) m = or4(m, w[u]);
  }
  for (; k < len; k += step) {
    const int32_t j = M.col[base + (int64_t)k * kSliceW];
    m = or4(m, *reinterpret_cast<const uint4 *>(chg + (int64_t)j * P.Gs + gq));
  }
  return m;
}

__device__ __forceinline__ uint4 live_mask(const BatchState &S, uint4 m, int gq) {
  const uint4 al = *reinterpret_cast<const uint4 *>(S.alive + gq);
  const uint4 fr = *reinterpret_cast<const uint4 *>(S.fresh + gq);
  m = or4(m, fr);
  return make_uint4(m.x & al.x, m.y & al.y, m.z & al.z, m.w & al.w);
}

__device__ __forceinline__ void bmark_body(const DevMatrix &M, const BatchState &S) {
  BCtrl *ctrl = S.ctrl;
  const BParams P = load_params(ctrl);
  if (P.err) return;
  const int p = P.round & 1;
  const bool first = P.round == 0;  // every live node is fresh
  const uint32_t *chg = S.chg[p];
  const int64_t nslots = S.nslots;
  const int64_t split_slots = (int64_t)M.nslices_split * kSliceW;
  const int lane = threadIdx.x & 31;
  // chunks of split rows (long): a warp per chunk, lanes strided over its
  // nonzeros; k_bmark_split makes them work items
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t cs = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
       cs < split_slots; cs += nwarps) {
    const int32_t row = M.chunk_row[cs];
    if (row < 0) continue;  // warp-uniform
    const int len = M.chunk_len[cs] & kLenMask;
    const int64_t base = M.slice_off[cs / kSliceW] + (cs % kSliceW);
    const bool used = d_isfinite(S.lhs[row]) || d_isfinite(S.rhs[row]);
    for (int gq = 0; gq < P.Gs; gq += 4) {
      uint4 m = make_uint4(0u, 0u, 0u, 0u);
      if (used) {
        if (first) {
          m = make_uint4(kFull, kFull, kFull, kFull);
        } else {
          m = chunk_mask(M, S, P, chg, base, len, lane, 32, gq);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            m.x |= __shfl_xor_sync(kFull, m.x, o);
            m.y |= __shfl_xor_sync(kFull, m.y, o);
            m.z |= __shfl_xor_sync(kFull, m.z, o);
            m.w |= __shfl_xor_sync(kFull, m.w, o);
          }
        }
        m = live_mask(S, m, gq);
      }
      if (lane == 0) *reinterpret_cast<uint4 *>(S.cmask + cs * P.Gs + gq) = m;
    }
  }
  // whole rows: a thread per chunk (block-uniform loop: warp_append needs
  // every lane)
  for (int64_t c0 = split_slots + (int64_t)blockIdx.x * blockDim.x; c0 < nslots;
       c0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cs = c0 + threadIdx.x;
    int32_t row = -1, len = 0;
    int64_t base = 0;
    bool used = false;  // a free row (both sides infinite) has no candidates
                        // and cannot be infeasible: it is never processed
    if (cs < nslots) {
      row = M.chunk_row[cs];
      if (row >= 0) {
        len = M.chunk_len[cs] & kLenMask;
        base = M.slice_off[cs / kSliceW] + (cs % kSliceW);
        used = d_isfinite(S.lhs[row]) || d_isfinite(S.rhs[row]);
      }
    }
    for (int gq = 0; gq < P.Gs; gq += 4) {
      uint4 m = make_uint4(0u, 0u, 0u, 0u);
      if (row >= 0) {
        if (used) {
          m = first ? make_uint4(kFull, kFull, kFull, kFull)
                    : chunk_mask(M, S, P, chg, base, len, 0, 1, gq);
          m = live_mask(S, m, gq);
        }
        *reinterpret_cast<uint4 *>(S.cmask + cs * P.Gs + gq) = m;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int g = gq + u;
        if (g < P.G)  // uniform
          warp_append<int32_t>(used && word4(m, u) != 0u, (int32_t)cs,
                               S.items + (int64_t)g * nslots, &ctrl->icount[g]);
      }
    }
  }
}

// All chunks of a split row get the OR of their masks (the row's activity
// needs every chunk), and become work items.  Block per split row.
__device__ __forceinline__ void bmark_split_body(const DevMatrix &M, const BatchState &S) {
  BCtrl *ctrl = S.ctrl;
  const BParams P = load_params(ctrl);
  if (P.err) return;
  constexpr int kW = kThreads / 32;
  __shared__ uint4 s_m[kW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nslots = S.nslots;
  // block per split row (block-uniform loop): the block's threads stride
  // over the row's chunks, a row of hundreds of chunks would otherwise be
  // one warp's serial chain
  for (int s = blockIdx.x; s < M.nsplit_rows; s += gridDim.x) {
    const int32_t q0 = M.split_cbeg[s], q1 = M.split_cbeg[s + 1];
    for (int gq = 0; gq < P.Gs; gq += 4) {
      uint4 m = make_uint4(0u, 0u, 0u, 0u);
      for (int32_t q = q0 + threadIdx.x; q < q1; q += kThreads)
        m = or4(m, *reinterpret_cast<const uint4 *>(S.cmask + (int64_t)M.split_cidx[q] * P.Gs + gq));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        m.x |= __shfl_xor_sync(kFull, m.x, o);
        m.y |= __shfl_xor_sync(kFull, m.y, o);
        m.z |= __shfl_xor_sync(kFull, m.z, o);
        m.w |= __shfl_xor_sync(kFull, m.w, o);
      }
      if (lane == 0) s_m[warp] = m;
      __syncthreads();
      m = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int k = 0; k < kW; ++k) m = or4(m, s_m[k]);
      __syncthreads();  // s_m is reused by the next group quad
      for (int32_t q = q0 + threadIdx.x; q < q1; q += kThreads)
        *reinterpret_cast<uint4 *>(S.cmask + (int64_t)M.split_cidx[q] * P.Gs + gq) = m;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int g = gq + u;
        if (g >= P.G || word4(m, u) == 0u) continue;  // block-uniform
        for (int32_t qb = q0 + warp * 32; qb < q1; qb += kThreads) {  // warp-uniform
          const int32_t q = qb + lane;
          warp_append<int32_t>(q < q1, q < q1 ? M.split_cidx[q] : 0,
                               S.items + (int64_t)g * nslots, &ctrl->icount[g]);
        }
      }
    }
  }
}

// -------------------------------------------------------------- k_bact --

template <bool kCo>
__device__ __forceinline__ void bact_body(const DevMatrix &M, const BatchState &S,
                                          PairBuf *s_pairs) {
  BCtrl *ctrl = S.ctrl;
  const BParams P = load_params(ctrl);
  if (P.err) return;
  const int p = P.round & 1;
  const int lane = threadIdx.x & 31;
  // regions of the work list: lane g holds the item count of group g
  const int cnt = lane < P.G ? ctrl->icount[lane] : 0;
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  const int excl = incl - cnt;
  const int64_t split_slots = (int64_t)M.nslices_split * kSliceW;
  const int nw = gridDim.x * kActWarps;
  PairQueue pq{&s_pairs[threadIdx.x >> 5], 0};
  uint32_t *chg_next = S.chg[p ^ 1];
  for (int it = blockIdx.x * kActWarps + (threadIdx.x >> 5); it < total; it += nw) {
    const int g = __popc(__ballot_sync(kFull, lane < P.G && it >= incl));
    const int off = __shfl_sync(kFull, excl, g);
    const int64_t cs = S.items[(int64_t)g * S.nslots + (it - off)];
    const int node = g * 32 + lane;
    const uint32_t mask = S.cmask[cs * P.Gs + g];
    const bool on = ((mask >> lane) & 1u) != 0u;
    const int32_t row = M.chunk_row[cs];
    const int32_t lenf = M.chunk_len[cs];
    const int len = lenf & kLenMask;
    const bool exact = (lenf & kExactFlag) != 0;
    const int64_t base = M.slice_off[cs / kSliceW] + (cs % kSliceW);
    const double lhs = S.lhs[row], rhs = S.rhs[row];
    const bool need_min = d_isfinite(rhs), need_max = d_isfinite(lhs);
    const BAct r = chunk_activity<kCo>(M, S, base, len, node, need_min, need_max, !exact, P);
    if (cs < split_slots) {
      BPartial pt;
      pt.minfin = r.minfin;
      pt.maxfin = r.maxfin;
      pt.mininf = r.mininf;
      pt.maxinf = r.maxinf;
      pt.tr = r.tr;
      pt.tl = r.tl;
      S.part[cs * P.Bp + node] = pt;
      continue;
    }
    RowView rv;
    rv.minfin = r.minfin;
    rv.maxfin = r.maxfin;
    rv.lhs = lhs;
    rv.rhs = rhs;
    rv.mininf = r.mininf;
    rv.maxinf = r.maxinf;
    rv.exact = exact ? 1 : 0;
    const bool infeas = row_sides_eval(rv, r.tr, r.tl, P.eps_feas);
    note_nodes(S.inf_bits, g, on && infeas);
    const bool go = on && rv.act != 0;
    if (!__any_sync(kFull, go)) continue;
    chunk_candidates<kCo>(M, S, base, len, node, go, row, rv, P, pq, chg_next);
  }
  drain_pairs<kCo>(pq, M, S, P, chg_next);
}

// ---------------------------------------------------------- split rows --

// Block per (split row, node group), block-uniform loop: each of the eight
// warps sums a contiguous eighth of the row's chunk partials in chunk order
// (four pieces' loads in flight at a time), and warp 0 adds the eight sums in
// warp order, a fixed association whatever the scheduling; then Step 2 and
// the screen thresholds of the row for the group's nodes.
__device__ __forceinline__ void bcombine_body(const DevMatrix &M, const BatchState &S) {
  const BParams P = load_params(S.ctrl);
  if (P.err) return;
  constexpr int kW = kThreads / 32;
  __shared__ BPartial s_sum[kW][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t pairs = (int64_t)M.nsplit_rows * P.G;
  for (int64_t w = blockIdx.x; w < pairs; w += gridDim.x) {
    const int s = (int)(w / P.G), g = (int)(w % P.G);
    const int32_t q0 = M.split_cbeg[s], q1 = M.split_cbeg[s + 1];
    const int64_t c0 = M.split_cidx[q0];
    const uint32_t mask = S.cmask[c0 * P.Gs + g];
    if (mask == 0u) {  // block-uniform
      if (threadIdx.x == 0) S.srow_act[(int64_t)s * P.Gs + g] = 0u;
      continue;
    }
    const int node = g * 32 + lane;
    BPartial acc;
    acc.minfin = acc.maxfin = 0.0;
    acc.mininf = acc.maxinf = 0;
    acc.tr = acc.tl = -f_inf();
    auto add = [&](const BPartial &pt) {
      acc.minfin += pt.minfin;
      acc.maxfin += pt.maxfin;
      acc.mininf += pt.mininf;
      acc.maxinf += pt.maxinf;
      acc.tr = fmaxf(acc.tr, pt.tr);
      acc.tl = fmaxf(acc.tl, pt.tl);
    };
    const int32_t span = (q1 - q0 + kW - 1) / kW;
    const int32_t qa = min(q1, q0 + warp * span), qb = min(q1, qa + span);
    int32_t q = qa;
    for (; q + 4 <= qb; q += 4) {
      BPartial pt[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) pt[u] = S.part[(int64_t)M.split_cidx[q + u] * P.Bp + node];
#pragma unroll
      for (int u = 0; u < 4; ++u) add(pt[u]);
    }
    for (; q < qb; ++q) add(S.part[(int64_t)M.split_cidx[q] * P.Bp + node]);
    s_sum[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
      const bool on = ((mask >> lane) & 1u) != 0u;
      const int32_t row = M.split_row[s];
      RowView rv;
      rv.minfin = rv.maxfin = 0.0;
      rv.mininf = rv.maxinf = 0;
      float tr = -f_inf(), tl = -f_inf();
#pragma unroll
      for (int k = 0; k < kW; ++k) {
        const BPartial &pt = s_sum[k][lane];
        rv.minfin += pt.minfin;
        rv.maxfin += pt.maxfin;
        rv.mininf += pt.mininf;
        rv.maxinf += pt.maxinf;
        tr = fmaxf(tr, pt.tr);
        tl = fmaxf(tl, pt.tl);
      }
      rv.lhs = S.lhs[row];
      rv.rhs = S.rhs[row];
      rv.exact = (M.chunk_len[c0] & kExactFlag) ? 1 : 0;
      const bool infeas = row_sides_eval(rv, tr, tl, P.eps_feas);
      note_nodes(S.inf_bits, g, on && infeas);
      BRowTot tt;
      tt.minfin = rv.minfin;
      tt.maxfin = rv.maxfin;
      tt.mininf = rv.mininf;
      tt.maxinf = rv.maxinf;
      tt.thr_r = rv.thr_r;
      tt.thr_l = rv.thr_l;
      S.rowtot[(int64_t)s * P.Bp + node] = tt;
      const unsigned act = __ballot_sync(kFull, on && rv.act != 0);
      if (lane == 0) S.srow_act[(int64_t)s * P.Gs + g] = act;
    }
    __syncthreads();  // s_sum is reused by the block's next pair
  }
}

template <bool kCo>
__device__ __forceinline__ void bcand_split_body(const DevMatrix &M, const BatchState &S,
                                                 PairBuf *s_pairs) {
  BCtrl *ctrl = S.ctrl;
  const BParams P = load_params(ctrl);
  if (P.err) return;
  const int p = P.round & 1;
  const int lane = threadIdx.x & 31;
  const int64_t pairs = (int64_t)M.nslices_split * kSliceW * P.G;
  const int nw = gridDim.x * (blockDim.x >> 5);
  PairQueue pq{&s_pairs[threadIdx.x >> 5], 0};
  uint32_t *chg_next = S.chg[p ^ 1];
  for (int64_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < pairs; w += nw) {
    const int64_t cs = w / P.G;
    const int g = (int)(w % P.G);
    const int32_t s = M.chunk_sidx[cs];
    if (s < 0) continue;
    const uint32_t act = S.srow_act[(int64_t)s * P.Gs + g];
    if (act == 0u) continue;
    const int node = g * 32 + lane;
    const bool on = ((act >> lane) & 1u) != 0u;
    const int32_t row = M.chunk_row[cs];
    const int32_t lenf = M.chunk_len[cs];
    const BRowTot t = S.rowtot[(int64_t)s * P.Bp + node];
    RowView rv;
    rv.minfin = t.minfin;
    rv.maxfin = t.maxfin;
    rv.lhs = S.lhs[row];
    rv.rhs = S.rhs[row];
    rv.mininf = t.mininf;
    rv.maxinf = t.maxinf;
    rv.thr_r = t.thr_r;
    rv.thr_l = t.thr_l;
    rv.exact = (lenf & kExactFlag) ? 1 : 0;
    rv.act = on ? 1 : 0;
    const int64_t base = M.slice_off[cs / kSliceW] + (cs % kSliceW);
    chunk_candidates<kCo>(M, S, base, lenf & kLenMask, node, on, row, rv, P, pq, chg_next);
  }
  drain_pairs<kCo>(pq, M, S, P, chg_next);
}

// ----------------------------------------------------------- k_bfinish --

// Commits the entries improved this round (the next state becomes the
// current one) and tests them for crossing bounds (Sec. 1.1, remark after
// Step 3).  The entries are those marked in this round's change mask, which
// the candidate kernels set; a warp reads 32 consecutive mask words and
// commits each nonzero word with one lane per node of its group, so that the
// state is read and written in contiguous runs.  The previous round's mask
// (read by this round's marking) is cleared for reuse.  The last block to
// arrive counts the round for every live node, ends the nodes that stopped
// (no change, infeasible, or the cap) and sets the WHILE condition.
__device__ __forceinline__ void bfinish_commit(const BatchState &S, int32_t n,
                                               const BParams &P, uint32_t *s_chg,
                                               uint32_t *s_inf) {
  const int p = P.round & 1;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < kMaxGroups) {
    s_chg[threadIdx.x] = 0u;
    s_inf[threadIdx.x] = 0u;
  }
  __syncthreads();
  if (!P.err) {
    const uint32_t *chg_next = S.chg[p ^ 1];
    uint32_t *chg_cur = S.chg[p];
    const int64_t words = (int64_t)n * P.Gs;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;  // 32 words per warp
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < words;
         w0 += wstride) {
      uint32_t c = 0u;
      if (w0 + lane < words) {
        c = chg_next[w0 + lane];
        if (chg_cur[w0 + lane] != 0u) chg_cur[w0 + lane] = 0u;
      }
      unsigned nz = __ballot_sync(kFull, c != 0u);
      while (nz != 0u) {
        // up to four nonzero words per step, their loads in flight together
        int k[4];
        uint32_t wd[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          k[u] = nz != 0u ? __ffs(nz) - 1 : 0;
          const uint32_t v = __shfl_sync(kFull, c, k[u]);
          wd[u] = nz != 0u ? v : 0u;
          nz &= nz - 1u;
        }
        longlong2 kk[4];
        bool isint[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t w = w0 + k[u];
          const int64_t j = w / P.Gs;
          const int node = (int)(w % P.Gs) * 32 + lane;
          kk[u] = make_longlong2(0, 0);
          isint[u] = false;
          if ((wd[u] >> lane) & 1u) {
            kk[u] = reinterpret_cast<const longlong2 *>(S.nkey)[j * P.Bp + node];
            isint[u] = S.vt[j] != 0;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t w = w0 + k[u];
          const int64_t j = w / P.Gs;
          const int g = (int)(w % P.Gs);
          const int node = g * 32 + lane;
          if ((wd[u] >> lane) & 1u) {
            const double L = val_of_key(kk[u].x), U = val_of_key(kk[u].y);
            put_entry(S, j * P.Bp + node, L, U, isint[u], P.tau_dn, P.eps_dn);
            if (kk[u].x > kk[u].y) {  // L > U in key order: test the crossing exactly
              const bool cross = isint[u] ? (L > U) : (L > U + P.eps_feas * d_max1abs(U));
              if (cross) atomicOr(&s_inf[g], 1u << lane);
            }
          }
          if (lane == 0 && wd[u] != 0u) atomicOr(&s_chg[g], wd[u]);
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < P.G) {
    if (s_chg[threadIdx.x]) atomicOr(&S.chg_bits[threadIdx.x], s_chg[threadIdx.x]);
    if (s_inf[threadIdx.x]) atomicOr(&S.inf_bits[threadIdx.x], s_inf[threadIdx.x]);
  }
}

// End of a round, one block, after every block's commit: counts the round
// for every live node, ends the nodes that stopped (no change, infeasible,
// or the cap), resets the per-round counters and sets the loop condition
// (the graph's WHILE handle when use_cond).
__device__ __forceinline__ void bfinish_decide(const BatchState &S, const BParams &P,
                                               cudaGraphConditionalHandle handle,
                                               int use_cond) {
  BCtrl *ctrl = S.ctrl;
  const int p = P.round & 1;
  const int32_t r = P.round + 1;
  const volatile uint32_t *chg_bits = S.chg_bits;
  const volatile uint32_t *inf_bits = S.inf_bits;
  int live = 0;
  // warp-uniform trip count (Bp and the block are multiples of 32): the
  // lanes of a warp are the 32 nodes of one group, whose live mask is a ballot
  for (int node = threadIdx.x; node < P.Bp; node += blockDim.x) {
    int32_t d = S.node_done[node];
    if (!d && !P.err) {
      // each node counts its own rounds (nodes admitted later start at 0)
      const uint32_t b = 1u << (node & 31);
      const int32_t rn = S.node_rounds[node] + 1;
      S.node_rounds[node] = rn;
      if (inf_bits[node >> 5] & b) d = 1;
      else if (!(chg_bits[node >> 5] & b)) d = 1;
      else if (rn >= P.max_rounds) {
        d = 1;
        S.node_status[node] = 1;
      }
    }
    S.node_done[node] = d;
    const unsigned w = __ballot_sync(kFull, d == 0);
    if ((threadIdx.x & 31) == 0) S.alive[node >> 5] = w;
    live |= w != 0u;
  }
  for (int g = P.G + (int)threadIdx.x; g < P.Gs; g += blockDim.x) S.alive[g] = 0u;
  live = __syncthreads_or(live);
  if (threadIdx.x < kMaxGroups) {
    ctrl->icount[threadIdx.x] = 0;
    S.chg_bits[threadIdx.x] = 0u;
    S.fresh[threadIdx.x] = 0u;
  }
  if (threadIdx.x == 0) {
    volatile BCtrl *vc = ctrl;
    vc->round = r;
    const int32_t cont = (live && !P.err) ? 1 : 0;
    vc->any_alive = cont;
    vc->blocks_done = 0;
    __threadfence();
    if (use_cond) cudaGraphSetConditional(handle, (unsigned)cont);
  }
  (void)p;
}

// ------------------------------------------------- round kernels (graph) --

__global__ void __launch_bounds__(kThreads) k_bmark(DevMatrix M, BatchState S) {
  bmark_body(M, S);
}

__global__ void __launch_bounds__(kThreads) k_bmark_split(DevMatrix M, BatchState S) {
  bmark_split_body(M, S);
}

// Four blocks of eight warps per SM (64 registers, a few spilled): the
// kernel waits on gathers, and 32 resident warps hide more of that latency
// than 24 warps without spills do (7% faster on a dense first round).
__global__ void __launch_bounds__(kActWarps * 32, 4) k_bact(DevMatrix M, BatchState S) {
  __shared__ PairBuf s_pairs[kActWarps];
  bact_body<false>(M, S, s_pairs);
}

__global__ void __launch_bounds__(kThreads) k_bcombine(DevMatrix M, BatchState S) {
  bcombine_body(M, S);
}

__global__ void __launch_bounds__(kThreads, 3) k_bcand_split(DevMatrix M, BatchState S) {
  __shared__ PairBuf s_pairs[kThreads / 32];
  bcand_split_body<false>(M, S, s_pairs);
}

// Commit of every block, then the last block to arrive ends the round.
__global__ void __launch_bounds__(kThreads)
k_bfinish(BatchState S, int32_t n, cudaGraphConditionalHandle handle, int use_cond) {
  __shared__ uint32_t s_chg[kMaxGroups], s_inf[kMaxGroups];
  __shared__ int s_last;
  const BParams P = load_params(S.ctrl);
  bfinish_commit(S, n, P, s_chg, s_inf);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&S.ctrl->blocks_done, 1u);
    s_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  bfinish_decide(S, P, handle, use_cond);
}

// ------------------------------------------------ round loop (persistent) --

// Grid barrier of the persistent loop over the batch's control block: as
// the single-instance loop's, a block that waits more than `limit` sleeps of
// 64 ns records DP_ERR_TIMEOUT and leaves, and every block returns false
// once an error is recorded.  The fences make each phase's writes (plain
// stores and atomics) visible to every block of the next phase.
__device__ __forceinline__ bool bgrid_sync(BCtrl *c, long long limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = &c->bar_gen;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(&c->bar_count, 1u) == gridDim.x - 1) {
      *(volatile unsigned *)&c->bar_count = 0u;  // all arrived; none leaves before gen moves
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      long long it = 0;
      while (*gen == g) {
        if (++it > limit) {
          atomicExch(&c->err, DP_ERR_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ((volatile BCtrl *)c)->err == 0;
}

// The batch's whole round loop in one cooperative launch (Sec. 3.7: one
// kernel for all rounds).  Each phase is the body of the graph kernel of
// the same name, grid-strided over the resident blocks, with a grid barrier
// between phases instead of a kernel boundary; block 0 ends each round.
// Four blocks per SM, as k_bact.
__global__ void __launch_bounds__(kThreads, 4) k_bpersistent(DevMatrix M, BatchState S) {
  __shared__ PairBuf s_pairs[kThreads / 32];
  __shared__ uint32_t s_chg[kMaxGroups], s_inf[kMaxGroups];
  BCtrl *ctrl = S.ctrl;
  if (((volatile BCtrl *)ctrl)->err) return;  // set before the launch: uniform
  const long long lim = ctrl->wait_limit;
  const bool split = M.nsplit_rows > 0;
  for (;;) {
    bmark_body(M, S);
    if (!bgrid_sync(ctrl, lim)) return;
    if (split) {
      bmark_split_body(M, S);
      if (!bgrid_sync(ctrl, lim)) return;
    }
    bact_body<true>(M, S, s_pairs);
    if (!bgrid_sync(ctrl, lim)) return;
    if (split) {
      bcombine_body(M, S);
      if (!bgrid_sync(ctrl, lim)) return;
      bcand_split_body<true>(M, S, s_pairs);
      if (!bgrid_sync(ctrl, lim)) return;
    }
    const BParams P = load_params(ctrl);
    bfinish_commit(S, M.n, P, s_chg, s_inf);
    if (!bgrid_sync(ctrl, lim)) return;
    if (blockIdx.x == 0) bfinish_decide(S, P, 0, 0);
    if (!bgrid_sync(ctrl, lim)) return;
    if (!((volatile BCtrl *)ctrl)->any_alive) return;
  }
}

// ---------------------------------------------------- prologue/epilogue --

// Normalises node-major bounds (lb[node*n + j]) into the node-minor state,
// 32 variables x 32 nodes per tile through shared memory so that both the
// reads and the writes are coalesced.  |v| >= thr becomes +-inf, integer
// bounds are rounded (ceil(lb - eps_int), floor(ub + eps_int)); NaN and
// contradictory infinities set ctrl->err.  Padding nodes get [0, 0].
__global__ void __launch_bounds__(kThreads)
k_bprologue_bounds(BatchState S, int32_t n, int32_t count, int32_t Bp, const double *lb,
                   const double *ub, const uint8_t *vartype, double eps_int, double tau_rel,
                   double eps_feas, double thr) {
  __shared__ double sL[32][33], sU[32][33];
  const double pinf = __longlong_as_double(0x7FF0000000000000ll);
  const long long k_thr = cmp_key(thr), k_mthr = cmp_key(-thr);
  const float tau_dn = f32_dn(tau_rel), eps_dn = f32_dn(eps_int);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int G = Bp / 32;
  const int64_t tiles_x = ((int64_t)n + 31) / 32;
  const int64_t tiles = tiles_x * G;
  bool bad = false;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t j0 = (t % tiles_x) * 32;
    const int g = (int)(t / tiles_x);
    for (int yy = ty; yy < 32; yy += kThreads / 32) {
      const int node = g * 32 + yy;
      const int64_t j = j0 + tx;
      double L = 0.0, U = 0.0;
      if (node < count && j < n) {
        L = lb[(int64_t)node * n + j];
        U = ub[(int64_t)node * n + j];
        // comparisons with +-thr on order-preserving keys (integer pipe;
        // the same decisions as the binary64 comparisons for non-NaN values)
        if (d_isnan(L) || d_isnan(U) || cmp_key(L) >= k_thr || cmp_key(U) <= k_mthr) {
          bad = true;
          L = 0.0;
          U = 0.0;
        }
        if (cmp_key(L) <= k_mthr) L = -pinf;
        if (cmp_key(U) >= k_thr) U = pinf;
        const bool isint = vartype[j] != 0;
        if (isint) {
          if (d_isfinite(L)) L = d_ceil_int(L - eps_int);
          if (d_isfinite(U)) U = d_floor_int(U + eps_int);
        }
        // Bounds that already cross: the crossing test of round 1 covers
        // every variable, and tightening cannot undo a crossing, so the
        // node is flagged now and ends after its first round.
        if (cmp_key(L) > cmp_key(U) && (isint || L > U + eps_feas * d_max1abs(U)))
          atomicOr(&S.inf_bits[node >> 5], 1u << (node & 31));
      }
      sL[yy][tx] = L;
      sU[yy][tx] = U;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += kThreads / 32) {
      const int64_t j = j0 + yy;
      if (j < n) {
        const int64_t e = j * Bp + g * 32 + tx;
        const double L = sL[tx][yy], U = sU[tx][yy];
        put_entry(S, e, L, U, vartype[j] != 0, tau_dn, eps_dn);
        reinterpret_cast<longlong2 *>(S.nkey)[e] = make_longlong2(key_of(L), key_of(U));
      }
    }
    __syncthreads();
  }
  if (bad) atomicExch(&S.ctrl->err, DP_ERR_NAN_INPUT);
}

// Variable types, normalised sides, per-node state and the live masks.
__global__ void k_bprologue_misc(BatchState S, int32_t m, int32_t n, int32_t count, int32_t Bp,
                                 const uint8_t *vartype, const double *lhs, const double *rhs,
                                 double thr) {
  const double pinf = __longlong_as_double(0x7FF0000000000000ll);
  const int Gs = ((Bp / 32) + 3) & ~3;
  int64_t total = n > m ? n : m;
  if (total < Bp) total = Bp;
  if (total < kMaxGroups) total = kMaxGroups;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) S.vt[i] = vartype[i] ? 1 : 0;
    if (i < m) {
      double l = lhs[i], r = rhs[i];
      if (d_isnan(l) || d_isnan(r) || l >= thr || r <= -thr) {
        atomicExch(&S.ctrl->err, DP_ERR_NAN_INPUT);
        l = 0.0;
        r = 0.0;
      }
      if (l <= -thr) l = -pinf;
      if (r >= thr) r = pinf;
      S.lhs[i] = l;
      S.rhs[i] = r;
    }
    if (i < kMaxGroups) {
      S.inf_bits[i] = 0u;
      S.chg_bits[i] = 0u;
    }
    if (i < Bp) {
      S.node_rounds[i] = 0;
      S.node_status[i] = 0;
      S.node_done[i] = i < count ? 0 : 1;
    }
    if (i < kMaxGroups) {
      const int64_t lo = i * 32;
      uint32_t w = 0u;
      for (int b = 0; b < 32; ++b)
        if (i < Gs && lo + b < count) w |= 1u << b;
      S.alive[i] = w;
      S.fresh[i] = w;
    }
  }
}

__global__ void __launch_bounds__(kThreads)
k_bepilogue(BatchState S, int32_t n, int32_t count, int32_t Bp, double *lb_out,
            double *ub_out) {
  __shared__ double sL[32][33], sU[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int G = Bp / 32;
  const int64_t tiles_x = ((int64_t)n + 31) / 32;
  const int64_t tiles = tiles_x * G;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t j0 = (t % tiles_x) * 32;
    const int g = (int)(t / tiles_x);
    for (int yy = ty; yy < 32; yy += kThreads / 32) {
      const int64_t j = j0 + yy;
      double2 b = make_double2(0.0, 0.0);
      if (j < n) b = S.cur[j * Bp + g * 32 + tx];
      sL[tx][yy] = b.x;
      sU[tx][yy] = b.y;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += kThreads / 32) {
      const int node = g * 32 + yy;
      const int64_t j = j0 + tx;
      if (node < count && j < n) {
        lb_out[(int64_t)node * n + j] = sL[yy][tx];
        ub_out[(int64_t)node * n + j] = sU[yy][tx];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------- slots (request serving) --
//
// A long-running batch whose nodes are independent requests: between rounds
// finished nodes are read out and their slots refilled with new requests,
// which start with every row active (fresh) and count their own rounds.

// Per-node state of newly admitted slots.  Thread per admitted slot.
__global__ void k_bslot_reset(BatchState S, const int32_t *slots, int32_t count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int node = slots[i];
  const uint32_t b = 1u << (node & 31);
  S.node_done[node] = 0;
  S.node_rounds[node] = 0;
  S.node_status[node] = 0;
  atomicAnd(&S.inf_bits[node >> 5], ~b);
  atomicOr(&S.alive[node >> 5], b);
  atomicOr(&S.fresh[node >> 5], b);
}

// Bounds of newly admitted slots: staged request vectors (slot i's lb at
// stage + 2*i*n, its ub n entries later; already validated) normalised
// into the slot's node column.  A crossing input flags the node.
__global__ void __launch_bounds__(kThreads)
k_bslot_fill(BatchState S, const int32_t *slots, int32_t count, const double *stage, int32_t n,
             int32_t Bp, double eps_int, double tau_rel, double eps_feas, double thr) {
  const double pinf = __longlong_as_double(0x7FF0000000000000ll);
  const long long k_thr = cmp_key(thr), k_mthr = cmp_key(-thr);
  const float tau_dn = f32_dn(tau_rel), eps_dn = f32_dn(eps_int);
  const int64_t total = (int64_t)count * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / n, j = t % n;
    const int node = slots[i];
    double L = stage[2 * i * n + j], U = stage[(2 * i + 1) * n + j];
    if (cmp_key(L) <= k_mthr) L = -pinf;
    if (cmp_key(U) >= k_thr) U = pinf;
    const bool isint = S.vt[j] != 0;
    if (isint) {
      if (d_isfinite(L)) L = d_ceil_int(L - eps_int);
      if (d_isfinite(U)) U = d_floor_int(U + eps_int);
    }
    if (cmp_key(L) > cmp_key(U) && (isint || L > U + eps_feas * d_max1abs(U)))
      atomicOr(&S.inf_bits[node >> 5], 1u << (node & 31));
    const int64_t e = j * Bp + node;
    put_entry(S, e, L, U, isint, tau_dn, eps_dn);
    reinterpret_cast<longlong2 *>(S.nkey)[e] = make_longlong2(key_of(L), key_of(U));
  }
}

// Bounds of finished slots into contiguous vectors (slot i's lb at
// out + 2*i*n, its ub n entries later).
__global__ void __launch_bounds__(kThreads)
k_bslot_extract(BatchState S, const int32_t *slots, int32_t count, double *out, int32_t n,
                int32_t Bp) {
  const int64_t total = (int64_t)count * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / n, j = t % n;
    const double2 b = S.cur[j * Bp + slots[i]];
    out[2 * i * n + j] = b.x;
    out[(2 * i + 1) * n + j] = b.y;
  }
}

// Sides, types and the empty per-node state of a serving batch (no node
// occupied yet).
__global__ void k_bslots_init(BatchState S, int32_t m, int32_t n, int32_t Bp,
                              const uint8_t *vartype, const double *lhs, const double *rhs,
                              double thr) {
  const double pinf = __longlong_as_double(0x7FF0000000000000ll);
  int64_t total = n > m ? n : m;
  if (total < Bp) total = Bp;
  if (total < kMaxGroups) total = kMaxGroups;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) S.vt[i] = vartype[i] ? 1 : 0;
    if (i < m) {
      double l = lhs[i], r = rhs[i];
      if (l <= -thr) l = -pinf;
      if (r >= thr) r = pinf;
      S.lhs[i] = l;
      S.rhs[i] = r;
    }
    if (i < Bp) {
      S.node_rounds[i] = 0;
      S.node_status[i] = 0;
      S.node_done[i] = 1;
    }
    if (i < kMaxGroups) {
      S.inf_bits[i] = 0u;
      S.chg_bits[i] = 0u;
      S.alive[i] = 0u;
      S.fresh[i] = 0u;
    }
  }
}

int grid_for(int64_t work, int threads, int max_blocks) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

}  // namespace

cudaError_t launch_batch_prologue(const DevMatrix &M, const BatchState &S, int32_t count,
                                  const double *lb, const double *ub, const uint8_t *vartype,
                                  const double *lhs, const double *rhs, double eps_int,
                                  double tau_rel, double eps_feas, double thr, int num_sms,
                                  cudaStream_t st) {
  const int32_t Bp = (count + 31) / 32 * 32;
  const int64_t tiles = (((int64_t)M.n + 31) / 32) * (Bp / 32);
  int64_t total = M.n > M.m ? M.n : M.m;
  if (total < Bp) total = Bp;
  if (total < kMaxGroups) total = kMaxGroups;
  k_bprologue_misc<<<grid_for(total, kThreads, num_sms * 16), kThreads, 0, st>>>(
      S, M.m, M.n, count, Bp, vartype, lhs, rhs, thr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || M.n == 0) return e;
  int nb = (int)(tiles < (int64_t)num_sms * 16 ? tiles : (int64_t)num_sms * 16);
  k_bprologue_bounds<<<nb, kThreads, 0, st>>>(S, M.n, count, Bp, lb, ub, vartype, eps_int,
                                              tau_rel, eps_feas, thr);
  return cudaGetLastError();
}

cudaError_t launch_batch_epilogue(const DevMatrix &M, const BatchState &S, int32_t count,
                                  double *lb_out, double *ub_out, int num_sms,
                                  cudaStream_t st) {
  if (M.n == 0 || count == 0) return cudaSuccess;
  const int32_t Bp = (count + 31) / 32 * 32;
  const int64_t tiles = (((int64_t)M.n + 31) / 32) * (Bp / 32);
  int nb = (int)(tiles < (int64_t)num_sms * 16 ? tiles : (int64_t)num_sms * 16);
  k_bepilogue<<<nb, kThreads, 0, st>>>(S, M.n, count, Bp, lb_out, ub_out);
  return cudaGetLastError();
}

cudaError_t launch_batch_persistent(const DevMatrix &M, const BatchState &S, int num_sms,
                                    cudaStream_t st) {
  int per_sm = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bpersistent, kThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  DevMatrix m = M;
  BatchState s = S;
  void *args[] = {&m, &s};
  return cudaLaunchCooperativeKernel((const void *)k_bpersistent, dim3(num_sms * per_sm),
                                     dim3(kThreads), args, 0, st);
}

cudaError_t launch_batch_round(const DevMatrix &M, const BatchState &S,
                               cudaGraphConditionalHandle handle, int use_cond, int num_sms,
                               cudaStream_t st, cudaEvent_t *ev) {
  cudaError_t e;
  const int64_t nslots = (int64_t)M.nslices * kSliceW;
  const bool split = M.nsplit_rows > 0;
  auto mark = [&](int k) {
    if (ev) cudaEventRecord(ev[k], st);
  };
  // grid-stride over the chunks: at most the blocks resident at once
  static int mark_blocks_per_sm = 0;
  if (mark_blocks_per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bmark, kThreads, 0) != cudaSuccess ||
        b < 1)
      b = 4;
    mark_blocks_per_sm = b;
  }
  mark(0);
  k_bmark<<<grid_for(nslots, kThreads, num_sms * mark_blocks_per_sm), kThreads, 0, st>>>(M, S);
  mark(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  mark(2);
  if (split)
    k_bmark_split<<<grid_for((int64_t)M.nsplit_rows * kThreads, kThreads, num_sms * 4), kThreads,
                    0, st>>>(M, S);
  mark(3);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  mark(4);
  k_bact<<<num_sms * 4, kActWarps * 32, 0, st>>>(M, S);
  mark(5);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  mark(6);
  if (split) k_bcombine<<<num_sms * 4, kThreads, 0, st>>>(M, S);
  mark(7);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  mark(8);
  if (split) k_bcand_split<<<num_sms * 3, kThreads, 0, st>>>(M, S);
  mark(9);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  mark(10);
  k_bfinish<<<num_sms * 4, kThreads, 0, st>>>(S, M.n, handle, use_cond);
  mark(11);
  return cudaGetLastError();
}

cudaError_t launch_slots_init(const DevMatrix &M, const BatchState &S, int32_t Bp,
                              const uint8_t *vartype, const double *lhs, const double *rhs,
                              double thr, int num_sms, cudaStream_t st) {
  int64_t total = M.n > M.m ? M.n : M.m;
  if (total < Bp) total = Bp;
  if (total < kMaxGroups) total = kMaxGroups;
  k_bslots_init<<<grid_for(total, kThreads, num_sms * 8), kThreads, 0, st>>>(S, M.m, M.n, Bp,
                                                                             vartype, lhs, rhs, thr);
  return cudaGetLastError();
}

cudaError_t launch_slots_admit(const DevMatrix &M, const BatchState &S, int32_t Bp,
                               const int32_t *slots, int32_t count, const double *stage,
                               double eps_int, double tau_rel, double eps_feas, double thr,
                               int num_sms, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_bslot_reset<<<(count + 127) / 128, 128, 0, st>>>(S, slots, count);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || M.n == 0) return e;
  k_bslot_fill<<<grid_for((int64_t)count * M.n, kThreads, num_sms * 8), kThreads, 0, st>>>(
      S, slots, count, stage, M.n, Bp, eps_int, tau_rel, eps_feas, thr);
  return cudaGetLastError();
}

cudaError_t launch_slots_extract(const DevMatrix &M, const BatchState &S, int32_t Bp,
                                 const int32_t *slots, int32_t count, double *out,
                                 int num_sms, cudaStream_t st) {
  if (count <= 0 || M.n == 0) return cudaSuccess;
  k_bslot_extract<<<grid_for((int64_t)count * M.n, kThreads, num_sms * 8), kThreads, 0, st>>>(
      S, slots, count, out, M.n, Bp);
  return cudaGetLastError();
}

}  // namespace dp
