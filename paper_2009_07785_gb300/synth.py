"""Seeded synthetic constraint systems  lhs <= A x <= rhs,  lb <= x <= ub.

These stand in for the MIPLIB 2017 instances the paper measures on (Sec. 4.1),
which are not available here.  Every instance is built around a feasible
point x* inside the bounds: rhs = A x* + slack, lhs = -inf or A x* - slack,
so propagation never proves infeasibility on a generated instance (only on
node fixings).  This module draws inputs only; it holds none of the
propagation arithmetic, and both the CUDA path and the CPU oracle consume
what it returns.

Workloads (sizes, distributions; seeds are 2009_07785 + 100*config + k):
  tiny     m=2,000   n=1,500   lengths U{2..10}, integer coefficients
  medium   m=200k    n=150k    Zipf(1.5) lengths clipped to 2..24 plus 15
                               knapsack rows of 20k..50k nonzeros, 30%
                               set-partitioning rows, log-uniform coefficients
  large    m=2M      n=1.5M    97.2% U{2..12}, 2.7% U{13..400}, 100 rows
                               U{401..100k} (~30M nonzeros), tiny's value
                               distributions
  nodes    branch-and-bound node bound vectors over an instance (1-5% of the
           integer variables fixed to a random value of their domain)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2009_07785


def seed_for(config: int, k: int = 0) -> int:
    return SEED_BASE + 100 * config + k


@dataclass
class Instance:
    name: str
    m: int
    n: int
    row_ptr: np.ndarray  # int64 [m+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]
    lb: np.ndarray       # float64 [n]
    ub: np.ndarray       # float64 [n]
    vartype: np.ndarray  # uint8 [n], 1 = integer
    lhs: np.ndarray      # float64 [m]
    rhs: np.ndarray      # float64 [m]
    xstar: np.ndarray    # float64 [n], a feasible point
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def problem(self):
        """The arrays a propagation call takes, in argument order."""
        return self.lb, self.ub, self.vartype, self.lhs, self.rhs


def _distinct_columns(rng: np.random.Generator, lengths: np.ndarray, n: int) -> np.ndarray:
    """Distinct uniformly random columns per row, sorted within each row."""
    m = lengths.size
    nnz = int(lengths.sum())
    row_of = np.repeat(np.arange(m, dtype=np.int64), lengths)
    cols = rng.integers(0, n, size=nnz, dtype=np.int64)
    for _ in range(64):
        key = row_of * n + cols
        key.sort()
        cols = key - row_of * n
        dup = np.zeros(nnz, dtype=bool)
        dup[1:] = key[1:] == key[:-1]
        nd = int(dup.sum())
        if nd == 0:
            return cols.astype(np.int32)
        cols[dup] = rng.integers(0, n, size=nd, dtype=np.int64)
    raise RuntimeError("could not draw distinct columns (rows longer than n?)")


def _row_ptr(lengths: np.ndarray) -> np.ndarray:
    rp = np.zeros(lengths.size + 1, dtype=np.int64)
    np.cumsum(lengths, out=rp[1:])
    return rp


def _rowdot(row_ptr, col, val, x) -> np.ndarray:
    """A x for the feasible point (the generator's own matrix-vector product)."""
    prod = val * x[col]
    m = row_ptr.size - 1
    out = np.zeros(m)
    nz = np.diff(row_ptr) > 0
    out[nz] = np.add.reduceat(prod, row_ptr[:-1][nz])
    return out


def _tiny_like_vars(rng, n: int, int_frac=0.6, inf_frac=0.1):
    """Variable types and bounds of the tiny workload: 60% integer (half
    binary [0,1], half [0,U] with U in 1..20); continuous lb 0, ub U[1,100]
    with 10% ub = +inf; x* uniform inside the bounds ([0,100] when ub=inf)."""
    vt = (rng.random(n) < int_frac).astype(np.uint8)
    lb = np.zeros(n)
    ub = np.empty(n)
    isint = vt == 1
    binary = isint & (rng.random(n) < 0.5)
    gen = isint & ~binary
    ub[binary] = 1.0
    ub[gen] = rng.integers(1, 21, size=int(gen.sum())).astype(float)
    cont = ~isint
    ub[cont] = rng.uniform(1.0, 100.0, size=int(cont.sum()))
    inf = cont & (rng.random(n) < inf_frac)
    ub[inf] = np.inf
    x = np.empty(n)
    x[isint] = np.floor(rng.random(int(isint.sum())) * (ub[isint] + 1.0))
    x[isint] = np.minimum(x[isint], ub[isint])
    cfin = cont & ~inf
    x[cfin] = rng.random(int(cfin.sum())) * ub[cfin]
    x[inf] = rng.random(int(inf.sum())) * 100.0
    return vt, lb, ub, x


def _sides(rng, row_ptr, col, val, x, ranged_frac=0.1, slack_mean=2.0):
    ax = _rowdot(row_ptr, col, val, x)
    m = ax.size
    rhs = ax + rng.exponential(slack_mean, size=m)
    lhs = np.full(m, -np.inf)
    ranged = rng.random(m) < ranged_frac
    lhs[ranged] = ax[ranged] - rng.exponential(slack_mean, size=int(ranged.sum()))
    return lhs, rhs


def tiny(seed: int | None = None, m: int = 2000, n: int = 1500) -> Instance:
    """The tiny workload (2,000 x 1,500, ~12k nonzeros)."""
    seed = seed_for(0) if seed is None else seed
    rng = np.random.default_rng(seed)
    lengths = rng.integers(2, 11, size=m)
    col = _distinct_columns(rng, lengths, n)
    mag = rng.integers(1, 11, size=col.size).astype(float)
    val = np.where(rng.random(col.size) < 0.5, -mag, mag)
    vt, lb, ub, x = _tiny_like_vars(rng, n)
    rp = _row_ptr(lengths)
    lhs, rhs = _sides(rng, rp, col, val, x)
    return Instance("tiny", m, n, rp, col, val, lb, ub, vt, lhs, rhs, x, seed)


def large(seed: int | None = None, scale: float = 1.0) -> Instance:
    """The large workload (2M x 1.5M, ~30M nonzeros); `scale` shrinks m and n
    (and the long-row count) proportionally for smaller test cases."""
    seed = seed_for(2) if seed is None else seed
    rng = np.random.default_rng(seed)
    m = max(64, int(round(2_000_000 * scale)))
    n = max(64, int(round(1_500_000 * scale)))
    nlong = max(1, int(round(100 * scale)))
    nmed = int(round(0.027 * m))
    nshort = m - nmed - nlong
    maxlong = min(100_000, n // 2)
    lengths = np.concatenate([
        rng.integers(2, 13, size=nshort),
        rng.integers(13, min(401, n // 2) + 1, size=nmed),
        rng.integers(min(401, maxlong), maxlong + 1, size=nlong),
    ])
    rng.shuffle(lengths)
    col = _distinct_columns(rng, lengths, n)
    mag = rng.integers(1, 11, size=col.size).astype(float)
    val = np.where(rng.random(col.size) < 0.5, -mag, mag)
    vt, lb, ub, x = _tiny_like_vars(rng, n)
    rp = _row_ptr(lengths)
    lhs, rhs = _sides(rng, rp, col, val, x)
    return Instance("large", m, n, rp, col, val, lb, ub, vt, lhs, rhs, x, seed,
                    meta={"scale": scale})


def medium(seed: int | None = None, scale: float = 1.0) -> Instance:
    """The medium irregular workload (200k x 150k, ~2M nonzeros).

    Bulk row lengths are Zipf(1.5) clipped to 2..24 plus 15 planted knapsack
    rows of 20k..50k nonzeros (positive coefficients, rhs only).  30% of the
    rows are set-partitioning rows (+1 over binaries, lhs = rhs = 1, exactly
    one binary of the row at 1 in x*).  Other coefficients have random sign
    and magnitude 10^U[-2,3].  50% integer variables (half binary), 5% of the
    non-binary variables get one infinite side.
    """
    seed = seed_for(1) if seed is None else seed
    rng = np.random.default_rng(seed)
    m = max(64, int(round(200_000 * scale)))
    n = max(64, int(round(150_000 * scale)))
    nknap = max(1, int(round(15 * scale)))
    kmax = min(50_000, max(8, n // 3))
    kmin = min(20_000, kmax)
    # variables
    vt = (rng.random(n) < 0.5).astype(np.uint8)
    isint = vt == 1
    binary = isint & (rng.random(n) < 0.5)
    gen = isint & ~binary
    cont = ~isint
    lb = np.zeros(n)
    ub = np.empty(n)
    ub[binary] = 1.0
    ub[gen] = rng.integers(1, 21, size=int(gen.sum())).astype(float)
    ub[cont] = rng.uniform(1.0, 100.0, size=int(cont.sum()))
    x = np.empty(n)
    x[gen] = np.minimum(np.floor(rng.random(int(gen.sum())) * (ub[gen] + 1.0)), ub[gen])
    x[cont] = rng.random(int(cont.sum())) * ub[cont]
    bins = np.flatnonzero(binary)
    ones = bins[rng.random(bins.size) < 0.1]
    if ones.size == 0:
        ones = bins[:1]
    zeros = np.setdiff1d(bins, ones)
    x[bins] = 0.0
    x[ones] = 1.0
    # one infinite side on 5% of the non-binary variables (x* stays finite)
    nb = np.flatnonzero(~binary)
    pick = nb[rng.random(nb.size) < 0.05]
    up = rng.random(pick.size) < 0.5
    ub[pick[up]] = np.inf
    lbinf = pick[~up]
    lb[lbinf] = -np.inf
    # rows
    nsp = int(round(0.3 * m))
    nother = m - nsp - nknap
    zl = np.clip(rng.zipf(1.5, size=nsp + nother), 2, 24)
    sp_len = np.minimum(zl[:nsp], max(2, zeros.size + 1))
    other_len = zl[nsp:]
    knap_len = rng.integers(kmin, kmax + 1, size=nknap)
    # set-partitioning rows: one binary at 1 plus len-1 binaries at 0
    sp_rows = []
    for ln in sp_len:
        c = np.concatenate([[rng.choice(ones)], rng.choice(zeros, size=int(ln) - 1, replace=False)])
        sp_rows.append(np.sort(c))
    sp_col = np.concatenate(sp_rows).astype(np.int32) if sp_rows else np.zeros(0, np.int32)
    other_col = _distinct_columns(rng, other_len, n)
    knap_col = _distinct_columns(rng, knap_len, n)
    other_val = (np.where(rng.random(other_col.size) < 0.5, -1.0, 1.0) *
                 10.0 ** rng.uniform(-2.0, 3.0, size=other_col.size))
    knap_val = 10.0 ** rng.uniform(-2.0, 3.0, size=knap_col.size)
    # knapsack rows must stay bounded above on x*: use finite-x* vars only
    lengths = np.concatenate([sp_len, other_len, knap_len])
    col = np.concatenate([sp_col, other_col, knap_col])
    val = np.concatenate([np.ones(sp_col.size), other_val, knap_val])
    kind = np.concatenate([np.zeros(nsp, np.int8), np.ones(nother, np.int8), np.full(nknap, 2, np.int8)])
    # shuffle row order
    perm = rng.permutation(m)
    rp0 = _row_ptr(lengths)
    seg = [np.arange(rp0[i], rp0[i + 1]) for i in perm]
    idx = np.concatenate(seg) if seg else np.zeros(0, np.int64)
    lengths = lengths[perm]
    col = col[idx]
    val = val[idx]
    kind = kind[perm]
    rp = _row_ptr(lengths)
    # x* for lb = -inf variables: somewhere below ub
    x[lbinf] = ub[lbinf] - rng.random(lbinf.size) * 100.0
    x[np.isinf(ub) & ~binary] = rng.random(int((np.isinf(ub) & ~binary).sum())) * 100.0
    x[isint] = np.floor(x[isint])  # integer variables need an integral x*
    lhs, rhs = _sides(rng, rp, col, val, x)
    sp = kind == 0
    lhs[sp] = 1.0
    rhs[sp] = 1.0
    lhs[kind == 2] = -np.inf
    return Instance("medium", m, n, rp, col, val, lb, ub, vt, lhs, rhs, x, seed,
                    meta={"scale": scale, "row_kind": kind})


def node_bounds(inst: Instance, count: int, seed: int, lo_frac=0.01, hi_frac=0.05):
    """Branch-and-bound node bound vectors: each fixes a random 1-5% of the
    integer variables (with finite bounds) to a random value of their domain.
    Returns (lb[count, n], ub[count, n])."""
    rng = np.random.default_rng(seed)
    ints = np.flatnonzero((inst.vartype == 1) & np.isfinite(inst.lb) & np.isfinite(inst.ub))
    LB = np.repeat(inst.lb[None, :], count, axis=0)
    UB = np.repeat(inst.ub[None, :], count, axis=0)
    for b in range(count):
        k = max(1, int(round(rng.uniform(lo_frac, hi_frac) * ints.size)))
        pick = rng.choice(ints, size=min(k, ints.size), replace=False)
        lo = np.ceil(inst.lb[pick])
        hi = np.floor(inst.ub[pick])
        v = lo + np.floor(rng.random(pick.size) * (hi - lo + 1.0))
        LB[b, pick] = v
        UB[b, pick] = v
    return LB, UB


def node_bounds_at_point(inst: Instance, count: int, seed: int, lo_frac=0.01, hi_frac=0.05):
    """Node bound vectors that fix a random 1-5% of the integer variables to
    their value in the instance's feasible point x* (every node stays
    feasible, as nodes on the path to a solution do).  Returns
    (lb[count, n], ub[count, n])."""
    rng = np.random.default_rng(seed)
    ints = np.flatnonzero((inst.vartype == 1) & np.isfinite(inst.lb) & np.isfinite(inst.ub))
    LB = np.repeat(inst.lb[None, :], count, axis=0)
    UB = np.repeat(inst.ub[None, :], count, axis=0)
    for b in range(count):
        k = max(1, int(round(rng.uniform(lo_frac, hi_frac) * ints.size)))
        pick = rng.choice(ints, size=min(k, ints.size), replace=False)
        LB[b, pick] = inst.xstar[pick]
        UB[b, pick] = inst.xstar[pick]
    return LB, UB


def small_random(rng: np.random.Generator, m: int, n: int, maxlen: int, int_frac=0.6,
                 coef=(1, 10), inf_frac=0.1, ranged_frac=0.2, slack_mean=2.0,
                 pure_integer=False, bounded=False) -> Instance:
    """Small random instances for exhaustive tests (same recipe as tiny)."""
    lengths = rng.integers(0 if m > 1 else 1, maxlen + 1, size=m)
    lengths = np.minimum(lengths, n)
    col = _distinct_columns(rng, lengths, n)
    mag = rng.integers(coef[0], coef[1] + 1, size=col.size).astype(float)
    val = np.where(rng.random(col.size) < 0.5, -mag, mag)
    vt, lb, ub, x = _tiny_like_vars(rng, n, int_frac=1.0 if pure_integer else int_frac,
                                    inf_frac=0.0 if bounded else inf_frac)
    rp = _row_ptr(lengths)
    lhs, rhs = _sides(rng, rp, col, val, x, ranged_frac=ranged_frac, slack_mean=slack_mean)
    return Instance("small", m, n, rp, col, val, lb, ub, vt, lhs, rhs, x, 0)
