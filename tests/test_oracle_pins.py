"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

None of these compare the oracle with itself:
  * closed forms derived by hand (tests/golden/closed_forms.json, each case
    with its citation and derivation);
  * the cascade pattern of Sec. 2.2: exact round counts for the round-
    synchronous and the sequential algorithm;
  * brute-force enumeration of tiny pure-integer systems (soundness: every
    feasible point stays inside the tightened bounds; an infeasibility
    verdict means there is no feasible point);
  * single-row continuous systems: the propagated bounds equal the LP
    projection computed by scipy's HiGHS; multi-row: they contain it;
  * the unique limit point (Sec. 1.1): the sequential Alg. 1 oracle, written
    separately in the Eq. 3 form, reaches the same bounds;
  * invariants: bounds only shrink (Sec. 3.5) and the generator's feasible
    point x* stays inside them in every round;
  * permutation invariance of the limit (App. B).
"""
import itertools
import json
from pathlib import Path

import numpy as np
import pytest

from paper_2009_07785_gb300 import synth

GOLDEN = Path(__file__).resolve().parent / "golden" / "closed_forms.json"


def _num(v):
    if isinstance(v, str):
        return float(v)
    return float(v)


def build_case(case):
    names = [v[0] for v in case["vars"]]
    idx = {nm: i for i, nm in enumerate(names)}
    n = len(names)
    vt = np.array([1 if v[1] == "int" else 0 for v in case["vars"]], np.uint8)
    lb = np.array([_num(v[2]) for v in case["vars"]])
    ub = np.array([_num(v[3]) for v in case["vars"]])
    rp, col, val, lhs, rhs = [0], [], [], [], []
    for lo, hi, coefs in case["rows"]:
        for nm, a in coefs.items():
            col.append(idx[nm])
            val.append(float(a))
        rp.append(len(col))
        lhs.append(_num(lo))
        rhs.append(_num(hi))
    inst = synth.Instance(case["name"], len(case["rows"]), n, np.array(rp, np.int64),
                          np.array(col, np.int32), np.array(val, np.float64), lb, ub, vt,
                          np.array(lhs), np.array(rhs), np.zeros(n))
    exp_lb = np.array([_num(case["expect"][nm][0]) for nm in names])
    exp_ub = np.array([_num(case["expect"][nm][1]) for nm in names])
    return inst, exp_lb, exp_ub


def load_cases():
    return json.loads(GOLDEN.read_text())["cases"]


@pytest.mark.parametrize("case", load_cases(), ids=lambda c: c["name"])
def test_closed_forms(orc, case):
    inst, elb, eub = build_case(case)
    r = orc.propagate_instance(inst)
    assert r.infeasible == case["infeasible"]
    assert r.rounds == case["rounds"]
    assert np.array_equal(r.lb, elb), (r.lb, elb)
    assert np.array_equal(r.ub, eub), (r.ub, eub)


def cascade(m, reverse=False):
    """x_{k+1} - x_k <= 0 for k = 0..m-1, x_0 fixed at 0, others integer in
    [0,10]: each constraint can only tighten after the previous one did
    (the cascading pattern of Sec. 2.2)."""
    n = m + 1
    rows = range(m - 1, -1, -1) if reverse else range(m)
    rp, col, val = [0], [], []
    for k in rows:
        col += [k + 1, k]
        val += [1.0, -1.0]
        rp.append(len(col))
    lb = np.zeros(n)
    ub = np.full(n, 10.0)
    ub[0] = 0.0
    return synth.Instance("cascade", m, n, np.array(rp, np.int64), np.array(col, np.int32),
                          np.array(val), lb, ub, np.ones(n, np.uint8), np.full(m, -np.inf),
                          np.zeros(m), np.zeros(n))


@pytest.mark.parametrize("m", [1, 5, 40])
def test_cascade_round_counts(orc, m):
    """Sec. 2.2: the parallel algorithm needs m rounds (plus the final no-change
    round); the sequential one needs one sweep (plus a check) in forward order
    and m sweeps in reverse order."""
    inst = cascade(m)
    r = orc.propagate_instance(inst)
    assert r.rounds == m + 1 and r.infeasible == 0
    assert np.all(r.ub == 0.0) and np.all(r.lb == 0.0)
    s = orc.propagate_seq_instance(inst)
    assert s.rounds == 2 and np.all(s.ub == 0.0)
    rev = cascade(m, reverse=True)
    assert orc.propagate_instance(rev).rounds == m + 1
    assert orc.propagate_seq_instance(rev).rounds == m + 1


def test_cascade_cap(orc):
    inst = cascade(30)
    r = orc.propagate_instance(inst, {"max_rounds": 10})
    assert r.rounds == 10 and r.status == 1 and r.infeasible == 0
    assert r.ub[10] == 0.0 and r.ub[11] == 10.0


def enumerate_points(inst):
    lo = np.ceil(inst.lb - 1e-9).astype(int)
    hi = np.floor(inst.ub + 1e-9).astype(int)
    pts = np.array(list(itertools.product(*[range(a, b + 1) for a, b in zip(lo, hi)])), float)
    if pts.size == 0:
        return pts.reshape(0, inst.n)
    A = np.zeros((inst.m, inst.n))
    for i in range(inst.m):
        for k in range(inst.row_ptr[i], inst.row_ptr[i + 1]):
            A[i, inst.col[k]] += inst.val[k]
    act = pts @ A.T
    ok = np.all((act >= inst.lhs - 1e-9) & (act <= inst.rhs + 1e-9), axis=1)
    return pts[ok]


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_soundness(orc, seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 7))
    m = int(rng.integers(1, 5))
    inst = synth.small_random(rng, m, n, maxlen=n, pure_integer=True, bounded=True,
                              slack_mean=0.7, ranged_frac=0.4)
    # cap domains at 0..3 so enumeration stays small
    inst.ub = np.minimum(inst.ub, 3.0)
    # shift sides so that some instances become infeasible
    if seed % 3 == 0:
        inst.rhs = inst.rhs - rng.uniform(0, 6, size=m)
    feas = enumerate_points(inst)
    r = orc.propagate_instance(inst)
    if r.infeasible:
        assert feas.shape[0] == 0, "infeasibility claimed but a feasible point exists"
    else:
        assert np.all(feas >= r.lb - 1e-9) and np.all(feas <= r.ub + 1e-9), \
            "a feasible point was cut off"
    # the sequential algorithm agrees on the verdict when both are conclusive
    s = orc.propagate_seq_instance(inst)
    if not r.infeasible and not s.infeasible:
        assert np.array_equal(r.lb, s.lb) and np.array_equal(r.ub, s.ub)


def _lp_bounds(inst, j):
    linprog = pytest.importorskip("scipy.optimize").linprog
    A = np.zeros((inst.m, inst.n))
    for i in range(inst.m):
        for k in range(inst.row_ptr[i], inst.row_ptr[i + 1]):
            A[i, inst.col[k]] += inst.val[k]
    A_ub, b_ub = [], []
    for i in range(inst.m):
        if np.isfinite(inst.rhs[i]):
            A_ub.append(A[i])
            b_ub.append(inst.rhs[i])
        if np.isfinite(inst.lhs[i]):
            A_ub.append(-A[i])
            b_ub.append(-inst.lhs[i])
    bnds = [(None if not np.isfinite(l) else l, None if not np.isfinite(u) else u)
            for l, u in zip(inst.lb, inst.ub)]
    c = np.zeros(inst.n)
    c[j] = 1.0
    lo = linprog(c, A_ub=np.array(A_ub), b_ub=np.array(b_ub), bounds=bnds, method="highs")
    hi = linprog(-c, A_ub=np.array(A_ub), b_ub=np.array(b_ub), bounds=bnds, method="highs")
    return lo, hi


@pytest.mark.parametrize("seed", range(25))
def test_single_row_equals_lp_projection(orc, seed):
    """For one linear row over a box, propagation computes the exact
    projection of the feasible set onto each variable."""
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(1, 7))
    inst = synth.small_random(rng, 1, n, maxlen=n, int_frac=0.0, bounded=True, ranged_frac=0.5)
    inst.val = rng.uniform(0.5, 5.0, size=inst.val.size) * np.sign(inst.val)
    x = inst.xstar
    ax = float(np.sum(inst.val * x[inst.col]))
    inst.rhs = np.array([ax + rng.exponential(1.0)])
    inst.lhs = np.array([ax - rng.exponential(1.0) if rng.random() < 0.5 else -np.inf])
    r = orc.propagate_instance(inst, {"tau_rel": 0.0})
    assert not r.infeasible
    for j in range(n):
        lo, hi = _lp_bounds(inst, j)
        assert lo.status == 0 and hi.status == 0
        assert abs(r.lb[j] - lo.fun) <= 1e-7 * max(1, abs(lo.fun)), (j, r.lb[j], lo.fun)
        assert abs(r.ub[j] + hi.fun) <= 1e-7 * max(1, abs(hi.fun)), (j, r.ub[j], -hi.fun)


@pytest.mark.parametrize("seed", range(10))
def test_multi_row_contains_lp_projection(orc, seed):
    rng = np.random.default_rng(3000 + seed)
    inst = synth.small_random(rng, 6, 5, maxlen=4, int_frac=0.0, bounded=True)
    r = orc.propagate_instance(inst)
    assert not r.infeasible
    for j in range(inst.n):
        lo, hi = _lp_bounds(inst, j)
        assert lo.status == 0 and hi.status == 0
        assert r.lb[j] <= lo.fun + 1e-7 * max(1, abs(lo.fun))
        assert r.ub[j] >= -hi.fun - 1e-7 * max(1, abs(hi.fun))


@pytest.mark.parametrize("seed", range(12))
def test_limit_point_matches_sequential(orc, seed):
    """Sec. 1.1: one limit point.  Pure-integer bounded systems: exact; mixed
    systems: within the comparison tolerance of Sec. 4.3."""
    rng = np.random.default_rng(4000 + seed)
    pure = seed % 2 == 0
    inst = synth.small_random(rng, 300, 200, maxlen=8, pure_integer=pure, bounded=pure)
    r = orc.propagate_instance(inst)
    s = orc.propagate_seq_instance(inst)
    assert r.infeasible == 0 and s.infeasible == 0
    if pure:
        assert np.array_equal(r.lb, s.lb) and np.array_equal(r.ub, s.ub)
    else:
        for a, b in ((s.lb, r.lb), (s.ub, r.ub)):
            same = (a == b) | (np.abs(a - b) <= 1e-8 + 1e-5 * np.abs(b))
            assert same.all()


def test_limit_point_tiny_workload(orc):
    inst = synth.tiny()
    r = orc.propagate_instance(inst)
    s = orc.propagate_seq_instance(inst)
    assert r.status == 0 and r.infeasible == 0 and s.infeasible == 0
    assert s.rounds <= r.rounds
    for a, b in ((s.lb, r.lb), (s.ub, r.ub)):
        assert ((a == b) | (np.abs(a - b) <= 1e-8 + 1e-5 * np.abs(b))).all()


@pytest.mark.parametrize("maker", ["tiny", "medium"])
def test_invariants_every_round(orc, maker):
    inst = synth.tiny() if maker == "tiny" else synth.medium(scale=0.05)
    r = orc.propagate_instance(inst, trace=True)
    assert r.infeasible == 0
    L0, U0, _, _ = orc.normalise(inst.m, inst.n, inst.lb, inst.ub, inst.vartype, inst.lhs, inst.rhs)
    prev_l, prev_u = L0, U0
    for t in range(r.rounds):
        l, u = r.trace_lb[t], r.trace_ub[t]
        assert np.all(l >= prev_l) and np.all(u <= prev_u), "a bound widened"
        assert np.all(inst.xstar >= l - 1e-9 * np.maximum(1, np.abs(l)))
        assert np.all(inst.xstar <= u + 1e-9 * np.maximum(1, np.abs(u)))
        prev_l, prev_u = l, u


def test_permutation_invariance(orc):
    """App. B: the limit does not depend on the order of rows and columns."""
    rng = np.random.default_rng(77)
    inst = synth.small_random(rng, 400, 300, maxlen=6, pure_integer=True, bounded=True)
    r = orc.propagate_instance(inst)
    pr = rng.permutation(inst.m)
    pc = rng.permutation(inst.n)
    inv = np.empty_like(pc)
    inv[pc] = np.arange(inst.n)
    lens = np.diff(inst.row_ptr)[pr]
    rp = np.zeros(inst.m + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    idx = np.concatenate([np.arange(inst.row_ptr[i], inst.row_ptr[i + 1]) for i in pr])
    col = inv[inst.col[idx]].astype(np.int32)
    q = synth.Instance("perm", inst.m, inst.n, rp, col, inst.val[idx], inst.lb[pc], inst.ub[pc],
                       inst.vartype[pc], inst.lhs[pr], inst.rhs[pr], inst.xstar[pc])
    rq = orc.propagate_instance(q)
    assert np.array_equal(rq.lb, r.lb[pc]) and np.array_equal(rq.ub, r.ub[pc])


def test_round_analysis_quiet_on_integer_rows(orc):
    """Integer coefficients and bounds: sums are exact, so no decision is a tie."""
    rng = np.random.default_rng(9)
    inst = synth.small_random(rng, 500, 300, maxlen=8, pure_integer=True, bounded=True)
    L, U, lhs, rhs = orc.normalise(inst.m, inst.n, inst.lb, inst.ub, inst.vartype, inst.lhs, inst.rhs)
    rr = orc.round_(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, L, U, inst.vartype, lhs, rhs,
                    analysis=True)
    assert rr.changed
    assert rr.lb_tie.sum() == 0 and rr.ub_tie.sum() == 0 and rr.inf_tie == 0


def test_rejects_nan(orc):
    inst = synth.tiny(m=20, n=15)
    inst.lb = inst.lb.copy()
    inst.lb[3] = np.nan
    with pytest.raises(ValueError):
        orc.propagate_instance(inst)


def _reorder_rows(row_ptr, col, val, rng, mode):
    """The same matrix with every row's nonzeros in another order (reversed
    or shuffled): the row sums of Eq. 2 are then taken in another order."""
    col2, val2 = col.copy(), val.copy()
    for i in range(len(row_ptr) - 1):
        b, e = int(row_ptr[i]), int(row_ptr[i + 1])
        perm = np.arange(b, e)[::-1] if mode == "reversed" else rng.permutation(np.arange(b, e))
        col2[b:e], val2[b:e] = col[perm], val[perm]
    return col2, val2


@pytest.mark.parametrize("mode", ["reversed", "shuffled"])
def test_reordering_error_bound_covers_other_summation_orders(orc, mode):
    """The round analysis bounds how far a bound may move when the row sums
    are taken in another order.  Summing every row in another order (the
    same arithmetic, only reassociated) must move each new bound by at most
    that bound, must leave integer bounds and acceptance decisions alone
    unless flagged as a tie (and few flagged decisions may actually flip),
    and the bound must not be vacuous: over the instance the largest
    observed move is within 10^3 of it."""
    rng = np.random.default_rng(2024 if mode == "reversed" else 2025)
    inst = synth.medium(seed=synth.seed_for(1, 17), scale=0.02)  # fractional coefficients
    L, U, lhs, rhs = orc.normalise(inst.m, inst.n, inst.lb, inst.ub, inst.vartype, inst.lhs,
                                   inst.rhs)
    ratio_max, checked, ties_used = 0.0, 0, 0
    for _ in range(4):  # the first rounds, from the oracle's own states
        a = orc.round_(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, L, U, inst.vartype,
                       lhs, rhs, analysis=True)
        c2, v2 = _reorder_rows(inst.row_ptr, inst.col, inst.val, rng, mode)
        b = orc.round_(inst.m, inst.n, inst.row_ptr, c2, v2, L, U, inst.vartype, lhs, rhs)
        for new_a, new_b, err, tie in ((a.lb, b.lb, a.lb_err, a.lb_tie), (a.ub, b.ub, a.ub_err,
                                                                            a.ub_tie)):
            tie = tie.astype(bool)
            isint = inst.vartype.astype(bool)
            with np.errstate(invalid="ignore"):
                d = np.abs(new_a - new_b)
            both_inf = np.isinf(new_a) & (new_a == new_b)
            within = both_inf | np.where(isint, d == 0.0, d <= err)
            # a move beyond the bound is a decision that went the other way,
            # which only a tie may do
            assert np.all(within | tie), "a bound moved beyond its error bound without a tie"
            ties_used += int((~within).sum())
            sel = ~isint & ~both_inf & (err > 0)
            checked += int(sel.sum())
            if sel.any():
                ratio_max = max(ratio_max, float((d[sel] / err[sel]).max()))
        assert b.infeasible == a.infeasible or a.inf_tie
        if not a.changed:
            break
        L, U = a.lb, a.ub
    assert checked > 100
    assert ties_used <= 5  # decisions that actually went the other way
    assert ratio_max >= 1e-3, f"the error bound is over 10^3 times the largest move ({ratio_max})"
