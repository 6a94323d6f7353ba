"""The binary32 screen at its margins.

The round kernels skip the binary64 candidate work of a nonzero when a
binary32 test proves that its candidate cannot be applied.  The test is
sound only if its margins cover every rounding of the binary64 formulas.
Here each row's exact candidate lands within a few ulps of its acceptance
threshold (Sec. 1.1 last paragraph: the improvement threshold; Step 3:
integer rounding), on both sides of it, with bound magnitudes from 1 to
1e18, widths of 0 and 1e-12, coefficients from 2^-119 to 2^119 and
one- and two-nonzero rows, so that a margin too tight would prune a
candidate the oracle applies.  Every row fits one chunk, so the GPU must
agree with the oracle bit for bit.
"""
import numpy as np
import pytest
import torch

from paper_2009_07785_gb300 import synth
from test_gpu_parity import dev

pytestmark = pytest.mark.gpu

TAU = 1e-6
EPS_INT = 1e-6


def _nudge(x, k):
    """x moved by k ulps (k may be negative)."""
    for _ in range(abs(k)):
        x = np.nextafter(x, np.inf if k > 0 else -np.inf)
    return x


def margin_instance(seed, narrow=False):
    """Rows a*x (+ b*y) <= rhs (or lhs <= a*x + b*y) whose candidate for x
    lies within 4 ulps of the threshold it is compared with.  With `narrow`
    a fifth of the variables have width 0 or 1e-12 relative, so that applied
    candidates also meet the crossing test at its margin (the feasibility
    tolerance equals the improvement threshold)."""
    rng = np.random.default_rng(seed)
    rows = []  # (cols, vals, lhs, rhs)
    lb, ub, vt = [], [], []

    def var(lo, hi, is_int):
        lb.append(lo)
        ub.append(hi)
        vt.append(1 if is_int else 0)
        return len(lb) - 1

    exps = [-119, -90, -40, -1, 0, 1, 7, 40, 90, 119]
    mags = [1.0, 37.5, 1e6, 1e12, 1e15, 1e18]
    for k in range(-4, 5):
        for e in exps:
            for M in mags:
                a = float(np.ldexp(1.0 + rng.random(), e)) * (1 if rng.random() < 0.5 else -1)
                is_int = rng.random() < 0.25 and M <= 1e15
                two = rng.random() < 0.5
                if is_int:
                    L = -float(np.floor(M * rng.random()))
                    U = L + float(rng.integers(1, 1000))
                else:
                    L = -M * rng.random()
                    U = L + M * (0.5 + rng.random())
                if narrow and rng.random() < 0.1 and not is_int:
                    U = L  # width 0: a fixed variable
                elif narrow and rng.random() < 0.1 and not is_int:
                    U = L + 1e-12 * max(1.0, abs(L))
                j = var(L, U, is_int)
                # the threshold the candidate meets: an upper candidate for
                # x (a > 0 from the right-hand side, a < 0 from the left)
                # against U - tau*max(1,|U|), a lower one against L +
                # tau*max(1,|L|); integer candidates after rounding
                use_rhs = rng.random() < 0.7
                upper = (a > 0) == use_rhs
                if is_int:  # floor(c + eps) < U  iff  c < U - eps
                    T = U - EPS_INT if upper else L + EPS_INT
                else:
                    T = U - TAU * max(1.0, abs(U)) if upper else L + TAU * max(1.0, abs(L))
                T = _nudge(T, k)
                cols, vals, res = [j], [a], 0.0
                if two and a * T != 0.0:
                    # the other term is of the order of a*T, so that the side
                    # a*T + res keeps the candidate within a few ulps of T
                    b = abs(a * T) * float(rng.uniform(0.05, 0.2))
                    yl = float(np.round(rng.uniform(-5, 5), 3))
                    y = var(yl, yl + 10.0, False)
                    cols.append(y)
                    vals.append(b)
                    # residual of x: the other term at the bound the side uses
                    res = b * (yl if use_rhs else yl + 10.0)
                side = a * T + res
                if not np.isfinite(side) or abs(side) >= 1e20:
                    continue
                rows.append((cols, vals, side if not use_rhs else -np.inf,
                             side if use_rhs else np.inf))
    order = rng.permutation(len(rows))
    rp, col, val, lhs, rhs = [0], [], [], [], []
    for i in order:
        c, v, l, r = rows[i]
        col += c
        val += v
        rp.append(len(col))
        lhs.append(l)
        rhs.append(r)
    n = len(lb)
    lb, ub = np.array(lb), np.array(ub)
    return synth.Instance("screen-margins", len(rp) - 1, n, np.array(rp, np.int64),
                          np.array(col, np.int32), np.array(val, np.float64), lb, ub,
                          np.array(vt, np.uint8), np.array(lhs), np.array(rhs), np.zeros(n))


@pytest.mark.parametrize("narrow", [False, True])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_screen_margins_bit_exact(gpu, orc, seed, narrow):
    dp, ctx = gpu
    inst = margin_instance(seed, narrow)
    L0, U0, lhs0, rhs0 = orc.normalise(inst.m, inst.n, inst.lb, inst.ub, inst.vartype, inst.lhs,
                                       inst.rhs)
    o1 = orc.round_(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, L0, U0, inst.vartype,
                    lhs0, rhs0)
    applied = int((o1.lb != L0).sum() + (o1.ub != U0).sum())
    # both outcomes occur at the margin: some candidates applied, many not
    assert applied > 20 and applied < inst.n, applied
    d = [dev(a) for a in inst.problem()]
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        assert mat.info()["split_rows"] == 0
        r1 = dp.dp_propagate(ctx, mat, *d, params=dp.dp_params_default(max_rounds=1))
        assert np.array_equal(r1.lb.cpu().numpy(), o1.lb)
        assert np.array_equal(r1.ub.cpu().numpy(), o1.ub)
        assert r1.infeasible == o1.infeasible
        r = dp.dp_propagate(ctx, mat, *d)
        o = orc.propagate_instance(inst)
        assert r.rounds == o.rounds and r.infeasible == o.infeasible
        assert np.array_equal(r.lb.cpu().numpy(), o.lb) and np.array_equal(r.ub.cpu().numpy(), o.ub)
    if not narrow:
        assert not o1.infeasible  # wide bounds never cross
    print(f"seed {seed}: {inst.m} rows at the acceptance margin, {applied} candidates applied")
