"""Problem sets (dp_matrix_load_set + dp_propagate_set): many distinct
matrices of uneven size in one device-side round loop.  Every problem must
end exactly where the oracle ends on that problem alone -- its own round
count, infeasibility flag and cap status, bounds bit-exact where no row is
split across threads (else within tests/parity.py's tolerance) -- and where
dp_propagate ends on that problem loaded alone."""
import numpy as np
import pytest
import torch

from paper_2009_07785_gb300 import synth
from parity import compare_bounds

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def problems(k=12, seed=41):
    """Uneven problems: tiny-like and medium-like of several sizes, some with
    node fixings (a few infeasible), one with long rows."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        kind = i % 3
        if kind == 0:
            m = int(rng.integers(50, 900))
            p = synth.tiny(seed=synth.seed_for(5, i), m=m, n=max(10, int(m * 0.75)))
        elif kind == 1:
            p = synth.medium(seed=synth.seed_for(5, i), scale=float(rng.uniform(0.002, 0.02)))
        else:
            p = synth.small_random(rng, int(rng.integers(100, 400)), int(rng.integers(80, 300)), 60)
        if i % 4 == 3:  # a branch-and-bound node of it
            LB, UB = synth.node_bounds(p, 1, seed=i, lo_frac=0.05, hi_frac=0.2)
            p.lb, p.ub = LB[0], UB[0]
        out.append(p)
    return out


def concat(ps, attr):
    return np.concatenate([getattr(p, attr) for p in ps])


def run_set(dp, ctx, ps, chunk=0, params=None, sides=False):
    with dp.MatrixSet(ctx, ps, chunk, sides=sides) as ms:
        assert ms.count == len(ps)
        r = dp.dp_propagate_set(ctx, ms, dev(concat(ps, "lb")), dev(concat(ps, "ub")),
                                dev(concat(ps, "vartype")), dev(concat(ps, "lhs")),
                                dev(concat(ps, "rhs")), params=params)
        lb, ub = r.lb.cpu().numpy(), r.ub.cpu().numpy()
        return ms.var_off.copy(), lb, ub, r


@pytest.mark.parametrize("chunk", [0, 16])
def test_set_matches_oracle_per_problem(gpu, orc, chunk):
    dp, ctx = gpu
    ps = problems()
    off, lb, ub, r = run_set(dp, ctx, ps, chunk)
    n_inf = 0
    for k, p in enumerate(ps):
        o = orc.propagate_instance(p)
        sl = slice(off[k], off[k + 1])
        assert r.infeasible[k] == o.infeasible, k
        assert r.rounds[k] == o.rounds, (k, r.rounds[k], o.rounds)
        assert r.cap_hit[k] == o.status, k
        nbad, _, det = compare_bounds(lb[sl], ub[sl], o.lb, o.ub, p.vartype)
        assert nbad == 0, f"problem {k}: {det}"
        if chunk == 0 and not (p.row_ptr[1:] - p.row_ptr[:-1] > 256).any():
            assert np.array_equal(lb[sl], o.lb) and np.array_equal(ub[sl], o.ub), k
        n_inf += o.infeasible
    assert n_inf > 0 and r.rounds.max() > 2 and len(set(r.rounds.tolist())) > 2


def test_set_equals_problems_alone(gpu):
    dp, ctx = gpu
    ps = problems(8, seed=43)
    off, lb, ub, r = run_set(dp, ctx, ps, chunk=16, sides=True)
    for k, p in enumerate(ps):
        with dp.Matrix(ctx, p.m, p.n, p.row_ptr, p.col, p.val, 16) as mat:
            a = dp.dp_propagate(ctx, mat, dev(p.lb), dev(p.ub), dev(p.vartype), dev(p.lhs),
                                dev(p.rhs))
        sl = slice(off[k], off[k + 1])
        assert a.rounds == r.rounds[k] and a.infeasible == r.infeasible[k]
        assert np.array_equal(a.lb.cpu().numpy(), lb[sl]) and np.array_equal(a.ub.cpu().numpy(), ub[sl])


def test_set_round_cap_and_zero_rounds(gpu, orc):
    dp, ctx = gpu
    ps = problems(6, seed=47)
    off, lb, ub, r = run_set(dp, ctx, ps, params=dp.dp_params_default(max_rounds=2))
    for k, p in enumerate(ps):
        o = orc.propagate_instance(p, {"max_rounds": 2})
        assert r.rounds[k] == o.rounds and r.cap_hit[k] == o.status
    assert r.cap_hit.any()
    off, lb, ub, r = run_set(dp, ctx, ps, params=dp.dp_params_default(max_rounds=0))
    assert (r.rounds == 0).all()
    for k, p in enumerate(ps):
        L, U, _, _ = orc.normalise(p.m, p.n, p.lb, p.ub, p.vartype, p.lhs, p.rhs)
        sl = slice(off[k], off[k + 1])
        assert np.array_equal(lb[sl], L) and np.array_equal(ub[sl], U)


def test_set_offsets_and_plain_matrix(gpu):
    dp, ctx = gpu
    ps = problems(3, seed=53)
    with dp.MatrixSet(ctx, ps) as ms:
        assert list(ms.row_off) == [0] + list(np.cumsum([p.m for p in ps]))
        assert list(ms.var_off) == [0] + list(np.cumsum([p.n for p in ps]))
    p = ps[0]
    with dp.Matrix(ctx, p.m, p.n, p.row_ptr, p.col, p.val) as mat:
        with pytest.raises(dp.DomPropError) as e:
            dp.dp_propagate_set(ctx, mat, dev(p.lb), dev(p.ub), dev(p.vartype), dev(p.lhs),
                                dev(p.rhs))
        assert e.value.code == dp.DP_ERR_INVALID_ARG
