"""The batched round loops as one persistent cooperative kernel
(dp_propagate_nodes_persistent, dp_propagate_set_persistent; Sec. 3.7's
single-kernel loop).  Each must end exactly where the graph-driven call
ends -- bounds bit for bit, round counts, infeasibility and cap flags --
and therefore where the oracle ends on each node or problem alone; its
grid barrier's bounded wait must run out cleanly when cut to one sleep.
"""
import numpy as np
import pytest
import torch

from paper_2009_07785_gb300 import synth
from parity import compare_bounds
from test_gpu_sets import concat, problems

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def node_args(inst, LB, UB):
    return [dev(LB), dev(UB), dev(inst.vartype), dev(inst.lhs), dev(inst.rhs)]


def same_nodes(a, b):
    assert np.array_equal(a.rounds, b.rounds)
    assert np.array_equal(a.infeasible, b.infeasible)
    assert np.array_equal(a.cap_hit, b.cap_hit)
    assert a.status == b.status
    assert torch.equal(a.lb, b.lb) and torch.equal(a.ub, b.ub)


@pytest.mark.parametrize("case", ["tiny", "medium_split", "medium_chunk16"])
def test_nodes_persistent_equals_graph_and_oracle(gpu, orc, case):
    dp, ctx = gpu
    if case == "tiny":
        inst, chunk, count = synth.tiny(), 0, 72
    else:
        inst = synth.medium(scale=0.01)
        chunk, count = (0, 40) if case == "medium_split" else (16, 40)
    LB, UB = synth.node_bounds(inst, count, seed=synth.seed_for(3, 7))
    LB2, UB2 = synth.node_bounds_at_point(inst, count, seed=synth.seed_for(3, 8))
    LB, UB = np.vstack([LB, LB2]), np.vstack([UB, UB2])
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val, chunk,
                   lhs=inst.lhs, rhs=inst.rhs) as mat:
        if case != "tiny":
            assert mat.info()["split_rows"] > 0
        args = node_args(inst, LB, UB)
        g = dp.dp_propagate_nodes(ctx, mat, *args)
        p = dp.dp_propagate_nodes_persistent(ctx, mat, *args)
        same_nodes(g, p)
        p2 = dp.dp_propagate_nodes_persistent(ctx, mat, *args)  # a second call, same state
        same_nodes(g, p2)
    lb, ub = p.lb.cpu().numpy(), p.ub.cpu().numpy()
    exact = case == "tiny"
    for k in range(0, LB.shape[0], 7):
        o = orc.propagate(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, LB[k], UB[k],
                          inst.vartype, inst.lhs, inst.rhs)
        assert p.rounds[k] == o.rounds and p.infeasible[k] == o.infeasible, f"node {k}"
        if exact:
            assert np.array_equal(lb[k], o.lb) and np.array_equal(ub[k], o.ub), f"node {k}"
        else:
            nbad, _, det = compare_bounds(lb[k], ub[k], o.lb, o.ub, inst.vartype)
            assert nbad == 0, f"node {k}: {det}"
    assert p.infeasible.any() and (p.rounds > 3).any()


@pytest.mark.parametrize("max_rounds", [0, 1, 3])
def test_nodes_persistent_round_cap(gpu, max_rounds):
    dp, ctx = gpu
    inst = synth.tiny()
    LB, UB = synth.node_bounds_at_point(inst, 33, seed=synth.seed_for(3, 9))
    prm = dp.dp_params_default(max_rounds=max_rounds)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        args = node_args(inst, LB, UB)
        g = dp.dp_propagate_nodes(ctx, mat, *args, params=prm)
        p = dp.dp_propagate_nodes_persistent(ctx, mat, *args, params=prm)
        same_nodes(g, p)
    assert int(p.rounds.max()) <= max_rounds


@pytest.mark.parametrize("chunk", [0, 16])
def test_set_persistent_equals_graph_and_oracle(gpu, orc, chunk):
    dp, ctx = gpu
    ps = problems()
    arrays = [dev(concat(ps, a)) for a in ("lb", "ub", "vartype", "lhs", "rhs")]
    with dp.MatrixSet(ctx, ps, chunk) as ms:
        g = dp.dp_propagate_set(ctx, ms, *arrays)
        p = dp.dp_propagate_set_persistent(ctx, ms, *arrays)
        off = ms.var_off.copy()
    assert np.array_equal(g.rounds, p.rounds) and np.array_equal(g.infeasible, p.infeasible)
    assert np.array_equal(g.cap_hit, p.cap_hit)
    assert torch.equal(g.lb, p.lb) and torch.equal(g.ub, p.ub)
    lb, ub = p.lb.cpu().numpy(), p.ub.cpu().numpy()
    for k, q in enumerate(ps):
        o = orc.propagate_instance(q)
        assert p.rounds[k] == o.rounds and p.infeasible[k] == o.infeasible, f"problem {k}"
        s = slice(off[k], off[k + 1])
        nbad, _, det = compare_bounds(lb[s], ub[s], o.lb, o.ub, q.vartype)
        assert nbad == 0, f"problem {k}: {det}"


def test_nodes_persistent_wait_runs_out_and_context_survives(gpu):
    dp, ctx = gpu
    inst = synth.tiny()
    LB, UB = synth.node_bounds_at_point(inst, 40, seed=synth.seed_for(3, 10))
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        args = node_args(inst, LB, UB)
        ref = dp.dp_propagate_nodes(ctx, mat, *args)
        dp.dp_ctx_set_wait_limit(ctx, 1)
        try:
            with pytest.raises(dp.DomPropError) as e:
                dp.dp_propagate_nodes_persistent(ctx, mat, *args)
            assert e.value.code == dp.DP_ERR_TIMEOUT
        finally:
            dp.dp_ctx_set_wait_limit(ctx, 0)
        same_nodes(ref, dp.dp_propagate_nodes_persistent(ctx, mat, *args))
        same_nodes(ref, dp.dp_propagate_nodes(ctx, mat, *args))


def test_set_persistent_wait_runs_out_and_context_survives(gpu):
    dp, ctx = gpu
    ps = problems(k=6)
    arrays = [dev(concat(ps, a)) for a in ("lb", "ub", "vartype", "lhs", "rhs")]
    with dp.MatrixSet(ctx, ps, 0) as ms:
        ref = dp.dp_propagate_set(ctx, ms, *arrays)
        dp.dp_ctx_set_wait_limit(ctx, 1)
        try:
            with pytest.raises(dp.DomPropError) as e:
                dp.dp_propagate_set_persistent(ctx, ms, *arrays)
            assert e.value.code == dp.DP_ERR_TIMEOUT
        finally:
            dp.dp_ctx_set_wait_limit(ctx, 0)
        p = dp.dp_propagate_set_persistent(ctx, ms, *arrays)
        assert np.array_equal(ref.rounds, p.rounds)
        assert torch.equal(ref.lb, p.lb) and torch.equal(ref.ub, p.ub)


def test_nodes_persistent_two_launches(gpu):
    """1100 nodes: more than one launch's 1024, run as two persistent launches."""
    dp, ctx = gpu
    inst = synth.tiny()
    LB, UB = synth.node_bounds(inst, 1100, seed=9)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        args = node_args(inst, LB, UB)
        same_nodes(dp.dp_propagate_nodes(ctx, mat, *args),
                   dp.dp_propagate_nodes_persistent(ctx, mat, *args))


def test_nodes_persistent_edges(gpu):
    """Crossing input bounds, empty rows (one infeasible), a matrix without
    rows, and a NaN input: the persistent loop ends where the graph ends."""
    dp, ctx = gpu
    rng = np.random.default_rng(17)
    inst = synth.small_random(rng, 200, 150, maxlen=6)
    LB, UB = synth.node_bounds(inst, 40, seed=4)
    ints = np.flatnonzero(inst.vartype == 1)
    LB[3, ints[0]] = UB[3, ints[0]] + 1.0
    rp = np.concatenate([inst.row_ptr, [inst.row_ptr[-1]] * 2]).astype(np.int64)
    e = synth.Instance("empty_rows", inst.m + 2, inst.n, rp, inst.col, inst.val, inst.lb, inst.ub,
                       inst.vartype, np.concatenate([inst.lhs, [-np.inf, -np.inf]]),
                       np.concatenate([inst.rhs, [1.0, -1.0]]), inst.xstar)
    for q in (inst, e):
        with dp.Matrix(ctx, q.m, q.n, q.row_ptr, q.col, q.val) as mat:
            args = node_args(q, LB, UB)
            g = dp.dp_propagate_nodes(ctx, mat, *args)
            p = dp.dp_propagate_nodes_persistent(ctx, mat, *args)
            same_nodes(g, p)
            assert p.infeasible[3] == 1
    n = 50
    lb, ub = np.zeros((33, n)), np.ones((33, n))
    with dp.Matrix(ctx, 0, n, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0)) as mat:
        args = [dev(lb), dev(ub), dev(np.zeros(n, np.uint8)), dev(np.zeros(0)), dev(np.zeros(0))]
        same_nodes(dp.dp_propagate_nodes(ctx, mat, *args),
                   dp.dp_propagate_nodes_persistent(ctx, mat, *args))
    t = synth.tiny(m=100, n=80)
    LB, UB = synth.node_bounds(t, 40, seed=2)
    LB[37, 5] = np.nan
    with dp.Matrix(ctx, t.m, t.n, t.row_ptr, t.col, t.val) as mat:
        with pytest.raises(dp.DomPropError) as ei:
            dp.dp_propagate_nodes_persistent(ctx, mat, *node_args(t, LB, UB))
        assert ei.value.code == dp.DP_ERR_NAN_INPUT
        LB[37, 5] = 0.0
        args = node_args(t, LB, UB)
        same_nodes(dp.dp_propagate_nodes(ctx, mat, *args),
                   dp.dp_propagate_nodes_persistent(ctx, mat, *args))
