"""Batched branch-and-bound nodes (dp_propagate_nodes) vs the oracle, node by
node: every node of a batch must end exactly where the oracle ends when it
propagates that node alone (same infeasibility flag, same round count, same
cap status; bounds bit-exact where no row is split across threads, else
within the tolerance of tests/parity.py).  Also: a node's result does not
depend on the other nodes of its batch."""
import numpy as np
import pytest
import torch

from paper_2009_07785_gb300 import synth
from parity import compare_bounds

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_nodes(dp, ctx, mat, inst, LB, UB, params=None, on_host=False):
    args = [LB, UB, inst.vartype, inst.lhs, inst.rhs]
    if not on_host:
        args = [dev(a) for a in args]
    r = dp.dp_propagate_nodes(ctx, mat, *args, params=params)
    lb = r.lb.cpu().numpy() if isinstance(r.lb, torch.Tensor) else r.lb
    ub = r.ub.cpu().numpy() if isinstance(r.ub, torch.Tensor) else r.ub
    return lb, ub, r


def check_nodes(dp, ctx, mat, inst, orc, LB, UB, params=None, exact=True, on_host=False):
    p = dp.dp_params_default(**params) if params else None
    lb, ub, r = run_nodes(dp, ctx, mat, inst, LB, UB, p, on_host)
    assert lb.shape == LB.shape
    n_inf = 0
    for k in range(LB.shape[0]):
        o = orc.propagate(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, LB[k], UB[k],
                          inst.vartype, inst.lhs, inst.rhs, params)
        assert r.infeasible[k] == o.infeasible, f"node {k}"
        assert r.rounds[k] == o.rounds, f"node {k}: rounds {r.rounds[k]} vs {o.rounds}"
        assert r.cap_hit[k] == o.status, f"node {k}"
        if exact:
            assert np.array_equal(lb[k], o.lb) and np.array_equal(ub[k], o.ub), f"node {k}"
        else:
            nbad, _, det = compare_bounds(lb[k], ub[k], o.lb, o.ub, inst.vartype)
            assert nbad == 0, f"node {k}: {det}"
        n_inf += o.infeasible
    assert (r.status == dp.DP_CAP_HIT) == bool(r.cap_hit.any())
    return r, n_inf


def test_nodes_tiny_bit_exact(gpu, orc):
    """40 nodes (a padded second node group); some fixings are infeasible."""
    dp, ctx = gpu
    inst = synth.tiny()
    LB, UB = synth.node_bounds(inst, 40, seed=synth.seed_for(3, 1))
    LB2, UB2 = synth.node_bounds(inst, 8, seed=synth.seed_for(3, 2), lo_frac=0.05, hi_frac=0.2)
    LB, UB = np.vstack([LB, LB2]), np.vstack([UB, UB2])
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        assert mat.info()["split_rows"] == 0
        r, n_inf = check_nodes(dp, ctx, mat, inst, orc, LB, UB)
        assert n_inf > 0 and (r.infeasible == 0).sum() > 0
        assert r.rounds.max() > 2


def test_nodes_root_equals_single_instance(gpu, orc):
    """The unbranched root as a batch of one node is dp_propagate."""
    dp, ctx = gpu
    inst = synth.tiny()
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        r1 = dp.dp_propagate(ctx, mat, dev(inst.lb), dev(inst.ub), dev(inst.vartype),
                             dev(inst.lhs), dev(inst.rhs))
        lb, ub, rn = run_nodes(dp, ctx, mat, inst, inst.lb[None, :], inst.ub[None, :])
        assert rn.rounds[0] == r1.rounds and rn.infeasible[0] == r1.infeasible
        assert np.array_equal(lb[0], r1.lb.cpu().numpy())
        assert np.array_equal(ub[0], r1.ub.cpu().numpy())


def test_nodes_host_pointers(gpu, orc):
    dp, ctx = gpu
    inst = synth.tiny(m=500, n=400)
    LB, UB = synth.node_bounds(inst, 33, seed=5)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        check_nodes(dp, ctx, mat, inst, orc, LB, UB, on_host=True)


@pytest.mark.parametrize("chunk", [8, 16])
def test_nodes_split_rows(gpu, orc, chunk):
    """Rows longer than `chunk` are split into pieces whose partial
    activities are combined in piece order."""
    dp, ctx = gpu
    rng = np.random.default_rng(5)
    big = synth.small_random(rng, 300, 400, 60)
    LB, UB = synth.node_bounds(big, 36, seed=6)
    with dp.Matrix(ctx, big.m, big.n, big.row_ptr, big.col, big.val, chunk) as mat:
        assert mat.info()["split_rows"] > 0
        check_nodes(dp, ctx, mat, big, orc, LB, UB, exact=False)


def test_nodes_medium_scaled(gpu, orc):
    """Config-1-like matrix (knapsack rows split, set partitioning rows)."""
    dp, ctx = gpu
    inst = synth.medium(scale=0.1)
    LB, UB = synth.node_bounds(inst, 64, seed=synth.seed_for(3, 3))
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        assert mat.info()["split_rows"] > 0
        check_nodes(dp, ctx, mat, inst, orc, LB, UB, exact=False)


def test_nodes_independent_of_batch(gpu):
    """A node's result is the same alone, in a batch of 70, and in a batch
    larger than one launch (1100 nodes: two launches)."""
    dp, ctx = gpu
    inst = synth.tiny(m=300, n=200)
    LB, UB = synth.node_bounds(inst, 1100, seed=9)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        lb, ub, r = run_nodes(dp, ctx, mat, inst, LB, UB)
        lb70, ub70, r70 = run_nodes(dp, ctx, mat, inst, LB[1000:1070], UB[1000:1070])
        assert np.array_equal(lb70, lb[1000:1070]) and np.array_equal(ub70, ub[1000:1070])
        assert np.array_equal(r70.rounds, r.rounds[1000:1070])
        for k in (0, 31, 32, 1023, 1024, 1099):
            r1 = dp.dp_propagate(ctx, mat, dev(LB[k]), dev(UB[k]), dev(inst.vartype),
                                 dev(inst.lhs), dev(inst.rhs))
            assert r1.rounds == r.rounds[k] and r1.infeasible == r.infeasible[k]
            assert np.array_equal(r1.lb.cpu().numpy(), lb[k])
            assert np.array_equal(r1.ub.cpu().numpy(), ub[k])


def test_nodes_round_cap_and_zero_rounds(gpu, orc):
    dp, ctx = gpu
    inst = synth.tiny(m=600, n=500)
    LB, UB = synth.node_bounds(inst, 32, seed=12)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        r, _ = check_nodes(dp, ctx, mat, inst, orc, LB, UB, params={"max_rounds": 2})
        assert r.cap_hit.any()
        lb, ub, r0 = run_nodes(dp, ctx, mat, inst, LB, UB, dp.dp_params_default(max_rounds=0))
        assert (r0.rounds == 0).all() and (r0.infeasible == 0).all()
        for k in range(LB.shape[0]):
            L, U, _, _ = orc.normalise(inst.m, inst.n, LB[k], UB[k], inst.vartype, inst.lhs,
                                       inst.rhs)
            assert np.array_equal(lb[k], L) and np.array_equal(ub[k], U)


def test_nodes_crossing_input_and_empty_rows(gpu, orc):
    """Nodes whose input bounds already cross, and rows without nonzeros
    (infeasible when 0 is outside [lhs, rhs])."""
    dp, ctx = gpu
    rng = np.random.default_rng(17)
    inst = synth.small_random(rng, 200, 150, maxlen=6)
    LB, UB = synth.node_bounds(inst, 40, seed=4)
    ints = np.flatnonzero(inst.vartype == 1)
    LB[3, ints[0]] = UB[3, ints[0]] + 1.0
    conts = np.flatnonzero((inst.vartype == 0) & np.isfinite(inst.ub))
    LB[35, conts[0]] = UB[35, conts[0]] + 0.5
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        r, _ = check_nodes(dp, ctx, mat, inst, orc, LB, UB)
        assert r.infeasible[3] == 1 and r.infeasible[35] == 1
    # two empty rows, one of them infeasible (0 > rhs)
    rp = np.concatenate([inst.row_ptr, [inst.row_ptr[-1]] * 2]).astype(np.int64)
    e = synth.Instance("empty_rows", inst.m + 2, inst.n, rp, inst.col, inst.val, inst.lb, inst.ub,
                       inst.vartype, np.concatenate([inst.lhs, [-np.inf, -np.inf]]),
                       np.concatenate([inst.rhs, [1.0, -1.0]]), inst.xstar)
    with dp.Matrix(ctx, e.m, e.n, e.row_ptr, e.col, e.val) as mat:
        r, n_inf = check_nodes(dp, ctx, mat, e, orc, LB[:5], UB[:5])
        assert n_inf == 5


def test_nodes_nan_rejected_and_context_survives(gpu):
    dp, ctx = gpu
    inst = synth.tiny(m=100, n=80)
    LB, UB = synth.node_bounds(inst, 40, seed=2)
    LB[37, 5] = np.nan
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        with pytest.raises(dp.DomPropError) as ei:
            run_nodes(dp, ctx, mat, inst, LB, UB)
        assert ei.value.code == dp.DP_ERR_NAN_INPUT
        LB[37, 5] = 0.0
        _, _, r = run_nodes(dp, ctx, mat, inst, LB, UB)
        assert r.rounds.min() >= 1


def test_nodes_no_rows(gpu):
    dp, ctx = gpu
    n = 50
    lb, ub = np.zeros((33, n)), np.ones((33, n))
    with dp.Matrix(ctx, 0, n, np.zeros(1, np.int64), np.zeros(0, np.int32),
                   np.zeros(0)) as mat:
        r = dp.dp_propagate_nodes(ctx, mat, dev(lb), dev(ub), dev(np.zeros(n, np.uint8)),
                                  dev(np.zeros(0)), dev(np.zeros(0)))
        assert (r.rounds == 1).all() and (r.infeasible == 0).all()
        assert np.array_equal(r.lb.cpu().numpy(), lb)


def test_nodes_hostloop_matches_graph_loop(gpu):
    dp, ctx = gpu
    rng = np.random.default_rng(8)
    big = synth.small_random(rng, 300, 400, 60)
    LB, UB = synth.node_bounds(big, 40, seed=8)
    with dp.Matrix(ctx, big.m, big.n, big.row_ptr, big.col, big.val, 16) as mat:
        lb, ub, r = run_nodes(dp, ctx, mat, big, LB, UB)
        h = dp.dp_propagate_nodes_hostloop(ctx, mat, dev(LB), dev(UB), dev(big.vartype),
                                           dev(big.lhs), dev(big.rhs))
        assert np.array_equal(h.lb.cpu().numpy(), lb) and np.array_equal(h.ub.cpu().numpy(), ub)
        assert np.array_equal(h.rounds, r.rounds) and np.array_equal(h.infeasible, r.infeasible)
        assert h.kernel_launches[0] == r.rounds.max() and all(t >= 0 for t in h.kernel_ms)


def test_autotune_nodes_picks_a_measured_layout(gpu, orc):
    """The batched-node autotuner times every distinct split length from 32
    up and returns the fastest; nodes on its layout still match the oracle."""
    dp, ctx = gpu
    inst = synth.medium(scale=0.02)
    LB, UB = synth.node_bounds_at_point(inst, 8, seed=4)
    t = dp.dp_autotune_nodes(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val, LB, UB,
                             inst.vartype, inst.lhs, inst.rhs)
    chunks = [e["chunk"] for e in t["entries"]]
    us = [e["us_per_round"] for e in t["entries"]]
    assert chunks[0] == 32 and chunks == sorted(set(chunks)) and len(chunks) >= 3
    assert min(us) > 0 and t["best"]["us_per_round"] == min(us)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val,
                   t["best"]["chunk"]) as mat:
        lb, ub, r = run_nodes(dp, ctx, mat, inst, LB, UB)
    for k in range(LB.shape[0]):
        o = orc.propagate(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, LB[k], UB[k],
                          inst.vartype, inst.lhs, inst.rhs)
        assert r.rounds[k] == o.rounds and r.infeasible[k] == o.infeasible, k
        nbad, _, det = compare_bounds(lb[k], ub[k], o.lb, o.ub, inst.vartype)
        assert nbad == 0, det
