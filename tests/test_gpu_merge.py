"""Merge-path layout (dp_matrix_load_merge): the same propagation with the
activity pass balanced over equal segments of the merged row-end/nonzero
sequence.  Rows inside one segment are summed in CSR order (bit-exact with
the oracle); rows split across segments within the tolerance of
tests/parity.py.  Round counts and infeasibility agree with the oracle
either way."""
import numpy as np
import pytest
import torch

from paper_2009_07785_gb300 import synth
from test_gpu_parity import check_full, dev, gpu_full, replay

pytestmark = pytest.mark.gpu


def merge_matrix(dp, ctx, inst, ipt, sides=False):
    kw = {"lhs": inst.lhs, "rhs": inst.rhs} if sides else {}
    return dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val, merge_ipt=ipt, **kw)


def test_single_segment_bit_exact(gpu, orc):
    """Fewer than ipt items: one segment, no split row, the oracle's sums."""
    dp, ctx = gpu
    inst = synth.tiny(m=300, n=250)
    assert inst.m + inst.nnz <= 4096
    with merge_matrix(dp, ctx, inst, 4096) as mat:
        assert mat.info()["split_rows"] == 0
        check_full(dp, ctx, mat, inst, orc, exact=True)
        rounds, ties = replay(dp, ctx, mat, inst, orc)
        assert rounds > 2 and ties == 0


@pytest.mark.parametrize("ipt", [4, 7, 16, 64, 512])
def test_tiny_split_rows(gpu, orc, ipt):
    """Small segments split most rows into two or more pieces (the one-lane
    combination) and long rows into many (the warp combination)."""
    dp, ctx = gpu
    inst = synth.tiny(seed=synth.seed_for(0, 3), m=1500, n=1100)
    with merge_matrix(dp, ctx, inst, ipt) as mat:
        assert mat.info()["split_rows"] > 0
        replay(dp, ctx, mat, inst, orc)
        check_full(dp, ctx, mat, inst, orc, exact=False)
    rng = np.random.default_rng(ipt)
    big = synth.small_random(rng, 300, 400, 120)  # empty rows and rows of 100+
    with merge_matrix(dp, ctx, big, ipt, sides=True) as mat:
        replay(dp, ctx, mat, big, orc)
        check_full(dp, ctx, mat, big, orc, exact=False)


def test_medium_and_large_scaled(gpu, orc):
    dp, ctx = gpu
    for inst in (synth.medium(scale=0.05), synth.large(scale=0.02)):
        with merge_matrix(dp, ctx, inst, 32, sides=True) as mat:
            assert mat.info()["split_rows"] > 0
            replay(dp, ctx, mat, inst, orc)
            check_full(dp, ctx, mat, inst, orc, exact=False)


def test_equals_sliced_layout(gpu):
    """Same rounds and infeasibility as the sliced layout; bounds bit-identical
    where neither layout splits a row."""
    dp, ctx = gpu
    inst = synth.tiny(m=300, n=250)
    args = [dev(a) for a in inst.problem()]
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as a, \
            merge_matrix(dp, ctx, inst, 4096, sides=True) as b:
        ra = dp.dp_propagate(ctx, a, *args)
        rb = dp.dp_propagate(ctx, b, *args)
        assert ra.rounds == rb.rounds and ra.infeasible == rb.infeasible
        assert torch.equal(ra.lb, rb.lb) and torch.equal(ra.ub, rb.ub)


def test_node_fixings_caps_and_crossing_inputs(gpu, orc):
    """Branch-and-bound node bounds (some infeasible), the round cap, zero
    rounds, and input bounds that already cross."""
    dp, ctx = gpu
    inst = synth.tiny(seed=synth.seed_for(0, 5), m=1200, n=900)
    LB, UB = synth.node_bounds(inst, 6, seed=2, lo_frac=0.05, hi_frac=0.2)
    with merge_matrix(dp, ctx, inst, 16) as mat:
        infeasible = 0
        for k in range(LB.shape[0]):
            g_lb, g_ub, r = gpu_full(dp, ctx, mat, inst, lb=LB[k], ub=UB[k])
            o = orc.propagate(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, LB[k], UB[k],
                              inst.vartype, inst.lhs, inst.rhs)
            assert r.rounds == o.rounds and r.infeasible == o.infeasible, k
            infeasible += o.infeasible
        assert infeasible > 0
        check_full(dp, ctx, mat, inst, orc, params={"max_rounds": 2}, exact=False)
        lb0, ub0, r = gpu_full(dp, ctx, mat, inst, dp.dp_params_default(max_rounds=0))
        L, U, _, _ = orc.normalise(inst.m, inst.n, inst.lb, inst.ub, inst.vartype, inst.lhs,
                                   inst.rhs)
        assert r.rounds == 0 and np.array_equal(lb0, L) and np.array_equal(ub0, U)
        lb = inst.lb.copy()
        ub = inst.ub.copy()
        j = int(np.flatnonzero(inst.vartype == 0)[0])
        lb[j], ub[j] = 5.0, 4.0  # crossing on input: found by round 1
        _, _, r = gpu_full(dp, ctx, mat, inst, lb=lb, ub=ub)
        o = orc.propagate(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, lb, ub,
                          inst.vartype, inst.lhs, inst.rhs)
        assert r.infeasible == 1 == o.infeasible and r.rounds == o.rounds


def test_launch_shapes_and_hostloop(gpu, orc):
    dp, ctx = gpu
    inst = synth.medium(scale=0.02)
    args = [dev(a) for a in inst.problem()]
    with merge_matrix(dp, ctx, inst, 64, sides=True) as mat:
        ref = dp.dp_propagate(ctx, mat, *args)
        mat.set_launch(4)
        r4 = dp.dp_propagate(ctx, mat, *args)
        h = dp.dp_propagate_hostloop(ctx, mat, *args)
        for r in (r4, h):
            assert r.rounds == ref.rounds and r.infeasible == ref.infeasible
            assert torch.equal(r.lb, ref.lb) and torch.equal(r.ub, ref.ub)
        o = orc.propagate_instance(inst)
        assert ref.rounds == o.rounds


def test_entry_points_that_need_the_sliced_layout(gpu):
    dp, ctx = gpu
    inst = synth.tiny(m=200, n=150)
    with merge_matrix(dp, ctx, inst, 16) as mat:
        args = [dev(a) for a in inst.problem()]
        for call in (lambda: dp.dp_propagate_persistent(ctx, mat, *args),
                     lambda: dp.dp_propagate_nodes(ctx, mat, dev(inst.lb[None]),
                                                   dev(inst.ub[None]), *args[2:])):
            with pytest.raises(dp.DomPropError) as e:
                call()
            assert e.value.code == dp.DP_ERR_INVALID_ARG
        with dp.Server(ctx, slots=32) as srv:
            with pytest.raises(dp.DomPropError) as e:
                srv.add_matrix(mat, inst.vartype, inst.lhs, inst.rhs)
            assert e.value.code == dp.DP_ERR_INVALID_ARG
    for ipt in (3, 4097):
        with pytest.raises(dp.DomPropError) as e:
            merge_matrix(dp, ctx, inst, ipt)
        assert e.value.code == dp.DP_ERR_INVALID_ARG
