"""Failure detection without faulting the GPU.

* The persistent round loop's grid barrier is a bounded wait: with the limit
  cut to one sleep the wait runs out, the call returns DP_ERR_TIMEOUT, every
  block leaves, and the same context then propagates correctly.
* Device allocations can be made to fail on the host (the k-th allocation
  from now on): loading a matrix and the first batched-node call (which
  allocates its workspace) return DP_ERR_OOM at every failure point, hold no
  device memory afterwards, and succeed once the failure point lies beyond
  their last allocation.
"""
import numpy as np
import pytest
import torch

from paper_2009_07785_gb300 import synth

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_persistent_wait_runs_out_and_context_survives(gpu, orc):
    dp, ctx = gpu
    inst = synth.tiny()
    d = [dev(a) for a in inst.problem()]
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        dp.dp_ctx_set_wait_limit(ctx, 1)
        try:
            with pytest.raises(dp.DomPropError) as e:
                dp.dp_propagate_persistent(ctx, mat, *d)
            assert e.value.code == dp.DP_ERR_TIMEOUT
        finally:
            dp.dp_ctx_set_wait_limit(ctx, 0)
        # the context, the matrix and the persistent loop work again
        r = dp.dp_propagate_persistent(ctx, mat, *d)
        o = orc.propagate_instance(inst)
        assert r.rounds == o.rounds and r.infeasible == o.infeasible
        assert np.array_equal(r.lb.cpu().numpy(), o.lb) and np.array_equal(r.ub.cpu().numpy(), o.ub)
        g = dp.dp_propagate(ctx, mat, *d)
        assert g.rounds == o.rounds


def test_wait_limit_rejects_negative(gpu):
    dp, ctx = gpu
    with pytest.raises(dp.DomPropError) as e:
        dp.dp_ctx_set_wait_limit(ctx, -1)
    assert e.value.code == dp.DP_ERR_INVALID_ARG


def _fail_at_every_point(dp, make, max_points=200):
    """Runs make() with the k-th allocation failing, k = 1, 2, ... until it
    succeeds; every failure must be DP_ERR_OOM and leave the library's live
    allocations where they were.  Returns (successful result, points)."""
    for k in range(1, max_points + 1):
        before = dp.dp_debug_live_allocs()
        dp.dp_debug_fail_alloc(k)
        try:
            out = make()
        except dp.DomPropError as e:
            assert e.code == dp.DP_ERR_OOM, (k, e.code)
            assert dp.dp_debug_live_allocs() == before, f"failure point {k} leaked"
            continue
        finally:
            dp.dp_debug_fail_alloc(0)
        return out, k
    raise AssertionError("never succeeded")


def test_matrix_load_allocation_failures(gpu, orc):
    dp, ctx = gpu
    inst = synth.medium(scale=0.01)  # has split rows: every allocation kind
    base = dp.dp_debug_live_allocs()
    mat, points = _fail_at_every_point(
        dp, lambda: dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val))
    assert points > 10
    try:
        r = dp.dp_propagate(ctx, mat, *[dev(a) for a in inst.problem()])
        o = orc.propagate_instance(inst)
        assert r.rounds == o.rounds and r.infeasible == o.infeasible
    finally:
        mat.close()
    assert dp.dp_debug_live_allocs() == base


def test_nodes_workspace_allocation_failures(gpu):
    dp, ctx = gpu
    inst = synth.tiny()
    LB, UB = synth.node_bounds(inst, 40, seed=5)
    args = [dev(LB), dev(UB), dev(inst.vartype), dev(inst.lhs), dev(inst.rhs)]
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as ref_mat:
        ref = dp.dp_propagate_nodes(ctx, ref_mat, *args)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        got, points = _fail_at_every_point(dp, lambda: dp.dp_propagate_nodes(ctx, mat, *args))
        assert points > 5
        assert np.array_equal(got.rounds, ref.rounds)
        assert np.array_equal(got.infeasible, ref.infeasible)
        assert torch.equal(got.lb, ref.lb) and torch.equal(got.ub, ref.ub)
