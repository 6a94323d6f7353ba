"""GPU path vs the CPU oracle through the C ABI, element by element.

Two comparison modes:
  * replay: every GPU round r starts from the GPU's own state after round
    r-1 (dp_propagate with max_rounds=1) and is compared with the oracle's
    round from that same state, so differences cannot accumulate;
  * full run: both sides propagate to the fixed point independently; bounds,
    round count and the infeasibility flag must agree.
Tolerances are those of tests/parity.py.
"""
import numpy as np
import pytest
import torch

from paper_2009_07785_gb300 import synth
from parity import compare_bounds

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy() if isinstance(t, torch.Tensor) else t


def gpu_full(dp, ctx, mat, inst, params=None, lb=None, ub=None, on_host=False):
    args = [inst.lb if lb is None else lb, inst.ub if ub is None else ub, inst.vartype, inst.lhs,
            inst.rhs]
    if not on_host:
        args = [dev(a) for a in args]
    r = dp.dp_propagate(ctx, mat, *args, params=params)
    return host(r.lb), host(r.ub), r


def replay(dp, ctx, mat, inst, orc, max_rounds=100, params=None):
    """Round-by-round comparison; returns (rounds, ties)."""
    q = dict(params or {})
    L, U, lhs, rhs = orc.normalise(inst.m, inst.n, inst.lb, inst.ub, inst.vartype, inst.lhs,
                                   inst.rhs, q)
    p1 = dp.dp_params_default(max_rounds=1, **{k: v for k, v in q.items() if k != "max_rounds"})
    d_vt, d_lhs, d_rhs = dev(inst.vartype), dev(lhs), dev(rhs)
    ties = 0
    for r in range(1, max_rounds + 1):
        res = dp.dp_propagate(ctx, mat, dev(L), dev(U), d_vt, d_lhs, d_rhs, params=p1)
        o = orc.round_(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, L, U, inst.vartype, lhs,
                       rhs, q, analysis=True)
        g_lb, g_ub = host(res.lb), host(res.ub)
        nbad, nt, det = compare_bounds(g_lb, g_ub, o.lb, o.ub, inst.vartype, o.lb_err, o.ub_err,
                                       o.lb_tie, o.ub_tie)
        ties += nt
        assert nbad == 0, f"round {r}: {nbad} bounds differ: {det}"
        assert res.rounds == 1
        if not o.inf_tie:
            assert res.infeasible == o.infeasible, f"round {r}: infeasible flag differs"
        assert (res.status == dp.DP_CAP_HIT) == (bool(o.changed) and not o.infeasible), f"round {r}"
        if o.infeasible or not o.changed:
            return r, ties
        L, U = g_lb, g_ub
    return max_rounds, ties


def check_full(dp, ctx, mat, inst, orc, params=None, exact=True, **kw):
    g_lb, g_ub, r = gpu_full(dp, ctx, mat, inst,
                             dp.dp_params_default(**params) if params else None, **kw)
    o = orc.propagate_instance(inst, params)
    assert r.infeasible == o.infeasible
    assert r.rounds == o.rounds, (r.rounds, o.rounds)
    assert (r.status == dp.DP_CAP_HIT) == bool(o.status)
    if exact:
        assert np.array_equal(g_lb, o.lb) and np.array_equal(g_ub, o.ub)
    else:
        nbad, _, det = compare_bounds(g_lb, g_ub, o.lb, o.ub, inst.vartype)
        assert nbad == 0, det
    return r


def test_tiny_full_bit_exact(gpu, orc):
    dp, ctx = gpu
    inst = synth.tiny()
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        assert mat.info()["split_rows"] == 0
        r = check_full(dp, ctx, mat, inst, orc, exact=True)
        assert r.rounds > 2


def test_tiny_host_pointers(gpu, orc):
    dp, ctx = gpu
    inst = synth.tiny()
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        check_full(dp, ctx, mat, inst, orc, exact=True, on_host=True)


def test_tiny_replay_bit_exact(gpu, orc):
    dp, ctx = gpu
    inst = synth.tiny()
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        rounds, ties = replay(dp, ctx, mat, inst, orc)
        assert rounds > 2 and ties == 0


@pytest.mark.parametrize("chunk", [8, 16])
def test_tiny_split_rows(gpu, orc, chunk):
    """Rows longer than `chunk` are split across lanes and combined."""
    dp, ctx = gpu
    inst = synth.tiny(seed=synth.seed_for(0, 7), m=600, n=400)
    rp = inst.row_ptr
    # make some rows long so that several chunks and slices are involved
    rng = np.random.default_rng(5)
    big = synth.small_random(rng, 300, 400, 60)
    with dp.Matrix(ctx, big.m, big.n, big.row_ptr, big.col, big.val, chunk) as mat:
        assert mat.info()["split_rows"] > 0
        replay(dp, ctx, mat, big, orc)
        check_full(dp, ctx, mat, big, orc, exact=False)
    with dp.Matrix(ctx, inst.m, inst.n, rp, inst.col, inst.val, chunk) as mat:
        replay(dp, ctx, mat, inst, orc)


# replayed decisions the oracle flags as ties may go either way; a few per
# workload are expected with fractional data, many would point at a bug
TIE_BUDGET = 20


def test_medium_scaled(gpu, orc):
    dp, ctx = gpu
    inst = synth.medium(scale=0.1)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        assert mat.info()["split_rows"] > 0
        _, ties = replay(dp, ctx, mat, inst, orc)
        assert ties <= TIE_BUDGET
        check_full(dp, ctx, mat, inst, orc, exact=False)


def test_large_scaled(gpu, orc):
    dp, ctx = gpu
    inst = synth.large(scale=0.02)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        assert mat.info()["split_rows"] > 0
        _, ties = replay(dp, ctx, mat, inst, orc)
        assert ties <= TIE_BUDGET
        check_full(dp, ctx, mat, inst, orc, exact=False)


def test_side_ordered_layout_bit_exact(gpu, orc):
    """Rows ordered by side pattern (dp_matrix_load_sides): warps whose rows
    all have an infinite side skip that side's activity; results unchanged."""
    dp, ctx = gpu
    inst = synth.tiny()
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val,
                   lhs=inst.lhs, rhs=inst.rhs) as mat:
        check_full(dp, ctx, mat, inst, orc, exact=True)
        rounds, ties = replay(dp, ctx, mat, inst, orc)
        assert ties == 0


@pytest.mark.parametrize("chunk", [0, 16])
def test_side_hints_never_change_results(gpu, orc, chunk):
    """Hints that disagree with the sides of the call (finite where the call
    has infinite sides and the reverse) change the order only."""
    dp, ctx = gpu
    rng = np.random.default_rng(23)
    inst = synth.small_random(rng, 600, 500, 40, ranged_frac=0.5)
    wrong_l = np.where(np.isfinite(inst.lhs), -np.inf, 0.0)
    wrong_r = np.where(np.isfinite(inst.rhs), np.inf, 0.0)
    for hl, hr in ((inst.lhs, inst.rhs), (wrong_l, wrong_r)):
        with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val, chunk,
                       lhs=hl, rhs=hr) as mat:
            replay(dp, ctx, mat, inst, orc)
            check_full(dp, ctx, mat, inst, orc, exact=(chunk == 0))


def test_large_scaled_side_ordered(gpu, orc):
    dp, ctx = gpu
    inst = synth.large(scale=0.02)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val,
                   lhs=inst.lhs, rhs=inst.rhs) as mat:
        _, ties = replay(dp, ctx, mat, inst, orc)
        assert ties <= TIE_BUDGET
        check_full(dp, ctx, mat, inst, orc, exact=False)


def test_launch_shapes_bit_identical(gpu, orc):
    """Both block shapes of the round kernels give the same bits."""
    dp, ctx = gpu
    inst = synth.tiny()
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        a = gpu_full(dp, ctx, mat, inst)
        mat.set_launch(4)
        b = gpu_full(dp, ctx, mat, inst)
        check_full(dp, ctx, mat, inst, orc, exact=True)
        mat.set_launch(8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2].rounds == b[2].rounds


def test_autotune_picks_a_measured_configuration(gpu, orc):
    dp, ctx = gpu
    inst = synth.medium(scale=0.05)
    t = dp.dp_autotune(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val, inst.lb, inst.ub,
                       inst.vartype, inst.lhs, inst.rhs, rounds=3)
    us = [e["us_per_round"] for e in t["entries"]]
    assert len(us) >= 4 and min(us) > 0 and t["best"]["us_per_round"] == min(us)
    assert {e["round_warps"] for e in t["entries"]} == {4, 8}
    b = t["best"]
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val, b["chunk"],
                   lhs=inst.lhs, rhs=inst.rhs) as mat:
        mat.set_launch(b["round_warps"])
        check_full(dp, ctx, mat, inst, orc, exact=False)


def test_persistent_loop_bit_exact(gpu, orc):
    """The persistent (cooperative) round loop gives the graph loop's bits
    and the oracle's (tiny: bit-exact) results, including the round count,
    the cap status and infeasibility."""
    dp, ctx = gpu
    inst = synth.tiny()
    d = [dev(a) for a in (inst.lb, inst.ub, inst.vartype, inst.lhs, inst.rhs)]
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        r = dp.dp_propagate_persistent(ctx, mat, *d)
        o = orc.propagate_instance(inst)
        assert r.rounds == o.rounds and r.infeasible == o.infeasible
        assert np.array_equal(host(r.lb), o.lb) and np.array_equal(host(r.ub), o.ub)
        for q in ({"max_rounds": 2}, {"max_rounds": 0}):
            rp = dp.dp_propagate_persistent(ctx, mat, *d, params=dp.dp_params_default(**q))
            rg = dp.dp_propagate(ctx, mat, *d, params=dp.dp_params_default(**q))
            assert rp.rounds == rg.rounds and rp.status == rg.status
            assert np.array_equal(host(rp.lb), host(rg.lb))
    LB, UB = synth.node_bounds(inst, 6, seed=11, lo_frac=0.05, hi_frac=0.2)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        for b in range(6):
            rp = dp.dp_propagate_persistent(ctx, mat, dev(LB[b]), dev(UB[b]), *d[2:])
            rg = dp.dp_propagate(ctx, mat, dev(LB[b]), dev(UB[b]), *d[2:])
            assert rp.rounds == rg.rounds and rp.infeasible == rg.infeasible
            assert np.array_equal(host(rp.lb), host(rg.lb)) and np.array_equal(host(rp.ub), host(rg.ub))


def test_persistent_loop_large_scaled_equals_graph(gpu):
    dp, ctx = gpu
    inst = synth.large(scale=0.05)
    d = [dev(a) for a in (inst.lb, inst.ub, inst.vartype, inst.lhs, inst.rhs)]
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val,
                   lhs=inst.lhs, rhs=inst.rhs) as mat:
        assert mat.info()["split_rows"] > 0
        rg = dp.dp_propagate(ctx, mat, *d)
        rp = dp.dp_propagate_persistent(ctx, mat, *d)
        assert rp.rounds == rg.rounds and rp.infeasible == rg.infeasible
        assert np.array_equal(host(rp.lb), host(rg.lb)) and np.array_equal(host(rp.ub), host(rg.ub))


def test_value_compression_lossless(gpu, orc):
    """Small-integer coefficients can be read as int8 (off by default);
    results are bit-identical with compression on and off, and equal the
    oracle."""
    dp, ctx = gpu
    inst = synth.tiny()
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        b0 = gpu_full(dp, ctx, mat, inst)  # default: binary64 values
        assert mat.set_compression(True)
        a = gpu_full(dp, ctx, mat, inst)
        assert np.array_equal(a[0], b0[0]) and np.array_equal(a[1], b0[1])
        check_full(dp, ctx, mat, inst, orc, exact=True)
        assert not mat.set_compression(False)
        b = gpu_full(dp, ctx, mat, inst)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2].rounds == b[2].rounds
    # every small integer value, both signs, through the kernels' conversion
    rng = np.random.default_rng(3)
    big = synth.small_random(rng, 400, 300, 30, coef=(1, 127))
    with dp.Matrix(ctx, big.m, big.n, big.row_ptr, big.col, big.val, 16) as mat:
        assert mat.set_compression(True)
        replay(dp, ctx, mat, big, orc)
    med = synth.medium(scale=0.01)  # fractional coefficients: no int8 copy
    with dp.Matrix(ctx, med.m, med.n, med.row_ptr, med.col, med.val) as mat:
        assert not mat.set_compression(True)
