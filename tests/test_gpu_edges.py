"""Edge cases and error paths of the CUDA path, through the C ABI."""
import numpy as np
import pytest
import torch

import test_oracle_pins as pins
from paper_2009_07785_gb300 import synth
from parity import compare_bounds

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(dp, ctx, inst, params=None, chunk=0, on_host=False):
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val, chunk) as mat:
        args = list(inst.problem())
        if not on_host:
            args = [dev(a) for a in args]
        r = dp.dp_propagate(ctx, mat, *args, params=params)
        lb = r.lb.cpu().numpy() if isinstance(r.lb, torch.Tensor) else r.lb
        ub = r.ub.cpu().numpy() if isinstance(r.ub, torch.Tensor) else r.ub
        return lb, ub, r


@pytest.mark.parametrize("case", pins.load_cases(), ids=lambda c: c["name"])
@pytest.mark.parametrize("chunk", [0, 8])
def test_closed_forms_on_gpu(gpu, case, chunk):
    dp, ctx = gpu
    inst, elb, eub = pins.build_case(case)
    lb, ub, r = run(dp, ctx, inst, chunk=chunk)
    assert r.infeasible == case["infeasible"]
    assert r.rounds == case["rounds"]
    assert np.array_equal(lb, elb) and np.array_equal(ub, eub), (lb, ub)


@pytest.mark.parametrize("m", [1, 5, 40])
def test_cascade_on_gpu(gpu, m):
    dp, ctx = gpu
    lb, ub, r = run(dp, ctx, pins.cascade(m))
    assert r.rounds == m + 1 and r.status == dp.DP_OK
    assert np.all(ub == 0.0)


def test_round_cap(gpu):
    dp, ctx = gpu
    lb, ub, r = run(dp, ctx, pins.cascade(30), params=dp.dp_params_default(max_rounds=10))
    assert r.rounds == 10 and r.status == dp.DP_CAP_HIT and r.infeasible == 0
    assert ub[10] == 0.0 and ub[11] == 10.0


def test_zero_rounds_returns_normalised_input(gpu, orc):
    dp, ctx = gpu
    inst = synth.tiny(m=50, n=40)
    inst.lb = inst.lb + 0.3  # integer bounds get rounded
    lb, ub, r = run(dp, ctx, inst, params=dp.dp_params_default(max_rounds=0))
    L, U, _, _ = orc.normalise(inst.m, inst.n, inst.lb, inst.ub, inst.vartype, inst.lhs, inst.rhs)
    assert r.rounds == 0 and r.status == dp.DP_OK
    assert np.array_equal(lb, L) and np.array_equal(ub, U)


def test_no_rows(gpu):
    dp, ctx = gpu
    n = 7
    inst = synth.Instance("empty", 0, n, np.zeros(1, np.int64), np.zeros(0, np.int32),
                          np.zeros(0), np.zeros(n), np.full(n, 3.5), np.ones(n, np.uint8),
                          np.zeros(0), np.zeros(0), np.zeros(n))
    lb, ub, r = run(dp, ctx, inst)
    assert r.rounds == 1 and r.infeasible == 0
    assert np.all(ub == 3.0) and np.all(lb == 0.0)


def test_empty_rows_and_unused_columns(gpu, orc):
    dp, ctx = gpu
    rng = np.random.default_rng(3)
    inst = synth.small_random(rng, 500, 800, maxlen=6)  # lengths 0..6: empty rows occur
    assert (np.diff(inst.row_ptr) == 0).any()
    inst.lhs = np.where(np.diff(inst.row_ptr) == 0, -np.inf, inst.lhs)
    inst.rhs = np.where(np.diff(inst.row_ptr) == 0, 1.0, inst.rhs)
    lb, ub, r = run(dp, ctx, inst)
    o = orc.propagate_instance(inst)
    assert r.rounds == o.rounds and r.infeasible == o.infeasible
    assert np.array_equal(lb, o.lb) and np.array_equal(ub, o.ub)


def test_nan_input_is_rejected_and_context_survives(gpu):
    dp, ctx = gpu
    inst = synth.tiny(m=30, n=20)
    bad = inst.lb.copy()
    bad[5] = np.nan
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        with pytest.raises(dp.DomPropError) as e:
            dp.dp_propagate(ctx, mat, dev(bad), *[dev(a) for a in inst.problem()[1:]])
        assert e.value.code == dp.DP_ERR_NAN_INPUT
        r = dp.dp_propagate(ctx, mat, *[dev(a) for a in inst.problem()])
        assert r.status == dp.DP_OK


@pytest.mark.parametrize("defect", ["zero_coef", "col_range", "row_ptr", "nan_coef"])
def test_bad_csr_rejected(gpu, defect):
    dp, ctx = gpu
    inst = synth.tiny(m=30, n=20)
    rp, col, val = inst.row_ptr.copy(), inst.col.copy(), inst.val.copy()
    if defect == "zero_coef":
        val[3] = 0.0
    elif defect == "col_range":
        col[3] = inst.n
    elif defect == "row_ptr":
        rp[5], rp[6] = rp[6], rp[5]
    else:
        val[3] = np.nan
    with pytest.raises(dp.DomPropError) as e:
        dp.Matrix(ctx, inst.m, inst.n, rp, col, val)
    assert e.value.code == dp.DP_ERR_BAD_CSR


def test_node_fixings_infeasibility(gpu, orc):
    """Branch-and-bound node fixings make some nodes infeasible; the flag,
    the round of detection and the bounds must match the oracle."""
    dp, ctx = gpu
    inst = synth.tiny()
    LB, UB = synth.node_bounds(inst, 24, seed=11, lo_frac=0.05, hi_frac=0.2)
    seen_inf = 0
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        for b in range(LB.shape[0]):
            r = dp.dp_propagate(ctx, mat, dev(LB[b]), dev(UB[b]), dev(inst.vartype),
                                dev(inst.lhs), dev(inst.rhs))
            o = orc.propagate(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, LB[b], UB[b],
                              inst.vartype, inst.lhs, inst.rhs)
            assert r.infeasible == o.infeasible and r.rounds == o.rounds
            assert np.array_equal(r.lb.cpu().numpy(), o.lb)
            assert np.array_equal(r.ub.cpu().numpy(), o.ub)
            seen_inf += o.infeasible
    assert seen_inf > 0


def test_unbounded_and_free_variables(gpu, orc):
    dp, ctx = gpu
    rng = np.random.default_rng(21)
    inst = synth.small_random(rng, 400, 300, maxlen=5, int_frac=0.3, inf_frac=0.5)
    free = rng.random(inst.n) < 0.2
    inst.lb = np.where(free, -np.inf, inst.lb)
    lb, ub, r = run(dp, ctx, inst)
    o = orc.propagate_instance(inst)
    assert r.rounds == o.rounds and r.infeasible == o.infeasible
    assert np.array_equal(lb, o.lb) and np.array_equal(ub, o.ub)


@pytest.mark.parametrize("chunk", [0, 8])
def test_coefficients_outside_screen_range(gpu, orc, chunk):
    """Rows with |a| outside [2^-120, 2^120] skip the binary32 screen."""
    dp, ctx = gpu
    rng = np.random.default_rng(5)
    inst = synth.small_random(rng, 300, 200, maxlen=12, int_frac=0.0, bounded=True)
    k = rng.choice(inst.nnz, 20, replace=False)
    inst.val = inst.val.copy()
    inst.val[k] *= 1e-40
    lb, ub, r = run(dp, ctx, inst, chunk=chunk)
    o = orc.propagate_instance(inst)
    assert r.rounds == o.rounds and r.infeasible == o.infeasible
    nbad, _, det = compare_bounds(lb, ub, o.lb, o.ub, inst.vartype)
    assert nbad == 0, det


def test_threshold_parameters_respected(gpu, orc):
    dp, ctx = gpu
    inst = synth.tiny(m=400, n=300)
    for q in ({"tau_rel": 0.0}, {"tau_rel": 1e-3}, {"eps_int": 0.0}, {"eps_feas": 0.0},
              {"inf_threshold": 50.0}):
        if "inf_threshold" in q:  # keep the sides valid under the lower threshold
            inst.rhs = np.where(inst.rhs <= -49.0, -49.0, inst.rhs)
            inst.lhs = np.where(inst.lhs >= 49.0, 49.0, inst.lhs)
        lb, ub, r = run(dp, ctx, inst, params=dp.dp_params_default(**q))
        o = orc.propagate_instance(inst, q)
        assert r.rounds == o.rounds and r.infeasible == o.infeasible, q
        assert np.array_equal(lb, o.lb) and np.array_equal(ub, o.ub), q


def test_resume_is_a_fixed_point(gpu):
    """Checkpoint/resume: the state is the bound vector; propagating the
    result again changes nothing in one round."""
    dp, ctx = gpu
    inst = synth.tiny()
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        r1 = dp.dp_propagate(ctx, mat, *[dev(a) for a in inst.problem()])
        r2 = dp.dp_propagate(ctx, mat, r1.lb, r1.ub, dev(inst.vartype), dev(inst.lhs),
                             dev(inst.rhs))
        assert r2.rounds == 1 and r2.status == dp.DP_OK
        assert torch.equal(r1.lb, r2.lb) and torch.equal(r1.ub, r2.ub)


def test_mixed_host_device_and_repeatability(gpu):
    dp, ctx = gpu
    inst = synth.tiny()
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        d_lb = torch.empty(inst.n, dtype=torch.float64, device="cuda")
        h_ub = np.empty(inst.n)
        ref = None
        for _ in range(3):
            r = dp.dp_propagate(ctx, mat, inst.lb, dev(inst.ub), inst.vartype, dev(inst.lhs),
                                inst.rhs, lb_out=d_lb, ub_out=h_ub)
            cur = (d_lb.cpu().numpy().copy(), h_ub.copy(), r.rounds)
            if ref is not None:
                assert np.array_equal(cur[0], ref[0]) and np.array_equal(cur[1], ref[1])
                assert cur[2] == ref[2]
            ref = cur


def test_hostloop_matches_graph_loop(gpu):
    dp, ctx = gpu
    inst = synth.medium(scale=0.05)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        args = [dev(a) for a in inst.problem()]
        a = dp.dp_propagate(ctx, mat, *args)
        b = dp.dp_propagate_hostloop(ctx, mat, *args)
        assert a.rounds == b.rounds and a.infeasible == b.infeasible
        assert torch.equal(a.lb, b.lb) and torch.equal(a.ub, b.ub)
        assert b.kernel_launches[0] == b.rounds and b.kernel_ms[0] > 0


def test_two_matrices_one_context(gpu, orc):
    dp, ctx = gpu
    i1, i2 = synth.tiny(), synth.small_random(np.random.default_rng(8), 700, 500, maxlen=20)
    with dp.Matrix(ctx, i1.m, i1.n, i1.row_ptr, i1.col, i1.val) as m1, \
            dp.Matrix(ctx, i2.m, i2.n, i2.row_ptr, i2.col, i2.val, 8) as m2:
        for _ in range(2):
            for inst, mat in ((i1, m1), (i2, m2)):
                r = dp.dp_propagate(ctx, mat, *[dev(a) for a in inst.problem()])
                o = orc.propagate_instance(inst)
                assert r.rounds == o.rounds
                nbad, _, det = compare_bounds(r.lb.cpu().numpy(), r.ub.cpu().numpy(), o.lb, o.ub,
                                              inst.vartype)
                assert nbad == 0, det
