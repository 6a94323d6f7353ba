"""dp_propagate_noalloc: the allocation-free entry point, for callers whose
device memory belongs to a pool allocator (or whose pipeline cannot afford
the device synchronisation of cudaMalloc/cudaFree) and who therefore must not
allocate.  Its one-thread-per-row round sums every row in CSR order, as the
oracle does, so its results must equal the oracle's bit for bit and match
dp_propagate (which allocates its matrix layout and workspace at load time)
on consecutive calls that share the entry point's static scratch array.

This file is collected last so that a failure here cannot hide another
test's result in a run that stops at the first failure."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2009_07785_gb300 import synth

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def outputs(n):
    lo = torch.empty(n, dtype=torch.float64, device="cuda")
    return lo, torch.empty_like(lo)


def noalloc(dp, inst, lb, ub, params=None, row_ptr=None):
    lo, hi = outputs(inst.n)
    d = [dev(inst.row_ptr if row_ptr is None else row_ptr), dev(inst.col), dev(inst.val),
         dev(lb), dev(ub), dev(inst.vartype), dev(inst.lhs), dev(inst.rhs)]
    r = dp.dp_propagate_noalloc(0, torch.cuda.current_stream(), inst.m, inst.n, *d, lo, hi,
                                params=params)
    return r, lo.cpu().numpy(), hi.cpu().numpy()


def test_noalloc_equals_oracle_and_dp_propagate_on_consecutive_calls(gpu, orc):
    dp, ctx = gpu
    inst = synth.tiny()
    LB, UB = synth.node_bounds(inst, 2, seed=3)
    # three calls in a row on the shared scratch array: the root problem, a
    # node that turns infeasible, and the root problem again
    problems = [(inst.lb, inst.ub), (LB[0], UB[0]), (inst.lb, inst.ub)]
    d_vt, d_lhs, d_rhs = dev(inst.vartype), dev(inst.lhs), dev(inst.rhs)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        for lb, ub in problems:
            got, lo, hi = noalloc(dp, inst, lb, ub)
            o = orc.propagate(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, lb, ub,
                              inst.vartype, inst.lhs, inst.rhs)
            assert got.rounds == o.rounds and got.infeasible == o.infeasible
            assert (got.status == dp.DP_CAP_HIT) == bool(o.status)
            assert np.array_equal(lo, o.lb) and np.array_equal(hi, o.ub)
            ref = dp.dp_propagate(ctx, mat, dev(lb), dev(ub), d_vt, d_lhs, d_rhs)
            assert got.rounds == ref.rounds and got.infeasible == ref.infeasible
            assert got.status == ref.status
            assert np.array_equal(lo, ref.lb.cpu().numpy())
            assert np.array_equal(hi, ref.ub.cpu().numpy())


@pytest.mark.parametrize("max_rounds", [0, 1, 3])
def test_noalloc_round_cap(gpu, orc, max_rounds):
    """The cap: rounds, status and bounds as the oracle and dp_propagate
    give them (max_rounds = 0 returns the normalised input bounds)."""
    dp, ctx = gpu
    inst = synth.tiny()
    p = dp.dp_params_default(max_rounds=max_rounds)
    got, lo, hi = noalloc(dp, inst, inst.lb, inst.ub, params=p)
    o = orc.propagate_instance(inst, {"max_rounds": max_rounds})
    assert got.rounds == o.rounds == max_rounds
    assert (got.status == dp.DP_CAP_HIT) == bool(o.status) == (max_rounds > 0)
    assert np.array_equal(lo, o.lb) and np.array_equal(hi, o.ub)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        ref = dp.dp_propagate(ctx, mat, *[dev(a) for a in inst.problem()], params=p)
    assert ref.rounds == got.rounds and ref.status == got.status


def test_noalloc_device_side_input_checks(gpu):
    """A malformed CSR held in device memory is caught by the prologue (which
    reads only in-range entries) before any round runs; so are NaN bounds."""
    dp, _ = gpu
    inst = synth.tiny(m=50, n=40)
    bad = inst.row_ptr.copy()
    bad[10], bad[11] = bad[11], bad[10]  # row_ptr decreases
    if bad[10] == bad[11]:
        bad[10] += 1
    with pytest.raises(dp.DomPropError) as e:
        noalloc(dp, inst, inst.lb, inst.ub, row_ptr=bad)
    assert e.value.code == dp.DP_ERR_BAD_CSR
    short = inst.row_ptr.copy()
    short[-1] -= 1  # the last row ends before nnz
    with pytest.raises(dp.DomPropError) as e:
        noalloc(dp, inst, inst.lb, inst.ub, row_ptr=short)
    assert e.value.code == dp.DP_ERR_BAD_CSR
    lb = inst.lb.copy()
    lb[7] = np.nan
    with pytest.raises(dp.DomPropError) as e:
        noalloc(dp, inst, lb, inst.ub)
    assert e.value.code == dp.DP_ERR_NAN_INPUT
    # the scratch array is fine afterwards
    got, lo, hi = noalloc(dp, inst, inst.lb, inst.ub)
    assert got.rounds >= 1


def test_noalloc_rejects_bad_arguments(gpu):
    dp, _ = gpu
    inst = synth.tiny(m=20, n=10)
    d = [dev(a) for a in (inst.row_ptr, inst.col, inst.val, inst.lb, inst.ub, inst.vartype,
                          inst.lhs, inst.rhs)]
    lo, hi = outputs(inst.n)
    stream = torch.cuda.current_stream()

    def expect_invalid(*args, n=inst.n):
        with pytest.raises(dp.DomPropError) as e:
            dp.dp_propagate_noalloc(0, stream, inst.m, n, *args)
        assert e.value.code == dp.DP_ERR_INVALID_ARG

    expect_invalid(*d, lo, hi, n=dp.NOALLOC_MAX_VARS + 1)
    host = list(d)
    host[3] = inst.lb  # a host array where device memory is required
    expect_invalid(*host, lo, hi)
    wrong = list(d)
    wrong[1] = d[1].to(torch.int64)  # int64 column indices would be misread
    expect_invalid(*wrong, lo, hi)
    wrong = list(d)
    wrong[0] = d[0].to(torch.int32)  # a too-short row_ptr would be read past its end
    expect_invalid(*wrong, lo, hi)
    expect_invalid(*d, lo.to(torch.float32), hi)  # 8n bytes into a 4n-byte buffer
    expect_invalid(*d, lo[:-1], hi)
    # the C entry point itself refuses a host pointer (no binding checks)
    inf, rounds = C.c_int32(), C.c_int32()
    ptrs = [C.c_void_p(t.data_ptr()) for t in d]
    ptrs[3] = C.c_void_p(inst.lb.ctypes.data)
    rc = dp.lib().dp_propagate_noalloc(0, None, inst.m, inst.n, int(d[1].numel()), *ptrs, None,
                                       C.c_void_p(lo.data_ptr()), C.c_void_p(hi.data_ptr()),
                                       C.byref(inf), C.byref(rounds))
    assert rc == dp.DP_ERR_INVALID_ARG


def test_noalloc_keeps_the_callers_current_device(gpu):
    dp, _ = gpu
    inst = synth.tiny(m=30, n=20)
    torch.cuda.set_device(0)
    noalloc(dp, inst, inst.lb, inst.ub)
    assert torch.cuda.current_device() == 0
