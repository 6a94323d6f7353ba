"""dp_propagate_noalloc: the allocation-free entry point, for callers whose
device memory belongs to a pool allocator (or whose pipeline cannot afford
the device synchronisation of cudaMalloc/cudaFree) and who therefore must not
allocate.  Its results must equal those of dp_propagate, which allocates its
matrix layout and workspace at load time, on consecutive calls that share
the entry point's static scratch array."""
import numpy as np
import pytest
import torch

from paper_2009_07785_gb300 import synth
from parity import compare_bounds

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_dp_propagate_on_consecutive_calls(gpu):
    dp, ctx = gpu
    inst = synth.tiny()
    LB, UB = synth.node_bounds(inst, 1, seed=3)
    problems = [(inst.lb, inst.ub), (LB[0], UB[0])]  # two different calls in a row
    d_rp, d_col, d_val = dev(inst.row_ptr), dev(inst.col), dev(inst.val)
    d_vt, d_lhs, d_rhs = dev(inst.vartype), dev(inst.lhs), dev(inst.rhs)
    stream = torch.cuda.current_stream()
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        for lb, ub in problems:
            ref = dp.dp_propagate(ctx, mat, dev(lb), dev(ub), d_vt, d_lhs, d_rhs)
            lo = torch.empty(inst.n, dtype=torch.float64, device="cuda")
            hi = torch.empty_like(lo)
            got = dp.dp_propagate_noalloc(0, stream, inst.m, inst.n, d_rp, d_col, d_val, dev(lb),
                                          dev(ub), d_vt, d_lhs, d_rhs, lo, hi)
            assert got.rounds == ref.rounds and got.infeasible == ref.infeasible
            assert got.status == ref.status
            nbad, _, det = compare_bounds(lo.cpu().numpy(), hi.cpu().numpy(),
                                          ref.lb.cpu().numpy(), ref.ub.cpu().numpy(),
                                          inst.vartype)
            assert nbad == 0, det


def test_noalloc_rejects_oversize_and_host_pointers(gpu):
    dp, _ = gpu
    inst = synth.tiny(m=20, n=10)
    d = [dev(a) for a in (inst.row_ptr, inst.col, inst.val, inst.lb, inst.ub, inst.vartype,
                          inst.lhs, inst.rhs)]
    lo = torch.empty(inst.n, dtype=torch.float64, device="cuda")
    hi = torch.empty_like(lo)
    with pytest.raises(dp.DomPropError) as e:
        dp.dp_propagate_noalloc(0, None, inst.m, dp.NOALLOC_MAX_VARS + 1, *d, lo, hi)
    assert e.value.code == dp.DP_ERR_INVALID_ARG
    host = list(d)
    host[3] = inst.lb  # a host array where device memory is required
    with pytest.raises(dp.DomPropError) as e:
        dp.dp_propagate_noalloc(0, None, inst.m, inst.n, *host, lo, hi)
    assert e.value.code == dp.DP_ERR_INVALID_ARG
