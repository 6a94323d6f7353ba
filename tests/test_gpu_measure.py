"""The access-floor measurement: the round's memory access pattern without
its arithmetic takes a positive time no longer than the round kernel itself
on the same matrix, and is refused for the merge-path layout."""
import numpy as np
import pytest
import torch

from paper_2009_07785_gb300 import synth

pytestmark = pytest.mark.gpu


def test_access_floor_below_round_kernel(gpu):
    dp, ctx = gpu
    inst = synth.large(scale=0.05)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in inst.problem()]
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val,
                   lhs=inst.lhs, rhs=inst.rhs) as mat:
        floor = dp.dp_matrix_access_floor(ctx, mat, 3)
        hl = dp.dp_propagate_hostloop(ctx, mat, *d, params=dp.dp_params_default(max_rounds=3))
        k_round_us = hl.kernel_ms[0] / hl.kernel_launches[0] * 1e3
        assert 0.0 < floor <= k_round_us * 1.05, (floor, k_round_us)
        # a propagation after the measurement is unaffected
        r = dp.dp_propagate(ctx, mat, *d)
        assert r.rounds > 1
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val, merge_ipt=64) as mm:
        with pytest.raises(dp.DomPropError) as e:
            dp.dp_matrix_access_floor(ctx, mm, 1)
        assert e.value.code == dp.DP_ERR_INVALID_ARG
