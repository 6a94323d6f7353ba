"""Parity at the benchmark sizes: the medium workload (m=200k, ~2M nonzeros)
in full, the 256 branch-and-bound nodes the batched benchmark propagates over
it (both node sets, node by node against the oracle), and the first rounds of
the large workload (m=2M, ~29.6M nonzeros) in the launch shape the benchmark
runs (row split length 256, 4 warps per block).  Tolerances are those of
tests/parity.py; the oracle runs in threads (its C calls release the GIL),
one node per call.
"""
from concurrent.futures import ThreadPoolExecutor
import os

import numpy as np
import pytest
import torch

from paper_2009_07785_gb300 import synth
from parity import compare_bounds
from test_gpu_parity import check_full, dev, replay

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

# replayed decisions the oracle flags as ties may go either way; a handful
# per workload is expected (fractional coefficients), many would mean a bug
TIE_BUDGET = 20


@pytest.fixture(scope="module")
def medium():
    return synth.medium()


def test_medium_full_size(gpu, orc, medium):
    dp, ctx = gpu
    inst = medium
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val,
                   lhs=inst.lhs, rhs=inst.rhs) as mat:
        assert mat.info()["split_rows"] > 0
        rounds, ties = replay(dp, ctx, mat, inst, orc)
        assert rounds > 5 and ties <= TIE_BUDGET, (rounds, ties)
        check_full(dp, ctx, mat, inst, orc, exact=False)


def _oracle_nodes(orc, inst, LB, UB):
    def one(k):
        return orc.propagate(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, LB[k], UB[k],
                             inst.vartype, inst.lhs, inst.rhs)

    with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        return list(ex.map(one, range(LB.shape[0])))


@pytest.mark.parametrize("node_set", ["random_values", "feasible_point_values"])
@pytest.mark.parametrize("chunk", [128, 256])
def test_medium_256_nodes(gpu, orc, medium, node_set, chunk):
    """The batched benchmark's two node sets (same seed, 256 nodes) on the
    medium matrix in both row split lengths its autotuner picks."""
    dp, ctx = gpu
    inst = medium
    seed = synth.seed_for(3, 0)
    make = synth.node_bounds if node_set == "random_values" else synth.node_bounds_at_point
    LB, UB = make(inst, 256, seed=seed)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val, chunk,
                   lhs=inst.lhs, rhs=inst.rhs) as mat:
        r = dp.dp_propagate_nodes(ctx, mat, dev(LB), dev(UB), dev(inst.vartype),
                                  dev(inst.lhs), dev(inst.rhs))
        lb, ub = r.lb.cpu().numpy(), r.ub.cpu().numpy()
    refs = _oracle_nodes(orc, inst, LB, UB)
    for k, o in enumerate(refs):
        assert r.infeasible[k] == o.infeasible, f"node {k}"
        assert r.rounds[k] == o.rounds, f"node {k}: rounds {r.rounds[k]} vs {o.rounds}"
        assert r.cap_hit[k] == o.status, f"node {k}"
        nbad, _, det = compare_bounds(lb[k], ub[k], o.lb, o.ub, inst.vartype)
        assert nbad == 0, f"node {k}: {det}"
    if node_set == "feasible_point_values":
        assert not r.infeasible.any() and r.rounds.mean() > 5


def test_large_first_rounds_bench_shape(gpu, orc):
    """Rounds 1-3 of the large workload replayed against the oracle (each GPU
    round from the GPU's own state), at split length 256 and 4 warps per
    block: the early rounds queue and re-read the most."""
    dp, ctx = gpu
    inst = synth.large()
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val, 256,
                   lhs=inst.lhs, rhs=inst.rhs) as mat:
        mat.set_launch(4)
        info = mat.info()
        assert info["split_rows"] > 10000
        rounds, ties = replay(dp, ctx, mat, inst, orc, max_rounds=3)
        assert rounds == 3 and ties <= TIE_BUDGET, (rounds, ties)
