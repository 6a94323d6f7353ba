"""Serving with continuous batching (dp_server_*): every request's result is
the one the request gets alone -- bit for bit the batched path's result for
that node, and the oracle's within the parity tolerance -- however requests
arrive, share slots and matrices, or wait for memory."""
import time

import numpy as np
import pytest
import torch

from paper_2009_07785_gb300 import synth
from parity import compare_bounds

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def pool(dp, ctx):
    """Three resident matrices of different shapes (one with split rows)."""
    rng = np.random.default_rng(31)
    insts = [synth.tiny(m=600, n=450), synth.medium(scale=0.01),
             synth.small_random(rng, 300, 400, 60)]
    mats = [dp.Matrix(ctx, i.m, i.n, i.row_ptr, i.col, i.val, 16 if k == 2 else 0)
            for k, i in enumerate(insts)]
    return insts, mats


def drain(srv, want, timeout_s=60.0):
    got = []
    t0 = time.time()
    while len(got) < want:
        got += srv.poll(256, wait_us=2000)
        assert time.time() - t0 < timeout_s, f"{len(got)} of {want} completions"
    return got


def alone(dp, ctx, mat, inst, lb, ub, params=None):
    r = dp.dp_propagate_nodes(ctx, mat, dev(lb[None]), dev(ub[None]), dev(inst.vartype),
                              dev(inst.lhs), dev(inst.rhs), params=params)
    return r.lb.cpu().numpy()[0], r.ub.cpu().numpy()[0], r


def test_serving_mixed_arrivals_equal_alone(gpu, orc):
    dp, ctx = gpu
    insts, mats = pool(dp, ctx)
    nodes = [synth.node_bounds(i, 40, seed=100 + k, lo_frac=0.01, hi_frac=0.08)
             for k, i in enumerate(insts)]
    rng = np.random.default_rng(7)
    plan = [(int(rng.integers(3)), int(rng.integers(40))) for _ in range(150)]
    with dp.Server(ctx, slots=32) as srv:
        ids = [srv.add_matrix(m, i.vartype, i.lhs, i.rhs) for m, i in zip(mats, insts)]
        meta = {}
        for q, (k, b) in enumerate(plan):  # bursts with pauses, so requests
            tag = srv.submit(ids[k], nodes[k][0][b], nodes[k][1][b])  # join running batches
            meta[tag] = (k, b)
            if q % 17 == 0:
                time.sleep(0.002)
        got = drain(srv, len(plan))
        st = srv.stats()
    assert st["completed"] == len(plan) and st["admissions"] == len(plan)
    assert st["max_active_slots"] <= 32
    checked = set()
    for c in got:
        k, b = meta[c["tag"]]
        inst, mat = insts[k], mats[k]
        lb, ub, r = alone(dp, ctx, mat, inst, nodes[k][0][b], nodes[k][1][b])
        assert np.array_equal(c["lb"], lb) and np.array_equal(c["ub"], ub), (k, b)
        assert c["rounds"] == r.rounds[0] and c["infeasible"] == r.infeasible[0]
        assert (c["status"] == dp.DP_CAP_HIT) == bool(r.cap_hit[0])
        if (k, b) not in checked and len(checked) < 30:
            checked.add((k, b))
            o = orc.propagate(inst.m, inst.n, inst.row_ptr, inst.col, inst.val,
                              nodes[k][0][b], nodes[k][1][b], inst.vartype, inst.lhs, inst.rhs)
            assert c["rounds"] == o.rounds and c["infeasible"] == o.infeasible
            nbad, _, det = compare_bounds(c["lb"], c["ub"], o.lb, o.ub, inst.vartype)
            assert nbad == 0, det
    for m in mats:
        m.close()


def test_serving_recycles_slots_and_counts_rounds_per_request(gpu, orc):
    """100 requests through 32 slots of one matrix: slots are refilled as
    nodes finish, and each request's round count is its own."""
    dp, ctx = gpu
    inst = synth.tiny(m=800, n=600)
    LB, UB = synth.node_bounds_at_point(inst, 100, seed=3)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        with dp.Server(ctx, slots=32) as srv:
            mid = srv.add_matrix(mat, inst.vartype, inst.lhs, inst.rhs)
            tags = [srv.submit(mid, LB[b], UB[b]) for b in range(100)]
            got = {c["tag"]: c for c in drain(srv, 100)}
            st = srv.stats()
        assert st["max_active_slots"] <= 32 and st["rounds"] > 0
        for b, t in enumerate(tags):
            o = orc.propagate(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, LB[b], UB[b],
                              inst.vartype, inst.lhs, inst.rhs)
            c = got[t]
            assert c["rounds"] == o.rounds and c["infeasible"] == o.infeasible
            assert np.array_equal(c["lb"], o.lb) and np.array_equal(c["ub"], o.ub)
            assert c["done_us"] >= c["arrival_us"]


def test_serving_memory_budget_evicts_idle_matrices(gpu):
    """A budget that holds one matrix's workspace at a time: requests for
    the other matrix wait until the first goes idle, then take its memory."""
    dp, ctx = gpu
    a, b = synth.tiny(m=500, n=400, seed=11), synth.tiny(m=500, n=400, seed=12)
    ma = dp.Matrix(ctx, a.m, a.n, a.row_ptr, a.col, a.val)
    mb = dp.Matrix(ctx, b.m, b.n, b.row_ptr, b.col, b.val)
    LA, UA = synth.node_bounds(a, 8, seed=1)
    LB, UB = synth.node_bounds(b, 8, seed=2)
    with dp.Server(ctx, slots=32) as probe:  # one matrix's workspace size
        ip = probe.add_matrix(ma, a.vartype, a.lhs, a.rhs)
        probe.submit(ip, LA[0], UA[0])
        drain(probe, 1)
        one = probe.stats()["device_bytes"]
    budget = one * 3 // 2
    with dp.Server(ctx, slots=32, mem_budget=budget) as srv:
        ia = srv.add_matrix(ma, a.vartype, a.lhs, a.rhs)
        ib = srv.add_matrix(mb, b.vartype, b.lhs, b.rhs)
        ta = [srv.submit(ia, LA[k], UA[k]) for k in range(8)]
        got = {c["tag"]: c for c in drain(srv, 8)}
        tb = [srv.submit(ib, LB[k], UB[k]) for k in range(8)]
        got.update({c["tag"]: c for c in drain(srv, 8)})
        st = srv.stats()
    assert st["evictions"] >= 1 and st["workspaces_allocated"] >= 2
    assert 0 < st["device_bytes"] <= budget
    for k in range(8):
        lb, ub, _ = alone(dp, ctx, ma, a, LA[k], UA[k])
        assert np.array_equal(got[ta[k]]["lb"], lb) and np.array_equal(got[ta[k]]["ub"], ub)
        lb, ub, _ = alone(dp, ctx, mb, b, LB[k], UB[k])
        assert np.array_equal(got[tb[k]]["lb"], lb) and np.array_equal(got[tb[k]]["ub"], ub)
    ma.close()
    mb.close()


def test_serving_round_cap_and_bad_requests(gpu, orc):
    dp, ctx = gpu
    inst = synth.tiny(m=600, n=500)
    LB, UB = synth.node_bounds_at_point(inst, 16, seed=5)
    p = dp.dp_params_default(max_rounds=2)
    with dp.Matrix(ctx, inst.m, inst.n, inst.row_ptr, inst.col, inst.val) as mat:
        with dp.Server(ctx, slots=32, params=p) as srv:
            mid = srv.add_matrix(mat, inst.vartype, inst.lhs, inst.rhs)
            bad = LB[0].copy()
            bad[3] = np.nan
            with pytest.raises(dp.DomPropError) as e:
                srv.submit(mid, bad, UB[0])
            assert e.value.code == dp.DP_ERR_NAN_INPUT
            with pytest.raises(dp.DomPropError) as e:
                srv.submit(mid + 5, LB[0], UB[0])
            assert e.value.code == dp.DP_ERR_INVALID_ARG
            tags = [srv.submit(mid, LB[b], UB[b]) for b in range(16)]
            got = {c["tag"]: c for c in drain(srv, 16)}
        caps = 0
        for b, t in enumerate(tags):
            o = orc.propagate(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, LB[b], UB[b],
                              inst.vartype, inst.lhs, inst.rhs, {"max_rounds": 2})
            c = got[t]
            assert c["rounds"] == o.rounds and (c["status"] == dp.DP_CAP_HIT) == bool(o.status)
            assert np.array_equal(c["lb"], o.lb) and np.array_equal(c["ub"], o.ub)
            caps += o.status
        assert caps > 0
