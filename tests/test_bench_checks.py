"""The benchmark's own checks, on the CPU: the full-size parity object it
puts in its JSON line must flag every kind of mismatch the tolerance rules
of the GPU tests flag (integer bounds and the infeasibility flag exact,
continuous bounds within 1e-9 relative / 1e-12 absolute, equal infinities),
and pass the oracle's own results."""
import numpy as np
import pytest

import bench
from paper_2009_07785_gb300 import synth


@pytest.fixture(scope="module")
def solved(orc):
    inst = synth.tiny()
    return inst, orc.propagate_instance(inst)


def check(inst, o, lb=None, ub=None, rounds=None, infeasible=None):
    return bench.parity_vs_oracle(inst, o.lb.copy() if lb is None else lb,
                                  o.ub.copy() if ub is None else ub,
                                  o.rounds if rounds is None else rounds,
                                  o.infeasible if infeasible is None else infeasible, o)


def test_oracle_against_itself_passes(solved):
    inst, o = solved
    p = check(inst, o)
    assert p["ok"] and p["n_bad"] == 0 and p["bounds_compared"] == 2 * inst.n
    assert p["max_rel_diff_continuous"] == 0.0


def test_integer_bound_off_by_one_is_flagged(solved):
    inst, o = solved
    j = int(np.flatnonzero((inst.vartype == 1) & np.isfinite(o.ub))[0])
    ub = o.ub.copy()
    ub[j] += 1.0
    p = check(inst, o, ub=ub)
    assert not p["ok"] and p["n_bad"] == 1


def test_integer_bound_must_be_exact(solved):
    inst, o = solved
    j = int(np.flatnonzero((inst.vartype == 1) & np.isfinite(o.lb) & (o.lb != 0))[0])
    lb = o.lb.copy()
    lb[j] = np.nextafter(lb[j], np.inf)  # one ulp: within 1e-9, but integer
    assert check(inst, o, lb=lb)["n_bad"] == 1


def test_continuous_tolerance(solved):
    inst, o = solved
    cont = np.flatnonzero((inst.vartype == 0) & np.isfinite(o.ub) & (np.abs(o.ub) > 1.0))
    j = int(cont[0])
    ub = o.ub.copy()
    ub[j] = o.ub[j] * (1 + 1e-10)
    p = check(inst, o, ub=ub)
    assert p["ok"] and 0.0 < p["max_rel_diff_continuous"] < 1e-9
    ub[j] = o.ub[j] * (1 + 1e-8)
    assert check(inst, o, ub=ub)["n_bad"] == 1


def test_infinity_mismatch_is_flagged(solved):
    inst, o = solved
    j = int(np.flatnonzero((inst.vartype == 0) & np.isfinite(o.ub))[0])
    ub = o.ub.copy()
    ub[j] = np.inf
    assert check(inst, o, ub=ub)["n_bad"] == 1
    j2 = int(np.flatnonzero(np.isinf(o.ub))[0])
    ub = o.ub.copy()
    ub[j2] = 1e19
    assert check(inst, o, ub=ub)["n_bad"] == 1


def test_rounds_and_infeasibility_must_match(solved):
    inst, o = solved
    assert not check(inst, o, rounds=o.rounds + 1)["ok"]
    assert not check(inst, o, infeasible=1 - int(o.infeasible))["ok"]


def test_gpu_test_comparison_flags_one_sided_infinity():
    """The GPU tests' helper (tests/parity.py) applies the same rule."""
    from parity import compare_bounds

    o_lb = np.array([0.0, -np.inf, 1.0])
    o_ub = np.array([np.inf, 5.0, 2.0])
    vt = np.zeros(3, np.uint8)
    assert compare_bounds(o_lb.copy(), o_ub.copy(), o_lb, o_ub, vt)[0] == 0
    g_ub = o_ub.copy()
    g_ub[0] = 1e19  # the oracle's bound is infinite
    assert compare_bounds(o_lb.copy(), g_ub, o_lb, o_ub, vt)[0] == 1
    g_lb = o_lb.copy()
    g_lb[1] = -1e30
    assert compare_bounds(g_lb, o_ub.copy(), o_lb, o_ub, vt)[0] == 1
