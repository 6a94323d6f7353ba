"""Planted mistakes in a copy of the oracle (on the CPU): each plausible
slip -- a dropped term, a wrong sign, a wrong rounding direction, a skipped
rule -- must make at least one pin fail.  This shows the pins constrain the
oracle, not merely agree with it."""
import shutil

import numpy as np
import pytest

import test_oracle_pins as pins
from paper_2009_07785_gb300 import synth

MUTANTS = {
    "min_activity_uses_wrong_bound": ("double bmin = (a > 0.0) ? L[j] : U[j];\n      double bmax = (a > 0.0) ? U[j] : L[j];\n      if (isinf(bmin)) {",
                                      "double bmin = (a < 0.0) ? L[j] : U[j];\n      double bmax = (a > 0.0) ? U[j] : L[j];\n      if (isinf(bmin)) {"),
    "residual_sign": ("resmin = fma(-a, bmin, minfin[i]);", "resmin = fma(a, bmin, minfin[i]);"),
    "no_one_infinity_rule": ("else if (mininf[i] == 1 && isinf(bmin))", "else if (0)"),
    "lower_rounding_direction": ("lc = ceil(lc - eps_int);", "lc = floor(lc - eps_int);"),
    "upper_rounding_epsilon_sign": ("uc = floor(uc + eps_int);", "uc = floor(uc - eps_int);"),
    "step2_dropped": ("if (sfin_max < thr) *infeasible = 1;", ""),
    "threshold_ignored": ("accept = lc > thr;", "accept = lc > L[j];"),
    "round_count_off_by_one": ("*rounds = r;", "*rounds = r - 1;"),
    "lhs_side_dropped": ("if (isfinite(lhs[i]) && isfinite(resmax)) { lc = (lhs[i] - resmax) / a;",
                         "if (0) { lc = (lhs[i] - resmax) / a;"),
    # the infinity-threshold readings: >= turned into >, a dropped discard,
    # a sign slip on the -inf_threshold side
    "input_ub_threshold_strict": ("if (ub[j] >= inf_threshold) ub[j] = INFINITY;",
                                  "if (ub[j] > inf_threshold) ub[j] = INFINITY;"),
    "input_lb_threshold_strict": ("if (lb[j] <= -inf_threshold) lb[j] = -INFINITY;",
                                  "if (lb[j] < -inf_threshold) lb[j] = -INFINITY;"),
    "input_rhs_threshold_strict": ("if (rhs[i] >= inf_threshold) rhs[i] = INFINITY;",
                                   "if (rhs[i] > inf_threshold) rhs[i] = INFINITY;"),
    "input_lhs_threshold_sign": ("if (lhs[i] <= -inf_threshold) lhs[i] = -INFINITY;",
                                 "if (-lhs[i] <= -inf_threshold) lhs[i] = -INFINITY;"),
    "upper_candidate_threshold_strict": ("if (isfinite(uc) && fabs(uc) >= inf_threshold) {",
                                         "if (isfinite(uc) && fabs(uc) > inf_threshold) {"),
    "lower_candidate_threshold_strict": ("if (isfinite(lc) && fabs(lc) >= inf_threshold) {",
                                         "if (isfinite(lc) && fabs(lc) > inf_threshold) {"),
    "upper_candidate_discard_dropped": ("        uc = INFINITY;\n      } else if", "        ;\n      } else if"),
    "lower_candidate_discard_dropped": ("        lc = -INFINITY;\n      } else if", "        ;\n      } else if"),
    "live_reads_in_candidates": ("      double bmin = (a > 0.0) ? L[j] : U[j];\n      double bmax = (a > 0.0) ? U[j] : L[j];\n\n      /* residual",
                                 "      double bmin = (a > 0.0) ? Lnew[j] : Unew[j];\n      double bmax = (a > 0.0) ? Unew[j] : Lnew[j];\n\n      /* residual"),
}


def failures(o):
    bad = []
    for case in pins.load_cases():
        inst, elb, eub = pins.build_case(case)
        try:
            r = pins_propagate(o, inst)
        except Exception as e:  # noqa: BLE001
            bad.append(f"{case['name']}: {e}")
            continue
        if (r.infeasible != case["infeasible"] or r.rounds != case["rounds"]
                or not np.array_equal(r.lb, elb) or not np.array_equal(r.ub, eub)):
            bad.append(case["name"])
    for m in (1, 5):
        r = pins_propagate(o, pins.cascade(m))
        if r.rounds != m + 1 or not np.all(r.ub == 0):
            bad.append(f"cascade{m}")
    for seed in range(12):
        rng = np.random.default_rng(1000 + seed)
        n = int(rng.integers(2, 7))
        m = int(rng.integers(1, 5))
        inst = synth.small_random(rng, m, n, maxlen=n, pure_integer=True, bounded=True,
                                  slack_mean=0.7, ranged_frac=0.4)
        inst.ub = np.minimum(inst.ub, 3.0)
        if seed % 3 == 0:
            inst.rhs = inst.rhs - rng.uniform(0, 6, size=m)
        feas = pins.enumerate_points(inst)
        r = pins_propagate(o, inst)
        if r.infeasible and feas.shape[0]:
            bad.append(f"brute{seed}: false infeasible")
        if not r.infeasible and not (np.all(feas >= r.lb - 1e-9) and np.all(feas <= r.ub + 1e-9)):
            bad.append(f"brute{seed}: cut off a point")
    return bad


def pins_propagate(o, inst):
    import oracle
    return oracle.propagate_instance(inst, oracle=o)


@pytest.fixture(scope="module")
def good(orc):
    return orc.Oracle()


def test_unmutated_oracle_passes(good):
    assert failures(good) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(orc, tmp_path, name):
    old, new = MUTANTS[name]
    for f in orc.SOURCES:
        shutil.copy(orc.HERE / f, tmp_path / f)
    src = (tmp_path / "dp_oracle.c").read_text()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    (tmp_path / "dp_oracle.c").write_text(src.replace(old, new))
    lib = orc.build(force=True, sources_dir=tmp_path, out=tmp_path / "mut.so")
    assert failures(orc.Oracle(lib)), f"mutant {name} survived every pin"
