"""Comparison helpers for GPU-vs-oracle parity tests.

Tolerance (written here, used by every parity test): integer-variable bounds
and the infeasibility flag must match exactly; continuous bounds within
max(1e-12, 1e-9 |oracle|), widened only by the oracle's rigorous bound on the
reordering error of that value (nonzero only for rows the GPU splits across
threads).  A decision the oracle flags as a tie (within that error bound of
a rounding or acceptance threshold) may go either way.
"""
from __future__ import annotations

import numpy as np

REL = 1e-9
ABS = 1e-12


def close_cont(g, o, err):
    """Equal (including equal infinities), or both finite and within the
    tolerance: an infinite bound on one side only is a different result,
    never a rounding difference (the relative tolerance of an infinite
    oracle value would otherwise be infinite)."""
    same = (g == o)
    tol = np.maximum(np.maximum(ABS, REL * np.abs(o)), err)
    with np.errstate(invalid="ignore"):
        fin = np.isfinite(g) & np.isfinite(o) & (np.abs(g - o) <= tol)
    return same | fin


def compare_bounds(g_lb, g_ub, o_lb, o_ub, vartype, lb_err=None, ub_err=None, lb_tie=None,
                   ub_tie=None):
    """Returns (n_bad, n_tie_used, details) comparing GPU and oracle bounds."""
    n = g_lb.size
    lb_err = np.zeros(n) if lb_err is None else lb_err
    ub_err = np.zeros(n) if ub_err is None else ub_err
    lb_tie = np.zeros(n, bool) if lb_tie is None else lb_tie.astype(bool)
    ub_tie = np.zeros(n, bool) if ub_tie is None else ub_tie.astype(bool)
    isint = vartype.astype(bool)
    ok_l = np.where(isint, g_lb == o_lb, close_cont(g_lb, o_lb, lb_err))
    ok_u = np.where(isint, g_ub == o_ub, close_cont(g_ub, o_ub, ub_err))
    bad_l = ~ok_l & ~lb_tie
    bad_u = ~ok_u & ~ub_tie
    ties = int((~ok_l & lb_tie).sum() + (~ok_u & ub_tie).sum())
    nbad = int(bad_l.sum() + bad_u.sum())
    details = ""
    if nbad:
        idx = np.flatnonzero(bad_l | bad_u)[:8]
        details = "; ".join(f"j={j} int={int(isint[j])} lb g={g_lb[j]!r} o={o_lb[j]!r} "
                            f"ub g={g_ub[j]!r} o={o_ub[j]!r}" for j in idx)
    return nbad, ties, details
