"""CPU oracle for round-synchronous domain propagation (arXiv 2009.07785).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it.

The arithmetic lives in plain C (``dp_oracle.c``: Alg. 2 with round-
synchronous reads; ``dp_oracle_seq.c``: Alg. 1, sequential with constraint
marking), compiled with gcc -O2 -ffp-contract=off so binary64 rounding is
exactly what the source says.  This module only builds the shared object and
marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess
from dataclasses import dataclass
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SOURCES = ["dp_oracle.c", "dp_oracle_seq.c"]
BUILD = HERE / "_build"
LIB = BUILD / "liboracle.so"

DEFAULTS = dict(max_rounds=100, eps_int=1e-6, tau_rel=1e-6, eps_feas=1e-6, inf_threshold=1e20)


def build(force: bool = False, sources_dir: Path | None = None, out: Path | None = None) -> Path:
    """Compiles the oracle with gcc.  `sources_dir`/`out` let a test compile
    a modified copy of the sources (to show that the pins catch mistakes)."""
    src = Path(sources_dir) if sources_dir else HERE
    target = Path(out) if out else LIB
    files = [src / s for s in SOURCES]
    if not force and target.exists() and all(f.stat().st_mtime <= target.stat().st_mtime for f in files):
        return target
    target.parent.mkdir(parents=True, exist_ok=True)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("gcc is required to build the oracle")
    tmp = target.with_suffix(f".{os.getpid()}.tmp")
    cmd = [cc, "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11",
           "-o", str(tmp), *map(str, files), "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"oracle build failed:\n{r.stderr}")
    os.replace(tmp, target)
    return target


class Oracle:
    """ctypes view of one compiled oracle library."""

    def __init__(self, path: Path | None = None):
        path = Path(path) if path else build()
        L = C.CDLL(str(path))
        vp, i32, d = C.c_void_p, C.c_int32, C.c_double
        L.orc_round.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, d, d, d, d, vp, vp,
                                C.POINTER(i32), C.POINTER(i32), vp, vp, vp, vp, C.POINTER(i32)]
        L.orc_round.restype = C.c_int
        L.orc_propagate.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, d, d, d, d,
                                    vp, vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), vp, vp]
        L.orc_propagate.restype = C.c_int
        L.orc_seq_propagate.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, d, d, d, d,
                                        vp, vp, C.POINTER(i32), C.POINTER(i32)]
        L.orc_seq_propagate.restype = C.c_int
        L.orc_normalise.argtypes = [i32, i32, vp, vp, vp, vp, vp, d, d]
        L.orc_normalise.restype = C.c_int
        self.L = L


_default = None


def _orc() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default


def _a(x, dt):
    return np.ascontiguousarray(x, dtype=dt)


def _p(x):
    return x.ctypes.data if x is not None else None


@dataclass
class PropResult:
    lb: np.ndarray
    ub: np.ndarray
    infeasible: int
    rounds: int
    status: int
    trace_lb: np.ndarray | None = None
    trace_ub: np.ndarray | None = None


@dataclass
class RoundResult:
    lb: np.ndarray
    ub: np.ndarray
    changed: int
    infeasible: int
    lb_tie: np.ndarray | None = None
    ub_tie: np.ndarray | None = None
    lb_err: np.ndarray | None = None
    ub_err: np.ndarray | None = None
    inf_tie: int = 0


def _csr(row_ptr, col, val):
    return _a(row_ptr, np.int64), _a(col, np.int32), _a(val, np.float64)


def _params(p):
    q = dict(DEFAULTS)
    if p:
        q.update(p)
    return q


def normalise(m, n, lb, ub, vartype, lhs, rhs, params=None, oracle: Oracle | None = None):
    """Input normalisation before round 1 (infinities, integer rounding)."""
    o = oracle or _orc()
    q = _params(params)
    lb, ub, lhs, rhs = (_a(x, np.float64).copy() for x in (lb, ub, lhs, rhs))
    vt = _a(vartype, np.uint8)
    rc = o.L.orc_normalise(m, n, _p(lb), _p(ub), _p(vt), _p(lhs), _p(rhs), q["eps_int"],
                           q["inf_threshold"])
    if rc != 0:
        raise ValueError(f"oracle rejected the input ({rc})")
    return lb, ub, lhs, rhs


def propagate(m, n, row_ptr, col, val, lb, ub, vartype, lhs, rhs, params=None, trace=False,
              oracle: Oracle | None = None) -> PropResult:
    """Alg. 2 to its fixed point (round-synchronous Jacobi rounds)."""
    o = oracle or _orc()
    q = _params(params)
    rp, ci, va = _csr(row_ptr, col, val)
    lb, ub, lhs, rhs = (_a(x, np.float64) for x in (lb, ub, lhs, rhs))
    vt = _a(vartype, np.uint8)
    lo, hi = np.empty(n), np.empty(n)
    inf, rounds, status = C.c_int32(), C.c_int32(), C.c_int32()
    tl = th = None
    if trace:
        tl = np.empty((max(q["max_rounds"], 1), n))
        th = np.empty((max(q["max_rounds"], 1), n))
    rc = o.L.orc_propagate(m, n, _p(rp), _p(ci), _p(va), _p(lb), _p(ub), _p(vt), _p(lhs), _p(rhs),
                           q["max_rounds"], q["eps_int"], q["tau_rel"], q["eps_feas"],
                           q["inf_threshold"], _p(lo), _p(hi), C.byref(inf), C.byref(rounds),
                           C.byref(status), _p(tl), _p(th))
    if rc != 0:
        raise ValueError(f"oracle rejected the input ({rc})")
    r = rounds.value
    return PropResult(lo, hi, inf.value, r, status.value,
                      tl[:r] if trace else None, th[:r] if trace else None)


def round_(m, n, row_ptr, col, val, L, U, vartype, lhs, rhs, params=None, analysis=False,
           oracle: Oracle | None = None) -> RoundResult:
    """One round from state (L, U); lhs/rhs/L/U must already be normalised.
    With analysis=True also returns the tie flags and error bounds that a
    parity test needs when another implementation sums in another order."""
    o = oracle or _orc()
    q = _params(params)
    rp, ci, va = _csr(row_ptr, col, val)
    L, U, lhs, rhs = (_a(x, np.float64) for x in (L, U, lhs, rhs))
    vt = _a(vartype, np.uint8)
    Ln, Un = np.empty(n), np.empty(n)
    ch, inf, itie = C.c_int32(), C.c_int32(), C.c_int32()
    lt = ut = le = ue = None
    if analysis:
        lt, ut = np.zeros(n, np.uint8), np.zeros(n, np.uint8)
        le, ue = np.zeros(n), np.zeros(n)
    rc = o.L.orc_round(m, n, _p(rp), _p(ci), _p(va), _p(L), _p(U), _p(vt), _p(lhs), _p(rhs),
                       q["eps_int"], q["tau_rel"], q["eps_feas"], q["inf_threshold"], _p(Ln), _p(Un),
                       C.byref(ch), C.byref(inf), _p(lt), _p(ut), _p(le), _p(ue),
                       C.byref(itie) if analysis else None)
    if rc != 0:
        raise ValueError(f"oracle round failed ({rc})")
    return RoundResult(Ln, Un, ch.value, inf.value, lt, ut, le, ue, itie.value)


def propagate_seq(m, n, row_ptr, col, val, lb, ub, vartype, lhs, rhs, params=None,
                  oracle: Oracle | None = None) -> PropResult:
    """Alg. 1: sequential propagation with constraint marking."""
    o = oracle or _orc()
    q = _params(params)
    rp, ci, va = _csr(row_ptr, col, val)
    lb, ub, lhs, rhs = (_a(x, np.float64) for x in (lb, ub, lhs, rhs))
    vt = _a(vartype, np.uint8)
    lo, hi = np.empty(n), np.empty(n)
    inf, rounds = C.c_int32(), C.c_int32()
    rc = o.L.orc_seq_propagate(m, n, _p(rp), _p(ci), _p(va), _p(lb), _p(ub), _p(vt), _p(lhs),
                               _p(rhs), q["max_rounds"], q["eps_int"], q["tau_rel"], q["eps_feas"],
                               q["inf_threshold"], _p(lo), _p(hi), C.byref(inf), C.byref(rounds))
    if rc != 0:
        raise ValueError(f"sequential oracle rejected the input ({rc})")
    return PropResult(lo, hi, inf.value, rounds.value, 0)


def propagate_instance(inst, params=None, trace=False, **kw) -> PropResult:
    return propagate(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, inst.lb, inst.ub,
                     inst.vartype, inst.lhs, inst.rhs, params, trace, **kw)


def propagate_seq_instance(inst, params=None, **kw) -> PropResult:
    return propagate_seq(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, inst.lb, inst.ub,
                         inst.vartype, inst.lhs, inst.rhs, params, **kw)
