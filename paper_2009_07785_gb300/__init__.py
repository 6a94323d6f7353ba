"""GB300 domain propagation (arXiv 2009.07785) -- Python binding of libdomprop.

Thin ctypes marshalling over the C ABI declared in ``include/domprop.h``; the
functions keep the C names.  Every step of the propagation runs in the CUDA
library: if ``_lib/libdomprop.so`` is missing this module raises instead of
falling back to anything else.

Inputs may be numpy arrays (host memory) or torch tensors (host or CUDA);
outputs are allocated on the same side as ``lb`` unless given.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_lib" / "libdomprop.so"

DP_OK = 0
DP_CAP_HIT = 1
DP_ERR_INVALID_ARG = -1
DP_ERR_BAD_CSR = -2
DP_ERR_NAN_INPUT = -3
DP_ERR_OOM = -4
DP_ERR_CUDA = -5
DP_ERR_TIMEOUT = -6

# exported symbols, in header order
SYMBOLS = ("dp_params_default", "dp_strerror", "dp_create", "dp_destroy", "dp_matrix_load",
           "dp_matrix_load_sides", "dp_matrix_load_merge", "dp_matrix_load_set",
           "dp_matrix_set_offsets", "dp_matrix_set_launch", "dp_matrix_set_compression",
           "dp_autotune", "dp_autotune_nodes", "dp_matrix_free", "dp_matrix_info", "dp_propagate",
           "dp_propagate_hostloop",
           "dp_propagate_noalloc", "dp_propagate_nodes", "dp_propagate_set",
           "dp_propagate_persistent", "dp_propagate_nodes_persistent",
           "dp_propagate_set_persistent",
           "dp_propagate_nodes_hostloop", "dp_server_create", "dp_server_add_matrix",
           "dp_server_submit", "dp_server_poll", "dp_server_stats_get", "dp_server_clock_us",
           "dp_server_destroy", "dp_ctx_set_wait_limit", "dp_debug_fail_alloc",
           "dp_debug_live_allocs", "dp_matrix_access_floor")


class dp_params(C.Structure):
    _fields_ = [("max_rounds", C.c_int32), ("reserved0", C.c_int32), ("eps_int", C.c_double),
                ("tau_rel", C.c_double), ("eps_feas", C.c_double), ("inf_threshold", C.c_double)]


class dp_tune_entry(C.Structure):
    _fields_ = [("chunk", C.c_int32), ("round_warps", C.c_int32), ("us_per_round", C.c_float),
                ("reserved", C.c_int32)]


class dp_server_config(C.Structure):
    _fields_ = [("slots", C.c_int32), ("reserved0", C.c_int32), ("mem_budget", C.c_int64),
                ("params", dp_params)]


class dp_completion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("status", C.c_int32), ("infeasible", C.c_int32),
                ("rounds", C.c_int32), ("matrix", C.c_int32), ("arrival_us", C.c_double),
                ("done_us", C.c_double)]


class dp_server_stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in
                ("submitted", "completed", "in_system", "rounds", "slot_rounds", "admissions",
                 "max_active_slots", "workspaces_allocated", "evictions", "device_bytes")]


_lib = None


def lib() -> C.CDLL:
    """Loads libdomprop.so (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(str(LIB_PATH))
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)
    L.dp_params_default.argtypes = [C.POINTER(dp_params)]
    L.dp_params_default.restype = C.c_int
    L.dp_strerror.argtypes = [C.c_int]
    L.dp_strerror.restype = C.c_char_p
    L.dp_create.argtypes = [C.POINTER(vp), C.c_int, vp]
    L.dp_create.restype = C.c_int
    L.dp_destroy.argtypes = [vp]
    L.dp_destroy.restype = None
    L.dp_matrix_load.argtypes = [vp, i32, i32, i64, vp, vp, vp, i32, C.POINTER(vp)]
    L.dp_matrix_load.restype = C.c_int
    L.dp_matrix_load_sides.argtypes = [vp, i32, i32, i64, vp, vp, vp, i32, vp, vp, C.POINTER(vp)]
    L.dp_matrix_load_sides.restype = C.c_int
    L.dp_matrix_load_merge.argtypes = [vp, i32, i32, i64, vp, vp, vp, i32, vp, vp, C.POINTER(vp)]
    L.dp_matrix_load_merge.restype = C.c_int
    L.dp_matrix_load_set.argtypes = [vp, i32, vp, vp, vp, vp, vp, i32, vp, vp, C.POINTER(vp)]
    L.dp_matrix_load_set.restype = C.c_int
    L.dp_matrix_set_offsets.argtypes = [vp, C.POINTER(i32), vp, vp]
    L.dp_matrix_set_offsets.restype = C.c_int
    L.dp_matrix_set_launch.argtypes = [vp, i32]
    L.dp_matrix_set_launch.restype = C.c_int
    L.dp_matrix_set_compression.argtypes = [vp, i32, C.POINTER(i32)]
    L.dp_matrix_set_compression.restype = C.c_int
    L.dp_autotune.argtypes = [vp, i32, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp,
                              C.POINTER(dp_params), i32, C.POINTER(dp_tune_entry), i32,
                              C.POINTER(i32), C.POINTER(dp_tune_entry)]
    L.dp_autotune.restype = C.c_int
    L.dp_autotune_nodes.argtypes = [vp, i32, i32, i64, vp, vp, vp, i32, vp, vp, vp, vp, vp,
                                    C.POINTER(dp_params), C.POINTER(dp_tune_entry), i32,
                                    C.POINTER(i32), C.POINTER(dp_tune_entry)]
    L.dp_autotune_nodes.restype = C.c_int
    L.dp_propagate_set.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.POINTER(dp_params), vp, vp, vp,
                                   vp, vp]
    L.dp_propagate_set.restype = C.c_int
    L.dp_propagate_set_persistent.argtypes = L.dp_propagate_set.argtypes
    L.dp_propagate_set_persistent.restype = C.c_int
    L.dp_propagate_persistent.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.POINTER(dp_params), vp,
                                          vp, C.POINTER(i32), C.POINTER(i32)]
    L.dp_propagate_persistent.restype = C.c_int
    L.dp_matrix_free.argtypes = [vp]
    L.dp_matrix_free.restype = None
    L.dp_matrix_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64),
                                 C.POINTER(i64), C.POINTER(i32)]
    L.dp_matrix_info.restype = C.c_int
    L.dp_propagate.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.POINTER(dp_params), vp, vp,
                               C.POINTER(i32), C.POINTER(i32)]
    L.dp_propagate.restype = C.c_int
    L.dp_propagate_hostloop.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.POINTER(dp_params), vp, vp,
                                        C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_float),
                                        C.POINTER(i32)]
    L.dp_propagate_hostloop.restype = C.c_int
    L.dp_matrix_access_floor.argtypes = [vp, vp, i32, C.POINTER(C.c_float)]
    L.dp_matrix_access_floor.restype = C.c_int
    L.dp_ctx_set_wait_limit.argtypes = [vp, i64]
    L.dp_ctx_set_wait_limit.restype = C.c_int
    L.dp_debug_fail_alloc.argtypes = [i32]
    L.dp_debug_fail_alloc.restype = C.c_int
    L.dp_debug_live_allocs.argtypes = []
    L.dp_debug_live_allocs.restype = i64
    L.dp_propagate_noalloc.argtypes = [C.c_int, vp, i32, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp,
                                       C.POINTER(dp_params), vp, vp, C.POINTER(i32),
                                       C.POINTER(i32)]
    L.dp_propagate_noalloc.restype = C.c_int
    L.dp_propagate_nodes.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, C.POINTER(dp_params), vp, vp,
                                     vp, vp, vp]
    L.dp_propagate_nodes.restype = C.c_int
    L.dp_propagate_nodes_persistent.argtypes = L.dp_propagate_nodes.argtypes
    L.dp_propagate_nodes_persistent.restype = C.c_int
    L.dp_propagate_nodes_hostloop.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp,
                                              C.POINTER(dp_params), vp, vp, vp, vp, vp,
                                              C.POINTER(C.c_float), C.POINTER(i32)]
    L.dp_propagate_nodes_hostloop.restype = C.c_int
    L.dp_server_create.argtypes = [vp, C.POINTER(dp_server_config), C.POINTER(vp)]
    L.dp_server_create.restype = C.c_int
    L.dp_server_add_matrix.argtypes = [vp, vp, vp, vp, vp, C.POINTER(i32)]
    L.dp_server_add_matrix.restype = C.c_int
    L.dp_server_submit.argtypes = [vp, i32, vp, vp, vp, vp, C.c_uint64, C.c_double]
    L.dp_server_submit.restype = C.c_int
    L.dp_server_poll.argtypes = [vp, C.POINTER(dp_completion), i32, C.POINTER(i32), i32]
    L.dp_server_poll.restype = C.c_int
    L.dp_server_stats_get.argtypes = [vp, C.POINTER(dp_server_stats)]
    L.dp_server_stats_get.restype = C.c_int
    L.dp_server_clock_us.argtypes = []
    L.dp_server_clock_us.restype = C.c_double
    L.dp_server_destroy.argtypes = [vp]
    L.dp_server_destroy.restype = C.c_int
    _lib = L
    return L


class DomPropError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {dp_strerror(code)} ({code})")
        self.code = code


def dp_strerror(code: int) -> str:
    return lib().dp_strerror(int(code)).decode()


def dp_params_default(**overrides) -> dp_params:
    p = dp_params()
    lib().dp_params_default(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise DomPropError(rc, where)
    return rc


def _ptr(x):
    """Raw address of a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


class Context:
    """A dp_ctx: one GPU and the stream all library work is issued on."""

    def __init__(self, device: int = 0, stream=None):
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        h = C.c_void_p()
        _check(lib().dp_create(C.byref(h), int(device), C.c_void_p(stream) if stream else None),
               "dp_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            lib().dp_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def dp_matrix_access_floor(ctx: Context, mat: Matrix, reps: int = 5) -> float:
    """Microseconds of the round's memory access pattern on this matrix
    without its arithmetic (fastest of `reps` launches)."""
    us = C.c_float()
    _check(lib().dp_matrix_access_floor(ctx.handle, mat.handle, int(reps), C.byref(us)),
           "dp_matrix_access_floor")
    return float(us.value)


def dp_ctx_set_wait_limit(ctx: Context, sleeps: int) -> None:
    """Bound (in ~64 ns sleeps; 0 = the default, about 2 s) on a persistent-
    loop block's wait at a grid barrier before DP_ERR_TIMEOUT."""
    _check(lib().dp_ctx_set_wait_limit(ctx.handle, int(sleeps)), "dp_ctx_set_wait_limit")


def dp_debug_fail_alloc(k: int) -> None:
    """Test hook: the k-th device allocation of the library from now on fails
    with DP_ERR_OOM (k = 0 disarms)."""
    _check(lib().dp_debug_fail_alloc(int(k)), "dp_debug_fail_alloc")


def dp_debug_live_allocs() -> int:
    """Device allocations the library holds now (process-wide)."""
    return int(lib().dp_debug_live_allocs())


def dp_create(device: int = 0, stream=None) -> Context:
    return Context(device, stream)


def dp_destroy(ctx: Context) -> None:
    ctx.close()


class Matrix:
    """A dp_matrix: a CSR constraint matrix resident on the GPU."""

    def __init__(self, ctx: Context, m: int, n: int, row_ptr, col_idx, val, chunk: int = 0,
                 lhs=None, rhs=None, merge_ipt: int | None = None):
        """lhs/rhs (optional, host): the row sides known at load time, used
        only to order rows by side pattern (dp_matrix_load_sides).  With
        merge_ipt > 0 the matrix gets the merge-path layout with that many
        items per thread (dp_matrix_load_merge; `chunk` is then unused)."""
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        h = C.c_void_p()
        nnz = int(row_ptr[-1]) if m > 0 else 0
        if merge_ipt is not None:
            if lhs is not None:
                lhs = np.ascontiguousarray(lhs, dtype=np.float64)
                rhs = np.ascontiguousarray(rhs, dtype=np.float64)
            _check(lib().dp_matrix_load_merge(ctx.handle, int(m), int(n), nnz, _ptr(row_ptr),
                                              _ptr(col_idx), _ptr(val), int(merge_ipt),
                                              _ptr(lhs) if lhs is not None else None,
                                              _ptr(rhs) if rhs is not None else None,
                                              C.byref(h)), "dp_matrix_load_merge")
        elif lhs is None and rhs is None:
            _check(lib().dp_matrix_load(ctx.handle, int(m), int(n), nnz, _ptr(row_ptr),
                                        _ptr(col_idx), _ptr(val), int(chunk), C.byref(h)),
                   "dp_matrix_load")
        else:
            lhs = np.ascontiguousarray(lhs, dtype=np.float64)
            rhs = np.ascontiguousarray(rhs, dtype=np.float64)
            _check(lib().dp_matrix_load_sides(ctx.handle, int(m), int(n), nnz, _ptr(row_ptr),
                                              _ptr(col_idx), _ptr(val), int(chunk), _ptr(lhs),
                                              _ptr(rhs), C.byref(h)), "dp_matrix_load_sides")
        self.handle = h
        self.ctx = ctx
        self.m, self.n = int(m), int(n)

    def set_launch(self, round_warps: int) -> None:
        """Warps per block of the round kernels (4 or 8)."""
        _check(lib().dp_matrix_set_launch(self.handle, int(round_warps)), "dp_matrix_set_launch")

    def set_compression(self, on: bool) -> bool:
        """Reads the int8 copy of small-integer coefficients (lossless) when
        on and available; returns whether it is active."""
        act = C.c_int32()
        _check(lib().dp_matrix_set_compression(self.handle, 1 if on else 0, C.byref(act)),
               "dp_matrix_set_compression")
        return bool(act.value)

    def info(self) -> dict:
        m, n, s = C.c_int32(), C.c_int32(), C.c_int32()
        nnz, pad = C.c_int64(), C.c_int64()
        _check(lib().dp_matrix_info(self.handle, C.byref(m), C.byref(n), C.byref(nnz),
                                    C.byref(pad), C.byref(s)), "dp_matrix_info")
        return {"m": m.value, "n": n.value, "nnz": nnz.value, "padded_slots": pad.value,
                "split_rows": s.value}

    def close(self):
        if self.handle:
            lib().dp_matrix_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def dp_matrix_set_launch(mat: Matrix, round_warps: int) -> None:
    mat.set_launch(round_warps)


def dp_matrix_set_compression(mat: Matrix, on: bool) -> bool:
    return mat.set_compression(on)


def dp_autotune(ctx: Context, m: int, n: int, row_ptr, col_idx, val, lb, ub, vartype, lhs, rhs,
                params: dp_params | None = None, rounds: int = 4) -> dict:
    """Times `rounds` rounds of the problem for each row split length and
    block shape; returns {"best": {...}, "entries": [...]}."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    ent = (dp_tune_entry * 16)()
    cnt = C.c_int32()
    best = dp_tune_entry()
    nnz = int(row_ptr[-1]) if m > 0 else 0
    _check(lib().dp_autotune(ctx.handle, int(m), int(n), nnz, _ptr(row_ptr), _ptr(col_idx),
                             _ptr(val), _ptr(lb), _ptr(ub), _ptr(vartype), _ptr(lhs), _ptr(rhs),
                             C.byref(params) if params is not None else None, int(rounds), ent,
                             16, C.byref(cnt), C.byref(best)), "dp_autotune")
    conv = lambda e: {"chunk": e.chunk, "round_warps": e.round_warps,
                      "us_per_round": e.us_per_round}
    return {"best": conv(best), "entries": [conv(ent[i]) for i in range(min(cnt.value, 16))]}


def dp_autotune_nodes(ctx: Context, m: int, n: int, row_ptr, col_idx, val, lb, ub, vartype,
                      lhs, rhs, params: dp_params | None = None) -> dict:
    """Times the batched propagation of the node bound vectors lb, ub
    ([nodes, n]) for each row split length; returns {"best": {...},
    "entries": [...]} as dp_autotune (round_warps 0)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    nodes = int(lb.shape[0])
    ent = (dp_tune_entry * 16)()
    cnt = C.c_int32()
    best = dp_tune_entry()
    nnz = int(row_ptr[-1]) if m > 0 else 0
    _check(lib().dp_autotune_nodes(ctx.handle, int(m), int(n), nnz, _ptr(row_ptr), _ptr(col_idx),
                                   _ptr(val), nodes, _ptr(lb), _ptr(ub), _ptr(vartype), _ptr(lhs),
                                   _ptr(rhs), C.byref(params) if params is not None else None,
                                   ent, 16, C.byref(cnt), C.byref(best)), "dp_autotune_nodes")
    conv = lambda e: {"chunk": e.chunk, "us_per_round": e.us_per_round}
    return {"best": conv(best), "entries": [conv(ent[i]) for i in range(min(cnt.value, 16))]}


class MatrixSet(Matrix):
    """A dp_matrix holding several independent problems (dp_matrix_load_set):
    their block-diagonal union, propagated per problem by dp_propagate_set.
    row_off / var_off give each problem's first row and variable."""

    def __init__(self, ctx: Context, problems, chunk: int = 0, sides: bool = False):
        """problems: sequence of (m, n, row_ptr, col_idx, val) or objects with
        those attributes (and lhs, rhs when sides=True)."""
        ps = [p if isinstance(p, tuple) else (p.m, p.n, p.row_ptr, p.col, p.val)
              for p in problems]
        k = len(ps)
        rp = [np.ascontiguousarray(p[2], dtype=np.int64) for p in ps]
        ci = [np.ascontiguousarray(p[3], dtype=np.int32) for p in ps]
        va = [np.ascontiguousarray(p[4], dtype=np.float64) for p in ps]
        m = np.asarray([p[0] for p in ps], dtype=np.int32)
        n = np.asarray([p[1] for p in ps], dtype=np.int32)
        P64, P32, PD = C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_double)
        rpa = (P64 * k)(*[a.ctypes.data_as(P64) for a in rp])
        cia = (P32 * k)(*[a.ctypes.data_as(P32) for a in ci])
        vaa = (PD * k)(*[a.ctypes.data_as(PD) for a in va])
        lh = rh = None
        keep = []
        if sides:
            ls = [np.ascontiguousarray(p.lhs, dtype=np.float64) for p in problems]
            rs = [np.ascontiguousarray(p.rhs, dtype=np.float64) for p in problems]
            keep = ls + rs
            lh = (PD * k)(*[a.ctypes.data_as(PD) for a in ls])
            rh = (PD * k)(*[a.ctypes.data_as(PD) for a in rs])
        h = C.c_void_p()
        _check(lib().dp_matrix_load_set(ctx.handle, k, m.ctypes.data, n.ctypes.data, rpa, cia, vaa,
                                        int(chunk), lh, rh, C.byref(h)), "dp_matrix_load_set")
        del keep
        self.handle = h
        self.ctx = ctx
        self.m, self.n = int(m.sum()), int(n.sum())
        self.count = k
        cnt = C.c_int32()
        self.row_off = np.zeros(k + 1, dtype=np.int32)
        self.var_off = np.zeros(k + 1, dtype=np.int32)
        _check(lib().dp_matrix_set_offsets(h, C.byref(cnt), self.row_off.ctypes.data,
                                           self.var_off.ctypes.data), "dp_matrix_set_offsets")


def dp_matrix_load_set(ctx: Context, problems, chunk: int = 0, sides: bool = False) -> MatrixSet:
    return MatrixSet(ctx, problems, chunk, sides)


def dp_matrix_set_offsets(mset: MatrixSet) -> tuple:
    return mset.row_off, mset.var_off


@dataclass
class SetResult:
    lb: object
    ub: object
    infeasible: np.ndarray
    rounds: np.ndarray
    cap_hit: np.ndarray
    status: int


def dp_propagate_set(ctx: Context, mset: MatrixSet, lb, ub, vartype, lhs, rhs,
                     params: dp_params | None = None, lb_out=None, ub_out=None) -> SetResult:
    """Propagates every problem of a set; arrays are the problems' arrays
    concatenated in problem order.  Per-problem flags and round counts."""
    return _set(ctx, mset, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out, False)


def dp_propagate_set_persistent(ctx: Context, mset: MatrixSet, lb, ub, vartype, lhs, rhs,
                                params: dp_params | None = None, lb_out=None,
                                ub_out=None) -> SetResult:
    """dp_propagate_set with the round loop in one persistent cooperative
    kernel; same results."""
    return _set(ctx, mset, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out, True)


def _set(ctx, mset, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out, persistent):
    if lb_out is None:
        lb_out = _like(lb, mset.n)
    if ub_out is None:
        ub_out = _like(lb, mset.n)
    k = max(getattr(mset, "count", 0), 1)  # a plain matrix is rejected by the library
    inf = np.zeros(k, dtype=np.int32)
    rounds = np.zeros(k, dtype=np.int32)
    cap = np.zeros(k, dtype=np.int32)
    name = "dp_propagate_set_persistent" if persistent else "dp_propagate_set"
    rc = _check(getattr(lib(), name)(ctx.handle, mset.handle, _ptr(lb), _ptr(ub), _ptr(vartype),
                                     _ptr(lhs), _ptr(rhs),
                                     C.byref(params) if params is not None else None,
                                     _ptr(lb_out), _ptr(ub_out), inf.ctypes.data,
                                     rounds.ctypes.data, cap.ctypes.data), name)
    return SetResult(lb_out, ub_out, inf, rounds, cap, rc)


def dp_matrix_load(ctx: Context, m: int, n: int, row_ptr, col_idx, val, chunk: int = 0) -> Matrix:
    return Matrix(ctx, m, n, row_ptr, col_idx, val, chunk)


def dp_matrix_load_sides(ctx: Context, m: int, n: int, row_ptr, col_idx, val, chunk: int,
                         lhs, rhs) -> Matrix:
    return Matrix(ctx, m, n, row_ptr, col_idx, val, chunk, lhs, rhs)


def dp_matrix_load_merge(ctx: Context, m: int, n: int, row_ptr, col_idx, val,
                         items_per_thread: int, lhs=None, rhs=None) -> Matrix:
    return Matrix(ctx, m, n, row_ptr, col_idx, val, lhs=lhs, rhs=rhs,
                  merge_ipt=items_per_thread)


def dp_matrix_free(mat: Matrix) -> None:
    mat.close()


def dp_matrix_info(mat: Matrix) -> dict:
    return mat.info()


@dataclass
class Result:
    lb: object
    ub: object
    infeasible: int
    rounds: int
    status: int  # DP_OK or DP_CAP_HIT
    kernel_ms: tuple | None = None        # host loop only: per-kernel totals
    kernel_launches: tuple | None = None  # host loop only: per-kernel counts


KERNELS = ("round", "combine", "cand_split", "cand_queue", "finish")


def _like(x, n):
    if isinstance(x, np.ndarray):
        return np.empty(n, dtype=np.float64)
    import torch
    return torch.empty(n, dtype=torch.float64, device=x.device)


def dp_propagate(ctx: Context, mat: Matrix, lb, ub, vartype, lhs, rhs, params: dp_params | None = None,
                 lb_out=None, ub_out=None) -> Result:
    """Runs round-synchronous propagation to its fixed point (or the cap)."""
    n = mat.n
    if lb_out is None:
        lb_out = _like(lb, n)
    if ub_out is None:
        ub_out = _like(lb, n)
    inf, rounds = C.c_int32(), C.c_int32()
    rc = _check(lib().dp_propagate(ctx.handle, mat.handle, _ptr(lb), _ptr(ub), _ptr(vartype),
                                   _ptr(lhs), _ptr(rhs), C.byref(params) if params is not None else None,
                                   _ptr(lb_out), _ptr(ub_out), C.byref(inf), C.byref(rounds)),
                "dp_propagate")
    return Result(lb_out, ub_out, inf.value, rounds.value, rc)


def dp_propagate_persistent(ctx: Context, mat: Matrix, lb, ub, vartype, lhs, rhs,
                            params: dp_params | None = None, lb_out=None, ub_out=None) -> Result:
    """Same as dp_propagate, with the round loop in one persistent
    (cooperative) kernel instead of the graph's WHILE node."""
    n = mat.n
    if lb_out is None:
        lb_out = _like(lb, n)
    if ub_out is None:
        ub_out = _like(lb, n)
    inf, rounds = C.c_int32(), C.c_int32()
    rc = _check(lib().dp_propagate_persistent(
        ctx.handle, mat.handle, _ptr(lb), _ptr(ub), _ptr(vartype), _ptr(lhs), _ptr(rhs),
        C.byref(params) if params is not None else None, _ptr(lb_out), _ptr(ub_out),
        C.byref(inf), C.byref(rounds)), "dp_propagate_persistent")
    return Result(lb_out, ub_out, inf.value, rounds.value, rc)


def dp_propagate_hostloop(ctx: Context, mat: Matrix, lb, ub, vartype, lhs, rhs,
                          params: dp_params | None = None, lb_out=None, ub_out=None,
                          timing: bool = True) -> Result:
    """Same result as dp_propagate, with the round loop on the host (one
    stream synchronisation per round) and per-kernel CUDA-event timings."""
    n = mat.n
    if lb_out is None:
        lb_out = _like(lb, n)
    if ub_out is None:
        ub_out = _like(lb, n)
    inf, rounds = C.c_int32(), C.c_int32()
    ms = (C.c_float * len(KERNELS))()
    cnt = (C.c_int32 * len(KERNELS))()
    rc = _check(lib().dp_propagate_hostloop(
        ctx.handle, mat.handle, _ptr(lb), _ptr(ub), _ptr(vartype), _ptr(lhs), _ptr(rhs),
        C.byref(params) if params is not None else None, _ptr(lb_out), _ptr(ub_out),
        C.byref(inf), C.byref(rounds), ms if timing else None, cnt), "dp_propagate_hostloop")
    return Result(lb_out, ub_out, inf.value, rounds.value, rc,
                  tuple(ms) if timing else None, tuple(cnt))


NOALLOC_MAX_VARS = 1 << 20


def dp_propagate_noalloc(device: int, stream, m: int, n: int, row_ptr, col_idx, val, lb, ub,
                         vartype, lhs, rhs, lb_out, ub_out,
                         params: dp_params | None = None) -> Result:
    """Allocation-free propagation over a CSR matrix and problem already in
    device memory (all array arguments are CUDA tensors; lb_out/ub_out are
    caller-allocated).  For callers that must not allocate device memory;
    its scratch is a fixed static device array (n <= NOALLOC_MAX_VARS)."""
    import torch

    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    m, n = int(m), int(n)
    want = torch.device("cuda", int(device))
    nnz = int(col_idx.numel()) if isinstance(col_idx, torch.Tensor) else -1
    spec = (("row_ptr", row_ptr, torch.int64, m + 1), ("col_idx", col_idx, torch.int32, nnz),
            ("val", val, torch.float64, nnz), ("lb", lb, torch.float64, n),
            ("ub", ub, torch.float64, n), ("vartype", vartype, torch.uint8, n),
            ("lhs", lhs, torch.float64, m), ("rhs", rhs, torch.float64, m),
            ("lb_out", lb_out, torch.float64, n), ("ub_out", ub_out, torch.float64, n))
    for name, t, dt, numel in spec:
        # the C entry point reads raw device pointers: the element type, length
        # and device must be right here, nothing converts them
        if not (isinstance(t, torch.Tensor) and t.device == want and t.dtype == dt
                and t.numel() == numel and t.is_contiguous()):
            raise DomPropError(DP_ERR_INVALID_ARG,
                               f"dp_propagate_noalloc: {name} must be a contiguous {dt} tensor "
                               f"of {numel} elements on {want}")
    inf, rounds = C.c_int32(), C.c_int32()
    rc = _check(lib().dp_propagate_noalloc(
        int(device), C.c_void_p(stream) if stream else None, int(m), int(n), nnz, _ptr(row_ptr),
        _ptr(col_idx), _ptr(val), _ptr(lb), _ptr(ub), _ptr(vartype), _ptr(lhs), _ptr(rhs),
        C.byref(params) if params is not None else None, _ptr(lb_out), _ptr(ub_out),
        C.byref(inf), C.byref(rounds)), "dp_propagate_noalloc")
    return Result(lb_out, ub_out, inf.value, rounds.value, rc)


@dataclass
class NodesResult:
    lb: object            # [count, n] bounds after each node's last round
    ub: object
    infeasible: np.ndarray  # int32 [count]
    rounds: np.ndarray      # int32 [count]
    cap_hit: np.ndarray     # int32 [count]: stopped by the round cap
    status: int             # DP_OK or DP_CAP_HIT (some node hit the cap)
    kernel_ms: tuple | None = None        # host loop only: per-stage totals
    kernel_launches: tuple | None = None  # host loop only: per-stage counts


NODE_STAGES = ("mark", "mark_split", "act", "combine", "cand_split", "finish")


def dp_propagate_nodes(ctx: Context, mat: Matrix, lb, ub, vartype, lhs, rhs,
                       params: dp_params | None = None, lb_out=None, ub_out=None) -> NodesResult:
    """Propagates a batch of branch-and-bound nodes over one matrix.  lb, ub
    are [count, n] (node-major; numpy or torch, host or CUDA); each node's
    result equals dp_propagate on that node alone."""
    return _nodes(ctx, mat, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out, None)


def dp_propagate_nodes_persistent(ctx: Context, mat: Matrix, lb, ub, vartype, lhs, rhs,
                                  params: dp_params | None = None, lb_out=None,
                                  ub_out=None) -> NodesResult:
    """dp_propagate_nodes with the round loop in one persistent cooperative
    kernel; same results."""
    return _nodes(ctx, mat, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out, "persistent")


def dp_propagate_nodes_hostloop(ctx: Context, mat: Matrix, lb, ub, vartype, lhs, rhs,
                                params: dp_params | None = None, lb_out=None,
                                ub_out=None) -> NodesResult:
    """dp_propagate_nodes with a host-driven round loop and per-stage
    CUDA-event timings (NodesResult.kernel_ms / kernel_launches, in the order
    of NODE_STAGES)."""
    return _nodes(ctx, mat, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out, "hostloop")


def _nodes(ctx, mat, lb, ub, vartype, lhs, rhs, params, lb_out, ub_out, mode):
    """mode: None (the graph), "hostloop" or "persistent"."""
    count = int(lb.shape[0]) if len(lb.shape) == 2 else 0
    if len(lb.shape) != 2 or tuple(ub.shape) != tuple(lb.shape) or int(lb.shape[1]) != mat.n:
        raise ValueError("lb and ub must both have shape [count, n]")
    if lb_out is None:
        lb_out = _like(lb, (count, mat.n))
    if ub_out is None:
        ub_out = _like(lb, (count, mat.n))
    inf = np.zeros(max(count, 1), dtype=np.int32)
    rounds = np.zeros(max(count, 1), dtype=np.int32)
    cap = np.zeros(max(count, 1), dtype=np.int32)
    args = (ctx.handle, mat.handle, count, _ptr(lb), _ptr(ub), _ptr(vartype), _ptr(lhs),
            _ptr(rhs), C.byref(params) if params is not None else None, _ptr(lb_out),
            _ptr(ub_out), inf.ctypes.data, rounds.ctypes.data, cap.ctypes.data)
    if mode == "hostloop":
        ms = (C.c_float * len(NODE_STAGES))()
        cnt = (C.c_int32 * len(NODE_STAGES))()
        rc = _check(lib().dp_propagate_nodes_hostloop(*args, ms, cnt),
                    "dp_propagate_nodes_hostloop")
        return NodesResult(lb_out, ub_out, inf[:count], rounds[:count], cap[:count], rc,
                           tuple(ms), tuple(cnt))
    name = "dp_propagate_nodes_persistent" if mode == "persistent" else "dp_propagate_nodes"
    rc = _check(getattr(lib(), name)(*args), name)
    return NodesResult(lb_out, ub_out, inf[:count], rounds[:count], cap[:count], rc)


# ------------------------------------------------------------------ serving --

class Server:
    """A dp_server: resident matrices and a request loop with continuous
    batching (see include/domprop.h).  Requests are numpy float64 host
    arrays; the binding keeps them alive until their completion is polled."""

    def __init__(self, ctx: Context, slots: int = 64, mem_budget: int = 0,
                 params: dp_params | None = None):
        cfg = dp_server_config()
        cfg.slots = int(slots)
        cfg.mem_budget = int(mem_budget)
        cfg.params = params if params is not None else dp_params_default()
        h = C.c_void_p()
        _check(lib().dp_server_create(ctx.handle, C.byref(cfg), C.byref(h)), "dp_server_create")
        self.handle = h
        self.ctx = ctx
        self._n = {}
        self._live = {}
        self._next_tag = 1

    def add_matrix(self, mat: Matrix, vartype, lhs, rhs) -> int:
        mid = C.c_int32()
        self._keep = getattr(self, "_keep", []) + [mat]
        _check(lib().dp_server_add_matrix(self.handle, mat.handle, _ptr(vartype), _ptr(lhs),
                                          _ptr(rhs), C.byref(mid)), "dp_server_add_matrix")
        self._n[mid.value] = mat.n
        return mid.value

    def submit(self, matrix_id: int, lb, ub, lb_out=None, ub_out=None, tag: int | None = None,
               arrival_us: float = 0.0) -> int:
        n = self._n.get(matrix_id, 0)  # an unknown id is rejected by the library
        lb = np.ascontiguousarray(lb, dtype=np.float64)
        ub = np.ascontiguousarray(ub, dtype=np.float64)
        if lb_out is None:
            lb_out = np.empty(n)
        if ub_out is None:
            ub_out = np.empty(n)
        if tag is None:
            tag = self._next_tag
            self._next_tag += 1
        _check(lib().dp_server_submit(self.handle, int(matrix_id), _ptr(lb), _ptr(ub),
                                      _ptr(lb_out), _ptr(ub_out), int(tag), float(arrival_us)),
               "dp_server_submit")
        self._live[int(tag)] = (lb, ub, lb_out, ub_out)
        return int(tag)

    def poll(self, max_count: int = 1024, wait_us: int = 0) -> list:
        buf = (dp_completion * max_count)()
        cnt = C.c_int32()
        _check(lib().dp_server_poll(self.handle, buf, max_count, C.byref(cnt), int(wait_us)),
               "dp_server_poll")
        out = []
        for i in range(cnt.value):
            c = buf[i]
            lb, ub, lo, hi = self._live.pop(int(c.tag))
            out.append({"tag": int(c.tag), "status": c.status, "infeasible": c.infeasible,
                        "rounds": c.rounds, "matrix": c.matrix, "arrival_us": c.arrival_us,
                        "done_us": c.done_us, "lb": lo, "ub": hi})
        return out

    def stats(self) -> dict:
        st = dp_server_stats()
        _check(lib().dp_server_stats_get(self.handle, C.byref(st)), "dp_server_stats_get")
        return {k: getattr(st, k) for k, _ in dp_server_stats._fields_}

    def close(self) -> int:
        rc = 0
        if self.handle:
            rc = lib().dp_server_destroy(self.handle)
            self.handle = None
        return rc

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def dp_server_create(ctx: Context, slots: int = 64, mem_budget: int = 0,
                     params: dp_params | None = None) -> Server:
    return Server(ctx, slots, mem_budget, params)


def dp_server_add_matrix(server: Server, mat: Matrix, vartype, lhs, rhs) -> int:
    return server.add_matrix(mat, vartype, lhs, rhs)


def dp_server_submit(server: Server, matrix_id: int, lb, ub, lb_out=None, ub_out=None,
                     tag: int | None = None, arrival_us: float = 0.0) -> int:
    return server.submit(matrix_id, lb, ub, lb_out, ub_out, tag, arrival_us)


def dp_server_poll(server: Server, max_count: int = 1024, wait_us: int = 0) -> list:
    return server.poll(max_count, wait_us)


def dp_server_stats_get(server: Server) -> dict:
    return server.stats()


def dp_server_clock_us() -> float:
    return lib().dp_server_clock_us()


def dp_server_destroy(server: Server) -> int:
    return server.close()
