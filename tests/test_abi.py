"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/domprop.h declares (no GPU needed: only host-only helpers are
called)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def declared():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names |= set(re.findall(r"\b(dp_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2009_07785_gb300 import _build

    path = _build.build()
    return ctypes.CDLL(str(path))


def test_header_declares_entry_points():
    assert {"dp_create", "dp_matrix_load", "dp_propagate", "dp_destroy"} <= declared()


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in sorted(declared()) if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_2009_07785_gb300 as dp

    assert set(dp.SYMBOLS) == declared()
    for s in dp.SYMBOLS:
        assert hasattr(dp, s), s


def test_host_only_helpers(lib):
    import paper_2009_07785_gb300 as dp

    p = dp.dp_params_default()
    assert p.max_rounds == 100 and p.eps_int == 1e-6 and p.tau_rel == 1e-6
    assert p.eps_feas == 1e-6 and p.inf_threshold == 1e20
    assert dp.dp_strerror(dp.DP_ERR_BAD_CSR).startswith("malformed")
    assert dp.lib().dp_params_default(None) == dp.DP_ERR_INVALID_ARG


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_2009_07785_gb300 as dp

    monkeypatch.setattr(dp, "_lib", None)
    monkeypatch.setattr(dp, "LIB_PATH", tmp_path / "nope.so")
    with pytest.raises(RuntimeError):
        dp.lib()


def test_product_path_does_not_import_the_oracle():
    for f in list((ROOT / "paper_2009_07785_gb300").rglob("*.py")) + \
            list((ROOT / "paper_2009_07785_gb300" / "csrc").glob("*")):
        text = f.read_text(errors="ignore")
        assert "import oracle" not in text and "from oracle" not in text, f
        assert "dp_oracle" not in text, f


def test_generator_is_deterministic():
    import numpy as np

    from paper_2009_07785_gb300 import synth

    a, b = synth.tiny(), synth.tiny()
    for x, y in zip((a.row_ptr, a.col, a.val, a.lb, a.ub, a.lhs, a.rhs),
                    (b.row_ptr, b.col, b.val, b.lb, b.ub, b.lhs, b.rhs)):
        assert np.array_equal(x, y)
    lens = np.diff(a.row_ptr)
    assert a.m == 2000 and a.n == 1500 and lens.min() >= 2 and lens.max() <= 10
    for i in range(a.m):
        c = a.col[a.row_ptr[i]:a.row_ptr[i + 1]]
        assert np.unique(c).size == c.size
    ax = np.array([np.dot(a.val[a.row_ptr[i]:a.row_ptr[i + 1]], a.xstar[a.col[a.row_ptr[i]:a.row_ptr[i + 1]]])
                   for i in range(a.m)])
    assert np.all(ax <= a.rhs) and np.all(ax >= a.lhs)


def test_host_side_argument_checks(lib):
    """Entry points reject null handles before touching a device."""
    import paper_2009_07785_gb300 as dp

    L = dp.lib()
    assert L.dp_matrix_set_launch(None, 4) == dp.DP_ERR_INVALID_ARG
    best = dp.dp_tune_entry()
    assert L.dp_autotune(None, 0, 0, 0, None, None, None, None, None, None, None, None, None, 4,
                         None, 0, None, best) == dp.DP_ERR_INVALID_ARG
    assert L.dp_propagate_set(None, None, None, None, None, None, None, None, None, None, None,
                              None, None) == dp.DP_ERR_INVALID_ARG
    out = ctypes.c_void_p(1)
    for ipt in (3, 16, 4097):  # null context, and item counts outside 4..4096
        assert L.dp_matrix_load_merge(None, 0, 0, 0, None, None, None, ipt, None, None,
                                      ctypes.byref(out)) == dp.DP_ERR_INVALID_ARG
        assert out.value is None
    best = dp.dp_tune_entry()
    for nodes in (0, 4):  # null context, and no nodes
        assert L.dp_autotune_nodes(None, 0, 0, 0, None, None, None, nodes, None, None, None, None,
                                   None, None, None, 0, None, best) == dp.DP_ERR_INVALID_ARG


def test_profile_summaries_parse():
    """The bench reads k_round's DRAM traffic from the committed summaries:
    each names the kernel sources it was taken from and a byte count."""
    import bench

    files = sorted((Path(__file__).resolve().parents[1] / "profiles").glob("ncu_k_round_large_chunk*.md"))
    assert files
    for f in files:
        kv = bench.read_summary(f)
        assert re.fullmatch(r"[0-9a-f]{16}", kv["kernel_source_sha256_16"])
        assert float(kv["dram_bytes_per_launch_full_size"]) > 1e8
