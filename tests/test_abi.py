"""The C-ABI library builds, loads without a GPU, and exports every entry
point include/grb.h declares; the Python binding covers all of them."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "grb.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:grb_info|const char\*)\s+(grb_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_14211_gb300 import _build

    try:
        _build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    import paper_2509_14211_gb300 as grb

    return grb.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("grb_matrix_build_csr", "grb_vector_new", "grb_apply", "grb_mxv", "grb_ewise_add",
                 "grb_ewise_mult", "grb_reduce", "grb_wait", "grb_iterate_begin", "grb_iterate_end"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    import paper_2509_14211_gb300 as grb

    assert sorted(grb.symbols()) == _declared()
    for n in _declared():
        assert callable(getattr(grb, n))


def _declared_debug():
    with open(os.path.join(ROOT, "include", "grb_debug.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^grb_info\s+(grb_\w+)\s*\(", text, flags=re.M)))


def test_checked_build_exports_the_debug_calls(lib):
    """libgrb_checked.so (the same sources with -DGRB_CHECK_BOUNDS) exports
    everything include/grb.h and include/grb_debug.h declare; the release
    library exports none of the debug calls."""
    import ctypes

    from paper_2509_14211_gb300 import _build

    debug = _declared_debug()
    assert debug == ["grb_debug_check_csr", "grb_debug_set_col"]
    checked = ctypes.CDLL(_build.LIB_CHECKED)
    missing = [n for n in _declared() + debug if not hasattr(checked, n)]
    assert not missing, missing
    assert not [n for n in debug if hasattr(lib, n)]


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_2509_14211_gb300 as grb

    monkeypatch.setattr(grb, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(grb, "_lib", None)
    with pytest.raises(ImportError):
        grb.load()


def test_block_diagonal_edges_offsets_each_graph(lib):
    """The graph-batch input: per-graph edge lists stacked with each graph's
    vertex ids offset by the vertices before it; vptr marks the blocks (an
    edgeless member keeps its block)."""
    import numpy as np

    import paper_2509_14211_gb300 as grb

    graphs = [(3, [0, 1, 2], [1, 2, 0]), (2, [], []), (4, [3, 0], [0, 3])]
    n, src, dst, vptr = grb.block_diagonal_edges(graphs)
    assert n == 9 and vptr.tolist() == [0, 3, 5, 9]
    assert src.dtype == np.int32 and dst.dtype == np.int32
    assert src.tolist() == [0, 1, 2, 8, 5] and dst.tolist() == [1, 2, 0, 5, 8]
    for k in range(len(graphs)):
        lo, hi = vptr[k], vptr[k + 1]
        inside = (src >= lo) & (src < hi)
        assert np.all((dst[inside] >= lo) & (dst[inside] < hi))   # no edge leaves its block


def test_binding_constants_match_the_header():
    """The binding's size limits are the header's."""
    import paper_2509_14211_gb300 as grb

    with open(os.path.join(ROOT, "include", "grb.h")) as f:
        text = f.read()
    m = re.search(r"#define GRB_FUSED_INDEX_LIMIT (\d+)LL", text)
    assert m and int(m.group(1)) == grb.GRB_FUSED_INDEX_LIMIT == (1 << 31) - (1 << 24)
    m = re.search(r"#define GRB_HOT_BYTES_MAX (\d+)", text)
    assert m and int(m.group(1)) == grb.GRB_HOT_BYTES_MAX
