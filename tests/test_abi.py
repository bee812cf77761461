"""The C-ABI library loads and exports every symbol include/xlb.h declares;
argument validation happens on the host before any CUDA call (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2311_16080_gb300 import build as B
from paper_2311_16080_gb300 import xlb as X


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(X.LIB_PATH):
        B.build()
    return X.load()


def _declared(repo_root):
    src = open(os.path.join(repo_root, "include", "xlb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xlb_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary(repo_root):
    names = _declared(repo_root)
    for n in ("xlb_create", "xlb_set_mask", "xlb_step", "xlb_macroscopic", "xlb_adjoint_step"):
        assert n in names


def test_every_declared_symbol_is_exported(lib, repo_root):
    for name in _declared(repo_root):
        assert hasattr(ctypes.CDLL(X.LIB_PATH), name), name
    assert set(_declared(repo_root)) <= set(X._PROTOS), "binding misses a declared entry point"


def test_invalid_arguments_rejected_on_host(lib):
    out = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(8, 8, 8)
    assert lib.xlb_create(ctypes.byref(out), 7, dims, 1.0, 1, 0, None) == X.XLB_ERR_ARG
    assert b"lattice" in lib.xlb_last_error(None)
    assert lib.xlb_create(ctypes.byref(out), 19, dims, 2.5, 1, 0, None) == X.XLB_ERR_ARG
    assert lib.xlb_create(ctypes.byref(out), 19, dims, 1.0, X.XLB_COLL_KBC, 0, None) == X.XLB_ERR_UNSUPPORTED
    assert lib.xlb_create(ctypes.byref(out), 9, dims, 1.0, 1, 0, None) == X.XLB_ERR_ARG  # D2Q9 needs nz = 1
    assert lib.xlb_create(ctypes.byref(out), 19, dims, 1.0, 1, 5, None) == X.XLB_ERR_ARG
    bad = (ctypes.c_int64 * 3)(0, 8, 8)
    assert lib.xlb_create(ctypes.byref(out), 19, bad, 1.0, 1, 0, None) == X.XLB_ERR_ARG
    assert out.value is None
    with pytest.raises(X.XlbError):
        X.xlb_create(27, (4, 4, 4), 1.0, X.XLB_COLL_BGK, 9)


def test_status_strings_and_host_helpers(lib):
    assert X.xlb_status_string(0) == "XLB_OK"
    assert X.xlb_status_string(5) == "XLB_ERR_TIMEOUT"
    # Eq. 4 with dt = 1: omega = 1 / (3 nu + 1/2)
    assert abs(X.xlb_omega_from_nu(0.1) - 1.25) < 1e-15
    X.xlb_destroy(None)


def test_lattice_table_matches_figure_1(lib):
    """The library's direction order (host call, no GPU) is Figure 1's, with
    the standard weights; it is the order xlb_set_wall_distances expects."""
    import os
    from paper_2311_16080_gb300 import xlb as X
    gold, cur = {}, None
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "lattice_velocities.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line.strip("[]")
            gold[cur] = []
        else:
            gold[cur].append(tuple(int(v) for v in line.split()))
    wsets = {9: {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}, 19: {0: 1 / 3, 1: 1 / 18, 2: 1 / 36},
             27: {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}}
    for q in (9, 19, 27):
        c, w = X.xlb_lattice_table(q)
        g = gold[f"D{2 if q == 9 else 3}Q{q}"]
        d = len(g[0])
        g = [(0,) * d] + g          # the rest velocity comes first
        assert [tuple(int(v) for v in row[:d]) for row in c] == g
        assert all(abs(w[i] - wsets[q][int((c[i] ** 2).sum())]) < 1e-16 for i in range(q))
    with pytest.raises(X.XlbError):
        X.xlb_lattice_table(15)
