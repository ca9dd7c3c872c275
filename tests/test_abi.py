"""CPU checks of the C-ABI library: it builds, loads, exports every symbol include/gdi.h declares,
and rejects malformed graphs with the documented error codes (validation runs before any CUDA call)."""
import os
import re

import numpy as np
import pytest

import paper_1908_00210_gb300 as P
from gdi_synth import erdos_renyi, from_edges

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    P.build()
    return P.load()


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gdi_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_and_binding_agree(lib):
    from paper_1908_00210_gb300.learn import MPNN_EXPORTS
    decl = declared_functions()
    assert decl, "no declarations found"
    assert sorted(P.EXPORTS + MPNN_EXPORTS) == decl
    for name in decl:
        assert hasattr(lib, name), name


def test_error_strings(lib):
    for code in range(0, -12, -1):
        assert lib.gdi_strerror(code)
    assert lib.gdi_strerror(-99) == b"unknown error"


def _create(g, **kw):
    return P.Annealer(g, **kw)


def test_rejects_self_loop(lib):
    g = from_edges(4, np.array([0, 1]), np.array([1, 2]))
    col = g.col.copy()
    col[0] = 0   # vertex 0 -> 0
    g.col = col
    with pytest.raises(P.GdiError) as e:
        _create(g)
    assert e.value.code in (-3, -2)


def test_rejects_duplicate_and_asymmetric(lib):
    g = from_edges(4, np.array([0, 1, 2]), np.array([1, 2, 3]))
    bad = g.col.copy()
    # row 1 = [0, 2] -> [0, 0]: duplicate
    bad[g.row_ptr[1] + 1] = 0
    g2 = type(g)(n=g.n, row_ptr=g.row_ptr, col=bad, w=g.w)
    with pytest.raises(P.GdiError) as e:
        _create(g2)
    assert e.value.code == -4
    w = g.w.copy()
    w[0] = -1    # (0,1) weight -1 but (1,0) weight +1
    g3 = type(g)(n=g.n, row_ptr=g.row_ptr, col=g.col, w=w)
    with pytest.raises(P.GdiError) as e:
        _create(g3)
    assert e.value.code == -2


def test_rejects_bad_weights_and_colouring(lib):
    g = erdos_renyi(30, 0.2, 3)
    g.w = g.w * 2
    with pytest.raises(P.GdiError) as e:
        _create(g)
    assert e.value.code == -1
    g = erdos_renyi(30, 0.2, 3)
    with pytest.raises(P.GdiError) as e:
        _create(g, color=np.zeros(30, np.int32))
    assert e.value.code == -5


def test_rejects_bad_model(lib):
    g = erdos_renyi(30, 0.2, 3)
    for kw in (dict(B=0), dict(A=-1), dict(W=-2), dict(replicas=0)):
        with pytest.raises(P.GdiError) as e:
            _create(g, **kw)
        assert e.value.code == -1
