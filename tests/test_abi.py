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


def test_rank_space_helper_matches_its_definition(lib):
    """gdi_rank_space: classes by colour, inside a class by splitmix64 of the vertex id; rank-space
    CSR with the weight sign in bit 31 (derived here independently of the library)."""
    import oracle
    from gdi_synth import splitmix64
    g = erdos_renyi(400, 0.04, 21, signed=True)
    rs = P.rank_space(g)
    color = oracle.greedy_color(g)
    vert = np.lexsort((splitmix64(np.arange(g.n, dtype=np.uint64)), color))
    assert np.array_equal(rs.vert_of, vert)
    counts = np.bincount(color)
    assert np.array_equal(rs.class_ptr, np.concatenate([[0], np.cumsum(counts[counts > 0])]))
    assert rs.max_class == counts.max() and rs.max_degree == np.diff(g.row_ptr).max()
    rank = np.empty(g.n, np.int64)
    rank[vert] = np.arange(g.n)
    for r in (0, 17, 399):
        v = vert[r]
        nb = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        w = g.w[g.row_ptr[v]:g.row_ptr[v + 1]]
        exp = rank[nb].astype(np.uint32) | np.where(w < 0, 0x80000000, 0).astype(np.uint32)
        assert np.array_equal(rs.col[rs.row_ptr[r]:rs.row_ptr[r + 1]], exp)
    bad = from_edges(3, np.array([0]), np.array([1]))
    bad.col = bad.col.copy()
    bad.col[0] = 0
    with pytest.raises(P.GdiError):
        P.rank_space(bad)


def test_table_helper_matches_the_oracle_table(lib):
    """gdi_build_table equals the oracle's table (Metropolis rows dE = 1.. while non-zero; paper rows
    thr(-1, 0, +1))."""
    import oracle
    tab, off, temp, mr = P.build_table(P.Schedule(sweeps=40, t0=12.0, t1=0.2))
    ecap, thr = oracle.table(oracle.METROPOLIS, 12.0, 0.2, 0, 0, 40)
    for s in range(40):
        row = thr[s, ecap + 1:]
        assert np.array_equal(tab[off[s]:off[s + 1]], row[row > 0].astype(np.uint32))
        assert temp[s] == np.float32(12.0 * (0.2 / 12.0) ** (s / 39))
    assert mr == max(np.diff(off))
    tab, off, temp, mr = P.build_table(P.Schedule(sweeps=10, mode=P.GDI_PAPER_PF, pf0=0.2, pf1=0.01))
    _, thr = oracle.table(oracle.PAPER_PF, 0, 0, 0.2, 0.01, 10)
    assert mr == 3 and np.array_equal(tab.reshape(10, 3), thr.astype(np.uint32))
