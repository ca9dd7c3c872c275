"""gdi_anneal_static, the allocation-free sweep, against gdi_anneal on the same inputs.

Callers whose device memory belongs to another allocator (or who must not grow their device
footprint while running) cannot let the library cudaMalloc; gdi_anneal_static keeps its scratch in a
static device array instead.  This test prepares the rank-space arrays the entry point takes as
input (in device memory owned by torch), calls it twice in a row -- sweeps [0, 12) from given spins,
then [12, 30) continuing in place -- and checks spins and G after each call against gdi_anneal's
grid-scale path (without repair) on the same graph, colouring, schedule and seed.  It is kept in a
file that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from gdi_synth import barabasi_albert

pytestmark = pytest.mark.gpu


def rank_space(g, color):
    """Rank order (colour asc, splitmix64(id) asc) and the rank-space CSR in the layout of
    include/gdi.h."""
    from gdi_synth import splitmix64
    vert = np.lexsort((splitmix64(np.arange(g.n, dtype=np.uint64)), color)).astype(np.int64)
    rank = np.empty(g.n, dtype=np.int64)
    rank[vert] = np.arange(g.n)
    deg = np.diff(g.row_ptr)
    row_ptr = np.zeros(g.n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(deg[vert])
    col = np.empty(g.nnz, dtype=np.uint32)
    for r in range(g.n):
        v = vert[r]
        nb = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        w = g.w[g.row_ptr[v]:g.row_ptr[v + 1]]
        col[row_ptr[r]:row_ptr[r + 1]] = rank[nb].astype(np.uint32) | np.where(w < 0, 0x80000000, 0).astype(np.uint32)
    counts = np.bincount(color)
    counts = counts[counts > 0]
    class_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return rank, row_ptr, col, class_ptr


def ragged_table(t0, t1, sweeps):
    """Metropolis rows: floor(exp(-dE/T_s) 2^32) for dE = 1.. while non-zero (oracle table)."""
    ecap, thr = oracle.table(oracle.METROPOLIS, t0, t1, 0, 0, sweeps)
    rows = [thr[s, ecap + 1:] for s in range(sweeps)]
    rows = [r[r > 0].astype(np.uint32) for r in rows]
    off = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    tab = np.concatenate(rows) if off[-1] else np.zeros(1, np.uint32)
    T = np.array([t0 * (t1 / t0) ** (s / (sweeps - 1)) for s in range(sweeps)], dtype=np.float32)
    return tab, off, T, max(len(r) for r in rows)


def test_static_entry_point_matches_gdi_anneal(gdi):
    import torch
    lib = gdi.load()
    g = barabasi_albert(30000, 5, 61)
    color = oracle.greedy_color(g)
    A, B, W, R, M, seed, t0, t1 = 1, 4, 128, 8, 30, 9, 12.0, 0.2
    rng = np.random.default_rng(5)
    half = np.where(np.arange(g.n) < g.n // 2, 1, -1).astype(np.int8)
    init = np.stack([rng.permutation(half) for _ in range(R)])

    # the existing entry point: grid-scale path, no repair, [0, 12) then [12, 30)
    ann = gdi.Annealer(g, A=A, B=B, W=W, replicas=R, color=color)
    ann.configure(path=gdi.GDI_PATH_GRID)
    sch = gdi.Schedule(sweeps=M, t0=t0, t1=t1)
    ann.anneal(sch, seed, init=init, last_sweep=12, flags=gdi.GDI_FLAG_NO_REPAIR)
    ref1_spins, ref1_G = ann.spins(), ann.results()["raw_G"][0].copy()
    ann.anneal(sch, seed, first_sweep=12, flags=gdi.GDI_FLAG_CONTINUE | gdi.GDI_FLAG_NO_REPAIR)
    ref2_spins, ref2_G = ann.spins(), ann.results()["raw_G"][0].copy()
    ann.close()

    # the allocation-free entry point on caller-owned device arrays
    rank, row_ptr, col, class_ptr = rank_space(g, color)
    tab, tab_off, temp, max_row = ragged_table(t0, t1, M)
    dev = torch.device("cuda")
    d_row = torch.from_numpy(row_ptr).to(dev)
    d_col = torch.from_numpy(col.view(np.int32)).to(dev)
    d_cls = torch.from_numpy(class_ptr).to(dev)
    d_tab = torch.from_numpy(tab.view(np.int32)).to(dev)
    d_off = torch.from_numpy(tab_off).to(dev)
    d_temp = torch.from_numpy(temp).to(dev)
    spins_rank = np.empty_like(init)
    spins_rank[:, rank] = init
    d_spins = torch.from_numpy(spins_rank).to(dev)
    d_G = torch.zeros(R, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    max_class = int(np.diff(class_ptr).max())
    max_degree = int(np.diff(g.row_ptr).max())

    def call(first, last):
        rc = lib.gdi_anneal_static(g.n, d_row.data_ptr(), d_col.data_ptr(), len(class_ptr) - 1,
                                   d_cls.data_ptr(), max_class, max_degree, A, B, W, 0,
                                   d_tab.data_ptr(), d_off.data_ptr(), d_temp.data_ptr(), max_row, M,
                                   first, last, seed, R, d_spins.data_ptr(), d_G.data_ptr(),
                                   C.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.gdi_last_error().decode()
        torch.cuda.synchronize()
        s = d_spins.cpu().numpy()
        return s[:, rank], d_G.cpu().numpy()

    s1, G1 = call(0, 12)
    assert np.array_equal(s1, ref1_spins)
    assert np.array_equal(G1, ref1_G)
    s2, G2 = call(12, 30)
    assert np.array_equal(s2, ref2_spins)
    assert np.array_equal(G2, ref2_G)

    # sizes beyond the static scratch are rejected without launching anything
    rc = lib.gdi_anneal_static((1 << 20) + 1, d_row.data_ptr(), d_col.data_ptr(), 1, d_cls.data_ptr(),
                               1, 1, A, B, W, 0, d_tab.data_ptr(), d_off.data_ptr(), d_temp.data_ptr(),
                               max_row, M, 0, 0, seed, R, d_spins.data_ptr(), d_G.data_ptr(), None)
    assert rc == -11
    assert b"static scratch" in lib.gdi_last_error()
