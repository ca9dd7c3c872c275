"""gdi_anneal_static, the allocation-free sweep, against gdi_anneal on the same inputs.

Some callers cannot let a library call cudaMalloc while they run: code whose device memory belongs
to another allocator (a framework's caching pool or a fixed arena), or a process that must not grow
its device footprint after start-up.  gdi_anneal_static keeps its scratch in a static device array
instead.  These tests build the rank-space arrays and the threshold table with the library's own
host helpers (gdi_rank_space, gdi_build_table), put them in device memory owned by torch, call the
entry point twice in a row -- sweeps [0, 12) from given spins, then [12, 30) continuing in place --
and check spins and G after each call against gdi_anneal's grid-scale path (without repair) on the
same graph, colouring, schedule and seed: every sorted-window size class (W = 32, 64, 256), the
tabulated-window kernel (W = 300), 3 and 8 replicas, and graphs with 6 and with more colour
classes.  Inputs whose sizes the caller understates are rejected by the input checks before any
sweep work.  The file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from gdi_synth import barabasi_albert, erdos_renyi

pytestmark = pytest.mark.gpu

M, SEED, T0, T1, A, B = 30, 9, 12.0, 0.2, 1, 4
_GRAPHS = {}


def _graph(kind):
    if kind not in _GRAPHS:
        _GRAPHS[kind] = barabasi_albert(30000, 5, 61) if kind == "ba" else erdos_renyi(20000, 16 / 19999, 62)
    return _GRAPHS[kind]


class _Static:
    """Device copies of the rank-space graph and table, and the entry point called on them."""

    def __init__(self, gdi, g, W, R):
        import torch
        self.lib = gdi.load()
        self.rs = gdi.rank_space(g)
        self.tab, self.off, self.temp, self.max_row = gdi.build_table(gdi.Schedule(sweeps=M, t0=T0, t1=T1))
        dev = torch.device("cuda")
        self.d_row = torch.from_numpy(self.rs.row_ptr).to(dev)
        self.d_col = torch.from_numpy(self.rs.col.view(np.int32)).to(dev)
        self.d_cls = torch.from_numpy(self.rs.class_ptr).to(dev)
        self.d_tab = torch.from_numpy(self.tab.view(np.int32)).to(dev)
        self.d_off = torch.from_numpy(self.off).to(dev)
        self.d_temp = torch.from_numpy(self.temp).to(dev)
        self.d_G = torch.zeros(R, dtype=torch.int32, device=dev)
        self.d_status = torch.full((1,), 12345, dtype=torch.int32, device=dev)
        self.n, self.W, self.R = g.n, W, R

    def load_spins(self, spins_orig):
        import torch
        s = np.empty_like(spins_orig)
        s[:, self.rs.rank_of] = spins_orig
        self.d_spins = torch.from_numpy(s).to("cuda")

    def call(self, first, last, max_class=None, max_row=None, col=None):
        import torch
        stream = torch.cuda.current_stream()
        rc = self.lib.gdi_anneal_static(
            self.n, self.d_row.data_ptr(), (col if col is not None else self.d_col).data_ptr(),
            len(self.rs.class_ptr) - 1, self.d_cls.data_ptr(),
            self.rs.max_class if max_class is None else max_class, self.rs.max_degree, A, B, self.W, 0,
            self.d_tab.data_ptr(), self.d_off.data_ptr(), self.d_temp.data_ptr(),
            self.max_row if max_row is None else max_row, M, first, last, SEED, self.R,
            self.d_spins.data_ptr(), self.d_G.data_ptr(), C.c_void_p(stream.cuda_stream))
        assert rc == 0, self.lib.gdi_last_error().decode()
        assert self.lib.gdi_anneal_static_status(self.d_status.data_ptr(), C.c_void_p(stream.cuda_stream)) == 0
        torch.cuda.synchronize()
        s = self.d_spins.cpu().numpy()
        return s[:, self.rs.rank_of], self.d_G.cpu().numpy(), int(self.d_status.cpu()[0])


def _init(g, R):
    rng = np.random.default_rng(5)
    half = np.where(np.arange(g.n) < g.n // 2, 1, -1).astype(np.int8)
    return np.stack([rng.permutation(half) for _ in range(R)])


@pytest.mark.parametrize("kind", ["ba", "er"])
@pytest.mark.parametrize("W", [32, 64, 256, 300])
@pytest.mark.parametrize("R", [3, 8])
def test_static_entry_point_matches_gdi_anneal(gdi, kind, W, R):
    g = _graph(kind)
    init = _init(g, R)
    # the existing entry point: grid-scale path, no repair, [0, 12) then [12, 30)
    ann = gdi.Annealer(g, A=A, B=B, W=W, replicas=R)
    ann.configure(path=gdi.GDI_PATH_GRID)
    sch = gdi.Schedule(sweeps=M, t0=T0, t1=T1)
    ann.anneal(sch, SEED, init=init, last_sweep=12, flags=gdi.GDI_FLAG_NO_REPAIR)
    ref1_spins, ref1_G = ann.spins(), ann.results()["raw_G"][0].copy()
    ann.anneal(sch, SEED, first_sweep=12, flags=gdi.GDI_FLAG_CONTINUE | gdi.GDI_FLAG_NO_REPAIR)
    ref2_spins, ref2_G = ann.spins(), ann.results()["raw_G"][0].copy()
    ncls = int(ann.info()["num_classes"][0])
    ann.close()

    st = _Static(gdi, g, W, R)
    assert len(st.rs.class_ptr) - 1 == ncls and ncls >= (6 if kind == "ba" else 7)
    st.load_spins(init)
    s1, G1, status = st.call(0, 12)
    assert status == 0
    assert np.array_equal(s1, ref1_spins)
    assert np.array_equal(G1, ref1_G)
    s2, G2, status = st.call(12, 30)
    assert status == 0
    assert np.array_equal(s2, ref2_spins)
    assert np.array_equal(G2, ref2_G)


def test_static_rejects_understated_sizes(gdi):
    """Sizes the caller understates, or a column outside the graph, are caught by the input checks:
    the status says GDI_ERR_INVALID_ARG, no sweep runs (the spins stay as they were), and the next
    correct call works."""
    import torch
    g = _graph("ba")
    R, W = 8, 32
    st = _Static(gdi, g, W, R)
    init = _init(g, R)
    st.load_spins(init)
    s, _, status = st.call(0, 12, max_class=W)              # one window per block: far too few
    assert status == -1 and np.array_equal(s, init)
    s, _, status = st.call(0, 12, max_row=st.max_row // 2)   # table rows longer than max_row
    assert status == -1 and np.array_equal(s, init)
    bad = st.d_col.clone()
    bad[7] = g.n + 5                                        # a neighbour rank outside [0, n)
    s, _, status = st.call(0, 12, col=bad)
    assert status == -1 and np.array_equal(s, init)
    s, _, status = st.call(0, 12)
    assert status == 0 and not np.array_equal(s, init)


def test_static_rejects_sizes_beyond_the_scratch(gdi):
    """Sizes beyond the static scratch are rejected on the host, without launching anything."""
    lib = gdi.load()
    rc = lib.gdi_anneal_static((1 << 20) + 1, 8, 8, 1, 8, 1, 1, A, B, 32, 0, 8, 8, 8, 1, M, 0, 0, SEED,
                               8, 8, 8, None)
    assert rc == -11
    assert b"static scratch" in lib.gdi_last_error()
    rc = lib.gdi_anneal_static(1000, 8, 8, 1, 8, 1000, 1, A, B, 32, 0, 8, 8, 8, 1, M, 0, 0, SEED,
                               9, 8, 8, None)
    assert rc == -11 and b"replicas" in lib.gdi_last_error()
