"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit-exact.

Compared after every sweep: the state digest, G and the cut; at the end: raw/final G, raw/final
cut and every spin.  Inputs are seeded synthetic graphs shaped like the paper's workloads.
"""
import numpy as np
import pytest

import oracle
from gdi_synth import (barabasi_albert, batch_union, er_batch, erdos_renyi, from_edges,
                       random_geometric, star_graph, torus2d)

pytestmark = pytest.mark.gpu


def run_both(gdi, g, *, A, B, W, sweeps, t0, t1, seed, replicas=1, mode=0, pf0=0.2, pf1=0.01,
             color=None, init=None, first_sweep=0, last_sweep=0, repair=True, trace=True):
    flags = (gdi.GDI_FLAG_TRACE if trace else 0) | (0 if repair else gdi.GDI_FLAG_NO_REPAIR)
    ann = gdi.Annealer(g, A=A, B=B, W=W, replicas=replicas, color=color)
    sch = gdi.Schedule(sweeps=sweeps, t0=t0, t1=t1, mode=mode, pf0=pf0, pf1=pf1)
    ann.anneal(sch, seed, init=init, flags=flags, first_sweep=first_sweep, last_sweep=last_sweep)
    res = ann.results()
    spins = ann.spins()
    tr = ann.trace() if trace else None
    ref = oracle.anneal(g, A=A, B=B, W=W, mode=mode, t0=t0, t1=t1, pf0=pf0, pf1=pf1, sweeps=sweeps,
                        seed=seed, replicas=replicas, color=color, init=init, first_sweep=first_sweep,
                        last_sweep=last_sweep, trace=trace, repair=repair)
    ann.close()
    return res, spins, tr, ref


def assert_parity(res, spins, tr, ref, s_lo=0, s_hi=None):
    if tr is not None:
        d, G, c = tr
        sl = slice(s_lo, s_hi)
        for r in range(ref.digest.shape[0]):
            bad = np.nonzero((d[r, sl] != ref.digest[r, sl]) | (G[r, sl] != ref.G_trace[r, sl]) |
                             (c[r, sl] != ref.cut_trace[r, sl]))[0]
            assert bad.size == 0, f"replica {r}: first mismatch at sweep {s_lo + bad[0]}: " \
                f"G {G[r, s_lo + bad[0]]} vs {ref.G_trace[r, s_lo + bad[0]]}, " \
                f"cut {c[r, s_lo + bad[0]]} vs {ref.cut_trace[r, s_lo + bad[0]]}"
    assert np.array_equal(res["raw_G"][0], ref.raw_G)
    assert np.array_equal(res["final_G"][0], ref.final_G)
    assert np.array_equal(res["raw_cut"][0], ref.raw_cut)
    assert np.array_equal(res["final_cut"][0], ref.final_cut)
    assert np.array_equal(spins, ref.spins)


def test_er800_full_config(gdi):
    """ER n=800 p=0.06 (unit weights, greedy colouring), W=64, Metropolis 3.0 -> 0.05 in units of
    B, 1000 sweeps, seed 1, one replica: every sweep bit-exact."""
    g = erdos_renyi(800, 0.06, 1001)
    out = run_both(gdi, g, A=1, B=4, W=64, sweeps=1000, t0=12.0, t1=0.2, seed=1)
    assert_parity(*out)


def test_torus_replicas_prefix(gdi):
    """Torus 100x100 with +-1 weights, checkerboard, W=1024, all 64 replicas for the first 40
    sweeps of the 5000-sweep schedule (repair on the partial state)."""
    g = torus2d(100, 2002)
    out = run_both(gdi, g, A=1, B=4, W=1024, sweeps=5000, t0=12.0, t1=0.2, seed=7, replicas=64,
                   color=g.color, last_sweep=40)
    assert_parity(*out, s_lo=0, s_hi=40)


def test_batched_er_instances(gdi):
    """24 ER instances of mixed size, density and weights (one replica each), one launch."""
    gs = er_batch(24, 3000, n_lo=200, n_hi=700)
    inst_ptr, u = batch_union(gs)
    A, B, W, M, t0, t1, seed = 1, 4, 256, 150, 12.0, 0.2, 99
    ann = gdi.Annealer(u, A=A, B=B, W=W, replicas=1, inst_ptr=inst_ptr)
    ann.anneal(gdi.Schedule(sweeps=M, t0=t0, t1=t1), seed, flags=gdi.GDI_FLAG_TRACE)
    res = ann.results()
    spins = ann.spins()
    d, G, c = ann.trace()
    for q, g in enumerate(gs):
        ref = oracle.anneal(g, A=A, B=B, W=W, t0=t0, t1=t1, sweeps=M, seed=seed, instance=q)
        assert np.array_equal(d[q], ref.digest[0]), f"instance {q}"
        assert np.array_equal(G[q], ref.G_trace[0])
        assert res["final_cut"][q, 0] == ref.final_cut[0]
        assert res["final_G"][q, 0] == ref.final_G[0]
        assert np.array_equal(spins[0, inst_ptr[q]:inst_ptr[q + 1]], ref.spins[0])
    ann.close()


@pytest.mark.parametrize("W", [1, 7, 0])
def test_window_sizes(gdi, W):
    g = erdos_renyi(300, 0.05, 77, signed=True)
    out = run_both(gdi, g, A=1, B=4, W=W, sweeps=60, t0=12.0, t1=0.2, seed=5, replicas=3)
    assert_parity(*out)


def test_paper_pf_mode(gdi):
    g = erdos_renyi(500, 0.02, 55)
    out = run_both(gdi, g, A=2, B=1, W=32, sweeps=200, t0=1, t1=1, seed=11, mode=1, pf0=0.2,
                   pf1=0.0002, replicas=2)
    assert_parity(*out)


def test_no_balance_term(gdi):
    g = random_geometric(400, 0.08, 3)
    out = run_both(gdi, g, A=0, B=3, W=0, sweeps=50, t0=9.0, t1=0.15, seed=4)
    assert_parity(*out)


@pytest.mark.parametrize("case", ["n2", "odd", "isolated", "star", "one_class", "negative"])
def test_edge_cases(gdi, case):
    if case == "n2":
        g = from_edges(2, np.array([0]), np.array([1]))
    elif case == "odd":
        g = erdos_renyi(101, 0.08, 12)
    elif case == "isolated":
        g = from_edges(50, np.array([0, 1, 2, 10]), np.array([1, 2, 3, 11]))
    elif case == "star":
        g = star_graph(601)          # hub degree 600 >> W
    elif case == "one_class":
        g = from_edges(9, np.zeros(0), np.zeros(0))
    else:
        g = erdos_renyi(200, 0.05, 13)
        g.w = -g.w
    out = run_both(gdi, g, A=1, B=4, W=16, sweeps=40, t0=12.0, t1=0.2, seed=3, replicas=2)
    assert_parity(*out)


def test_bad_start_exact_fallback(gdi):
    """All spins start at +1 (G = n): the first windows flip thousands of spins at once, which takes
    the exact counting path of the window selection instead of the shared-memory histogram."""
    g = barabasi_albert(10000, 5, 8)
    init = np.ones((1, g.n), dtype=np.int8)
    out = run_both(gdi, g, A=1, B=4, W=0, sweeps=6, t0=12.0, t1=0.2, seed=2, init=init)
    assert_parity(*out)


def test_resume_continue(gdi):
    """Anneal sweeps [0, 30) then [30, 80) with GDI_FLAG_CONTINUE == one call over [0, 80)."""
    g = erdos_renyi(400, 0.03, 31)
    sch = gdi.Schedule(sweeps=80, t0=12.0, t1=0.2)
    a = gdi.Annealer(g, A=1, B=4, W=32, replicas=2)
    a.anneal(sch, 8, last_sweep=30, flags=gdi.GDI_FLAG_NO_REPAIR)
    a.anneal(sch, 8, first_sweep=30, flags=gdi.GDI_FLAG_CONTINUE)
    got = a.spins()
    ref = oracle.anneal(g, A=1, B=4, W=32, t0=12.0, t1=0.2, sweeps=80, seed=8, replicas=2)
    assert np.array_equal(got, ref.spins)
    a.close()


def test_user_init_spins(gdi):
    g = erdos_renyi(333, 0.04, 41)
    rng = np.random.default_rng(0)
    init = np.where(rng.random((2, g.n)) < 0.5, 1, -1).astype(np.int8)
    out = run_both(gdi, g, A=1, B=4, W=64, sweeps=30, t0=12.0, t1=0.2, seed=6, replicas=2, init=init)
    assert_parity(*out)


@pytest.mark.parametrize("W,mode,A", [(64, 0, 1), (1, 0, 1), (0, 1, 2), (16, 1, 1)])
def test_standard_mode_matches_stale_oracle(gdi, W, mode, A):
    """Algorithm 2 (GDI_FLAG_STANDARD): every spin reads all n spins for the balance term and the
    spins of a window decide on the window-start state; bit-exact to the oracle's stale reading,
    in both table modes, for one spin per window and for whole classes."""
    g = erdos_renyi(700, 0.03, 77, signed=True)
    ann = gdi.Annealer(g, A=A, B=4, W=W, replicas=3)
    ann.configure(path=gdi.GDI_PATH_CTA)
    sch = gdi.Schedule(sweeps=60, t0=12.0, t1=0.2, mode=mode, pf0=0.2, pf1=0.001)
    ann.anneal(sch, 9, flags=gdi.GDI_FLAG_TRACE | gdi.GDI_FLAG_STANDARD)
    res, spins, tr = ann.results(), ann.spins(), ann.trace()
    ann.close()
    ref = oracle.anneal(g, A=A, B=4, W=W, mode=mode, t0=12.0, t1=0.2, pf0=0.2, pf1=0.001, sweeps=60,
                        seed=9, replicas=3, stale=True)
    assert_parity(res, spins, tr, ref)


def test_standard_mode_rejected_on_grid_path(gdi):
    g = erdos_renyi(300, 0.05, 78)
    ann = gdi.Annealer(g, A=1, B=4, W=16, replicas=1)
    ann.configure(path=gdi.GDI_PATH_GRID)
    with pytest.raises(gdi.GdiError):
        ann.anneal(gdi.Schedule(sweeps=4), 1, flags=gdi.GDI_FLAG_STANDARD)
    ann.close()


@pytest.mark.parametrize("W", [4, 8, 32, 64, 256])
def test_cta_sorted_walk_and_ordered_tail(gdi, W):
    """CTA-resident sorted kernel: one-sided starts (all +1, all -1) make G leave the stage maps'
    lattice in the first sweeps, so the walk stops at a window and the rest of the class replays in
    rank order; W = 4 gives classes of 200 windows (more than the walk keeps), replayed in order
    throughout.  Bit-exact to the oracle after every sweep."""
    g = torus2d(40, 45)
    init = np.stack([np.ones(g.n), -np.ones(g.n),
                     np.where(np.arange(g.n) % 3 == 0, -1, 1)]).astype(np.int8)
    kw = dict(A=1, B=4, W=W, t0=2.0, t1=0.2, sweeps=12, seed=17, color=g.color)
    ann = gdi.Annealer(g, A=1, B=4, W=W, replicas=3, color=g.color)
    ann.configure(path=gdi.GDI_PATH_CTA)
    ann.anneal(gdi.Schedule(sweeps=12, t0=2.0, t1=0.2), 17, init=init, flags=gdi.GDI_FLAG_TRACE)
    res, spins, tr = ann.results(), ann.spins(), ann.trace()
    assert ann.last_launch()["path"] == gdi.GDI_PATH_CTA
    ann.close()
    ref = oracle.anneal(g, replicas=3, init=init, **kw)
    assert_parity(res, spins, tr, ref)


def test_cta_sorted_32bit_columns(gdi):
    """An instance above 32,767 vertices on the CTA-resident sorted kernel: the neighbour sums read
    the 32-bit columns (smaller instances read the 16-bit copy)."""
    g = barabasi_albert(40000, 5, 47)
    kw = dict(A=1, B=4, W=64, t0=12.0, t1=0.2, sweeps=6, seed=23)
    ann = gdi.Annealer(g, A=1, B=4, W=64, replicas=2)
    ann.configure(path=gdi.GDI_PATH_CTA)
    ann.anneal(gdi.Schedule(sweeps=6, t0=12.0, t1=0.2), 23, flags=gdi.GDI_FLAG_TRACE)
    res, spins, tr = ann.results(), ann.spins(), ann.trace()
    assert ann.last_launch()["path"] == gdi.GDI_PATH_CTA
    ann.close()
    ref = oracle.anneal(g, replicas=2, **kw)
    assert_parity(res, spins, tr, ref)
