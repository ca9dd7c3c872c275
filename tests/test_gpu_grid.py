"""GPU parity of the grid-scale path (one instance over every SM) against the CPU oracle."""
import numpy as np
import pytest

import oracle
from gdi_synth import barabasi_albert, erdos_renyi, torus2d

pytestmark = pytest.mark.gpu


def grid_vs_oracle(gdi, g, *, A=1, B=4, W=64, sweeps=30, t0=12.0, t1=0.2, seed=3, replicas=8,
                   last_sweep=0, init=None, color=None, mode=0, pf0=0.2, pf1=0.01, grid_limit=0,
                   repair=True):
    ann = gdi.Annealer(g, A=A, B=B, W=W, replicas=replicas, color=color)
    ann.configure(path=gdi.GDI_PATH_GRID, grid_limit=grid_limit)
    sch = gdi.Schedule(sweeps=sweeps, t0=t0, t1=t1, mode=mode, pf0=pf0, pf1=pf1)
    flags = gdi.GDI_FLAG_TRACE | (0 if repair else gdi.GDI_FLAG_NO_REPAIR)
    ann.anneal(sch, seed, init=init, last_sweep=last_sweep, flags=flags)
    res = ann.results()
    spins = ann.spins()
    d, G, c = ann.trace()
    launch = ann.last_launch()
    ann.close()
    ref = oracle.anneal(g, A=A, B=B, W=W, t0=t0, t1=t1, sweeps=sweeps, seed=seed, replicas=replicas,
                        last_sweep=last_sweep, init=init, color=color, mode=mode, pf0=pf0, pf1=pf1,
                        repair=repair)
    hi = last_sweep if last_sweep > 0 else sweeps
    for r in range(replicas):
        bad = np.nonzero((d[r, :hi] != ref.digest[r, :hi]) | (G[r, :hi] != ref.G_trace[r, :hi]) |
                         (c[r, :hi] != ref.cut_trace[r, :hi]))[0]
        assert bad.size == 0, f"replica {r}: first mismatch at sweep {bad[0]}: G {G[r, bad[0]]} vs " \
            f"{ref.G_trace[r, bad[0]]}, cut {c[r, bad[0]]} vs {ref.cut_trace[r, bad[0]]}"
    assert np.array_equal(res["raw_G"][0], ref.raw_G)
    assert np.array_equal(res["raw_cut"][0], ref.raw_cut)
    assert np.array_equal(res["final_G"][0], ref.final_G)
    assert np.array_equal(res["final_cut"][0], ref.final_cut)
    assert np.array_equal(spins, ref.spins)
    assert launch["path"] == gdi.GDI_PATH_GRID
    return launch


def test_grid_ba_small(gdi):
    g = barabasi_albert(20000, 5, 44)
    grid_vs_oracle(gdi, g, W=64, sweeps=25, replicas=8)


def test_grid_two_replica_groups_odd_n(gdi):
    g = erdos_renyi(9001, 0.001, 45, signed=True)
    grid_vs_oracle(gdi, g, W=256, sweeps=12, replicas=11)


def test_grid_torus_paper_mode(gdi):
    g = torus2d(60, 46)
    grid_vs_oracle(gdi, g, W=128, sweeps=40, replicas=3, color=g.color, mode=1, pf0=0.2, pf1=0.001)


def test_grid_few_blocks(gdi):
    """Fewer blocks than SMs: more windows per block, same results."""
    g = barabasi_albert(30000, 5, 47)
    grid_vs_oracle(gdi, g, W=128, sweeps=8, replicas=4, grid_limit=37)


def test_grid_bad_start_takes_exact_fallback(gdi):
    """All spins +1 (G = n): the block tables cannot cover the first classes, so the chain takes the
    exact fallback; results stay bit-exact."""
    g = barabasi_albert(20000, 5, 48)
    init = np.ones((2, g.n), dtype=np.int8)
    launch = grid_vs_oracle(gdi, g, W=64, sweeps=4, replicas=2, init=init)
    assert launch["fallbacks"] > 0


@pytest.mark.parametrize("W", [1, 3, 33, 200])
def test_grid_sorted_window_sizes(gdi, W):
    """Windows of 1 to 8 members per lane (and ragged last windows) on the sorted-window path."""
    g = erdos_renyi(12000, 0.0008, 50 + W, signed=True)
    grid_vs_oracle(gdi, g, W=W, sweeps=6, replicas=3)


def test_grid_sorted_far_from_class_start(gdi):
    """All spins +1 on 10^5 vertices: inside the first classes G moves by far more than the stored
    window values cover (|G - c| > 32000), so windows replay through the exact counting path."""
    g = barabasi_albert(100_000, 5, 51)
    init = np.ones((2, g.n), dtype=np.int8)
    launch = grid_vs_oracle(gdi, g, W=256, sweeps=2, replicas=2, init=init)
    assert launch["fallbacks"] > 0


@pytest.mark.parametrize("W", [300, 1024])
def test_grid_tabulated_large_windows(gdi, W):
    """W > 256 takes the tabulated-window path (histogram tables, chain blocks)."""
    g = barabasi_albert(20000, 5, 52)
    grid_vs_oracle(gdi, g, W=W, sweeps=8, replicas=5)


def test_grid_tabulated_bad_start(gdi):
    g = barabasi_albert(20000, 5, 53)
    init = np.ones((3, g.n), dtype=np.int8)
    launch = grid_vs_oracle(gdi, g, W=512, sweeps=3, replicas=3, init=init)
    assert launch["fallbacks"] > 0


def test_grid_ba_1m_first_sweeps(gdi):
    """The full-size workload (BA n = 10^6, m = 5, 8 replicas, W = 256, 500-sweep schedule), checked
    on its first 2 sweeps (then repaired) against the oracle."""
    g = barabasi_albert(1_000_000, 5, 4004)
    grid_vs_oracle(gdi, g, W=256, sweeps=500, replicas=8, last_sweep=2, seed=1)


def test_bounded_waits_report_timeout_and_context_recovers(gdi):
    """Failure detection without a GPU fault: the host closes the grid barrier's gate word before
    the launch, so no block's wait can end; every wait gives up after a short bounded poll,
    the anneal reports GDI_ERR_TIMEOUT, and the same context then anneals normally (bit-exact)."""
    g = barabasi_albert(20000, 5, 60)
    ann = gdi.Annealer(g, A=1, B=4, W=64, replicas=2)
    ann.configure(path=gdi.GDI_PATH_GRID)
    sch = gdi.Schedule(sweeps=6, t0=12.0, t1=0.2)
    ann.inject_wait_failure(spin_limit=1 << 14)
    ann.anneal(sch, 3)
    with pytest.raises(gdi.GdiError) as err:
        ann.results()
    assert err.value.code == -9          # GDI_ERR_TIMEOUT
    ann.anneal(sch, 3, flags=gdi.GDI_FLAG_TRACE)
    res, spins = ann.results(), ann.spins()
    ann.close()
    ref = oracle.anneal(g, A=1, B=4, W=64, t0=12.0, t1=0.2, sweeps=6, seed=3, replicas=2)
    assert np.array_equal(spins, ref.spins)
    assert np.array_equal(res["final_cut"][0], ref.final_cut)
