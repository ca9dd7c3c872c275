"""Batched launch: many instances in one persistent launch, launch configuration chosen by the
autotuner without changing any result, and CUDA-graph capture of an anneal."""
import numpy as np
import pytest

import oracle
from gdi_synth import barabasi_albert, batch_union, er_batch

pytestmark = pytest.mark.gpu


def _run(gdi, u, inst_ptr, sch, seed, block=0, grid=0, autotune=False):
    ann = gdi.Annealer(u, A=1, B=4, W=256, replicas=2, inst_ptr=inst_ptr)
    tuned = None
    if autotune:
        tuned = ann.autotune(sch, probe_sweeps=5)
    elif block or grid:
        ann.configure(path=gdi.GDI_PATH_CTA, block=block, grid_limit=grid)
    ann.anneal(sch, seed, flags=gdi.GDI_FLAG_TRACE)
    out = (ann.trace()[0].copy(), ann.spins().copy(), ann.results()["final_cut"].copy(), ann.last_launch())
    ann.close()
    return out, tuned


def test_results_do_not_depend_on_launch_configuration(gdi):
    gs = er_batch(40, 7000, n_lo=150, n_hi=900)
    inst_ptr, u = batch_union(gs)
    sch = gdi.Schedule(sweeps=60, t0=12.0, t1=0.2)
    ref, _ = _run(gdi, u, inst_ptr, sch, 17)
    for block, grid in [(128, 0), (1024, 0), (256, 7), (512, 152)]:
        got, _ = _run(gdi, u, inst_ptr, sch, 17, block=block, grid=grid)
        assert np.array_equal(got[0], ref[0]), (block, grid)
        assert np.array_equal(got[1], ref[1]), (block, grid)
        assert got[3]["grid"] <= (grid or 10 ** 9)
    got, tuned = _run(gdi, u, inst_ptr, sch, 17, autotune=True)
    assert tuned["block"] in (128, 256, 512, 1024) and tuned["ms"] > 0
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    # and the oracle agrees on a few instances
    for q in (0, 13, 39):
        r = oracle.anneal(gs[q], A=1, B=4, W=256, t0=12.0, t1=0.2, sweeps=60, seed=17, instance=q,
                          replicas=2)
        assert np.array_equal(ref[2][q], r.final_cut)
        assert np.array_equal(ref[1][:, inst_ptr[q]:inst_ptr[q + 1]], r.spins)


def test_grid_path_autotune_keeps_results(gdi):
    g = barabasi_albert(40000, 5, 71)
    sch = gdi.Schedule(sweeps=20, t0=12.0, t1=0.2)
    a = gdi.Annealer(g, A=1, B=4, W=128, replicas=8)
    a.configure(path=gdi.GDI_PATH_GRID)
    a.anneal(sch, 3, flags=gdi.GDI_FLAG_TRACE)
    d0, s0 = a.trace()[0].copy(), a.spins().copy()
    tuned = a.autotune(sch, probe_sweeps=4)
    a.anneal(sch, 3, flags=gdi.GDI_FLAG_TRACE)
    assert np.array_equal(a.trace()[0], d0) and np.array_equal(a.spins(), s0)
    assert tuned["grid"] > 0
    a.close()


@pytest.mark.parametrize("grid_path", [False, True])
def test_cuda_graph_replay_equals_direct_anneal(gdi, grid_path):
    import torch
    if grid_path:
        g = barabasi_albert(40000, 5, 72)
        a = gdi.Annealer(g, A=1, B=4, W=128, replicas=8)
        a.configure(path=gdi.GDI_PATH_GRID)
    else:
        gs = er_batch(30, 8000, n_lo=200, n_hi=600)
        inst_ptr, g = batch_union(gs)
        a = gdi.Annealer(g, A=1, B=4, W=64, replicas=3, inst_ptr=inst_ptr)
    sch = gdi.Schedule(sweeps=40, t0=12.0, t1=0.2)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a.anneal(sch, 21, stream=stream)
    ref_spins, ref_cut = a.spins().copy(), a.results()["final_cut"].copy()
    ms, n = a.kernel_ms()
    assert ms > 0 and n == 1
    graph = a.capture_graph(sch, 21, stream)
    with pytest.raises(gdi.GdiError):
        a.kernel_ms()          # a captured anneal records no timing events
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(a.spins(), ref_spins)
        assert np.array_equal(a.results()["final_cut"], ref_cut)
    a.close()


def test_kernel_time_counts_sweep_launches(gdi):
    """The sweep kernel is timed alone: one launch per group of 8 replicas on the grid path, one on
    the CTA path, each shorter than the whole anneal measured around it."""
    import torch
    g = barabasi_albert(30000, 5, 73)
    a = gdi.Annealer(g, A=1, B=4, W=64, replicas=11)
    a.configure(path=gdi.GDI_PATH_GRID)
    sch = gdi.Schedule(sweeps=20, t0=12.0, t1=0.2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    a.anneal(sch, 5, stream=torch.cuda.current_stream())
    e1.record()
    torch.cuda.synchronize()
    ms, n = a.kernel_ms()
    assert n == 2 and 0 < ms < e0.elapsed_time(e1)
    a.configure(path=gdi.GDI_PATH_CTA)
    small = barabasi_albert(3000, 4, 74)
    b = gdi.Annealer(small, A=1, B=4, W=64, replicas=4)
    b.anneal(sch, 5)
    ms2, n2 = b.kernel_ms()
    assert n2 == 1 and ms2 > 0
    a.close()
    b.close()


@pytest.mark.parametrize("n,replicas,want", [(1000, 8, "cta"), (20000, 8, "grid"), (20000, 608, "cta")])
def test_auto_path_follows_cost_model(gdi, n, replicas, want):
    """One instance: the automatic path is the CTA-resident one for small graphs or many replicas
    (one block per replica fills the GPU) and the grid-scale one for a few replicas of a larger
    graph (every SM on one replica group); results are bit-exact either way."""
    g = barabasi_albert(n, 5, 90 + n)
    sch = gdi.Schedule(sweeps=6, t0=12.0, t1=0.2)
    a = gdi.Annealer(g, A=1, B=4, W=256, replicas=replicas)
    a.anneal(sch, 5)
    path = a.last_launch()["path"]
    cut = a.results()["final_cut"][0]
    a.close()
    assert path == (gdi.GDI_PATH_GRID if want == "grid" else gdi.GDI_PATH_CTA)
    if replicas <= 8:
        ref = oracle.anneal(g, A=1, B=4, W=256, t0=12.0, t1=0.2, sweeps=6, seed=5, replicas=replicas)
        assert np.array_equal(cut, ref.final_cut)


def test_autotune_under_auto_path(gdi):
    g = barabasi_albert(20000, 5, 73)
    sch = gdi.Schedule(sweeps=20, t0=12.0, t1=0.2)
    a = gdi.Annealer(g, A=1, B=4, W=256, replicas=8)
    a.anneal(sch, 3, flags=gdi.GDI_FLAG_TRACE)
    d0 = a.trace()[0].copy()
    tuned = a.autotune(sch, probe_sweeps=4)
    a.anneal(sch, 3, flags=gdi.GDI_FLAG_TRACE)
    assert np.array_equal(a.trace()[0], d0) and tuned["ms"] > 0
    a.close()
