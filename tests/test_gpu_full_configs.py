"""GPU parity at the full sizes of the benchmark configurations, on outputs the oracle can
compute one at a time: every replica (or a sample of replicas / instances) of the full schedule is
replayed by the oracle in spawned worker processes and compared bit for bit -- digest, G and cut
after every sweep, then raw/final G, raw/final cut and every spin."""
import multiprocessing as mp

import numpy as np
import pytest

import oracle
from gdi_synth import barabasi_albert, batch_union, er_batch, torus2d

pytestmark = pytest.mark.gpu


def _check_replica(res, spins, tr, ref, r, q=0):
    d, G, c = tr
    k = 0
    bad = np.nonzero((d[r] != ref.digest[k]) | (G[r] != ref.G_trace[k]) | (c[r] != ref.cut_trace[k]))[0]
    assert bad.size == 0, f"replica {r}: first mismatch at sweep {bad[0]}"
    assert res["raw_G"][q, r] == ref.raw_G[k] and res["final_G"][q, r] == ref.final_G[k]
    assert res["raw_cut"][q, r] == ref.raw_cut[k] and res["final_cut"][q, r] == ref.final_cut[k]
    assert np.array_equal(spins[r], ref.spins[k])


def test_ba1m_500_sweeps_windows_every_replica(gdi):
    """BA n = 10^6, m = 5, 8 replicas, W = 256, the 500-sweep schedule (the benchmark's anneal).
    The GPU runs it whole, and also in two parts (resumed with GDI_FLAG_CONTINUE); the oracle
    replays three 6-sweep windows of every replica -- the first sweeps, the middle of the schedule
    and its end with the repair -- each started from the GPU's own spins at the window start."""
    g = barabasi_albert(1_000_000, 5, 4004)
    sch = gdi.Schedule(sweeps=500, t0=12.0, t1=0.2)
    ann = gdi.Annealer(g, A=1, B=4, W=256, replicas=8)
    ann.anneal(sch, 1, flags=gdi.GDI_FLAG_TRACE)
    res, spins, tr = ann.results(), ann.spins(), ann.trace()
    assert ann.last_launch()["path"] == gdi.GDI_PATH_GRID
    starts = {}
    for k in (247, 494):
        ann.anneal(sch, 1, last_sweep=k, flags=gdi.GDI_FLAG_NO_REPAIR)
        starts[k] = ann.spins()
    ann.anneal(sch, 1, first_sweep=494, flags=gdi.GDI_FLAG_CONTINUE)
    assert np.array_equal(ann.spins(), spins)                # the two-part run equals the whole one
    ann.close()
    kw = dict(A=1, B=4, W=256, t0=12.0, t1=0.2, sweeps=500, seed=1)
    d, G, c = tr
    for k0, k1, init in ((0, 6, None), (247, 253, starts[247]), (494, 500, starts[494])):
        last = k1 == 500
        if init is None:
            refs = oracle.anneal_parallel(g, replica_ids=range(8), processes=8, first_sweep=k0,
                                          last_sweep=k1, repair=last, **kw)
        else:
            refs = _replay_from(g, init, k0, k1, last, kw)
        sl = slice(k0, k1)
        for r, ref in enumerate(refs):
            assert np.array_equal(d[r, sl], ref.digest[0, sl]), f"replica {r}, sweeps {k0}-{k1}"
            assert np.array_equal(G[r, sl], ref.G_trace[0, sl]) and np.array_equal(c[r, sl], ref.cut_trace[0, sl])
            if last:
                assert res["raw_G"][0, r] == ref.raw_G[0] and res["final_G"][0, r] == ref.final_G[0]
                assert res["raw_cut"][0, r] == ref.raw_cut[0] and res["final_cut"][0, r] == ref.final_cut[0]
                assert np.array_equal(spins[r], ref.spins[0])


def _replay_job(args):
    g, init_r, k0, k1, last, r, kw = args
    return oracle.anneal(g, replicas=1, first_replica=r, init=init_r[None, :], first_sweep=k0, last_sweep=k1,
                         repair=last, **kw)


def _replay_from(g, init, k0, k1, last, kw):
    with mp.get_context("spawn").Pool(8) as pool:
        return pool.map(_replay_job, [(g, init[r], k0, k1, last, r, kw) for r in range(8)])


def test_ba1m_all_500_sweeps_every_replica(gdi):
    """The whole 500-sweep anneal of all 8 replicas replayed by the oracle (about 5 minutes of
    oracle time on 8 host cores): every sweep's digest, G and cut, then the repair and every spin."""
    g = barabasi_albert(1_000_000, 5, 4004)
    kw = dict(A=1, B=4, W=256, t0=12.0, t1=0.2, sweeps=500, seed=1)
    ann = gdi.Annealer(g, A=1, B=4, W=256, replicas=8)
    ann.anneal(gdi.Schedule(sweeps=500, t0=12.0, t1=0.2), 1, flags=gdi.GDI_FLAG_TRACE)
    res, spins, tr = ann.results(), ann.spins(), ann.trace()
    ann.close()
    refs = oracle.anneal_parallel(g, replica_ids=range(8), processes=8, **kw)
    for r in range(8):
        _check_replica(res, spins, tr, refs[r], r)


def test_torus_all_5000_sweeps_sampled_replicas(gdi):
    """Torus 100 x 100 (+-1 weights, checkerboard), 64 replicas, W = 256, 5000 sweeps: replicas
    0, 21, 42 and 63 replayed by the oracle over the whole schedule."""
    g = torus2d(100, 2002)
    kw = dict(A=1, B=4, W=256, t0=12.0, t1=0.2, sweeps=5000, seed=1, color=g.color)
    ann = gdi.Annealer(g, A=1, B=4, W=256, replicas=64, color=g.color)
    ann.anneal(gdi.Schedule(sweeps=5000, t0=12.0, t1=0.2), 1, flags=gdi.GDI_FLAG_TRACE)
    res, spins, tr = ann.results(), ann.spins(), ann.trace()
    ann.close()
    ids = [0, 21, 42, 63]
    refs = oracle.anneal_parallel(g, replica_ids=ids, processes=4, **kw)
    for r, ref in zip(ids, refs):
        _check_replica(res, spins, tr, ref, r)


def _er_chunk(args):
    lo, hi = args
    return er_batch(hi - lo, 3000 + lo, n_lo=800, n_hi=3000)


def _oracle_instance(args):
    g, q = args
    return oracle.anneal(g, A=1, B=4, W=256, t0=12.0, t1=0.2, sweeps=2000, seed=11, instance=q)


def test_batched_4096_instances_graph_replay(gdi):
    """4,096 ER instances (n ~ U[800, 3000], mean degree ~ U[3, 48], unit or +-1 weights), one
    replica each, 2000 sweeps: autotuned, captured into a CUDA graph and replayed; eight instances
    (the first, the last, the smallest, the largest and four others) replayed by the oracle."""
    import torch
    with mp.get_context("spawn").Pool(16) as pool:
        parts = pool.map(_er_chunk, [(i, min(4096, i + 256)) for i in range(0, 4096, 256)])
    gs = [g for part in parts for g in part]
    inst_ptr, u = batch_union(gs)
    ann = gdi.Annealer(u, A=1, B=4, W=256, replicas=1, inst_ptr=inst_ptr)
    sch = gdi.Schedule(sweeps=2000, t0=12.0, t1=0.2)
    ann.autotune(gdi.Schedule(sweeps=2000, t0=12.0, t1=0.2), probe_sweeps=20)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ann.anneal(sch, 11, stream=stream, flags=gdi.GDI_FLAG_TRACE)
    graph = ann.capture_graph(sch, 11, stream, flags=gdi.GDI_FLAG_TRACE)
    graph.replay()
    torch.cuda.synchronize()
    res, spins, (d, G, c) = ann.results(), ann.spins(), ann.trace()
    ann.close()
    ns = np.diff(inst_ptr)
    pick = sorted({0, 4095, int(np.argmin(ns)), int(np.argmax(ns)), 1000, 2047, 3001, 3500})
    with mp.get_context("spawn").Pool(len(pick)) as pool:
        refs = pool.map(_oracle_instance, [(gs[q], q) for q in pick])
    for q, ref in zip(pick, refs):
        assert np.array_equal(d[q], ref.digest[0]) and np.array_equal(G[q], ref.G_trace[0]), f"instance {q}"
        assert np.array_equal(c[q], ref.cut_trace[0]), f"instance {q}"
        assert res["final_cut"][q, 0] == ref.final_cut[0] and res["final_G"][q, 0] == ref.final_G[0]
        assert res["raw_cut"][q, 0] == ref.raw_cut[0] and res["raw_G"][q, 0] == ref.raw_G[0]
        assert np.array_equal(spins[0, inst_ptr[q]:inst_ptr[q + 1]], ref.spins[0])
