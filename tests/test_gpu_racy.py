"""GDI_FLAG_RACY (Algorithm 3 as printed: every spin of a colour class decides on the G it reads and
adds its change atomically).  Not deterministic, so the checks are the exact invariants the racy
path must keep, and one case that makes it deterministic: with A = 0 no decision depends on G,
and the racy path must equal the serialised oracle bit for bit."""
import numpy as np
import pytest

import oracle
from gdi_synth import barabasi_albert

pytestmark = pytest.mark.gpu


def test_racy_keeps_g_and_cut_exact(gdi):
    g = barabasi_albert(20000, 5, 81)
    sch = gdi.Schedule(sweeps=60, t0=12.0, t1=0.2)
    ann = gdi.Annealer(g, A=1, B=4, W=256, replicas=8)
    ann.anneal(sch, 9, flags=gdi.GDI_FLAG_RACY | gdi.GDI_FLAG_NO_REPAIR)
    res, spins = ann.results(), ann.spins()
    assert ann.last_launch()["path"] == gdi.GDI_PATH_GRID
    # the atomically tracked magnetisation is the sum of the spins, the cut that of the spins
    assert np.array_equal(res["raw_G"][0], spins.astype(np.int64).sum(axis=1))
    assert all(res["raw_cut"][0, r] == oracle.cut(g, spins[r]) for r in range(8))
    ann.anneal(sch, 9, flags=gdi.GDI_FLAG_RACY)
    res, spins = ann.results(), ann.spins()
    ann.close()
    assert np.all(np.abs(res["final_G"][0]) == g.n % 2)
    assert np.array_equal(res["final_G"][0], spins.astype(np.int64).sum(axis=1))
    assert all(res["final_cut"][0, r] == oracle.cut(g, spins[r]) for r in range(8))


def test_racy_without_balance_term_equals_oracle(gdi):
    """A = 0: every threshold is +-infinity (flip or not, whatever G is), so the order of the
    atomics cannot matter and the racy path is the serialised one."""
    g = barabasi_albert(20000, 5, 82)
    sch = gdi.Schedule(sweeps=30, t0=12.0, t1=0.2)
    ann = gdi.Annealer(g, A=0, B=4, W=256, replicas=4)
    ann.anneal(sch, 6, flags=gdi.GDI_FLAG_RACY | gdi.GDI_FLAG_TRACE)
    res, spins, (d, G, c) = ann.results(), ann.spins(), ann.trace()
    ann.close()
    ref = oracle.anneal(g, A=0, B=4, W=256, t0=12.0, t1=0.2, sweeps=30, seed=6, replicas=4)
    assert np.array_equal(d, ref.digest) and np.array_equal(G, ref.G_trace) and np.array_equal(c, ref.cut_trace)
    assert np.array_equal(spins, ref.spins)
    assert np.array_equal(res["final_cut"][0], ref.final_cut)
