"""Pins of the FP64 network oracle (CPU): finite differences, invariances, exact balance."""
import numpy as np
import pytest

import oracle
from oracle import mpnn
from gdi_synth import batch_union, erdos_renyi, random_geometric


def _batch():
    gs = [erdos_renyi(40, 0.12, 3), random_geometric(35, 0.3, 4), erdos_renyi(29, 0.2, 5)]
    gp, u = batch_union(gs)
    return gs, gp, u


def _params(seed=0, scale=0.3):
    _, total = mpnn.param_layout()
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(total) * scale).astype(np.float32)


def _labels(gp, seed=1):
    rng = np.random.default_rng(seed)
    y = np.empty(gp[-1], dtype=np.int8)
    for g in range(len(gp) - 1):
        n = gp[g + 1] - gp[g]
        s = np.where(np.arange(n) < n // 2, 1, -1)
        y[gp[g]:gp[g + 1]] = rng.permutation(s)
    return y


def test_backward_matches_finite_differences():
    """Central differences of the float64 loss w.r.t. the effective (BF16-valued) parameters."""
    gs, gp, u = _batch()
    X = mpnn.features(gp, np.arange(len(gs), dtype=np.uint32), u.row_ptr, u.col, 77, 3)
    y = _labels(gp)
    P = mpnn.effective_params(_params())
    lam = 0.3
    z, cache = mpnn.forward(P, u.row_ptr, u.col, X)
    L, dz, _ = mpnn.loss(gp, z, y, lam)
    grads = mpnn.backward(P, u.row_ptr, u.col, cache, dz)
    rng = np.random.default_rng(3)
    h = 1e-6
    for key in ("Ws1", "Wn1", "b1", "Ws2", "Wn3", "b3", "wo", "bo"):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in P[key].shape)
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[key][idx] += h
            Pm[key][idx] -= h
            Lp = mpnn.loss(gp, mpnn.forward(Pp, u.row_ptr, u.col, X)[0], y, lam)[0]
            Lm = mpnn.loss(gp, mpnn.forward(Pm, u.row_ptr, u.col, X)[0], y, lam)[0]
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - grads[key][idx]) <= 1e-6 + 1e-4 * abs(fd), (key, idx, fd, grads[key][idx])


def test_loss_is_invariant_to_label_sign():
    gs, gp, u = _batch()
    X = mpnn.features(gp, np.arange(len(gs), dtype=np.uint32), u.row_ptr, u.col, 5, 2)
    P = mpnn.effective_params(_params(1))
    z, _ = mpnn.forward(P, u.row_ptr, u.col, X)
    y = _labels(gp)
    a = mpnn.loss(gp, z, y, 0.1)
    b = mpnn.loss(gp, z, (-y).astype(np.int8), 0.1)
    assert a[0] == pytest.approx(b[0], rel=1e-12)
    assert np.allclose(a[1], b[1], rtol=1e-12, atol=0)


def test_forward_is_permutation_equivariant():
    """Relabelling the vertices (with the same input rows) permutes the logits."""
    g = erdos_renyi(50, 0.1, 8)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((g.n, mpnn.FIN))
    P = mpnn.effective_params(_params(2))
    z, _ = mpnn.forward(P, g.row_ptr, g.col, X)
    perm = rng.permutation(g.n)          # new id of old vertex v is perm[v]
    from gdi_synth import from_edges
    uu, vv, ww = g.edges()
    h = from_edges(g.n, perm[uu], perm[vv], ww)
    X2 = np.empty_like(X)
    X2[perm] = X
    z2, _ = mpnn.forward(P, h.row_ptr, h.col, X2)
    assert np.allclose(z2[perm], z, rtol=1e-12, atol=1e-12)


def test_features_are_centred_and_scaled():
    gs, gp, u = _batch()
    X = mpnn.features(gp, np.array([7, 8, 9], dtype=np.uint32), u.row_ptr, u.col, 11, 4)
    for g in range(len(gs)):
        s = slice(gp[g], gp[g + 1])
        assert np.allclose(X[s, :8].mean(axis=0), 0, atol=1e-12)
        assert np.allclose((X[s, :8] ** 2).mean(axis=0), 1, atol=1e-9)
        deg = np.diff(gs[g].row_ptr)
        assert np.allclose(X[s, 8], np.log1p(deg))
        assert np.allclose(X[s, 10:], 0)


def test_rounding_is_exactly_balanced_and_ordered():
    rng = np.random.default_rng(5)
    gp = np.array([0, 10, 21, 21 + 8], dtype=np.int64)
    z = rng.standard_normal(gp[-1]).astype(np.float32)
    z[3] = z[4]                          # a tie inside graph 0
    s = mpnn.round_balanced(gp, z)
    for g in range(3):
        sg = s[gp[g]:gp[g + 1]]
        n = gp[g + 1] - gp[g]
        assert (sg == 1).sum() == n // 2
        zg = z[gp[g]:gp[g + 1]]
        assert zg[sg == 1].min() >= zg[sg == -1].max()


def test_adam_step_closed_form():
    """One step from m = v = 0 moves every parameter by lr * sign(g) (up to eps)."""
    p = np.array([0.5, -1.0, 2.0])
    g = np.array([0.3, -2.0, 1e-3])
    p1, m, v = mpnn.adam_step(p, g, np.zeros(3), np.zeros(3), 0.01, 0.9, 0.999, 1e-12, 1)
    assert np.allclose(p1, p - 0.01 * np.sign(g), atol=1e-9)
