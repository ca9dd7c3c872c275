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


# ------------------------------------------------------------------ closed-form pins ----------
def _star(m):
    from gdi_synth import star_graph
    return star_graph(m + 1)            # vertex 0 is the hub, 1..m the leaves


def test_mean_aggregate_closed_forms():
    """D^-1 A X: on K_n every vertex gets (sum - own) / (n - 1); on a star the hub gets the mean of
    the leaves and every leaf the hub's row; an isolated vertex gets 0."""
    from gdi_synth import from_edges
    rng = np.random.default_rng(11)
    n = 7
    u, v = np.triu_indices(n, 1)
    k = from_edges(n, u, v)
    X = rng.standard_normal((n, 3))
    Y = mpnn.mean_aggregate(k.row_ptr, k.col, X)
    assert np.allclose(Y, (X.sum(axis=0) - X) / (n - 1), rtol=0, atol=1e-13)
    s = _star(5)
    X = rng.standard_normal((6, 2))
    Y = mpnn.mean_aggregate(s.row_ptr, s.col, X)
    assert np.allclose(Y[0], X[1:].mean(axis=0), atol=1e-13)
    assert np.allclose(Y[1:], np.broadcast_to(X[0], (5, 2)), atol=1e-13)
    iso = from_edges(3, np.array([0]), np.array([1]))     # vertex 2 has no neighbour
    Y = mpnn.mean_aggregate(iso.row_ptr, iso.col, np.ones((3, 1)))
    assert Y[2, 0] == 0.0 and Y[0, 0] == 1.0


def test_mean_aggregate_transpose_is_the_adjoint():
    """<D^-1 A X, Y> = <X, (D^-1 A)^T Y> for any X, Y (the transposed operator of the backward)."""
    g = erdos_renyi(60, 0.08, 12)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((g.n, 4))
    Y = rng.standard_normal((g.n, 4))
    lhs = np.sum(mpnn.mean_aggregate(g.row_ptr, g.col, X) * Y)
    rhs = np.sum(X * mpnn.mean_aggregate_T(g.row_ptr, g.col, Y))
    assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.parametrize("n,k,t", [(12, 1, 1), (12, 3, 5), (31, 2, 40), (16, 8, 3)])
def test_lazy_walk_multiplies_cycle_fourier_modes(n, k, t):
    """On the cycle C_n, D^-1/2 A D^-1/2 = A / 2 has the Fourier modes cos(2 pi k i / n + phi) as
    eigenvectors with eigenvalue cos(2 pi k / n); t lazy steps multiply them by
    ((1 + cos(2 pi k / n)) / 2)^t."""
    from gdi_synth import from_edges
    i = np.arange(n)
    c = from_edges(n, i, (i + 1) % n)
    theta = 2 * np.pi * k / n
    X = np.stack([np.cos(theta * i + 0.3), np.sin(theta * i - 1.1)], axis=1)
    Y = X.copy()
    for _ in range(t):
        Y = mpnn.lazy_walk(c.row_ptr, c.col, Y)
    assert np.allclose(Y, X * ((1 + np.cos(theta)) / 2) ** t, rtol=0, atol=1e-12)


def test_lazy_walk_star_eigenvectors():
    """Star K_{1,m} (not regular): D^-1/2 A D^-1/2 fixes sqrt(deg) (eigenvalue 1), maps
    sqrt(deg) * (+1 hub, -1 leaves) to its negative (eigenvalue -1, so a lazy step gives 0), and
    annihilates a difference of two leaves (eigenvalue 0, a lazy step halves it)."""
    m = 6
    s = _star(m)
    sq = np.sqrt(np.diff(s.row_ptr).astype(np.float64))
    top = sq[:, None]
    bip = (sq * np.where(np.arange(m + 1) == 0, 1.0, -1.0))[:, None]
    dif = np.zeros((m + 1, 1))
    dif[1], dif[2] = 1.0, -1.0
    assert np.allclose(mpnn.lazy_walk(s.row_ptr, s.col, top), top, atol=1e-13)
    assert np.allclose(mpnn.lazy_walk(s.row_ptr, s.col, bip), 0.0, atol=1e-13)
    assert np.allclose(mpnn.lazy_walk(s.row_ptr, s.col, dif), 0.5 * dif, atol=1e-13)


def _golden_mpnn():
    import os
    fx = {"w": [], "b": [], "v": []}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "mpnn_path4_forward.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *vals = line.split()
        if k in ("w", "b", "v"):
            fx[k].append(vals)
        else:
            fx[k] = vals
    return fx


def test_forward_hand_derived_path4():
    """tests/golden/mpnn_path4_forward.txt: a 3-layer forward pass worked out by hand (mean
    aggregation, self and neighbour weights, biases, ReLU clipping, output layer, rounding)."""
    from gdi_synth import from_edges
    fx = _golden_mpnn()
    eu, ev = zip(*[tuple(map(int, e.split("-"))) for e in fx["edges"]])
    g = from_edges(4, np.array(eu), np.array(ev))
    _, total = mpnn.param_layout()
    P = mpnn.unpack(np.zeros(total))
    P = {k: v.copy() for k, v in P.items()}
    for name, i, j, val in fx["w"]:
        P[name][int(i), int(j)] = float(val)
    for name, i, val in fx["b"] + fx["v"]:
        P[name][int(i)] = float(val)
    X = np.zeros((4, mpnn.FIN))
    X[:, 0] = list(map(float, fx["x0"]))
    X[:, 1] = list(map(float, fx["x1"]))
    z, cache = mpnn.forward(P, g.row_ptr, g.col, X)
    for (l, ch) in ((1, 0), (1, 1), (1, 2), (1, 3), (2, 0), (2, 1), (3, 5), (3, 6)):
        assert cache[l - 1][2][:, ch].tolist() == list(map(float, fx[f"h{l}_{ch}"])), (l, ch)
    others = np.ones(mpnn.HID, bool)
    others[[5, 6]] = False
    assert np.all(cache[2][2][:, others] == 0)
    assert z.tolist() == list(map(float, fx["z"]))
    s = mpnn.round_balanced(np.array([0, 4]), z.astype(np.float32))
    assert s.tolist() == list(map(int, fx["spins"]))
    # the same numbers through the float32 -> BF16 path the GPU uses (every value is BF16-exact)
    flat = mpnn.flat_grads(P).astype(np.float32)
    z2, _ = mpnn.forward(mpnn.effective_params(flat), g.row_ptr, g.col, X)
    assert z2.tolist() == z.tolist()


@pytest.mark.parametrize("c,lam", [(0.0, 0.3), (0.7, 0.0), (-1.3, 0.25)])
def test_loss_closed_form_for_constant_logits(c, lam):
    """Balanced labels and constant logits z = c: both signs give (softplus(c) + softplus(-c)) / 2
    = log(2 cosh(c / 2)), and the balance term is lam tanh(c)^2 (z = 0: log 2)."""
    gp = np.array([0, 6, 14], dtype=np.int64)
    y = np.array([1, -1, 1, -1, -1, 1] + [1, 1, -1, -1, 1, -1, 1, -1], dtype=np.int8)
    z = np.full(14, c)
    L, _, _ = mpnn.loss(gp, z, y, lam)
    assert L == pytest.approx(np.log(2 * np.cosh(c / 2)) + lam * np.tanh(c) ** 2, rel=1e-12)


def test_feature_alignment_and_noise_mask():
    """ALIGN flips whole noise channels so that each has a non-negative inner product with channel 0
    inside every graph (and changes nothing else); NO_NOISE zeroes the noise channels only."""
    gs, gp, u = _batch()
    ids = np.array([3, 4, 5], dtype=np.uint32)
    X0 = mpnn.features(gp, ids, u.row_ptr, u.col, 21, 6)
    Xa = mpnn.features(gp, ids, u.row_ptr, u.col, 21, 6, mpnn.ALIGN)
    Xn = mpnn.features(gp, ids, u.row_ptr, u.col, 21, 6, mpnn.NO_NOISE)
    assert np.array_equal(np.abs(Xa), np.abs(X0)) and np.array_equal(Xa[:, 8:], X0[:, 8:])
    for g in range(len(gs)):
        s = slice(gp[g], gp[g + 1])
        dots = Xa[s, :8].T @ Xa[s, 0]
        assert np.all(dots >= 0)
        for c in range(8):                       # each channel is the unaligned one or its negative
            assert np.array_equal(Xa[s, c], X0[s, c]) or np.array_equal(Xa[s, c], -X0[s, c])
    assert np.all(Xn[:, :8] == 0) and np.array_equal(Xn[:, 8:], X0[:, 8:])
