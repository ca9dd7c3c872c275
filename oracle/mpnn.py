"""FP64 reference of the learned warm start's network -- TEST INFRASTRUCTURE ONLY.

Plain numpy, float64, written from the definitions (no blocking, no fusion), and sharing no code
with the CUDA kernels.  The network's weights are taken as BF16 (round-to-nearest-even of the
float32 master values), exactly as the GPU path uses them; everything else is float64.

    features  X = [diffused Philox +-1 noise (8 channels, centred, unit RMS per graph, optionally
                   sign-aligned to channel 0 per graph),
                   log(1 + deg), deg / mean deg, 0 x 6]
    layer l   H_l = ReLU(H_{l-1} Ws_l + (D^-1 A H_{l-1}) Wn_l + b_l),  l = 1, 2, 3
    logits    z = H_3 wo + bo
    loss      mean over graphs of min(mean softplus(-y z), mean softplus(y z)) + lam (mean tanh z)^2
    rounding  the floor(n/2) largest logits of a graph (ties: smaller vertex id) -> +1

Parity status: the backward pass is pinned by central finite differences of the loss
(tests/test_mpnn_oracle.py); features, forward and rounding are restatements of the definitions
above, pinned by invariances (permutation equivariance, sign invariance of the loss, balance of
the rounding) rather than by external values.
"""
from __future__ import annotations

import numpy as np

from . import philox4x32_10_many

HID = 64
FIN = 16
NRAND = 8
LAYER_DIMS = [(FIN, HID), (HID, HID), (HID, HID)]


# ------------------------------------------------------------------ parameter layout ----------
def param_layout():
    """Offsets of the flat parameter vector: per layer Ws [din x 64], Wn [din x 64], b [64];
    then wo [64], bo [1]."""
    off = {}
    o = 0
    for l, (din, dout) in enumerate(LAYER_DIMS, start=1):
        off[f"Ws{l}"] = (o, (din, dout)); o += din * dout
        off[f"Wn{l}"] = (o, (din, dout)); o += din * dout
        off[f"b{l}"] = (o, (dout,)); o += dout
    off["wo"] = (o, (HID,)); o += HID
    off["bo"] = (o, (1,)); o += 1
    return off, o


def unpack(flat):
    off, _ = param_layout()
    return {k: np.asarray(flat[o:o + int(np.prod(s))]).reshape(s) for k, (o, s) in off.items()}


def bf16_round(x):
    """float32 -> nearest BF16 value (ties to even), returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def effective_params(flat32):
    """Weights as the network uses them: BF16-rounded matrices and wo, float32 biases."""
    P = unpack(np.asarray(flat32, dtype=np.float32))
    out = {}
    for k, v in P.items():
        out[k] = v.astype(np.float64) if k.startswith("b") else bf16_round(v)
    return out


# ------------------------------------------------------------------ graph operators -----------
def _adj(row_ptr, col):
    n = len(row_ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    return rows, np.asarray(col, dtype=np.int64), np.diff(row_ptr).astype(np.float64)


def _matrix(rows, cols, vals, n):
    """The n x n sparse matrix with entries vals at (rows, cols) (a library sparse product serves as
    the matrix-times-block step below)."""
    import scipy.sparse as sp
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def mean_aggregate(row_ptr, col, X):
    """D^-1 A X: every vertex gets the mean of its neighbours' rows (0 for an isolated vertex)."""
    rows, cols, deg = _adj(row_ptr, col)
    return np.asarray(_matrix(rows, cols, 1.0 / deg[rows], len(deg)) @ np.asarray(X, dtype=np.float64))


def mean_aggregate_T(row_ptr, col, X):
    """(D^-1 A)^T X for a symmetric A: Y_j = sum_{i in N(j)} X_i / deg_i."""
    rows, cols, deg = _adj(row_ptr, col)
    return np.asarray(_matrix(rows, cols, 1.0 / deg[rows], len(deg)).T @ np.asarray(X, dtype=np.float64))


def walk_matrix(row_ptr, col):
    """D^-1/2 A D^-1/2 of the graph."""
    rows, cols, deg = _adj(row_ptr, col)
    return _matrix(rows, cols, 1.0 / np.sqrt(deg[rows] * deg[cols]), len(deg))


def lazy_walk(row_ptr, col, X, S=None):
    """One lazy step of the normalised walk: 0.5 X + 0.5 D^-1/2 A D^-1/2 X (S: that matrix, if
    already built)."""
    if S is None:
        S = walk_matrix(row_ptr, col)
    X = np.asarray(X, dtype=np.float64)
    return 0.5 * X + 0.5 * np.asarray(S @ X)


# ------------------------------------------------------------------ features ------------------
ALIGN, NO_NOISE = 1, 2


def features(graph_ptr, graph_id, row_ptr, col, seed, steps, flags=0):
    """Input features; flags & ALIGN: noise channel c >= 1 times the sign of its inner product with
    channel 0 inside each graph (sign 0 -> +1); flags & NO_NOISE: noise channels 0."""
    N = len(row_ptr) - 1
    R = np.zeros((N, NRAND))
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    for g in range(len(graph_ptr) - 1):
        # counter (local vertex, channel, graph id, tag); word 0's top bit gives the sign
        n = int(graph_ptr[g + 1] - graph_ptr[g])
        ctr = np.zeros((n, NRAND, 4), dtype=np.uint32)
        ctr[:, :, 0] = np.arange(n, dtype=np.uint32)[:, None]
        ctr[:, :, 1] = np.arange(NRAND, dtype=np.uint32)[None, :]
        ctr[:, :, 2] = graph_id[g]
        ctr[:, :, 3] = 0x4D504E4E
        w = philox4x32_10_many(ctr.reshape(-1, 4), key)[:, 0].reshape(n, NRAND)
        R[graph_ptr[g]:graph_ptr[g + 1]] = np.where(w >> np.uint32(31), -1.0, 1.0)
    S = walk_matrix(row_ptr, col)
    for _ in range(steps):
        R = lazy_walk(row_ptr, col, R, S)
    X = np.zeros((N, FIN))
    deg = np.diff(row_ptr).astype(np.float64)
    for g in range(len(graph_ptr) - 1):
        s = slice(graph_ptr[g], graph_ptr[g + 1])
        r = R[s] - R[s].mean(axis=0)
        rms = np.sqrt((r ** 2).mean(axis=0)) + 1e-12
        sign = np.ones(NRAND)
        if flags & ALIGN:
            sign[1:] = np.where(r[:, 1:].T @ r[:, 0] < 0, -1.0, 1.0)
        if flags & NO_NOISE:
            sign[:] = 0.0
        X[s, :NRAND] = sign * (r / rms)
        X[s, NRAND] = np.log1p(deg[s])
        md = deg[s].mean()
        X[s, NRAND + 1] = deg[s] / md if md > 0 else 0.0
    return X


# ------------------------------------------------------------------ forward / loss / backward -
def forward(P, row_ptr, col, X):
    """Returns logits z and the cache of every layer's (input, aggregate, output)."""
    cache = []
    h = X
    for l in (1, 2, 3):
        agg = mean_aggregate(row_ptr, col, h)
        out = np.maximum(h @ P[f"Ws{l}"] + agg @ P[f"Wn{l}"] + P[f"b{l}"], 0.0)
        cache.append((h, agg, out))
        h = out
    z = h @ P["wo"] + P["bo"][0]
    return z, cache


def _softplus(x):
    return np.logaddexp(0.0, x)


def loss(graph_ptr, z, y, lam):
    """Total loss and dL/dz (and the chosen sign per graph)."""
    G = len(graph_ptr) - 1
    L = 0.0
    dz = np.zeros_like(z)
    signs = np.zeros(G)
    for g in range(G):
        s = slice(graph_ptr[g], graph_ptr[g + 1])
        n = graph_ptr[g + 1] - graph_ptr[g]
        zg, yg = z[s], y[s].astype(np.float64)
        l1 = _softplus(-yg * zg).mean()
        l2 = _softplus(yg * zg).mean()
        m = np.tanh(zg).mean()
        sg = 1.0 if l1 <= l2 else -1.0
        signs[g] = sg
        L += (min(l1, l2) + lam * m * m) / G
        t = sg * yg
        sig = 1.0 / (1.0 + np.exp(t * zg))                 # sigmoid(-t z)
        dz[s] = (-t * sig + lam * 2.0 * m * (1.0 - np.tanh(zg) ** 2)) / (n * G)
    return L, dz, signs


def backward(P, row_ptr, col, cache, dz):
    """Gradients (same keys as P) of the loss whose dL/dz is given."""
    grads = {}
    h3 = cache[-1][2]
    grads["wo"] = h3.T @ dz
    grads["bo"] = np.array([dz.sum()])
    dh = np.outer(dz, P["wo"])
    for l in (3, 2, 1):
        h_in, agg, out = cache[l - 1]
        dpre = dh * (out > 0)
        grads[f"Ws{l}"] = h_in.T @ dpre
        grads[f"Wn{l}"] = agg.T @ dpre
        grads[f"b{l}"] = dpre.sum(axis=0)
        dh = dpre @ P[f"Ws{l}"].T + mean_aggregate_T(row_ptr, col, dpre @ P[f"Wn{l}"].T)
    return grads


def flat_grads(grads):
    off, total = param_layout()
    out = np.zeros(total)
    for k, (o, s) in off.items():
        out[o:o + int(np.prod(s))] = np.asarray(grads[k]).ravel()
    return out


def adam_step(p, g, m, v, lr, b1, b2, eps, t):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p, m, v


def round_balanced(graph_ptr, z):
    s = np.empty(len(z), dtype=np.int8)
    for g in range(len(graph_ptr) - 1):
        a, b = graph_ptr[g], graph_ptr[g + 1]
        n = b - a
        order = np.lexsort((np.arange(n), -np.asarray(z[a:b], dtype=np.float64)))
        sg = -np.ones(n, dtype=np.int8)
        sg[order[:n // 2]] = 1
        s[a:b] = sg
    return s
