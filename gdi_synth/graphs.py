"""Graph generators: Erdos-Renyi (Batagelj-Brandes skip sampling), 2-D torus, Barabasi-Albert
(Batagelj-Brandes linear-time preferential attachment), random geometric, and batched ER.

All graphs are simple, undirected and returned as a symmetric CSR over vertices 0..n-1 with
rows sorted by neighbour id. Weights are int32 (+1 unit, or +-1 signed) and symmetric.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


@dataclass
class CSRGraph:
    n: int
    row_ptr: np.ndarray            # int64 [n+1]
    col: np.ndarray                # int32 [nnz]
    w: np.ndarray                  # int32 [nnz]
    name: str = ""
    color: np.ndarray | None = None   # optional int32 [n] colouring supplied by the generator
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def max_degree(self) -> int:
        return int(np.diff(self.row_ptr).max()) if self.n else 0

    def edges(self):
        """Undirected edge list (u < v) with weights."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))
        m = rows < self.col
        return rows[m], self.col[m].astype(np.int64), self.w[m]


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied elementwise to uint64 input (Steele, Lea, Flood 2014)."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _MASK64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
        return z ^ (z >> np.uint64(31))


def _bits(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    base = splitmix64(np.array([(seed * 0x100000001B3 + stream) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        return splitmix64((idx.astype(np.uint64) * np.uint64(0xD1B54A32D192ED03)) ^ base)


def uniform01(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits, a pure function of (seed, stream, idx)."""
    return (_bits(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _uint_below(seed: int, stream: int, idx: np.ndarray, bound: np.ndarray) -> np.ndarray:
    """Integers in [0, bound) (bound >= 1) via the high 64x64 product (Lemire's mapping, no rejection)."""
    b = _bits(seed, stream, idx)
    hi_b = b >> np.uint64(32)
    lo_b = b & np.uint64(0xFFFFFFFF)
    bound = bound.astype(np.uint64)
    # floor(b * bound / 2^64) computed in 32-bit halves (bound < 2^32)
    with np.errstate(over="ignore"):
        t = lo_b * bound
        t = (t >> np.uint64(32)) + hi_b * bound
    return (t >> np.uint64(32)).astype(np.int64)


def from_edges(n: int, u: np.ndarray, v: np.ndarray, w: np.ndarray | None = None, name: str = "") -> CSRGraph:
    """Build a simple symmetric CSR from an undirected edge list (self-loops and duplicates dropped;
    for a duplicate pair the first weight in input order is kept)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if w is None:
        w = np.ones(u.shape[0], dtype=np.int32)
    w = np.asarray(w, dtype=np.int32)
    keep = u != v
    u, v, w = u[keep], v[keep], w[keep]
    a = np.minimum(u, v)
    b = np.maximum(u, v)
    key = a * n + b
    _, first = np.unique(key, return_index=True)
    first.sort()
    a, b, w = a[first], b[first], w[first]
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    ww = np.concatenate([w, w])
    order = np.lexsort((dst, src))
    src, dst, ww = src[order], dst[order], ww[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return CSRGraph(n=n, row_ptr=row_ptr, col=dst.astype(np.int32), w=ww.astype(np.int32), name=name)


def _pair_from_linear(L: np.ndarray):
    """Map a linear index over pairs (v, u) with u < v, ordered by v then u, back to (v, u)."""
    v = np.floor((1.0 + np.sqrt(1.0 + 8.0 * L.astype(np.float64))) / 2.0).astype(np.int64)
    # exact integer correction of the float estimate
    for _ in range(2):
        base = v * (v - 1) // 2
        v = np.where(base > L, v - 1, v)
        base = v * (v - 1) // 2
        v = np.where(L - base >= v, v + 1, v)
    u = L - v * (v - 1) // 2
    return v, u


def erdos_renyi(n: int, p: float, seed: int, signed: bool = False, name: str | None = None) -> CSRGraph:
    """G(n, p) by Batagelj-Brandes geometric skip sampling over the n(n-1)/2 vertex pairs.
    signed=True draws each edge weight +1 or -1 with equal probability."""
    total = n * (n - 1) // 2
    if p <= 0 or total == 0:
        g = from_edges(n, np.zeros(0), np.zeros(0), name=name or f"er_{n}_{p}")
        return g
    if p >= 1:
        L = np.arange(total, dtype=np.int64)
    else:
        lq = np.log1p(-p)
        chunks = []
        pos = -1
        k0 = 0
        expect = int(total * p * 1.1) + 64
        while True:
            idx = np.arange(k0, k0 + expect, dtype=np.int64)
            r = uniform01(seed, 1, idx)
            skip = np.floor(np.log1p(-r) / lq).astype(np.int64)
            steps = np.cumsum(skip + 1) + pos
            inside = steps < total
            chunks.append(steps[inside])
            if not inside.all():
                break
            pos = int(steps[-1])
            k0 += expect
        L = np.concatenate(chunks)
    v, u = _pair_from_linear(L)
    if signed:
        w = np.where(uniform01(seed, 2, np.arange(L.shape[0])) < 0.5, 1, -1).astype(np.int32)
    else:
        w = None
    g = from_edges(n, u, v, w, name=name or f"er_n{n}_p{p}")
    g.meta.update(dict(kind="er", n=n, p=p, seed=seed, signed=signed))
    return g


def torus2d(L: int, seed: int, signed: bool = True, name: str | None = None) -> CSRGraph:
    """L x L periodic square lattice (4-regular for L >= 3). Vertex (x, y) has id y*L + x.
    Horizontal edge of (x, y) has index 2*id, vertical edge 2*id+1; signed weights are drawn per edge.
    For even L the generator also returns the checkerboard colouring (x + y) & 1."""
    ids = np.arange(L * L, dtype=np.int64)
    x = ids % L
    y = ids // L
    right = y * L + (x + 1) % L
    down = ((y + 1) % L) * L + x
    u = np.concatenate([ids, ids])
    v = np.concatenate([right, down])
    eidx = np.concatenate([2 * ids, 2 * ids + 1])
    if signed:
        w = np.where(uniform01(seed, 3, eidx) < 0.5, 1, -1).astype(np.int32)
    else:
        w = np.ones(eidx.shape[0], dtype=np.int32)
    g = from_edges(L * L, u, v, w, name=name or f"torus{L}x{L}")
    if L % 2 == 0:
        g.color = ((x + y) & 1).astype(np.int32)
    g.meta.update(dict(kind="torus", L=L, seed=seed, signed=signed))
    return g


def barabasi_albert(n: int, m: int, seed: int, name: str | None = None) -> CSRGraph:
    """Preferential attachment by the Batagelj-Brandes linear-time method: vertices 0..m form a
    complete core K_{m+1}; each later vertex v appends m edge slots (v, M[r]) where r is uniform over
    all earlier slot positions of the endpoint list M. Self-loops and repeated pairs are dropped."""
    core_u, core_v = np.triu_indices(m + 1, k=1)
    core = np.empty(2 * core_u.shape[0], dtype=np.int64)
    core[0::2] = core_u
    core[1::2] = core_v
    c = core.shape[0]
    nv = n - (m + 1)
    if nv <= 0:
        return from_edges(n, core_u, core_v, name=name or f"ba_n{n}_m{m}")
    k = np.arange(nv * m, dtype=np.int64)
    vert = (m + 1) + k // m
    pos = c + 2 * k                      # slot position holding the new vertex
    r = _uint_below(seed, 4, k, pos + 1)  # uniform over [0, pos] -> earlier slots plus own slot
    total = c + 2 * nv * m
    # value lookup: even offsets beyond the core hold the new vertex; odd ones point back to r
    ptr = np.empty(total, dtype=np.int64)
    val = np.full(total, -1, dtype=np.int64)
    val[:c] = core
    ptr[:c] = np.arange(c)
    val[pos] = vert
    ptr[pos] = pos
    ptr[pos + 1] = r
    # pointer jumping until every slot points at a resolved position
    resolved = val >= 0
    while True:
        t = ptr[~resolved]
        if t.size == 0:
            break
        ptr[~resolved] = ptr[t]
        newly = val[ptr] >= 0
        val[~resolved & newly] = val[ptr[~resolved & newly]]
        resolved = val >= 0
    u = np.concatenate([core_u, vert])
    v = np.concatenate([core_v, val[pos + 1]])
    g = from_edges(n, u, v, name=name or f"ba_n{n}_m{m}")
    g.meta.update(dict(kind="ba", n=n, m=m, seed=seed))
    return g


def random_geometric(n: int, radius: float, seed: int, name: str | None = None) -> CSRGraph:
    """n points uniform in the unit square; an edge joins points closer than radius."""
    pts = np.stack([uniform01(seed, 5, np.arange(n)), uniform01(seed, 6, np.arange(n))], axis=1)
    cells = max(1, int(1.0 / max(radius, 1e-9)))
    cx = np.minimum((pts[:, 0] * cells).astype(np.int64), cells - 1)
    cy = np.minimum((pts[:, 1] * cells).astype(np.int64), cells - 1)
    cid = cy * cells + cx
    order = np.argsort(cid, kind="stable")
    us, vs = [], []
    r2 = radius * radius
    starts = np.searchsorted(cid[order], np.arange(cells * cells))
    ends = np.searchsorted(cid[order], np.arange(cells * cells), side="right")
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            ny = cy + dy
            nx = cx + dx
            ok = (ny >= 0) & (ny < cells) & (nx >= 0) & (nx < cells)
            idx = np.nonzero(ok)[0]
            nc = ny[idx] * cells + nx[idx]
            cnt = ends[nc] - starts[nc]
            rep = np.repeat(idx, cnt)
            offs = np.concatenate([order[starts[c]:ends[c]] for c in nc]) if idx.size else np.zeros(0, np.int64)
            d = pts[rep] - pts[offs]
            close = (d * d).sum(1) < r2
            m = close & (rep < offs)
            us.append(rep[m])
            vs.append(offs[m])
    g = from_edges(n, np.concatenate(us), np.concatenate(vs), name=name or f"rgg_n{n}_r{radius:.4f}")
    g.meta.update(dict(kind="rgg", n=n, radius=radius, seed=seed))
    return g


def path_graph(n: int, w=None) -> CSRGraph:
    u = np.arange(n - 1)
    return from_edges(n, u, u + 1, w, name=f"path{n}")


def star_graph(n: int) -> CSRGraph:
    u = np.zeros(n - 1, dtype=np.int64)
    return from_edges(n, u, np.arange(1, n), name=f"star{n}")


def er_batch(count: int, seed0: int, n_lo: int = 800, n_hi: int = 3000,
             d_lo: float = 3.0, d_hi: float = 48.0):
    """Independent ER instances: instance i uses seed seed0 + i; n ~ U[n_lo, n_hi],
    average degree d ~ U[d_lo, d_hi] (p = d / (n - 1)); weights unit or +-1 by a fair coin."""
    out = []
    for i in range(count):
        s = seed0 + i
        n = n_lo + int(_uint_below(s, 7, np.array([0]), np.array([n_hi - n_lo + 1]))[0])
        d = d_lo + (d_hi - d_lo) * float(uniform01(s, 8, np.array([0]))[0])
        signed = bool(uniform01(s, 9, np.array([0]))[0] < 0.5)
        g = erdos_renyi(n, d / (n - 1), s, signed=signed, name=f"er_batch_{s}")
        out.append(g)
    return out


def batch_union(graphs):
    """Disjoint union of graphs: returns (inst_ptr int64 [k+1], CSRGraph over all vertices)."""
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    inst_ptr = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    nnzs = np.array([g.nnz for g in graphs], dtype=np.int64)
    eoff = np.concatenate([[0], np.cumsum(nnzs)])
    N = int(inst_ptr[-1])
    row_ptr = np.empty(N + 1, dtype=np.int64)
    col = np.empty(int(eoff[-1]), dtype=np.int32)
    w = np.empty(int(eoff[-1]), dtype=np.int32)
    color = None
    if all(g.color is not None for g in graphs):
        color = np.concatenate([g.color for g in graphs]).astype(np.int32)
    for i, g in enumerate(graphs):
        row_ptr[inst_ptr[i]:inst_ptr[i + 1]] = g.row_ptr[:-1] + eoff[i]
        col[eoff[i]:eoff[i + 1]] = g.col + inst_ptr[i]
        w[eoff[i]:eoff[i + 1]] = g.w
    row_ptr[N] = eoff[-1]
    return inst_ptr, CSRGraph(n=N, row_ptr=row_ptr, col=col, w=w, name=f"batch{len(graphs)}", color=color)
