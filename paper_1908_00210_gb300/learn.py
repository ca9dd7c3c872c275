"""Learned warm start: a message-passing network that predicts where annealing should start.

Every computation runs in libgdi.so's kernels (include/gdi_mpnn.h); this module only holds device
buffers (torch tensors) and calls the C ABI.  The plain random-start annealer produces the training
labels and judges the result: a graph is "reached" when an anneal from the network's exactly
balanced prediction, started at a low temperature, matches the median cut of full random-start
anneals.

    python -m paper_1908_00210_gb300.learn --train 1024 --test 128 --out results.json
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import os
import time
from dataclasses import dataclass

import numpy as np

from . import _binding as B

HID = 64
FIN = 16
LAYER_DIMS = [(FIN, HID), (HID, HID), (HID, HID)]

MPNN_EXPORTS = ["gdi_mpnn_features", "gdi_mpnn_aggregate", "gdi_mpnn_dense_fwd", "gdi_mpnn_dense_bwd",
                "gdi_mpnn_wgrad", "gdi_mpnn_out_fwd", "gdi_mpnn_out_bwd", "gdi_mpnn_loss",
                "gdi_mpnn_adam", "gdi_mpnn_to_bf16", "gdi_mpnn_round"]

_L = None


def lib():
    global _L
    if _L is None:
        L = B.load()
        vp, i32, i64, f32, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_uint64
        L.gdi_mpnn_features.argtypes = [i64, i32, vp, vp, vp, vp, u64, i32, i32, vp, vp, vp]
        L.gdi_mpnn_aggregate.argtypes = [i64, vp, vp, vp, i32, vp, i32, i32, vp]
        L.gdi_mpnn_dense_fwd.argtypes = [i64, vp, vp, i32, vp, vp, vp, vp, vp]
        L.gdi_mpnn_dense_bwd.argtypes = [i64, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.gdi_mpnn_wgrad.argtypes = [i64, vp, i32, vp, i32, vp, vp, vp]
        L.gdi_mpnn_out_fwd.argtypes = [i64, vp, vp, vp, vp, vp]
        L.gdi_mpnn_out_bwd.argtypes = [i64, vp, vp, vp, vp]
        L.gdi_mpnn_loss.argtypes = [i32, vp, vp, vp, f32, vp, vp, vp, vp]
        L.gdi_mpnn_adam.argtypes = [i64, vp, vp, vp, vp, vp, f32, f32, f32, f32, i32, vp]
        L.gdi_mpnn_to_bf16.argtypes = [i64, vp, vp, vp]
        L.gdi_mpnn_round.argtypes = [i32, vp, i32, vp, vp, vp]
        for n in MPNN_EXPORTS:
            getattr(L, n).restype = C.c_int
        _L = L
    return _L


def _ok(rc, what):
    if rc != 0:
        raise B.GdiError(rc, what)


def param_layout():
    off, o = {}, 0
    for l, (din, dout) in enumerate(LAYER_DIMS, start=1):
        off[f"Ws{l}"] = (o, din * dout); o += din * dout
        off[f"Wn{l}"] = (o, din * dout); o += din * dout
        off[f"b{l}"] = (o, dout); o += dout
    off["wo"] = (o, HID); o += HID
    off["bo"] = (o, 1); o += 1
    return off, o


def init_params(seed: int = 0) -> np.ndarray:
    """Glorot-uniform matrices, zero biases (float32 master weights)."""
    off, total = param_layout()
    rng = np.random.default_rng(seed)
    p = np.zeros(total, dtype=np.float32)
    for l, (din, dout) in enumerate(LAYER_DIMS, start=1):
        a = math.sqrt(6.0 / (din + dout))
        for k in ("Ws", "Wn"):
            o, n = off[f"{k}{l}"]
            p[o:o + n] = rng.uniform(-a, a, n)
    o, n = off["wo"]
    p[o:o + n] = rng.uniform(-math.sqrt(6 / (HID + 1)), math.sqrt(6 / (HID + 1)), n)
    return p


@dataclass
class GraphBatch:
    """A disjoint union of graphs resident on the device."""
    N: int
    G: int
    max_n: int
    graph_ptr_h: np.ndarray
    row_ptr: "object"
    col: "object"
    graph_ptr: "object"
    graph_id: "object"
    graphs: list

    @staticmethod
    def from_graphs(graphs, graph_ids=None, device="cuda"):
        import torch
        from gdi_synth import batch_union
        gp, u = batch_union(graphs)
        ids = np.arange(len(graphs), dtype=np.uint32) if graph_ids is None else np.asarray(graph_ids, dtype=np.uint32)
        return GraphBatch(N=int(u.n), G=len(graphs), max_n=int(max(g.n for g in graphs)), graph_ptr_h=gp,
                          row_ptr=torch.from_numpy(u.row_ptr).to(device),
                          col=torch.from_numpy(u.col).to(device),
                          graph_ptr=torch.from_numpy(gp).to(device),
                          graph_id=torch.from_numpy(ids.view(np.int32)).to(device), graphs=list(graphs))


class MPNN:
    """Parameters, optimiser state and activation buffers of the network on the device."""

    def __init__(self, params: np.ndarray | None = None, seed: int = 0, lr: float = 1e-3,
                 lam: float = 0.1, feat_seed: int = 0x9E3779B9, steps: int = 256, feat_flags: int = 0):
        import torch
        self.torch = torch
        off, total = param_layout()
        self.off, self.P = off, total
        p = init_params(seed) if params is None else np.asarray(params, dtype=np.float32)
        self.params = torch.from_numpy(p.copy()).cuda()
        self.params_bf16 = torch.zeros(total, dtype=torch.int16, device="cuda")
        self.grads = torch.zeros(total, dtype=torch.float32, device="cuda")
        self.m = torch.zeros_like(self.grads)
        self.v = torch.zeros_like(self.grads)
        self.step = 0
        self.lr, self.lam, self.feat_seed, self.steps = lr, lam, feat_seed, steps
        self.feat_flags = feat_flags          # GDI_MPNN_ALIGN | GDI_MPNN_NO_NOISE
        _ok(lib().gdi_mpnn_to_bf16(total, self.params.data_ptr(), self.params_bf16.data_ptr(), self._st()), "to_bf16")

    def _st(self):
        return C.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def _pf(self, key):      # float32 master slice
        return self.params.data_ptr() + 4 * self.off[key][0]

    def _pb(self, key):      # bf16 slice
        return self.params_bf16.data_ptr() + 2 * self.off[key][0]

    def _gf(self, key):
        return self.grads.data_ptr() + 4 * self.off[key][0]

    # ---------------------------------------------------------------- forward / backward -----
    def features(self, b: GraphBatch):
        t = self.torch
        X = t.empty((b.N, FIN), dtype=t.float32, device="cuda")
        scratch = t.empty((2 * b.N * 8,), dtype=t.float32, device="cuda")
        _ok(lib().gdi_mpnn_features(b.N, b.G, b.graph_ptr.data_ptr(), b.graph_id.data_ptr(), b.row_ptr.data_ptr(),
                                    b.col.data_ptr(), self.feat_seed, self.steps, self.feat_flags, X.data_ptr(),
                                    scratch.data_ptr(),
                                    self._st()), "features")
        return X

    def forward(self, b: GraphBatch, X=None):
        t = self.torch
        L = lib()
        if X is None:
            X = self.features(b)
        cache = []
        h = X
        for l, (din, dout) in enumerate(LAYER_DIMS, start=1):
            agg = t.empty((b.N, din), dtype=t.float32, device="cuda")
            _ok(L.gdi_mpnn_aggregate(b.N, b.row_ptr.data_ptr(), b.col.data_ptr(), h.data_ptr(), din, agg.data_ptr(),
                                     0, 0, self._st()), "aggregate")
            out = t.empty((b.N, HID), dtype=t.float32, device="cuda")
            _ok(L.gdi_mpnn_dense_fwd(b.N, h.data_ptr(), agg.data_ptr(), din, self._pb(f"Ws{l}"), self._pb(f"Wn{l}"),
                                     self._pf(f"b{l}"), out.data_ptr(), self._st()), "dense_fwd")
            cache.append((h, agg, out, din))
            h = out
        z = t.empty((b.N,), dtype=t.float32, device="cuda")
        _ok(L.gdi_mpnn_out_fwd(b.N, h.data_ptr(), self._pb("wo"), self._pf("bo"), z.data_ptr(), self._st()), "out_fwd")
        return z, cache

    def loss_and_backward(self, b: GraphBatch, y, z, cache):
        """Loss (device scalar) and the gradients in self.grads."""
        t = self.torch
        L = lib()
        self.grads.zero_()
        loss = t.zeros(1, dtype=t.float32, device="cuda")
        stats = t.empty((b.G, 4), dtype=t.float32, device="cuda")
        dz = t.empty((b.N,), dtype=t.float32, device="cuda")
        _ok(L.gdi_mpnn_loss(b.G, b.graph_ptr.data_ptr(), z.data_ptr(), y.data_ptr(), self.lam, stats.data_ptr(),
                            dz.data_ptr(), loss.data_ptr(), self._st()), "loss")
        h3 = cache[-1][2]
        _ok(L.gdi_mpnn_wgrad(b.N, h3.data_ptr(), HID, dz.data_ptr(), 1, self._gf("wo"), self._gf("bo"), self._st()),
            "wgrad out")
        dh = t.empty((b.N, HID), dtype=t.float32, device="cuda")
        _ok(L.gdi_mpnn_out_bwd(b.N, self._pb("wo"), dz.data_ptr(), dh.data_ptr(), self._st()), "out_bwd")
        for l in (3, 2, 1):
            h_in, agg, out, din = cache[l - 1]
            dpre = t.empty((b.N, HID), dtype=t.float32, device="cuda")
            dxs = t.empty((b.N, din), dtype=t.float32, device="cuda")
            tt = t.empty((b.N, din), dtype=t.float32, device="cuda")
            _ok(L.gdi_mpnn_dense_bwd(b.N, din, self._pb(f"Ws{l}"), self._pb(f"Wn{l}"), out.data_ptr(), dh.data_ptr(),
                                     dpre.data_ptr(), dxs.data_ptr(), tt.data_ptr(), self._st()), "dense_bwd")
            _ok(L.gdi_mpnn_wgrad(b.N, h_in.data_ptr(), din, dpre.data_ptr(), HID, self._gf(f"Ws{l}"), self._gf(f"b{l}"),
                                 self._st()), "wgrad Ws")
            _ok(L.gdi_mpnn_wgrad(b.N, agg.data_ptr(), din, dpre.data_ptr(), HID, self._gf(f"Wn{l}"), None, self._st()),
                "wgrad Wn")
            if l > 1:
                _ok(L.gdi_mpnn_aggregate(b.N, b.row_ptr.data_ptr(), b.col.data_ptr(), tt.data_ptr(), din, dxs.data_ptr(),
                                         1, 1, self._st()), "aggregate T")
                dh = dxs
        return loss, stats

    def adam(self, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        _ok(lib().gdi_mpnn_adam(self.P, self.params.data_ptr(), self.grads.data_ptr(), self.m.data_ptr(),
                                self.v.data_ptr(), self.params_bf16.data_ptr(), self.lr, beta1, beta2, eps, self.step,
                                self._st()), "adam")

    def train_step(self, b: GraphBatch, y, X=None):
        z, cache = self.forward(b, X)
        loss, _ = self.loss_and_backward(b, y, z, cache)
        self.adam()
        return loss

    def predict_spins(self, b: GraphBatch):
        """Exactly balanced spins (int8, device [N]) from the network's logits."""
        t = self.torch
        z, _ = self.forward(b)
        s = t.empty((b.N,), dtype=t.int8, device="cuda")
        _ok(lib().gdi_mpnn_round(b.G, b.graph_ptr.data_ptr(), b.max_n, z.data_ptr(), s.data_ptr(), self._st()), "round")
        return s


# -------------------------------------------------------------------- data and evaluation -----
def make_graphs(count: int, seed0: int, n_lo=1000, n_hi=5000):
    """Half Erdos-Renyi (mean degree ~ U[3, 48]), half random geometric (mean degree ~ U[4, 32])."""
    from gdi_synth import erdos_renyi, random_geometric, uniform01
    out = []
    for i in range(count):
        s = seed0 + i
        u = uniform01(s, 11, np.arange(3))
        n = int(n_lo + u[0] * (n_hi - n_lo + 1))
        if i % 2 == 0:
            d = 3.0 + 45.0 * u[1]
            out.append(erdos_renyi(n, d / (n - 1), s, name=f"er{s}"))
        else:
            d = 4.0 + 28.0 * u[1]
            r = math.sqrt(d / (math.pi * (n - 1)))
            out.append(random_geometric(n, r, s, name=f"rgg{s}"))
    return out


def _graph_chunk(args):
    count, seed0, n_lo, n_hi = args
    return make_graphs(count, seed0, n_lo, n_hi)


def make_graphs_parallel(count: int, seed0: int, n_lo=1000, n_hi=5000, processes=16, chunk=256):
    """make_graphs in spawned worker processes (same graphs, same order); the graph of index i
    always comes from seed seed0 + i, so chunks keep the ER / RGG alternation only if `chunk` is
    even."""
    import multiprocessing as mp
    jobs = [(min(chunk, count - i), seed0 + i, n_lo, n_hi) for i in range(0, count, chunk)]
    with mp.get_context("spawn").Pool(processes) as pool:
        parts = pool.map(_graph_chunk, jobs)
    return [g for part in parts for g in part]


class Dataset:
    """Training graphs resident on the device as one disjoint union (CSR, features, labels), cut
    into batches of `batch` consecutive graphs without copying the graphs themselves."""

    def __init__(self, graphs, labels, model, batch=16, chunk=2048):
        import torch
        from gdi_synth import batch_union
        self.graphs = graphs
        gp, u = batch_union(graphs)
        self.gp = gp
        self.row_ptr_h = u.row_ptr
        self.row_ptr = torch.from_numpy(u.row_ptr).cuda()
        self.col = torch.from_numpy(u.col).cuda()
        self.y = torch.from_numpy(np.asarray(labels, dtype=np.int8)).cuda()
        self.X = torch.empty((int(gp[-1]), FIN), dtype=torch.float32, device="cuda")
        for g0 in range(0, len(graphs), chunk):      # features of every graph, once
            g1 = min(len(graphs), g0 + chunk)
            b = self.batch(g0, g1, with_x=False)
            self.X[int(gp[g0]):int(gp[g1])] = model.features(b)
        self.bsize = batch

    def batch(self, g0, g1, with_x=True):
        import torch
        v0, v1 = int(self.gp[g0]), int(self.gp[g1])
        e0, e1 = int(self.row_ptr_h[v0]), int(self.row_ptr_h[v1])
        b = GraphBatch(N=v1 - v0, G=g1 - g0, max_n=int(max(g.n for g in self.graphs[g0:g1])),
                       graph_ptr_h=self.gp[g0:g1 + 1] - v0,
                       row_ptr=(self.row_ptr[v0:v1 + 1] - e0).contiguous(),
                       col=(self.col[e0:e1] - v0).contiguous(),
                       graph_ptr=torch.from_numpy(self.gp[g0:g1 + 1] - v0).cuda(),
                       graph_id=torch.from_numpy(np.arange(g0, g1, dtype=np.int32)).cuda(),
                       graphs=self.graphs[g0:g1])
        return (b, self.X[v0:v1], self.y[v0:v1]) if with_x else b


def train_dataset(model: MPNN, ds: Dataset, *, epochs=10, seed=0, log=None):
    """Adam over the dataset's batches (consecutive groups of graphs, visited in a new random
    order every epoch)."""
    rng = np.random.default_rng(seed)
    starts = np.arange(0, len(ds.graphs), ds.bsize)
    history = []
    for ep in range(epochs):
        rng.shuffle(starts)
        tot = 0.0
        for g0 in starts:
            g1 = min(len(ds.graphs), g0 + ds.bsize)
            b, X, y = ds.batch(int(g0), int(g1))
            loss = model.train_step(b, y, X)
            tot += float(loss.item()) * (g1 - g0)
        history.append(tot / len(ds.graphs))
        if log:
            log(f"epoch {ep}: loss {history[-1]:.4f}")
    return history


def anneal_batch(graphs, *, sweeps, t0, t1, seed, replicas, init=None, A=1, Bc=4, W=256, stream=None):
    """Random-start (or given-start) anneal of every graph; returns (final_cut [G, R], spins [R, N],
    GPU milliseconds of the anneal kernel launch sequence)."""
    import torch
    from gdi_synth import batch_union
    gp, u = batch_union(graphs)
    ann = B.Annealer(u, A=A, B=Bc, W=W, replicas=replicas, inst_ptr=gp)
    sch = B.Schedule(sweeps=sweeps, t0=t0 * Bc, t1=t1 * Bc)
    st = stream or torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    if init is None:
        ann.anneal(sch, seed, stream=st)
    else:
        ann.anneal(sch, seed, init_device_ptr=init.data_ptr(), stream=st)
    e1.record(st)
    cut = ann.results()["final_cut"]
    ms = e0.elapsed_time(e1)
    spins = ann.spins()
    ann.close()
    return cut, spins, ms


def label_graphs(graphs, *, sweeps=2000, replicas=4, seed=1, chunk=2048, A=1, start=None, t0=3.0):
    """Labels = the best (lowest repaired cut) of `replicas` anneals, annealed `chunk` graphs per
    batched launch: plain random-start anneals from T = t0, or (start = a function of a list of
    graphs returning exactly balanced device spins) anneals from that start."""
    ys, bests = [], []
    for g0 in range(0, len(graphs), chunk):
        part = graphs[g0:g0 + chunk]
        init = None if start is None else start(part).repeat(replicas)
        cut, spins, _ = anneal_batch(part, sweeps=sweeps, t0=t0, t1=0.05, seed=seed, replicas=replicas, A=A,
                                     init=init)
        from gdi_synth import batch_union
        gp, _ = batch_union(part)
        y = np.empty(gp[-1], dtype=np.int8)
        for g in range(len(part)):
            best = int(np.argmin(cut[g]))
            y[gp[g]:gp[g + 1]] = spins[best, gp[g]:gp[g + 1]]
        ys.append(y)
        bests.append(cut.min(axis=1))
    return np.concatenate(ys), np.concatenate(bests)


def train(model: MPNN, graphs, labels, *, epochs=30, batch=16, seed=0, log=None):
    import torch
    from gdi_synth import batch_union
    rng = np.random.default_rng(seed)
    gp_all, _ = batch_union(graphs)
    history = []
    batches = []
    order = np.arange(len(graphs))
    for ep in range(epochs):
        rng.shuffle(order)
        tot = 0.0
        for k in range(0, len(order), batch):
            idx = order[k:k + batch]
            gb = GraphBatch.from_graphs([graphs[i] for i in idx], graph_ids=idx)
            y = np.concatenate([labels[gp_all[i]:gp_all[i + 1]] for i in idx])
            loss = model.train_step(gb, torch.from_numpy(y).cuda())
            tot += float(loss.item()) * len(idx)
        history.append(tot / len(graphs))
        if log:
            log(f"epoch {ep}: loss {history[-1]:.4f}")
    return history


LADDER = [25, 50, 100, 200, 400, 800, 1600, 2000]


def evaluate(model: MPNN, graphs, *, seeds=8, full_sweeps=2000, ladder=LADDER, t_low=0.5, log=None):
    """Time to reach the random-start median cut: learned start at T0 = t_low, random start at
    T0 = 3.0, random start at T0 = t_low (control), all ending at T = 0.05."""
    import torch
    ref_cut, _, full_ms = anneal_batch(graphs, sweeps=full_sweeps, t0=3.0, t1=0.05, seed=101, replicas=seeds)
    c_ref = np.median(ref_cut, axis=1)
    gb = GraphBatch.from_graphs(graphs, graph_ids=np.arange(len(graphs)) + 1_000_000)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    pred = model.predict_spins(gb)
    e1.record()
    torch.cuda.synchronize()
    infer_ms = e0.elapsed_time(e1)
    init = pred.repeat(seeds)            # [seeds * N]: every replica starts from the prediction
    ns = np.array([g.n for g in graphs], dtype=np.float64)
    share = ns / ns.sum()                # a graph's share of a batched launch's GPU time
    methods = {f"learned_T{t_low}": dict(t0=t_low, init=init), "random_T3.0": dict(t0=3.0, init=None),
               f"random_T{t_low}": dict(t0=t_low, init=None)}
    out = {"c_ref_median": float(np.median(c_ref)), "full_random_ms": full_ms, "infer_ms": infer_ms,
           "graphs": len(graphs), "seeds": seeds, "ladder": ladder}
    times = {}
    for name, m in methods.items():
        reached_at = np.full(len(graphs), -1)
        rung_ms = {}
        for M in ladder:
            cut, _, ms = anneal_batch(graphs, sweeps=M, t0=m["t0"], t1=0.05, seed=202, replicas=seeds, init=m["init"])
            rung_ms[M] = ms
            med = np.median(cut, axis=1)
            newly = (reached_at < 0) & (med <= c_ref)
            reached_at[newly] = M
            if log:
                log(f"{name} M={M}: reached {int((reached_at > 0).sum())}/{len(graphs)} ({ms:.1f} ms)")
        t = np.array([rung_ms[M] * share[g] if M > 0 else np.nan for g, M in enumerate(reached_at)])
        if name.startswith("learned"):
            t = t + infer_ms * share
        ok = reached_at > 0
        times[name] = np.where(ok, t, np.nan)
        out[name] = {"fraction_reached": float(ok.mean()),
                     "median_sweeps_to_cut": float(np.median(reached_at[ok])) if ok.any() else None,
                     "median_gpu_ms_to_cut": float(np.median(t[ok])) if ok.any() else None,
                     "total_gpu_ms_reached_graphs": float(np.nansum(t[ok])), "rung_ms": rung_ms}
    # paired comparison on the graphs that both the learned and the random start reach
    a, b = times[f"learned_T{t_low}"], times["random_T3.0"]
    both = np.isfinite(a) & np.isfinite(b)
    out["paired"] = {"graphs_both_reached": int(both.sum()),
                     "median_time_ratio_random_over_learned": float(np.median(b[both] / a[both])) if both.any() else None,
                     "learned_faster_fraction": float(np.mean(a[both] < b[both])) if both.any() else None}
    return out


def evaluate_many(starts, graphs, *, seeds=8, full_sweeps=2000, ladder=LADDER, A=1, log=None):
    """Like evaluate, for several learned starts at once: starts = {name: (model, t_low)}.  The
    target, the plain annealer's ladder (random start, T0 = 3.0) and a random-start control at every
    t_low are computed once."""
    import torch
    ref_cut, _, full_ms = anneal_batch(graphs, sweeps=full_sweeps, t0=3.0, t1=0.05, seed=101, replicas=seeds, A=A)
    c_ref = np.median(ref_cut, axis=1)
    ns = np.array([g.n for g in graphs], dtype=np.float64)
    share = ns / ns.sum()
    out = {"c_ref_median": float(np.median(c_ref)), "full_random_ms": full_ms, "graphs": len(graphs),
           "seeds": seeds, "ladder": ladder, "A": A}
    methods = {"random_T3.0": dict(t0=3.0, init=None, infer=0.0)}
    for t_low in sorted({st[-2] if st[0] == "spins" and len(st) > 3 else st[-1] for st in starts.values()}):
        methods[f"random_T{t_low}"] = dict(t0=t_low, init=None, infer=0.0)
    for name, st in starts.items():
        if st[0] == "spins":                         # a start given as spins (already computed)
            methods[name] = dict(t0=st[2], init=st[1].repeat(seeds), infer=st[3] if len(st) > 3 else 0.0)
            continue
        model, t_low = st
        gb = GraphBatch.from_graphs(graphs, graph_ids=np.arange(len(graphs)) + 1_000_000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        pred = model.predict_spins(gb)
        e1.record()
        torch.cuda.synchronize()
        methods[name] = dict(t0=t_low, init=pred.repeat(seeds), infer=e0.elapsed_time(e1))
    times = {}
    for name, m in methods.items():
        reached_at = np.full(len(graphs), -1)
        rung_ms, rung_reached = {}, {}
        for M in ladder:
            cut, _, ms = anneal_batch(graphs, sweeps=M, t0=m["t0"], t1=0.05, seed=202, replicas=seeds,
                                      init=m["init"], A=A)
            rung_ms[M] = ms
            med = np.median(cut, axis=1)
            newly = (reached_at < 0) & (med <= c_ref)
            reached_at[newly] = M
            rung_reached[M] = int((reached_at > 0).sum())
            if log:
                log(f"{name} M={M}: reached {rung_reached[M]}/{len(graphs)} ({ms:.1f} ms)")
        t = np.array([rung_ms[M] * share[g] if M > 0 else np.nan for g, M in enumerate(reached_at)])
        t = t + m["infer"] * share
        ok = reached_at > 0
        times[name] = np.where(ok, t, np.nan)
        out[name] = {"reached": rung_reached, "median_sweeps_to_cut": float(np.median(reached_at[ok])) if ok.any() else None,
                     "median_gpu_ms_to_cut": float(np.median(t[ok])) if ok.any() else None,
                     "infer_ms": m["infer"], "rung_ms": rung_ms}
    for name in starts:
        a, b = times[name], times["random_T3.0"]
        both = np.isfinite(a) & np.isfinite(b)
        out[name]["paired_vs_random_T3.0"] = {
            "graphs_both_reached": int(both.sum()),
            "median_time_ratio_random_over_learned": float(np.median(b[both] / a[both])) if both.any() else None,
            "learned_faster_fraction": float(np.mean(a[both] < b[both])) if both.any() else None}
    return out


def ablate(args, log):
    """One set of graphs and labels; a network per feature setting (diffusion steps), each
    evaluated at every start temperature against one shared plain-annealer reference."""
    import torch
    t0 = time.time()
    train_graphs = make_graphs_parallel(args.train, 500_000, processes=args.processes)
    test_graphs = make_graphs_parallel(args.test, 900_000, processes=args.processes)
    log(f"graphs generated in {time.time() - t0:.1f} s")
    torch.cuda.set_device(0)
    t0 = time.time()
    labels, _ = label_graphs(train_graphs, sweeps=args.label_sweeps, A=args.A)
    log(f"labels in {time.time() - t0:.1f} s")
    starts, losses = {}, {}
    for steps in [int(x) for x in args.ablate_steps.split(",")]:
        model = MPNN(seed=0, lr=args.lr, lam=args.lam, steps=steps)
        ds = Dataset(train_graphs, labels, model)
        t0 = time.time()
        losses[steps] = train_dataset(model, ds, epochs=args.epochs, log=log)
        log(f"steps {steps}: trained in {time.time() - t0:.1f} s")
        del ds
        for t_low in [float(x) for x in args.ablate_t.split(",")]:
            starts[f"learned_steps{steps}_T{t_low}"] = (model, t_low)
    res = evaluate_many(starts, test_graphs, A=args.A, log=log)
    res["train_loss"] = {str(k): v for k, v in losses.items()}
    res["train_graphs"] = args.train
    return res


def channel_spins(model: "MPNN", graphs, channel: int = 0):
    """Exactly balanced spins from one input feature channel alone (the diffused noise channel 0 is a
    cheap spectral embedding): the same rounding as the network's logits, applied to X[:, channel]."""
    import torch
    gb = GraphBatch.from_graphs(graphs, graph_ids=np.arange(len(graphs)) + 1_000_000)
    X = model.features(gb)
    z = X[:, channel].contiguous()
    s = torch.empty((gb.N,), dtype=torch.int8, device="cuda")
    _ok(lib().gdi_mpnn_round(gb.G, gb.graph_ptr.data_ptr(), gb.max_n, z.data_ptr(), s.data_ptr(), model._st()), "round")
    return s


def ablate_starts(args, log):
    """What the trained network adds: one set of graphs and labels; the held-out graphs annealed
    from (1) the rounded diffused noise channel 0 alone, (2) an untrained network, (3) a network
    trained without the noise channels, (4) the trained network, next to the plain annealer and the
    random start at the same low temperature.  Features sign-aligned per graph (GDI_MPNN_ALIGN)
    unless --no-align."""
    import torch
    t0 = time.time()
    train_graphs = make_graphs_parallel(args.train, 500_000, processes=args.processes)
    test_graphs = make_graphs_parallel(args.test, 900_000, processes=args.processes)
    log(f"graphs generated in {time.time() - t0:.1f} s")
    torch.cuda.set_device(0)
    t0 = time.time()
    flags = 0 if args.no_align else 1
    if args.label_start == "spectral":
        # labels refined from the network's own spectral input: the rounded noise channel 0,
        # annealed from T0 = t_low -- a target that is one good partition the features point to
        probe = MPNN(seed=0, steps=args.steps, feat_flags=flags)
        labels, _ = label_graphs(train_graphs, sweeps=args.label_sweeps, A=args.A, t0=args.t_low,
                                 start=lambda part: channel_spins(probe, part, 0))
    else:
        labels, _ = label_graphs(train_graphs, sweeps=args.label_sweeps, A=args.A)
    log(f"labels ({args.label_start} start) in {time.time() - t0:.1f} s")
    nets, losses = {}, {}
    for name, fl in (("trained", flags), ("trained_no_noise", flags | 2)):
        model = MPNN(seed=0, lr=args.lr, lam=args.lam, steps=args.steps, feat_flags=fl)
        ds = Dataset(train_graphs, labels, model)
        t0 = time.time()
        losses[name] = train_dataset(model, ds, epochs=args.epochs, log=log)
        log(f"{name}: trained in {time.time() - t0:.1f} s, loss {losses[name][0]:.4f} -> {losses[name][-1]:.4f}")
        del ds
        nets[name] = model
    untrained = MPNN(seed=0, lr=args.lr, lam=args.lam, steps=args.steps, feat_flags=flags)
    t = args.t_low
    starts = {"noise_channel0": ("spins", channel_spins(untrained, test_graphs, 0), t),
              "untrained": (untrained, t), "trained_no_noise": (nets["trained_no_noise"], t),
              "trained": (nets["trained"], t)}
    res = evaluate_many(starts, test_graphs, A=args.A, log=log)
    res["train_loss"] = losses
    res["train_graphs"] = args.train
    res["feature_flags"] = flags
    res["label_start"] = args.label_start
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--train", type=int, default=1024)
    ap.add_argument("--test", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--label-sweeps", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=256, help="lazy-walk diffusion steps of the features")
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lam", type=float, default=0.1)
    ap.add_argument("--t-low", type=float, default=0.5)
    ap.add_argument("--out", default="")
    ap.add_argument("--processes", type=int, default=16, help="host processes generating the graphs")
    ap.add_argument("--A", type=int, default=1, help="balance weight of the anneals (labels and evaluation)")
    ap.add_argument("--ablate-steps", default="", help="comma list of diffusion steps: ablation mode")
    ap.add_argument("--ablate-t", default="0.5", help="comma list of start temperatures (ablation mode)")
    ap.add_argument("--ablate-starts", action="store_true",
                    help="compare the trained network with the noise channel alone, an untrained network "
                         "and a network trained without the noise channels")
    ap.add_argument("--no-align", action="store_true", help="features without the per-graph sign alignment")
    ap.add_argument("--label-start", default="random", choices=["random", "spectral"],
                    help="training labels from random-start anneals (T0 = 3.0) or from anneals that start at "
                         "the rounded noise channel 0 (T0 = --t-low) (--ablate-starts)")
    args = ap.parse_args()
    log = lambda s: print(s, flush=True)  # noqa: E731
    if args.ablate_starts:
        res = ablate_starts(args, log)
        print(json.dumps({k: v for k, v in res.items() if k != "train_loss"}, default=str))
        if args.out:
            with open(args.out, "w") as f:
                json.dump(res, f, default=str, indent=1)
        return
    if args.ablate_steps:
        res = ablate(args, log)
        print(json.dumps({k: v for k, v in res.items() if k != "train_loss"}, default=str))
        if args.out:
            with open(args.out, "w") as f:
                json.dump(res, f, default=str, indent=1)
        return
    t0 = time.time()
    train_graphs = make_graphs_parallel(args.train, 500_000, processes=args.processes)
    test_graphs = make_graphs_parallel(args.test, 900_000, processes=args.processes)
    log(f"graphs generated in {time.time() - t0:.1f} s")
    import torch
    torch.cuda.set_device(0)
    t0 = time.time()
    labels, best = label_graphs(train_graphs, sweeps=args.label_sweeps)
    torch.cuda.synchronize()
    log(f"labels in {time.time() - t0:.1f} s")
    model = MPNN(seed=0, lr=args.lr, lam=args.lam, steps=args.steps)
    t0 = time.time()
    ds = Dataset(train_graphs, labels, model)
    torch.cuda.synchronize()
    log(f"features of the training graphs in {time.time() - t0:.1f} s")
    t0 = time.time()
    hist = train_dataset(model, ds, epochs=args.epochs, log=log)
    torch.cuda.synchronize()
    log(f"trained in {time.time() - t0:.1f} s")
    res = evaluate(model, test_graphs, log=log, t_low=args.t_low)
    res["train_loss"] = hist
    res["steps"] = args.steps
    res["train_graphs"] = args.train
    res["label_sweeps"] = args.label_sweeps
    print(json.dumps({k: v for k, v in res.items() if k != "train_loss"}, default=str))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, default=str, indent=1)


if __name__ == "__main__":
    main()
