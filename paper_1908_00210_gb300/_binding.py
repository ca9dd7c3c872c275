"""ctypes binding of libgdi.so (include/gdi.h): argument marshalling only.

Every step of the annealing path runs in the library's CUDA kernels; there is no Python or CPU
fallback.  If libgdi.so is missing, load() raises: build it with paper_1908_00210_gb300.build().
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgdi.so")

GDI_MEM_HOST, GDI_MEM_DEVICE = 0, 1
GDI_METROPOLIS, GDI_PAPER_PF = 0, 1
GDI_FLAG_TRACE, GDI_FLAG_NO_REPAIR, GDI_FLAG_CONTINUE, GDI_FLAG_RACY, GDI_FLAG_STANDARD = 1, 2, 4, 8, 16

ERRORS = {
    -1: "GDI_ERR_INVALID_ARG", -2: "GDI_ERR_NOT_SYMMETRIC", -3: "GDI_ERR_SELF_LOOP",
    -4: "GDI_ERR_DUP_EDGE", -5: "GDI_ERR_BAD_COLORING", -6: "GDI_ERR_OVERFLOW", -7: "GDI_ERR_OOM",
    -8: "GDI_ERR_CUDA", -9: "GDI_ERR_TIMEOUT", -10: "GDI_ERR_NOT_ANNEALED", -11: "GDI_ERR_TOO_LARGE",
}

# every entry point that include/gdi.h declares
EXPORTS = ["gdi_create", "gdi_anneal", "gdi_get_spins", "gdi_get_results", "gdi_cut", "gdi_balance",
           "gdi_get_trace", "gdi_configure", "gdi_last_launch", "gdi_info", "gdi_destroy",
           "gdi_strerror", "gdi_last_error", "gdi_anneal_static", "gdi_autotune", "gdi_kernel_time",
           "gdi_inject_wait_failure", "gdi_rank_space", "gdi_build_table", "gdi_anneal_static_status"]
GDI_PATH_AUTO, GDI_PATH_CTA, GDI_PATH_GRID = 0, 1, 2


class GdiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class gdi_graph(C.Structure):
    _fields_ = [("num_instances", C.c_int32), ("inst_ptr", C.c_void_p), ("num_vertices", C.c_int64),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("weight", C.c_void_p), ("color", C.c_void_p)]


class gdi_model(C.Structure):
    _fields_ = [("A", C.c_int32), ("B", C.c_int32), ("W", C.c_int32), ("replicas", C.c_int32)]


class gdi_schedule(C.Structure):
    _fields_ = [("mode", C.c_int32), ("t0", C.c_double), ("t1", C.c_double), ("pf0", C.c_double),
                ("pf1", C.c_double), ("sweeps", C.c_int32)]


class gdi_run(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("first_sweep", C.c_int32), ("last_sweep", C.c_int32),
                ("flags", C.c_int32), ("init_spins", C.c_void_p), ("init_mem", C.c_int32),
                ("stream", C.c_void_p)]


_lib = None


def load():
    """Load libgdi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1908_00210_gb300.build() "
                           "(nvcc, sm_103a); there is no fallback implementation")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    L.gdi_create.argtypes = [C.POINTER(vp), C.POINTER(gdi_graph), C.POINTER(gdi_model)]
    L.gdi_anneal.argtypes = [vp, C.POINTER(gdi_schedule), C.POINTER(gdi_run)]
    L.gdi_get_spins.argtypes = [vp, vp, i32]
    L.gdi_get_results.argtypes = [vp, vp, vp, vp, vp]
    L.gdi_cut.argtypes = [vp, i32, i32, vp]
    L.gdi_balance.argtypes = [vp, i32, i32, vp, vp]
    L.gdi_get_trace.argtypes = [vp, vp, vp, vp]
    L.gdi_info.argtypes = [vp, vp, vp, vp]
    L.gdi_configure.argtypes = [vp, i32, i32, i32]
    L.gdi_autotune.argtypes = [vp, C.POINTER(gdi_schedule), i32, vp, vp, vp]
    L.gdi_anneal_static.argtypes = [i32, vp, vp, i32, vp, i32, i32, i32, i32, i32, i32, vp, vp, vp,
                                    i32, i32, i32, i32, C.c_uint64, i32, vp, vp, vp]
    L.gdi_anneal_static_status.argtypes = [vp, vp]
    L.gdi_rank_space.argtypes = [C.POINTER(gdi_graph), vp, vp, vp, vp, vp, vp, vp]
    L.gdi_build_table.argtypes = [C.POINTER(gdi_schedule), vp, i64, vp, vp, vp, vp]
    L.gdi_last_launch.argtypes = [vp, vp, vp, vp, vp]
    L.gdi_kernel_time.argtypes = [vp, vp, vp]
    L.gdi_inject_wait_failure.argtypes = [vp, C.c_int64]
    L.gdi_destroy.argtypes = [vp]
    L.gdi_destroy.restype = None
    L.gdi_strerror.argtypes = [C.c_int]
    L.gdi_strerror.restype = C.c_char_p
    L.gdi_last_error.argtypes = []
    L.gdi_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("gdi_destroy", "gdi_strerror", "gdi_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(rc: int):
    if rc != 0:
        raise GdiError(rc, load().gdi_last_error().decode(errors="replace"))


def _ptr(a):
    return None if a is None else a.ctypes.data


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


@dataclass
class Schedule:
    """Annealing schedule (Section 5.2): Metropolis T geometric t0 -> t1, or the paper's P_f."""
    sweeps: int
    t0: float = 3.0
    t1: float = 0.05
    mode: int = GDI_METROPOLIS
    pf0: float = 0.2
    pf1: float = 0.01

    def c(self) -> gdi_schedule:
        return gdi_schedule(self.mode, self.t0, self.t1, self.pf0, self.pf1, self.sweeps)


class Annealer:
    """One gdi_ctx: a graph (or a batch of graphs) resident on the current CUDA device."""

    def __init__(self, graph, *, A: int = 1, B: int = 1, W: int = 0, replicas: int = 1,
                 color=None, inst_ptr=None):
        L = load()
        self.n = int(graph.n)
        self.replicas = int(replicas)
        rp = np.ascontiguousarray(graph.row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(graph.col, dtype=np.int32)
        w = np.ascontiguousarray(graph.w, dtype=np.int32) if getattr(graph, "w", None) is not None else None
        if color is None:
            color = getattr(graph, "color", None)
        colr = None if color is None else np.ascontiguousarray(color, dtype=np.int32)
        ip = None if inst_ptr is None else np.ascontiguousarray(inst_ptr, dtype=np.int64)
        self.num_instances = 1 if ip is None else len(ip) - 1
        g = gdi_graph(self.num_instances, _ptr(ip), self.n, _ptr(rp), _ptr(col), _ptr(w), _ptr(colr))
        m = gdi_model(A, B, W, replicas)
        h = C.c_void_p()
        _check(L.gdi_create(C.byref(h), C.byref(g), C.byref(m)))
        self._h = h
        self.sweeps = 0

    def close(self):
        if getattr(self, "_h", None):
            load().gdi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def anneal(self, schedule: Schedule, seed: int, *, init=None, init_device_ptr: int | None = None,
               flags: int = 0, first_sweep: int = 0, last_sweep: int = 0, stream=None):
        """Enqueue one anneal (asynchronous on `stream`)."""
        L = load()
        init_arr = None
        init_p, init_mem = None, GDI_MEM_HOST
        if init_device_ptr is not None:
            init_p, init_mem = init_device_ptr, GDI_MEM_DEVICE
        elif init is not None:
            init_arr = np.ascontiguousarray(init, dtype=np.int8).reshape(self.replicas, self.n)
            init_p = init_arr.ctypes.data
        run = gdi_run(seed & 0xFFFFFFFFFFFFFFFF, first_sweep, last_sweep, flags, init_p, init_mem,
                      _stream_handle(stream))
        s = schedule.c()
        _check(L.gdi_anneal(self._h, C.byref(s), C.byref(run)))
        self.sweeps = schedule.sweeps
        return self

    def spins(self) -> np.ndarray:
        out = np.empty((self.replicas, self.n), dtype=np.int8)
        _check(load().gdi_get_spins(self._h, out.ctypes.data, GDI_MEM_HOST))
        return out

    def spins_to_device(self, dev_ptr: int):
        _check(load().gdi_get_spins(self._h, dev_ptr, GDI_MEM_DEVICE))

    def results(self):
        k = self.num_instances * self.replicas
        rg = np.empty(k, np.int32)
        fg = np.empty(k, np.int32)
        rc = np.empty(k, np.int64)
        fc = np.empty(k, np.int64)
        _check(load().gdi_get_results(self._h, rg.ctypes.data, fg.ctypes.data, rc.ctypes.data, fc.ctypes.data))
        shp = (self.num_instances, self.replicas)
        return dict(raw_G=rg.reshape(shp), final_G=fg.reshape(shp), raw_cut=rc.reshape(shp),
                    final_cut=fc.reshape(shp))

    def cut(self, instance: int = 0, replica: int = 0) -> int:
        v = np.zeros(1, np.int64)
        _check(load().gdi_cut(self._h, instance, replica, v.ctypes.data))
        return int(v[0])

    def balance(self, instance: int = 0, replica: int = 0):
        a = np.zeros(1, np.int32)
        b = np.zeros(1, np.int32)
        _check(load().gdi_balance(self._h, instance, replica, a.ctypes.data, b.ctypes.data))
        return int(a[0]), int(b[0])

    def trace(self):
        k = self.num_instances * self.replicas
        d = np.empty((k, self.sweeps), np.uint64)
        g = np.empty((k, self.sweeps), np.int32)
        c = np.empty((k, self.sweeps), np.int64)
        _check(load().gdi_get_trace(self._h, d.ctypes.data, g.ctypes.data, c.ctypes.data))
        return d, g, c

    def configure(self, path: int = GDI_PATH_AUTO, block: int = 0, grid_limit: int = 0):
        _check(load().gdi_configure(self._h, path, block, grid_limit))
        return self

    def autotune(self, schedule: Schedule, probe_sweeps: int = 20):
        """Time candidate launch configurations on a schedule prefix and keep the fastest."""
        b = np.zeros(1, np.int32)
        g = np.zeros(1, np.int32)
        ms = np.zeros(1, np.float32)
        s = schedule.c()
        _check(load().gdi_autotune(self._h, C.byref(s), probe_sweeps, b.ctypes.data, g.ctypes.data, ms.ctypes.data))
        return dict(block=int(b[0]), grid=int(g[0]), ms=float(ms[0]))

    def capture_graph(self, schedule: Schedule, seed: int, stream, flags: int = 0):
        """Capture one anneal (random start) into a CUDA graph on `stream` (a torch.cuda.Stream);
        returns the torch.cuda.CUDAGraph, whose replay() re-runs it.  Call anneal() once with the
        same schedule before capturing so that every buffer and the table already exist."""
        import torch
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            self.anneal(schedule, seed, flags=flags, stream=torch.cuda.current_stream())
        return graph

    def last_launch(self):
        pa = np.zeros(1, np.int32)
        gr = np.zeros(1, np.int32)
        sm = np.zeros(1, np.int64)
        fb = np.zeros(1, np.int32)
        _check(load().gdi_last_launch(self._h, pa.ctypes.data, gr.ctypes.data, sm.ctypes.data, fb.ctypes.data))
        return dict(path=int(pa[0]), grid=int(gr[0]), smem=int(sm[0]), fallbacks=int(fb[0]))

    def inject_wait_failure(self, spin_limit: int = 1 << 16):
        """Make the next grid-scale anneal's device waits run out (test of failure detection)."""
        _check(load().gdi_inject_wait_failure(self._h, int(spin_limit)))

    def kernel_ms(self):
        """Device time (ms) of the last anneal's sweep-kernel launches and their number."""
        ms = np.zeros(1, np.float32)
        n = np.zeros(1, np.int32)
        _check(load().gdi_kernel_time(self._h, ms.ctypes.data, n.ctypes.data))
        return float(ms[0]), int(n[0])

    def info(self):
        nc = np.zeros(self.num_instances, np.int32)
        md = np.zeros(1, np.int32)
        ec = np.zeros(1, np.int32)
        _check(load().gdi_info(self._h, nc.ctypes.data, md.ctypes.data, ec.ctypes.data))
        return dict(num_classes=nc, max_degree=int(md[0]), ecap=int(ec[0]))


@dataclass
class RankSpace:
    """The rank-space layout of one graph (gdi_rank_space), as gdi_anneal_static takes it."""
    vert_of: np.ndarray      # int32 [n]: original vertex at rank r
    rank_of: np.ndarray      # int64 [n]: rank of original vertex v
    row_ptr: np.ndarray      # int64 [n + 1]
    col: np.ndarray          # uint32 [nnz]: neighbour rank | 0x80000000 for weight -1
    class_ptr: np.ndarray    # int32 [num_classes + 1]
    max_class: int
    max_degree: int


def rank_space(graph, color=None) -> RankSpace:
    """gdi_rank_space on one graph (host arrays; validation and colouring as gdi_create)."""
    L = load()
    n = int(graph.n)
    rp = np.ascontiguousarray(graph.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(graph.col, dtype=np.int32)
    w = np.ascontiguousarray(graph.w, dtype=np.int32) if getattr(graph, "w", None) is not None else None
    if color is None:
        color = getattr(graph, "color", None)
    colr = None if color is None else np.ascontiguousarray(color, dtype=np.int32)
    g = gdi_graph(1, None, n, _ptr(rp), _ptr(col), _ptr(w), _ptr(colr))
    vert = np.empty(n, np.int32)
    orp = np.empty(n + 1, np.int64)
    ocol = np.empty(int(rp[-1]), np.uint32)
    cls = np.empty(n + 1, np.int32)
    nc = np.zeros(1, np.int32)
    mc = np.zeros(1, np.int32)
    md = np.zeros(1, np.int32)
    _check(L.gdi_rank_space(C.byref(g), _ptr(vert), _ptr(orp), _ptr(ocol), _ptr(cls), _ptr(nc), _ptr(mc),
                            _ptr(md)))
    rank = np.empty(n, np.int64)
    rank[vert] = np.arange(n)
    return RankSpace(vert, rank, orp, ocol, cls[:int(nc[0]) + 1].copy(), int(mc[0]), int(md[0]))


def build_table(schedule: Schedule):
    """gdi_build_table: (tab uint32, tab_off int32 [M+1], temp float32 [M], max_row)."""
    L = load()
    s = schedule.c()
    ln = np.zeros(1, np.int64)
    mr = np.zeros(1, np.int32)
    _check(L.gdi_build_table(C.byref(s), None, 0, _ptr(ln), None, None, _ptr(mr)))
    tab = np.zeros(max(int(ln[0]), 1), np.uint32)
    off = np.zeros(schedule.sweeps + 1, np.int32)
    temp = np.zeros(schedule.sweeps, np.float32)
    _check(L.gdi_build_table(C.byref(s), _ptr(tab), len(tab), _ptr(ln), _ptr(off), _ptr(temp), _ptr(mr)))
    return tab, off, temp, int(mr[0])
