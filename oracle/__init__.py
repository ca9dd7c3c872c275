"""CPU oracle for the GDI annealer -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this package.
It wraps oracle/gdi_oracle.c (plain sequential C, built with gcc) through ctypes and shares no
code with the CUDA library in paper_1908_00210_gb300/.

Parity status of each function (what pins it, apart from itself):
  philox4x32_10      Triton's library Philox run by its CPU interpreter; uniformity and avalanche.
  greedy_color       properness + first-fit minimality checked by brute force in the tests.
  table              closed forms exp(-dE/T) and the P_f probabilities of Alg. 2/3.
  energy / cut       Eq. 3 with dense couplings J_ij = B w_ij / 2 - 2A (dense numpy), brute force.
  anneal             every flip decided by u < thr[s][clamp(dE at the running G)], with dE from
                     Eq. 4-6; W = 1 reduces to textbook single-spin Metropolis with the energy
                     recomputed from scratch (tests); W > 1 replayed with flip thresholds found by
                     scanning G with the energy recomputed from its definition, in both table
                     modes, for several replica and instance words; invariants (tracked G and cut
                     equal recomputation); brute-force optimum bound on n <= 20.
  bruteforce         exhaustive enumeration, checked on graphs with known bisection widths.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gdi_oracle.c")
_LIB = os.path.join(_HERE, "libgdi_oracle.so")

METROPOLIS = 0
PAPER_PF = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no SIMD intrinsics, portable across x86_64/aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("n", C.c_int32),
        ("row_ptr", C.c_void_p),
        ("col", C.c_void_p),
        ("w", C.c_void_p),
        ("color", C.c_void_p),
        ("A", C.c_int32), ("B", C.c_int32), ("W", C.c_int32),
        ("mode", C.c_int32),
        ("t0", C.c_double), ("t1", C.c_double), ("pf0", C.c_double), ("pf1", C.c_double),
        ("sweeps", C.c_int32),
        ("seed", C.c_uint64),
        ("instance", C.c_int32),
        ("replicas", C.c_int32),
        ("first_sweep", C.c_int32),
        ("last_sweep", C.c_int32),
        ("check_invariants", C.c_int32),
        ("first_replica", C.c_int32),
        ("stale", C.c_int32),
    ]


class _Out(C.Structure):
    _fields_ = [
        ("spins", C.c_void_p),
        ("use_init", C.c_int32),
        ("raw_G", C.c_void_p),
        ("final_G", C.c_void_p),
        ("raw_cut", C.c_void_p),
        ("final_cut", C.c_void_p),
        ("digest", C.c_void_p),
        ("G_trace", C.c_void_p),
        ("cut_trace", C.c_void_p),
        ("invariant_failures", C.c_int64),
        ("num_colors", C.c_int32),
        ("do_repair", C.c_int32),
        ("decision_mismatches", C.c_int64),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.oracle_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_philox4x32_10_many.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_table_ecap.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int]
        L.oracle_build_table.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                         C.c_int, C.c_int, C.c_void_p]
        L.oracle_greedy_color.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_cut.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_cut.restype = C.c_int64
        L.oracle_energy.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                    C.c_int32, C.c_void_p]
        L.oracle_energy.restype = C.c_int64
        L.oracle_bruteforce_bisection.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                                  C.c_void_p, C.c_void_p]
        L.oracle_anneal.argtypes = [C.POINTER(_Params), C.POINTER(_Out)]
        assert L.oracle_sizeof_params() == C.sizeof(_Params), "oracle_params layout mismatch"
        assert L.oracle_sizeof_out() == C.sizeof(_Out), "oracle_out layout mismatch"
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of counter ctr (4 x uint32) under key (2 x uint32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def philox4x32_10_many(ctr, key) -> np.ndarray:
    """Philox4x32-10 of every row of ctr ([n, 4] uint32) under one key: [n, 4] uint32."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    lib().oracle_philox4x32_10_many(len(c), _p(c), _p(k), _p(out))
    return out


def table(mode: int, t0: float, t1: float, pf0: float, pf1: float, sweeps: int):
    """(ecap, thr[sweeps, 2*ecap+1] uint64): accept a flip of energy change dE at sweep s iff
    u32 < thr[s, clamp(dE, -ecap, ecap) + ecap]."""
    ecap = lib().oracle_table_ecap(mode, t0, t1, pf0, pf1, sweeps)
    if ecap < 0:
        raise ValueError(f"bad schedule (code {ecap})")
    thr = np.zeros((sweeps, 2 * ecap + 1), dtype=np.uint64)
    lib().oracle_build_table(mode, t0, t1, pf0, pf1, sweeps, ecap, _p(thr))
    return ecap, thr


def greedy_color(g) -> np.ndarray:
    col = np.zeros(g.n, dtype=np.int32)
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    cc = np.ascontiguousarray(g.col, dtype=np.int32)
    lib().oracle_greedy_color(g.n, _p(rp), _p(cc), _p(col))
    return col


def cut(g, spins) -> int:
    s = np.ascontiguousarray(spins, dtype=np.int8)
    return int(lib().oracle_cut(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), _p(s)))


def energy(g, A: int, B: int, spins) -> int:
    s = np.ascontiguousarray(spins, dtype=np.int8)
    return int(lib().oracle_energy(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), A, B, _p(s)))


def bruteforce_bisection(g):
    best = np.zeros(1, dtype=np.int64)
    cnt = np.zeros(1, dtype=np.int64)
    rc = lib().oracle_bruteforce_bisection(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), _p(best), _p(cnt))
    if rc != 0:
        raise ValueError(f"bruteforce failed ({rc})")
    return int(best[0]), int(cnt[0])


@dataclass
class AnnealResult:
    spins: np.ndarray        # int8 [R, n], original vertex order, after repair
    raw_G: np.ndarray        # int32 [R]
    final_G: np.ndarray      # int32 [R]
    raw_cut: np.ndarray      # int64 [R]
    final_cut: np.ndarray    # int64 [R]
    digest: np.ndarray | None     # uint64 [R, sweeps]
    G_trace: np.ndarray | None    # int32 [R, sweeps]
    cut_trace: np.ndarray | None  # int64 [R, sweeps]
    invariant_failures: int
    num_colors: int


def anneal(g, *, A: int = 1, B: int = 1, W: int = 0, mode: int = METROPOLIS, t0: float = 3.0,
           t1: float = 0.05, pf0: float = 0.2, pf1: float = 0.01, sweeps: int = 100,
           seed: int = 1, instance: int = 0, replicas: int = 1, color=None, init=None,
           first_sweep: int = 0, last_sweep: int = 0, trace: bool = True,
           check_invariants: bool = False, repair: bool = True, first_replica: int = 0,
           stale: bool = False) -> AnnealResult:
    """Run the oracle annealer on one instance: replicas first_replica .. first_replica + replicas - 1
    (output row k is replica first_replica + k).  stale: every spin of a window decides on the G of
    the window start (the reference of the racy variant) instead of the running G."""
    n = g.n
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    cc = np.ascontiguousarray(g.col, dtype=np.int32)
    ww = np.ascontiguousarray(g.w, dtype=np.int32)
    colr = None if color is None else np.ascontiguousarray(color, dtype=np.int32)
    spins = np.zeros((replicas, n), dtype=np.int8)
    if init is not None:
        spins[:] = np.asarray(init, dtype=np.int8).reshape(replicas, n)
    raw_G = np.zeros(replicas, dtype=np.int32)
    final_G = np.zeros(replicas, dtype=np.int32)
    raw_cut = np.zeros(replicas, dtype=np.int64)
    final_cut = np.zeros(replicas, dtype=np.int64)
    dig = np.zeros((replicas, sweeps), dtype=np.uint64) if trace else None
    gtr = np.zeros((replicas, sweeps), dtype=np.int32) if trace else None
    ctr = np.zeros((replicas, sweeps), dtype=np.int64) if trace else None
    P = _Params(n, _p(rp), _p(cc), _p(ww), _p(colr), A, B, W, mode, t0, t1, pf0, pf1, sweeps,
                seed & 0xFFFFFFFFFFFFFFFF, instance, replicas, first_sweep, last_sweep,
                1 if check_invariants else 0, first_replica, 1 if stale else 0)
    O = _Out(_p(spins), 1 if init is not None else 0, _p(raw_G), _p(final_G), _p(raw_cut),
             _p(final_cut), _p(dig), _p(gtr), _p(ctr), 0, 0, 1 if repair else 0, 0)
    rc = lib().oracle_anneal(C.byref(P), C.byref(O))
    if rc != 0:
        raise ValueError(f"oracle_anneal failed with code {rc}")
    if O.decision_mismatches:
        raise AssertionError(f"oracle: {O.decision_mismatches} flips where the threshold order key "
                             "disagreed with the acceptance test")
    return AnnealResult(spins, raw_G, final_G, raw_cut, final_cut, dig, gtr, ctr,
                        int(O.invariant_failures), int(O.num_colors))


def _anneal_job(args):
    g, kw = args
    return anneal(g, **kw)


def anneal_parallel(g, *, replica_ids, processes: int = 8, **kw):
    """oracle.anneal for the replicas in replica_ids, one replica per task on a pool of `processes`
    spawned workers (never forked: the caller may already hold a GPU context).  Returns a list of
    AnnealResult, one per replica id, each with a single row."""
    import multiprocessing as mp
    jobs = [(g, dict(kw, replicas=1, first_replica=int(r))) for r in replica_ids]
    with mp.get_context("spawn").Pool(min(processes, len(jobs))) as pool:
        return pool.map(_anneal_job, jobs)
