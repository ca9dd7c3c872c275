"""Benchmark of the GDI annealing path (one JSON line on rank 0).

A step is one gdi_anneal of the workload: initial state, all sweeps (thresholds, window selection,
flips), exact-balance repair and cut, with the graph already resident on the device.  The metric
is spin-updates per second (one update = one spin of one replica visited in one sweep).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Multi-GPU runs (torchrun, one process per GPU) are replicas only: every rank anneals its own
replica set of the same graph with its own seed, no data-path collective (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# ---------------------------------------------------------------------------------------------
# Workloads: seeded synthetic stand-ins for the paper's G-set graphs (generators in gdi_synth)
WORKLOADS = {
    # Barabasi-Albert n = 10^6, m = 5, unit weights, greedy colouring (6 classes), 8 replicas,
    # 500 sweeps, window W = 256: the grid-scale path (every SM on one graph).  Algorithmic bytes
    # of one spin update in the pull form: 4 d (columns) + 4 (row pointer) + d (neighbour spins)
    # + 2 (own spin read and write) = 56 B for d = 10.  traffic: dram__bytes_read.sum +
    # dram__bytes_write.sum of one launch of the sweep kernel (ncu), traffic_l2 its
    # lts__t_bytes.sum; None when the kernel changed after the counters were taken.
    "ba1m_r8": dict(kind="ba", n=1_000_000, m=5, gseed=4004, A=1, B=4, W=256, replicas=8,
                    sweeps=500, t0=12.0, t1=0.2, seed=1,
                    roofline=dict(bound="hbm", bytes_per_update=56, traffic=53_390_000,
                                  traffic_l2=61_610_000_000,
                                  note="the graph stays L2-resident (DRAM traffic: the graph read once); "
                                       "the kernel is bound by its per-class chain of block waits and "
                                       "barriers, not by a memory unit")),
    # 2-D torus 100 x 100, +-1 weights, checkerboard colouring, 64 replicas, 5000 sweeps, window
    # W = 256: the CTA-resident path.  26 B per update: 4 x 4 B columns + 4 B row pointer + 4 x 1 B
    # spins + 2 B.
    "torus100_r64": dict(kind="torus", L=100, gseed=2002, A=1, B=4, W=256, replicas=64,
                         sweeps=5000, t0=12.0, t1=0.2, seed=1,
                         roofline=dict(bound="hbm", bytes_per_update=26, traffic=2_480_000,
                                       traffic_l2=54_630_000_000,
                                       note="a pair of blocks per replica on 128 of 152 SMs; the graph "
                                            "is L1/L2-resident (90 % L1 hits); issue- and barrier-bound")),
    # Erdos-Renyi n = 800, p = 0.06, unit weights, greedy colouring, 1000 sweeps, 1 replica: one
    # block holds the whole instance; latency-bound.  Bytes per update 4 d + 4 + d + 2 at d = 48.7.
    "er800": dict(kind="er", n=800, p=0.06, gseed=1001, A=1, B=4, W=64, replicas=1, sweeps=1000,
                  t0=12.0, t1=0.2, seed=1,
                  roofline=dict(bound="hbm", bytes_per_update=249.5, traffic=655_620, traffic_l2=11_920_000,
                                note="one block on one SM: latency-bound (19 colour classes of about "
                                     "42 vertices per sweep)")),
    # 4,096 Erdos-Renyi instances, n ~ U[800, 3000], mean degree ~ U[3, 48], unit or +-1 weights,
    # one replica each, 2000 sweeps, one persistent launch (CTA-resident, autotuned).  Bytes per
    # update at the batch's mean degree d = 25.5: 4 d + 4 + d + 2 = 134 B.
    "batched4096": dict(kind="batch", count=4096, gseed=3000, n_lo=800, n_hi=3000, A=1, B=4, W=256,
                        replicas=1, sweeps=2000, t0=12.0, t1=0.2, seed=11,
                        roofline=dict(bound="hbm", bytes_per_update=134, traffic=685_297_000_000,
                                      traffic_l2=1_850_000_000_000,
                                      note="the 4,096 graphs do not fit in L2: DRAM traffic is about a "
                                           "third of the algorithmic bytes, at 6 % of the measured HBM "
                                           "bandwidth; latency-bound")),
}
DEFAULT_WORKLOAD = "ba1m_r8"


def _er_chunk(args):
    from gdi_synth import er_batch
    count, seed0, n_lo, n_hi = args
    return er_batch(count, seed0, n_lo=n_lo, n_hi=n_hi)


def make_graph(wl):
    """The workload's graph; for a batch, the disjoint union (with .inst_ptr and .parts)."""
    from gdi_synth import barabasi_albert, batch_union, erdos_renyi, torus2d
    if wl["kind"] == "batch":
        import multiprocessing as mp
        jobs = [(min(256, wl["count"] - i), wl["gseed"] + i, wl["n_lo"], wl["n_hi"])
                for i in range(0, wl["count"], 256)]
        with mp.get_context("spawn").Pool(min(16, len(jobs))) as pool:
            parts = [g for part in pool.map(_er_chunk, jobs) for g in part]
        inst_ptr, u = batch_union(parts)
        u.inst_ptr = inst_ptr
        u.parts = parts
        return u
    if wl["kind"] == "ba":
        return barabasi_albert(wl["n"], wl["m"], wl["gseed"])
    if wl["kind"] == "torus":
        return torus2d(wl["L"], wl["gseed"], signed=True)
    if wl["kind"] == "er":
        return erdos_renyi(wl["n"], wl["p"], wl["gseed"])
    raise ValueError(wl["kind"])


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def rd():
            for line in self.proc.stdout:
                self.rows.append([x.strip() for x in line.split(",")])
        self.thread = threading.Thread(target=rd, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
def oracle_throughput(g, wl, seconds: float = 12.0, processes: int | None = None):
    """The oracle as it stands, timed on the host cores on a bounded sample of the workload: each
    worker process anneals up to 4 replicas of the graph (for a batch: 4 of its instances, a
    different set per process) for as many sweeps of the same schedule as fit the time budget, and
    repeats the whole anneal with other seeds while the budget lasts when the schedule is shorter
    than it.  The cost of a sweep and of a call's setup come from two probes (1 and 3 sweeps).
    Returns (updates/s, cores, sample text)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = processes or os.cpu_count() or 1
    R = min(4, wl["replicas"])
    parts = getattr(g, "parts", None)
    sets = [_inst_set(parts, k) for k in range(cores)] if parts else [None] * cores
    probe = []
    for sw in (1, 3):
        t = time.perf_counter()
        _oracle_worker((g if parts is None else sets[0], wl, R, sw, 0, 0.0))
        probe.append(time.perf_counter() - t)
    per_sweep = max((probe[1] - probe[0]) / 2, 1e-5)
    setup = max(probe[0] - per_sweep, 0.0)
    sweeps = int(max(1, min(wl["sweeps"], (seconds - setup) / per_sweep)))
    # a schedule shorter than the budget is annealed again (other seeds) until the budget is spent
    budget = 0.0 if sweeps < wl["sweeps"] else seconds
    ctx = mp.get_context("spawn")
    args = [(g if parts is None else sets[k], wl, R, sweeps, k, budget) for k in range(cores)]
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        done = pool.map(_oracle_worker, args)
    dt = time.perf_counter() - t0
    reps = sum(done) / len(done)
    if parts is None:
        updates = sum(done) * R * sweeps * g.n
        sample = (f"{cores} processes x {reps:.1f} anneals x {R} replicas x first {sweeps} of {wl['sweeps']} "
                  f"sweeps x {g.n} spins = {updates:.3e} updates in {dt:.1f} s")
    else:
        updates = sum(d * R * sweeps * sum(x.n for x in st) for d, st in zip(done, sets))
        sample = (f"{cores} processes x {reps:.1f} anneals x 4 instances of the batch x {R} replica x first "
                  f"{sweeps} of {wl['sweeps']} sweeps = {updates:.3e} updates in {dt:.1f} s")
    return updates / dt, cores, sample


def _inst_set(parts, k):
    """Instances 4k .. 4k + 3 of a batch (mod its size): the oracle sample of worker k."""
    return [parts[(4 * k + j) % len(parts)] for j in range(4)]


def _oracle_worker(a):
    """Anneal the sample once, then again with other seeds while the time budget lasts; returns
    the number of anneals."""
    g, wl, R, sweeps, k, budget = a
    import oracle
    t_end = time.perf_counter() + budget
    rep = 0
    while rep == 0 or time.perf_counter() < t_end:
        for x in (g if isinstance(g, list) else [g]):
            oracle.anneal(x, A=wl["A"], B=wl["B"], W=wl["W"], t0=wl["t0"], t1=wl["t1"], sweeps=wl["sweeps"],
                          seed=wl["seed"] + 1000 * k + 100_000 * rep, replicas=R, color=x.color,
                          last_sweep=sweeps, trace=False, repair=False)
        rep += 1
    return rep


# ---------------------------------------------------------------------------------------------
def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def job_throughput(world, updates_per_rank, ms_per_step):
    """Whole-job spin-updates/s: every rank anneals its own replica set (weak scaling), and the
    step time is the slowest rank's."""
    return world * updates_per_rank / (ms_per_step / 1e3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, wl, rank, world):
    if rank != 0:
        return
    g = make_graph(wl)
    for _ in range(args.warmup):
        oracle_throughput(g, wl, seconds=2.0)
    vals, samples = [], []
    cores = 1
    for _ in range(args.steps):
        v, cores, s = oracle_throughput(g, wl, seconds=8.0)
        vals.append(v)
        samples.append(s)
    value = statistics.mean(vals)
    updates_per_step = wl["replicas"] * wl["sweeps"] * g.n
    line = {"impl": "reference", "metric": "spin-updates/s", "value": value, "unit": "spin-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * updates_per_step / value,
            "ms_per_step_note": "extrapolated: the oracle anneals a bounded sample of the step's sweeps and "
                                "replicas; the whole step at the measured rate",
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": config_of(args.workload, wl, g),
            "cpu_baseline": {"value": value, "unit": "spin-updates/s", "cores": cores,
                             "kind": "oracle", "sample": samples[-1]},
            "e2e": {"value": value, "unit": "spin-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(name, wl, g):
    c = {"workload": name, "n": g.n, "nnz": g.nnz, "replicas": wl["replicas"],
         "sweeps": wl["sweeps"], "A": wl["A"], "B": wl["B"], "W": wl["W"],
         "schedule": f"metropolis T {wl['t0']}->{wl['t1']} (3.0->0.05 in units of B)",
         "l2": "L2 flushed (256 MiB write) before every timed step",
         "parallelism": "replicas" if wl["kind"] != "batch" else "instances"}
    if wl["kind"] == "batch":
        c["instances"] = wl["count"]
    return c


def run_ours(args, wl, rank, world, local):
    import torch
    import paper_1908_00210_gb300 as P
    torch.cuda.set_device(local)
    P.load()
    g = make_graph(wl)
    dev_props = torch.cuda.get_device_properties(local)
    stream = torch.cuda.Stream()
    seed = wl["seed"] + 7919 * rank
    sch = P.Schedule(sweeps=wl["sweeps"], t0=wl["t0"], t1=wl["t1"])
    t_create = time.perf_counter()
    ann = P.Annealer(g, A=wl["A"], B=wl["B"], W=wl["W"], replicas=wl["replicas"],
                     inst_ptr=getattr(g, "inst_ptr", None))
    create_s = time.perf_counter() - t_create
    # CTA-resident workloads: block size and blocks per SM by the library's autotuner (results do
    # not depend on them); the grid-scale workload keeps one 768-thread block per SM
    if wl["kind"] == "ba":
        tuned = None
    elif args.block:
        ann.configure(block=args.block)
        tuned = dict(block=args.block, grid=0, ms=None)
    else:
        tuned = ann.autotune(sch, probe_sweeps=20)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    updates = wl["replicas"] * wl["sweeps"] * g.n

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ann.anneal(sch, seed, stream=stream)
            ann.results()
    launch_path = ann.last_launch()["path"] if args.warmup > 0 else 0
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    wall0 = time.perf_counter()
    ms = []
    kms, klaunch = 0.0, 0                               # the sweep kernel alone (library events)
    launches = 0
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.fill_(1)                              # evict the working set from L2
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ann.anneal(sch, seed, stream=stream)
            e1.record(stream)
            launches += launches_per_anneal(launch_path, wl["replicas"])
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            k_ms, k_n = ann.kernel_ms()
            kms += k_ms
            klaunch += k_n
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    res = ann.results()
    launch = ann.last_launch()
    total_ms = sum(ms)
    total_ms = allreduce_max(total_ms, world)
    ms_per_step = total_ms / args.steps
    value = job_throughput(world, updates, ms_per_step)

    # end to end through the public API with host buffers: the step's input (balanced initial spins
    # of every replica) is copied from pinned host memory, the spins and results are read back
    rng = np.random.default_rng(1234 + rank)
    init_t = torch.empty((wl["replicas"], g.n), dtype=torch.int8, pin_memory=True)
    init_np = init_t.numpy()
    half = np.ones(g.n, dtype=np.int8)
    half[g.n // 2:] = -1
    for r in range(wl["replicas"]):
        init_np[r] = rng.permutation(half)
    e2e_ms = []
    h2d = init_np.nbytes
    d2h = wl["replicas"] * g.n + 24 * wl["replicas"]
    for _ in range(0 if args.quick else max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ann.anneal(sch, seed, init=init_np, stream=stream)
        ann.spins()
        ann.results()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    if not e2e_ms:
        e2e_ms = [float("nan")]
    e2e_value = job_throughput(world, updates, statistics.median(e2e_ms))

    if rank != 0:
        return
    pk = peaks()
    rf = wl["roofline"]
    # roofline of the dominant kernel: algorithmic bytes (ops) of one launch / its mean duration,
    # from CUDA events recorded by the library around each sweep-kernel launch on this stream
    kernel_ms = kms / max(1, klaunch)
    rate = updates * args.steps / max(1, klaunch) / (kernel_ms / 1e3)
    if rf["bound"] == "hbm":
        peak = float(pk.get("hbm_gbs", 6800.0))
        achieved = rf["bytes_per_update"] * rate / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": rf.get("traffic"),
                "algorithmic_bytes_per_update": rf["bytes_per_update"], "kernel_ms_per_launch": kernel_ms,
                "achieved_note": "algorithmic bytes (pull-form gather of every update) / sweep-kernel time",
                "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
        if rf.get("traffic_l2"):
            # lts__t_bytes.sum of one launch (ncu) over the launch's duration
            roof["traffic_l2"] = rf["traffic_l2"]
            roof["achieved_l2_gbs"] = rf["traffic_l2"] / (kernel_ms / 1e3) / 1e9
        if rf.get("note"):
            roof["note"] = rf["note"]
    else:
        sm_max = float(pk.get("sm_max_mhz", 2070.0))
        peak = dev_props.multi_processor_count * 128 * sm_max * 1e6 / 1e12
        achieved = rf["ops_per_update"] * rate / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                "frac": achieved / peak, "traffic": rf.get("traffic"), "ops_per_update": rf["ops_per_update"],
                "kernel_ms_per_launch": kernel_ms,
                "peak_note": "SMs x 128 int32 lanes x max SM clock (derived)"}
    try:
        if args.quick:
            raise RuntimeError("skipped (--quick)")
        cpu_v, cores, sample = oracle_throughput(g, wl, seconds=12.0)
        cpu = {"value": cpu_v, "unit": "spin-updates/s", "cores": cores, "kind": "oracle", "sample": sample}
    except Exception as ex:  # the baseline is reported, not required
        cpu = {"value": None, "unit": "spin-updates/s", "cores": 0, "kind": "oracle",
               "sample": f"failed: {ex!r}"[:200]}
    line = {
        "metric": "spin-updates/s", "value": value, "unit": "spin-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": config_of(args.workload, wl, g),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "spin-updates/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "clocks": clk, "gpu_launches": launches,
        "wall_s_timed_region": wall,
        "launch": launch,
        "autotune": tuned,
        "create_s": create_s,
        "result": {"final_cut_median": float(np.median(res["final_cut"])),
                   "final_G_max_abs": int(np.abs(res["final_G"]).max()),
                   "raw_G_max_abs": int(np.abs(res["raw_G"]).max())},
    }
    print(json.dumps(line), flush=True)
    ann.close()



def launches_per_anneal(path: int, replicas: int) -> int:
    """Kernels of one gdi_anneal: grid path = initial spins, then per group of 8 replicas pack,
    sweep kernel, raw cut, unpack, five repair kernels, pack and final cut; CTA path = initial
    spins and the persistent sweep kernel (cut and repair inside it)."""
    if path == 2:
        return 1 + 11 * ((replicas + 7) // 8)
    return 2


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sweeps", type=int, default=0,
                    help="profiling only: override the workload's sweep count")
    ap.add_argument("--quick", action="store_true",
                    help="profiling only: skip the CPU baseline and the end-to-end leg")
    ap.add_argument("--block", type=int, default=0,
                    help="profiling only: CTA-resident threads per block instead of the autotuner's "
                         "choice (128/256/512/1024; full occupancy)")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.sweeps > 0:
        wl["sweeps"] = args.sweeps
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, wl, rank, world)
    else:
        run_ours(args, wl, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
