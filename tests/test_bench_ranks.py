"""Host logic of bench.py's multi-rank run (replicas only, weak scaling), on CPU with gloo: two
ranks meet at the barriers, take the step time as the maximum over ranks, and report the whole
job's throughput; the reference arm prints on rank 0 only."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, step_ms, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w, _ = bench.dist_setup(world)
    bench.barrier(w)
    slowest = bench.allreduce_max(step_ms[rank], w)
    bench.barrier(w)
    q.put((r, w, slowest, bench.job_throughput(w, 1000, slowest)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    step_ms = [2.0, 5.0]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, step_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slower rank's time; the job did 2 x 1000 updates in 5 ms
    assert got == [(0, 2, 5.0, 2 * 1000 / 5e-3), (1, 2, 5.0, 2 * 1000 / 5e-3)]


def test_reference_arm_prints_on_rank_zero_only(capsys):
    import argparse
    import bench
    args = argparse.Namespace(gpus=2, steps=1, warmup=0, workload=bench.DEFAULT_WORKLOAD,
                              impl="reference", sweeps=0, quick=True)
    bench.run_reference(args, dict(bench.WORKLOADS[bench.DEFAULT_WORKLOAD]), rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_job_throughput_is_weak_scaling():
    import bench
    assert bench.job_throughput(1, 4e9, 100.0) == pytest.approx(4e10)
    assert bench.job_throughput(8, 4e9, 100.0) == pytest.approx(3.2e11)


def test_oracle_baseline_sample_fills_its_budget():
    """The CPU baseline times the oracle on a bounded sample: a schedule shorter than the budget is
    annealed again with other seeds until the budget is spent, and the sample text states what ran."""
    import bench
    from gdi_synth import erdos_renyi
    g = erdos_renyi(120, 0.05, 3)
    wl = dict(A=1, B=4, W=16, t0=12.0, t1=0.2, sweeps=20, seed=1, replicas=1)
    v, cores, sample = bench.oracle_throughput(g, wl, seconds=1.0, processes=2)
    assert v > 0 and cores == 2
    assert "first 20 of 20 sweeps" in sample
    anneals = float(sample.split(" x ")[1].split()[0])
    assert anneals > 1.0            # the whole schedule takes far less than the budget
