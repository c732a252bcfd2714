"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2).

bench.py runs one independent replica per GPU (the pencils of one problem
are not distributed: every configuration fits one GPU), so the only
cross-rank step is the timing reduction: the job's rate is the units of all
ranks over the slowest rank's time.  Here two gloo ranks with different
local times must agree on that rate, and the reference arm must print
nothing on ranks other than 0.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    rate, secs = bench.job_rate(1000.0, 1.0 + rank, world, device="cpu")
    out.put((rank, rate, secs))
    dist.destroy_process_group()


def test_job_rate_is_max_over_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, secs in res:
        assert secs == 2.0                       # the slower rank's time
        assert rate == world * 1000.0 / 2.0      # all ranks' units over it


def test_single_rank_rate_and_reference_arm_on_other_ranks(monkeypatch):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    assert bench.job_rate(10.0, 0.5, 1) == (20.0, 0.5)
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(workload=bench.WORKLOAD, steps=1, warmup=3, gpus=2)
    assert bench.run_reference(args) is None
