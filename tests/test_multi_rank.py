"""The N > 1 bench path on CPU: two gloo ranks (spawned processes on 127.0.0.1).

The method has no exchange step, so several GPUs run independent replicas; the
only cross-rank operation is the max over ranks of the timed region.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = bench.max_over_ranks(1.5 + rank)        # rank 1 is the slow replica
        out[rank] = (elapsed, bench.job_throughput(10, world, elapsed))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            assert out[r][0] == 2.5
            assert out[r][1] == pytest.approx(20 / 2.5)


def test_reference_arm_runs_on_rank0_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"gpus": 2, "steps": 1, "warmup": 3, "workload": "tfim_L12"})()
    assert bench.run_reference(args) == 0        # returns at once, no oracle work


def test_single_process_max_is_identity():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
