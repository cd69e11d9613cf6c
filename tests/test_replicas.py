"""bench.py's multi-GPU form: independent replicas, one process per GPU.  The
whole-job number is the units of all ranks over the slowest rank's time, and
the reference arm runs on rank 0 only.  Checked with two gloo ranks on the CPU
(the collective is the same call the NCCL run makes)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = [100.0, 250.0][rank]
        pairs_local = [455.0, 470.0][rank]
        value, ms = bench.job_throughput(pairs_local, ms_local, dist, "cpu")
        out[rank] = (value, ms)
        # the reference arm: ranks other than 0 return at once, without work
        class A:
            steps, warmup = 1, 0
        if rank != 0:
            assert bench.run_reference(A()) == 0
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_summed_units():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in (0, 1):
        value, ms = out[r]
        assert ms == 250.0
        assert value == pytest.approx((455.0 + 470.0) / 0.25)


def test_single_process_throughput():
    import bench
    assert bench.job_throughput(455.0, 200.0) == (455.0 / 0.2, 200.0)
