"""Replicas on several GPUs (`bench.py --gpus N` under torchrun): every rank runs the whole
workload and the job's time is the slowest rank's. The bookkeeping runs here on CPU with
two gloo ranks (the GPU path uses NCCL for the same two calls)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, torch.device("cpu"))
    q.put((rank, ms, bench.whole_job_mvis(4_128_768, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_with_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 15.0                                   # the slower rank's time on both
        assert value == pytest.approx(2 * 4_128_768 / 15e-3 / 1e6)


def test_single_process_keeps_its_own_time():
    import bench
    assert bench.max_over_ranks(7.5, torch.device("cpu")) == 7.5
    assert bench.whole_job_mvis(1_000_000, 1, 1.0) == pytest.approx(1000.0)
