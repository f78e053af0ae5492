"""Host-side logic of the multi-rank benchmark on CPU (gloo, world size 2):
independent replicas per rank, max-over-ranks timing, whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    p = bench.replica_problem("cavity256_v32", rank)
    t = bench.max_over_ranks(1.5 + rank, world, "cpu")
    out[rank] = (p.instance, p.seed, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == 0 and out[1][0] == 1          # distinct Philox instances
    assert out[0][1] == out[1][1]                     # same workload otherwise
    assert out[0][2] == out[1][2] == 2.5              # every rank sees the max


def test_job_throughput_is_whole_job():
    import bench
    assert bench.job_throughput(100, 10, 4, 2.0) == 2000.0
