"""The multi-process path of bench.py on CPU (gloo, world size 2): every rank
times its own replica and the job's duration is the maximum over ranks, so the
reported throughput is (units of all ranks) / (slowest rank's time)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local = 10.0 * (rank + 1)  # rank 1 is the slow one
    out[rank] = bench.job_ms(local)
    env = bench.dist_env()
    assert env == (ws, rank, 0) or env[:2] == (ws, rank)
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_max_over_two_gloo_ranks():
    ws = 2
    port = free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(worker, args=(ws, port, out), nprocs=ws, join=True)
    assert out[0] == 20.0 and out[1] == 20.0


def test_single_process_job_time_is_local():
    import bench
    assert bench.job_ms(12.5) == 12.5
