"""The multi-GPU path of the benchmark is "replicas only": independent transforms,
one per rank, with collectives used just for the barrier and the max over the
ranks' times. Its host logic runs here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow replica
    dist.barrier()
    job_ms = bench.reduce_max_ms(dist, local_ms, torch.device("cpu"))
    value = bench.whole_job_value(world, 1e9, job_ms / 2)  # 2 steps
    q.put((rank, job_ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_max_over_ranks_and_whole_job_value():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, job_ms, value in res:
        assert job_ms == pytest.approx(15.0)           # the slowest replica
        assert value == pytest.approx(2 * 1e9 / 7.5e-3 / 1e9)  # both replicas' work over the job time
