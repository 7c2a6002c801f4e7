"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): every
rank owns different seeded captures, the job time is the slowest rank's, and
the whole-job throughput counts every rank's volumes. No GPU and no
collective on the data path (the captures are independent)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_s = 1.0 + 0.5 * rank                      # the second rank is slower
    worst = bench.reduce_max(local_s, dist, "cpu")
    value = bench.whole_job_throughput(world, 10, worst)
    q.put((rank, worst, value, bench.capture_index_for(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_aggregate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [1.5, 1.5]                 # max over ranks seen by all
    assert out[0][2] == pytest.approx(2 * 10 / 1.5)           # all ranks' units / slowest time
    assert out[0][3] != out[1][3]                             # distinct captures per rank


def test_single_process_without_group():
    assert bench.reduce_max(2.5, None, "cpu") == 2.5
    assert bench.whole_job_throughput(1, 100, 0.5) == 200.0
