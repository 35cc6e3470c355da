"""Host side of the multi-GPU replicas (no data-path collective): the job's
throughput over two gloo ranks on the CPU, and the dealing of a coil batch."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2403_07666_b300.replicas import job_throughput, shard_coils


def test_shard_coils_partitions_and_balances():
    sizes = [2160, 41472, 5000, 5000, 34020, 8000, 12000, 2160, 7000]
    for world in (1, 2, 3, 4, 8):
        parts = [shard_coils(sizes, world, r) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    with pytest.raises(ValueError):
        shard_coils(sizes, 2, 2)


def test_single_rank_throughput():
    v, s = job_throughput(2.0, 100.0)
    assert v == 50.0 and s == 2.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs = [1.5, 3.0][rank]
    units = [96000.0 * 50, 96000.0 * 50][rank]
    out[rank] = job_throughput(secs, units, dist)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        v, s = out[r]
        assert s == 3.0
        assert v == 2 * 96000.0 * 50 / 3.0
