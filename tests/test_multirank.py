"""The multi-rank host logic of bench.py on CPU with the gloo backend
(world size 2): the batched workload's shards and the max-over-ranks time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, sizes, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shard = bench.shard_by_nnz(sizes, world)[rank]
    mine = float(sum(sizes[i] for i in shard))
    out[rank] = (shard, mine, bench.max_over_ranks(mine, world))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_partition_and_balance():
    sizes = [int(1000 * 1.07 ** (i % 37)) + i for i in range(256)]
    for world in (1, 2, 3, 8):
        shards = bench.shard_by_nnz(sizes, world)
        flat = sorted(i for sh in shards for i in sh)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in sh) for sh in shards]
        assert max(loads) - min(loads) <= max(sizes)
        assert shards == bench.shard_by_nnz(sizes, world)  # deterministic


def test_two_gloo_ranks_agree():
    sizes = [5, 17, 3, 11, 8, 13, 2, 7]
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), sizes, out), nprocs=world, start_method="spawn")
    shards = [out[r][0] for r in range(world)]
    assert sorted(i for sh in shards for i in sh) == list(range(len(sizes)))
    loads = [out[r][1] for r in range(world)]
    assert all(out[r][2] == max(loads) for r in range(world))
