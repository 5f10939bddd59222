"""Multi-process host logic on CPU (gloo, world size 2): the benchmark's
rank setup and max / sum reduction over ranks, and the partition of a batch
of independent cells over ranks (computed by every rank on its own; no
data-path collective)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from paper_1603_08893_gb300.shard import cell_cost, partition_cells
    r, w, dist = bench.dist_setup(world)
    assert (r, w) == (rank, world) and dist is not None
    t, s = bench.reduce_max_sum(dist, 1.5 + rank, 10.0 * (rank + 1))
    assert t == 1.5 + (world - 1)
    assert s == 10.0 * world * (world + 1) / 2
    rng = np.random.default_rng(7)
    shapes = [(int(n),) * 3 for n in rng.choice([15, 21, 27, 33, 45, 63], 40)]
    parts = partition_cells(shapes, world)
    everyone = [None] * world
    dist.all_gather_object(everyone, parts)
    assert all(p == parts for p in everyone)          # the same partition on every rank
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(shapes)))           # disjoint and complete
    loads = [sum(cell_cost(shapes[i]) for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(cell_cost(sh) for sh in shapes)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)


def test_partition_single_rank_and_errors():
    sys.path.insert(0, ROOT)
    from paper_1603_08893_gb300.shard import partition_cells
    assert partition_cells([(3, 3, 3), (5, 5, 5)], 1) == [[0, 1]]
    assert partition_cells([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        partition_cells([(3, 3, 3)], 0)
