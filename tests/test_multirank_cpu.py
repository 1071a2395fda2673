"""The N-process path of bench.py on CPU (gloo, world size 2): the work shards by image with no
collective in the data path (replicas only), each rank draws its own disjoint, seeded images, and
the step time is the largest over the ranks."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    images, Ms, pk, W0s, ndims, Gs = bench.make_workload("c3", rank, n=6)
    digest = np.array([float(np.sum(im.astype(np.int64) * (1 + np.arange(im.size).reshape(im.shape) % 7)))
                       for im in images])
    t = torch.tensor(digest, dtype=torch.float64)
    gathered = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(gathered, t)
    slowest = bench.max_over_ranks(10.0 + rank, world, "cpu")
    if rank == 0:
        out.put(([g.numpy() for g in gathered], slowest, [im.shape for im in images], list(Ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_images_and_report_the_slowest():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    digests, slowest, shapes, Ms = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert slowest == 11.0
    assert not np.array_equal(digests[0], digests[1])          # disjoint shards
    sys.path.insert(0, ROOT)
    import bench
    images, Ms0, _, _, _, _ = bench.make_workload("c3", 0, n=6)
    assert [im.shape for im in images] == shapes and list(Ms0) == Ms   # seeded: rank 0 reproduces
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
