"""Host logic of the multi-rank benchmark path on two gloo ranks (CPU).

Each rank synthesises its own quasars on a replica of the box: catalogues
must differ, ids must be disjoint, and the timing reduction must return the
maximum over ranks on every rank.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    import bench
    import skewer_inputs as si

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = si.shrink(si.workload("batched"), n_q=2000)
    w2, pos, ids = bench.rank_catalogue(w, rank)
    gathered = [torch.zeros(len(ids), dtype=torch.int64) for _ in range(world)]
    dist.all_gather(gathered, torch.from_numpy(ids.astype(np.int64)))
    first = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(first, torch.from_numpy(pos[0].copy()))
    ms = bench.max_over_ranks([10.0 + rank, 5.0 - rank], dist, "cpu")
    out[rank] = (sorted(set(np.concatenate([g.numpy() for g in gathered]).tolist())) ==
                 list(range(world * len(ids))),
                 not torch.equal(first[0], first[1]), ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_catalogues_are_disjoint_and_timing_takes_the_max():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        disjoint, differ, ms = res[rank]
        assert disjoint and differ
        assert ms == [11.0, 5.0]


def test_single_process_reduction_is_identity():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([1.5, 2.5], None, "cpu") == [1.5, 2.5]
