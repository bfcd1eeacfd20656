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


def _merge_worker(rank, world, port, out):
    """Each rank takes the oracle statistics of its half of a tiny catalogue,
    then the ranks exchange raw sums and merge them with mk_stats_merge."""
    import sys

    sys.path.insert(0, ROOT)
    import oracle
    import paper_2310_18996_gb300 as mk
    import skewer_inputs as si

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = si.workload("tiny")
    d, e = si.gaussian_box(w["n"], w["cell"], w["seed_box"], backend="numpy")
    pos, ids = si.catalogue(w, n_q=120)
    half = slice(0, 50) if rank == 0 else slice(50, 120)  # uneven halves
    o = oracle.run_skewers(w, d, e, pos[half], ids[half])
    st = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    merged = mk.merge_stats_across_ranks(st, w, dist)
    out[rank] = {k: np.asarray(v) for k, v in merged.items()}
    dist.barrier()
    dist.destroy_process_group()


def _dead_rank_worker(rank, world, port, out):
    """Rank 1 leaves after joining the group, before the statistics exchange
    (a killed process); rank 0 must get an error from the exchange, not hang."""
    import datetime
    import sys
    import time

    sys.path.insert(0, ROOT)
    import oracle
    import paper_2310_18996_gb300 as mk
    import skewer_inputs as si

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(0)  # no shutdown of the process group: its peer sees a dead rank
    w = si.workload("tiny")
    d, e = si.gaussian_box(w["n"], w["cell"], w["seed_box"], backend="numpy")
    pos, ids = si.catalogue(w, n_q=20)
    o = oracle.run_skewers(w, d, e, pos, ids)
    st = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    t0 = time.monotonic()
    try:
        mk.merge_stats_across_ranks(st, w, dist)
        out[rank] = ("merged", time.monotonic() - t0)
    except RuntimeError as ex:  # gloo reports the lost peer (or the group's timeout)
        out[rank] = ("error: " + str(ex)[:200], time.monotonic() - t0)


def test_statistics_merge_with_a_dead_rank_fails_without_hanging():
    """A rank that dies before the exchange of raw sums: the surviving rank's
    merge raises within the process group's 10 s timeout instead of waiting
    forever, so the job can report the failure."""
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_dead_rank_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    status, seconds = res[0]
    assert status.startswith("error"), status
    assert seconds < 60


def test_two_rank_statistics_merge_equals_union():
    """Sec. 3 runs the mocks in independent slices; statistics of the whole
    catalogue follow from the slices' raw sums.  Two gloo ranks, each with the
    oracle statistics of part of the catalogue, merged through one all-gather
    and mk_stats_merge, equal the oracle statistics of the union computed in
    one process."""
    import sys

    sys.path.insert(0, ROOT)
    import oracle
    import skewer_inputs as si

    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_merge_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    w = si.workload("tiny")
    d, e = si.gaussian_box(w["n"], w["cell"], w["seed_box"], backend="numpy")
    pos, ids = si.catalogue(w, n_q=120)
    o = oracle.run_skewers(w, d, e, pos, ids)
    ref = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    assert ref["n_seg"].sum() > 0 and np.count_nonzero(ref["sums"][:, 0]) >= 3
    for rank in (0, 1):
        got = res[rank]
        for k in ("sums", "p1d_sum", "n_seg"):  # raw sums: a different FP64 addition order only
            np.testing.assert_allclose(got[k], ref[k], rtol=1e-12, atol=0)
        m = ref["sums"][:, 0] > 0
        for k in ("mean_flux", "sigma_f", "b_f", "beta_f"):
            np.testing.assert_allclose(got[k][m], ref[k][m], rtol=1e-10, atol=0, err_msg=k)
        ms = ref["n_seg"] > 0
        for k in ("p1d_f", "p1d_df"):
            np.testing.assert_allclose(got[k][ms], ref[k][ms], rtol=1e-12, atol=0, err_msg=k)
    for k in got:  # every rank holds the same merged result
        assert np.array_equal(res[0][k], res[1][k])


def test_statistics_merge_rejects_bad_arguments():
    import ctypes as C
    import sys

    sys.path.insert(0, ROOT)
    import paper_2310_18996_gb300 as mk

    b = mk.StatBins(n_z=4, z_lo=2.0, dz=0.2, n_k=8, n_fft=256)
    parts = (mk.StatsOut * 2)()
    out = mk.StatsOut()
    L = mk.lib()
    assert L.mk_stats_merge(parts, 0, C.byref(b), C.byref(out)) == mk.MK_EINVAL
    assert L.mk_stats_merge(None, 1, C.byref(b), C.byref(out)) == mk.MK_EINVAL
    bad = mk.StatBins(n_z=4, z_lo=2.0, dz=0.2, n_k=7, n_fft=256)
    assert L.mk_stats_merge(parts, 2, C.byref(bad), C.byref(out)) == mk.MK_EINVAL
    assert L.mk_stats_merge(parts, 2, C.byref(b), C.byref(out)) == mk.MK_OK
    assert np.ctypeslib.as_array(out.mean_flux).sum() == 0.0  # empty parts: no derived statistics
