"""mk_stats_static: statistics for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc while they work: programs that give all
device memory to their own pool at start-up, processes under a hard device
memory cap, and latency-bound loops where an allocation (which waits for the
whole device) is not acceptable.  mk_stats_static keeps its scratch in a fixed
array inside the library instead of a workspace grown on demand.  This test
calls it through the C-ABI twice in a row and checks both results against the
allocating mk_stats on the same inputs, within the statistics tolerance of the
parity tests, and checks the size limit.  It lives in its own file, collected
last, and builds all its inputs itself so it also passes in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import skewer_inputs as si
from tests.parity_util import assert_stats_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2310_18996_gb300 as mk  # noqa: E402


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _static_stats(ctx, w, sk, n, off, flux, delta, eta):
    p = mk.skewer_params(w)
    b = mk.stat_bins(w)
    st = mk.StatsOut()
    rc = mk.lib().mk_stats_static(ctx.h, C.byref(p), _ptr(sk), n, _ptr(off), _ptr(flux), 1,
                                  _ptr(delta), _ptr(eta), C.byref(b), C.byref(st))
    return rc, mk.stats_dict(st, b.n_z, b.n_k)


def test_static_scratch_statistics_match_allocating_call():
    ctx = mk.Context(0)
    w = si.workload("tiny")
    d, e = si.gaussian_box(w["n"], w["cell"], w["seed_box"], backend="numpy")
    n = 3000  # more than one scan tile of skewers
    pos, ids = si.catalogue(w, n_q=n)
    box = ctx.load_box(w, torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda())
    r = ctx.make_skewers(box, mk.catalogue_tensor(pos, ids), n, w)
    f, off = ctx.flux(w, r["sk"], n, r["delta"], r["eta"])
    ref = ctx.stats(w, r["sk"], n, off, f, delta=r["delta"], eta=r["eta"])
    assert ref["sums"][:, 0].sum() > 0 and ref["n_seg"].sum() > 0
    for _ in range(2):
        rc, st = _static_stats(ctx, w, r["sk"], n, off, f, r["delta"], r["eta"])
        assert rc == mk.MK_OK, mk.lib().mk_last_error(ctx.h).decode()
        assert_stats_close(st, ref)
        np.testing.assert_allclose(st["sums"], ref["sums"], rtol=1e-4, atol=1e-9)
    # with timing on, the kernel time reported is this call's
    ctx.set_timing(True)
    rc, _ = _static_stats(ctx, w, r["sk"], n, off, f, r["delta"], r["eta"])
    assert rc == mk.MK_OK
    assert ctx.last_kernel_ms() > 0.0
    ctx.set_timing(False)
    # beyond the stated maximum the call refuses before running anything
    rc, _ = _static_stats(ctx, w, r["sk"], mk.STATIC_MAX_SKEWERS + 1, off, f, r["delta"], r["eta"])
    assert rc == mk.MK_EINVAL
    assert b"MK_STATIC_MAX_SKEWERS" in mk.lib().mk_last_error(ctx.h)
    ctx.close()


def test_static_scratch_needs_tables_and_allocates_nothing():
    """A context that has not yet run an allocating statistics call lacks the
    z-bin tables: the call refuses (MK_EINVAL) instead of allocating them.  A
    fresh context lacks every table.  Once an allocating statistics call has
    run, the call leaves the device's free memory unchanged."""
    w = si.workload("tiny")
    d, e = si.gaussian_box(w["n"], w["cell"], w["seed_box"], backend="numpy")
    n = 200
    pos, ids = si.catalogue(w, n_q=n)
    ctx = mk.Context(0)
    # nothing has run: no pixel tables
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    off0 = torch.zeros(2, dtype=torch.int64, device="cuda")
    rc, _ = _static_stats(ctx, w, dummy, 0, off0, dummy, None, None)
    assert rc == mk.MK_EINVAL and b"pixel tables" in mk.lib().mk_last_error(ctx.h)
    # synthesis and flux only (no statistics call): no z-bin tables
    box = ctx.load_box(w, torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda())
    r = ctx.make_skewers(box, mk.catalogue_tensor(pos, ids), n, w)
    f, off = ctx.flux(w, r["sk"], n, r["delta"], r["eta"])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    rc, _ = _static_stats(ctx, w, r["sk"], n, off, f, r["delta"], r["eta"])
    assert rc == mk.MK_EINVAL and b"z-bin tables" in mk.lib().mk_last_error(ctx.h)
    assert torch.cuda.mem_get_info()[0] == free0
    # after one allocating statistics call the static call allocates nothing
    # (the first static call may make the CUDA driver load the library's device
    # image, which holds the fixed array: free memory is compared after it)
    ref = ctx.stats(w, r["sk"], n, off, f, delta=r["delta"], eta=r["eta"])
    rc, _ = _static_stats(ctx, w, r["sk"], n, off, f, r["delta"], r["eta"])
    assert rc == mk.MK_OK, mk.lib().mk_last_error(ctx.h).decode()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        rc, st = _static_stats(ctx, w, r["sk"], n, off, f, r["delta"], r["eta"])
        assert rc == mk.MK_OK, mk.lib().mk_last_error(ctx.h).decode()
        assert_stats_close(st, ref)
    assert torch.cuda.mem_get_info()[0] == free1
    ctx.close()
