"""GPU path vs the FP64 oracle, element by element, through the C-ABI.

Sizes: the 64^3 / 500-quasar workload in full (several FFT segments per
skewer and a ragged tail), the 512^3 / 100k and 1024^3 / 1M workloads on
sampled skewers in the launch configuration the benchmark times, plus
edge cases (empty catalogue, zero-length skewers, capacity overflow, bad
arguments, every supported FFT length, both box layouts).
"""
import math

import numpy as np
import pytest

import oracle
import skewer_inputs as si
from tests.parity_util import (TOL_STAT, assert_field_close, assert_flux_close, assert_stats_close,
                               box_numpy, oracle_subset, ragged)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2310_18996_gb300 as mk  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = mk.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def tiny():
    w = si.workload("tiny")
    d, e = box_numpy(w)
    pos, ids = si.catalogue(w)
    orc = oracle.run_skewers(w, d, e, pos, ids, n_threads=16)
    st = oracle.stats(w, orc["j_lo"], orc["offsets"], orc["offsets_out"], orc["flux"], orc["delta"], orc["eta"])
    dev = dict(d=torch.from_numpy(d).cuda(), e=torch.from_numpy(e).cuda(),
               qso=mk.catalogue_tensor(pos, ids))
    return dict(w=w, d=d, e=e, pos=pos, ids=ids, orc=orc, st=st, dev=dev)


def records(sk, n):
    return mk.skewer_records(sk, n)


# ------------------------------------------------------------------ tiny workload, full
def test_geometry_matches_oracle_exactly(ctx, tiny):
    w, o = tiny["w"], tiny["orc"]
    box = ctx.load_box(w, tiny["dev"]["d"], tiny["dev"]["e"])
    sk, off, total = ctx.plan(box, tiny["dev"]["qso"], len(tiny["ids"]), w)
    rec = records(sk, len(tiny["ids"]))
    np.testing.assert_array_equal(rec["n"], o["npix"])
    np.testing.assert_array_equal(rec["j_lo"], o["j_lo"])
    np.testing.assert_array_equal(off.cpu().numpy(), o["offsets"])
    np.testing.assert_array_equal(rec["offset"], o["offsets"][:-1])
    assert total == o["offsets"][-1]


def load(ctx, w, d, e, layout):
    if layout == "planar":
        return ctx.load_box(w, d, e)
    if layout == "interleaved":
        return ctx.load_box(w, ctx.pack_box(d, e), None)
    if layout == "halo":
        return ctx.load_box(w, ctx.pack_box(d, e, halo=True), None, layout=mk.BOX_HALO)
    return ctx.load_box(w, ctx.pack_box(d, e, padded=True), None, layout=mk.BOX_PADDED)


def test_padded_pack_repeats_the_periodic_box(ctx, tiny):
    d, e = tiny["dev"]["d"], tiny["dev"]["e"]
    n = tiny["w"]["n"]
    p = ctx.pack_box(d, e, padded=True).view(n + 1, n + 1, n + 1, 2)
    torch.cuda.synchronize()
    idx = torch.arange(n + 1, device="cuda") % n
    ref_d = d.view(n, n, n)[idx][:, idx][:, :, idx]
    ref_e = e.view(n, n, n)[idx][:, idx][:, :, idx]
    assert torch.equal(p[..., 0], ref_d) and torch.equal(p[..., 1], ref_e)


def test_halo_pack_repeats_the_periodic_box(ctx, tiny):
    d, e = tiny["dev"]["d"], tiny["dev"]["e"]
    n = tiny["w"]["n"]
    p = ctx.pack_box(d, e, halo=True).view(n + 6, n + 6, n + 6, 2)
    torch.cuda.synchronize()
    idx = (torch.arange(n + 6, device="cuda") - 3) % n
    ref_d = d.view(n, n, n)[idx][:, idx][:, :, idx]
    ref_e = e.view(n, n, n)[idx][:, idx][:, :, idx]
    assert torch.equal(p[..., 0], ref_d) and torch.equal(p[..., 1], ref_e)


@pytest.mark.parametrize("layout", ["planar", "interleaved", "padded", "halo"])
def test_pre_fgpa_fields_match_oracle(ctx, tiny, layout):
    w, o, dv = tiny["w"], tiny["orc"], tiny["dev"]
    box = load(ctx, w, dv["d"], dv["e"], layout)
    r = ctx.make_skewers(box, dv["qso"], len(tiny["ids"]), w)
    ctx.sync()
    assert_field_close(r["delta"].cpu().numpy(), o["delta"], "delta_tot")
    assert_field_close(r["eta"].cpu().numpy(), o["eta"], "eta")


@pytest.mark.parametrize("rebin", [1, 3])
def test_flux_matches_oracle(ctx, tiny, rebin):
    w, dv = tiny["w"], tiny["dev"]
    box = ctx.load_box(w, dv["d"], dv["e"])
    n = len(tiny["ids"])
    r = ctx.make_skewers(box, dv["qso"], n, w)
    f, off = ctx.flux(w, r["sk"], n, r["delta"], r["eta"], rebin=rebin)
    o = tiny["orc"] if rebin == 1 else oracle.run_skewers(w, tiny["d"], tiny["e"], tiny["pos"], tiny["ids"],
                                                          rebin=rebin, n_threads=16)
    np.testing.assert_array_equal(off.cpu().numpy(), o["offsets_out"])
    assert_flux_close(f[: o["offsets_out"][-1]].cpu().numpy(), o["flux"])
    if rebin > 1:
        st_o = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"],
                            rebin=rebin)
        st_g = ctx.stats(w, r["sk"], n, off, f, rebin=rebin, delta=r["delta"], eta=r["eta"])
        assert_stats_close(st_g, st_o)


@pytest.mark.parametrize("n_fft,cap", [(256, 1), (1024, 2)])
def test_long_register_carry_matches_oracle(ctx, tiny, n_fft, cap):
    """The whole tiny workload through one or two CTAs: every team runs
    hundreds of consecutive segments, carrying its pixel sums in registers
    across segments and z bins (flushed at bin ends), in the fused pass, the
    statistics pass and the tuning pass."""
    w = si.shrink(tiny["w"], n_fft=n_fft)
    dv = tiny["dev"]
    n = len(tiny["ids"])
    o = oracle.run_skewers(w, tiny["d"], tiny["e"], tiny["pos"], tiny["ids"], n_threads=16)
    so = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    box = ctx.load_box(w, ctx.pack_box(dv["d"], dv["e"], padded=True), None, layout=mk.BOX_PADDED)
    ctx.set_grid_cap(cap)
    try:
        st, g = ctx.run(box, dv["qso"], n, w, flags=mk.STATS | mk.STORE_FIELDS | mk.STORE_FLUX)
        tot = int(o["offsets"][-1])
        assert_field_close(g["delta"][:tot].cpu().numpy(), o["delta"], "delta_tot")
        assert_flux_close(g["flux"][:tot].cpu().numpy(), o["flux"])
        assert_stats_close(st, so)
        st2 = ctx.stats(w, g["sk"], n, g["offsets"], g["flux"], delta=g["delta"], eta=g["eta"])
        assert_stats_close(st2, so)
        st3 = ctx.flux_stats(w, g["sk"], n, g["offsets"], g["delta"], g["eta"])
        assert_stats_close(st3, so)
    finally:
        ctx.set_grid_cap(0)
    # segments per team: the carry spans hundreds of segments
    segs = int(np.sum((o["npix"] + n_fft - 1) // n_fft))
    teams = cap * (256 // (n_fft // 8))
    assert segs / teams >= 100


def test_split_statistics_match_oracle(ctx, tiny):
    w, dv = tiny["w"], tiny["dev"]
    box = ctx.load_box(w, dv["d"], dv["e"])
    n = len(tiny["ids"])
    r = ctx.make_skewers(box, dv["qso"], n, w)
    f, off = ctx.flux(w, r["sk"], n, r["delta"], r["eta"])
    st = ctx.stats(w, r["sk"], n, off, f, delta=r["delta"], eta=r["eta"])
    assert_stats_close(st, tiny["st"])
    # without the fields the flux statistics are unchanged
    st2 = ctx.stats(w, r["sk"], n, off, f)
    np.testing.assert_array_equal(st2["mean_flux"], st["mean_flux"])
    np.testing.assert_array_equal(st2["p1d_sum"], st["p1d_sum"])


def test_tuning_pass_matches_oracle_and_split_path(ctx, tiny):
    w, dv = tiny["w"], tiny["dev"]
    box = ctx.load_box(w, dv["d"], dv["e"])
    n = len(tiny["ids"])
    r = ctx.make_skewers(box, dv["qso"], n, w)
    st = ctx.flux_stats(w, r["sk"], n, r["offsets"], r["delta"], r["eta"])
    assert_stats_close(st, tiny["st"])
    f, off = ctx.flux(w, r["sk"], n, r["delta"], r["eta"])
    st2 = ctx.stats(w, r["sk"], n, off, f, delta=r["delta"], eta=r["eta"])
    for k in ("sums", "p1d_sum", "n_seg"):
        np.testing.assert_array_equal(st[k], st2[k])
    # other FGPA parameters on the same stored fields
    w2 = dict(w)
    w2["node_b"] = [1.2 + 0.05 * i for i in range(len(w["node_z"]))]
    w2["node_c"] = [0.7] * len(w["node_z"])
    o2 = oracle.run_skewers(w2, tiny["d"], tiny["e"], tiny["pos"], tiny["ids"], n_threads=16)
    so2 = oracle.stats(w2, o2["j_lo"], o2["offsets"], o2["offsets_out"], o2["flux"], o2["delta"], o2["eta"])
    st3 = ctx.flux_stats(w2, r["sk"], n, r["offsets"], r["delta"], r["eta"])
    assert_stats_close(st3, so2)


def test_tuning_pass_unaligned_fields_match_oracle(ctx, tiny):
    """Stored fields that do not start on a 16-byte boundary cannot be staged
    with 16-byte asynchronous copies; the pass then runs the unstaged kernel,
    which must give the same statistics."""
    w, dv = tiny["w"], tiny["dev"]
    box = ctx.load_box(w, dv["d"], dv["e"])
    n = len(tiny["ids"])
    r = ctx.make_skewers(box, dv["qso"], n, w)
    tot = r["total"]
    d1 = torch.empty(tot + 1, dtype=torch.float32, device="cuda")
    e1 = torch.empty(tot + 1, dtype=torch.float32, device="cuda")
    d1[1:] = r["delta"]
    e1[1:] = r["eta"]
    assert d1[1:].data_ptr() % 16 != 0 and r["delta"].data_ptr() % 16 == 0
    st_u = ctx.flux_stats(w, r["sk"], n, r["offsets"], d1[1:], e1[1:])
    assert_stats_close(st_u, tiny["st"])
    st_a = ctx.flux_stats(w, r["sk"], n, r["offsets"], r["delta"], r["eta"])
    for k in ("sums", "p1d_sum", "n_seg"):
        np.testing.assert_array_equal(st_u[k], st_a[k])


def test_injected_faults_leave_the_context_usable(tiny):
    """Host-side error paths (mk_inject_fault): on a fresh context an injected
    workspace allocation failure makes the fused run return MK_ENOMEM, and an
    injected launch failure makes the tuning pass and the fused run return
    MK_ECUDA; each time the next call on the same context is correct."""
    c = mk.Context(0)  # fresh, so that the run must grow its workspaces
    try:
        w, dv = tiny["w"], tiny["dev"]
        box = c.load_box(w, dv["d"], dv["e"])
        n = len(tiny["ids"])
        c.inject_fault(mk.FAULT_ALLOC)
        with pytest.raises(mk.MkError) as ei:
            c.run(box, dv["qso"], n, w, flags=mk.STATS)
        assert ei.value.code == mk.MK_ENOMEM
        st, _ = c.run(box, dv["qso"], n, w, flags=mk.STATS)
        assert_stats_close(st, tiny["st"])
        r = c.make_skewers(box, dv["qso"], n, w)
        c.inject_fault(mk.FAULT_LAUNCH)
        with pytest.raises(mk.MkError) as ei:
            c.flux_stats(w, r["sk"], n, r["offsets"], r["delta"], r["eta"])
        assert ei.value.code == mk.MK_ECUDA
        assert_stats_close(c.flux_stats(w, r["sk"], n, r["offsets"], r["delta"], r["eta"]), tiny["st"])
        c.inject_fault(mk.FAULT_LAUNCH)
        with pytest.raises(mk.MkError) as ei:
            c.run(box, dv["qso"], n, w, flags=mk.STATS)
        assert ei.value.code == mk.MK_ECUDA
        st, _ = c.run(box, dv["qso"], n, w, flags=mk.STATS)
        assert_stats_close(st, tiny["st"])
        with pytest.raises(mk.MkError) as ei:
            c.inject_fault(7)
        assert ei.value.code == mk.MK_EINVAL
    finally:
        c.close()


def test_tuning_pass_wait_times_out_and_context_survives(ctx, tiny):
    """The tuning pass's one device wait (the mbarrier of each segment's bulk
    copies) is bounded: with the test hook no copy is issued, every team gives
    up after a short wait, the call reports MK_ETIMEOUT, and the next pass on
    the same context is correct."""
    w, dv = tiny["w"], tiny["dev"]
    box = ctx.load_box(w, dv["d"], dv["e"])
    n = len(tiny["ids"])
    r = ctx.make_skewers(box, dv["qso"], n, w)
    assert r["delta"].data_ptr() % 16 == 0 and r["eta"].data_ptr() % 16 == 0  # the staged kernel runs
    ctx.set_wait_test(True)
    try:
        with pytest.raises(mk.MkError) as ei:
            ctx.flux_stats(w, r["sk"], n, r["offsets"], r["delta"], r["eta"])
        assert ei.value.code == mk.MK_ETIMEOUT
    finally:
        ctx.set_wait_test(False)
    st = ctx.flux_stats(w, r["sk"], n, r["offsets"], r["delta"], r["eta"])
    assert_stats_close(st, tiny["st"])


@pytest.mark.parametrize("layout", ["planar", "padded"])
def test_fused_path_matches_split_path_and_oracle(ctx, tiny, layout):
    w, dv = tiny["w"], tiny["dev"]
    box = load(ctx, w, dv["d"], dv["e"], layout)
    n = len(tiny["ids"])
    st, o = ctx.run(box, dv["qso"], n, w, flags=mk.STATS | mk.STORE_FIELDS | mk.STORE_FLUX)
    r = ctx.make_skewers(box, dv["qso"], n, w)
    f, off = ctx.flux(w, r["sk"], n, r["delta"], r["eta"])
    tot = r["total"]
    assert torch.equal(o["delta"][:tot], r["delta"]) and torch.equal(o["eta"][:tot], r["eta"])
    assert torch.equal(o["flux"][:tot], f[:tot])
    assert_stats_close(st, tiny["st"])
    st_fast, _ = ctx.run(box, dv["qso"], n, w, flags=mk.STATS)
    for k in ("sums", "p1d_sum", "n_seg"):
        np.testing.assert_array_equal(st_fast[k], st[k])


@pytest.mark.parametrize("layout", ["planar", "padded"])
@pytest.mark.parametrize("n_fft", [512, 1024, 2048])
def test_other_fft_lengths(ctx, tiny, n_fft, layout):
    w = si.shrink(tiny["w"], n_fft=n_fft)
    idx = np.arange(0, 500, 7)
    pos, ids = tiny["pos"][idx], tiny["ids"][idx]
    o = oracle.run_skewers(w, tiny["d"], tiny["e"], pos, ids, n_threads=16)
    so = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    box = load(ctx, w, tiny["dev"]["d"], tiny["dev"]["e"], layout)
    st, g = ctx.run(box, mk.catalogue_tensor(pos, ids), len(ids), w,
                    flags=mk.STATS | mk.STORE_FIELDS | mk.STORE_FLUX)
    tot = o["offsets"][-1]
    assert_field_close(g["delta"][:tot].cpu().numpy(), o["delta"], "delta_tot")
    assert_field_close(g["eta"][:tot].cpu().numpy(), o["eta"], "eta")
    assert_flux_close(g["flux"][:tot].cpu().numpy(), o["flux"])
    assert_stats_close(st, so, check_fields=False)
    # the tuning pass over the stored fields: teams of N/8 threads (several
    # warps; at N = 2048 the whole CTA) stage the fields with bulk copies
    st2 = ctx.flux_stats(w, g["sk"], len(ids), g["offsets"], g["delta"], g["eta"])
    assert_stats_close(st2, so, check_fields=False)


@pytest.mark.parametrize("n_fft", [256, 2048])
def test_segments_crossing_many_z_bins(ctx, tiny, n_fft):
    # narrow z bins: a segment of N pixels crosses several bin edges (up to ~10
    # at N = 2048), inside one warp's pixels and between the warps of a team
    w = si.shrink(tiny["w"], n_fft=n_fft, n_zbins=32, z_bin_lo=1.8, dz_bin=0.05, n_kbins=8)
    idx = np.arange(0, 500, 3)
    pos, ids = tiny["pos"][idx], tiny["ids"][idx]
    o = oracle.run_skewers(w, tiny["d"], tiny["e"], pos, ids, n_threads=16)
    so = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    assert np.count_nonzero(so["sums"][:, 0]) >= 10
    box = load(ctx, w, tiny["dev"]["d"], tiny["dev"]["e"], "padded")
    st, g = ctx.run(box, mk.catalogue_tensor(pos, ids), len(ids), w,
                    flags=mk.STATS | mk.STORE_FLUX | mk.STORE_FIELDS)
    assert_flux_close(g["flux"][:o["offsets"][-1]].cpu().numpy(), o["flux"])
    assert_stats_close(st, so)
    # and the tuning pass over the stored fields, the same bin edges
    assert_stats_close(ctx.flux_stats(w, g["sk"], len(ids), g["offsets"], g["delta"], g["eta"]), so)


# ------------------------------------------------------------------ Gaussian-kernel interpolation (Sec. 2.3)
@pytest.mark.parametrize("n_fft,step", [(256, 1), (1024, 5)])
def test_gauss7_path_matches_oracle(ctx, tiny, n_fft, step):
    w = si.shrink(tiny["w"], n_fft=n_fft, interp=mk.INTERP_GAUSS7)
    idx = np.arange(0, 500, step)
    pos, ids = tiny["pos"][idx], tiny["ids"][idx]
    o = oracle.run_skewers(w, tiny["d"], tiny["e"], pos, ids, n_threads=16)
    so = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    box = load(ctx, w, tiny["dev"]["d"], tiny["dev"]["e"], "halo")
    st, g = ctx.run(box, mk.catalogue_tensor(pos, ids), len(ids), w,
                    flags=mk.STATS | mk.STORE_FIELDS | mk.STORE_FLUX)
    tot = o["offsets"][-1]
    assert_field_close(g["delta"][:tot].cpu().numpy(), o["delta"], "delta_tot")
    assert_field_close(g["eta"][:tot].cpu().numpy(), o["eta"], "eta")
    assert_flux_close(g["flux"][:tot].cpu().numpy(), o["flux"])
    assert_stats_close(st, so, check_fields=(step == 1))
    # the Gaussian average smooths: its eta differs from trilinear's
    w_tri = dict(w)
    w_tri["interp"] = mk.INTERP_TRILINEAR
    _, gt = ctx.run(box, mk.catalogue_tensor(pos, ids), len(ids), w_tri, flags=mk.STORE_FIELDS)
    assert not torch.equal(gt["eta"][:tot], g["eta"][:tot])


def test_gauss7_needs_a_halo_box(ctx, tiny):
    w = si.shrink(tiny["w"], interp=mk.INTERP_GAUSS7)
    box = load(ctx, w, tiny["dev"]["d"], tiny["dev"]["e"], "padded")
    with pytest.raises(mk.MkError) as e:
        ctx.run(box, tiny["dev"]["qso"], 10, w)
    assert e.value.code == mk.MK_EINVAL
    bad = dict(w)
    bad["interp"] = 2
    with pytest.raises(mk.MkError):
        ctx.run(load(ctx, w, tiny["dev"]["d"], tiny["dev"]["e"], "halo"), tiny["dev"]["qso"], 10, bad)


# ------------------------------------------------------------------ radial eta_par from six eta_pq boxes (Eq. eta)
@pytest.fixture(scope="module")
def tensor(tiny):
    w = si.shrink(tiny["w"], eta_mode=1)
    d, e6 = si.gaussian_box_tensor(w["n"], w["cell"], w["seed_box"])
    assert np.array_equal(d, tiny["d"])
    return dict(w=w, d=d, e6=e6, dev_d=torch.from_numpy(d).cuda(), dev_e6=torch.from_numpy(e6).cuda())


def test_tensor_pack_layout(ctx, tensor):
    n = tensor["w"]["n"]
    p = ctx.pack_box_tensor(tensor["dev_d"], tensor["dev_e6"]).view(n + 1, n + 1, n + 1, 8)
    torch.cuda.synchronize()
    idx = torch.arange(n + 1, device="cuda") % n
    pick = lambda b: b.view(n, n, n)[idx][:, idx][:, :, idx]
    assert torch.equal(p[..., 0], pick(tensor["dev_d"]))
    for c in range(6):
        assert torch.equal(p[..., 1 + c], pick(tensor["dev_e6"][c]))
    assert torch.count_nonzero(p[..., 7]) == 0


def test_tensor_eta_path_matches_oracle(ctx, tiny, tensor):
    w = tensor["w"]
    idx = np.arange(0, 500, 2)
    pos, ids = tiny["pos"][idx], tiny["ids"][idx]
    o = oracle.run_skewers(w, tensor["d"], tensor["e6"], pos, ids, n_threads=16)
    so = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    box = ctx.load_box(w, ctx.pack_box_tensor(tensor["dev_d"], tensor["dev_e6"]), None, layout=mk.BOX_TENSOR)
    st, g = ctx.run(box, mk.catalogue_tensor(pos, ids), len(ids), w,
                    flags=mk.STATS | mk.STORE_FIELDS | mk.STORE_FLUX)
    tot = o["offsets"][-1]
    assert_field_close(g["delta"][:tot].cpu().numpy(), o["delta"], "delta_tot")
    assert_field_close(g["eta"][:tot].cpu().numpy(), o["eta"], "eta_par")
    assert_flux_close(g["flux"][:tot].cpu().numpy(), o["flux"])
    assert_stats_close(st, so, check_fields=False)


def test_tensor_isotropic_diagonal_equals_single_box_path(ctx, tiny, tensor):
    w = tensor["w"]
    e = tiny["dev"]["e"]
    z = torch.zeros_like(e)
    iso = torch.stack([e, e, e, z, z, z])
    box6 = ctx.load_box(w, ctx.pack_box_tensor(tiny["dev"]["d"], iso), None, layout=mk.BOX_TENSOR)
    box1 = load(ctx, tiny["w"], tiny["dev"]["d"], e, "padded")
    n = 100
    _, g6 = ctx.run(box6, tiny["dev"]["qso"], n, w, flags=mk.STORE_FIELDS)
    _, g1 = ctx.run(box1, tiny["dev"]["qso"], n, tiny["w"], flags=mk.STORE_FIELDS)
    tot = int(tiny["orc"]["offsets"][n])
    assert torch.equal(g6["delta"][:tot], g1["delta"][:tot])
    # u_x^2 + u_y^2 + u_z^2 = 1 up to FP32 rounding of the weights
    assert_field_close(g6["eta"][:tot].cpu().numpy(), g1["eta"][:tot].cpu().numpy().astype(np.float64), "eta")


def test_saved_pre_production_round_trip(ctx, tiny, tmp_path):
    # Sec. 3: pre-FGPA skewers written once, post-production (FGPA and
    # statistics with other parameters) run from the file
    w, dv = tiny["w"], tiny["dev"]
    box = ctx.load_box(w, dv["d"], dv["e"])
    n = len(tiny["ids"])
    r = ctx.make_skewers(box, dv["qso"], n, w)
    f = tmp_path / "pre.mksk"
    ctx.save_skewers(str(f), r, n)
    assert f.stat().st_size == 24 + n * mk.SKEWER_BYTES + 8 * (n + 1) + 8 * r["total"]
    q, nq = ctx.load_skewers(str(f))
    assert nq == n and q["total"] == r["total"]
    assert torch.equal(q["sk"][: n * mk.SKEWER_BYTES], r["sk"][: n * mk.SKEWER_BYTES])
    assert torch.equal(q["offsets"], r["offsets"])
    tot = r["total"]
    assert torch.equal(q["delta"][:tot], r["delta"][:tot]) and torch.equal(q["eta"][:tot], r["eta"][:tot])
    w2 = dict(w)
    w2["node_b"] = [1.3] * len(w["node_z"])
    a = ctx.flux_stats(w2, r["sk"], n, r["offsets"], r["delta"], r["eta"])
    b = ctx.flux_stats(w2, q["sk"], n, q["offsets"], q["delta"], q["eta"])
    for k in ("sums", "p1d_sum", "n_seg"):
        np.testing.assert_array_equal(a[k], b[k])
    # a truncated or foreign file is refused, the context stays usable
    bad = tmp_path / "bad.mksk"
    bad.write_bytes(f.read_bytes()[:100])
    with pytest.raises(mk.MkError):
        ctx.load_skewers(str(bad))
    bad.write_bytes(b"NOTASKEW" + bytes(16))
    with pytest.raises(mk.MkError):
        ctx.load_skewers(str(bad))
    # records or offsets that do not tile the pixel arrays are refused
    raw = f.read_bytes()
    for at in (24 + mk.SKEWER_BYTES, 24 + n * mk.SKEWER_BYTES + 8):  # record 1's offset; offsets[1]
        v = int.from_bytes(raw[at:at + 8], "little") + 1
        bad.write_bytes(raw[:at] + v.to_bytes(8, "little") + raw[at + 8:])
        with pytest.raises(mk.MkError) as ei:
            ctx.load_skewers(str(bad))
        assert ei.value.code == mk.MK_EINVAL
    c = ctx.flux_stats(w2, q["sk"], n, q["offsets"], q["delta"], q["eta"])
    np.testing.assert_array_equal(c["sums"], a["sums"])


def test_flux_refuses_records_past_the_pixel_tables(ctx, tiny):
    # records whose pixels lie beyond the pixel tables (made for another pixel
    # length) set the range error instead of reading past the tables
    w, dv = tiny["w"], tiny["dev"]
    box = ctx.load_box(w, dv["d"], dv["e"])
    n = len(tiny["ids"])
    r = ctx.make_skewers(box, dv["qso"], n, w)
    ctx.sync()
    sk = r["sk"].clone()
    sk[: n * mk.SKEWER_BYTES].view(torch.int32).view(n, mk.SKEWER_BYTES // 4)[:, 3] = 1 << 30  # j_lo
    ctx.flux(w, sk, n, r["delta"], r["eta"])
    with pytest.raises(mk.MkError) as ei:
        ctx.sync()
    assert ei.value.code == mk.MK_ERANGE
    with pytest.raises(mk.MkError) as ei:  # the tuning pass (k_stats) checks them too
        ctx.flux_stats(w, sk, n, r["offsets"], r["delta"], r["eta"])
    assert ei.value.code == mk.MK_ERANGE
    f, _ = ctx.flux(w, r["sk"], n, r["delta"], r["eta"])
    ctx.sync()
    assert torch.isfinite(f[: r["total"]]).all()
    st = ctx.flux_stats(w, r["sk"], n, r["offsets"], r["delta"], r["eta"])
    assert st["sums"][:, 0].sum() > 0


def test_small_scale_field_is_whitened_philox_modes(ctx, tiny):
    # zero box: delta_tot is delta_S; each segment's DFT over its amplitude gives
    # back the oracle's modes
    w = tiny["w"]
    z = torch.zeros_like(tiny["dev"]["d"])
    box = ctx.load_box(w, z, z)
    idx = np.arange(5)
    r = ctx.make_skewers(box, mk.catalogue_tensor(tiny["pos"][idx], tiny["ids"][idx]), 5, w)
    ds = r["delta"].cpu().numpy().astype(np.float64)
    off = r["offsets"].cpu().numpy()
    N = w["n_fft"]
    for q in range(5):
        x = ragged(ds, off, q)
        for s in range(len(x) // N):
            X = np.fft.rfft(x[s * N:(s + 1) * N])
            ref = oracle.small_scale_modes(w, int(tiny["ids"][q]), s)
            # pixel errors below 2e-6 sigma give mode errors below 2e-6 of the
            # RMS mode amplitude sqrt(N) sigma (Parseval); allow 5x for the max
            rms = math.sqrt(np.mean(np.abs(ref[1:]) ** 2))
            np.testing.assert_allclose(X[1:], ref[1:], rtol=0, atol=1e-5 * rms)
            assert abs(X[0]) < 1e-5 * rms


def _p_s_nodes_workload(w):
    # three redshift nodes with 0.5x, 1x and 2.5x the small-scale power
    # (Sec. 2.6 tunes P_s at each z_t); segment windows fall on both sides of
    # the middle node and beyond the outer ones
    return si.shrink(w, p_s=np.stack([0.5 * w["p_s"], w["p_s"], 2.5 * w["p_s"]]), p_s_z=[2.1, 2.4, 2.8])


def test_z_dependent_small_scale_power_matches_oracle(ctx, tiny):
    w, dv = _p_s_nodes_workload(tiny["w"]), tiny["dev"]
    n = len(tiny["ids"])
    o = oracle.run_skewers(w, tiny["d"], tiny["e"], tiny["pos"], tiny["ids"], n_threads=16)
    so = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    box = load(ctx, w, dv["d"], dv["e"], "padded")
    st, g = ctx.run(box, dv["qso"], n, w, flags=mk.STATS | mk.STORE_FIELDS | mk.STORE_FLUX)
    tot = int(o["offsets"][-1])
    assert_field_close(g["delta"][:tot].cpu().numpy(), o["delta"], "delta_tot")
    assert_field_close(g["eta"][:tot].cpu().numpy(), o["eta"], "eta")
    assert_flux_close(g["flux"][:tot].cpu().numpy(), o["flux"])
    assert_stats_close(st, so)
    # the node tables change the field: it is not the one-table field
    st1, g1 = ctx.run(box, dv["qso"], n, tiny["w"], flags=mk.STATS | mk.STORE_FIELDS)
    d0, d1 = g["delta"][:tot].cpu().numpy(), g1["delta"][:tot].cpu().numpy()
    assert np.abs(d0 - d1).max() > 0.1
    # back on one table, the cached amplitudes are replaced again
    st2, g2 = ctx.run(box, dv["qso"], n, tiny["w"], flags=mk.STATS | mk.STORE_FIELDS)
    assert torch.equal(g2["delta"][:tot], g1["delta"][:tot])


def test_z_dependent_small_scale_power_modes(ctx, tiny):
    # zero box: each segment's DFT gives back the oracle's modes at the
    # power interpolated to the mean z of its window
    w = _p_s_nodes_workload(tiny["w"])
    z = torch.zeros_like(tiny["dev"]["d"])
    box = ctx.load_box(w, z, z)
    idx = np.arange(6)
    r = ctx.make_skewers(box, mk.catalogue_tensor(tiny["pos"][idx], tiny["ids"][idx]), 6, w)
    ds = r["delta"].cpu().numpy().astype(np.float64)
    off = r["offsets"].cpu().numpy()
    rec = records(r["sk"], 6)
    N = w["n_fft"]
    for q in range(6):
        x = ragged(ds, off, q)
        for s in range(len(x) // N):
            X = np.fft.rfft(x[s * N:(s + 1) * N])
            ref = oracle.small_scale_modes(w, int(tiny["ids"][q]), s, j0=int(rec["j_lo"][q]) + s * N)
            rms = math.sqrt(np.mean(np.abs(ref[1:]) ** 2))
            np.testing.assert_allclose(X[1:], ref[1:], rtol=0, atol=1e-5 * rms)


def test_z_dependent_small_scale_power_rejects_bad_nodes(ctx, tiny):
    box = ctx.load_box(tiny["w"], tiny["dev"]["d"], tiny["dev"]["e"])
    w = si.shrink(_p_s_nodes_workload(tiny["w"]), p_s_z=[2.1, 2.1, 2.8])
    with pytest.raises(mk.MkError) as ei:
        ctx.run(box, tiny["dev"]["qso"], 10, w)
    assert ei.value.code == mk.MK_EINVAL
    with pytest.raises(ValueError):
        mk.skewer_params(si.shrink(tiny["w"], p_s_z=[2.0, 3.0]))


def test_graph_replay_and_autotune_match_direct_launch(ctx, tiny):
    w, dv = tiny["w"], tiny["dev"]
    box = load(ctx, w, dv["d"], dv["e"], "padded")
    n = len(tiny["ids"])
    flags = mk.STATS | mk.STORE_FLUX
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        st_tuned, o = ctx.run(box, dv["qso"], n, w, flags=flags | mk.AUTOTUNE, capacity=tiny["orc"]["offsets"][-1])
        threads, occ, tuned = ctx.launch_config(w["n_fft"], flags=flags, layout=mk.BOX_PADDED)
        assert tuned and threads in (128, 256) and occ in (2, 3, 4)
        st_direct, _ = ctx.run(box, dv["qso"], n, w, flags=flags, outputs=o, capacity=o["flux"].numel())
        f_direct = o["flux"].clone()
        o["flux"].zero_()
        st_g1, _ = ctx.run(box, dv["qso"], n, w, flags=flags | mk.GRAPH, outputs=o, capacity=o["flux"].numel())
        st_g2, _ = ctx.run(box, dv["qso"], n, w, flags=flags | mk.GRAPH, outputs=o, capacity=o["flux"].numel())
        # a changed argument (the FGPA nodes) must re-capture, not replay
        w2 = dict(w)
        w2["node_b"] = [1.5] * len(w["node_z"])
        st_g3, _ = ctx.run(box, dv["qso"], n, w2, flags=flags | mk.GRAPH, outputs=o, capacity=o["flux"].numel())
        st_d3, _ = ctx.run(box, dv["qso"], n, w2, flags=flags, outputs=o, capacity=o["flux"].numel())
    torch.cuda.synchronize()
    for st in (st_g1, st_g2):
        for k in ("sums", "p1d_sum", "n_seg"):
            np.testing.assert_array_equal(st[k], st_direct[k])
    for k in ("sums", "p1d_sum", "n_seg"):
        np.testing.assert_array_equal(st_g3[k], st_d3[k])
    assert not np.array_equal(st_g3["mean_flux"], st_g1["mean_flux"])
    assert_stats_close(st_tuned, tiny["st"], check_fields=False)
    assert_stats_close(st_direct, tiny["st"], check_fields=False)
    tot = tiny["orc"]["offsets"][-1]
    assert_flux_close(f_direct[:tot].cpu().numpy(), tiny["orc"]["flux"])


def test_flux_stored_into_pinned_host_memory(ctx, tiny):
    w, dv = tiny["w"], tiny["dev"]
    box = load(ctx, w, dv["d"], dv["e"], "padded")
    n = len(tiny["ids"])
    tot = int(tiny["orc"]["offsets"][-1])
    host = torch.full((tot,), float("nan"), dtype=torch.float32).pin_memory()
    st_h, _ = ctx.run(box, dv["qso"], n, w, flags=mk.STATS | mk.STORE_FLUX, capacity=tot, outputs={"flux": host})
    st_d, o = ctx.run(box, dv["qso"], n, w, flags=mk.STATS | mk.STORE_FLUX, capacity=tot)
    torch.cuda.synchronize()
    assert torch.equal(host, o["flux"][:tot].cpu())
    for k in ("sums", "p1d_sum", "n_seg"):
        np.testing.assert_array_equal(st_h[k], st_d[k])


@pytest.mark.parametrize("n_chunks", [1, 5])
def test_host_pipelined_run_matches_device_run(ctx, tiny, n_chunks):
    w, dv = tiny["w"], tiny["dev"]
    box = load(ctx, w, dv["d"], dv["e"], "padded")
    n = len(tiny["ids"])
    off = tiny["orc"]["offsets"]
    tot = int(off[-1])
    hq = mk.catalogue_tensor(tiny["pos"], tiny["ids"], device="cpu").pin_memory()
    hf = torch.full((tot + 7,), float("nan"), dtype=torch.float32).pin_memory()
    st_h, total = ctx.run_host(box, hq, n, w, hf, n_chunks=n_chunks)
    assert total == tot
    st_d, o = ctx.run(box, dv["qso"], n, w, flags=mk.STATS | mk.STORE_FLUX, capacity=tot)
    torch.cuda.synchronize()
    assert torch.equal(hf[:tot], o["flux"][:tot].cpu())
    assert torch.isnan(hf[tot:]).all()
    np.testing.assert_array_equal(st_h["sums"][:, 0], st_d["sums"][:, 0])
    np.testing.assert_array_equal(st_h["n_seg"], st_d["n_seg"])
    assert_stats_close(st_h, tiny["st"])
    # more slices than quasars (empty slices), no statistics
    rb = mk.QSO_DTYPE.itemsize
    hf.fill_(float("nan"))
    st3, t3 = ctx.run_host(box, hq[: 3 * rb], 3, w, hf, n_chunks=n_chunks + 4, stats=False)
    assert st3 is None and t3 == off[3]
    assert torch.equal(hf[:t3], o["flux"][:t3].cpu())
    # a flux array too small is refused before anything is written
    hf.fill_(float("nan"))
    with pytest.raises(mk.MkError) as e:
        ctx.run_host(box, hq, n, w, hf[: tot - 1], n_chunks=n_chunks)
    assert e.value.code == mk.MK_ERANGE and torch.isnan(hf).all()


def test_graph_needs_a_non_default_stream(ctx, tiny):
    w, dv = tiny["w"], tiny["dev"]
    box = ctx.load_box(w, dv["d"], dv["e"])
    with torch.cuda.stream(torch.cuda.default_stream()):
        with pytest.raises(mk.MkError) as ei:
            ctx.run(box, dv["qso"], 10, w, flags=mk.STATS | mk.GRAPH)
    assert ei.value.code == mk.MK_EINVAL


# ------------------------------------------------------------------ edge cases
def test_empty_catalogue_and_zero_length_skewers(ctx, tiny):
    w, dv = tiny["w"], tiny["dev"]
    box = ctx.load_box(w, dv["d"], dv["e"])
    q0 = mk.catalogue_tensor(np.zeros((0, 3)), np.zeros(0, np.uint64))
    st, o = ctx.run(box, q0, 0, w, flags=mk.STATS)
    assert o["offsets"][0].item() == 0 and st["sums"].sum() == 0
    # quasars too close (forest below z = 0) or at the observer give n = 0
    pos = np.array([[10.0, 0.0, 0.0], [0.0, 0.0, 0.0], tiny["pos"][0]])
    ids = np.array([7, 8, 9], np.uint64)
    sk, off, total = ctx.plan(box, mk.catalogue_tensor(pos, ids), 3, w)
    rec = records(sk, 3)
    assert rec["n"][0] == 0 and rec["n"][1] == 0 and rec["n"][2] == tiny["orc"]["npix"][0]
    r = ctx.make_skewers(box, mk.catalogue_tensor(pos, ids), 3, w)
    o2 = oracle.run_skewers(w, tiny["d"], tiny["e"], pos, ids)
    assert_field_close(r["delta"].cpu().numpy(), o2["delta"], "delta_tot")


def test_capacity_overflow_is_reported_and_context_survives(ctx, tiny):
    w, dv = tiny["w"], tiny["dev"]
    box = ctx.load_box(w, dv["d"], dv["e"])
    n = 20
    qso = mk.catalogue_tensor(tiny["pos"][:n], tiny["ids"][:n])
    sk, off, total = ctx.plan(box, qso, n, w)
    small = torch.empty(total // 2, dtype=torch.float32, device="cuda")
    p = mk.skewer_params(w)
    import ctypes as C
    rc = mk.lib().mk_make_skewers(ctx.h, box.handle, C.c_void_p(qso.data_ptr()), n, C.byref(p),
                                  C.c_void_p(sk.data_ptr()), C.c_void_p(off.data_ptr()),
                                  C.c_void_p(small.data_ptr()), C.c_void_p(small.data_ptr()),
                                  total // 2, None)
    assert rc == mk.MK_OK
    with pytest.raises(mk.MkError) as ei:
        ctx.sync()
    assert ei.value.code == mk.MK_ERANGE
    ctx.sync()  # cleared
    r = ctx.make_skewers(box, qso, n, w)
    assert r["total"] == total


def test_invalid_arguments(ctx, tiny):
    w = si.shrink(tiny["w"], n_fft=300)
    box = ctx.load_box(tiny["w"], tiny["dev"]["d"], tiny["dev"]["e"])
    with pytest.raises(mk.MkError) as ei:
        ctx.plan(box, tiny["dev"]["qso"], 10, w)
    assert ei.value.code == mk.MK_EINVAL
    bad = dict(tiny["w"])
    bad["n"] = 48
    with pytest.raises(mk.MkError):
        ctx.load_box(bad, tiny["dev"]["d"], tiny["dev"]["e"])
    nodes = mk.fgpa_nodes(tiny["w"])
    nodes.z[3] = nodes.z[2]
    with pytest.raises(mk.MkError):
        ctx.run(box, tiny["dev"]["qso"], 10, tiny["w"], nodes=nodes)


# ------------------------------------------------------------------ full-size workloads, sampled
def _full_size_check(ctx, w, n_sample, seed, lognormal=False, layout="padded"):
    torch.cuda.empty_cache()
    d, e = si.gaussian_box(w["n"], w["cell"], w["seed_box"], backend="torch")
    dh = d.cpu().numpy()
    pos, ids = si.catalogue(w, delta=dh if lognormal else None)
    qso = mk.catalogue_tensor(pos, ids)
    eh = e.cpu().numpy()
    box = load(ctx, w, d, e, layout)
    del d, e
    st, g = ctx.run(box, qso, len(ids), w, flags=mk.STATS | mk.STORE_FLUX | mk.STORE_FIELDS)
    rec = records(g["sk"], len(ids))
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(ids), n_sample, replace=False))
    o = oracle_subset(w, dh, eh, pos, ids, idx)
    np.testing.assert_array_equal(rec["n"][idx], o["npix"])
    np.testing.assert_array_equal(rec["j_lo"][idx], o["j_lo"])
    off = g["offsets"].cpu().numpy()
    for k, q in enumerate(idx):
        a, b = off[q], off[q + 1]
        assert_field_close(g["delta"][a:b].cpu().numpy(), ragged(o["delta"], o["offsets"], k), f"delta q{q}")
        assert_field_close(g["eta"][a:b].cpu().numpy(), ragged(o["eta"], o["offsets"], k), f"eta q{q}")
        assert_flux_close(g["flux"][a:b].cpu().numpy(), ragged(o["flux"], o["offsets"], k), f"flux q{q}")
    # whole-catalogue statistics: the fused pass equals the split pass over the
    # stored fields, and the mean flux per z bin equals an FP64 reduction of
    # the stored flux binned with the oracle's pixel redshifts
    tot = int(off[-1])
    st2 = ctx.stats(w, g["sk"], len(ids), g["offsets"], g["flux"], delta=g["delta"], eta=g["eta"])
    np.testing.assert_array_equal(st2["sums"][:, 0], st["sums"][:, 0])
    # both passes add FP32 partial sums with compensation in different orders:
    # agreement to 1e-8 of the pixel count (pixel values are O(1)) or 1e-6 relative
    assert np.all(np.abs(st2["sums"] - st["sums"]) <= 1e-6 * np.abs(st["sums"]) + 1e-8 * st["sums"][:, :1])
    np.testing.assert_allclose(st2["p1d_sum"], st["p1d_sum"], rtol=1e-6)
    jl = torch.from_numpy(rec["j_lo"].astype(np.int64)).cuda()
    nn = torch.from_numpy(rec["n"].astype(np.int64)).cuda()
    owner = torch.repeat_interleave(torch.arange(len(ids), device="cuda"), nn)
    J = jl[owner] + (torch.arange(tot, device="cuda") - g["offsets"][:-1][owner])
    jmax = int(J.max().item()) + 1
    jmin = int(J.min().item())
    zt = np.zeros(jmax)
    for j in range(jmin, jmax):
        zt[j] = oracle.pixel_z(w, j)
    zb = torch.floor((torch.from_numpy(zt).cuda()[J] - w["z_bin_lo"]) / w["dz_bin"]).long()
    ok = (zb >= 0) & (zb < w["n_zbins"])
    fsum = torch.zeros(w["n_zbins"], dtype=torch.float64, device="cuda")
    cnt = torch.zeros(w["n_zbins"], dtype=torch.float64, device="cuda")
    fsum.index_add_(0, zb[ok], g["flux"][:tot][ok].double())
    cnt.index_add_(0, zb[ok], torch.ones_like(fsum[zb[ok]]))
    np.testing.assert_array_equal(cnt.cpu().numpy(), st["sums"][:, 0])
    m = cnt.cpu().numpy() > 0
    np.testing.assert_allclose(st["mean_flux"][m], (fsum / cnt).cpu().numpy()[m], rtol=TOL_STAT)
    # every statistic of the sampled skewers against the oracle: (1) the
    # statistics pass over the sampled skewers' stored fields and flux,
    # gathered into compact arrays; (2) the fused pass over the sampled
    # quasars on the full-size box, in one CTA, so that each team carries its
    # pixel sums across many segments and z bins
    so = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    assert so["n_seg"].sum() > 0
    sel = torch.cat([torch.arange(int(off[q]), int(off[q + 1]), device="cuda") for q in idx])
    rc = rec[idx].copy()
    rc["offset"] = o["offsets"][:-1]
    sk_c = torch.from_numpy(rc.view(np.uint8).reshape(-1).copy()).cuda()
    off_c = torch.from_numpy(o["offsets"].astype(np.int64)).cuda()
    st_c = ctx.stats(w, sk_c, len(idx), off_c, g["flux"][sel].contiguous(), delta=g["delta"][sel].contiguous(),
                     eta=g["eta"][sel].contiguous())
    assert_stats_close(st_c, so)
    ctx.set_grid_cap(1)
    try:
        st_f, _ = ctx.run(box, mk.catalogue_tensor(pos[idx], ids[idx]), len(idx), w, flags=mk.STATS)
    finally:
        ctx.set_grid_cap(0)
    assert_stats_close(st_f, so)
    del g, box
    torch.cuda.empty_cache()


def test_scale_workload_sampled(ctx):
    _full_size_check(ctx, si.workload("scale"), 24, 5, lognormal=True)


def test_batched_workload_sampled(ctx):
    _full_size_check(ctx, si.workload("batched"), 40, 6)


def test_batched_workload_sampled_z_dependent_p_s(ctx):
    # the P_S node tables at the 12 bin centres (the instance the Sec. 2.6
    # tuning runs), full size, sampled skewers against the oracle
    w = si.workload("batched")
    zs = [w["z_bin_lo"] + (i + 0.5) * w["dz_bin"] for i in range(w["n_zbins"])]
    ps = np.stack([np.asarray(w["p_s"]) * (1.0 + 0.3 * (z - 2.6)) for z in zs])
    _full_size_check(ctx, si.shrink(w, p_s=ps, p_s_z=zs), 16, 9)


def test_scale_workload_sampled_tensor(ctx):
    w = si.shrink(si.workload("scale"), eta_mode=1)
    torch.cuda.empty_cache()
    d, e6 = si.gaussian_box_tensor(w["n"], w["cell"], w["seed_box"], backend="torch")
    dh, eh = d.cpu().numpy(), e6.cpu().numpy()
    pos, ids = si.catalogue(w, delta=dh)
    box = ctx.load_box(w, ctx.pack_box_tensor(d, e6), None, layout=mk.BOX_TENSOR)
    del d, e6
    torch.cuda.empty_cache()
    st, g = ctx.run(box, mk.catalogue_tensor(pos, ids), len(ids), w,
                    flags=mk.STATS | mk.STORE_FLUX | mk.STORE_FIELDS)
    rec = records(g["sk"], len(ids))
    idx = np.sort(np.random.default_rng(8).choice(len(ids), 16, replace=False))
    o = oracle_subset(w, dh, eh, pos, ids, idx)
    np.testing.assert_array_equal(rec["n"][idx], o["npix"])
    off = g["offsets"].cpu().numpy()
    for k, q in enumerate(idx):
        a, b = off[q], off[q + 1]
        assert_field_close(g["eta"][a:b].cpu().numpy(), ragged(o["eta"], o["offsets"], k), f"eta_par q{q}")
        assert_flux_close(g["flux"][a:b].cpu().numpy(), ragged(o["flux"], o["offsets"], k), f"flux q{q}")
    del g, box
    torch.cuda.empty_cache()


def test_batched_workload_sampled_gauss7(ctx):
    w = si.shrink(si.workload("batched"), interp=mk.INTERP_GAUSS7)
    _full_size_check(ctx, w, 24, 7, layout="halo")
