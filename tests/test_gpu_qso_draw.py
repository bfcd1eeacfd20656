"""Quasars from lognormal quasar-density boxes (mk_draw_qso, Sec. 2.2 and
App. A) against the oracle's voxel loop, on seeded Gaussian boxes and on the
whole chain: P_q tables (mk_lognormal_pk), three boxes from one white noise
(mk_synth_box) and the draw.

A voxel's decision is u0 < P; the library takes it in FP32 with coefficients
interpolated from an r table, the oracle in FP64.  Decisions may differ only
where u0 lies within a small relative distance of P: the catalogues agree
everywhere else, voxel by voxel."""
import math

import numpy as np
import pytest

import oracle
from oracle import box_synth, lognormal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2310_18996_gb300 as mk  # noqa: E402

OM = 0.3147


@pytest.fixture(scope="module")
def ctx():
    c = mk.Context(0)
    yield c
    c.close()


def params(n, cell, seed, xi_m5=0.6, nbar=2e-3):
    return dict(n=n, cell=cell, origin=(4300.0 - n * cell / 2, -n * cell / 2, -n * cell / 2), z_box=(1.9, 2.75, 3.6),
                bias=(3.7, 2.33, 1.7), xi_m5=xi_m5, nbar=[nbar * (1 + 0.1 * j) for j in range(12)], nbar_z0=1.5,
                nbar_dz=0.25, seed=seed, omega_m=OM)


def records(cat):
    a = cat.cpu().numpy().view(mk.QSO_DTYPE)
    return a["id"].astype(np.int64), a["pos"]


def compare(ids, pos, ref, rel):
    P, u = ref["P"], ref["u"]
    border = np.abs(u - P) <= rel * np.maximum(P, 1e-12)
    a, b = set(ids.tolist()), set(ref["ids"].astype(np.int64).tolist())
    diff = np.array(sorted(a ^ b), dtype=np.int64)
    assert np.all(border[diff]), f"{diff.size} decisions differ, {np.count_nonzero(~border[diff])} away from u0 = P"
    common = np.array(sorted(a & b), dtype=np.int64)
    gi = {v: i for i, v in enumerate(ids.tolist())}
    oi = {v: i for i, v in enumerate(ref["ids"].astype(np.int64).tolist())}
    gp = pos[[gi[v] for v in common]]
    op = ref["pos"][[oi[v] for v in common]]
    np.testing.assert_allclose(gp, op, rtol=0, atol=1e-9)
    assert np.all(np.diff(ids) > 0)
    return diff.size


def test_draw_matches_oracle_on_gaussian_boxes(ctx):
    n, cell = 64, 2.19
    q = params(n, cell, seed=0x5EED_0001)
    rng = np.random.default_rng(4)
    boxes = [(rng.standard_normal((n, n, n)) * s).astype(np.float32) for s in (0.8, 0.6, 0.5)]
    cat, cnt = ctx.draw_qso(q, [torch.from_numpy(b).cuda() for b in boxes], stride=1)
    ids, pos = records(cat)
    ref = oracle.qso_draw(q, boxes)
    assert cnt == ids.size and ref["count"] > 1000
    nd = compare(ids, pos, ref, rel=1e-5)
    assert nd <= 3 and abs(cnt - ref["count"]) <= nd


def test_draw_chain_from_one_white_noise(ctx):
    # P_m -> P_q,i (B_i = b_q^2(z_i) G^2(z_i)) -> three delta_q boxes of one seed -> draw
    n, cell, seed = 128, 2.19, 91
    dk = 2 * math.pi * math.sqrt(3) / cell / 1990
    k = dk * np.arange(2000)
    pm = np.where(k > 0, 30.0 * k ** 0.96 * np.exp(-(k / 1.5) ** 2), 0.0)
    q = params(n, cell, seed=0x5EED_0002, xi_m5=float(lognormal.xi_of_pk(pm, dk, 5.0)[0]))
    B = [(3.7 * ((1 + z) / 3.33) ** 1.7) ** 2 * oracle.growth(OM, z) ** 2 for z in q["z_box"]]
    g_boxes, o_boxes = [], []
    for Bi in B:
        pq = mk.lognormal_pk(pm, dk, Bi)
        g_boxes.append(ctx.synth_box(n, cell, seed, pq, dk, layout=mk.BOX_INTERLEAVED))
        d, _ = box_synth.synth_box(n, cell, seed, dk, lognormal.lognormal_pk(pm, dk, Bi))
        o_boxes.append(d.astype(np.float32))
    cat, cnt = ctx.draw_qso(q, g_boxes, stride=2)
    ids, pos = records(cat)
    ref = oracle.qso_draw(q, o_boxes)
    assert ref["count"] > 5000
    nd = compare(ids, pos, ref, rel=2e-4)
    assert nd <= 20


def test_capacity_overflow_reports_count(ctx):
    n, cell = 32, 2.19
    q = params(n, cell, seed=3)
    z = torch.zeros(n ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(mk.MkError) as ei:
        ctx.draw_qso(q, [z, z, z], stride=1, capacity=5)
    assert ei.value.code == mk.MK_ERANGE
    cat, cnt = ctx.draw_qso(q, [z, z, z], stride=1)
    ref = oracle.qso_draw(q, [np.zeros((n, n, n), np.float32)] * 3)
    assert cnt == ref["count"]  # uniform P: no decision near its threshold in practice


def test_large_box_counts_follow_the_mean_density(ctx):
    # 512^3 of Gaussian boxes: the count per z slab follows nbar(z) V within Poisson noise
    n, cell = 512, 2.19
    q = params(n, cell, seed=17, nbar=1e-4)
    gen = torch.Generator(device="cuda").manual_seed(5)
    boxes = [torch.randn(n ** 3, generator=gen, device="cuda") * 0.5 for _ in range(3)]
    cat, cnt = ctx.draw_qso(q, boxes, stride=1)
    ids, pos = records(cat)
    r = np.linalg.norm(pos, axis=1)
    assert cnt > 100000
    # expected count: sum over voxels of nbar(z(r)) cell^3 (E[p] / E[p] = 1), from the voxel centres
    x = (np.arange(n) + 0.5) * cell
    cz = q["origin"][2] + x
    cy = q["origin"][1] + x
    cx = q["origin"][0] + x
    rr = np.sqrt(cx[None, None, :] ** 2 + cy[None, :, None] ** 2 + cz[:, None, None] ** 2).ravel()
    rs = np.linspace(rr.min(), rr.max(), 400)
    zs = np.array([oracle.z_of_distance(OM, v) for v in rs])
    zv = np.interp(rr, rs, zs)
    nb = np.interp(zv, q["nbar_z0"] + q["nbar_dz"] * np.arange(len(q["nbar"])), q["nbar"])
    expect = nb.sum() * cell ** 3
    assert abs(cnt - expect) < 5 * math.sqrt(expect) + 1e-3 * expect


def test_cosmo_eval_matches_oracle(ctx):
    for z in (0.0, 1.9, 2.75, 3.6, 6.0):
        dc, g = ctx.cosmo_eval(z)
        assert abs(dc - oracle.comoving_distance(OM, z)) <= 1e-9 * max(dc, 1.0)
        assert abs(g / oracle.growth(OM, z) - 1) < 1e-9
    with pytest.raises(mk.MkError):
        ctx.cosmo_eval(-0.5)
