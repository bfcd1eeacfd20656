"""The Sec. 2.6 tuning of a, b sigma_g and P_S in the library (mk_tune_ps) against
the same procedure on the oracle (oracle/ps_tuning.py), on the 64^3 workload.

The target is the oracle's statistics of the catalogue synthesised at hidden
parameters: seeded b*(z), c*(z), a*(z) = 0.25 ((1+z)/3)^3.5 and a seeded
P_S*(k, z) of the same form as the benchmark's.
"""
import ctypes as C
import math

import numpy as np
import pytest

import oracle
import skewer_inputs as si
from oracle import ps_tuning
from tests.parity_util import box_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2310_18996_gb300 as mk  # noqa: E402

NTHREADS = 16


@pytest.fixture(scope="module")
def ctx():
    c = mk.Context(0)
    yield c
    c.close()


def _hidden(w, seed):
    """Seeded hidden parameters at the bin centres: power laws b*, c*, a fixed
    a*(z) and P_S*(k, z) = P_S(k) (1 + A (z - 2.6)) (k / k_8)^t."""
    rng = np.random.default_rng(seed)
    b0, bb, c0, bc, amp, tilt = (rng.uniform(lo, hi) for lo, hi in
                                 ((1.3, 1.9), (-0.5, 0.5), (0.7, 1.3), (-0.5, 0.5), (-0.4, 0.4), (-0.3, 0.3)))
    zs = [w["z_bin_lo"] + (i + 0.5) * w["dz_bin"] for i in range(w["n_zbins"])]
    b = [b0 * ((1 + z) / 3.3) ** bb for z in zs]
    c = [c0 * ((1 + z) / 3.3) ** bc for z in zs]
    la = [math.log(0.25 * ((1 + z) / 3.0) ** 3.5) for z in zs]
    n = w["n_fft"]
    m = np.arange(n // 2 + 1, dtype=np.float64)
    shape = np.where(m > 0, (np.maximum(m, 1.0) / (n // 8)) ** tilt, 1.0)
    ps = np.stack([np.asarray(w["p_s"]) * shape * (1.0 + amp * (z - 2.6)) for z in zs])
    return zs, la, b, c, ps


def _start(w):
    return np.tile(np.asarray(w["p_s"], dtype=np.float64), (w["n_zbins"], 1))


def _target_from_oracle(w, d, e, pos, ids, seed):
    zs, la, b, c, ps = _hidden(w, seed)
    ws = dict(w, p_s=ps, p_s_z=zs, node_ln_a=la, node_b=b, node_c=c)
    o = oracle.run_skewers(ws, d, e, pos, ids, n_threads=NTHREADS)
    st = oracle.stats(ws, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    t = mk.TuneTarget()
    active = 0
    for i in range(w["n_zbins"]):
        if st["n_seg"][i] >= 20:
            active |= 1 << i
        t.mean_flux[i] = st["mean_flux"][i]
        t.beta[i] = st["beta_f"][i]
        for k in range(w["n_kbins"]):
            t.p1d[i][k] = st["p1d_df"][i][k]
    t.use_beta, t.k_lo, t.k_hi, t.active = 1, 0, w["n_kbins"], active
    t.tol_mean_flux, t.tol_p1d, t.tol_beta = 1e-3, 0.02, 0.02
    odict = dict(mean_flux=st["mean_flux"], p1d=st["p1d_df"], beta=st["beta_f"],
                 active=[bool((active >> i) & 1) for i in range(w["n_zbins"])])
    return t, odict


@pytest.fixture(scope="module")
def case():
    w = si.workload("tiny")
    d, e = box_numpy(w)
    pos, ids = si.catalogue(w)
    pos, ids = pos[:250], ids[:250]
    t, odict = _target_from_oracle(w, d, e, pos, ids, seed=7)
    dev = dict(d=torch.from_numpy(d).cuda(), e=torch.from_numpy(e).cuda(), qso=mk.catalogue_tensor(pos, ids))
    return dict(w=w, d=d, e=e, pos=pos, ids=ids, t=t, odict=odict, dev=dev)


def test_tune_ps_matches_oracle_procedure(ctx, case):
    w, dv = case["w"], case["dev"]
    box = ctx.load_box(w, dv["d"], dv["e"])
    p0 = _start(w)
    nd, ps, rep = mk.tune_ps(ctx, box, dv["qso"], len(case["ids"]), w, case["t"], p0, n_outer=1, n_inner=2)
    ref = ps_tuning.tune_ps(w, case["d"], case["e"], case["pos"], case["ids"], case["odict"], p0,
                            n_outer=1, n_inner=2, n_threads=NTHREADS)
    assert rep.passes == ref["passes"] == 4
    nz = w["n_zbins"]
    act = np.array(case["odict"]["active"])
    assert act.sum() >= 5
    # fit of (a, b sigma_g) and c from beta: host arithmetic on the same target
    np.testing.assert_allclose(np.exp([nd.ln_a[i] for i in range(nz)]), ref["a"], rtol=1e-8)
    np.testing.assert_allclose([rep.bsigma[i] for i in range(nz)], ref["s"], rtol=1e-8)
    np.testing.assert_allclose([nd.c[i] for i in range(nz)], ref["c"], rtol=1e-12)
    # b from sigma_g of the synthesised pixels (fields within 2e-6 of the oracle)
    np.testing.assert_allclose([nd.b[i] for i in range(nz)], ref["b"], rtol=2e-5)
    # two ratio updates from P1D within 1e-4 of the oracle's
    np.testing.assert_allclose(ps, ref["p_s"], rtol=2e-3)
    # untuned nodes copy the nearest tuned node
    src = ps_tuning._follow(act)
    for i in range(nz):
        np.testing.assert_array_equal(ps[i], ps[src[i]])
    # the last pass
    o = ref["stats"]
    m = act
    g_p1d_err = rep.max_rel_p1d
    o_p1d_err = np.max(np.abs(o["p1d_df"][m] / case["odict"]["p1d"][m] - 1))
    assert abs(g_p1d_err - o_p1d_err) < 2e-3
    assert abs(rep.max_abs_dfbar - np.max(np.abs(o["mean_flux"][m] - case["odict"]["mean_flux"][m]))) < 2e-4


def test_tune_ps_reduces_p1d_error_and_oracle_agrees(ctx, case):
    w, dv = case["w"], case["dev"]
    box = ctx.load_box(w, dv["d"], dv["e"])
    p0 = _start(w)
    nd, ps, rep = mk.tune_ps(ctx, box, dv["qso"], len(case["ids"]), w, case["t"], p0, n_outer=2, n_inner=5)
    hist = np.array(rep.max_rel_p1d_pass[: rep.passes])
    assert rep.passes == 2 * 6 + 1
    # the ratio iteration lowers the P1D error well below the start's
    assert hist[-1] < 0.5 * hist[0]
    # the oracle at the tuned parameters sees the same errors the library reports
    nz = w["n_zbins"]
    ws = dict(w, p_s=ps, p_s_z=[nd.z[i] for i in range(nz)], node_ln_a=[nd.ln_a[i] for i in range(nz)],
              node_b=[nd.b[i] for i in range(nz)], node_c=[nd.c[i] for i in range(nz)])
    o = oracle.run_skewers(ws, case["d"], case["e"], case["pos"], case["ids"], n_threads=NTHREADS)
    st = oracle.stats(ws, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    m = np.array(case["odict"]["active"])
    err = np.max(np.abs(st["p1d_df"][m] / case["odict"]["p1d"][m] - 1))
    assert abs(err - rep.max_rel_p1d) < 2e-3
    dfb = np.max(np.abs(st["mean_flux"][m] - case["odict"]["mean_flux"][m]))
    assert abs(dfb - rep.max_abs_dfbar) < 2e-4


def test_tune_ps_rejects_bad_arguments(ctx, case):
    w, dv = case["w"], case["dev"]
    box = ctx.load_box(w, dv["d"], dv["e"])
    p0 = _start(w)
    n = len(case["ids"])
    t = mk.TuneTarget()
    C.pointer(t)[0] = case["t"]
    t.use_beta = 0
    with pytest.raises(mk.MkError):
        mk.tune_ps(ctx, box, dv["qso"], n, w, t, p0, n_outer=1, n_inner=1)
    with pytest.raises(mk.MkError):
        mk.tune_ps(ctx, box, dv["qso"], n, w, case["t"], p0, n_outer=0, n_inner=1)
    with pytest.raises(mk.MkError):
        mk.tune_ps(ctx, box, dv["qso"], n, w, case["t"], p0, n_outer=12, n_inner=10)  # > 128 passes
    C.pointer(t)[0] = case["t"]
    for k in range(w["n_kbins"]):  # sigma_F above sqrt(F (1 - F)) in the first active bin
        t.p1d[case["odict"]["active"].index(True)][k] = 1e3
    with pytest.raises(mk.MkError):
        mk.tune_ps(ctx, box, dv["qso"], n, w, t, p0, n_outer=1, n_inner=1)
