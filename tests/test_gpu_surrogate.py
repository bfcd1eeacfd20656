"""Surrogate MLP kernels against the FP64 oracle, and tuning of a, b, c.

The MLP gradients of the GPU (BF16 weights, FP32 activations and
accumulation) are compared with the oracle's FP64 gradients evaluated at the
same BF16-rounded weights.  Tuning: both methods must reach a reachable
seeded target on stored skewers, and the tuned parameters are re-checked by
the oracle pipeline.
"""
import math

import numpy as np
import pytest

import oracle
import skewer_inputs as si
from tests.parity_util import box_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2310_18996_gb300 as mk  # noqa: E402
from paper_2310_18996_gb300 import tuning  # noqa: E402

DIMS = (4, 128, 128, 128, 35)


def weight_mask():
    m = np.zeros(mk.MLP_NPARAM, bool)
    o = 0
    for l in range(4):
        nw = DIMS[l + 1] * DIMS[l]
        m[o:o + nw] = True
        o += nw + DIMS[l + 1]
    return m


def effective_params(master, bf16):
    """The values the kernels use: BF16 weights, FP32 biases, as FP64."""
    w = (bf16.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return np.where(weight_mask(), w, master.astype(np.float64))


@pytest.fixture(scope="module")
def ctx():
    c = mk.Context(0)
    yield c
    c.close()


def test_mlp_forward_and_gradient_match_oracle(ctx):
    """Tensor-core inference and training gradients against the oracle at the
    same BF16 weights.  Inference takes each hidden activation as two BF16
    terms (~16 bits), so it matches the plain FP64 forward to 1e-4; the
    gradient follows the training precision (one BF16 term per activation
    and backward operand) and is compared with the oracle's BF16 path."""
    rng = np.random.default_rng(11)
    mlp = mk.Mlp(ctx, max_batch=512, seed=3)
    p = (rng.standard_normal(mk.MLP_NPARAM) * 0.15).astype(np.float32)
    mlp.set_params(p)
    master, b16 = mlp.get_params()
    np.testing.assert_array_equal(master, p)
    eff = effective_params(master, b16)
    assert np.max(np.abs(eff - p)[weight_mask()] / np.maximum(np.abs(p[weight_mask()]), 1e-30)) <= 2.0 ** -8
    n = 300  # two passes of the 256-sample cluster, the second ragged
    x = rng.standard_normal((n, 4)).astype(np.float32)
    t = rng.standard_normal((n, 35)).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = mlp.forward(xd).cpu().numpy()
    yo = oracle.mlp_forward(eff, x.astype(np.float64))
    scale = np.abs(yo).max()
    np.testing.assert_allclose(y, yo, rtol=1e-4, atol=1e-5 * scale)
    # one BF16 term per activation would be ~100x further off
    yq = oracle.mlp_forward(eff, x.astype(np.float64), bf16=True)
    assert np.abs(y - yo).max() < 0.1 * np.abs(yq - yo).max()
    loss, g = mlp.loss_grad(xd, td)
    lo, go = oracle.mlp_loss_grad(eff, x.astype(np.float64), t.astype(np.float64), bf16=True)
    assert loss == pytest.approx(lo, rel=1e-5)
    # BF16 operands on both sides; FP32 against FP64 accumulation and the
    # occasional rounding flip: 1e-2 relative per entry, 1e-3 in norm
    big = np.abs(go) > 1e-2 * np.abs(go).max()
    np.testing.assert_allclose(g[big], go[big], rtol=1e-2)
    assert np.linalg.norm(g - go) <= 1e-3 * np.linalg.norm(go)
    # the same weights through the plain FP64 oracle: BF16 operands move the
    # gradient by far more than the kernels' own error
    _, g64 = oracle.mlp_loss_grad(eff, x.astype(np.float64), t.astype(np.float64))
    assert np.linalg.norm(g - go) < 0.5 * np.linalg.norm(g64 - go)
    mlp.close()


def test_mlp_adam_steps_match_oracle(ctx):
    """mk_mlp_adam_step on a seeded gradient, one and three steps, against the
    oracle's Adam (Kingma & Ba 2015, Algorithm 1) in FP64: FP32 master
    weights to 1e-6 relative, plus the FP32 rounding of each step: the
    update lr u (|u| = 1 for a repeated gradient) to a few ulp of lr, and
    the subtraction p - lr u to half an ulp of |p| + lr, which is relative to
    the operands, not the result; the BF16 copy is the master rounded."""
    rng = np.random.default_rng(21)
    p0 = (rng.standard_normal(mk.MLP_NPARAM) * 0.1).astype(np.float32)
    g = (rng.standard_normal(mk.MLP_NPARAM) * 10.0 ** rng.uniform(-9, 0, mk.MLP_NPARAM)).astype(np.float32)
    g[:50] = 0.0  # no gradient: the parameter stays
    gd = torch.from_numpy(g).cuda()
    mlp = mk.Mlp(ctx, max_batch=64, seed=1)
    mlp.set_params(p0)
    po, mo, vo = p0.astype(np.float64), np.zeros(mk.MLP_NPARAM), np.zeros(mk.MLP_NPARAM)
    lr = 3e-3
    for step in (1, 2, 3):
        mlp.adam_step(gd, lr)
        oracle.adam_step(po, mo, vo, g.astype(np.float64), step, lr)
        if step in (1, 3):
            master, b16 = mlp.get_params()
            bound = 1e-6 * np.abs(po) + step * 2.0 ** -24 * (np.abs(p0) + step * lr + 8 * lr)
            assert np.all(np.abs(master - po) <= bound), np.max(np.abs(master - po) / bound)
            assert np.array_equal(master[:50], p0[:50])
            want = torch.from_numpy(master).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
            np.testing.assert_array_equal(b16, want)
    mlp.close()


def test_mlp_training_step_is_gradient_then_adam(ctx):
    """One training step of the cluster kernel equals the gradient of
    mk_mlp_loss_grad followed by mk_mlp_adam_step (the same update), up to
    the order in which the step's shuffled samples are summed."""
    rng = np.random.default_rng(7)
    n = 200
    x = torch.from_numpy(rng.standard_normal((n, 4)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((n, 35)).astype(np.float32)).cuda()
    a = mk.Mlp(ctx, max_batch=256, seed=9)
    b = mk.Mlp(ctx, max_batch=256, seed=9)
    a.train(x, t, batch=n, epochs=1, lr=1e-3, seed=0)   # one step over every sample
    _, g = b.loss_grad(x, t)
    b.adam_step(torch.from_numpy(g).cuda(), 1e-3)
    pa, _ = a.get_params()
    pb, _ = b.get_params()
    p0, _ = mk.Mlp(ctx, max_batch=1, seed=9).get_params()
    assert np.abs(pa - p0).max() > 5e-4  # the step moved the weights by about lr
    np.testing.assert_allclose(pa, pb, rtol=1e-6, atol=1e-9)
    a.close()
    b.close()


def test_mlp_training_fits_a_smooth_map(ctx):
    rng = np.random.default_rng(12)
    n = 20000
    x = rng.uniform(-1.5, 1.5, (n, 4)).astype(np.float32)
    k = rng.standard_normal((4, 35)) * 0.8
    t = np.sin(x @ k).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    mlp = mk.Mlp(ctx, max_batch=1024, seed=5)
    l0, _ = mlp.loss_grad(xd[:1024], td[:1024])
    losses = mlp.train(xd, td, batch=512, epochs=30, lr=3e-3, seed=1)
    assert np.all(np.isfinite(losses))
    l1, _ = mlp.loss_grad(xd[:1024], td[:1024])
    assert l1 < 0.05 * l0, (l0, l1, losses[-3:])
    mlp.close()


@pytest.fixture(scope="module")
def stored(ctx):
    w = si.workload("tiny")
    d, e = box_numpy(w)
    pos, ids = si.catalogue(w)
    box = ctx.load_box(w, torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda())
    r = ctx.make_skewers(box, mk.catalogue_tensor(pos, ids), len(ids), w)
    return dict(w=w, d=d, e=e, pos=pos, ids=ids, r=r, box=box)


def _check_with_oracle(stored, nd, target):
    w = dict(stored["w"])
    w["node_z"] = [nd.z[i] for i in range(nd.count)]
    w["node_ln_a"] = [nd.ln_a[i] for i in range(nd.count)]
    w["node_b"] = [nd.b[i] for i in range(nd.count)]
    w["node_c"] = [nd.c[i] for i in range(nd.count)]
    o = oracle.run_skewers(w, stored["d"], stored["e"], stored["pos"], stored["ids"], n_threads=16)
    so = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    for i in range(w["n_zbins"]):
        if not (target.active >> i) & 1:
            continue
        assert abs(so["mean_flux"][i] - target.mean_flux[i]) <= 1.05 * target.tol_mean_flux
        rel = so["p1d_df"][i][target.k_lo:target.k_hi] / np.array(target.p1d[i][target.k_lo:target.k_hi]) - 1
        assert np.max(np.abs(rel)) <= 1.05 * target.tol_p1d


def test_plain_and_surrogate_tuning_reach_the_target(ctx, stored):
    # the surrogate (trained here on constant-parameter passes) must reach the
    # target in at most half the full passes of the plain method
    w, r = stored["w"], stored["r"]
    n = len(stored["ids"])
    target, hidden = tuning.make_target(ctx, w, r["sk"], n, r["offsets"], r["delta"], r["eta"], seed=5)
    assert bin(target.active).count("1") >= 6
    nd0 = tuning.start_nodes(w)
    nd_p, rep_p = mk.tune(ctx, w, r["sk"], n, r["offsets"], r["delta"], r["eta"], target, nd0,
                          method=mk.TUNE_PLAIN, max_passes=120)
    assert rep_p.converged, (rep_p.passes, rep_p.max_abs_dfbar, rep_p.max_rel_p1d, rep_p.max_rel_beta)
    _check_with_oracle(stored, nd_p, target)
    # surrogate trained on constant-parameter passes over the same stored skewers
    hx, ht = mk.surrogate_labels(ctx, w, r["sk"], n, r["offsets"], r["delta"], r["eta"], n_draws=2000, seed=9)
    assert hx.shape[0] > 10000
    mlp = mk.Mlp(ctx, max_batch=1024, seed=2)
    norm, losses = mlp.fit(hx, ht, batch=256, epochs=200, lr=2e-3, seed=4)
    assert losses[-1] < 1e-3 * losses[0]
    nd_s, rep_s = mk.tune(ctx, w, r["sk"], n, r["offsets"], r["delta"], r["eta"], target, nd0,
                          method=mk.TUNE_SURROGATE, mlp=mlp, norm=norm, max_passes=40)
    assert rep_s.converged, (rep_s.passes, rep_s.max_abs_dfbar, rep_s.max_rel_p1d, rep_s.max_rel_beta)
    assert 2 * rep_s.passes <= rep_p.passes, (rep_s.passes, rep_p.passes)
    assert rep_s.calib_passes == 0
    _check_with_oracle(stored, nd_s, target)
    # calibrated on a labelled subset: the first half of the skewers, relabelled
    hx2, ht2 = mk.surrogate_labels(ctx, w, r["sk"], n // 2, r["offsets"], r["delta"], r["eta"], n_draws=2000,
                                   seed=9)
    norm2, _ = mlp.fit(hx2, ht2, batch=256, epochs=200, lr=2e-3, seed=4)
    norm2.calib_skewers = n // 2
    nd_c, rep_c = mk.tune(ctx, w, r["sk"], n, r["offsets"], r["delta"], r["eta"], target, nd0,
                          method=mk.TUNE_SURROGATE, mlp=mlp, norm=norm2, max_passes=40)
    assert rep_c.converged and rep_c.calib_passes == 1, (rep_c.passes, rep_c.calib_passes)
    assert 2 * rep_c.passes <= rep_p.passes, (rep_c.passes, rep_p.passes)
    _check_with_oracle(stored, nd_c, target)
    mlp.close()
