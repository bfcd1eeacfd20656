"""Gaussian box synthesis on the GPU (mk_synth_box) against the oracle
(oracle/box_synth.py): every voxel at 128^3 and 256^3, every layout, and at
512^3 and 1024^3 the properties that hold at any size (mode-space relations
and the shell power), checked with torch FFTs on the device."""
import math

import numpy as np
import pytest

from oracle import box_synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2310_18996_gb300 as mk  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = mk.Context(0)
    yield c
    c.close()


def table(cell, n_tab=2000):
    # smooth power law with a cut-off, out beyond the corner of the k grid
    dk = 2.0 * math.pi * math.sqrt(3.0) / cell / (n_tab - 10)
    k = dk * np.arange(n_tab)
    return dk, np.where(k > 0, 40.0 * k ** 0.96 * np.exp(-(k / 1.5) ** 2) * (1.0 + 0.05 * np.sin(15.0 * k)), 0.0)


U32 = 2.0 ** -24  # unit roundoff of FP32


def fft_error_bound(n):
    """Worst-case relative error, in the 2-norm over the n^3 voxels, of an
    FP32 box made by one forward and one inverse 3D FFT (Higham, Accuracy and
    Stability of Numerical Algorithms, 2nd ed., Thm. 24.2: a radix-2 FFT of
    length 2^t has ||err|| / ||y|| <= t eta / (1 - t eta), eta = mu + g4 (sqrt 2
    + mu), g4 = 4u / (1 - 4u), mu the twiddle error; twiddles are FP64 values
    rounded to FP32, mu = u).  Both 3D transforms together take
    t = 2 * 3 * log2 n radix-2-equivalent stages; the filter adds one rounding."""
    t = 2 * 3 * int(round(math.log2(n)))
    g4 = 4 * U32 / (1 - 4 * U32)
    eta = U32 + g4 * (math.sqrt(2.0) + U32)
    return t * eta / (1 - t * eta) + U32


def close(gpu, ref, what, rel=2e-5):
    """Every voxel within rel x RMS of the oracle's box, and the RMS error
    within the worst-case FFT bound.  rel: the rounding errors of the FFT
    stages act as independent noise of RMS ~ u sqrt(t) per voxel (t stages),
    so the largest of n^3 voxel errors is ~ sqrt(2 ln n^3) ~ 6 times that,
    ~2.4e-6 x RMS at n = 256; 2e-5 leaves a factor 8 for the constant."""
    gpu = np.asarray(gpu, dtype=np.float64)
    n = round(ref.size ** (1.0 / 3.0))
    rms = math.sqrt(np.mean(ref ** 2))
    err = np.abs(gpu - ref)
    assert err.max() <= rel * rms, f"{what}: max error {err.max():.3e} > {rel:.0e} x RMS {rms:.3e}"
    rms_err = math.sqrt(np.mean(err ** 2))
    bound = fft_error_bound(n)
    assert rms_err <= bound * rms, f"{what}: RMS error {rms_err / rms:.3e} x RMS > bound {bound:.3e}"


def pairs(out, n):
    return out.view(n, n, n, 2).cpu().numpy()


@pytest.mark.parametrize("n,cell,seed", [(128, 2.0, 5), (256, 1.0, 0x1234_5678_9ABC)])
def test_interleaved_box_matches_oracle(ctx, n, cell, seed):
    dk, tab = table(cell)
    out = ctx.synth_box(n, cell, seed, tab, dk, layout=mk.BOX_INTERLEAVED)
    torch.cuda.synchronize()
    g = pairs(out, n)
    d, e = box_synth.synth_box(n, cell, seed, dk, tab)
    close(g[..., 0], d, "delta")
    close(g[..., 1], e, "eta_xx")


def test_padded_and_halo_layouts_repeat_the_box(ctx):
    n, cell, seed = 128, 2.0, 9
    dk, tab = table(cell)
    g = pairs(ctx.synth_box(n, cell, seed, tab, dk, layout=mk.BOX_INTERLEAVED), n)
    p = ctx.synth_box(n, cell, seed, tab, dk, layout=mk.BOX_PADDED).view(n + 1, n + 1, n + 1, 2).cpu().numpy()
    idx = np.arange(n + 1) % n
    np.testing.assert_array_equal(p, g[np.ix_(idx, idx, idx)])
    h = ctx.synth_box(n, cell, seed, tab, dk, layout=mk.BOX_HALO).view(n + 6, n + 6, n + 6, 2).cpu().numpy()
    idx = (np.arange(n + 6) - 3) % n
    np.testing.assert_array_equal(h, g[np.ix_(idx, idx, idx)])
    d = ctx.synth_box(n, cell, seed, tab, dk, layout=mk.BOX_PLANAR).view(n, n, n).cpu().numpy()
    np.testing.assert_array_equal(d, g[..., 0])


def test_tensor_box_matches_oracle(ctx):
    n, cell, seed = 128, 1.5, 21
    dk, tab = table(cell)
    t = ctx.synth_box(n, cell, seed, tab, dk, layout=mk.BOX_TENSOR).view(n + 1, n + 1, n + 1, 8).cpu().numpy()
    d, eta = box_synth.synth_box(n, cell, seed, dk, tab, tensor=True)
    close(t[:n, :n, :n, 0], d, "delta")
    for c in range(6):
        close(t[:n, :n, :n, 1 + c], eta[c], f"eta {box_synth.PAIRS[c]}")
    assert np.all(t[..., 7] == 0.0)
    idx = np.arange(n + 1) % n
    np.testing.assert_array_equal(t, t[np.ix_(idx, idx, idx)])
    # the first record slots are the interleaved pair of the same seed
    g = pairs(ctx.synth_box(n, cell, seed, tab, dk, layout=mk.BOX_INTERLEAVED), n)
    np.testing.assert_array_equal(t[:n, :n, :n, :2], g)


@pytest.mark.parametrize("n", [512, 1024])
def test_large_box_mode_relations_and_power(ctx, n):
    cell = 1.0
    dk, tab = table(cell)
    out = ctx.synth_box(n, cell, 77, tab, dk, layout=mk.BOX_INTERLEAVED)
    v = out.view(n, n, n, 2)
    D = torch.fft.fftn(v[..., 0].contiguous())
    E = torch.fft.fftn(v[..., 1].contiguous())
    del out, v
    k1 = 2.0 * math.pi * torch.fft.fftfreq(n, d=cell, device=D.device)
    kx, ky, kz = k1[None, None, :], k1[None, :, None], k1[:, None, None]
    k2 = kx * kx + ky * ky + kz * kz
    # eta_xx modes = -(k_x^2 / k^2) delta modes
    mu2 = torch.where(k2 > 0, kx * kx / torch.where(k2 > 0, k2, 1.0), torch.zeros_like(k2))
    rms = torch.sqrt(torch.mean(D.abs() ** 2)).item()
    assert (E + mu2 * D).abs().max().item() < 1e-4 * rms
    del E, mu2
    # zero mode and Nyquist planes are empty
    h = n // 2
    assert D[0, 0, 0].abs().item() < 1e-4 * rms
    for plane in (D[h], D[:, h], D[:, :, h]):
        assert plane.abs().max().item() < 1e-4 * rms
    # shell power |D|^2 cell^3 / n^3 averages to P(k) (5 sigma in each shell)
    kk = torch.sqrt(k2)
    del k2
    for lo, hi in ((0.05, 0.1), (0.3, 0.35), (1.0, 1.02), (2.0, 2.01)):
        m = (kk >= lo) & (kk < hi)
        ks = kk[m].double().cpu().numpy()
        pw = (D[m].abs().double() ** 2 * cell ** 3 / n ** 3).cpu().numpy()
        ratio = np.mean(pw / np.interp(ks, dk * np.arange(tab.size), tab))
        assert abs(ratio - 1) < 5 / math.sqrt(ks.size), (lo, ratio, ks.size)


def test_bad_arguments(ctx):
    dk, tab = table(1.0)
    for n in (64, 100):
        with pytest.raises(mk.MkError):
            ctx.synth_box(n, 1.0, 1, tab, dk, layout=mk.BOX_INTERLEAVED)
    with pytest.raises(mk.MkError):
        ctx.synth_box(128, -1.0, 1, tab, dk, layout=mk.BOX_INTERLEAVED)
    with pytest.raises(mk.MkError):
        ctx.synth_box(128, 1.0, 1, -tab - 1.0, dk, layout=mk.BOX_INTERLEAVED)
    w = torch.empty(2 * 129 ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(mk.MkError):  # padded output on top of its own scratch
        ctx._check(mk.lib().mk_synth_box(ctx.h, 128, 1.0, 1, mk._dp(tab), tab.size, dk, mk.BOX_PADDED,
                                         mk._ptr(w), None, mk._ptr(w)))
    t = torch.empty(8 * 129 ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(mk.MkError):  # tensor output without the mode buffer
        ctx._check(mk.lib().mk_synth_box(ctx.h, 128, 1.0, 1, mk._dp(tab), tab.size, dk, mk.BOX_TENSOR,
                                         mk._ptr(w), None, mk._ptr(t)))


def test_box_2048_in_core_moments(ctx):
    # 2048^3 (68.7 GB of pairs, in place): the sample moments of delta and
    # eta_xx match the ensemble expectations of the realised discrete spectrum,
    #   <delta^2> = sum_k P / V,  <eta_xx^2> = sum_k mu^4 P / V,  <delta eta_xx> = -sum_k mu^2 P / V,
    # summed over the kept modes (no zero mode, no Nyquist planes), V = (n cell)^3
    n, cell = 2048, 2.0
    if torch.cuda.mem_get_info()[0] < 80e9:
        pytest.skip("needs 80 GB of free device memory")
    dk, tab = table(cell)
    out = ctx.synth_box(n, cell, 2048, tab, dk, layout=mk.BOX_INTERLEAVED)
    v = out.view(n, n * n, 2)
    s = torch.zeros(3, dtype=torch.float64, device=out.device)
    for z in range(0, n, 64):
        blk = v[z:z + 64].double()
        d, e = blk[..., 0], blk[..., 1]
        s += torch.stack([(d * d).sum(), (e * e).sum(), (d * e).sum()])
    s = (s / float(n) ** 3).cpu().numpy()
    del out, v
    torch.cuda.empty_cache()
    k1 = 2.0 * math.pi * torch.fft.fftfreq(n, d=cell, device="cuda", dtype=torch.float64)
    keep = torch.ones(n, dtype=torch.bool, device="cuda")
    keep[n // 2] = False
    kx, ky = k1[None, :], k1[:, None]
    ptab = torch.from_numpy(tab).cuda()
    e = torch.zeros(3, dtype=torch.float64, device="cuda")
    for iz in range(n):
        if iz == n // 2:
            continue
        kz = k1[iz]
        k2 = kx * kx + ky * ky + kz * kz
        u = torch.sqrt(k2) / dk
        j = torch.clamp(u.floor().long(), max=tab.size - 2)
        p = ptab[j] + (u - j) * (ptab[j + 1] - ptab[j])
        m = keep[None, :] & keep[:, None] & (k2 > 0)
        mu2 = torch.where(k2 > 0, kx * kx / torch.where(k2 > 0, k2, 1.0), torch.zeros_like(k2))
        p = torch.where(m, p, torch.zeros_like(p))
        e += torch.stack([p.sum(), (mu2 * mu2 * p).sum(), -(mu2 * p).sum()])
    e = (e / (n * cell) ** 3).cpu().numpy()
    np.testing.assert_allclose(s, e, rtol=2e-3)
