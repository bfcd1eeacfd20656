"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against a closed form, a published value, an
independent library routine, or a brute-force/statistical property, so that
a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.  No GPU is used.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats as sst
from scipy.optimize import brentq
from scipy.special import hyp2f1, roots_hermitenorm

import oracle
import skewer_inputs as si
from oracle import targets

OM = 0.3147
CH = 2997.92458
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NTHREADS = max(1, min(8, os.cpu_count() or 1))


# ------------------------------------------------------------ independent cosmology
def dc_closed(om, z):
    """D_C for flat LCDM via int_0^X (1 + c x^3)^-1/2 dx = X 2F1(1/2,1/3;4/3;-c X^3)."""
    ol = 1.0 - om
    c = om / ol
    F = lambda x: x * hyp2f1(0.5, 1.0 / 3.0, 4.0 / 3.0, -c * x ** 3)
    return CH / math.sqrt(ol) * (F(1.0 + z) - F(1.0))


def growth_closed(om, z):
    """Linear growth D(a) ~ a 2F1(1/3, 1; 11/6; -a^3 OL/OM), normalised at z = 0."""
    ol = 1.0 - om
    D = lambda a: a * hyp2f1(1.0 / 3.0, 1.0, 11.0 / 6.0, -a ** 3 * ol / om)
    return D(1.0 / (1.0 + z)) / D(1.0)


def z_closed(om, r):
    return brentq(lambda z: dc_closed(om, z) - r, 0.0, 20.0, xtol=1e-15, rtol=1e-15)


# ------------------------------------------------------------ cosmology
@pytest.mark.parametrize("z", [0.05, 0.5, 1.0, 1.8, 2.5, 3.3, 5.0, 9.0])
def test_einstein_de_sitter_closed_forms(z):
    # Omega_M = 1: D_C = 2 c/H0 (1 - (1+z)^-1/2), G = 1/(1+z)
    assert oracle.comoving_distance(1.0, z) == pytest.approx(
        2 * CH * (1 - 1 / math.sqrt(1 + z)), rel=1e-12)
    assert oracle.growth(1.0, z) == pytest.approx(1 / (1 + z), rel=1e-12)


@pytest.mark.parametrize("z", [0.3, 1.57, 1.8, 2.23, 3.0, 3.94, 4.5, 7.0])
def test_lcdm_distance_and_growth_hypergeometric(z):
    assert oracle.comoving_distance(OM, z) == pytest.approx(dc_closed(OM, z), rel=1e-12)
    assert oracle.growth(OM, z) == pytest.approx(growth_closed(OM, z), rel=1e-11)


def test_z_of_distance_inverts():
    for r in [100.0, 1000.0, 3000.0, 3800.1, 4687.6, 5500.0]:
        z = oracle.z_of_distance(OM, r)
        assert z == pytest.approx(z_closed(OM, r), abs=1e-12)


# ------------------------------------------------------------ Philox + Box-Muller
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_box_muller_normals_distribution():
    e = []
    for c in range(6000):
        w = oracle.philox4x32_10([c, 5, 0, 0], [77, 13])
        e += list(oracle.box_muller(w[0], w[1])) + list(oracle.box_muller(w[2], w[3]))
    e = np.array(e)
    n = e.size
    assert abs(e.mean()) < 4 / math.sqrt(n)
    assert abs(e.var() - 1) < 4 * math.sqrt(2 / n)
    assert sst.kstest(e, "norm").pvalue > 1e-3
    # the two outputs of a pair are independent
    assert abs(np.corrcoef(e[0::2], e[1::2])[0, 1]) < 4 / math.sqrt(n / 2)


def test_box_muller_extreme_words():
    # x = 0 gives the largest radius sqrt(-2 ln(2^-33)); angle 2 pi 2^-33 ~ 0
    e1, e2 = oracle.box_muller(0, 0)
    assert e1 == pytest.approx(math.sqrt(66 * math.log(2)), rel=1e-12)
    assert abs(e2) < 1e-8
    # u2 = 1/4 (x2 = 2^30 - 1/2 -> just under a quarter turn): e1 ~ 0, e2 ~ radius
    e1, e2 = oracle.box_muller(0x80000000, 0x40000000)
    rad = math.sqrt(-2 * math.log((0x80000000 + 0.5) / 2 ** 32))
    assert e2 == pytest.approx(rad, rel=1e-12) and abs(e1) < 1e-8


# ------------------------------------------------------------ DFT
@pytest.mark.parametrize("n", [8, 64, 256])
def test_dft_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n)
    np.testing.assert_allclose(oracle.dft_forward_real(x), np.fft.rfft(x), atol=1e-11 * n)
    X = rng.standard_normal(n // 2 + 1) + 1j * rng.standard_normal(n // 2 + 1)
    np.testing.assert_allclose(oracle.dft_inverse_hermitian(X, n), np.fft.irfft(X, n),
                               atol=1e-12 * n)


# ------------------------------------------------------------ trilinear
def test_trilinear_reproduces_linear_field():
    n = 16
    i = np.arange(n) + 0.5
    box = (1.0 * i[None, None, :] + 0.5 * i[None, :, None] - 0.25 * i[:, None, None])
    box = box.astype(np.float32)  # dyadic values: exact in FP32
    rng = np.random.default_rng(3)
    for _ in range(200):
        c = rng.uniform(0.5, n - 0.5, 3)
        assert oracle.trilinear(box, c) == pytest.approx(c[0] + 0.5 * c[1] - 0.25 * c[2],
                                                         abs=1e-12)


def test_trilinear_single_voxel_is_tent_product_with_wrap():
    n = 8
    rng = np.random.default_rng(4)
    for v in [(0, 0, 0), (3, 5, 7), (7, 0, 2)]:
        box = np.zeros((n, n, n), np.float32)
        box[v[2], v[1], v[0]] = 1.0
        for _ in range(100):
            c = rng.uniform(-2.0, n + 2.0, 3)
            expect = 1.0
            for d in range(3):
                dist = (c[d] - (v[d] + 0.5)) % n
                dist = min(dist, n - dist)
                expect *= max(0.0, 1.0 - dist)
            assert oracle.trilinear(box, c) == pytest.approx(expect, abs=1e-13)


# ------------------------------------------------------------ Gaussian-kernel average (Sec. 2.3)
def _theta_window_sum():
    # sum_{|m|<=3} exp(-m^2/2) from the Jacobi theta identity
    # sum_{m in Z} exp(-m^2/2) = sqrt(2 pi) (1 + 2 sum_k exp(-2 pi^2 k^2)), minus the tail |m| >= 4
    full = math.sqrt(2.0 * math.pi) * (1.0 + 2.0 * sum(math.exp(-2.0 * math.pi ** 2 * k * k) for k in (1, 2)))
    tail = 2.0 * sum(math.exp(-0.5 * m * m) for m in range(4, 40))
    return full - tail


def test_gauss7_constant_field():
    box = np.full((16, 16, 16), 0.75, np.float32)
    rng = np.random.default_rng(21)
    for _ in range(50):
        c = rng.uniform(-3.0, 19.0, 3)
        assert oracle.gauss7(box, c) == pytest.approx(0.75, rel=1e-14)


def test_gauss7_single_voxel_weights_window_and_wrap():
    n = 16
    s0 = _theta_window_sum()
    assert s0 == pytest.approx(2.50594988, abs=1e-8)
    box = np.zeros((n, n, n), np.float32)
    v = (5, 9, 12)
    box[v[2], v[1], v[0]] = 1.0
    ctr = np.array(v, float) + 0.5
    assert oracle.gauss7(box, ctr) == pytest.approx(s0 ** -3, rel=1e-12)
    # one and two voxels away along different axes
    assert oracle.gauss7(box, ctr + [1, 0, 0]) == pytest.approx(math.exp(-0.5) / s0 ** 3, rel=1e-12)
    assert oracle.gauss7(box, ctr + [0, -2, 1]) == pytest.approx(math.exp(-2.5) / s0 ** 3, rel=1e-12)
    # 3 voxels away is inside the 7^3 window, 4 is outside
    assert oracle.gauss7(box, ctr + [0, 0, 3]) == pytest.approx(math.exp(-4.5) / s0 ** 3, rel=1e-12)
    assert oracle.gauss7(box, ctr + [4, 0, 0]) == 0.0
    assert oracle.gauss7(box, ctr + [0, -4, 2]) == 0.0
    # periodic wrap: voxel 0 seen from the centre of voxel n - 1
    box2 = np.zeros((n, n, n), np.float32)
    box2[0, 0, 0] = 1.0
    assert oracle.gauss7(box2, [n - 0.5, 0.5, 0.5]) == pytest.approx(math.exp(-0.5) / s0 ** 3, rel=1e-12)


def test_gauss7_linear_field_centres_and_face_bias():
    # f = x on voxel centres (no wrap inside the window): symmetric windows give
    # the centre value exactly; on a voxel face the window (containing voxel
    # +-3) reaches 3.5 cells ahead and 2.5 behind, a bias sum(d w)/sum(w) > 0
    n = 32
    i = np.arange(n) + 0.5
    box = np.broadcast_to(i[None, None, :], (n, n, n)).astype(np.float32).copy()
    for x in (8.5, 11.5, 20.5):
        assert oracle.gauss7(box, [x, 12.3, 17.9]) == pytest.approx(x, abs=1e-12)
    ds = [-2.5, -1.5, -0.5, 0.5, 1.5, 2.5, 3.5]
    wts = [math.exp(-0.5 * d * d) for d in ds]
    bias = sum(d * w for d, w in zip(ds, wts)) / sum(wts)
    assert bias == pytest.approx(3.5 * math.exp(-6.125) / sum(wts), rel=1e-3)  # the unmatched far voxel
    assert oracle.gauss7(box, [14.0, 12.3, 17.9]) == pytest.approx(14.0 + bias, abs=1e-12)


def test_gauss7_separable_field_is_product_of_axis_averages():
    n = 16
    rng = np.random.default_rng(22)
    gx, gy, gz = (rng.uniform(0.5, 1.5, n) for _ in range(3))
    box = (gz[:, None, None] * gy[None, :, None] * gx[None, None, :]).astype(np.float64)
    box32 = box.astype(np.float32)

    def avg1(g, c):  # 1D normalised Gaussian average over the 7 voxels around floor(c)
        ic = math.floor(c)
        ks = range(ic - 3, ic + 4)
        w = [math.exp(-0.5 * ((k + 0.5) - c) ** 2) for k in ks]
        return sum(wi * g[k % n] for wi, k in zip(w, ks)) / sum(w)

    for _ in range(40):
        c = rng.uniform(-2.0, n + 2.0, 3)
        expect = avg1(gx, c[0]) * avg1(gy, c[1]) * avg1(gz, c[2])
        # the box holds FP32-rounded products
        assert oracle.gauss7(box32, c) == pytest.approx(expect, rel=2e-7)


def test_skewer_fields_gauss7_constant_box_is_growth_times_constant():
    w = si.shrink(si.workload("tiny"), interp=1)
    n = w["n"]
    d = np.full((n, n, n), 0.5, np.float32)
    e = np.full((n, n, n), -0.25, np.float32)
    pos, ids = si.catalogue(w, n_q=3)
    o = oracle.run_skewers(w, d, e, pos, ids, n_threads=1)
    zj = np.array([oracle.pixel_z(w, j) for j in range(o["j_lo"][0], o["j_lo"][0] + o["npix"][0])])
    g = np.array([oracle.growth(w["omega_m"], z) for z in zj])
    k = o["offsets"][1]
    np.testing.assert_allclose(o["eta"][:k], -0.25 * g, rtol=1e-12)


# ------------------------------------------------------------ radial eta_par from six eta_pq boxes (Eq. eta)
_PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def test_eta_tensor_constant_components_give_u_c_u():
    w = si.shrink(si.workload("tiny"), eta_mode=1)
    n = w["n"]
    cvals = [0.3, -0.2, 0.5, 0.11, -0.07, 0.05]
    d = np.zeros((n, n, n), np.float32)
    e6 = np.stack([np.full((n, n, n), v, np.float32) for v in cvals])
    pos, ids = si.catalogue(w, n_q=4)
    o = oracle.run_skewers(w, d, e6, pos, ids, n_threads=1)
    cm = np.zeros((3, 3))
    for (a, b), v in zip(_PAIRS, np.float32(cvals).astype(np.float64)):
        cm[a, b] = cm[b, a] = v
    for q in range(4):
        u = pos[q] / np.linalg.norm(pos[q])
        js = range(o["j_lo"][q], o["j_lo"][q] + o["npix"][q])
        g = np.array([oracle.growth(w["omega_m"], oracle.pixel_z(w, j)) for j in js])
        np.testing.assert_allclose(o["eta"][o["offsets"][q]:o["offsets"][q + 1]], g * (u @ cm @ u), rtol=1e-12)


def test_eta_tensor_isotropic_diagonal_equals_single_box():
    w1 = si.workload("tiny")
    w6 = si.shrink(w1, eta_mode=1)
    d, e = si.gaussian_box(w1["n"], w1["cell"], w1["seed_box"])
    z = np.zeros_like(e)
    pos, ids = si.catalogue(w1, n_q=6)
    o1 = oracle.run_skewers(w1, d, e, pos, ids, n_threads=1)
    o6 = oracle.run_skewers(w6, d, np.stack([e, e, e, z, z, z]), pos, ids, n_threads=1)
    np.testing.assert_allclose(o6["eta"], o1["eta"], rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(o6["delta"], o1["delta"])


def test_eta_tensor_sightline_along_x_reduces_to_xx():
    w1 = si.workload("tiny")
    w6 = si.shrink(w1, eta_mode=1)
    d, e6 = si.gaussian_box_tensor(w1["n"], w1["cell"], w1["seed_box"])
    pos = np.array([[3900.0, 0.0, 0.0], [4300.0, 0.0, 0.0]])
    ids = np.array([7, 8], dtype=np.uint64)
    o1 = oracle.run_skewers(w1, d, e6[0], pos, ids, n_threads=1)
    o6 = oracle.run_skewers(w6, d, e6, pos, ids, n_threads=1)
    assert o6["offsets"][-1] > 1000
    np.testing.assert_allclose(o6["eta"], o1["eta"], rtol=1e-12, atol=1e-14)


def test_eta_tensor_inputs_trace_and_xx():
    d, e = si.gaussian_box(16, seed=5)
    d2, e6 = si.gaussian_box_tensor(16, seed=5)
    np.testing.assert_array_equal(d, d2)
    np.testing.assert_array_equal(e, e6[0])
    # sum_p k_p k_p / k^2 = 1: the trace is -delta (the zero mode of both vanishes)
    np.testing.assert_allclose(e6[0] + e6[1] + e6[2], -d, atol=1e-6)


# ------------------------------------------------------------ z-dependent small-scale power (Sec. 2.6)
def test_p_s_nodes_identical_tables_equal_one_table():
    w1 = si.workload("tiny")
    w2 = si.shrink(w1, p_s=np.stack([w1["p_s"], w1["p_s"]]), p_s_z=[2.0, 3.0])
    d, e = si.gaussian_box(w1["n"], w1["cell"], w1["seed_box"])
    pos, ids = si.catalogue(w1, n_q=5)
    o1 = oracle.run_skewers(w1, d, e, pos, ids, n_threads=1)
    o2 = oracle.run_skewers(w2, d, e, pos, ids, n_threads=1)
    np.testing.assert_allclose(o2["delta"], o1["delta"], rtol=1e-13, atol=1e-15)  # (1-w) P + w P rounds


def test_p_s_nodes_interpolate_power_at_window_mean_z():
    # tables P0 at z = 2.2 and 4 P0 at z = 2.6: every mode of a segment scales by
    # sqrt((1 - w) + 4 w), w from the mean pixel z of its n_fft window (clamped)
    w1 = si.workload("tiny")
    w2 = si.shrink(w1, p_s=np.stack([w1["p_s"], 4.0 * w1["p_s"]]), p_s_z=[2.2, 2.6])
    n = w1["n_fft"]
    for qid, j0 in ((7, 17000), (9, 19200), (11, 20000), (3, 22000)):
        zbar = np.mean([oracle.pixel_z(w1, j) for j in range(j0, j0 + n)])
        wz = min(max((zbar - 2.2) / 0.4, 0.0), 1.0)
        ref = oracle.small_scale_modes(w1, qid, 1, j0)
        got = oracle.small_scale_modes(w2, qid, 1, j0)
        np.testing.assert_allclose(got, ref * math.sqrt((1.0 - wz) + 4.0 * wz), rtol=1e-12, atol=1e-300)
    # the four windows cover below, inside and above the node range
    zs = [np.mean([oracle.pixel_z(w1, j) for j in range(j0, j0 + n)]) for j0 in (17000, 22000)]
    assert zs[0] < 2.2 and zs[1] > 2.6


# ------------------------------------------------------------ tuning of a, b sigma_g and P_s (Sec. 2.6)
from oracle import ps_tuning  # noqa: E402


def test_gauss_moments_without_dispersion():
    for a in (0.3, 1.2):
        f, sf = ps_tuning.fgpa_gauss_moments(a, 0.0)
        assert abs(f - math.exp(-a)) < 1e-14 and sf < 1e-7


@pytest.mark.parametrize("a,s", [(0.5, 0.3), (0.2, 0.25), (0.05, 0.35)])
def test_gauss_moments_lognormal_series(a, s):
    # E[exp(-t X)] = sum_n (-t)^n E[X^n] / n!, X lognormal with E[X^n] = exp(n^2 s^2 / 2):
    # t = a gives F-bar, t = 2a gives E[F^2]; the terms are below 1e-14 by n = 30
    def series(t):
        return sum((-t) ** n * math.exp(0.5 * n * n * s * s) / math.factorial(n) for n in range(31))
    f, sf = ps_tuning.fgpa_gauss_moments(a, s)
    m1, m2 = series(a), series(2.0 * a)
    assert abs(f - m1) < 1e-12
    assert abs(sf - math.sqrt(m2 - m1 * m1)) < 1e-10


def test_gauss_moments_monte_carlo():
    rng = np.random.default_rng(2310)
    a, s = 0.8, 1.5
    x = rng.standard_normal(4_000_000)
    f = np.exp(-a * np.exp(s * x))
    got, gsf = ps_tuning.fgpa_gauss_moments(a, s)
    se = f.std() / math.sqrt(f.size)
    assert abs(got - f.mean()) < 5 * se
    assert abs(gsf - f.std()) < 5 * se * 2


@pytest.mark.parametrize("a,s", [(0.3, 0.8), (1.2, 1.6), (0.08, 2.4)])
def test_fit_a_bsigma_recovers_parameters(a, s):
    f, sf = ps_tuning.fgpa_gauss_moments(a, s)
    a2, s2 = ps_tuning.fit_a_bsigma(f, sf)
    assert abs(a2 / a - 1) < 1e-7 and abs(s2 / s - 1) < 1e-7
    with pytest.raises(ValueError):
        ps_tuning.fit_a_bsigma(f, math.sqrt(f * (1 - f)))


def test_sigma_f_from_white_p1d():
    # white noise of variance v: every mode has P = v dr, and the DC-free
    # variance within a segment is v (N - 1) / N
    v, dr, n, fbar = 0.04, 0.6, 256, 0.7
    got = ps_tuning.sigma_f_from_p1d(fbar, np.full(32, v * dr), n, dr)
    assert abs(got - fbar * math.sqrt(v * (n - 1) / n)) < 1e-15


def test_sigma_f_from_p1d_is_the_segment_variance():
    # Parseval on real segments, binned like the statistics (equal-count k
    # bins of the P1D modes): the mode sum misses only Nyquist's share
    rng = np.random.default_rng(5)
    n, dr, nk = 256, 0.2, 32
    x = rng.standard_normal((400, n)) * np.exp(-np.arange(n) / 300.0)
    X = np.fft.rfft(x, axis=1)
    p = (dr / n) * np.abs(X[:, 1:]) ** 2              # modes 1..N/2
    pb = p.mean(axis=0).reshape(nk, -1).mean(axis=1)  # k-bin means
    var = np.mean(np.var(x, axis=1))
    got = ps_tuning.sigma_f_from_p1d(1.0, pb, n, dr) ** 2
    nyq_err = abs(p[:, -1].mean() - pb[-1]) / (n * dr)
    assert abs(got - var) <= nyq_err + 1e-12 * var


def test_sigma_g2_from_pixel_sums():
    # one z bin over every pixel of a tiny run: the bin's sums give the
    # variance of delta_tot + c eta over those pixels
    w = si.shrink(si.workload("tiny"), n_zbins=1, z_bin_lo=0.0, dz_bin=11.0)
    d, e = si.gaussian_box(w["n"], w["cell"], w["seed_box"])
    pos, ids = si.catalogue(w, n_q=20)
    o = oracle.run_skewers(w, d, e, pos, ids, n_threads=NTHREADS)
    st = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    for c in (0.0, 0.8, -1.3):
        ref = np.var(o["delta"] + c * o["eta"])
        assert abs(ps_tuning.sigma_g2(st["sums"][0], c) / ref - 1) < 1e-10


def test_mode_bins():
    np.testing.assert_array_equal(ps_tuning.mode_bins(256, 256, 1, 32)[1:], (np.arange(1, 129) - 1) // 4)
    mb = ps_tuning.mode_bins(1024, 256, 1, 32)   # 4 P_s modes per P1D mode
    assert mb[1] == 0 and mb[512] == 31 and mb[16] == 0 and mb[18] == 1
    mb = ps_tuning.mode_bins(256, 256, 3, 32)    # rebin 3: k beyond the P1D range -> last bin
    assert mb[1] == 0 and mb[2] == 1 and np.all(mb[43:] == 31)


def test_follow_nearest_tuned_node():
    np.testing.assert_array_equal(ps_tuning._follow(np.array([0, 1, 1, 0, 0, 1, 0], bool)),
                                  [1, 1, 2, 2, 5, 5, 5])


# ------------------------------------------------------------ geometry
def test_geometry_forest_window():
    w = si.workload("tiny")
    pos, ids = si.catalogue(w, n_q=25)
    jl, npx, zq = oracle.geometry(w, pos)
    for k in range(25):
        zq_ref = z_closed(OM, float(np.linalg.norm(pos[k])))
        assert zq[k] == pytest.approx(zq_ref, abs=1e-12)
        lam = lambda J: w["lambda_lya"] * (1 + z_closed(OM, (J + 0.5) * w["dr"]))
        lo, hi = w["lrf_min"] * (1 + zq_ref), w["lrf_max"] * (1 + zq_ref)
        assert npx[k] > 1500
        assert lo <= lam(jl[k]) < hi and lo <= lam(jl[k] + npx[k] - 1) < hi
        assert lam(jl[k] - 1) < lo and lam(jl[k] + npx[k]) >= hi


def test_geometry_cuts_and_truncation():
    w = si.workload("batched")
    pos, ids = si.catalogue(w, n_q=60)
    jl, npx, zq = oracle.geometry(w, pos)
    for k in range(60):
        zq_ref = z_closed(OM, float(np.linalg.norm(pos[k])))
        r_hi = dc_closed(OM, (1 + zq_ref) * w["lrf_max"] / w["lambda_lya"] - 1)
        z_lo = max((1 + zq_ref) * w["lrf_min"] / w["lambda_lya"] - 1,
                   w["lobs_min"] / w["lambda_lya"] - 1)
        r_lo = dc_closed(OM, z_lo)
        full = math.ceil(r_hi / w["dr"] - 0.5) - math.ceil(r_lo / w["dr"] - 0.5)
        if full < w["n_min"]:
            assert npx[k] == 0
            continue
        assert npx[k] == min(full, w["n_max"])
        # the red end is always kept: last pixel is the last one below r_hi
        assert (jl[k] + npx[k] - 0.5) * w["dr"] < r_hi <= (jl[k] + npx[k] + 0.5) * w["dr"]
        assert w["lambda_lya"] * (1 + z_closed(OM, (jl[k] + 0.5) * w["dr"])) >= w["lobs_min"]


def test_skewer_path_reproduces_linear_field_times_growth():
    # A box large enough that the forests stay inside it: trilinear must give
    # the linear field at the pixel position, scaled by G(z) of the pixel.
    n, cell = 64, 20.0
    w = si.shrink(si.workload("tiny"), n=n)
    w["cell"] = cell
    w["origin"] = (3400.0, -640.0, -640.0)
    i = np.arange(n) + 0.5
    box = (0.5 * i[None, None, :] - 0.25 * i[None, :, None] + 0.125 * i[:, None, None])
    box = box.astype(np.float32)
    zero = np.zeros_like(box)
    for q in [np.array([4000.0, 30.0, -20.0]), np.array([4100.0, -200.0, 150.0])]:
        jl, npx, _ = oracle.geometry(w, q[None, :])
        dl, et, ds = oracle.skewer_fields(w, box, zero, q, 9, int(jl[0]), int(npx[0]))
        u = q / np.linalg.norm(q)
        for j in range(0, int(npx[0]), 97):
            r = (jl[0] + j + 0.5) * w["dr"]
            c = (r * u - np.array(w["origin"])) / cell
            assert np.all((c > 0.5) & (c < n - 0.5))
            g = growth_closed(OM, z_closed(OM, r))
            assert dl[j] == pytest.approx(g * (0.5 * c[0] - 0.25 * c[1] + 0.125 * c[2]),
                                          rel=1e-11)
            assert et[j] == 0.0


# ------------------------------------------------------------ small-scale field
def test_small_scale_modes_are_whitened_philox_normals():
    w = si.workload("tiny")
    n = w["n_fft"]
    for qid, seg in [(0, 0), (17, 3), (2 ** 33 + 5, 1)]:
        X = oracle.small_scale_modes(w, qid, seg)
        x = oracle.small_scale_segment(w, qid, seg)
        np.testing.assert_allclose(np.fft.rfft(x)[1:], X[1:], rtol=1e-9, atol=1e-9)
        assert abs(np.fft.rfft(x)[0]) < 1e-9
        amp = np.sqrt(n * w["p_s"] / w["dr"])
        for m in [1, 2, 3, 77, n // 2 - 1]:
            ww = oracle.philox4x32_10([m >> 1, seg, qid >> 32, 0],
                                      [w["seed_noise"], qid & 0xFFFFFFFF])
            e1, e2 = oracle.box_muller(*(ww[2:4] if m & 1 else ww[0:2]))
            assert X[m] == pytest.approx(amp[m] * (e1 + 1j * e2) / math.sqrt(2), rel=1e-12)
        # the Nyquist mode uses words (0, 1) of counter 0, which mode 0 leaves free
        ww = oracle.philox4x32_10([0, seg, qid >> 32, 0], [w["seed_noise"], qid & 0xFFFFFFFF])
        e1, _ = oracle.box_muller(ww[0], ww[1])
        assert X[n // 2] == pytest.approx(amp[n // 2] * e1, rel=1e-12)


def test_small_scale_variance_closed_form():
    w = si.workload("tiny")
    n, dr, p = w["n_fft"], w["dr"], w["p_s"]
    expect = (2 * p[1:n // 2].sum() + p[n // 2]) / (n * dr)
    v = np.array([np.mean(oracle.small_scale_segment(w, q, s) ** 2)
                  for q in range(500) for s in range(3)])
    sem = v.std() / math.sqrt(v.size)   # segments are independent realisations
    assert abs(v.mean() - expect) < 5 * sem and sem < 0.01 * expect


# ------------------------------------------------------------ FGPA + statistics
def _gh_mean(f, sigma, order=80):
    x, wt = roots_hermitenorm(order)
    return float(np.sum(wt * f(sigma * x)) / math.sqrt(2 * math.pi))


def _const_nodes(w, a, b, c):
    w = dict(w)
    w["node_ln_a"] = [math.log(a)] * len(w["node_z"])
    w["node_b"] = [b] * len(w["node_z"])
    w["node_c"] = [c] * len(w["node_z"])
    return w


def test_fgpa_params_interpolation_and_clamp():
    w = si.workload("tiny")
    a, b, c = oracle.fgpa_params(w, 2.5)   # between nodes 2.4 and 2.6: ln a linear
    la = 0.5 * (math.log(0.01) + 4 * math.log(3.4)) + 0.5 * (math.log(0.01) + 4 * math.log(3.6))
    assert a == pytest.approx(math.exp(la), rel=1e-13) and b == 1.6 and c == 1.0
    assert oracle.fgpa_params(w, 1.0)[0] == pytest.approx(0.01 * 2.8 ** 4, rel=1e-13)
    assert oracle.fgpa_params(w, 9.0)[0] == pytest.approx(0.01 * 5.0 ** 4, rel=1e-13)


def test_mean_flux_matches_gauss_hermite_on_pure_small_scale_field():
    w = _const_nodes(si.workload("tiny"), 0.3, 1.6, 1.0)
    n, dr, p = w["n_fft"], w["dr"], w["p_s"]
    sig = math.sqrt((2 * p[1:n // 2].sum() + p[n // 2]) / (n * dr))
    pos, ids = si.catalogue(w, n_q=80)
    zero = np.zeros((w["n"],) * 3, np.float32)
    out = oracle.run_skewers(w, zero, zero, pos, ids, n_threads=NTHREADS)
    fbar = out["flux"].mean()
    expect = _gh_mean(lambda g: np.exp(-0.3 * np.exp(1.6 * g)), sig)
    assert fbar == pytest.approx(expect, abs=4e-3)


def test_stein_bias_and_beta_on_gaussian_eta_box():
    # delta box zero, eta box Gaussian: regression of F on (delta_tot, eta)
    # has coefficients E[T'(g)] (1, c), i.e. beta_F = c, b_F = E[T']/Fbar.
    a, b, c = 0.4, 1.6, 0.7
    w = _const_nodes(si.workload("tiny"), a, b, c)
    _, eta_box = si.gaussian_box(w["n"], w["cell"], w["seed_box"])
    zero = np.zeros_like(eta_box)
    pos, ids = si.catalogue(w, n_q=250)
    out = oracle.run_skewers(w, zero, eta_box, pos, ids, n_threads=NTHREADS)
    st = oracle.stats(w, out["j_lo"], out["offsets"], out["offsets_out"], out["flux"],
                      out["delta"], out["eta"])
    n, dr, p = w["n_fft"], w["dr"], w["p_s"]
    var_s = (2 * p[1:n // 2].sum() + p[n // 2]) / (n * dr)
    checked = 0
    for zb in range(w["n_zbins"]):
        s = st["sums"][zb]
        if s[0] < 60000:
            continue
        var_e = s[6] / s[0] - (s[4] / s[0]) ** 2
        sig = math.sqrt(var_s + c * c * var_e)
        T = lambda g: np.exp(-a * np.exp(b * g))
        Tp = lambda g: -a * b * np.exp(b * g) * np.exp(-a * np.exp(b * g))
        assert st["beta_f"][zb] == pytest.approx(c, rel=0.05)
        assert st["b_f"][zb] == pytest.approx(_gh_mean(Tp, sig) / _gh_mean(T, sig), rel=0.05)
        checked += 1
    assert checked >= 3


def test_regression_and_mean_flux_exact_on_manufactured_pixels():
    # F = alpha + k_d d + k_e e exactly  =>  b_F = k_d/Fbar, beta_F = k_e/k_d.
    w = si.workload("tiny")
    rng = np.random.default_rng(5)
    n = 3000
    j_lo = np.array([int(dc_closed(OM, 2.15) / w["dr"])], np.int32)
    d, e = rng.standard_normal(n), rng.standard_normal(n)
    F = 0.6 + 0.05 * d - 0.02 * e
    off = np.array([0, n], np.int64)
    st = oracle.stats(w, j_lo, off, off, F, d, e)
    zpix = np.array([z_closed(OM, (j_lo[0] + j + 0.5) * w["dr"]) for j in range(n)])
    zb = np.floor((zpix - w["z_bin_lo"]) / w["dz_bin"]).astype(int)
    for b in np.unique(zb):
        m = zb == b
        fbar = F[m].mean()
        assert st["sums"][b][0] == m.sum()
        assert st["mean_flux"][b] == pytest.approx(fbar, rel=1e-13)
        assert st["sigma_f"][b] == pytest.approx(F[m].std(), rel=1e-9)
        if m.sum() > 10:
            assert st["b_f"][b] == pytest.approx(0.05 / fbar, rel=1e-9)
            assert st["beta_f"][b] == pytest.approx(-0.02 / 0.05, rel=1e-9)


def test_p1d_single_mode_lands_in_its_bin_with_parseval_normalisation():
    w = si.workload("tiny")
    N, dr = w["n_fft"], w["dr"]
    j_lo = np.array([int(dc_closed(OM, 2.19) / dr)], np.int32)
    for m0 in [1, 4, 5, 37, N // 2 - 1]:
        j = np.arange(N)
        F = 0.7 + 0.1 * np.cos(2 * np.pi * m0 * j / N + 0.3)
        off = np.array([0, N], np.int64)
        st = oracle.stats(w, j_lo, off, off, F)
        zb = int(np.argmax(st["n_seg"]))
        assert st["n_seg"][zb] == 1 and st["n_seg"].sum() == 1
        kb = (m0 - 1) * w["n_kbins"] // (N // 2)
        row = st["p1d_sum"][zb]
        assert row[kb] == pytest.approx(dr * N * 0.1 ** 2 / 4, rel=1e-10)
        assert np.sum(np.delete(row, kb)) < 1e-20
        per_bin = (N // 2) / w["n_kbins"]
        assert st["p1d_df"][zb][kb] == pytest.approx(
            row[kb] / per_bin / st["mean_flux"][zb] ** 2, rel=1e-12)


def test_p1d_parseval_random_segment():
    w = si.workload("tiny")
    N, dr = w["n_fft"], w["dr"]
    rng = np.random.default_rng(8)
    F = rng.uniform(0.0, 1.0, N)
    j_lo = np.array([int(dc_closed(OM, 2.61) / dr)], np.int32)
    off = np.array([0, N], np.int64)
    st = oracle.stats(w, j_lo, off, off, F)
    total = st["p1d_sum"].sum()
    nyq = dr / N * np.sum(F * (-1.0) ** np.arange(N)) ** 2
    assert 2 * total - nyq == pytest.approx(dr * np.sum((F - F.mean()) ** 2), rel=1e-11)


def test_p1d_recovers_small_scale_power_in_linear_regime():
    # zero box, F = exp(-a e^{b g}) with a b small: P1D_F ~ (a b)^2 P_S.
    a, b = 1e-3, 0.1
    w = _const_nodes(si.workload("tiny"), a, b, 1.0)
    pos, ids = si.catalogue(w, n_q=200)
    zero = np.zeros((w["n"],) * 3, np.float32)
    out = oracle.run_skewers(w, zero, zero, pos, ids, n_threads=NTHREADS)
    st = oracle.stats(w, out["j_lo"], out["offsets"], out["offsets_out"], out["flux"])
    nseg = st["n_seg"]
    pooled = (st["p1d_f"] * nseg[:, None]).sum(0) / nseg.sum()
    N = w["n_fft"]
    ps = w["p_s"][1:N // 2 + 1].reshape(w["n_kbins"], -1).mean(1)
    ratio = pooled / ((a * b) ** 2 * ps)
    assert nseg.sum() > 1000
    assert np.all(np.abs(ratio - 1) < 0.06), ratio


def test_rebin_is_boxcar_mean_with_tail_dropped():
    w = si.workload("tiny")
    pos, ids = si.catalogue(w, n_q=3)
    d, e = si.gaussian_box(w["n"], w["cell"], w["seed_box"])
    o1 = oracle.run_skewers(w, d, e, pos, ids, rebin=1)
    o3 = oracle.run_skewers(w, d, e, pos, ids, rebin=3)
    for k in range(3):
        n = o1["npix"][k]
        f1 = o1["flux"][o1["offsets"][k]:o1["offsets"][k + 1]]
        f3 = o3["flux"][o3["offsets_out"][k]:o3["offsets_out"][k + 1]]
        assert f3.size == n // 3
        np.testing.assert_allclose(f3, f1[:3 * (n // 3)].reshape(-1, 3).mean(1), rtol=1e-14)


# ------------------------------------------------------------ paper targets
def test_table3_target_rows():
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLDEN, "table3_targets.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for z, beta, beff in rows:
        # printed z_eff has 3 decimals: allow its rounding plus the last printed digit
        db = abs(targets.beta_target(z + 5e-4) - targets.beta_target(z - 5e-4)) / 2
        de = abs(targets.b_eff_target(z + 5e-4) - targets.b_eff_target(z - 5e-4)) / 2
        assert abs(targets.beta_target(z) - beta) <= 5e-4 + db
        assert abs(targets.b_eff_target(z) - beff) <= 5e-5 + de


# ------------------------------------------------------------ surrogate MLP
def test_gelu_is_x_times_normal_cdf():
    from scipy.special import ndtr
    for x in [-6.0, -1.3, -0.2, 0.0, 0.5, 1.0, 2.7, 8.0]:
        assert oracle.gelu(x) == pytest.approx(x * ndtr(x), rel=1e-13, abs=1e-300)


def _mlp_params(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(oracle.MLP_NPARAM) * scale


def test_mlp_zero_hidden_weights_give_the_output_bias():
    p = np.zeros(oracle.MLP_NPARAM)
    b3 = np.arange(35) * 0.1 - 1.0
    p[-35:] = b3
    y = oracle.mlp_forward(p, np.random.default_rng(1).standard_normal((7, 4)))
    np.testing.assert_allclose(y, np.tile(b3, (7, 1)), atol=0)


def test_mlp_single_path_closed_form():
    # one live path x0 -> h1[0] -> h2[0] -> h3[0] -> y[j]: y_j = v_j G(w3 G(w2 G(w1 x0)))
    dims = oracle.MLP_DIMS
    p = np.zeros(oracle.MLP_NPARAM)
    offs, o = [], 0
    for l in range(4):
        offs.append(o)
        o += dims[l + 1] * dims[l] + dims[l + 1]
    w1, w2, w3 = 0.7, -1.3, 0.9
    p[offs[0] + 0] = w1                      # W0[0][0]
    p[offs[1] + 0] = w2                      # W1[0][0]
    p[offs[2] + 0] = w3                      # W2[0][0]
    v = np.linspace(-1, 1, 35)
    p[offs[3]:offs[3] + 35 * 128].reshape(35, 128)[:, 0] = v   # W3[:, 0]
    from scipy.special import ndtr
    G = lambda z: z * ndtr(z)
    for x0 in [-1.5, 0.3, 2.0]:
        y = oracle.mlp_forward(p, np.array([[x0, 5.0, -2.0, 1.0]]))[0]
        np.testing.assert_allclose(y, v * G(w3 * G(w2 * G(w1 * x0))), rtol=1e-12, atol=1e-15)


def test_mlp_gradient_matches_central_differences():
    p = _mlp_params(3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((6, 4))
    t = rng.standard_normal((6, 35))
    loss, g = oracle.mlp_loss_grad(p, x, t)
    y = oracle.mlp_forward(p, x)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-13)
    idx = np.concatenate([rng.choice(oracle.MLP_NPARAM, 60, replace=False),
                          [0, 511, 512, 639, 640, 17151, 17152, 33663, 33664, 38178]])
    h = 1e-4  # truncation ~h^2, round-off ~1e-16/h: both well below the tolerance
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_loss_grad(pp, x, t)[0] - oracle.mlp_loss_grad(pm, x, t)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=2e-6, abs=1e-9), i


def _bf16_torch(x):
    """x -> FP32 -> BF16 through torch's conversions (round to nearest even)."""
    import torch
    return torch.tensor(float(x), dtype=torch.float64).to(torch.float32).to(torch.bfloat16).double().item()


def test_bf16_rounding_is_nearest_even_via_fp32():
    # ties between BF16 neighbours go to the even one; above a tie rounds up
    assert oracle.bf16(1.0 + 2.0 ** -8) == 1.0
    assert oracle.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert oracle.bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7
    assert oracle.bf16(-(1.0 + 3 * 2.0 ** -9)) == -(1.0 + 2.0 ** -7)
    rng = np.random.default_rng(31)
    for x in np.concatenate([rng.standard_normal(200) * 10.0 ** rng.integers(-6, 6, 200), [0.0, 2.0 ** -130]]):
        assert oracle.bf16(x) == _bf16_torch(x), x


def test_adam_first_steps_in_closed_form():
    # step 1: m_hat = g, v_hat = g^2, so p moves by -lr g / (|g| + eps); eps sits
    # outside the root, so a gradient of 1e-9 moves p by lr / 11, not ~lr 1e-5
    lr, eps = 1e-3, 1e-8
    g1 = np.array([0.5, -2.0, 1e-9, 0.0, 3e-4])
    p = np.array([0.1, -0.2, 0.3, 0.4, 0.0])
    m, v = np.zeros(5), np.zeros(5)
    p0 = p.copy()
    oracle.adam_step(p, m, v, g1, 1, lr)
    np.testing.assert_allclose(p, p0 - lr * g1 / (np.abs(g1) + eps), rtol=1e-15, atol=1e-18)
    assert p[2] == pytest.approx(0.3 - lr / 11.0, rel=1e-12) and p[3] == 0.4
    # step 2 with another gradient: m = 0.09 g1 + 0.1 g2, v = 0.000999 g1^2 +
    # 0.001 g2^2, bias corrections 1 - 0.9^2 = 0.19 and 1 - 0.999^2 = 0.001999
    g2 = np.array([-0.25, 1.0, 2e-9, 1.0, 3e-4])
    p1 = p.copy()
    oracle.adam_step(p, m, v, g2, 2, lr)
    mh = (0.09 * g1 + 0.1 * g2) / 0.19
    vh = (0.000999 * g1 ** 2 + 0.001 * g2 ** 2) / 0.001999
    np.testing.assert_allclose(p, p1 - lr * mh / (np.sqrt(vh) + eps), rtol=1e-14, atol=1e-18)
    np.testing.assert_allclose(m, 0.09 * g1 + 0.1 * g2, rtol=1e-15)
    np.testing.assert_allclose(v, 0.000999 * g1 ** 2 + 0.001 * g2 ** 2, rtol=1e-15)


def _single_path_params(w1, w2, w3, v):
    dims = oracle.MLP_DIMS
    p = np.zeros(oracle.MLP_NPARAM)
    offs, o = [], 0
    for l in range(4):
        offs.append(o)
        o += dims[l + 1] * dims[l] + dims[l + 1]
    p[offs[0]] = w1
    p[offs[1]] = w2
    p[offs[2]] = w3
    p[offs[3]:offs[3] + 35 * 128].reshape(35, 128)[:, 0] = v
    return p, offs


def test_mlp_bf16_operands_single_path_closed_form():
    """The BF16-operand forward and backward on one live path x0 -> h0 -> h1
    -> h2 -> y, with the roundings written out: hidden activations, the
    output gradient and each dz are BF16; the output y is not rounded."""
    from scipy.special import ndtr
    G = lambda z: z * ndtr(z)
    dG = lambda z: ndtr(z) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)
    q = _bf16_torch
    w1, w2, w3 = 0.7, -1.3, 0.9
    v = np.linspace(-1, 1, 35)
    p, offs = _single_path_params(w1, w2, w3, v)
    x0 = 1.37
    x = np.array([[x0, 5.0, -2.0, 1.0]])
    t = np.random.default_rng(5).standard_normal((1, 35))
    z0 = w1 * x0
    h0 = q(G(z0))
    z1 = w2 * h0
    h1 = q(G(z1))
    z2 = w3 * h1
    h2 = q(G(z2))
    y = v * h2
    np.testing.assert_allclose(oracle.mlp_forward(p, x, bf16=True)[0], y, rtol=1e-14, atol=1e-16)
    loss, g = oracle.mlp_loss_grad(p, x, t, bf16=True)
    assert loss == pytest.approx(np.mean((y - t[0]) ** 2), rel=1e-13)
    dy = np.array([q(2.0 * (y[j] - t[0, j]) / 35.0) for j in range(35)])
    dz2 = q(np.dot(v, dy) * dG(z2))
    dz1 = q(w3 * dz2 * dG(z1))
    dz0 = q(w2 * dz1 * dG(z0))
    w3_block = g[offs[3]:offs[3] + 35 * 128].reshape(35, 128)
    np.testing.assert_allclose(w3_block[:, 0], dy * h2, rtol=1e-14, atol=1e-18)
    np.testing.assert_allclose(g[offs[3] + 35 * 128:offs[3] + 35 * 128 + 35], dy, rtol=1e-14, atol=1e-18)
    assert g[offs[2]] == pytest.approx(dz2 * h1, rel=1e-13)                 # W2[0][0]
    assert g[offs[2] + 128 * 128] == pytest.approx(dz2, rel=1e-13)          # b2[0]
    assert g[offs[1]] == pytest.approx(dz1 * h0, rel=1e-13)                 # W1[0][0]
    assert g[offs[0]] == pytest.approx(dz0 * x0, rel=1e-13)                 # W0[0][0]
    assert g[offs[0] + 1] == pytest.approx(dz0 * 5.0, rel=1e-13)            # W0[0][1]
    assert g[offs[0] + 128 * 4] == pytest.approx(dz0, rel=1e-13)            # b0[0]
    # every other hidden unit is dead: G(0) = 0, so no other weight moves
    # except the first-layer row of unit 0 and the output layer's column 0
    mask = np.ones(oracle.MLP_NPARAM, bool)
    mask[offs[0]:offs[0] + 4] = False
    mask[offs[0] + 512] = False
    mask[offs[1]] = mask[offs[1] + 128 * 128] = False
    mask[offs[2]] = mask[offs[2] + 128 * 128] = False
    mask[offs[3]:] = False
    # dead units still pass gradient to their biases through GELU'(0) = 1/2
    # times a zero dh, so their gradients are exactly zero
    assert np.all(g[mask] == 0.0)
    # without BF16 operands the same path gives the unrounded closed form
    loss64, g64 = oracle.mlp_loss_grad(p, x, t)
    assert g64[offs[2]] != g[offs[2]]


# ------------------------------------------------------------ Gaussian box synthesis (Sec. 2.1)
from oracle import box_synth  # noqa: E402


def test_box_noise_is_philox_box_muller_and_normal():
    n, seed = 32, 0x1234_5678_9ABC
    r = oracle.box_noise(seed, n).ravel()
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for v in (0, 1, 2, 3, 4, 4097, n ** 3 - 1):
        g = v // 4
        w = oracle.philox4x32_10((g & 0xFFFFFFFF, g >> 32, 0, 0), key)
        e = oracle.box_muller(w[0], w[1]) + oracle.box_muller(w[2], w[3])
        assert r[v] == e[v % 4]
    assert sst.kstest(r, "norm").pvalue > 1e-3
    assert abs(r.mean()) < 5 / math.sqrt(r.size)


def _white(n, cell, p0):
    return 0.5, np.full(int(2 * math.pi * math.sqrt(3) / cell / 0.5) + 3, p0)


def test_box_white_spectrum_variance():
    # P = p0 at every k: var(delta) = p0 / cell^3 times the kept mode fraction
    # ((n - 1)^3 - 1) / n^3 (no zero mode, no Nyquist planes)
    n, cell, p0 = 32, 2.0, 3.0
    dk, tab = _white(n, cell, p0)
    d, _ = box_synth.synth_box(n, cell, 99, dk, tab)
    expect = p0 / cell ** 3 * ((n - 1) ** 3 - 1) / n ** 3
    assert abs(d.var() / expect - 1) < 5 * math.sqrt(2.0 / n ** 3)
    assert abs(d.mean()) < 1e-12


def test_box_shell_power_matches_table():
    # |DFT(delta)_k|^2 cell^3 / n^3 averages to P(k) in shells (5 sigma)
    n, cell = 48, 1.5
    dk = 0.01
    ks = dk * np.arange(600)
    tab = (ks + 0.05) ** -1.5
    D = box_synth.delta_modes(n, cell, 7, dk, tab)
    kx, ky, kz = box_synth._wavenumbers(n, cell)
    k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2).ravel()
    pw = (np.abs(D) ** 2 * cell ** 3 / n ** 3).ravel()
    ptab = np.interp(k, ks, tab)
    keep = pw > 0
    edges = np.linspace(0.3, 1.8, 7)
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = keep & (k >= lo) & (k < hi)
        ratio = pw[m] / ptab[m]
        assert abs(ratio.mean() - 1) < 5 / math.sqrt(m.sum())


def test_box_eta_trace_is_minus_delta_and_boxes_are_real():
    n, cell = 32, 1.0
    dk = 0.02
    tab = np.exp(-dk * np.arange(400))
    d, eta = box_synth.synth_box(n, cell, 3, dk, tab, tensor=True)
    np.testing.assert_allclose(eta[0] + eta[1] + eta[2], -d, atol=1e-12 * np.abs(d).max())
    D = box_synth.delta_modes(n, cell, 3, dk, tab)
    z = np.fft.ifftn(D)
    assert np.abs(z.imag).max() < 1e-12 * np.abs(z.real).max()


def test_box_eta_isotropic_moments():
    # isotropic Gaussian field: <eta_xx^2> = <mu^4> sigma^2 = sigma^2/5,
    # <eta_xy^2> = sigma^2/15, <delta eta_xx> = -sigma^2/3 (sampling and grid
    # anisotropy within 3 %)
    n, cell = 64, 1.0
    dk = 0.01
    ks = dk * np.arange(600)
    tab = np.where((ks > 1.0) & (ks < 2.6), 1.0, 0.0)
    d, eta = box_synth.synth_box(n, cell, 11, dk, tab, tensor=True)
    s2 = d.var()
    for i in range(3):
        assert abs(np.mean(eta[i] ** 2) / (s2 / 5) - 1) < 0.03
        assert abs(np.mean(d * eta[i]) / (-s2 / 3) - 1) < 0.03
    for i in range(3, 6):
        assert abs(np.mean(eta[i] ** 2) / (s2 / 15) - 1) < 0.03


def test_box_eta_axes_by_finite_differences():
    # d_x^2 eta_yy = d_y^2 eta_xx = d_x d_y eta_xy (all -d_x^2 d_y^2 lap^-1 delta),
    # checked with central differences on a smooth box; a swapped axis breaks it
    n, cell = 64, 1.0
    dk = 0.005
    ks = dk * np.arange(200)
    tab = np.exp(-(ks / 0.25) ** 2)
    _, eta = box_synth.synth_box(n, cell, 5, dk, tab, tensor=True)

    def d2(f, ax):
        return np.roll(f, -1, ax) - 2 * f + np.roll(f, 1, ax)

    def d1(f, ax):
        return 0.5 * (np.roll(f, -1, ax) - np.roll(f, 1, ax))

    X, Y, Z = 2, 1, 0
    a = d2(eta[1], X)
    b = d2(eta[0], Y)
    c = d1(d1(eta[3], X), Y)
    scale = np.abs(a).max()
    assert np.abs(a - b).max() < 0.05 * scale
    assert np.abs(a - c).max() < 0.05 * scale
    # the same identity with z in place of y: d_x^2 eta_zz = d_z^2 eta_xx
    assert np.abs(d2(eta[2], X) - d2(eta[0], Z)).max() < 0.05 * np.abs(d2(eta[2], X)).max()
    # and it fails if eta_yy were taken for eta_zz
    assert np.abs(d2(eta[1], X) - d2(eta[0], Z)).max() > 0.2 * scale


# ------------------------------------------------------------ lognormal quasar field (Sec. 2.2, App. A)
from oracle import lognormal  # noqa: E402


def _gauss_pk(s, n=3000, kmax=12.0):
    # P(k) = (2 pi s^2)^(3/2) exp(-k^2 s^2 / 2)  <->  xi(r) = exp(-r^2 / (2 s^2))
    dk = kmax / (n - 1)
    k = dk * np.arange(n)
    return dk, (2 * math.pi * s * s) ** 1.5 * np.exp(-0.5 * (k * s) ** 2)


def test_xi_of_gaussian_spectrum_is_gaussian():
    s = 4.0
    dk, pk = _gauss_pk(s)
    r = np.array([0.0, 1.0, 3.0, 5.0, 8.0, 12.0])
    np.testing.assert_allclose(lognormal.xi_of_pk(pk, dk, r), np.exp(-r ** 2 / (2 * s * s)), atol=1e-10)


def test_lognormal_pk_second_order_closed_form():
    # ln(1 + B xi) = B xi - B^2 xi^2 / 2 + O(B^3), and xi^2 is the Gaussian of
    # width s / sqrt 2: P_q = B P - (B^2 / 2)(pi s^2)^(3/2) exp(-k^2 s^2 / 4) + O(B^3)
    s, B = 4.0, 1e-3
    dk, pk = _gauss_pk(s)
    k = dk * np.arange(pk.size)
    got = lognormal.lognormal_pk(pk, dk, B)
    ref = B * pk - 0.5 * B * B * (math.pi * s * s) ** 1.5 * np.exp(-0.25 * (k * s) ** 2)
    m = k < 0.8
    scale = B * pk[0]
    assert np.abs(got[m] - ref[m]).max() < 2 * B ** 3 * pk[0] * 3 + 1e-9 * scale


def test_qso_draw_uniform_field_follows_mean_density():
    # delta_q = 0: p = sum of the weights = 1 and E[p] = 1, so every voxel has
    # P = nbar cell^3; the count is binomial and positions stay in their voxel
    n, cell = 32, 2.19
    q = dict(n=n, cell=cell, origin=(3700.0 - n * cell / 2, -n * cell / 2, -n * cell / 2), z_box=(1.9, 2.75, 3.6),
             bias=(3.7, 2.33, 1.7), xi_m5=0.5, nbar=[2e-3] * 10, nbar_z0=1.5, nbar_dz=0.5, seed=7, omega_m=OM)
    z = np.zeros((n, n, n), np.float32)
    r = oracle.qso_draw(q, [z, z, z])
    P = 2e-3 * cell ** 3
    np.testing.assert_allclose(r["P"], P, rtol=1e-12)
    assert abs(r["count"] - n ** 3 * P) < 5 * math.sqrt(n ** 3 * P * (1 - P))
    ids = r["ids"].astype(np.int64)
    assert np.all(np.diff(ids) > 0)
    idx = np.stack([ids % n, (ids // n) % n, ids // (n * n)], axis=1)
    cell_of = np.floor((r["pos"] - np.asarray(q["origin"])) / cell)
    np.testing.assert_array_equal(cell_of, idx)
    assert np.all((r["u"] < r["P"]).sum() == r["count"])


def test_qso_draw_exponent_weights_at_the_middle_box():
    # a voxel at z = z_2 has t12 = 1 and t23 = 0: p = p_2 = exp(delta_2) (a_2 = 1),
    # E[p] = exp(sigma_2^2 / 2), whatever lambda is
    n, cell, om = 16, 2.19, OM
    z2 = 2.75
    r2 = dc_closed(om, z2)
    rng = np.random.default_rng(3)
    b = [rng.standard_normal((n, n, n)).astype(np.float32) * 0.3 for _ in range(3)]
    # put voxel (x=0, y=n/2, z=n/2) of the box centred on the axis at distance r2
    origin = (r2 - 0.5 * cell, -n * cell / 2, -n * cell / 2)
    q = dict(n=n, cell=cell, origin=origin, z_box=(1.9, z2, 3.6), bias=(3.7, 2.33, 1.7), xi_m5=0.7,
             nbar=[1e-3] * 10, nbar_z0=1.5, nbar_dz=0.5, seed=1, omega_m=om)
    res = oracle.qso_draw(q, b)
    v = (n // 2 * n + n // 2) * n
    s2 = float(np.mean(b[1].astype(np.float64) ** 2))
    ref = 1e-3 * cell ** 3 * math.exp(float(b[1].ravel()[v])) / math.exp(0.5 * s2)
    assert abs(res["P"][v] / ref - 1) < 1e-6  # the voxel centre sits within 1e-6 of z_2 in its weights


def test_qso_draw_expected_count_is_nbar_volume():
    # Gaussian boxes: E[P] = nbar cell^3 in every voxel when P stays below 1
    n, cell = 32, 2.19
    rng = np.random.default_rng(11)
    b = [rng.standard_normal((n, n, n)).astype(np.float32) * 0.5 for _ in range(3)]
    q = dict(n=n, cell=cell, origin=(4000.0, -n * cell / 2, -n * cell / 2), z_box=(1.9, 2.75, 3.6),
             bias=(3.7, 2.33, 1.7), xi_m5=0.4, nbar=[1e-3] * 10, nbar_z0=1.5, nbar_dz=0.5, seed=2, omega_m=OM)
    r = oracle.qso_draw(q, b)
    exp_mean = 1e-3 * cell ** 3
    assert abs(r["P"].mean() / exp_mean - 1) < 0.02
    assert abs(r["count"] - r["P"].sum()) < 5 * math.sqrt(r["P"].sum())


def test_dfbar_dlna_is_the_slope_of_the_moments():
    for a, s in ((0.3, 0.8), (1.2, 1.6), (0.05, 2.2)):
        h = 1e-5
        fd = (ps_tuning.fgpa_gauss_moments(a * math.exp(h), s)[0]
              - ps_tuning.fgpa_gauss_moments(a * math.exp(-h), s)[0]) / (2 * h)
        assert abs(ps_tuning.dfbar_dlna(a, s) - fd) < 1e-8
