"""FP64 restatement of the paper's tuning of a, b and P_s (Sec. 2.6).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: tests and the
benchmark's reference leg may call it; the library never does.

The steps, in the order Sec. 2.6 gives them:

1. c at each tuning redshift is the target beta (beta = f c with f = 1).
2. g is Gaussian, so F-bar and sigma_F depend only on a and b sigma_g; a and
   b sigma_g are fitted to the target F-bar and to the target sigma_F, the
   latter from the integral of the target P1D.
3. sigma_g^2 = sigma_L^2 + sigma_S^2 + c^2 sigma_eta^2 + 2 c cov(delta_L, eta)
   is measured on the skewers; b = (b sigma_g) / sigma_g.
4. P_s is iterated with the ratio P_s <- P_s * P1D_target / P1D_measured in
   each k bin, one full synthesis pass per iteration (ten in the paper).
5. The outer loop repeats 3-4 (five times in the paper).

Readings (the library takes the same ones; each is one line here):

- tuning redshifts are the z-bin centres; a bin with no P1D segment is not
  tuned and its node copies the nearest tuned node (ties: the lower);
- sigma_F target: F-bar* sqrt(sum over all DFT modes m = 1..N-1 of P1D*(k_m)
  / (N dr_out)), the mode sum taken from the equal-count k-bin means, the
  Nyquist mode's power read as the last bin's mean;
- sigma_g^2 is the population variance of delta_tot + c eta over the pixels of
  the bin (delta_tot = G delta_L + delta_S already holds sigma_L^2 + sigma_S^2
  and the covariance), so no separate box moments are needed;
- a P_s mode m of an N_fft-pixel segment takes the ratio of the k bin that
  holds P1D mode round(m N_p1d R / N_fft), clamped to 1 .. N_p1d / 2;
- the outer loop re-derives b from sigma_g and, after the first loop, takes
  one Newton step in ln a on the pass's mean flux (slope from the Gaussian
  model), the paper's small adjustments of a that keep F-bar; the bias-driven
  adjustments of b follow from a correlation-function prediction (out of scope).

Moments use composite Simpson over xi in [-12, 12]; the fit of (a, s) nests
two bisections, each on a quantity that is monotone in its variable.
"""
from __future__ import annotations

import numpy as np

import oracle

_XI = np.linspace(-12.0, 12.0, 12001)
_SIMPSON = np.ones_like(_XI)
_SIMPSON[1:-1:2] = 4.0
_SIMPSON[2:-1:2] = 2.0
_SIMPSON *= (_XI[1] - _XI[0]) / 3.0
_PHI = np.exp(-0.5 * _XI ** 2)
_PHI /= np.sum(_SIMPSON * _PHI)  # the rule integrates the density to exactly 1


def fgpa_gauss_moments(a, s):
    """F-bar and sigma_F of F = exp(-a exp(s xi)), xi ~ N(0, 1) (Eq. FGPA with
    b g Gaussian of dispersion s = b sigma_g)."""
    f = np.exp(-a * np.exp(s * _XI))
    m1 = float(np.sum(_SIMPSON * _PHI * f))
    m2 = float(np.sum(_SIMPSON * _PHI * f * f))
    return m1, float(np.sqrt(max(m2 - m1 * m1, 0.0)))


def dfbar_dlna(a, s):
    """d F-bar / d ln a of F = exp(-a exp(s xi)): -E[tau F], tau = a exp(s xi)."""
    tau = a * np.exp(s * _XI)
    return float(-np.sum(_SIMPSON * _PHI * tau * np.exp(-tau)))


def _bisect(fn, lo, hi, n=80):
    """Root of an increasing fn on [lo, hi] by bisection."""
    for _ in range(n):
        mid = 0.5 * (lo + hi)
        if fn(mid) < 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def fit_a_bsigma(fbar, sigma_f):
    """(a, b sigma_g) with fgpa_gauss_moments(a, s) = (fbar, sigma_f).

    At fixed s, F-bar falls as ln a grows; at F-bar held fixed, sigma_F grows
    with s (up to sqrt(F-bar (1 - F-bar)) as s -> infinity)."""
    if not (0.0 < fbar < 1.0) or not (0.0 < sigma_f < np.sqrt(fbar * (1.0 - fbar))):
        raise ValueError("no (a, s) gives this mean flux and sigma_F")

    def ln_a_at(s):
        return _bisect(lambda la: fbar - fgpa_gauss_moments(np.exp(la), s)[0], -40.0, 40.0, 70)

    s = _bisect(lambda s: fgpa_gauss_moments(np.exp(ln_a_at(s)), s)[1] - sigma_f, 1e-6, 12.0, 60)
    return float(np.exp(ln_a_at(s))), float(s)


def sigma_f_from_p1d(fbar, p1d_df, n_fft_p1d, dr_out):
    """Target sigma_F from the integral (a DFT-mode sum) of P1D_dF bin means."""
    p = np.asarray(p1d_df, dtype=np.float64)
    q = (n_fft_p1d // 2) // p.size
    total = 2.0 * q * p.sum() - p[-1]  # modes 1..N-1: twice 1..N/2, Nyquist once
    return fbar * np.sqrt(total / (n_fft_p1d * dr_out))


def sigma_g2(sums, c):
    """Population variance of delta_tot + c eta from one z bin's pixel sums
    (0 count, 3 d, 4 e, 5 d^2, 6 e^2, 7 d e)."""
    n = sums[0]
    md, me = sums[3] / n, sums[4] / n
    vd = sums[5] / n - md * md
    ve = sums[6] / n - me * me
    cv = sums[7] / n - md * me
    return vd + c * c * ve + 2.0 * c * cv


def mode_bins(n_fft, n_fft_p1d, rebin, n_k):
    """k bin of each P_s mode m = 0..n_fft/2 (entry 0 unused: X_0 = 0)."""
    q = (n_fft_p1d // 2) // n_k
    out = np.zeros(n_fft // 2 + 1, dtype=np.int64)
    for m in range(1, n_fft // 2 + 1):
        mp = int(np.floor(m * n_fft_p1d * rebin / n_fft + 0.5))
        mp = min(max(mp, 1), n_fft_p1d // 2)
        out[m] = (mp - 1) // q
    return out


def _follow(active):
    """Index of the node each node copies: itself when tuned, else the nearest
    tuned node (ties: the lower)."""
    idx = np.flatnonzero(active)
    src = np.arange(active.size)
    for i in range(active.size):
        if not active[i] and idx.size:
            src[i] = idx[np.argmin(np.abs(idx - i))]
    return src


def _pass(w, d, e, pos, ids, nodes, p_s, rebin, n_threads):
    wp = dict(w)
    wp.update(node_ln_a=list(np.log(nodes["a"])), node_b=list(nodes["b"]), node_c=list(nodes["c"]),
              p_s=p_s.copy(), p_s_z=list(nodes["z"]))
    o = oracle.run_skewers(wp, d, e, pos, ids, rebin=rebin, n_threads=n_threads)
    return oracle.stats(wp, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"],
                        rebin=rebin)


def tune_ps(w, d, e, pos, ids, target, p_s0, n_outer=5, n_inner=10, rebin=1, n_threads=1):
    """The Sec. 2.6 procedure on the oracle; returns the nodes, P_s tables,
    the last pass's statistics and the pass count.

    target: dict with per-bin "mean_flux", "p1d" (P1D_dF, n_k bins) and
    "beta", and "active" (bool per bin).  p_s0: (n_z, n_fft/2 + 1) start."""
    nz, nk = w["n_zbins"], w["n_kbins"]
    z = w["z_bin_lo"] + (np.arange(nz) + 0.5) * w["dz_bin"]
    active = np.asarray(target["active"], dtype=bool)
    src = _follow(active)
    dr_out = w["dr"] * rebin
    # steps 1-2
    c = np.array([float(target["beta"][i]) for i in range(nz)])
    a = np.ones(nz)
    s = np.ones(nz)
    for i in np.flatnonzero(active):
        sf = sigma_f_from_p1d(target["mean_flux"][i], target["p1d"][i][:nk], w["n_fft_p1d"], dr_out)
        a[i], s[i] = fit_a_bsigma(target["mean_flux"][i], sf)
    a, s, c = a[src], s[src], c[src]
    b = np.ones(nz)
    p_s = np.array(p_s0, dtype=np.float64).reshape(nz, w["n_fft"] // 2 + 1).copy()
    mb = mode_bins(w["n_fft"], w["n_fft_p1d"], rebin, nk)
    passes = 0
    for o in range(n_outer):
        # step 3 (and, after the first outer loop, a Newton step in ln a on this
        # pass's mean flux: the paper's small adjustments of a that keep F-bar)
        st = _pass(w, d, e, pos, ids, dict(z=z, a=a, b=b, c=c), p_s, rebin, n_threads)
        passes += 1
        for i in np.flatnonzero(active):
            b[i] = s[i] / np.sqrt(sigma_g2(st["sums"][i], c[i]))
            if o > 0:
                slope = dfbar_dlna(a[i], s[i])
                if slope < 0.0:
                    a[i] *= np.exp(np.clip((st["mean_flux"][i] - target["mean_flux"][i]) / -slope, -0.5, 0.5))
        a = a[src]
        b = b[src]
        # step 4
        for _ in range(n_inner):
            st = _pass(w, d, e, pos, ids, dict(z=z, a=a, b=b, c=c), p_s, rebin, n_threads)
            passes += 1
            for i in np.flatnonzero(active):
                ratio = np.asarray(target["p1d"][i][:nk]) / st["p1d_df"][i][:nk]
                p_s[i, 1:] *= ratio[mb[1:]]
            p_s = p_s[src]
    st = _pass(w, d, e, pos, ids, dict(z=z, a=a, b=b, c=c), p_s, rebin, n_threads)
    passes += 1
    return dict(z=z, a=a, b=b, c=c, s=s, p_s=p_s, stats=st, passes=passes)
