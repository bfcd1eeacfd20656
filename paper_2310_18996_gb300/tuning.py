"""Targets and helpers for tuning a(z), b(z), c(z) (Sec. 2.6).

The tuning target of this library is reachable by construction: hidden
parameters b*(z) = b0 ((1+z)/3.3)^beta_b and c*(z) = c0 ((1+z)/3.3)^beta_c
(seeded coefficients) and a*(z) solved so that the mean flux of the stored
skewers equals exp(-0.0025 (1+z)^3.7); the P1D and beta_F targets are then
the statistics of one pass at (a*, b*, c*).  Every pass runs in the library
(mk_flux_stats); this module only updates the 12 node values between passes.
"""
from __future__ import annotations

import math

import numpy as np

from . import FgpaNodes, TuneTarget, stat_bins


def mean_flux_target(z):
    return math.exp(-0.0025 * (1.0 + z) ** 3.7)


def node_z(w):
    b = stat_bins(w)
    return [b.z_lo + (i + 0.5) * b.dz for i in range(b.n_z)]


def nodes(zs, ln_a, b, c):
    nd = FgpaNodes()
    nd.count = len(zs)
    for i, z in enumerate(zs):
        nd.z[i], nd.ln_a[i], nd.b[i], nd.c[i] = z, ln_a[i], b[i], c[i]
    return nd


def hidden_parameters(w, seed):
    """Seeded power laws b*(z), c*(z) at the bin-centre nodes."""
    rng = np.random.default_rng(seed)
    b0, beta_b = rng.uniform(1.3, 1.9), rng.uniform(-0.5, 0.5)
    c0, beta_c = rng.uniform(0.7, 1.3), rng.uniform(-0.5, 0.5)
    zs = node_z(w)
    b = [b0 * ((1 + z) / 3.3) ** beta_b for z in zs]
    c = [c0 * ((1 + z) / 3.3) ** beta_c for z in zs]
    return zs, b, c


def solve_mean_flux(ctx, w, sk, n_sk, offsets, delta, eta, zs, b, c, ln_a0=None, iters=12):
    """ln a per node such that the mean flux per bin meets the target (secant on ln a)."""
    nz = len(zs)
    la = np.array(ln_a0 if ln_a0 is not None else [math.log(0.2)] * nz, dtype=np.float64)
    tgt = np.array([mean_flux_target(z) for z in zs])
    prev_la, prev_f = None, None
    st = None
    for _ in range(iters):
        st = ctx.flux_stats(w, sk, n_sk, offsets, delta, eta, nodes=nodes(zs, la, b, c))
        f = st["mean_flux"]
        if prev_la is None:
            new = la + 0.3 * np.sign(f - tgt)  # the flux falls as a grows
        else:
            slope = (f - prev_f) / np.where(np.abs(la - prev_la) > 1e-12, la - prev_la, 1e-12)
            new = np.where(np.abs(slope) > 1e-9, la - (f - tgt) / np.where(np.abs(slope) > 1e-9, slope, 1.0), la)
            new = np.clip(new, la - 1.0, la + 1.0)
        prev_la, prev_f = la, f
        la = new
    st = ctx.flux_stats(w, sk, n_sk, offsets, delta, eta, nodes=nodes(zs, la, b, c))
    return la, st


def fill_inactive(vals, active):
    """Values of bins without data follow the nearest active bin (ties: the lower)."""
    idx = [i for i in range(len(vals)) if (active >> i) & 1]
    out = list(vals)
    for i in range(len(vals)):
        if not (active >> i) & 1 and idx:
            j = min(idx, key=lambda k: (abs(k - i), k))
            out[i] = vals[j]
    return out


def make_target(ctx, w, sk, n_sk, offsets, delta, eta, seed=5, tol_mean_flux=1e-3, tol_p1d=0.02,
                tol_beta=0.02, k_lo=0, k_hi=32, min_segments=20):
    """(TuneTarget, hidden FgpaNodes): a reachable seeded target on these skewers.

    Bins with fewer than min_segments P1D segments are inactive; their nodes
    follow the nearest active node, as mk_tune's do."""
    zs, b, c = hidden_parameters(w, seed)
    la, st = solve_mean_flux(ctx, w, sk, n_sk, offsets, delta, eta, zs, b, c)
    active = 0
    for i in range(len(zs)):
        if (st["n_seg"][i] >= min_segments and st["sums"][i][0] > 0
                and np.all(st["p1d_df"][i][k_lo:k_hi] > 0)):
            active |= 1 << i
    la, b, c = (fill_inactive(list(v), active) for v in (la, b, c))
    st = ctx.flux_stats(w, sk, n_sk, offsets, delta, eta, nodes=nodes(zs, la, b, c))
    t = TuneTarget()
    for i in range(len(zs)):
        t.mean_flux[i] = st["mean_flux"][i]
        t.beta[i] = st["beta_f"][i]
        for k in range(len(st["p1d_df"][i])):
            t.p1d[i][k] = st["p1d_df"][i][k]
    t.use_beta = 1
    t.k_lo, t.k_hi = k_lo, k_hi
    t.active = active
    t.tol_mean_flux, t.tol_p1d, t.tol_beta = tol_mean_flux, tol_p1d, tol_beta
    return t, nodes(zs, la, b, c)


def start_nodes(w, ln_a=math.log(0.2), b=1.6, c=1.0):
    zs = node_z(w)
    n = len(zs)
    return nodes(zs, [ln_a] * n, [b] * n, [c] * n)


# ------------------------------------------------------------ small-scale power (Sec. 2.6)
def hidden_small_scale_power(w, seed):
    """Seeded P_S*(k, z) = P_S(k) (1 + A (z - 2.6)) (k / k_8)^t at the bin-centre
    nodes, A in [-0.4, 0.4], t in [-0.3, 0.3], k_8 the mode n_fft/8; P_S(k) is
    the workload's table.  Shape (n_z, n_fft/2 + 1)."""
    rng = np.random.default_rng(seed + 1000)
    amp, tilt = rng.uniform(-0.4, 0.4), rng.uniform(-0.3, 0.3)
    n = w["n_fft"]
    p0 = np.asarray(w["p_s"], dtype=np.float64).reshape(-1, n // 2 + 1)[0]
    m = np.arange(n // 2 + 1, dtype=np.float64)
    shape = np.where(m > 0, (np.maximum(m, 1.0) / (n // 8)) ** tilt, 1.0)
    return np.stack([p0 * shape * (1.0 + amp * (z - 2.6)) for z in node_z(w)])


def start_small_scale_power(w):
    """The workload's one P_S table at every bin-centre node: (n_z, n_fft/2 + 1)."""
    n = w["n_fft"]
    p0 = np.asarray(w["p_s"], dtype=np.float64).reshape(-1, n // 2 + 1)[0]
    return np.tile(p0, (len(node_z(w)), 1))


def make_ps_target(ctx, box, qso, n_qso, w, seed=5, **kw):
    """(TuneTarget, hidden FgpaNodes, hidden P_S tables): the statistics of the
    catalogue synthesised with the seeded hidden P_S*(k, z) and the hidden
    a*, b*, c* of make_target (on skewers stored at P_S*)."""
    ps = hidden_small_scale_power(w, seed)
    ws = dict(w, p_s=ps, p_s_z=node_z(w))
    r = ctx.make_skewers(box, qso, n_qso, ws)
    t, nd = make_target(ctx, ws, r["sk"], n_qso, r["offsets"], r["delta"], r["eta"], seed=seed, **kw)
    del r
    return t, nd, ps
