"""Seeded synthetic inputs shared by the oracle tests and the CUDA library.

This module holds the workload recipes (box size, cell, observer placement,
quasar placement, small-scale power table, FGPA node values, statistic bins)
and the generators for the Gaussian boxes and quasar catalogues.  It holds
none of the skewer-synthesis arithmetic: no cosmology, no geometry, no
interpolation, no FGPA, no statistics.  Distances that stand for redshift
ranges are literal numbers (comoving Mpc/h in the Table 1 cosmology).

Box recipe (the paper's Sec. 2 box synthesis, used here only to make inputs):
white noise N(0,1) per voxel -> 3D FFT -> multiply by sqrt(P(k)/V_cell) ->
inverse FFT, with P(k) = A k^0.96 exp(-(k/1.5)^2) (1 + 0.05 sin(150 k)) and A
fixed so that the voxel variance (1/V) sum_{k != 0} P(k) is 1; the
line-of-sight velocity-gradient box is eta = IFFT[-(k_x^2/k^2) delta_hat].
"""
from __future__ import annotations

import math

import numpy as np

OMEGA_M = 0.3147          # Table 1
LAMBDA_LYA = 1215.67      # Angstrom
CELL = 2.19               # Mpc/h (Sec. 2)
DR = 0.2                  # Mpc/h (Sec. 2.3)
OBSERVER_TO_BOX_CENTRE = 3800.0  # Mpc/h along +x

# comoving distances [Mpc/h] standing for redshifts in the Table 1 cosmology
DIST_Z = {1.8: 3373.74, 2.0: 3581.23, 2.04: 3620.44, 3.5: 4687.67,
          3.8: 4845.95, 4.0: 4943.61}

NODE_Z = [1.8 + 0.2 * i for i in range(12)]


def power_shape(k):
    """Unnormalised 3D power spectrum of the synthetic boxes (k in h/Mpc)."""
    k = np.asarray(k, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        p = k ** 0.96 * np.exp(-(k / 1.5) ** 2) * (1.0 + 0.05 * np.sin(150.0 * k))
    return np.where(k > 0, p, 0.0)


def small_scale_power(n_fft, dr=DR):
    """P_S(k_m) = 0.1 k^-1 exp(-(k/5)^2) on k_m = 2 pi m/(n_fft dr), m = 0..n_fft/2."""
    m = np.arange(n_fft // 2 + 1, dtype=np.float64)
    k = 2.0 * np.pi * m / (n_fft * dr)
    with np.errstate(divide="ignore"):
        p = 0.1 / k * np.exp(-(k / 5.0) ** 2)
    p[0] = 0.0
    return p


def _base(name, n, n_q, n_fft, seeds, **kw):
    L = n * CELL
    w = dict(
        name=name, omega_m=OMEGA_M, lambda_lya=LAMBDA_LYA, n=n, cell=CELL,
        origin=(OBSERVER_TO_BOX_CENTRE - 0.5 * L, -0.5 * L, -0.5 * L),
        dr=DR, lrf_min=1040.0, lrf_max=1200.0, lobs_min=0.0, n_min=0, n_max=0,
        n_fft=n_fft, p_s=small_scale_power(n_fft), n_q=n_q,
        seed_box=seeds[0], seed_cat=seeds[1], seed_noise=seeds[2],
        # FGPA nodes: a = 0.01 (1+z)^4, b = 1.6, c = 1 sampled at 12 z nodes
        node_z=list(NODE_Z),
        node_ln_a=[math.log(0.01) + 4.0 * math.log(1.0 + z) for z in NODE_Z],
        node_b=[1.6] * len(NODE_Z), node_c=[1.0] * len(NODE_Z),
        # statistics: 12 z bins centred on the nodes, 32 k bins
        n_zbins=12, z_bin_lo=1.7, dz_bin=0.2, n_kbins=32, n_fft_p1d=n_fft,
        rebin=1,
    )
    w.update(kw)
    return w


def workload(name):
    """Recipe of a named workload (sizes, seeds, tables); no arithmetic of the method."""
    if name == "tiny":       # 64^3 box, 500 quasars at z 2.0-3.5, N_fft 256
        return _base(name, 64, 500, 256, (1001, 2001, 3001), placement="uniform",
                     x_range=(DIST_Z[2.0], DIST_Z[3.5]))
    if name == "scale":      # 512^3 box, 100k lognormal-selected quasars at z 1.8-3.8
        return _base(name, 512, 100_000, 1024, (1002, 2002, 3002), placement="lognormal",
                     x_range=(DIST_Z[1.8], DIST_Z[3.8]))
    if name == "batched":    # 1024^3 box, 1M quasars, 200-1500 px skewers, N_fft 256
        return _base(name, 1024, 1_000_000, 256, (1003, 2003, 3003), placement="uniform",
                     x_range=(DIST_Z[2.04], DIST_Z[4.0]), lobs_min=3600.0, n_min=200,
                     n_max=1500)
    raise KeyError(name)


def shrink(w, n=None, n_q=None, **kw):
    """Same recipe with a smaller box and/or catalogue (test sizes)."""
    w = dict(w)
    if n is not None:
        L = n * w["cell"]
        w["n"] = n
        w["origin"] = (OBSERVER_TO_BOX_CENTRE - 0.5 * L, -0.5 * L, -0.5 * L)
    if n_q is not None:
        w["n_q"] = n_q
    if "n_fft" in kw:
        kw.setdefault("p_s", small_scale_power(kw["n_fft"], w["dr"]))
        kw.setdefault("n_fft_p1d", kw["n_fft"])
    w.update(kw)
    return w


# ------------------------------------------------------------------ boxes
def _box_numpy(n, cell, seed):
    rng = np.random.default_rng(seed)
    wn = rng.standard_normal((n, n, n))                 # [z][y][x], x fastest
    wk = np.fft.rfftn(wn)
    kx = 2.0 * np.pi * np.fft.rfftfreq(n, d=cell)
    ky = 2.0 * np.pi * np.fft.fftfreq(n, d=cell)
    k2 = kx[None, None, :] ** 2 + ky[None, :, None] ** 2 + ky[:, None, None] ** 2
    p = power_shape(np.sqrt(k2))
    mult = np.full(kx.size, 2.0)
    mult[0] = 1.0
    if n % 2 == 0:
        mult[-1] = 1.0
    amp = 1.0 / (np.sum(p * mult[None, None, :]) / (n ** 3 * cell ** 3))
    dk = wk * np.sqrt(amp * p / cell ** 3)
    with np.errstate(divide="ignore", invalid="ignore"):
        mu2 = np.where(k2 > 0, kx[None, None, :] ** 2 / k2, 0.0)
    delta = np.fft.irfftn(dk, s=(n, n, n), axes=(0, 1, 2)).astype(np.float32)
    eta = np.fft.irfftn(-mu2 * dk, s=(n, n, n), axes=(0, 1, 2)).astype(np.float32)
    return delta, eta


def _box_torch(n, cell, seed, device):
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    wn = torch.randn((n, n, n), generator=g, device=device, dtype=torch.float32)
    wk = torch.fft.rfftn(wn)
    del wn
    kx = (2.0 * math.pi * torch.fft.rfftfreq(n, d=cell, device=device, dtype=torch.float64))
    ky = (2.0 * math.pi * torch.fft.fftfreq(n, d=cell, device=device, dtype=torch.float64))
    k2 = kx[None, None, :] ** 2 + ky[None, :, None] ** 2 + ky[:, None, None] ** 2
    k = torch.sqrt(k2)
    p = torch.where(k > 0, k.pow(0.96) * torch.exp(-(k / 1.5) ** 2)
                    * (1.0 + 0.05 * torch.sin(150.0 * k)), torch.zeros_like(k))
    del k
    mult = torch.full((kx.numel(),), 2.0, device=device, dtype=torch.float64)
    mult[0] = 1.0
    mult[-1] = 1.0
    amp = 1.0 / (torch.sum(p * mult[None, None, :]).item() / (n ** 3 * cell ** 3))
    s = torch.sqrt(amp * p / cell ** 3).to(torch.float32)
    del p
    mu2 = torch.where(k2 > 0, kx[None, None, :] ** 2 / torch.where(k2 > 0, k2, 1.0),
                      torch.zeros_like(k2)).to(torch.float32)
    del k2
    wk.mul_(s)
    del s
    delta = torch.fft.irfftn(wk, s=(n, n, n))
    wk.mul_(-mu2)
    del mu2
    eta = torch.fft.irfftn(wk, s=(n, n, n))
    del wk
    return delta.contiguous(), eta.contiguous()


ETA_PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))  # xx, yy, zz, xy, xz, yz


def _tensor_numpy(n, cell, seed):
    delta, eta_xx = _box_numpy(n, cell, seed)
    rng = np.random.default_rng(seed)
    wn = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(wn)
    kx = 2.0 * np.pi * np.fft.rfftfreq(n, d=cell)
    ky = 2.0 * np.pi * np.fft.fftfreq(n, d=cell)
    ks = (kx[None, None, :], ky[None, :, None], ky[:, None, None])  # k_x, k_y, k_z
    k2 = ks[0] ** 2 + ks[1] ** 2 + ks[2] ** 2
    p = power_shape(np.sqrt(k2))
    mult = np.full(kx.size, 2.0)
    mult[0] = 1.0
    if n % 2 == 0:
        mult[-1] = 1.0
    amp = 1.0 / (np.sum(p * mult[None, None, :]) / (n ** 3 * cell ** 3))
    dk = wk * np.sqrt(amp * p / cell ** 3)
    eta = np.empty((6, n, n, n), np.float32)
    eta[0] = eta_xx
    with np.errstate(divide="ignore", invalid="ignore"):
        for c, (a, b) in enumerate(ETA_PAIRS[1:], start=1):
            m = np.where(k2 > 0, ks[a] * ks[b] / k2, 0.0)
            eta[c] = np.fft.irfftn(-m * dk, s=(n, n, n), axes=(0, 1, 2)).astype(np.float32)
    return delta, eta


def _tensor_torch(n, cell, seed, device):
    import torch

    delta, eta_xx = _box_torch(n, cell, seed, device)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    wk = torch.fft.rfftn(torch.randn((n, n, n), generator=g, device=device, dtype=torch.float32))
    kx = (2.0 * math.pi * torch.fft.rfftfreq(n, d=cell, device=device, dtype=torch.float64))
    ky = (2.0 * math.pi * torch.fft.fftfreq(n, d=cell, device=device, dtype=torch.float64))
    ks = (kx[None, None, :], ky[None, :, None], ky[:, None, None])
    k2 = ks[0] ** 2 + ks[1] ** 2 + ks[2] ** 2
    k = torch.sqrt(k2)
    p = torch.where(k > 0, k.pow(0.96) * torch.exp(-(k / 1.5) ** 2)
                    * (1.0 + 0.05 * torch.sin(150.0 * k)), torch.zeros_like(k))
    del k
    mult = torch.full((kx.numel(),), 2.0, device=device, dtype=torch.float64)
    mult[0] = 1.0
    mult[-1] = 1.0
    amp = 1.0 / (torch.sum(p * mult[None, None, :]).item() / (n ** 3 * cell ** 3))
    wk.mul_(torch.sqrt(amp * p / cell ** 3).to(torch.float32))
    del p
    safe = torch.where(k2 > 0, k2, torch.ones_like(k2))
    eta = torch.empty((6, n, n, n), device=device, dtype=torch.float32)
    eta[0] = eta_xx
    del eta_xx
    for c, (a, b) in enumerate(ETA_PAIRS[1:], start=1):
        m = torch.where(k2 > 0, ks[a] * ks[b] / safe, torch.zeros_like(k2)).to(torch.float32)
        eta[c] = torch.fft.irfftn(wk * (-m), s=(n, n, n))
        del m
    return delta.contiguous(), eta


def gaussian_box_tensor(n, cell=CELL, seed=0, backend="numpy", device="cuda"):
    """delta and the six velocity-gradient boxes eta_pq = IFFT[-(k_p k_q/k^2) delta_hat]
    (Eq. eta with the fixtures' sign, f = 1), shape (6, n, n, n) in the order
    xx, yy, zz, xy, xz, yz.  delta and eta_xx equal gaussian_box's delta and eta."""
    if backend == "numpy":
        return _tensor_numpy(n, cell, seed)
    if backend == "torch":
        return _tensor_torch(n, cell, seed, device)
    raise ValueError(backend)


def gaussian_box(n, cell=CELL, seed=0, backend="numpy", device="cuda"):
    """(delta, eta) FP32 boxes of shape (n, n, n), index [z][y][x] (x fastest)."""
    if backend == "numpy":
        return _box_numpy(n, cell, seed)
    if backend == "torch":
        return _box_torch(n, cell, seed, device)
    raise ValueError(backend)


# ------------------------------------------------------------- catalogues
def catalogue(w, delta=None, n_q=None):
    """Quasar positions in the observer frame (float64, (n_q, 3)) and ids (uint64).

    "uniform": x uniform over the workload's distance range, y and z uniform
    across the box face.  "lognormal": a voxel drawn with weight
    exp(delta) 1[delta > 0], the position uniform inside it, then the
    periodic replica along x whose distance falls in the range (one drawn at
    random when several do).
    """
    n_q = w["n_q"] if n_q is None else n_q
    rng = np.random.default_rng(w["seed_cat"])
    L = w["n"] * w["cell"]
    lo, hi = w["x_range"]
    if w["placement"] == "uniform":
        x = rng.uniform(lo, hi, n_q)
        y = rng.uniform(-0.5 * L, 0.5 * L, n_q)
        z = rng.uniform(-0.5 * L, 0.5 * L, n_q)
    elif w["placement"] == "lognormal":
        if delta is None:
            raise ValueError("lognormal placement needs the delta box")
        d = np.asarray(delta, dtype=np.float64).ravel()
        wt = np.where(d > 0, np.exp(d), 0.0)
        wt /= wt.sum()
        vox = rng.choice(d.size, size=n_q, p=wt)
        n = w["n"]
        ix, iy, iz = vox % n, (vox // n) % n, vox // (n * n)
        off = rng.uniform(0.0, 1.0, (n_q, 3))
        bx = (ix + off[:, 0]) * w["cell"] + w["origin"][0]
        y = (iy + off[:, 1]) * w["cell"] + w["origin"][1]
        z = (iz + off[:, 2]) * w["cell"] + w["origin"][2]
        kmin = np.ceil((lo - bx) / L)
        kmax = np.floor((hi - bx) / L)
        pick = kmin + np.floor(rng.uniform(0.0, 1.0, n_q) * (kmax - kmin + 1))
        x = bx + pick * L
    else:
        raise ValueError(w["placement"])
    pos = np.stack([x, y, z], axis=1)
    ids = np.arange(n_q, dtype=np.uint64)
    return pos, ids


def node_arrays(w):
    """FGPA node table of the workload as four float64 arrays (z, ln a, b, c)."""
    return (np.asarray(w["node_z"], np.float64), np.asarray(w["node_ln_a"], np.float64),
            np.asarray(w["node_b"], np.float64), np.asarray(w["node_c"], np.float64))
