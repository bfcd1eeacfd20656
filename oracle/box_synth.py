"""FP64 restatement of the Gaussian box synthesis (Sec. 2.1, Eq. deltaL, Eq. eta).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``.

The density contrast is white noise filtered in Fourier space by the square
root of the power spectrum; the velocity-gradient boxes multiply the same
modes by -k_p k_q / k^2 (with f = 1 and the sign of the synthetic fixtures).
With V = (n cell)^3 and the unnormalised DFT, <|DFT(delta)_k|^2> = n^3 P(k) /
cell^3 and <|DFT(noise)_k|^2> = n^3, so the filter is sqrt(P(k) / cell^3).

Readings (the library takes the same ones):

- the noise is ``oracle.box_noise`` (Philox4x32-10 + Box-Muller per voxel);
- P(k) is the caller's table at k_i = i dk, i = 0 .. n_tab - 1, linear in
  between and 0 beyond the last entry;
- the k = 0 mode and every mode with an index n/2 on any axis (the Nyquist
  planes) are zero, so that the spectrum is exactly Hermitian and every
  filter, odd or even in k_p, gives a real box;
- k along an axis at index j is 2 pi (j or j - n) / (n cell), the wrapped
  frequency.

numpy's FFTs serve as the library primitive for each transform.
"""
from __future__ import annotations

import numpy as np

import oracle

PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))  # eta_xx, yy, zz, xy, xz, yz


def _wavenumbers(n, cell):
    k1 = 2.0 * np.pi * np.fft.fftfreq(n, d=cell)
    return k1[None, None, :], k1[None, :, None], k1[:, None, None]  # k_x, k_y, k_z on [z][y][x]


def power_interp(k, dk, table):
    table = np.asarray(table, dtype=np.float64)
    kmax = dk * (table.size - 1)
    p = np.interp(k, dk * np.arange(table.size), table)
    return np.where(k <= kmax, p, 0.0)


def delta_modes(n, cell, seed, dk, table):
    """DFT of the density box: noise modes times sqrt(P / cell^3), with the
    k = 0 mode and the Nyquist planes zero."""
    r = oracle.box_noise(seed, n)
    R = np.fft.fftn(r)
    kx, ky, kz = _wavenumbers(n, cell)
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    D = R * np.sqrt(power_interp(k, dk, table) / cell ** 3)
    D[0, 0, 0] = 0.0
    h = n // 2
    D[h, :, :] = 0.0
    D[:, h, :] = 0.0
    D[:, :, h] = 0.0
    return D


def synth_box(n, cell, seed, dk, table, tensor=False):
    """(delta, eta): eta is eta_xx (n, n, n), or with tensor the six eta_pq in
    the order xx, yy, zz, xy, xz, yz (6, n, n, n)."""
    D = delta_modes(n, cell, seed, dk, table)
    ks = _wavenumbers(n, cell)
    k2 = ks[0] ** 2 + ks[1] ** 2 + ks[2] ** 2
    inv = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    delta = np.fft.ifftn(D).real
    pairs = PAIRS if tensor else PAIRS[:1]
    eta = np.stack([np.fft.ifftn(-ks[a] * ks[b] * inv * D).real for a, b in pairs])
    return delta, (eta if tensor else eta[0])
