"""FP64 restatement of the lognormal quasar field (Sec. 2.2, App. A).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``.

- ``xi_of_pk``: xi(r) = (1 / 2 pi^2) int P(k) k^2 j0(k r) dk, the trapezoid rule
  on the table k_i = i dk.
- ``lognormal_pk``: the power spectrum of the Gaussian field delta_q whose
  exponential has correlation B xi_m (the paper takes P_q as the Fourier
  transform of ln[1 + b_q^2 xi_m]): xi_m on r_j = j pi / k_max, then
  P_q(k_i) = 4 pi int ln(1 + B xi_m(r)) r^2 j0(k_i r) dr by the trapezoid rule on r_j,
  negative values (ringing of the finite sums where P_q is small) set to 0.
- The voxel draw itself is ``oracle.qso_draw`` (plain C loop).

Both sums are written as matrix products over the whole grid (numpy), with
j0(x) = sin(x)/x through ``np.sinc``.
"""
from __future__ import annotations

import numpy as np


def _trap(n):
    w = np.ones(n)
    w[0] = w[-1] = 0.5
    return w


def _j0(x):
    return np.sinc(x / np.pi)


def xi_of_pk(pk, dk, r):
    pk = np.asarray(pk, dtype=np.float64)
    k = dk * np.arange(pk.size)
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    f = _trap(pk.size) * dk * pk * k * k
    return _j0(np.outer(r, k)) @ f / (2.0 * np.pi ** 2)


def lognormal_pk(pk, dk, B):
    pk = np.asarray(pk, dtype=np.float64)
    n = pk.size
    k = dk * np.arange(n)
    dr = np.pi / (dk * (n - 1))
    r = dr * np.arange(n)
    xi = xi_of_pk(pk, dk, r)
    arg = 1.0 + B * xi
    if np.any(arg <= 0.0):
        raise ValueError("1 + B xi <= 0")
    g = _trap(n) * dr * np.log(arg) * r * r
    return np.maximum(4.0 * np.pi * (_j0(np.outer(k, r)) @ g), 0.0)  # a spectrum: ringing below 0 is cut
