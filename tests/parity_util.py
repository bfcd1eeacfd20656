"""Shared helpers of the GPU parity tests (tolerances, oracle runs, boxes)."""
import os

import numpy as np

import oracle
import skewer_inputs as si

# Tolerances: delta/eta 2e-6 relative to max(|x|, field RMS); F 1e-5
# absolute; mean flux and P1D 1e-4 relative.
TOL_FIELD = 2e-6
TOL_FLUX = 1e-5
TOL_STAT = 1e-4
NTHREADS = max(1, min(16, os.cpu_count() or 1))


def assert_field_close(gpu, orc, what):
    gpu = np.asarray(gpu, dtype=np.float64)
    orc = np.asarray(orc, dtype=np.float64)
    assert gpu.shape == orc.shape, what
    if orc.size == 0:
        return
    sigma = np.sqrt(np.mean(orc ** 2))
    err = np.abs(gpu - orc) / np.maximum(np.abs(orc), sigma)
    worst = int(np.argmax(err))
    assert err[worst] <= TOL_FIELD, f"{what}: rel err {err[worst]:.3g} at {worst} ({gpu[worst]} vs {orc[worst]})"


def assert_flux_close(gpu, orc, what="flux"):
    gpu = np.asarray(gpu, dtype=np.float64)
    orc = np.asarray(orc, dtype=np.float64)
    assert gpu.shape == orc.shape
    if orc.size:
        err = np.abs(gpu - orc)
        assert err.max() <= TOL_FLUX, f"{what}: abs err {err.max():.3g}"


def assert_stats_close(g, o, check_fields=True):
    np.testing.assert_array_equal(g["sums"][:, 0], o["sums"][:, 0])   # pixel counts
    np.testing.assert_array_equal(g["n_seg"], o["n_seg"])              # segment counts
    m = o["sums"][:, 0] > 0
    np.testing.assert_allclose(g["mean_flux"][m], o["mean_flux"][m], rtol=TOL_STAT)
    np.testing.assert_allclose(g["sigma_f"][m], o["sigma_f"][m], rtol=TOL_STAT)
    ms = o["n_seg"] > 0
    np.testing.assert_allclose(g["p1d_f"][ms], o["p1d_f"][ms], rtol=TOL_STAT)
    np.testing.assert_allclose(g["p1d_df"][ms], o["p1d_df"][ms], rtol=TOL_STAT)
    if check_fields:
        big = o["sums"][:, 0] > 1000
        np.testing.assert_allclose(g["b_f"][big], o["b_f"][big], rtol=TOL_STAT)
        np.testing.assert_allclose(g["beta_f"][big], o["beta_f"][big], rtol=TOL_STAT)


def ragged(values, offsets, i):
    return values[offsets[i]:offsets[i + 1]]


def oracle_subset(w, dbox, ebox, pos, ids, idx, rebin=1):
    """Oracle outputs for the quasars idx (a subset of the catalogue)."""
    return oracle.run_skewers(w, dbox, ebox, pos[idx], ids[idx], rebin=rebin, n_threads=NTHREADS)


def box_numpy(w):
    return si.gaussian_box(w["n"], w["cell"], w["seed_box"], backend="numpy")
