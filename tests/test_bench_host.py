"""Host arithmetic of the benchmark line (CPU): the algorithmic bytes that the
roofline fraction divides by, against a brute-force count of the voxels that
each skewer's trilinear stencils touch."""
import numpy as np

import bench

CORNERS = np.array([[a, b, c] for a in (0, 1) for b in (0, 1) for c in (0, 1)], dtype=np.int64)


def distinct_stencil_voxels(p0, step, npix):
    # voxels (floor(p) + {0, 1})^3 over the pixel positions p0 + j step (cell units)
    j = np.arange(npix, dtype=np.float64)[:, None]
    base = np.floor(p0[None, :] + j * step[None, :]).astype(np.int64)
    v = (base[:, None, :] + CORNERS[None, :, :]).reshape(-1, 3)
    return len(np.unique(v, axis=0))


def sight_lines(rng, n, max_deg):
    # unit vectors within max_deg of the x axis
    c = rng.uniform(np.cos(np.radians(max_deg)), 1.0, n)
    phi = rng.uniform(0, 2 * np.pi, n)
    s = np.sqrt(1 - c * c)
    return np.stack([c, s * np.cos(phi), s * np.sin(phi)], axis=1)


def test_algorithmic_bytes_count_the_trilinear_tube():
    rng = np.random.default_rng(11)
    w = dict(dr=0.2, cell=2.19)
    u = np.concatenate([sight_lines(rng, 48, 20.0), sight_lines(rng, 16, 90.0)])
    pos = u * rng.uniform(3600.0, 6000.0, (len(u), 1))
    npix = rng.integers(200, 1501, len(u))
    npix[:3] = (0, 1, 2)  # empty and tiny skewers
    brute = 0
    for k in range(len(u)):
        if npix[k] == 0:
            continue
        p0 = rng.uniform(0.0, 1000.0, 3)
        brute += distinct_stencil_voxels(p0, u[k] * w["dr"] / w["cell"], int(npix[k]))
    per_skewer = 32 + 72 + 72 + 16
    expect = brute * 8.0 + npix.sum() * 4.0 + per_skewer * len(u)
    got = bench.algorithmic_bytes(pos, npix, w)
    # the closed form counts 4 new voxels per cell-face crossing; crossings of
    # two faces at one step share 2 voxels, which it does not subtract
    assert 0.0 <= got / expect - 1.0 < 0.02


def test_algorithmic_bytes_of_an_axis_aligned_skewer_are_exact():
    # along x with step 1/4 cell from 0.5: positions up to 100.25, 100 cell
    # faces crossed, 8 voxels and then 4 more per face
    w = dict(dr=0.25, cell=1.0)
    npix = np.array([400])
    pos = np.array([[5000.0, 0.0, 0.0]])
    brute = distinct_stencil_voxels(np.array([0.5, 0.5, 0.5]), np.array([0.25, 0.0, 0.0]), 400)
    assert brute == 8 + 4 * 100
    got = bench.algorithmic_bytes(pos, npix, w)
    assert abs(got - ((8 + 4 * 100) * 8.0 + 400 * 4.0 + 192)) < 1e-9
