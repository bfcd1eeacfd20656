"""FP64 CPU oracle for Lyman-alpha skewer synthesis (arXiv 2310.18996).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference``) may import
this package.  It shares no code with ``paper_2310_18996_gb300`` and never
imports it; both sides read their inputs from ``skewer_inputs``.

The arithmetic lives in ``oracle.c`` (plain C, double precision, built with
gcc); this module compiles it on first use and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle.h")]
_lock = threading.Lock()
_lib = None

MAX_NODES = 32
MAX_ZBINS = 32
MAX_KBINS = 64
NSUM = 10


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no fast-math: IEEE double throughout)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC[0], "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class Cfg(C.Structure):
    _fields_ = [
        ("omega_m", C.c_double), ("lambda_lya", C.c_double),
        ("n", C.c_int32), ("cell", C.c_double), ("origin", C.c_double * 3),
        ("dr", C.c_double), ("lrf_min", C.c_double), ("lrf_max", C.c_double),
        ("lobs_min", C.c_double), ("n_min", C.c_int32), ("n_max", C.c_int32),
        ("n_fft", C.c_int32), ("p_s", C.POINTER(C.c_double)), ("seed", C.c_uint32),
        ("interp", C.c_int32), ("eta_mode", C.c_int32),
        ("p_s_nodes", C.c_int32), ("p_s_z", C.POINTER(C.c_double)),
    ]


class Nodes(C.Structure):
    _fields_ = [("count", C.c_int32), ("z", C.c_double * MAX_NODES),
                ("ln_a", C.c_double * MAX_NODES), ("b", C.c_double * MAX_NODES),
                ("c", C.c_double * MAX_NODES)]


class Bins(C.Structure):
    _fields_ = [("n_z", C.c_int32), ("z_lo", C.c_double), ("dz", C.c_double),
                ("n_k", C.c_int32), ("n_fft", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [
        ("sums", (C.c_double * NSUM) * MAX_ZBINS),
        ("p1d_sum", (C.c_double * MAX_KBINS) * MAX_ZBINS),
        ("n_seg", C.c_double * MAX_ZBINS),
        ("mean_flux", C.c_double * MAX_ZBINS),
        ("sigma_f", C.c_double * MAX_ZBINS),
        ("p1d_f", (C.c_double * MAX_KBINS) * MAX_ZBINS),
        ("p1d_df", (C.c_double * MAX_KBINS) * MAX_ZBINS),
        ("b_f", C.c_double * MAX_ZBINS),
        ("beta_f", C.c_double * MAX_ZBINS),
    ]


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i32, i64, u32, u64 = C.c_double, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
            P = C.POINTER
            sig = {
                "orc_hubble_e": (d, [d, d]),
                "orc_comoving_distance": (d, [d, d]),
                "orc_z_of_distance": (d, [d, d]),
                "orc_growth": (d, [d, d]),
                "orc_philox4x32_10": (None, [P(u32), P(u32), P(u32)]),
                "orc_box_muller": (None, [u32, u32, P(d), P(d)]),
                "orc_box_noise": (None, [C.c_uint64, i32, P(d)]),
                "orc_qso_draw": (i64, [d, P(C.c_float), P(C.c_float), P(C.c_float), i32, i32, d, P(d), P(d),
                                       P(d), d, P(d), i32, d, d, C.c_uint64, P(d), P(d), P(u64), P(d), i64]),
                "orc_dft_forward_real": (None, [P(d), i32, P(d), P(d)]),
                "orc_dft_inverse_hermitian": (None, [P(d), P(d), i32, P(d)]),
                "orc_geometry": (C.c_int, [P(Cfg), P(d), P(i32), P(i32), P(d)]),
                "orc_pixel_z": (d, [P(Cfg), i64]),
                "orc_trilinear": (d, [P(C.c_float), i32, P(d)]),
                "orc_gauss7": (d, [P(C.c_float), i32, P(d)]),
                "orc_small_scale_modes": (None, [P(Cfg), u64, i32, i64, P(d), P(d)]),
                "orc_small_scale_segment": (None, [P(Cfg), u64, i32, i64, P(d)]),
                "orc_skewer_fields": (C.c_int, [P(Cfg), P(C.c_float), P(C.c_float), P(d), u64,
                                                i32, i32, P(d), P(d), P(d)]),
                "orc_fgpa_params": (None, [P(Nodes), d, P(d), P(d), P(d)]),
                "orc_fgpa": (d, [d, d, d, d, d]),
                "orc_run_skewers": (i64, [P(Cfg), P(C.c_float), P(C.c_float), P(d), P(u64), i64,
                                          P(Nodes), i32, P(i32), P(i32), P(i64), P(d), P(d),
                                          P(d), P(i64), P(d), i32]),
                "orc_stats_zero": (None, [P(Stats)]),
                "orc_stats_accumulate": (C.c_int, [P(Cfg), P(Bins), i32, P(i32), P(i64),
                                                   P(i64), i64, P(d), P(d), P(d), P(Stats)]),
                "orc_stats_finalize": (None, [P(Bins), P(Stats)]),
                "orc_mlp_forward": (None, [P(d), P(d), i64, P(d), C.c_int]),
                "orc_mlp_loss_grad": (d, [P(d), P(d), P(d), i64, P(d), C.c_int]),
                "orc_bf16": (d, [d]),
                "orc_adam_step": (None, [P(d), P(d), P(d), P(d), i64, i64, d, d, d, d]),
                "orc_gelu": (d, [d]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


# ---------------------------------------------------------------- scalars
def hubble_e(om, z):
    return lib().orc_hubble_e(om, z)


def comoving_distance(om, z):
    return lib().orc_comoving_distance(om, z)


def z_of_distance(om, r):
    return lib().orc_z_of_distance(om, r)


def growth(om, z):
    return lib().orc_growth(om, z)


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def box_muller(x1, x2):
    e1, e2 = C.c_double(), C.c_double()
    lib().orc_box_muller(int(x1) & 0xFFFFFFFF, int(x2) & 0xFFFFFFFF, C.byref(e1), C.byref(e2))
    return e1.value, e2.value


def box_noise(seed, n):
    """White noise of the synthetic box, shape (n, n, n) as [z][y][x]."""
    out = np.zeros(n * n * n)
    lib().orc_box_noise(int(seed) & 0xFFFFFFFFFFFFFFFF, int(n), _p(out, C.c_double))
    return out.reshape(n, n, n)


def dft_forward_real(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.size
    re = np.zeros(n // 2 + 1)
    im = np.zeros(n // 2 + 1)
    lib().orc_dft_forward_real(_p(x, C.c_double), n, _p(re, C.c_double), _p(im, C.c_double))
    return re + 1j * im


def dft_inverse_hermitian(X, n):
    re = np.ascontiguousarray(np.real(X), dtype=np.float64)
    im = np.ascontiguousarray(np.imag(X), dtype=np.float64)
    out = np.zeros(n)
    lib().orc_dft_inverse_hermitian(_p(re, C.c_double), _p(im, C.c_double), n,
                                    _p(out, C.c_double))
    return out


def trilinear(box, c):
    box = np.ascontiguousarray(box, dtype=np.float32)
    cc = np.ascontiguousarray(c, dtype=np.float64)
    return lib().orc_trilinear(_p(box, C.c_float), box.shape[0], _p(cc, C.c_double))


def gauss7(box, c):
    """Gaussian-kernel average over 7^3 voxels (Sec. 2.3) at cell coordinate c."""
    box = np.ascontiguousarray(box, dtype=np.float32)
    cc = np.ascontiguousarray(c, dtype=np.float64)
    return lib().orc_gauss7(_p(box, C.c_float), box.shape[0], _p(cc, C.c_double))


# ---------------------------------------------------------------- structs
def make_cfg(w):
    """Build the C config from a workload dict (see skewer_inputs.workload)."""
    ps = np.ascontiguousarray(w["p_s"], dtype=np.float64)
    cfg = Cfg()
    cfg.omega_m = w["omega_m"]
    cfg.lambda_lya = w["lambda_lya"]
    cfg.n = w["n"]
    cfg.cell = w["cell"]
    for d in range(3):
        cfg.origin[d] = w["origin"][d]
    cfg.dr = w["dr"]
    cfg.lrf_min, cfg.lrf_max = w["lrf_min"], w["lrf_max"]
    cfg.lobs_min = w.get("lobs_min", 0.0)
    cfg.n_min, cfg.n_max = w.get("n_min", 0), w.get("n_max", 0)
    cfg.n_fft = w["n_fft"]
    cfg.p_s = _p(ps, C.c_double)
    cfg.seed = w["seed_noise"] & 0xFFFFFFFF
    cfg.interp = w.get("interp", 0)
    cfg.eta_mode = w.get("eta_mode", 0)
    psz = np.ascontiguousarray(w.get("p_s_z", []), dtype=np.float64)
    cfg.p_s_nodes = len(psz)
    if cfg.p_s_nodes >= 2:
        assert ps.size == cfg.p_s_nodes * (w["n_fft"] // 2 + 1), "p_s needs one table per p_s_z node"
        cfg.p_s_z = _p(psz, C.c_double)
    cfg._keep = (ps, psz)  # keep the tables alive with the struct
    return cfg


def make_nodes(w):
    nd = Nodes()
    z = np.asarray(w["node_z"], dtype=np.float64)
    nd.count = z.size
    for i in range(z.size):
        nd.z[i] = z[i]
        nd.ln_a[i] = w["node_ln_a"][i]
        nd.b[i] = w["node_b"][i]
        nd.c[i] = w["node_c"][i]
    return nd


def make_bins(w):
    b = Bins()
    b.n_z, b.z_lo, b.dz = w["n_zbins"], w["z_bin_lo"], w["dz_bin"]
    b.n_k, b.n_fft = w["n_kbins"], w["n_fft_p1d"]
    return b


# ---------------------------------------------------------------- drivers
def geometry(w, qpos):
    cfg = make_cfg(w)
    qpos = np.ascontiguousarray(qpos, dtype=np.float64).reshape(-1, 3)
    n = qpos.shape[0]
    jl = np.zeros(n, np.int32)
    npx = np.zeros(n, np.int32)
    zq = np.zeros(n)
    for i in range(n):
        a, b, z = C.c_int32(), C.c_int32(), C.c_double()
        lib().orc_geometry(C.byref(cfg), _p(qpos[i], C.c_double), C.byref(a), C.byref(b),
                           C.byref(z))
        jl[i], npx[i], zq[i] = a.value, b.value, z.value
    return jl, npx, zq


def pixel_z(w, j):
    cfg = make_cfg(w)
    return lib().orc_pixel_z(C.byref(cfg), int(j))


def small_scale_modes(w, qid, seg, j0=0):
    cfg = make_cfg(w)
    n = w["n_fft"]
    re = np.zeros(n // 2 + 1)
    im = np.zeros(n // 2 + 1)
    lib().orc_small_scale_modes(C.byref(cfg), int(qid), int(seg), int(j0), _p(re, C.c_double),
                                _p(im, C.c_double))
    return re + 1j * im


def small_scale_segment(w, qid, seg, j0=0):
    cfg = make_cfg(w)
    out = np.zeros(w["n_fft"])
    lib().orc_small_scale_segment(C.byref(cfg), int(qid), int(seg), int(j0), _p(out, C.c_double))
    return out


def skewer_fields(w, dbox, ebox, q, qid, j_lo, npix):
    cfg = make_cfg(w)
    dbox = np.ascontiguousarray(dbox, dtype=np.float32)
    ebox = np.ascontiguousarray(ebox, dtype=np.float32)
    q = np.ascontiguousarray(q, dtype=np.float64)
    dl, et, ds = np.zeros(npix), np.zeros(npix), np.zeros(npix)
    lib().orc_skewer_fields(C.byref(cfg), _p(dbox, C.c_float), _p(ebox, C.c_float),
                            _p(q, C.c_double), int(qid), int(j_lo), int(npix),
                            _p(dl, C.c_double), _p(et, C.c_double), _p(ds, C.c_double))
    return dl, et, ds


def fgpa_params(w, z):
    nd = make_nodes(w)
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    lib().orc_fgpa_params(C.byref(nd), float(z), C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def run_skewers(w, dbox, ebox, qpos, ids, rebin=1, flux=True, n_threads=1):
    """Geometry, fields, FGPA and rebin for a catalogue; ragged FP64 outputs."""
    cfg = make_cfg(w)
    nd = make_nodes(w)
    dbox = np.ascontiguousarray(dbox, dtype=np.float32)
    ebox = np.ascontiguousarray(ebox, dtype=np.float32)
    qpos = np.ascontiguousarray(qpos, dtype=np.float64).reshape(-1, 3)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    nq = qpos.shape[0]
    jl = np.zeros(nq, np.int32)
    npx = np.zeros(nq, np.int32)
    off = np.zeros(nq + 1, np.int64)
    offo = np.zeros(nq + 1, np.int64)
    L = lib()
    total = L.orc_run_skewers(C.byref(cfg), _p(dbox, C.c_float), _p(ebox, C.c_float),
                              _p(qpos, C.c_double), _p(ids, C.c_uint64), nq, C.byref(nd),
                              rebin, _p(jl, C.c_int32), _p(npx, C.c_int32),
                              _p(off, C.c_int64), None, None, None, _p(offo, C.c_int64),
                              None, n_threads)
    if total < 0:
        raise ValueError("oracle geometry failed")
    dt, et = np.zeros(total), np.zeros(total)
    ff = np.zeros(total) if flux else None
    fo = np.zeros(int(offo[-1])) if flux else None
    L.orc_run_skewers(C.byref(cfg), _p(dbox, C.c_float), _p(ebox, C.c_float),
                      _p(qpos, C.c_double), _p(ids, C.c_uint64), nq, C.byref(nd), rebin,
                      _p(jl, C.c_int32), _p(npx, C.c_int32), _p(off, C.c_int64),
                      _p(dt, C.c_double), _p(et, C.c_double), _p(ff, C.c_double),
                      _p(offo, C.c_int64), _p(fo, C.c_double), n_threads)
    return dict(j_lo=jl, npix=npx, offsets=off, delta=dt, eta=et, flux_fine=ff,
                offsets_out=offo, flux=fo)


def stats(w, j_lo, offsets_fine, offsets_out, flux_out, delta=None, eta=None, rebin=1):
    """FP64 statistics (sums, mean flux, P1D, b_F, beta_F) of ragged flux."""
    cfg = make_cfg(w)
    bins = make_bins(w)
    st = Stats()
    L = lib()
    L.orc_stats_zero(C.byref(st))
    j_lo = np.ascontiguousarray(j_lo, dtype=np.int32)
    offf = np.ascontiguousarray(offsets_fine, dtype=np.int64)
    offo = np.ascontiguousarray(offsets_out, dtype=np.int64)
    fo = np.ascontiguousarray(flux_out, dtype=np.float64)
    dd = None if delta is None else np.ascontiguousarray(delta, dtype=np.float64)
    ee = None if eta is None else np.ascontiguousarray(eta, dtype=np.float64)
    rc = L.orc_stats_accumulate(C.byref(cfg), C.byref(bins), rebin, _p(j_lo, C.c_int32),
                                _p(offf, C.c_int64), _p(offo, C.c_int64), j_lo.size,
                                _p(fo, C.c_double), _p(dd, C.c_double), _p(ee, C.c_double),
                                C.byref(st))
    if rc != 0:
        raise ValueError("oracle stats: bad binning")
    L.orc_stats_finalize(C.byref(bins), C.byref(st))
    nz, nk = bins.n_z, bins.n_k
    arr = lambda a: np.ctypeslib.as_array(a)
    return dict(
        sums=arr(st.sums)[:nz].copy(), p1d_sum=arr(st.p1d_sum)[:nz, :nk].copy(),
        n_seg=arr(st.n_seg)[:nz].copy(), mean_flux=arr(st.mean_flux)[:nz].copy(),
        sigma_f=arr(st.sigma_f)[:nz].copy(), p1d_f=arr(st.p1d_f)[:nz, :nk].copy(),
        p1d_df=arr(st.p1d_df)[:nz, :nk].copy(), b_f=arr(st.b_f)[:nz].copy(),
        beta_f=arr(st.beta_f)[:nz].copy())


# ---------------------------------------------------------------- surrogate MLP
MLP_DIMS = (4, 128, 128, 128, 35)
MLP_NPARAM = 38179


def gelu(x):
    return lib().orc_gelu(float(x))


def mlp_forward(params, x, bf16=False):
    """FP64 forward of the 4-128-128-128-35 GELU MLP; x (n, 4) -> (n, 35).
    bf16: hidden activations rounded to BF16 (the tensor-core operands of
    training)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 4)
    y = np.zeros((x.shape[0], 35))
    lib().orc_mlp_forward(_p(p, C.c_double), _p(x, C.c_double), x.shape[0], _p(y, C.c_double), int(bf16))
    return y


def mlp_loss_grad(params, x, t, bf16=False):
    """Mean squared error and its gradient (FP64) at params; bf16: the
    forward's and backward's tensor-core operands rounded to BF16."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 4)
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1, 35)
    g = np.zeros(MLP_NPARAM)
    loss = lib().orc_mlp_loss_grad(_p(p, C.c_double), _p(x, C.c_double), _p(t, C.c_double),
                                   x.shape[0], _p(g, C.c_double), int(bf16))
    return loss, g


def bf16(x):
    """x rounded to FP32, then to BF16 (nearest even), as a float."""
    return lib().orc_bf16(float(x))


def adam_step(p, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) in place on FP64 arrays."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib().orc_adam_step(_p(p, C.c_double), _p(m, C.c_double), _p(v, C.c_double), _p(g, C.c_double),
                        p.size, int(t), lr, b1, b2, eps)


def qso_draw(q, boxes, stride=1, capacity=None):
    """Quasars from three quasar-density boxes (Sec. 2.2, App. A); q holds n,
    cell, origin, z_box, bias, xi_m5, nbar, nbar_z0, nbar_dz, seed, omega_m.
    Returns ids, positions, and P and u0 of every voxel."""
    n = int(q["n"])
    nv = n ** 3
    cap = nv if capacity is None else int(capacity)
    bx = [np.ascontiguousarray(b, dtype=np.float32).ravel() for b in boxes]
    pout = np.zeros(nv)
    uout = np.zeros(nv)
    ids = np.zeros(max(cap, 1), dtype=np.uint64)
    pos = np.zeros((max(cap, 1), 3))
    og = np.ascontiguousarray(q["origin"], dtype=np.float64)
    zq = np.ascontiguousarray(q["z_box"], dtype=np.float64)
    bl = np.ascontiguousarray(q["bias"], dtype=np.float64)
    nb = np.ascontiguousarray(q["nbar"], dtype=np.float64)
    cnt = lib().orc_qso_draw(q["omega_m"], _p(bx[0], C.c_float), _p(bx[1], C.c_float), _p(bx[2], C.c_float),
                             int(stride), n, q["cell"], _p(og, C.c_double), _p(zq, C.c_double),
                             _p(bl, C.c_double), q["xi_m5"], _p(nb, C.c_double), nb.size, q["nbar_z0"],
                             q["nbar_dz"], int(q["seed"]) & 0xFFFFFFFFFFFFFFFF, _p(pout, C.c_double),
                             _p(uout, C.c_double), _p(ids, C.c_uint64), _p(pos, C.c_double), cap)
    k = min(cnt, cap)
    return dict(count=int(cnt), ids=ids[:k].copy(), pos=pos[:k].copy(), P=pout, u=uout)
