"""GB300-native Lyman-alpha skewer synthesis (arXiv 2310.18996).

Thin ctypes binding over ``libmockskewer.so`` (declared in
``include/mockskewer.h``).  This module only marshals arguments: every step
of the path runs in the library's CUDA kernels.  PyTorch supplies device
memory and the stream.  There is no CPU fallback: importing succeeds without
a GPU, but creating a :class:`Context` needs the compiled library and a CUDA
device and raises otherwise.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

from . import build as _build

MK_OK, MK_EINVAL, MK_ECUDA, MK_ENOMEM, MK_ETIMEOUT, MK_ERANGE = range(6)
FAULT_NONE, FAULT_ALLOC, FAULT_LAUNCH = range(3)
MAX_NODES, MAX_ZBINS, MAX_KBINS, NSUM = 32, 32, 64, 10
STATIC_MAX_SKEWERS = 131072
BOX_PLANAR, BOX_INTERLEAVED, BOX_PADDED, BOX_HALO, BOX_TENSOR = 0, 1, 2, 3, 4
INTERP_TRILINEAR, INTERP_GAUSS7 = 0, 1
GAUSS7_VARIANT = 16  # mk_launch_config: layout + 16 for the Gaussian-kernel instance
STORE_FIELDS, STORE_FLUX, STATS, AUTOTUNE, GRAPH = 1, 2, 4, 8, 16

EXPORTS = ["mk_create", "mk_destroy", "mk_last_error", "mk_set_stream", "mk_sync", "mk_load_box",
           "mk_free_box", "mk_pack_box", "mk_pack_box_padded", "mk_pack_box_halo", "mk_pack_box_tensor", "mk_make_skewers", "mk_run_host", "mk_flux", "mk_stats", "mk_run",
           "mk_set_timing", "mk_last_kernel_ms", "mk_stats_static", "mk_stats_merge", "mk_launch_config",
           "mk_flux_stats",
           "mk_mlp_create", "mk_mlp_destroy", "mk_mlp_set_params", "mk_mlp_get_params", "mk_mlp_forward",
           "mk_mlp_loss_grad", "mk_mlp_train", "mk_surrogate_labels", "mk_surrogate_fit", "mk_tune",
           "mk_fgpa_gauss_moments", "mk_fit_a_bsigma", "mk_tune_ps", "mk_synth_box", "mk_xi_of_pk",
           "mk_lognormal_pk", "mk_draw_qso", "mk_cosmo_eval", "mk_save_skewers", "mk_load_skewers",
           "mk_set_grid_cap", "mk_mlp_adam_step", "mk_set_wait_test", "mk_inject_fault"]


class MkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mockskewer error {code}: {msg}")
        self.code = code


class Cosmo(C.Structure):
    _fields_ = [("omega_m", C.c_double), ("lambda_lya", C.c_double)]


class BoxDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("layout", C.c_int32), ("cell", C.c_double),
                ("origin", C.c_double * 3)]


class SkewerParams(C.Structure):
    _fields_ = [("dr", C.c_double), ("lrf_min", C.c_double), ("lrf_max", C.c_double),
                ("lobs_min", C.c_double), ("n_min", C.c_int32), ("n_max", C.c_int32),
                ("n_fft", C.c_int32), ("seed", C.c_uint32), ("h_p_s", C.POINTER(C.c_double)),
                ("interp", C.c_int32), ("p_s_nodes", C.c_int32), ("h_p_s_z", C.POINTER(C.c_double))]


class FgpaNodes(C.Structure):
    _fields_ = [("count", C.c_int32), ("z", C.c_double * MAX_NODES),
                ("ln_a", C.c_double * MAX_NODES), ("b", C.c_double * MAX_NODES),
                ("c", C.c_double * MAX_NODES)]


class StatBins(C.Structure):
    _fields_ = [("n_z", C.c_int32), ("z_lo", C.c_double), ("dz", C.c_double),
                ("n_k", C.c_int32), ("n_fft", C.c_int32)]


class StatsOut(C.Structure):
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


class SurrogateSpace(C.Structure):
    _fields_ = [("ln_a_min", C.c_double), ("ln_a_max", C.c_double), ("b_min", C.c_double),
                ("b_max", C.c_double), ("c_min", C.c_double), ("c_max", C.c_double),
                ("dln_a_dz_max", C.c_double), ("db_dz_max", C.c_double), ("dc_dz_max", C.c_double)]


class SurrogateNorm(C.Structure):
    _fields_ = [("x_mean", C.c_double * 4), ("x_std", C.c_double * 4),
                ("t_mean", C.c_double * 35), ("t_std", C.c_double * 35), ("calib_skewers", C.c_int64)]


class TuneTarget(C.Structure):
    _fields_ = [("mean_flux", C.c_double * MAX_ZBINS),
                ("p1d", (C.c_double * MAX_KBINS) * MAX_ZBINS),
                ("beta", C.c_double * MAX_ZBINS), ("use_beta", C.c_int32),
                ("k_lo", C.c_int32), ("k_hi", C.c_int32), ("active", C.c_uint32),
                ("tol_mean_flux", C.c_double), ("tol_p1d", C.c_double), ("tol_beta", C.c_double)]


PS_TUNE_MAX_PASSES = 128


class QsoDrawParams(C.Structure):
    _fields_ = [("n", C.c_int32), ("cell", C.c_double), ("origin", C.c_double * 3), ("z_box", C.c_double * 3),
                ("bias", C.c_double * 3), ("xi_m5", C.c_double), ("h_nbar", C.POINTER(C.c_double)),
                ("n_nbar", C.c_int32), ("nbar_z0", C.c_double), ("nbar_dz", C.c_double), ("seed", C.c_uint64)]


class PsTuneReport(C.Structure):
    _fields_ = [("passes", C.c_int32), ("gpu_ms", C.c_double), ("wall_ms", C.c_double),
                ("sigma_f_target", C.c_double * MAX_ZBINS), ("bsigma", C.c_double * MAX_ZBINS),
                ("sigma_g", C.c_double * MAX_ZBINS), ("max_abs_dfbar", C.c_double),
                ("max_rel_p1d", C.c_double), ("max_rel_beta", C.c_double),
                ("max_rel_p1d_pass", C.c_double * PS_TUNE_MAX_PASSES)]


class TuneReport(C.Structure):
    _fields_ = [("converged", C.c_int32), ("passes", C.c_int32), ("iterations", C.c_int32),
                ("gpu_ms", C.c_double), ("wall_ms", C.c_double), ("max_abs_dfbar", C.c_double),
                ("max_rel_p1d", C.c_double), ("max_rel_beta", C.c_double), ("calib_passes", C.c_int32)]


MLP_NPARAM = 38179
TUNE_PLAIN, TUNE_SURROGATE = 0, 1
SKEWER_BYTES = 72  # sizeof(mk_skewer)
QSO_DTYPE = np.dtype([("pos", np.float64, 3), ("id", np.uint64)])  # mk_qso, 32 bytes
SKEWER_DTYPE = np.dtype([("offset", np.int64), ("n", np.int32), ("j_lo", np.int32), ("p0", np.int64, 3),
                         ("step", np.int64, 3), ("id", np.uint64)])  # mk_skewer

_lib = None
_lock = threading.Lock()


def lib():
    """Load libmockskewer.so (building it in-tree if needed); raises on failure."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            vp, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
            P = C.POINTER
            sig = {
                "mk_create": (C.c_int, [P(vp), C.c_int, vp, P(Cosmo)]),
                "mk_destroy": (None, [vp]),
                "mk_last_error": (C.c_char_p, [vp]),
                "mk_set_stream": (C.c_int, [vp, vp]),
                "mk_sync": (C.c_int, [vp]),
                "mk_load_box": (C.c_int, [vp, P(vp), P(BoxDesc), vp, vp]),
                "mk_free_box": (None, [vp]),
                "mk_pack_box": (C.c_int, [vp, i64, vp, vp, vp]),
                "mk_pack_box_padded": (C.c_int, [vp, i32, vp, vp, vp]),
                "mk_pack_box_halo": (C.c_int, [vp, i32, vp, vp, vp]),
                "mk_pack_box_tensor": (C.c_int, [vp, i32, vp, vp, vp]),
                "mk_synth_box": (C.c_int, [vp, i32, C.c_double, C.c_uint64, P(C.c_double), i32, C.c_double,
                                           i32, vp, vp, vp]),
                "mk_run_host": (C.c_int, [vp, vp, vp, i64, P(SkewerParams), P(FgpaNodes), P(StatBins), u32,
                                          i32, vp, i64, P(i64), P(StatsOut)]),
                "mk_make_skewers": (C.c_int, [vp, vp, vp, i64, P(SkewerParams), vp, vp, vp, vp,
                                              i64, P(i64)]),
                "mk_flux": (C.c_int, [vp, P(SkewerParams), vp, i64, vp, vp, P(FgpaNodes), i32, vp,
                                      vp, i64]),
                "mk_stats": (C.c_int, [vp, P(SkewerParams), vp, i64, vp, vp, i32, vp, vp,
                                       P(StatBins), P(StatsOut)]),
                "mk_run": (C.c_int, [vp, vp, vp, i64, P(SkewerParams), P(FgpaNodes), P(StatBins),
                                     u32, vp, vp, vp, vp, vp, i64, P(StatsOut)]),
                "mk_stats_static": (C.c_int, [vp, P(SkewerParams), vp, i64, vp, vp, i32, vp, vp,
                                              P(StatBins), P(StatsOut)]),
                "mk_stats_merge": (C.c_int, [P(StatsOut), i32, P(StatBins), P(StatsOut)]),
                "mk_launch_config": (C.c_int, [vp, i32, i32, i32, u32, P(i32), P(i32)]),
                "mk_flux_stats": (C.c_int, [vp, P(SkewerParams), vp, i64, vp, vp, vp, P(FgpaNodes),
                                            P(StatBins), P(StatsOut)]),
                "mk_mlp_create": (C.c_int, [vp, P(vp), i64, C.c_uint64]),
                "mk_mlp_destroy": (None, [vp]),
                "mk_mlp_set_params": (C.c_int, [vp, P(C.c_float)]),
                "mk_mlp_get_params": (C.c_int, [vp, P(C.c_float), P(C.c_uint16)]),
                "mk_mlp_forward": (C.c_int, [vp, vp, i64, vp]),
                "mk_mlp_loss_grad": (C.c_int, [vp, vp, vp, i64, P(C.c_double), P(C.c_float)]),
                "mk_mlp_adam_step": (C.c_int, [vp, vp, C.c_float]),
                "mk_mlp_train": (C.c_int, [vp, vp, vp, i64, i32, i32, C.c_float, C.c_uint64,
                                           P(C.c_double)]),
                "mk_surrogate_labels": (C.c_int, [vp, P(SkewerParams), vp, i64, vp, vp, vp, P(StatBins),
                                                  P(SurrogateSpace), i32, C.c_uint64, P(C.c_double),
                                                  P(C.c_double), P(i64)]),
                "mk_surrogate_fit": (C.c_int, [vp, P(C.c_double), P(C.c_double), i64, i32, i32,
                                               C.c_float, C.c_uint64, P(SurrogateNorm),
                                               P(C.c_double)]),
                "mk_tune": (C.c_int, [vp, P(SkewerParams), vp, i64, vp, vp, vp, P(StatBins),
                                      P(TuneTarget), i32, vp, P(SurrogateNorm), i32, P(FgpaNodes),
                                      P(TuneReport)]),
                "mk_fgpa_gauss_moments": (C.c_int, [C.c_double, C.c_double, P(C.c_double), P(C.c_double)]),
                "mk_fit_a_bsigma": (C.c_int, [C.c_double, C.c_double, P(C.c_double), P(C.c_double)]),
                "mk_tune_ps": (C.c_int, [vp, vp, vp, i64, P(SkewerParams), P(StatBins), P(TuneTarget), i32,
                                         i32, vp, vp, P(C.c_double), P(FgpaNodes), P(PsTuneReport)]),
                "mk_xi_of_pk": (C.c_int, [P(C.c_double), i32, C.c_double, P(C.c_double), i32, P(C.c_double)]),
                "mk_lognormal_pk": (C.c_int, [P(C.c_double), i32, C.c_double, C.c_double, P(C.c_double)]),
                "mk_draw_qso": (C.c_int, [vp, P(QsoDrawParams), P(vp), i32, vp, i64, P(i64)]),
                "mk_cosmo_eval": (C.c_int, [vp, C.c_double, P(C.c_double), P(C.c_double)]),
                "mk_save_skewers": (C.c_int, [vp, C.c_char_p, vp, i64, vp, vp, vp]),
                "mk_load_skewers": (C.c_int, [vp, C.c_char_p, vp, i64, vp, vp, vp, i64, P(i64), P(i64)]),
                "mk_set_grid_cap": (C.c_int, [vp, i32]),
                "mk_set_wait_test": (C.c_int, [vp, i32]),
                "mk_inject_fault": (C.c_int, [vp, i32]),
                "mk_set_timing": (C.c_int, [vp, C.c_int]),
                "mk_last_kernel_ms": (C.c_int, [vp, P(C.c_double)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


# ------------------------------------------------------------------ struct builders
def skewer_params(w):
    ps = np.ascontiguousarray(w["p_s"], dtype=np.float64)
    p = SkewerParams(dr=w["dr"], lrf_min=w["lrf_min"], lrf_max=w["lrf_max"],
                     lobs_min=w.get("lobs_min", 0.0), n_min=w.get("n_min", 0),
                     n_max=w.get("n_max", 0), n_fft=w["n_fft"],
                     seed=w["seed_noise"] & 0xFFFFFFFF,
                     h_p_s=ps.ctypes.data_as(C.POINTER(C.c_double)), interp=w.get("interp", 0))
    psz = np.ascontiguousarray(w.get("p_s_z", []), dtype=np.float64)
    if psz.size >= 2:  # one P_s table per redshift node
        if ps.size != psz.size * (w["n_fft"] // 2 + 1):
            raise ValueError("p_s needs one table of n_fft/2 + 1 values per p_s_z node")
        p.p_s_nodes = psz.size
        p.h_p_s_z = psz.ctypes.data_as(C.POINTER(C.c_double))
    p._keep = (ps, psz)
    return p


def fgpa_nodes(w):
    nd = FgpaNodes()
    z = list(w["node_z"])
    nd.count = len(z)
    for i in range(len(z)):
        nd.z[i], nd.ln_a[i], nd.b[i], nd.c[i] = z[i], w["node_ln_a"][i], w["node_b"][i], w["node_c"][i]
    return nd


def stat_bins(w):
    return StatBins(n_z=w["n_zbins"], z_lo=w["z_bin_lo"], dz=w["dz_bin"], n_k=w["n_kbins"],
                    n_fft=w["n_fft_p1d"])


def stats_dict(st, n_z, n_k):
    a = np.ctypeslib.as_array
    return dict(sums=a(st.sums)[:n_z].copy(), p1d_sum=a(st.p1d_sum)[:n_z, :n_k].copy(),
                n_seg=a(st.n_seg)[:n_z].copy(), mean_flux=a(st.mean_flux)[:n_z].copy(),
                sigma_f=a(st.sigma_f)[:n_z].copy(), p1d_f=a(st.p1d_f)[:n_z, :n_k].copy(),
                p1d_df=a(st.p1d_df)[:n_z, :n_k].copy(), b_f=a(st.b_f)[:n_z].copy(),
                beta_f=a(st.beta_f)[:n_z].copy())


RAW_KEYS = ("sums", "p1d_sum", "n_seg")


def raw_sums_vector(st):
    """The raw sums of a statistics dict (sums, p1d_sum, n_seg of its n_z bins)
    as one flat FP64 array: what ranks exchange before mk_stats_merge."""
    return np.concatenate([np.asarray(st[k], dtype=np.float64).ravel() for k in RAW_KEYS])


def raw_sums_from_vector(v, n_z, n_k):
    v = np.asarray(v, dtype=np.float64)
    a, b = n_z * NSUM, n_z * NSUM + n_z * n_k
    return {"sums": v[:a].reshape(n_z, NSUM), "p1d_sum": v[a:b].reshape(n_z, n_k), "n_seg": v[b:b + n_z]}


def stats_merge(parts, w):
    """mk_stats_merge: statistics of the union of catalogue parts from each
    part's raw sums (dicts with sums, p1d_sum, n_seg), added in list order."""
    b = stat_bins(w)
    arr = (StatsOut * len(parts))()
    for i, prt in enumerate(parts):
        a = np.ctypeslib.as_array
        a(arr[i].sums)[:b.n_z] = prt["sums"]
        a(arr[i].p1d_sum)[:b.n_z, :b.n_k] = prt["p1d_sum"]
        a(arr[i].n_seg)[:b.n_z] = prt["n_seg"]
    out = StatsOut()
    rc = lib().mk_stats_merge(arr, len(parts), C.byref(b), C.byref(out))
    if rc != MK_OK:
        raise MkError(rc, "mk_stats_merge: bad arguments")
    return stats_dict(out, b.n_z, b.n_k)


def merge_stats_across_ranks(st, w, dist, device="cpu"):
    """Catalogue-wide statistics of a run split over the ranks of a process
    group: one all-gather of every rank's raw sums (n_z (11 + n_k) FP64
    values), then mk_stats_merge over the parts in rank order, so that every
    rank gets the same result whatever the collective's summation order."""
    import torch

    b = stat_bins(w)
    v = torch.from_numpy(raw_sums_vector(st)).to(device)
    parts = [torch.empty_like(v) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, v)
    return stats_merge([raw_sums_from_vector(p.cpu().numpy(), b.n_z, b.n_k) for p in parts], w)


def catalogue_tensor(pos, ids, device="cuda"):
    """mk_qso records (pos FP64 x3, id) as a uint8 device tensor."""
    import torch

    rec = np.zeros(len(ids), dtype=QSO_DTYPE)
    rec["pos"] = np.asarray(pos, dtype=np.float64)
    rec["id"] = np.asarray(ids, dtype=np.uint64)
    return torch.from_numpy(rec.view(np.uint8)).to(device)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ objects
class Box:
    def __init__(self, ctx, handle, desc, keep):
        self._ctx, self.handle, self.desc, self._keep = ctx, handle, desc, keep

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mk_free_box(self.handle)
            self.handle = None


class Context:
    """A library context on one CUDA device; calls run on torch's current stream."""

    def __init__(self, device=0, omega_m=0.3147, lambda_lya=1215.67):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("mockskewer needs a CUDA device (no CPU fallback)")
        self._torch = torch
        self.device = device
        L = lib()
        h = C.c_void_p()
        cos = Cosmo(omega_m=omega_m, lambda_lya=lambda_lya)
        with torch.cuda.device(device):
            rc = L.mk_create(C.byref(h), device, C.c_void_p(torch.cuda.current_stream().cuda_stream),
                             C.byref(cos))
        if rc != MK_OK:
            raise MkError(rc, "mk_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().mk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != MK_OK:
            raise MkError(rc, lib().mk_last_error(self.h).decode())

    def _stream(self):
        s = self._torch.cuda.current_stream(self.device).cuda_stream
        self._check(lib().mk_set_stream(self.h, C.c_void_p(s)))

    def sync(self):
        self._check(lib().mk_sync(self.h))

    def set_timing(self, on=True):
        self._check(lib().mk_set_timing(self.h, 1 if on else 0))

    def launch_config(self, n_fft, layout=BOX_INTERLEAVED, big_box=False, flags=STATS):
        """(threads, occupancy, tuned) of the fused kernel variant."""
        t, o = C.c_int32(), C.c_int32()
        rc = lib().mk_launch_config(self.h, n_fft, layout, 1 if big_box else 0, flags, C.byref(t), C.byref(o))
        if rc not in (MK_OK, MK_ERANGE):
            self._check(rc)
        return t.value, o.value, rc == MK_OK

    def set_grid_cap(self, max_ctas=0):
        """At most max_ctas CTAs for the persistent kernels (0: no cap)."""
        self._check(lib().mk_set_grid_cap(self.h, int(max_ctas)))

    def inject_fault(self, kind):
        """Test hook: the next step of this kind fails once (mk_inject_fault)."""
        self._check(lib().mk_inject_fault(self.h, int(kind)))

    def set_wait_test(self, on):
        """Test hook: the tuning pass's bounded device wait runs out (mk_set_wait_test)."""
        self._check(lib().mk_set_wait_test(self.h, int(bool(on))))

    def last_kernel_ms(self):
        ms = C.c_double()
        self._check(lib().mk_last_kernel_ms(self.h, C.byref(ms)))
        return ms.value

    # boxes
    def load_box(self, w, delta, eta=None, layout=None):
        """Register a box (torch float32 tensors on the device) with the recipe's geometry."""
        if layout is None:
            layout = BOX_PLANAR if eta is not None else BOX_INTERLEAVED
        desc = BoxDesc(n=w["n"], layout=layout, cell=w["cell"])
        for d in range(3):
            desc.origin[d] = w["origin"][d]
        h = C.c_void_p()
        self._check(lib().mk_load_box(self.h, C.byref(h), C.byref(desc), _ptr(delta), _ptr(eta)))
        return Box(self, h, desc, (delta, eta))

    def pack_box(self, delta, eta, padded=False, halo=False):
        """Interleaved (delta, eta) pairs; padded=True: the MK_BOX_PADDED layout
        ((n+1)^3 pairs with a periodic ghost layer), for load_box(..., layout=BOX_PADDED);
        halo=True: the MK_BOX_HALO layout ((n+6)^3 pairs, periodic margin of 3)."""
        torch = self._torch
        self._stream()
        if padded or halo:
            n = round(delta.numel() ** (1.0 / 3.0))
            m = n + (6 if halo else 1)
            out = torch.empty(2 * m ** 3, dtype=torch.float32, device=delta.device)
            fn = lib().mk_pack_box_halo if halo else lib().mk_pack_box_padded
            self._check(fn(self.h, n, _ptr(delta), _ptr(eta), _ptr(out)))
            return out
        out = torch.empty(delta.numel() * 2, dtype=torch.float32, device=delta.device)
        self._check(lib().mk_pack_box(self.h, delta.numel(), _ptr(delta), _ptr(eta), _ptr(out)))
        return out

    def pack_box_tensor(self, delta, eta6):
        """delta (n^3) and the six eta_pq boxes ((6, n, n, n): xx, yy, zz, xy, xz, yz)
        into the MK_BOX_TENSOR layout, for load_box(..., layout=BOX_TENSOR)."""
        torch = self._torch
        n = round(delta.numel() ** (1.0 / 3.0))
        out = torch.empty(8 * (n + 1) ** 3, dtype=torch.float32, device=delta.device)
        self._stream()
        self._check(lib().mk_pack_box_tensor(self.h, n, _ptr(delta), _ptr(eta6), _ptr(out)))
        return out

    def synth_box(self, n, cell, seed, pk, dk, layout=BOX_PADDED, work=None):
        """Gaussian delta and eta boxes of side n (Sec. 2.1) from the P(k) table
        pk (at k = i dk) and a seed, in `layout` (BOX_INTERLEAVED, BOX_PADDED,
        BOX_HALO or BOX_TENSOR), for load_box(..., layout=layout)."""
        torch = self._torch
        dev = torch.device("cuda", self.device)
        pk = np.ascontiguousarray(pk, dtype=np.float64)
        side, stride = {BOX_PLANAR: (n, 1), BOX_INTERLEAVED: (n, 2), BOX_PADDED: (n + 1, 2), BOX_HALO: (n + 6, 2),
                        BOX_TENSOR: (n + 1, 8)}[layout]
        if work is None:
            work = torch.empty(2 * n ** 3, dtype=torch.float32, device=dev)
        out = work if layout == BOX_INTERLEAVED else torch.empty(stride * side ** 3, dtype=torch.float32,
                                                                   device=dev)
        spec = torch.empty(2 * n ** 3, dtype=torch.float32, device=dev) if layout == BOX_TENSOR else None
        self._stream()
        self._check(lib().mk_synth_box(self.h, n, cell, int(seed) & 0xFFFFFFFFFFFFFFFF, _dp(pk), pk.size, dk,
                                       layout, _ptr(work), _ptr(spec), _ptr(out)))
        return out

    def save_skewers(self, path, r, n_sk):
        """Write stored pre-FGPA skewers (make_skewers' dict) to `path`."""
        self._stream()
        self._check(lib().mk_save_skewers(self.h, os.fsencode(path), _ptr(r["sk"]), n_sk, _ptr(r["offsets"]),
                                          _ptr(r["delta"]), _ptr(r["eta"])))

    def load_skewers(self, path):
        """Read a file of save_skewers into new device tensors: dict(sk, offsets,
        delta, eta, total) and the skewer count."""
        torch = self._torch
        ns, tp = C.c_int64(), C.c_int64()
        self._check(lib().mk_load_skewers(self.h, os.fsencode(path), None, 0, None, None, None, 0, C.byref(ns),
                                          C.byref(tp)))
        dev = torch.device("cuda", self.device)
        r = dict(sk=torch.empty(max(ns.value, 1) * SKEWER_BYTES, dtype=torch.uint8, device=dev),
                 offsets=torch.empty(ns.value + 1, dtype=torch.int64, device=dev),
                 delta=torch.empty(max(tp.value, 1), dtype=torch.float32, device=dev),
                 eta=torch.empty(max(tp.value, 1), dtype=torch.float32, device=dev), total=tp.value)
        self._stream()
        self._check(lib().mk_load_skewers(self.h, os.fsencode(path), _ptr(r["sk"]), ns.value, _ptr(r["offsets"]),
                                          _ptr(r["delta"]), _ptr(r["eta"]), tp.value, C.byref(ns), C.byref(tp)))
        return r, ns.value

    def cosmo_eval(self, z):
        """(D_C(z), G(z)) of the context's cosmology."""
        dc, g = C.c_double(), C.c_double()
        self._check(lib().mk_cosmo_eval(self.h, z, C.byref(dc), C.byref(g)))
        return dc.value, g.value

    def draw_qso(self, q, boxes, stride=2, capacity=None):
        """Quasars from three quasar-density boxes (Sec. 2.2, App. A); q: dict with
        n, cell, origin, z_box, bias, xi_m5, nbar, nbar_z0, nbar_dz, seed.  boxes:
        three device tensors (stride 2: mk_synth_box interleaved pairs).  Returns
        (catalogue tensor of mk_qso records, count)."""
        torch = self._torch
        n = int(q["n"])
        cap = int(capacity) if capacity is not None else max(16, int(4 * n ** 3 * max(q["nbar"]) * q["cell"] ** 3) + 4096)
        out = torch.empty(max(cap, 1) * QSO_DTYPE.itemsize, dtype=torch.uint8, device=boxes[0].device)
        nb = np.ascontiguousarray(q["nbar"], dtype=np.float64)
        p = QsoDrawParams(n=n, cell=q["cell"], xi_m5=q["xi_m5"], h_nbar=_dp(nb), n_nbar=nb.size,
                          nbar_z0=q["nbar_z0"], nbar_dz=q["nbar_dz"], seed=int(q["seed"]) & 0xFFFFFFFFFFFFFFFF)
        for d in range(3):
            p.origin[d], p.z_box[d], p.bias[d] = q["origin"][d], q["z_box"][d], q["bias"][d]
        ptrs = (C.c_void_p * 3)(*[b.data_ptr() for b in boxes])
        cnt = C.c_int64()
        self._stream()
        rc = lib().mk_draw_qso(self.h, C.byref(p), ptrs, stride, _ptr(out), cap, C.byref(cnt))
        self._check(rc)
        return out[: cnt.value * QSO_DTYPE.itemsize], cnt.value

    # skewers
    def plan(self, box, qso, n_qso, w):
        """Geometry only: (skewer records, offsets, total pixels)."""
        torch = self._torch
        sk = torch.empty(max(n_qso, 1) * SKEWER_BYTES, dtype=torch.uint8, device=qso.device)
        off = torch.empty(n_qso + 1, dtype=torch.int64, device=qso.device)
        total = C.c_int64()
        p = skewer_params(w)
        self._stream()
        self._check(lib().mk_make_skewers(self.h, box.handle, _ptr(qso), n_qso, C.byref(p), _ptr(sk),
                                          _ptr(off), None, None, 0, C.byref(total)))
        return sk, off, total.value

    def make_skewers(self, box, qso, n_qso, w):
        """Pre-FGPA skewers: dict(sk, offsets, delta, eta) as device tensors."""
        torch = self._torch
        sk, off, total = self.plan(box, qso, n_qso, w)
        d = torch.empty(max(total, 1), dtype=torch.float32, device=qso.device)
        e = torch.empty(max(total, 1), dtype=torch.float32, device=qso.device)
        p = skewer_params(w)
        self._stream()
        self._check(lib().mk_make_skewers(self.h, box.handle, _ptr(qso), n_qso, C.byref(p), _ptr(sk),
                                          _ptr(off), _ptr(d), _ptr(e), total, None))
        return dict(sk=sk, offsets=off, delta=d[:total], eta=e[:total], total=total)

    def flux(self, w, sk, n_sk, delta, eta, rebin=1, nodes=None, capacity=None):
        torch = self._torch
        total = delta.numel()
        cap = total // rebin if capacity is None else capacity
        f = torch.empty(max(cap, 1), dtype=torch.float32, device=delta.device)
        off = torch.empty(n_sk + 1, dtype=torch.int64, device=delta.device)
        p = skewer_params(w)
        nd = fgpa_nodes(w) if nodes is None else nodes
        self._stream()
        self._check(lib().mk_flux(self.h, C.byref(p), _ptr(sk), n_sk, _ptr(delta), _ptr(eta), C.byref(nd),
                                  rebin, _ptr(f), _ptr(off), cap))
        return f, off

    def stats(self, w, sk, n_sk, offsets_out, flux, rebin=1, delta=None, eta=None):
        p = skewer_params(w)
        b = stat_bins(w)
        st = StatsOut()
        self._stream()
        self._check(lib().mk_stats(self.h, C.byref(p), _ptr(sk), n_sk, _ptr(offsets_out), _ptr(flux),
                                   rebin, _ptr(delta), _ptr(eta), C.byref(b), C.byref(st)))
        return stats_dict(st, b.n_z, b.n_k)

    def flux_stats(self, w, sk, n_sk, offsets, delta, eta, nodes=None):
        """Tuning pass: FGPA of stored fields and their statistics (no flux stored)."""
        p = skewer_params(w)
        nd = fgpa_nodes(w) if nodes is None else nodes
        b = stat_bins(w)
        st = StatsOut()
        self._stream()
        self._check(lib().mk_flux_stats(self.h, C.byref(p), _ptr(sk), n_sk, _ptr(offsets), _ptr(delta),
                                        _ptr(eta), C.byref(nd), C.byref(b), C.byref(st)))
        return stats_dict(st, b.n_z, b.n_k)

    def run(self, box, qso, n_qso, w, flags=STATS, capacity=0, outputs=None, nodes=None):
        """The fused path; returns (stats dict or None, dict of device tensors)."""
        torch = self._torch
        o = dict(outputs or {})
        if "sk" not in o:
            o["sk"] = torch.empty(max(n_qso, 1) * SKEWER_BYTES, dtype=torch.uint8, device=qso.device)
            o["offsets"] = torch.empty(n_qso + 1, dtype=torch.int64, device=qso.device)
        if (flags & (STORE_FIELDS | STORE_FLUX)) and capacity == 0:
            _, _, capacity = self.plan(box, qso, n_qso, w)
        if flags & STORE_FIELDS and "delta" not in o:
            o["delta"] = torch.empty(max(capacity, 1), dtype=torch.float32, device=qso.device)
            o["eta"] = torch.empty(max(capacity, 1), dtype=torch.float32, device=qso.device)
        if flags & STORE_FLUX and "flux" not in o:
            o["flux"] = torch.empty(max(capacity, 1), dtype=torch.float32, device=qso.device)
        p = skewer_params(w)
        nd = fgpa_nodes(w) if nodes is None else nodes
        b = stat_bins(w)
        st = StatsOut()
        self._stream()
        self._check(lib().mk_run(self.h, box.handle, _ptr(qso), n_qso, C.byref(p), C.byref(nd),
                                 C.byref(b), flags, _ptr(o["sk"]), _ptr(o["offsets"]),
                                 _ptr(o.get("delta")), _ptr(o.get("eta")), _ptr(o.get("flux")),
                                 capacity, C.byref(st)))
        return (stats_dict(st, b.n_z, b.n_k) if flags & STATS else None), o

    def run_host(self, box, host_qso, n_qso, w, host_flux, n_chunks=8, stats=True, nodes=None):
        """The fused pass from a host catalogue to a host flux array, pipelined in
        n_chunks slices (mk_run_host).  host_qso: catalogue_tensor bytes in
        page-locked host memory; host_flux: page-locked float32 tensor of at
        least the total pixel count.  Returns (stats dict or None, total pixels)."""
        p = skewer_params(w)
        nd = fgpa_nodes(w) if nodes is None else nodes
        b = stat_bins(w)
        st = StatsOut()
        total = C.c_int64()
        self._stream()
        self._check(lib().mk_run_host(self.h, box.handle, _ptr(host_qso), n_qso, C.byref(p), C.byref(nd),
                                      C.byref(b), STATS if stats else 0, n_chunks, _ptr(host_flux),
                                      host_flux.numel(), C.byref(total), C.byref(st)))
        return (stats_dict(st, b.n_z, b.n_k) if stats else None), total.value


def skewer_records(sk, n):
    """Host view of mk_skewer records (offset, n, j_lo, p0[3], step[3], id)."""
    return sk[: n * SKEWER_BYTES].cpu().numpy().view(SKEWER_DTYPE)


# ------------------------------------------------------------------ surrogate and tuning
def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Mlp:
    """The surrogate MLP (4-128-128-128-35, GELU) bound to a Context."""

    def __init__(self, ctx, max_batch=4096, seed=0):
        self.ctx = ctx
        h = C.c_void_p()
        ctx._stream()
        ctx._check(lib().mk_mlp_create(ctx.h, C.byref(h), max_batch, seed))
        self.h = h
        self.max_batch = max_batch

    def close(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.mk_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == MLP_NPARAM
        self.ctx._stream()
        self.ctx._check(lib().mk_mlp_set_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float))))

    def get_params(self):
        p = np.zeros(MLP_NPARAM, np.float32)
        b = np.zeros(MLP_NPARAM, np.uint16)
        self.ctx._stream()
        self.ctx._check(lib().mk_mlp_get_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float)),
                                                b.ctypes.data_as(C.POINTER(C.c_uint16))))
        return p, b

    def forward(self, x):
        torch = self.ctx._torch
        y = torch.empty((x.shape[0], 35), dtype=torch.float32, device=x.device)
        self.ctx._stream()
        self.ctx._check(lib().mk_mlp_forward(self.h, _ptr(x), x.shape[0], _ptr(y)))
        return y

    def loss_grad(self, x, t):
        g = np.zeros(MLP_NPARAM, np.float32)
        loss = C.c_double()
        self.ctx._stream()
        self.ctx._check(lib().mk_mlp_loss_grad(self.h, _ptr(x), _ptr(t), x.shape[0], C.byref(loss),
                                               g.ctypes.data_as(C.POINTER(C.c_float))))
        return loss.value, g

    def adam_step(self, grad, lr):
        """One Adam step with a device gradient (MLP_NPARAM float32 values)."""
        self.ctx._stream()
        self.ctx._check(lib().mk_mlp_adam_step(self.h, _ptr(grad), lr))

    def train(self, x, t, batch=2048, epochs=10, lr=2e-3, seed=0):
        losses = np.zeros(max(epochs, 1))
        self.ctx._stream()
        self.ctx._check(lib().mk_mlp_train(self.h, _ptr(x), _ptr(t), x.shape[0], batch, epochs, lr, seed,
                                           _dp(losses)))
        return losses[:epochs]

    def fit(self, hx, ht, batch=2048, epochs=10, lr=2e-3, seed=0):
        """Normalise raw samples, train; returns (SurrogateNorm, per-epoch loss)."""
        hx = np.ascontiguousarray(hx, dtype=np.float64)
        ht = np.ascontiguousarray(ht, dtype=np.float64)
        norm = SurrogateNorm()
        losses = np.zeros(max(epochs, 1))
        self.ctx._stream()
        self.ctx._check(lib().mk_surrogate_fit(self.h, _dp(hx), _dp(ht), hx.shape[0], batch, epochs, lr, seed,
                                               C.byref(norm), _dp(losses)))
        return norm, losses[:epochs]


def surrogate_labels(ctx, w, sk, n_sk, offsets, delta, eta, n_draws, seed=0, space=None, slopes=None):
    """Raw surrogate training samples x (n, 4) and t (n, 35) from tuning passes.
    slopes: (d ln a/dz, db/dz, dc/dz) maxima for linear-in-z draws (None: constant)."""
    sp = space or SurrogateSpace(ln_a_min=math.log(1e-3), ln_a_max=math.log(3.0), b_min=1.0, b_max=2.2,
                                 c_min=0.5, c_max=1.5)
    if slopes is not None:
        sp.dln_a_dz_max, sp.db_dz_max, sp.dc_dz_max = slopes
    p = skewer_params(w)
    b = stat_bins(w)
    hx = np.zeros((n_draws * b.n_z, 4))
    ht = np.zeros((n_draws * b.n_z, 35))
    cnt = C.c_int64()
    ctx._stream()
    ctx._check(lib().mk_surrogate_labels(ctx.h, C.byref(p), _ptr(sk), n_sk, _ptr(offsets), _ptr(delta),
                                         _ptr(eta), C.byref(b), C.byref(sp), n_draws, seed, _dp(hx), _dp(ht),
                                         C.byref(cnt)))
    return hx[:cnt.value], ht[:cnt.value]


def tune(ctx, w, sk, n_sk, offsets, delta, eta, target, nodes, method=TUNE_PLAIN, mlp=None, norm=None,
         max_passes=60):
    """Run mk_tune; returns (FgpaNodes, TuneReport)."""
    p = skewer_params(w)
    b = stat_bins(w)
    rep = TuneReport()
    nd = FgpaNodes()
    C.pointer(nd)[0] = nodes
    ctx._stream()
    ctx._check(lib().mk_tune(ctx.h, C.byref(p), _ptr(sk), n_sk, _ptr(offsets), _ptr(delta), _ptr(eta),
                             C.byref(b), C.byref(target), method, mlp.h if mlp else None,
                             C.byref(norm) if norm is not None else None, max_passes, C.byref(nd),
                             C.byref(rep)))
    return nd, rep


def fgpa_gauss_moments(a, s):
    """(F-bar, sigma_F) of exp(-a exp(s xi)), xi ~ N(0, 1) (Sec. 2.6)."""
    f, sf = C.c_double(), C.c_double()
    rc = lib().mk_fgpa_gauss_moments(a, s, C.byref(f), C.byref(sf))
    if rc != MK_OK:
        raise MkError(rc, "mk_fgpa_gauss_moments: bad argument")
    return f.value, sf.value


def fit_a_bsigma(fbar, sigma_f):
    """(a, b sigma_g) reaching (F-bar, sigma_F) for a Gaussian field (Sec. 2.6)."""
    a, s = C.c_double(), C.c_double()
    rc = lib().mk_fit_a_bsigma(fbar, sigma_f, C.byref(a), C.byref(s))
    if rc != MK_OK:
        raise MkError(rc, "mk_fit_a_bsigma: no (a, b sigma_g) reaches this mean flux and sigma_F")
    return a.value, s.value


def tune_ps(ctx, box, qso, n_qso, w, target, p_s0, n_outer=5, n_inner=10):
    """Run mk_tune_ps (the Sec. 2.6 procedure); returns (FgpaNodes, P_S tables
    of shape (n_z, n_fft/2 + 1), PsTuneReport)."""
    torch = ctx._torch
    p = skewer_params(w)
    b = stat_bins(w)
    ps = np.array(p_s0, dtype=np.float64).reshape(b.n_z, w["n_fft"] // 2 + 1).copy()
    sk = torch.empty(max(n_qso, 1) * SKEWER_BYTES, dtype=torch.uint8, device=qso.device)
    off = torch.empty(n_qso + 1, dtype=torch.int64, device=qso.device)
    nd = FgpaNodes()
    rep = PsTuneReport()
    ctx._stream()
    ctx._check(lib().mk_tune_ps(ctx.h, box.handle, _ptr(qso), n_qso, C.byref(p), C.byref(b), C.byref(target),
                                n_outer, n_inner, _ptr(sk), _ptr(off), _dp(ps), C.byref(nd), C.byref(rep)))
    return nd, ps, rep


def xi_of_pk(pk, dk, r):
    """xi(r) of a tabulated isotropic power spectrum (host)."""
    pk = np.ascontiguousarray(pk, dtype=np.float64)
    r = np.ascontiguousarray(np.atleast_1d(r), dtype=np.float64)
    out = np.zeros(r.size)
    rc = lib().mk_xi_of_pk(_dp(pk), pk.size, dk, _dp(r), r.size, _dp(out))
    if rc != MK_OK:
        raise MkError(rc, "mk_xi_of_pk: bad argument")
    return out


def lognormal_pk(pk, dk, B):
    """Spectrum of the Gaussian field whose exponential has correlation B xi(r) (host)."""
    pk = np.ascontiguousarray(pk, dtype=np.float64)
    out = np.zeros(pk.size)
    rc = lib().mk_lognormal_pk(_dp(pk), pk.size, dk, B, _dp(out))
    if rc != MK_OK:
        raise MkError(rc, "mk_lognormal_pk: bad argument or 1 + B xi <= 0")
    return out
