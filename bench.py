#!/usr/bin/env python
"""Skewer-synthesis throughput on GB300: skewer pixels per second.

A step is one pass of the whole path over the 1024^3-cell box and its 1M-quasar
catalogue (skewers of 200-1500 pixels): geometry, trilinear gather, growth,
small-scale field, FGPA, flux store and FP64 statistics, issued through the
C-ABI (mk_run).  The box (8.6 GB) and catalogue are resident in HBM when the
timed region starts; the box is larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank synthesises
its own 1M-quasar catalogue on its own copy of the box (weak scaling, no
data-path collective).  --impl reference times the FP64 CPU oracle on bounded
samples of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import skewer_inputs as si  # noqa: E402

WORKLOAD = "batched"
METRIC = "skewer_pixels_per_s"
UNIT = "pixels/s"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def profiled_traffic(total_px):
    """DRAM bytes per fused-kernel launch from the committed ncu record, scaled
    by pixels, or None when the kernel sources changed since it was taken."""
    import hashlib

    p = os.path.join(ROOT, "profiles", "k_skewer_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    h = hashlib.sha256()
    for src in rec["sources"]:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != rec["sha256"]:
        return None
    return rec["dram_bytes_per_pixel"] * total_px


def workload_config(w, n_q):
    """The `config` of both arms' JSON lines (the same workload)."""
    return {"workload": f"{w['n']}^3 box (delta+eta FP32 pairs, periodic ghost layer), {n_q} quasars "
                        "z 2.04-4.0, 200-1500 px skewers, N_fft 256",
            "skewers_per_gpu": n_q, "l2": "inputs larger than L2 (8.6 GB box)",
            "outputs": "flux + FP64 statistics (mean flux, sigma_F, P1D, b_F, beta_F in 12 z bins)"}


def profiled_kernel_record():
    """The fused kernel's committed ncu record (instruction counts per pixel,
    issue activity), or None when the kernel sources changed since it was taken."""
    import hashlib

    p = os.path.join(ROOT, "profiles", "k_skewer_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    h = hashlib.sha256()
    for src in rec["sources"]:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    return rec if h.hexdigest() == rec["sha256"] else None


def algorithmic_bytes(pos, npix, w):
    """Bytes a launch must move: each skewer's distinct trilinear voxels (8 B,
    a (delta, eta) pair), its flux (4 B/pixel), catalogue and record traffic."""
    u = np.abs(pos / np.linalg.norm(pos, axis=1, keepdims=True))
    vox = 4.0 * w["dr"] * u.sum(axis=1) / w["cell"] * npix + 8.0 * (npix > 0)
    per_skewer = 32 + 72 + 72 + 16  # catalogue read, record write + read, offsets
    return float(np.sum(vox) * 8.0 + np.sum(npix) * 4.0 + per_skewer * len(npix))


# ---------------------------------------------------------------- oracle legs
def oracle_rate(w, dh, eh, pos, ids, target_s, threads):
    """Oracle pixels/s on a bounded sample (skewers taken in catalogue order)."""
    import oracle

    # calibrate the time per skewer (fields, flux and statistics) on a few
    # skewers, then time a sample sized to take about target_s
    n0 = 64
    t = time.perf_counter()
    o = oracle.run_skewers(w, dh, eh, pos[:n0], ids[:n0], n_threads=threads)
    oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    per_sk = (time.perf_counter() - t) / n0
    n = int(min(len(ids) - n0, max(n0, target_s / max(per_sk, 1e-9))))
    t = time.perf_counter()
    o = oracle.run_skewers(w, dh, eh, pos[n0:n0 + n], ids[n0:n0 + n], n_threads=threads)
    st = oracle.stats(w, o["j_lo"], o["offsets"], o["offsets_out"], o["flux"], o["delta"], o["eta"])
    dt = time.perf_counter() - t
    px = int(o["offsets"][-1])
    return px / dt, px, n, dt


def rank_catalogue(w, rank):
    """Rank `rank`'s own quasars: a catalogue seed of its own and ids offset by
    rank * n_q, so that ranks synthesise disjoint sets of skewers (weak scaling)
    on identical box replicas."""
    w = dict(w)
    w["seed_cat"] = w["seed_cat"] + 7919 * rank
    pos, ids = si.catalogue(w)
    return w, pos, ids + np.uint64(rank * w["n_q"])


def max_over_ranks(values, dist, device):
    """Elementwise maximum of per-rank timings (identity without a process group)."""
    if dist is None:
        return list(values)
    import torch

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def make_inputs(w, rank, device, box_n=None, n_q=None):
    w = si.shrink(w, n=box_n, n_q=n_q)
    w, pos, ids = rank_catalogue(w, rank)
    d, e = si.gaussian_box(w["n"], w["cell"], w["seed_box"], backend="torch", device=device)
    return w, d, e, pos, ids


def run_reference(args, rank):
    if rank != 0:
        return
    import torch

    w = si.workload(WORKLOAD)
    device = "cuda:0" if torch.cuda.is_available() else "cpu"
    w, d, e, pos, ids = make_inputs(w, 0, device)
    dh, eh = d.cpu().numpy(), e.cpu().numpy()
    del d, e
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_rate(w, dh, eh, pos, ids, 2.0, threads)
    rates, pxs, secs = [], 0, 0.0
    for s in range(args.steps):
        r, px, n, dt = oracle_rate(w, dh, eh, pos, ids, 6.0, threads)
        rates.append(r)
        pxs += px
        secs += dt
    value = pxs / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(w, len(ids)),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"each step ~6 s of skewers in catalogue order (fields, flux, statistics); "
                                   f"{pxs} pixels over {args.steps} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- tuning A/B
def surrogate_leg(ctx, mk, w, r, n_q, target, nd0, dev, draws, held, epochs, source, slopes):
    """Train the surrogate on constant-parameter passes over 100k quasars (the
    first 100k stored skewers of the benchmark catalogue, "subset", or a
    separate 512^3 box with its own 100k quasars, "box512"), measure it on
    `held` fresh draws, and run the surrogate-driven tuning of the benchmark
    catalogue with it (every accepted set verified by full plain passes)."""
    import torch

    if source == "subset":
        ws, n_lab = w, 100_000
        rs = {"sk": r["sk"], "offsets": r["offsets"], "delta": r["delta"], "eta": r["eta"]}
    else:
        ws = si.shrink(w, n=512, n_q=100_000)
        ws["seed_box"], ws["seed_cat"] = w["seed_box"] + 1, w["seed_cat"] + 1
        d, e = si.gaussian_box(ws["n"], ws["cell"], ws["seed_box"], backend="torch", device=dev)
        pos, ids = si.catalogue(ws)
        bs = ctx.load_box(ws, ctx.pack_box(d, e, padded=True), None, layout=mk.BOX_PADDED)
        del d, e
        rs = ctx.make_skewers(bs, mk.catalogue_tensor(pos, ids, dev), len(ids), ws)
        n_lab = len(ids)
    t0 = time.perf_counter()
    hx, ht = mk.surrogate_labels(ctx, ws, rs["sk"], n_lab, rs["offsets"], rs["delta"], rs["eta"],
                                 n_draws=draws, seed=11, slopes=slopes)
    t_lab = time.perf_counter() - t0
    mlp = mk.Mlp(ctx, max_batch=1024, seed=3)
    t0 = time.perf_counter()
    norm, losses = mlp.fit(hx, ht, batch=256, epochs=epochs, lr=2e-3, seed=5)
    t_fit = time.perf_counter() - t0
    # one calibration pass over the first 100k skewers of the catalogue being
    # tuned: for the subset those are the labelled skewers (the surrogate's own
    # error, free of sample variance); for the 512^3 box it also measures the
    # box-to-box offset
    norm.calib_skewers = 100_000
    vx, vt = mk.surrogate_labels(ctx, ws, rs["sk"], n_lab, rs["offsets"], rs["delta"], rs["eta"],
                                 n_draws=held, seed=12, slopes=slopes)
    xm, xs = np.ctypeslib.as_array(norm.x_mean), np.ctypeslib.as_array(norm.x_std)
    tm, ts = np.ctypeslib.as_array(norm.t_mean), np.ctypeslib.as_array(norm.t_std)
    xin = torch.from_numpy(((vx - xm) / xs).astype(np.float32)).to(dev)
    pred = torch.cat([mlp.forward(xin[i:i + 1024].contiguous()) for i in range(0, xin.shape[0], 1024)])
    pred = pred.double().cpu().numpy() * ts + tm
    err = pred - vt
    held_out = {"draws": held, "samples": int(vx.shape[0]),
                "mean_flux_rms": float(np.sqrt(np.mean(err[:, 0] ** 2))),
                "mean_flux_max": float(np.abs(err[:, 0]).max()),
                "beta_rel_rms": float(np.sqrt(np.mean((err[:, 2] / vt[:, 2]) ** 2))),
                "ln_p1d_rms": float(np.sqrt(np.mean(err[:, 3:] ** 2)))}
    _, rep_s = mk.tune(ctx, w, r["sk"], n_q, r["offsets"], r["delta"], r["eta"], target, nd0,
                       method=mk.TUNE_SURROGATE, mlp=mlp, norm=norm, max_passes=60)
    mlp.close()
    del rs
    torch.cuda.empty_cache()
    return rep_s, {"source": source, "box": "1024^3 (first 100k skewers)" if source == "subset" else "512^3",
                   "quasars": 100_000, "draws": draws, "samples": int(hx.shape[0]), "epochs": epochs,
                   "profiles": ("linear in z, slopes up to d ln a/dz, db/dz, dc/dz = "
                                f"{slopes[0]}, {slopes[1]}, {slopes[2]}" if slopes else "constant"),
                   "label_s": t_lab, "fit_s": t_fit, "final_loss": float(losses[-1]) if len(losses) else None,
                   "held_out": held_out}


def tuning_ab(ctx, mk, box, qso, n_q, w, dev, legs, epochs, slopes=None):
    """Plain vs surrogate tuning of ln a, b, c at the 12 z nodes on the stored
    skewers of the benchmark catalogue; one surrogate run per (source, draws,
    held-out draws) leg."""
    import torch
    from paper_2310_18996_gb300 import tuning

    r = ctx.make_skewers(box, qso, n_q, w)  # stored pre-FGPA skewers (untimed)
    target, _ = tuning.make_target(ctx, w, r["sk"], n_q, r["offsets"], r["delta"], r["eta"], seed=7)
    nd0 = tuning.start_nodes(w)
    _, rep_p = mk.tune(ctx, w, r["sk"], n_q, r["offsets"], r["delta"], r["eta"], target, nd0,
                       method=mk.TUNE_PLAIN, max_passes=200)

    def rep(x):
        return {"converged": bool(x.converged), "passes": x.passes, "calib_passes": x.calib_passes,
                "gpu_ms": x.gpu_ms, "wall_ms": x.wall_ms,
                "max_abs_dfbar": x.max_abs_dfbar, "max_rel_p1d": x.max_rel_p1d, "max_rel_beta": x.max_rel_beta}

    out = {"workload": "stored skewers of the benchmark catalogue (1024^3, 1M quasars), 12 z nodes, target "
                       "Fbar = exp(-0.0025 (1+z)^3.7) +- 1e-3, P1D and beta_F of seeded hidden power laws +- 2%",
           "plain": rep(rep_p)}
    for name, source, draws, held in legs:
        rep_s, info = surrogate_leg(ctx, mk, w, r, n_q, target, nd0, dev, draws, held, epochs, source, slopes)
        out[name] = {"surrogate": rep(rep_s), "training": info,
                     "gpu_time_ratio_plain_over_surrogate": rep_p.gpu_ms / max(rep_s.gpu_ms, 1e-9),
                     "wall_time_ratio_including_training":
                         rep_p.wall_ms / (rep_s.wall_ms + 1000.0 * (info["label_s"] + info["fit_s"]))}
    del r
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- box synthesis (Sec. 2.1)
def box_synth_leg(ctx, mk, w, dev, peak, reps=3):
    """mk_synth_box at the benchmark's box size into the padded layout the
    fused pass reads, against the fixture's torch/cuFFT synthesis plus
    mk_pack_box_padded; CUDA events on the current stream, one untimed run each."""
    import torch

    n, cell = w["n"], w["cell"]
    dk = 2.0 * np.pi * np.sqrt(3.0) / cell / 4000.0
    tab = si.power_shape(dk * np.arange(4011))
    work = torch.empty(2 * n ** 3, dtype=torch.float32, device=dev)
    out = torch.empty(2 * (n + 1) ** 3, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def lib_once(seed):
        ctx._stream()
        ctx._check(mk.lib().mk_synth_box(ctx.h, n, cell, seed, mk._dp(tab), tab.size, dk, mk.BOX_PADDED,
                                         mk._ptr(work), None, mk._ptr(out)))

    def torch_once(seed):
        d, e = si.gaussian_box(n, cell, seed, backend="torch", device=dev)
        ctx.pack_box(d, e, padded=True)
        del d, e

    res = {}
    big = None
    if n == 1024 and torch.cuda.mem_get_info()[0] > work.numel() * 4 * 8 + out.numel() * 4 * 8 + 20e9:
        # a 2048^3 box and its padded copy (137 GB) in core on one GPU
        w2 = torch.empty(2 * 2048 ** 3, dtype=torch.float32, device=dev)
        o2 = torch.empty(2 * 2049 ** 3, dtype=torch.float32, device=dev)

        def big_once(seed):
            ctx._stream()
            ctx._check(mk.lib().mk_synth_box(ctx.h, 2048, cell, seed, mk._dp(tab), tab.size, dk, mk.BOX_PADDED,
                                             mk._ptr(w2), None, mk._ptr(o2)))

        big_once(1)
        torch.cuda.synchronize()
        e0.record(st)
        big_once(2)
        e1.record(st)
        e1.synchronize()
        big = e0.elapsed_time(e1)
        del w2, o2
        torch.cuda.empty_cache()
    for name, fn in (("library", lib_once), ("torch_cufft_fixture", torch_once)):
        fn(1)
        torch.cuda.synchronize()
        e0.record(st)
        for r in range(reps):
            fn(2 + r)
        e1.record(st)
        e1.synchronize()
        res[name] = e0.elapsed_time(e1) / reps
    del work, out
    torch.cuda.empty_cache()
    # the quasar chain (Sec. 2.2, App. A): three delta_q boxes of one white noise,
    # then the voxel draw at nbar = 1e-4 (h/Mpc)^3 (about 1.1M quasars at 1024^3)
    zb = (1.9, 2.75, 3.6)
    pq = []
    for z in zb:
        g = ctx.cosmo_eval(z)[1]
        pq.append(mk.lognormal_pk(tab, dk, (3.7 * ((1 + z) / 3.33) ** 1.7) ** 2 * g * g))
    q = dict(n=n, cell=cell, origin=w["origin"], z_box=zb, bias=(3.7, 2.33, 1.7),
             xi_m5=float(mk.xi_of_pk(tab, dk, 5.0)[0]), nbar=[1e-4] * 20, nbar_z0=1.0, nbar_dz=0.25, seed=77)
    wq = torch.empty(2 * n ** 3, dtype=torch.float32, device=dev)
    boxes = [torch.empty(n ** 3, dtype=torch.float32, device=dev) for _ in range(3)]

    def synth3_once(seed):
        for i in range(3):
            ctx._stream()
            ctx._check(mk.lib().mk_synth_box(ctx.h, n, cell, seed, mk._dp(pq[i]), pq[i].size, dk, mk.BOX_PLANAR,
                                             mk._ptr(wq), None, mk._ptr(boxes[i])))

    synth3_once(5)  # untimed run
    ctx.draw_qso(q, boxes, stride=1)
    torch.cuda.synchronize()
    e0.record(st)
    synth3_once(6)
    e1.record(st)
    e1.synchronize()
    synth3 = e0.elapsed_time(e1)
    t0 = time.perf_counter()
    _, cnt = ctx.draw_qso(q, boxes, stride=1)
    draw_ms = 1000.0 * (time.perf_counter() - t0)
    del boxes, wq
    torch.cuda.empty_cache()
    # bytes of the five passes: noise+x (write), y, z (read+write each), inverse y,
    # inverse x (read, padded write)
    b = 8.0 * n ** 3 * (1 + 2 + 2 + 2 + 1) + 8.0 * (n + 1) ** 3
    return {"box": f"{n}^3, cell {cell}, delta + eta_xx into the padded layout",
            "ms": res["library"], "fixture_ms": res["torch_cufft_fixture"],
            "pass_bytes": b, "achieved_gbs": b / (res["library"] * 1e6), "frac_of_hbm_peak": b / (res["library"] * 1e6) / peak,
            "design": "5 passes: Philox noise + FFT x | FFT y | FFT z, filter, inverse z | inverse y | inverse x + layout",
            "box_2048_padded_ms": big,
            "qso_chain": {"what": "three quasar-density boxes (z 1.9, 2.75, 3.6) from one white noise, delta "
                                  "alone (planar), then mk_draw_qso (App. A) at nbar 1e-4 (h/Mpc)^3",
                          "synth_3_boxes_ms": synth3, "draw_wall_ms": draw_ms, "quasars": cnt,
                          "draw_note": "wall time of the synchronous call: box moments, r table on the host, "
                                       "count pass, host scan, write pass"}}


# ---------------------------------------------------------------- Sec. 2.6 P_S tuning
def ps_tuning_leg(ctx, mk, box, qso, n_q, w, n_outer, n_inner):
    """The paper's procedure (mk_tune_ps): a, b sigma_g fitted to F-bar and the
    P1D integral, c from beta, b from the measured sigma_g, then ratio
    iterations of P_S(k, z) at the 12 nodes, every pass a fused synthesis of
    the whole catalogue.  Target: the statistics of the catalogue synthesised
    at seeded hidden a*, b*, c* and P_S*(k, z)."""
    import torch
    from paper_2310_18996_gb300 import tuning

    target, _, _ = tuning.make_ps_target(ctx, box, qso, n_q, w, seed=7)
    torch.cuda.empty_cache()
    p0 = tuning.start_small_scale_power(w)
    nd, ps, rep = mk.tune_ps(ctx, box, qso, n_q, w, target, p0, n_outer=n_outer, n_inner=n_inner)
    hist = [round(float(rep.max_rel_p1d_pass[i]), 5) for i in range(rep.passes)]
    return {"workload": f"{w['n']}^3 box, {n_q} quasars, 12 z nodes (bin centres), P_S at each node, every pass "
                        "a fused synthesis of the catalogue (mk_run, statistics only)",
            "target": "statistics at seeded hidden a*, b*, c* power laws and P_S*(k, z) = P_S(k) (1 + A (z - 2.6)) "
                      "(k / k_8)^t; start: the workload's P_S at every node",
            "outer": n_outer, "inner": n_inner, "passes": rep.passes, "gpu_ms": rep.gpu_ms,
            "ms_per_pass": rep.gpu_ms / max(rep.passes, 1), "wall_ms": rep.wall_ms,
            "max_abs_dfbar": rep.max_abs_dfbar, "max_rel_p1d": rep.max_rel_p1d, "max_rel_beta": rep.max_rel_beta,
            "max_rel_p1d_first_pass": hist[0] if hist else None,
            "max_rel_p1d_end_of_outer_loop": [hist[min(len(hist) - 1, (k + 1) * (n_inner + 1) - 1)]
                                              for k in range(n_outer)] if hist else None}


# ---------------------------------------------------------------- GPU arm
def run_gb300(args, rank, world, local_rank):
    import torch

    import paper_2310_18996_gb300 as mk

    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    w, d, e, pos, ids = make_inputs(si.workload(WORKLOAD), rank, dev, args.box_n, args.n_q)
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    dh = eh = None
    if want_cpu:
        dh, eh = d.cpu().numpy(), e.cpu().numpy()
    ctx = mk.Context(local_rank)
    packed = ctx.pack_box(d, e, padded=True)
    halo = None if args.no_gauss7 else ctx.pack_box(d, e, halo=True)  # for the Gaussian-kernel path
    torch.cuda.synchronize()
    del d, e
    torch.cuda.empty_cache()
    box = ctx.load_box(w, packed, None, layout=mk.BOX_PADDED)
    n_q = len(ids)
    rec_np = np.zeros(n_q, dtype=mk.QSO_DTYPE)
    rec_np["pos"] = pos
    rec_np["id"] = ids
    host_cat = torch.from_numpy(rec_np.view(np.uint8)).pin_memory()
    qso = host_cat.to(dev)
    sk, off, total = ctx.plan(box, qso, n_q, w)
    npix = mk.skewer_records(sk, n_q)["n"].astype(np.int64)
    flux = torch.empty(total, dtype=torch.float32, device=dev)
    outs = {"sk": sk, "offsets": off, "flux": flux}
    flags = mk.STATS | mk.STORE_FLUX
    stream = torch.cuda.Stream(device=dev)  # graphs cannot be captured on the legacy stream
    torch.cuda.set_stream(stream)

    def step(extra=mk.GRAPH):
        return ctx.run(box, qso, n_q, w, flags=flags | extra, capacity=total, outputs=outs)

    # warm-up: the first call tunes the launch shape, the next capture the graph
    step(mk.AUTOTUNE)
    for _ in range(args.warmup):
        step()
    threads, occ, tuned = ctx.launch_config(w["n_fft"], flags=flags, layout=mk.BOX_PADDED)
    # kernel-only time of the fused kernel (direct launches, CUDA events on the stream)
    ctx.set_timing(True)
    kern = []
    for _ in range(max(3, args.steps // 2)):
        step(0)
        kern.append(ctx.last_kernel_ms())
    ctx.set_timing(False)
    kms = float(np.mean(kern))
    clocks = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        st, _ = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms, kms = max_over_ranks([ms, kms], dist, dev)
    value = world * total / (ms / 1000.0)

    # end to end through the public API with host buffers: each step takes the
    # catalogue from pinned host memory and returns the flux to pinned host
    # memory plus the statistics.  mk_run_host pipelines it (slices computed
    # while the previous slice's flux crosses the host link); the plain
    # sequence (catalogue H2D, mk_run, one flux D2H) is timed beside it.
    host_flux = torch.empty(total, dtype=torch.float32).pin_memory()
    e2e_steps = 0 if args.no_e2e else max(3, args.steps // 2)
    qdev = torch.empty_like(qso)

    def e2e_loop(pipelined):
        t0 = time.perf_counter()
        for it in range(e2e_steps + 1):
            if it == 1:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            if pipelined:
                ctx.run_host(box, host_cat, n_q, w, host_flux, n_chunks=args.e2e_chunks)
            else:
                qdev.copy_(host_cat, non_blocking=True)
                ctx.run(box, qdev, n_q, w, flags=flags | mk.GRAPH, capacity=total, outputs=outs)
                host_flux.copy_(flux, non_blocking=True)
                torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1000.0 / e2e_steps

    e2e_ms = e2e_copy_ms = float("nan")
    if e2e_steps:
        e2e_copy_ms = e2e_loop(False)
        host_flux.zero_()
        e2e_ms = e2e_loop(True)
        k = min(total, 1 << 24)  # the pipelined flux equals the device-resident flux
        if not torch.equal(host_flux[:k].to(dev), flux[:k]) or not torch.equal(host_flux[-k:].to(dev), flux[-k:]):
            raise RuntimeError("pipelined host flux differs from the device-resident flux")
    e2e_ms, e2e_copy_ms = max_over_ranks([e2e_ms, e2e_copy_ms], dist, dev)

    def variant_leg(wv, box_v, layout_code):
        """The same fused step on another box layout / interpolation: autotuned
        launch, kernel-only time, graph-replayed steps."""
        def vstep(extra=mk.GRAPH):
            return ctx.run(box_v, qso, n_q, wv, flags=flags | extra, capacity=total, outputs=outs)

        vstep(mk.AUTOTUNE)
        for _ in range(args.warmup):
            vstep()
        vt, vo, _ = ctx.launch_config(w["n_fft"], layout=layout_code, flags=flags)
        ctx.set_timing(True)
        vk = []
        for _ in range(max(3, args.steps // 2)):
            vstep(0)
            vk.append(ctx.last_kernel_ms())
        ctx.set_timing(False)
        torch.cuda.synchronize()
        v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        for _ in range(args.steps):
            vstep()
        v1.record(stream)
        torch.cuda.synchronize()
        vms, vkms = max_over_ranks([v0.elapsed_time(v1) / args.steps, float(np.mean(vk))], dist, dev)
        return {"value": world * total / (vms / 1000.0), "unit": UNIT, "ms_per_step": vms, "kernel_ms": vkms,
                "launch": f"{vt} threads/CTA, occupancy target {vo}"}

    # the same step as separate passes (a1-a5 storing delta, eta; FGPA + rebin;
    # statistics), the shape of a per-stage pipeline, for comparison with the fused launch
    split = None
    if rank == 0 and world == 1 and not args.no_split:
        def split_once():
            r = ctx.make_skewers(box, qso, n_q, w)
            f, off = ctx.flux(w, r["sk"], n_q, r["delta"], r["eta"])
            return ctx.stats(w, r["sk"], n_q, off, f)

        split_once()
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        s0.record(stream)
        for _ in range(reps):
            split_once()
        s1.record(stream)
        torch.cuda.synchronize()
        sms = s0.elapsed_time(s1) / reps
        split = {"value": total / (sms / 1000.0), "unit": UNIT, "ms_per_step": sms,
                 "path": "mk_make_skewers (plan + pass storing delta_tot, eta) -> mk_flux -> mk_stats, "
                         "8 B/px stored and re-read, flux stored and re-read"}
        torch.cuda.empty_cache()

    # the same catalogue as launches over batches of 500 quasars (the size of the
    # 64^3 / 500-quasar case), each a fused pass with its own statistics read back
    batched = None
    if rank == 0 and world == 1 and not args.no_split:
        nb = 500
        cap_b = nb * 2300
        ob = {"sk": torch.empty(nb * mk.SKEWER_BYTES, dtype=torch.uint8, device=dev),
              "offsets": torch.empty(nb + 1, dtype=torch.int64, device=dev),
              "flux": torch.empty(cap_b, dtype=torch.float32, device=dev)}
        rb = mk.QSO_DTYPE.itemsize

        def batched_once():
            for b0 in range(0, n_q, nb):
                m = min(nb, n_q - b0)
                ctx.run(box, qso[b0 * rb:(b0 + m) * rb], m, w, flags=flags, capacity=cap_b, outputs=ob)

        batched_once()
        torch.cuda.synchronize()
        b0e, b1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0e.record(stream)
        batched_once()
        b1e.record(stream)
        torch.cuda.synchronize()
        bms = b0e.elapsed_time(b1e)
        batched = {"value": total / (bms / 1000.0), "unit": UNIT, "ms_per_step": bms, "launches": (n_q + nb - 1) // nb,
                   "path": "mk_run (fused, statistics read back) per batch of 500 quasars, no graph"}

    # the same sight lines at distances that make the skewer lengths uniform in
    # [200, 1500] pixels (each quasar's distance bisected on the library's geometry)
    uni = None
    if rank == 0 and world == 1 and not args.no_split:
        rng_u = np.random.default_rng(17)
        target = rng_u.integers(200, 1501, n_q)
        udir = pos / np.linalg.norm(pos, axis=1, keepdims=True)
        lo = np.full(n_q, ctx.cosmo_eval(1.9)[0])
        hi = np.full(n_q, ctx.cosmo_eval(4.6)[0])
        for _ in range(44):
            mid = 0.5 * (lo + hi)
            sk_m, _, _ = ctx.plan(box, mk.catalogue_tensor(udir * mid[:, None], ids, dev), n_q, w)
            nm = mk.skewer_records(sk_m, n_q)["n"]
            short = nm < target
            lo = np.where(short, mid, lo)
            hi = np.where(short, hi, mid)
        qu = mk.catalogue_tensor(udir * hi[:, None], ids, dev)
        sk_u, off_u, tot_u = ctx.plan(box, qu, n_q, w)
        nu = mk.skewer_records(sk_u, n_q)["n"]
        ou = {"sk": sk_u, "offsets": off_u, "flux": torch.empty(tot_u, dtype=torch.float32, device=dev)}

        def ustep(extra=mk.GRAPH):
            return ctx.run(box, qu, n_q, w, flags=flags | extra, capacity=tot_u, outputs=ou)

        ustep(mk.AUTOTUNE)
        for _ in range(args.warmup):
            ustep()
        torch.cuda.synchronize()
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        for _ in range(args.steps):
            ustep()
        u1.record(stream)
        torch.cuda.synchronize()
        ums = u0.elapsed_time(u1) / args.steps
        uni = {"value": tot_u / (ums / 1000.0), "unit": UNIT, "ms_per_step": ums, "pixels_per_step": int(tot_u),
               "lengths": f"min {int(nu.min())}, max {int(nu.max())}, mean {float(nu.mean()):.1f}, "
                          f"{float(np.mean(nu == target)):.3f} exactly on target",
               "catalogue": "the benchmark's 1M sight lines, each quasar's distance set so that its skewer "
                            "has a length drawn uniformly from [200, 1500] pixels"}
        del ou
        torch.cuda.empty_cache()

    # the paper's Gaussian-kernel interpolation (7^3 voxels, Sec. 2.3) on the
    # same catalogue: the same fused step with the other gather
    gauss = None
    if halo is not None:
        wg = dict(w)
        wg["interp"] = mk.INTERP_GAUSS7
        gauss = variant_leg(wg, ctx.load_box(wg, halo, None, layout=mk.BOX_HALO), mk.BOX_HALO + mk.GAUSS7_VARIANT)
        gauss.update({"interp": "Gaussian kernel over 7^3 voxels, sigma = one voxel (Sec. 2.3)",
                      "box": f"{w['n']}^3 (delta, eta) pairs with a periodic margin of 3"})
        del halo
        torch.cuda.empty_cache()
    # the radial eta_par of Eq. eta from the six velocity-gradient boxes
    tens = None
    if not args.no_tensor:
        wt = dict(w)
        wt["eta_mode"] = 1
        td, te6 = si.gaussian_box_tensor(w["n"], w["cell"], w["seed_box"], backend="torch", device=dev)
        tpacked = ctx.pack_box_tensor(td, te6)
        torch.cuda.synchronize()
        del td, te6
        torch.cuda.empty_cache()
        tens = variant_leg(wt, ctx.load_box(wt, tpacked, None, layout=mk.BOX_TENSOR), mk.BOX_TENSOR)
        tens.update({"eta": "u_p u_q eta_pq from six velocity-gradient boxes (Eq. eta), trilinear",
                     "box": f"{w['n']}^3 points of (delta, 6 eta_pq), 32 B each"})
        del tpacked
        torch.cuda.empty_cache()

    peak, peak_kind = measured_peaks()
    alg = algorithmic_bytes(pos, npix, w)
    achieved = alg / (kms / 1000.0) / 1e9
    tune = None
    if rank == 0 and world == 1 and not args.no_tuning:
        slopes = None if args.surrogate_slopes == "none" else tuple(float(v) for v in args.surrogate_slopes.split(","))
        legs = [("surrogate_subset", "subset", args.surrogate_draws, max(args.surrogate_draws // 10, 10))]
        if args.config4_draws > 0:
            legs.append(("surrogate_512", "box512", args.config4_draws, args.config4_held))
        tune = tuning_ab(ctx, mk, box, qso, n_q, w, dev, legs, args.surrogate_epochs, slopes)
    boxs = None
    if rank == 0 and world == 1 and not args.no_box_synth and w["n"] in (128, 256, 512, 1024):
        boxs = box_synth_leg(ctx, mk, w, dev, peak)
    pst = None
    if rank == 0 and world == 1 and not args.no_ps_tuning:
        pst = ps_tuning_leg(ctx, mk, box, qso, n_q, w, args.ps_outer, args.ps_inner)
    merged = None
    if dist:  # catalogue-wide statistics: one all-gather of the raw sums, then mk_stats_merge
        mst = mk.merge_stats_across_ranks(st, w, dist, device=dev)
        merged = {"ranks": world, "pixels": int(mst["sums"][:, 0].sum()), "p1d_segments": int(mst["n_seg"].sum()),
                  "mean_flux": [round(float(x), 6) for x in mst["mean_flux"]],
                  "how": "all-gather of each rank's raw sums (sums, p1d_sum, n_seg), mk_stats_merge in rank order"}
    cpu = None
    if want_cpu:
        cores = os.cpu_count() or 1
        rate, px, n, dt = oracle_rate(w, dh, eh, pos, ids, args.cpu_seconds, cores)
        rate1, px1, n1, dt1 = oracle_rate(w, dh, eh, pos, ids, args.cpu_seconds / 3.0, 1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} skewers ({px} pixels) of the same catalogue, {dt:.1f} s, fields+flux+stats",
               "one_core": {"value": rate1, "cores": 1, "sample": f"{n1} skewers ({px1} pixels), {dt1:.1f} s"}}
    if rank == 0:
        prof = profiled_kernel_record()
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic(total), "peak_kind": peak_kind,
                "kernel": f"k_skewer<256,padded> {threads} threads/CTA, occupancy "
                          f"target {occ}{' (autotuned)' if tuned else ''}", "kernel_ms": kms,
                "algorithmic_bytes": alg, "algorithmic_bytes_per_pixel": alg / total}
        if prof:  # the compute side, from the committed ncu record of the same kernel source
            roof.update({k: prof[k] for k in ("warp_inst_per_px", "thread_inst_per_px", "issue_active",
                                              "alu_pipe_active", "fma_pipe_active") if k in prof})
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(w, n_q),
            "pixels_per_step_per_gpu": int(total),
            "roofline": roof,
            "e2e": {"value": world * total / (e2e_ms / 1000.0), "unit": UNIT,
                    "h2d_bytes_per_step": int(host_cat.numel()),
                    "d2h_bytes_per_step": int(total * 4 + mk.C.sizeof(mk.StatsOut)),
                    "ms_per_step": e2e_ms,
                    "method": f"mk_run_host: catalogue H2D from pinned memory, {args.e2e_chunks} slices, each "
                              "slice's flux copied to pinned host memory while the next is computed",
                    "sequential_ms_per_step": e2e_copy_ms},
            "gpu_launches": 6 * args.steps,  # per step: geometry, 3 scan passes, fused kernel, finalize
            "launch": "CUDA graph per step (mk_run MK_GRAPH), fused persistent kernel, launch shape autotuned",
            "clocks": clk,
        }
        if cpu:
            line["cpu_baseline"] = cpu
        # the other legs; the tuning A/B last, so that the end of the line carries it
        for key, val in (("gauss7", gauss), ("eta_tensor", tens), ("split_path", split),
                         ("batched_launches", batched), ("uniform_lengths", uni), ("box_synth", boxs),
                         ("ps_tuning", pst), ("stats_merge", merged), ("tuning", tune)):
            if val:
                line[key] = val
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=16)
    ap.add_argument("--no-gauss7", action="store_true")
    ap.add_argument("--no-tensor", action="store_true")
    ap.add_argument("--no-tuning", action="store_true")
    ap.add_argument("--no-ps-tuning", action="store_true")
    ap.add_argument("--no-box-synth", action="store_true")
    ap.add_argument("--no-split", action="store_true")
    ap.add_argument("--ps-outer", type=int, default=5, help="outer loops of the Sec. 2.6 P_S tuning")
    ap.add_argument("--ps-inner", type=int, default=10, help="P_S ratio iterations per outer loop")
    ap.add_argument("--surrogate-draws", type=int, default=8000)
    ap.add_argument("--surrogate-epochs", type=int, default=300)
    ap.add_argument("--surrogate-slopes", default="1.8,0.45,0.45",
                    help="maxima of d ln a/dz, db/dz, dc/dz of the training profiles, or 'none'")
    ap.add_argument("--config4-draws", type=int, default=20000,
                    help="draws of the surrogate labelled on a separate 512^3 box (0: leg off)")
    ap.add_argument("--config4-held", type=int, default=2000, help="held-out draws of that surrogate")
    ap.add_argument("--box-n", type=int, default=None, help="smaller box (profiling runs)")
    ap.add_argument("--n-q", type=int, default=None, help="fewer quasars (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_gb300(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
