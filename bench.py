#!/usr/bin/env python
"""Benchmark of the FW-H hot path on GB300: panel x source-step x observer
evaluations per second for the 32768-panel x 2048-step x 72-observer convected
dipole (sphere r=1.5, M0=0.5, AoA=10 deg, dt=0.01), mixed precision, with the
plain FP64 form, the end-to-end C-ABI call on host buffers and the FP64 CPU
oracle timed beside it.

One step = one fwh_forward: integrand preparation + forward scatter over the
whole surface, all 2048 source steps and all observers, inputs resident in
HBM (1.34 GB of FP32 fields and 4.3 GB of prepared series: both larger than
the 129 MB L2, so no flush is needed between steps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own observer set (the circle rotated by a
rank-dependent angle): the observer dimension is independent, so there is no
data-path collective and the scaling is weak.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FW-H panel·τ·observer evals/s, mixed vs FP64 at ≤1e-4 rel L2; % roofline"
UNIT = "evals/s"
FLOP_PER_EVAL = 40          # 20 FMA: 8 + 8 (signal, spline moment) + 4 (interpolation)
# FP32 FMA roof: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP64 FMA roof: nominal GB300 FP64 rate
FP64_PEAK_TFLOPS = 1.25


def hbm_peak_gbs():
    """HBM copy bandwidth measured on these GB300s (GB/s), else an earlier
    GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"
PROFILE = os.path.join(ROOT, "profiles", "forward_kernel_workload2.md")
KERNEL_SRC = os.path.join(ROOT, "paper_2312_16263_gb300", "csrc", "fwh_forward.cu")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the extra legs (workloads 1, 3, 4 backward, 5 batched, PSD)")
    ap.add_argument("--profile-case", action="store_true",
                    help="small case for ncu: workload 2 with --nt steps, two forward calls")
    ap.add_argument("--nt", type=int, default=512)
    ap.add_argument("--profile-backward", action="store_true",
                    help="small case for ncu: the 16384-panel x 1024-step x 36-observer dipole, "
                         "two forward + backward calls")
    ap.add_argument("--profile-batch", action="store_true",
                    help="small case for ncu: one contour surface of the eight-surface set "
                         "(16384 panels x 2048 steps x 1024 observers) through fwh_forward, "
                         "the single-grid and the persistent batched forms, twice each")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tile-config", type=int, default=-1,
                    help="forward tile configuration index (-1: the library default)")
    return ap.parse_args()


def profile_backward(args):
    """Two fwh_forward + fwh_backward calls on the 16384 x 1024 x 36 dipole
    (about 2.5 GB on the device): the capture target for the adjoint kernels."""
    import torch
    from __graft_entry__ import build
    build()
    from paper_2312_16263_gb300 import FWH
    from fwh_inputs import workload
    w = workload(4)
    s = FWH.from_workload(w, args.precision)
    f = w.fields(device="cuda:0", dtype="float32" if args.precision == "mixed" else "float64")
    p = s.forward(f)
    g = 2.0 * p
    for _ in range(2):
        gf = s.backward(f, g)
    torch.cuda.synchronize()
    s.check()
    print(json.dumps({"profile_backward": w.name, "precision": args.precision,
                      "max_abs_grad": float(gf.abs().max())}))


def profile_case(args):
    """Two fwh_forward calls on workload 2 cut to --nt source steps (about
    1.4 GB on the device at nt=512): the capture target for ncu --set full."""
    import torch
    from __graft_entry__ import build
    build()
    from paper_2312_16263_gb300 import FWH
    w = rank_workload(0, 1)
    w.nt = args.nt
    s = FWH.from_workload(w, args.precision)
    if args.tile_config >= 0:
        s.set_tile_config(args.tile_config)
    f = w.fields(device="cuda:0", dtype="float32" if args.precision == "mixed" else "float64")
    out = torch.empty((s.O, w.nt), dtype=torch.float64, device="cuda:0")
    for _ in range(2):
        s.forward(f, out)
    torch.cuda.synchronize()
    s.check()
    print(json.dumps({"profile_case": w.name, "nt": w.nt, "precision": args.precision,
                      "max_abs": float(out.abs().max())}))


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, ws: int) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_workload(rank: int, ws: int):
    import numpy as np
    from fwh_inputs import observers_circle, workload
    w = workload(2)
    if rank > 0:  # rotate the 72-observer circle: a distinct, equally sized set
        ang = 2 * np.pi / 72 * rank / ws
        c, s = np.cos(ang), np.sin(ang)
        w.observers = observers_circle(100.0, 72) @ np.array([[c, s, 0], [-s, c, 0], [0, 0, 1]])
    return w


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.idx = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        load = [v for v in sm if mx and v > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_fma_peaks():
    """FP32 and FP64 FMA throughput of this GPU (TFLOP/s) from the library's
    FMA-chain probe (fwh_fma_peak), taken before the timed region."""
    import ctypes
    from paper_2312_16263_gb300 import _abi
    lib = _abi.load()
    out = {}
    for name, prec in (("fp32", _abi.FWH_MIXED), ("fp64", _abi.FWH_FP64)):
        v = ctypes.c_double(0.0)
        _abi.check(lib.fwh_fma_peak(prec, ctypes.byref(v), None))
        out[name] = v.value
    return out


def profile_traffic():
    """DRAM bytes per forward launch from the committed ncu summary, if that
    summary was taken on the current kernel source (hash match), else None."""
    if not os.path.exists(PROFILE):
        return None
    txt = open(PROFILE).read()
    h = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != h:
        return None
    return float(t.group(1))


def cpu_baseline(w, target_s=15.0):
    """The FP64 oracle as it stands, on all host cores, on a bounded sample of
    the same workload: all panels and source steps for a subset of the
    observers, sized from a two-observer probe to take about target_s."""
    import numpy as np
    from oracle import Oracle
    from oracle.oracle import max_threads
    f = w.fields("float32").double().numpy()
    orc = Oracle.from_workload(w)
    n_all = w.observers.shape[0]
    t0 = time.perf_counter()
    orc.forward(f, w.observers[:2])
    per_obs = (time.perf_counter() - t0) / 2
    n_obs = int(min(n_all, max(2, round(target_s / max(per_obs, 1e-6)))))
    pick = np.linspace(0, n_all, n_obs, endpoint=False).astype(int)
    t0 = time.perf_counter()
    p, ts, nv = orc.forward(f, w.observers[pick])
    dt = time.perf_counter() - t0
    evals = w.surface.n_panels * w.nt * len(pick)
    return {"value": evals / dt, "unit": UNIT, "cores": max_threads(), "kind": "oracle",
            "sample": f"{len(pick)} of {n_all} observers (evenly spaced), all "
                      f"{w.surface.n_panels} panels x {w.nt} steps ({evals:.3g} evals, "
                      f"{dt:.1f} s)"}, (pick, p, nv)


def _time_calls(fn, n, warm=2):
    """Average ms of fn() over n calls (CUDA events on the current stream)."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def _oracle_leg(w, f64_host, pick):
    """The oracle on a sample of observers: (p_ref, nv_ref, evals/s, threads)."""
    from oracle import Oracle
    from oracle.oracle import max_threads
    orc = Oracle.from_workload(w)
    t0 = time.perf_counter()
    p_ref, _, nv_ref = orc.forward(f64_host, w.observers[pick])
    dt_s = time.perf_counter() - t0
    return p_ref, nv_ref, w.surface.n_panels * w.nt * len(pick) / dt_s, max_threads()


def extra_legs(dev):
    """Workloads 1 (plain FP64), 3 (mixed and FP64), 4 (backward), 5 (eight
    surfaces, batched) and the PSD of workload 2's signals, each timed with
    CUDA events on inputs resident in HBM, with the error against the oracle on
    a sample of observers and the oracle's rate on this host beside it.
    Returns a dict of keys for the JSON line."""
    import numpy as np
    import torch
    from fwh_inputs import batch_workloads, workload
    from paper_2312_16263_gb300 import FWH, batch_forward, welch_psd
    out = {}
    # workload 1: plain FP64 (and mixed), every observer against the oracle
    w = workload(1)
    f = w.fields(device=dev, dtype="float64")
    p_ref, nv_ref, orate, thr = _oracle_leg(w, f.cpu().numpy(), np.arange(w.observers.shape[0]))
    # the same on one host core
    from oracle import Oracle
    t0 = time.perf_counter()
    Oracle.from_workload(w).forward(f.cpu().numpy(), w.observers, threads=1)
    orate1 = w.evals / (time.perf_counter() - t0)
    leg = {"workload": w.name, "evals": w.evals, "oracle_evals_per_s": orate, "oracle_cores": thr,
           "oracle_evals_per_s_1core": orate1}
    for prec in ("fp64", "mixed"):
        s = FWH.from_workload(w, prec)
        fx = f if prec == "fp64" else f.float()
        o = torch.empty((s.O, w.nt), dtype=torch.float64, device=dev)
        ms = _time_calls(lambda: s.forward(fx, o), 20)
        _, nv = s.window(w.nt)
        # few observers: the series bytes per call (one row per panel and
        # sample per observer group; 64 B mixed, 128 B FP64) against HBM too
        groups = -(-w.observers.shape[0] // 36)
        xbytes = (64 if prec == "mixed" else 128) * w.surface.n_panels * w.nt * groups
        leg[prec] = {"ms": ms, "evals_per_s": w.evals / (ms / 1e3),
                     "series_bytes": xbytes,
                     "hbm_frac": xbytes / (ms / 1e3) / 1e9 / hbm_peak_gbs()[0],
                     "rel_l2_vs_oracle": rel_l2_stats(o.cpu().numpy(), nv, p_ref, nv_ref,
                                                      np.arange(w.observers.shape[0]))}
        s.check()
        s.close()
    out["workload1"] = leg
    # workload 3: the contour with broadband fields, two observers against the oracle
    w = workload(3)
    f = w.fields(device=dev, dtype="float32")
    pick = np.array([0, 23])
    p_ref, nv_ref, orate, thr = _oracle_leg(w, f.double().cpu().numpy(), pick)
    leg = {"workload": w.name, "evals": w.evals, "oracle_evals_per_s": orate, "oracle_cores": thr,
           "oracle_sample": "observers 0 and 23, all panels and steps"}
    for prec in ("mixed", "fp64"):
        s = FWH.from_workload(w, prec)
        fx = f if prec == "mixed" else f.double()
        o = torch.empty((s.O, w.nt), dtype=torch.float64, device=dev)
        ms = _time_calls(lambda: s.forward(fx, o), 5 if prec == "mixed" else 2, warm=1)
        _, nv = s.window(w.nt)
        leg[prec] = {"ms": ms, "evals_per_s": w.evals / (ms / 1e3),
                     "rel_l2_vs_oracle": rel_l2_stats(o.cpu().numpy(), nv, p_ref, nv_ref, pick)}
        s.check()
        s.close()
        del fx
    out["workload3"] = leg
    del f
    # workload 4: the adjoint (d sum p^2 / d fields), against the oracle's FP64 adjoint
    from oracle import Oracle
    w = workload(4)
    f = w.fields(device=dev, dtype="float32")
    leg = {"workload": w.name, "evals": w.evals}
    s64 = FWH.from_workload(w, "fp64")
    g_p = 2.0 * s64.forward(f.double())
    t0 = time.perf_counter()
    g_ref = Oracle.from_workload(w).backward(f.double().cpu().numpy(), w.observers,
                                             g_p.cpu().numpy())
    leg["oracle_evals_per_s"] = w.evals / (time.perf_counter() - t0)
    for prec in ("mixed", "fp64"):
        s = FWH.from_workload(w, prec)
        fx = f if prec == "mixed" else f.double()
        gout = torch.empty_like(fx)
        ms = _time_calls(lambda: s.backward(fx, g_p, gout), 20 if prec == "mixed" else 2,
                         warm=3 if prec == "mixed" else 1)
        g = gout.double().cpu().numpy()
        leg[prec] = {"ms": ms, "evals_per_s": w.evals / (ms / 1e3),
                     "grad_rel_l2_vs_oracle": float(np.linalg.norm(g - g_ref) /
                                                    np.linalg.norm(g_ref))}
        s.check()
        s.close()
    s64.close()
    out["backward"] = leg
    del f, g_p
    torch.cuda.empty_cache()
    # workload 5: eight uneven surfaces in one graph-captured call (whole
    # records, pipelined form), one fwh_forward call per surface, the single
    # grid and persistent forms, and the series streamed through a ring of two
    # 512-sample segments per surface (four rounds); the smallest surface
    # against the oracle
    ws5 = batch_workloads()
    surfs = [FWH.from_workload(x, "mixed") for x in ws5]
    fields = [x.fields(device=dev, dtype="float32") for x in ws5]
    ev5 = sum(x.evals for x in ws5)
    outs = batch_forward(surfs, fields)
    ms_b = _time_calls(lambda: batch_forward(surfs, fields, outs), 3, warm=1)
    surfs[0].check()
    free_b = torch.cuda.mem_get_info()[0]
    small = len(ws5) - 1
    pick = np.array([0, ws5[small].observers.shape[0] // 2])
    p_ref, nv_ref, orate, thr = _oracle_leg(ws5[small], fields[small].double().cpu().numpy(), pick)
    _, nv = surfs[small].window(ws5[small].nt)
    err_b = rel_l2_stats(outs[small].cpu().numpy(), nv, p_ref, nv_ref, pick)
    ms_s = _time_calls(lambda: [sx.forward(fx, ox) for sx, fx, ox in zip(surfs, fields, outs)],
                       2, warm=1)
    # the other launch forms over the same items: one grid, the persistent
    # work-queue kernel
    ms_f, err_f = {}, {}
    for form in ("grid", "persistent"):
        surfs[0].set_batch_options(0, form)
        outs_p = batch_forward(surfs, fields)
        ms_f[form] = _time_calls(lambda: batch_forward(surfs, fields, outs_p), 3, warm=1)
        surfs[0].check()
        err_f[form] = rel_l2_stats(outs_p[small].cpu().numpy(), nv, p_ref, nv_ref, pick)
        del outs_p
    # the ring: series of 1024 samples per surface instead of 4096 (the
    # handles' whole-record buffers are released first, so the free memory
    # below is what a streamed call needs)
    for sx in surfs:
        sx.close()
    surfs = [FWH.from_workload(x, "mixed") for x in ws5]
    surfs[0].set_batch_options(1024, "pipelined")
    outs_r = batch_forward(surfs, fields)
    ms_r = _time_calls(lambda: batch_forward(surfs, fields, outs_r), 3, warm=1)
    surfs[0].check()
    free_r = torch.cuda.mem_get_info()[0]
    err_r = rel_l2_stats(outs_r[small].cpu().numpy(), nv, p_ref, nv_ref, pick)
    out["batch"] = {"workload": "eight surfaces, 524288 panels x 4096 steps x 1024 observers each",
                    "evals": ev5, "ms": ms_b, "evals_per_s": ev5 / (ms_b / 1e3),
                    "form": "pipelined: whole records, one launch per surface, each "
                            "surface's prep under the scatters before it",
                    "per_surface_calls_ms": ms_s, "per_surface_evals_per_s": ev5 / (ms_s / 1e3),
                    "grid_ms": ms_f["grid"], "grid_evals_per_s": ev5 / (ms_f["grid"] / 1e3),
                    "persistent_ms": ms_f["persistent"],
                    "persistent_evals_per_s": ev5 / (ms_f["persistent"] / 1e3),
                    "grid_vs_oracle_rel_l2": err_f["grid"],
                    "persistent_vs_oracle_rel_l2": err_f["persistent"],
                    "streamed_ms": ms_r, "streamed_evals_per_s": ev5 / (ms_r / 1e3),
                    "streamed_form": "pipelined, ring of 2 x 512 samples per surface, 4 rounds",
                    "device_free_gb_whole_records": free_b / 1e9,
                    "device_free_gb_streamed": free_r / 1e9,
                    "mixed_vs_oracle_rel_l2": err_b, "streamed_vs_oracle_rel_l2": err_r,
                    "oracle_evals_per_s": orate,
                    "oracle_sample": f"surface {small} ({ws5[small].surface.n_panels} panels), "
                                     "2 observers"}
    del outs_r
    for sx in surfs:
        sx.close()
    del surfs, fields, outs
    torch.cuda.empty_cache()
    out["moving"] = moving_leg(dev)
    return out


def moving_leg(dev):
    """The general moving-surface form (Sec. II B, fwh_forward_moving, FP64): a
    sphere of 8192 panels spinning at 0.3 c0 around a stationary monopole,
    2048 steps, 16 observers at rest; the oracle on one observer."""
    import numpy as np
    import torch
    from fwh_inputs.geometry import observers_fibonacci, uv_sphere
    from oracle.oracle import forward_moving
    from paper_2312_16263_gb300 import moving_forward
    nt, dt, Om, c0, A, om = 2048, 0.02, 0.3, 1.0, 1e-4, np.pi
    s = uv_sphere(1.0, 64, 128)
    P = s.n_panels
    tau = torch.arange(nt, dtype=torch.float64, device=dev) * dt
    c, sn = torch.cos(Om * tau), torch.sin(Om * tau)
    rot = torch.zeros((nt, 3, 3), dtype=torch.float64, device=dev)
    rot[:, 0, 0], rot[:, 0, 1], rot[:, 1, 0], rot[:, 1, 1], rot[:, 2, 2] = c, -sn, sn, c, 1.0
    y = torch.einsum("tij,pj->tpi", rot, torch.as_tensor(s.centroids, device=dev)).contiguous()
    n = torch.einsum("tij,pj->tpi", rot, torch.as_tensor(s.normals, device=dev)).contiguous()
    v = torch.cross(torch.tensor([0.0, 0.0, Om], dtype=torch.float64, device=dev).expand_as(y), y,
                    dim=-1).contiguous()
    # stationary monopole (linear acoustics) sampled on the moving panels
    r = torch.linalg.norm(y, dim=-1)
    ph = om * (tau[:, None] - r / c0)
    amp = A / (4 * np.pi * r)
    e_re, e_im = amp * torch.cos(ph), amp * torch.sin(ph)
    dr_re = -e_re / r + om / c0 * e_im          # Re[e (-1/r - i om/c0)]
    p = om * e_im                                # -Re[i om e], rho0 = 1
    f = torch.empty((nt, 5, P), dtype=torch.float64, device=dev)
    f[:, 0] = p / (c0 * c0)
    f[:, 1:4] = (dr_re[..., None] * y / r[..., None]).permute(0, 2, 1)
    f[:, 4] = p
    obs = observers_fibonacci(15.0, 16, np.zeros(3))
    out = torch.empty((16, nt), dtype=torch.float64, device=dev)
    ms = _time_calls(lambda: moving_forward(y, n, v, s.areas, c0, 1.0, dt, f, obs, out=out), 3,
                     warm=1)
    _, ts, nv = moving_forward(y, n, v, s.areas, c0, 1.0, dt, f, obs, out=out)
    t0 = time.perf_counter()
    p_ref, _, nv_ref = forward_moving(y.cpu().numpy(), n.cpu().numpy(), v.cpu().numpy(), s.areas,
                                      c0, 1.0, dt, f.cpu().numpy(), obs[:1])
    orate = P * nt / (time.perf_counter() - t0)
    k = int(min(nv[0], nv_ref[0]))
    err = float(np.linalg.norm(out[0, :k].cpu().numpy() - p_ref[0, :k]) /
                np.linalg.norm(p_ref[0, :k]))
    evals = P * nt * 16
    return {"workload": "sphere 8192 panels spinning at 0.3 c0 around a monopole, 2048 steps, "
                        "16 observers at rest (FP64)",
            "evals": evals, "ms": ms, "evals_per_s": evals / (ms / 1e3),
            "rel_l2_vs_oracle_observer0": err, "oracle_evals_per_s": orate}


def rel_l2_stats(p_gpu, nv_gpu, p_ref, nv_ref, idx):
    import numpy as np
    errs = []
    for k, o in enumerate(idx):
        n = int(min(nv_gpu[o], nv_ref[k]))
        ref = p_ref[k, :n]
        errs.append(float(np.linalg.norm(p_gpu[o, :n] - ref) / np.linalg.norm(ref)))
    return {"max": max(errs), "median": statistics.median(errs)}


def run_reference(args, ws, rank):
    """Reference arm: the FP64 CPU oracle (the paper ships no GPU code), timed
    as it stands on the host cores, one bounded sample (one observer of the
    same workload, all panels and steps) per step."""
    if rank != 0:
        return
    import numpy as np
    from oracle import Oracle
    from oracle.oracle import max_threads
    w = rank_workload(0, 1)
    f = w.fields("float32").double().numpy()
    orc = Oracle.from_workload(w)
    evals = w.surface.n_panels * w.nt
    for i in range(args.warmup):
        orc.forward(f, w.observers[i % 72:i % 72 + 1])
    times = []
    for i in range(args.steps):
        o = (7 * i) % 72
        t0 = time.perf_counter()
        orc.forward(f, w.observers[o:o + 1])
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = evals / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "panels": w.surface.n_panels, "nt": w.nt,
                       "observers_per_step": 1, "sample": "one observer per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": max_threads(),
                             "kind": "oracle", "sample": "1 of 72 observers per step, all "
                             f"{w.surface.n_panels} panels x {w.nt} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_batch(args):
    """fwh_forward, then a batch of that one surface as one grid and as the
    persistent work queue (same items, same kernel code), twice each in that
    order (about 4 GB on the device): the capture target for comparing the
    three launches (k_forward* launches 4 to 6 are the second round)."""
    import torch
    from __graft_entry__ import build
    build()
    from fwh_inputs import batch_workloads
    from paper_2312_16263_gb300 import FWH, batch_forward
    w = batch_workloads(scale=0.25, nt=2048)[1]
    s = FWH.from_workload(w, "mixed")
    f = w.fields(device="cuda:0", dtype="float32")
    out = torch.empty((s.O, w.nt), dtype=torch.float64, device="cuda:0")
    res = {}
    for _ in range(2):
        s.forward(f, out)
        for form in ("grid", "persistent"):
            s.set_batch_options(0, form)
            res[form] = batch_forward([s], [f])[0]
    torch.cuda.synchronize()
    s.check()
    print(json.dumps({"profile_batch": w.name, "P": w.surface.n_panels, "nt": w.nt,
                      "O": int(s.O), "max_diff": max(float((r - out).abs().max())
                                                     for r in res.values())}))


def main():
    args = parse_args()
    if args.profile_backward:
        profile_backward(args)
        return
    if args.profile_case:
        profile_case(args)
        return
    if args.profile_batch:
        profile_batch(args)
        return
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import numpy as np
    import torch

    from __graft_entry__ import build
    build()
    from paper_2312_16263_gb300 import FWH

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    peaks = measured_fma_peaks()
    w = rank_workload(rank, ws)
    evals = w.evals
    s = FWH.from_workload(w, "mixed")
    f = w.fields(device=dev, dtype="float32")
    out = torch.empty((s.O, w.nt), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        s.forward(f, out)
    torch.cuda.synchronize()
    s.check()
    s.set_timing(True)
    s.timing_totals(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            s.forward(f, out)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
    ms_step = e0.elapsed_time(e1) / args.steps
    tt = s.timing_totals(reset=True)
    s.set_timing(False)
    s.check()
    ms_max = max_over_ranks(ms_step, ws)
    value = evals * ws / (ms_max / 1e3)
    fwd_ms = tt["forward_ms"] / max(1, tt["calls"])
    prep_ms = tt["prep_ms"] / max(1, tt["calls"])
    achieved = evals * FLOP_PER_EVAL / (fwd_ms / 1e3) / 1e12
    # series prep: FP32 fields read once, FP32 series rows (16 values per panel
    # and padded step) written once
    ntp = (w.nt + 255) // 256 * 256
    prep_bytes = w.nt * 5 * w.surface.n_panels * 4 + w.surface.n_panels * ntp * 16 * 4
    hbm_gbs, hbm_src = hbm_peak_gbs()
    traffic = profile_traffic()
    p_mixed = out.cpu().numpy()
    _, nv = s.window(w.nt)

    # plain FP64 form on the same workload
    s64 = FWH.from_workload(w, "fp64")
    f64 = f.double()
    out64 = torch.empty_like(out)
    s64.forward(f64, out64)
    torch.cuda.synchronize()
    s64.set_timing(True)
    s64.timing_totals(reset=True)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(args.fp64_steps):
        s64.forward(f64, out64)
    a1.record(stream)
    torch.cuda.synchronize()
    ms64 = a0.elapsed_time(a1) / args.fp64_steps
    tt64 = s64.timing_totals(reset=True)
    fwd64 = tt64["forward_ms"] / max(1, tt64["calls"])
    p64 = out64.cpu().numpy()
    s64.check()
    s64.close()
    del f64, out64
    den = np.linalg.norm(p64, axis=1)
    rel_mixed_fp64 = np.linalg.norm(p_mixed - p64, axis=1) / np.where(den > 0, den, 1)

    # end to end through the C ABI with host buffers (pinned), copies timed
    fh = f.cpu().pin_memory()
    oh = torch.empty((s.O, w.nt), dtype=torch.float64).pin_memory()
    s.forward(fh, oh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        s.forward(fh, oh)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e_ms_max = max_over_ranks(e2e_s * 1e3, ws)
    # the host path scatters shorter time segments (overlapped with the copy),
    # which splits FP32 per-bin partial sums differently: equal to FP32 rounding
    e2e_den = np.linalg.norm(p_mixed, axis=1)
    e2e_rel = np.linalg.norm(oh.numpy() - p_mixed, axis=1) / np.where(e2e_den > 0, e2e_den, 1)
    assert e2e_rel.max() <= 1e-5, e2e_rel.max()
    clocks = clk.summary()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (analytic convected x1-dipole, A=0.01, omega=4 pi)",
        "config": {"workload": w.name, "panels": w.surface.n_panels, "nt": w.nt,
                   "observers_per_gpu": s.O, "precision": "mixed (FP32 series and integrand "
                   "arithmetic, FP64 arrival times/weights and output)",
                   "l2": "inputs larger than L2 (1.34 GB fields, 4.3 GB series per step)",
                   "parallelism": f"observer sets x{ws}, no collective"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": traffic,
                     "kernel": "k_forward (forward scatter)",
                     "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 flop x 2.07 GHz",
                     "peak_measured": peaks["fp32"],
                     "frac_of_measured": achieved / peaks["fp32"],
                     "peak_measured_source": "FMA-chain probe fwh_fma_peak (FP32)",
                     "kernel_ms": fwd_ms, "prep_ms": prep_ms,
                     "flop_per_eval": FLOP_PER_EVAL},
        "fp64": {"value": evals * ws / (max_over_ranks(ms64, ws) / 1e3), "unit": UNIT,
                 "ms_per_step": ms64, "kernel_ms": fwd64,
                 "achieved_tflops": evals * FLOP_PER_EVAL / (fwd64 / 1e3) / 1e12,
                 "peak_tflops": FP64_PEAK_TFLOPS, "peak_source": "nominal GB300 FP64",
                 "frac": evals * FLOP_PER_EVAL / (fwd64 / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                 "peak_measured": peaks["fp64"],
                 "frac_of_measured": evals * FLOP_PER_EVAL / (fwd64 / 1e3) / 1e12 / peaks["fp64"]},
        "accuracy": {"mixed_vs_fp64_rel_l2_max": float(rel_mixed_fp64.max()),
                     "mixed_vs_fp64_rel_l2_median": float(np.median(rel_mixed_fp64))},
        "e2e": {"value": evals * ws / (e2e_ms_max / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(fh.numel() * fh.element_size()),
                "d2h_bytes_per_step": int(oh.numel() * oh.element_size()),
                "ms_per_step": e2e_ms_max},
        "prep": {"bound": "hbm", "kernels": "k_prep_iir_int (interior blocks) + k_prep_iir "
                 "(record ends)", "ms": prep_ms, "bytes": prep_bytes,
                 "achieved": prep_bytes / (prep_ms / 1e3) / 1e9, "peak": hbm_gbs,
                 "unit": "GB/s", "frac": prep_bytes / (prep_ms / 1e3) / 1e9 / hbm_gbs,
                 "peak_source": hbm_src},
        # per step: the two prep kernels and the forward scatter
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    # PSD of the far-field signals (Sec. IV C): Welch, 512-sample segments
    from paper_2312_16263_gb300 import welch_psd
    from oracle.psd import observer_psd
    psd_ms = _time_calls(lambda: welch_psd(out, 1.0 / w.dt, 512, nv), 20)
    psd_gpu = welch_psd(out, 1.0 / w.dt, 512, nv).cpu().numpy()
    psd_ref = observer_psd(p_mixed, nv, 1.0 / w.dt, 512)
    line["psd"] = {"kernel": "k_psd", "ms": psd_ms, "signals": int(s.O), "nperseg": 512,
                   "rel_err_vs_oracle_max": float(np.nanmax(np.abs(psd_gpu - psd_ref)) /
                                                  np.nanmax(np.abs(psd_ref)))}
    if rank == 0 and ws == 1 and not args.no_extra:
        del fh, oh
        torch.cuda.empty_cache()
        try:
            line.update(extra_legs(dev))
        except Exception as e:  # the extra keys never cost the headline line
            line["extra_legs_error"] = f"{type(e).__name__}: {e}"[:500]
            torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb, (pick, p_ref, nv_ref) = cpu_baseline(w)
        line["cpu_baseline"] = cb
        line["accuracy"]["mixed_vs_oracle_rel_l2"] = rel_l2_stats(p_mixed, nv, p_ref, nv_ref, pick)
        line["accuracy"]["fp64_vs_oracle_rel_l2"] = rel_l2_stats(p64, nv, p_ref, nv_ref, pick)
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
