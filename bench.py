#!/usr/bin/env python
"""Benchmark of the hot path: eps(p) build + adjoint-gradient VJP.

One step = one pass of the whole path over the 3D two-etch grating
(600 x 200 x 120 Yee cells, 3 components, 60 etched boxes, 120 edge
parameters): host FP64 parameter map, binner, eps/fill build, band VJP over
the complex64 forward/adjoint fields, deterministic finalize.  The
parameters change every step (as in an optimiser loop), so nothing is cached
across steps.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead, on a bounded sample of the same workload.  Under torchrun each rank
runs its own replica (the path shards across designs with no collective).
"""
from __future__ import annotations

import argparse
import math
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "grid cells/s for eps(p)+VJP gradient"
WORKLOAD = ("3D two-etch grating: Yee grid 600x200x120, Ex/Ey/Ez, dx=dy=40 nm, dz=20 nm, "
            "220 nm slab, 2 etch depths x 30 teeth (60 exact-overlap boxes), 120 edge params, "
            "complex64 fwd+adj fields (6 arrays, seeded plane waves x Gaussian)")


def reduce_max(x: float, dist, device) -> float:
    """The largest of x over the ranks (the slowest replica's time); x itself
    with one rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, units_per_rank: float, ms: float) -> float:
    """Whole-job throughput of `world` replicas that each process
    `units_per_rank` units per step, with the max-over-ranks step time."""
    return world * units_per_rank / (ms * 1e-3)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampler (SM clock, max clock, throttle reasons) run alongside
    the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms",
                 "50", "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        import statistics
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def crop(desc, k0, nzs, j0=0, nys=None):
    """The same design restricted to z-planes [k0, k0 + nzs) and y-rows
    [j0, j0 + nys) (bounded CPU samples)."""
    d = dict(desc)
    g = dict(desc["grid"])
    n = list(g["n"])
    n[2] = nzs
    if nys is not None:
        n[1] = nys
    g["n"] = tuple(n)
    o = list(g["o"])
    o[1] = o[1] + j0 * g["d"][1]
    o[2] = o[2] + k0 * g["d"][2]
    g["o"] = tuple(o)
    d["grid"] = g
    return d


def _oracle_box(desc, ef, ea, w, target_s):
    """A block of z-planes (through the middle of the grid) and y-rows whose
    oracle fill + gradient take about `target_s` on this host.  The oracle
    runs its z-planes in parallel, so the probe takes one plane per thread;
    shorter targets keep the planes and drop y-rows."""
    from oracle import oracle as O
    nx, ny, nz = desc["grid"]["n"]
    kc = nz // 2
    probe = max(1, min(nz, O.num_threads()))
    k0 = max(0, kc - probe // 2)
    t0 = time.perf_counter()
    O.fill(crop(desc, k0, probe))
    O.grad(crop(desc, k0, probe), ef[:, k0:k0 + probe].copy(), ea[:, k0:k0 + probe].copy(), w)
    t1 = max(time.perf_counter() - t0, 1e-3)
    if target_s >= t1:  # whole multiples of the thread count keep every thread busy
        planes = int(max(1, min(nz, probe * math.ceil(target_s / t1))))
        return max(0, kc - planes // 2), planes, 0, ny
    rows = int(max(1, ny * target_s / t1))
    return k0, probe, (ny - rows) // 2, rows


def _sample(desc, ef, ea, box):
    k0, nzs, j0, nys = box
    return (crop(desc, k0, nzs, j0, nys), ef[:, k0:k0 + nzs, j0:j0 + nys].copy(),
            ea[:, k0:k0 + nzs, j0:j0 + nys].copy())


def _sample_text(desc, box):
    nx, ny, nz = desc["grid"]["n"]
    k0, nzs, j0, nys = box
    return ("%d of %d z-planes x %d of %d y-rows (%d cells x %d components) through the middle "
            "of the grid" % (nzs, nz, nys, ny, nx * nys * nzs, desc["grid"]["ncomp"]))


def oracle_sample(desc, ef, ea, w, target_s=15.0):
    """Time the oracle (fill + gradient, as it stands) on a block through the
    slab, about `target_s` of CPU work.  Returns (cells/s, cores, description,
    timings: the box, the fill's and the gradient's seconds, the fill)."""
    from oracle import oracle as O
    nx = desc["grid"]["n"][0]
    box = _oracle_box(desc, ef, ea, w, target_s)
    sub, efs, eas = _sample(desc, ef, ea, box)
    t0 = time.perf_counter()
    f = O.fill(sub)
    t1 = time.perf_counter()
    O.grad(sub, efs, eas, w)
    dt = time.perf_counter() - t0
    cells = nx * box[1] * box[3]
    timings = {"box": box, "fill_s": t1 - t0, "grad_s": dt - (t1 - t0), "fill": f}
    return cells / dt, O.num_threads(), "%s; one oracle fill + one oracle gradient, %.1f s" % (
        _sample_text(desc, box), dt), timings


def oracle_methods(desc, ef, ea, w, timings, gpu_value, target_1core_s=5.0):
    """The oracle's two host methods on this workload, in cells/s of the whole
    step (cells of the sample over its time):
    - analytic: the VJP of Sec. 3 (one eps evaluation and one reverse sweep),
      from the timed sample on all cores, and on one core on a smaller block;
    - fd: the finite-difference baseline of Sec. 2 -- n + 1 eps builds and n
      multiply-reduces for n parameters -- extrapolated from the timed build
      and from four multiply-reduces timed on the sample (z = Re(w E_adj E_fwd)
      formed once, then one dot product with a fill difference per parameter).
    analytic_over_fd is the ratio of the two on the same host (the comparison
    of Secs. 6.1 and 6.3); the GPU's speed-up over each is value / method."""
    import numpy as np
    from oracle import oracle as O
    nx, ny, nz = desc["grid"]["n"]
    k0, nzs, j0, nys = timings["box"]
    cells = nx * nzs * nys
    t_fill, t_grad = timings["fill_s"], timings["grad_s"]
    n = len(desc["params"])
    analytic = cells / (t_fill + t_grad)
    # FD's multiply-reduce on the sample's arrays
    _, efs, eas = _sample(desc, ef, ea, timings["box"])
    f = np.asarray(timings["fill"], dtype=np.float64)
    wv = np.asarray(w, dtype=np.complex128).reshape(-1, 1, 1, 1)
    t0 = time.perf_counter()
    z = np.real(wv * eas.astype(np.complex128) * efs.astype(np.complex128))
    t_z = time.perf_counter() - t0
    t0 = time.perf_counter()
    for _ in range(4):
        float(np.vdot(z.ravel(), f.ravel()))
    t_dot = (time.perf_counter() - t0) / 4
    t_fd = t_z + (n + 1) * t_fill + n * t_dot
    # the analytic method on one core: the same z-planes as the sample above
    # (the same mix of slab and cladding cells), fewer y-rows, sized from a
    # one-row probe to about target_1core_s
    threads = O.num_threads()
    O.set_threads(1)
    try:
        jp = j0 + nys // 2
        sub, es, as_ = _sample(desc, ef, ea, (k0, nzs, jp, 1))
        t0 = time.perf_counter()
        O.fill(sub)
        O.grad(sub, es, as_, w)
        tp = max(time.perf_counter() - t0, 1e-3)
        rows = int(max(1, min(nys, target_1core_s / tp)))
        j1 = j0 + (nys - rows) // 2
        box1 = (k0, nzs, j1, rows)
        sub, es, as_ = _sample(desc, ef, ea, box1)
        t0 = time.perf_counter()
        O.fill(sub)
        O.grad(sub, es, as_, w)
        t1c = time.perf_counter() - t0
    finally:
        O.set_threads(threads)
    one_core = nx * nzs * rows / t1c
    return {
        "unit": "cells/s", "params": n,
        "analytic_all_cores": {"value": analytic, "cores": threads,
                               "sample": _sample_text(desc, timings["box"])},
        "analytic_one_core": {"value": one_core, "cores": 1, "sample": _sample_text(desc, box1)},
        "fd_all_cores": {"value": cells / t_fd, "cores": threads,
                         "how": "(n + 1) timed oracle fills + n dot products of z with a fill "
                                "difference, extrapolated from one fill and four dot products "
                                "on the sample"},
        "analytic_over_fd": t_fd / (t_fill + t_grad),  # the paper's AD-vs-FD comparison, one host
        "gpu_over_analytic": gpu_value / analytic, "gpu_over_analytic_one_core": gpu_value / one_core,
        "gpu_over_fd": gpu_value / (cells / t_fd)}


def grid_of(args):
    """The grating's grid: 600x200x120 unless --grid NXxNYxNZ asks for another."""
    g = getattr(args, "grid", "") or "600x200x120"
    return tuple(int(v) for v in g.split("x"))


def workload_name(n):
    if tuple(n) == (600, 200, 120):
        return WORKLOAD
    return WORKLOAD.replace("600x200x120", "%dx%dx%d" % tuple(n))


def make_inputs(n=(600, 200, 120)):
    import numpy as np
    from paper_2311_05646_gb300 import inputs as I
    desc = I.grating_3d(n=tuple(n))
    ef = I.plane_wave_field(desc, 22)
    ea = I.plane_wave_field(desc, 23)
    w = np.full(3, -2j, dtype=np.complex64)  # Eq. 1: w = -2 i omega, omega = 1
    return desc, ef, ea, w


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    desc, ef, ea, w = make_inputs(grid_of(args))
    from oracle import oracle as O
    nx, ny, nz = desc["grid"]["n"]
    # bounded sample per step: z-planes through the slab, sized so that the
    # whole run (warm-up + timed steps) takes about two minutes
    per_step = min(2.0, 120.0 / max(1, args.steps + args.warmup))
    box = _oracle_box(desc, ef, ea, w, per_step)
    sub, efs, eas = _sample(desc, ef, ea, box)
    p0 = desc["params"]
    for k in range(args.warmup):
        O.fill(sub, p0 + 0.01 * (k % 2))
        O.grad(sub, efs, eas, w, params=p0 + 0.01 * (k % 2))
    t0 = time.perf_counter()
    for k in range(args.steps):
        O.fill(sub, p0 + 0.01 * (k % 2))
        O.grad(sub, efs, eas, w, params=p0 + 0.01 * (k % 2))
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    cells = nx * box[1] * box[3]
    value = cells / dt
    sample = "%s per step: one oracle fill + one oracle gradient" % _sample_text(desc, box)
    line = {"metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(grid_of(args)), "sample": sample},
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": O.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _traffic(kernel, tile=None, grid=(600, 200, 120)):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when the kernel source (or the tile shape, or the grid) differs from
    the one the counters were taken on."""
    if tuple(grid) != (600, 200, 120):
        return None
    try:
        import hashlib
        tr = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
        src = open(os.path.join(ROOT, "paper_2311_05646_gb300", "csrc", "adg_kernels.cu"), "rb").read()
        if tile is not None and list(tr.get("tile", [])) != list(tile):
            return None
        if tr.get("source_sha256") == hashlib.sha256(src).hexdigest() and kernel in tr.get("kernels", {}):
            return tr["kernels"][kernel]["dram_bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        pass
    return None


def run_adg(args):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_2311_05646_gb300 import adg

    desc, ef_h, ea_h, w = make_inputs(grid_of(args))
    nx, ny, nz = desc["grid"]["n"]
    C = desc["grid"]["ncomp"]
    cells = nx * ny * nz
    ctx = adg.Context(local)
    efd = torch.from_numpy(ef_h).cuda()
    ead = torch.from_numpy(ea_h).cuda()
    # the tile shape: given, the library's default, or (default) the project's
    # autotuner, which times each candidate shape on this design and fields
    # before the benchmark starts
    tuned = False
    if args.tile:
        tile = tuple(int(v) for v in args.tile.split("x"))
    elif args.no_tune:
        tile = None
    else:
        from paper_2311_05646_gb300.tuning import Autotuner
        tile = Autotuner(ctx, reps=16).best(desc, fields=(efd, ead))
        tuned = True
    design = adg.Design(ctx, desc, tile=tile)
    fill = torch.empty(design.shape, dtype=torch.float32, device="cuda")
    eps = torch.empty_like(fill)
    g = torch.zeros(design.n_params, dtype=torch.float32, device="cuda")
    p0 = desc["params"].copy()
    params = [p0 + 0.01 * (k % 2) for k in range(2)]  # alternate: every step re-bins
    stream = torch.cuda.current_stream()

    def step(k):
        p = params[k % 2]
        adg.adg_build_eps(design, p, eps, fill=fill, stream=stream)
        adg.adg_grad(design, p, efd, ead, w, g, stream=stream)

    for k in range(args.warmup):
        step(k)
    adg.adg_sync(ctx, stream)

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    for k in range(50):  # keep the GPU busy while the sampler starts
        step(k)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks.stop()
    adg.adg_sync(ctx, stream)
    ms = e0.elapsed_time(e1) / args.steps
    # per-kernel times: the same steps again with every launch bracketed by
    # events (kept out of the timed loop above)
    adg.adg_profile_read(ctx, reset=True)
    adg.adg_profile_enable(ctx, True)
    for k in range(min(args.steps, 200)):
        step(k)
    torch.cuda.synchronize()
    adg.adg_profile_enable(ctx, False)
    prof = adg.adg_profile_read(ctx, reset=True)
    adg.adg_sync(ctx, stream)
    ms = reduce_max(ms, dist, "cuda")
    stats = adg.adg_design_stats(design, stream)
    value = replica_value(world, cells, ms)

    # roofline of the dominant kernel (HBM-bound): algorithmic bytes / launch
    # the build writes fill + eps (fp32) of every sample: constant tiles by a
    # streaming fill, band tiles by program evaluation, in one kernel
    bytes_build = cells * C * 4 * 2
    # E_fwd + E_adj complex64 of the samples whose Jacobian row can be nonzero
    bytes_vjp = stats["active_samples"] * 16
    kern = {"build": bytes_build, "vjp": bytes_vjp}
    dom = max(kern, key=lambda k: prof[k][1])
    n_l, tot_ms = prof[dom]
    avg_ms = tot_ms / max(n_l, 1)
    achieved = kern[dom] / (avg_ms * 1e-3) / 1e9
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    fill_warps = int(tile[3]) if tile is not None and len(tile) > 3 else 1
    opts = list(stats["tile"]) + ([fill_warps] if fill_warps > 1 else [])
    traffic = _traffic(dom, opts, (nx, ny, nz))
    roof = {"bound": "hbm", "kernel": "k_" + dom, "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "algorithmic_bytes_per_launch": kern[dom],
            "peak_source": "measured" if peaks else "fallback",
            "note": ("the VJP reads the fields only of the samples where d eps / d p can be "
                     "nonzero, so it is latency-bound, not HBM-bound; the HBM-bound kernels are "
                     "the build (kernels.build: fill + eps of every sample) and the dense field "
                     "stream (dense_vjp.stream_*)") if dom == "vjp" else
                    ("the build writes fill + eps of every sample; its band tiles (program "
                     "evaluation, latency-bound) and the constant-tile stream run in separate "
                     "warps; the VJP (kernels.vjp) reads the fields only where d eps / d p can "
                     "be nonzero and is latency-bound")}
    # the whole step against the same peak: its algorithmic bytes (fill + eps
    # of every sample, the fields of the active samples) over the step time
    step_bytes = bytes_build + bytes_vjp
    step_roof = {"algorithmic_bytes": step_bytes, "ms": ms,
                 "achieved_GBps": step_bytes / (ms * 1e-3) / 1e9,
                 "frac_of_measured_hbm": step_bytes / (ms * 1e-3) / 1e9 / peak,
                 "floor_ms": step_bytes / (peak * 1e9) * 1e3}
    kernels = {k: {"launches": v[0], "ms_total": v[1],
                   "us_per_launch": 1e3 * v[1] / max(v[0], 1)} for k, v in prof.items() if v[0]}
    for k in kern:
        if k not in kernels:
            continue
        a = kern[k] / (kernels[k]["us_per_launch"] * 1e-6) / 1e9
        kernels[k]["GBps"] = a
        kernels[k]["frac_of_measured_hbm"] = a / peak
    # kernels launched in the timed region: the profiled steps' count per step
    launches = int(round(sum(v[0] for v in prof.values()) / min(args.steps, 200) * args.steps))

    # the dense form of the gradient (every cell's fields streamed for the
    # material-level derivatives) against the plain one, each call timed alone
    dense = None
    if not args.no_dense:
        gm = torch.zeros(2, dtype=torch.float64, device="cuda")
        p = params[0]
        adg.adg_build_eps(design, p, eps, fill=fill, stream=stream)
        nd = max(20, min(args.steps, 200))

        def t_calls(fn):
            for _ in range(5):
                fn()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(nd):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / nd

        ms_plain = t_calls(lambda: adg.adg_grad(design, p, efd, ead, w, g, stream=stream))
        adg.adg_profile_read(ctx, reset=True)
        adg.adg_profile_enable(ctx, True)
        ms_dense = t_calls(lambda: adg.adg_grad_dense(design, p, efd, ead, w, fill, g, gm,
                                                      stream=stream))
        adg.adg_profile_enable(ctx, False)
        dprof = adg.adg_profile_read(ctx, reset=True)
        adg.adg_sync(ctx, stream)
        stream_bytes = cells * C * (8 + 8 + 4)  # E_fwd, E_adj complex64 + fill fp32
        n_l, tot = dprof["dense"]
        us_k = 1e3 * tot / max(n_l, 1)
        dense = {"grad_ms": ms_dense, "plain_grad_ms": ms_plain,
                 "cells_per_s": world * cells / (ms_dense * 1e-3),
                 "outputs": "g (band VJP) + dL/d eps_bg, dL/d eps_fg (every cell)",
                 "stream_kernel": "k_dense (+ fixed-order sum)",
                 "stream_bytes_per_launch": stream_bytes, "stream_us_per_launch": us_k,
                 "stream_GBps": stream_bytes / (us_k * 1e-6) / 1e9,
                 "stream_frac_of_measured_hbm": stream_bytes / (us_k * 1e-6) / 1e9 / peak,
                 "stream_traffic": _traffic("dense", opts, (nx, ny, nz)),
                 "call_GBps": (stream_bytes + kern["vjp"]) / (ms_dense * 1e-3) / 1e9,
                 "call_frac_of_measured_hbm": (stream_bytes + kern["vjp"]) / (ms_dense * 1e-3) / 1e9 / peak,
                 "vjp_us_per_launch": 1e3 * dprof["vjp"][1] / max(dprof["vjp"][0], 1)}

    # the topology special case (Sec. 3.1) on the same grid and fields: every
    # (x, y) pixel of the grid a parameter, broadcast over 16 z cells through
    # the slab; both kernels are HBM streams
    topo = None
    if not args.no_dense:
        z0 = max(0, nz // 2 - 8)
        region = (0, 0, nx, ny, z0, min(nz, z0 + 16))
        npix = nx * ny
        nsamp = npix * (region[5] - region[4]) * C
        vt = torch.randn(npix, dtype=torch.float32, device="cuda")
        gt = torch.empty(npix, dtype=torch.float32, device="cuda")
        et = torch.empty_like(eps)
        nt = 50

        def t_topo(fn):
            for _ in range(5):
                fn()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(nt):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / nt

        us_e = 1e3 * t_topo(lambda: adg.adg_topo_eps(ctx, (nx, ny, nz), C, region, vt, 2.085, 10.025,
                                                      et, stream=stream))
        us_g = 1e3 * t_topo(lambda: adg.adg_topo_grad(ctx, (nx, ny, nz), C, region, vt, 10.025, efd,
                                                       ead, w, gt, stream=stream))
        b_e, b_g = nsamp * 4 + npix * 4, nsamp * 16 + npix * 8
        topo = {"region": list(region), "pixels": npix, "samples": nsamp,
                "eps_us": us_e, "eps_GBps": b_e / (us_e * 1e-6) / 1e9,
                "eps_frac_of_measured_hbm": b_e / (us_e * 1e-6) / 1e9 / peak,
                "grad_us": us_g, "grad_GBps": b_g / (us_g * 1e-6) / 1e9,
                "grad_frac_of_measured_hbm": b_g / (us_g * 1e-6) / 1e9 / peak,
                "bytes": {"eps": b_e, "grad": b_g}}

    # the paper's comparison (Sec. 3, Sec. 6): the finite-difference gradient
    # -- two builds per parameter with the library's own exact mesher and a
    # dot product with Re(w E_adj E) -- against the AutoDiff gradient, on the
    # same GPU, fields and parameters
    fdc = None
    if not args.no_dense:
        gfd = torch.zeros_like(g)
        gad = torch.zeros_like(g)
        adg.adg_grad(design, p0, efd, ead, w, gad, stream=stream)
        adg.adg_grad_fd(design, p0, efd, ead, w, 0.5, gfd, stream=stream)
        adg.adg_sync(ctx, stream)
        torch.cuda.synchronize()
        nf = 3
        e0.record(stream)
        for _ in range(nf):
            adg.adg_grad_fd(design, p0, efd, ead, w, 0.5, gfd, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_fd = e0.elapsed_time(e1) / nf
        e0.record(stream)
        for _ in range(nf * 20):
            adg.adg_grad(design, params[_ % 2], efd, ead, w, gad, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_ad = e0.elapsed_time(e1) / (nf * 20)
        adg.adg_grad(design, p0, efd, ead, w, gad, stream=stream)
        adg.adg_sync(ctx, stream)
        ga, gf = gad.double(), gfd.double()
        fdc = {"params": int(design.n_params), "h_nm": 0.5, "fd_builds": 2 * int(design.n_params),
               "fd_ms": ms_fd, "ad_ms": ms_ad, "ad_speedup": ms_fd / ms_ad,
               "fd_vs_ad_rel_l2": float((gf - ga).norm() / ga.norm())}

    # the union over non-binary material levels (App. B, Alg. 1) on the same
    # grid and fields: four sets of overlapping circles and boxes at four
    # material levels; the per-sample pass of Alg. 1 is an HBM stream (K fills
    # in, eps out; or K fills and the two fields in, K cotangents out)
    levels = None
    if not args.no_dense:
        from paper_2311_05646_gb300 import inputs as I
        lvm = I.nonbinary_circles(n=(nx, ny, nz), d=desc["grid"]["d"], per_level=8,
                                  levels=(1.9, 5.0, 9.0, 10.025), eps_bg=2.085, seed=91)
        sets = [adg.Design(ctx, dd) for dd in lvm["sets"]]
        pl = lvm["sets"][0]["params"]
        gl = torch.zeros(sets[0].n_params, dtype=torch.float32, device="cuda")
        nl = 20

        def t_lv(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            adg.adg_profile_read(ctx, reset=True)
            adg.adg_profile_enable(ctx, True)
            e0.record(stream)
            for _ in range(nl):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            adg.adg_profile_enable(ctx, False)
            pr = adg.adg_profile_read(ctx, reset=True)
            return e0.elapsed_time(e1) / nl, 1e3 * pr["levels"][1] / max(pr["levels"][0], 1)

        ms_le, us_ke = t_lv(lambda: adg.adg_levels_eps(sets, lvm["levels"], lvm["eps_bg"], pl, eps,
                                                        stream=stream))
        ms_lg, us_kg = t_lv(lambda: adg.adg_levels_grad(sets, lvm["levels"], pl, efd, ead, w, gl,
                                                         stream=stream))
        adg.adg_sync(ctx, stream)
        K, ns = len(sets), cells * C
        b_e, b_g = ns * (4 * K + 4), ns * (8 * K + 16)
        levels = {"sets": K, "params": int(sets[0].n_params), "samples": ns,
                  "eps_ms": ms_le, "grad_ms": ms_lg,
                  "pass_kernel": "k_levels",
                  "eps_pass_us": us_ke, "eps_pass_GBps": b_e / (us_ke * 1e-6) / 1e9,
                  "eps_pass_frac_of_measured_hbm": b_e / (us_ke * 1e-6) / 1e9 / peak,
                  "cot_pass_us": us_kg, "cot_pass_GBps": b_g / (us_kg * 1e-6) / 1e9,
                  "cot_pass_frac_of_measured_hbm": b_g / (us_kg * 1e-6) / 1e9 / peak,
                  "bytes": {"eps_pass": b_e, "cot_pass": b_g}}
        del sets

    # Prop. 2 / Sec. 6.3 on the same grid and fields: hexagonal holes through
    # the slab; the exact mesher's volume-averaged fill of the whole layer,
    # the FD gradient that re-meshes each parameter's region twice, and the
    # AutoDiffGeo gradient of the same holes as Poly2D hexagons
    mesh = None
    if not args.no_dense:
        from paper_2311_05646_gb300 import inputs as I
        spec = I.hex_hole_lattice(n=(nx, ny, nz), d=desc["grid"]["d"], holes=(max(1, nx // 30), 6),
                                  R=260.0, ncomp=C)
        hdesc = spec["desc"]
        hp = hdesc["params"]
        hdes = adg.Design(ctx, hdesc)
        layer = I.hex_layer(spec, hp)
        hfill = torch.empty_like(fill)
        mh = 0.5
        plus, minus, regions = I.hex_fd_layers(spec, hp, mh)
        plus, minus = adg.MeshLayers(plus), adg.MeshLayers(minus)  # the layouts, marshalled once
        hdeps = -(hdesc["eps_fg"] - hdesc["eps_bg"])
        gfd = torch.zeros(hdes.n_params, dtype=torch.float32, device="cuda")
        gad = torch.zeros_like(gfd)

        def t_mesh(fn, reps):
            fn()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        ms_mf = t_mesh(lambda: adg.adg_mesh_fill(ctx, hdesc["grid"], layer, hfill, stream=stream), 10)
        ms_fd = t_mesh(lambda: adg.adg_mesh_grad_fd(ctx, hdesc["grid"], plus, minus, regions, mh,
                                                    hdeps, efd, ead, w, gfd, stream=stream), 3)
        ms_ad = t_mesh(lambda: adg.adg_grad(hdes, hp, efd, ead, w, gad, stream=stream), 20)
        ga, gf = gad.double(), gfd.double()
        rsamp = sum(C * r[2] * r[3] * (r[5] - r[4]) for r in regions)
        mesh = {"holes": len(spec["centres"]), "params": int(hdes.n_params), "h_nm": mh,
                "mesh_fill_ms": ms_mf, "fd_exact_ms": ms_fd, "fd_meshes": 2 * int(hdes.n_params),
                "fd_region_samples": int(rsamp),
                "fd_region_fraction_of_grid": rsamp / (hdes.n_params * cells * C),
                "ad_ms": ms_ad, "ad_speedup": ms_fd / ms_ad,
                "ad_vs_fd_exact_rel_l2": float((ga - gf).norm() / gf.norm())}
        del hdes

    # end to end through the public API: host (pinned) fields in, eps + g out
    e2e = None
    if not args.no_e2e:
        efp = torch.from_numpy(ef_h).pin_memory()
        eap = torch.from_numpy(ea_h).pin_memory()
        eps_h = torch.empty(design.shape, dtype=torch.float32).pin_memory()
        g_h = torch.empty(design.n_params, dtype=torch.float32).pin_memory()
        ne = max(3, min(args.steps, 20))

        # Copies on their own streams: the host link carries one direction at
        # a time per stream, so the read-back of step k (D2H) runs while the
        # fields of step k+1 come in (H2D).  Events keep the buffers safe: the
        # fields are not overwritten before the VJP that reads them is done,
        # nor eps before its read-back is done.
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        state = {"comp": None, "out": None}

        def e2e_step(k):
            if state["comp"] is not None:
                s_in.wait_event(state["comp"])
            with torch.cuda.stream(s_in):
                efd.copy_(efp, non_blocking=True)
                ead.copy_(eap, non_blocking=True)
            ev_in = torch.cuda.Event()
            ev_in.record(s_in)
            stream.wait_event(ev_in)
            if state["out"] is not None:
                stream.wait_event(state["out"])
            step(k)
            ev_comp = torch.cuda.Event()
            ev_comp.record(stream)
            s_out.wait_event(ev_comp)
            with torch.cuda.stream(s_out):
                eps_h.copy_(eps, non_blocking=True)
                g_h.copy_(g, non_blocking=True)
            ev_out = torch.cuda.Event()
            ev_out.record(s_out)
            state["comp"], state["out"] = ev_comp, ev_out

        for k in range(2):
            e2e_step(k)
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        s_in.wait_event(e0)
        state["comp"] = state["out"] = None
        for k in range(ne):
            e2e_step(k)
        stream.wait_event(state["out"])
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms_e = reduce_max(e0.elapsed_time(e1) / ne, dist, "cuda")
        e2e = {"value": replica_value(world, cells, ms_e), "unit": "cells/s",
               "h2d_bytes_per_step": int(efp.numel() * 8 * 2),
               "d2h_bytes_per_step": int(eps_h.numel() * 4 + g_h.numel() * 4),
               "ms_per_step": ms_e}

    # the other configurations: the batched launch, the served mix, the 2D TE
    # design (launch-bound) and the taper through autograd, each with its own
    # clock record
    systems = {}
    if rank == 0 and world == 1 and not args.no_systems:
        systems["te2d"] = measure_te2d(ctx, device=local)
        systems["taper_autograd"] = measure_taper_autograd(ctx, device=local)
        systems["batch"] = measure_batch(ctx, 256, device=local)
        systems["serve"] = measure_serve(ctx, device=local)

    cpu = None
    methods = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample, timings = oracle_sample(desc, ef_h, ea_h, w)
        cpu = {"value": v, "unit": "cells/s", "cores": cores, "kind": "oracle", "sample": sample}
        methods = oracle_methods(desc, ef_h, ea_h, w, timings, value)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(grid_of(args)), "cells_per_design": cells,
                       "components": C,
                       "params": int(design.n_params), "parallelism": "replicas" if world > 1 else "single",
                       "outputs": "fill + eps (fp32) + gradient",
                       "vjp": "band tiles only (tiles crossed by an edge band)",
                       "tile": list(stats["tile"]), "tile_autotuned": tuned,
                       "build_fill_warps": fill_warps,
                       "program_tiles": stats["program_tiles"],
                       "tiles": stats["tiles"], "band_cells": stats["band_cells"],
                       "vjp_active_samples": stats["active_samples"],
                       "l2": "inputs larger than L2 (fields 691 MB + outputs 346 MB per step)"},
            "roofline": roof, "step_roofline": step_roof, "kernels": kernels,
            "gpu_launches": launches,
            "cpu_baseline": cpu, "oracle_methods": methods, "e2e": e2e, "dense_vjp": dense,
            "topology": topo,
            "fd_vs_ad": fdc, "levels": levels, "prop2_mesher": mesh,
            "batch": systems.get("batch"), "serve": systems.get("serve"),
            "te2d": systems.get("te2d"), "taper_autograd": systems.get("taper_autograd"),
            "clocks": clocks.summary(),
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _device_fields(desc, seed):
    """Seeded complex64 fields generated on the device (large batched / served
    workloads; the values do not steer the work, only the shapes do)."""
    import torch
    C = desc["grid"]["ncomp"]
    nx, ny, nz = desc["grid"]["n"]
    g = torch.Generator(device="cuda").manual_seed(int(seed))
    return (torch.randn((C, nz, ny, nx), dtype=torch.complex64, device="cuda", generator=g),
            torch.randn((C, nz, ny, nx), dtype=torch.complex64, device="cuda", generator=g))


def _timed_events(fn, steps, warm, sync):
    """Device time per call (CUDA events on the current stream) and host wall
    time per call, after `warm` untimed calls."""
    import torch
    for k in range(warm):
        fn(k)
    sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    for k in range(steps):
        fn(k)
    e1.record()
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / steps
    sync()
    return e0.elapsed_time(e1) / steps, wall * 1e3


BATCH_TUNE_CANDIDATES = [(32, 4, 4), (32, 8, 4), (32, 4, 2), (32, 8, 2)]


def measure_batch(ctx, designs_n=256, steps=5, warmup=3, tune=True, device=0):
    """Batched persistent launch: designs_n random designs of uneven grid size
    and primitive count; eps build + gradient for all of them per step, as
    one graph-captured job table versus one launch sequence per design.  Both
    tile policies are timed -- the library's default tile, and the
    autotuner's tile per size class -- and the faster is the headline."""
    import numpy as np
    import torch

    from paper_2311_05646_gb300 import adg
    from paper_2311_05646_gb300 import inputs as I
    from paper_2311_05646_gb300.tuning import Autotuner

    descs = [I.random_design(4100 + k) for k in range(designs_n)]
    cells = sum(int(np.prod(desc["grid"]["n"])) for desc in descs)
    params = [[desc["params"], desc["params"] + 0.01] for desc in descs]
    w = np.full(3, -2j, dtype=np.complex64)
    bufs = []
    for k, desc in enumerate(descs):
        ef, ea = _device_fields(desc, 9000 + k)
        sh = I.field_shape(desc)
        eps = torch.empty(sh, dtype=torch.float32, device="cuda")
        fill = torch.empty_like(eps)
        g = torch.zeros(len(desc["params"]), dtype=torch.float32, device="cuda")
        bufs.append((ef, ea, eps, fill, g))
    sync = lambda: (torch.cuda.synchronize(), adg.adg_sync(ctx))  # noqa: E731

    def run_policy(tiles):
        designs = [adg.Design(ctx, desc, tile=t) for desc, t in zip(descs, tiles)]

        def batched(k):
            items = []
            for i, d in enumerate(designs):
                ef, ea, eps, fill, g = bufs[i]
                items.append(adg.BatchItem(d, params[i][k % 2], eps=eps, fill=fill, efwd=ef,
                                           eadj=ea, w=w, grad=g))
            return adg.adg_batch_submit(ctx, items, graph=True)

        def per_design(k):
            for i, d in enumerate(designs):
                ef, ea, eps, fill, g = bufs[i]
                p = params[i][k % 2]
                adg.adg_build_eps(d, p, eps, fill=fill)
                adg.adg_grad(d, p, ef, ea, w, g)

        clocks = Clocks(device)
        clocks.start()
        ms_b, wall_b = _timed_events(batched, steps, warmup, sync)
        ms_d, wall_d = _timed_events(per_design, steps, warmup, sync)
        clocks.stop()
        # per-kernel device time of one batched step (direct launches, events around each)
        adg.adg_profile_read(ctx, reset=True)
        adg.adg_profile_enable(ctx, True)
        items = []
        for i, d in enumerate(designs):
            ef, ea, eps, fill, g = bufs[i]
            items.append(adg.BatchItem(d, params[i][0], eps=eps, fill=fill, efwd=ef, eadj=ea, w=w,
                                       grad=g))
        adg.adg_batch_wait(ctx, adg.adg_batch_submit(ctx, items, graph=False))
        torch.cuda.synchronize()
        adg.adg_profile_enable(ctx, False)
        prof = {k: round(1e3 * v[1] / max(v[0], 1), 1)
                for k, v in adg.adg_profile_read(ctx, reset=True).items() if v[0]}
        for d in designs:
            d.close()
        n = len(designs)
        return {"gradients_per_s": n / (ms_b * 1e-3), "ms_per_step": ms_b,
                "host_wall_ms_per_step": wall_b, "cells_per_s": cells / (ms_b * 1e-3),
                "one_launch_per_design": {"gradients_per_s": n / (ms_d * 1e-3),
                                          "ms_per_step": ms_d, "host_wall_ms_per_step": wall_d},
                "speedup_vs_per_design": ms_d / ms_b, "batched_kernels_us": prof,
                "clocks": clocks.summary()}

    out = {"designs": len(descs), "cells_total": cells,
           "workload": "%d random designs, grids U[128,512]x[64,256]x[32,96], 10-400 primitives "
                       "(boxes, circles r 80-200 nm, 16-64-gons), unions/differences, complex64 "
                       "fields" % len(descs),
           "steps": steps, "warmup": warmup}
    out["default_tile"] = run_policy([None] * len(descs))
    if tune:
        tuner = Autotuner(ctx, candidates=BATCH_TUNE_CANDIDATES)
        t0 = time.perf_counter()
        tiles = [tuner.best(desc) for desc in descs]
        out["autotuned_tile"] = run_policy(tiles)
        out["autotuned_tile"]["tuning_s"] = time.perf_counter() - t0
        out["autotuned_tile"]["size_classes"] = len(tuner.cache)
    best = max((k for k in ("default_tile", "autotuned_tile") if k in out),
               key=lambda k: out[k]["gradients_per_s"])
    out["headline_tiles"] = best
    out["gradients_per_s"] = out[best]["gradients_per_s"]
    out["speedup_vs_per_design"] = out[best]["speedup_vs_per_design"]
    del bufs
    torch.cuda.empty_cache()
    return out


def run_batch(args):
    import torch

    from paper_2311_05646_gb300 import adg
    torch.cuda.set_device(0)
    ctx = adg.Context(0)
    b = measure_batch(ctx, args.designs, args.steps, max(args.warmup, 3), tune=args.tune)
    best = b[b["headline_tiles"]]
    line = {"metric": "gradients/s (eps build + VJP gradient per design)",
            "value": b["gradients_per_s"], "unit": "gradients/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": b["workload"], "cells_total": b["cells_total"],
                                            "tiles": b["headline_tiles"]},
            "batch": b, "clocks": best["clocks"]}
    print(json.dumps(line))
    return 0


def _serve_clients(I, np, rng, n, iterations):
    """The served mix: the largest client a 20 x 20 hole lattice in 1000 x
    1000 x 80 (1200 parameters), the others 2D 400 x 400 or 3D hole lattices
    of log-uniform size; fields made on the device at admission."""
    from paper_2311_05646_gb300 import serve as S
    cl = []
    for k in range(n):
        if k == 0:
            desc = I.hole_lattice(n=(1000, 1000, 80), holes=20, seed=51)
        elif rng.uniform() < 0.5:
            desc = I.hole_lattice(n=(400, 400, 1), d=(40.0, 40.0, 40.0), holes=8, ncomp=1,
                                  seed=51 + k)
        else:
            sx = int(np.exp(rng.uniform(np.log(128), np.log(1000))))
            sy = int(np.exp(rng.uniform(np.log(128), np.log(1000))))
            sz = int(np.exp(rng.uniform(np.log(32), np.log(80))))
            desc = I.hole_lattice(n=(sx, sy, sz), holes=int(np.clip(sx // 50, 2, 20)), seed=51 + k)
        cl.append(S.Client(cid=k, desc=desc, w=np.full(desc["grid"]["ncomp"], -2j),
                           iterations=iterations,
                           make_fields=(lambda desc=desc, k=k: _device_fields(desc, 7000 + k))))
    return cl


def measure_serve(ctx, clients_n=12, iterations=50, mem_gb=40.0, rates=(0.5, 0.8, 0.95),
                  tune=True, device=0):
    """Served requests: clients (designs) arrive as a Poisson process and run
    `iterations` optimiser iterations each (an eps build, then a gradient,
    then the parameter step); fields stay resident; admission is gated by
    the bytes libadg reports plus the clients' buffers against a memory
    budget and the device's free memory; batches form continuously.  First
    saturated (all clients at once), then Poisson arrivals at each rate x the
    saturated request rate: p50 / p99 request latency and gradients/s."""
    import numpy as np
    import torch

    from paper_2311_05646_gb300 import inputs as I
    from paper_2311_05646_gb300 import serve as S

    rng = np.random.default_rng(51)
    tuner = None
    if tune:
        from paper_2311_05646_gb300.tuning import Autotuner
        tuner = Autotuner(ctx)
    budget = int(mem_gb * 2 ** 30)

    def run(clients, arrivals):
        srv = S.Server(ctx, mem_budget_bytes=budget, max_inflight=2, tuner=tuner)
        clocks = Clocks(device)
        clocks.start()
        t0 = time.perf_counter()
        order = sorted(zip(arrivals, range(len(clients))))
        nxt = 0
        peak = 0
        while nxt < len(order) or not srv.idle():
            now = time.perf_counter() - t0
            while nxt < len(order) and order[nxt][0] <= now:
                srv.arrive(clients[order[nxt][1]], time.perf_counter())
                nxt += 1
            peak = max(peak, srv.used)
            if not srv.poll():
                time.sleep(20e-6)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clocks.stop()
        grads = sum(1 for r in srv.completed if r.op == "grad")
        lat = S.latency_stats(srv.completed)
        return {"gradients_per_s": grads / wall, "requests": len(srv.completed),
                "p50_ms": lat["p50_ms"], "p99_ms": lat["p99_ms"], "mean_ms": lat.get("mean_ms"),
                "batches": srv.batches, "wall_s": wall, "peak_admitted_bytes": peak,
                "clocks": clocks.summary()}

    t0 = time.perf_counter()
    clients = _serve_clients(I, np, rng, clients_n, iterations)
    if tuner is not None:
        for c in clients:
            tuner.best(c.desc)
        torch.cuda.synchronize()
    tuning_s = time.perf_counter() - t0
    sat = run(clients, [0.0] * len(clients))
    out = {"workload": "%d clients x %d iterations (eps build + gradient), hole lattices: 2D "
                       "400x400 or 3D up to 1000x1000x80 (20x20 holes, 1200 params)"
                       % (clients_n, iterations),
           "mem_budget_gb": mem_gb, "tiles_autotuned": tuner is not None, "tuning_s": tuning_s,
           "saturated": sat, "poisson": {}}
    for lam in rates:
        clients = _serve_clients(I, np, np.random.default_rng(51), clients_n, iterations)
        rate_clients = lam * sat["gradients_per_s"] / iterations
        arr = np.cumsum(rng.exponential(1.0 / rate_clients, len(clients)))
        arr -= arr[0]
        out["poisson"]["%.2f" % lam] = run(clients, list(arr))
    torch.cuda.empty_cache()
    return out


def run_serve(args):
    import torch

    from paper_2311_05646_gb300 import adg
    torch.cuda.set_device(0)
    ctx = adg.Context(0)
    sv = measure_serve(ctx, args.clients, args.iterations, args.mem_gb, tune=not args.no_tune)
    mid = sv["poisson"]["0.80"]
    line = {"metric": "served gradients/s with p50/p99 request latency",
            "value": mid["gradients_per_s"], "unit": "gradients/s", "n_gpus": 1,
            "steps": mid["requests"], "warmup": 0,
            "ms_per_step": 1e3 * mid["wall_s"] / max(mid["requests"], 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": sv["workload"],
                                            "arrivals": "Poisson at 0.8 x saturated"},
            "latency_ms": {"p50": mid["p50_ms"], "p99": mid["p99_ms"]},
            "serve": sv, "clocks": mid["clocks"]}
    print(json.dumps(line))
    return 0


def measure_te2d(ctx, steps=2000, warmup=50, device=0):
    """The 2D TE single design (200 x 100 cells, 20 nm, a waveguide box minus a
    20-tooth grating, 40 edge parameters, Ez fields of seeded plane waves):
    launch-bound, so reported as the device time and host wall time per eps
    build + gradient, with the parameters alternating (every step re-bins)."""
    import torch

    from paper_2311_05646_gb300 import adg
    from paper_2311_05646_gb300 import inputs as I
    desc = I.grating_2d("fit")
    d = adg.Design(ctx, desc)
    ef = torch.from_numpy(I.plane_wave_field(desc, 12)).cuda()
    ea = torch.from_numpy(I.plane_wave_field(desc, 13)).cuda()
    w = I.seeded_w(1, 5)
    eps = torch.empty(d.shape, dtype=torch.float32, device="cuda")
    fill = torch.empty_like(eps)
    g = torch.zeros(d.n_params, dtype=torch.float32, device="cuda")
    ps = [desc["params"], desc["params"] + 0.01]

    def step(k):
        adg.adg_build_eps(d, ps[k % 2], eps, fill=fill)
        adg.adg_grad(d, ps[k % 2], ef, ea, w, g)

    clocks = Clocks(device)
    clocks.start()
    ms, wall = _timed_events(step, steps, warmup, lambda: (torch.cuda.synchronize(), adg.adg_sync(ctx)))
    clocks.stop()
    cells = 200 * 100
    d.close()
    return {"workload": "2D TE grating 200x100 (Ez), 40 edge params", "cells": cells,
            "device_us_per_step": 1e3 * ms, "host_us_per_step": 1e3 * wall,
            "cells_per_s": cells / (ms * 1e-3), "steps": steps, "clocks": clocks.summary()}


def measure_taper_autograd(ctx, steps=20, warmup=3, device=0):
    """The differentiable taper through torch.autograd: eps = eps_of(design, p)
    on the 800 x 300 x 100 grid (two 64-vertex graph boundaries, 128
    parameters, sigmoid k = 4 / dx), then eps.backward(G) with a fixed real
    cotangent: the forward keeps only p, the backward recomputes fill."""
    import numpy as np
    import torch

    from paper_2311_05646_gb300 import adg
    from paper_2311_05646_gb300 import inputs as I
    from paper_2311_05646_gb300.autograd import eps_of
    desc = I.taper_3d()
    d = adg.Design(ctx, desc)
    gen = torch.Generator(device="cuda").manual_seed(12)
    G = torch.randn(d.shape, dtype=torch.float32, device="cuda", generator=gen)
    p = torch.tensor(desc["params"], dtype=torch.float64, requires_grad=True)

    def step(k):
        with torch.no_grad():
            p.add_(0.01 if k % 2 else -0.01)  # new parameters every step (re-binning)
        p.grad = None
        eps = eps_of(d, p)
        eps.backward(G)

    clocks = Clocks(device)
    clocks.start()
    ms, wall = _timed_events(step, steps, warmup, lambda: (torch.cuda.synchronize(), adg.adg_sync(ctx)))
    clocks.stop()
    cells = int(np.prod(desc["grid"]["n"]))
    d.close()
    return {"workload": "taper 800x300x100, 3 components, 128 vertex-offset params, autograd "
                        "forward + backward", "cells": cells, "ms_per_step": ms,
            "host_ms_per_step": wall, "cells_per_s": cells / (ms * 1e-3), "steps": steps,
            "clocks": clocks.summary()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="adg", choices=["adg", "reference"])
    ap.add_argument("--tile", default="")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--workload", default="grating3d", choices=["grating3d", "batch", "serve"])
    ap.add_argument("--grid", default="")  # grating3d: NXxNYxNZ (default 600x200x120)
    ap.add_argument("--designs", type=int, default=256)
    ap.add_argument("--tune", action="store_true")  # batch: autotune tiles per size class
    ap.add_argument("--no-tune", action="store_true")  # grating: the library's default tile
    ap.add_argument("--clients", type=int, default=12)
    ap.add_argument("--iterations", type=int, default=50)
    ap.add_argument("--mem-gb", type=float, default=40.0)
    ap.add_argument("--no-systems", action="store_true")  # skip batch / serve / TE / taper entries
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_adg(args)


if __name__ == "__main__":
    sys.exit(main())
