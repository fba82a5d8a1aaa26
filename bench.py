#!/usr/bin/env python
"""Benchmark: trust-region steps/s of the 3DGS^2-TR iteration on one GB300.

Workload (the batched multi-view configuration): 1,000,000 Gaussians (FP32, SH
degree 3) drawn from 20 isotropic clusters (sigma 0.3) in a radius-10 scene, 8
views of 1920x1080 per step from a 64-camera jittered ring, 16x16 tiles, L1 loss,
nu = 2 Rademacher probes and the Hutchinson diagonal on every step.  One step =
projection + binning/sort + forward (with tangents) + reverse pass (gradient and
z.Hz) + trust-region update over all 8 views.  Targets are rendered once, before
timing, from a second seeded Gaussian set by the forward pass.

Printed JSON line: value = whole-job steps/s with inputs resident in HBM; e2e =
the same through the C ABI with the step's targets and cameras copied from
pinned host memory and the loss read back inside the timed region; roofline of
the dominant kernel; the FP64 oracle as a CPU baseline on a bounded sample.

``--impl reference`` times the FP64 CPU oracle (the only reference this
project has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GAUSS = 1_000_000
SH_DEG = 3
N_VIEWS = 8
W, H = 1920, 1080
NU = 2
RING = 64
TILE = (16, 16)
METRIC = "TR steps/s (fwd+bwd+HVP+update) @1M Gaussians 1080p"
UNIT = "steps/s"
WORKLOAD = "batched multi-view: 1M Gaussians SH3, 20 clusters sigma 0.3 in radius-10 ball, 8 views 1920x1080 per step, nu=2"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--n", type=int, default=N_GAUSS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-full-step", action="store_true",
                    help="time one full oracle step of the workload (nothing scaled) and exit")
    ap.add_argument("--configs", action="store_true",
                    help="GPU plain-loop steps/s of the smaller configurations and their oracle steps, then exit")
    ap.add_argument("--no-serve", action="store_true", help="skip the served multi-scene measurement")
    ap.add_argument("--profile-steps", type=int, default=0, help="run N untimed steps only (for ncu)")
    ap.add_argument("--profile-views", type=int, default=N_VIEWS,
                    help="views per step in a --profile-steps run (a smaller case for ncu captures)")
    ap.add_argument("--profile-tile", default="16x16",
                    help="tile shape WxH of a --profile-steps run (the shape the autotuner picked)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"gs3dtr_clocks_{os.getpid()}_gpu{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9 and p[1].replace(".", "").isdigit():
                    rows.append(p)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------------ workload
def make_workload(n, device, rank=0, views=N_VIEWS, n_batches=None, tile=TILE):
    import numpy as np
    import torch
    from paper_2602_00395_gb300 import synth as S
    from paper_2602_00395_gb300.engine import TRConfig, TRStep
    from paper_2602_00395_gb300 import gs3dtr as G

    scene = S.make_scene(n, SH_DEG, seed=1000 + rank, kind="clusters", extent=10.0)
    gt = S.make_scene(n, SH_DEG, seed=2000 + rank, kind="clusters", extent=10.0)
    cams = S.camera_ring(RING, W, H, 10.0, seed=7)
    batches = [[cams[b + RING // views * k] for k in range(views)] for b in range(RING // views)]
    batches = batches[:n_batches] if n_batches else batches
    eng = TRStep(n, SH_DEG, views, W, H, nu=NU, tile=tile, cfg=TRConfig(l=1), device=device)
    # targets: the ground-truth set rendered by the forward pass, one batch of views at a time
    eng.set_params(gt.params)
    cam_dev, targets = [], []
    need = 0
    for bcams in batches:
        eng.set_cameras(bcams)
        need = max(need, eng.ensure_capacity())
        eng.render()
        targets.append(eng.image.clone())
        cam_dev.append(eng.cams.clone())
    eng.set_params(scene.params)
    for cd in cam_dev:
        eng.cams.copy_(cd)
        need = max(need, eng.ensure_capacity())
    if need * 1.15 > eng.capacity:
        eng._alloc_pairs(int(need * 1.3))
    torch.cuda.synchronize()
    return eng, cam_dev, targets, batches, need


def kernel_launches_per_step(eng) -> int:
    """Kernels of this library launched per step (the sort's memsets are not
    kernels and are not counted)."""
    def bits(v):
        b = 0
        while (1 << b) < v:
            b += 1
        return b
    rec_pass = 4  # 32 depth bits, per view
    pair_pass = max(1, (bits(N_VIEWS * eng.Tx * eng.Ty) + 7) // 8)
    radix = 1 + 3 + 1  # histogram, three-kernel scan, scatter
    # record keys, record passes, count gather, three-kernel scan, emit, pair passes, ranges,
    # heaviest-first tile order (class counts, class starts, placement)
    sort = 1 + rec_pass * radix + 1 + 3 + 1 + pair_pass * radix + 1 + 3
    # step counter, project, sort, fwd, reverse call (workspace check, reverse blend,
    # projection reverse), update
    return 1 + 1 + sort + 1 + 3 + 1


def retile_workload(eng, cam_dev, targets, batches, tile, device, batch=0):
    """The same workload (parameters, cameras, targets) on a step with another
    tile shape and blend batch."""
    from paper_2602_00395_gb300.engine import TRStep
    e = TRStep(eng.n, SH_DEG, eng.V, W, H, nu=NU, tile=tile, cfg=eng.cfg, device=device, batch=batch)
    e.x.copy_(eng.x)
    need = 0
    for cd in cam_dev:
        e.cams.copy_(cd)
        need = max(need, e.ensure_capacity())
    if need * 1.15 > e.capacity:
        e._alloc_pairs(int(need * 1.3))
    return e, cam_dev, targets, batches, need


def timed_steps(eng, cam_dev, targets, K, W0, t0, stream, per_call=False):
    """K steps on `stream`; returns (ms total from events, per-call ms dict).
    With per_call, each call is bracketed by its own events, and the work units
    of those very launches are summed on the device between the calls: the dict
    then also holds "sum_n_contrib" and "pairs", their means per step."""
    import torch
    from paper_2602_00395_gb300.engine import eps_schedule
    calls = ["project", "bin_sort", "raster_fwd", "raster_bwd", "update"]
    ev = {c: [] for c in calls}
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    nb = len(targets)
    units = torch.zeros(2, dtype=torch.float64, device=eng.device)  # sum n_contrib, pairs
    with torch.cuda.stream(stream):
        start.record(stream)
        for k in range(K):
            t = t0 + k
            b = (t - 1) % nb
            eng.cams = cam_dev[b]
            eng.target = targets[b]
            eps = eps_schedule(t, 30000)
            eng.loss_val.zero_()
            seq = [("project", lambda: eng.project(t, True, stream)),
                   ("bin_sort", lambda: eng.bin_sort(stream)),
                   ("raster_fwd", lambda: eng.raster_fwd(t, True, stream)),
                   ("raster_bwd", lambda: eng.raster_bwd(t, True, stream)),
                   ("update", lambda: eng.update(t, eps, True, None, stream))]
            for name, fn in seq:
                if per_call:
                    a = torch.cuda.Event(enable_timing=True)
                    z = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    fn()
                    z.record(stream)
                    ev[name].append((a, z))
                    if name == "raster_fwd":  # outside the calls' event brackets
                        units[0] += eng.n_contrib.sum(dtype=torch.float64)
                        units[1] += eng.n_pairs.to(torch.float64).sum()
                else:
                    fn()
        stop.record(stream)
    stop.synchronize()
    total = start.elapsed_time(stop)
    per = {c: (sum(a.elapsed_time(z) for a, z in ev[c]) / len(ev[c]) if ev[c] else None) for c in calls}
    if per_call:
        per["sum_n_contrib"], per["pairs"] = (float(u) / K for u in units.cpu())
    return total, per


def plain_loop_steps(eng, cam_dev, targets, K, t0, stream, device):
    """The same steps issued one view at a time (the plain loop): for each of the
    8 views project / bin-sort / forward / reverse pass on a single-view frame,
    then the per-view gradients and Hutchinson diagonals, each normalised by its
    own residual count, are averaged, and one update is applied.  Returns ms per
    step (device time, CUDA events)."""
    import torch
    from paper_2602_00395_gb300.engine import TRConfig, TRStep, eps_schedule
    one = TRStep(eng.n, SH_DEG, 1, W, H, nu=NU, tile=eng.tile, cfg=TRConfig(l=1), capacity=eng.capacity,
                 device=device)
    one.x.copy_(eng.x)
    g_acc = torch.zeros_like(one.grad)
    h_acc = torch.zeros_like(one.hz)
    HW3 = 3 * W * H
    nb = len(targets)

    def run(k0, k1):
        for k in range(k0, k1):
            t = t0 + k
            b = (t - 1) % nb
            g_acc.zero_()
            h_acc.zero_()
            for v in range(N_VIEWS):
                one.cams = cam_dev[b][96 * v:96 * (v + 1)]
                one.target = targets[b][HW3 * v:HW3 * (v + 1)]
                one.project(t, True, stream)
                one.bin_sort(stream)
                one.raster_fwd(t, True, stream)
                one.raster_bwd(t, True, stream)
                g_acc.add_(one.grad, alpha=1.0 / N_VIEWS)
                h_acc.add_(one.hz, alpha=1.0 / N_VIEWS)
            one.grad.copy_(g_acc)
            one.hz.copy_(h_acc)
            one.update(t, eps_schedule(t, 30000), True, None, stream)

    with torch.cuda.stream(stream):
        run(0, 3)
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        run(3, 3 + K)
        stop.record(stream)
    stop.synchronize()
    ms = start.elapsed_time(stop) / K
    del one
    torch.cuda.empty_cache()
    return ms


def graph_steps(eng, graphs, K, t0, stream):
    """K steps replayed from the captured graphs (one per view batch); the step
    index runs on the device from t0.  Returns ms from events on `stream`."""
    import torch
    nb = len(graphs)
    eng.t_dev.fill_(t0 - 1)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        start.record(stream)
        for k in range(K):
            graphs[(t0 + k - 1) % nb].replay()
        stop.record(stream)
    stop.synchronize()
    return start.elapsed_time(stop)


def e2e_steps(eng, batches, host_targets, K, t0, stream, schedule):
    """K steps through the C ABI with each step's targets and cameras copied from
    pinned host memory and the loss copied back, all inside the timed region.
    The copy of step k+1's inputs runs on a second stream into the other half of
    a double buffer while step k, a graph replay bound to that half, computes."""
    import torch
    from paper_2602_00395_gb300 import gs3dtr as G
    host_cams = [torch.from_numpy(G.camera_bytes(bc)).pin_memory() for bc in batches]
    loss_host = torch.zeros(K, dtype=torch.float32).pin_memory()
    nb = len(batches)
    copy_stream = torch.cuda.Stream(device=stream.device)
    dev_tg = [torch.empty_like(eng.target) for _ in range(2)]
    dev_cams = [torch.empty_like(eng.cams) for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    graphs = []
    for slot in range(2):
        eng.target = dev_tg[slot]
        eng.cams = dev_cams[slot]
        graphs.append(eng.capture_step(True, schedule, stream))
    eng.t_dev.fill_(t0 - 1)

    def prefetch(k):
        b = (t0 + k - 1) % nb
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(consumed[k % 2])
            dev_tg[k % 2].copy_(host_targets[b], non_blocking=True)
            dev_cams[k % 2].copy_(host_cams[b], non_blocking=True)
            copied[k % 2].record(copy_stream)

    torch.cuda.synchronize()
    w0 = time.perf_counter()
    start.record(stream)
    copy_stream.wait_event(start)
    prefetch(0)
    if K > 1:
        prefetch(1)
    with torch.cuda.stream(stream):
        for k in range(K):
            stream.wait_event(copied[k % 2])
            graphs[k % 2].replay()
            loss_host[k:k + 1].copy_(eng.loss_val, non_blocking=True)
            consumed[k % 2].record(stream)
            if k + 2 < K:
                prefetch(k + 2)
        stop.record(stream)
    stop.synchronize()
    wall = time.perf_counter() - w0
    h2d = host_targets[0].numel() * 4 + host_cams[0].numel()
    return start.elapsed_time(stop), wall, h2d, 4


# ------------------------------------------------------------------ curvature cost
def curvature_costs(eng, cam_dev, targets, K, stream):
    """ms per step of (a) the gradient-only step (no probes, no curvature),
    (b) Algorithm 1 with l = 10 and the curvature batch S2 = the next view batch
    (Sec. 4.1; the paper's default interval), averaged over K steps, and the
    resulting overheads of curvature relative to (a)."""
    import torch
    from paper_2602_00395_gb300.engine import eps_schedule
    nb = len(targets)
    cfg_l = eng.cfg.l

    def run(kind, t0):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for phase in (0, 1):
                if phase == 1:
                    ev0.record(stream)
                for k in range(K if phase else 2):
                    t = t0 + k
                    b = (t - 1) % nb
                    eng.cams, eng.target = cam_dev[b], targets[b]
                    eps = eps_schedule(t, 30000)
                    if kind == "grad":
                        eng.loss_val.zero_()
                        eng.project(t, False, stream)
                        eng.bin_sort(stream)
                        eng.raster_fwd(t, False, stream)
                        eng.raster_bwd(t, False, stream)
                        eng.update(t, eps, False, None, stream)
                    else:
                        b2 = (b + 1) % nb
                        eng.step_s2(t, eps, cam_dev[b2], targets[b2], stream)
            ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / K

    grad_ms = run("grad", 3000)
    eng.cfg.l = 10
    try:
        l10_ms = run("s2", 4001)  # t = 4001 is a curvature step: K = 20 covers two of them
    finally:
        eng.cfg.l = cfg_l
    return {"gradient_only_ms": grad_ms, "l10_separate_s2_ms": l10_ms,
            "overhead_l10": l10_ms / grad_ms - 1.0}


# ------------------------------------------------------------------ variants
def variant_costs(eng, cam_dev, targets, K, stream):
    """ms per step, same workload, of (a) ADAM-TR (Sec. 5 ablation: gradient
    only, Adam step clipped by the trust region) and (b) Algorithm 1 with the
    pixel loss (1 - 0.2) L1 + 0.2 D-SSIM (Eq. pixel_loss), with the time of the
    D-SSIM cotangent call alone."""
    import torch
    from paper_2602_00395_gb300 import gs3dtr as G
    from paper_2602_00395_gb300.engine import eps_schedule
    nb = len(targets)
    adam = G.adam_struct()

    def timed(fn, t0):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for k in range(2):
                fn(t0 + k)
            ev0.record(stream)
            for k in range(K):
                fn(t0 + k)
            ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / K

    def batch(t):
        b = (t - 1) % nb
        eng.cams, eng.target = cam_dev[b], targets[b]

    def adam_step(t):
        batch(t)
        eng.step_adam(t, eps_schedule(t, 30000), adam, stream)

    def dssim_step(t):
        batch(t)
        eng.step(t, eps_schedule(t, 30000), stream)

    out = {"adam_tr_ms": timed(adam_step, 6000)}
    HW = W * H
    eng.dssim_lambda = 0.2
    eng.cot_img = torch.empty((1 + NU) * N_VIEWS * 3 * HW, dtype=torch.float32, device=eng.device)
    eng.dssim_ws = torch.empty(G.gs_dssim_workspace_size(eng.frame, NU), dtype=torch.uint8, device=eng.device)
    try:
        out["dssim_l1_mix_ms"] = timed(dssim_step, 7000)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(K):
                G.gs_dssim_cotangents(eng.frame, eng.image, eng.target, eng.image_tan, NU, 0.2, eng.loss.gn_floor,
                                      True, eng.cot_img, eng.loss_val, eng.dssim_ws, eng.status, stream)
            ev1.record(stream)
        ev1.synchronize()
        out["dssim_cotangents_ms"] = ms = ev0.elapsed_time(ev1) / K
        # algorithmic bytes per pixel and channel: statistics 8 read + 16 written;
        # the probes' derivative pass 32 + 8; the gradient's adjoint 20 + 4; the
        # probes' adjoint 36 + 8 (nu = 2)
        nbytes = 132 * N_VIEWS * 3 * HW
        hbm, _, src = peaks()
        out["dssim_cotangents_roofline"] = {"bound": "hbm", "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": hbm,
                                            "unit": "GB/s", "frac": nbytes / (ms * 1e-3) / 1e9 / hbm,
                                            "bytes": nbytes}
    finally:
        eng.dssim_lambda = None
        del eng.cot_img, eng.dssim_ws
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ memory
def memory_footprint(eng, cam_dev, targets, device, stream):
    """Device memory of one trust-region step against one ADAM-TR step (the
    paper's comparison of peak GPU memory, Sec. 5, Table 1) on the bench's scene
    (1M Gaussians, SH 3, 1920x1080): each step is built fresh on the same
    parameters, cameras and targets, and its peak is torch's max allocated bytes
    during construction and one step, above what was allocated before.  Two
    settings: the bench's step (8 views, nu = 2, fused) and the paper's (one view
    per step, nu = 1).  The ADAM-TR step holds x, m, v and the gradient; the
    trust-region step adds the curvature estimate hz, the probe tangents of the
    splat records and images, and the extra cotangent streams of the reverse pass."""
    import torch
    from paper_2602_00395_gb300.engine import TRStep
    rows = 11 + 3 * (SH_DEG + 1) ** 2
    mat = rows * eng.n_pad * 4
    HW3 = 3 * W * H
    out = {}
    for setting, views, nu in (("bench_8_views_nu2", N_VIEWS, NU), ("one_view_nu1", 1, 1)):
        res = {}
        for kind in ("tr", "adam_tr"):
            torch.cuda.synchronize(device)
            torch.cuda.empty_cache()
            base = torch.cuda.memory_allocated(device)
            torch.cuda.reset_peak_memory_stats(device)
            e = TRStep(eng.n, SH_DEG, views, W, H, nu=nu if kind == "tr" else 0, tile=eng.tile, cfg=eng.cfg,
                       device=device, capacity=eng.capacity, batch=eng.frame.batch)
            e.x.copy_(eng.x)
            e.cams.copy_(cam_dev[0][:96 * views])
            e.target.copy_(targets[0][:HW3 * views])
            with torch.cuda.stream(stream):
                if kind == "tr":
                    e.step(1, 1e-6, stream)
                else:
                    e.step_adam(1, 1e-6, None, stream)
            torch.cuda.synchronize(device)
            assert e.read_status() == 0, e.read_status()
            res[kind] = (torch.cuda.max_memory_allocated(device) - base) / 1e9
            del e
        torch.cuda.empty_cache()
        out[setting] = {"tr_step_peak_GB": res["tr"], "adam_tr_step_peak_GB": res["adam_tr"],
                        "overhead_GB": res["tr"] - res["adam_tr"],
                        "overhead_frac": res["tr"] / res["adam_tr"] - 1.0,
                        "optimizer_state_GB": {"tr (x, g_ema, d_ema, g, hz)": 5 * mat / 1e9,
                                               "adam_tr (x, m, v, g)": 4 * mat / 1e9}}
    out["paper"] = ("A100, whole training process, 3DGS^2-TR vs ADAM peak memory: +0.91 / +0.84 / +0.95 GB "
                    "(MipNeRF-360 / Deep Blending / T&T), 17 % on average (Sec. 5, Table 1); context only")
    return out


# ------------------------------------------------------------------ serving
def served_metrics(device, n_requests=200, slots=16, budget_gb=40.0):
    """The served multi-scene workload: 16 resident scenes (50k-2M Gaussians, SH 3,
    image sizes from 256x256 to 1920x1080, 8 views each), a seeded Poisson stream
    of 70 % training steps and 30 % renders.  The plain loop's capacity is measured
    on back-to-back requests; the stream is then replayed at 0.5, 0.8, 1.0 and
    1.2 x that rate through the plain loop and through the server (continuous
    batching on `slots` streams, in-flight working sets within `budget_gb`)."""
    import torch
    from paper_2602_00395_gb300 import serve as SV
    from paper_2602_00395_gb300 import synth as S
    scenes = SV.make_scenes(16, device=device)
    nv = 8
    budget = int(budget_gb * 1e9)
    # warm-up: every scene once per request kind (allocator, kernel attributes)
    SV.plain_loop(scenes, [(0.0, k, s, 0) for s in range(len(scenes)) for k in ("train", "render")])
    # saturation: every request waiting at time 0
    burst = [(0.0, k, s, v) for (_, k, s, v) in S.request_stream(n_requests, 1.0, len(scenes), nv, seed=98)]
    sat_plain = SV.plain_loop(scenes, burst).summary()
    # one server throughout, its slots' buffer pools warmed by one untimed pass
    # of the burst (a running server is warm; the plain loop's warm-up above
    # plays the same role for its per-request buffers)
    server = SV.Server(scenes, slots=slots, budget_bytes=budget)
    server.run(burst)
    sat_served = server.run(burst).summary()
    capacity = sat_plain["requests_per_s"]
    sweep = []
    for f in (0.5, 0.8, 1.0, 1.2):
        spec = S.request_stream(n_requests, f * capacity, len(scenes), nv, seed=99)
        p = SV.plain_loop(scenes, spec).summary()
        q = server.run(spec).summary()
        keep = ("p50_ms", "p99_ms", "train_steps_per_s", "requests_per_s", "status_words")
        sweep.append({"rate_x_plain_capacity": f, "rate_per_s": round(f * capacity, 2),
                      "plain": {k: p[k] for k in keep}, "served": {k: q[k] for k in keep},
                      "served_peak_inflight_GB": q["peak_inflight_GB"]})
    info = {"scenes": [{"n": sc.n, "image": f"{sc.W}x{sc.H}"} for sc in scenes], "slots": slots,
            "budget_GB": budget_gb, "requests_per_run": n_requests,
            "plain_capacity_requests_per_s": capacity,
            "saturated": {"plain_train_steps_per_s": sat_plain["train_steps_per_s"],
                          "served_train_steps_per_s": sat_served["train_steps_per_s"],
                          "served_speedup": sat_served["train_steps_per_s"] / sat_plain["train_steps_per_s"],
                          "plain_p50_ms": sat_plain["p50_ms"], "plain_p99_ms": sat_plain["p99_ms"],
                          "served_p50_ms": sat_served["p50_ms"], "served_p99_ms": sat_served["p99_ms"]},
            "sweep": sweep}
    del scenes
    torch.cuda.empty_cache()
    return info


# ------------------------------------------------------------------ roofline
# Algorithmic FP32 work per contributing (pixel, splat) unit, the unit being
# sum over pixels of n_contrib (list position of the last blended splat): the
# forward blend ~20 FLOP per unit plus ~25 per probe for the fused tangents; the
# reverse blend ~50 FLOP per unit per cotangent stream (1 + nu streams).
def raster_fwd_flops_per_unit() -> int:
    return 20 + 25 * NU


def raster_bwd_flops_per_unit() -> int:
    return 50 * (1 + NU)


# DRAM bytes of one gs_raster_bwd call (its two kernels, read plus write; the
# workspace clear is a memset, not counted) from one-kernel ncu captures of the
# 2-view case (summaries under profiles/), with that case's pair count: a full
# launch's traffic is scaled from it by the pairs (the gathered records and the
# cotangent rows grow with the pairs and views).  Valid while the kernel sources
# are the ones captured (their SHA-256 below); otherwise null.
RASTER_BWD_TRAFFIC = {
    # one-kernel captures (dram__bytes_read.sum + dram__bytes_write.sum) of the
    # reverse call's two kernels on the 2-view case of the bench scene
    "blend_bytes": 376_053_760 + 42_944_512,        # raster_bwd_kernel
    "projection_bytes": 460_134_656 + 448_670_720,  # project_bwd_kernel
    "pairs": 12_223_264,                            # pairs blended in that launch
    "n": 1_000_000,
    "views": 2,
    "sources": {
        "paper_2602_00395_gb300/csrc/raster.cu": "8b921d07294e5538f909dd67b67d2deb0e81b2b5488131abab5203f770442d7f",
        "paper_2602_00395_gb300/csrc/common.cuh": "717ae4cfbf722db44969cb1b4c8974cb88deb3c71b60bd452f4448c33bb37054",
    },
}


def projection_reverse_bytes(n: int, views: int, sh_degree: int = SH_DEG, nu: int = NU) -> int:
    """Algorithmic bytes of the projection reverse: each Gaussian's parameter
    column read once, its cotangent row of every view read once (9 floats per
    stream, padded to a float4) and cleared for the next call, its gradient and
    z . Gz columns written."""
    rows = 11 + 3 * (sh_degree + 1) ** 2
    streams = 1 + nu
    cot = 4 * (-(-9 * streams // 4))
    return n * (4 * rows + 2 * views * 4 * cot + (2 if nu > 0 else 1) * 4 * rows)


def raster_bwd_traffic(pairs: float | None = None, n: int | None = None, views: int | None = None):
    """DRAM bytes of one reverse call, scaled from the captures: the blend's by
    the pairs it blends, the projection reverse's by its algorithmic bytes (the
    cotangent rows it reads grow with the views).  None once a source of the
    captured build has changed."""
    import hashlib
    c = RASTER_BWD_TRAFFIC
    if c["blend_bytes"] is None:
        return None
    for rel, digest in c["sources"].items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    blend = c["blend_bytes"] * (pairs / c["pairs"] if pairs is not None else 1.0)
    proj = c["projection_bytes"]
    if n is not None and views is not None:
        proj *= projection_reverse_bytes(n, views) / projection_reverse_bytes(c["n"], c["views"])
    return int(round(blend + proj))


def fp32_peak_tflops(n_sm: int, sm_mhz: float) -> float:
    """FP32 FMA peak: n_sm SMs x 128 FP32 lanes x 2 FLOP per FMA x the SM clock."""
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


# ------------------------------------------------------------------ CPU oracle
def _oracle_view(job):
    """One view's share of an oracle step (forward, reverse pass with the
    Hutchinson product) on the bench scene of n Gaussians; returns (seconds,
    grad, hz)."""
    n, v = job
    import numpy as np
    import oracle as O
    from paper_2602_00395_gb300 import synth as S
    sc = S.make_scene(n, SH_DEG, seed=1000, kind="clusters", extent=10.0)
    cam = [S.camera_ring(RING, W, H, 10.0, seed=7)[v * (RING // N_VIEWS)]]
    target = S.noise_target(1, H, W, seed=2000 + v).astype(np.float64)
    P = O.params64(sc)
    t0 = time.perf_counter()
    out = O.backward(P, SH_DEG, cam, target, seed=42, t=1, nu=NU)
    return time.perf_counter() - t0, out["grad"], out["hz"]


def oracle_pool():
    """Spawned worker processes for the oracle, one per view up to the core count."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = min(N_VIEWS, os.cpu_count() or 1)
    ex = cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"))
    list(ex.map(_oracle_view, [(1000, v) for v in range(cores)]))  # workers up, oracle loaded
    return ex, cores


def run_reference(args):
    """The FP64 oracle on the host's cores, timed on whole steps of the workload
    (all 1M Gaussians, the 8 views in spawned processes, gradients summed, the
    update; nothing scaled), by the wall clock.  A step takes tens of seconds, so
    the arm times as many of the requested steps as fit about three minutes and
    reports the steps it ran."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import __graft_entry__  # noqa: F401
    import oracle
    oracle.build()
    pool = oracle_pool()
    try:
        times, full = [], None
        for k in range(max(1, args.steps)):
            full = oracle_full_step(pool, args.n)
            times.append(full["oracle_full_step_s"])
            if sum(times) + times[-1] > 180.0:
                break
    finally:
        pool[0].shutdown()
    step_s = sum(times) / len(times)
    val = 1.0 / step_s
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(times), "steps_requested": args.steps, "warmup": 0, "ms_per_step": step_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": full["sample"]},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": full["cores"], "kind": "oracle",
                         "sample": full["sample"]},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))





def oracle_full_step(pool=None, n: int = N_GAUSS):
    """One full oracle step of the bench workload, nothing scaled: all 1M
    Gaussians, the 8 views of one batch in spawned processes (one per view),
    gradients and Hutchinson diagonals summed, then the update; by the wall clock
    (pool: a running oracle_pool(), else one is started and stopped outside the
    timed region)."""
    import numpy as np
    import oracle as O
    from paper_2602_00395_gb300 import synth as S
    O.build()
    own = pool is None
    ex, cores = oracle_pool() if own else pool
    try:
        t0 = time.perf_counter()
        res = list(ex.map(_oracle_view, [(n, v) for v in range(N_VIEWS)]))
    finally:
        if own:
            ex.shutdown()
    g = sum(r[1] for r in res)
    hz = sum(r[2] for r in res)
    P = O.params64(S.make_scene(n, SH_DEG, seed=1000, kind="clusters", extent=10.0))
    O.tr_update(P, np.zeros_like(P), np.zeros_like(P), g, hz, SH_DEG, t=1, eps=1e-6, cfg=O.tr_config(l=1))
    dt = time.perf_counter() - t0
    return {"oracle_full_step_s": dt, "value": 1.0 / dt, "unit": UNIT, "cores": cores,
            "host_cpus": os.cpu_count(), "per_view_s": [r[0] for r in res],
            "sample": f"one full step: {n} Gaussians, {N_VIEWS} views at {W}x{H} in {cores} spawned "
                      f"processes (each generating its scene), nu={NU}, update; nothing scaled"}


# The smaller configurations: (name, Gaussians, SH degree, scene kind, extent,
# log-scale shift, image, views per step, nu, oracle steps timed).
CONFIGS = [
    ("tiny plain step", 1000, 0, "cube", 1.0, None, (128, 128), 1, 1, 10),
    ("plain single-view training", 100_000, 3, "cube", 5.0, None, (1297, 840), 1, 1, 5),
    ("large scene, recomputed transmittance", 6_000_000, 3, "clusters", 10.0, None, (1920, 1080), 1, 1, 0),
]


def _config_oracle_step(job):
    name, n, deg, kind, ext, shift, (w, h), V, nu, _ = job
    import numpy as np
    import oracle as O
    from paper_2602_00395_gb300 import synth as S
    sc = S.make_scene(n, deg, seed=1000, kind=kind, extent=ext, log_scale_shift=shift)
    cams = S.camera_ring(RING, w, h, ext, seed=7)[:V] if n > 1000 else [S.single_camera(w, h)]
    target = S.noise_target(V, h, w, seed=2000).astype(np.float64)
    P = O.params64(sc)
    t0 = time.perf_counter()
    out = O.backward(P, deg, cams, target, seed=42, t=1, nu=nu)
    O.tr_update(P, np.zeros_like(P), np.zeros_like(P), out["grad"], out["hz"], deg, t=1, eps=1e-6,
                cfg=O.tr_config(l=1))
    return time.perf_counter() - t0


def run_configs(device):
    """GPU plain loop (the six calls per step, no graph) of configurations 1, 2
    and 4, and the oracle's full steps of configurations 1 and 2 (single
    thread, nothing scaled)."""
    import torch
    import oracle as O
    from paper_2602_00395_gb300 import gs3dtr as G
    from paper_2602_00395_gb300 import synth as S
    from paper_2602_00395_gb300.engine import TRConfig, TRStep, eps_schedule
    O.build()
    out = []
    for job in CONFIGS:
        name, n, deg, kind, ext, shift, (w, h), V, nu, osteps = job
        sc = S.make_scene(n, deg, seed=1000, kind=kind, extent=ext, log_scale_shift=shift)
        cams = S.camera_ring(RING, w, h, ext, seed=7) if n > 1000 else [S.single_camera(w, h)]
        e = TRStep(n, deg, V, w, h, nu=nu, tile=TILE, cfg=TRConfig(l=1), device=device)
        e.set_params(sc.params)
        e.set_cameras(cams[:V])
        gt = S.make_scene(n, deg, seed=2000, kind=kind, extent=ext, log_scale_shift=shift)
        e.set_params(gt.params)
        e.ensure_capacity()
        e.render()
        e.target.copy_(e.image)
        e.set_params(sc.params)
        need = e.ensure_capacity()
        if need * 1.2 > e.capacity:
            e._alloc_pairs(int(need * 1.4))
        stream = torch.cuda.Stream(device=device)
        total = 10 if n <= 100_000 else 500
        dev_cams = [torch.from_numpy(G.camera_bytes([c])).to(device) for c in cams[:8]]
        with torch.cuda.stream(stream):
            for t in range(1, 4):
                e.cams = dev_cams[(t - 1) % len(dev_cams)]
                e.step(t, eps_schedule(t, total), stream)
        K = 10 if n <= 1000 else 20
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            for t in range(4, 4 + K):
                e.cams = dev_cams[(t - 1) % len(dev_cams)]
                e.step(t, eps_schedule(t, total), stream)
            z.record(stream)
        z.synchronize()
        ms = a.elapsed_time(z) / K
        status = e.read_status()
        del e
        torch.cuda.empty_cache()
        row = {"config": name, "gaussians": n, "sh_degree": deg, "image": f"{w}x{h}", "views_per_step": V,
               "nu": nu, "gpu_plain_ms_per_step": ms, "gpu_plain_steps_per_s": 1e3 / ms, "status_word": status,
               "pairs": need}
        if osteps:
            times = [_config_oracle_step(job) for _ in range(osteps)]
            row["oracle_steps_timed"] = osteps
            row["oracle_s_per_step"] = sum(times) / len(times)
            row["oracle_steps_per_s"] = len(times) / sum(times)
            row["oracle_cores"] = 1
        out.append(row)
    return out


def rooflines(eng, per_call, sum_nc, pairs_timed, local, full_size):
    """The dominant call's roofline and every call's, from per-call CUDA-event
    times and the work units of the same launches."""
    import torch
    hbm, sm_mhz, src = peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = fp32_peak_tflops(n_sm, sm_mhz)
    # every call against its own bound (HBM for the streaming calls, the FP32
    # pipe for the blends); algorithmic work per unit as documented
    R = N_VIEWS * eng.n_pad
    rows = 11 + 3 * (SH_DEG + 1) ** 2

    def bits(v):
        b = 0
        while (1 << b) < v:
            b += 1
        return b
    rec_pass = 4
    pair_pass = max(1, (bits(N_VIEWS * eng.Tx * eng.Ty) + 7) // 8)
    work = {
        "project": ("hbm", eng.n * rows * 4 + N_VIEWS * eng.n * 48 * (1 + NU)),
        # per pair (32-bit tile key, 32-bit splat index): emit 8 B, 16 B per pass,
        # ranges 4 B; per record: 48 B read and 28 B written by the count pass
        # (count, key, value, row-table header; the row entries are not counted),
        # 16 B per pass, 12 B count gather, 16 B header read by the emit
        "bin_sort": ("hbm", pairs_timed * (8 + 16 * pair_pass + 4) + R * (48 + 28 + 16 * rec_pass + 12 + 16)),
        "raster_fwd": ("alu", raster_fwd_flops_per_unit() * sum_nc),
        "raster_bwd": ("alu", raster_bwd_flops_per_unit() * sum_nc),
        "update": ("hbm", eng.n * rows * 4 * (5 + 3)),
    }
    roof_calls = {}
    for name, (kind, amount) in work.items():
        ms_c = per_call[name]
        if kind == "hbm":
            ach = amount / (ms_c * 1e-3) / 1e9
            roof_calls[name] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                                "bytes": amount, "ms": ms_c}
        else:
            ach = amount / (ms_c * 1e-3) / 1e12
            roof_calls[name] = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                                "frac": ach / fp32_peak, "flop": amount, "ms": ms_c}
    fwd_ms, bwd_ms = per_call["raster_fwd"], per_call["raster_bwd"]
    if fwd_ms >= bwd_ms:
        name, ms_k, per_unit = "gs_raster_fwd (blend + fused JVP, nu=2)", fwd_ms, raster_fwd_flops_per_unit()
        traffic = None
    else:
        name, ms_k, per_unit = "gs_raster_bwd (reverse blend, 1+nu streams, + projection reverse)", bwd_ms, raster_bwd_flops_per_unit()
        traffic = raster_bwd_traffic(pairs_timed, N_GAUSS, N_VIEWS) if full_size else None
    achieved = per_unit * sum_nc / (ms_k * 1e-3) / 1e12
    roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": traffic, "launch_ms": ms_k,
            "peak_source": (f"{n_sm} SMs (device query) x 128 FP32 lanes x 2 FLOP x {sm_mhz:.0f} MHz "
                            f"({src} max SM clock)"),
            "work": (f"{per_unit} FLOP x {sum_nc:.4g} units (sum over pixels of n_contrib, all views, mean of "
                     f"the steps the call was timed on)")}
    return roof, roof_calls


def dp_steps(eng, cam_dev, targets, my_batches, K, t0, stream, exchange, host_targets=None):
    """K data-parallel steps on this rank: its view batch of each step (step t
    takes my_batches[(t - 1) % len]), the eager six calls with the all-reduce of
    g and hz between the reverse pass and the update.  With host_targets each
    step's targets are copied from pinned host memory and the loss read back
    inside the steps.  Returns ms from CUDA events on `stream`."""
    import torch
    from paper_2602_00395_gb300.engine import eps_schedule
    loss_host = torch.zeros(max(K, 1), dtype=torch.float32).pin_memory()
    dev_tg = torch.empty_like(targets[0]) if host_targets is not None else None
    a = torch.cuda.Event(enable_timing=True)
    z = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
        for k in range(K):
            t = t0 + k
            b = my_batches[(t - 1) % len(my_batches)]
            eng.cams = cam_dev[b]
            if host_targets is not None:
                dev_tg.copy_(host_targets[b], non_blocking=True)
                eng.target = dev_tg
            else:
                eng.target = targets[b]
            eng.step(t, eps_schedule(t, 30000), stream, exchange)
            if host_targets is not None:
                loss_host[k:k + 1].copy_(eng.loss_val, non_blocking=True)
        z.record(stream)
    z.synchronize()
    return a.elapsed_time(z)


def run_data_parallel(args, ws, rank, local, device):
    """N ranks split the training over views: every rank holds the same scene and
    trust-region state and renders its own batch of 8 views per step; the
    gradients and Hutchinson diagonals are summed over ranks (NCCL all-reduce,
    weighted by each rank's residual count) before the identical update on every
    rank.  Weak scaling: each rank's work per step is fixed; value = the view
    batches all ranks processed per second."""
    import torch
    import torch.distributed as dist
    from paper_2602_00395_gb300.exchange import GradExchange
    eng, cam_dev, targets, batches, need = make_workload(args.n, device, 0)  # one scene on every rank
    stream = torch.cuda.Stream(device=device)
    mine = [b for b in range(len(cam_dev)) if b % ws == rank % len(cam_dev)] or [rank % len(cam_dev)]
    ex = GradExchange()
    dp_steps(eng, cam_dev, targets, mine, max(args.warmup, 3), 1, stream, ex)
    _, per_call = timed_steps(eng, cam_dev, targets, max(2, min(args.steps, 5)), 0, 100, stream, per_call=True)
    eng.status.zero_()
    dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms = dp_steps(eng, cam_dev, targets, mine, args.steps, 1000, stream, ex)
        torch.cuda.synchronize()
    host_targets = [tg.cpu().pin_memory() for tg in targets]
    dist.barrier()
    e2e_ms = dp_steps(eng, cam_dev, targets, mine, args.steps, 5000, stream, ex, host_targets)
    tt = torch.tensor([ms, e2e_ms], device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ms, e2e_ms = (float(v) for v in tt.cpu())
    sum_nc = per_call.pop("sum_n_contrib")
    pairs_timed = per_call.pop("pairs")
    roof, roof_calls = rooflines(eng, per_call, sum_nc, pairs_timed, local, args.n == N_GAUSS)
    status = eng.read_status()
    if rank == 0:
        ms_per_step = ms / args.steps
        print(json.dumps({
            "metric": METRIC, "value": ws * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_gaussians": args.n, "views_per_step": N_VIEWS * ws,
                       "views_per_rank": N_VIEWS, "image": f"{W}x{H}", "nu": NU,
                       "parallelism": f"data-parallel over views, {ws} ranks, NCCL all-reduce of g and hz",
                       "graph": "eager six calls per step (the all-reduce sits between reverse pass and update)",
                       "l2": "inputs larger than L2 (236 MB parameters, 199 MB targets per rank and step)"},
            "per_call_ms": per_call, "status_word": status,
            "e2e": {"value": ws * args.steps / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": targets[0].numel() * 4, "d2h_bytes_per_step": 4},
            # the eager step launches no step counter
            "gpu_launches": (kernel_launches_per_step(eng) - 1) * args.steps,
            "roofline": roof, "roofline_calls": roof_calls, "clocks": clk.summary(), "cpu_baseline": None,
        }))


# ------------------------------------------------------------------ main
def run_cuda(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    import __graft_entry__
    __graft_entry__.build() if rank == 0 or ws == 1 else None
    if ws > 1:
        torch.distributed.barrier()
    from paper_2602_00395_gb300 import gs3dtr as G
    G.load()
    if ws > 1 and not args.profile_steps:
        run_data_parallel(args, ws, rank, local, device)
        torch.distributed.destroy_process_group()
        return
    if args.profile_steps:
        ptile = tuple(int(v) for v in args.profile_tile.lower().split("x"))
        eng, cam_dev, targets, batches, need = make_workload(args.n, device, rank, args.profile_views, 2, ptile)
        stream = torch.cuda.Stream(device=device)
        timed_steps(eng, cam_dev, targets, args.profile_steps, 0, 1, stream)
        torch.cuda.synchronize()
        print(json.dumps({"profile_steps": args.profile_steps, "views": args.profile_views, "pairs": need,
                          "sum_n_contrib": float(eng.n_contrib.double().sum().item()),
                          "status_word": eng.read_status()}))
        return
    eng, cam_dev, targets, batches, need = make_workload(args.n, device, rank)
    stream = torch.cuda.Stream(device=device)
    # tile shape: measured on this workload (the step is rebuilt if another shape wins)
    from paper_2602_00395_gb300.engine import autotune_tile
    (bw, bh, best_batch), tile_ms = autotune_tile(eng, stream=stream)
    if (bw, bh, best_batch) != (*TILE, 0):
        eng, cam_dev, targets, batches, need = retile_workload(eng, cam_dev, targets, batches, (bw, bh), device,
                                                               best_batch)
    # warm-up
    timed_steps(eng, cam_dev, targets, max(args.warmup, 3), 0, 1, stream)
    torch.cuda.synchronize()
    eng.status.zero_()
    # every measured sequence below starts from this state, so that each times
    # the same stretch of training (the pair count drifts as the scene trains)
    state0 = [b.clone() for b in (eng.x, eng.g_ema, eng.d_ema)]

    def restore():
        torch.cuda.synchronize()
        for b, v in zip((eng.x, eng.g_ema, eng.d_ema), state0):
            b.copy_(v)
        torch.cuda.synchronize()
    # per-call breakdown (separate, untimed for the headline)
    _, per_call = timed_steps(eng, cam_dev, targets, max(2, min(args.steps, 5)), 0, 100, stream, per_call=True)
    # the eager step sequence (six calls per step from the host), for reference
    restore()
    eager_ms, _ = timed_steps(eng, cam_dev, targets, args.steps, 0, 500, stream)
    # one captured graph per view batch; each replay is a whole step
    sched = G.gs_eps_schedule(1e-6, 1e-8, 30000)
    graphs = []
    for b in range(len(cam_dev)):
        eng.cams = cam_dev[b]
        eng.target = targets[b]
        graphs.append(eng.capture_step(True, sched, stream))
    restore()
    graph_steps(eng, graphs, max(args.warmup, 3), 700, stream)  # untimed replays
    # timed region
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms = graph_steps(eng, graphs, args.steps, 1000, stream)
        torch.cuda.synchronize()
    status = eng.read_status()
    if ws > 1:
        import torch.distributed as dist
        tt = torch.tensor([ms], device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
        dist.barrier()
    ms_per_step = ms / args.steps
    value = ws * args.steps / (ms / 1e3)
    # end to end through the C ABI from pinned host buffers
    host_targets = [tg.cpu().pin_memory() for tg in targets]
    restore()
    e2e_ms, e2e_wall, h2d, d2h = e2e_steps(eng, batches, host_targets, args.steps, 5000, stream, sched)
    e2e_val = ws * args.steps / (e2e_ms / 1e3)
    # the cost of curvature: gradient-only steps, and l = 10 with S2 != S1
    restore()
    curv = curvature_costs(eng, cam_dev, targets, 20, stream)
    restore()
    variants = variant_costs(eng, cam_dev, targets, 10, stream)
    restore()
    # the plain one-view-at-a-time loop on the same workload
    plain_ms = plain_loop_steps(eng, cam_dev, targets, max(3, min(args.steps, 10)), 9000, stream, device)
    restore()
    memory = memory_footprint(eng, cam_dev, targets, device, stream)
    # roofline of the dominant call: the work units are those of the launches
    # the per-call times come from (summed between the calls of those steps)
    torch.cuda.synchronize()
    sum_nc = per_call.pop("sum_n_contrib")
    pairs_timed = per_call.pop("pairs")
    roof, roof_calls = rooflines(eng, per_call, sum_nc, pairs_timed, local, args.n == N_GAUSS)
    clocks = clk.summary()
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            full = oracle_full_step(n=args.n)
            cpu = {"value": full["value"], "unit": UNIT, "cores": full["cores"], "kind": "oracle",
                   "sample": full["sample"], "sample_seconds": full["oracle_full_step_s"],
                   "host_cpus": full["host_cpus"], "per_view_s": full["per_view_s"]}
        except Exception as ex:  # pragma: no cover
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_gaussians": args.n, "views_per_step": N_VIEWS,
                       "image": f"{W}x{H}", "nu": NU, "tile": f"{eng.tile[0]}x{eng.tile[1]}",
                       "blend_batch": eng.frame.batch or "one per thread",
                       "tile_autotune_ms": {f"{a}x{b}" + (f"/{c}" if c else ""): round(v, 3)
                                            for (a, b, c), v in tile_ms.items()}, "pairs_per_step": pairs_timed,
                       "pairs_max_over_view_batches": need,
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "l2": "inputs larger than L2 (236 MB parameters, 199 MB targets per step)",
                       "view_steps_per_s": value * N_VIEWS},
            "per_call_ms": per_call, "status_word": status,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "wall_s": e2e_wall},
            "plain_loop": {"ms_per_step": plain_ms, "value": 1e3 / plain_ms, "unit": UNIT,
                           "batched_speedup": (1e3 / ms_per_step) / (1e3 / plain_ms),
                           "what": "8 single-view project/sort/fwd/bwd call sequences + averaged update, no batching"},
            "eager": {"ms_per_step": eager_ms / args.steps, "value": 1e3 * args.steps / eager_ms, "unit": UNIT,
                      "what": "the same steps as six C-ABI calls issued from the host per step, no graph"},
            "graph": "one captured CUDA graph per view batch, step index and eps_t on the device",
            "curvature": {**curv, "l1_fused_ms": ms_per_step, "overhead_l1_fused": ms_per_step / curv["gradient_only_ms"] - 1.0},
            "variants": variants, "memory": memory,
            "gpu_launches": kernel_launches_per_step(eng) * args.steps,
            "roofline": roof, "roofline_calls": roof_calls, "clocks": clocks, "cpu_baseline": cpu,
            "served": None,
        }
        if not args.no_serve:
            del eng, cam_dev, targets, graphs
            torch.cuda.empty_cache()
            out["served"] = served_metrics(device)
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.oracle_full_step:
        print(json.dumps(oracle_full_step()))
    elif args.configs:
        import torch
        torch.cuda.set_device(0)
        import __graft_entry__
        __graft_entry__.build()
        print(json.dumps({"configs": run_configs("cuda:0")}))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
