"""One 3DGS^2-TR training iteration over the C ABI (Algorithm 1 of arXiv 2602.00395).

``TRStep`` owns the device buffers of one scene and one frame (views of a fixed
size) and issues the six library calls of an iteration on a stream:

    gs_project(x, probes)        -> splat records and probe tangents
    gs_bin_sort                  -> sorted (tile, depth) pairs, tile ranges
    gs_raster_fwd(probes)        -> image, final T, n_contrib, image tangents J z_k
    gs_raster_bwd(+ tangents)    -> gradient g and Hutchinson diagonal hz (S2 = S1)
    gs_tr_update                 -> EMAs, Newton step, SHD radius, clip, update

All arithmetic runs in libgs3dtr.so; this module holds buffers and the host
loop (step counter, eps schedule).  Nothing here synchronises the stream except
``ensure_capacity``, which sizes the pair buffer once outside any timed region.
"""
from __future__ import annotations

import contextlib
import math
from dataclasses import dataclass, field

import torch

from . import gs3dtr as G
from . import synth


@dataclass
class TRConfig:
    theta1: float = 0.9
    theta2: float = 0.999
    d_floor: float = 1e-12
    color_floor: float = 1e-2
    l: int = 10
    mean_exact: int = 0

    def struct(self) -> G.gs_tr_config:
        return G.gs_tr_config(self.theta1, self.theta2, self.d_floor, self.color_floor, self.l, self.mean_exact)


def eps_schedule(t: int, total: int, eps0: float = 1e-6, eps1: float = 1e-8) -> float:
    """Exponential decay of the trust-region parameter from eps0 to eps1 over the run (Sec. 5)."""
    if total <= 1:
        return eps0
    return eps0 * (eps1 / eps0) ** ((t - 1) / (total - 1))


class TRStep:
    def __init__(self, n: int, sh_degree: int, n_views: int, width: int, height: int, *, nu: int = 1,
                 tile=(16, 16), capacity: int | None = None, loss_kind: int = G.GS_LOSS_L1,
                 gn_floor: float = 1e-3, cfg: TRConfig | None = None, probe_seed: int = 42,
                 device: str = "cuda", state=None, zero_init: bool = True, dssim_lambda: float | None = None,
                 footprint_bins: bool = True, batch: int = 0):
        """state: optional (x, g_ema, d_ema) tensors of shape rows x n_pad that the
        step uses in place of its own (a scene's resident parameters and trust-region
        state, shared by the short-lived steps of a serving loop).  zero_init=False
        leaves the buffers that the calls overwrite before reading (records,
        images, gradient, curvature, target, cameras) uninitialised, which saves a
        fill per buffer when steps are created per request.  dssim_lambda: the
        pixel loss (1 - lambda) L1 + lambda D-SSIM of Eq. pixel_loss instead of L1.
        footprint_bins: bin each splat into the tiles its alpha >= 1/255 footprint
        box reaches within its 3DGS tile square (False: the whole square); the
        images and derivatives are the same, the pairs fewer.  batch: records a
        tile's block stages per step of its list in the blends (0: one per
        thread; else a multiple of 32 up to 512)."""
        G.load()
        self.n, self.deg, self.V, self.W, self.H, self.nu = n, sh_degree, n_views, width, height, nu
        self.n_pad = synth.pad_count(n)
        self.rows = synth.n_rows(sh_degree)
        self.tile = tile
        self.device = torch.device(device)
        self.cfg = cfg or TRConfig()
        self.loss = G.gs_loss(loss_kind, gn_floor)
        self.probe_seed = probe_seed
        self.frame = G.frame_struct(n_views, width, height, *tile, footprint_bins=footprint_bins, batch=batch)
        self.Tx = -(-width // tile[0])
        self.Ty = -(-height // tile[1])
        f32 = dict(dtype=torch.float32, device=self.device)
        z = lambda *s: torch.zeros(*s, **f32)
        w = z if zero_init else (lambda *s: torch.empty(*s, **f32))  # buffers written before read
        if state is not None:
            self.x, self.g_ema, self.d_ema = state
            assert all(t.shape == (self.rows, self.n_pad) and t.dtype == torch.float32 for t in state)
        else:
            self.x = z(self.rows, self.n_pad)
            self.g_ema = z(self.rows, self.n_pad)
            self.d_ema = z(self.rows, self.n_pad)
        self.grad = w(self.rows, self.n_pad)
        # the curvature buffers exist only for a step with probes (nu > 0); a
        # gradient-only step (ADAM-TR) holds x, its two moments and the gradient
        self.hz = w(self.rows, self.n_pad) if nu > 0 else None
        self.cams = (torch.zeros if zero_init else torch.empty)(96 * n_views, dtype=torch.uint8, device=self.device)
        self.rec = w(n_views * self.n_pad * 12)
        self.tan = w((1 + nu) * n_views * self.n_pad * 12 if nu > 0 else 4)  # each record again, then its probes
        HW = width * height
        self.image = w(n_views * 3 * HW)
        self.final_T = w(n_views * HW)
        self.n_contrib = (torch.zeros if zero_init else torch.empty)(n_views * HW, dtype=torch.int32,
                                                                    device=self.device)
        self.image_tan = w(nu * n_views * 3 * HW if nu > 0 else 4)
        self.target = w(n_views * 3 * HW)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.loss_val = z(1)
        zi = torch.zeros if zero_init else torch.empty  # gs_bin_sort clears both before use
        self.ranges = zi(2 * n_views * self.Tx * self.Ty, dtype=torch.int32, device=self.device)
        self.n_pairs = zi(1, dtype=torch.int32, device=self.device)
        self.order = zi(n_views * self.Tx * self.Ty, dtype=torch.int32, device=self.device)  # heaviest tiles first
        self.bwd_ws = torch.empty(G.gs_raster_bwd_workspace_size(self.n_pad, self.frame, nu), dtype=torch.uint8,
                                  device=self.device)
        self.dssim_lambda = dssim_lambda
        if dssim_lambda is not None:
            self.cot_img = torch.empty((1 + nu) * n_views * 3 * HW, dtype=torch.float32, device=self.device)
            self.dssim_ws = torch.empty(G.gs_dssim_workspace_size(self.frame, nu), dtype=torch.uint8,
                                        device=self.device)
        self._alloc_pairs(capacity or max(1 << 16, 8 * n * n_views))
        self.t = 0
        self.t_dev = torch.zeros(1, dtype=torch.int64, device=self.device)  # step index of captured graphs

    # ------------------------------------------------------------ buffers
    def _alloc_pairs(self, capacity: int) -> None:
        self.capacity = int(capacity)
        self.keys = torch.empty(self.capacity, dtype=torch.int32, device=self.device)
        self.vals = torch.empty(self.capacity, dtype=torch.int32, device=self.device)
        # the forward pass's block masks of the pairs, read by the reverse passes
        self.masks = torch.empty(self.capacity, dtype=torch.uint8, device=self.device)
        self.masks_valid = False  # set by a forward pass, cleared by the next bin-sort
        self.sort_ws = torch.empty(G.gs_bin_sort_workspace_size(self.n_pad, self.frame, self.capacity),
                                   dtype=torch.uint8, device=self.device)

    def set_params(self, params) -> None:
        p = torch.as_tensor(params, dtype=torch.float32)
        self.x.zero_()
        self.x[:, : p.shape[1]].copy_(p[:, : self.n_pad].to(self.device))

    def set_cameras(self, cams) -> None:
        assert len(cams) == self.V and all(c.width == self.W and c.height == self.H for c in cams)
        self.cams.copy_(torch.from_numpy(G.camera_bytes(cams)).to(self.device))

    def set_target(self, target) -> None:
        self.target.copy_(torch.as_tensor(target, dtype=torch.float32).reshape(-1).to(self.device))

    # ------------------------------------------------------------ structs
    def P(self, t) -> G.gs_params:
        return G.params_struct(t, self.n, self.deg)

    def proj(self) -> G.gs_projected:
        return G.gs_projected(self.rec.data_ptr(), self.tan.data_ptr())

    def sorted(self, masks: bool = True) -> G.gs_sorted:
        """The sorted pairs; with masks, the block-mask buffer (the forward pass
        writes it, a reverse pass reads it)."""
        return G.gs_sorted(self.keys.data_ptr(), self.vals.data_ptr(), self.ranges.data_ptr(),
                           self.n_pairs.data_ptr(), self.capacity, self.order.data_ptr(),
                           self.masks.data_ptr() if masks else None)

    def sorted_rev(self) -> G.gs_sorted:
        """The sorted pairs for a reverse pass: the masks only if a forward pass
        has written them for the current sort."""
        return self.sorted(self.masks_valid)

    def probe(self, t: int | None, device_t: bool = False) -> G.gs_probe | None:
        if self.nu == 0:
            return None
        return G.probe_struct(self.probe_seed, t or 0, self.nu, self.t_dev if device_t else None)

    # ------------------------------------------------------------ calls
    def project(self, t: int | None = None, probes: bool = True, stream=None) -> None:
        pr = self.probe(t) if (probes and t is not None) else None
        G.gs_project(self.P(self.x), self.cams, self.frame, pr, self.proj(), self.status, stream)

    def bin_sort(self, stream=None) -> None:
        G.gs_bin_sort(self.proj(), self.n_pad, self.frame, self.sort_ws, self.sorted(), self.status, stream)
        self.masks_valid = False

    def raster_fwd(self, t: int | None = None, probes: bool = True, stream=None) -> None:
        pr = self.probe(t) if (probes and t is not None) else None
        G.gs_raster_fwd(self.proj(), self.sorted(), self.n_pad, self.frame, pr, self.image, self.final_T,
                        self.n_contrib, self.image_tan if pr else None, self.status, stream)
        self.masks_valid = True

    def raster_bwd(self, t: int | None = None, probes: bool = True, stream=None) -> None:
        pr = self.probe(t) if (probes and t is not None) else None
        if self.dssim_lambda is not None:  # D-SSIM: the cotangent images first, then the reverse pass
            nu = pr.nu if pr else 0
            G.gs_dssim_cotangents(self.frame, self.image, self.target, self.image_tan if pr else None, nu,
                                  self.dssim_lambda, self.loss.gn_floor, True, self.cot_img, self.loss_val,
                                  self.dssim_ws, self.status, stream)
            self.raster_bwd_cotangent(self.cot_img, t if pr else None, True, stream)
            return
        G.gs_raster_bwd(self.P(self.x), self.cams, self.frame, self.proj(), self.sorted_rev(), self.image,
                        self.target, self.final_T, self.n_contrib, self.image_tan if pr else None, pr, self.loss,
                        self.P(self.grad), self.P(self.hz) if pr else None, self.loss_val, self.bwd_ws,
                        self.status, stream)

    def raster_bwd_cotangent(self, cot, t: int | None = None, want_grad: bool = True, stream=None) -> None:
        """Reverse pass from caller-formed cotangent images (GS_LOSS_COTANGENT):
        cot is S x V x 3 x H x W (dL/dC first when want_grad, then one vector per
        probe when t is given); grad and/or hz are written."""
        pr = self.probe(t) if t is not None else None
        loss = G.gs_loss(G.GS_LOSS_COTANGENT, self.loss.gn_floor)
        if want_grad:
            G.gs_raster_bwd(self.P(self.x), self.cams, self.frame, self.proj(), self.sorted_rev(), self.image, cot,
                            self.final_T, self.n_contrib, None, pr, loss, self.P(self.grad),
                            self.P(self.hz) if pr else None, None, self.bwd_ws, self.status, stream)
        else:
            G.gs_hvp_diag(self.P(self.x), self.cams, self.frame, self.proj(), self.sorted_rev(), self.image, cot,
                          self.final_T, self.n_contrib, None, pr, loss, self.P(self.hz), self.bwd_ws, self.status,
                          stream)

    def hvp_weighted(self, t: int, weights, stream=None) -> None:
        """Hutchinson diagonal of J^T diag(weights) J (GS_LOSS_WEIGHTED): the
        reverse pass forms weights * J z_k from the image tangents of the last
        forward pass with the probes of step t; weights is V x 3 x H x W."""
        pr = self.probe(t)
        loss = G.gs_loss(G.GS_LOSS_WEIGHTED, self.loss.gn_floor)
        G.gs_hvp_diag(self.P(self.x), self.cams, self.frame, self.proj(), self.sorted_rev(), self.image, weights,
                      self.final_T, self.n_contrib, self.image_tan, pr, loss, self.P(self.hz), self.bwd_ws,
                      self.status, stream)

    def hvp_diag(self, t: int, stream=None) -> None:
        pr = self.probe(t)
        if self.dssim_lambda is not None:
            G.gs_dssim_cotangents(self.frame, self.image, self.target, self.image_tan, pr.nu, self.dssim_lambda,
                                  self.loss.gn_floor, False, self.cot_img, None, self.dssim_ws, self.status, stream)
            self.raster_bwd_cotangent(self.cot_img, t, False, stream)
            return
        G.gs_hvp_diag(self.P(self.x), self.cams, self.frame, self.proj(), self.sorted_rev(), self.image, self.target,
                      self.final_T, self.n_contrib, self.image_tan, pr, self.loss, self.P(self.hz), self.bwd_ws,
                      self.status, stream)

    def update(self, t: int, eps: float, with_hz: bool = True, eta_out=None, stream=None) -> None:
        G.gs_tr_update(self.P(self.x), self.P(self.g_ema), self.P(self.d_ema), self.P(self.grad),
                       self.P(self.hz) if with_hz else None, self.cfg.struct(), t, eps,
                       self.P(eta_out) if eta_out is not None else None, self.status, stream)

    def update_adam(self, t: int, eps: float, adam=None, eta_out=None, stream=None) -> None:
        """ADAM-TR update (Sec. 5 ablation); g_ema and d_ema hold Adam's m and v."""
        G.gs_adam_tr_update(self.P(self.x), self.P(self.g_ema), self.P(self.d_ema), self.P(self.grad),
                            self.cfg.struct(), adam or G.adam_struct(), t, eps,
                            self.P(eta_out) if eta_out is not None else None, self.status, stream)

    def step_adam(self, t: int, eps: float, adam=None, stream=None) -> None:
        """One ADAM-TR iteration: the gradient of the frame's views, then the
        Adam step clipped by the Hellinger trust region (no curvature)."""
        self.loss_val.zero_()
        self.project(t, probes=False, stream=stream)
        self.bin_sort(stream)
        self.raster_fwd(t, probes=False, stream=stream)
        self.raster_bwd(t, probes=False, stream=stream)
        self.update_adam(t, eps, adam, None, stream)

    # ------------------------------------------------------------ composite
    def render(self, stream=None) -> None:
        self.project(None, probes=False, stream=stream)
        self.bin_sort(stream)
        self.raster_fwd(None, probes=False, stream=stream)

    def step_s2(self, t: int, eps: float, s2_cams, s2_target, stream=None) -> None:
        """One iteration of Algorithm 1 with the curvature mini-batch S2 drawn
        apart from S1 (Sec. 4.1): the gradient comes from the frame's views
        (self.cams / self.target); on curvature steps ((t - 1) % l == 0) the
        Hutchinson product comes from S2's views (same count, so the |S| factors
        cancel), by a second projection with the probes, a forward pass with the
        tangents and gs_hvp_diag.  s2_cams / s2_target are device tensors laid out
        as self.cams / self.target."""
        hvp = self.nu > 0 and ((t - 1) % self.cfg.l) == 0
        self.loss_val.zero_()
        self.project(t, probes=False, stream=stream)
        self.bin_sort(stream)
        self.raster_fwd(t, probes=False, stream=stream)
        self.raster_bwd(t, probes=False, stream=stream)
        if hvp:
            cams1, target1 = self.cams, self.target
            self.cams, self.target = s2_cams, s2_target
            try:
                self.project(t, probes=True, stream=stream)
                self.bin_sort(stream)
                self.raster_fwd(t, probes=True, stream=stream)
                self.hvp_diag(t, stream)
            finally:
                self.cams, self.target = cams1, target1
        self.update(t, eps, with_hz=hvp, stream=stream)

    def step_device(self, hvp: bool, schedule: G.gs_eps_schedule, stream=None) -> None:
        """One step of Algorithm 1 whose index lives in device memory (self.t_dev):
        advance it, then the six calls reading it there, so that the sequence can
        be captured once as a CUDA graph and replayed for successive steps.
        `hvp` fixes whether the captured step carries the probes (every step for
        l = 1; capture one graph of each kind for l > 1)."""
        G.gs_step_advance(self.t_dev, stream)
        self.loss_val.zero_()
        pr = self.probe(None, device_t=True) if hvp else None
        G.gs_project(self.P(self.x), self.cams, self.frame, pr, self.proj(), self.status, stream)
        self.bin_sort(stream)
        G.gs_raster_fwd(self.proj(), self.sorted(), self.n_pad, self.frame, pr, self.image, self.final_T,
                        self.n_contrib, self.image_tan if pr else None, self.status, stream)
        self.masks_valid = True
        G.gs_raster_bwd(self.P(self.x), self.cams, self.frame, self.proj(), self.sorted_rev(), self.image,
                        self.target, self.final_T, self.n_contrib, self.image_tan if pr else None, pr, self.loss,
                        self.P(self.grad), self.P(self.hz) if pr else None, self.loss_val, self.bwd_ws,
                        self.status, stream)
        G.gs_tr_update_dev(self.P(self.x), self.P(self.g_ema), self.P(self.d_ema), self.P(self.grad),
                           self.P(self.hz) if pr else None, self.cfg.struct(), self.t_dev, schedule, None,
                           self.status, stream)

    def capture_step(self, hvp: bool, schedule: G.gs_eps_schedule, stream=None):
        """A CUDA graph of step_device; each replay advances self.t_dev by one.
        Capturing runs nothing.  Make one eager step first (it sets the kernels'
        shared-memory attributes, which capture cannot record)."""
        s = stream or torch.cuda.Stream(device=self.device)
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize(self.device)
        with torch.cuda.graph(g, stream=s):
            self.step_device(hvp, schedule, s)
        return g

    def step(self, t: int, eps: float, stream=None, exchange=None) -> None:
        """One iteration of Algorithm 1 on the frame's views (S1 = S2).  With an
        exchange (exchange.GradExchange) the step's views are this rank's share
        of a data-parallel step: after the reverse pass the gradient and the
        Hutchinson diagonal are summed over ranks, each weighted by its share of
        the residual count (Sec. 4.1 normalises by m over all views), and every
        rank then applies the same update."""
        hvp = self.nu > 0 and ((t - 1) % self.cfg.l) == 0
        self.loss_val.zero_()
        self.project(t, probes=hvp, stream=stream)
        self.bin_sort(stream)
        self.raster_fwd(t, probes=hvp, stream=stream)
        self.raster_bwd(t, probes=hvp, stream=stream)
        if exchange is not None:
            with torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext():
                exchange(3 * self.W * self.H * self.V, self.grad, self.hz if hvp else None)
        self.update(t, eps, with_hz=hvp, stream=stream)

    def ensure_capacity(self, headroom: float = 1.25) -> int:
        """Project and bin once, read the pair count (one host sync) and grow the pair buffer if needed."""
        self.project(None, probes=False)
        self.bin_sort()
        torch.cuda.synchronize(self.device)
        need = int(self.n_pairs.item())
        if need > self.capacity:
            self._alloc_pairs(int(need * headroom) + 1024)
            self.status.zero_()
        return need

    def read_status(self) -> int:
        return int(self.status.item())


def autotune_tile(eng: TRStep, candidates=((16, 16), (32, 8), (8, 32), (16, 8), (32, 16), (16, 32)),
                  batches=(0, 64, 256), steps: int = 3, stream=None) -> tuple[tuple[int, int, int], dict]:
    """Pick the tile shape, then the blends' per-block record batch for it, with
    the shortest step on the caller's own workload: each candidate is a TRStep
    with the same parameters, cameras, targets and probes that runs one untimed
    and `steps` timed steps (CUDA events), starting from copies of eng's state so
    that eng is left unchanged.  Returns (tile_w, tile_h, batch) and the ms per
    step of every candidate, keyed (tile_w, tile_h, batch)."""
    s = stream or torch.cuda.Stream(device=eng.device)
    times = {}

    def run(tile, batch):
        e = TRStep(eng.n, eng.deg, eng.V, eng.W, eng.H, nu=eng.nu, tile=tile, cfg=eng.cfg,
                   probe_seed=eng.probe_seed, device=str(eng.device),
                   footprint_bins=bool(eng.frame.footprint_bins), batch=batch)
        for dst, src in ((e.x, eng.x), (e.g_ema, eng.g_ema), (e.d_ema, eng.d_ema), (e.cams, eng.cams),
                         (e.target, eng.target)):
            dst.copy_(src)
        e.ensure_capacity()
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            e.step(1, 1e-6, s)
            start.record(s)
            for t in range(2, 2 + steps):
                e.step(t, 1e-6, s)
            stop.record(s)
        stop.synchronize()
        times[(tile[0], tile[1], batch)] = start.elapsed_time(stop) / steps
        del e
        torch.cuda.empty_cache()

    for tile in candidates:
        run(tile, 0)
    best_tile = min(candidates, key=lambda t: times[(t[0], t[1], 0)])
    for batch in batches:
        if batch:
            run(best_tile, batch)
    best = min((k for k in times if (k[0], k[1]) == tuple(best_tile)), key=times.get)
    return best, times


@dataclass
class BatchEntry:
    """One request of a batch: one view of a resident scene.  x, g_ema, d_ema are
    the scene's rows x n_pad state (updated in place by a training step), cam its
    camera (96 bytes on the device), target its 3 x H x W target image (device)."""
    x: torch.Tensor
    g_ema: torch.Tensor
    d_ema: torch.Tensor
    n: int
    cam: torch.Tensor
    target: torch.Tensor | None = None
    t: int = 1
    eps: float = 1e-6


class BatchStep:
    """Training steps or renders of several requests of one image size in shared
    launches (gs_project_batch, gs_bin_sort, gs_raster_fwd, gs_raster_bwd_batch,
    gs_tr_update_batch): request b is view b of the batch frame, its splat
    records in slot b of one set of buffers.  Each request keeps its own
    objective (m = 3 H W), probes (its scene's step t) and update; its image is
    images()[b].  Buffers are allocated for the batch at construction (on the
    current stream, from PyTorch's caching allocator), or taken from `pool`, a
    dict of buffers that a caller keeps per stream and that grow as needed:
    consecutive batches on one stream then reuse them (and the reverse pass
    finds its workspace already clear).  A pooled batch's outputs (images())
    are valid until the next batch with the same pool starts."""

    def __init__(self, entries: list[BatchEntry], width: int, height: int, *, sh_degree: int = 3, nu: int = 1,
                 tile=(16, 16), capacity: int, train: bool = True, loss_kind: int = G.GS_LOSS_L1,
                 gn_floor: float = 1e-3, cfg: TRConfig | None = None, probe_seed: int = 42, device: str = "cuda",
                 footprint_bins: bool = True, batch: int = 0, pool: dict | None = None):
        G.load()
        self.pool = pool
        assert 1 <= len(entries) <= G.GS_BATCH_MAX
        self.entries, self.B, self.W, self.H, self.deg = entries, len(entries), width, height, sh_degree
        self.train, self.nu = train, (nu if train else 0)
        self.cfg = cfg or TRConfig()
        self.loss = G.gs_loss(loss_kind, gn_floor)
        self.probe_seed = probe_seed
        self.device = torch.device(device)
        self.rows = synth.n_rows(sh_degree)
        self.n_pad = max(e.x.shape[1] for e in entries)
        self.frame = G.frame_struct(self.B, width, height, *tile, footprint_bins=footprint_bins, batch=batch)
        Tx, Ty = -(-width // tile[0]), -(-height // tile[1])
        f32, i32, u8 = torch.float32, torch.int32, torch.uint8
        buf = self._buf
        HW, B = width * height, self.B
        self.rec = buf("rec", B * self.n_pad * 12, f32)
        self.tan = buf("tan", (1 + self.nu) * B * self.n_pad * 12 if self.nu else 4, f32)
        self.image = buf("image", B * 3 * HW, f32)
        self.final_T = buf("final_T", B * HW, f32)
        self.n_contrib = buf("n_contrib", B * HW, i32)
        self.image_tan = buf("image_tan", self.nu * B * 3 * HW if self.nu else 4, f32)
        self.status = buf("status", 1, i32).zero_()
        self.ranges = buf("ranges", 2 * B * Tx * Ty, i32)
        self.order = buf("order", B * Tx * Ty, i32)
        self.n_pairs = buf("n_pairs", 1, i32)
        self.capacity = int(capacity)
        self.keys = buf("keys", self.capacity, i32)
        self.vals = buf("vals", self.capacity, i32)
        self.masks = buf("masks", self.capacity, u8)  # written by the forward pass, read by the reverse
        self.sort_ws = buf("sort_ws", G.gs_bin_sort_workspace_size(self.n_pad, self.frame, self.capacity), u8)
        self.cams = torch.cat([e.cam for e in entries])
        if train:
            self.target = buf("target", B * 3 * HW, f32)
            self.loss_val = buf("loss_val", B, f32).zero_()
            self.grads = [buf(f"grad{b}", self.rows * e.x.shape[1], f32).view(self.rows, e.x.shape[1])
                          for b, e in enumerate(entries)]
            self.hzs = ([buf(f"hz{b}", self.rows * e.x.shape[1], f32).view(self.rows, e.x.shape[1])
                         for b, e in enumerate(entries)] if self.nu else None)
            self.bwd_ws = buf("bwd_ws", G.gs_raster_bwd_workspace_size(self.n_pad, self.frame, self.nu), u8)

    def _buf(self, name: str, numel: int, dtype) -> torch.Tensor:
        """A device buffer of numel elements: a new one, or the front of the pool's
        buffer of that name (replaced by a larger one when too small)."""
        if self.pool is None:
            return torch.empty(numel, dtype=dtype, device=self.device)
        t = self.pool.get(name)
        if t is None or t.dtype != dtype or t.numel() < numel:
            t = torch.empty(max(numel, 1), dtype=dtype, device=self.device)
            self.pool[name] = t
        return t[:numel]

    @staticmethod
    def working_bytes(n_pads: list[int], width: int, height: int, *, sh_degree: int = 3, nu: int = 1,
                      tile=(16, 16), capacity: int, train: bool = True) -> int:
        """Device bytes the buffers of a batch of scenes with these row pitches take."""
        B, n_pad, rows, HW = len(n_pads), max(n_pads), synth.n_rows(sh_degree), width * height
        nu = nu if train else 0
        frame = G.frame_struct(B, width, height, *tile)
        Tx, Ty = -(-width // tile[0]), -(-height // tile[1])
        b = B * n_pad * 48 * (1 + (1 + nu if nu else 0)) + B * HW * 4 * (3 + 1 + 1 + 3 * nu) + B * Tx * Ty * 12
        b += capacity * 9  # keys, values, block masks
        b += G.gs_bin_sort_workspace_size(n_pad, frame, capacity) + 96 * B
        if train:
            b += B * HW * 12 + G.gs_raster_bwd_workspace_size(n_pad, frame, nu)
            b += sum(rows * p * 4 * (1 + (1 if nu else 0)) for p in n_pads)
        return int(b)

    def items(self) -> list:
        out = []
        for b, e in enumerate(self.entries):
            P = lambda t: G.params_struct(t, e.n, self.deg)
            hvp = 1 if (self.nu and (e.t - 1) % self.cfg.l == 0) else 0
            if self.train:
                out.append(G.gs_batch_item(P(e.x), P(self.grads[b]), P(self.hzs[b]) if self.nu else G.gs_params(),
                                           P(e.g_ema), P(e.d_ema), self.cams.data_ptr() + 96 * b, e.t, e.eps, hvp))
            else:
                out.append(G.gs_batch_item(P(e.x), G.gs_params(), G.gs_params(), G.gs_params(), G.gs_params(),
                                           self.cams.data_ptr() + 96 * b, max(e.t, 1), e.eps, 0))
        return out

    def run(self, stream=None) -> None:
        """The batch's calls on `stream`: a training step of every request (or a render)."""
        items = self.items()
        pr = G.probe_struct(self.probe_seed, 0, self.nu) if self.nu else None
        proj = G.gs_projected(self.rec.data_ptr(), self.tan.data_ptr())
        srt = G.gs_sorted(self.keys.data_ptr(), self.vals.data_ptr(), self.ranges.data_ptr(),
                          self.n_pairs.data_ptr(), self.capacity, self.order.data_ptr(), self.masks.data_ptr())
        G.gs_project_batch(items, self.n_pad, self.frame, pr, proj, self.status, stream)
        G.gs_bin_sort(proj, self.n_pad, self.frame, self.sort_ws, srt, self.status, stream)
        G.gs_raster_fwd(proj, srt, self.n_pad, self.frame, pr, self.image, self.final_T, self.n_contrib,
                        self.image_tan if pr else None, self.status, stream)
        if not self.train:
            return
        HW3 = 3 * self.W * self.H
        with torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext():
            for b, e in enumerate(self.entries):
                self.target[HW3 * b: HW3 * (b + 1)].copy_(e.target, non_blocking=True)
            self.loss_val.zero_()
        G.gs_raster_bwd_batch(items, self.n_pad, self.frame, proj, srt, self.image, self.target, self.final_T,
                              self.n_contrib, self.image_tan if pr else None, pr, self.loss, self.loss_val,
                              self.bwd_ws, self.status, stream)
        G.gs_tr_update_batch(items, self.cfg.struct(), self.status, stream)

    def images(self) -> torch.Tensor:
        return self.image.view(self.B, 3, self.H, self.W)

    def read_status(self) -> int:
        return int(self.status.item())
