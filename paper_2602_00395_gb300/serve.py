"""Serving loop: many resident scenes, training-step and render requests,
continuous batching on the GPU.

* A Scene keeps its parameters and trust-region state (x, g_ema, d_ema), its
  cameras and its target images resident in HBM, and a host step counter.
* A request is one training step of Algorithm 1 on one view of a scene
  (projection, binning, forward, reverse pass with the Hutchinson probes,
  update) or one render (projection, binning, forward).  The working buffers
  of a batch of requests (records, pairs, images, cotangents, gradients,
  curvature) come from its slot's pool: each slot (stream) keeps the buffers
  of its batches and grows them as needed, so that a batch allocates nothing
  once the slot has seen a batch as large, and the reverse pass finds its
  workspace already clear.  The budget bounds the working sets of the
  batches in flight (the pools keep, per slot, the largest seen).
* Admission: a request that has arrived is started when a slot (a CUDA stream)
  is free, its scene has no request in flight (a training step changes the
  scene), and its batch's working set fits the HBM budget left by the batches
  in flight.  Requests are taken in arrival order; one that cannot start does not
  hold back later ones for other scenes, and no later request of its own scene
  overtakes it.
* Continuous batching: waiting requests of one kind and one image size start
  together as one batch in shared launches (gs_project_batch, gs_bin_sort,
  gs_raster_fwd, gs_raster_bwd_batch, gs_tr_update_batch; engine.BatchStep):
  each request is one view of the batch frame with its own scene, objective,
  probes and update, so that many small requests fill one set of launches
  instead of each paying for a full sequence of small kernels.  A batch of
  training steps holds at most one request per scene (a step changes its
  scene); renders of one scene may share a batch.  Every batch runs on its own
  stream, so batches overlap on the device, and a request that arrives while
  others run starts as soon as a slot and memory free up.  Each request keeps
  its own result, equal to the one it gets alone.
* Latency of a request = completion (its end event observed by the host) minus
  arrival, both on the host clock.

The plain loop serves the same stream one request at a time on one stream.

Across GPUs the served workload shards by scene with no collective: rank r
holds the scenes whose id is r modulo the world size (`scene_shard`) and serves
the requests for them (`shard_requests`); a request names its scene by its
global id.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import gs3dtr as G
from . import synth
from .engine import BatchEntry, BatchStep, TRConfig, TRStep, eps_schedule


@dataclass
class Request:
    rid: int
    arrival: float
    kind: str  # "train" or "render"
    scene: int
    view: int
    start: float = math.nan
    done: float = math.nan
    nbytes: int = 0
    image: object = None  # rendered image (device tensor), when results are kept
    rejected: bool = False  # working set larger than the whole budget
    batch: int = 1  # requests started together with this one (itself included)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Scene:
    """A resident scene: parameters and trust-region state, cameras and targets."""

    def __init__(self, sid: int, n: int, width: int, height: int, *, n_views: int = 8, nu: int = 1,
                 tile=(16, 16), total_steps: int = 30000, device: str = "cuda"):
        self.sid, self.n, self.W, self.H, self.nu, self.tile = sid, n, width, height, nu, tile
        self.deg, self.total_steps, self.device = 3, total_steps, torch.device(device)
        self.cfg = TRConfig(l=1)
        self.t = 0
        # the served-workload recipe: uniform cube of radius 5, log-scales shifted
        # by (1/3) ln(1e5 / N) so that the pairs per Gaussian stay comparable
        shift = math.log(5.0) + math.log(1e5 / n) / 3.0
        sc = synth.make_scene(n, self.deg, seed=1000 + sid, kind="cube", extent=5.0, log_scale_shift=shift)
        gt = synth.make_scene(n, self.deg, seed=2000 + sid, kind="cube", extent=5.0, log_scale_shift=shift)
        cams = synth.camera_ring(64, width, height, 5.0, seed=7 + sid)[:: 64 // n_views][:n_views]
        self.cams = torch.from_numpy(G.camera_bytes(cams)).to(self.device)
        # targets rendered from the ground-truth set, one view at a time
        eng = TRStep(n, self.deg, 1, width, height, nu=nu, tile=tile, cfg=self.cfg, device=device)
        eng.set_params(gt.params)
        self.targets = []
        self.need = 0
        for v in range(n_views):
            eng.cams = self.cams[96 * v: 96 * (v + 1)]
            self.need = max(self.need, eng.ensure_capacity())
            eng.render()
            self.targets.append(eng.image.clone())
        eng.set_params(sc.params)
        for v in range(n_views):
            eng.cams = self.cams[96 * v: 96 * (v + 1)]
            self.need = max(self.need, eng.ensure_capacity())
        self.capacity = int(self.need * 1.25) + 1024
        self.x, self.g_ema, self.d_ema = eng.x, eng.g_ema, eng.d_ema
        del eng
        torch.cuda.synchronize(self.device)

    @property
    def resident_bytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in (self.x, self.g_ema, self.d_ema, self.cams, *self.targets))

    def working_bytes(self, kind: str, n_views: int = 1) -> int:
        """Device bytes of the working buffers of a request over n_views views (as
        TRStep allocates them)."""
        n_pad, rows, HW, V = synth.pad_count(self.n), synth.n_rows(self.deg), self.W * self.H, n_views
        frame = G.frame_struct(V, self.W, self.H, *self.tile)
        cap = self.capacity * V
        b = V * n_pad * 12 * 4 * (2 + max(self.nu, 1))                   # records, their copies + tangents
        b += V * HW * 4 * (3 + 1 + 1 + 3 * max(self.nu, 1) + 3)          # image, T, n_contrib, tangents, target slot
        b += cap * 9 + G.gs_bin_sort_workspace_size(n_pad, frame, cap)  # keys, values, block masks
        b += G.gs_raster_bwd_workspace_size(n_pad, frame, self.nu) + 2 * rows * n_pad * 4  # cotangents, grad, hz
        return int(b)

    def make_step(self, n_views: int = 1) -> TRStep:
        """Working buffers for one request over n_views views, on the current
        stream, sharing the resident state."""
        return TRStep(self.n, self.deg, n_views, self.W, self.H, nu=self.nu, tile=self.tile,
                      capacity=self.capacity * n_views, cfg=self.cfg, device=str(self.device),
                      state=(self.x, self.g_ema, self.d_ema), zero_init=False)

    def enqueue(self, req: Request, stream) -> TRStep:
        """Issue the request's calls on `stream`; returns the step that owns its buffers."""
        with torch.cuda.stream(stream):
            e = self.make_step()
            e.cams = self.cams[96 * req.view: 96 * (req.view + 1)]
            e.target = self.targets[req.view]
            if req.kind == "train":
                self.t += 1
                e.step(self.t, eps_schedule(self.t, self.total_steps), stream)
            else:
                e.render(stream)
        return e

    def entry(self, req: Request) -> BatchEntry:
        """The batch entry of a request of this scene; a training step takes the
        scene's next step index."""
        cam = self.cams[96 * req.view: 96 * (req.view + 1)]
        if req.kind == "train":
            self.t += 1
            return BatchEntry(self.x, self.g_ema, self.d_ema, self.n, cam, self.targets[req.view], self.t,
                              eps_schedule(self.t, self.total_steps))
        return BatchEntry(self.x, self.g_ema, self.d_ema, self.n, cam, None, max(self.t, 1))


@dataclass
class ServeResult:
    requests: list
    wall_s: float
    mode: str
    slots: int = 1
    budget_bytes: int = 0
    peak_inflight_bytes: int = 0
    statuses: list = field(default_factory=list)

    def summary(self) -> dict:
        served = [r for r in self.requests if not r.rejected]
        lat = np.array([r.latency for r in served]) * 1e3
        n_train = sum(r.kind == "train" for r in served)
        return {"mode": self.mode, "requests": len(served), "rejected": len(self.requests) - len(served),
                "train_steps": n_train,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "wall_s": self.wall_s,
                "train_steps_per_s": n_train / self.wall_s, "requests_per_s": len(self.requests) / self.wall_s,
                "slots": self.slots, "budget_GB": self.budget_bytes / 1e9,
                "peak_inflight_GB": self.peak_inflight_bytes / 1e9,
                "status_words": sorted(set(self.statuses))}


def scene_shard(n_scenes: int, rank: int = 0, world: int = 1) -> list[int]:
    """Scene ids held by `rank` of `world` ranks: id % world == rank."""
    return [s for s in range(n_scenes) if s % world == rank]


def shard_requests(stream_spec, rank: int = 0, world: int = 1) -> list:
    """The requests (arrival, kind, scene, view) that `rank` serves: those for
    its scenes, in arrival order."""
    return [q for q in stream_spec if q[2] % world == rank]


def _by_sid(scenes) -> dict:
    return {sc.sid: sc for sc in scenes}


def _requests(stream_spec) -> list[Request]:
    return [Request(i, a, k, s, v) for i, (a, k, s, v) in enumerate(stream_spec)]


def plain_loop(scenes: list[Scene], stream_spec, stream=None, keep_results: bool = False) -> ServeResult:
    """One request at a time, in arrival order, on one stream (each waits for the
    previous to finish and for its own arrival)."""
    s = stream or torch.cuda.Stream()
    reqs = _requests(stream_spec)
    scenes = _by_sid(scenes)
    statuses = []
    t0 = time.perf_counter()
    for r in reqs:
        while time.perf_counter() - t0 < r.arrival:
            pass
        r.start = time.perf_counter() - t0
        e = scenes[r.scene].enqueue(r, s)
        s.synchronize()
        r.done = time.perf_counter() - t0
        statuses.append(e.read_status())
        if keep_results and r.kind == "render":
            r.image = e.image
        del e
    return ServeResult(reqs, time.perf_counter() - t0, "plain", statuses=statuses)


class Server:
    """Continuous batching of requests over resident scenes (see the module text)."""

    def __init__(self, scenes: list[Scene], slots: int = 4, budget_bytes: int | None = None, max_batch: int = 8,
                 max_pad_ratio: float | None = 4.0):
        """max_pad_ratio: a request joins a batch only if its scene's Gaussian
        count is within this factor of the batch's first (every slot of a batch
        is padded to the largest scene); None for any."""
        self.scenes = _by_sid(scenes)
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        # each slot's batch buffers, reused by its next batch (a slot runs one
        # batch at a time, so the reuse follows the previous batch's end)
        self.pools = [dict() for _ in range(slots)]
        self.budget = budget_bytes if budget_bytes is not None else 1 << 62
        self.max_batch = max(1, min(max_batch, G.GS_BATCH_MAX))
        self.max_pad_ratio = max_pad_ratio
        # each slot's status word lands here by an asynchronous copy on the slot's
        # stream, so that reading it never synchronises with requests in flight
        self.status_host = torch.zeros(slots, dtype=torch.int32).pin_memory()

    def batch_bytes(self, reqs: list) -> int:
        scs = [self.scenes[r.scene] for r in reqs]
        s0 = scs[0]
        return BatchStep.working_bytes([synth.pad_count(sc.n) for sc in scs], s0.W, s0.H, sh_degree=s0.deg,
                                       nu=s0.nu, tile=s0.tile, capacity=sum(sc.capacity for sc in scs),
                                       train=reqs[0].kind == "train")

    def start(self, batch: list, stream, pool: dict | None = None) -> BatchStep:
        scs = [self.scenes[r.scene] for r in batch]
        s0 = scs[0]
        with torch.cuda.stream(stream):
            bs = BatchStep([sc.entry(r) for sc, r in zip(scs, batch)], s0.W, s0.H, sh_degree=s0.deg, nu=s0.nu,
                           tile=s0.tile, capacity=sum(sc.capacity for sc in scs), train=batch[0].kind == "train",
                           cfg=s0.cfg, device=str(s0.device), pool=pool)
            bs.run(stream)
        return bs

    def run(self, stream_spec, keep_results: bool = False) -> ServeResult:
        reqs = _requests(stream_spec)
        waiting = deque()
        upcoming = deque(reqs)
        free = list(range(len(self.streams)))
        inflight = {}  # slot -> (requests, batch step, end event, bytes)
        busy = set()
        used = peak = 0
        statuses = []
        t0 = time.perf_counter()
        while upcoming or waiting or inflight:
            now = time.perf_counter() - t0
            # completions
            for slot in list(inflight):
                batch, bs, ev, nb = inflight[slot]
                if ev.query():
                    done = time.perf_counter() - t0
                    statuses.append(int(self.status_host[slot]))
                    for j, r in enumerate(batch):
                        r.done = done
                        if keep_results and r.kind == "render":
                            r.image = bs.images()[j].clone()  # the slot's buffers are reused
                    for r in batch:
                        busy.discard(r.scene)
                    used -= nb
                    free.append(slot)
                    del inflight[slot]
            while upcoming and upcoming[0].arrival <= now:
                waiting.append(upcoming.popleft())
            # admissions, in arrival order: a request starts with the later ones
            # of its kind and image size that may join it; a scene whose earliest
            # waiting request cannot start admits none of its later ones
            started = False
            blocked = set()
            taken = set()
            for r in list(waiting):
                if not free:
                    break
                if r.rid in taken:
                    continue
                sc = self.scenes[r.scene]
                if self.batch_bytes([r]) > self.budget:  # can never fit: rejected at once
                    r.rejected = True
                    r.start = r.done = time.perf_counter() - t0
                    waiting.remove(r)
                    continue
                if r.scene in busy or r.scene in blocked or used + self.batch_bytes([r]) > self.budget:
                    blocked.add(r.scene)
                    continue
                batch = [r]
                later_blocked = set(blocked)
                after = False
                for q in waiting:
                    if len(batch) >= self.max_batch:
                        break
                    if q is r:
                        after = True
                        continue
                    if not after or q.rid in taken:
                        continue
                    qs = self.scenes[q.scene]
                    near_size = (self.max_pad_ratio is None
                                 or max(qs.n, sc.n) <= self.max_pad_ratio * max(1, min(qs.n, sc.n)))
                    joins = (q.kind == r.kind and (qs.W, qs.H) == (sc.W, sc.H) and near_size and q.scene not in busy
                             and q.scene not in later_blocked
                             and (q.kind == "render" or all(b.scene != q.scene for b in batch))
                             and used + self.batch_bytes(batch + [q]) <= self.budget)
                    if joins:
                        batch.append(q)
                    else:
                        later_blocked.add(q.scene)  # none of its later requests may overtake q
                nb = self.batch_bytes(batch)
                slot = free.pop()
                st = self.streams[slot]
                start = time.perf_counter() - t0
                for q in batch:
                    q.nbytes, q.start, q.batch = nb, start, len(batch)
                bs = self.start(batch, st, self.pools[slot])
                with torch.cuda.stream(st):
                    self.status_host[slot: slot + 1].copy_(bs.status, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(st)
                inflight[slot] = (batch, bs, ev, nb)
                for q in batch:
                    busy.add(q.scene)
                used += nb
                peak = max(peak, used)
                for q in batch:
                    waiting.remove(q)
                    taken.add(q.rid)
                started = True
            if not started and not inflight and waiting and not free:
                raise RuntimeError("no slot can ever be freed")  # unreachable: inflight empty means free slots
            if not started:
                time.sleep(2e-5)
        res = ServeResult(reqs, time.perf_counter() - t0, "served", len(self.streams), min(self.budget, 1 << 62),
                          peak, statuses)
        return res


def make_scenes(n_scenes: int = 16, *, device: str = "cuda", budget_bytes: int | None = None, seed: int = 5000,
                n_views: int = 8, n_max: int = 2_000_000, rank: int = 0, world: int = 1) -> list[Scene]:
    """The served workload's resident scenes of `rank` (see scene_shard); scenes
    are admitted in order while their resident bytes fit `budget_bytes` (the
    rest are not loaded)."""
    scenes = []
    used = 0
    mine = set(scene_shard(n_scenes, rank, world))
    for sid, (n, W, H) in enumerate(synth.served_scene_specs(n_scenes, seed=seed, n_max=n_max)):
        if sid not in mine:
            continue
        sc = Scene(sid, n, W, H, n_views=n_views, device=device)
        if budget_bytes is not None and used + sc.resident_bytes > budget_bytes:
            del sc
            break
        used += sc.resident_bytes
        scenes.append(sc)
    return scenes
