"""A training step captured once as a CUDA graph and replayed gives the eager
steps' results: the step index is read on the device (gs_probe.t_device,
gs_tr_update_dev) and advanced inside the graph (gs_step_advance), with
eps_t of the exponential schedule of Sec. 5 evaluated on the device.

The reverse pass adds with float atomics, so two runs agree to rounding, not
bit for bit; the tolerance covers that.
"""
import math

import numpy as np
import pytest

from paper_2602_00395_gb300 import synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _engine(l):
    from paper_2602_00395_gb300.engine import TRConfig, TRStep
    sc = S.make_scene(1500, 1, seed=31, extent=1.0, log_scale_shift=math.log(2.0))
    cams = S.camera_ring(2, 160, 120, 1.0, seed=4, ring_factor=4.0)
    e = TRStep(sc.n, 1, 2, 160, 120, nu=2, cfg=TRConfig(l=l))
    e.set_cameras(cams)
    e.set_params(sc.params)
    e.set_target(S.smooth_target(2, 120, 160, seed=8))
    e.ensure_capacity()
    return e


def _state(e):
    return [b.clone() for b in (e.x, e.g_ema, e.d_ema)]


def _close(a, b):
    for u, v in zip(a, b):
        scale = float(v.abs().max()) + 1e-30
        assert float((u - v).abs().max()) <= 1e-4 * scale


@pytest.mark.parametrize("l", [1, 2])
def test_graph_replay_matches_eager_steps(l):
    from paper_2602_00395_gb300 import gs3dtr as G
    from paper_2602_00395_gb300.engine import eps_schedule
    total, K = 40, 4
    e = _engine(l)
    x0 = _state(e)
    # eager reference
    for t in range(1, K + 1):
        e.step(t, eps_schedule(t, total))
    torch.cuda.synchronize()
    assert e.read_status() == 0
    ref = _state(e)
    # the same steps replayed from a graph per step kind
    for b, v in zip((e.x, e.g_ema, e.d_ema), x0):
        b.copy_(v)
    sched = G.gs_eps_schedule(1e-6, 1e-8, total)
    graphs = {hvp: e.capture_step(hvp, sched) for hvp in ({True} if l == 1 else {True, False})}
    e.t_dev.zero_()
    for t in range(1, K + 1):
        graphs[(t - 1) % l == 0].replay()
    torch.cuda.synchronize()
    assert int(e.t_dev.item()) == K
    assert e.read_status() == 0
    _close(_state(e), ref)


def test_device_schedule_matches_host_schedule():
    """eps_t on the device equals the host schedule: one update from a zero state
    moves each parameter by exactly its radius when the Newton step is clipped."""
    from paper_2602_00395_gb300 import gs3dtr as G
    from paper_2602_00395_gb300.engine import eps_schedule
    e = _engine(1)
    total = 17
    for t in (1, 5, 17):
        eta_h = torch.zeros_like(e.x)
        eta_d = torch.zeros_like(e.x)
        x_saved = e.x.clone()
        e.grad.fill_(1.0)
        e.hz.fill_(1e-30)
        e.g_ema.zero_()
        e.d_ema.zero_()
        e.update(t, eps_schedule(t, total), True, eta_h)
        e.x.copy_(x_saved)
        e.g_ema.zero_()
        e.d_ema.zero_()
        e.t_dev.fill_(t)
        G.gs_tr_update_dev(e.P(e.x), e.P(e.g_ema), e.P(e.d_ema), e.P(e.grad), e.P(e.hz), e.cfg.struct(), e.t_dev,
                           G.gs_eps_schedule(1e-6, 1e-8, total), e.P(eta_d), e.status)
        e.x.copy_(x_saved)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(eta_d[:, : e.n].cpu().numpy(), eta_h[:, : e.n].cpu().numpy())


def test_tile_autotuner_times_every_shape_and_leaves_the_step_unchanged():
    """Every tile shape with the default batch, then the batches for the fastest
    shape; the pick is the fastest of those."""
    from paper_2602_00395_gb300.engine import autotune_tile
    e = _engine(1)
    before = _state(e)
    best, times = autotune_tile(e, candidates=((16, 16), (32, 8), (16, 8)), batches=(0, 32, 256), steps=2)
    shapes = [(16, 16), (32, 8), (16, 8)]
    fastest = min(shapes, key=lambda s: times[(*s, 0)])
    assert set(times) == {(*s, 0) for s in shapes} | {(*fastest, 32), (*fastest, 256)}
    assert all(v > 0 for v in times.values())
    assert (best[0], best[1]) == fastest and times[best] == min(v for k, v in times.items() if k[:2] == fastest)
    for u, v in zip(_state(e), before):
        assert torch.equal(u, v)
