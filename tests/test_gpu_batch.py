"""Several requests in shared launches (gs_project_batch, gs_bin_sort and
gs_raster_fwd on the batch frame, gs_raster_bwd_batch, gs_tr_update_batch): each
request of a batch of scenes with uneven Gaussian counts gets what it gets
alone -- its image bit for bit, its gradient, Hutchinson diagonal and updated
trust-region state within FP32 rounding of the order of the reverse pass's
atomics -- and one batched request agrees with the oracle."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_00395_gb300 import synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

W, H, DEG = 97, 75, 1
GROUPS = {"mean": slice(0, 3), "log_scale": slice(3, 6), "quat": slice(6, 10), "opacity": slice(10, 11),
          "sh": slice(11, None)}


def _scenes():
    out = []
    for k, n in enumerate((2999, 1201, 333)):
        sc = S.make_scene(n, DEG, seed=1100 + k, kind="cube", extent=1.0, log_scale_shift=math.log(1.5))
        cam = S.camera_ring(8, W, H, 1.0, seed=7 + k, ring_factor=3.0)[k]
        tg = S.noise_target(1, H, W, seed=2100 + k)
        out.append((sc, cam, tg, 3 + 2 * k))  # each scene at its own step index
    return out


def _close(a, b, tol, what):
    for name, sl in GROUPS.items():
        scale = max(np.abs(b[sl]).max(), 1e-30)
        assert np.abs(a[sl] - b[sl]).max() <= tol * scale, (what, name)


@pytest.mark.parametrize("nu", [1, 2])
def test_batched_training_step_equals_each_request_alone(nu):
    from paper_2602_00395_gb300 import gs3dtr as G
    from paper_2602_00395_gb300.engine import BatchEntry, BatchStep, TRConfig, TRStep
    cfg = TRConfig(l=2)
    scenes = _scenes()
    alone = []
    for sc, cam, tg, t in scenes:
        e = TRStep(sc.n, DEG, 1, W, H, nu=nu, cfg=cfg)
        e.set_cameras([cam])
        e.set_params(sc.params)
        e.set_target(tg)
        e.ensure_capacity()
        e.step(t, 1e-5)
        torch.cuda.synchronize()
        assert e.read_status() == 0
        alone.append(dict(x=e.x.clone(), ge=e.g_ema.clone(), de=e.d_ema.clone(), grad=e.grad.clone(),
                          hz=e.hz.clone(), image=e.image.clone(), loss=float(e.loss_val.item()),
                          cap=e.capacity))
        del e
    entries = []
    for (sc, cam, tg, t) in scenes:
        x = torch.zeros(S.n_rows(DEG), sc.n_pad, device="cuda")
        x[:, : sc.params.shape[1]].copy_(torch.from_numpy(sc.params))
        entries.append(BatchEntry(x, torch.zeros_like(x), torch.zeros_like(x), sc.n,
                                  torch.from_numpy(G.camera_bytes([cam])).cuda(),
                                  torch.from_numpy(tg.reshape(-1)).cuda(), t, 1e-5))
    bs = BatchStep(entries, W, H, sh_degree=DEG, nu=nu, capacity=sum(a["cap"] for a in alone), cfg=cfg)
    bs.run()
    torch.cuda.synchronize()
    assert bs.read_status() == 0
    imgs = bs.images().cpu().numpy()
    for b, (a, ent) in enumerate(zip(alone, entries)):
        n = scenes[b][0].n
        assert np.array_equal(imgs[b].reshape(-1), a["image"].cpu().numpy())
        assert abs(float(bs.loss_val[b]) - a["loss"]) <= 1e-6 * a["loss"]
        _close(bs.grads[b][:, :n].cpu().numpy(), a["grad"][:, :n].cpu().numpy(), 1e-5, f"grad {b}")
        _close(bs.hzs[b][:, :n].cpu().numpy(), a["hz"][:, :n].cpu().numpy(), 1e-5, f"hz {b}")
        # the update: the same step within the rounding of the gradient
        for name, got, ref in (("x", ent.x, a["x"]), ("g_ema", ent.g_ema, a["ge"]), ("d_ema", ent.d_ema, a["de"])):
            d = (got - ref)[:, :n].abs().max().item()
            scale = max(ref[:, :n].abs().max().item(), 1e-30)
            assert d <= 1e-5 * scale, (b, name, d, scale)


def test_batched_request_matches_oracle():
    from paper_2602_00395_gb300 import gs3dtr as G
    from paper_2602_00395_gb300.engine import BatchEntry, BatchStep, TRConfig
    scenes = _scenes()
    entries = []
    for (sc, cam, tg, t) in scenes:
        x = torch.zeros(S.n_rows(DEG), sc.n_pad, device="cuda")
        x[:, : sc.params.shape[1]].copy_(torch.from_numpy(sc.params))
        entries.append(BatchEntry(x, torch.zeros_like(x), torch.zeros_like(x), sc.n,
                                  torch.from_numpy(G.camera_bytes([cam])).cuda(),
                                  torch.from_numpy(tg.reshape(-1)).cuda(), t, 1e-5))
    bs = BatchStep(entries, W, H, sh_degree=DEG, nu=2, capacity=1 << 20, cfg=TRConfig(l=1))
    bs.run()
    torch.cuda.synchronize()
    assert bs.read_status() == 0
    b = 1
    sc, cam, tg, t = scenes[b]
    ref = O.backward(O.params64(sc), DEG, [cam], tg.astype(np.float64), seed=42, t=t, nu=2, masses=True)
    g = bs.grads[b][:, : sc.n].cpu().numpy()
    h = bs.hzs[b][:, : sc.n].cpu().numpy()
    for name, sl in GROUPS.items():
        ga = ref["grad_allow"][sl]
        assert np.all(np.abs(g[sl] - ref["grad"][sl]) <= 1e-4 * np.abs(ref["grad"][sl]).max() + ga), name
        ha = ref["hz_sens"][sl] + ref["hz_allow"][sl]
        assert np.all(np.abs(h[sl] - ref["hz"][sl]) <= 1e-3 * np.abs(ref["hz"][sl]).max() + ha), name


def test_batched_render_equals_each_render_alone():
    from paper_2602_00395_gb300 import gs3dtr as G
    from paper_2602_00395_gb300.engine import BatchEntry, BatchStep, TRStep
    scenes = _scenes()
    entries, alone = [], []
    for (sc, cam, tg, t) in scenes:
        e = TRStep(sc.n, DEG, 1, W, H, nu=0)
        e.set_cameras([cam])
        e.set_params(sc.params)
        e.ensure_capacity()
        e.render()
        alone.append(e.image.clone())
        entries.append(BatchEntry(e.x.clone(), e.g_ema, e.d_ema, sc.n, e.cams.clone()))
    bs = BatchStep(entries, W, H, sh_degree=DEG, capacity=1 << 20, train=False)
    bs.run()
    torch.cuda.synchronize()
    assert bs.read_status() == 0
    for b, img in enumerate(alone):
        assert torch.equal(bs.images()[b].reshape(-1), img)
