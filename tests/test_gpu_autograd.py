"""torch.autograd over the C-ABI rasteriser: the gradient of a scalar function of
the rendered images equals the oracle's J^T w and finite differences of the CUDA
forward on a 2k-Gaussian scene, and the Gauss-Newton diagonal estimate equals the
oracle's Hutchinson diagonal under the same probes.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_00395_gb300 import synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GROUPS = {"mean": slice(0, 3), "log_scale": slice(3, 6), "quat": slice(6, 10), "opacity": slice(10, 11),
          "sh": slice(11, None)}


def _setup(n=2000, deg=1, nu=2):
    from paper_2602_00395_gb300.engine import TRStep
    sc = S.make_scene(n, deg, seed=55, extent=1.0, log_scale_shift=math.log(1.5))
    cams = S.camera_ring(2, 96, 72, 1.0, seed=9, ring_factor=3.0)
    e = TRStep(n, deg, 2, 96, 72, nu=nu)
    e.set_cameras(cams)
    e.set_params(sc.params)
    e.ensure_capacity()
    return sc, cams, e


def _close(gpu, ref, tol, what):
    for name, sl in GROUPS.items():
        scale = np.abs(ref[sl]).max()
        assert np.abs(gpu[sl] - ref[sl]).max() <= tol * scale, (what, name)


def test_autograd_gradient_matches_oracle():
    from paper_2602_00395_gb300.autograd import render
    sc, cams, e = _setup()
    w = torch.from_numpy(np.random.default_rng(1).normal(size=(2, 3, 72, 96)).astype(np.float32)).cuda()
    params = e.x.clone().requires_grad_(True)
    img = render(params, e)
    (img * w).sum().backward()
    torch.cuda.synchronize()
    assert e.read_status() == 0
    # the oracle's L2 objective with target = image - m w has gradient J^T w
    P = O.params64(sc)
    ref_img = O.render(P, sc.sh_degree, cams, with_margin=False)["image"]
    m = ref_img.size
    ref = O.backward(P, sc.sh_degree, cams, ref_img - m * w.cpu().numpy().astype(np.float64), loss_kind=1)
    _close(params.grad[:, : sc.n].cpu().numpy(), ref["grad"], 1e-4, "grad")


def test_autograd_gradient_matches_finite_differences_of_the_cuda_forward():
    """Central differences of sum(w * render(x)) in FP32 on the SH colour rows of
    sampled Gaussians of the 2k-Gaussian scene.  The image is linear in these rows
    (up to the clamp of negative colour), so the differences are exact up to
    rounding; the geometric rows move pixels across the alpha >= 1/255 threshold,
    which FP32 differences cannot step over (the oracle test covers them)."""
    from paper_2602_00395_gb300.autograd import render
    sc, cams, e = _setup()
    w = torch.from_numpy(np.random.default_rng(2).uniform(0.5, 1.5, size=(2, 3, 72, 96)).astype(np.float32)).cuda()
    params = e.x.clone().requires_grad_(True)
    (render(params, e) * w).sum().backward()
    g = params.grad.clone()
    f = lambda p: float((render(p, e) * w).double().sum())
    rng = np.random.default_rng(3)
    cols = rng.choice(sc.n, 12, replace=False)
    agree = total = 0
    gscale = float(g[:, : sc.n].abs().max())
    for i in cols:
        for r, h in [(r, 1e-2) for r in range(11, 11 + 3 * (sc.sh_degree + 1) ** 2)]:
            pp, pm = params.detach().clone(), params.detach().clone()
            pp[r, i] += h
            pm[r, i] -= h
            fd = (f(pp) - f(pm)) / (2 * h)
            total += 1
            agree += abs(fd - float(g[r, i])) <= 2e-2 * abs(float(g[r, i])) + 1e-3 * gscale
    # a perturbation may flip a discrete decision of the blend (a threshold, a tile)
    assert agree >= 0.9 * total, (agree, total)


def test_gauss_newton_diagonal_matches_oracle():
    """Uniform weights 1/m: the Hutchinson diagonal of J^T J / m, the oracle's L2
    curvature at a zero residual."""
    from paper_2602_00395_gb300.autograd import gn_diagonal
    sc, cams, e = _setup()
    t = 3
    m = 2 * 3 * 72 * 96
    params = e.x.clone()
    hz = gn_diagonal(params, torch.full((2, 3, 72, 96), 1.0 / m, device="cuda"), e, t)
    torch.cuda.synchronize()
    assert e.read_status() == 0 and not hz.requires_grad
    P = O.params64(sc)
    ref_img = O.render(P, sc.sh_degree, cams, with_margin=False)["image"]
    ref = O.backward(P, sc.sh_degree, cams, ref_img, loss_kind=1, seed=42, t=t, nu=2)
    _close(hz[:, : sc.n].cpu().numpy(), ref["hz"], 1e-3, "hz")


def test_gauss_newton_diagonal_with_l1_weights_matches_oracle():
    """The weights of the L1 objective of Sec. 3.2, 1/(4 max(|r|, delta))/m, formed
    in PyTorch from the differentiable render; the library weights and pulls
    back J z_k (GS_LOSS_WEIGHTED).  Compared with the oracle's L1 Hutchinson
    diagonal under the same probes: 1e-3 of each group's largest entry, each
    entry within 1e-3 of the mass of its sum, plus the oracle's bound on how far
    an entry moves when the residuals move by their FP32 rounding."""
    from paper_2602_00395_gb300.autograd import gn_diagonal, render
    sc, cams, e = _setup()
    t = 5
    m = 2 * 3 * 72 * 96
    target = S.smooth_target(2, 72, 96, seed=2011)
    tg = torch.from_numpy(target).cuda()
    params = e.x.clone().requires_grad_(True)
    img = render(params, e)
    w = 1.0 / (4.0 * torch.clamp((img.detach() - tg).abs(), min=1e-3)) / m
    hz = gn_diagonal(params, w, e, t)
    torch.cuda.synchronize()
    assert e.read_status() == 0
    P = O.params64(sc)
    ref = O.backward(P, sc.sh_degree, cams, target.astype(np.float64), loss_kind=0, seed=42, t=t, nu=2, masses=True)
    h = hz[:, : sc.n].cpu().numpy()
    for name, sl in GROUPS.items():
        err = np.abs(h[sl] - ref["hz"][sl])
        scale = np.abs(ref["hz"][sl]).max()
        assert np.all(err <= 1e-3 * scale + ref["hz_sens"][sl]), name
        assert np.all(err <= 1e-3 * ref["hz_mass"][sl] + ref["hz_sens"][sl]), name
