"""Single-Gaussian fit (Fig. 3): a Gaussian started from a small perturbation of a
ground-truth Gaussian is fitted to the ground truth's renders from three views,
by the trust-region method (Algorithm 1, Hutchinson curvature with two probes)
and by Adam (ADAM-TR with radii too large to clip).  Both recover the ground
truth; the trust-region path deforms the Gaussian much less per step.

Deformation is the squared Hellinger distance between consecutive Gaussians
(opacity as mass), evaluated by the oracle's closed form; the targets are the
oracle's renders of the ground truth.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_00395_gb300 import synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _gt():
    p = np.zeros((14, 1))
    p[3:6, 0] = (-1.6, -2.0, -1.8)
    q = np.array([0.2, -0.1, 0.3, 0.9])
    p[6:10, 0] = q / np.linalg.norm(q)
    p[10, 0] = 1.0
    p[11:14, 0] = (np.array([0.8, 0.4, 0.2]) - 0.5) / 0.28209479177387814
    return p


def _perturbed(p):
    d = p.copy()
    d[0:3, 0] += (0.06, -0.05, 0.04)
    d[3:6, 0] += (0.25, -0.2, 0.15)
    d[6:10, 0] += (0.05, 0.04, -0.03, 0.0)
    d[10, 0] -= 0.6
    d[11:14, 0] += 0.3
    return d


def _gauss(p):
    s = np.exp(p[3:6, 0])
    R = O.quat_to_rotmat(p[6:10, 0] / np.linalg.norm(p[6:10, 0]))
    return p[0:3, 0], R @ np.diag(s * s) @ R.T, 1.0 / (1.0 + math.exp(-p[10, 0]))


def _h2(a, b):
    return O.hellinger(*_gauss(a), *_gauss(b))


def _fit(kind, steps=300):
    from paper_2602_00395_gb300 import gs3dtr as G
    from paper_2602_00395_gb300.engine import TRConfig, TRStep
    cams = S.camera_ring(3, 64, 64, 0.5, seed=3, ring_factor=6.0)
    gt = _gt()
    target = O.render(gt, 0, cams)["image"].astype(np.float32)
    e = TRStep(1, 0, 3, 64, 64, nu=2, cfg=TRConfig(l=1))
    e.set_cameras(cams)
    e.set_params(_perturbed(gt).astype(np.float32))
    e.set_target(target)
    e.ensure_capacity()
    adam = G.adam_struct(lr=(1e-2, 1e-2, 1e-2, 5e-2, 1e-2, 1e-2))
    traj, losses = [e.x[:, :1].cpu().numpy().astype(np.float64)], []
    for t in range(1, steps + 1):
        if kind == "tr":
            e.step(t, 1e-5)
        else:
            e.step_adam(t, 1e6, adam)  # radii far above every Adam step: plain Adam
        traj.append(e.x[:, :1].cpu().numpy().astype(np.float64))
        losses.append(float(e.loss_val.item()))
    assert e.read_status() == 0
    return gt, traj, losses


@pytest.fixture(scope="module")
def fits():
    return {k: _fit(k) for k in ("tr", "adam")}


@pytest.mark.parametrize("kind", ["tr", "adam"])
def test_both_recover_the_ground_truth(fits, kind):
    gt, traj, losses = fits[kind]
    assert losses[-1] <= 0.1 * losses[0]
    # the mean starts 0.06 off; where it lands within a few 1e-3 varies from run
    # to run with the order of the reverse pass's float atomics
    assert np.abs(traj[-1][0:3, 0] - gt[0:3, 0]).max() <= 5e-3
    assert _h2(traj[-1], gt) <= 0.1 * _h2(traj[0], gt)


def test_trust_region_deforms_much_less_per_step(fits):
    step_max = {k: max(_h2(a, b) for a, b in zip(tr, tr[1:])) for k, (_, tr, _) in fits.items()}
    assert step_max["tr"] <= 0.25 * step_max["adam"], step_max
