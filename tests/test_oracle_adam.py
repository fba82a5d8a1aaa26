"""Pins of the oracle's ADAM-TR update (the trust-region clip of Sec. 4.2 applied
to Adam, the paper's ablation in Sec. 5).

* With radii far above the Adam steps (eps so large that no parameter is
  clipped), three steps equal torch.optim.Adam's, parameter groups and moments
  included.
* With radii that bite, every change is the Adam step clipped to +-eta of x_t.
"""
import numpy as np
import pytest

import oracle as O
from paper_2602_00395_gb300 import synth as S

torch = pytest.importorskip("torch")

GROUPS = [slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 14), slice(14, None)]


def _scene(deg=3, n=40, seed=3):
    return O.params64(S.make_scene(n, deg, seed=seed))


def test_unclipped_steps_equal_torch_adam():
    deg = 3
    P = _scene(deg)
    adam = O.adam_config()
    rng = np.random.default_rng(0)
    grads = [rng.normal(size=P.shape) * 10.0 ** rng.uniform(-4, -1) for _ in range(3)]
    x, m, v = P.copy(), np.zeros_like(P), np.zeros_like(P)
    for t, g in enumerate(grads, start=1):
        x, m, v, eta = O.adam_tr_update(x, m, v, g, deg, t=t, eps=1e6, adam=adam)
        assert np.all(eta >= 1e2)  # no clip can bite
    params = [torch.tensor(P[sl], dtype=torch.float64, requires_grad=True) for sl in GROUPS]
    opt = torch.optim.Adam([{"params": [p], "lr": float(adam[3 + q])} for q, p in enumerate(params)],
                           betas=(float(adam[0]), float(adam[1])), eps=float(adam[2]))
    for g in grads:
        for p, sl in zip(params, GROUPS):
            p.grad = torch.tensor(g[sl], dtype=torch.float64)
        opt.step()
    ref = np.concatenate([p.detach().numpy() for p in params])
    np.testing.assert_allclose(x, ref, rtol=1e-12, atol=1e-15)
    m_ref = np.concatenate([opt.state[p]["exp_avg"].numpy() for p in params])
    v_ref = np.concatenate([opt.state[p]["exp_avg_sq"].numpy() for p in params])
    np.testing.assert_allclose(m, m_ref, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(v, v_ref, rtol=1e-12, atol=1e-300)


def test_clipped_steps_are_adam_steps_clipped_to_the_radius():
    deg = 1
    P = _scene(deg, n=60, seed=8)
    rng = np.random.default_rng(1)
    g = rng.normal(size=P.shape) * 1e-2
    t, eps = 1, 1e-7
    x1, m1, v1, eta = O.adam_tr_update(P, np.zeros_like(P), np.zeros_like(P), g, deg, t=t, eps=eps)
    eta_ref = O.shd_radius(P, deg, eps, O.tr_config())
    np.testing.assert_array_equal(eta, eta_ref)
    adam = O.adam_config()
    group = [0] * 3 + [1] * 3 + [2] * 4 + [3] + [4] * 3 + [5] * (P.shape[0] - 14)
    lr = np.array([adam[3 + q] for q in group])
    step = -lr[:, None] * (m1 / (1 - adam[0])) / (np.sqrt(v1 / (1 - adam[1])) + adam[2])
    dx = x1 - P
    clipped = np.abs(step) > eta
    assert clipped.any() and (~clipped).any()
    # dx = x_{t+1} - x_t carries the rounding of x (a few ulps of |x|)
    ulp = 4e-16 * np.abs(P)
    assert np.all(np.abs(np.abs(dx[clipped]) - eta[clipped]) <= 1e-12 * eta[clipped] + ulp[clipped])
    assert np.all(np.abs(dx[~clipped] - step[~clipped]) <= 1e-12 * np.abs(step[~clipped]) + ulp[~clipped])
