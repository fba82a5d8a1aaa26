"""Pins of the oracle's D-SSIM objective (Eq. pixel_loss with D-SSIM = 1 - SSIM,
Sec. 3.2 least-squares form with m = 6 H W per view).

* The SSIM map equals one computed here with scipy.ndimage filters (same
  11 x 11, sigma 1.5 window, zero outside the image); SSIM(x, x) = 1; symmetry.
* The adjoint (VJP) and the directional derivative (JVP) of the map equal
  central differences of the scipy map.
* The objective's gradient equals central differences of the objective evaluated
  from the oracle's render and the scipy map.
* The Hutchinson diagonal equals z . (G z) with G = (1/m) J_F^T J_F built from the
  oracle's image Jacobian and the scipy map's Jacobian (by differences).
"""
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle as O
from paper_2602_00395_gb300 import synth as S

C1, C2 = 1e-4, 9e-4


def _window():
    g = np.exp(-np.arange(-5, 6) ** 2 / (2 * 1.5 ** 2))
    g /= g.sum()
    return np.outer(g, g)


def scipy_ssim(x, y):
    w = _window()
    f = lambda a: ndimage.correlate(a, w, mode="constant", cval=0.0)
    mx, my = f(x), f(y)
    sx2, sy2, sxy = f(x * x) - mx * mx, f(y * y) - my * my, f(x * y) - mx * my
    return (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sx2 + sy2 + C2))


def _images(seed=0, H=14, W=17):
    rng = np.random.default_rng(seed)
    x = ndimage.gaussian_filter(rng.uniform(size=(H, W)), 1.0)
    y = np.clip(x + 0.1 * rng.normal(size=(H, W)), 0, 1)
    return x, y


def test_ssim_map_matches_scipy_and_its_invariants():
    x, y = _images()
    S_o = O.ssim(x, y)[0]
    np.testing.assert_allclose(S_o, scipy_ssim(x, y), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(O.ssim(x, x)[0], 1.0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(O.ssim(y, x)[0], S_o, rtol=1e-12, atol=1e-14)


def test_ssim_adjoint_and_directional_derivative_match_differences():
    x, y = _images(1)
    rng = np.random.default_rng(2)
    a = rng.normal(size=x.shape)
    d = rng.normal(size=x.shape)
    vjp = O.ssim_vjp(x, y, a)
    h = 1e-6
    for q in rng.choice(x.size, 25, replace=False):
        e = np.zeros(x.size)
        e[q] = h
        e = e.reshape(x.shape)
        fd = ((a * scipy_ssim(x + e, y)).sum() - (a * scipy_ssim(x - e, y)).sum()) / (2 * h)
        assert abs(fd - vjp.flat[q]) <= 1e-6 * max(1.0, abs(fd))
    jvp = O.ssim_jvp(x, y, d)
    fd = (scipy_ssim(x + h * d, y) - scipy_ssim(x - h * d, y)) / (2 * h)
    np.testing.assert_allclose(jvp, fd, rtol=1e-5, atol=1e-7)


def _tiny(deg=1, n=12, W=16, H=16):
    sc = S.make_scene(n, deg, seed=23, extent=0.5, log_scale_shift=math.log(4.0))
    cam = S.Camera(S.look_at((3.0, 0.4, 0.3)), **S.pinhole(W, H))
    return O.params64(sc), cam


def _objective(P, deg, cam, tg, lam):
    img = O.render(P, deg, [cam], with_margin=False)["image"][0]
    m = 6 * img.shape[1] * img.shape[2]
    s = sum((1 - scipy_ssim(img[c], tg[0, c])).sum() for c in range(3))
    return ((1 - lam) * np.abs(img - tg[0]).sum() + lam * s) / (2 * m)


def test_dssim_gradient_matches_finite_differences():
    deg, lam = 1, 0.2
    P, cam = _tiny(deg)
    tg = S.smooth_target(1, 16, 16, seed=4).astype(np.float64)
    out = O.backward(P, deg, [cam], tg, loss_kind=2, lam=lam)
    assert abs(out["loss"] - _objective(P, deg, cam, tg, lam)) <= 1e-12 * abs(out["loss"])
    g = out["grad"]
    sig0 = O.signature(P, deg, [cam])
    rng = np.random.default_rng(5)
    checked = 0
    for c in rng.choice(P.size, 80, replace=False):
        r, i = divmod(c, P.shape[1])
        h = 1e-5 * max(1.0, abs(P[r, i]))
        Pp, Pm = P.copy(), P.copy()
        Pp[r, i] += h
        Pm[r, i] -= h
        if not (np.array_equal(O.signature(Pp, deg, [cam]), sig0) and np.array_equal(O.signature(Pm, deg, [cam]), sig0)):
            continue
        img_p = O.render(Pp, deg, [cam], with_margin=False)["image"]
        img_m = O.render(Pm, deg, [cam], with_margin=False)["image"]
        if not np.array_equal(np.sign(img_p - tg), np.sign(img_m - tg)):
            continue  # an L1 residual changes sign inside the step
        fd = (_objective(Pp, deg, cam, tg, lam) - _objective(Pm, deg, cam, tg, lam)) / (2 * h)
        assert abs(fd - g[r, i]) <= 1e-6 * np.abs(g).max() + 1e-6 * abs(g[r, i]), (r, i, fd, g[r, i])
        checked += 1
    assert checked >= 50


def test_dssim_hutchinson_diagonal_equals_exact_gauss_newton_products():
    deg, lam, nu, t, seed, floor = 0, 0.2, 2, 3, 11, 1e-3
    P, cam = _tiny(deg, n=8, W=12, H=12)
    tg = S.smooth_target(1, 12, 12, seed=6).astype(np.float64)
    out = O.backward(P, deg, [cam], tg, loss_kind=2, lam=lam, nu=nu, seed=seed, t=t, gn_floor=floor)
    img = O.render(P, deg, [cam], with_margin=False)["image"][0]
    J = O.jacobian(P, deg, [cam])  # (3 H W) x (rows n), image Jacobian
    H, W = 12, 12
    m = 6 * H * W
    # SSIM Jacobian of each channel by central differences of the scipy map
    JS = np.zeros((3 * H * W, 3 * H * W))
    h = 1e-6
    for c in range(3):
        for q in range(H * W):
            e = np.zeros(H * W)
            e[q] = h
            e = e.reshape(H, W)
            col = (scipy_ssim(img[c] + e, tg[0, c]) - scipy_ssim(img[c] - e, tg[0, c])) / (2 * h)
            JS[c * H * W:(c + 1) * H * W, c * H * W + q] = col.ravel()
    r = (img - tg[0]).ravel()
    Sv = np.concatenate([scipy_ssim(img[c], tg[0, c]).ravel() for c in range(3)])
    w_l1 = (1 - lam) / (4 * np.maximum(np.abs(r), floor)) / m
    w_s = lam / (4 * np.maximum(1 - Sv, floor)) / m
    G = J.T @ (w_l1[:, None] * J) + (JS @ J).T @ (w_s[:, None] * (JS @ J))
    rows, n = P.shape
    hz = np.zeros(rows * n)
    for k in range(nu):
        z = O.probe_matrix(seed, t, k, rows, n).ravel()
        hz += z * (G @ z) / nu
    np.testing.assert_allclose(out["hz"].ravel(), hz, rtol=1e-6, atol=1e-9 * np.abs(hz).max())
