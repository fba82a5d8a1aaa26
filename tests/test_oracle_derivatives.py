"""Pins of the oracle's derivatives (Sec. 4.1) on tiny scenes (<= 50 Gaussians, 32x32).

* reverse-mode gradient vs central finite differences of the objective
  (components whose +-h perturbation changes a discrete decision are skipped and
  counted);
* forward-mode image Jacobian vs finite differences of the image, and the
  gradient vs J^T w, the GN product vs J^T diag(w) J z from the same J;
* Hutchinson's estimator: mean over many probes converges to diag(G) within
  the variance bound computed from the exact G;
* for the L2 objective at a zero-residual point the Gauss-Newton diagonal equals
  the finite-difference Hessian diagonal.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_00395_gb300 import synth as S


def tiny(deg, n=30, seed=21, W=32, H=32):
    sc = S.make_scene(n, deg, seed=seed, extent=0.5, log_scale_shift=math.log(4.0))
    cam = S.Camera(S.look_at((3.0, 0.4, 0.3)), **S.pinhole(W, H))
    return O.params64(sc), cam


def objective(P, deg, cam, tg, loss_kind):
    img = O.render(P, deg, [cam], with_margin=False)["image"]
    r = img - tg
    m = r.size
    return (np.abs(r).sum() if loss_kind == 0 else (r * r).sum()) / (2 * m), np.sign(r)


@pytest.mark.parametrize("deg,loss_kind", [(0, 0), (3, 0), (1, 1)])
def test_gradient_matches_finite_differences(deg, loss_kind):
    P, cam = tiny(deg)
    tg = S.smooth_target(1, 32, 32, seed=5).astype(np.float64)
    out = O.backward(P, deg, [cam], tg, loss_kind=loss_kind)
    g = out["grad"]
    sig0 = O.signature(P, deg, [cam])
    rows, n = P.shape
    checked = skipped = 0
    group_max = np.abs(g).max(axis=1, keepdims=True)
    for r in range(rows):
        for i in range(n):
            h = 1e-5 * max(1.0, abs(P[r, i]))
            Pp, Pm = P.copy(), P.copy()
            Pp[r, i] += h
            Pm[r, i] -= h
            fp, sp = objective(Pp, deg, cam, tg, loss_kind)
            fm, sm = objective(Pm, deg, cam, tg, loss_kind)
            same = (np.array_equal(O.signature(Pp, deg, [cam]), sig0) and
                    np.array_equal(O.signature(Pm, deg, [cam]), sig0) and
                    (loss_kind == 1 or np.array_equal(sp, sm)))
            if not same:
                skipped += 1
                continue
            fd = (fp - fm) / (2 * h)
            tol = 1e-6 * max(group_max[r, 0], 1e-30) + 1e-6 * abs(g[r, i])
            assert abs(fd - g[r, i]) <= tol, (r, i, fd, g[r, i])
            checked += 1
    assert checked > 0.9 * rows * n, (checked, skipped)
    assert np.count_nonzero(g) > 0.5 * rows * n


def _fd_jacobian_columns(P, deg, cam, cols, h=1e-6):
    rows, n = P.shape
    out = []
    for c in cols:
        r, i = divmod(c, n)
        Pp, Pm = P.copy(), P.copy()
        Pp[r, i] += h
        Pm[r, i] -= h
        ip = O.render(Pp, deg, [cam], with_margin=False)["image"].ravel()
        im = O.render(Pm, deg, [cam], with_margin=False)["image"].ravel()
        same = (np.array_equal(O.signature(Pp, deg, [cam]), O.signature(P, deg, [cam])) and
                np.array_equal(O.signature(Pm, deg, [cam]), O.signature(P, deg, [cam])))
        out.append(((ip - im) / (2 * h), same))
    return out


def test_forward_mode_jacobian_matches_finite_differences():
    P, cam = tiny(3, n=12, W=24, H=24)
    J = O.jacobian(P, 3, [cam])
    rows, n = P.shape
    rng = np.random.default_rng(0)
    cols = rng.choice(rows * n, size=120, replace=False)
    ok = 0
    for c, (fd, same) in zip(cols, _fd_jacobian_columns(P, 3, cam, cols)):
        if not same:
            continue
        scale = max(np.abs(J[:, c]).max(), 1e-12)
        assert np.abs(fd - J[:, c]).max() <= 1e-6 * scale + 1e-9, c
        ok += 1
    assert ok > 100


@pytest.mark.parametrize("loss_kind", [0, 1])
def test_gradient_and_gn_product_agree_with_exact_jacobian(loss_kind):
    deg, nu = 1, 2
    P, cam = tiny(deg, n=15, W=24, H=24)
    tg = S.noise_target(1, 24, 24, seed=3).astype(np.float64)
    J = O.jacobian(P, deg, [cam])
    out = O.backward(P, deg, [cam], tg, loss_kind=loss_kind, gn_floor=1e-3, seed=77, t=5, nu=nu,
                     want_tangents=True)
    img = O.render(P, deg, [cam], with_margin=False)["image"].ravel()
    r = img - tg.ravel()
    m = r.size
    rows, n = P.shape
    if loss_kind == 0:
        w = np.sign(r) / (2 * m)
        lam = 1.0 / (4 * np.maximum(np.abs(r), 1e-3)) / m
    else:
        w = r / m
        lam = np.full_like(r, 1.0 / m)
    g = (J.T @ w).reshape(rows, n)
    np.testing.assert_allclose(out["grad"], g, atol=1e-12 * np.abs(g).max() + 1e-15)
    hz = np.zeros(rows * n)
    for k in range(nu):
        z = O.probe_matrix(77, 5, k, rows, n).ravel()
        np.testing.assert_allclose(out["image_tangent"][k].ravel(), J @ z, atol=1e-10)
        hz += z * (J.T @ (lam * (J @ z))) / nu
    np.testing.assert_allclose(out["hz"], hz.reshape(rows, n), atol=1e-10 * np.abs(hz).max())


def test_hutchinson_mean_converges_to_gn_diagonal():
    """E[z . G z] = diag(G); over K probes each entry lies within 5 sigma of it."""
    P, cam = tiny(0, n=10, W=20, H=20)
    J = O.jacobian(P, 0, [cam])
    G = J.T @ J / J.shape[0]
    K = 10000
    rng = np.random.default_rng(123)
    Z = rng.choice([-1.0, 1.0], size=(K, G.shape[0]))
    est = (Z * (Z @ G.T)).mean(0)
    off = G - np.diag(np.diag(G))
    sigma = np.sqrt((off ** 2).sum(1) / K)
    assert np.all(np.abs(est - np.diag(G)) <= 5 * sigma + 1e-15)


def test_gn_diagonal_is_hessian_diagonal_at_zero_residual():
    deg = 0
    P, cam = tiny(deg, n=12, W=24, H=24)
    tg = O.render(P, deg, [cam], with_margin=False)["image"]
    J = O.jacobian(P, deg, [cam])
    m = J.shape[0]
    d_gn = (J ** 2).sum(0) / m
    rows, n = P.shape
    sig0 = O.signature(P, deg, [cam])
    rng = np.random.default_rng(4)
    checked = 0
    for c in rng.choice(rows * n, size=60, replace=False):
        r, i = divmod(c, n)
        h = 1e-4 * max(1.0, abs(P[r, i]))
        Pp, Pm = P.copy(), P.copy()
        Pp[r, i] += h
        Pm[r, i] -= h
        if not (np.array_equal(O.signature(Pp, deg, [cam]), sig0) and np.array_equal(O.signature(Pm, deg, [cam]), sig0)):
            continue
        gp = O.backward(Pp, deg, [cam], tg, loss_kind=1)["grad"][r, i]
        gm = O.backward(Pm, deg, [cam], tg, loss_kind=1)["grad"][r, i]
        hess = (gp - gm) / (2 * h)
        assert abs(hess - d_gn[c]) <= 1e-5 * max(d_gn.max(), 1e-30) + 1e-5 * abs(d_gn[c]), (c, hess, d_gn[c])
        checked += 1
    assert checked > 40


def test_hvp_stream_uses_regenerated_probes():
    """The probe entries used by the oracle's HVP are the published-hash Rademacher values."""
    deg = 0
    P, cam = tiny(deg, n=8, W=16, H=16)
    tg = S.noise_target(1, 16, 16, seed=9).astype(np.float64)
    out = O.backward(P, deg, [cam], tg, seed=5, t=2, nu=1, want_tangents=True)
    rows, n = P.shape
    z = O.probe_matrix(5, 2, 0, rows, n)
    np.testing.assert_allclose(out["image_tangent"][0], O.jvp(P, deg, [cam], z), atol=1e-13)


def test_sampled_entry_points_reproduce_the_full_ones():
    """The sampled pixel and sampled-Gaussian paths (used at full workload size)
    agree with the full-frame oracle functions."""
    deg, nu = 1, 2
    sc = S.make_scene(200, deg, seed=44, extent=0.7, log_scale_shift=math.log(2.0))
    cams = S.camera_ring(2, 48, 40, 0.7, seed=5, ring_factor=5.0)
    tg = S.noise_target(2, 40, 48, seed=6).astype(np.float64)
    P = O.params64(sc)
    full = O.render(P, deg, cams)
    bw = O.backward(P, deg, cams, tg, seed=9, t=3, nu=nu, want_tangents=True)
    rng = np.random.default_rng(0)
    xs, ys = rng.integers(0, 48, 60), rng.integers(0, 40, 60)
    for v in range(2):
        px = O.render_pixels(P, deg, cams[v], xs, ys, seed=9, t=3, nu=nu)
        np.testing.assert_allclose(px["rgb"], full["image"][v][:, ys, xs].T, atol=1e-15)
        np.testing.assert_allclose(px["final_T"], full["final_T"][v][ys, xs], atol=1e-15)
        np.testing.assert_array_equal(px["n_contrib"], full["n_contrib"][v][ys, xs])
        np.testing.assert_allclose(px["margin"], full["margin"][v][ys, xs])
        for k in range(nu):
            np.testing.assert_allclose(px["jz"][:, k, :], bw["image_tangent"][k, v][:, ys, xs].T, atol=1e-14)
    smp = rng.choice(sc.n, 25, replace=False)
    out = O.backward_sampled(P, deg, cams, tg, smp, seed=9, t=3, nu=nu)
    np.testing.assert_allclose(out["grad"], bw["grad"][:, smp].T, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(out["hz"], bw["hz"][:, smp].T, rtol=1e-10, atol=1e-14)
