"""Pins of the oracle's FP32 comparability bounds (test infrastructure of the
parity tests, not of the method):

  * the flip bound of the blend (Sec. 3.1 thresholds): a decision that sits on
    its threshold is reported, and when a perturbation far below the rounding
    window pushes it to either side, the colour moves by no more than the bound;
    one case for each kind of flip (the 1/255 skip, the 1e-4 termination, the
    order of two splats of equal depth);
  * the mass of a gradient entry's sum: at least the entry, and equal to it
    where every term has the same sign;
  * the Hutchinson entries' sensitivity to the residuals: moving every residual
    by up to its bound moves the entries by no more than hz_sens.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_00395_gb300 import synth as S

W, H = 64, 48
PX, PY = 32, 24  # the pixel under test; its centre is (32.5, 24.5)


def _cam():
    return S.single_camera(W, H)


def _scene(specs):
    """Degree-0 Gaussians: (y, z, depth_x, log_scale, logit, colour) each; the
    camera sits at +x and looks at the origin, so x sets the depth."""
    n = len(specs)
    P = np.zeros((14, n))
    for i, (y, z, x, ls, logit, col) in enumerate(specs):
        P[0:3, i] = (x, y, z)
        P[3:6, i] = ls
        P[6:10, i] = (0.0, 0.0, 0.0, 1.0)
        P[10, i] = logit
        P[11:14, i] = (np.asarray(col) - 0.5) / 0.28209479177387814  # colour under the degree-0 basis
    return P


def _alpha_at(P, i, cam):
    s = O.project(P, 0, cam)
    dx, dy = s["mx"][i] - (PX + 0.5), s["my"][i] - (PY + 0.5)
    power = -0.5 * (s["A"][i] * dx * dx + s["C"][i] * dy * dy) - s["B"][i] * dx * dy
    return s["o"][i], math.exp(power)


def _logit(p):
    return math.log(p / (1.0 - p))


def _pixel(r):
    return r["image"][0][:, PY, PX], r["impact"][0][PY, PX]


def test_skip_flip_is_bounded():
    cam = _cam()
    P = _scene([(0.0, 0.0, 0.5, -2.5, 0.0, (0.9, 0.2, 0.1)),
                (0.03, -0.02, 0.0, -2.5, 0.0, (0.1, 0.8, 0.3)),
                (0.0, 0.01, -0.5, -2.0, 1.0, (0.2, 0.3, 0.9))])
    # tune the middle splat so that its alpha at the pixel is exactly 1/255
    _, G = _alpha_at(P, 1, cam)
    P[10, 1] = _logit((1.0 / 255.0) / G)
    c0, impact = _pixel(O.render(P, 0, [cam]))
    assert impact > 0.0
    side = []
    for d in (-1e-9, 1e-9):
        Q = P.copy()
        Q[10, 1] += d
        side.append(_pixel(O.render(Q, 0, [cam]))[0])
    moved = np.abs(side[1] - side[0]).max()
    assert moved > 1e-6  # the splat is blended on one side only
    assert moved <= impact
    assert np.abs(c0 - side[0]).max() <= impact and np.abs(c0 - side[1]).max() <= impact


def test_termination_flip_is_bounded():
    cam = _cam()
    # alphas 0.96, 0.97, then a third splat that brings T exactly to 1e-4, then one more
    P = _scene([(0.0, 0.0, 0.6, -1.5, 0.0, (0.9, 0.1, 0.1)),
                (0.0, 0.0, 0.3, -1.5, 0.0, (0.1, 0.9, 0.1)),
                (0.0, 0.0, 0.0, -1.5, 0.0, (0.1, 0.1, 0.9)),
                (0.0, 0.0, -0.3, -1.5, 0.0, (0.8, 0.8, 0.8))])
    for i, a in enumerate((0.96, 0.97, None, 0.5)):
        _, G = _alpha_at(P, i, cam)
        if a is not None:
            P[10, i] = _logit(a / G)
    _, G = _alpha_at(P, 2, cam)
    P[10, 2] = _logit((1.0 - 1e-4 / ((1 - 0.96) * (1 - 0.97))) / G)
    _, impact = _pixel(O.render(P, 0, [cam]))
    assert impact >= 1.2e-3 * 0.5  # T in front of the third splat (1.2e-3) times a colour
    side = []
    for d in (-1e-9, 1e-9):
        Q = P.copy()
        Q[10, 2] += d
        side.append(_pixel(O.render(Q, 0, [cam]))[0])
    moved = np.abs(side[1] - side[0]).max()
    assert moved > 1e-5  # blended on one side, the walk stops before it on the other
    assert moved <= impact


def test_depth_swap_is_bounded():
    cam = _cam()
    A = (0.0, 0.0, 0.0, -2.0, 0.5, (0.9, 0.1, 0.1))
    B = (0.01, 0.0, 0.0, -2.2, 1.0, (0.1, 0.2, 0.9))
    one = O.render(_scene([A, B]), 0, [cam])
    two = O.render(_scene([B, A]), 0, [cam])  # equal depths sort by index: the other order
    (c1, i1), (c2, i2) = _pixel(one), _pixel(two)
    moved = np.abs(c1 - c2).max()
    assert moved > 1e-4
    assert moved <= i1 and moved <= i2


def test_gradient_mass_bounds_the_entry_and_equals_it_without_cancellation():
    cam = _cam()
    P = _scene([(0.02, -0.01, 0.0, -2.0, 0.3, (0.6, 0.4, 0.5))])
    img = O.render(P, 0, [cam], with_margin=False)["image"]
    # L2 objective with every residual +1: dL/dC = 1/m > 0 at every pixel, so
    # the DC colour rows sum terms Y_0 a T / m of one sign
    r = O.backward(P, 0, [cam], img - 1.0, loss_kind=1, masses=True)
    g, m = r["grad"], r["grad_mass"]
    assert np.all(m >= np.abs(g) * (1 - 1e-12))
    np.testing.assert_allclose(m[11:14], np.abs(g[11:14]), rtol=1e-12)
    # the mean's image-plane rows cancel across the footprint
    assert np.all(m[1:3, 0] > 10 * np.abs(g[1:3, 0]))


def test_hutchinson_sensitivity_bounds_residual_moves():
    sc = S.make_scene(200, 1, seed=12, extent=1.0, log_scale_shift=math.log(1.5))
    cam = S.single_camera(48, 40)
    P = O.params64(sc)
    target = S.smooth_target(1, 40, 48, seed=2012).astype(np.float64)
    base = O.render(P, 1, [cam])
    r0 = O.backward(P, 1, [cam], target, loss_kind=0, seed=3, t=2, nu=1, masses=True)
    assert r0["hz_sens"].max() > 0
    # residuals near the Gauss-Newton floor are where the weight is sensitive
    near = (np.abs(base["image"] - target) > 1e-3) & (np.abs(base["image"] - target) < 3e-3)
    assert near.any()
    rng = np.random.default_rng(4)
    e = np.minimum(base["err"], 1e-5)[:, None, :, :] * np.ones((1, 3, 1, 1))
    signs = [rng.choice([-1.0, 1.0], size=target.shape) for _ in range(3)]
    signs.append(np.sign(base["image"] - target))  # every |r| grows: the bound is reached
    for s in signs:
        r1 = O.backward(P, 1, [cam], target - 0.999 * e * s, loss_kind=0, seed=3, t=2, nu=1)
        moved = np.abs(r1["hz"] - r0["hz"])
        assert np.all(moved <= 1.02 * r0["hz_sens"] + 1e-15 * np.abs(r0["hz"]).max())
    on = r0["hz_sens"] > 0
    assert (moved[on] / r0["hz_sens"][on]).max() > 0.9


def _skip_scene():
    cam = _cam()
    P = _scene([(0.0, 0.0, 0.5, -2.5, 0.0, (0.9, 0.2, 0.1)),
                (0.03, -0.02, 0.0, -2.5, 0.0, (0.1, 0.8, 0.3)),
                (0.0, 0.01, -0.5, -2.0, 1.0, (0.2, 0.3, 0.9))])
    _, G = _alpha_at(P, 1, cam)
    P[10, 1] = _logit((1.0 / 255.0) / G)
    return P, 1


def _termination_scene():
    cam = _cam()
    P = _scene([(0.0, 0.0, 0.6, -1.5, 0.0, (0.9, 0.1, 0.1)),
                (0.0, 0.0, 0.3, -1.5, 0.0, (0.1, 0.9, 0.1)),
                (0.0, 0.0, 0.0, -1.5, 0.0, (0.1, 0.1, 0.9)),
                (0.0, 0.0, -0.3, -1.5, 0.0, (0.8, 0.8, 0.8))])
    for i, a in enumerate((0.96, 0.97, None, 0.5)):
        _, G = _alpha_at(P, i, cam)
        if a is not None:
            P[10, i] = _logit(a / G)
    _, G = _alpha_at(P, 2, cam)
    P[10, 2] = _logit((1.0 - 1e-4 / ((1 - 0.96) * (1 - 0.97))) / G)
    return P, 2


@pytest.mark.parametrize("make", [_skip_scene, _termination_scene])
def test_gradient_allowances_bound_the_flips(make):
    """At a skip or termination decision on its threshold, the gradient on either
    side of the flip differs by no more than the oracle's allowances (flips of a
    Gaussian's own decisions, terminations in front of it, and the rounding)."""
    cam = _cam()
    P, k = make()
    target = np.full((1, 3, H, W), 0.25)
    r0 = O.backward(P, 0, [cam], target, loss_kind=1, masses=True)
    bound = r0["grad_allow"] + r0["grad_round"]
    assert bound.max() > 0
    side = []
    for d in (-1e-9, 1e-9):
        Q = P.copy()
        Q[10, k] += d
        side.append(O.backward(Q, 0, [cam], target, loss_kind=1)["grad"])
    moved = np.abs(side[1] - side[0])
    assert moved.max() > 0
    assert np.all(moved <= bound + 1e-12 * np.abs(r0["grad"]).max())


def _one_pixel(P, **kw):
    return O.render_pixels(P, 0, _cam(), [PX], [PY], seed=3, t=2, nu=2, **kw)


def _swap_scene():
    A = (0.0, 0.0, 0.0, -2.0, 0.5, (0.9, 0.1, 0.1))
    B = (0.01, 0.0, 0.0, -2.2, 1.0, (0.1, 0.2, 0.9))
    return _scene([A, B]), _scene([B, A])


@pytest.mark.parametrize("make", [_skip_scene, _termination_scene])
def test_outcomes_hold_both_sides_of_a_flip(make):
    """A decision on its threshold gives two outcomes; each of them is what the
    blend gives when a perturbation far below the rounding window pushes the
    decision to that side (colour, T and the image tangents), and the last one is
    the FP64 result."""
    P, k = make()
    r = _one_pixel(P, outcomes=16)
    assert r["n_leaves"][0] == 2
    L = r["n_leaves"][0]
    np.testing.assert_array_equal(r["leaf_rgb"][0, L - 1], r["rgb"][0])
    np.testing.assert_array_equal(r["leaf_T"][0, L - 1], r["final_T"][0])
    np.testing.assert_allclose(r["leaf_jz"][0, L - 1], r["jz"][0], rtol=0, atol=1e-15)
    hit = set()
    for d in (-1e-9, 1e-9):
        Q = P.copy()
        Q[10, k] += d
        s = _one_pixel(Q)
        err = [max(np.abs(r["leaf_rgb"][0, l] - s["rgb"][0]).max(), abs(r["leaf_T"][0, l] - s["final_T"][0]),
                   np.abs(r["leaf_jz"][0, l] - s["jz"][0]).max()) for l in range(L)]
        assert min(err) <= 1e-8, err
        hit.add(int(np.argmin(err)))
    assert hit == {0, 1}  # the two sides reach different outcomes


def test_outcomes_hold_both_orders_of_equal_depths():
    one, two = _swap_scene()
    r = _one_pixel(one, outcomes=16)
    assert r["n_leaves"][0] == 2
    other = _one_pixel(two)
    err = [np.abs(r["leaf_rgb"][0, l] - other["rgb"][0]).max() for l in range(2)]
    assert min(err) <= 1e-12 and max(err) > 1e-4
    np.testing.assert_array_equal(r["leaf_rgb"][0, 1], r["rgb"][0])


def test_outcomes_without_a_near_decision_are_the_fp64_result():
    """Where no decision is within rounding of its threshold there is one
    outcome, the blend itself; the leaf cap reports -1 when there are more."""
    sc = S.make_scene(300, 1, seed=21, extent=1.0)
    cam = S.single_camera(W, H)
    P = O.params64(sc)
    rng = np.random.default_rng(8)
    xs, ys = rng.integers(0, W, 200), rng.integers(0, H, 200)
    r = O.render_pixels(P, 1, cam, xs, ys, seed=3, t=2, nu=1, outcomes=8)
    firm = (r["impact"] == 0) & (r["t_impact"] == 0)
    assert firm.sum() > 150
    assert np.all(r["n_leaves"][firm] == 1)
    np.testing.assert_array_equal(r["leaf_rgb"][firm, 0], r["rgb"][firm])
    np.testing.assert_array_equal(r["leaf_T"][firm, 0], r["final_T"][firm])
    np.testing.assert_allclose(r["leaf_jz"][firm, 0], r["jz"][firm], rtol=0, atol=1e-15)
    assert np.all(r["rest"][firm] == 0)
    P2, _ = _skip_scene()
    assert _one_pixel(P2, outcomes=1)["n_leaves"][0] == -1


def test_outcomes_cover_every_pixel_of_a_scene():
    """On every pixel of a small scene: at least one outcome, the last one the
    FP64 blend bit for bit, every T in [0, 1], and a single outcome wherever
    the flip bound is zero."""
    sc = S.make_scene(400, 1, seed=23, extent=1.0, log_scale_shift=math.log(1.5))
    cam = S.single_camera(40, 32)
    P = O.params64(sc)
    ys, xs = np.mgrid[0:32, 0:40]
    xs, ys = xs.ravel(), ys.ravel()
    r = O.render_pixels(P, 1, cam, xs, ys, outcomes=64)
    nl = r["n_leaves"]
    assert np.all(nl >= 1)
    last = nl - 1
    k = np.arange(len(xs))
    np.testing.assert_array_equal(r["leaf_rgb"][k, last], r["rgb"])
    np.testing.assert_array_equal(r["leaf_T"][k, last], r["final_T"])
    valid = np.arange(r["leaf_T"].shape[1])[None, :] < nl[:, None]
    assert np.all((r["leaf_T"][valid] >= 0.0) & (r["leaf_T"][valid] <= 1.0))
    firm = (r["impact"] == 0) & (r["t_impact"] == 0)
    assert np.all(nl[firm] == 1)


@pytest.mark.parametrize("side", ["added", "dropped"])
def test_outcomes_hold_both_sides_of_a_membership_flip(side):
    """3DGS tile squares (the oracle's default binning): a bright splat of
    radius 10 px whose square ends exactly on a tile boundary, so whether the
    tile beyond lists it is within FP32 rounding, while its alpha at the pixel
    just past the boundary is above 1/255.  "added": the square starts at
    x = 32 (mx - r = 32), FP64 leaves tile 1 out and FP32 may list the splat
    there (pixel 31); "dropped": it ends so that (mx + r + 15) / 16 = 4
    (mx + r = 49), FP64 lists it in tile 3 and FP32 may not (pixel 48).  That
    pixel has two outcomes, with and without the splat; moving the splat by a
    few FP32 ulps either way reproduces each."""
    cam = _cam()

    def scene(y):
        return _scene([(y, 0.0, 0.0, -1.5, 3.0, (0.9, 0.2, 0.1)),
                       (0.0, 0.0, -0.6, -1.0, 0.0, (0.2, 0.3, 0.8))])

    def edge(y):  # the square's end, minus the boundary it is put on
        s = O.project(scene(y), 0, cam)
        mx, r = s["mx"][0], s["radius"][0]
        return mx - r - 32.0 if side == "added" else mx + r - 49.0

    a, b = (0.5, 1.0) if side == "added" else (0.3, 0.6)  # secant solve of edge(y) = 0
    fa, fb = edge(a), edge(b)
    for _ in range(60):
        if fb == 0.0 or fa == fb:
            break
        a, b, fa = b, b - fb * (b - a) / (fb - fa), fb
        fb = edge(b)
    assert abs(fb) < 1e-9 and O.project(scene(b), 0, cam)["radius"][0] == 10
    px = 31 if side == "added" else 48
    r = O.render_pixels(scene(b), 0, cam, [px], [24], outcomes=16)
    assert r["n_leaves"][0] == 2 and r["flip_kinds"][0] & 4
    np.testing.assert_array_equal(r["leaf_rgb"][0, 1], r["rgb"][0])  # the last outcome is the FP64 blend
    hit = set()
    for d in (-2e-6, 2e-6):  # about 2.8e-5 px, several FP32 ulps of mx
        s = O.render_pixels(scene(b + d), 0, cam, [px], [24])
        err = [np.abs(r["leaf_rgb"][0, l] - s["rgb"][0]).max() for l in range(2)]
        assert min(err) <= 1e-6, err
        hit.add(int(np.argmin(err)))
    assert hit == {0, 1}
    assert np.abs(r["leaf_rgb"][0, 0] - r["leaf_rgb"][0, 1]).max() > 1e-3
