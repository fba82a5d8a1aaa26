"""Pins of the oracle's projection, binning and blending (Sec. 3.1).

Projection: the exact pinhole image of the mean, the closed-form footprint of
an isotropic Gaussian on the optical axis, and a Monte-Carlo projection of
samples (EWA is the linearisation of that projection).  Binning: a brute-force
interval test over every tile and numpy's lexicographic sort; the footprint box
that narrows the 3DGS tile square leaves every image equal to a per-pixel blend
over the depth-sorted splats with the square alone.  Blending: single
splat, two coincident splats, and the telescoping identity C = c (1 - T) for
splats that share one colour.
"""
import math

import numpy as np
import pytest
from scipy.special import expit

import oracle as O
from paper_2602_00395_gb300 import synth as S


def _cam(W=1000, H=800, dist=4.0):
    return S.Camera(S.look_at((dist, 0.3, -0.2)), **S.pinhole(W, H))


def _one(mu, log_s, q, logit, sh):
    K = len(sh)
    P = np.zeros((11 + 3 * K, 1))
    P[0:3, 0] = mu
    P[3:6, 0] = log_s
    P[6:10, 0] = q
    P[10, 0] = logit
    P[11:, 0] = np.asarray(sh, np.float64).reshape(-1)
    return P


def _to_world(cam, pc):
    V = np.asarray(cam.viewmat)
    return V[:3, :3].T @ (np.asarray(pc) - V[:3, 3])


def test_mean_depth_opacity_match_pinhole():
    rng = np.random.default_rng(0)
    cam = _cam()
    V = np.asarray(cam.viewmat)
    for _ in range(20):
        pc = np.array([rng.uniform(-1, 1), rng.uniform(-0.8, 0.8), rng.uniform(2, 6)])
        mu = _to_world(cam, pc)
        logit = rng.normal()
        P = _one(mu, [-3, -3, -3], [0, 0, 0, 1], logit, [[0.1, 0.2, 0.3]])
        s = O.project(P, 0, cam)
        assert s["valid"][0] == 1
        np.testing.assert_allclose(s["mx"][0], cam.fx * pc[0] / pc[2] + cam.cx, rtol=1e-13)
        np.testing.assert_allclose(s["my"][0], cam.fy * pc[1] / pc[2] + cam.cy, rtol=1e-13)
        np.testing.assert_allclose(s["depth"][0], (V[:3, :3] @ mu + V[:3, 3])[2], rtol=1e-13)
        np.testing.assert_allclose(s["o"][0], expit(logit), rtol=1e-13)


def test_isotropic_on_axis_is_a_circle_of_predicted_radius():
    cam = _cam()
    for z, ls in ((3.0, -3.0), (5.0, -2.0), (2.5, -4.5)):
        mu = _to_world(cam, [0.0, 0.0, z])
        P = _one(mu, [ls] * 3, [0.2, -0.1, 0.4, 0.8], 0.0, [[0.0, 0.0, 0.0]])
        s = O.project(P, 0, cam)
        var = (cam.fx * math.exp(ls) / z) ** 2 + 0.3  # J Sigma J^T = (f/z)^2 s^2 I on the axis
        np.testing.assert_allclose(s["A"][0], 1 / var, rtol=1e-12)
        np.testing.assert_allclose(s["C"][0], 1 / var, rtol=1e-12)
        assert abs(s["B"][0]) < 1e-12 / var
        # lambda_max = mid + sqrt(max(0.1, mid^2 - det)) and mid^2 = det for a circle
        lam = var + math.sqrt(0.1)
        np.testing.assert_allclose(s["radius_raw"][0], 3 * math.sqrt(lam), rtol=1e-12)
        assert s["radius"][0] == math.ceil(3 * math.sqrt(lam))


def test_ewa_covariance_matches_monte_carlo_projection():
    """Sigma' - 0.3 I is the covariance of the pinhole image of samples, to first order."""
    rng = np.random.default_rng(1)
    cam = _cam()
    V = np.asarray(cam.viewmat)
    for pc in ([0.7, -0.45, 4.0], [-0.9, 0.6, 3.0]):
        mu = _to_world(cam, pc)
        log_s = np.log([0.006, 0.002, 0.004])
        q = rng.normal(size=4)
        P = _one(mu, log_s, q, 0.0, [[0, 0, 0]])
        s = O.project(P, 0, cam)
        conic = np.array([[s["A"][0], s["B"][0]], [s["B"][0], s["C"][0]]])
        cov_ewa = np.linalg.inv(conic) - 0.3 * np.eye(2)
        R = O.quat_to_rotmat(q)
        Sig = R @ np.diag(np.exp(2 * log_s)) @ R.T
        x = rng.multivariate_normal(mu, Sig, size=400000)
        xc = x @ V[:3, :3].T + V[:3, 3]
        uv = np.stack([cam.fx * xc[:, 0] / xc[:, 2] + cam.cx, cam.fy * xc[:, 1] / xc[:, 2] + cam.cy], 1)
        cov_mc = np.cov(uv.T)
        assert np.abs(cov_ewa - cov_mc).max() < 0.02 * np.abs(cov_mc).max(), (cov_ewa, cov_mc)
        np.testing.assert_allclose(uv.mean(0), [s["mx"][0], s["my"][0]], atol=0.01)


def test_degree0_colour_is_view_independent():
    c0 = 0.5 / math.sqrt(math.pi)
    sh = [[0.3, -0.2, 1.1]]
    P = _one([0.1, 0.2, 0.0], [-3] * 3, [0, 0, 0, 1], 0.0, sh)
    for cam in S.camera_ring(6, 64, 48, 1.0):
        s = O.project(P, 0, cam)
        np.testing.assert_allclose([s["r"][0], s["g"][0], s["b"][0]],
                                   np.maximum(c0 * np.array(sh[0]) + 0.5, 0.0), rtol=1e-13)


def test_behind_near_plane_is_culled():
    cam = _cam()
    P = _one(_to_world(cam, [0, 0, 0.1]), [-3] * 3, [0, 0, 0, 1], 0.0, [[0, 0, 0]])
    assert O.project(P, 0, cam)["valid"][0] == 0


# ---------------------------------------------------------------- binning
def _half(bits):
    return float(np.array([bits], np.uint16).view(np.float16)[0])


F = np.float32


def _row_span(mx, my, A, B, C, hx, hy, x0, x1, ty, tw, th, Tx):
    """Tiles [a, b) of row ty narrowed to the footprint ellipse, in FP32 with one
    rounding per operation in the order of the binning rule."""
    if not (hx > 0 and hy > 0 and hx < 65536 and hy < 65536 and A > 0 and C > 0):
        return x0, x1
    rho = min(max(F(-B) / F(np.sqrt(F(A) * F(C))), F(-1)), F(1))
    q = max(F(0), F(1) - rho * rho)
    mgn = F(F(0.01) * hx) + F(0.5)
    vlo = F(F(ty * th) - my) / hy
    vhi = F(F((ty + 1) * th) - my) / hy
    if vhi < -1 or vlo > 1:
        return x0, x0
    vr = min(max(rho, vlo), vhi)
    vl = min(max(-rho, vlo), vhi)
    sr = F(np.sqrt(max(F(0), q * F(F(1) - vr * vr))))
    sl = F(np.sqrt(max(F(0), q * F(F(1) - vl * vl))))
    xr = F(F(mx + F(hx * F(rho * vr + sr))) + mgn)
    xl = F(F(mx + F(hx * F(rho * vl - sl))) - mgn)
    cl = lambda f: 0 if not f > 0 else (Tx if f > Tx else int(f))
    a = max(x0, cl(np.floor(F(xl / F(tw)))))
    b = min(x1, cl(F(np.floor(F(xr / F(tw))) + F(1))))
    return a, max(a, b)


def _brute_tiles(mx, my, r, ext, conic, W, H, tw, th):
    """Tiles whose pixel interval [t*tw, (t+1)*tw) meets (m - r, m + r - 1] and
    [m - h, m + h] on both axes (h the footprint half-extent; FP32 sums), each
    row then narrowed to the ellipse (conic None: the rectangle)."""
    Tx, Ty = -(-W // tw), -(-H // th)
    out = []
    if r <= 0:
        return out
    hx, hy = F(_half(int(ext) & 0xFFFF)), F(_half(int(ext) >> 16))
    mx, my = F(mx), F(my)
    lo_x, hi_x = mx - F(r), mx + F(r - 1)
    lo_y, hi_y = my - F(r), my + F(r - 1)
    with np.errstate(invalid="ignore", over="ignore"):
        flo_x, fhi_x = mx - hx, mx + hx
        flo_y, fhi_y = my - hy, my + hy
    cols = [tx for tx in range(Tx) if tx * tw <= hi_x and (tx + 1) * tw > lo_x and tx * tw <= fhi_x
            and (tx + 1) * tw > flo_x]
    rows = [ty for ty in range(Ty) if ty * th <= hi_y and (ty + 1) * th > lo_y and ty * th <= fhi_y
            and (ty + 1) * th > flo_y]
    if not cols or not rows:
        return out
    for ty in rows:
        a, b = cols[0], cols[-1] + 1
        if conic is not None:
            with np.errstate(invalid="ignore", over="ignore", divide="ignore"):
                a, b = _row_span(mx, my, F(conic[0]), F(conic[1]), F(conic[2]), hx, hy, a, b, ty, tw, th, Tx)
        out.extend(ty * Tx + tx for tx in range(a, b))
    return out


@pytest.mark.parametrize("W,H,tw,th,n", [(128, 128, 16, 16, 300), (97, 53, 16, 8, 200), (61, 45, 8, 8, 150)])
def test_binning_against_brute_force_and_lexsort(W, H, tw, th, n):
    mx, my, r, d, ext, conic = S.projected_records(n, W, H, seed=W + n, max_radius=40)
    keys, vals, ranges = O.bin_sort(mx, my, r, d, W, H, tw, th, extents=ext, conic=conic)
    Tx, Ty = -(-W // tw), -(-H // th)
    expect = []
    for i in range(n):
        for tile in _brute_tiles(mx[i], my[i], int(r[i]), ext[i], conic[:, i], W, H, tw, th):
            key = (tile << 32) | int(np.float32(d[i]).view(np.uint32))
            expect.append((key, i))
    ek = np.array([k for k, _ in expect], np.uint64)
    ev = np.array([v for _, v in expect], np.uint32)
    order = np.lexsort((ev, ek))
    np.testing.assert_array_equal(keys, ek[order])
    np.testing.assert_array_equal(vals, ev[order])
    # ranges: every tile's [start, end) holds exactly its keys
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    for t in range(Tx * Ty):
        s, e = ranges[t]
        sel = np.nonzero(tiles == t)[0]
        if len(sel) == 0:
            assert s == e
        else:
            assert (s, e) == (sel[0], sel[-1] + 1)
    # the rows narrow the box, and without extents the 3DGS square is binned
    n_box = sum(len(_brute_tiles(mx[i], my[i], int(r[i]), ext[i], None, W, H, tw, th)) for i in range(n))
    assert len(keys) < n_box
    k2, _, _ = O.bin_sort(mx, my, r, d, W, H, tw, th)
    n_square = sum(len(_brute_tiles(mx[i], my[i], int(r[i]), 0x7C007C00, None, W, H, tw, th)) for i in range(n))
    assert len(k2) == n_square > n_box


def _extents(A, B, C, o):
    """Footprint half-extents as the projection stores them: sqrt(tau C/det) and
    sqrt(tau A/det), tau = 2 ln(255 o), widened 0.1 % + 0.01 px, rounded up to
    half precision, packed (x low)."""
    tau = 2 * np.log(255 * o)
    det = A * C - B * B
    h = []
    for v in (np.sqrt(tau * C / det), np.sqrt(tau * A / det)):
        x = v * 1.001 + 0.01
        hv = np.float16(x)
        hv = np.where(hv.astype(np.float64) < x, np.nextafter(hv, np.float16(np.inf)), hv)
        h.append(np.asarray(hv, np.float16).view(np.uint16).astype(np.uint32))
    return h[0] | (h[1] << np.uint32(16))


def test_footprint_tiles_cover_every_pixel_the_splat_reaches():
    """Random splats (correlations up to 0.995, opacities up to 0.99): every tile
    with a pixel centre where o exp(-d^T Q d / 2) >= 1/255 (FP64) is among the
    splat's tiles, and the tiles are fewer than the 3DGS square's."""
    rng = np.random.default_rng(12)
    W, H, tw, th, n = 256, 192, 16, 16, 400
    sig = np.exp(rng.uniform(np.log(0.7), np.log(40.0), size=(2, n)))
    corr = rng.uniform(-0.995, 0.995, size=n)
    cov = np.array([[sig[0] ** 2, corr * sig[0] * sig[1]], [corr * sig[0] * sig[1], sig[1] ** 2]])
    cov[0, 0] += 0.3
    cov[1, 1] += 0.3
    det = cov[0, 0] * cov[1, 1] - cov[0, 1] ** 2
    A, B, C = cov[1, 1] / det, -cov[0, 1] / det, cov[0, 0] / det
    o = rng.uniform(0.005, 0.99, size=n)
    mid = 0.5 * (cov[0, 0] + cov[1, 1])
    lam = mid + np.sqrt(np.maximum(0.1, mid * mid - det))
    r = np.ceil(3 * np.sqrt(lam)).astype(np.int32)
    mx = rng.uniform(-20, W + 20, n).astype(np.float32)
    my = rng.uniform(-20, H + 20, n).astype(np.float32)
    ext = _extents(A, B, C, o)
    conic = np.stack([A, B, C]).astype(np.float32)
    keys, vals, _ = O.bin_sort(mx, my, r, np.ones(n, np.float32), W, H, tw, th, extents=ext, conic=conic)
    have = set(zip(vals.tolist(), (keys >> np.uint64(32)).astype(np.int64).tolist()))
    Tx = -(-W // tw)
    ys, xs = np.mgrid[0:H, 0:W] + 0.5
    n_square = 0
    for i in range(n):
        dx, dy = mx[i] - xs, my[i] - ys
        a = o[i] * np.exp(-0.5 * (A[i] * dx * dx + C[i] * dy * dy) - B[i] * dx * dy)
        # the 3DGS square bounds where a splat is blended at all
        x0, x1 = max(0, int(np.floor((mx[i] - r[i]) / tw))), min(Tx, int(np.floor((mx[i] + r[i] + tw - 1) / tw)))
        y0, y1 = max(0, int(np.floor((my[i] - r[i]) / th))), min(-(-H // th), int(np.floor((my[i] + r[i] + th - 1) / th)))
        n_square += max(0, x1 - x0) * max(0, y1 - y0)
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                if (a[ty * th:(ty + 1) * th, tx * tw:(tx + 1) * tw] >= 1 / 255).any():
                    assert (i, ty * Tx + tx) in have, (i, tx, ty)
    assert len(keys) < 0.8 * n_square


def _square_blend(s, W, H, tw, th):
    """Per-pixel front-to-back blend (Sec. 3.1) over every valid splat in (FP32
    depth, index) order whose 3DGS tile square holds the pixel's tile: no lists."""
    valid = np.nonzero(s["valid"] > 0)[0]
    order = valid[np.lexsort((valid, s["depth"][valid].astype(np.float32)))]
    img, T_out = np.zeros((3, H, W)), np.ones((H, W))
    tiles = {int(i): set(_brute_tiles(s["mx"][i], s["my"][i], int(s["radius"][i]), 0x7C007C00, None, W, H, tw, th))
             for i in order}
    Tx = -(-W // tw)
    rgb = np.stack([s["r"], s["g"], s["b"]])
    for y in range(H):
        for x in range(W):
            tile = (y // th) * Tx + x // tw
            T = 1.0
            for i in order:
                if tile not in tiles[int(i)]:
                    continue
                dx, dy = s["mx"][i] - (x + 0.5), s["my"][i] - (y + 0.5)
                power = -0.5 * (s["A"][i] * dx * dx + s["C"][i] * dy * dy) - s["B"][i] * dx * dy
                if power > 0:
                    continue
                alpha = min(0.99, s["o"][i] * math.exp(power))
                if alpha < 1 / 255:
                    continue
                Tn = T * (1 - alpha)
                if Tn < 1e-4:
                    break
                img[:, y, x] += rgb[:, i] * alpha * T
                T = Tn
            T_out[y, x] = T
    return img, T_out


@pytest.mark.parametrize("tw,th", [(16, 16), (8, 8)])
def test_footprint_box_binning_leaves_the_image_unchanged(tw, th):
    """Elongated, rotated splats of all opacities: the footprint box drops tiles
    (fewer pairs than the 3DGS square gives) and no pixel changes."""
    W, H = 56, 44
    sc = S.make_scene(120, 1, seed=77, extent=0.7, log_scale_shift=math.log(2.5))
    P = O.params64(sc)
    rng = np.random.default_rng(3)
    P[3, :] += rng.uniform(-1.2, 1.2, sc.n)  # anisotropy
    P[10, :] = rng.uniform(-6.0, 5.0, sc.n)  # opacities from 0.0025 to 0.993
    cam = S.Camera(S.look_at((3.2, 0.5, -0.4)), **S.pinhole(W, H))
    s = O.project(P, 1, cam)
    square = O.render(P, 1, [cam], tw, th)
    with O.footprint_bins():
        box = O.render(P, 1, [cam], tw, th)
    img, T = _square_blend(s, W, H, tw, th)
    n_square = sum(len(_brute_tiles(s["mx"][i], s["my"][i], int(s["radius"][i]), 0x7C007C00, None, W, H, tw, th))
                   for i in np.nonzero(s["valid"] > 0)[0])
    assert square["n_pairs"] == n_square
    assert box["n_pairs"] < 0.9 * n_square
    assert T.min() < 0.2 and np.abs(img).max() > 0.3
    for out in (square, box):
        np.testing.assert_allclose(out["image"][0], img, rtol=0, atol=1e-12)
        np.testing.assert_allclose(out["final_T"][0], T, rtol=0, atol=1e-12)


# ----------------------------------------------------------------- blending
def _tiny_cam(W=32, H=32):
    return S.Camera(S.look_at((4.0, 0.0, 0.0)), **S.pinhole(W, H))


def test_single_splat_closed_form():
    cam = _tiny_cam()
    mu = _to_world(cam, [0.05, -0.02, 3.5])
    sh = [[0.4, -0.3, 0.9]]
    P = _one(mu, [-2.3, -2.9, -2.6], [0.3, 0.1, -0.2, 0.9], 0.8, sh)
    s = O.project(P, 0, cam)
    out = O.render(P, 0, [cam])
    ys, xs = np.mgrid[0:32, 0:32] + 0.5
    dx, dy = s["mx"][0] - xs, s["my"][0] - ys
    power = -0.5 * (s["A"][0] * dx ** 2 + s["C"][0] * dy ** 2) - s["B"][0] * dx * dy
    a = np.minimum(0.99, s["o"][0] * np.exp(power))
    inside = np.zeros((32, 32), bool)
    r = int(s["radius"][0])
    # only pixels of tiles in the splat's rectangle can see it
    x0, x1 = max(0, math.floor((np.float32(s["mx"][0]) - r) / 16)), min(2, math.floor((np.float32(s["mx"][0]) + r + 15) / 16))
    y0, y1 = max(0, math.floor((np.float32(s["my"][0]) - r) / 16)), min(2, math.floor((np.float32(s["my"][0]) + r + 15) / 16))
    inside[y0 * 16:y1 * 16, x0 * 16:x1 * 16] = True
    a = np.where((a >= 1 / 255) & inside, a, 0.0)
    rgb = np.array([s["r"][0], s["g"][0], s["b"][0]])
    np.testing.assert_allclose(out["image"][0], rgb[:, None, None] * a[None], atol=1e-14)
    np.testing.assert_allclose(out["final_T"][0], 1 - a, atol=1e-14)


def test_two_coincident_splats_blend_in_depth_order():
    cam = _tiny_cam()
    near = _to_world(cam, [0.0, 0.0, 3.0])
    far = _to_world(cam, [0.0, 0.0, 3.6])
    c1, c2 = [0.9, 0.1, 0.0], [0.0, 0.2, 0.8]
    P = np.concatenate([_one(far, [-1.8] * 3, [0, 0, 0, 1], 0.5, [c2]),
                        _one(near, [-1.8 + math.log(3.0 / 3.6)] * 3, [0, 0, 0, 1], -0.3, [c1])], axis=1)
    s = O.project(P, 0, cam)
    out = O.render(P, 0, [cam])
    px = 16  # pixel (16, 16) centre is (16.5, 16.5); means project to (16, 16)
    ys, xs = px + 0.5, px + 0.5
    def alpha(i):
        dx, dy = s["mx"][i] - xs, s["my"][i] - ys
        return min(0.99, s["o"][i] * math.exp(-0.5 * (s["A"][i] * dx * dx + s["C"][i] * dy * dy) - s["B"][i] * dx * dy))
    a_near, a_far = alpha(1), alpha(0)
    rgb = lambda i: np.array([s["r"][i], s["g"][i], s["b"][i]])
    expect = rgb(1) * a_near + rgb(0) * a_far * (1 - a_near)
    np.testing.assert_allclose(out["image"][0][:, px, px], expect, rtol=1e-13)
    np.testing.assert_allclose(out["final_T"][0][px, px], (1 - a_near) * (1 - a_far), rtol=1e-13)


def test_shared_colour_telescopes_to_one_minus_T():
    """If every splat has colour c then sum c a_i T_i = c (1 - T_final)."""
    sc = S.make_scene(400, 0, seed=5, extent=0.8, log_scale_shift=math.log(2.0))
    P = O.params64(sc)
    c0 = 0.5 / math.sqrt(math.pi)
    c = np.array([0.7, 0.3, 0.55])
    P[11:14, :] = ((c - 0.5) / c0)[:, None]
    out = O.render(P, 0, [_tiny_cam(48, 40)])
    img, T = out["image"][0], out["final_T"][0]
    assert T.min() < 0.05  # some pixels are nearly opaque
    np.testing.assert_allclose(img, c[:, None, None] * (1 - T)[None], atol=1e-13)
    # termination: T never drops below 1e-4
    assert T.min() >= 1e-4
