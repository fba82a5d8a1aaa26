"""FP64 CPU oracle for one 3DGS^2-TR iteration (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
import this package; the product path never does.  The arithmetic lives in
``gs_oracle.cpp`` (plain C++, FP64); this module only marshals numpy arrays.

Parameter matrices are float64 [rows, n] (no padding), rows as in the
package's synthetic-scene layout: 0..2 mean, 3..5 log-scale, 6..9 quaternion
(x, y, z, w), 10 opacity logit, 11 + 3k + c SH coefficient k of channel c.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CXXFLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile gs_oracle.cpp into liboracle.so (g++, a few seconds)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", *CXXFLAGS, "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            d, i64, u64, i32 = C.c_double, C.c_long, C.c_uint64, C.c_int
            P = C.c_void_p
            L.or_splitmix64.restype = u64
            L.or_splitmix64.argtypes = [u64]
            L.or_rademacher.restype = d
            L.or_rademacher.argtypes = [u64, C.c_int64, i32, u64]
            L.or_sh_basis.argtypes = [i32, P, P]
            L.or_sh_absmax.argtypes = [i32, P]
            L.or_quat_to_rotmat.argtypes = [P, P]
            L.or_project.argtypes = [P, i64, i64, i32, P, P]
            L.or_set_footprint_bins.argtypes = [i32]
            L.or_bin_sort.restype = i64
            L.or_bin_sort.argtypes = [i32, i64, P, P, P, P, P, P, P, P, i32, i32, i32, i32, P, P, i64, P]
            L.or_render.restype = i64
            L.or_render.argtypes = [P, i64, i64, i32, P, i32, i32, i32, P, P, P, P, P, P, P, P]
            L.or_jvp.argtypes = [P, i64, i64, i32, P, i32, i32, i32, P, P]
            L.or_jacobian.argtypes = [P, i64, i64, i32, P, i32, i32, i32, P]
            L.or_backward_dssim.restype = d
            L.or_backward_dssim.argtypes = [P, i64, i64, i32, P, i32, i32, i32, P, d, d, u64, C.c_int64, i32,
                                            P, P, P, P, P, P, P, P, P]
            L.or_ssim.argtypes = [P, P, i32, i32, P, P, P, P]
            L.or_ssim_vjp.argtypes = [P, P, i32, i32, P, P]
            L.or_ssim_jvp.argtypes = [P, P, i32, i32, P, P]
            L.or_backward.restype = d
            L.or_backward.argtypes = [P, i64, i64, i32, P, i32, i32, i32, P, i32, d, u64, C.c_int64, i32,
                                      P, P, P, P, P, P, P, P, P, P, P]
            L.or_shd_radius.argtypes = [P, i64, i64, i32, d, P, P]
            L.or_tr_update.argtypes = [P, P, P, P, P, i64, i64, i32, P, C.c_int64, d, P]
            L.or_adam_tr_update.argtypes = [P, P, P, P, i64, i64, i32, P, P, C.c_int64, d, P]
            L.or_project_tangent.argtypes = [P, i64, i64, i32, P, P, P]
            L.or_render_pixels.argtypes = [P, i64, i64, i32, P, i32, i32, i64, P, P, u64, C.c_int64, i32, P, P, P,
                                           P, P, P, P, P, P, i32, d, P, P, P, P, P, P]
            L.or_backward_sampled.argtypes = [P, i64, i64, i32, P, i32, i32, i32, P, i32, d, u64, C.c_int64, i32,
                                              i64, P, P, P, P, d, P, P, P, P, P, P, P]
            L.or_signature.argtypes = [P, i64, i64, i32, P, i32, i32, i32, P]
            L.or_hellinger.restype = d
            L.or_hellinger.argtypes = [P, P, d, P, P, d]
            L.or_rotation_beta.argtypes = [P, P, P]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def camera_array(cams) -> np.ndarray:
    """24 doubles per camera: viewmat (16, row-major), fx, fy, cx, cy, near, width, height, 0."""
    out = np.zeros((len(cams), 24))
    for k, c in enumerate(cams):
        out[k, :16] = np.asarray(c.viewmat, np.float64).reshape(16)
        out[k, 16:23] = [c.fx, c.fy, c.cx, c.cy, c.near, c.width, c.height]
    return out


def params64(scene_or_params, n: int | None = None) -> np.ndarray:
    """float64 [rows, n] copy of a scene's parameters with the padding dropped."""
    if hasattr(scene_or_params, "params"):
        return _f64(scene_or_params.params[:, : scene_or_params.n])
    a = np.asarray(scene_or_params)
    return _f64(a if n is None else a[:, :n])


# ---------------------------------------------------------------- primitives
def splitmix64(x: int) -> int:
    return int(lib().or_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def rademacher(seed: int, t: int, k: int, j: int) -> float:
    return float(lib().or_rademacher(seed, t, k, j))


def sh_basis(deg: int, direction) -> np.ndarray:
    d = _f64(direction)
    Y = np.zeros(16)
    lib().or_sh_basis(deg, _p(d), _p(Y))
    return Y[: (deg + 1) ** 2]


def sh_absmax(deg: int) -> np.ndarray:
    Y = np.zeros(16)
    lib().or_sh_absmax(deg, _p(Y))
    return Y[: (deg + 1) ** 2]


def quat_to_rotmat(q) -> np.ndarray:
    q = _f64(q)
    R = np.zeros(9)
    lib().or_quat_to_rotmat(_p(q), _p(R))
    return R.reshape(3, 3)


def hellinger(mu1, S1, Z1, mu2, S2, Z2) -> float:
    return float(lib().or_hellinger(_p(_f64(mu1)), _p(_f64(S1)), Z1, _p(_f64(mu2)), _p(_f64(S2)), Z2))


def rotation_beta(q, s) -> np.ndarray:
    b = np.zeros(4)
    lib().or_rotation_beta(_p(_f64(q)), _p(_f64(s)), _p(b))
    return b


# --------------------------------------------------------------- pipeline
SPLAT_FIELDS = ("mx", "my", "A", "B", "C", "o", "r", "g", "b", "depth", "radius_raw", "radius", "valid")


def project(P: np.ndarray, deg: int, cam) -> dict:
    P = _f64(P)
    rows, n = P.shape
    out = np.zeros((n, 13))
    ca = camera_array([cam])
    lib().or_project(_p(P), n, n, deg, _p(ca), _p(out))
    return {f: out[:, k] for k, f in enumerate(SPLAT_FIELDS)}


def project_tangent(P: np.ndarray, deg: int, cam, direction: np.ndarray) -> np.ndarray:
    """n x 9 tangents of (mx, my, A, B, C, o, r, g, b) along a parameter direction (rows x n)."""
    P = _f64(P)
    rows, n = P.shape
    d = _f64(direction)
    out = np.zeros((n, 9))
    lib().or_project_tangent(_p(P), n, n, deg, _p(camera_array([cam])), _p(d), _p(out))
    return out


def probe_matrix(seed: int, t: int, k: int, rows: int, n: int) -> np.ndarray:
    """Rademacher probe k of step t as a rows x n matrix (row r of Gaussian i is
    entry j = i * rows + r)."""
    z = np.empty(rows * n)
    L = lib()
    for j in range(rows * n):
        z[j] = L.or_rademacher(seed, t, k, j)
    return z.reshape(n, rows).T.copy()


@contextlib.contextmanager
def footprint_bins(on: bool = True):
    """Within the block, renders, JVPs, Jacobians and backward passes bin each
    splat into its 3DGS tile square narrowed to its footprint box (the GPU
    frame's footprint_bins = 1); outside it, into the whole square."""
    L = lib()
    L.or_set_footprint_bins(int(on))
    try:
        yield
    finally:
        L.or_set_footprint_bins(0)


def bin_sort(mx, my, radius, depth, width: int, height: int, tw: int = 16, th: int = 16, extents=None,
             conic=None):
    """Pairs and tile ranges from FP32 splat records; arrays are [V, n] (or [n]).
    `extents` are the records' footprint half-extents as packed halves (uint32,
    x in the low 16 bits) and `conic` their (A, B, C), [3, V, n] (or [3, n]);
    without extents the 3DGS square is binned."""
    mx = np.ascontiguousarray(np.atleast_2d(mx), np.float32)
    my = np.ascontiguousarray(np.atleast_2d(my), np.float32)
    rad = np.ascontiguousarray(np.atleast_2d(radius), np.int32)
    dp = np.ascontiguousarray(np.atleast_2d(depth), np.float32)
    ext = None if extents is None else np.ascontiguousarray(np.atleast_2d(extents), np.uint32)
    V, n = mx.shape
    if conic is None:
        cA, cB, cC = (np.zeros((V, n), np.float32) for _ in range(3))
    else:
        cA, cB, cC = (np.ascontiguousarray(np.asarray(c, np.float32).reshape(V, n)) for c in conic)
    T = ((width + tw - 1) // tw) * ((height + th - 1) // th)
    ranges = np.zeros((V * T, 2), np.uint32)
    L = lib()
    pe = None if ext is None else _p(ext)
    args = (V, n, _p(mx), _p(my), _p(cA), _p(cB), _p(cC), _p(rad), pe, _p(dp), width, height, tw, th)
    P = L.or_bin_sort(*args, None, None, 0, _p(ranges))
    keys = np.zeros(max(P, 1), np.uint64)
    vals = np.zeros(max(P, 1), np.uint32)
    L.or_bin_sort(*args, _p(keys), _p(vals), P, _p(ranges))
    return keys[:P], vals[:P], ranges


def render(P: np.ndarray, deg: int, cams, tw: int = 16, th: int = 16, with_margin: bool = True):
    """Image, final T, n_contrib; with_margin adds the decision margin, the bounds
    ``impact`` / ``t_impact`` on what FP32 flips of the blend's decisions can do to
    each pixel's colour and final T, ``err`` on the colour's own FP32 rounding,
    and the n_contrib range they allow."""
    P = _f64(P)
    rows, n = P.shape
    ca = camera_array(cams)
    V = len(cams)
    H, W = cams[0].height, cams[0].width
    img = np.zeros((V, 3, H, W))
    T = np.zeros((V, H, W))
    nc = np.zeros((V, H, W), np.int32)
    mg = np.zeros((V, H, W)) if with_margin else None
    rng = np.zeros((V, H, W, 2), np.int32) if with_margin else None
    imp = np.zeros((V, H, W)) if with_margin else None
    timp = np.zeros((V, H, W)) if with_margin else None
    err = np.zeros((V, H, W)) if with_margin else None
    pairs = lib().or_render(_p(P), n, n, deg, _p(ca), V, tw, th, _p(img), _p(T), _p(nc), _p(mg), _p(rng),
                            _p(imp), _p(timp), _p(err))
    out = dict(image=img, final_T=T, n_contrib=nc, margin=mg, n_pairs=int(pairs), impact=imp, t_impact=timp,
               err=err)
    if with_margin:
        out["n_contrib_lo"], out["n_contrib_hi"] = rng[..., 0], rng[..., 1]
    return out


def jvp(P: np.ndarray, deg: int, cams, direction: np.ndarray, tw: int = 16, th: int = 16) -> np.ndarray:
    P = _f64(P)
    rows, n = P.shape
    d = _f64(direction)
    ca = camera_array(cams)
    V = len(cams)
    H, W = cams[0].height, cams[0].width
    out = np.zeros((V, 3, H, W))
    lib().or_jvp(_p(P), n, n, deg, _p(ca), V, tw, th, _p(d), _p(out))
    return out


def signature(P: np.ndarray, deg: int, cams, tw: int = 16, th: int = 16) -> np.ndarray:
    """Per-pixel hash of the blend's discrete decisions (contributors, caps, clamps)."""
    P = _f64(P)
    rows, n = P.shape
    ca = camera_array(cams)
    V = len(cams)
    H, W = cams[0].height, cams[0].width
    out = np.zeros((V, H, W), np.uint64)
    lib().or_signature(_p(P), n, n, deg, _p(ca), V, tw, th, _p(out))
    return out


def jacobian(P: np.ndarray, deg: int, cams, tw: int = 16, th: int = 16) -> np.ndarray:
    """dC/dx: rows = V*3*H*W image entries, columns = rows_p * n parameters (index r*n + i)."""
    P = _f64(P)
    rows, n = P.shape
    ca = camera_array(cams)
    V = len(cams)
    H, W = cams[0].height, cams[0].width
    J = np.zeros((V * 3 * H * W, rows * n))
    lib().or_jacobian(_p(P), n, n, deg, _p(ca), V, tw, th, _p(J))
    return J


def backward(P: np.ndarray, deg: int, cams, target: np.ndarray, *, loss_kind: int = 0,
             gn_floor: float = 1e-3, seed: int = 42, t: int = 1, nu: int = 0,
             tw: int = 16, th: int = 16, want_tangents: bool = False, lam: float = 0.2, masses: bool = False):
    """Objective, gradient (rows x n) and, if nu > 0, the Hutchinson diagonal (rows x n).
    loss_kind 0: L1, 1: L2, 2: (1 - lam) L1 + lam D-SSIM (res_margin not computed).
    masses: also grad_mass / hz_mass, per entry the sum of the absolute values of
    the terms that form it (the scale its FP32 rounding is measured against),
    for the L1 loss hz_sens, the bound on how far each Hutchinson entry moves
    when each residual moves by its pixel's FP32 rounding bound, and
    grad_allow / hz_allow, how far each entry may move when a decision of its
    Gaussian's own (or, for the L1 gradient, a residual sign) flips in FP32,
    and grad_round / hz_round, the rounding its terms carry under the oracle's
    model of the FP32 records."""
    P = _f64(P)
    rows, n = P.shape
    ca = camera_array(cams)
    V = len(cams)
    H, W = cams[0].height, cams[0].width
    tg = _f64(target)
    grad = np.zeros((rows, n))
    hz = np.zeros((rows, n)) if nu > 0 else None
    it = np.zeros((nu, V, 3, H, W)) if (want_tangents and nu > 0) else None
    rm = np.zeros((V, H, W))
    gm = np.zeros((rows, n)) if masses else None
    hm = np.zeros((rows, n)) if (masses and nu > 0) else None
    hs = np.zeros((rows, n)) if (masses and nu > 0 and loss_kind == 0) else None
    ga = np.zeros((rows, n)) if masses else None
    ha = np.zeros((rows, n)) if (masses and nu > 0) else None
    gr = np.zeros((rows, n)) if masses else None
    hr = np.zeros((rows, n)) if (masses and nu > 0) else None
    if loss_kind == 2:
        f = lib().or_backward_dssim(_p(P), n, n, deg, _p(ca), V, tw, th, _p(tg), lam, gn_floor, seed, t, nu,
                                    _p(grad), _p(hz), _p(it), _p(gm), _p(hm), _p(ga), _p(ha), _p(gr), _p(hr))
        rm = None
    else:
        f = lib().or_backward(_p(P), n, n, deg, _p(ca), V, tw, th, _p(tg), loss_kind, gn_floor, seed, t, nu,
                              _p(grad), _p(hz), _p(it), _p(rm), _p(gm), _p(hm), _p(hs), _p(ga), _p(ha), _p(gr),
                              _p(hr))
    return dict(loss=float(f), grad=grad, hz=hz, image_tangent=it, res_margin=rm, grad_mass=gm, hz_mass=hm,
                hz_sens=hs, grad_allow=ga, hz_allow=ha, grad_round=gr, hz_round=hr)


def ssim(x: np.ndarray, y: np.ndarray):
    """SSIM map of one channel (H x W) and its partials by mx, E[x^2], E[xy]."""
    x, y = _f64(x), _f64(y)
    H, W = x.shape
    out = [np.zeros((H, W)) for _ in range(4)]
    lib().or_ssim(_p(x), _p(y), H, W, *[_p(o) for o in out])
    return tuple(out)


def ssim_vjp(x: np.ndarray, y: np.ndarray, a: np.ndarray) -> np.ndarray:
    x, y, a = _f64(x), _f64(y), _f64(a)
    out = np.zeros_like(x)
    lib().or_ssim_vjp(_p(x), _p(y), x.shape[0], x.shape[1], _p(a), _p(out))
    return out


def ssim_jvp(x: np.ndarray, y: np.ndarray, d: np.ndarray) -> np.ndarray:
    x, y, d = _f64(x), _f64(y), _f64(d)
    out = np.zeros_like(x)
    lib().or_ssim_jvp(_p(x), _p(y), x.shape[0], x.shape[1], _p(d), _p(out))
    return out


def tr_config(theta1=0.9, theta2=0.999, d_floor=1e-12, color_floor=1e-2, l=10, mean_exact=0) -> np.ndarray:
    return np.array([theta1, theta2, d_floor, color_floor, l, mean_exact], np.float64)


def shd_radius(P: np.ndarray, deg: int, eps: float, cfg=None) -> np.ndarray:
    P = _f64(P)
    rows, n = P.shape
    cfg = tr_config() if cfg is None else _f64(cfg)
    eta = np.zeros((rows, n))
    lib().or_shd_radius(_p(P), n, n, deg, eps, _p(cfg), _p(eta))
    return eta


def tr_update(x, g_ema, d_ema, grad, hz, deg: int, t: int, eps: float, cfg=None):
    """Algorithm 1 update for step t; returns new (x, g_ema, d_ema, eta) as float64 copies."""
    x, g, d = _f64(x).copy(), _f64(g_ema).copy(), _f64(d_ema).copy()
    gr = _f64(grad)
    h = None if hz is None else _f64(hz)
    rows, n = x.shape
    cfg = tr_config() if cfg is None else _f64(cfg)
    eta = np.zeros_like(x)
    lib().or_tr_update(_p(x), _p(g), _p(d), _p(gr), _p(h), n, n, deg, _p(cfg), t, eps, _p(eta))
    return x, g, d, eta


def adam_config(beta1=0.9, beta2=0.999, eps_adam=1e-15,
                lr=(1.6e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4)) -> np.ndarray:
    """beta1, beta2, eps_adam and the learning rates of the row groups (mean,
    log-scale, quaternion, opacity logit, SH DC, SH rest)."""
    return np.array([beta1, beta2, eps_adam, *lr], np.float64)


def adam_tr_update(x, m, v, grad, deg: int, t: int, eps: float, cfg=None, adam=None):
    """ADAM-TR update for step t; returns new (x, m, v, eta) as float64 copies."""
    x, m, v = _f64(x).copy(), _f64(m).copy(), _f64(v).copy()
    gr = _f64(grad)
    rows, n = x.shape
    cfg = tr_config() if cfg is None else _f64(cfg)
    adam = adam_config() if adam is None else _f64(adam)
    eta = np.zeros_like(x)
    lib().or_adam_tr_update(_p(x), _p(m), _p(v), _p(gr), n, n, deg, _p(cfg), _p(adam), t, eps, _p(eta))
    return x, m, v, eta


# ------------------------------------------------------------- sampled outputs
def render_pixels(P: np.ndarray, deg: int, cam, xs, ys, *, seed: int = 42, t: int = 1, nu: int = 0,
                  tw: int = 16, th: int = 16, outcomes: int = 0, branch_min: float = 1e-7):
    """Colour, T, n_contrib (and the range the tile sets within rounding allow),
    margin and (nu > 0) image tangents at chosen pixels of one view.

    outcomes > 0: also every result an FP32 blend may reach when the decisions
    within rounding of their thresholds go either way (at most `outcomes` per
    pixel; flips whose bound is at most branch_min are summed instead):
    n_leaves (-1 where there are more), leaf_rgb (k x outcomes x 3), leaf_T,
    leaf_jz (k x outcomes x nu x 3), rest / t_rest (the largest summed bounds).
    The FP64 result is the last leaf of each pixel."""
    P = _f64(P)
    rows, n = P.shape
    xs = np.ascontiguousarray(xs, np.int32)
    ys = np.ascontiguousarray(ys, np.int32)
    k = len(xs)
    rgb = np.zeros((k, 3))
    T = np.zeros(k)
    nc = np.zeros(k, np.int32)
    mg = np.zeros(k)
    jz = np.zeros((k, max(nu, 1), 3))
    rng = np.zeros((k, 2), np.int32)
    imp = np.zeros(k)
    timp = np.zeros(k)
    kinds = np.zeros(k, np.int32)
    L = max(int(outcomes), 1)
    nl = np.zeros(k, np.int32)
    lrgb = np.zeros((k, L, 3))
    lT = np.zeros((k, L))
    ljz = np.zeros((k, L, max(nu, 1), 3))
    rest = np.zeros(k)
    trest = np.zeros(k)
    want = outcomes > 0
    lib().or_render_pixels(_p(P), n, n, deg, _p(camera_array([cam])), tw, th, k, _p(xs), _p(ys), seed, t, nu,
                           _p(rgb), _p(T), _p(nc), _p(mg), _p(jz), _p(rng), _p(imp), _p(timp), _p(kinds), L,
                           float(branch_min), _p(nl) if want else None, _p(lrgb), _p(lT), _p(ljz), _p(rest),
                           _p(trest))
    out = dict(rgb=rgb, final_T=T, n_contrib=nc, margin=mg, jz=jz[:, :nu], n_contrib_lo=rng[:, 0],
               n_contrib_hi=rng[:, 1], impact=imp, t_impact=timp, flip_kinds=kinds)
    if want:
        out.update(n_leaves=nl, leaf_rgb=lrgb, leaf_T=lT, leaf_jz=ljz[:, :, :nu], rest=rest, t_rest=trest)
    return out


def match_outcomes(ref: dict, rgb, final_T, jz=None, *, img_tol: float = 1e-5, jz_tol=None,
                   flip_max: float = 5e-6):
    """Which sampled pixels of an FP32 evaluation equal one of the oracle's
    outcomes (render_pixels with outcomes > 0).

    rgb (k x 3), final_T (k), jz (k x nu x 3, optional, with jz_tol a bound per
    probe).  A pixel is resolved when its outcomes are complete and the flips
    summed instead of enumerated are bounded by flip_max (colour and T); it
    matches when one outcome is within img_tol in colour and T (and jz_tol in
    the tangents).  Returns (resolved, matched, leaf): leaf is the index of the
    first matching outcome, -1 where none; the FP64 result is the last one."""
    nl = ref["n_leaves"]
    resolved = (nl > 0) & (ref["rest"] <= flip_max) & (ref["t_rest"] <= flip_max)
    k, L = ref["leaf_T"].shape
    valid = np.arange(L)[None, :] < nl[:, None]
    ok = np.abs(ref["leaf_rgb"] - np.asarray(rgb)[:, None, :]).max(axis=2) <= img_tol
    ok &= np.abs(ref["leaf_T"] - np.asarray(final_T)[:, None]) <= img_tol
    if jz is not None:
        tol = np.broadcast_to(np.asarray(jz_tol, np.float64), (ref["leaf_jz"].shape[2],))
        ok &= (np.abs(ref["leaf_jz"] - np.asarray(jz)[:, None]) <= tol[None, None, :, None]).all(axis=(2, 3))
    ok &= valid
    matched = ok.any(axis=1)
    leaf = np.where(matched, ok.argmax(axis=1), -1)
    return resolved, matched, leaf


def backward_sampled(P: np.ndarray, deg: int, cams, target: np.ndarray, samples, *, loss_kind: int = 0,
                     gn_floor: float = 1e-3, seed: int = 42, t: int = 1, nu: int = 0, tw: int = 16, th: int = 16,
                     eps_img: float = 1e-5):
    """Gradient and Hutchinson rows of chosen Gaussians over a full frame of views,
    with comparability flags, the masses of the entries' sums (grad_mass,
    hz_mass) and hz_sens, the largest change of each Hutchinson entry when each
    residual moves by the FP32 rounding bound of its pixel's colour (capped at
    eps_img), and grad_allow / hz_allow, how far each entry may move when a
    decision of the sample's own (or a residual sign, for the gradient) flips in
    FP32 somewhere in its footprint, and grad_round / hz_round, the rounding its
    terms carry under the oracle's model of the FP32 records.  eps_img: the
    image tolerance."""
    P = _f64(P)
    rows, n = P.shape
    tg = _f64(target)
    smp = np.ascontiguousarray(samples, np.int64)
    k = len(smp)
    grad = np.zeros((k, rows))
    hz = np.zeros((k, rows))
    flag = np.zeros(k, np.int32)
    gm, hm, hs, ga, ha, gr, hr = (np.zeros((k, rows)) for _ in range(7))
    h = (lambda a: a) if nu > 0 else (lambda a: None)
    lib().or_backward_sampled(_p(P), n, n, deg, _p(camera_array(cams)), len(cams), tw, th, _p(tg), loss_kind,
                              gn_floor, seed, t, nu, k, _p(smp), _p(grad), _p(h(hz)), _p(flag), eps_img, _p(gm),
                              _p(h(hm)), _p(h(hs)), _p(ga), _p(h(ha)), _p(gr), _p(h(hr)))
    return dict(grad=grad, hz=h(hz), flag=flag, grad_mass=gm, hz_mass=h(hm), hz_sens=h(hs), grad_allow=ga,
                hz_allow=h(ha), grad_round=gr, hz_round=h(hr))
