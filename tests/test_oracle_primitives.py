"""Pins of the oracle's primitives against facts fixed outside the oracle.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand) fails it: published outputs of
SplitMix64, scipy's rotation matrices and spherical harmonics, closed-form
maxima, 3-D quadrature of the Hellinger integral, finite differences of the
rotation trace, and the Taylor ratios of the trust-region bounds.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy import special

import oracle as O


# ------------------------------------------------------------------- RNG
def test_splitmix64_published_sequence():
    # SplitMix64 seeded with 0: first outputs as published with the reference
    # implementation (Vigna, splitmix64.c); state advances by the golden gamma.
    gamma = 0x9E3779B97F4A7C15
    expected = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [O.splitmix64((k * gamma) & 0xFFFFFFFFFFFFFFFF) for k in range(3)]
    assert got == expected


def test_rademacher_balanced_and_independent_of_probe():
    z0 = np.array([O.rademacher(42, 3, 0, j) for j in range(20000)])
    z1 = np.array([O.rademacher(42, 3, 1, j) for j in range(20000)])
    z2 = np.array([O.rademacher(42, 4, 0, j) for j in range(20000)])
    for z in (z0, z1, z2):
        assert set(np.unique(z)) == {-1.0, 1.0}
        assert abs(z.mean()) < 4 / math.sqrt(len(z))
    # distinct probes and steps are uncorrelated
    assert abs((z0 * z1).mean()) < 4 / math.sqrt(len(z0))
    assert abs((z0 * z2).mean()) < 4 / math.sqrt(len(z0))


# -------------------------------------------------------------- rotation
def test_rotation_matches_scipy_and_is_orthonormal():
    rng = np.random.default_rng(0)
    for _ in range(50):
        q = rng.normal(size=4) * rng.uniform(0.2, 3.0)
        R = O.quat_to_rotmat(q)
        Rs = Rotation.from_quat(q / np.linalg.norm(q)).as_matrix()  # scalar-last (x, y, z, w)
        np.testing.assert_allclose(R, Rs, atol=1e-13)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(R) - 1.0) < 1e-13


# ------------------------------------------------------------------- SH
def _real_sh_scipy(l, m, theta, phi):
    """Real SH from scipy's complex Y_l^m (orthonormal, Condon-Shortley phase)."""
    if m == 0:
        return special.sph_harm_y(l, 0, theta, phi).real
    Y = special.sph_harm_y(l, abs(m), theta, phi)
    if m > 0:
        return math.sqrt(2) * (-1) ** m * Y.real
    return math.sqrt(2) * (-1) ** m * Y.imag


def test_sh_basis_matches_scipy_up_to_fixed_signs():
    rng = np.random.default_rng(1)
    dirs = rng.normal(size=(200, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    ours = np.array([O.sh_basis(3, d) for d in dirs])  # [200, 16]
    theta = np.arccos(np.clip(dirs[:, 2], -1, 1))
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            ref = np.array([_real_sh_scipy(l, m, th, ph) for th, ph in zip(theta, phi)])
            # one sign per basis function, the same for every direction
            s = np.sign(np.dot(ours[:, k], ref))
            assert s != 0
            np.testing.assert_allclose(ours[:, k], s * ref, atol=1e-12, err_msg=f"k={k} l={l} m={m}")
            k += 1


def test_sh_absmax_closed_forms():
    # max over the unit sphere of |Y_k|, derived by hand from each polynomial:
    c0 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3 / (4 * math.pi))
    c2a, c2b, c2c = 0.5 * math.sqrt(15 / math.pi), 0.25 * math.sqrt(5 / math.pi), 0.25 * math.sqrt(15 / math.pi)
    c3a, c3b = 0.25 * math.sqrt(35 / (2 * math.pi)), 0.5 * math.sqrt(105 / math.pi)
    c3c, c3d, c3e = 0.25 * math.sqrt(21 / (2 * math.pi)), 0.25 * math.sqrt(7 / math.pi), 0.25 * math.sqrt(105 / math.pi)
    expected = [
        c0,
        c1, c1, c1,
        c2a / 2, c2a / 2, 2 * c2b, c2a / 2, c2c,        # |xy|<=1/2, |3z^2-1|<=2, |x^2-y^2|<=1
        c3a, c3b / (3 * math.sqrt(3)),                   # rho^3 sin 3phi <= 1; |xyz| <= 3^-3/2
        c3c * 16 / math.sqrt(135),                       # sqrt(1-z^2)|5z^2-1| max at z^2 = 11/15
        2 * c3d,                                         # |z(5z^2-3)| <= 2
        c3c * 16 / math.sqrt(135),
        c3e * 2 / (3 * math.sqrt(3)),                    # |z|(1-z^2) <= 2/(3 sqrt 3)
        c3a,
    ]
    np.testing.assert_allclose(O.sh_absmax(3), expected, rtol=1e-9)


# -------------------------------------------------------------- Hellinger
def _gauss_density(pts, mu, S):
    d = pts - mu
    Si = np.linalg.inv(S)
    q = np.einsum("...i,ij,...j->...", d, Si, d)
    return np.exp(-0.5 * q) / math.sqrt((2 * math.pi) ** 3 * np.linalg.det(S))


def _rand_spd(rng, scale):
    A = rng.normal(size=(3, 3))
    Q, _ = np.linalg.qr(A)
    return Q @ np.diag(rng.uniform(0.3, 1.0, 3) * scale) ** 2 @ Q.T


def test_hellinger_closed_form_matches_quadrature():
    rng = np.random.default_rng(3)
    g = np.linspace(-3.0, 3.0, 121)
    h = g[1] - g[0]
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X, Y, Z], -1)
    for _ in range(4):
        S1, S2 = _rand_spd(rng, 0.5), _rand_spd(rng, 0.5)
        mu1, mu2 = rng.normal(0, 0.2, 3), rng.normal(0, 0.2, 3)
        Z1, Z2 = rng.uniform(0.3, 2.0, 2)
        G1 = Z1 * _gauss_density(pts, mu1, S1)
        G2 = Z2 * _gauss_density(pts, mu2, S2)
        quad = 0.5 * np.sum((np.sqrt(G1) - np.sqrt(G2)) ** 2) * h ** 3
        closed = O.hellinger(mu1, S1.ravel(), Z1, mu2, S2.ravel(), Z2)
        assert abs(closed - quad) < 2e-4 * max(Z1, Z2), (closed, quad)


def test_hellinger_invariants():
    rng = np.random.default_rng(4)
    for _ in range(20):
        S1, S2 = _rand_spd(rng, 1.0), _rand_spd(rng, 1.0)
        mu1, mu2 = rng.normal(size=3), rng.normal(size=3)
        assert abs(O.hellinger(mu1, S1.ravel(), 1.3, mu1, S1.ravel(), 1.3)) < 1e-14
        a = O.hellinger(mu1, S1.ravel(), 1.0, mu2, S2.ravel(), 1.0)
        b = O.hellinger(mu2, S2.ravel(), 1.0, mu1, S1.ravel(), 1.0)
        assert abs(a - b) < 1e-14
        assert 0.0 <= a <= 1.0


# ----------------------------------------------------------- rotation beta
def _trace_T(q, s, c, a):
    R0 = Rotation.from_quat(q / np.linalg.norm(q)).as_matrix()
    q2 = q.copy()
    q2[c] += a
    R1 = Rotation.from_quat(q2 / np.linalg.norm(q2)).as_matrix()
    dR = R0.T @ R1
    S2 = np.diag(s ** 2)
    return np.trace(np.linalg.inv(S2) @ dR @ S2 @ dR.T)


def test_rotation_beta_matches_second_difference_of_trace():
    rng = np.random.default_rng(5)
    for _ in range(10):
        q = rng.normal(size=4) * rng.uniform(0.5, 2.0)
        s = np.exp(rng.normal(-3, 0.7, 3))
        beta = O.rotation_beta(q, s)
        for c in range(4):
            a = 1e-4 * np.linalg.norm(q)
            fd = (_trace_T(q, s, c, a) - 2 * _trace_T(q, s, c, 0.0) + _trace_T(q, s, c, -a)) / a ** 2
            assert abs(fd - beta[c]) <= 1e-5 * max(abs(beta).max(), 1e-12) + 1e-6, (c, fd, beta[c])


def test_rotation_beta_zero_for_isotropic():
    q = np.array([0.3, -0.4, 0.5, 0.7])
    np.testing.assert_allclose(O.rotation_beta(q, np.array([0.2, 0.2, 0.2])), 0.0, atol=1e-12)


# ---------------------------------------------------- trust-region radii
def _gauss_of(P, i, deg):
    mu = P[0:3, i]
    s = np.exp(P[3:6, i])
    R = Rotation.from_quat(P[6:10, i] / np.linalg.norm(P[6:10, i])).as_matrix()
    S = R @ np.diag(s ** 2) @ R.T
    alpha = 1 / (1 + math.exp(-P[10, i]))
    return mu, S, alpha, np.prod(s)


def _normalised_h2(P0, P1, i, deg, colour_channel=None):
    """H^2(G, G') / det(S) with mass alpha det(Sigma)^1/2 (times the DC colour for colour moves)."""
    mu0, S0, a0, dS0 = _gauss_of(P0, i, deg)
    mu1, S1, a1, dS1 = _gauss_of(P1, i, deg)
    Z0 = a0 * math.sqrt(np.linalg.det(S0))
    Z1 = a1 * math.sqrt(np.linalg.det(S1))
    if colour_channel is not None:
        c0 = 0.5 / math.sqrt(math.pi)
        Z0 *= c0 * P0[11 + colour_channel, i] + 0.5
        Z1 *= c0 * P1[11 + colour_channel, i] + 0.5
    return O.hellinger(mu0, S0.ravel(), Z0, mu1, S1.ravel(), Z1) / dS0


def _one_gaussian(seed=6, axis_aligned=False):
    rng = np.random.default_rng(seed)
    P = np.zeros((14, 1))
    P[0:3, 0] = rng.normal(size=3)
    P[3:6, 0] = [-2.5, -3.1, -2.0]
    q = rng.normal(size=4)
    P[6:10, 0] = [0, 0, 0, 1.0] if axis_aligned else q / np.linalg.norm(q) * 1.7
    P[10, 0] = 0.4
    P[11:14, 0] = [0.6, 0.2, -0.3]
    return P


@pytest.mark.parametrize("what,row,ratio", [
    ("scale", 3, 0.75), ("scale", 5, 0.75),
    ("opacity", 10, 0.5),
    ("colour", 11, 0.5), ("colour", 13, 0.5),
    ("rotation", 6, 0.5), ("rotation", 7, 0.5), ("rotation", 8, 0.5), ("rotation", 9, 0.5),
])
def test_radius_taylor_ratios(what, row, ratio):
    """At |step| = eta the normalised H^2 equals ratio * eps as eps -> 0 (Appendix B)."""
    eps = 1e-9
    P = _one_gaussian()
    eta = O.shd_radius(P, 0, eps)
    for sgn in (+1, -1):
        P1 = P.copy()
        P1[row, 0] += sgn * eta[row, 0]
        ch = (row - 11) % 3 if what == "colour" else None
        r = _normalised_h2(P, P1, 0, 0, ch) / eps
        assert abs(r - ratio) < 2e-3, (what, row, sgn, r)


def test_mean_radius_exact_on_axis_aligned_covariance():
    eps = 1e-7
    P = _one_gaussian(axis_aligned=True)
    for exact in (0, 1):
        eta = O.shd_radius(P, 0, eps, O.tr_config(mean_exact=exact))
        for c in range(3):
            P1 = P.copy()
            P1[c, 0] += eta[c, 0]
            assert abs(_normalised_h2(P, P1, 0, 0) / eps - 1.0) < 1e-6


def test_mean_radius_paper_vs_exact_on_rotated_covariance():
    eps = 1e-7
    P = _one_gaussian()
    eta_exact = O.shd_radius(P, 0, eps, O.tr_config(mean_exact=1))
    eta_paper = O.shd_radius(P, 0, eps, O.tr_config(mean_exact=0))
    ratios = []
    for c in range(3):
        P1 = P.copy()
        P1[c, 0] += eta_exact[c, 0]
        assert abs(_normalised_h2(P, P1, 0, 0) / eps - 1.0) < 1e-6
        P2 = P.copy()
        P2[c, 0] += eta_paper[c, 0]
        ratios.append(_normalised_h2(P, P2, 0, 0) / eps)
    # the printed bound uses Sigma_cc where 1/(Sigma^-1)_cc is exact; Sigma_cc >= 1/(Sigma^-1)_cc
    assert all(r >= 1.0 - 1e-9 for r in ratios) and max(ratios) > 1.0


def test_radius_infinite_when_alpha_below_eps():
    P = _one_gaussian()
    P[10, 0] = -12.0  # alpha ~ 6e-6
    eta = O.shd_radius(P, 0, 1e-4)
    assert np.all(np.isinf(eta[0:3, 0])) and np.all(np.isinf(eta[6:10, 0]))
    assert np.all(np.isfinite(eta[3:6, 0])) and np.isfinite(eta[10, 0])


# ----------------------------------------------------------- TR update
def test_update_is_exact_newton_on_separable_quadratic():
    """f = 1/2 sum h_j (x_j - x*_j)^2: with theta1 = theta2 = 0 and no clipping
    (eps >> alpha), one step lands on x* (Algorithm 1 with exact z.Hz = h)."""
    rng = np.random.default_rng(8)
    n, deg = 7, 0
    x = rng.normal(size=(14, n))
    x[10] = -6.0  # alpha ~ 2.5e-3, far below eps: mean/rotation radii unbounded
    xs = x + rng.normal(0, 1e-3, size=x.shape)
    xs[10] = x[10]
    h = rng.uniform(0.5, 2.0, size=x.shape)
    g = h * (x - xs)
    cfg = O.tr_config(theta1=0.0, theta2=0.0, l=1)
    x1, ge, de, eta = O.tr_update(x, np.zeros_like(x), np.zeros_like(x), g, h, deg, t=1, eps=10.0, cfg=cfg)
    assert np.all(eta > 1e-2)
    np.testing.assert_allclose(x1, xs, rtol=0, atol=1e-12)


def test_update_ema_interval_and_clip():
    rng = np.random.default_rng(9)
    n, deg = 5, 0
    x = rng.normal(size=(14, n))
    g = rng.normal(size=x.shape)
    hz = rng.uniform(1.0, 2.0, size=x.shape)
    cfg = O.tr_config(theta1=0.9, theta2=0.999, l=3)
    ge0 = rng.normal(size=x.shape)
    de0 = rng.uniform(0.1, 1.0, size=x.shape)
    eps = 1e-6
    for t, upd in ((1, True), (2, False), (3, False), (4, True)):
        x1, ge, de, eta = O.tr_update(x, ge0, de0, g, hz, deg, t=t, eps=eps, cfg=cfg)
        np.testing.assert_allclose(ge, 0.9 * ge0 + 0.1 * g, rtol=1e-15)
        np.testing.assert_allclose(de, 0.999 * de0 + 0.001 * hz if upd else de0, rtol=1e-15)
        step = np.clip(-ge / np.maximum(de, 1e-12), -eta, eta)
        np.testing.assert_allclose(x1 - x, step, atol=1e-15)
        np.testing.assert_allclose(eta, O.shd_radius(x, deg, eps, cfg), rtol=1e-15)


def test_update_vanishes_as_eps_goes_to_zero():
    rng = np.random.default_rng(10)
    x = rng.normal(size=(14, 6))
    g = rng.normal(size=x.shape) * 1e3
    hz = np.full(x.shape, 1e-3)
    steps = []
    for eps in (1e-6, 1e-8, 1e-10, 1e-12):
        x1, *_ = O.tr_update(x, np.zeros_like(x), np.zeros_like(x), g, hz, 0, t=1, eps=eps)
        steps.append(np.abs(x1 - x).max())
    assert all(b < a for a, b in zip(steps, steps[1:]))
    assert steps[-1] < 1e-4
