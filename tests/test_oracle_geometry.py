"""Pins of the oracle's sphere geometry (Sec. 3.1, App. A) against facts that
do not depend on the oracle: orthonormality, the geodesic-distance property of
the azimuthal equidistant chart, finite differences, numpy's sinc and
Cholesky."""
import math

import numpy as np
import pytest


def _random_units(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    # include the poles and near-antipodal frames of the basis construction
    extra = np.array([[0, 0, 1.0], [0, 0, -1.0], [1.0, 0, 0], [0, 1.0, 0],
                      [1e-9, 0, -1.0], [0, 1e-7, -1.0]])
    extra /= np.linalg.norm(extra, axis=1, keepdims=True)
    return np.concatenate([v, extra])


def test_basis_is_rotation_taking_mu_to_z(orc):
    for mu in _random_units(200, 1):
        R = orc.basis(mu)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-13
        assert np.allclose(R @ mu, [0, 0, 1], atol=1e-14)


def test_sinc_matches_numpy(orc):
    for r in [0.0, 1e-9, 1e-5, 9.9e-5, 1e-4, 0.3, 1.0, 2.5, math.pi - 1e-9]:
        # numpy's sinc is the normalised one: sinc(x) = sin(pi x)/(pi x)
        assert abs(orc.sinc(r) - np.sinc(r / math.pi)) < 1e-15


def test_log_length_is_geodesic_distance(orc):
    """|log_mu(w)| equals the great-circle angle between mu and w (Sec. 3.1)."""
    mus = _random_units(50, 2)
    ws = _random_units(50, 3)
    for mu in mus:
        for w in ws:
            nu, anti, th, _ = orc.log_map(mu, w)
            if anti:
                continue
            ang = math.acos(max(-1.0, min(1.0, float(np.dot(mu, w)))))
            # acos loses accuracy near 0 and pi, compare through the chord too
            chord = np.linalg.norm(mu - w)
            assert abs(np.linalg.norm(nu) - ang) < 1e-7
            assert abs(2 * math.sin(np.linalg.norm(nu) / 2) - chord) < 1e-14


def test_exp_log_round_trip(orc):
    rng = np.random.default_rng(4)
    for mu in _random_units(100, 5):
        w = rng.normal(size=3)
        w /= np.linalg.norm(w)
        nu, anti, _, _ = orc.log_map(mu, w)
        assert not anti
        assert np.allclose(orc.exp_map(mu, nu), w, atol=2e-15)
        # and the other way round, inside the injectivity radius
        r = rng.uniform(0, math.pi - 1e-3)
        phi = rng.uniform(0, 2 * math.pi)
        nu = np.array([r * math.cos(phi), r * math.sin(phi)])
        nu2, anti, _, _ = orc.log_map(mu, orc.exp_map(mu, nu))
        assert not anti
        assert np.allclose(nu2, nu, atol=1e-12)


def test_exp_traces_geodesic(orc):
    """exp_mu(t e) stays at angle t from mu, on one great circle."""
    for mu in _random_units(20, 6):
        e = np.array([0.6, -0.8])
        pts = np.array([orc.exp_map(mu, t * e) for t in np.linspace(0.0, 3.0, 13)])
        assert np.allclose(pts @ mu, np.cos(np.linspace(0.0, 3.0, 13)), atol=1e-14)
        # all points lie in the plane spanned by mu and the first step
        n = np.cross(mu, pts[1])
        n /= np.linalg.norm(n)
        assert np.allclose(pts @ n, 0.0, atol=1e-14)


def test_log_map_antipode_flag(orc):
    mu = np.array([0.0, 0.6, 0.8])
    _, anti, th, _ = orc.log_map(mu, -mu)
    assert anti and abs(th - math.pi) < 1e-15
    nu, anti, th, _ = orc.log_map(mu, mu)
    assert not anti and th == 0.0 and np.all(nu == 0.0)


def _fd_jexp(orc, mu, nu, h=1e-6):
    J = np.zeros((3, 2))
    for c in range(2):
        e = np.zeros(2)
        e[c] = h
        J[:, c] = (orc.exp_map(mu, nu + e) - orc.exp_map(mu, nu - e)) / (2 * h)
    return J


def test_jexp_matches_finite_differences(orc):
    rng = np.random.default_rng(7)
    for mu in _random_units(40, 8):
        for r in [0.0, 1e-5, 5e-3, 0.2, 1.0, 2.5]:
            phi = rng.uniform(0, 2 * math.pi)
            nu = r * np.array([math.cos(phi), math.sin(phi)])
            assert np.allclose(orc.jexp(mu, nu), _fd_jexp(orc, mu, nu), atol=2e-9)


def test_printed_jexp_would_fail_finite_differences(orc):
    """App. A's printed J_exp (extra sinc in entry (1,2), missing square in
    (2,2)) disagrees with differentiation of Eq. (exp); this pins the reading
    that the corrected form is the intended one."""
    mu = np.array([0.0, 0.0, 1.0])
    nu = np.array([0.7, -0.4])
    r = np.linalg.norm(nu)
    s = math.sin(r) / r
    c = (math.cos(r) - s) / r ** 2
    printed = np.array([[s + nu[0] ** 2 * c, s + nu[0] * nu[1] * c],
                        [s + nu[1] * nu[0] * c, s + nu[1] * c],
                        [-nu[0] * s, -nu[1] * s]])
    R = orc.basis(mu)
    fd = _fd_jexp(orc, mu, nu)
    assert np.abs(R.T @ printed - fd).max() > 0.1
    assert np.allclose(orc.jexp(mu, nu), fd, atol=1e-9)


def test_jlog_inverts_jexp_on_tangent_plane(orc):
    rng = np.random.default_rng(9)
    for mu in _random_units(40, 10):
        for r in [1e-6, 1e-2, 0.4, 1.5, 2.8]:
            phi = rng.uniform(0, 2 * math.pi)
            nu = r * np.array([math.cos(phi), math.sin(phi)])
            w = orc.exp_map(mu, nu)
            assert np.allclose(orc.jlog(mu, w) @ orc.jexp(mu, nu), np.eye(2), atol=1e-9)
            # finite differences of log along the sphere
            for c in range(2):
                e = np.zeros(2)
                e[c] = 1e-6
                a, _, _, _ = orc.log_map(mu, orc.exp_map(mu, nu + e))
                b, _, _, _ = orc.log_map(mu, orc.exp_map(mu, nu - e))
                assert np.allclose((a - b) / 2e-6, e / 1e-6, atol=1e-8)


def test_jlog_at_centre_is_projection(orc):
    for mu in _random_units(20, 11):
        R = orc.basis(mu)
        assert np.allclose(orc.jlog(mu, mu), R[:2], atol=1e-15)


def test_cholesky5_matches_numpy(orc):
    rng = np.random.default_rng(12)
    idx = [(i, j) for i in range(5) for j in range(i + 1)]
    for _ in range(50):
        A = rng.normal(size=(5, 5))
        S = A @ A.T + 0.1 * np.eye(5)
        L, bad = orc.cholesky5(np.array([S[i, j] for i, j in idx]))
        assert not bad
        Ln = np.linalg.cholesky(S)
        assert np.allclose(L, [Ln[i, j] for i, j in idx], rtol=1e-12, atol=1e-13)
    S = np.diag([1.0, 1.0, -1e-3, 1.0, 1.0])
    _, bad = orc.cholesky5(np.array([S[i, j] for i, j in idx]))
    assert bad
