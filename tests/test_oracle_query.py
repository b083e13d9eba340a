"""Pins of the oracle's query side (conditioning, pdf, sampling; Sec. 3.1-3.3)
against the textbook Gaussian conditional, quadrature over the sphere and the
plane, a chi-square test and a closed-form integral."""
import math

import numpy as np
import pytest
from scipy import stats

PK = [(i, j) for i in range(5) for j in range(i + 1)]


def _unpack(Lp):
    L = np.zeros((5, 5))
    for p, (i, j) in enumerate(PK):
        L[i, j] = Lp[p]
    return L


def _mixture(seed, K, dir_sd=(0.3, 0.9), cross=0.4):
    rng = np.random.default_rng(seed)
    pi = rng.dirichlet(np.ones(K))
    mu_x = rng.uniform(0.3, 0.7, size=(K, 3))
    mu_w = rng.normal(size=(K, 3))
    mu_w /= np.linalg.norm(mu_w, axis=1, keepdims=True)
    L = np.zeros((K, 15))
    for k in range(K):
        diag = np.concatenate([rng.uniform(0.05, 0.2, 3), rng.uniform(*dir_sd, 2)])
        for p, (i, j) in enumerate(PK):
            L[k, p] = diag[i] if i == j else cross * rng.normal() * diag[i]
    return pi, mu_x, mu_w, L


def test_condition_matches_dense_textbook_conditional(orc):
    K = 5
    pi, mu_x, mu_w, L = _mixture(1, K)
    rng = np.random.default_rng(2)
    qx = rng.uniform(0.3, 0.7, size=(20, 3)).astype(np.float32)
    region = np.zeros(20, dtype=np.int32)
    cpi, cm, cL = orc.condition(K, pi[None], mu_x[None], mu_w[None], L[None], qx, region)
    for q in range(20):
        x = qx[q].astype(np.float64)
        wts = np.zeros(K)
        for k in range(K):
            Lk = _unpack(L[k])
            S = Lk @ Lk.T
            Sxx, Svx, Svv = S[:3, :3], S[3:, :3], S[3:, 3:]
            m = Svx @ np.linalg.solve(Sxx, x - mu_x[k])
            C = Svv - Svx @ np.linalg.solve(Sxx, Svx.T)
            wts[k] = pi[k] * stats.multivariate_normal(mu_x[k], Sxx).pdf(x)
            assert np.allclose(cm[q, k], m, rtol=1e-10, atol=1e-12)
            D = np.array([[cL[q, k, 0], 0.0], [cL[q, k, 1], cL[q, k, 2]]])
            assert np.allclose(D @ D.T, C, rtol=1e-10, atol=1e-14)
        assert np.allclose(cpi[q], wts / wts.sum(), rtol=1e-9, atol=1e-15)


def _disk_mass(m, C, n_r=160, n_phi=320):
    """P(|nu| < pi) for nu ~ N(m, C), by polar quadrature on the plane."""
    xr, wr = np.polynomial.legendre.leggauss(n_r)
    rho = (xr + 1) * math.pi / 2
    wr = wr * math.pi / 2
    phi = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    P = np.stack([np.outer(rho, np.cos(phi)), np.outer(rho, np.sin(phi))], -1)
    dens = stats.multivariate_normal(m, C).pdf(P.reshape(-1, 2)).reshape(n_r, n_phi)
    return float(np.sum(dens * rho[:, None] * wr[:, None]) * 2 * math.pi / n_phi)


def _polar_grid(axis, n_a, n_phi):
    """Quadrature nodes/weights over the sphere in polar angle alpha around
    `axis` (Gauss-Legendre in alpha with the sin(alpha) area factor), so that a
    1/(pi - theta) singularity at the pole is integrated smoothly."""
    xa, wa = np.polynomial.legendre.leggauss(n_a)
    al = (xa + 1) * math.pi / 2
    wa = wa * math.pi / 2 * np.sin(al)
    phi = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    t = np.cross(axis, [1.0, 0, 0] if abs(axis[0]) < 0.9 else [0, 1.0, 0])
    t /= np.linalg.norm(t)
    b = np.cross(axis, t)
    A = np.repeat(al, n_phi)
    P = np.tile(phi, n_a)
    dirs = (np.cos(A)[:, None] * axis + (np.sin(A) * np.cos(P))[:, None] * t
            + (np.sin(A) * np.sin(P))[:, None] * b)
    return dirs, np.repeat(wa, n_phi) * 2 * math.pi / n_phi


def test_pdf_integrates_to_in_disk_mass(orc):
    """The solid-angle pdf (p^t / sinc, Sec. 3.1) integrates over the sphere to
    the conditioned mixture's planar mass inside |nu| < pi (computed on the
    plane); the paper's literal p^t * sinc would not."""
    K = 3
    pi, mu_x, mu_w, L = _mixture(3, K, dir_sd=(0.6, 1.3))
    x = np.array([0.5, 0.45, 0.55], dtype=np.float32)
    cpi, cm, cL = orc.condition(K, pi[None], mu_x[None], mu_w[None], L[None], x[None],
                                np.zeros(1, np.int32))
    expected, total, literal = 0.0, 0.0, 0.0
    for k in range(K):
        D = np.array([[cL[0, k, 0], 0.0], [cL[0, k, 1], cL[0, k, 2]]])
        expected += cpi[0, k] * _disk_mass(cm[0, k], D @ D.T)
        # component k alone (its conditional is the same with weight 1),
        # integrated on a grid whose pole is its antipode
        dirs, wts = _polar_grid(-mu_w[k], 700, 1400)
        Q = dirs.shape[0]
        one = (np.ones((1, 1)), mu_x[None, k:k + 1], mu_w[None, k:k + 1], L[None, k:k + 1])
        p = orc.pdf(1, *one, np.repeat(x[None], Q, 0), np.zeros(Q, np.int32), dirs)
        total += cpi[0, k] * float(np.sum(p * wts))
        th = np.arccos(np.clip(dirs @ mu_w[k], -1, 1))
        literal += cpi[0, k] * float(np.sum(p * np.sinc(th / math.pi) ** 2 * wts))
    assert 0.9 < expected < 0.999          # the lobes are wide enough to matter
    assert abs(total - expected) < 1e-6, (total, expected)
    assert abs(literal - expected) > 0.05
    # the mixture pdf is the weighted sum of the conditioned components
    dirs, _ = _polar_grid([0.3, -0.2, 0.9], 20, 40)
    Q = dirs.shape[0]
    pm = orc.pdf(K, pi[None], mu_x[None], mu_w[None], L[None], np.repeat(x[None], Q, 0),
                 np.zeros(Q, np.int32), dirs)
    parts = sum(cpi[0, k] * orc.pdf(1, np.ones((1, 1)), mu_x[None, k:k + 1], mu_w[None, k:k + 1],
                                    L[None, k:k + 1], np.repeat(x[None], Q, 0),
                                    np.zeros(Q, np.int32), dirs) for k in range(K))
    assert np.allclose(pm, parts, rtol=1e-12)


def _equal_area_bins(dirs, n_z, n_phi):
    z = np.clip(dirs[:, 2], -1, 1)
    iz = np.minimum(((z + 1) / 2 * n_z).astype(int), n_z - 1)
    ph = np.mod(np.arctan2(dirs[:, 1], dirs[:, 0]), 2 * math.pi)
    ip = np.minimum((ph / (2 * math.pi) * n_phi).astype(int), n_phi - 1)
    return iz * n_phi + ip


def _bin_masses(orc, K, params, x, n_z, n_phi, sub=6):
    """Integral of the pdf over each equal-area bin (Gauss-Legendre in z and phi)."""
    xs, ws = np.polynomial.legendre.leggauss(sub)
    out = np.zeros(n_z * n_phi)
    zs = []
    for iz in range(n_z):
        z0, z1 = -1 + 2 * iz / n_z, -1 + 2 * (iz + 1) / n_z
        for ip in range(n_phi):
            p0, p1 = 2 * math.pi * ip / n_phi, 2 * math.pi * (ip + 1) / n_phi
            z = (xs + 1) / 2 * (z1 - z0) + z0
            p = (xs + 1) / 2 * (p1 - p0) + p0
            Z, P = np.meshgrid(z, p, indexing="ij")
            W = np.outer(ws, ws) * (z1 - z0) / 2 * (p1 - p0) / 2
            s = np.sqrt(1 - Z * Z)
            zs.append((np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3), W.reshape(-1)))
    dirs = np.concatenate([d for d, _ in zs])
    wts = np.concatenate([w for _, w in zs])
    Q = dirs.shape[0]
    p = orc.pdf(K, *params, np.repeat(x[None], Q, 0), np.zeros(Q, np.int32), dirs)
    return (p * wts).reshape(n_z * n_phi, -1).sum(1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sample_histogram_chi_square(orc, seed):
    K = 3
    pi, mu_x, mu_w, L = _mixture(10 + seed, K, dir_sd=(0.4, 1.1))
    params = (pi[None], mu_x[None], mu_w[None], L[None])
    x = np.array([0.5, 0.5, 0.5], dtype=np.float32)
    N = 200_000
    u = np.random.default_rng(100 + seed).random((N, 3), dtype=np.float32)
    out = orc.sample(K, *params, np.repeat(x[None], N, 0), np.zeros(N, np.int32), u)
    n_z, n_phi = 16, 32
    mass = _bin_masses(orc, K, params, x, n_z, n_phi)
    valid = out["valid"].astype(bool)
    counts = np.bincount(_equal_area_bins(out["dir"][valid], n_z, n_phi), minlength=n_z * n_phi)
    obs = np.append(counts, (~valid).sum()).astype(float)
    exp = np.append(mass, 1.0 - mass.sum()) * N
    # merge sparse bins into one
    small = exp < 5
    obs = np.append(obs[~small], obs[small].sum())
    exp = np.append(exp[~small], exp[small].sum())
    if exp[-1] == 0:
        obs, exp = obs[:-1], exp[:-1]
    chi2 = float(np.sum((obs - exp) ** 2 / exp))
    pval = stats.chi2.sf(chi2, obs.size - 1)
    assert pval > 1e-3, (chi2, obs.size, pval)


def test_sampling_estimator_unbiased(orc):
    """E[1_valid f(w)/p(w)] = int f dw; f(w) = exp(k (a.w - 1)) integrates to
    2 pi (1 - e^{-2k}) / k.  Discarded samples count as zero (Sec. 3.1)."""
    K = 4
    pi, mu_x, mu_w, L = _mixture(20, K, dir_sd=(0.5, 1.0))
    params = (pi[None], mu_x[None], mu_w[None], L[None])
    x = np.array([0.45, 0.5, 0.55], dtype=np.float32)
    N = 200_000
    u = np.random.default_rng(21).random((N, 3), dtype=np.float32)
    out = orc.sample(K, *params, np.repeat(x[None], N, 0), np.zeros(N, np.int32), u)
    kappa = 2.0
    a = mu_w[np.argmax(pi)]
    est = np.zeros(N)
    v = out["valid"].astype(bool)
    est[v] = np.exp(kappa * (out["dir"][v] @ a - 1.0)) / out["pdf"][v]
    truth = 2 * math.pi * (1 - math.exp(-2 * kappa)) / kappa
    se = est.std() / math.sqrt(N)
    assert abs(est.mean() - truth) < 4 * se, (est.mean(), truth, se)
    # the sampler's reported pdf is the pdf of the returned direction
    p2 = orc.pdf(K, *params, np.repeat(x[None], 1000, 0), np.zeros(1000, np.int32),
                 out["dir"][:1000])
    assert np.allclose(np.where(out["valid"][:1000] == 1, p2, 0.0), out["pdf"][:1000], rtol=1e-12)
