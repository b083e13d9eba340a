"""The oracle's product sampling (Sec. 3.5, Eq. product-distribution; top-2
BSDF pruning of Sec. 4.1) against finite differences, the pointwise product
of the two Gaussians, quadrature over the sphere and a Monte Carlo
estimator."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as orc
from oracle import product as prod


def _unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


def _log_map_np(mu, dirs):
    """log_mu of many directions (numpy restatement for quadrature)."""
    R = orc.basis(mu)
    w = dirs @ R.T
    s = np.hypot(w[:, 0], w[:, 1])
    th = np.arctan2(s, w[:, 2])
    g = np.where(s > 0, th / np.where(s > 0, s, 1.0), 1.0)
    return np.stack([g * w[:, 0], g * w[:, 1]], 1), th


def _case(seed, K=3, J=4):
    rng = np.random.default_rng(seed)
    mu_w = np.array([_unit(rng.normal(size=3)) for _ in range(K)])
    cpi = rng.dirichlet(np.ones(K))
    cm = rng.normal(scale=0.1, size=(K, 2))
    cL = np.column_stack([rng.uniform(0.2, 0.5, K), rng.normal(scale=0.05, size=K), rng.uniform(0.2, 0.5, K)])
    bw = rng.uniform(0.1, 1.0, J)
    bmu = np.array([_unit(mu_w[j % K] + rng.normal(scale=0.6, size=3)) for j in range(J)])
    bL = np.column_stack([rng.uniform(0.1, 0.4, J), rng.normal(scale=0.05, size=J), rng.uniform(0.1, 0.4, J)])
    return cpi, cm, cL, mu_w, bw, bmu, bL


def test_transport_jacobian_matches_finite_differences():
    rng = np.random.default_rng(1)
    for _ in range(10):
        mu1, mu2 = _unit(rng.normal(size=3)), _unit(rng.normal(size=3))
        if mu1 @ mu2 < -0.5:
            continue
        J = prod.transport(mu1, mu2)
        h = 1e-6
        F = np.zeros((2, 2))
        for c in range(2):
            e = np.zeros(2)
            e[c] = h
            a = orc.log_map(mu1, orc.exp_map(mu2, e))[0]
            b = orc.log_map(mu1, orc.exp_map(mu2, -e))[0]
            F[:, c] = (a - b) / (2 * h)
        assert np.abs(J - F).max() < 1e-7


def test_pair_is_the_pointwise_product_of_the_two_gaussians():
    cpi, cm, cL, mu_w, bw, bmu, bL = _case(2)
    prs = prod.pairs(cpi, cm, cL, mu_w, bw, bmu, bL)
    raw = []
    for k in range(len(cpi)):
        D = np.array([[cL[k, 0], 0], [cL[k, 1], cL[k, 2]]])
        for j in prod.top2(bw):
            nu2 = orc.log_map(mu_w[k], bmu[j])[0]
            L2 = np.array([[bL[j, 0], 0], [bL[j, 1], bL[j, 2]]])
            Jt = prod.transport(mu_w[k], bmu[j])
            raw.append((k, j, nu2, D @ D.T, Jt @ L2 @ L2.T @ Jt.T))
    rng = np.random.default_rng(3)
    ratios = []
    for (k, w, mean, P), (k2, j, nu2, S1, S2) in zip(prs, raw):
        assert k == k2
        for nu in rng.normal(scale=0.4, size=(5, 2)):
            lhs = w * stats.multivariate_normal(mean, P).pdf(nu)
            rhs = (cpi[k] * bw[j] * stats.multivariate_normal(cm[k], S1).pdf(nu)
                   * stats.multivariate_normal(nu2, S2).pdf(nu))
            ratios.append(lhs / rhs)
    # one common constant (the mixture's normaliser) for every pair and point
    ratios = np.asarray(ratios)
    assert np.abs(ratios / ratios[0] - 1.0).max() < 1e-9


def test_pruning_keeps_the_two_largest_lobes():
    assert prod.top2([0.1, 0.5, 0.3, 0.5]) == [1, 3]
    assert prod.top2([0.2, 0.2, 0.2]) == [0, 1]
    assert prod.top2([0.7]) == [0]
    cpi, cm, cL, mu_w, bw, bmu, bL = _case(4, J=4)
    bw = np.array([0.9, 0.01, 0.8, 0.02])
    a = prod.pairs(cpi, cm, cL, mu_w, bw, bmu, bL)
    b = prod.pairs(cpi, cm, cL, mu_w, bw[[0, 2]], bmu[[0, 2]], bL[[0, 2]])
    assert len(a) == len(b) and all(np.allclose(x[2], y[2]) and abs(x[1] - y[1]) < 1e-14 for x, y in zip(a, b))


def _polar_grid(axis, n_a, n_phi):
    xa, wa = np.polynomial.legendre.leggauss(n_a)
    al = (xa + 1) * math.pi / 2
    wa = wa * math.pi / 2 * np.sin(al)
    phi = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    axis = _unit(axis)
    t = _unit(np.cross(axis, [1.0, 0, 0] if abs(axis[0]) < 0.9 else [0, 1.0, 0]))
    b = np.cross(axis, t)
    A, P = np.repeat(al, n_phi), np.tile(phi, n_a)
    d = (np.cos(A)[:, None] * axis + (np.sin(A) * np.cos(P))[:, None] * t + (np.sin(A) * np.sin(P))[:, None] * b)
    return d, np.repeat(wa, n_phi) * 2 * math.pi / n_phi


def _disk_mass(m, C, n_r=160, n_phi=320):
    xr, wr = np.polynomial.legendre.leggauss(n_r)
    rho = (xr + 1) * math.pi / 2
    wr = wr * math.pi / 2
    phi = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    Pn = np.stack([np.outer(rho, np.cos(phi)), np.outer(rho, np.sin(phi))], -1)
    dens = stats.multivariate_normal(m, C).pdf(Pn.reshape(-1, 2)).reshape(n_r, n_phi)
    return float(np.sum(dens * rho[:, None] * wr[:, None]) * 2 * math.pi / n_phi)


def test_pdf_integrates_to_the_pairs_in_disk_mass():
    """Each pair's density on the sphere (chart Gaussian / sinc) integrates to
    its planar mass inside |nu| < pi; pdf_at is the sum of the pairs."""
    cpi, cm, cL, mu_w, bw, bmu, bL = _case(5)
    prs = prod.pairs(cpi, cm, cL, mu_w, bw, bmu, bL)
    total, expected = 0.0, 0.0
    for k, w, mean, P in prs:
        dirs, wts = _polar_grid(-mu_w[k], 500, 1000)     # pole at the antipode of mu_k
        nu, th = _log_map_np(mu_w[k], dirs)
        dens = w * stats.multivariate_normal(mean, P).pdf(nu) / np.where(th > 0, np.sin(th) / th, 1.0)
        dens[th >= math.pi] = 0.0
        total += float(np.sum(dens * wts))
        expected += w * _disk_mass(mean, P)
    assert 0.8 < expected < 1.0 and abs(total - expected) < 1e-6, (total, expected)
    rng = np.random.default_rng(6)
    for om in [_unit(v) for v in rng.normal(size=(5, 3))]:
        s = 0.0
        for k, w, mean, P in prs:
            nu, th = _log_map_np(mu_w[k], om[None])
            if th[0] < math.pi:
                s += w * stats.multivariate_normal(mean, P).pdf(nu[0]) / (math.sin(th[0]) / th[0])
        assert abs(prod.pdf_at(prs, mu_w, om) - s) < 1e-12 * max(1.0, s)


def test_sampling_estimator_is_unbiased():
    """E[f(omega) / p(omega)] over product samples equals the integral of f
    over the region the product mixture covers (f: a smooth lobe)."""
    cpi, cm, cL, mu_w, bw, bmu, bL = _case(7, K=2, J=3)
    prs = prod.pairs(cpi, cm, cL, mu_w, bw, bmu, bL)
    axis = _unit(mu_w[0] + mu_w[1])

    def f(om):
        return np.exp(4.0 * (om @ axis - 1.0))

    u = orc.uniforms(11, 20000)
    vals = []
    for q in range(u.shape[0]):
        om, p, ok, _ = prod.sample(prs, mu_w, u[q])
        vals.append(f(om) / p if ok and p > 0 else 0.0)
    vals = np.asarray(vals)
    est, se = vals.mean(), vals.std() / math.sqrt(vals.size)
    dirs, wts = _polar_grid(axis, 400, 800)
    truth = float(np.sum(f(dirs) * wts))               # f is negligible where p = 0 here
    assert abs(est - truth) < 4 * se + 1e-3 * truth, (est, truth, se)
