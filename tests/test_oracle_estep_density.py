"""Pin of the oracle's solid-angle E-step density (Sec. 3.1 Eq. solidangle-pdf
used inside Sec. 3.2 Eq. em-ss-computation, ``estep_density = 1``).

The per-sample log-likelihood of the solid-angle E-step is
    l(x, w) = log sum_k pi_k N_5((x - mu_k^x, log_{mu_k} w); 0, Sigma_k) / sinc|nu_k|.
Every joint Gaussian factors into its spatial marginal times the conditional of
the direction given the position, so
    exp l(x, w) = [sum_l pi_l N_3(x; mu_l^x, Sigma_l^xx)] * p(w | x),
where p(w | x) is the conditioned mixture's solid-angle pdf.  The oracle's query
side computes p(w | x) with code of its own (conditioning pinned against the
dense textbook conditional, the pdf pinned by quadrature over the sphere), and
the spatial marginal is evaluated here with scipy.  A dropped, inverted or
sign-flipped Jacobian term in the E-step breaks the identity by log(theta /
sin theta), which the lobes below make as large as several units.

The second test integrates exp l over the sphere at a fixed position: it equals
the spatial marginal times the conditioned mixture's planar mass inside
|nu| < pi, computed on the plane.
"""
import math

import numpy as np
from scipy import stats

from test_oracle_query import PK, _disk_mass, _polar_grid, _unpack


def _mixture(seed, K):
    """K components with wide directional lobes (std 0.7 to 1.4 rad), so that
    samples reach far into each chart where theta / sin(theta) is large."""
    rng = np.random.default_rng(seed)
    pi = rng.dirichlet(np.ones(K))
    mu_x = rng.uniform(0.35, 0.65, size=(K, 3))
    mu_w = rng.normal(size=(K, 3))
    mu_w /= np.linalg.norm(mu_w, axis=1, keepdims=True)
    L = np.zeros((K, 15))
    for k in range(K):
        diag = np.concatenate([rng.uniform(0.08, 0.2, 3), rng.uniform(0.7, 1.4, 2)])
        for p, (i, j) in enumerate(PK):
            L[k, p] = diag[i] if i == j else 0.4 * rng.normal() * diag[i]
    return pi, mu_x, mu_w, L


def _spatial_marginal(pi, mu_x, L, x):
    """sum_k pi_k N_3(x; mu_k^x, A_k A_k^T) with A_k the spatial block of L_k."""
    tot = 0.0
    for k in range(len(pi)):
        Lk = _unpack(L[k])
        S = Lk @ Lk.T
        tot += pi[k] * stats.multivariate_normal(mu_x[k], S[:3, :3]).pdf(x)
    return tot


def _samples(xs, dirs, w=None):
    M = xs.shape[0]
    s = np.zeros((7, M), np.float32)
    s[0:3] = xs.T
    s[3:6] = dirs.T
    s[6] = 1.0 if w is None else w
    return s


def test_solid_angle_loglik_is_marginal_times_conditioned_pdf(orc):
    K = 3
    pi, mu_x, mu_w, L = _mixture(5, K)
    rng = np.random.default_rng(6)
    M = 400
    xs = rng.uniform(0.3, 0.7, size=(M, 3)).astype(np.float32)
    d = rng.normal(size=(M, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    dirs = d.astype(np.float32)
    s = _samples(xs, dirs)
    out = orc.estep_region(orc.config(K, estep_density=1), pi, mu_x, mu_w, L, s)
    out_t = orc.estep_region(orc.config(K, estep_density=0), pi, mu_x, mu_w, L, s)
    p = orc.pdf(K, pi[None], mu_x[None], mu_w[None], L[None], xs, np.zeros(M, np.int32),
                dirs.astype(np.float64))
    marg = np.array([_spatial_marginal(pi, mu_x, L, xs[i].astype(np.float64)) for i in range(M)])
    expect = np.log(marg) + np.log(p)
    # the FP32 directions are unit length to ~6e-8, which the two sides treat
    # slightly differently; the identity holds to that level
    assert np.allclose(out["loglik"], expect, rtol=0, atol=1e-6)
    # the lobes are wide: the Jacobian term matters by far more than the tolerance
    gap = np.abs(out["loglik"] - out_t["loglik"])
    assert gap.max() > 1.0 and np.median(gap) > 0.05


def test_solid_angle_likelihood_integrates_to_marginal_times_disk_mass(orc):
    K = 2
    pi, mu_x, mu_w, L = _mixture(9, K)
    x = np.array([0.48, 0.52, 0.5], dtype=np.float32)
    cpi, cm, cL = orc.condition(K, pi[None], mu_x[None], mu_w[None], L[None], x[None],
                                np.zeros(1, np.int32))
    marg = _spatial_marginal(pi, mu_x, L, x.astype(np.float64))
    total, expected = 0.0, 0.0
    for k in range(K):
        D = np.array([[cL[0, k, 0], 0.0], [cL[0, k, 1], cL[0, k, 2]]])
        expected += cpi[0, k] * _disk_mass(cm[0, k], D @ D.T)
        # component k's share of exp(l) on a grid whose pole is its antipode
        # (the 1 / sinc singularity sits there)
        dirs, wts = _polar_grid(-mu_w[k], 500, 1000)
        Q = dirs.shape[0]
        s = _samples(np.repeat(x[None], Q, 0), dirs.astype(np.float32))
        one = orc.estep_region(orc.config(1, estep_density=1), np.ones(1), mu_x[k:k + 1],
                               mu_w[k:k + 1], L[k:k + 1], s)
        Lk = _unpack(L[k])
        mk = stats.multivariate_normal(mu_x[k], (Lk @ Lk.T)[:3, :3]).pdf(x.astype(np.float64))
        # exp(l) of the single component is N_3(x) * (its conditional pdf); weight
        # it by pi_k and integrate over the sphere
        total += pi[k] * float(np.sum(np.exp(one["loglik"]) * wts))
        assert mk > 0
    assert 0.8 < expected < 0.999          # wide lobes: part of the mass lies beyond |nu| = pi
    assert abs(total - marg * expected) < 1e-6 * marg * expected, (total, marg * expected)
