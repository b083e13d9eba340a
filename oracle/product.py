"""Product sampling of the conditioned radiance mixture with a BSDF mixture
(Sec. 3.5 "Product Sampling from Mixed-Orientation Gaussians", Eq.
product-distribution; Sec. 4.1 "Pruning before product sampling").

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): plain FP64 per-query
loops, shared with nothing on the CUDA path.

Per query: the radiance mixture conditioned on the position (weights pi'_k,
chart of mu_k, offset mean m_k, factor D_k: or_condition) and J BSDF lobes
(weight w_j, unit mean direction mu2_j in the same frame, factor L2_j of the
lobe's covariance in its own chart, Duff basis).  Readings:
  * pruning keeps the two lobes of largest weight (lower index on ties), in
    increasing lobe index; with J = 1 the one lobe;
  * every pair (k, j) is formed in the chart of mu_k: the lobe's mean is
    nu2 = log_{mu_k}(mu2_j) and its covariance J S2 J^T with
    J = J_log_{mu_k}(mu2_j) J_exp_{mu2_j}(0) (first order, Eq.
    product-distribution); a lobe at the antipode of mu_k gives no pair;
  * the product of N(nu; m_k, S1) and N(nu; nu2, S2') is the Gaussian of
    covariance P = S1 (S1 + S2')^-1 S2' and mean S2' (S1 + S2')^-1 m_k +
    S1 (S1 + S2')^-1 nu2, scaled by N(m_k; nu2, S1 + S2'); the pair's weight
    is pi'_k w_j times that scale, the mixture normalised over the pairs;
  * pairs are ordered by k, then lobe index; u0 picks one by inverse CDF,
    Box-Muller on (1 - u1, u2) draws in its chart, |nu| >= pi is discarded
    (valid = 0, pdf 0), otherwise omega = exp_{mu_k}(nu);
  * the pdf on the sphere of the product mixture is
    sum over pairs of weight * N(log_{mu_k}(omega); mean, P) / sinc|nu_k|,
    pairs with |log_{mu_k}(omega)| >= pi (or the antipode) contributing 0.
"""
from __future__ import annotations

import numpy as np

import oracle as orc


def top2(w):
    """Indices of the two largest weights, lower index first on ties, sorted."""
    J = len(w)
    if J == 1:
        return [0]
    order = sorted(range(J), key=lambda j: (-float(w[j]), j))
    return sorted(order[:2])


def _gauss2(d, S):
    det = S[0, 0] * S[1, 1] - S[0, 1] * S[1, 0]
    Si = np.array([[S[1, 1], -S[0, 1]], [-S[1, 0], S[0, 0]]]) / det
    return np.exp(-0.5 * d @ Si @ d) / (2.0 * np.pi * np.sqrt(det))


def transport(mu1, mu2):
    """J of nu1 = log_{mu1}(exp_{mu2}(nu2)) at nu2 = 0 (2 x 2)."""
    return orc.jlog(mu1, mu2) @ orc.jexp(mu2, np.zeros(2))


def pairs(cpi, cm, cL, mu_w, bw, bmu, bL):
    """Product mixture of one query: list of (k, weight, mean, P), weights
    normalised; cpi (K,), cm (K, 2), cL (K, 3), mu_w (K, 3); bw (J,),
    bmu (J, 3), bL (J, 3)."""
    out = []
    K = len(cpi)
    for k in range(K):
        D = np.array([[cL[k, 0], 0.0], [cL[k, 1], cL[k, 2]]])
        S1 = D @ D.T
        for j in top2(bw):
            nu2, anti, _, _ = orc.log_map(mu_w[k], bmu[j])
            if anti or np.hypot(*nu2) >= np.pi:
                continue
            L2 = np.array([[bL[j, 0], 0.0], [bL[j, 1], bL[j, 2]]])
            Jt = transport(mu_w[k], bmu[j])
            S2 = Jt @ L2 @ L2.T @ Jt.T
            S = S1 + S2
            Sinv = np.linalg.inv(S)
            P = S1 @ Sinv @ S2
            P = 0.5 * (P + P.T)
            mean = S2 @ Sinv @ cm[k] + S1 @ Sinv @ nu2
            wgt = cpi[k] * bw[j] * _gauss2(cm[k] - nu2, S)
            out.append((k, wgt, mean, P))
    tot = sum(p[1] for p in out)
    if not tot > 0.0:
        return []
    return [(k, w / tot, m, P) for k, w, m, P in out]


def pdf_at(prs, mu_w, omega):
    p = 0.0
    for k, w, mean, P in prs:
        nu, anti, _, _ = orc.log_map(mu_w[k], omega)
        r = np.hypot(*nu)
        if anti or r >= np.pi:
            continue
        p += w * _gauss2(nu - mean, P) / orc.sinc(r)
    return p


def sample(prs, mu_w, u):
    """(omega, pdf, valid, pair index) for uniforms u = (u0, u1, u2)."""
    if not prs:
        return np.array([0.0, 0.0, 1.0]), 0.0, 0, -1
    cum = np.cumsum([p[1] for p in prs])
    t = float(u[0]) * cum[-1]
    idx = int(np.searchsorted(cum, t, side="right"))
    idx = min(idx, len(prs) - 1)
    k, w, mean, P = prs[idx]
    rad = np.sqrt(-2.0 * np.log(1.0 - float(u[1])))
    z = rad * np.array([np.cos(2.0 * np.pi * float(u[2])), np.sin(2.0 * np.pi * float(u[2]))])
    C = np.linalg.cholesky(P)
    nu = mean + C @ z
    if np.hypot(*nu) >= np.pi:
        return np.array([0.0, 0.0, 1.0]), 0.0, 0, idx
    omega = orc.exp_map(mu_w[k], nu)
    return omega, pdf_at(prs, mu_w, omega), 1, idx


def margin(prs, u0):
    """Distance of u0 to the nearest pair CDF boundary (ties and rounding)."""
    if not prs:
        return 1.0
    cum = np.cumsum([p[1] for p in prs]) / sum(p[1] for p in prs)
    return float(np.min(np.abs(cum[:-1] - u0))) if len(cum) > 1 else 1.0
