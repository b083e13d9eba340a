"""Pins of the oracle's MAP objective and its analytic gradient (derived from
Sec. 3.2 Eq. em-ss-computation and Sec. 4.3's MAP priors) against central
finite differences in FP64, and of its stationary point against the M-step."""
import numpy as np
import pytest

from paper_2111_13094_gb300 import synthetic as syn


def _setup(orc, seed=0, R=2, K=3, M=300, density=0):
    truth = syn.batched_truth(seed, R, K=K, parallax=True)
    b = syn.batched_round(seed, R, np.full(R, M), 0, truth)
    cfg = orc.config(K, estep_density=density, prior_scale_mode=1)
    st = orc.State(R, K)
    orc.init_regions(cfg, b.offsets, b.samples, b.extent, syn.init_uniforms(seed, R, 1), st)
    orc.fit_regions(orc.config(K, eta_mode=1), b.offsets, b.samples, 3, st)
    st.n_seen[:] = M
    beta = np.full(R, 0.05)            # large, so the prior terms are exercised
    return cfg, b, st, beta


@pytest.mark.parametrize("density", [0, 1])
def test_gradient_matches_central_differences(orc, density):
    cfg, b, st, beta = _setup(orc, density=density)
    R, K = st.R, st.K
    F0, gd, gL, ga = orc.objective(cfg, b.offsets, b.samples, st, prior_scale=beta)
    h = 1e-6

    def F(stx, delta=None):
        return orc.objective(cfg, b.offsets, b.samples, stx, prior_scale=beta, delta=delta,
                             grads=False)

    zero = np.zeros((R, K, 5))
    for r in range(R):
        for k in range(K):
            for c in range(5):
                dp, dm = zero.copy(), zero.copy()
                dp[r, k, c], dm[r, k, c] = h, -h
                fd = (F(st, dp)[r] - F(st, dm)[r]) / (2 * h)
                assert abs(fd - gd[r, k, c]) < 1e-6 * max(1.0, abs(fd)), (r, k, c, fd, gd[r, k, c])
            for p in range(15):
                sp, sm = st.copy(), st.copy()
                sp.L[r, k, p] += h
                sm.L[r, k, p] -= h
                fd = (F(sp)[r] - F(sm)[r]) / (2 * h)
                assert abs(fd - gL[r, k, p]) < 1e-6 * max(1.0, abs(fd)), (r, k, p, fd, gL[r, k, p])
            # logits: pi = softmax(a), perturb a_k
            a = np.log(st.pi[r])
            ap, am = a.copy(), a.copy()
            ap[k] += h
            am[k] -= h
            sp, sm = st.copy(), st.copy()
            sp.pi[r] = np.exp(ap) / np.exp(ap).sum()
            sm.pi[r] = np.exp(am) / np.exp(am).sum()
            fd = (F(sp)[r] - F(sm)[r]) / (2 * h)
            assert abs(fd - ga[r, k]) < 1e-6 * max(1.0, abs(fd)), (r, k, fd, ga[r, k])


def test_euclidean_m_step_is_stationary_point(orc):
    """After a Euclidean MAP-EM step from a converged state, the gradient of the
    objective vanishes (the M-step of Sec. 4.3 maximises it)."""
    rng = np.random.default_rng(3)
    K, N = 3, 2000
    X = np.concatenate([rng.normal(0.3, 0.05, (N // 2, 5)), rng.normal(0.7, 0.08, (N // 2, 5))])
    s = np.zeros((7, N), np.float32)
    s[0:3] = X[:, :3].T
    s[3:5] = X[:, 3:].T
    s[6] = rng.lognormal(0, 1, N)
    cfg = orc.config(K, euclid=1, eta_mode=1, prior_scale_mode=1)
    st = orc.State(1, K)
    st.pi[:] = 1 / K
    st.mu_x[0] = rng.uniform(0.3, 0.7, (K, 3))
    st.mu_w[0, :, :2] = rng.uniform(0.3, 0.7, (K, 2))
    st.L[0] = np.array([0.2 if i == j else 0.0 for i in range(5) for j in range(i + 1)])
    beta = np.array([1e-3])
    orc.fit_regions(cfg, [0, N], s, 500, st, prior_scale=beta)
    _, gd, gL, ga = orc.objective(cfg, [0, N], s, st, prior_scale=beta)
    assert np.abs(gd).max() < 1e-7 and np.abs(gL).max() < 1e-6 and np.abs(ga).max() < 1e-9
