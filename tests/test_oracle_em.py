"""Pins of the oracle's EM (Sec. 3.2, 3.4, 4.2, 4.3) against closed forms,
invariants and parameter recovery from data with a known generating mixture."""
import math

import numpy as np
import pytest

from paper_2111_13094_gb300 import synthetic as syn

PK = [(i, j) for i in range(5) for j in range(i + 1)]


def _unpack(Lp):
    L = np.zeros(Lp.shape[:-1] + (5, 5))
    for p, (i, j) in enumerate(PK):
        L[..., i, j] = Lp[..., p]
    return L


def _pack(M):
    return np.stack([M[..., i, j] for i, j in PK], -1)


def _state(orc, pi, mu_x, mu_w, L):
    R, K = pi.shape
    st = orc.State(R, K)
    st.set_params(pi, mu_x, mu_w, L)
    return st


def _samples(x, d, w):
    s = np.zeros((7, x.shape[0]), np.float32)
    s[0:3] = x.T
    s[3:6] = d.T
    s[6] = w
    return s


def test_defaults_are_paper_constants(orc):
    from conftest import read_constants
    c = read_constants()
    cfg = orc.config(16)
    assert cfg.prior_q == c["prior_q_times_K"]
    assert cfg.prior_a == c["prior_a_times_K"]
    assert cfg.prior_B_pos == c["prior_B_pos_over_a"]
    assert cfg.prior_B_dir == c["prior_B_dir_over_a"]
    assert cfg.eta_alpha == c["eta_alpha"] and cfg.eta_beta == c["eta_beta"]
    assert cfg.min_samples == c["min_samples"]


def test_k1_euclidean_is_weighted_mean_and_covariance(orc):
    """One component, Euclidean directions: one MAP-EM step gives the weighted
    mean and (beta B + weighted covariance) / (beta a + 1) (Sec. 3.2, 4.3)."""
    rng = np.random.default_rng(0)
    N = 5000
    X = rng.normal(size=(N, 5)) @ rng.normal(size=(5, 5)) * 0.1 + 0.5
    w = rng.lognormal(0, 1.5, N).astype(np.float32)
    d = np.zeros((N, 3))
    d[:, :2] = X[:, 3:]
    s = _samples(X[:, :3], d, w)
    Xf = np.concatenate([s[0:3].T, s[3:5].T], 1).astype(np.float64)
    beta = 0.37
    cfg = orc.config(1, euclid=1, eta_mode=1, prior_scale_mode=1)
    st = _state(orc, np.ones((1, 1)), np.zeros((1, 1, 3)), np.zeros((1, 1, 3)),
                _pack(np.eye(5))[None, None])
    orc.fit_regions(cfg, [0, N], s, 1, st, prior_scale=np.array([beta]))
    wt = s[6].astype(np.float64)
    mean = np.average(Xf, axis=0, weights=wt)
    cov = np.cov(Xf.T, aweights=wt, bias=True)
    a = cfg.prior_a / 1
    B = a * np.diag([cfg.prior_B_pos] * 3 + [cfg.prior_B_dir] * 2)
    Sig = (beta * B + cov) / (beta * a + 1.0)
    assert st.status[0] == 0
    assert np.allclose(st.mu_x[0, 0], mean[:3], rtol=1e-12, atol=1e-13)
    assert np.allclose(st.mu_w[0, 0, :2], mean[3:], rtol=1e-12, atol=1e-13)
    Lf = _unpack(st.L[0, 0])
    assert np.allclose(Lf @ Lf.T, Sig, rtol=1e-10, atol=1e-14)
    assert st.pi[0, 0] == 1.0


def test_k1_great_circle_mean_and_variance(orc):
    """Directions on one great circle through mu: the new mean is the exp of the
    weighted mean angle along the circle, and the first-order chart change keeps
    the variance along the circle equal to the weighted variance of the angles
    (Sec. 3.2 Eq. tangent-space-mu-update, Sec. 3.4)."""
    rng = np.random.default_rng(1)
    N = 4000
    mu = np.array([0.2, -0.4, 0.8])
    mu /= np.linalg.norm(mu)
    e = np.cross(mu, [1.0, 0, 0])
    e /= np.linalg.norm(e)
    t = rng.normal(0.35, 0.2, N)
    d = np.cos(t)[:, None] * mu + np.sin(t)[:, None] * e
    x = rng.uniform(0.4, 0.6, size=(N, 3))
    w = rng.lognormal(0, 1.0, N).astype(np.float32)
    s = _samples(x, d, w)
    # angles of the stored (float32) directions, measured independently
    dd = s[3:6].T.astype(np.float64)
    ts = np.arctan2(dd @ e, dd @ mu)
    wt = s[6].astype(np.float64)
    tbar = np.average(ts, weights=wt)
    vt = np.average((ts - tbar) ** 2, weights=wt)
    cfg = orc.config(1, eta_mode=1, prior_scale_mode=1)
    L0 = _pack(np.diag([0.1, 0.1, 0.1, 0.5, 0.5]))
    st = _state(orc, np.ones((1, 1)), np.full((1, 1, 3), 0.5), mu[None, None], L0[None, None])
    orc.fit_regions(cfg, [0, N], s, 1, st, prior_scale=np.array([1e-9]))
    assert st.status[0] == 0
    expect = math.cos(tbar) * mu + math.sin(tbar) * e
    assert np.allclose(st.mu_w[0, 0], expect, atol=1e-12)
    R = orc.basis(st.mu_w[0, 0])
    P = R[:2].T
    Lf = _unpack(st.L[0, 0])
    Sw = P @ (Lf @ Lf.T)[3:, 3:] @ P.T
    e_new = -math.sin(tbar) * mu + math.cos(tbar) * e
    assert np.allclose(Sw, vt * np.outer(e_new, e_new), atol=1e-9)


def _objective(orc, cfg, off, s, st, beta):
    return orc.objective(cfg, off, s, st, prior_scale=np.full(len(off) - 1, beta), grads=False)


def test_map_objective_never_decreases_euclidean(orc):
    """Euclidean MAP-EM ascends the MAP objective exactly (Sec. 4.3, Gauvain-Lee)."""
    rng = np.random.default_rng(2)
    K, N = 4, 3000
    centres = rng.uniform(0.2, 0.8, size=(K, 5))
    lab = rng.integers(0, K, N)
    X = centres[lab] + 0.08 * rng.normal(size=(N, 5))
    d = np.zeros((N, 3))
    d[:, :2] = X[:, 3:]
    s = _samples(X[:, :3], d, rng.lognormal(0, 1.5, N).astype(np.float32))
    cfg = orc.config(K, euclid=1, eta_mode=1, prior_scale_mode=1)
    st = _state(orc, np.full((1, K), 1 / K), rng.uniform(0.3, 0.7, (1, K, 3)),
                np.concatenate([rng.uniform(0.3, 0.7, (1, K, 2)), np.zeros((1, K, 1))], 2),
                np.tile(_pack(0.3 * np.eye(5)), (1, K, 1)))
    beta = 1.0 / N
    off = [0, N]
    F = [_objective(orc, cfg, off, s, st, beta)[0]]
    for _ in range(25):
        orc.fit_regions(cfg, off, s, 1, st, prior_scale=np.array([beta]))
        assert st.status[0] == 0
        F.append(_objective(orc, cfg, off, s, st, beta)[0])
    F = np.array(F)
    assert np.all(np.diff(F) >= -1e-12 * np.abs(F[1:]))
    assert F[-1] > F[0] + 1.0


def test_map_objective_tangent_slack_is_small(orc):
    """On the sphere the M-step is exact up to the first-order chart change;
    the objective may only dip by that slack."""
    b = syn.single_region(seed=3, N=8000, K=8)
    K = 8
    cfg = orc.config(K, eta_mode=1, prior_scale_mode=1)
    st = orc.State(1, K)
    orc.init_regions(cfg, b.offsets, b.samples, b.extent, syn.init_uniforms(3, 1, 1), st)
    beta = 1.0 / b.N
    F = [_objective(orc, cfg, b.offsets, b.samples, st, beta)[0]]
    for _ in range(20):
        orc.fit_regions(cfg, b.offsets, b.samples, 1, st, prior_scale=np.array([beta]))
        F.append(_objective(orc, cfg, b.offsets, b.samples, st, beta)[0])
    F = np.array(F)
    worst = np.max(np.maximum(0.0, -np.diff(F)))
    assert worst <= 1e-6 * np.abs(F).max(), (worst, F)
    assert F[-1] > F[0]


def _lobe_region(orc, delta, N=40000, sd=(0.25, 0.12), seed=4):
    """Antithetic (symmetric) directions around a true mean; the model's
    current mean is off by `delta` rad."""
    rng = np.random.default_rng(seed)
    mu_t = np.array([0.3, 0.5, 0.6])
    mu_t /= np.linalg.norm(mu_t)
    half = rng.normal(size=(N // 2, 2)) * np.array(sd)
    nu = np.concatenate([half, -half])
    Rt = orc.basis(mu_t)
    d = np.array([orc.exp_map(mu_t, v) for v in nu])
    x = np.full((N, 3), 0.5) + 0.01 * np.concatenate([rng.normal(size=(N // 2, 3))] * 2)
    s = _samples(x, d, np.ones(N, np.float32))
    mu0 = orc.exp_map(mu_t, np.array([delta, 0.5 * delta]))
    return s, mu0, Rt


def test_first_order_covariance_update_is_second_order_accurate(orc):
    """First-order chart change (Sec. 3.4, Fig. covariance-foreign d) against the
    accurate two-pass update (Eq. tangent-space-sigma-update): the gap shrinks
    quadratically with the mean step; the naive update (no chart change) only
    linearly."""
    gaps, naive = [], []
    for delta in [0.2, 0.1, 0.05]:
        s, mu0, _ = _lobe_region(orc, delta)
        N = s.shape[1]
        L0 = _pack(np.diag([0.02, 0.02, 0.02, 0.4, 0.4]))
        out = {}
        for mode in (0, 1):
            cfg = orc.config(1, eta_mode=1, prior_scale_mode=1, cov_update=mode)
            st = _state(orc, np.ones((1, 1)), np.full((1, 1, 3), 0.5), mu0[None, None], L0[None, None])
            orc.fit_regions(cfg, [0, N], s, 1, st, prior_scale=np.array([1e-9]))
            R = orc.basis(st.mu_w[0, 0])
            Lf = _unpack(st.L[0, 0])
            out[mode] = R[:2].T @ (Lf @ Lf.T)[3:, 3:] @ R[:2]       # world-frame tensor
        gaps.append(np.abs(out[0] - out[1]).max())
        # naive: centred covariance of the old-chart coordinates, no chart change
        cfg = orc.config(1, eta_mode=1)
        e = orc.estep_region(cfg, np.ones(1), np.full((1, 3), 0.5), mu0[None], L0[None], s)
        S0, S1, S2 = e["s0"][0], e["s1"][0], _unpack(e["s2"][0])
        C = S2 / S0 - np.outer(S1 / S0, S1 / S0)
        R0 = orc.basis(mu0)
        naive.append(np.abs(R0[:2].T @ C[3:, 3:] @ R0[:2] - out[1]).max())
    r1, r2 = gaps[0] / gaps[1], gaps[1] / gaps[2]
    assert 3.0 < r1 < 5.5 and 3.0 < r2 < 5.5, gaps
    n1, n2 = naive[0] / naive[1], naive[1] / naive[2]
    assert n1 < 3.0 and n2 < 3.0, naive             # has a first-order term
    assert all(g < 0.2 * n for g, n in zip(gaps, naive)), (gaps, naive)


def _frame_free(orc, mu_w, L):
    """World-frame covariance blocks of a fitted component."""
    R = orc.basis(mu_w)
    P = R[:2].T
    Lf = _unpack(L)
    S = Lf @ Lf.T
    return S[:3, :3], P @ S[3:, 3:] @ P.T, S[:3, 3:] @ P.T


def test_parameter_recovery_from_known_mixture(orc):
    """EM started near a known 4-component mixture converges to it within
    statistical error (frame-free comparison of all parameters)."""
    rng = np.random.default_rng(5)
    K = 4
    gt = syn.ground_truth(rng, 1, K, parallax=True)
    # well-separated truth: distinct corners in space, spread weights
    gt.mu_x[0] = np.array([[0.25, 0.25, 0.25], [0.75, 0.25, 0.7], [0.3, 0.75, 0.6], [0.7, 0.7, 0.3]])
    gt.pi[0] = np.array([0.2, 0.3, 0.25, 0.25])
    N = 160_000
    s = syn.draw(rng, gt, [N])
    # start: truth means displaced by ~half a std, covariances inflated
    cfg = orc.config(K, eta_mode=1)
    st = orc.State(1, K)
    st.pi[0] = 1.0 / K
    for k in range(K):
        C = gt.cov[0, k]
        st.mu_x[0, k] = gt.mu_x[0, k] + 0.5 * np.sqrt(np.diag(C)[:3]) * rng.normal(size=3)
        st.mu_w[0, k] = orc.exp_map(gt.mu_w[0, k], 0.5 * np.sqrt(np.diag(C)[3:]) * rng.normal(size=2))
        st.L[0, k] = _pack(np.diag(np.sqrt(1.5 * np.diag(C))))
    orc.fit_regions(cfg, [0, N], s, 40, st)
    assert st.status[0] == 0
    wt = s[6].astype(np.float64)
    neff = wt.sum() ** 2 / (wt ** 2).sum()
    for k in range(K):
        C = gt.cov[0, k]
        E = np.stack([gt.e1[0, k], gt.e2[0, k]], 1)
        nk = neff * gt.pi[0, k]
        assert abs(st.pi[0, k] - gt.pi[0, k]) < 5 * math.sqrt(gt.pi[0, k] / neff) + 1e-3
        sx = np.sqrt(np.diag(C)[:3])
        assert np.all(np.abs(st.mu_x[0, k] - gt.mu_x[0, k]) < 5 * sx / math.sqrt(nk))
        ang = math.acos(min(1.0, float(st.mu_w[0, k] @ gt.mu_w[0, k])))
        assert ang < 5 * np.sqrt(np.diag(C)[3:]).max() / math.sqrt(nk)
        Sxx, Sww, Sxw = _frame_free(orc, st.mu_w[0, k], st.L[0, k])
        tol = 6.0 / math.sqrt(nk)
        assert np.allclose(Sxx, C[:3, :3], atol=tol * np.abs(C[:3, :3]).max())
        Tww = E @ C[3:, 3:] @ E.T
        assert np.allclose(Sww, Tww, atol=tol * np.abs(Tww).max())
        Txw = C[:3, 3:] @ E.T
        assert np.allclose(Sxw, Txw, atol=tol * math.sqrt(np.abs(C[:3, :3]).max() * np.abs(Tww).max()))


def test_fit_from_paper_init_approaches_truth_likelihood(orc):
    """16-component truth, N = 65,536, 20 iterations from the initialisation of
    Sec. 4.3 / App. B-C: the held-out mean log-likelihood is close to the
    generating mixture's."""
    b = syn.single_region(seed=0, N=65536, K=16)
    K = 16
    cfg = orc.config(K, eta_mode=1)
    st = orc.State(1, K)
    orc.init_regions(cfg, b.offsets, b.samples, b.extent, syn.init_uniforms(0, 1, 2), st)
    orc.fit_regions(cfg, b.offsets, b.samples, 20, st)
    assert st.status[0] == 0
    held = syn.draw(np.random.default_rng(99), b.truth, [20000])
    fit_ll = orc.estep_region(cfg, st.pi[0], st.mu_x[0], st.mu_w[0], st.L[0], held)["loglik"]
    # the truth expressed in the oracle's charts
    gt = b.truth
    Lt = np.zeros((K, 15))
    for k in range(K):
        R = orc.basis(gt.mu_w[0, k])
        T = np.eye(5)
        T[3:, 3:] = R[:2] @ np.stack([gt.e1[0, k], gt.e2[0, k]], 1)
        Lt[k] = _pack(np.linalg.cholesky(T @ gt.cov[0, k] @ T.T))
    tru_ll = orc.estep_region(cfg, gt.pi[0], gt.mu_x[0], gt.mu_w[0], Lt, held)["loglik"]
    gap = tru_ll.mean() - fit_ll.mean()
    assert gap < 0.35, gap
    assert np.isfinite(fit_ll).all()


def test_stepwise_average_has_plain_em_fixed_point(orc):
    """Robbins-Monro averaging over repeated identical batches converges to the
    plain EM fixed point (Sec. 4.3), and the averaged mean weight is W/M."""
    b = syn.single_region(seed=6, N=4000, K=4)
    K = 4
    st0 = orc.State(1, K)
    orc.init_regions(orc.config(K), b.offsets, b.samples, b.extent, syn.init_uniforms(6, 1, 1), st0)
    beta = 1.0 / b.N
    plain = st0.copy()
    orc.fit_regions(orc.config(K, eta_mode=1, prior_scale_mode=1), b.offsets, b.samples, 400,
                    plain, prior_scale=np.array([beta]))
    rm = st0.copy()
    cfg = orc.config(K, eta_mode=0, prior_scale_mode=1)
    for _ in range(400):
        orc.fit_regions(cfg, b.offsets, b.samples, 1, rm, prior_scale=np.array([beta]))
    assert rm.step_j[0] == 400 and rm.n_seen[0] == 400 * b.N
    assert np.allclose(rm.pi, plain.pi, atol=2e-4)
    assert np.allclose(rm.mu_x, plain.mu_x, atol=2e-4)
    assert np.allclose(rm.mu_w, plain.mu_w, atol=2e-4)
    assert np.allclose(rm.L, plain.L, atol=2e-4)
    Wm = b.samples[6].astype(np.float64).mean()
    assert abs(rm.Wbar[0] - Wm) < 1e-12 * Wm


def test_first_stepwise_step_is_plain_em(orc):
    b = syn.single_region(seed=7, N=3000, K=4)
    st0 = orc.State(1, 4)
    orc.init_regions(orc.config(4), b.offsets, b.samples, b.extent, syn.init_uniforms(7, 1, 1), st0)
    a, p = st0.copy(), st0.copy()
    orc.fit_regions(orc.config(4, eta_mode=0), b.offsets, b.samples, 1, a)
    orc.fit_regions(orc.config(4, eta_mode=1), b.offsets, b.samples, 1, p)
    for f in ("pi", "mu_x", "mu_w", "L", "S0", "S2"):
        assert np.array_equal(getattr(a, f), getattr(p, f))


def test_resume_is_bit_identical(orc):
    truth = syn.batched_truth(8, 8, K=4)
    counts = syn.region_counts(8, 8, 64, 2000)
    batches = [syn.batched_round(8, 8, counts, r, truth) for r in range(4)]
    cfg = orc.config(4)
    st = orc.State(8, 4)
    orc.init_regions(cfg, batches[0].offsets, batches[0].samples, batches[0].extent,
                     syn.init_uniforms(8, 8, 1), st)
    a = st.copy()
    for bt in batches:
        orc.fit_regions(cfg, bt.offsets, bt.samples, 1, a)
    b = st.copy()
    for bt in batches[:2]:
        orc.fit_regions(cfg, bt.offsets, bt.samples, 1, b)
    c = b.copy()                      # "checkpoint"
    for bt in batches[2:]:
        orc.fit_regions(cfg, bt.offsets, bt.samples, 1, c)
    for f in orc.State.FIELDS:
        assert np.array_equal(getattr(a, f), getattr(c, f)), f


def test_region_status_codes(orc):
    rng = np.random.default_rng(9)
    K = 2
    counts = [10, 100, 100, 100]
    N = sum(counts)
    off = syn.offsets_from_counts(counts)
    x = rng.uniform(0.4, 0.6, (N, 3))
    d = rng.normal(size=(N, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    w = rng.lognormal(0, 1, N).astype(np.float32)
    w[off[2]:off[3]] = 0.0                       # region 2: zero weight
    w[off[3] + 5] = np.nan                       # region 3: non-finite
    s = _samples(x, d, w)
    st = orc.State(4, K)
    st.pi[:] = 0.5
    st.mu_x[:] = 0.5
    st.mu_w[:] = [0, 0, 1.0]
    st.L[:] = _pack(np.diag([0.1, 0.1, 0.1, 0.5, 0.5]))
    before = st.copy()
    orc.fit_regions(orc.config(K), off, s, 1, st)
    assert list(st.status) == [1, 0, 4, 3]
    for r in (0, 2, 3):
        assert np.array_equal(st.L[r], before.L[r]) and st.n_seen[r] == 0
    # collapsed covariance (identical samples, zero prior scale): the MAP
    # covariance is 0; the numerical floor adds 1e-6 B / a and flags the region
    x2 = np.zeros((50, 3)) + 0.5
    s2 = _samples(x2, np.tile([0, 0, 1.0], (50, 1)), np.ones(50, np.float32))
    st2 = orc.State(1, 1)
    st2.pi[:] = 1
    st2.mu_x[:] = 0.5
    st2.mu_w[:] = [0, 0, 1.0]
    st2.L[:] = _pack(np.eye(5) * 0.1)
    cfg = orc.config(1, prior_scale_mode=1)
    orc.fit_regions(cfg, [0, 50], s2, 1, st2, prior_scale=np.zeros(1))
    assert st2.status[0] == 7 and st2.step_j[0] == 1
    floor = 1e-6 * np.array([cfg.prior_B_pos] * 3 + [cfg.prior_B_dir] * 2)
    assert np.allclose(st2.L[0, 0, [0, 2, 5, 9, 14]], np.sqrt(floor), rtol=1e-6)
