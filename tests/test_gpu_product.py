"""GPU product sampling (Sec. 3.5 product of the conditioned radiance mixture
with the BSDF mixture; top-2 pruning of Sec. 4.1) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle as orc
from oracle import product as prod
from gpu_util import PDF_RTOL, gpu_state
from paper_2111_13094_gb300 import api
from paper_2111_13094_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _mixtures(seed, dims, K):
    pi, mu_x, mu_w, L = syn.random_mixtures(seed, dims, K)
    ost = orc.State(int(np.prod(dims)), K)
    ost.set_params(pi, mu_x, mu_w, L)
    return ost


def _oracle_pairs(ost, K, qx, reg, bw, bmu, bL):
    cpi, cm, cL = orc.condition(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, qx, reg)
    mw = ost.mu_w.reshape(ost.R, K, 3)
    out = []
    for q in range(qx.shape[0]):
        mu_w = mw[reg[q]]
        out.append((prod.pairs(cpi[q], cm[q], cL[q], mu_w, bw[q].astype(np.float64), bmu[q].astype(np.float64),
                               bL[q].astype(np.float64)), mu_w))
    return out


def _transport_gain(ost, K, reg, bw, bmu):
    """Per query: theta / sin(theta) of every formed pair (component mean to
    lobe mean), in the oracle's pair order, and its maximum.  The first-order
    transport J_log has entries of this size, so FP32 rounding of the inputs
    alone moves a pair's Gaussian by about eps * theta / sin(theta): near the
    antipode of a component's chart the product is ill-conditioned and the
    parity bounds scale with this gain (1 for a lobe at the chart centre)."""
    mw = ost.mu_w.reshape(ost.R, K, 3)
    gains, gmax = [], np.ones(len(reg))
    for q in range(len(reg)):
        g = []
        for k in range(K):
            for j in prod.top2(bw[q]):
                nu2, anti, _, _ = orc.log_map(mw[reg[q], k], bmu[q, j].astype(np.float64))
                r = float(np.hypot(*nu2))
                if anti or r >= np.pi:
                    continue
                g.append(r / np.sin(r) if r > 1e-8 else 1.0)
        gains.append(g)
        gmax[q] = max(g, default=1.0)
    return gains, gmax


EPS32 = 2.0 ** -24


def _pdf_condition(pr, mu_w, gains, om):
    """First-order FP32 condition number kappa of the product pdf at om, from
    FP64 oracle quantities: the pdf's relative error is about u * kappa
    (u = 2^-24).  A pair that contributes to the density at om is evaluated in
    the chart of its component, |nu| up to pi away from the chart centre, with
    the narrowed product factor C: an O(u |nu|) error in nu moves its log-density
    by |y| |nu| / sigma_min (y = C^-1 (nu - mean)).  A pair that carries
    weight moves the normalisation through its transport (gain^2, the
    covariance J S2 J^T)."""
    terms, tot = [], 0.0
    for (k, w, mean, P), g in zip(pr, gains):
        nu, anti, _, _ = orc.log_map(mu_w[k], om)
        r = float(np.hypot(*nu))
        if anti or r >= np.pi:
            continue
        C = np.linalg.cholesky(P)
        y = np.linalg.solve(C, nu - mean)
        c = w * np.exp(-0.5 * y @ y) / (2 * np.pi * C[0, 0] * C[1, 1]) / orc.sinc(r)
        smin = float(np.sqrt(np.linalg.eigvalsh(P)[0]))
        terms.append((c, 1.0 + np.linalg.norm(y) * (1.0 + r + np.linalg.norm(mean)) / smin + g * g))
        tot += c
    kw = max((1.0 + g * g for (_, w, _, _), g in zip(pr, gains) if w > 1e-3), default=1.0)
    return max(kw, max((kp for c, kp in terms if c > 1e-3 * tot), default=1.0))


def _angle(a, b):
    a = a / np.linalg.norm(a, axis=1, keepdims=True)
    b = b / np.linalg.norm(b, axis=1, keepdims=True)
    return 2 * np.arcsin(np.clip(np.linalg.norm(a - b, axis=1) / 2, 0, 1))


def _dev(*a):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]


def _sorted(qx, reg):
    """The queries ordered by region (stable): warps then hold one or two
    regions and take the thread-per-query path (K <= 16)."""
    o = np.argsort(reg, kind="stable")
    return np.ascontiguousarray(qx[o]), np.ascontiguousarray(reg[o])


@pytest.mark.parametrize("order", ["given", "sorted"])
@pytest.mark.parametrize("K,J", [(2, 1), (16, 3), (32, 4)])
def test_product_sample_matches_oracle(K, J, order):
    dims = (4, 4, 2)
    ost = _mixtures(21, dims, K)
    cfg = api.config(K)
    st = gpu_state(ost, cfg)
    Q = {2: 4000, 16: 2500, 32: 1500}[K]
    qx = syn.query_points(22, Q)
    reg = syn.grid_region(qx, dims)
    if order == "sorted":
        qx, reg = _sorted(qx, reg)
    bw, bmu, bL = syn.bsdf_lobes(23, Q, J)
    u = np.random.default_rng(24).random((Q, 3), dtype=np.float32)
    tq, tr, tw, tm, tl, tu = _dev(qx, reg, bw, bmu, bL, u)
    d, p, v = api.product_sample(cfg, st, tq, tw, tm, tl, region=tr, uniforms=tu)
    d, p, v = d.cpu().numpy().astype(np.float64), p.cpu().numpy(), v.cpu().numpy()
    prs = _oracle_pairs(ost, K, qx, reg, bw, bmu, bL)
    gains, gq = _transport_gain(ost, K, reg, bw, bmu)
    od, ov, marg, po = np.zeros((Q, 3)), np.zeros(Q, np.uint8), np.zeros(Q), np.zeros(Q)
    gsel = np.ones(Q)
    for q, (pr, mu_w) in enumerate(prs):
        om, _, ok, idx = prod.sample(pr, mu_w, u[q].astype(np.float64))
        od[q], ov[q], marg[q] = om, ok, prod.margin(pr, float(u[q, 0]))
        gsel[q] = gains[q][idx] if idx >= 0 else 1.0
        po[q] = prod.pdf_at(pr, mu_w, d[q]) if v[q] else 0.0
    same = marg > 1e-5                                   # the pair choice is unique
    assert same.mean() > 0.99
    assert np.array_equal(v[same], ov[same])
    ok = same & (ov == 1)
    assert ok.sum() > 0.9 * Q
    # direction: the query contract (1e-4 rad) where the drawn pair's gain is
    # at most 20, growing with the gain beyond
    ang = _angle(d[ok], od[ok])
    assert np.all(ang <= 5e-6 * np.maximum(20.0, gsel[ok])), np.quantile(ang, [0.5, 0.999, 1.0])
    # the reported pdf equals the FP64 product pdf of the returned direction:
    # within 32 u kappa for every query, PDF_RTOL for 99 % of them
    vv = v == 1
    rel = np.abs(p[vv] - po[vv]) / po[vv]
    kap = np.array([_pdf_condition(prs[q][0], prs[q][1], gains[q], d[q]) for q in np.flatnonzero(vv)])
    assert np.quantile(rel, 0.99) < PDF_RTOL, np.quantile(rel, [0.5, 0.99, 0.999, 1.0])
    assert np.all(rel <= 32 * EPS32 * kap), np.quantile(rel / (EPS32 * kap), [0.5, 0.999, 1.0])
    assert np.all(p[~vv] == 0)


@pytest.mark.parametrize("order", ["given", "sorted"])
def test_product_pdf_entry_matches_oracle(order):
    K, J = 16, 3
    dims = (2, 2, 2)
    ost = _mixtures(25, dims, K)
    cfg = api.config(K)
    st = gpu_state(ost, cfg)
    Q = 4000
    qx = syn.query_points(26, Q)
    reg = syn.grid_region(qx, dims)
    if order == "sorted":
        qx, reg = _sorted(qx, reg)
    bw, bmu, bL = syn.bsdf_lobes(27, Q, J)
    rng = np.random.default_rng(28)
    dirs = rng.normal(size=(Q, 3))
    dirs[: Q // 2] = bmu[: Q // 2, 1] + 0.2 * dirs[: Q // 2]     # half of them near the glossy lobe
    dirs = (dirs / np.linalg.norm(dirs, axis=1, keepdims=True)).astype(np.float32)
    tq, tr, tw, tm, tl, td = _dev(qx, reg, bw, bmu, bL, dirs)
    p = api.product_pdf(cfg, st, tq, td, tw, tm, tl, region=tr).cpu().numpy()
    prs = _oracle_pairs(ost, K, qx, reg, bw, bmu, bL)
    po = np.array([prod.pdf_at(pr, mu_w, dirs[q].astype(np.float64)) for q, (pr, mu_w) in enumerate(prs)])
    gains, _ = _transport_gain(ost, K, reg, bw, bmu)
    big = po > 1e-6 * po.max()
    rel = np.abs(p[big] - po[big]) / po[big]
    kap = np.array([_pdf_condition(prs[q][0], prs[q][1], gains[q], dirs[q].astype(np.float64))
                    for q in np.flatnonzero(big)])
    assert np.quantile(rel, 0.99) < PDF_RTOL, np.quantile(rel, [0.5, 0.99, 0.999, 1.0])
    assert np.all(rel <= 32 * EPS32 * kap), np.quantile(rel / (EPS32 * kap), [0.5, 0.999, 1.0])
    assert np.abs(p - po).max() < 1e-4 * po.max()


@pytest.mark.parametrize("order", ["given", "sorted"])
def test_product_philox_and_grid_paths_are_exact(order):
    K, J = 16, 2
    dims = (4, 4, 4)
    ost = _mixtures(29, dims, K)
    cfg = api.config(K)
    st = gpu_state(ost, cfg)
    Q = 20000
    qx = syn.query_points(30, Q)
    reg = syn.grid_region(qx, dims)
    if order == "sorted":
        qx, reg = _sorted(qx, reg)
    bw, bmu, bL = syn.bsdf_lobes(31, Q, J)
    u = orc.uniforms(99, Q)
    tq, tr, tw, tm, tl, tu = _dev(qx, reg, bw, bmu, bL, u)
    a = api.product_sample(cfg, st, tq, tw, tm, tl, region=tr, uniforms=tu)
    b = api.product_sample(cfg, st, tq, tw, tm, tl, grid=api.Grid((0, 0, 0), (1, 1, 1), dims), seed=99)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_product_edge_cases():
    """Empty batch; a lobe at the exact antipode of a component gives no pair
    with it; a zero-weight lobe gives pairs of zero weight."""
    K = 4
    dims = (1, 1, 1)
    pi, mu_x, mu_w, L = syn.random_mixtures(32, dims, K)
    mu_w[0, 1] = [0.0, 0.0, 1.0]                                        # chart basis exact in FP32
    ost = orc.State(1, K)
    ost.set_params(pi, mu_x, mu_w, L)
    cfg = api.config(K)
    st = gpu_state(ost, cfg)
    e = torch.empty(0, 3, device="cuda")
    d, p, v = api.product_sample(cfg, st, e, torch.empty(0, 2, device="cuda"), torch.empty(0, 2, 3, device="cuda"),
                                 torch.empty(0, 2, 3, device="cuda"),
                                 grid=api.Grid((0, 0, 0), (1, 1, 1), dims))
    assert d.shape == (0, 3) and p.numel() == 0 and v.numel() == 0
    Q = 64
    qx = np.full((Q, 3), 0.5, np.float32)
    reg = np.zeros(Q, np.int32)
    mw = ost.mu_w.reshape(K, 3)
    bw = np.tile(np.array([[0.0, 1.0]], np.float32), (Q, 1))          # lobe 0 has no weight
    bmu = np.zeros((Q, 2, 3), np.float32)
    bmu[:, 0] = mw[0]
    bmu[:, 1] = [0.0, 0.0, -1.0]                                       # antipode of component 1
    bL = np.tile(np.array([[[0.2, 0.0, 0.2]]], np.float32), (Q, 2, 1))
    u = np.random.default_rng(33).random((Q, 3), dtype=np.float32)
    tq, tr, tw, tm, tl, tu = _dev(qx, reg, bw, bmu, bL, u)
    d, p, v = api.product_sample(cfg, st, tq, tw, tm, tl, region=tr, uniforms=tu)
    prs = _oracle_pairs(ost, K, qx, reg, bw, bmu, bL)
    live = [(k, w) for k, w, _, _ in prs[0][0] if w > 0]
    assert len(live) == K - 1 and all(k != 1 for k, _ in live)
    d, p, v = d.cpu().numpy().astype(np.float64), p.cpu().numpy(), v.cpu().numpy()
    po = np.array([prod.pdf_at(prs[q][0], mw, d[q]) if v[q] else 0.0 for q in range(Q)])
    vv = v == 1
    assert vv.mean() > 0.9
    gains, _ = _transport_gain(ost, K, reg, bw, bmu)
    kap = np.array([_pdf_condition(prs[q][0], mw, gains[q], d[q]) for q in range(Q)])
    assert np.all(np.abs(p[vv] - po[vv]) <= 32 * EPS32 * kap[vv] * po[vv])
