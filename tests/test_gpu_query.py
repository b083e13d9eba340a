"""GPU query path (condition, sample, pdf) against the FP64 oracle, on small
cases and on sampled outputs of the 16M-query / 65,536-region workload."""
import math

import numpy as np
import pytest
import torch
from scipy import stats

import oracle as orc
from gpu_util import EPS32, PDF_RTOL, assert_pdf_close, gpu_state, pdf_kappa
from paper_2111_13094_gb300 import api
from paper_2111_13094_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _mixtures(seed, dims, K):
    pi, mu_x, mu_w, L = syn.random_mixtures(seed, dims, K)
    R = int(np.prod(dims))
    ost = orc.State(R, K)
    ost.set_params(pi, mu_x, mu_w, L)
    return ost


def _queries(seed, Q, dims):
    qx = syn.query_points(seed, Q)
    return qx, syn.grid_region(qx, dims)


@pytest.mark.parametrize("K", [1, 3, 16, 32])
def test_condition_matches_oracle(K):
    dims = (4, 4, 2)
    ost = _mixtures(1, dims, K)
    cfg = api.config(K)
    st = gpu_state(ost, cfg)
    qx, reg = _queries(2, 3000, dims)
    cpi, cm, cL = api.condition(cfg, st, torch.from_numpy(qx).cuda(), region=torch.from_numpy(reg).cuda())
    opi, om, oL = orc.condition(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, qx, reg)
    assert np.abs(cpi.cpu().numpy() - opi).max() < 2e-5
    assert np.abs(cm.cpu().numpy() - om).max() < 1e-5 * max(1.0, np.abs(om).max())
    assert np.allclose(cL.cpu().numpy(), oL, rtol=1e-6)


def _angle(a, b):
    a = a / np.linalg.norm(a, axis=1, keepdims=True)
    b = b / np.linalg.norm(b, axis=1, keepdims=True)
    return 2 * np.arcsin(np.clip(np.linalg.norm(a - b, axis=1) / 2, 0, 1))


@pytest.mark.parametrize("K", [2, 16, 32])
def test_sample_and_pdf_match_oracle(K):
    dims = (4, 4, 4)
    ost = _mixtures(3, dims, K)
    cfg = api.config(K)
    st = gpu_state(ost, cfg)
    Q = 20000
    qx, reg = _queries(4, Q, dims)
    u = np.random.default_rng(5).random((Q, 3), dtype=np.float32)
    d, p, v = api.sample(cfg, st, torch.from_numpy(qx).cuda(), region=torch.from_numpy(reg).cuda(),
                         uniforms=torch.from_numpy(u).cuda())
    d, p, v = d.cpu().numpy(), p.cpu().numpy(), v.cpu().numpy()
    o = orc.sample(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, qx, reg, u)
    same = o["margin"] > 1e-5                          # component choice is unique
    assert same.mean() > 0.999
    assert np.array_equal(v[same], o["valid"][same])
    ok = same & (o["valid"] == 1)
    assert _angle(d[ok].astype(np.float64), o["dir"][ok]).max() < 1e-4
    # the reported pdf equals the FP64 pdf of the returned (FP32) direction
    po = orc.pdf(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, qx, reg, d.astype(np.float64))
    vv = v == 1
    rel = assert_pdf_close(p[vv], po[vv], ost, K, qx[vv], reg[vv], d[vv].astype(np.float64))
    print(K, "pdf rel quantiles", np.quantile(rel, [0.5, 0.99, 0.999, 1.0]))
    assert np.all(p[~vv] == 0)


def test_pdf_entry_matches_oracle():
    K = 16
    dims = (2, 2, 2)
    ost = _mixtures(6, dims, K)
    cfg = api.config(K)
    st = gpu_state(ost, cfg)
    Q = 20000
    qx, reg = _queries(7, Q, dims)
    rng = np.random.default_rng(8)
    dirs = rng.normal(size=(Q, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    dirs = dirs.astype(np.float32)
    p = api.pdf(cfg, st, torch.from_numpy(qx).cuda(), torch.from_numpy(dirs).cuda(),
                region=torch.from_numpy(reg).cuda()).cpu().numpy()
    po = orc.pdf(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, qx, reg, dirs.astype(np.float64))
    big = po > 1e-6 * po.max()
    rel = assert_pdf_close(p[big], po[big], ost, K, qx[big], reg[big], dirs[big].astype(np.float64))
    print("pdf entry rel quantiles", np.quantile(rel, [0.5, 0.99, 0.999, 1.0]))
    assert np.abs(p - po).max() < 1e-5 * po.max()


def test_philox_and_grid_paths_are_exact():
    """Device Philox uniforms equal the oracle's bit for bit, and the grid
    lookup gives the generator's cell ids."""
    K = 16
    dims = (8, 4, 4)
    ost = _mixtures(9, dims, K)
    cfg = api.config(K)
    st = gpu_state(ost, cfg)
    Q = 50000
    qx, reg = _queries(10, Q, dims)
    tq = torch.from_numpy(qx).cuda()
    u = orc.uniforms(1234, Q)
    a = api.sample(cfg, st, tq, region=torch.from_numpy(reg).cuda(), uniforms=torch.from_numpy(u).cuda())
    b = api.sample(cfg, st, tq, grid=api.Grid((0, 0, 0), (1, 1, 1), dims), seed=1234)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_sample_histogram_chi_square_on_gpu():
    K = 3
    rng = np.random.default_rng(11)
    pi = rng.dirichlet(np.ones(K))[None]
    mu_x = rng.uniform(0.3, 0.7, (1, K, 3))
    mu_w = rng.normal(size=(1, K, 3))
    mu_w /= np.linalg.norm(mu_w, axis=2, keepdims=True)
    L = np.zeros((1, K, 15))
    for k in range(K):
        diag = np.concatenate([rng.uniform(0.05, 0.2, 3), rng.uniform(0.4, 1.1, 2)])
        for i in range(5):
            for j in range(i + 1):
                L[0, k, i * (i + 1) // 2 + j] = diag[i] if i == j else 0.4 * rng.normal() * diag[i]
    ost = orc.State(1, K)
    ost.set_params(pi, mu_x, mu_w, L)
    cfg = api.config(K)
    st = gpu_state(ost, cfg)
    N = 1_000_000
    x = np.tile(np.array([[0.5, 0.5, 0.5]], np.float32), (N, 1))
    d, p, v = api.sample(cfg, st, torch.from_numpy(x).cuda(), region=torch.zeros(N, dtype=torch.int32).cuda(),
                         seed=77)
    d, v = d.cpu().numpy(), v.cpu().numpy().astype(bool)
    n_z, n_phi, sub = 12, 24, 6
    xs, ws = np.polynomial.legendre.leggauss(sub)
    mass = np.zeros(n_z * n_phi)
    dirs, wts = [], []
    for iz in range(n_z):
        z0, z1 = -1 + 2 * iz / n_z, -1 + 2 * (iz + 1) / n_z
        for ip in range(n_phi):
            p0, p1 = 2 * math.pi * ip / n_phi, 2 * math.pi * (ip + 1) / n_phi
            Z, P = np.meshgrid((xs + 1) / 2 * (z1 - z0) + z0, (xs + 1) / 2 * (p1 - p0) + p0, indexing="ij")
            s = np.sqrt(1 - Z * Z)
            dirs.append(np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3))
            wts.append((np.outer(ws, ws) * (z1 - z0) / 2 * (p1 - p0) / 2).reshape(-1))
    dirs, wts = np.concatenate(dirs), np.concatenate(wts)
    pq = orc.pdf(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, np.repeat(x[:1], len(dirs), 0),
                 np.zeros(len(dirs), np.int32), dirs)
    mass = (pq * wts).reshape(n_z * n_phi, -1).sum(1)
    dd = d[v].astype(np.float64)
    iz = np.minimum(((dd[:, 2] + 1) / 2 * n_z).astype(int), n_z - 1)
    ph = np.mod(np.arctan2(dd[:, 1], dd[:, 0]), 2 * math.pi)
    ip = np.minimum((ph / (2 * math.pi) * n_phi).astype(int), n_phi - 1)
    counts = np.bincount(iz * n_phi + ip, minlength=n_z * n_phi)
    obs = np.append(counts, (~v).sum()).astype(float)
    exp = np.append(mass, 1 - mass.sum()) * N
    keep = exp >= 5
    obs = np.append(obs[keep], obs[~keep].sum())
    exp = np.append(exp[keep], exp[~keep].sum())
    if exp[-1] <= 0:
        obs, exp = obs[:-1], exp[:-1]
    chi2 = float(np.sum((obs - exp) ** 2 / exp))
    assert stats.chi2.sf(chi2, obs.size - 1) > 1e-3, chi2


def test_query_workload_16M_sampled_against_oracle():
    """16M query positions uniform in the unit cube, 65,536 grid regions with
    K = 16 mixtures, one Philox draw per query; 20,000 sampled queries are
    recomputed by the oracle."""
    K = 16
    dims = (64, 32, 32)
    ost = _mixtures(12, dims, K)
    cfg = api.config(K)
    st = gpu_state(ost, cfg)
    Q = 16 * 2 ** 20
    qx = syn.query_points(13, Q)
    tq = torch.from_numpy(qx).cuda()
    # the launch configuration the benchmark times: queries as given, binned by
    # region in the library's workspace
    d, p, v = api.sample(cfg, st, tq, grid=api.Grid((0, 0, 0), (1, 1, 1), dims), seed=99,
                         ws=api.query_workspace(st.R, Q))
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(14).choice(Q, 20000, replace=False))
    u = orc.uniforms(99, Q)[idx]
    reg = syn.grid_region(qx[idx], dims)
    o = orc.sample(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, qx[idx], reg, u)
    dg = d[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    vg = v[torch.from_numpy(idx).cuda()].cpu().numpy()
    pg = p[torch.from_numpy(idx).cuda()].cpu().numpy()
    same = o["margin"] > 1e-5
    assert np.array_equal(vg[same], o["valid"][same])
    ok = same & (o["valid"] == 1)
    assert _angle(dg[ok], o["dir"][ok]).max() < 1e-4
    po = orc.pdf(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, qx[idx], reg, dg)
    vv = vg == 1
    assert_pdf_close(pg[vv], po[vv], ost, K, qx[idx][vv], reg[vv], dg[vv])
    # discard rate (|nu| >= pi) is small, as the paper reports for its lobes
    assert 1.0 - v.float().mean().item() < 0.01


@pytest.mark.parametrize("K", [3, 16, 32])
def test_binned_entry_points_match_the_oracle(K):
    """sdmm_sample_binned / sdmm_pdf_binned (queries in any order, binned by
    region inside the library) against the oracle on the same queries and
    uniforms: validity, directions and pdfs under the sampling tolerances,
    with region ids (including ids out of range: valid = 0, pdf = 0) and with
    the grid lookup; a short workspace is rejected."""
    dims = (8, 4, 4)
    ost = _mixtures(21, dims, K)
    cfg = api.config(K)
    st = gpu_state(ost, cfg)
    Q = 40000
    qx, reg = _queries(22, Q, dims)
    reg = reg.copy()
    reg[::997] = -1
    tq, tr = torch.from_numpy(qx).cuda(), torch.from_numpy(reg).cuda()
    ws = api.query_workspace(st.R, Q)
    grid = api.Grid((0, 0, 0), (1, 1, 1), dims)
    u = orc.uniforms(77, Q)
    good = reg >= 0
    o = orc.sample(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, qx[good], reg[good], u[good])
    same = o["margin"] > 1e-5
    for kw, sel in ((dict(region=tr), good), (dict(grid=grid), np.ones(Q, bool))):
        dt, pt, vt = api.sample(cfg, st, tq, seed=77, ws=ws, **kw)
        # the binned pdf entry at the sampled directions
        pe = api.pdf(cfg, st, tq, dt, ws=ws, **kw).cpu().numpy()[good]
        d, p, v = dt.cpu().numpy(), pt.cpu().numpy(), vt.cpu().numpy()
        if "region" in kw:
            assert not v[~good].any() and not p[~good].any()
        d, p, v = d[good], p[good], v[good]
        assert np.array_equal(v[same], o["valid"][same])
        ok = same & (o["valid"] == 1)
        assert _angle(d[ok].astype(np.float64), o["dir"][ok]).max() < 1e-4
        vv = v == 1
        po = orc.pdf(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, qx[good][vv], reg[good][vv], d[vv].astype(np.float64))
        assert_pdf_close(p[vv], po, ost, K, qx[good][vv], reg[good][vv], d[vv].astype(np.float64))
        assert_pdf_close(pe[vv], po, ost, K, qx[good][vv], reg[good][vv], d[vv].astype(np.float64))
    if K <= 16:                                       # the binned path needs its workspace
        with pytest.raises(api.SdmmError):
            api.sample(cfg, st, tq, seed=77, region=tr, ws=ws[: ws.numel() // 2])


@pytest.mark.parametrize("K", [2, 16])
def test_empty_and_ragged_query_batches(K):
    """No queries (every entry point returns empty outputs); 37 queries of one
    region (one warp plus a ragged tail, all through the thread-per-query
    path) and the same 37 queries through the library's binning, where the
    bin is padded to two warps: both agree with the oracle."""
    dims = (2, 2, 2)
    ost = _mixtures(41, dims, K)
    cfg = api.config(K)
    st = gpu_state(ost, cfg)
    grid = api.Grid((0, 0, 0), (1, 1, 1), dims)
    e = torch.empty(0, 3, device="cuda")
    ws0 = api.query_workspace(st.R, 0)
    for kw in (dict(grid=grid), dict(grid=grid, ws=ws0)):
        d, p, v = api.sample(cfg, st, e, seed=1, **kw)
        assert d.shape == (0, 3) and p.numel() == 0 and v.numel() == 0
        assert api.pdf(cfg, st, e, e, **kw).numel() == 0
    Q = 37
    rng = np.random.default_rng(42)
    qx = (0.5 * rng.random((Q, 3)) + np.array([0.5, 0.0, 0.5])).astype(np.float32)   # all in cell (1, 0, 1)
    reg = syn.grid_region(qx, dims)
    assert np.all(reg == reg[0])
    u = orc.uniforms(43, Q)
    o = orc.sample(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, qx, reg, u)
    same = o["margin"] > 1e-5
    tq = torch.from_numpy(qx).cuda()
    ws = api.query_workspace(st.R, Q)
    for kw in (dict(region=torch.from_numpy(reg).cuda()), dict(grid=grid, ws=ws)):
        d, p, v = (t.cpu().numpy() for t in api.sample(cfg, st, tq, seed=43, **kw))
        assert np.array_equal(v[same], o["valid"][same])
        ok = same & (o["valid"] == 1)
        assert _angle(d[ok].astype(np.float64), o["dir"][ok]).max() < 1e-4
        vv = v == 1
        po = orc.pdf(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, qx[vv], reg[vv], d[vv].astype(np.float64))
        assert_pdf_close(p[vv], po, ost, K, qx[vv], reg[vv], d[vv].astype(np.float64))


def _far_mixture(seed, K):
    """One region's K components with narrow positions (std 1e-3 to 4e-3) and
    weak position-direction coupling, so that a position tenths away from
    every mean is tens to hundreds of standard deviations out while the
    conditional mean m = L21 z stays well inside the chart."""
    pi, mu_x, mu_w, L = syn.random_mixtures(seed, (1, 1, 1), K)
    for i in range(5):
        for j in range(min(i + 1, 3)):
            L[..., i * (i + 1) // 2 + j] *= 0.02 if i < 3 else 0.002
    ost = orc.State(1, K)
    ost.set_params(pi, mu_x, mu_w, L)
    return ost


def _spatial_terms(ost, K, qx):
    """Per query and component, in FP64: |z_k|^2 with z_k = A_k^-1 (x - mu_k),
    and log2 of pi_k N_3(x; mu_k, A_k A_k^T) less the region's bound (its
    largest log2 of pi_k / ((2 pi)^(3/2) det A_k))."""
    Lp = ost.L.reshape(K, 15)
    mu = ost.mu_x.reshape(K, 3)
    pi = ost.pi.reshape(K)
    z2 = np.empty((qx.shape[0], K))
    cx = np.empty(K)
    for k in range(K):
        A = np.zeros((3, 3))
        for i in range(3):
            for j in range(i + 1):
                A[i, j] = Lp[k, i * (i + 1) // 2 + j]
        z = np.linalg.solve(A, (qx.astype(np.float64) - mu[k]).T)
        z2[:, k] = (z * z).sum(axis=0)
        cx[k] = np.log(pi[k]) - np.log(np.diag(A)).sum() - 1.5 * np.log(2 * np.pi)
    lw2 = (cx[None, :] - 0.5 * z2 - cx.max()) / np.log(2.0)
    return z2, lw2


@pytest.mark.parametrize("K", [3, 16])
def test_far_positions_take_the_exact_maximum(K):
    """Positions far from every component of their region: every conditioned
    weight pi_k N_3(x) lies more than 2^110 below the region's bound, so the
    weights shifted by the bound underflow and the kernel redoes them with the
    exact per-query maximum (a broken redo gives pdf 0 and valid 0 for all).
    Validity and directions match the oracle where its component choice has a
    margin of 1e-2 (the FP32 weights of near-tied components differ from the
    FP64 ones by about eps |z|^2); each pdf, of the sample entry and of the pdf
    entry at the same direction, is within 32 eps times its condition number,
    here the direction part plus the largest |z_k|^2 of the components that
    carry 1e-3 of the conditioned weight (the rounding of their spatial
    Mahalanobis terms)."""
    ost = _far_mixture(61, K)
    qx = syn.query_points(62, 6000)
    z2, lw2 = _spatial_terms(ost, K, qx)
    far = lw2.max(axis=1) < -110.0
    assert far.mean() > 0.9
    qx = np.ascontiguousarray(qx[far])
    z2, lw2 = z2[far], lw2[far]
    Q = qx.shape[0]
    reg = np.zeros(Q, np.int32)
    cfg = api.config(K)
    st = gpu_state(ost, cfg)
    tq, tr = torch.from_numpy(qx).cuda(), torch.from_numpy(reg).cuda()
    dt, pt, vt = api.sample(cfg, st, tq, region=tr, seed=63)
    pe = api.pdf(cfg, st, tq, dt, region=tr).cpu().numpy()
    d, p, v = dt.cpu().numpy(), pt.cpu().numpy(), vt.cpu().numpy()
    o = orc.sample(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, qx, reg, orc.uniforms(63, Q))
    same = o["margin"] > 1e-2
    assert same.mean() > 0.9
    assert np.array_equal(v[same], o["valid"][same])
    assert v.mean() > 0.5
    ok = same & (o["valid"] == 1)
    assert _angle(d[ok].astype(np.float64), o["dir"][ok]).max() < 1e-4
    vv = np.flatnonzero(v == 1)
    po = orc.pdf(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, qx[vv], reg[vv], d[vv].astype(np.float64))
    w = np.exp2(lw2[vv] - lw2[vv].max(axis=1, keepdims=True))
    w /= w.sum(axis=1, keepdims=True)
    zc2 = np.where(w >= 1e-3, z2[vv], 0.0).max(axis=1)
    for pg in (p[vv], pe[vv]):
        rel = np.abs(pg - po) / po
        assert np.all(np.isfinite(rel))
        print(K, "far-position pdf rel quantiles", np.quantile(rel, [0.5, 0.99, 1.0]))
        for q in np.flatnonzero(rel >= PDF_RTOL):
            kap = pdf_kappa(ost, K, qx[vv[q]], 0, d[vv[q]].astype(np.float64))
            assert rel[q] < 32 * EPS32 * (kap + zc2[q]), (q, rel[q], kap, zc2[q])
