"""Helpers shared by the GPU parity tests: move seeded inputs and oracle
states to the device and compare results with stated tolerances."""
import numpy as np
import torch

import oracle as orc
from paper_2111_13094_gb300 import api
from paper_2111_13094_gb300 import synthetic as syn

# tolerances of the parity contract (GPU FP32 vs FP64 oracle)
LOGLIK_RTOL = 1e-4     # per-sample log-likelihood, relative (floor 1)
PARAM_RTOL = 1e-3      # parameters, relative to each block's magnitude
PDF_RTOL = 1e-5        # pdf at the GPU's direction, re-evaluated in FP64


def dev_batch(b) -> api.SampleBatch:
    return api.SampleBatch(torch.from_numpy(np.ascontiguousarray(b.samples)).cuda(),
                           torch.from_numpy(np.ascontiguousarray(b.offsets)).cuda())


def gpu_state(ost: orc.State, cfg) -> api.MixtureState:
    st = api.MixtureState(ost.R, ost.K)
    for f in orc.State.FIELDS:
        getattr(st, f).copy_(torch.from_numpy(getattr(ost, f)))
    api.prepare(cfg, st)
    return st


def host(st: api.MixtureState) -> orc.State:
    o = orc.State(st.R, st.K)
    for f in orc.State.FIELDS:
        getattr(o, f)[...] = getattr(st, f).cpu().numpy()
    return o


def block_err(g, o, ok=None):
    """max over components of max|g - o| / max(|o|) within the component."""
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    if o.ndim == 2:
        g, o = g[..., None], o[..., None]
    scale = np.maximum(np.abs(o).max(axis=-1, keepdims=True), 1e-12)
    e = (np.abs(g - o) / scale).max(axis=-1)
    if ok is not None:
        e = e[ok]
    return float(e.max()) if e.size else 0.0


def assert_params_close(g: orc.State, o: orc.State, regions=None, rtol=PARAM_RTOL, L_rtol=None):
    ok = (o.status == 0)
    if regions is not None:
        ok = ok & np.isin(np.arange(o.R), regions)
    assert np.array_equal(g.status[ok], o.status[ok])
    # weights: relative to the region's largest weight
    pe = np.abs(g.pi - o.pi)[ok].max(initial=0.0) / max(o.pi[ok].max(initial=1.0), 1e-12)
    assert pe < rtol, ("pi", pe)
    # positions: relative to the spread of the region's means (its cell size)
    for r in np.where(ok)[0]:
        span = max(np.ptp(o.mu_x[r], axis=0).max(), 1e-3)
        assert np.abs(g.mu_x[r] - o.mu_x[r]).max() < rtol * span, ("mu_x", r)
    assert np.abs(g.mu_w - o.mu_w)[ok].max(initial=0.0) < rtol, "mu_w"
    e = block_err(g.L[ok], o.L[ok])
    assert e < (rtol if L_rtol is None else L_rtol), ("L", e)


def oracle_init(seed, b, K, cfg_over=None):
    cfg = orc.config(K, **(cfg_over or {}))
    n_pos = K // 8 if K % 8 == 0 else 1
    ost = orc.State(b.R, K)
    orc.init_regions(cfg, b.offsets, b.samples, b.extent, syn.init_uniforms(seed, b.R, n_pos), ost)
    return ost


def loglik_err(g, o, mask=None):
    g = np.asarray(g, np.float64)
    e = np.abs(g - o) / np.maximum(1.0, np.abs(o))
    if mask is not None:
        e = e[mask]
    return float(e.max()) if e.size else 0.0


EPS32 = 2.0 ** -24


def pdf_kappa(ost, K, x, r, om):
    """First-order FP32 condition number of the conditioned mixture's pdf at
    direction om (FP64 oracle quantities).  A component contributes
    pi'_k N_2(y_k) g_k with nu_k = log_{mu_k}(om), y_k = D_k^-1 (nu_k - m_k),
    g_k = theta/sin(theta).  Rounding the chart coordinates of om moves nu_k by
    about eps (1 + g_k theta_k) (the log map's gain), so y_k by that over the
    smallest singular value of D_k, and the exponent -|y|^2/2 by |y_k| times
    that, plus its own rounding eps |y_k|^2:
        kappa = max_k 1 + (1 + g_k theta_k) |y_k| / s_min(D_k) + |y_k|^2
    over the components carrying at least 1e-3 of the pdf.  The pdf's relative
    error is about eps * kappa."""
    cpi, cm, cL = orc.condition(K, ost.pi, ost.mu_x, ost.mu_w, ost.L, x[None].astype(np.float32),
                                np.array([r], np.int32))
    mw = ost.mu_w.reshape(ost.R, K, 3)[r]
    terms, kap = [], []
    for k in range(K):
        nu, anti, th, sn = orc.log_map(mw[k], om)
        D = np.array([[cL[0, k, 0], 0.0], [cL[0, k, 1], cL[0, k, 2]]])
        if anti or np.hypot(*nu) >= np.pi:
            continue
        g = th / sn if sn > 0 else 1.0
        y = np.linalg.solve(D, nu - cm[0, k])
        ny = float(np.linalg.norm(y))
        smin = float(np.linalg.svd(D, compute_uv=False).min())
        terms.append(cpi[0, k] * np.exp(-0.5 * ny * ny) / (2 * np.pi * abs(np.linalg.det(D))) * g)
        kap.append(1.0 + (1.0 + g * th) * ny / smin + ny * ny)
    if not terms:
        return 1.0
    p = sum(terms)
    return max((kk for t, kk in zip(terms, kap) if t >= 1e-3 * p), default=1.0)


def assert_pdf_close(p_gpu, p_oracle, ost, K, qx, reg, dirs, bulk=0.999):
    """pdf parity: every value within max(PDF_RTOL, 32 eps kappa) of the FP64
    pdf at the same direction, and the contract PDF_RTOL itself for the bulk."""
    rel = np.abs(p_gpu - p_oracle) / p_oracle
    assert np.mean(rel < PDF_RTOL) >= bulk, np.quantile(rel, [0.5, 0.99, 0.999, 1.0])
    for q in np.flatnonzero(rel >= PDF_RTOL):
        kap = pdf_kappa(ost, K, qx[q], int(reg[q]), dirs[q])
        assert rel[q] < 32 * EPS32 * kap, (q, rel[q], kap)
    return rel
