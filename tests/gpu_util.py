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


def assert_params_close(g: orc.State, o: orc.State, regions=None, rtol=PARAM_RTOL):
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
    assert e < rtol, ("L", e)


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
