"""Contraction-form E-step on the tensor cores (split 3xBF16, TF32, split
3xTF32, three-piece 6xBF16) against the FP64 oracle on the same inputs, one
EM step of ragged regions for K = 16 and 32.  The split-TF32 and 6xBF16
forms meet the parity contract; the other two are bounded (precision
sweep).  The two contract forms also with the solid-angle E-step density."""
import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import LOGLIK_RTOL, PARAM_RTOL, assert_params_close, block_err, dev_batch, gpu_state, host, \
    loglik_err, oracle_init
from paper_2111_13094_gb300 import api
from paper_2111_13094_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

# FP32-level rounding of the direction quadratic T2 of the contraction form,
# relative to the log density it enters multiplied by g^2 (solid-angle test)
EPS_T2 = 1e-6

MODES = {"3xbf16": api.PREC_TC_3XBF16, "tf32": api.PREC_TC_TF32, "3xtf32": api.PREC_TC_3XTF32,
         "6xbf16": api.PREC_TC_6XBF16}


def _errors(K, prec, seed, counts=(16, 200, 3001, 9000), iters=1, density=0):
    truth = syn.batched_truth(seed, len(counts), K=K, parallax=True)
    b = syn.batched_round(seed, len(counts), np.asarray(counts), 0, truth)
    ost = oracle_init(seed, b, K)
    gcfg = api.config(K, precision=prec, estep_density=density)
    st = gpu_state(ost, gcfg)
    oll = orc.fit_regions(orc.config(K, estep_density=density), b.offsets, b.samples, iters, ost,
                          want_loglik=True)
    ll = torch.zeros(b.N, dtype=torch.float32, device="cuda")
    api.fit_regions(gcfg, dev_batch(b), iters, st, api.workspace(gcfg, b.R, b.N), loglik=ll)
    g = host(st)
    ok = ost.status == 0
    e = {"loglik": loglik_err(ll.cpu().numpy(), oll),
         "pi": float(np.abs(g.pi - ost.pi)[ok].max()),
         "mu_x": float(np.abs(g.mu_x - ost.mu_x)[ok].max()),
         "mu_w": float(np.abs(g.mu_w - ost.mu_w)[ok].max()),
         "L": block_err(g.L[ok], ost.L[ok]),
         "status": list(g.status), "ostatus": list(ost.status)}
    return e, g, ost


@pytest.mark.parametrize("K", [16, 32])
@pytest.mark.parametrize("mode", list(MODES))
def test_tc_estep_one_step(K, mode):
    e, g, ost = _errors(K, MODES[mode], 200 + K)
    print(f"K={K} {mode}: {e}")
    assert e["status"] == e["ostatus"] and 6 not in e["status"]
    if mode in ("3xtf32", "6xbf16"):
        assert e["loglik"] < LOGLIK_RTOL
        assert_params_close(g, ost)
    elif mode == "3xbf16":
        # about one extra decimal digit lost to the expanded quadratic forms
        assert e["loglik"] < 5e-4 and e["L"] < 5e-3
    else:
        # plain TF32 (10-bit mantissa) misses the 1e-4 contract by design;
        # bound it so that a broken kernel still fails
        assert 1e-3 < e["loglik"] < 0.5 and e["L"] < 0.05


def _antipode_weight(seed, K, counts):
    """Per sample, lambda_i = sum_k r_ik g_ik^2 at the initial state (FP64
    oracle), g = theta / sin(theta).  The contraction form evaluates the
    direction quadratic of the Mahalanobis term as g^2 T2 with T2 a product
    of direction features and coefficients (Sec. 3.1 log map in the expanded
    form), so the FP32-level rounding of T2 reaches the log density
    multiplied by g^2, which grows as 1 / sin^2 near a component's antipode;
    the solid-angle density weights those components up by g."""
    truth = syn.batched_truth(seed, len(counts), K=K, parallax=True)
    b = syn.batched_round(seed, len(counts), np.asarray(counts), 0, truth)
    ost = oracle_init(seed, b, K)
    cfg = orc.config(K, estep_density=api.DENSITY_SOLID_ANGLE)
    lam = np.zeros(b.N)
    for r in range(b.R):
        o0, o1 = int(b.offsets[r]), int(b.offsets[r + 1])
        if ost.status[r] != 0 or o1 == o0:
            continue
        s = b.samples[:, o0:o1]
        out = orc.estep_region(cfg, ost.pi[r], ost.mu_x[r], ost.mu_w[r], ost.L[r], s)
        w = s[3:6].T.astype(np.float64)
        w /= np.linalg.norm(w, axis=1, keepdims=True)
        sin = np.linalg.norm(np.cross(w[:, None, :], ost.mu_w[r][None, :, :]), axis=2)
        cos = np.einsum("mc,kc->mk", w, ost.mu_w[r])
        th = np.arctan2(sin, cos)
        g = np.where(sin > 0, th / np.maximum(sin, 1e-300), 1.0)
        lam[o0:o1] = np.sum(out["resp"] * g * g, axis=1)
    return lam


@pytest.mark.parametrize("K", [16, 32])
@pytest.mark.parametrize("mode", ["3xtf32", "6xbf16"])
def test_tc_estep_solid_angle_density(K, mode):
    """The solid-angle E-step density (Sec. 3.1 Eq. solidangle-pdf inside
    Sec. 3.2 Eq. em-ss-computation: p^t / sinc |nu|) in the contraction
    forms that meet the contract: one EM step against the oracle's.  The
    per-sample log-likelihood is held to the 1e-4 contract plus the
    conditioning of the contraction form near a component's antipode,
    EPS_T2 * sum_k r_k g_k^2 (see _antipode_weight)."""
    counts = (16, 200, 3001, 9000)
    seed = 300 + K
    truth = syn.batched_truth(seed, len(counts), K=K, parallax=True)
    b = syn.batched_round(seed, len(counts), np.asarray(counts), 0, truth)
    ost = oracle_init(seed, b, K)
    dens = api.DENSITY_SOLID_ANGLE
    gcfg = api.config(K, precision=MODES[mode], estep_density=dens)
    st = gpu_state(ost, gcfg)
    lam = _antipode_weight(seed, K, counts)
    oll = orc.fit_regions(orc.config(K, estep_density=dens), b.offsets, b.samples, 1, ost, want_loglik=True)
    ll = torch.zeros(b.N, dtype=torch.float32, device="cuda")
    api.fit_regions(gcfg, dev_batch(b), 1, st, api.workspace(gcfg, b.R, b.N), loglik=ll)
    g = host(st)
    assert list(g.status) == list(ost.status)
    err = np.abs(ll.cpu().numpy().astype(np.float64) - oll)
    live = np.isfinite(oll)
    floor = LOGLIK_RTOL * np.maximum(1.0, np.abs(oll))
    over = live & (err > floor)
    ratio = np.where(over, (err - floor) / np.maximum(lam, 1e-300), 0.0)
    print(f"K={K} {mode} solid angle: max err {err[live].max():.3g}; {int(over.sum())} of {b.N} samples "
          f"above 1e-4, their (err - 1e-4) / lambda at most {ratio.max():.3g}; lambda max {lam.max():.3g}")
    assert np.all(err[live] <= floor[live] + EPS_T2 * lam[live])
    # L: the statistics are uncentred feature moments in split BF16, whose
    # cancellation in the direction block (about 1 / sigma_dir^2) the
    # solid-angle weights g = theta / sin(theta) > 1 enlarge; measured 1.75e-3
    # here, held to the 3xBF16 bound
    assert_params_close(g, ost, L_rtol=5e-3)
