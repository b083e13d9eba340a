"""GPU MAP objective and its hand-written adjoint against the FP64 oracle's
value, its analytic gradient and central finite differences; the autograd
wrapper; sampled regions of the 1,024 x 16,384 workload."""
import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import dev_batch, gpu_state, oracle_init
from paper_2111_13094_gb300 import api
from paper_2111_13094_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _case(seed, R, K, M):
    truth = syn.batched_truth(seed, R, K=K, parallax=True)
    b = syn.batched_round(seed, R, np.full(R, M), 0, truth)
    ost = oracle_init(seed, b, K)
    orc.fit_regions(orc.config(K, eta_mode=1), b.offsets, b.samples, 3, ost)
    return b, ost


def _rel(g, o):
    return float(np.abs(g - o).max() / max(np.abs(o).max(), 1e-30))


@pytest.mark.parametrize("K", [4, 16])
def test_objective_and_gradient_match_oracle(K):
    b, ost = _case(50 + K, 6, K, 3000)
    beta = np.full(b.R, 0.02)
    ocfg = orc.config(K, prior_scale_mode=1)
    F, gd, gL, ga = orc.objective(ocfg, b.offsets, b.samples, ost, prior_scale=beta)
    gcfg = api.config(K, prior_scale_mode=api.PRIOR_SCALE_ARRAY)
    st = gpu_state(ost, gcfg)
    ws = api.workspace(gcfg, b.R, b.N)
    batch = dev_batch(b)
    tb = torch.from_numpy(beta).cuda()
    Fg = api.objective(gcfg, batch, st, ws, prior_scale=tb).cpu().numpy()
    assert np.abs(Fg - F).max() < 1e-5 * max(1.0, np.abs(F).max())
    dF = torch.linspace(0.5, 1.5, b.R, dtype=torch.float64).cuda()
    g = api.objective_backward(gcfg, batch, st, dF, ws, prior_scale=tb)
    sc = dF.cpu().numpy()
    assert _rel(g[0].cpu().numpy(), sc[:, None, None] * gd) < 1e-3
    assert _rel(g[1].cpu().numpy(), sc[:, None, None] * gL) < 1e-3
    assert _rel(g[2].cpu().numpy(), sc[:, None] * ga) < 1e-3


def test_adjoint_against_fp64_finite_differences():
    """A few gradient entries of the GPU adjoint against central differences
    (step 1e-6) of the FP64 objective."""
    K = 4
    b, ost = _case(60, 2, K, 2000)
    beta = np.full(b.R, 0.02)
    ocfg = orc.config(K, prior_scale_mode=1)
    gcfg = api.config(K, prior_scale_mode=api.PRIOR_SCALE_ARRAY)
    st = gpu_state(ost, gcfg)
    ws = api.workspace(gcfg, b.R, b.N)
    gd, gL, ga = (t.cpu().numpy() for t in api.objective_backward(
        gcfg, dev_batch(b), st, torch.ones(b.R, dtype=torch.float64).cuda(), ws,
        prior_scale=torch.from_numpy(beta).cuda()))
    h = 1e-6
    F = lambda s, dl=None: orc.objective(ocfg, b.offsets, b.samples, s, prior_scale=beta, delta=dl,
                                         grads=False)
    for (r, k, c) in [(0, 0, 0), (0, 1, 3), (1, 2, 4), (1, 3, 1)]:
        dp, dm = np.zeros((b.R, K, 5)), np.zeros((b.R, K, 5))
        dp[r, k, c], dm[r, k, c] = h, -h
        fd = (F(ost, dp)[r] - F(ost, dm)[r]) / (2 * h)
        assert abs(gd[r, k, c] - fd) < 1e-3 * max(1.0, np.abs(gd[r]).max())
    for (r, k, p) in [(0, 0, 0), (0, 2, 7), (1, 1, 14), (1, 3, 9)]:
        sp, sm = ost.copy(), ost.copy()
        sp.L[r, k, p] += h
        sm.L[r, k, p] -= h
        fd = (F(sp)[r] - F(sm)[r]) / (2 * h)
        assert abs(gL[r, k, p] - fd) < 1e-3 * max(1.0, np.abs(gL[r]).max())


def test_autograd_function_gradients():
    K = 8
    b, ost = _case(70, 3, K, 2500)
    beta = torch.full((b.R,), 0.01, dtype=torch.float64).cuda()
    gcfg = api.config(K, prior_scale_mode=api.PRIOR_SCALE_ARRAY)
    st = gpu_state(ost, gcfg)
    ws = api.workspace(gcfg, b.R, b.N)
    batch = dev_batch(b)
    rng = np.random.default_rng(0)
    delta_np = 0.01 * rng.normal(size=(b.R, K, 5))
    delta = torch.tensor(delta_np, dtype=torch.float64, device="cuda", requires_grad=True)
    L = torch.tensor(ost.L, dtype=torch.float64, device="cuda", requires_grad=True)
    logits = torch.tensor(np.log(ost.pi), dtype=torch.float64, device="cuda", requires_grad=True)
    F = api.map_objective(gcfg, batch, st, ws, delta, L, logits, prior_scale=beta)
    w = torch.arange(1, b.R + 1, dtype=torch.float64, device="cuda")
    (F * w).sum().backward()
    ocfg = orc.config(K, prior_scale_mode=1)
    Fo, gd, gL, ga = orc.objective(ocfg, b.offsets, b.samples, ost, prior_scale=beta.cpu().numpy(),
                                   delta=delta_np)
    assert np.abs(F.detach().cpu().numpy() - Fo).max() < 1e-5 * max(1.0, np.abs(Fo).max())
    wn = w.cpu().numpy()
    assert _rel(delta.grad.cpu().numpy(), wn[:, None, None] * gd) < 1e-3
    assert _rel(L.grad.cpu().numpy(), wn[:, None, None] * gL) < 1e-3
    assert _rel(logits.grad.cpu().numpy(), wn[:, None] * ga) < 1e-3


def test_objective_workload_1024_regions_sampled():
    """1,024 regions x 16,384 samples, K = 16: objective and adjoint for all
    regions on the GPU; four regions recomputed by the oracle."""
    K, R, M = 16, 1024, 16384
    truth = syn.batched_truth(80, R, K=K)
    b = syn.batched_round(80, R, np.full(R, M), 0, truth)
    gcfg = api.config(K)
    st = api.MixtureState(R, K)
    batch = dev_batch(b)
    api.init_regions(gcfg, batch, torch.from_numpy(b.extent.astype(np.float64)).cuda(),
                     torch.from_numpy(syn.init_uniforms(80, R, 2)).cuda(), st)
    ws = api.workspace(gcfg, R, b.N)
    api.fit_regions(gcfg, batch, 1, st, ws)
    Fg = api.objective(gcfg, batch, st, ws).cpu().numpy()
    g = [t.cpu().numpy() for t in api.objective_backward(gcfg, batch, st, torch.ones(R, dtype=torch.float64).cuda(), ws)]
    pick = np.array([0, 17, 500, 1023])
    sub_off = syn.offsets_from_counts(np.full(len(pick), M))
    sub = np.concatenate([b.samples[:, b.offsets[r]:b.offsets[r + 1]] for r in pick], axis=1)
    ost = orc.State(len(pick), K)
    for f in orc.State.FIELDS:
        getattr(ost, f)[...] = getattr(st, f).cpu().numpy()[pick]
    F, gd, gL, ga = orc.objective(orc.config(K), sub_off, sub, ost)
    assert np.abs(Fg[pick] - F).max() < 1e-5 * max(1.0, np.abs(F).max())
    assert _rel(g[0][pick], gd) < 1e-3
    assert _rel(g[1][pick], gL) < 1e-3
    assert _rel(g[2][pick], ga) < 1e-3
