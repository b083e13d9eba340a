"""Euclidean ablation of the directional coordinates (nu = (w_x - mu_x,
w_y - mu_y), no change of variables, the mean translated in x and y) on the
GPU, SIMT and contraction forms, against the oracle's Euclidean mode on the
same inputs; the paths that need tangent charts reject it."""
import numpy as np
import pytest
import torch

import oracle as orc
from gpu_util import LOGLIK_RTOL, assert_params_close, dev_batch, gpu_state, host, loglik_err, oracle_init
from paper_2111_13094_gb300 import api
from paper_2111_13094_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _run(K, prec, seed, counts, iters, chunk=0):
    truth = syn.batched_truth(seed, len(counts), K=K, parallax=True)
    b = syn.batched_round(seed, len(counts), np.asarray(counts), 0, truth)
    ost = oracle_init(seed, b, K)
    gcfg = api.config(K, precision=prec, dir_coords=api.DIR_EUCLIDEAN, chunk=chunk)
    st = gpu_state(ost, gcfg)
    oll = orc.fit_regions(orc.config(K, euclid=1), b.offsets, b.samples, iters, ost, want_loglik=True)
    ll = torch.zeros(b.N, dtype=torch.float32, device="cuda")
    api.fit_regions(gcfg, dev_batch(b), iters, st, api.workspace(gcfg, b.R, b.N), loglik=ll)
    return b, host(st), ost, ll.cpu().numpy(), oll


@pytest.mark.parametrize("K,iters", [(1, 1), (3, 1), (16, 1), (32, 1), (3, 2), (16, 2)])
def test_simt_matches_oracle(K, iters):
    counts = [10, 17, 257, 3001, 6000]                  # skipped, tiny, ragged, several units
    b, g, ost, ll, oll = _run(K, api.PREC_FP32, 300 + K, counts, iters, chunk=256)
    assert list(g.status) == list(ost.status)
    mask = np.zeros(b.N, bool)
    mask[b.offsets[1]:] = True
    assert loglik_err(ll, oll, mask) < LOGLIK_RTOL
    assert_params_close(g, ost)
    ok = ost.status == 0
    # the ablation moves the mean off the sphere (translation in x and y only)
    assert np.abs(np.linalg.norm(ost.mu_w.reshape(-1, 3), axis=1) - 1.0)[np.repeat(ok, K)].max() > 1e-6
    # ... and leaves its z coordinate where the initialisation put it
    assert np.array_equal(g.mu_w.reshape(-1, 3)[:, 2], ost.mu_w.reshape(-1, 3)[:, 2])


@pytest.mark.parametrize("K", [16, 32])
@pytest.mark.parametrize("prec", [api.PREC_TC_6XBF16, api.PREC_TC_3XTF32])
def test_contraction_form_matches_oracle(K, prec):
    b, g, ost, ll, oll = _run(K, prec, 320 + K, [16, 200, 3001, 9000], 1)
    assert list(g.status) == list(ost.status)
    assert loglik_err(ll, oll) < LOGLIK_RTOL
    assert_params_close(g, ost)


def test_tangent_only_paths_reject_the_ablation():
    K = 16
    cfg = api.config(K, dir_coords=api.DIR_EUCLIDEAN)
    st = api.MixtureState(1, K)
    qx = torch.full((8, 3), 0.5, device="cuda")
    with pytest.raises(api.SdmmError):
        api.sample(cfg, st, qx, region=torch.zeros(8, dtype=torch.int32, device="cuda"))
    with pytest.raises(api.SdmmError):
        api.workspace(api.config(K, dir_coords=api.DIR_EUCLIDEAN, cov_update=api.COV_TWO_PASS,
                                 eta_mode=api.ETA_ONE), 1, 1024)
    with pytest.raises(api.SdmmError):
        api.workspace(api.config(K, dir_coords=2), 1, 1024)
