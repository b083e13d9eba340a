"""sdmm_fit_regions_noalloc: the fit for callers that may not allocate device
memory (for example a plugin whose host application owns all device
allocations, or code inside an allocator callback).  It uses the library's
fixed scratch array instead of a caller workspace.

These tests call it through the C ABI and check it against the workspace
entry point, sdmm_fit_regions, on two calls in a row (the second call runs on
scratch that still holds the first call's contents), and check that a problem
too large for the fixed scratch is rejected before any launch.  This file is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import LOGLIK_RTOL, PARAM_RTOL, assert_params_close, dev_batch, gpu_state, host, oracle_init
from paper_2111_13094_gb300 import _lib, api
from paper_2111_13094_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _noalloc(cfg, batch, iters, state, loglik=None, prior_scale=None):
    lib = _lib.load()
    sm = batch.c()
    st = state.c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.sdmm_fit_regions_noalloc(ctypes.byref(cfg), ctypes.byref(sm), int(iters),
                                        None if prior_scale is None else ctypes.c_void_p(prior_scale.data_ptr()),
                                        ctypes.byref(st),
                                        None if loglik is None else ctypes.c_void_p(loglik.data_ptr()),
                                        stream)


def test_noalloc_fit_matches_workspace_fit_on_two_calls():
    K, R = 16, 7
    counts = np.array([10, 16, 300, 2100, 5000, 9001, 40000])     # skipped, tiny, ragged, many units
    truth = syn.batched_truth(91, R, K=K, parallax=True)
    batches = [syn.batched_round(91, R, counts, r, truth) for r in range(2)]
    ost = oracle_init(91, batches[0], K)
    cfg = api.config(K)
    ref = gpu_state(ost, cfg)
    new = gpu_state(ost, cfg)
    ws = api.workspace(cfg, R, int(counts.sum()))
    for call, b in enumerate(batches):               # two calls in a row
        db = dev_batch(b)
        ll_ref = torch.zeros(b.N, dtype=torch.float32, device="cuda")
        ll_new = torch.zeros(b.N, dtype=torch.float32, device="cuda")
        api.fit_regions(cfg, db, 2, ref, ws, loglik=ll_ref)
        assert _noalloc(cfg, db, 2, new, loglik=ll_new) == 0, _lib.load().sdmm_last_error()
        torch.cuda.synchronize()
        g_ref, g_new = host(ref), host(new)
        assert list(g_new.status) == list(g_ref.status) == [1, 0, 0, 0, 0, 0, 0]
        assert_params_close(g_new, g_ref, rtol=PARAM_RTOL)
        for f in ("S0", "S2", "Wbar"):
            a, e = getattr(g_new, f), getattr(g_ref, f)
            assert np.abs(a - e).max() <= 1e-6 * max(1.0, np.abs(e).max()), (call, f)
        assert np.array_equal(g_new.n_seen, g_ref.n_seen) and np.array_equal(g_new.step_j, g_ref.step_j)
        o = b.offsets[1]
        a, e = ll_new[o:].cpu().numpy().astype(np.float64), ll_ref[o:].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(a - e) / np.maximum(1.0, np.abs(e))) < LOGLIK_RTOL


def test_noalloc_rejects_problems_larger_than_its_scratch():
    K, R = 16, 20000                                  # 20,000 one-sample regions
    counts = np.ones(R, dtype=np.int64)
    cfg = api.config(K)
    need = api.workspace_bytes(cfg, R, R)
    assert need > _lib.SDMM_NOALLOC_SCRATCH_BYTES
    samples = torch.zeros(7, R, dtype=torch.float32, device="cuda")
    samples[5] = 1.0
    batch = api.SampleBatch(samples, torch.from_numpy(syn.offsets_from_counts(counts)).cuda())
    st = api.MixtureState(R, K)
    before = st.status.clone()
    assert _noalloc(cfg, batch, 1, st) == 5            # SDMM_ERR_WORKSPACE, nothing launched
    msg = _lib.load().sdmm_last_error().decode()
    assert str(need) in msg and str(_lib.SDMM_NOALLOC_SCRATCH_BYTES) in msg
    torch.cuda.synchronize()
    assert torch.equal(st.status, before)
