"""sdmm_fit_regions_noalloc: the fit for callers that may not allocate device
memory (for example a plugin whose host application owns all device
allocations, or code inside an allocator callback).  It uses the library's
fixed scratch array instead of a caller workspace.

These tests call it through the C ABI and check it against the workspace
entry point, sdmm_fit_regions, bit for bit: on two calls in a row (the second
call runs on scratch that still holds the first call's contents), on a smaller
problem right after a larger one (a different scratch layout), with the
two-pass covariance update and with the 6xBF16 contraction form; and check
that a problem too large for the fixed scratch is rejected before any launch.
This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import dev_batch, gpu_state, host, oracle_init
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


def _bits(t):
    """The tensor's bytes as integers (NaN-carrying records compare bit for bit)."""
    return t.contiguous().view(torch.uint8)


def _assert_same(a, b):
    for f in api.MixtureState.FIELDS:
        assert torch.equal(_bits(getattr(a, f)), _bits(getattr(b, f))), f


def _problem(seed, counts, K=16):
    R = len(counts)
    truth = syn.batched_truth(seed, R, K=K, parallax=True)
    batches = [syn.batched_round(seed, R, np.asarray(counts), r, truth) for r in range(2)]
    return batches, oracle_init(seed, batches[0], K)


def _both(cfg, b, iters, ref, new, ws):
    """One call of each entry point on the same state; bit-identical results."""
    db = dev_batch(b)
    ll_ref = torch.zeros(b.N, dtype=torch.float32, device="cuda")
    ll_new = torch.zeros(b.N, dtype=torch.float32, device="cuda")
    api.fit_regions(cfg, db, iters, ref, ws, loglik=ll_ref)
    assert _noalloc(cfg, db, iters, new, loglik=ll_new) == 0, _lib.load().sdmm_last_error()
    torch.cuda.synchronize()
    _assert_same(new, ref)
    assert torch.equal(_bits(ll_new), _bits(ll_ref))


def test_noalloc_fit_matches_workspace_fit_on_two_calls():
    """Two calls in a row (the second runs on scratch that still holds the
    first's contents), then a smaller problem (fewer regions and work units,
    so a different scratch layout) right after the larger one: each result
    equals sdmm_fit_regions' bit for bit (same work units, same order of
    every sum)."""
    K = 16
    counts = [10, 16, 300, 2100, 5000, 9001, 40000]     # skipped, tiny, ragged, many units
    batches, ost = _problem(91, counts, K)
    cfg = api.config(K)
    ref, new = gpu_state(ost, cfg), gpu_state(ost, cfg)
    ws = api.workspace(cfg, len(counts), int(np.sum(counts)))
    for b in batches:
        _both(cfg, b, 2, ref, new, ws)
    assert list(host(new).status) == [1, 0, 0, 0, 0, 0, 0]
    small, ost2 = _problem(92, [700, 40, 3000], K)
    ref2, new2 = gpu_state(ost2, cfg), gpu_state(ost2, cfg)
    _both(cfg, small[0], 1, ref2, new2, api.workspace(cfg, 3, small[0].N))


@pytest.mark.parametrize("kw", [dict(cov_update=1, eta_mode=1), dict(precision=4)],
                         ids=["two_pass_update", "tensor_core_6xbf16"])
def test_noalloc_other_fit_variants(kw):
    """The accurate two-pass covariance update (second-pass scratch) and the
    6xBF16 contraction form (coefficient tables, unit ranges) through the
    fixed scratch: bit-identical to the workspace entry point."""
    K = 16
    counts = [500, 2500, 9000]
    batches, ost = _problem(93, counts, K)
    cfg = api.config(K, **kw)
    ref, new = gpu_state(ost, cfg), gpu_state(ost, cfg)
    ws = api.workspace(cfg, len(counts), int(np.sum(counts)))
    for b in batches:
        _both(cfg, b, 1, ref, new, ws)


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
