"""The tensor-core helpers (shared-memory layout, descriptors, tcgen05.mma,
commit, TMEM read-out) against an FP64 product of the same rounded
operands, for BF16 (kind::f16) and TF32 (kind::tf32) tiles."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2111_13094_gb300 import _lib

pytestmark = pytest.mark.gpu


def _round_tf32(x):
    """Round FP32 to TF32 (10 explicit mantissa bits), nearest, ties away."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x1000) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32)


def _run(kind, N, Kd, variant, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(128, Kd)).astype(np.float32)
    B = rng.normal(size=(N, Kd)).astype(np.float32)
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    D = torch.full((128, N), float("nan"), device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    lib = _lib.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.sdmm_tc_selftest(kind, N, Kd, ctypes.c_void_p(tA.data_ptr()), ctypes.c_void_p(tB.data_ptr()),
                                ctypes.c_void_p(D.data_ptr()), variant, ctypes.c_void_p(st.data_ptr()), s)
    assert code == 0, lib.sdmm_last_error()
    torch.cuda.synchronize()
    assert int(st.item()) == 0, "MMA did not complete"
    if kind == 0:
        Ar = tA.bfloat16().double().cpu().numpy()
        Br = tB.bfloat16().double().cpu().numpy()
    else:
        Ar, Br = _round_tf32(A).astype(np.float64), _round_tf32(B).astype(np.float64)
    ref = Ar @ Br.T
    return D.cpu().numpy().astype(np.float64), ref


@pytest.mark.parametrize("kind,Kd", [(0, 16), (0, 32), (0, 64), (1, 8), (1, 32)])
@pytest.mark.parametrize("N", [16, 96, 256])
def test_tc_tile_matches_fp64_product(kind, N, Kd):
    D, ref = _run(kind, N, Kd, variant=0)
    err = np.abs(D - ref).max()
    assert err < 1e-4 * max(1.0, np.abs(ref).max()), err


@pytest.mark.parametrize("variant", [2, 4, 6])          # A and/or B staged MN-major (BF16)
@pytest.mark.parametrize("N,Kd", [(32, 64), (96, 32), (128, 64)])
def test_tc_mn_major_tiles(variant, N, Kd):
    D, ref = _run(0, N, Kd, variant=variant)
    assert np.abs(D - ref).max() < 1e-4 * max(1.0, np.abs(ref).max())


def test_tc_swapped_offsets_are_detected():
    """The diagnostic variants that swap the two descriptor offsets must give a
    wrong product: the tests above would catch a wrong layout reading."""
    for variant in (1, 10):
        D, ref = _run(0, 96, 32, variant=variant)
        assert np.abs(D - ref).max() > 1.0


def _wait(limit_ns, arrive):
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    el = torch.zeros(1, dtype=torch.int64, device="cuda")
    lib = _lib.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.sdmm_wait_selftest(limit_ns, arrive, ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(el.data_ptr()), s)
    assert code == 0, lib.sdmm_last_error()
    torch.cuda.synchronize()
    return int(st.item()), int(el.item())


def test_bounded_wait_gives_up_and_the_context_survives():
    """The E-step's bounded mbarrier wait on a barrier nothing completes: it
    gives up after its limit, reports it, and the GPU stays usable; with an
    arrival it completes at once."""
    status, elapsed = _wait(2_000_000, 0)            # 2 ms limit, nobody arrives
    assert status == 1 and 2_000_000 <= elapsed < 1_000_000_000
    status, elapsed = _wait(2_000_000, 1)
    assert status == 0 and elapsed < 2_000_000
    x = torch.arange(1024, device="cuda", dtype=torch.float32)   # the context still runs work
    assert float(x.sum().item()) == 1024 * 1023 / 2
    lib = _lib.load()
    assert lib.sdmm_wait_selftest(0, 0, None, None, None) == 1   # argument errors come from the host
