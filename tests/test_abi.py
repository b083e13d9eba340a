"""The C-ABI library builds for sm_103a, loads, exports every symbol that
include/sdmm.h declares, and rejects bad arguments on the host (no GPU)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    with open(os.path.join(ROOT, "include", "sdmm.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sdmm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2111_13094_gb300 import _lib
    return _lib.load()


def test_header_and_binding_agree(lib):
    from paper_2111_13094_gb300 import _lib
    assert _declared() == sorted(_lib.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm_103a():
    from paper_2111_13094_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.LIB)


def test_config_defaults_are_paper_constants(lib):
    from conftest import read_constants
    from paper_2111_13094_gb300 import api
    c = read_constants()
    cfg = api.config(16)
    assert cfg.K == 16 and cfg.min_samples == c["min_samples"]
    assert cfg.prior_q == c["prior_q_times_K"] and cfg.prior_a == c["prior_a_times_K"]
    assert cfg.prior_B_pos == c["prior_B_pos_over_a"] and cfg.prior_B_dir == c["prior_B_dir_over_a"]
    assert cfg.eta_alpha == c["eta_alpha"] and cfg.eta_beta == c["eta_beta"]


def test_host_validation_errors(lib):
    from paper_2111_13094_gb300 import _lib, api
    n = ctypes.c_size_t()
    assert lib.sdmm_fit_workspace_size(ctypes.byref(api.config(0)), 1, 10, ctypes.byref(n)) == 1
    assert b"K = 0" in lib.sdmm_last_error()
    assert lib.sdmm_fit_workspace_size(ctypes.byref(api.config(33)), 1, 10, ctypes.byref(n)) == 4
    assert lib.sdmm_fit_workspace_size(ctypes.byref(api.config(16, chunk=300)), 1, 10, ctypes.byref(n)) == 1
    assert lib.sdmm_fit_workspace_size(ctypes.byref(api.config(16)), 0, 10, ctypes.byref(n)) == 1
    assert lib.sdmm_fit_workspace_size(ctypes.byref(api.config(16, chunk=256)), 4, 1000, ctypes.byref(n)) == 0
    assert n.value % 256 == 0 and n.value >= (1000 // 256 + 1 + 4) * (16 * 21 + 2) * 4
    # null state / samples are rejected before any CUDA call
    cfg = api.config(4)
    assert lib.sdmm_fit_regions(ctypes.byref(cfg), None, 1, None, None, None, None, 0, None) == 1
    sm = _lib.Samples()
    sm.R, sm.N = 1, 0
    assert lib.sdmm_fit_regions(ctypes.byref(cfg), ctypes.byref(sm), 1, None, None, None, None, 0, None) == 1
    assert lib.sdmm_prepare(ctypes.byref(cfg), 1, None, None, None, None) == 1
    g = _lib.Grid()
    assert lib.sdmm_condition(ctypes.byref(cfg), None, 1, 1, None, None, ctypes.byref(g), None, None, None, None) == 1
    assert lib.sdmm_fit_plan_destroy(None) == 0
    # the accurate (two-pass) covariance update: plain EM on the FP32 SIMT path only
    assert lib.sdmm_fit_workspace_size(ctypes.byref(api.config(16, cov_update=2)), 1, 10, ctypes.byref(n)) == 1
    assert lib.sdmm_fit_workspace_size(ctypes.byref(api.config(16, cov_update=1)), 1, 10, ctypes.byref(n)) == 4
    assert b"eta_mode" in lib.sdmm_last_error()
    assert lib.sdmm_fit_workspace_size(ctypes.byref(api.config(16, cov_update=1, eta_mode=1, precision=4)),
                                       1, 10, ctypes.byref(n)) == 4
    assert lib.sdmm_fit_workspace_size(ctypes.byref(api.config(16, cov_update=1, eta_mode=1)), 1, 10,
                                       ctypes.byref(n)) == 0
    # the Euclidean ablation: fit only, FP32 SIMT, 6xBF16 or 3xTF32, first-order update
    for prec, want in ((0, 0), (4, 0), (3, 0), (1, 4), (2, 4)):
        assert lib.sdmm_fit_workspace_size(ctypes.byref(api.config(16, dir_coords=1, precision=prec)), 1, 10,
                                           ctypes.byref(n)) == want, prec
    assert lib.sdmm_fit_workspace_size(ctypes.byref(api.config(16, dir_coords=1, cov_update=1, eta_mode=1)), 1, 10,
                                       ctypes.byref(n)) == 4
    assert lib.sdmm_fit_workspace_size(ctypes.byref(api.config(16, dir_coords=2)), 1, 10, ctypes.byref(n)) == 1
    assert lib.sdmm_condition(ctypes.byref(api.config(16, dir_coords=1)), None, 1, 1, None, None, ctypes.byref(g),
                              None, None, None, None) in (1, 4)


def test_noalloc_scratch_constant_matches_the_header():
    from paper_2111_13094_gb300 import _lib
    with open(os.path.join(ROOT, "include", "sdmm.h")) as f:
        src = f.read()
    m = re.search(r"#define\s+SDMM_NOALLOC_SCRATCH_BYTES\s+\(([^)]*)\)", src)
    assert m is not None
    value = eval(m.group(1).replace("u", ""), {})          # e.g. 16u * 1024u * 1024u
    assert value == _lib.SDMM_NOALLOC_SCRATCH_BYTES


def test_binned_query_workspace_checks(lib):
    from paper_2111_13094_gb300 import _lib, api
    n = ctypes.c_size_t()
    assert lib.sdmm_query_workspace_size(65536, 1 << 24, ctypes.byref(n)) == 0
    assert n.value >= 4 * (65536 + 1) + 12 * (1 << 24) and n.value % 256 == 0
    assert lib.sdmm_query_workspace_size(0, 10, ctypes.byref(n)) == 1
    assert lib.sdmm_query_workspace_size(4, -1, ctypes.byref(n)) == 1
    assert lib.sdmm_sample_binned(ctypes.byref(api.config(16)), None, 1, 1, None, None, None, 0, None, None, None,
                                  None, None, 0, None) == 1
