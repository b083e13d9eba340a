"""The log map's scale g = theta / sin(theta) used by the SIMT E-step
(g_of_cos in csrc/common.cuh): its coefficients, evaluated in FP32 exactly as
the kernel does, against numpy over all angles in [0, pi)."""
import os
import re

import numpy as np

from conftest import ROOT


def _coefficients(name="g_of_cos"):
    src = open(os.path.join(ROOT, "paper_2111_13094_gb300", "csrc", "common.cuh")).read()
    body = src[src.index(f"float {name}("):]
    body = body[:body.index("return")]
    first = re.search(r"float p = (-?[0-9.e-]+)f;", body).group(1)
    rest = re.findall(r"p = fmaf\(p, t, (-?[0-9.e-]+)f\)", body)
    return [np.float32(first)] + [np.float32(x) for x in rest]


def _g_of_cos_f32(c, rs, coef):
    c = c.astype(np.float32)
    t = (np.float32(1) - np.abs(c)).astype(np.float32)
    p = np.full_like(t, coef[0])
    for cj in coef[1:]:
        p = (p * t + cj).astype(np.float32)
    neg = (np.float32(3.14159274) * rs.astype(np.float32) - p).astype(np.float32)
    return np.where(c < 0, neg, p)


def test_g_of_cos_accuracy():
    coef = _coefficients()
    assert len(coef) == 10 and coef[-1] == np.float32(1.0)
    th = np.linspace(0.0, np.pi, 2_000_001)[:-1]
    c32 = np.cos(th).astype(np.float32)
    s32 = np.sin(th).astype(np.float32)
    # the kernel's inputs: c and 1/sin from the FP32 direction (rsqrt of u^2 + v^2)
    rs = np.where(s32 > 0, 1.0 / np.maximum(s32.astype(np.float64), 1e-300), np.inf)
    got = _g_of_cos_f32(c32, rs, coef).astype(np.float64)
    cd, sd = c32.astype(np.float64), s32.astype(np.float64)
    ang = np.arctan2(sd, cd)
    ref = np.where(sd > 0, ang / np.where(sd > 0, sd, 1.0), 1.0)
    rel = np.abs(got - ref) / ref
    # P alone is within 9.5e-8; the pi / sin branch adds the rounding of pi and of the
    # subtraction (largest just past pi / 2, where pi rs - P halves): about 3 FP32 ulp
    assert rel[cd >= 0].max() < 1.5e-7
    assert rel[cd < 0].max() < 4e-7
    # the chart centre is exact
    assert _g_of_cos_f32(np.array([1.0]), np.array([np.inf]), coef)[0] == np.float32(1.0)


def test_g_of_cos_fit_accuracy():
    """The degree-7 form of the fit's E-step: within 6e-7 for c >= 0 and
    within 1e-6 past pi / 2 (the pi / sin branch)."""
    coef = _coefficients("g_of_cos_fit")
    assert len(coef) == 8 and coef[-1] == np.float32(1.0)
    th = np.linspace(0.0, np.pi, 2_000_001)[:-1]
    c32 = np.cos(th).astype(np.float32)
    s32 = np.sin(th).astype(np.float32)
    rs = np.where(s32 > 0, 1.0 / np.maximum(s32.astype(np.float64), 1e-300), np.inf)
    got = _g_of_cos_f32(c32, rs, coef).astype(np.float64)
    cd, sd = c32.astype(np.float64), s32.astype(np.float64)
    ang = np.arctan2(sd, cd)
    ref = np.where(sd > 0, ang / np.where(sd > 0, sd, 1.0), 1.0)
    rel = np.abs(got - ref) / ref
    assert rel[cd >= 0].max() < 6e-7
    assert rel[cd < 0].max() < 1e-6
    assert _g_of_cos_f32(np.array([1.0]), np.array([np.inf]), coef)[0] == np.float32(1.0)
