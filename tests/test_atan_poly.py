"""The arctangent used by the kernels (atan2_pos in csrc/common.cuh): its
coefficients, evaluated in FP32 exactly as the kernel does, against numpy's
arctan2 over all angles in [0, pi]."""
import os
import re

import numpy as np

from conftest import ROOT


def _coefficients():
    src = open(os.path.join(ROOT, "paper_2111_13094_gb300", "csrc", "common.cuh")).read()
    body = src[src.index("float atan2_pos"):]
    body = body[:body.index("return p;")]
    first = re.search(r"float p = (-?[0-9.e-]+)f;", body).group(1)
    rest = re.findall(r"p = fmaf\(p, u, (-?[0-9.e-]+)f\)", body)
    return [np.float32(first)] + [np.float32(x) for x in rest]


def _atan2_pos_f32(s, c, coef):
    s = s.astype(np.float32)
    c = c.astype(np.float32)
    ac = np.abs(c)
    mn, mx = np.minimum(s, ac), np.maximum(s, ac)
    t = np.where(mx > 0, mn / np.where(mx > 0, mx, 1), 0).astype(np.float32)
    u = (t * t).astype(np.float32)
    p = np.full_like(t, coef[0])
    for cj in coef[1:]:
        p = (p * u + cj).astype(np.float32)
    p = (p * t).astype(np.float32)
    p = np.where(s > ac, np.float32(1.57079637) - p, p).astype(np.float32)
    p = np.where(c < 0, np.float32(3.14159274) - p, p).astype(np.float32)
    return p


def test_atan2_pos_accuracy():
    coef = _coefficients()
    assert len(coef) == 8 and coef[-1] == np.float32(1.0)
    th = np.linspace(0.0, np.pi, 2_000_001)
    s, c = np.sin(th), np.cos(th)
    s32, c32 = s.astype(np.float32), c.astype(np.float32)
    got = _atan2_pos_f32(s32, c32, coef).astype(np.float64)
    ref = np.arctan2(s32.astype(np.float64), c32.astype(np.float64))
    # about 2.5 FP32 ulp of the result everywhere (polynomial 2.1e-7 plus division and fix-up rounding)
    pos = ref > 0
    assert np.max(np.abs(got[pos] - ref[pos]) / ref[pos]) < 3e-7
    assert got[~pos].max() == 0.0
