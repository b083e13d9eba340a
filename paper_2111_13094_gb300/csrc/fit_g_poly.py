"""Derives the polynomial for the log map's scale g = theta / sin(theta) used
by the SIMT E-step (g_of_cos in common.cuh).

For a unit direction with c = cos(theta) in [0, 1], g is written
P(t) = 1 + sum_{j>=1} c_j t^j in t = 1 - c (P(0) = 1: g = 1 at the chart
centre).  acos(c) / sqrt(1 - c^2) is analytic on (-1, 1], so a modest degree
reaches FP32 accuracy on t in [0, 1]; the coefficients minimise the maximum
relative error by iteratively reweighted least squares (Lawson's algorithm)
on Chebyshev nodes.  For c < 0 the kernel uses
acos(c) = pi - acos(-c), i.e. g = pi / sin(theta) - P(1 - |c|).

    python paper_2111_13094_gb300/csrc/fit_g_poly.py [degree]
"""
import sys

import numpy as np


def target(t):
    c = 1.0 - t
    s = np.sqrt(np.maximum(1.0 - c * c, 0.0))
    out = np.ones_like(t)
    nz = s > 0
    out[nz] = np.arccos(c[nz]) / s[nz]
    return out


def fit(deg=11, nodes=6000, iters=100):
    k = np.arange(nodes)
    t = (1 - np.cos(np.pi * (k + 0.5) / nodes)) / 2          # Chebyshev nodes on [0, 1]
    f = target(t)
    A = np.stack([t ** j for j in range(1, deg + 1)], 1)
    y = f - 1.0
    w = np.ones(nodes) / nodes
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], y * sw, rcond=None)
        e = np.abs(A @ c - y) / f
        w *= e / e.max() + 1e-4
        w /= w.sum()
    return np.concatenate([[1.0], c])                        # ascending powers of t


def horner_f32(coef, t):
    cf = np.asarray(coef, np.float32)
    p = np.full_like(t, cf[-1])
    for cj in cf[-2::-1]:
        p = (p * t + cj).astype(np.float32)
    return p


def max_rel_error_f32(coef):
    t = np.linspace(0.0, 1.0, 400001).astype(np.float32)
    p = horner_f32(coef, t).astype(np.float64)
    ref = target(t.astype(np.float64))
    return float(np.max(np.abs(p / ref - 1.0)))


if __name__ == "__main__":
    deg = int(sys.argv[1]) if len(sys.argv) > 1 else 11
    c = fit(deg)
    print("coefficients, highest power first (float32):",
          ", ".join("%.9gf" % float(np.float32(x)) for x in c[::-1]))
    print(f"degree {deg}: max relative error {max_rel_error_f32(c):.3e} (FP32 Horner)")
