"""Derives the arctangent polynomial used by the kernels (atan_poly in
common.cuh).

atan(t) on t in [0, 1] is written t * P(t^2), P of degree 7 in u = t^2.  The
coefficients minimise the maximum relative error |t P(t^2) / atan(t) - 1| by
iteratively reweighted least squares (Lawson's algorithm) on Chebyshev nodes,
with the leading coefficient fixed to 1 so that small angles keep full
relative accuracy.  Octant reduction in the kernel maps any atan2(s, c) with
s >= 0 onto this interval.

    python paper_2111_13094_gb300/csrc/fit_atan_poly.py
"""
import numpy as np


def fit(deg=8, nodes=6000, iters=80):
    k = np.arange(nodes)
    u = (1 - np.cos(np.pi * (k + 0.5) / nodes)) / 2
    t = np.sqrt(u)
    f = np.ones_like(u)
    nz = t > 0
    f[nz] = np.arctan(t[nz]) / t[nz]                  # target P(u) = atan(t)/t
    # P(u) = 1 + sum_{j>=1} c_j u^j ; fit the remainder
    A = np.stack([u ** j for j in range(1, deg)], 1)
    y = f - 1.0
    w = np.ones(nodes) / nodes
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], y * sw, rcond=None)
        e = np.abs(A @ c - y) / f                      # relative error of atan
        w *= e / e.max() + 1e-4
        w /= w.sum()
    return np.concatenate([[1.0], c])


def max_rel_error_f32(c):
    t = np.linspace(1e-6, 1.0, 400001).astype(np.float32)
    u = t * t
    cf = np.asarray(c, np.float32)
    p = np.zeros_like(t)
    for cj in cf[::-1]:
        p = (p * u + cj).astype(np.float32)
    a = (t * p).astype(np.float64)
    ref = np.arctan(t.astype(np.float64))
    return float(np.max(np.abs(a / ref - 1.0))), float(np.max(np.abs(a - ref)))


if __name__ == "__main__":
    c = fit()
    rel, ab = max_rel_error_f32(c)
    print("coefficients (float32):", ", ".join("%.9gf" % float(np.float32(x)) for x in c))
    print(f"max relative error {rel:.3e}, max absolute error {ab:.3e} (FP32 Horner)")
