"""Pins of the oracle's mixture initialisation (Sec. 4.3 "Initialization",
App. B, App. C) against scipy's chi-square quantile and numpy's weighted
inverse-CDF pick."""
import math

import numpy as np
from scipy import stats

from conftest import read_constants
from paper_2111_13094_gb300 import synthetic as syn


def _pick(p, u):
    c = np.cumsum(p)
    return int(np.searchsorted(c, u * c[-1], side="right"))


def test_init_structure_and_seeds(orc):
    const = read_constants()
    b = syn.batched_round(1, 8, syn.region_counts(1, 8, 20, 3000), 0, syn.batched_truth(1, 8, K=16))
    K = 16
    u = syn.init_uniforms(1, b.R, 2)
    st = orc.State(b.R, K)
    st.S0[:] = 7.0
    st.n_seen[:] = 5
    orc.init_regions(orc.config(K), b.offsets, b.samples, b.extent, u, st)
    q = stats.chi2.ppf(const["init_mass_quantile"], 3)
    corners = np.array([[sx, sy, sz] for sz in (1, -1) for sy in (1, -1) for sx in (1, -1)]) / math.sqrt(3)
    for r in range(b.R):
        o, M = b.offsets[r], b.offsets[r + 1] - b.offsets[r]
        assert st.status[r] == 0 and st.n_seen[r] == 0 and np.all(st.S0[r] == 0)
        x = b.samples[0:3, o:o + M].T.astype(np.float64)
        w = np.clip(b.samples[6, o:o + M].astype(np.float64),
                    const["init_weight_clamp_lo"], const["init_weight_clamp_hi"])
        i1 = _pick(w, u[r, 0])
        i2 = _pick(w * np.linalg.norm(x - x[i1], axis=1), u[r, 1])
        assert np.allclose(st.mu_x[r, :8], x[i1]) and np.allclose(st.mu_x[r, 8:], x[i2])
        assert np.allclose(st.pi[r], 1 / K)
        for j in range(2):
            assert np.allclose(st.mu_w[r, 8 * j:8 * j + 8], corners, atol=1e-15)
        L = st.L[r]
        diag = L[:, [0, 2, 5, 9, 14]]
        rst = 2 * b.extent[r] / 2
        assert np.allclose(diag[:, :3], rst / math.sqrt(q), rtol=1e-12)
        assert np.allclose(diag[:, 3:] ** 2, const["init_dir_var_times_8"] / 8, rtol=1e-12)
        off = np.delete(L, [0, 2, 5, 9, 14], axis=1)
        assert np.all(off == 0)


def test_init_skips_small_regions(orc):
    counts = [15, 16]
    b = syn.batched_round(2, 2, counts, 0, syn.batched_truth(2, 2, K=8))
    st = orc.State(2, 8)
    orc.init_regions(orc.config(8), b.offsets, b.samples, b.extent, syn.init_uniforms(2, 2, 1), st)
    assert list(st.status) == [1, 0]
