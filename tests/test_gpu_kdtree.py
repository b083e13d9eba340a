"""The GPU kD-tree (Sec. 4.2 refinement and binning, Sec. 4.3 pre-
subdivision) against the oracle: lookups, sample order, offsets and parents
must agree exactly (index work)."""
import numpy as np
import pytest
import torch

from oracle import kdtree as kd
from gpu_util import dev_batch, host, oracle_init
from paper_2111_13094_gb300 import api
from paper_2111_13094_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _scene(seed, N, clusters=12):
    """Positions clustered like path vertices on surfaces (many points in a
    few places), directions and weights of the usual recipe."""
    rng = np.random.default_rng([seed, 77])
    c = rng.random((clusters, 3))
    sd = rng.uniform(0.005, 0.08, size=clusters)
    k = rng.integers(0, clusters, size=N)
    s = np.zeros((7, N), np.float32)
    s[:3] = np.clip(c[k].T + sd[k] * rng.normal(size=(3, N)), 0.0, 1.0).astype(np.float32)
    w = rng.normal(size=(3, N))
    w /= np.linalg.norm(w, axis=0)
    s[3:6] = w.astype(np.float32)
    s[6] = rng.lognormal(0.0, 1.5, size=N).astype(np.float32)
    return s


@pytest.mark.parametrize("levels", [0, 1, 3])
def test_grid_lookup_matches_oracle(levels):
    t = api.KdTree(4096, 4096).grid(levels)
    ot = kd.grid(levels)
    assert t.n_leaves == ot.n_leaves
    pts = np.random.default_rng(levels).random((3, 20000)).astype(np.float32)
    pts[:, :3] = [[0.5, 0.25, 0.0], [0.5, 0.75, 1.0], [0.125, 0.5, 0.999]]   # on planes and faces
    got = t.lookup(torch.from_numpy(pts).cuda()).cpu().numpy()
    assert np.array_equal(got, kd.lookup(ot, pts))


@pytest.mark.parametrize("N,levels", [(60000, 3), (8193, 3), (100, 1), (60000, 4), (9000, 4)])
def test_binning_matches_oracle(N, levels):
    """Up to 1024 leaves (levels <= 3: 8^levels) the binning is one counting
    pass that moves the streams; beyond (levels = 4: 4096 leaves) two 8-bit
    passes on (leaf, index) and a gather.  Both keep each leaf's samples in
    their input order; N spans whole and ragged tiles."""
    s = _scene(1, N)
    t = api.KdTree(1 << 14, 1 << 13).grid(levels)
    b = t.bin(torch.from_numpy(s).cuda())
    out, off, _ = kd.bin_samples(kd.grid(levels), s)
    assert np.array_equal(b.offsets.cpu().numpy(), off)
    assert np.array_equal(b.samples.cpu().numpy(), out)


@pytest.mark.parametrize("N,c,levels", [(60000, 1000, 1), (300000, 16000, 3), (5000, 100, 0)])
def test_refinement_matches_oracle(N, c, levels):
    s = _scene(2 + levels, N)
    t = api.KdTree(1 << 17, 1 << 16).grid(levels)
    b = t.bin(torch.from_numpy(s).cuda())
    ot = kd.grid(levels)
    ob, ooff, _ = kd.bin_samples(ot, s)
    nt, out, noff, parent = kd.refine(ot, ob, ooff, c)
    rb, rparent = t.refine(b, c=c)
    assert t.n_leaves == nt.n_leaves > kd.grid(levels).n_leaves
    assert np.array_equal(rb.offsets.cpu().numpy(), noff)
    assert np.array_equal(rb.samples.cpu().numpy(), out)
    assert np.array_equal(rparent.cpu().numpy(), parent)
    pts = np.concatenate([np.random.default_rng(9).random((3, 20000)).astype(np.float32), s[:3, :20000]], axis=1)
    assert np.array_equal(t.lookup(torch.from_numpy(pts).cuda()).cpu().numpy(), kd.lookup(nt, pts))
    # refining again with the same c splits nothing
    rb2, p2 = t.refine(rb, c=c)
    assert np.array_equal(rb2.offsets.cpu().numpy(), noff) and np.array_equal(p2.cpu().numpy(), np.arange(len(noff) - 1))


def test_refine_reports_small_capacities():
    s = _scene(5, 50000)
    t = api.KdTree(64, 32).grid(1)
    b = t.bin(torch.from_numpy(s).cuda())
    with pytest.raises(api.SdmmError):
        t.refine(b, c=100)


def test_gather_then_fit_on_refined_leaves():
    """Bin, refine, copy the parents' mixtures into the new leaves, fit."""
    K = 16
    s = _scene(6, 200000)
    t = api.KdTree(1 << 16, 1 << 15).grid(1)
    b = t.bin(torch.from_numpy(s).cuda())
    cfg = api.config(K)
    st = api.MixtureState(t.n_leaves, K)
    api.init_regions(cfg, b, torch.full((t.n_leaves,), 0.5, dtype=torch.float64).cuda(),
                     torch.from_numpy(syn.init_uniforms(6, t.n_leaves, 2)).cuda(), st)
    rb, parent = t.refine(b, c=16000)
    st2 = api.gather_regions(st, parent)
    g, g2 = host(st), host(st2)
    p = parent.cpu().numpy()
    for f in ("pi", "mu_x", "mu_w", "L", "n_seen", "status"):
        assert np.array_equal(getattr(g2, f), getattr(g, f)[p]), f
    assert torch.equal(st2.etab, st.etab[parent])
    ws = api.workspace(cfg, rb.R, rb.N)
    api.fit_regions(cfg, rb, 1, st2, ws)
    stat = st2.status.cpu().numpy()
    counts = np.diff(rb.offsets.cpu().numpy())
    assert np.all(stat[counts >= 16] != 2)                       # fitted regions are updated
