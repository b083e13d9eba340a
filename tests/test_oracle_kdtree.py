"""The oracle's kD-tree (Sec. 4.2 "Refinement of the spatial kD-tree",
Sec. 4.3 pre-subdivision) against brute force and the paper's rule."""
import numpy as np
import pytest

from oracle import kdtree as kd


def _morton(i, j, k, levels):
    r = 0
    for b in range(levels - 1, -1, -1):
        r = (r << 3) | (((i >> b) & 1) << 2) | (((j >> b) & 1) << 1) | ((k >> b) & 1)
    return r


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_grid_cells_are_morton_numbered(levels):
    t = kd.grid(levels)
    n = 1 << levels
    assert t.n_leaves == n ** 3
    ijk = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), 0).reshape(3, -1)
    centres = ((ijk + 0.5) / n).astype(np.float32)
    got = kd.lookup(t, centres)
    want = np.array([_morton(i, j, k, levels) for i, j, k in ijk.T])
    assert np.array_equal(got, want)


def _samples(rng, N, spread=(1.0, 1.0, 1.0)):
    s = np.zeros((7, N), np.float32)
    s[:3] = (rng.random((3, N)) * np.asarray(spread)[:, None]).astype(np.float32)
    s[5] = 1.0
    s[6] = rng.random(N).astype(np.float32)
    return s


def test_binning_is_a_stable_sort_by_cell():
    rng = np.random.default_rng(1)
    t = kd.grid(2)
    s = _samples(rng, 5000)
    out, off, order = kd.bin_samples(t, s)
    leaf = kd.lookup(t, s[:3])
    for r in range(t.n_leaves):
        idx = np.where(leaf == r)[0]                 # brute force: original order within the cell
        assert np.array_equal(order[off[r]:off[r + 1]], idx)
    assert np.array_equal(out, s[:, order]) and off[-1] == 5000


def _planes(t):
    return [(n, t.axis[n], t.split[n]) for n in range(len(t.axis)) if t.axis[n] >= 0]


def test_refine_splits_at_the_mean_along_the_axis_of_largest_variance():
    rng = np.random.default_rng(2)
    # one root leaf; positions stretched along y: the first plane is on y at the mean
    t = kd.grid(0)
    s = _samples(rng, 3000, spread=(0.2, 0.9, 0.4))
    nt, out, off, parent = kd.refine(t, s, np.array([0, 3000]), c=1000)
    assert nt.axis[0] == 1
    assert abs(nt.split[0] - float(np.mean(s[1].astype(np.float64)))) < 1e-9
    # every internal node: plane = mean of its vertices along their largest-variance axis
    def check(node, idx):
        if nt.axis[node] < 0:
            assert idx.size <= 1000
            return
        x = s[:3, idx].astype(np.float64)
        a = int(np.argmax(x.var(axis=1)))
        assert nt.axis[node] == a
        assert abs(nt.split[node] - x[a].mean()) < 1e-9
        go = s[a, idx].astype(np.float64) < nt.split[node]
        check(nt.left[node], idx[go])
        check(nt.left[node] + 1, idx[~go])
    check(0, np.arange(3000))
    # leaves in tree order, samples grouped and stable, parents = the one input leaf
    leaf = kd.lookup(nt, out[:3])
    assert np.array_equal(leaf, np.repeat(np.arange(len(off) - 1), np.diff(off)))
    assert np.all(parent == 0) and sorted(map(tuple, out.T.tolist())) == sorted(map(tuple, s.T.tolist()))


def test_refine_threshold_is_strictly_more_than_c():
    rng = np.random.default_rng(3)
    t = kd.grid(0)
    s = _samples(rng, 500)
    assert kd.refine(t, s, np.array([0, 500]), c=500)[0].n_leaves == 1        # M = c: kept
    assert kd.refine(t, s, np.array([0, 500]), c=499)[0].n_leaves >= 2        # M = c + 1: split


def test_identical_positions_are_not_split():
    t = kd.grid(0)
    s = np.zeros((7, 100), np.float32)
    s[:3] = 0.25
    s[5] = 1.0
    nt, out, off, parent = kd.refine(t, s, np.array([0, 100]), c=10)
    assert nt.n_leaves == 1 and np.array_equal(off, [0, 100])


def test_refine_keeps_cell_membership_and_copies_parents():
    rng = np.random.default_rng(4)
    t = kd.grid(1)
    s = _samples(rng, 20000)
    b, off, _ = kd.bin_samples(t, s)
    nt, out, noff, parent = kd.refine(t, b, off, c=700)
    assert nt.n_leaves == len(noff) - 1 > t.n_leaves
    old_leaf = kd.lookup(t, out[:3])
    new_leaf = kd.lookup(nt, out[:3])
    assert np.array_equal(new_leaf, np.repeat(np.arange(nt.n_leaves), np.diff(noff)))
    assert np.array_equal(old_leaf, parent[new_leaf])          # every new leaf lies in its parent
    assert np.all(np.diff(noff) <= 700)
