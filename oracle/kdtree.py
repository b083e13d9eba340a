"""Spatial kD-tree of the regions: lookup, binning and refinement (Sec. 4.2
"Refinement of the spatial kD-tree", Sec. 4.3 "Initialization").

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): a plain, sequential
numpy statement of what the CUDA path computes, shared with nothing on that
path.

Tree: node arrays axis (split axis 0..2, -1 for a leaf), split (float64
split position; x[axis] < split goes left), left (first child; the second is
left + 1), leaf (leaf index of a leaf node).  Leaves are numbered in tree
order (left before right), so the samples of leaf r form the r-th contiguous
segment when samples are sorted by leaf.

Readings (the paper fixes the rule, not its arithmetic):
  * a leaf is split when it holds more than c vertices (M > c);
  * "largest variation" is the population variance of the vertex positions
    along each axis, the lowest axis on ties; the plane is at the mean;
  * mean and variance come from fixed-point sums: q = floor(clamp(x, 0, 1)
    2^32) and q2 = floor(clamp(x, 0, 1)^2 2^32), summed exactly as integers,
    mean = (S / M) / 2^32, variance = (S2 / M) / 2^32 - mean^2 in FP64, so
    that every implementation places the plane identically (positions are
    normalised to the scene's bounding box, Sec. 4.3);
  * a split that would leave one side empty is not made (all positions equal
    along the axis);
  * children are redistributed stably (original order kept within a leaf);
  * the pre-subdivision of Sec. 4.3 splits every axis at the centre of its
    cell, x then y then z, `levels` times (3 levels: 8 x 8 x 8 cells).
"""
from __future__ import annotations

import numpy as np

TWO32 = 4294967296.0


class Tree:
    def __init__(self):
        self.axis, self.split, self.left, self.leaf = [], [], [], []

    def node(self, axis=-1, split=0.0, left=-1, leaf=-1):
        self.axis.append(axis)
        self.split.append(split)
        self.left.append(left)
        self.leaf.append(leaf)
        return len(self.axis) - 1

    @property
    def n_leaves(self):
        return sum(1 for a in self.axis if a < 0)

    def copy(self):
        t = Tree()
        t.axis, t.split, t.left, t.leaf = list(self.axis), list(self.split), list(self.left), list(self.leaf)
        return t


def grid(levels: int) -> Tree:
    """Regular pre-subdivision of [0,1]^3: 2^levels cells per axis."""
    t = Tree()
    root = t.node()
    counter = [0]

    def build(n, lo, hi, depth):
        if depth == 3 * levels:
            t.leaf[n] = counter[0]
            counter[0] += 1
            return
        a = depth % 3
        mid = 0.5 * (lo[a] + hi[a])
        l = t.node()
        r = t.node()
        t.axis[n], t.split[n], t.left[n] = a, mid, l
        lhi = list(hi)
        lhi[a] = mid
        rlo = list(lo)
        rlo[a] = mid
        build(l, lo, lhi, depth + 1)
        build(r, rlo, hi, depth + 1)

    build(root, [0.0, 0.0, 0.0], [1.0, 1.0, 1.0], 0)
    return t


def lookup(t: Tree, pos: np.ndarray) -> np.ndarray:
    """Leaf of every point (pos: (3, Q) float32), by descent from the root."""
    Q = pos.shape[1]
    out = np.empty(Q, dtype=np.int32)
    for i in range(Q):
        n = 0
        while t.axis[n] >= 0:
            n = t.left[n] if float(pos[t.axis[n], i]) < t.split[n] else t.left[n] + 1
        out[i] = t.leaf[n]
    return out


def bin_samples(t: Tree, samples: np.ndarray):
    """Samples (7, N) sorted by leaf (stable), and the leaf offsets."""
    leaf = lookup(t, samples[:3])
    order = np.argsort(leaf, kind="stable")
    counts = np.bincount(leaf, minlength=t.n_leaves)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return samples[:, order], offsets, order


def _plane(x: np.ndarray):
    """(axis, split) of a vertex set x (3, M) by the fixed-point rule."""
    xc = np.clip(x.astype(np.float64), 0.0, 1.0)
    q = np.floor(xc * TWO32).astype(np.uint64)
    q2 = np.floor(xc * xc * TWO32).astype(np.uint64)
    M = x.shape[1]
    best, axis, split = -1.0, 0, 0.0
    for a in range(3):
        S = int(q[a].sum(dtype=np.uint64))
        S2 = int(q2[a].sum(dtype=np.uint64))
        mean = (float(S) / float(M)) / TWO32
        var = (float(S2) / float(M)) / TWO32 - mean * mean
        if var > best:
            best, axis, split = var, a, mean
    return axis, split


def refine(t: Tree, samples: np.ndarray, offsets: np.ndarray, c: int):
    """Split every leaf holding more than c vertices, recursively (Sec. 4.2).

    samples: (7, N) sorted by leaf; offsets: (n_leaves + 1,).  Returns the
    new tree, the samples sorted by the new leaves, the new offsets, and for
    every new leaf the leaf it came from (its mixture is copied from there).
    """
    t = t.copy()
    # leaves in tree order, with their nodes
    leaf_node = {}
    for n, a in enumerate(t.axis):
        if a < 0:
            leaf_node[t.leaf[n]] = n
    R = len(leaf_node)
    new_cols, new_counts, parent = [], [], []

    def split(node, idx, src):
        x = samples[:3, idx]
        M = idx.size
        if M > c:
            a, s = _plane(x)
            go_left = x[a].astype(np.float64) < s
            nl = int(go_left.sum())
            if 0 < nl < M:
                l = t.node()
                r = t.node()
                t.axis[node], t.split[node], t.left[node], t.leaf[node] = a, s, l, -1
                split(l, idx[go_left], src)
                split(r, idx[~go_left], src)
                return
        t.leaf[node] = len(new_counts)
        new_cols.append(idx)
        new_counts.append(M)
        parent.append(src)

    for r in range(R):
        split(leaf_node[r], np.arange(offsets[r], offsets[r + 1]), r)
    order = np.concatenate(new_cols) if new_cols else np.zeros(0, np.int64)
    new_off = np.concatenate([[0], np.cumsum(new_counts)]).astype(np.int64)
    return t, samples[:, order], new_off, np.asarray(parent, dtype=np.int64)
