"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws data: it holds none of the fitting or query
arithmetic and imports neither the CUDA library nor the oracle, so both can
be fed the same arrays.  Random numbers that the method itself consumes
(initialisation seeds, sampling uniforms) are generated here and passed in as
inputs.

Ground-truth mixtures follow the synthetic recipe of the workloads:
  * K components, weights ~ Dirichlet(1);
  * spatial means uniform in [0.1, 0.9]^3 of the region's cell, isotropic
    spatial std U(0.05, 0.2) x cell size;
  * directional means uniform on the sphere; tangent-plane lobes with per-axis
    angular std U(0.05, 0.5) rad and a random in-plane rotation;
  * optional "parallax": a random position/direction cross-covariance;
  * sample weights log-normal(0, 1.5).
Directions are drawn by walking a geodesic of length |nu| from the lobe
centre along the tangent direction (nu_1 e1 + nu_2 e2)/|nu|, where (e1, e2)
is a frame the generator picks by Gram-Schmidt; draws with |nu| >= pi are
redrawn.  The frame is reported so that tests can express the ground truth
without reference to any chart convention.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

FIELDS = ("px", "py", "pz", "ox", "oy", "oz", "w")


@dataclass
class GroundTruth:
    """Frame-free description of R regions x K components (FP64)."""
    pi: np.ndarray        # (R, K)
    mu_x: np.ndarray      # (R, K, 3)
    mu_w: np.ndarray      # (R, K, 3) unit
    e1: np.ndarray        # (R, K, 3) tangent frame used for the lobe
    e2: np.ndarray        # (R, K, 3)
    cov: np.ndarray       # (R, K, 5, 5) joint covariance of (x, nu) in frame (e1, e2)

    @property
    def R(self):
        return self.pi.shape[0]

    @property
    def K(self):
        return self.pi.shape[1]


def _unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _frame(rng, mu):
    """Gram-Schmidt tangent frame at each unit vector in mu (n, 3)."""
    a = rng.normal(size=mu.shape)
    e1 = a - np.sum(a * mu, axis=1, keepdims=True) * mu
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(mu, e1)
    return e1, e2


def ground_truth(rng, R, K, cell_lo=None, cell_size=None, parallax=False) -> GroundTruth:
    cell_lo = np.zeros((R, 3)) if cell_lo is None else np.asarray(cell_lo, float).reshape(R, 3)
    h = np.ones(R) if cell_size is None else np.broadcast_to(np.asarray(cell_size, float), (R,))
    pi = rng.dirichlet(np.ones(K), size=R)
    mu_x = cell_lo[:, None, :] + h[:, None, None] * rng.uniform(0.1, 0.9, size=(R, K, 3))
    sx = h[:, None] * rng.uniform(0.05, 0.2, size=(R, K))
    mu_w = _unit(rng, R * K)
    e1, e2 = _frame(rng, mu_w)
    sig = rng.uniform(0.05, 0.5, size=(R * K, 2))
    ang = rng.uniform(0.0, math.pi, size=R * K)
    c, s = np.cos(ang), np.sin(ang)
    rot = np.stack([np.stack([c, -s], -1), np.stack([s, c], -1)], -2)      # (RK, 2, 2)
    lnu = rot * sig[:, None, :]                                         # (RK, 2, 2)
    F = np.zeros((R * K, 5, 5))
    F[:, :3, :3] = sx.reshape(-1)[:, None, None] * np.eye(3)
    F[:, 3:, 3:] = lnu
    if parallax:
        # direction noise partly driven by position noise: nu = Lnu (rho G z_x
        # + sqrt(1 - rho^2) z_nu), correlation up to 0.6 (positive definite
        # by construction)
        rho = rng.uniform(0.0, 0.6, size=R * K)
        G = rng.normal(size=(R * K, 2, 3)) / math.sqrt(3.0)
        F[:, 3:, :3] = lnu @ (rho[:, None, None] * G)
        F[:, 3:, 3:] = lnu * np.sqrt(1.0 - rho ** 2)[:, None, None]
    cov = F @ np.swapaxes(F, 1, 2)
    return GroundTruth(pi=pi, mu_x=mu_x, mu_w=mu_w.reshape(R, K, 3),
                       e1=e1.reshape(R, K, 3), e2=e2.reshape(R, K, 3),
                       cov=cov.reshape(R, K, 5, 5))


def _component_index(u, reg, gt: GroundTruth):
    R, K = gt.R, gt.K
    cum = np.cumsum(gt.pi, axis=1)
    cum[:, -1] = 1.0
    glob = (cum + np.arange(R)[:, None]).reshape(-1)
    k = np.searchsorted(glob, reg + u, side="right") - reg * K
    return reg * K + np.minimum(k, K - 1)


def draw(rng, gt: GroundTruth, counts) -> np.ndarray:
    """Samples of every region, concatenated region by region: (7, N) float32."""
    counts = np.asarray(counts, dtype=np.int64)
    R, K = gt.R, gt.K
    N = int(counts.sum())
    reg = np.repeat(np.arange(R), counts)
    rk = _component_index(rng.random(N), reg, gt)
    chol = np.linalg.cholesky(gt.cov.reshape(R * K, 5, 5))
    mux = gt.mu_x.reshape(-1, 3)
    out = np.empty((7, N), dtype=np.float32)
    x = np.empty((N, 3))
    nu = np.empty((N, 2))
    todo = np.arange(N)
    while todo.size:
        z = rng.normal(size=(todo.size, 5))
        idx = rk[todo]
        v = np.zeros((todo.size, 5))
        for i in range(5):                      # v = chol z, row by row
            for j in range(i + 1):
                v[:, i] += chol[idx, i, j] * z[:, j]
        x[todo] = mux[idx] + v[:, :3]
        nu[todo] = v[:, 3:]
        todo = todo[np.hypot(nu[todo, 0], nu[todo, 1]) >= math.pi]
    r = np.hypot(nu[:, 0], nu[:, 1])
    safe = np.where(r > 0, r, 1.0)
    e1 = gt.e1.reshape(-1, 3)[rk]
    e2 = gt.e2.reshape(-1, 3)[rk]
    mu = gt.mu_w.reshape(-1, 3)[rk]
    cr, sr = np.cos(r), np.sin(r) / safe
    d = cr[:, None] * mu + (sr * nu[:, 0])[:, None] * e1 + (sr * nu[:, 1])[:, None] * e2
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    out[0:3] = x.T
    out[3:6] = d.T
    out[6] = rng.lognormal(0.0, 1.5, size=N)
    return out


def draw_torch(seed, gt: GroundTruth, counts, device="cuda", block=1 << 22):
    """The same recipe as draw() with torch on `device` (a different random
    stream, same distribution), for workloads too large to draw on the host.
    Returns a (7, N) float32 tensor.  Works in blocks of `block` samples."""
    import torch
    counts = np.asarray(counts, dtype=np.int64)
    R, K = gt.R, gt.K
    N = int(counts.sum())
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = dict(dtype=torch.float64, device=device)
    reg_all = torch.repeat_interleave(torch.arange(R, device=device),
                                      torch.as_tensor(counts, device=device))
    cum = torch.as_tensor(np.cumsum(gt.pi, axis=1), **f64)
    cum[:, -1] = 1.0
    glob = (cum + torch.arange(R, **f64)[:, None]).reshape(-1)
    chol = torch.as_tensor(np.linalg.cholesky(gt.cov.reshape(R * K, 5, 5)), **f64)
    mux = torch.as_tensor(gt.mu_x.reshape(-1, 3), **f64)
    E1 = torch.as_tensor(gt.e1.reshape(-1, 3), **f64)
    E2 = torch.as_tensor(gt.e2.reshape(-1, 3), **f64)
    MU = torch.as_tensor(gt.mu_w.reshape(-1, 3), **f64)
    out = torch.empty(7, N, dtype=torch.float32, device=device)
    for b0 in range(0, N, block):
        b1 = min(N, b0 + block)
        n = b1 - b0
        reg = reg_all[b0:b1]
        u = torch.rand(n, generator=g, **f64)
        k = torch.searchsorted(glob, reg.to(torch.float64) + u, right=True) - reg * K
        rk = reg * K + torch.clamp(k, max=K - 1)
        x = torch.empty(n, 3, **f64)
        nu = torch.empty(n, 2, **f64)
        todo = torch.arange(n, device=device)
        while todo.numel():
            z = torch.randn(todo.numel(), 5, generator=g, **f64)
            v = torch.einsum("nij,nj->ni", chol[rk[todo]], z)
            x[todo] = mux[rk[todo]] + v[:, :3]
            nu[todo] = v[:, 3:]
            todo = todo[torch.hypot(nu[todo, 0], nu[todo, 1]) >= math.pi]
        r = torch.hypot(nu[:, 0], nu[:, 1])
        safe = torch.where(r > 0, r, torch.ones_like(r))
        sr = torch.sin(r) / safe
        d = (torch.cos(r)[:, None] * MU[rk] + (sr * nu[:, 0])[:, None] * E1[rk]
             + (sr * nu[:, 1])[:, None] * E2[rk])
        d = d / torch.linalg.norm(d, dim=1, keepdim=True)
        w = torch.exp(1.5 * torch.randn(n, generator=g, **f64))
        out[0:3, b0:b1] = x.T.to(torch.float32)
        out[3:6, b0:b1] = d.T.to(torch.float32)
        out[6, b0:b1] = w.to(torch.float32)
    return out


def offsets_from_counts(counts) -> np.ndarray:
    counts = np.asarray(counts, dtype=np.int64)
    off = np.zeros(counts.size + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off


@dataclass
class Batch:
    samples: np.ndarray    # (7, N) float32: px, py, pz, ox, oy, oz, w
    offsets: np.ndarray    # (R + 1,) int64
    extent: np.ndarray     # (R,) longest side of each region's cell
    truth: GroundTruth

    @property
    def R(self):
        return self.offsets.size - 1

    @property
    def N(self):
        return int(self.offsets[-1])


def single_region(seed=0, N=65536, K=16, parallax=False) -> Batch:
    """One region on the unit cube, N samples from a K-component truth."""
    rng = np.random.default_rng([seed, 0])
    gt = ground_truth(rng, 1, K, parallax=parallax)
    s = draw(rng, gt, [N])
    return Batch(s, offsets_from_counts([N]), np.ones(1), gt)


def region_grid(R):
    """Cells of a near-cubic grid of R regions over the unit cube."""
    n = round(R ** (1.0 / 3.0))
    dims = None
    for a in range(max(1, n - 2), n + 3):
        for b in range(a, n + 3):
            if R % (a * b) == 0:
                c = R // (a * b)
                cand = sorted((a, b, c), reverse=True)
                if dims is None or max(cand) - min(cand) < max(dims) - min(dims):
                    dims = tuple(cand)
    if dims is None:
        dims = (R, 1, 1)
    idx = np.arange(R)
    ijk = np.stack([idx % dims[0], (idx // dims[0]) % dims[1], idx // (dims[0] * dims[1])], 1)
    size = 1.0 / np.array(dims, float)
    return ijk * size, np.broadcast_to(size.max(), (R,)).copy(), dims


def region_counts(seed, R, m_lo=256, m_hi=65536):
    """Per-region sample counts, log-uniform in [m_lo, m_hi]."""
    rng = np.random.default_rng([seed, 1])
    return np.floor(np.exp(rng.uniform(math.log(m_lo), math.log(m_hi), size=R))).astype(np.int64)


def batched_truth(seed, R, K=16, parallax=False) -> GroundTruth:
    rng = np.random.default_rng([seed, 2])
    lo, h, _ = region_grid(R)
    return ground_truth(rng, R, K, cell_lo=lo, cell_size=h, parallax=parallax)


def batched_round(seed, R, counts, round_index, truth: GroundTruth) -> Batch:
    """A fresh batch of every region's samples for one stepwise-EM round."""
    rng = np.random.default_rng([seed, 3, round_index])
    s = draw(rng, truth, counts)
    _, h, _ = region_grid(R)
    return Batch(s, offsets_from_counts(counts), h, truth)


def init_uniforms(seed, R, per_region):
    """Uniforms consumed by the k-means++ seeding of the initialisation."""
    return np.random.default_rng([seed, 4]).random((R, per_region))


def random_mixtures(seed, dims=(64, 32, 32), K=16):
    """Per-cell K-component 5-D mixtures for the query workload.

    Returns (pi, mu_x, mu_w, L) with L a random lower-triangular factor in the
    (x, nu) order: position block with std U(0.05, 0.2) x cell size, direction
    block with std U(0.05, 0.5) rad, and random cross terms.
    """
    rng = np.random.default_rng([seed, 5])
    R = int(np.prod(dims))
    idx = np.arange(R)
    ijk = np.stack([idx % dims[0], (idx // dims[0]) % dims[1], idx // (dims[0] * dims[1])], 1)
    h = 1.0 / np.array(dims, float)
    lo = ijk * h
    pi = rng.dirichlet(np.ones(K), size=R)
    mu_x = lo[:, None, :] + h[None, None, :] * rng.uniform(0.1, 0.9, size=(R, K, 3))
    mu_w = _unit(rng, R * K).reshape(R, K, 3)
    L = np.zeros((R, K, 15))
    sx = h.max() * rng.uniform(0.05, 0.2, size=(R, K, 3))
    sd = rng.uniform(0.05, 0.5, size=(R, K, 2))
    diag = np.concatenate([sx, sd], axis=2)
    for i in range(5):
        L[:, :, i * (i + 1) // 2 + i] = diag[:, :, i]
        for j in range(i):
            L[:, :, i * (i + 1) // 2 + j] = 0.3 * rng.normal(size=(R, K)) * diag[:, :, i]
    return pi, mu_x, mu_w, L


def query_points(seed, Q):
    return np.random.default_rng([seed, 6]).random((Q, 3), dtype=np.float32)


def grid_region(qx, dims):
    """Cell index of each position on a uniform grid over the unit cube."""
    d = np.asarray(dims)
    ijk = np.clip(np.floor(np.asarray(qx, np.float64) * d).astype(np.int64), 0, d - 1)
    return (ijk[:, 0] + d[0] * (ijk[:, 1] + d[1] * ijk[:, 2])).astype(np.int32)


def bsdf_lobes(seed, Q, J=3):
    """Per-query BSDF mixtures of J lobes for product sampling.

    Lobe 0 is wide (a diffuse-like lobe about a random normal, std U(0.6, 0.9)
    rad), lobe 1 narrow (a glossy lobe about a random direction in the normal's
    hemisphere, std U(0.03, 0.3) rad), further lobes random with std
    U(0.05, 0.6) rad; weights U(0.05, 1).  Returns float32 (w (Q, J),
    mu (Q, J, 3), L (Q, J, 3)) with L the lower-triangular factor
    (l00, l10, l11) of each lobe's covariance in its own chart.
    """
    rng = np.random.default_rng([seed, 7])
    n = _unit(rng, Q)
    mu = _unit(rng, Q * J).reshape(Q, J, 3)
    sd = rng.uniform(0.05, 0.6, size=(Q, J, 2))
    sd[:, 0] = rng.uniform(0.6, 0.9, size=(Q, 2))
    mu[:, 0] = n
    if J > 1:
        r = mu[:, 1]
        r = np.where((np.sum(r * n, axis=1) < 0)[:, None], -r, r)
        mu[:, 1] = r
        sd[:, 1] = rng.uniform(0.03, 0.3, size=(Q, 2))
    L = np.stack([sd[..., 0], 0.3 * rng.normal(size=(Q, J)) * sd[..., 1], sd[..., 1]], axis=2)
    w = rng.uniform(0.05, 1.0, size=(Q, J))
    return w.astype(np.float32), mu.astype(np.float32), L.astype(np.float32)
