"""Python API over the C ABI of include/sdmm.h.

PyTorch provides device memory and streams; every computation runs in the
CUDA library.  The functions here only build the argument structs from
tensors and check the returned status.  There is no CPU fallback: without
the library or a GPU the calls raise.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import SdmmError, check  # noqa: F401  (SdmmError: raised by every call)

__all__ = ["config", "MixtureState", "SampleBatch", "Grid", "workspace", "workspace_bytes",
           "init_regions", "fit_regions", "fit_regions_noalloc", "prepare", "condition", "sample", "pdf", "objective",
           "objective_backward", "FitPlan", "autotune", "MapObjective", "map_objective"]

ETA_ROBBINS_MONRO, ETA_ONE = 0, 1
DENSITY_TANGENT, DENSITY_SOLID_ANGLE = 0, 1
PRIOR_SCALE_SEEN, PRIOR_SCALE_ARRAY = 0, 1
PREC_FP32, PREC_TC_3XBF16, PREC_TC_TF32, PREC_TC_3XTF32, PREC_TC_6XBF16 = 0, 1, 2, 3, 4
COV_FIRST_ORDER, COV_TWO_PASS = 0, 1
DIR_TANGENT, DIR_EUCLIDEAN = 0, 1


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def config(K: int, **kw) -> _lib.Config:
    """The paper's constants for K components (Sec. 4.2, 4.3), with overrides."""
    c = _lib.Config()
    _lib.load().sdmm_config_default(ctypes.byref(c), int(K))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


class MixtureState:
    """Parameters, averaged statistics and derived tables of R x K components."""

    FIELDS = ("pi", "mu_x", "mu_w", "L", "S0", "S2", "Wbar", "n_seen", "step_j", "status",
              "etab", "qtab")

    def __init__(self, R: int, K: int, device="cuda"):
        self.R, self.K = int(R), int(K)
        f64 = dict(dtype=torch.float64, device=device)
        self.pi = torch.zeros(R, K, **f64)
        self.mu_x = torch.zeros(R, K, 3, **f64)
        self.mu_w = torch.zeros(R, K, 3, **f64)
        self.L = torch.zeros(R, K, 15, **f64)
        self.S0 = torch.zeros(R, K, **f64)
        self.S2 = torch.zeros(R, K, 15, **f64)
        self.Wbar = torch.zeros(R, **f64)
        self.n_seen = torch.zeros(R, dtype=torch.int64, device=device)
        self.step_j = torch.zeros(R, dtype=torch.int32, device=device)
        self.status = torch.zeros(R, dtype=torch.int32, device=device)
        self.etab = torch.zeros(R, K, _lib.SDMM_ETAB_FLOATS, dtype=torch.float32, device=device)
        self.qtab = torch.zeros(R, K, _lib.SDMM_QTAB_FLOATS, dtype=torch.float32, device=device)

    def c(self) -> _lib.State:
        return _lib.State(*[getattr(self, f).data_ptr() for f in self.FIELDS])

    def set_params(self, pi, mu_x, mu_w, L):
        for name, v in (("pi", pi), ("mu_x", mu_x), ("mu_w", mu_w), ("L", L)):
            getattr(self, name).copy_(torch.as_tensor(v, dtype=torch.float64))

    def state_dict(self):
        return {f: getattr(self, f).clone() for f in self.FIELDS if f not in ("etab", "qtab")}

    def load_state_dict(self, d, cfg=None, stream=None):
        for f, v in d.items():
            getattr(self, f).copy_(v)
        if cfg is not None:
            prepare(cfg, self, stream=stream)


@dataclass
class SampleBatch:
    """FP32 samples (7, N) = (px, py, pz, ox, oy, oz, w), sorted by region,
    with int64 offsets (R + 1) on the device."""
    samples: torch.Tensor
    offsets: torch.Tensor

    def __post_init__(self):
        if self.samples.dtype != torch.float32 or self.samples.dim() != 2 or self.samples.shape[0] != 7:
            raise ValueError("samples must be a float32 tensor of shape (7, N)")
        if self.offsets.dtype != torch.int64:
            raise ValueError("offsets must be int64")
        self.samples = self.samples.contiguous()

    @property
    def R(self):
        return self.offsets.numel() - 1

    @property
    def N(self):
        return self.samples.shape[1]

    def c(self) -> _lib.Samples:
        s = self.samples
        base = s.data_ptr()
        st = s.stride(0) * s.element_size()
        return _lib.Samples(*[base + i * st for i in range(7)], self.offsets.data_ptr(), self.R, self.N)


class KdTree:
    """The spatial kD-tree of the regions (Sec. 4.2, Sec. 4.3) on the device:
    node arrays with capacity `cap_nodes`, at most `cap_leaves` leaves."""

    def __init__(self, cap_nodes: int, cap_leaves: int, device="cuda"):
        self.axis = torch.full((cap_nodes,), -1, dtype=torch.int32, device=device)
        self.split = torch.zeros(cap_nodes, dtype=torch.float64, device=device)
        self.left = torch.full((cap_nodes,), -1, dtype=torch.int32, device=device)
        self.leaf = torch.full((cap_nodes,), -1, dtype=torch.int32, device=device)
        self._c = _lib.KdTree(self.axis.data_ptr(), self.split.data_ptr(), self.left.data_ptr(),
                              self.leaf.data_ptr(), 0, 0, int(cap_nodes), int(cap_leaves))

    @property
    def n_nodes(self):
        return self._c.n_nodes

    @property
    def n_leaves(self):
        return self._c.n_leaves

    def grid(self, levels: int, stream=None):
        """Pre-subdivision: 2^levels cells per axis (3: the paper's 8 x 8 x 8)."""
        check(_lib.load().sdmm_kdtree_grid(ctypes.byref(self._c), int(levels), _stream(stream)), "sdmm_kdtree_grid")
        return self

    def lookup(self, pos: torch.Tensor, stream=None) -> torch.Tensor:
        """Leaf of each point; pos: float32 (3, Q)."""
        pos = pos.contiguous()
        Q = pos.shape[1]
        out = torch.empty(Q, dtype=torch.int32, device=pos.device)
        st = pos.stride(0) * pos.element_size()
        b = pos.data_ptr()
        check(_lib.load().sdmm_kdtree_lookup(ctypes.byref(self._c), Q, b, b + st, b + 2 * st, _ptr(out),
                                             _stream(stream)), "sdmm_kdtree_lookup")
        return out

    def _run(self, samples: torch.Tensor, offsets, c, stream):
        samples = samples.contiguous()
        N = samples.shape[1]
        n = ctypes.c_size_t()
        check(_lib.load().sdmm_kdtree_workspace_size(ctypes.byref(self._c), N, ctypes.byref(n)),
              "sdmm_kdtree_workspace_size")
        ws = torch.empty(max(1, n.value), dtype=torch.uint8, device=samples.device)
        out = torch.empty_like(samples)
        out_off = torch.empty(self._c.cap_leaves + 1, dtype=torch.int64, device=samples.device)
        base, st = out.data_ptr(), out.stride(0) * out.element_size()
        ob = _lib.SampleBuffers(*[base + i * st for i in range(7)], out_off.data_ptr(), 0, 0)
        sb, sst = samples.data_ptr(), samples.stride(0) * samples.element_size()
        off = offsets if offsets is not None else torch.zeros(2, dtype=torch.int64, device=samples.device)
        si = _lib.Samples(*[sb + i * sst for i in range(7)], off.data_ptr(),
                          self._c.n_leaves if offsets is not None else 1, N)
        return out, out_off, ob, si, ws

    def bin(self, samples: torch.Tensor, stream=None) -> "SampleBatch":
        """Samples (7, N) in any order, sorted by leaf (stable), with the leaf offsets."""
        out, out_off, ob, si, ws = self._run(samples, None, None, stream)
        check(_lib.load().sdmm_kdtree_bin(ctypes.byref(self._c), ctypes.byref(si), ctypes.byref(ob), _ptr(ws),
                                          ws.numel(), _stream(stream)), "sdmm_kdtree_bin")
        return SampleBatch(out, out_off[: ob.R + 1].clone())

    def refine(self, batch: "SampleBatch", c: int = 16000, stream=None):
        """Split every leaf holding more than c samples (Sec. 4.2); returns the
        samples sorted by the new leaves and, per new leaf, the leaf it came from."""
        out, out_off, ob, si, ws = self._run(batch.samples, batch.offsets, c, stream)
        parent = torch.empty(self._c.cap_leaves, dtype=torch.int64, device=out.device)
        check(_lib.load().sdmm_kdtree_refine(ctypes.byref(self._c), int(c), ctypes.byref(si), ctypes.byref(ob),
                                             _ptr(parent), _ptr(ws), ws.numel(), _stream(stream)),
              "sdmm_kdtree_refine")
        return SampleBatch(out, out_off[: ob.R + 1].clone()), parent[: ob.R].clone()


def gather_regions(state: "MixtureState", src: torch.Tensor, stream=None) -> "MixtureState":
    """A new state whose region r is a copy of region src[r] of `state`."""
    src = src.to(torch.int64).contiguous()
    out = MixtureState(src.numel(), state.K, device=state.pi.device)
    check(_lib.load().sdmm_gather_regions(state.K, src.numel(), _ptr(src), ctypes.byref(state.c()),
                                          ctypes.byref(out.c()), _stream(stream)), "sdmm_gather_regions")
    return out


def Grid(lo, hi, dims) -> _lib.Grid:
    g = _lib.Grid()
    for c in range(3):
        g.lo[c], g.hi[c], g.dims[c] = float(lo[c]), float(hi[c]), int(dims[c])
    return g


def workspace_bytes(cfg, R: int, N: int) -> int:
    n = ctypes.c_size_t()
    check(_lib.load().sdmm_fit_workspace_size(ctypes.byref(cfg), int(R), int(N), ctypes.byref(n)),
          "sdmm_fit_workspace_size")
    return n.value


def workspace(cfg, R: int, N: int, device="cuda") -> torch.Tensor:
    return torch.empty(workspace_bytes(cfg, R, N), dtype=torch.uint8, device=device)


def validate_samples(batch: SampleBatch, unit_tol=1e-5, stream=None):
    """Counts of bad samples: (directions not unit length within unit_tol,
    weights negative or not finite, positions not finite), int64 on the device."""
    counts = torch.empty(3, dtype=torch.int64, device=batch.samples.device)
    sm = batch.c()
    check(_lib.load().sdmm_validate_samples(ctypes.byref(sm), float(unit_tol), _ptr(counts), _stream(stream)),
          "sdmm_validate_samples")
    return counts


def init_regions(cfg, batch: SampleBatch, extent, uniforms, state: MixtureState, stream=None):
    sm = batch.c()
    st = state.c()
    check(_lib.load().sdmm_init_regions(ctypes.byref(cfg), ctypes.byref(sm), _ptr(extent),
                                        _ptr(uniforms), ctypes.byref(st), _stream(stream)),
          "sdmm_init_regions")


def fit_regions(cfg, batch: SampleBatch, iters: int, state: MixtureState, ws: torch.Tensor,
                prior_scale=None, loglik=None, stream=None):
    sm = batch.c()
    st = state.c()
    check(_lib.load().sdmm_fit_regions(ctypes.byref(cfg), ctypes.byref(sm), int(iters), _ptr(prior_scale),
                                       ctypes.byref(st), _ptr(loglik), _ptr(ws), ws.numel(),
                                       _stream(stream)), "sdmm_fit_regions")


def fit_regions_noalloc(cfg, batch: SampleBatch, iters: int, state: MixtureState, prior_scale=None,
                        loglik=None, stream=None):
    """fit_regions without a workspace, for callers that may not allocate
    device memory: the library's fixed scratch array is used instead (size
    limit and sharing rules in include/sdmm.h, sdmm_fit_regions_noalloc)."""
    sm = batch.c()
    st = state.c()
    check(_lib.load().sdmm_fit_regions_noalloc(ctypes.byref(cfg), ctypes.byref(sm), int(iters),
                                               _ptr(prior_scale), ctypes.byref(st), _ptr(loglik),
                                               _stream(stream)), "sdmm_fit_regions_noalloc")


def prepare(cfg, state: MixtureState, logits=None, delta=None, stream=None):
    st = state.c()
    check(_lib.load().sdmm_prepare(ctypes.byref(cfg), state.R, ctypes.byref(st), _ptr(logits),
                                   _ptr(delta), _stream(stream)), "sdmm_prepare")


def _grid_arg(grid):
    return None if grid is None else ctypes.byref(grid)


def condition(cfg, state: MixtureState, qx, region=None, grid=None, stream=None):
    Q, K = qx.shape[0], cfg.K
    dev = qx.device
    cpi = torch.empty(Q, K, dtype=torch.float32, device=dev)
    cm = torch.empty(Q, K, 2, dtype=torch.float32, device=dev)
    cL = torch.empty(Q, K, 3, dtype=torch.float32, device=dev)
    st = state.c()
    check(_lib.load().sdmm_condition(ctypes.byref(cfg), ctypes.byref(st), state.R, Q, _ptr(qx),
                                     _ptr(region), _grid_arg(grid), _ptr(cpi), _ptr(cm), _ptr(cL),
                                     _stream(stream)), "sdmm_condition")
    return cpi, cm, cL


def query_workspace(R: int, Q: int, device="cuda") -> torch.Tensor:
    """Workspace of the binned query entry points (sdmm_query_workspace_size)."""
    n = ctypes.c_size_t()
    check(_lib.load().sdmm_query_workspace_size(int(R), int(Q), ctypes.byref(n)), "sdmm_query_workspace_size")
    return torch.empty(max(int(n.value), 1), dtype=torch.uint8, device=device)


def sample(cfg, state: MixtureState, qx, region=None, grid=None, seed=0, uniforms=None, out=None,
           stream=None, ws=None):
    """Guided directions, pdfs and validity flags; with `ws` (query_workspace)
    the queries are binned by region inside the library (sdmm_sample_binned)."""
    Q = qx.shape[0]
    dev = qx.device
    if out is None:
        out = (torch.empty(Q, 3, dtype=torch.float32, device=dev),
               torch.empty(Q, dtype=torch.float32, device=dev),
               torch.empty(Q, dtype=torch.uint8, device=dev))
    d, p, v = out
    st = state.c()
    if ws is not None:
        check(_lib.load().sdmm_sample_binned(ctypes.byref(cfg), ctypes.byref(st), state.R, Q, _ptr(qx),
                                             _ptr(region), _grid_arg(grid), ctypes.c_uint64(seed), _ptr(uniforms),
                                             _ptr(d), _ptr(p), _ptr(v), _ptr(ws), ws.numel(), _stream(stream)),
              "sdmm_sample_binned")
        return d, p, v
    check(_lib.load().sdmm_sample(ctypes.byref(cfg), ctypes.byref(st), state.R, Q, _ptr(qx),
                                  _ptr(region), _grid_arg(grid), ctypes.c_uint64(seed), _ptr(uniforms),
                                  _ptr(d), _ptr(p), _ptr(v), _stream(stream)), "sdmm_sample")
    return d, p, v


def _lobes(bsdf_w, bsdf_mu, bsdf_L):
    w = bsdf_w.to(torch.float32).contiguous()
    mu = bsdf_mu.to(torch.float32).contiguous()
    L = bsdf_L.to(torch.float32).contiguous()
    if w.dim() != 2 or mu.shape != (*w.shape, 3) or L.shape != (*w.shape, 3):
        raise ValueError("BSDF lobes: w (Q, J), mu (Q, J, 3), L (Q, J, 3)")
    return (w, mu, L), _lib.BsdfLobes(w.data_ptr(), mu.data_ptr(), L.data_ptr(), w.shape[1])


def product_sample(cfg, state: MixtureState, qx, bsdf_w, bsdf_mu, bsdf_L, region=None, grid=None, seed=0,
                   uniforms=None, stream=None):
    """Directions from the product of each query's conditioned radiance
    mixture and its BSDF lobes (Sec. 3.5; the two largest lobes, Sec. 4.1):
    (dir (Q, 3), pdf (Q,), valid (Q,) uint8)."""
    qx = qx.contiguous()
    Q = qx.shape[0]
    keep, lobes = _lobes(bsdf_w, bsdf_mu, bsdf_L)
    d = torch.empty(Q, 3, dtype=torch.float32, device=qx.device)
    p = torch.empty(Q, dtype=torch.float32, device=qx.device)
    v = torch.empty(Q, dtype=torch.uint8, device=qx.device)
    check(_lib.load().sdmm_product_sample(ctypes.byref(cfg), ctypes.byref(state.c()), state.R, Q, _ptr(qx),
                                          _ptr(region), _grid_arg(grid), ctypes.byref(lobes), int(seed),
                                          _ptr(uniforms), _ptr(d), _ptr(p), _ptr(v), _stream(stream)),
          "sdmm_product_sample")
    return d, p, v


def product_pdf(cfg, state: MixtureState, qx, dirs, bsdf_w, bsdf_mu, bsdf_L, region=None, grid=None, stream=None):
    """Density on the sphere of the product mixture at the given directions."""
    qx = qx.contiguous()
    dirs = dirs.contiguous()
    Q = qx.shape[0]
    keep, lobes = _lobes(bsdf_w, bsdf_mu, bsdf_L)
    p = torch.empty(Q, dtype=torch.float32, device=qx.device)
    check(_lib.load().sdmm_product_pdf(ctypes.byref(cfg), ctypes.byref(state.c()), state.R, Q, _ptr(qx),
                                       _ptr(region), _grid_arg(grid), ctypes.byref(lobes), _ptr(dirs), _ptr(p),
                                       _stream(stream)),
          "sdmm_product_pdf")
    return p


def pdf(cfg, state: MixtureState, qx, dirs, region=None, grid=None, out=None, stream=None, ws=None):
    Q = qx.shape[0]
    p = out if out is not None else torch.empty(Q, dtype=torch.float32, device=qx.device)
    st = state.c()
    if ws is not None:
        check(_lib.load().sdmm_pdf_binned(ctypes.byref(cfg), ctypes.byref(st), state.R, Q, _ptr(qx), _ptr(region),
                                          _grid_arg(grid), _ptr(dirs), _ptr(p), _ptr(ws), ws.numel(),
                                          _stream(stream)), "sdmm_pdf_binned")
        return p
    check(_lib.load().sdmm_pdf(ctypes.byref(cfg), ctypes.byref(st), state.R, Q, _ptr(qx), _ptr(region),
                               _grid_arg(grid), _ptr(dirs), _ptr(p), _stream(stream)), "sdmm_pdf")
    return p


def objective(cfg, batch: SampleBatch, state: MixtureState, ws, prior_scale=None, stream=None):
    F = torch.empty(state.R, dtype=torch.float64, device=ws.device)
    sm = batch.c()
    st = state.c()
    check(_lib.load().sdmm_objective(ctypes.byref(cfg), ctypes.byref(sm), _ptr(prior_scale),
                                     ctypes.byref(st), _ptr(F), _ptr(ws), ws.numel(), _stream(stream)),
          "sdmm_objective")
    return F


def objective_backward(cfg, batch: SampleBatch, state: MixtureState, dF, ws, prior_scale=None,
                       stream=None):
    R, K = state.R, state.K
    dev = ws.device
    gd = torch.empty(R, K, 5, dtype=torch.float32, device=dev)
    gL = torch.empty(R, K, 15, dtype=torch.float32, device=dev)
    ga = torch.empty(R, K, dtype=torch.float32, device=dev)
    sm = batch.c()
    st = state.c()
    check(_lib.load().sdmm_objective_backward(ctypes.byref(cfg), ctypes.byref(sm), _ptr(prior_scale),
                                              ctypes.byref(st), _ptr(dF), _ptr(gd), _ptr(gL), _ptr(ga),
                                              _ptr(ws), ws.numel(), _stream(stream)),
          "sdmm_objective_backward")
    return gd, gL, ga


class FitPlan:
    """A fit step sequence captured once as a CUDA graph and replayed per batch."""

    def __init__(self, cfg, R: int, N_max: int, iters: int, state: MixtureState, ws, stream=None):
        self._lib = _lib.load()
        self.cfg, self.state, self.ws = cfg, state, ws
        self._st = state.c()
        h = ctypes.c_void_p()
        check(self._lib.sdmm_fit_plan_create(ctypes.byref(cfg), int(R), int(N_max), int(iters),
                                             ctypes.byref(self._st), _ptr(ws), ws.numel(), _stream(stream),
                                             ctypes.byref(h)), "sdmm_fit_plan_create")
        self.h = h

    def run(self, batch: SampleBatch, prior_scale=None, loglik=None, stream=None):
        sm = batch.c()
        check(self._lib.sdmm_fit_plan_run(self.h, ctypes.byref(sm), _ptr(prior_scale), _ptr(loglik),
                                          _stream(stream)), "sdmm_fit_plan_run")

    def staging_bytes(self) -> int:
        n = ctypes.c_size_t()
        check(self._lib.sdmm_fit_plan_staging_size(self.h, ctypes.byref(n)), "sdmm_fit_plan_staging_size")
        return n.value

    def run_host(self, batch: SampleBatch, staging, prior_scale=None, loglik=None, stream=None):
        """Run on a batch in (pinned) host memory: its copy into a slot of the
        device `staging` buffer overlaps the previous run's replay."""
        if batch.samples.is_cuda or batch.offsets.is_cuda:
            raise ValueError("run_host takes a batch in host memory")
        sm = batch.c()
        check(self._lib.sdmm_fit_plan_run_host(self.h, ctypes.byref(sm), _ptr(staging), staging.numel(),
                                               _ptr(prior_scale), _ptr(loglik), _stream(stream)),
              "sdmm_fit_plan_run_host")

    def enable_timing(self, capacity: int):
        check(self._lib.sdmm_fit_plan_enable_timing(self.h, int(capacity)), "sdmm_fit_plan_enable_timing")

    def timing(self, max_records: int = 65536):
        buf = (ctypes.c_float * max_records)()
        n = ctypes.c_int32()
        check(self._lib.sdmm_fit_plan_timing(self.h, buf, max_records, ctypes.byref(n)),
              "sdmm_fit_plan_timing")
        return [buf[i] for i in range(n.value)]

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._lib.sdmm_fit_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(cfg, batch: SampleBatch, state: MixtureState, ws, stream=None):
    sm = batch.c()
    st = state.c()
    c, g = ctypes.c_int32(), ctypes.c_int32()
    ms = ctypes.c_float()
    check(_lib.load().sdmm_autotune(ctypes.byref(cfg), ctypes.byref(sm), ctypes.byref(st), _ptr(ws),
                                    ws.numel(), _stream(stream), ctypes.byref(c), ctypes.byref(g),
                                    ctypes.byref(ms)), "sdmm_autotune")
    return c.value, g.value, ms.value


class MapObjective(torch.autograd.Function):
    """F_r(delta, L, logits): the weighted MAP objective of each region, with
    pi = softmax(logits) and each component evaluated at the in-chart mean
    offset delta (density N(d - delta; 0, L L^T)).  Forward and backward run
    the library's kernels; the inputs are written into `state` (L, pi) before
    each evaluation."""

    @staticmethod
    def forward(ctx, delta, L, logits, cfg, batch, state, ws, prior_scale):
        state.L.copy_(L.detach())
        prepare(cfg, state, logits=logits.detach().contiguous(), delta=delta.detach().contiguous())
        F = objective(cfg, batch, state, ws, prior_scale)
        ctx.save_for_backward(delta.detach(), L.detach(), logits.detach())
        ctx.extra = (cfg, batch, state, ws, prior_scale)
        return F

    @staticmethod
    def backward(ctx, gF):
        delta, L, logits = ctx.saved_tensors
        cfg, batch, state, ws, prior_scale = ctx.extra
        state.L.copy_(L)
        prepare(cfg, state, logits=logits.contiguous(), delta=delta.contiguous())
        gd, gL, ga = objective_backward(cfg, batch, state, gF.to(torch.float64).contiguous(), ws,
                                        prior_scale)
        return (gd.to(delta.dtype), gL.to(L.dtype), ga.to(logits.dtype), None, None, None, None, None)


def map_objective(cfg, batch, state, ws, delta, L, logits, prior_scale=None):
    return MapObjective.apply(delta, L, logits, cfg, batch, state, ws, prior_scale)
