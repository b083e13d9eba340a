"""FP64 CPU oracle of the SDMM hot path, loaded through ctypes.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The oracle is a plain C library
(``oracle/*.c``, FP64, unblocked loops in the paper's order) that shares no
code with the CUDA library.  This module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["geom.c", "em.c", "query.c", "philox.c"]
LIB_PATH = os.path.join(_HERE, "liboracle_sdmm.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP64, no contraction)."""
    srcs = [os.path.join(_HERE, s) for s in SOURCES]
    if not force and os.path.exists(LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "sdmm_oracle.h")])
        if os.path.getmtime(LIB_PATH) >= newest:
            return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class OrConfig(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("min_samples", ctypes.c_int32),
                ("eta_mode", ctypes.c_int32), ("estep_density", ctypes.c_int32),
                ("euclid", ctypes.c_int32), ("cov_update", ctypes.c_int32),
                ("prior_scale_mode", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("eta_alpha", ctypes.c_double), ("eta_beta", ctypes.c_double),
                ("prior_q", ctypes.c_double), ("prior_a", ctypes.c_double),
                ("prior_B_pos", ctypes.c_double), ("prior_B_dir", ctypes.c_double)]


class OrState(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("pi", "mu_x", "mu_w", "L", "S0", "S2", "Wbar", "n_seen", "step_j", "status")]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB_PATH)
            L.or_sinc.restype = ctypes.c_double
            L.or_sinc.argtypes = [ctypes.c_double]
            for n in ("or_basis", "or_exp_map", "or_jexp", "or_jlog"):
                getattr(L, n).restype = None
            L.or_log_map.restype = ctypes.c_int
            L.or_cholesky5.restype = ctypes.c_int
            L.or_config_default.restype = None
            L.or_config_default.argtypes = [ctypes.POINTER(OrConfig), ctypes.c_int]
            L.or_estep_region.argtypes = [ctypes.POINTER(OrConfig), ctypes.c_int] + [_P] * 5 + \
                [_I64] + [_P] * 7 + [_P] * 6
            L.or_fit_regions.argtypes = [ctypes.POINTER(OrConfig), _I64, _P] + [_P] * 7 + \
                [ctypes.c_int, _P, ctypes.POINTER(OrState), _P]
            L.or_init_regions.argtypes = [ctypes.POINTER(OrConfig), _I64, _P] + [_P] * 4 + \
                [_P, _P, ctypes.POINTER(OrState)]
            L.or_objective.argtypes = [ctypes.POINTER(OrConfig), _I64, _P] + [_P] * 7 + \
                [_P, ctypes.POINTER(OrState), _P, _P, _P, _P, _P]
            L.or_condition.argtypes = [ctypes.c_int] + [_P] * 4 + [_I64] + [_P] * 5
            L.or_pdf.argtypes = [ctypes.c_int] + [_P] * 4 + [_I64] + [_P] * 4
            L.or_sample.argtypes = [ctypes.c_int] + [_P] * 4 + [_I64] + [_P] * 8
            L.or_philox4x32_10.argtypes = [_P, _P, _P]
            L.or_uniforms.argtypes = [ctypes.c_uint64, _I64, _P]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def config(K: int, **kw) -> OrConfig:
    c = OrConfig()
    lib().or_config_default(ctypes.byref(c), int(K))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


# ---------------------------------------------------------------- geometry
def sinc(r: float) -> float:
    return lib().or_sinc(float(r))


def basis(mu):
    R = np.zeros(9)
    lib().or_basis(_p(_f64(mu)), _p(R))
    return R.reshape(3, 3)


def log_map(mu, w):
    nu = np.zeros(2)
    th = ctypes.c_double()
    s = ctypes.c_double()
    anti = lib().or_log_map(_p(_f64(mu)), _p(_f64(w)), _p(nu), ctypes.byref(th), ctypes.byref(s))
    return nu, bool(anti), th.value, s.value


def exp_map(mu, nu):
    w = np.zeros(3)
    lib().or_exp_map(_p(_f64(mu)), _p(_f64(nu)), _p(w))
    return w


def jexp(mu, nu):
    J = np.zeros(6)
    lib().or_jexp(_p(_f64(mu)), _p(_f64(nu)), _p(J))
    return J.reshape(3, 2)


def jlog(mu, w):
    J = np.zeros(6)
    lib().or_jlog(_p(_f64(mu)), _p(_f64(w)), _p(J))
    return J.reshape(2, 3)


def cholesky5(S_packed):
    L = np.zeros(15)
    bad = lib().or_cholesky5(_p(_f64(S_packed)), _p(L))
    return L, bool(bad)


# ---------------------------------------------------------------- state
class State:
    """Mixture parameters and averaged statistics of R regions (numpy, FP64)."""

    def __init__(self, R: int, K: int):
        self.R, self.K = R, K
        self.pi = np.zeros((R, K))
        self.mu_x = np.zeros((R, K, 3))
        self.mu_w = np.zeros((R, K, 3))
        self.L = np.zeros((R, K, 15))
        self.S0 = np.zeros((R, K))
        self.S2 = np.zeros((R, K, 15))
        self.Wbar = np.zeros(R)
        self.n_seen = np.zeros(R, dtype=np.int64)
        self.step_j = np.zeros(R, dtype=np.int32)
        self.status = np.zeros(R, dtype=np.int32)

    FIELDS = ("pi", "mu_x", "mu_w", "L", "S0", "S2", "Wbar", "n_seen", "step_j", "status")

    def copy(self) -> "State":
        s = State(self.R, self.K)
        for f in self.FIELDS:
            setattr(s, f, getattr(self, f).copy())
        return s

    def c(self) -> OrState:
        return OrState(*[getattr(self, f).ctypes.data for f in self.FIELDS])

    def set_params(self, pi, mu_x, mu_w, L):
        self.pi[...] = pi
        self.mu_x[...] = mu_x
        self.mu_w[...] = mu_w
        self.L[...] = L


def _rows(samples):
    s = np.ascontiguousarray(samples, dtype=np.float32)
    assert s.shape[0] == 7
    return s, [s[i].ctypes.data_as(ctypes.c_void_p) for i in range(7)]


def estep_region(cfg, pi, mu_x, mu_w, L, samples, delta=None):
    K = cfg.K
    s, rows = _rows(samples)
    M = s.shape[1]
    loglik = np.zeros(M)
    resp = np.zeros((M, K))
    s0, s1, s2 = np.zeros(K), np.zeros((K, 5)), np.zeros((K, 15))
    W = ctypes.c_double()
    lib().or_estep_region(ctypes.byref(cfg), K, _p(_f64(pi)), _p(_f64(mu_x)), _p(_f64(mu_w)),
                          _p(_f64(L)), _p(None if delta is None else _f64(delta)), M, *rows,
                          _p(loglik), _p(resp), _p(s0), _p(s1), _p(s2), ctypes.byref(W))
    return dict(loglik=loglik, resp=resp, s0=s0, s1=s1, s2=s2, W=W.value)


def fit_regions(cfg, offsets, samples, iters, state: State, prior_scale=None, want_loglik=False):
    s, rows = _rows(samples)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    R = off.shape[0] - 1
    ll = np.zeros(s.shape[1]) if want_loglik else None
    ps = None if prior_scale is None else _f64(prior_scale)
    st = state.c()
    lib().or_fit_regions(ctypes.byref(cfg), R, _p(off), *rows, int(iters), _p(ps),
                         ctypes.byref(st), _p(ll))
    return ll


def init_regions(cfg, offsets, samples, extent, uniforms, state: State):
    s, rows = _rows(samples)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    R = off.shape[0] - 1
    ext = _f64(extent)
    u = _f64(uniforms)
    st = state.c()
    lib().or_init_regions(ctypes.byref(cfg), R, _p(off), rows[0], rows[1], rows[2], rows[6],
                          _p(ext), _p(u), ctypes.byref(st))


def objective(cfg, offsets, samples, state: State, prior_scale=None, delta=None, grads=True):
    s, rows = _rows(samples)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    R, K = off.shape[0] - 1, cfg.K
    F = np.zeros(R)
    gd = np.zeros((R, K, 5)) if grads else None
    gL = np.zeros((R, K, 15)) if grads else None
    ga = np.zeros((R, K)) if grads else None
    ps = None if prior_scale is None else _f64(prior_scale)
    dl = None if delta is None else _f64(delta)
    st = state.c()
    lib().or_objective(ctypes.byref(cfg), R, _p(off), *rows, _p(ps), ctypes.byref(st), _p(dl),
                       _p(F), _p(gd), _p(gL), _p(ga))
    return (F, gd, gL, ga) if grads else F


# ---------------------------------------------------------------- queries
def _params(K, pi, mu_x, mu_w, L):
    return [_f64(pi), _f64(mu_x), _f64(mu_w), _f64(L)]


def condition(K, pi, mu_x, mu_w, L, qx, region):
    P = _params(K, pi, mu_x, mu_w, L)
    qx = np.ascontiguousarray(qx, dtype=np.float32)
    region = np.ascontiguousarray(region, dtype=np.int32)
    Q = region.shape[0]
    cpi, cm, cL = np.zeros((Q, K)), np.zeros((Q, K, 2)), np.zeros((Q, K, 3))
    lib().or_condition(int(K), *[_p(a) for a in P], Q, _p(qx), _p(region), _p(cpi), _p(cm), _p(cL))
    return cpi, cm, cL


def pdf(K, pi, mu_x, mu_w, L, qx, region, dirs):
    P = _params(K, pi, mu_x, mu_w, L)
    qx = np.ascontiguousarray(qx, dtype=np.float32)
    region = np.ascontiguousarray(region, dtype=np.int32)
    d = _f64(dirs)
    Q = region.shape[0]
    out = np.zeros(Q)
    lib().or_pdf(int(K), *[_p(a) for a in P], Q, _p(qx), _p(region), _p(d), _p(out))
    return out


def sample(K, pi, mu_x, mu_w, L, qx, region, uniforms):
    P = _params(K, pi, mu_x, mu_w, L)
    qx = np.ascontiguousarray(qx, dtype=np.float32)
    region = np.ascontiguousarray(region, dtype=np.int32)
    u = np.ascontiguousarray(uniforms, dtype=np.float32)
    Q = region.shape[0]
    d, p = np.zeros((Q, 3)), np.zeros(Q)
    v = np.zeros(Q, dtype=np.uint8)
    comp = np.zeros(Q, dtype=np.int32)
    margin = np.zeros(Q)
    lib().or_sample(int(K), *[_p(a) for a in P], Q, _p(qx), _p(region), _p(u), _p(d), _p(p),
                    _p(v), _p(comp), _p(margin))
    return dict(dir=d, pdf=p, valid=v, comp=comp, margin=margin)


# ---------------------------------------------------------------- RNG
def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def uniforms(seed: int, Q: int):
    out = np.zeros((Q, 3), dtype=np.float32)
    lib().or_uniforms(ctypes.c_uint64(seed), int(Q), _p(out))
    return out
