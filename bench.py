"""Benchmark of the SDMM hot path on GB300.

Workload (one step): the batched stepwise fit of 4,096 regions x K = 16
components, sample counts log-uniform in [256, 65,536] per region, four
Robbins-Monro EM rounds with a fresh seeded batch each, starting from the
regions' initial state (restored by device-to-device copies at the start of
every step, inside the timed region), every round one persistent E-step
launch plus reductions replayed from a CUDA graph.  Inputs are resident in
HBM (about 1.38 GB per round, larger than L2) when the timed region starts.
`value` = sample-iterations per second over all ranks.

Also reported on the same line:
  * the E-step kernel's roofline (FP32 ALU bound) from CUDA events inside
    the replayed graph;
  * the tensor-core contraction form (6xBF16) on the same step;
  * the end-to-end rate through the public API with host buffers, beside a
    plain pinned host-to-device copy of the same bytes (its ceiling);
  * the query workload (16M guided queries over 65,536 grid regions) with its
    roofline, and product sampling;
  * the FP64 oracle on the host cores (`cpu_baseline`): single-threaded and
    over all cores, on a bounded sample of each workload; its results on that
    sample are the reference of the matched-error comparison of every GPU
    form (`accuracy`): per-sample log-likelihood and parameter errors after
    the step's four rounds, pdf errors of the queries;
  * the other workloads as sub-objects (`configs`): the single-region fit,
    the precision sweep (1,024 x 65,536, K = 16 and 32, every E-step form),
    the MAP objective and its adjoint, and the ablations (covariance update,
    E-step density, Euclidean directions).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EM sample-iterations/s and guided queries/s vs plain FP32 at matched log-lik"
UNIT = "sample-iterations/s"
K_COMP, ROUNDS = 16, 4
# work-unit size of the batched fit (the library's heuristic picks it for this
# workload too); the accuracy check fits its sample of regions with the same
# units, so every region's arithmetic is the timed run's
CHUNK = 4096
Q_DIMS, Q_COUNT = (64, 32, 32), 16 * 2 ** 20
# algorithmic FP32 work of the E-step + statistics per (sample, component):
# log map 23, Mahalanobis 39, log-sum-exp and responsibility 6, statistics 46
FLOPS_PER_PAIR = 114
# algorithmic FP32 work of a guided query: per component 32 (conditioning:
# offset 3, A^-1 e 9, log weight 7, C^T z 10, normalisation 3) + 39 (pdf at the
# sampled direction: chart coordinates 15, theta/sin(theta) 7, nu 2, offset 2,
# D^-1 4, Gaussian 6, weight and sum 3), per query 70 (component choice 32,
# Box-Muller 8, Gaussian draw 5, exp map 25)
FLOPS_PER_QUERY_COMPONENT, FLOPS_PER_QUERY = 71, 70
# bytes per sample of one E-step pass: 7 FP32 streams
BYTES_PER_SAMPLE = 28
# bytes per query: position in (12), direction + pdf + valid out (17)
BYTES_PER_QUERY = 29
# DRAM bytes per sample of the E-step kernel, read + write, from one ncu
# capture of a 512-region launch of the same kernel (traffic grows with the
# samples processed, so a full launch moves this times N); None for kernels
# without a capture of their current version
DRAM_BYTES_PER_SAMPLE = {"k_estep<16>": 29.10}
PREC = {"fp32": 0, "3xbf16": 1, "tf32": 2, "3xtf32": 3, "6xbf16": 4}
STATE_FIELDS = ("pi", "mu_x", "mu_w", "L", "S0", "S2", "Wbar", "n_seen", "step_j", "status")


# ---- multi-rank helpers (one process per GPU under torchrun; every rank fits
# its own regions, so the only cross-rank traffic is the timing barrier and a
# max-reduction of one number)
def rank_env():
    """(world, rank, local rank) from the torchrun environment; (1, 0, 0) without it."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(rank):
    """Seed of a rank's workload: distinct regions per rank (weak scaling)."""
    return 1 + 1000 * rank


def max_over_ranks(ms, world, device=None):
    """The slowest rank's elapsed time (all-reduce MAX, then a barrier)."""
    if world == 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units processed by all ranks per second of the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3)


def host_cores():
    """Cores this process may run on (read at runtime)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak(n_sm, peaks, src):
    mhz = peaks.get("sm_max_mhz", 2070.0)
    return (n_sm * 128 * 2 * mhz * 1e6 / 1e12,
            f"{n_sm} SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz ({src} max clock)")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU baseline legs: the FP64 oracle, as it stands, on the host cores.  These
# are the only functions here that run the oracle; their results on the
# sampled work double as the reference of the matched-error comparison.
def _or_fit_one(orc, K, rounds, extent, uni):
    """One region: the oracle's initialisation on round 0, then one stepwise
    round per batch.  Returns (initial state, final state, [loglik per
    round], seconds spent in the fit rounds)."""
    off = np.array([0, rounds[0].shape[1]], np.int64)
    cfg = orc.config(K)
    st = orc.State(1, K)
    orc.init_regions(cfg, off, rounds[0], np.array([extent]), np.array([uni]), st)
    s0 = st.copy()
    lls = []
    t0 = time.perf_counter()
    for s in rounds:
        lls.append(orc.fit_regions(cfg, np.array([0, s.shape[1]], np.int64), s, 1, st, want_loglik=True))
    return s0, st, lls, time.perf_counter() - t0


def cpu_baseline_fit(region_data, budget_s):
    """The oracle on whole regions of the batched fit, in the given (seeded)
    order until `budget_s` of single-threaded fit time, then the same regions
    again with one region per thread over every host core.  `region_data` is
    a list of (region id, [round batches (7, M_r)], extent, init uniforms)."""
    import oracle as orc
    done, t_single, used = [], 0.0, 0
    for r, rounds, ext, uni in region_data:
        s0, s1, lls, dt = _or_fit_one(orc, K_COMP, rounds, ext, uni)
        done.append((r, rounds, s0, s1, lls))
        t_single += dt
        used += 1
        if t_single > budget_s:
            break
    work = sum(ROUNDS * rounds[0].shape[1] for _, rounds, *_ in done)
    cores = host_cores()

    def refit(item):
        _, rounds, s0, _, _ = item
        st = s0.copy()
        cfg = orc.config(K_COMP)
        for s in rounds:
            orc.fit_regions(cfg, np.array([0, s.shape[1]], np.int64), s, 1, st)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(refit, sorted(done, key=lambda d: -d[1][0].shape[1])))
    t_multi = time.perf_counter() - t0
    res = {"value": work / t_single, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{used} whole regions of the workload in seeded order ({work // ROUNDS} samples per round), "
                     f"{ROUNDS} stepwise rounds each from the oracle's own initialisation, FP64, "
                     f"{t_single:.1f} s single-threaded",
           "threaded": {"value": work / t_multi, "unit": UNIT, "cores": cores,
                        "note": "one region per thread (ctypes releases the GIL), same regions and rounds"},
           "host_cores": cores}
    return res, done


def cpu_baseline_queries(params, qx, region, seed, budget_s):
    """The oracle's guided sampling (condition, draw, pdf) on the first
    queries of the workload, calibrated to about `budget_s` single-threaded,
    then over every host core in slices.  The uniforms of query i come from
    the oracle's own Philox generator with counter i and key `seed`, as the
    GPU draws them."""
    import oracle as orc
    pi, mu_x, mu_w, L = params
    uniforms = orc.uniforms(seed, min(len(region), 1 << 20))
    Qc = 2048
    t0 = time.perf_counter()
    orc.sample(K_COMP, pi, mu_x, mu_w, L, qx[:Qc], region[:Qc], uniforms[:Qc])
    per_q = (time.perf_counter() - t0) / Qc
    Qs = int(min(len(uniforms), max(Qc, budget_s / max(per_q, 1e-9))))
    t0 = time.perf_counter()
    out = orc.sample(K_COMP, pi, mu_x, mu_w, L, qx[:Qs], region[:Qs], uniforms[:Qs])
    t_single = time.perf_counter() - t0
    cores = host_cores()
    sl = np.array_split(np.arange(Qs), cores)

    def part(ix):
        orc.sample(K_COMP, pi, mu_x, mu_w, L, qx[ix], region[ix], uniforms[ix])

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(part, sl))
    t_multi = time.perf_counter() - t0
    res = {"value": Qs / t_single, "unit": "queries/s", "cores": 1, "kind": "oracle",
           "sample": f"the first {Qs} queries of the workload (condition + draw + pdf), FP64, "
                     f"{t_single:.1f} s single-threaded",
           "threaded": {"value": Qs / t_multi, "unit": "queries/s", "cores": cores}}
    return res, out, Qs


def cpu_baseline_pdf(params, qx, region, dirs):
    """The oracle's pdf at given directions (re-evaluation of GPU samples)."""
    import oracle as orc
    return orc.pdf(K_COMP, *params, qx, region, dirs)


def cpu_baseline_steps(K, offsets, samples, extent, uni, steps, cfg_kw=None, objective=False):
    """The oracle on a few regions: own initialisation, then `steps` EM steps
    (with `cfg_kw`); returns (initial state, final state, loglik of the last
    step, seconds of the steps) and, for `objective`, the objective and its
    gradient at the final state."""
    import oracle as orc
    cfg = orc.config(K, **(cfg_kw or {}))
    st = orc.State(len(offsets) - 1, K)
    orc.init_regions(orc.config(K), offsets, samples, extent, uni, st)
    s0 = st.copy()
    t0 = time.perf_counter()
    ll = orc.fit_regions(cfg, offsets, samples, steps, st, want_loglik=True)
    dt = time.perf_counter() - t0
    obj = None
    if objective:
        t1 = time.perf_counter()
        obj = orc.objective(orc.config(K), offsets, samples, st)
        obj = obj + (time.perf_counter() - t1,)
    return s0, st, ll, dt, obj


def run_reference(args):
    """The oracle alone on the fit workload: each step a bounded sample of
    whole regions (init + four stepwise rounds), over every host core."""
    _, rank, _ = rank_env()
    if rank != 0:                            # the oracle runs once, on rank 0
        return None
    import oracle as orc
    from paper_2111_13094_gb300 import synthetic as syn
    R = args.regions
    seed = rank_seed(0)
    counts = syn.region_counts(seed, R)
    truth = syn.batched_truth(seed, R, K=K_COMP)
    _, h, _ = syn.region_grid(R)
    uni = syn.init_uniforms(seed, R, 2)
    cores = host_cores()
    order = np.random.default_rng(seed).permutation(R)
    per_step = max(0.5, 60.0 / max(1, args.steps + args.warmup))

    def region_rounds(r, step):
        sub = syn.GroundTruth(truth.pi[r:r + 1], truth.mu_x[r:r + 1], truth.mu_w[r:r + 1],
                              truth.e1[r:r + 1], truth.e2[r:r + 1], truth.cov[r:r + 1])
        return [syn.draw(np.random.default_rng([seed, 7, int(r), step, j]), sub, [counts[r]])
                for j in range(ROUNDS)]


    def fit(item):
        r, rounds = item
        return _or_fit_one(orc, K_COMP, rounds, h[r], uni[r])[3]

    # the regions of one step, drawn once on the host (seeded order, about
    # per_step seconds of fitting over all cores); every step fits them again
    items, est = [], 0.0
    while est < per_step * cores and len(items) < R:
        r = int(order[len(items)])
        items.append((r, region_rounds(r, 0)))
        est += ROUNDS * counts[r] / 6.0e5
    step_work = sum(ROUNDS * counts[r] for r, _ in items)

    def one_step():
        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=cores) as ex:
            list(ex.map(fit, sorted(items, key=lambda it: -counts[it[0]])))
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        one_step()
    secs = sum(one_step() for _ in range(args.steps))
    work, regions = step_work * args.steps, len(items)
    v = work / secs
    N = int(counts.sum())
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": fit_config(R, N),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{regions} whole regions per step ({step_work // ROUNDS} samples per "
                                       f"round), init + {ROUNDS} stepwise rounds per region, FP64, one region "
                                       f"per thread on {cores} host cores"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fit_config(R_REGIONS, N):
    """The workload both arms report."""
    return {"workload": f"batched stepwise MAP-EM fit: {R_REGIONS} regions x K=16, sample counts "
                        "log-uniform in [256, 65536], 4 Robbins-Monro rounds per step with a "
                        "fresh batch each, starting from the regions' initial state, CUDA-graph "
                        "replay per round",
            "regions": R_REGIONS, "K": K_COMP, "rounds_per_step": ROUNDS,
            "samples_per_round": N, "per_rank": True,
            "l2": "inputs larger than L2 (about 1.38 GB per round)"}


# --------------------------------------------------------------------------
# GPU legs
def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _timed(fn, stream, reps=10, warm=3):
    import torch
    e0, e1 = _events()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _block_err(g, o):
    """max over components of max|g - o| / max(|o|) within the component."""
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    scale = np.maximum(np.abs(o).max(axis=-1, keepdims=True), 1e-12)
    e = (np.abs(g - o) / scale).max(axis=-1)
    return float(e.max()) if e.size else 0.0


def _param_errors(g, o):
    """Parameter errors of GPU arrays g against oracle arrays o (dicts with
    pi (S, K), mu_x (S, K, 3), mu_w (S, K, 3), L (S, K, 15), status (S,)),
    over every region, whatever its status."""
    span = np.maximum(np.ptp(o["mu_x"], axis=1).max(axis=1), 1e-3)
    return {"pi": float(np.abs(g["pi"] - o["pi"]).max() / max(o["pi"].max(), 1e-12)),
            "mu_x": float((np.abs(g["mu_x"] - o["mu_x"]).max(axis=(1, 2)) / span).max()),
            "mu_w": float(np.abs(g["mu_w"] - o["mu_w"]).max()),
            "L": _block_err(g["L"], o["L"]),
            "status_match": bool(np.array_equal(g["status"], o["status"])),
            "repaired_gpu": int(np.sum(g["status"] == 7)), "repaired_oracle": int(np.sum(o["status"] == 7))}


def _ll_err(g, o):
    e = np.abs(np.asarray(g, np.float64) - o) / np.maximum(1.0, np.abs(o))
    return float(e.max()) if e.size else 0.0, float(np.median(e)) if e.size else 0.0


def _to_gpu_state(api, torch, K, o, dev, cfg):
    st = api.MixtureState(o.R, K, device=dev)
    for f in STATE_FIELDS:
        getattr(st, f).copy_(torch.from_numpy(getattr(o, f)))
    api.prepare(cfg, st)
    return st


def _state_arrays(st):
    return {f: getattr(st, f).cpu().numpy() for f in ("pi", "mu_x", "mu_w", "L", "status")}


def fit_accuracy(api, torch, dev, done, forms):
    """Every GPU form on the sampled regions, from the oracle's initial state
    over the same four rounds (work units of CHUNK samples, as in the timed
    run): per-sample log-likelihood errors over all rounds, parameter errors
    and statuses after the last round, against the oracle's results."""
    S = len(done)
    counts = [[d[1][j].shape[1] for d in done] for j in range(ROUNDS)]
    batches = []
    for j in range(ROUNDS):
        s = np.concatenate([d[1][j] for d in done], axis=1)
        off = np.concatenate([[0], np.cumsum(counts[j])]).astype(np.int64)
        batches.append(api.SampleBatch(torch.from_numpy(np.ascontiguousarray(s)).to(dev),
                                       torch.from_numpy(off).to(dev)))
    o_init = _stack_states([d[2] for d in done])
    o_final = {f: np.concatenate([getattr(d[3], f) for d in done]) for f in ("pi", "mu_x", "mu_w", "L", "status")}
    ll_o = [np.concatenate([d[4][j] for d in done]) for j in range(ROUNDS)]
    out = {}
    for name in forms:
        cfg = api.config(K_COMP, precision=PREC[name], chunk=CHUNK)
        st = _to_gpu_state(api, torch, K_COMP, o_init, dev, cfg)
        ws = api.workspace(cfg, S, max(b.N for b in batches), device=dev)
        errs = []
        for j, b in enumerate(batches):
            ll = torch.empty(b.N, dtype=torch.float32, device=dev)
            api.fit_regions(cfg, b, 1, st, ws, loglik=ll)
            errs.append(np.abs(ll.cpu().numpy().astype(np.float64) - ll_o[j]) / np.maximum(1.0, np.abs(ll_o[j])))
        e = np.concatenate(errs)
        out[name] = {"loglik_max": float(e.max()), "loglik_median": float(np.median(e)),
                     "loglik_p999": float(np.quantile(e, 0.999)),
                     **_param_errors(_state_arrays(st), o_final)}
        del st, ws
    out["regions"] = S
    out["rounds"] = ROUNDS
    out["note"] = ("GPU forms from the oracle's initial state on the sampled regions, same four rounds, "
                   "work units of 4096 samples; log-likelihood error relative with floor 1 over every "
                   "sample of every round; parameters over every region after the last round")
    return out


class _StateStack:
    pass


def _stack_states(states):
    s = _StateStack()
    s.R = sum(x.R for x in states)
    for f in STATE_FIELDS:
        setattr(s, f, np.ascontiguousarray(np.concatenate([getattr(x, f) for x in states])))
    return s


def measure_e2e(args, batches, off, st, snap, plan, stream, world, N):
    """Same step through the public API with host buffers: each round's batch
    goes from pinned host memory through the plan's host entry point (its
    copy into a staging slot overlaps the previous round's replay), and the
    fitted parameters are read back.  Beside it, the ceiling: a plain pinned
    host-to-device copy of the same bytes on one stream."""
    import torch

    from paper_2111_13094_gb300 import api
    host_off = off.cpu().pin_memory()
    host = [api.SampleBatch(b.samples.cpu().pin_memory(), host_off) for b in batches]
    staging = torch.empty(plan.staging_bytes(), dtype=torch.uint8, device=off.device)
    params = (st.pi, st.mu_x, st.mu_w, st.L)
    out_host = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in params]

    def e2e_step():
        for f in STATE_FIELDS + ("etab", "qtab"):
            getattr(st, f).copy_(snap[f], non_blocking=True)
        for hb in host:
            plan.run_host(hb, staging)
        for o, t in zip(out_host, params):
            o.copy_(t, non_blocking=True)

    n = max(2, args.steps // 10)
    h2d = sum(hb.samples.numel() * hb.samples.element_size() + host_off.numel() * 8 for hb in host)
    d2h = sum(o.numel() * o.element_size() for o in out_host)
    # ceiling: the same host bytes copied to the device, nothing else; the
    # faster of one copy per batch and one copy per sample stream (the plan's
    # pattern), both on a side stream.  The host link is shared with the other
    # GPUs of the machine, so the end-to-end steps and the copies are timed in
    # alternation (each a mean over the same n rounds of the alternation).
    dst = [torch.empty_like(b.samples) for b in batches]
    side = torch.cuda.Stream()

    def copy_whole():
        with torch.cuda.stream(side):
            for d, hb in zip(dst, host):
                d.copy_(hb.samples, non_blocking=True)

    def copy_rows():
        with torch.cuda.stream(side):
            for d, hb in zip(dst, host):
                for q in range(7):
                    d[q].copy_(hb.samples[q], non_blocking=True)

    e2e_step()
    copy_whole()
    copy_rows()
    torch.cuda.synchronize()
    t_e2e, t_whole, t_rows = [], [], []
    for _ in range(n):
        t_e2e.append(_timed(e2e_step, stream, reps=1, warm=0))
        t_whole.append(_timed(copy_whole, side, reps=1, warm=0))
        t_rows.append(_timed(copy_rows, side, reps=1, warm=0))
    ms = float(np.mean(t_e2e))
    c_ms = min(float(np.mean(t_whole)), float(np.mean(t_rows)))
    copy_gbs = h2d / (c_ms * 1e-3) / 1e9
    e2e_gbs = h2d / (ms * 1e-3) / 1e9
    del staging, dst
    return {"value": world * ROUNDS * N / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": ms,
            "path": "sdmm_fit_plan_run_host: pinned host batch -> staging slot (copy stream) -> graph replay",
            "h2d_gbs": e2e_gbs,
            "ceiling": {"pinned_h2d_copy_gbs": copy_gbs, "copy_ms_per_step": c_ms,
                        "frac": e2e_gbs / copy_gbs,
                        "note": "plain pinned host-to-device copies of the step's four batches on a side "
                                "stream (the faster of one copy per batch and one per sample stream), "
                                "timed in alternation with the end-to-end steps"}}


def query_leg(args, api, torch, dev, stream, seed, world, cfg, peaks, src, n_sm, want_cpu):
    """16M guided queries over 65,536 grid regions: as given (grid lookup) and
    pre-sorted by region; roofline; oracle baseline and pdf errors on the
    first queries; product sampling with 3 BSDF lobes."""
    Q = args.queries
    Rq = int(np.prod(Q_DIMS))
    pi, mu_x, mu_w, L = syn_random_mixtures(seed)
    qst = api.MixtureState(Rq, K_COMP, device=dev)
    qst.set_params(torch.from_numpy(pi), torch.from_numpy(mu_x), torch.from_numpy(mu_w), torch.from_numpy(L))
    api.prepare(cfg, qst)
    from paper_2111_13094_gb300 import synthetic as syn
    qx_h = syn.query_points(seed, Q)
    qx = torch.from_numpy(qx_h).to(dev)
    grid = api.Grid((0, 0, 0), (1, 1, 1), Q_DIMS)
    out = (torch.empty(Q, 3, device=dev), torch.empty(Q, device=dev),
           torch.empty(Q, dtype=torch.uint8, device=dev))
    reg_h = syn.grid_region(qx_h, Q_DIMS)
    reg = torch.from_numpy(reg_h).to(dev)
    order = torch.argsort(reg)
    qx_b, reg_b = qx[order].contiguous(), reg[order].contiguous()
    qws = api.query_workspace(Rq, Q, device=dev)
    t_lib = _timed(lambda: api.sample(cfg, qst, qx, grid=grid, seed=7, out=out, ws=qws), stream)
    t_grid = _timed(lambda: api.sample(cfg, qst, qx, grid=grid, seed=7, out=out), stream)
    t_bin = _timed(lambda: api.sample(cfg, qst, qx_b, region=reg_b, seed=7, out=out), stream)
    api.sample(cfg, qst, qx, grid=grid, seed=7, out=out)
    torch.cuda.synchronize()
    disc = 1.0 - out[2].float().mean().item()
    peak, basis = fp32_peak(n_sm, peaks, src)
    flops = Q * (K_COMP * FLOPS_PER_QUERY_COMPONENT + FLOPS_PER_QUERY)

    def roof(ms):
        a = flops / (ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                "traffic": None, "kernel_ms": ms, "peak_basis": basis,
                "flops_per_query": K_COMP * FLOPS_PER_QUERY_COMPONENT + FLOPS_PER_QUERY,
                "hbm_gbs": Q * BYTES_PER_QUERY / (ms * 1e-3) / 1e9}

    qres = {"value": world * Q / (t_lib * 1e-3), "unit": "queries/s", "ms": t_lib,
            "path": "sdmm_sample_binned: queries as given (uniform positions), grid lookup, binned by region "
                    "in the library's workspace (counting sort), then one thread per query",
            "unbinned_value": world * Q / (t_grid * 1e-3), "unbinned_ms": t_grid,
            "presorted_value": world * Q / (t_bin * 1e-3), "presorted_ms": t_bin,
            "queries": Q, "regions": Rq, "K": K_COMP,
            "discard_rate": disc, "roofline": roof(t_lib), "presorted_roofline": roof(t_bin),
            "config": f"{Q} positions uniform in the unit cube, 64x32x32 grid regions, "
                      "condition + Philox draw + sample + pdf, FP32"}
    if want_cpu:
        cpu, o, Qs = cpu_baseline_queries((pi, mu_x, mu_w, L), qx_h, reg_h, 7, args.cpu_budget / 3)
        d = out[0][:Qs].cpu().numpy().astype(np.float64)
        p = out[1][:Qs].cpu().numpy().astype(np.float64)
        v = out[2][:Qs].cpu().numpy()
        # the oracle's pdf at the GPU's own FP32 direction
        p_o = cpu_baseline_pdf((pi, mu_x, mu_w, L), qx_h[:Qs], reg_h[:Qs], d)
        ok = (v == 1) & (p_o > 0)
        e = np.abs(p[ok] - p_o[ok]) / p_o[ok]
        margin_ok = o["margin"] > 1e-5
        dv = (v == o["valid"])
        cosang = np.clip(np.sum(d * o["dir"], axis=1), -1, 1)
        ang = np.arccos(cosang)[margin_ok & (o["valid"] == 1) & (v == 1)]
        qres["cpu_baseline"] = cpu
        qres["accuracy"] = {"queries": Qs, "pdf_rel_max": float(e.max()) if e.size else 0.0,
                            "pdf_rel_median": float(np.median(e)) if e.size else 0.0,
                            "pdf_rel_p999": float(np.quantile(e, 0.999)) if e.size else 0.0,
                            "valid_agree": float(dv.mean()),
                            "direction_rad_max_outside_margin": float(ang.max()) if ang.size else 0.0,
                            "direction_rad_p999_outside_margin": float(np.quantile(ang, 0.999)) if ang.size else 0.0,
                            "note": "pdf: GPU value against the oracle's pdf at the GPU's FP32 direction; "
                                    "directions against the oracle's sample where its component choice "
                                    "is more than 1e-5 from a CDF boundary"}
    bw, bmu, bL = (torch.from_numpy(a).to(dev) for a in syn.bsdf_lobes(seed, Q, 3))
    t_prod = _timed(lambda: api.product_sample(cfg, qst, qx, bw, bmu, bL, grid=grid, seed=7), stream)
    bw_b, bmu_b, bL_b = bw[order].contiguous(), bmu[order].contiguous(), bL[order].contiguous()
    t_prod_b = _timed(lambda: api.product_sample(cfg, qst, qx_b, bw_b, bmu_b, bL_b, region=reg_b, seed=7), stream)
    qres["product"] = {"value": world * Q / (t_prod * 1e-3), "unit": "queries/s", "kernel_ms": t_prod,
                       "presorted_value": world * Q / (t_prod_b * 1e-3), "presorted_kernel_ms": t_prod_b,
                       "config": f"the same {Q} queries, 3 BSDF lobes each (wide, narrow, random), "
                                 "2K pairs per query: condition + pair products + sample + product pdf, FP32; "
                                 "presorted: the queries ordered by region beforehand"}
    del bw, bmu, bL, bw_b, bmu_b, bL_b, qst, out, qws
    return qres


def syn_random_mixtures(seed):
    from paper_2111_13094_gb300 import synthetic as syn
    return syn.random_mixtures(seed, Q_DIMS, K_COMP)


def kdtree_leg(api, torch, dev, batch, N, peaks):
    tree = api.KdTree(1 << 20, 1 << 19, device=dev)
    raw = batch.samples
    times = []
    for _ in range(3):
        tree.grid(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        kb = tree.bin(raw)
        t1 = time.perf_counter()
        kr, kp = tree.refine(kb, c=16000)
        t2 = time.perf_counter()
        times.append((t1 - t0, t2 - t1))
    tb = float(np.median([a for a, _ in times])) * 1e3
    tr = float(np.median([b for _, b in times])) * 1e3
    # binning moves at least every sample's 7 streams once: 28 B read + 28 B written
    bin_gbs = 56.0 * N / (tb * 1e-3) / 1e9
    hbm = peaks.get("hbm_gbs", 6800.0)
    res = {"samples": N, "bin_ms": tb, "refine_ms": tr, "leaves_after": tree.n_leaves,
           "nodes_after": tree.n_nodes, "c": 16000,
           "bin_samples_per_s": N / (tb * 1e-3), "refine_samples_per_s": N / (tr * 1e-3),
           "bin_roofline": {"bound": "hbm", "achieved": bin_gbs, "peak": hbm, "unit": "GB/s",
                            "frac": bin_gbs / hbm, "bytes_per_sample": 56.0},
           "note": "host wall time of the synchronous calls (binning: leaf lookup, one stable counting "
                   "pass by leaf that moves the streams (up to 1024 leaves); refinement: rounds of stable "
                   "partitions, one 4-byte read-back per tree level)"}
    del tree, kb, kr, kp
    return res


# ---- the other workloads (each with its own oracle sample and errors)
def config_single_region(api, torch, dev, stream, want_cpu, seed=0, N=65536, K=16, iters=20):
    """Single region, N = 65,536, K = 16, 20 plain EM iterations (eta = 1)."""
    from paper_2111_13094_gb300 import synthetic as syn
    b = syn.single_region(seed, N, K)
    gcfg = api.config(K, eta_mode=1)
    batch = api.SampleBatch(torch.from_numpy(np.ascontiguousarray(b.samples)).to(dev),
                            torch.from_numpy(b.offsets).to(dev))
    ws = api.workspace(gcfg, 1, N, device=dev)
    res = {"config": "single region, N = 65,536, K = 16, 20 EM iterations (eta = 1), FP32"}
    uni = syn.init_uniforms(seed, 1, K // 8)
    if want_cpu:
        s0, s1, ll_o, dt, _ = cpu_baseline_steps(K, b.offsets, b.samples, b.extent, uni, iters,
                                                 cfg_kw={"eta_mode": 1})
        st = _to_gpu_state(api, torch, K, s0, dev, gcfg)
        snap = {f: getattr(st, f).clone() for f in STATE_FIELDS + ("etab", "qtab")}
        ll = torch.empty(N, dtype=torch.float32, device=dev)
        api.fit_regions(gcfg, batch, iters, st, ws, loglik=ll)
        torch.cuda.synchronize()
        m, med = _ll_err(ll.cpu().numpy(), ll_o)
        res["accuracy"] = {"loglik_max": m, "loglik_median": med,
                           **_param_errors(_state_arrays(st), {f: getattr(s1, f) for f in
                                                               ("pi", "mu_x", "mu_w", "L", "status")})}
        res["cpu_baseline"] = {"value": N * iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"the whole workload, {dt:.2f} s"}
    else:
        st = api.MixtureState(1, K, device=dev)
        api.init_regions(gcfg, batch, torch.from_numpy(np.asarray(b.extent, np.float64)).to(dev),
                         torch.from_numpy(uni).to(dev), st)
        snap = {f: getattr(st, f).clone() for f in STATE_FIELDS + ("etab", "qtab")}
    e0, e1 = _events()
    times = []
    for rep in range(8):
        for f, v in snap.items():
            getattr(st, f).copy_(v)
        torch.cuda.synchronize()
        e0.record(stream)
        api.fit_regions(gcfg, batch, iters, st, ws)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep >= 2:
            times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    res.update({"gpu_ms": ms, "value": N * iters / (ms * 1e-3), "unit": UNIT,
                "note": "one region fills few SMs: latency-bound"})
    return res


def config_precision_sweep(api, torch, dev, stream, want_cpu, R=1024, per=65536, Ks=(16, 32),
                           forms=("fp32", "6xbf16", "3xtf32", "3xbf16", "tf32"), check=4, reps=10, seed=11):
    """1,024 regions x 65,536 samples, K = 16 and 32: one EM round per form
    (graph replay) and its error after one step on `check` seeded regions."""
    from paper_2111_13094_gb300 import synthetic as syn
    rows = []
    for K in Ks:
        truth = syn.batched_truth(seed + K, R, K=K)
        counts = np.full(R, per, dtype=np.int64)
        N = int(counts.sum())
        offsets = syn.offsets_from_counts(counts)
        samples = syn.draw_torch(seed + K, truth, counts, device=dev)
        batch = api.SampleBatch(samples, torch.from_numpy(offsets).to(dev))
        _, h, _ = syn.region_grid(R)
        n_pos = K // 8
        uni = syn.init_uniforms(seed, R, n_pos)
        regions = np.sort(np.random.default_rng([seed, K, 7]).choice(R, size=min(check, R), replace=False))
        o = None
        if want_cpu:
            sub = np.concatenate([samples[:, offsets[r]:offsets[r + 1]].cpu().numpy() for r in regions], axis=1)
            sub_off = syn.offsets_from_counts(counts[regions])
            o = cpu_baseline_steps(K, sub_off, sub, h[regions], uni[regions], 1)
            sel = torch.from_numpy(np.concatenate([np.arange(offsets[r], offsets[r + 1]) for r in regions])).to(dev)
        for form in forms:
            cfg = api.config(K, precision=PREC[form])
            st = api.MixtureState(R, K, device=dev)
            api.init_regions(cfg, batch, torch.from_numpy(h.astype(np.float64)).to(dev),
                             torch.from_numpy(uni).to(dev), st)
            row = {"K": K, "form": form}
            ws = api.workspace(cfg, R, N, device=dev)
            if o is not None:
                s0, s1, ll_o, dt, _ = o
                idx = torch.from_numpy(regions).to(dev)
                for f in STATE_FIELDS:
                    getattr(st, f)[idx] = torch.from_numpy(getattr(s0, f)).to(dev)
                api.prepare(cfg, st)
                ll = torch.empty(N, dtype=torch.float32, device=dev)
                snap = {f: getattr(st, f).clone() for f in STATE_FIELDS + ("etab", "qtab")}
                api.fit_regions(cfg, batch, 1, st, ws, loglik=ll)
                torch.cuda.synchronize()
                m, med = _ll_err(ll[sel].cpu().numpy(), ll_o)
                g = {f: getattr(st, f)[idx].cpu().numpy() for f in ("pi", "mu_x", "mu_w", "L", "status")}
                row.update({"loglik_max": m, "loglik_median": med,
                            **_param_errors(g, {f: getattr(s1, f) for f in ("pi", "mu_x", "mu_w", "L", "status")})})
                row["oracle_s"] = dt
                for f, v in snap.items():
                    getattr(st, f).copy_(v)
            plan = api.FitPlan(cfg, R, N, 1, st, ws)
            for _ in range(3):
                plan.run(batch)
            plan.enable_timing(reps)
            ms = _timed(lambda: plan.run(batch), stream, reps=reps, warm=0)
            kern = plan.timing()
            row.update({"round_ms": ms, "estep_ms": float(np.mean(kern)) if len(kern) else None,
                        "value": N / (ms * 1e-3), "unit": UNIT})
            rows.append(row)
            plan.close()
            del plan, ws, st
            torch.cuda.empty_cache()
        del samples, batch
        torch.cuda.empty_cache()
    for K in Ks:
        base = [r for r in rows if r["K"] == K and r["form"] == "fp32"][0]
        for r in rows:
            if r["K"] == K:
                r["vs_fp32"] = base["round_ms"] / r["round_ms"]
    return {"config": f"precision sweep: {R} regions x {per} samples, K in {list(Ks)}, one EM round per "
                      f"graph replay; errors after one EM step on {check} seeded regions against the oracle",
            "rows": rows}


def config_objective(api, torch, dev, stream, want_cpu, seed=30, R=1024, M=16384, K=16, check=3, reps=10):
    """MAP objective and its adjoint, 1,024 regions x 16,384 samples, K = 16."""
    from paper_2111_13094_gb300 import synthetic as syn
    truth = syn.batched_truth(seed, R, K=K, parallax=True)
    counts = np.full(R, M, dtype=np.int64)
    N = R * M
    offsets = syn.offsets_from_counts(counts)
    samples = syn.draw_torch(seed, truth, counts, device=dev)
    batch = api.SampleBatch(samples, torch.from_numpy(offsets).to(dev))
    _, h, _ = syn.region_grid(R)
    gcfg = api.config(K)
    st = api.MixtureState(R, K, device=dev)
    uni = syn.init_uniforms(seed, R, K // 8)
    api.init_regions(gcfg, batch, torch.from_numpy(h.astype(np.float64)).to(dev), torch.from_numpy(uni).to(dev), st)
    ws = api.workspace(gcfg, R, N, device=dev)
    api.fit_regions(gcfg, batch, 3, st, ws)
    res = {"config": f"objective + adjoint, {R} regions x {M} samples, K = {K}"}
    dF = torch.ones(R, dtype=torch.float64, device=dev)
    if want_cpu:
        regions = np.sort(np.random.default_rng([seed, 9]).choice(R, size=check, replace=False))
        sub = np.concatenate([samples[:, offsets[r]:offsets[r + 1]].cpu().numpy() for r in regions], axis=1)
        sub_off = syn.offsets_from_counts(counts[regions])
        _, o, _, _, obj = cpu_baseline_steps(K, sub_off, sub, h[regions], uni[regions], 3, objective=True)
        F_o, gd_o, gL_o, ga_o, t_or = obj
        idx = torch.from_numpy(regions).to(dev)
        for f in STATE_FIELDS:
            getattr(st, f)[idx] = torch.from_numpy(getattr(o, f)).to(dev)
        api.prepare(gcfg, st)
        F = api.objective(gcfg, batch, st, ws)
        gd, gL, ga = api.objective_backward(gcfg, batch, st, dF, ws)
        torch.cuda.synchronize()

        def rel(g, ref):
            return float(np.abs(g - ref).max() / max(np.abs(ref).max(), 1e-30))

        Fg = F.cpu().numpy()[regions]
        res["accuracy"] = {"F": float(np.abs(Fg - F_o).max() / max(1.0, np.abs(F_o).max())),
                           "g_delta": rel(gd.cpu().numpy()[regions], gd_o), "g_L": rel(gL.cpu().numpy()[regions], gL_o),
                           "g_logit": rel(ga.cpu().numpy()[regions], ga_o), "regions": check}
        res["cpu_baseline"] = {"value": check * M / t_or, "unit": "samples/s (objective + gradient)", "cores": 1,
                               "kind": "oracle", "sample": f"{check} regions, {t_or:.2f} s"}
    f_ms = _timed(lambda: api.objective(gcfg, batch, st, ws), stream, reps=reps)
    b_ms = _timed(lambda: api.objective_backward(gcfg, batch, st, dF, ws), stream, reps=reps)
    res.update({"forward_ms": f_ms, "backward_ms": b_ms, "samples_per_s_forward": N / (f_ms * 1e-3),
                "samples_per_s_backward": N / (b_ms * 1e-3)})
    del samples, batch, ws, st
    torch.cuda.empty_cache()
    return res


def config_ablations(api, torch, dev, stream, want_cpu, R=1024, M=16384, K=16, reps=10):
    """Covariance update (first-order vs two-pass), E-step density (chart vs
    solid angle) and directions (tangent vs Euclidean): E-step or step times
    and, for the covariance update, the error against the oracle's two-pass
    update on three regions."""
    from paper_2111_13094_gb300 import synthetic as syn
    out = {}
    # covariance update, plain EM, 3 steps
    seed, steps, check = 40, 3, 3
    truth = syn.batched_truth(seed, R, K=K, parallax=True)
    counts = np.full(R, M, dtype=np.int64)
    N = R * M
    offsets = syn.offsets_from_counts(counts)
    samples = syn.draw_torch(seed, truth, counts, device=dev)
    batch = api.SampleBatch(samples, torch.from_numpy(offsets).to(dev))
    _, h, _ = syn.region_grid(R)
    uni = syn.init_uniforms(seed, R, K // 8)
    regions = np.sort(np.random.default_rng([seed, 9]).choice(R, size=check, replace=False))
    ref = None
    if want_cpu:
        sub = np.concatenate([samples[:, offsets[r]:offsets[r + 1]].cpu().numpy() for r in regions], axis=1)
        sub_off = syn.offsets_from_counts(counts[regions])
        o0, ref, _, _, _ = cpu_baseline_steps(K, sub_off, sub, h[regions], uni[regions], steps,
                                              cfg_kw={"eta_mode": 1, "cov_update": 1})
    cov = {"config": f"covariance update, {R} regions x {M} samples, K = {K}, plain EM, {steps} steps"}
    for name, mode in (("first_order", 0), ("two_pass", 1)):
        cfg = api.config(K, eta_mode=1, cov_update=mode)
        st = api.MixtureState(R, K, device=dev)
        api.init_regions(cfg, batch, torch.from_numpy(h.astype(np.float64)).to(dev), torch.from_numpy(uni).to(dev), st)
        idx = torch.from_numpy(regions).to(dev)
        if ref is not None:
            for f in STATE_FIELDS:
                getattr(st, f)[idx] = torch.from_numpy(getattr(o0, f)).to(dev)
            api.prepare(cfg, st)
        ws = api.workspace(cfg, R, N, device=dev)
        snap = {f: getattr(st, f).clone() for f in STATE_FIELDS + ("etab", "qtab")}
        api.fit_regions(cfg, batch, steps, st, ws)
        torch.cuda.synchronize()
        row = {}
        if ref is not None:
            row["L_error_vs_two_pass_oracle"] = _block_err(st.L[idx].cpu().numpy(), ref.L)

        def one():
            for f, v in snap.items():
                getattr(st, f).copy_(v)
            api.fit_regions(cfg, batch, 1, st, ws)

        row["step_ms"] = _timed(one, stream, reps=5)
        cov[name] = row
        del st, ws
    cov["time_ratio"] = cov["two_pass"]["step_ms"] / cov["first_order"]["step_ms"]
    out["covariance_update"] = cov
    del samples, batch
    # E-step density and directions: E-step kernel time from the plan's events
    for key, seed, MM, variants in (
            ("estep_density", 50, M, (("chart", {}), ("solid_angle", {"estep_density": 1}),
                                      ("6xbf16_chart", {"precision": 4}),
                                      ("6xbf16_solid_angle", {"precision": 4, "estep_density": 1}))),
            ("directions", 80, 65536, (("fp32_tangent", {}), ("fp32_euclidean", {"dir_coords": 1}),
                                       ("6xbf16_tangent", {"precision": 4}),
                                       ("6xbf16_euclidean", {"precision": 4, "dir_coords": 1})))):
        truth = syn.batched_truth(seed, R, K=K)
        counts = np.full(R, MM, dtype=np.int64)
        NN = R * MM
        samples = syn.draw_torch(seed, truth, counts, device=dev)
        batch = api.SampleBatch(samples, torch.from_numpy(syn.offsets_from_counts(counts)).to(dev))
        _, h, _ = syn.region_grid(R)
        res = {"config": f"E-step, {R} regions x {MM} samples, K = {K}"}
        for name, kw in variants:
            cfg = api.config(K, **kw)
            st = api.MixtureState(R, K, device=dev)
            api.init_regions(cfg, batch, torch.from_numpy(h.astype(np.float64)).to(dev),
                             torch.from_numpy(syn.init_uniforms(seed, R, K // 8)).to(dev), st)
            ws = api.workspace(cfg, R, NN, device=dev)
            plan = api.FitPlan(cfg, R, NN, 1, st, ws)
            for _ in range(3):
                plan.run(batch)
            plan.enable_timing(reps)
            for _ in range(reps):
                plan.run(batch)
            torch.cuda.synchronize()
            res[f"{name}_estep_ms"] = float(np.mean(plan.timing()))
            plan.close()
            del plan, ws, st
        out[key] = res
        del samples, batch
        torch.cuda.empty_cache()
    d = out["estep_density"]
    d["ratio"] = d["solid_angle_estep_ms"] / d["chart_estep_ms"]
    d["6xbf16_ratio"] = d["6xbf16_solid_angle_estep_ms"] / d["6xbf16_chart_estep_ms"]
    e = out["directions"]
    e["fp32_ratio"] = e["fp32_tangent_estep_ms"] / e["fp32_euclidean_estep_ms"]
    e["6xbf16_ratio"] = e["6xbf16_tangent_estep_ms"] / e["6xbf16_euclidean_estep_ms"]
    return out


def config_batching(api, torch, dev, stream, seed=0, R=512, K=16, reps=5):
    """The batched form against plain per-region fitting (the paper fits each
    kD-tree leaf on its own): one stepwise round of R regions of the batched
    workload's recipe, as one sdmm_fit_regions call (persistent work queue over
    all regions) and as R calls of one region each, on the same work units
    (chunk fixed), so both compute the same FP32 sums: the parameters must
    agree bit for bit, i.e. at equal log-likelihood error."""
    import ctypes

    from paper_2111_13094_gb300 import _lib
    from paper_2111_13094_gb300 import synthetic as syn
    lib = _lib.load()
    truth = syn.batched_truth(seed + 5, R, K=K)
    counts = syn.region_counts(seed + 5, R)
    b = syn.batched_round(seed + 5, R, counts, 0, truth)
    cfg = api.config(K, chunk=CHUNK)
    batch = api.SampleBatch(torch.from_numpy(np.ascontiguousarray(b.samples)).to(dev),
                            torch.from_numpy(b.offsets).to(dev))
    st = api.MixtureState(R, K, device=dev)
    api.init_regions(cfg, batch, torch.from_numpy(np.asarray(b.extent, np.float64)).to(dev),
                     torch.from_numpy(syn.init_uniforms(seed + 5, R, K // 8)).to(dev), st)
    snap = {f: getattr(st, f).clone() for f in STATE_FIELDS + ("etab", "qtab")}
    ws = api.workspace(cfg, R, b.N, device=dev)
    Mmax = int(np.max(counts))
    ws1 = api.workspace(cfg, 1, Mmax, device=dev)
    one_off = [torch.tensor([0, int(m)], dtype=torch.int64, device=dev) for m in counts]
    s = batch.samples
    row = s.stride(0) * s.element_size()
    off = b.offsets

    def region_state(r):
        ptrs = []
        for f in api.MixtureState.FIELDS:
            t = getattr(st, f)
            ptrs.append(t.data_ptr() + r * (t.numel() // R) * t.element_size())
        return _lib.State(*ptrs)

    def batched():
        api.fit_regions(cfg, batch, 1, st, ws, stream=stream)

    sm = [_lib.Samples(*[s.data_ptr() + q * row + int(off[r]) * s.element_size() for q in range(7)],
                       one_off[r].data_ptr(), 1, int(counts[r])) for r in range(R)]
    sts = [region_state(r) for r in range(R)]
    hs = ctypes.c_void_p(stream.cuda_stream)

    def per_region():
        for r in range(R):
            _lib.check(lib.sdmm_fit_regions(ctypes.byref(cfg), ctypes.byref(sm[r]), 1, None, ctypes.byref(sts[r]),
                                            None, ctypes.c_void_p(ws1.data_ptr()), ws1.numel(), hs),
                       "sdmm_fit_regions")

    def restore():
        for f, v in snap.items():
            getattr(st, f).copy_(v)

    res = {"config": f"one stepwise round of {R} regions (counts log-uniform in [256, 65536], "
                     f"{int(counts.sum())} samples), K = {K}, work units of {CHUNK} samples in both forms"}
    out = {}
    for name, fn in (("batched", batched), ("per_region", per_region)):
        times = []
        for rep in range(reps + 1):
            restore()
            torch.cuda.synchronize()
            e0, e1 = _events()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                times.append(e0.elapsed_time(e1))
        res[f"{name}_ms"] = float(np.mean(times))
        out[name] = {f: getattr(st, f).clone() for f in ("pi", "mu_x", "mu_w", "L", "status")}
    res["speedup"] = res["per_region_ms"] / res["batched_ms"]
    res["bit_identical"] = all(torch.equal(out["batched"][f], out["per_region"][f]) for f in out["batched"])
    res["value_batched"] = float(counts.sum()) / (res["batched_ms"] * 1e-3)
    res["value_per_region"] = float(counts.sum()) / (res["per_region_ms"] * 1e-3)
    res["unit"] = UNIT
    del ws, ws1, st, batch
    torch.cuda.empty_cache()
    return res


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2111_13094_gb300 import api
    from paper_2111_13094_gb300 import synthetic as syn

    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    seed = rank_seed(rank)                     # every rank fits its own regions (weak scaling)
    want_cpu = rank == 0 and world == 1 and not args.no_cpu

    # ---- inputs resident in HBM
    R_REGIONS = args.regions
    truth = syn.batched_truth(seed, R_REGIONS, K=K_COMP)
    counts = syn.region_counts(seed, R_REGIONS)
    N = int(counts.sum())
    off_h = syn.offsets_from_counts(counts)
    off = torch.from_numpy(off_h).to(dev)
    batches = [api.SampleBatch(syn.draw_torch(seed * 100 + r, truth, counts, device=dev), off)
               for r in range(ROUNDS)]
    _, h, _ = syn.region_grid(R_REGIONS)
    uni = syn.init_uniforms(seed, R_REGIONS, 2)
    prec = PREC[args.precision]
    peaks, src = _peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count

    def fit_leg(precision):
        """The timed step for one E-step form: restore the initial state, four
        rounds.  Returns (ms per step, E-step kernel ms per launch, status
        counts, state, snapshot, plan)."""
        cfg = api.config(K_COMP, precision=precision, chunk=CHUNK)
        st = api.MixtureState(R_REGIONS, K_COMP, device=dev)
        api.init_regions(cfg, batches[0], torch.from_numpy(h.astype(np.float64)).to(dev),
                         torch.from_numpy(uni).to(dev), st)
        snap = {f: getattr(st, f).clone() for f in STATE_FIELDS + ("etab", "qtab")}
        ws = api.workspace(cfg, R_REGIONS, N, device=dev)
        plan = api.FitPlan(cfg, R_REGIONS, N, 1, st, ws)
        torch.cuda.synchronize()

        def step():
            for f, v in snap.items():               # the step's initial state (device copies)
                getattr(st, f).copy_(v, non_blocking=True)
            for b in batches:
                plan.run(b)

        for _ in range(args.warmup):
            step()
        plan.enable_timing(args.steps * ROUNDS)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        e0, e1 = _events()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ck = clocks.stop()
        ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        kern = plan.timing()
        codes, cnt = torch.unique(st.status, return_counts=True)
        sc = {int(c): int(n) for c, n in zip(codes.cpu(), cnt.cpu())}
        return ms, (float(np.mean(kern)) if kern else float("nan")), sc, st, snap, plan, ws, ck, len(kern)

    ms, kms, status_counts, st, snap, plan, ws, ck, n_launch = fit_leg(prec)
    status_ok = status_counts.get(0, 0) == R_REGIONS
    value = whole_job_rate(args.steps * ROUNDS * N, world, ms)

    # ---- E-step kernel roofline (FP32 ALU bound)
    pairs = N * K_COMP
    achieved = pairs * FLOPS_PER_PAIR / (kms * 1e-3) / 1e12
    peak, basis = fp32_peak(n_sm, peaks, src)
    kname = "k_estep<16>" if prec == PREC["fp32"] else f"k_tc_estep<16,{args.precision}>"
    bps = DRAM_BYTES_PER_SAMPLE.get(kname)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": bps * N if bps is not None else None,
            "traffic_unit": "bytes per launch", "kernel": kname,
            "kernel_ms": kms, "launches_timed": n_launch,
            "algorithmic": f"{FLOPS_PER_PAIR} FP32 flops per (sample, component) x {N} samples x {K_COMP}",
            "peak_basis": basis,
            "hbm_gbs": N * BYTES_PER_SAMPLE / (kms * 1e-3) / 1e9,
            "hbm_frac": N * BYTES_PER_SAMPLE / (kms * 1e-3) / 1e9 / peaks.get("hbm_gbs", 6800.0)}

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args, batches, off, st, snap, plan, stream, world, N)
    plan.close()
    del plan, ws, st, snap
    torch.cuda.empty_cache()

    # ---- the tensor-core contraction form (three-piece BF16) on the same step
    tcres = None
    if prec == PREC["fp32"] and not args.no_tc:
        tms, tk, tsc, tst, tsnap, tplan, tws, _, _ = fit_leg(PREC["6xbf16"])
        tval = whole_job_rate(args.steps * ROUNDS * N, world, tms)
        tcres = {"precision": "6xbf16", "value": tval, "unit": UNIT, "ms_per_step": tms / args.steps,
                 "kernel": "k_tc_estep<16,6xbf16>", "kernel_ms": tk, "vs_fp32": tval / value,
                 "status_counts": tsc}
        tplan.close()
        del tplan, tws, tst, tsnap
        torch.cuda.empty_cache()

    # ---- oracle baseline on a seeded sample of whole regions, and the
    # matched-error comparison of every form on those regions
    cpu, accuracy = None, None
    if want_cpu:
        order = np.random.default_rng(seed).permutation(R_REGIONS)
        data = []
        for r in order[:1024]:
            o0, o1 = int(off_h[r]), int(off_h[r + 1])
            data.append((int(r), [b.samples[:, o0:o1].cpu().numpy() for b in batches], float(h[r]), uni[r]))
        cpu, done = cpu_baseline_fit(data, args.cpu_budget)
        accuracy = fit_accuracy(api, torch, dev, done, ("fp32", "6xbf16", "3xtf32"))
        if tcres is not None:
            tcres["accuracy"] = accuracy["6xbf16"]

    # ---- the spatial kD-tree on this round's samples: binning into the
    # pre-subdivided 8 x 8 x 8 grid, then refinement with c = 16,000 (Sec. 4.2)
    kdres = None if args.no_kdtree else kdtree_leg(api, torch, dev, batches[0], N, peaks)
    del batches
    torch.cuda.empty_cache()

    # ---- query workload: 16M guided queries over 65,536 grid regions
    qres = None
    if not args.no_queries:
        qres = query_leg(args, api, torch, dev, stream, seed, world, api.config(K_COMP), peaks, src, n_sm,
                         want_cpu)

    # ---- the other workloads
    configs = None
    if not args.no_configs and rank == 0:
        configs = {"single_region": config_single_region(api, torch, dev, stream, want_cpu),
                   "precision_sweep": config_precision_sweep(api, torch, dev, stream, want_cpu),
                   "objective": config_objective(api, torch, dev, stream, want_cpu),
                   "ablations": config_ablations(api, torch, dev, stream, want_cpu),
                   "batching": config_batching(api, torch, dev, stream)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded; shapes of the paper's leaves: K=16, log-uniform leaf sizes)",
                "config": dict(fit_config(R_REGIONS, N), all_regions_ok=status_ok, status_counts=status_counts,
                               precision=args.precision, chunk=CHUNK,
                               state_restore="12 device-to-device copies of the initial state (23 MB) at the "
                                             "start of every step, inside the timed region"),
                "clocks": ck, "e2e": e2e,
                "gpu_launches": args.steps * ROUNDS * (4 if prec == PREC["fp32"] else 5),
                "roofline": roof, "cpu_baseline": cpu, "accuracy": accuracy, "queries": qres,
                "tensor_core": tcres, "kdtree": kdres, "configs": configs}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="sdmm", choices=["sdmm", "reference"])
    ap.add_argument("--no-queries", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle legs (and so the accuracy check)")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="single-threaded oracle seconds of the fit leg")
    ap.add_argument("--regions", type=int, default=4096, help="regions of the fit workload")
    ap.add_argument("--no-tc", action="store_true", help="skip the tensor-core (6xBF16) comparison")
    ap.add_argument("--no-kdtree", action="store_true", help="skip the kD-tree binning/refinement timing")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads")
    ap.add_argument("--precision", default="fp32", choices=list(PREC),
                    help="E-step arithmetic: FP32 SIMT or a tensor-core contraction form")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--queries", type=int, default=Q_COUNT, help="queries of the query workload")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)        # at least 3 untimed steps, reported as run
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
