"""Benchmark of the SDMM hot path on GB300.

Workload (one step): the batched stepwise fit of 4,096 regions x K = 16
components, sample counts log-uniform in [256, 65,536] per region, four
Robbins-Monro EM rounds with a fresh seeded batch each, every round one
persistent E-step launch plus reductions replayed from a CUDA graph.  Inputs
are resident in HBM (about 1.35 GB per round, larger than L2) when the timed
region starts.  `value` = sample-iterations per second over all ranks.

Also reported on the same line: the end-to-end rate through the public API
with host buffers (H2D of each round's batch, D2H of the fitted parameters),
the E-step kernel's roofline (FP32 ALU bound) from CUDA events inside the
graph, the query workload (16M guided queries over 65,536 grid regions), and
the FP64 oracle timed on the host cores on a bounded sample.

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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EM sample-iterations/s and guided queries/s vs plain FP32 at matched log-lik"
UNIT = "sample-iterations/s"
K_COMP, ROUNDS = 16, 4
Q_DIMS, Q_COUNT = (64, 32, 32), 16 * 2 ** 20
# algorithmic FP32 work of the E-step + statistics per (sample, component):
# log map 23, Mahalanobis 39, log-sum-exp and responsibility 6, statistics 46
FLOPS_PER_PAIR = 114
# bytes per sample of one E-step pass: 7 FP32 streams
BYTES_PER_SAMPLE = 28
# DRAM bytes per sample of the FP32 E-step kernel, read + write, from one ncu
# capture of a 512-region launch of the same kernel (traffic grows with the
# samples processed, so a full launch moves this times N); None for kernels
# without a capture of their current version
DRAM_BYTES_PER_SAMPLE = {"k_accumulate<16,FIT>": 29.0}


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


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


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
def cpu_baseline(budget_s=15.0, seed=1, R_REGIONS=4096):
    """The FP64 oracle, as it stands, on a bounded sample of the fit workload
    (whole regions in seed order until the budget), single-threaded."""
    import oracle as orc
    from paper_2111_13094_gb300 import synthetic as syn
    truth = syn.batched_truth(seed, R_REGIONS, K=K_COMP)
    counts = syn.region_counts(seed, R_REGIONS)
    regions = np.random.default_rng(seed).permutation(R_REGIONS)
    done_samples, t_total, used = 0, 0.0, 0
    for r in regions:
        sub_truth = syn.GroundTruth(truth.pi[r:r + 1], truth.mu_x[r:r + 1], truth.mu_w[r:r + 1],
                                    truth.e1[r:r + 1], truth.e2[r:r + 1], truth.cov[r:r + 1])
        s = syn.draw(np.random.default_rng([seed, 7, int(r)]), sub_truth, [counts[r]])
        off = np.array([0, counts[r]], np.int64)
        st = orc.State(1, K_COMP)
        orc.init_regions(orc.config(K_COMP), off, s, np.array([1.0 / 16]), np.array([[0.3, 0.7]]), st)
        t0 = time.perf_counter()
        for _ in range(ROUNDS):
            orc.fit_regions(orc.config(K_COMP), off, s, 1, st)
        t_total += time.perf_counter() - t0
        done_samples += ROUNDS * int(counts[r])
        used += 1
        if t_total > budget_s:
            break
    return {"value": done_samples / t_total, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{used} of {R_REGIONS} regions ({done_samples // ROUNDS} samples), "
                      f"{ROUNDS} stepwise rounds each, FP64, single thread, {t_total:.1f} s"}


def fit_config(R_REGIONS, N):
    """The workload both arms report (the GPU arm adds its run's status counts)."""
    return {"workload": f"batched stepwise MAP-EM fit: {R_REGIONS} regions x K=16, sample counts "
                        "log-uniform in [256, 65536], 4 Robbins-Monro rounds per step with a "
                        "fresh batch each, CUDA-graph replay per round",
            "regions": R_REGIONS, "K": K_COMP, "rounds_per_step": ROUNDS,
            "samples_per_round": N, "per_rank": True,
            "l2": "inputs larger than L2 (about 1.35 GB per round)"}


def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:                            # the oracle runs once, on rank 0
        return None
    from paper_2111_13094_gb300 import synthetic as syn
    n_round = int(syn.region_counts(rank_seed(0), args.regions).sum())   # rank 0's workload, as the GPU arm
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(budget_s=per_step / 4)
    vals = []
    t0 = time.perf_counter()
    for i in range(args.steps):
        vals.append(cpu_baseline(budget_s=per_step, seed=1 + i))
    dt = time.perf_counter() - t0
    v = float(np.mean([x["value"] for x in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": fit_config(args.regions, n_round),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
def measure_e2e(args, batches, off, st, plan, stream, e0, e1, world, N):
    """Same step through the public API with host buffers: each round's batch
    goes from pinned host memory through the plan's host entry point (its
    copy into a staging slot overlaps the previous round's replay), and the
    fitted parameters are read back."""
    import torch

    from paper_2111_13094_gb300 import api
    host_off = off.cpu().pin_memory()
    host = [api.SampleBatch(b.samples.cpu().pin_memory(), host_off) for b in batches]
    staging = torch.empty(plan.staging_bytes(), dtype=torch.uint8, device=off.device)
    params = (st.pi, st.mu_x, st.mu_w, st.L)
    out_host = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in params]

    def e2e_step():
        for hb in host:
            plan.run_host(hb, staging)
        for o, t in zip(out_host, params):
            o.copy_(t, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    n = max(2, args.steps // 10)
    e0.record(stream)
    for _ in range(n):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    h2d = sum(hb.samples.numel() * hb.samples.element_size() + host_off.numel() * 8 for hb in host)
    d2h = sum(o.numel() * o.element_size() for o in out_host)
    del staging
    return {"value": world * ROUNDS * N / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": ms,
            "path": "sdmm_fit_plan_run_host: pinned host batch -> staging slot (copy stream) -> graph replay"}


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

    # ---- inputs resident in HBM
    R_REGIONS = args.regions
    truth = syn.batched_truth(seed, R_REGIONS, K=K_COMP)
    counts = syn.region_counts(seed, R_REGIONS)
    N = int(counts.sum())
    off = torch.from_numpy(syn.offsets_from_counts(counts)).to(dev)
    batches = [api.SampleBatch(syn.draw_torch(seed * 100 + r, truth, counts, device=dev), off)
               for r in range(ROUNDS)]
    _, h, _ = syn.region_grid(R_REGIONS)
    prec = {"fp32": api.PREC_FP32, "3xbf16": api.PREC_TC_3XBF16, "tf32": api.PREC_TC_TF32,
            "3xtf32": api.PREC_TC_3XTF32, "6xbf16": api.PREC_TC_6XBF16}[args.precision]
    cfg = api.config(K_COMP, precision=prec)
    st = api.MixtureState(R_REGIONS, K_COMP, device=dev)
    api.init_regions(cfg, batches[0], torch.from_numpy(h.astype(np.float64)).to(dev),
                     torch.from_numpy(syn.init_uniforms(seed, R_REGIONS, 2)).to(dev), st)
    ws = api.workspace(cfg, R_REGIONS, N, device=dev)
    plan = api.FitPlan(cfg, R_REGIONS, N, 1, st, ws)
    torch.cuda.synchronize()

    def step():
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
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    kern = plan.timing()
    codes, cnt = torch.unique(st.status, return_counts=True)
    status_counts = {int(c): int(n) for c, n in zip(codes.cpu(), cnt.cpu())}
    status_ok = status_counts.get(0, 0) == R_REGIONS
    value = whole_job_rate(args.steps * ROUNDS * N, world, ms)

    # ---- E-step kernel roofline (FP32 ALU bound)
    peaks, src = _peaks()
    kms = float(np.mean(kern)) if kern else float("nan")
    pairs = N * K_COMP
    achieved = pairs * FLOPS_PER_PAIR / (kms * 1e-3) / 1e12
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = n_sm * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    kname = "k_accumulate<16,FIT>" if prec == api.PREC_FP32 else f"k_tc_estep<16,{args.precision}>"
    bps = DRAM_BYTES_PER_SAMPLE.get(kname)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": bps * N if bps is not None else None,
            "traffic_unit": "bytes per launch",
            "kernel": kname,
            "kernel_ms": kms, "launches_timed": len(kern),
            "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x 2 flop x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz "
                          f"({src} max clock)",
            "hbm_gbs": N * BYTES_PER_SAMPLE / (kms * 1e-3) / 1e9,
            "hbm_frac": N * BYTES_PER_SAMPLE / (kms * 1e-3) / 1e9 / peaks.get("hbm_gbs", 6800.0)}

    # ---- the tensor-core contraction form (three-piece BF16, which meets the
    # parity contract) on the same resident batches, same steps
    tcres = None
    if prec == api.PREC_FP32 and not args.no_tc:
        tcfg = api.config(K_COMP, precision=api.PREC_TC_6XBF16)
        tst = api.MixtureState(R_REGIONS, K_COMP, device=dev)
        api.init_regions(tcfg, batches[0], torch.from_numpy(h.astype(np.float64)).to(dev),
                         torch.from_numpy(syn.init_uniforms(seed, R_REGIONS, 2)).to(dev), tst)
        tws = api.workspace(tcfg, R_REGIONS, N, device=dev)
        tplan = api.FitPlan(tcfg, R_REGIONS, N, 1, tst, tws)
        for _ in range(args.warmup):
            for b in batches:
                tplan.run(b)
        tplan.enable_timing(args.steps * ROUNDS)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0.record(stream)
        for _ in range(args.steps):
            for b in batches:
                tplan.run(b)
        e1.record(stream)
        torch.cuda.synchronize()
        tms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        tk = tplan.timing()
        c2, n2 = torch.unique(tst.status, return_counts=True)
        tval = whole_job_rate(args.steps * ROUNDS * N, world, tms)
        tcres = {"precision": "6xbf16", "value": tval, "unit": UNIT, "ms_per_step": tms / args.steps,
                 "kernel": "k_tc_estep<16,6xbf16>", "kernel_ms": float(np.mean(tk)) if tk else None,
                 "vs_fp32": tval / value,
                 "status_counts": {int(c): int(n) for c, n in zip(c2.cpu(), n2.cpu())},
                 "accuracy": "meets the 1e-4 log-likelihood / 1e-3 parameter contract against the FP64 "
                             "oracle at 1,024 x 65,536 (tests/precision_sweep.py)"}
        del tplan, tws, tst

    # ---- the spatial kD-tree on this round's samples: binning into the
    # pre-subdivided 8 x 8 x 8 grid, then refinement with c = 16,000 (Sec. 4.2)
    kdres = None
    if not args.no_kdtree:
        tree = api.KdTree(1 << 20, 1 << 19, device=dev)
        raw = batches[0].samples
        times = []
        for rep in range(3):
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
        kdres = {"samples": N, "bin_ms": tb, "refine_ms": tr, "leaves_after": tree.n_leaves,
                 "nodes_after": tree.n_nodes, "c": 16000,
                 "bin_samples_per_s": N / (tb * 1e-3), "refine_samples_per_s": N / (tr * 1e-3),
                 "bin_roofline": {"bound": "hbm", "achieved": bin_gbs, "peak": peaks.get("hbm_gbs", 6800.0),
                                  "unit": "GB/s", "frac": bin_gbs / peaks.get("hbm_gbs", 6800.0),
                                  "bytes_per_sample": 56.0},
                 "note": "host wall time of the synchronous calls (binning: leaf lookup, stable radix sort by "
                         "leaf, one gather; refinement: rounds of stable partitions, one 4-byte read-back per "
                         "tree level)"}
        del tree, kb, kr, kp

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args, batches, off, st, plan, stream, e0, e1, world, N)

    # ---- query workload: 16M guided queries over 65,536 grid regions
    qres = None
    if not args.no_queries:
        Rq = int(np.prod(Q_DIMS))
        pi, mu_x, mu_w, L = syn.random_mixtures(seed, Q_DIMS, K_COMP)
        qst = api.MixtureState(Rq, K_COMP, device=dev)
        qst.set_params(torch.from_numpy(pi), torch.from_numpy(mu_x), torch.from_numpy(mu_w),
                       torch.from_numpy(L))
        api.prepare(cfg, qst)
        qx = torch.from_numpy(syn.query_points(seed, Q_COUNT)).to(dev)
        grid = api.Grid((0, 0, 0), (1, 1, 1), Q_DIMS)
        out = (torch.empty(Q_COUNT, 3, device=dev), torch.empty(Q_COUNT, device=dev),
               torch.empty(Q_COUNT, dtype=torch.uint8, device=dev))
        reg = torch.from_numpy(syn.grid_region(qx.cpu().numpy(), Q_DIMS)).to(dev)
        order = torch.argsort(reg)
        qx_b, reg_b = qx[order].contiguous(), reg[order].contiguous()

        def timed(fn, reps=10):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        t_grid = timed(lambda: api.sample(cfg, qst, qx, grid=grid, seed=7, out=out))
        t_bin = timed(lambda: api.sample(cfg, qst, qx_b, region=reg_b, seed=7, out=out))
        disc = 1.0 - out[2].float().mean().item()
        qres = {"value": world * Q_COUNT / (t_grid * 1e-3), "unit": "queries/s",
                "binned_value": world * Q_COUNT / (t_bin * 1e-3), "kernel_ms": t_grid,
                "binned_kernel_ms": t_bin, "queries": Q_COUNT, "regions": Rq, "K": K_COMP,
                "discard_rate": disc,
                "config": "16M positions uniform in the unit cube, 64x32x32 grid regions, "
                          "condition + Philox draw + sample + pdf, FP32"}
        # product sampling with a 3-lobe BSDF mixture per query (top-2 lobes kept)
        bw, bmu, bL = (torch.from_numpy(a).to(dev) for a in syn.bsdf_lobes(seed, Q_COUNT, 3))
        t_prod = timed(lambda: api.product_sample(cfg, qst, qx, bw, bmu, bL, grid=grid, seed=7))
        bw_b, bmu_b, bL_b = bw[order].contiguous(), bmu[order].contiguous(), bL[order].contiguous()
        t_prod_b = timed(lambda: api.product_sample(cfg, qst, qx_b, bw_b, bmu_b, bL_b, region=reg_b, seed=7))
        qres["product"] = {"value": world * Q_COUNT / (t_prod * 1e-3), "unit": "queries/s", "kernel_ms": t_prod,
                           "binned_value": world * Q_COUNT / (t_prod_b * 1e-3), "binned_kernel_ms": t_prod_b,
                           "config": "the same 16M queries, 3 BSDF lobes each (wide, narrow, random), "
                                     "2K pairs per query: condition + pair products + sample + product pdf, FP32"}
        del bw, bmu, bL, bw_b, bmu_b, bL_b

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(budget_s=args.cpu_budget)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded; shapes of the paper's leaves: K=16, log-uniform leaf sizes)",
                "config": dict(fit_config(R_REGIONS, N), all_regions_ok=status_ok, status_counts=status_counts,
                               precision=args.precision),
                "clocks": ck, "e2e": e2e,
                "gpu_launches": args.steps * ROUNDS * (4 if prec == api.PREC_FP32 else 5),
                "roofline": roof, "cpu_baseline": cpu, "queries": qres, "tensor_core": tcres,
                "kdtree": kdres}
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
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--regions", type=int, default=4096, help="regions of the fit workload")
    ap.add_argument("--no-tc", action="store_true", help="skip the tensor-core (6xBF16) comparison")
    ap.add_argument("--no-kdtree", action="store_true", help="skip the kD-tree binning/refinement timing")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "3xbf16", "tf32", "3xtf32", "6xbf16"],
                    help="E-step arithmetic: FP32 SIMT or a tensor-core contraction form")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)        # at least 3 untimed steps, reported as run
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
