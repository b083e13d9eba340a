"""Precision sweep of the E-step on the config of 1,024 regions x 65,536
samples (K = 16 and 32): throughput of the FP32 SIMT form and of the
tensor-core contraction form in split 3xBF16, TF32, split 3xTF32 and
three-piece 6xBF16, each beside its error against the FP64 oracle on a
seeded sample of regions.

    python tests/precision_sweep.py [--regions 1024] [--per-region 65536]
                                    [--check 4] [--K 16 32] [--rounds 20]

Test infrastructure (it runs the oracle): prints a markdown table and one
JSON line.  For every mode the checked regions start from the oracle's own
initialisation of the same seeded samples; one EM step follows on both
sides and the per-sample log-likelihood and the parameters are compared.
The timing then replays one EM round (E-step, reduction, M-step) from a
CUDA graph on all regions.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle as orc  # noqa: E402
from gpu_util import block_err, host  # noqa: E402
from paper_2111_13094_gb300 import api  # noqa: E402
from paper_2111_13094_gb300 import synthetic as syn  # noqa: E402

MODES = {"fp32": api.PREC_FP32, "3xbf16": api.PREC_TC_3XBF16, "tf32": api.PREC_TC_TF32,
         "3xtf32": api.PREC_TC_3XTF32, "6xbf16": api.PREC_TC_6XBF16}


def _errors(g: orc.State, o: orc.State, regions, ll_g, ll_o):
    """Errors of the GPU state g against the oracle o on `regions` (indices
    into g), o holding those regions in order."""
    ok = o.status == 0
    rs = np.asarray(regions)[ok]
    oo = np.where(ok)[0]
    e_ll = np.abs(ll_g.astype(np.float64) - ll_o) / np.maximum(1.0, np.abs(ll_o))
    out = {"loglik_max": float(e_ll.max()), "loglik_median": float(np.median(e_ll))}
    out["pi"] = float(np.abs(g.pi[rs] - o.pi[oo]).max()) if rs.size else 0.0
    span = np.array([max(np.ptp(o.mu_x[r], axis=0).max(), 1e-3) for r in oo])
    out["mu_x"] = float((np.abs(g.mu_x[rs] - o.mu_x[oo]).max(axis=(1, 2)) / span).max()) if rs.size else 0.0
    out["mu_w"] = float(np.abs(g.mu_w[rs] - o.mu_w[oo]).max()) if rs.size else 0.0
    out["L"] = block_err(g.L[rs], o.L[oo])
    out["status_match"] = bool(np.array_equal(g.status[regions], o.status))
    return out


def run(R=1024, per=65536, K_list=(16, 32), modes=tuple(MODES), check=4, rounds=20, seed=11):
    dev = torch.device("cuda")
    results = []
    for K in K_list:
        truth = syn.batched_truth(seed + K, R, K=K)
        counts = np.full(R, per, dtype=np.int64)
        N = int(counts.sum())
        offsets = syn.offsets_from_counts(counts)
        samples = syn.draw_torch(seed + K, truth, counts, device=dev)
        batch = api.SampleBatch(samples, torch.from_numpy(offsets).to(dev))
        _, h, _ = syn.region_grid(R)
        regions = np.sort(np.random.default_rng([seed, K, 7]).choice(R, size=min(check, R), replace=False))
        # oracle side: the checked regions' samples, its own initialisation
        sub = np.concatenate([samples[:, offsets[r]:offsets[r + 1]].cpu().numpy() for r in regions], axis=1)
        sub_off = syn.offsets_from_counts(counts[regions])
        ocfg = orc.config(K)
        o0 = orc.State(len(regions), K)
        n_pos = K // 8
        orc.init_regions(ocfg, sub_off, sub, h[regions], syn.init_uniforms(seed, R, n_pos)[regions], o0)
        o1 = o0.copy()
        t0 = time.time()
        ll_o = orc.fit_regions(ocfg, sub_off, sub, 1, o1, want_loglik=True)
        t_oracle = time.time() - t0
        sel = np.concatenate([np.arange(offsets[r], offsets[r + 1]) for r in regions])
        for mode in modes:
            cfg = api.config(K, precision=MODES[mode])
            st = api.MixtureState(R, K, device=dev)
            api.init_regions(cfg, batch, torch.from_numpy(h.astype(np.float64)).to(dev),
                             torch.from_numpy(syn.init_uniforms(seed, R, n_pos)).to(dev), st)
            for f in orc.State.FIELDS:            # checked regions: the oracle's initial state
                getattr(st, f)[torch.from_numpy(regions).to(dev)] = torch.from_numpy(getattr(o0, f)).to(dev)
            api.prepare(cfg, st)
            ws = api.workspace(cfg, R, N, device=dev)
            ll = torch.empty(N, dtype=torch.float32, device=dev)
            api.fit_regions(cfg, batch, 1, st, ws, loglik=ll)
            torch.cuda.synchronize()
            err = _errors(host(st), o1, regions, ll[torch.from_numpy(sel).to(dev)].cpu().numpy(), ll_o)
            # timing: one EM round per graph replay on all regions
            plan = api.FitPlan(cfg, R, N, 1, st, ws)
            for _ in range(3):
                plan.run(batch)
            plan.enable_timing(rounds)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(rounds):
                plan.run(batch)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / rounds
            kern = plan.timing()
            k_ms = float(np.mean(kern)) if len(kern) else float("nan")
            results.append({"K": K, "mode": mode, "regions": R, "samples_per_region": per, "N": N,
                            "round_ms": ms, "estep_ms": k_ms, "sample_iterations_per_s": N / (ms * 1e-3),
                            "estep_samples_per_s": N / (k_ms * 1e-3), "checked_regions": [int(r) for r in regions],
                            "oracle_s": t_oracle, **err})
            del plan, ws, st, ll
            torch.cuda.empty_cache()
        del samples, batch
        torch.cuda.empty_cache()
    return results


def table(results):
    lines = ["| K | mode | E-step ms | round ms | sample-it/s | loglik err max | loglik err median | pi | mu_x | mu_w | L |",
             "|---|---|---|---|---|---|---|---|---|---|---|"]
    for r in results:
        lines.append(f"| {r['K']} | {r['mode']} | {r['estep_ms']:.3f} | {r['round_ms']:.3f} | "
                     f"{r['sample_iterations_per_s']:.3e} | {r['loglik_max']:.1e} | {r['loglik_median']:.1e} | "
                     f"{r['pi']:.1e} | {r['mu_x']:.1e} | {r['mu_w']:.1e} | {r['L']:.1e} |")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--regions", type=int, default=1024)
    ap.add_argument("--per-region", type=int, default=65536)
    ap.add_argument("--K", type=int, nargs="+", default=[16, 32])
    ap.add_argument("--modes", nargs="+", default=list(MODES))
    ap.add_argument("--check", type=int, default=4)
    ap.add_argument("--rounds", type=int, default=20)
    a = ap.parse_args()
    res = run(a.regions, a.per_region, a.K, a.modes, a.check, a.rounds)
    print(table(res))
    print(json.dumps(res))


if __name__ == "__main__":
    main()
