"""GPU timings and errors against the FP64 oracle for the single-region
fit (65,536 samples, K = 16, 20 plain EM iterations), the MAP objective and
its adjoint (1,024 regions x 16,384 samples, K = 16), the covariance
updates, the E-step density, and GPU timings of guided and product queries.

    python tests/measure_configs.py                 # everything
    python tests/measure_configs.py product --queries 1048576

Test infrastructure (it runs the oracle): prints a markdown table and one
JSON line.  Checked regions start from the oracle's own initialisation and
fit; the GPU receives those states, never the other way round.
"""
from __future__ import annotations

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
from gpu_util import block_err, dev_batch, gpu_state, host, loglik_err, oracle_init  # noqa: E402
from paper_2111_13094_gb300 import api  # noqa: E402
from paper_2111_13094_gb300 import synthetic as syn  # noqa: E402


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def single_region(seed=0, N=65536, K=16, iters=20, reps=10):
    b = syn.single_region(seed, N, K)
    ost = oracle_init(seed, b, K)
    o = ost.copy()
    ocfg = orc.config(K, eta_mode=1)
    t0 = time.time()
    ll_o = orc.fit_regions(ocfg, b.offsets, b.samples, iters, o, want_loglik=True)
    t_or = time.time() - t0
    gcfg = api.config(K, eta_mode=api.ETA_ONE)
    batch = dev_batch(b)
    ws = api.workspace(gcfg, 1, b.N)
    ll = torch.empty(b.N, dtype=torch.float32, device="cuda")
    st = gpu_state(ost, gcfg)
    api.fit_regions(gcfg, batch, iters, st, ws, loglik=ll)
    torch.cuda.synchronize()
    g = host(st)
    err = {"loglik": loglik_err(ll.cpu().numpy(), ll_o), "L": block_err(g.L[0], o.L[0]),
           "pi": float(np.abs(g.pi - o.pi).max()), "mu_w": float(np.abs(g.mu_w - o.mu_w).max())}
    e0, e1 = _events()
    times = []
    for _ in range(reps):
        st = gpu_state(ost, gcfg)
        torch.cuda.synchronize()
        e0.record()
        api.fit_regions(gcfg, batch, iters, st, ws)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    return {"config": "single region, N = 65,536, K = 16, 20 EM iterations (eta = 1)", "gpu_ms": ms,
            "sample_iterations_per_s": b.N * iters / (ms * 1e-3), "oracle_s": t_or,
            "oracle_sample_iterations_per_s": b.N * iters / t_or, **err}


def objective_adjoint(seed=30, R=1024, M=16384, K=16, check=3, reps=10):
    truth = syn.batched_truth(seed, R, K=K, parallax=True)
    counts = np.full(R, M, dtype=np.int64)
    N = R * M
    offsets = syn.offsets_from_counts(counts)
    dev = torch.device("cuda")
    samples = syn.draw_torch(seed, truth, counts, device=dev)
    batch = api.SampleBatch(samples, torch.from_numpy(offsets).to(dev))
    _, h, _ = syn.region_grid(R)
    gcfg = api.config(K)
    st = api.MixtureState(R, K, device=dev)
    api.init_regions(gcfg, batch, torch.from_numpy(h.astype(np.float64)).to(dev),
                     torch.from_numpy(syn.init_uniforms(seed, R, K // 8)).to(dev), st)
    ws = api.workspace(gcfg, R, N, device=dev)
    api.fit_regions(gcfg, batch, 3, st, ws)
    # checked regions: oracle initialisation and three oracle steps, handed to the GPU
    regions = np.sort(np.random.default_rng([seed, 9]).choice(R, size=check, replace=False))
    sub = np.concatenate([samples[:, offsets[r]:offsets[r + 1]].cpu().numpy() for r in regions], axis=1)
    sub_off = syn.offsets_from_counts(counts[regions])
    ocfg = orc.config(K)
    o = orc.State(check, K)
    orc.init_regions(ocfg, sub_off, sub, h[regions], syn.init_uniforms(seed, R, K // 8)[regions], o)
    orc.fit_regions(ocfg, sub_off, sub, 3, o)
    idx = torch.from_numpy(regions).to(dev)
    for f in orc.State.FIELDS:
        getattr(st, f)[idx] = torch.from_numpy(getattr(o, f)).to(dev)
    api.prepare(gcfg, st)
    t0 = time.time()
    F_o, gd_o, gL_o, ga_o = orc.objective(ocfg, sub_off, sub, o)
    t_or = time.time() - t0
    dF = torch.ones(R, dtype=torch.float64, device=dev)
    F = api.objective(gcfg, batch, st, ws)
    gd, gL, ga = api.objective_backward(gcfg, batch, st, dF, ws)
    torch.cuda.synchronize()

    def rel(g, ref):
        return float(np.abs(g - ref).max() / max(np.abs(ref).max(), 1e-30))

    Fg = F.cpu().numpy()[regions]
    err = {"F": float(np.abs(Fg - F_o).max() / max(1.0, np.abs(F_o).max())),
           "g_delta": rel(gd.cpu().numpy()[regions], gd_o), "g_L": rel(gL.cpu().numpy()[regions], gL_o),
           "g_logit": rel(ga.cpu().numpy()[regions], ga_o)}
    e0, e1 = _events()
    for _ in range(3):
        api.objective(gcfg, batch, st, ws)
        api.objective_backward(gcfg, batch, st, dF, ws)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        api.objective(gcfg, batch, st, ws)
    e1.record()
    torch.cuda.synchronize()
    f_ms = e0.elapsed_time(e1) / reps
    e0.record()
    for _ in range(reps):
        api.objective_backward(gcfg, batch, st, dF, ws)
    e1.record()
    torch.cuda.synchronize()
    b_ms = e0.elapsed_time(e1) / reps
    return {"config": "objective + adjoint, 1,024 regions x 16,384 samples, K = 16", "forward_ms": f_ms,
            "backward_ms": b_ms, "samples_per_s_forward": N / (f_ms * 1e-3),
            "samples_per_s_backward": N / (b_ms * 1e-3), "oracle_s_per_region": t_or / check,
            "oracle_samples_per_s": check * M / t_or, **err}


def covariance_updates(seed=40, R=1024, M=16384, K=16, check=3, steps=3, reps=5):
    """First-order vs accurate two-pass covariance update (plain EM): GPU time
    of an EM step and the covariance error of each against the oracle's
    two-pass update (the accurate reference) on checked regions."""
    truth = syn.batched_truth(seed, R, K=K, parallax=True)
    counts = np.full(R, M, dtype=np.int64)
    N = R * M
    offsets = syn.offsets_from_counts(counts)
    dev = torch.device("cuda")
    samples = syn.draw_torch(seed, truth, counts, device=dev)
    batch = api.SampleBatch(samples, torch.from_numpy(offsets).to(dev))
    _, h, _ = syn.region_grid(R)
    regions = np.sort(np.random.default_rng([seed, 9]).choice(R, size=check, replace=False))
    sub = np.concatenate([samples[:, offsets[r]:offsets[r + 1]].cpu().numpy() for r in regions], axis=1)
    sub_off = syn.offsets_from_counts(counts[regions])
    o0 = orc.State(check, K)
    orc.init_regions(orc.config(K), sub_off, sub, h[regions], syn.init_uniforms(seed, R, K // 8)[regions], o0)
    ref = o0.copy()
    orc.fit_regions(orc.config(K, eta_mode=1, cov_update=1), sub_off, sub, steps, ref)
    idx = torch.from_numpy(regions).to(dev)
    out = {"config": f"covariance update, {R} regions x {M} samples, K = {K}, plain EM, {steps} steps"}
    for name, mode in (("first_order", 0), ("two_pass", 1)):
        cfg = api.config(K, eta_mode=api.ETA_ONE, cov_update=mode)
        st = api.MixtureState(R, K, device=dev)
        api.init_regions(cfg, batch, torch.from_numpy(h.astype(np.float64)).to(dev),
                         torch.from_numpy(syn.init_uniforms(seed, R, K // 8)).to(dev), st)
        for f in orc.State.FIELDS:
            getattr(st, f)[idx] = torch.from_numpy(getattr(o0, f)).to(dev)
        api.prepare(cfg, st)
        ws = api.workspace(cfg, R, N, device=dev)
        snap = {f: getattr(st, f).clone() for f in orc.State.FIELDS}
        api.fit_regions(cfg, batch, steps, st, ws)
        torch.cuda.synchronize()
        g = host(st)
        err_L = block_err(g.L[regions], ref.L)
        e0, e1 = _events()
        times = []
        for _ in range(reps):
            for f in orc.State.FIELDS:
                getattr(st, f).copy_(snap[f])
            api.prepare(cfg, st)
            torch.cuda.synchronize()
            e0.record()
            api.fit_regions(cfg, batch, 1, st, ws)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        out[name] = {"step_ms": float(np.median(times)), "L_error_vs_two_pass_oracle": err_L}
    out["time_ratio"] = out["two_pass"]["step_ms"] / out["first_order"]["step_ms"]
    return out


def estep_density(seed=50, R=1024, M=16384, K=16, reps=10):
    """Cost of the change of variables in the E-step: one EM step with the
    chart density p^t (paper) and with the solid-angle density p^t / sinc."""
    truth = syn.batched_truth(seed, R, K=K)
    counts = np.full(R, M, dtype=np.int64)
    N = R * M
    dev = torch.device("cuda")
    samples = syn.draw_torch(seed, truth, counts, device=dev)
    batch = api.SampleBatch(samples, torch.from_numpy(syn.offsets_from_counts(counts)).to(dev))
    _, h, _ = syn.region_grid(R)
    out = {"config": f"E-step density, {R} regions x {M} samples, K = {K}"}
    for name, dens in (("chart", api.DENSITY_TANGENT), ("solid_angle", api.DENSITY_SOLID_ANGLE)):
        cfg = api.config(K, estep_density=dens)
        st = api.MixtureState(R, K, device=dev)
        api.init_regions(cfg, batch, torch.from_numpy(h.astype(np.float64)).to(dev),
                         torch.from_numpy(syn.init_uniforms(seed, R, K // 8)).to(dev), st)
        ws = api.workspace(cfg, R, N, device=dev)
        plan = api.FitPlan(cfg, R, N, 1, st, ws)
        for _ in range(3):
            plan.run(batch)
        plan.enable_timing(reps)
        for _ in range(reps):
            plan.run(batch)
        torch.cuda.synchronize()
        out[name] = {"estep_ms": float(np.mean(plan.timing()))}
        del plan, ws, st
    out["ratio"] = out["solid_angle"]["estep_ms"] / out["chart"]["estep_ms"]
    return out


def euclid_ablation(seed=80, R=1024, M=65536, K=16, reps=10):
    """E-step cost of the change of variables: the tangent-chart fit (paper)
    against the Euclidean ablation (no log map), for the FP32 SIMT form and
    the 6xBF16 contraction form, one EM step per run (GPU time of the E-step
    kernel from the plan's events)."""
    truth = syn.batched_truth(seed, R, K=K)
    counts = np.full(R, M, dtype=np.int64)
    N = R * M
    dev = torch.device("cuda")
    samples = syn.draw_torch(seed, truth, counts, device=dev)
    batch = api.SampleBatch(samples, torch.from_numpy(syn.offsets_from_counts(counts)).to(dev))
    _, h, _ = syn.region_grid(R)
    out = {"config": f"E-step, tangent vs Euclidean directions, {R} regions x {M} samples, K = {K}"}
    for pname, prec in (("fp32", api.PREC_FP32), ("6xbf16", api.PREC_TC_6XBF16)):
        for dname, dc in (("tangent", api.DIR_TANGENT), ("euclidean", api.DIR_EUCLIDEAN)):
            cfg = api.config(K, precision=prec, dir_coords=dc)
            st = api.MixtureState(R, K, device=dev)
            api.init_regions(cfg, batch, torch.from_numpy(h.astype(np.float64)).to(dev),
                             torch.from_numpy(syn.init_uniforms(seed, R, K // 8)).to(dev), st)
            ws = api.workspace(cfg, R, N, device=dev)
            plan = api.FitPlan(cfg, R, N, 1, st, ws)
            for _ in range(3):
                plan.run(batch)
            plan.enable_timing(reps)
            for _ in range(reps):
                plan.run(batch)
            torch.cuda.synchronize()
            out[f"{pname}_{dname}_estep_ms"] = float(np.mean(plan.timing()))
            plan.close()
            del plan, ws, st
        out[f"{pname}_ratio"] = out[f"{pname}_tangent_estep_ms"] / out[f"{pname}_euclidean_estep_ms"]
    return out


def product_queries(seed=60, Q=1 << 24, K=16, J=3, dims=(64, 32, 32), reps=10):
    """Guided queries with and without the BSDF product on the same positions
    (grid lookup, one Philox draw per query): GPU time per batch."""
    dev = torch.device("cuda")
    cfg = api.config(K)
    pi, mu_x, mu_w, L = syn.random_mixtures(seed, dims, K)
    st = api.MixtureState(int(np.prod(dims)), K, device=dev)
    st.set_params(torch.from_numpy(pi), torch.from_numpy(mu_x), torch.from_numpy(mu_w), torch.from_numpy(L))
    api.prepare(cfg, st)
    qx = torch.from_numpy(syn.query_points(seed, Q)).to(dev)
    bw, bmu, bL = (torch.from_numpy(a).to(dev) for a in syn.bsdf_lobes(seed, Q, J))
    grid = api.Grid((0, 0, 0), (1, 1, 1), dims)
    e0, e1 = _events()
    out = {"config": f"{Q} queries, {int(np.prod(dims))} grid regions, K = {K}, {J} BSDF lobes"}
    for name, fn in (("plain", lambda: api.sample(cfg, st, qx, grid=grid, seed=7)),
                     ("product", lambda: api.product_sample(cfg, st, qx, bw, bmu, bL, grid=grid, seed=7))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": ms, "queries_per_s": Q / (ms * 1e-3)}
    return out


def main():
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("which", nargs="*", default=[])
    ap.add_argument("--queries", type=int, default=1 << 24)
    args = ap.parse_args()
    if args.which == ["product"]:
        print(json.dumps(product_queries(Q=args.queries)))
        return
    if args.which == ["euclid"]:
        print(json.dumps(euclid_ablation()))
        return
    a = single_region()
    b = objective_adjoint()
    c = covariance_updates()
    d = estep_density()
    print("| config | GPU | error vs oracle | oracle (1 core) |")
    print("|---|---|---|---|")
    print(f"| {a['config']} | {a['gpu_ms']:.2f} ms ({a['sample_iterations_per_s']:.3e} sample-it/s) | "
          f"loglik {a['loglik']:.1e}, L {a['L']:.1e}, pi {a['pi']:.1e}, mu_w {a['mu_w']:.1e} | "
          f"{a['oracle_s']:.2f} s ({a['oracle_sample_iterations_per_s']:.3e} sample-it/s) |")
    print(f"| {b['config']} | forward {b['forward_ms']:.2f} ms, backward {b['backward_ms']:.2f} ms "
          f"({b['samples_per_s_backward']:.3e} samples/s) | F {b['F']:.1e}, grad delta {b['g_delta']:.1e}, "
          f"grad L {b['g_L']:.1e}, grad logit {b['g_logit']:.1e} | "
          f"{b['oracle_s_per_region']:.2f} s per region ({b['oracle_samples_per_s']:.3e} samples/s) |")
    for name in ("first_order", "two_pass"):
        print(f"| {c['config']}: {name} | {c[name]['step_ms']:.2f} ms per EM step | "
              f"L vs the accurate (two-pass) oracle {c[name]['L_error_vs_two_pass_oracle']:.1e} | — |")
    print(f"| {d['config']} | chart {d['chart']['estep_ms']:.2f} ms, solid angle {d['solid_angle']['estep_ms']:.2f} ms "
          f"per E-step ({d['ratio']:.2f}x) | (parity: tests/test_gpu_fit.py) | — |")
    print(json.dumps({"single_region": a, "objective": b, "covariance_updates": c, "estep_density": d}))


if __name__ == "__main__":
    main()
