"""Benchmark: one interior-point iteration on the 100^3 grid LP per step.

A step is one pass of the whole hot path on one GPU: constraint evaluation,
scaling D, assembly of the condensed matrix K = J^T D J + delta I, supernodal
Cholesky, predictor and corrector solves with FP64 refinement, direction
recovery, fraction-to-the-boundary step lengths, barrier update and the KKT
convergence test. The metric is throughput in algorithmic factor flops
(sum over columns of colcount^2) per second of step time, plus the
time-to-1e-6 KKT residual of a full solve.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one iteration of the cold-start solve to a 1e-6 KKT residual,
replayed from the iterate that iteration starts from (step k runs iteration
k mod T of the T-iteration solve), so the timed work is exactly the method's.
The method runs on one GPU; --gpus other than 1 is rejected.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "time-to-1e-6 KKT residual and factor TFLOP/s: mixed/learned vs FP64 on GB300"
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3, "tf32x3": 4}
# time-to-1e-6 forms beyond a fixed precision: (precision, CG steps per
# iteration above which ipm_solve moves to the split TF32 for the rest)
LADDERS = {"tf32_then_tf32x3": (2, 16)}
# DRAM bytes (read + written) of one factorisation, from a one-pass ncu capture
# of dram__bytes_read.sum and dram__bytes_write.sum over its launches (this
# build's kernels), keyed by (grid, precision): the roofline's "traffic"
FACTOR_TRAFFIC = {(100, "tf32x3"): 430.140e9 + 113.871e9}
DTYPE = {"fp64": "f64", "fp32": "f32+f64", "tf32": "tf32+f64", "bf16": "bf16+f64",
         "tf32x3": "tf32x3+f64"}
ORACLE_GRID = 24  # CPU sample: one oracle Newton direction on the 24^3 member of the family


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        if not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_direction_sample(grid: int, reps: int = 1):
    """Time the oracle's hot path (assembly + factor + solves of one Newton
    direction) on one host core; returns (seconds per direction, flops)."""
    import oracle
    oracle.build()
    lp = gen.grid_lp(grid, seed=1)
    perm = gen.nd_order_grid3d(grid)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    mt = lp.m + 2 * lp.n
    x = gen.uniform(21, lp.n, 0.5, 9.5)
    s = gen.uniform(22, mt, 0.01, 3.0)
    lam = gen.uniform(23, mt, 0.01, 3.0)
    w = np.zeros(mt)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.lp_direction(S, lp, x, s, lam, w, 1e-8, 1e-8)
        ts.append(time.perf_counter() - t0)
    return float(np.mean(ts)), S.flops, lp.n


def mpc_measure(steps: int = 3):
    """Batched MPC QPs (4096 instances, T ~ U{10..100}, 12 states, 4 inputs):
    autotuned launch shape, one persistent launch per batch replayed from a CUDA
    graph; solves per second for the FP32-factor (FP64-refined) and FP64 kernels."""
    import torch
    import paper_2508_16094_gb300 as gb
    mb = gen.mpc_batch(4096, seed=3)
    b = gb.BatchedMPC(mb)
    out = {"instances": mb.count, "stages": int(mb.T.sum())}
    for name, prec in (("fp32", gb.IPM_FP32), ("fp64", gb.IPM_FP64)):
        cfg, ms = b.ipm_mpc_autotune(precision=prec, tol=1e-6)
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            b.ipm_solve_batched(precision=prec, instances_per_cta=cfg.instances_per_cta,
                                ctas=cfg.ctas, tol=1e-6, stream=s.cuda_stream)
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / steps
        st = b.status.cpu().numpy()
        out[name] = {"ms_per_batch": round(t, 3), "solves_per_s": round(mb.count / (t * 1e-3), 1),
                     "converged": int((st == 0).sum()),
                     "max_kkt": float(f"{b.kkt.max().item():.3e}"),
                     "mean_iters": round(float(b.iters.float().mean().item()), 3),
                     "instances_per_cta": int(cfg.instances_per_cta), "ctas": int(cfg.ctas),
                     "autotune_ms": [round(x, 1) for x in ms]}
    return out


def forms_measure(G: int, train_seeds=(1001, 1002, 1003, 1004), seed: int = 1):
    """Time to a 1e-6 KKT residual from the cold start on the G^3 member of the
    grid-LP family for every form of the path: the FP64 factor, the split-TF32
    factor with FP64 refinement, and the latter with stale-factor skipping
    corrected by the trained network (learned = 1) or uncorrected (learned = 2,
    the E = 0 ablation). The network is first trained on the iterates of the
    method itself on other seeds of the same family."""
    import torch
    import paper_2508_16094_gb300 as gb
    from paper_2508_16094_gb300 import learned as GL
    perm = gen.nd_order_grid3d(G)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    lp = gen.grid_lp(G, seed=seed)
    jv, b, c = dev(lp.val), dev(lp.b), dev(lp.c)

    flops = []

    def mk(**kw):
        ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u,
                            options=gb.default_options(tol=1e-6, max_iter=200, **kw))
        flops.append(ctx.kkt_analyze(perm).flops)
        ctx.ipm_set_workspace()
        return ctx

    def run(ctx, **kw):
        ctx.ipm_set_options(warm_start=0, **kw)
        x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
        s = torch.empty(ctx.m_tot, dtype=torch.float64, device="cuda")
        lam = torch.empty(ctx.m_tot, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ctx.ipm_solve(jv, b, c, x, s, lam)
        torch.cuda.synchronize()
        return {"seconds": round(time.perf_counter() - t0, 4), "status": int(r.status),
                "iterations": int(r.iterations), "factorizations": int(r.factorizations),
                "learned_skips": int(r.learned_skips), "pcg_steps": int(r.pcg_steps),
                "kkt": float(f"{r.kkt:.3e}"), "objective": r.objective,
                "time_factor_s": round(r.time_factor_ms / 1e3, 4),
                "time_solve_s": round(r.time_solve_ms / 1e3, 4)}

    out = {"workload": f"grid LP {G}^3 (n={lp.n}), seed {seed}; network trained on seeds "
                       f"{list(train_seeds)} of the same family"}
    c64 = mk(precision=gb.IPM_FP64, storage_fp64=1)
    run(c64, max_iter=1)  # first-touch of the workspace and graphs
    out["fp64"] = run(c64, max_iter=200)
    c64.close()
    # the FP64 factor with its updates on the tensor cores (Ozaki slices)
    c64 = mk(precision=gb.IPM_FP64, storage_fp64=1, fp64_tc=1)
    run(c64, max_iter=1)
    out["fp64_tc"] = run(c64, max_iter=200)
    c64.close()
    ctx = mk(precision=gb.IPM_TF32X3, storage_fp64=0, learned_probes=4)
    run(ctx, max_iter=1, learned=0)
    out["tf32x3"] = run(ctx, max_iter=200, learned=0)
    t0 = time.perf_counter()
    samples = []
    for sd in train_seeds:
        lpt = gen.grid_lp(G, seed=sd)
        jt, bt, ct = dev(lpt.val), dev(lpt.b), dev(lpt.c)
        traj = GL.trajectory(ctx, jt, bt, ct, 60)
        samples += GL.collect(ctx, jt, bt, ct, traj, staleness=(1, 2, 3), seed=sd)
    hist = GL.train(ctx, samples, epochs=30, lr=3e-3)
    torch.cuda.synchronize()
    out["training"] = {"samples": len(samples), "seconds": time.perf_counter() - t0,
                       "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1]}
    out["tf32x3_learned"] = run(ctx, max_iter=200, learned=1)
    out["tf32x3_stale_E0"] = run(ctx, max_iter=200, learned=2)
    ctx.close()
    ref = out["fp64"]["objective"]
    for k in ("fp64_tc", "tf32x3", "tf32x3_learned", "tf32x3_stale_E0"):
        out[k]["objective_rel_diff_vs_fp64"] = float(
            f"{abs(out[k]['objective'] - ref) / max(1.0, abs(ref)):.2e}")
    out["flops"] = flops[0]
    return out


def nlp_measure(N: int, max_iter: int = 150):
    """Grid NLP (512^2 grid, cubic PDE constraint as inequality pairs, -1 <= v <= 1):
    the FP64 factor against the split-TF32 and BF16 factors with FP64 fallback
    (once a low-precision factor breaks down, FP64 for the rest), from the cold
    start, at most max_iter iterations towards a 1e-6 KKT residual."""
    import torch
    import paper_2508_16094_gb300 as gb
    P = gen.grid_nlp(N, seed=5)
    perm = gen.nd_order_grid_nlp(N)
    ut = torch.as_tensor(P.ut, dtype=torch.float64, device="cuda")
    out = {"workload": f"grid NLP {N}^2 (n = m = {P.n}), alpha 5e-3, |v| <= 1, seed 5",
           "max_iter": max_iter}
    for name, prec, tc in (("fp64", gb.IPM_FP64, 0), ("fp64_tc", gb.IPM_FP64, 1),
                           ("tf32x3", gb.IPM_TF32X3, 0), ("bf16", gb.IPM_BF16, 0)):
        o = gb.default_options(precision=prec, tol=1e-6, max_iter=max_iter, storage_fp64=1,
                               fallback_fp64=1, fp64_tc=tc)
        G = gb.GridNLP(N, perm=perm, options=o)
        n, mt = G.pat["n"], G.ctx.m_tot
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        s = torch.empty(mt, dtype=torch.float64, device="cuda")
        lam = torch.empty(mt, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = G.ipm_solve_grid_nlp(ut, x, s, lam)
        torch.cuda.synchronize()
        out[name] = {"seconds": round(time.perf_counter() - t0, 3), "status": int(r.status),
                     "iterations": int(r.iterations), "objective": r.objective,
                     "kkt": float(f"{r.kkt:.3e}"), "primal": float(f"{r.primal_res:.3e}"),
                     "dual": float(f"{r.dual_res:.3e}"), "fp64_fallbacks": int(r.fp64_fallbacks),
                     "factorizations": int(r.factorizations),
                     "regularizations": int(r.regularizations), "refine_steps": int(r.refine_steps),
                     "fp64_tc_rechecks": int(r.fp64_tc_rechecks),
                     "factor_flops": G.info.flops}
        G.ctx.close()
    for name in ("fp64_tc", "tf32x3", "bf16"):
        out[name]["objective_rel_diff_vs_fp64"] = float(
            f"{abs(out[name]['objective'] - out['fp64']['objective']) / max(1.0, abs(out['fp64']['objective'])):.2e}")
    return out


def learned_sweep(G: int, n_train: int = 64, n_test: int = 16, first_seed: int = 3001):
    """The learned correction's seed sweep on the G^3 member of the grid-LP
    family: the network is trained on the interior-point iterates of n_train
    seeds (staleness 1-3, 4 probes per sample), then n_test held-out seeds are
    solved from the cold start to KKT <= 1e-6 with the FP64 factor, the
    split-TF32 factor refactored every iteration, and the latter with the
    learned skip (learned = 1) and with the uncorrected stale factor (the
    E = 0 ablation, learned = 2). Per form: refactorisations skipped, the
    times, and their shifted geometric mean (shift 10 s, SGM10)."""
    import torch
    import paper_2508_16094_gb300 as gb
    from paper_2508_16094_gb300 import learned as GL
    perm = gen.nd_order_grid3d(G)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    lp0 = gen.grid_lp(G, seed=first_seed)

    def mk(**kw):
        ctx = gb.IpmContext(lp0.n, lp0.m, lp0.rowptr, lp0.col, lp0.l, lp0.u,
                            options=gb.default_options(tol=1e-6, max_iter=200, **kw))
        ctx.kkt_analyze(perm)
        ctx.ipm_set_workspace()
        return ctx

    def run(ctx, jv, b, c, **kw):
        ctx.ipm_set_options(warm_start=0, **kw)
        x = torch.empty(lp0.n, dtype=torch.float64, device="cuda")
        s = torch.empty(ctx.m_tot, dtype=torch.float64, device="cuda")
        lam = torch.empty(ctx.m_tot, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ctx.ipm_solve(jv, b, c, x, s, lam)
        torch.cuda.synchronize()
        return {"s": time.perf_counter() - t0, "status": int(r.status), "iters": int(r.iterations),
                "fact": int(r.factorizations), "skips": int(r.learned_skips),
                "pcg": int(r.pcg_steps), "obj": r.objective}

    ctx = mk(precision=gb.IPM_TF32X3, storage_fp64=0, learned_probes=4)
    t0 = time.perf_counter()
    samples = []
    train = [first_seed + k for k in range(n_train)]
    test = [first_seed + n_train + k for k in range(n_test)]
    for sd in train:
        lp = gen.grid_lp(G, seed=sd)
        jv, b, c = dev(lp.val), dev(lp.b), dev(lp.c)
        traj = GL.trajectory(ctx, jv, b, c, 60)
        samples += GL.collect(ctx, jv, b, c, traj, staleness=(1, 2, 3), seed=sd)
    t_collect = time.perf_counter() - t0
    hist = GL.train(ctx, samples, epochs=30, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0 - t_collect
    n_samples = len(samples)
    del samples
    c64 = mk(precision=gb.IPM_FP64, storage_fp64=1)
    lpw = gen.grid_lp(G, seed=test[0])
    run(c64, dev(lpw.val), dev(lpw.b), dev(lpw.c), max_iter=1)  # first touch
    run(ctx, dev(lpw.val), dev(lpw.b), dev(lpw.c), max_iter=1, learned=0)
    forms = {"fp64": (c64, {}), "tf32x3": (ctx, {"learned": 0}),
             "tf32x3_learned": (ctx, {"learned": 1}), "tf32x3_stale_E0": (ctx, {"learned": 2})}
    per = {k: [] for k in forms}
    for sd in test:
        lp = gen.grid_lp(G, seed=sd)
        jv, b, c = dev(lp.val), dev(lp.b), dev(lp.c)
        for name, (cx, kw) in forms.items():
            per[name].append(run(cx, jv, b, c, max_iter=200, **kw))
    c64.close()
    ctx.close()
    out = {"workload": f"grid LP {G}^3 family (n={lp0.n}): network trained on {n_train} seeds "
                       f"({n_samples} samples), evaluated on {n_test} held-out seeds to KKT <= 1e-6",
           "collect_s": round(t_collect, 1), "train_s": round(t_train, 1),
           "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1]}
    ref = [r["obj"] for r in per["fp64"]]
    for name, rs in per.items():
        ts = np.array([r["s"] for r in rs])
        out[name] = {"sgm10_s": round(float(np.exp(np.mean(np.log(ts + 10.0))) - 10.0), 4),
                     "mean_s": round(float(ts.mean()), 4), "converged": int(sum(r["status"] == 0 for r in rs)),
                     "refactorisations": int(sum(r["fact"] for r in rs)),
                     "skips": int(sum(r["skips"] for r in rs)), "pcg": int(sum(r["pcg"] for r in rs)),
                     "iterations": int(sum(r["iters"] for r in rs)),
                     "max_obj_rel_diff_vs_fp64": float(f"{max(abs(r['obj'] - o) / max(1.0, abs(o)) for r, o in zip(rs, ref)):.2e}")}
    return out


def world():
    """(world size, rank) from the launcher's environment (no process group:
    neither arm exchanges data between ranks)."""
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))


def run_reference(args, rank):
    """The oracle as it stands, on the host cores: each step one Newton direction
    of the 24^3 member of the grid-LP family. Under torchrun only rank 0 runs."""
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_direction_sample(ORACLE_GRID)
    ts = []
    flops = n = None
    for _ in range(args.steps):
        t, flops, n = oracle_direction_sample(ORACLE_GRID)
        ts.append(t)
    sec = float(np.sum(ts))
    val = flops * args.steps / sec / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"grid LP {ORACLE_GRID}^3 sample of the 100^3 family "
                                   "(one Newton direction per step)",
                       "parallelism": "single host core"},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": 1,
                             "host_cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"one oracle Newton direction (assembly, left-looking "
                                       f"Cholesky, solves) on the {ORACLE_GRID}^3 grid LP, "
                                       f"n={n}"},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def record_trajectory(ctx, jv, b, c, x, s, lam, max_iter=200):
    """The cold-start solve run one iteration per call: returns the iterate each
    iteration starts from (device copies) and the last call's result. Warm
    starts from the previous call's iterate reproduce the single solve's
    iterations (the regularisation starts from delta_p in both)."""
    ctx.ipm_set_options(max_iter=0, warm_start=0)
    r = ctx.ipm_solve(jv, b, c, x, s, lam)
    traj = []
    ctx.ipm_set_options(max_iter=1, warm_start=1)
    for _ in range(max_iter):
        traj.append((x.clone(), s.clone(), lam.clone()))
        r = ctx.ipm_solve(jv, b, c, x, s, lam)
        if r.status == 0:
            break
        if r.status != 7:
            raise RuntimeError(f"interior-point iteration failed: status {r.status}")
    return traj, r


def tti_run(ctx, jv, b, c, x, s, lam, prec, ref_obj=None, cg_escalate=0):
    """Cold start to the 1e-6 KKT residual in one ipm_solve call."""
    import torch
    # TF32/BF16 factors fall back to a split-TF32 refactorisation when their
    # PCG misses the acceptance tolerance (counted in "fallbacks"); with
    # cg_escalate also once an iteration needs more CG steps than that
    ctx.ipm_set_options(max_iter=200, warm_start=0, tol=1e-6, precision=prec, fallback_fp64=1,
                        cg_escalate=cg_escalate)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = ctx.ipm_solve(jv, b, c, x, s, lam)
    torch.cuda.synchronize()
    out = {"s": round(time.perf_counter() - t0, 4), "status": int(r.status),
           "iters": int(r.iterations), "pcg": int(r.pcg_steps), "kkt": float(f"{r.kkt:.3e}"),
           "fallbacks": int(r.fp64_fallbacks), "perturbed": int(r.perturbed_pivots),
           "regularizations": int(r.regularizations), "fp64_tc_rechecks": int(r.fp64_tc_rechecks),
           "obj": r.objective, "factor_s": round(r.time_factor_ms / 1e3, 4),
           "solve_s": round(r.time_solve_ms / 1e3, 4)}
    if ref_obj is not None:
        out["obj_rel_diff"] = float(f"{abs(r.objective - ref_obj) / max(1.0, abs(ref_obj)):.2e}")
    return out


def tti_fp64_tc(lp, perm, jv, b, c, ref_obj, bf16_peak):
    """The FP64 path measured: cold start to KKT <= 1e-6 with every factorisation
    in FP64, its dense updates on the tensor cores (Ozaki slices), in a context
    of its own (FP64 storage plus the slices)."""
    import torch
    import paper_2508_16094_gb300 as gb
    o = gb.default_options(precision=gb.IPM_FP64, storage_fp64=1, fp64_tc=1, tol=1e-6)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u, options=o)
    try:
        info = ctx.kkt_analyze(perm)
        ctx.ipm_set_workspace()
        x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
        s = torch.empty(ctx.m_tot, dtype=torch.float64, device="cuda")
        lam = torch.empty(ctx.m_tot, dtype=torch.float64, device="cuda")
        ctx.ipm_set_options(max_iter=1)  # first touch of the workspace
        ctx.ipm_solve(jv, b, c, x, s, lam)
        out = tti_run(ctx, jv, b, c, x, s, lam, gb.IPM_FP64, ref_obj)
        # one more factorisation of the last assembled matrix, timed alone
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.kkt_factor(gb.IPM_FP64)
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        out["factor_s_one"] = round(tf, 4)
        out["factor_tflops_fp64_equiv"] = round(info.flops / tf / 1e12, 2)
        # the same matrix factored on the FMA pipe (the slices left unused): the
        # FMA-pipe FP64 path's time to 1e-6 is this run's with each of its
        # factorisations replaced by one of those (the same 10 iterations)
        ctx.ipm_set_options(fp64_tc=0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.kkt_factor(gb.IPM_FP64)
        torch.cuda.synchronize()
        tm = time.perf_counter() - t0
        out["fma_factor_s_one"] = round(tm, 3)
        out["fma_factor_tflops"] = round(info.flops / tm / 1e12, 3)
        out["fma_path_s_estimate"] = round(out["s"] + out["iters"] * (tm - tf), 1)
        # its tensor work: 28 BF16 slice products per multiply-add, against the
        # measured BF16 burst peak (the factorisation timed alone)
        bp = 28 * info.flops / tf / 1e12
        out["roofline"] = {"bound": "tensor", "achieved": round(bp, 1), "peak": bf16_peak,
                           "unit": "TFLOP/s", "frac": round(bp / bf16_peak, 3),
                           "work": "28 BF16 products x sum colcount^2 per factorisation"}
        out["workspace_gb"] = round(info.workspace_bytes / 1e9, 1)
        return out
    except Exception as e:  # e.g. the slices do not fit next to the main context
        return {"error": str(e)[:160]}
    finally:
        ctx.close()
        torch.cuda.empty_cache()


def summary(tti, forms, nlp, mpc):
    """The headline figures, compact, for the end of the JSON line."""
    def pick(d, key):
        return {k: v[key] for k, v in d.items()
                if isinstance(v, dict) and key in v and k != "training"}
    out = {"tti_1e-6_s": pick(tti, "s")}
    if isinstance(tti.get("fp64_tc"), dict) and "fma_path_s_estimate" in tti["fp64_tc"]:
        out["tti_1e-6_s"]["fp64_fma_estimate"] = tti["fp64_tc"]["fma_path_s_estimate"]
    t = out["tti_1e-6_s"]
    if "fp64_tc" in t and "tf32_then_tf32x3" in t:
        out["fp64_tc_over_ladder"] = round(t["fp64_tc"] / t["tf32_then_tf32x3"], 2)
    if isinstance(tti.get("fp64_tc"), dict) and "factor_tflops_fp64_equiv" in tti["fp64_tc"]:
        out["fp64_tc_factor_tflops"] = tti["fp64_tc"]["factor_tflops_fp64_equiv"]
    if forms:
        out["forms_48_s"] = pick(forms, "seconds")
    if nlp:
        out["grid_nlp_s"] = pick(nlp, "seconds")
    if mpc:
        out["mpc_solves_per_s"] = {k: v["solves_per_s"] for k, v in mpc.items()
                                   if isinstance(v, dict) and "solves_per_s" in v}
    return out


def run_ours(args, ws, rank):
    import torch
    import paper_2508_16094_gb300 as gb

    if ws != 1 or args.gpus != 1:
        # one factorisation per iteration on one GPU: there is nothing to shard
        if rank == 0:
            print(json.dumps({"metric": METRIC, "error": "single-GPU method: bench.py runs on "
                              "one GPU only (--gpus 1, no torchrun)"}), flush=True)
        sys.exit(2)
    gb.build()
    torch.cuda.set_device(0)
    pk, pk_src = peaks()
    prec = PREC[args.precision]
    G = args.grid
    lp = gen.grid_lp(G, seed=1)
    perm = gen.nd_order_grid3d(G)
    opts = gb.default_options(precision=prec, tol=1e-6, storage_fp64=1 if prec == 0 else 0)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u, options=opts)
    t0 = time.perf_counter()
    info = ctx.kkt_analyze(perm)
    t_analyze = time.perf_counter() - t0
    ctx.ipm_set_workspace()
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    jv, b, c = dev(lp.val), dev(lp.b), dev(lp.c)
    mt = ctx.m_tot
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    s = torch.empty(mt, dtype=torch.float64, device="cuda")
    lam = torch.empty(mt, dtype=torch.float64, device="cuda")

    # the iterations of the cold-start solve to 1e-6, recorded once
    traj, rlast = record_trajectory(ctx, jv, b, c, x, s, lam)
    T = len(traj)

    def restore(i):
        xi, si, li = traj[i % T]
        x.copy_(xi)
        s.copy_(si)
        lam.copy_(li)

    # step k = iteration (k mod T) of that solve, from its own starting iterate
    ctx.ipm_set_options(max_iter=1, warm_start=1, tol=1e-6)
    for k in range(args.warmup):
        restore(k)
        ctx.ipm_solve(jv, b, c, x, s, lam)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    l0 = gb.kernel_launches()
    pcg = refine = 0
    fac_ms = sol_ms = 0.0
    with ClockSampler(0) as clk:
        ev0.record(stream)
        for k in range(args.steps):
            restore(k)
            r = ctx.ipm_solve(jv, b, c, x, s, lam)
            pcg += r.pcg_steps
            refine += r.refine_steps
            fac_ms += r.time_factor_ms
            sol_ms += r.time_solve_ms
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = gb.kernel_launches() - l0
    ms = ev0.elapsed_time(ev1)
    value = info.flops * args.steps / (ms * 1e-3) / 1e12

    # end to end through the C ABI with host buffers: every step copies its
    # inputs (J values, b, c and the starting iterate) from pinned host memory,
    # runs the same iteration and reads the new iterate back
    hj, hb, hc = (t.cpu().pin_memory() for t in (jv, b, c))
    htraj = [tuple(t.cpu().pin_memory() for t in it) for it in traj]
    hout = [torch.empty_like(t).pin_memory() for t in (htraj[0])]
    h2d = 8 * (jv.numel() + b.numel() + c.numel() + x.numel() + s.numel() + lam.numel())
    d2h = 8 * (x.numel() + s.numel() + lam.numel())
    torch.cuda.synchronize()
    ev0.record(stream)
    for k in range(args.steps):
        hx, hs, hl = htraj[k % T]
        for dst, src in ((jv, hj), (b, hb), (c, hc), (x, hx), (s, hs), (lam, hl)):
            dst.copy_(src, non_blocking=True)
        ctx.ipm_solve(jv, b, c, x, s, lam)
        for dst, src in zip(hout, (x, s, lam)):
            dst.copy_(src, non_blocking=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = ev0.elapsed_time(ev1)
    e2e_val = info.flops * args.steps / (e2e_ms * 1e-3) / 1e12

    # the factorisation chain alone (all launches of kkt_factor, both streams),
    # CUDA events on the library's stream
    restore(T // 2)
    ctx.ipm_solve(jv, b, c, x, s, lam)  # leaves K of a mid-trajectory iterate assembled
    fts = []
    for _ in range(2):
        ev0.record(stream)
        ctx.kkt_factor(prec)
        ev1.record(stream)
        torch.cuda.synchronize()
        fts.append(ev0.elapsed_time(ev1))
    t_fac = float(np.mean(fts))
    achieved = info.flops / (t_fac * 1e-3) / 1e12
    # peak of the contraction's dtype: measured BF16 burst x nominal ratio
    # (TF32 = 0.5); the split's three TF32 products are the implementation's
    # work, reported beside it as the tensor pipe's product rate
    ratio = {0: None, 1: None, 2: 0.5, 3: 1.0, 4: 0.5}[prec]
    if ratio is not None:
        peak = pk["bf16_tflops"] * ratio
        bound = "tensor"
        peak_note = f"{pk_src} bf16 burst x {ratio:g}" + (" (tf32)" if ratio == 0.5 else "")
    elif prec == 1:
        peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        bound, peak_note = "alu", "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"
    else:
        peak = 1.25
        bound, peak_note = "alu", "nominal FP64 rate (1.25 TFLOP/s)"
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": FACTOR_TRAFFIC.get((G, args.precision)),
            "kernel": "supernodal factorisation (all launches of kkt_factor)",
            "peak_source": peak_note, "duration_ms": round(t_fac, 3),
            "work": "sum over columns of colcount^2 (algorithmic)"}
    if prec == 4:
        roof["products_frac"] = 3 * achieved / peak

    # HBM rooflines of the solve and the assembly kernels, algorithmic bytes:
    # solve 2 x 4 B per entry of L (nnz(L): both sweeps read the factor once)
    # plus its three FP32 vectors; assembly 8 B per J value, per D entry and
    # per K entry written
    hbm = pk["hbm_gbs"]
    extra_roof = {}
    if prec != 0:
        t_sol = ctx.kkt_time_kernel(1, reps=5)
        sb = 2 * 4 * info.nnz_l + 4 * 3 * lp.n  # both sweeps read L once; a, b, x
        extra_roof["psolve_kernel"] = {"bound": "hbm", "achieved": sb / (t_sol * 1e-3) / 1e9,
                                       "peak": hbm, "unit": "GB/s",
                                       "frac": sb / (t_sol * 1e-3) / 1e9 / hbm,
                                       "ms": round(t_sol, 4), "bytes": sb}
    t_as = ctx.kkt_time_kernel(0, reps=5)
    ab = 8 * (int(lp.rowptr[-1]) + mt + info.nnz_k)
    extra_roof["assemble_kernel"] = {"bound": "hbm", "achieved": ab / (t_as * 1e-3) / 1e9,
                                     "peak": hbm, "unit": "GB/s",
                                     "frac": ab / (t_as * 1e-3) / 1e9 / hbm,
                                     "ms": round(t_as, 4), "bytes": ab}

    # time to a 1e-6 KKT residual from the cold start, every precision of the
    # factor on the 100^3 grid (the FP64 path in a context of its own, below)
    tti = {"workload": f"grid LP {G}^3 cold start to KKT <= 1e-6"}
    if args.tti:
        tti[args.precision] = tti_run(ctx, jv, b, c, x, s, lam, prec)
        ref = tti[args.precision]["obj"]
        for name in args.tti_forms.split(","):
            if not name or name == args.precision or name == "fp64":
                continue
            try:
                if name in LADDERS:
                    p0, esc = LADDERS[name]
                    tti[name] = tti_run(ctx, jv, b, c, x, s, lam, p0, ref, cg_escalate=esc)
                else:
                    tti[name] = tti_run(ctx, jv, b, c, x, s, lam, PREC[name], ref)
            except Exception as e:  # an unsupported precision is reported, not fatal
                tti[name] = {"error": str(e)[:120]}
        ctx.ipm_set_options(cg_escalate=0)
        if args.fp64_tc_tti:
            tti["fp64_tc"] = tti_fp64_tc(lp, perm, jv, b, c, ref, pk["bf16_tflops"])

    mpc = mpc_measure() if not args.no_mpc else None
    forms = forms_measure(args.forms_grid) if args.forms_grid > 0 else None
    nlp = nlp_measure(args.nlp_grid) if args.nlp_grid > 0 else None

    cpu = None
    if not args.no_cpu_baseline:
        sec, oflops, on = oracle_direction_sample(ORACLE_GRID, reps=3)
        cpu = {"value": oflops / sec / 1e12, "unit": "TFLOP/s", "cores": 1,
               "host_cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one oracle Newton direction (assembly, left-looking Cholesky, solves) "
                         f"on the {ORACLE_GRID}^3 member of the grid-LP family (n={on}), "
                         f"{sec:.1f} s on 1 of {os.cpu_count()} host cores"}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": f"grid LP {G}^3 (n=m={lp.n}, 7-point rows, N(0,1)+8 diagonal, "
                               f"bounds [0,10], ND ordering); step k = iteration k mod {T} of "
                               f"the cold-start solve to KKT <= 1e-6, from its own iterate",
                   "precision": args.precision, "parallelism": "single GPU",
                   "l2": "inputs larger than L2 (factor storage "
                         f"{info.factor_entries * (8 if prec == 0 else 4) / 1e9:.1f} GB)",
                   "factor_flops": info.flops, "nnz_l": info.nnz_l, "nsuper": info.nsuper,
                   "levels": info.nlevels, "analyze_s": round(t_analyze, 2),
                   "trajectory_iterations": T},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "mpc_batch": mpc,
        "grid_nlp": nlp,
        "time_to_kkt_1e-6_forms": forms,
        "rooflines_hbm": extra_roof,
        "ipm_step": {"pcg_steps": pcg / args.steps, "refine_steps": refine / args.steps,
                     "factor_ms": fac_ms / args.steps, "solve_ms": sol_ms / args.steps},
        "time_to_kkt_1e-6": tti,
    }
    line["summary"] = summary(tti, forms, nlp, mpc)  # last: the headline figures in the line's tail
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--learned-sweep", type=int, default=0, metavar="G",
                    help="only run the learned correction's seed sweep on the G^3 grid-LP family "
                         "(64 training and 16 held-out seeds) and print its JSON line")
    ap.add_argument("--no-fp64-tc-tti", dest="fp64_tc_tti", action="store_false",
                    help="skip the FP64 (tensor-core updates) time to 1e-6 on the bench grid")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--grid", type=int, default=100)
    ap.add_argument("--precision", choices=list(PREC), default="tf32x3")
    ap.add_argument("--no-tti", dest="tti", action="store_false")
    ap.add_argument("--tti-forms", default="tf32,bf16,tf32_then_tf32x3",
                    help="other factor precisions timed to 1e-6 on the bench grid")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mpc", action="store_true")
    ap.add_argument("--nlp-grid", type=int, default=512,
                    help="grid of the NLP comparison (0: skip)")
    ap.add_argument("--forms-grid", type=int, default=48,
                    help="grid of the FP64 / split-TF32 / learned time-to-1e-6 comparison (0: skip)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    ws, rank = world()
    if args.learned_sweep > 0:
        import paper_2508_16094_gb300 as gb
        gb.build()
        print(json.dumps({"learned_sweep": learned_sweep(args.learned_sweep)}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, ws, rank)


if __name__ == "__main__":
    main()
