"""Benchmark: one interior-point iteration on the 100^3 grid LP per step.

A step is one pass of the whole hot path on one GPU: constraint evaluation,
scaling D, assembly of the condensed matrix K = J^T D J + delta I, supernodal
Cholesky, predictor and corrector solves with FP64 refinement, direction
recovery, fraction-to-the-boundary step lengths, barrier update and the KKT
convergence test. The metric is throughput in algorithmic factor flops
(sum over columns of colcount^2) per second of step time, plus the
time-to-1e-6 KKT residual of a full solve.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs are independent replicas (one solve per GPU, no collective on
the data path): value = flops of all ranks / max over ranks of the time.
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
        out[name] = {"ms_per_batch": t, "solves_per_s": mb.count / (t * 1e-3),
                     "converged": int((st == 0).sum()), "max_kkt": float(b.kkt.max().item()),
                     "mean_iters": float(b.iters.float().mean().item()),
                     "instances_per_cta": int(cfg.instances_per_cta), "ctas": int(cfg.ctas),
                     "autotune_ms": [round(x, 3) for x in ms]}
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

    def mk(**kw):
        ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u,
                            options=gb.default_options(tol=1e-6, max_iter=200, **kw))
        ctx.kkt_analyze(perm)
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
        return {"seconds": time.perf_counter() - t0, "status": int(r.status),
                "iterations": int(r.iterations), "factorizations": int(r.factorizations),
                "learned_skips": int(r.learned_skips), "pcg_steps": int(r.pcg_steps),
                "refine_steps": int(r.refine_steps), "kkt": r.kkt, "objective": r.objective,
                "time_factor_s": r.time_factor_ms / 1e3, "time_solve_s": r.time_solve_ms / 1e3}

    out = {"workload": f"grid LP {G}^3 (n={lp.n}), seed {seed}; network trained on seeds "
                       f"{list(train_seeds)} of the same family"}
    c64 = mk(precision=gb.IPM_FP64, storage_fp64=1)
    run(c64, max_iter=1)  # first-touch of the workspace and graphs
    out["fp64"] = run(c64, max_iter=200)
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
    for k in ("tf32x3", "tf32x3_learned", "tf32x3_stale_E0"):
        out[k]["objective_rel_diff_vs_fp64"] = abs(out[k]["objective"] - ref) / max(1.0, abs(ref))
    return out


def nlp_measure(N: int, max_iter: int = 60):
    """Grid NLP (512^2 grid, cubic PDE constraint as inequality pairs, -1 <= v <= 1):
    the FP64 factor against the split-TF32 factor with FP64 fallback, from the
    cold start, at most max_iter iterations towards a 1e-6 KKT residual."""
    import torch
    import paper_2508_16094_gb300 as gb
    P = gen.grid_nlp(N, seed=5)
    perm = gen.nd_order_grid_nlp(N)
    ut = torch.as_tensor(P.ut, dtype=torch.float64, device="cuda")
    out = {"workload": f"grid NLP {N}^2 (n = m = {P.n}), alpha 5e-3, |v| <= 1, seed 5",
           "max_iter": max_iter}
    for name, prec in (("fp64", gb.IPM_FP64), ("tf32x3", gb.IPM_TF32X3)):
        o = gb.default_options(precision=prec, tol=1e-6, max_iter=max_iter, storage_fp64=1,
                               fallback_fp64=1)
        G = gb.GridNLP(N, perm=perm, options=o)
        n, mt = G.pat["n"], G.ctx.m_tot
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        s = torch.empty(mt, dtype=torch.float64, device="cuda")
        lam = torch.empty(mt, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = G.ipm_solve_grid_nlp(ut, x, s, lam)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "status": int(r.status),
                     "iterations": int(r.iterations), "objective": r.objective, "kkt": r.kkt,
                     "primal": r.primal_res, "dual": r.dual_res, "fp64_fallbacks": int(r.fp64_fallbacks),
                     "regularizations": int(r.regularizations), "refine_steps": int(r.refine_steps),
                     "factor_flops": G.info.flops}
        G.ctx.close()
    out["objective_rel_diff_tf32x3_vs_fp64"] = abs(out["tf32x3"]["objective"] - out["fp64"]["objective"]) / max(1.0, abs(out["fp64"]["objective"]))
    return out


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, ws, rank):
    """The oracle as it stands, on the host cores: each step one Newton direction
    of the 24^3 member of the grid-LP family."""
    if rank != 0:
        return
    t_w = [oracle_direction_sample(ORACLE_GRID)[0] for _ in range(args.warmup)]
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
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": f"one oracle Newton direction (assembly, left-looking "
                                       f"Cholesky, solves) on the {ORACLE_GRID}^3 grid LP, "
                                       f"n={n}"},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    del t_w
    print(json.dumps(line), flush=True)


def run_ours(args, ws, rank, local):
    import torch
    import paper_2508_16094_gb300 as gb

    gb.build()
    torch.cuda.set_device(local)
    pk, pk_src = peaks()
    prec = PREC[args.precision]
    G = args.grid
    lp = gen.grid_lp(G, seed=1 + (rank if args.vary_seed else 0))
    perm = gen.nd_order_grid3d(G)
    opts = gb.default_options(precision=prec, tol=1e-6, max_iter=args.warmup,
                              storage_fp64=1 if prec == 0 else 0)
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
    # warm-up iterations from the cold start
    ctx.ipm_set_options(max_iter=args.warmup, warm_start=0)
    ctx.ipm_solve(jv, b, c, x, s, lam)
    torch.cuda.synchronize()
    # timed iterations, continuing from the warm-up iterate
    ctx.ipm_set_options(max_iter=args.steps, warm_start=1, tol=0.0)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    l0 = gb.kernel_launches()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        res = ctx.ipm_solve(jv, b, c, x, s, lam)
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = gb.kernel_launches() - l0
    barrier(ws)
    ms = ev0.elapsed_time(ev1)
    steps_done = max(res.iterations, 1)
    ms_max = max_over_ranks(ws, ms)
    value = info.flops * steps_done * ws / (ms_max * 1e-3) / 1e12

    # factorisation alone (the dominant kernel chain), CUDA events on the same stream
    fts = []
    for _ in range(2):
        ev0.record(stream)
        ctx.kkt_factor(prec)
        ev1.record(stream)
        torch.cuda.synchronize()
        fts.append(ev0.elapsed_time(ev1))
    t_fac = float(np.mean(fts))
    achieved = info.flops / (t_fac * 1e-3) / 1e12
    if prec in (2, 3, 4):
        # tensor-core contraction: measured BF16 peak x nominal TF32/BF16 ratio (0.5);
        # the 3-term split issues three TF32 products per algorithmic one
        ratio = {2: 0.5, 3: 1.0, 4: 0.5 / 3.0}[prec]
        peak = pk["bf16_tflops"] * ratio
        bound = "tensor"
        peak_note = f"{pk_src} bf16 burst x {ratio:.4g}" + {2: " (tf32)", 3: "", 4: " (tf32, 3 products per flop)"}[prec]
    elif prec == 1:
        # FP32 FMA pipe: 152 SMs x 128 lanes x 2 flops x max SM clock
        peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        bound, peak_note = "alu", "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"
    else:
        peak = 1.25
        bound, peak_note = "alu", "nominal FP64 rate (1.25 TFLOP/s)"

    # end to end through the C ABI with host buffers: H2D of the step's inputs
    # (J values, b, c and the iterate) from pinned memory, one iteration, D2H
    # of the new iterate
    host = {k: t.cpu().pin_memory() for k, t in dict(jv=jv, b=b, c=c, x=x, s=s, lam=lam).items()}
    hout = {k: torch.empty_like(host[k]).pin_memory() for k in ("x", "s", "lam")}
    h2d = sum(t.numel() * 8 for t in host.values())
    d2h = sum(t.numel() * 8 for t in hout.values())
    ctx.ipm_set_options(max_iter=1)
    e2e_ms = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in host:
            {"jv": jv, "b": b, "c": c, "x": x, "s": s, "lam": lam}[k].copy_(host[k], non_blocking=True)
        r1 = ctx.ipm_solve(jv, b, c, x, s, lam)
        hout["x"].copy_(x, non_blocking=True)
        hout["s"].copy_(s, non_blocking=True)
        hout["lam"].copy_(lam, non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(ev0.elapsed_time(ev1) / max(r1.iterations, 1))
    e2e_val = info.flops * ws / (max_over_ranks(ws, float(np.mean(e2e_ms))) * 1e-3) / 1e12

    # time to a 1e-6 KKT residual from the cold start
    tti = None
    if args.tti:
        ctx.ipm_set_options(max_iter=200, warm_start=0, tol=1e-6)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rt = ctx.ipm_solve(jv, b, c, x, s, lam)
        torch.cuda.synchronize()
        tti = {"seconds": time.perf_counter() - t0, "status": int(rt.status),
               "iterations": int(rt.iterations), "kkt": rt.kkt, "objective": rt.objective,
               "refine_steps": int(rt.refine_steps), "pcg_steps": int(rt.pcg_steps),
               "fp64_fallbacks": int(rt.fp64_fallbacks),
               "time_factor_s": rt.time_factor_ms / 1e3, "time_solve_s": rt.time_solve_ms / 1e3}

    mpc = None
    if rank == 0 and not args.no_mpc:
        mpc = mpc_measure()
    forms = None
    if rank == 0 and args.forms_grid > 0:
        forms = forms_measure(args.forms_grid)
    nlp = None
    if rank == 0 and args.nlp_grid > 0:
        nlp = nlp_measure(args.nlp_grid)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        sec, oflops, on = oracle_direction_sample(ORACLE_GRID, reps=3)
        cpu = {"value": oflops / sec / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
               "sample": f"one oracle Newton direction (assembly, left-looking Cholesky, solves) "
                         f"on the {ORACLE_GRID}^3 member of the grid-LP family (n={on}), "
                         f"{sec:.1f} s on one host core"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
            "steps": steps_done, "warmup": args.warmup, "ms_per_step": ms_max / steps_done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": f"grid LP {G}^3 (n=m={lp.n}, 7-point rows, N(0,1)+8 diagonal, "
                                   f"bounds [0,10], ND ordering), one IPM iteration per step",
                       "precision": args.precision, "replicas": ws,
                       "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2 (factor storage "
                             f"{info.factor_entries * (8 if prec == 0 else 4) / 1e9:.1f} GB)",
                       "factor_flops": info.flops, "nnz_l": info.nnz_l, "nsuper": info.nsuper,
                       "levels": info.nlevels, "analyze_s": round(t_analyze, 2)},
            "roofline": {"bound": bound, "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "kernel": "supernodal factorisation (all launches of kkt_factor)",
                         "peak_source": peak_note, "duration_ms": t_fac},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "time_to_kkt_1e-6": tti,
            "mpc_batch": mpc,
            "time_to_kkt_1e-6_forms": forms,
            "grid_nlp": nlp,
            "ipm_step": {"refine_steps": int(res.refine_steps), "pcg_steps": int(res.pcg_steps),
                         "factor_ms": res.time_factor_ms / steps_done,
                         "solve_ms": res.time_solve_ms / steps_done},
        }
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--grid", type=int, default=100)
    ap.add_argument("--precision", choices=list(PREC), default="tf32x3")
    ap.add_argument("--no-tti", dest="tti", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--vary-seed", action="store_true")
    ap.add_argument("--no-mpc", action="store_true")
    ap.add_argument("--nlp-grid", type=int, default=512,
                    help="grid of the NLP comparison (0: skip)")
    ap.add_argument("--forms-grid", type=int, default=48,
                    help="grid of the FP64 / split-TF32 / learned time-to-1e-6 comparison (0: skip)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
