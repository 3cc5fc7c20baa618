"""Benchmark: LS solves/s at relres 1e-8 on one GB300 (mixed precision and
plain FP64), synthetic 2D workload of 256^2 unknowns, omega/2pi = 32.

One step = the whole hot path for one medium and one batch of incident waves:
medium update (moving-PML stencils + slab assembly), factorization of all slab
subproblems + interface maps, right-hand sides g = -omega^2 K(m u_I), flexible
GMRES(30) to relres 1e-8 with the sparsify-and-sweep preconditioner, true
residual.  The per-(n, omega) tables (kernel FFT, alpha/beta, physical PML
stencils) are built once when the solver is created, as the method allows.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun) runs independent replicas (the solve does not shard); rank 0
prints one JSON line.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "LS solves/s at relres 1e-8, mixed+batched vs plain FP64 on one GB300"
WORKLOAD = "2d_n256"
HBM_FALLBACK_GBS = 6800.0
# FP64 / FP32 CUDA-core peaks of a GB300 (derivation in the design notes):
# FP64 1.25 TFLOP/s nominal; FP32 152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return HBM_FALLBACK_GBS, "fallback"


def workload_cfg(name=WORKLOAD):
    w = synth.WORKLOADS[name]
    m, dirs = synth.make_workload(w)
    return w, m, dirs


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.rows, self.proc, self.index = [], None, index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 8:
                for k, v in zip(names, r[4:8]):
                    if v.strip().lower() == "active":
                        reasons.add(k)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ---------------------------------------------------------------- algorithmic work per kernel group
def _levels(K0):
    Ks, K = [], K0
    while K > 1:
        Ks.append(K)
        K = (K + 1) // 2
    return Ks


def cr_solve_work(K0, w, part, rows=None):
    """Complex MACs and factor entries (unpadded w x w blocks) of one cyclic-
    reduction solve of a slab of width w: forward over the rows that can be
    non-zero (all, or a column's neighbourhood for the interface maps), the top
    row, back substitution with only the first and last layers kept at level 0
    when `part`."""
    Ks = _levels(K0)
    w2 = w * w
    mac = ent = 0
    lo, hi = (0, K0 - 1) if rows is None else rows
    for l, K in enumerate(Ks):
        j0, j1 = lo | 1, min(hi, K - 1)
        nodd = (j1 - j0) // 2 + 1 if j0 <= j1 else 0
        e0 = max(0, lo - 1)
        e0 += e0 & 1
        e1 = min(K - 1, hi + 1)
        nev = (e1 - e0) // 2 + 1 if e0 <= e1 else 0
        mac += nodd * w2
        ent += nodd * w2
        per_even = 6 * w if l == 0 else 2 * w2
        mac += nev * per_even
        ent += nev * per_even
        lo, hi = (e0 // 2, e1 // 2) if nev else (1, 0)
    mac += w2
    ent += w2
    for l, K in enumerate(Ks):
        per_odd = (6 * w + (2 * w if part else w2)) if l == 0 else 2 * w2
        mac += (K // 2) * per_odd
        ent += (K // 2) * per_odd
    return mac, ent


def algorithmic(solver, R, prec_bytes):
    """Per-launch algorithmic bytes / flops of each kernel group (design notes,
    section on kernels and rooflines)."""
    n, L, nt, ns = solver.n, solver.fft_len, solver.n_tot, solver.n_slabs
    N = n * n
    ws = []
    for i in range(ns):
        _, nl, na = solver.slab_info(i)
        ws.append(na + nl)
    cb = 2 * prec_bytes
    a_mac = a_ent = e_mac = e_ent = 0
    for w in ws:
        m1, e1 = cr_solve_work(nt, w, True)
        m2, e2 = cr_solve_work(nt, w, False)
        a_mac, a_ent, e_mac, e_ent = a_mac + m1, a_ent + e1, e_mac + m2, e_ent + e2
    # interface maps: all n_tot unit columns of a slab side at once; forward
    # over the column windows of width 2^(l+1) - 1, dense back substitution,
    # then the tridiagonal coupling
    Ks = _levels(nt)
    if_mac = 0
    for side in (0, 1):
        for i in range(1, (ns - 1) if side == 0 else (ns - 2) + 1):
            w = ws[i]
            mac = 0
            for l, K in enumerate(Ks):
                wodd, wev = min(nt, 2 ** (l + 1) - 1), min(nt, 2 ** (l + 2) - 1)
                mac += (K // 2) * wodd * (w * w if l else w)
                mac += ((K + 1) // 2) * wev * (2 * w * w if l else 6 * w)
                mac += (K // 2) * nt * (2 * w * w if l else 8 * w)
            mac += nt * w * w + nt * nt * 3 * (2 if side == 0 else 1)
            if_mac += mac
    fft_flops = R * (n * 5 * L * math.log2(L) + L * 2 * 5 * L * math.log2(L) + n * 5 * L * math.log2(L))
    mv_bytes = R * (16 * N * 2) + 8 * N + 16 * L * L
    recur_bytes = (2 * max(ns - 2, 0) + max(ns - 1, 0)) * nt * nt * cb   # Lambda, Phi chains + Gamma (mu)
    factor_flops = sum(8 * 2 * nt * (3.5 + 4.0) * w ** 3 for w in ws)
    rhs_bytes = R * (nt * nt * cb + 16 * N)
    return {
        "slab_a": dict(bytes=a_ent * cb + rhs_bytes, flops=8 * a_mac * R, launches_per_apply=1),
        "slab_e": dict(bytes=e_ent * cb + rhs_bytes, flops=8 * e_mac * R, launches_per_apply=1),
        # one factorization per step: its launches are the step's iface launches
        "iface": dict(bytes=3 * ns * nt * nt * cb, flops=8 * if_mac, launches_per_apply=None),
        "matvec": dict(bytes=mv_bytes, flops=fft_flops, launches_per_apply=3),
        "recur": dict(bytes=recur_bytes * R, flops=recur_bytes // cb * 8 * R, launches_per_apply=3),
        "factor": dict(bytes=sum(nt * 3 * w * w * cb for w in ws), flops=factor_flops, launches_per_apply=None),
    }


# ---------------------------------------------------------------- our arm
def max_over_ranks(vals, dev, world):
    """Element-wise maximum of per-rank timings over all ranks (one all-reduce;
    a single rank returns its own values)."""
    if world <= 1:
        return [float(v) for v in vals]
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def run_ours(args, rank, world):
    import torch
    from paper_1705_09443_gb300 import GmresOptions, LSS_FP64, LSS_MIXED, LSSolver

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w, m, dirs = workload_cfg(args.workload)
    R = dirs.shape[0]
    n = w.n
    mt = torch.tensor(m, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2
    opts = GmresOptions(30, 1e-8, 300)
    results = {}
    arms = [a for a in (("mixed", LSS_MIXED), ("fp64", LSS_FP64)) if a[0] in args.arms.split(",")]
    for prec_name, prec in arms:
        solver = LSSolver(n, w.omega, mt, b_pml=w.b_pml, b_slab=w.b_slab, precision=prec)
        tuned = solver.autotune(R)   # launch parameters for this workload, picked by timing
        stream = torch.cuda.current_stream()

        def step():
            solver.set_medium(mt)
            solver.factor()
            g = solver.plane_wave_rhs(dirs)
            u, st = solver.solve(g, opts)
            return st

        for _ in range(args.warmup):
            st = step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clk = ClockSampler(dev.index)
        clk.start()
        total_ms = 0.0
        stats = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = step()
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            stats.append(st)
        torch.cuda.synchronize()
        clocks = clk.stop()
        # per-kernel-group breakdown and launch counts: the same steps again with
        # CUDA events around every kernel group (iterations then run launch by
        # launch, not from their graphs), outside the timed region
        solver.profile_read()
        solver.profile(True)
        for _ in range(args.steps):
            flush.zero_()
            step()
        solver.profile(False)
        prof_ms, prof_n = solver.profile_read()
        torch.cuda.synchronize()
        total_ms, = max_over_ranks([total_ms], dev, world)
        iters = [s["iters"] for st in stats for s in st]
        relres = max(s["relres_true"] for st in stats for s in st)
        conv = all(s["relres_true"] <= 1e-8 for st in stats for s in st)
        res = dict(value=(R * args.steps * world) / (total_ms / 1e3), ms_per_step=total_ms / args.steps,
                   iters=float(np.mean(iters)), relres_true_max=relres, converged=conv, clocks=clocks,
                   prof_ms={k: v / args.steps for k, v in prof_ms.items()},
                   prof_launches={k: v // args.steps for k, v in prof_n.items()},
                   gpu_launches=int(sum(prof_n.values())), solver=solver, autotune=tuned,
                   prec_bytes=8 if prec == LSS_FP64 else 4)
        # solve only (the metric's lss_solve time): factors in place, right-hand side resident
        solver.set_medium(mt)
        solver.factor()
        g = solver.plane_wave_rhs(dirs)
        for _ in range(args.warmup):
            solver.solve(g, opts)
        solve_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.solve(g, opts)
            e1.record(stream)
            e1.synchronize()
            solve_ms += e0.elapsed_time(e1)
        setup_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.set_medium(mt)
            solver.factor()
            e1.record(stream)
            e1.synchronize()
            setup_ms += e0.elapsed_time(e1)
        solve_ms, setup_ms = max_over_ranks([solve_ms, setup_ms], dev, world)
        graphs = solver.graph_count()
        # the same solves with every kernel launched one by one (no iteration graphs)
        solver.use_graphs(False)
        for _ in range(args.warmup):
            solver.solve(g, opts)
        nog_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.solve(g, opts)
            e1.record(stream)
            e1.synchronize()
            nog_ms += e0.elapsed_time(e1)
        solver.use_graphs(True)
        res["solve_only"] = {"value": (R * args.steps * world) / (solve_ms / 1e3), "unit": "solves/s",
                             "ms_per_solve_call": solve_ms / args.steps,
                             "iteration_graphs": {"captured": graphs[0], "refused": graphs[1]},
                             "without_iteration_graphs": {"value": (R * args.steps * world) / (nog_ms / 1e3),
                                                          "ms_per_solve_call": nog_ms / args.steps}}
        res["setup_factor_ms"] = setup_ms / args.steps
        # e2e: medium from pinned host memory, solution back to pinned host memory
        m_host = torch.tensor(m, dtype=torch.float64).pin_memory()
        u_host = torch.empty((R, n, n), dtype=torch.complex128).pin_memory()
        m_dev = torch.empty_like(mt)
        e2e_ms = 0.0
        for k in range(args.warmup + args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m_dev.copy_(m_host, non_blocking=True)
            solver.set_medium(m_dev)
            solver.factor()
            g = solver.plane_wave_rhs(dirs)
            u, st = solver.solve(g, opts)
            u_host.copy_(u, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            if k >= args.warmup:
                e2e_ms += e0.elapsed_time(e1)
        e2e_ms, = max_over_ranks([e2e_ms], dev, world)
        res["e2e"] = {"value": (R * args.steps * world) / (e2e_ms / 1e3), "unit": "solves/s",
                      "h2d_bytes_per_step": int(n * n * 8 + R * 16), "d2h_bytes_per_step": int(R * n * n * 16)}
        results[prec_name] = res
    if args.batched and "mixed" in results:
        results["batched"] = run_batched(args, dev, world)
    if args.ragged and "mixed" in results:
        results["ragged"] = run_ragged(args, dev, world)
    return w, R, results


def run_batched(args, dev, world):
    """Form (2), batching: the same medium with R plane waves per solve call, in
    mixed precision (set-up + factor + R-RHS solve per step); against it the
    plain FP64 arm above solves one right-hand side per call."""
    import torch
    from paper_1705_09443_gb300 import GmresOptions, LSS_MIXED, LSSolver
    wb, m, dirs = workload_cfg(args.batched)
    R = dirs.shape[0]
    mt = torch.tensor(m, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    opts = GmresOptions(30, 1e-8, 300)
    solver = LSSolver(wb.n, wb.omega, mt, b_pml=wb.b_pml, b_slab=wb.b_slab, precision=LSS_MIXED)
    tuned = solver.autotune(R)
    stream = torch.cuda.current_stream()

    def step():
        solver.set_medium(mt)
        solver.factor()
        g = solver.plane_wave_rhs(dirs)
        return solver.solve(g, opts)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    total = 0.0
    stats = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = step()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
        stats.append(st)
    g = solver.plane_wave_rhs(dirs)
    solve_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.solve(g, opts)
        e1.record(stream)
        e1.synchronize()
        solve_ms += e0.elapsed_time(e1)
    total, solve_ms = max_over_ranks([total, solve_ms], dev, world)
    # per-group breakdown of one step, outside the timed region
    solver.profile_read()
    solver.profile(True)
    step()
    solver.profile(False)
    prof_ms, _ = solver.profile_read()
    relres = max(s["relres_true"] for st in stats for s in st)
    return {"workload": args.batched, "R": R, "autotune": tuned, "breakdown_ms": prof_ms,
            "value": R * args.steps * world / (total / 1e3),
            "unit": "solves/s", "ms_per_step": total / args.steps,
            "solve_only": {"value": R * args.steps * world / (solve_ms / 1e3), "ms_per_solve_call": solve_ms / args.steps},
            "iters_mean": float(np.mean([s["iters"] for st in stats for s in st])), "relres_true_max": relres,
            "converged": all(s["relres_true"] <= 1e-8 for st in stats for s in st)}


def run_ragged(args, dev, world):
    """Form (2), ragged instances: independent problems with n uniform on
    {128..384}, omega/2pi = n/8, band-limited media, one plane wave each, all
    behind one batch context (instances run concurrently); against it the same
    instances solved one after another, each by its own context.  Mixed
    precision; a step is factor + plane-wave RHS + solve of every instance."""
    import torch
    from paper_1705_09443_gb300 import GmresOptions, LSS_MIXED, LSSolver, LSSolverBatch
    spec = dict(synth.RAGGED_32, count=args.ragged)
    ns = synth.ragged_sizes(**spec)
    inst = synth.ragged_instances(ns, spec["seed"])
    ms = [torch.tensor(m, dtype=torch.float64, device=dev) for _, m, _ in inst]
    oms = [2 * math.pi * f for f, _, _ in inst]
    dirs = np.stack([d for _, _, d in inst])
    opts = GmresOptions(30, 1e-8, 300)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    batch = LSSolverBatch(ns, oms, ms, precision=LSS_MIXED)
    batch.autotune(1)
    single = [LSSolver(n, om, m, precision=LSS_MIXED) for n, om, m in zip(ns, oms, ms)]
    for s in single:
        s.autotune(1)

    def step_batch():
        batch.factor()
        return batch.solve(batch.plane_wave_rhs(dirs), opts)[1]

    def step_seq():
        st = []
        for s, d in zip(single, dirs):
            s.factor()
            st.append(s.solve(s.plane_wave_rhs(d), opts)[1])
        return st

    out = {}
    for name, step in (("batch", step_batch), ("sequential", step_seq)):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        total, stats = 0.0, []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats.append(step())
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        total, = max_over_ranks([total], dev, world)
        flat = [x for st in stats for q in st for x in q]
        out[name] = {"value": len(ns) * args.steps * world / (total / 1e3), "ms_per_step": total / args.steps,
                     "iters_mean": float(np.mean([x["iters"] for x in flat])),
                     "relres_true_max": max(x["relres_true"] for x in flat),
                     "converged": all(x["relres_true"] <= 1e-8 for x in flat)}
    del batch, single
    return {"instances": len(ns), "n": ns, "unit": "instances solved/s",
            "step": "factor + plane-wave RHS + FGMRES solve of every instance (mixed precision)",
            **out["batch"], "sequential": out["sequential"],
            "batch_over_sequential": out["batch"]["value"] / out["sequential"]["value"]}


# DRAM traffic per launch group from ncu captures (profiles/iface_maps_2d_n256_mixed.md):
# key (kernel group, workload, precision).  Stale once those kernels change.
MEASURED_TRAFFIC = {("iface", "2d_n256", "mixed"): 2.444e9}


def roofline(res, hbm_peak, hbm_src, workload="2d_n256", prec="mixed"):
    """Roofline of the kernel group that takes the most time in the timed
    steps: algorithmic work per launch over its CUDA-event time per launch."""
    solver = res["solver"]
    alg = algorithmic(solver, 1, res["prec_bytes"])
    cats = {k: v for k, v in res["prof_ms"].items() if k in alg}
    dom = max(cats, key=lambda k: cats[k])
    launches = max(res["prof_launches"].get(dom, 1), 1)
    a = alg[dom]
    per = a["launches_per_apply"] or launches
    per_apply_ms = cats[dom] / max(launches // per, 1)
    if dom in ("recur", "slab_a", "slab_e"):
        achieved = a["bytes"] / (per_apply_ms / 1e3) / 1e9
        return dom, {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": None, "peak_source": hbm_src,
                     "per_launch_ms": per_apply_ms}
    achieved = a["flops"] / (per_apply_ms / 1e3) / 1e12
    peak = FP64_PEAK_TFLOPS if (res["prec_bytes"] == 8 or dom == "matvec") else FP32_PEAK_TFLOPS
    return dom, {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                 "traffic": MEASURED_TRAFFIC.get((dom, workload, prec)), "traffic_per": "one factorization",
                 "per_launch_ms": per_apply_ms,
                 "peak_source": "derived: FP64 1.25 TFLOP/s nominal; FP32 = 152 SMs x 128 FMA/clk x 2 x 2.07 GHz"}


# ---------------------------------------------------------------- oracle (CPU) arm
ORACLE_SNIPPET = r"""
import json, sys, time, math
sys.path.insert(0, {root!r})
import numpy as np
import synth
from oracle import lss_oracle as O
w = synth.WORKLOADS[{wl!r}]
m, dirs = synth.make_workload(w)
ts = []
for k in range({reps}):
    t0 = time.perf_counter()
    res, relres, pb, g = O.solve(w.n, w.omega, m, dirs[0], O.Params(b_pml=w.b_pml, b_slab=w.b_slab), tol=1e-8)
    ts.append(time.perf_counter() - t0)
print(json.dumps(dict(times=ts, iters=res.iters, relres=relres)))
"""


def run_oracle(wl, reps):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, wl=wl, reps=reps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched", default="2d_n256_r16",
                    help="workload of the batched mixed-precision line ('' to skip)")
    ap.add_argument("--ragged", type=int, default=32,
                    help="instances of the ragged batch line (0 to skip)")
    ap.add_argument("--arms", default="mixed,fp64",
                    help="precisions to run (mixed first; the JSON line needs both, profiling may take one)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    w = synth.WORKLOADS[args.workload]
    config = {"workload": f"2D LS, n={w.n} (N={w.n * w.n}), omega/2pi={w.freq:g}, {w.n_gauss} Gaussians "
                          f"width {w.width} c in {list(w.c_range)}, {w.n_rhs} plane wave(s), PML {w.b_pml}, "
                          f"slab {w.b_slab}, GMRES(30) tol 1e-8",
              "l2": "flushed (256 MB write) before every timed step",
              "per_omega_tables": "built once at solver creation (kernel FFT, alpha/beta, physical PML stencils)"}

    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.time()
        reps = max(1, min(args.steps, 2))
        out = run_oracle(args.workload, reps)
        v = 1.0 / float(np.mean(out["times"]))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
                "steps": reps, "warmup": 0, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                 "sample": f"{reps} full oracle solve(s) (setup + GMRES to 1e-8) of the benchmark "
                                           f"workload, numpy/scipy single thread"},
                "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "oracle_iters": out["iters"], "wall_s": time.time() - t0}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    cpu = None
    w, R, results = run_ours(args, rank, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle runs in a fresh interpreter (fork + exec), after the GPU timing
        out = run_oracle(args.workload, 1)
        cpu = {"value": 1.0 / out["times"][0], "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": "one full oracle solve (setup + GMRES to 1e-8) of the benchmark workload, "
                         "numpy/scipy, single thread", "oracle_iters": out["iters"]}
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    hbm, src = peaks()
    if "mixed" not in results or "fp64" not in results:
        for name, r in results.items():
            if name in ("batched", "ragged"):
                print(json.dumps({"leg": name, **r}))
                continue
            print(json.dumps({"arm": name, "value": r["value"], "ms_per_step": r["ms_per_step"],
                              "breakdown_ms": r["prof_ms"], "launches_per_step": r["prof_launches"]}))
        return
    mix, f64 = results["mixed"], results["fp64"]
    dom, roof = roofline(mix, hbm, src, args.workload, "mixed")
    line = {
        "metric": METRIC, "value": mix["value"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mix["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64 sweep / f64 matvec+Arnoldi", "data": "synthetic",
        "config": config, "e2e": mix["e2e"], "gpu_launches": mix["gpu_launches"],
        "clocks": mix["clocks"], "roofline": dict(kernel=dom, **roof), "cpu_baseline": cpu,
        "iters": mix["iters"], "relres_true_max": mix["relres_true_max"],
        "step": "set_medium + factor (setup) + plane-wave RHS + FGMRES solve, per medium and batch",
        "solve_only": mix["solve_only"], "setup_factor_ms": mix["setup_factor_ms"], "autotune": mix["autotune"],
        "plain_fp64": {"value": f64["value"], "ms_per_step": f64["ms_per_step"], "iters": f64["iters"],
                       "relres_true_max": f64["relres_true_max"], "e2e": f64["e2e"],
                       "solve_only": f64["solve_only"], "setup_factor_ms": f64["setup_factor_ms"],
                       "breakdown_ms": f64["prof_ms"], "clocks": f64["clocks"]},
        "mixed_over_fp64": mix["value"] / f64["value"],
        "batched": (dict(results["batched"], vs_plain_fp64=results["batched"]["value"] / f64["value"],
                         solve_only_vs_plain_fp64=results["batched"]["solve_only"]["value"]
                         / f64["solve_only"]["value"])
                    if "batched" in results else None),
        "ragged": results.get("ragged"),
        "breakdown_ms": mix["prof_ms"], "launches_per_step": mix["prof_launches"],
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
