"""Benchmark: LS solves/s at relres 1e-8, mixed precision + batching against
plain FP64, on one GB300.

Headline workload: 2D, n = 512 (N = 262144), omega/2pi = 64, band-limited
random medium (c in [0.8, 1.2]), 64 plane waves at angles 2 pi k/64 solved in
one call, FP32 preconditioner (slab factors, sweep) with FP64 operator,
Arnoldi, Givens and true residual.  One step = the whole hot path for one
medium and its batch of waves: medium update (moving-PML stencils + slab
assembly), factorization of all slab subproblems, right-hand sides
g = -omega^2 K(m u_I), flexible GMRES(30) to relres 1e-8, true residual.  The
per-(n, omega) tables (kernel FFT, alpha/beta, physical PML stencils) are built
once when the solver is created, as the method allows (Sec. 2.4 remark 3).

Against it: plain FP64 on the same workload, one right-hand side per solve call
(factorization once per medium).  Further legs: the n = 256 single-wave
workload in both precisions, the 3D n = 64 workload in both precisions, and 32
ragged instances in one batch context.

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
WORKLOAD = "2d_n512_r64"
HBM_FALLBACK_GBS = 6800.0
# CUDA-core peaks of a GB300 (the measured-peaks file holds HBM and bf16 only):
# FP64 1.25 TFLOP/s nominal (an FMA probe on the pool measured 1.19);
# FP32 = 152 SMs x 128 FP32 lanes x 2 flop/FMA x 2.07 GHz = 80.5 TFLOP/s.
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# TF32 tensor rate: half the measured dense bf16 rate (the nominal bf16:tf32
# ratio 2.25 : 1.125 PFLOP/s)
TF32_OVER_BF16 = 0.5


def peaks():
    """(HBM GB/s, bf16 TFLOP/s burst, source) from the measured-peaks file, else
    the fallback figures."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1900.0)), "measured"
        except Exception:
            pass
    return HBM_FALLBACK_GBS, 1900.0, "fallback"


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


# ---------------------------------------------------------------- algorithmic work (the method's, per unit)
def method_work(solver, prec_bytes):
    """The method's own work per unit for each step of the hot path, independent
    of how the kernels organise it:
      matvec    per operator application and right-hand side: compulsory bytes
                16N (u) + 8N (m) + 16N (result) + 16 (L/2+1)^d (the even kernel
                transform's distinct entries); FFT flops 2 * 5 L^d log2(L^d)
      sparsify  per application and right-hand side: 16N in, n_tot^d out
      sweep     per application: the dense block-LU factors D_k^{-1} of every
                slab read twice (forward and backward substitution) by each of
                the 2 l - 1 slab solves of Algorithm 2, sum n_y w^2 (2D, w x w
                blocks) or n_y M^2 (3D, M = w n_tot) entries per slab solve
      factor    per factorization: sum over slabs of n_y (8/3 + 8) b^3 real
                flops, b the block size (w in 2D, M in 3D)
      krylov    per Arnoldi step j (0-based) and right-hand side: the two
                Gram-Schmidt passes read the j + 1 basis vectors twice and
                read/write w: 16 N (4 (j + 1) + 4) bytes
    """
    n, L, nt, ns, d = solver.n, solver.fft_len, solver.n_tot, solver.n_slabs, solver.dim
    N = n ** d
    cb = 2 * prec_bytes
    blocks = []
    for i in range(ns):
        _, nl, na = solver.slab_info(i)
        w = na + nl
        blocks.append(w if d == 2 else w * nt)
    solves = [2] * (ns - 1) + [1]       # slabs 1..l-1 are solved in both sweeps, the last once
    sweep_entries = sum(2 * s * nt * b * b for s, b in zip(solves, blocks))
    return {
        "matvec": {"bytes": 16 * N + 8 * N + 16 * N + 16 * (L // 2 + 1) ** d,
                   "flops": 2 * 5 * L ** d * math.log2(L ** d)},
        "sparsify": {"bytes": 16 * N + cb * nt ** d},
        "sweep": {"bytes": sweep_entries * cb},
        "factor": {"flops": sum(nt * (8.0 / 3.0 + 8.0) * b ** 3 for b in blocks)},
        "krylov_step": lambda j: 16 * N * (4 * (j + 1) + 4),
    }


def group_roofline(solver, res, prec_bytes, R, iters_mean, hbm, bf16, tc=False):
    """Achieved rate of every kernel group of a step against its bound, from the
    per-group CUDA-event times of the profiling pass (ms per step) and the
    method's work per unit (method_work) times the units the step processed."""
    wk = method_work(solver, prec_bytes)
    ms, nl = res["prof_ms"], res["prof_launches"]
    d = solver.dim
    mv_per_call = 3 if d == 2 else 5
    out = {}
    # matvec: calls x R right-hand sides
    calls = nl.get("matvec", 0) / mv_per_call
    if ms.get("matvec", 0) > 0 and calls > 0:
        t = ms["matvec"] / 1e3
        fl = wk["matvec"]["flops"] * calls * R / t / 1e12
        by = wk["matvec"]["bytes"] * calls * R / t / 1e9
        out["matvec"] = {"bound": "alu", "achieved": fl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": fl / FP64_PEAK_TFLOPS, "hbm_GBs": by, "hbm_frac": by / hbm,
                         "units": f"{calls:.0f} operator applications x {R} RHS"}
    applies = nl.get("sparsify", 0) if d == 2 else nl.get("sparsify", 0) / 2
    if ms.get("sparsify", 0) > 0 and applies > 0:
        by = wk["sparsify"]["bytes"] * applies * R / (ms["sparsify"] / 1e3) / 1e9
        out["sparsify"] = {"bound": "hbm", "achieved": by, "peak": hbm, "unit": "GB/s", "frac": by / hbm}
    sweep_ms = sum(ms.get(k, 0.0) for k in ("slab_a", "recur", "slab_e"))
    if sweep_ms > 0 and applies > 0:
        by = wk["sweep"]["bytes"] * applies / (sweep_ms / 1e3) / 1e9
        out["sweep"] = {"bound": "hbm", "achieved": by, "peak": hbm, "unit": "GB/s", "frac": by / hbm,
                        "units": f"{applies:.0f} preconditioner applications (factor stream shared by {R} RHS)"}
    fac_ms = ms.get("factor", 0.0) + ms.get("iface", 0.0)
    if fac_ms > 0:
        fl = wk["factor"]["flops"] / (fac_ms / 1e3) / 1e12
        if prec_bytes == 8:
            peak, kind = FP64_PEAK_TFLOPS, "FP64 CUDA cores (nominal)"
        elif tc:
            peak, kind = bf16 * TF32_OVER_BF16 / 3.0, "3xTF32 tensor cores (measured bf16 / 2 / 3)"
        else:
            peak, kind = FP32_PEAK_TFLOPS, "FP32 CUDA cores (derived)"
        out["factor"] = {"bound": "alu" if not tc else "tensor", "achieved": fl, "peak": peak, "unit": "TFLOP/s",
                         "frac": fl / peak, "peak_kind": kind}
    if ms.get("krylov", 0) > 0:
        J = max(1, int(round(iters_mean)))
        by = sum(wk["krylov_step"](j) for j in range(J)) * R / (ms["krylov"] / 1e3) / 1e9
        out["krylov"] = {"bound": "hbm", "achieved": by, "peak": hbm, "unit": "GB/s", "frac": by / hbm}
    return out


# ---------------------------------------------------------------- timing helpers
def max_over_ranks(vals, dev, world):
    """Element-wise maximum of per-rank timings over all ranks (one all-reduce;
    a single rank returns its own values)."""
    if world <= 1:
        return [float(v) for v in vals]
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def timed(fn, steps, warmup, flush, stream):
    """CUDA-event milliseconds of `steps` calls of fn (after `warmup` untimed
    calls), L2 flushed (a write larger than L2) before each; returns (ms list,
    results)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts, outs = [], []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs.append(fn())
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return ts, outs


def profile_pass(solver, fn, reps):
    """Per-kernel-group CUDA-event times and launch counts per call of fn."""
    solver.profile_read()
    solver.profile(True)
    for _ in range(reps):
        fn()
    solver.profile(False)
    ms, n = solver.profile_read()
    return {k: v / reps for k, v in ms.items()}, {k: v / reps for k, v in n.items()}


FRONTS = 2   # sweeping fronts of the headline workload (--fronts); its FP64 arm and the oracle use the same
RECURSIVE = False   # 3D headline workloads: the recursive approach of Sec. 3.1 (--recursive)


def leg_fronts(w):
    """Fronts of a further leg: two in 2D (the setting of the paper's 2D
    experiments); one in 3D, where the middle slab padded on both sides has
    (b_slab + 2 b_aux) / (b_slab + b_aux) times the unknowns per block and its
    factorization becomes the critical path of the step."""
    return 2 if w.dim == 2 else 1


def make_solver(w, m_dev, prec, dev, fronts=None, recursive=None):
    from paper_1705_09443_gb300 import LSSolver
    return LSSolver(w.n, w.omega, m_dev, b_pml=w.b_pml, b_slab=w.b_slab, precision=prec,
                    fronts=FRONTS if fronts is None else fronts,
                    recursive=(RECURSIVE and w.dim == 3) if recursive is None else recursive)


# ---------------------------------------------------------------- our arm
def run_headline(args, dev, world, flush):
    """Mixed precision, all right-hand sides of the workload in one solve call;
    full steps timed; profiling pass; solve-only; error against FP64; e2e
    through the host-buffer entry point (the last three skipped with
    --only-headline)."""
    import torch
    from paper_1705_09443_gb300 import GmresOptions, LSS_FP64, LSS_MIXED
    w = synth.WORKLOADS[args.workload]
    m, dirs = synth.make_workload(w)
    R = dirs.shape[0]
    mt = torch.tensor(m, dtype=torch.float64, device=dev)
    opts = GmresOptions(30, 1e-8, 300)
    stream = torch.cuda.current_stream()
    s = make_solver(w, mt, LSS_MIXED, dev)
    tuned = s.autotune(R) if w.dim == 2 else None

    def step():
        s.set_medium(mt)
        s.factor()
        g = s.plane_wave_rhs(dirs)
        return s.solve(g, opts)[1]

    clk = ClockSampler(dev.index)
    step()
    clk.start()
    ts, stats = timed(step, args.steps, max(args.warmup - 1, 0), flush, stream)
    clocks = clk.stop()
    total_ms, = max_over_ranks([sum(ts)], dev, world)
    prof_ms, prof_n = profile_pass(s, step, 1)
    flat = [x for st in stats for x in st]
    iters = float(np.mean([x["iters"] for x in flat]))
    res = dict(value=R * args.steps * world / (total_ms / 1e3), ms_per_step=total_ms / args.steps,
               iters=iters, relres_true_max=max(x["relres_true"] for x in flat),
               converged=all(x["relres_true"] <= 1e-8 for x in flat), clocks=clocks, autotune=tuned,
               prof_ms=prof_ms, prof_launches=prof_n, gpu_launches_per_step=int(sum(prof_n.values())))
    if args.only_headline:
        res["solver"] = s
        return w, R, res
    # solve only (factors in place, right-hand sides resident)
    g = s.plane_wave_rhs(dirs)
    ts_s, _ = timed(lambda: s.solve(g, opts), args.steps, 1, flush, stream)
    sv_ms, = max_over_ranks([sum(ts_s)], dev, world)
    res["solve_only"] = {"value": R * args.steps * world / (sv_ms / 1e3), "unit": "solves/s",
                         "ms_per_solve_call": sv_ms / args.steps}
    # error of the mixed solutions against FP64 solutions at relres 1e-12 (GPU
    # FP64 path, equal to the oracle's to 1e-10 in the parity tests), sampled
    u32, _ = s.solve(g, opts)
    s64 = make_solver(w, mt, LSS_FP64, dev)
    pick = list(range(0, R, max(1, R // 4)))[:4]
    u64, _ = s64.solve(g[pick].contiguous(), GmresOptions(30, 1e-12, 400))
    errs = [float(torch.linalg.vector_norm(u32[p] - u64[q]) / torch.linalg.vector_norm(u64[q]))
            for q, p in enumerate(pick)]
    res["error_vs_fp64"] = {"max": max(errs), "per_rhs": dict(zip([int(p) for p in pick], errs)),
                            "reference": "FP64 GPU solve to relres 1e-12 of the same right-hand sides"}
    del s64
    # e2e through the C ABI with host buffers: m (pinned host) -> device, set-up,
    # factorization, lss_solve_host (g from pinned host, u back to pinned host)
    m_host = torch.tensor(m, dtype=torch.float64).pin_memory()
    g_host = g.cpu().pin_memory()
    u_host = torch.empty_like(g_host).pin_memory()
    m_dev = torch.empty_like(mt)

    def e2e_step():
        m_dev.copy_(m_host, non_blocking=True)
        s.set_medium(m_dev)
        s.factor()
        return s.solve_host(g_host, u_host, opts)

    ts_e, _ = timed(e2e_step, args.steps, 1, flush, stream)
    e2e_ms, = max_over_ranks([sum(ts_e)], dev, world)
    res["e2e"] = {"value": R * args.steps * world / (e2e_ms / 1e3), "unit": "solves/s",
                  "h2d_bytes_per_step": int(m_host.numel() * 8 + g_host.numel() * 16),
                  "d2h_bytes_per_step": int(u_host.numel() * 16),
                  "path": "pinned host m -> lss_set_medium, lss_factor, lss_solve_host (host g in, host u out)"}
    res["solver"] = s
    return w, R, res


def run_plain_fp64(args, dev, world, flush, w, R):
    """Plain FP64 on the same workload, one right-hand side per solve call: the
    set-up + factorization once per medium plus R single-RHS solves; the solves
    are timed on a sample of the R right-hand sides and scaled to R."""
    import torch
    from paper_1705_09443_gb300 import GmresOptions, LSS_FP64
    m, dirs = synth.make_workload(w)
    mt = torch.tensor(m, dtype=torch.float64, device=dev)
    opts = GmresOptions(30, 1e-8, 300)
    stream = torch.cuda.current_stream()
    s = make_solver(w, mt, LSS_FP64, dev)

    def setup():
        s.set_medium(mt)
        s.factor()

    ts_f, _ = timed(setup, max(1, min(args.steps, 3)), 1, flush, stream)
    nsamp = min(R, args.fp64_sample)
    pick = [int(round(k * R / nsamp)) % R for k in range(nsamp)]
    gs = [s.plane_wave_rhs(dirs[p:p + 1]) for p in pick]
    it = iter(range(10 ** 9))
    ts_s, stats = timed(lambda: s.solve(gs[next(it) % nsamp], opts)[1], nsamp, 1, flush, stream)
    f_ms, s_ms = max_over_ranks([float(np.mean(ts_f)), float(np.mean(ts_s))], dev, world)
    step_ms = f_ms + R * s_ms
    flat = [x for st in stats for x in st]
    prof_ms, prof_n = profile_pass(s, lambda: s.solve(gs[0], opts), 1)
    return s, {"value": R * world / (step_ms / 1e3), "unit": "solves/s", "ms_per_step": step_ms,
               "setup_factor_ms": f_ms, "ms_per_single_rhs_solve": s_ms, "rhs_sample": nsamp,
               "iters": float(np.mean([x["iters"] for x in flat])),
               "relres_true_max": max(x["relres_true"] for x in flat),
               "step": f"set-up + factorization once, then {R} single-RHS FGMRES solves "
                       f"(timed on {nsamp} of them, scaled to {R})",
               "solve_breakdown_ms": prof_ms, "solve_launches": prof_n}


def run_leg(args, dev, world, flush, wname, prec, steps, warmup, recursive=False):
    """A full-step leg (set-up + factor + RHS + solve) on another workload
    (3D: with the recursive approach of Sec. 3.1 when asked)."""
    import torch
    from paper_1705_09443_gb300 import GmresOptions
    w = synth.WORKLOADS[wname]
    m, dirs = synth.make_workload(w)
    R = dirs.shape[0]
    mt = torch.tensor(m, dtype=torch.float64, device=dev)
    opts = GmresOptions(30, 1e-8, 300)
    stream = torch.cuda.current_stream()
    s = make_solver(w, mt, prec, dev, fronts=leg_fronts(w), recursive=recursive)
    if w.dim == 2:
        s.autotune(R)

    def step():
        s.set_medium(mt)
        s.factor()
        return s.solve(s.plane_wave_rhs(dirs), opts)[1]

    ts, stats = timed(step, steps, warmup, flush, stream)
    tot, = max_over_ranks([sum(ts)], dev, world)
    g = s.plane_wave_rhs(dirs)
    ts_s, _ = timed(lambda: s.solve(g, opts), steps, 0, flush, stream)
    ts_f, _ = timed(lambda: (s.set_medium(mt), s.factor()), 1, 0, flush, stream)
    prof_ms, prof_n = profile_pass(s, step, 1)
    flat = [x for st in stats for x in st]
    out = {"workload": wname, "precision": "mixed" if prec else "fp64", "R": R, "fronts": leg_fronts(w),
           "slab_solver": ("recursive (inner sweep along x2)" if recursive else
                           "block elimination of the whole slab along x2" if w.dim == 3 else
                           "block LU on 16-wide slabs, cyclic reduction on the others" if R >= 16 else
                           "block cyclic reduction"),
           "value": R * steps * world / (tot / 1e3), "unit": "solves/s", "ms_per_step": tot / steps,
           "solve_only": {"value": R * steps * world / (sum(ts_s) / 1e3), "ms_per_solve_call": sum(ts_s) / steps},
           "setup_factor_ms": float(ts_f[0]), "iters": float(np.mean([x["iters"] for x in flat])),
           "relres_true_max": max(x["relres_true"] for x in flat),
           "converged": all(x["relres_true"] <= 1e-8 for x in flat),
           "breakdown_ms": prof_ms, "launches_per_step": prof_n}
    return s, out


def run_ragged(args, dev, world, flush):
    """Form (2), ragged instances: independent problems with n uniform on
    {128..384}, omega/2pi = n/8, band-limited media, one plane wave each, all
    behind one batch context, solved by the lockstep driver (one set of Krylov
    vectors with a segment per instance); beside it the threaded driver (each
    instance's own solve on a host thread) and the same instances solved one
    after another, each by its own context.  Mixed precision; a step is
    factor + plane-wave RHS + solve of every instance."""
    import torch
    from paper_1705_09443_gb300 import GmresOptions, LSS_MIXED, LSSolver, LSSolverBatch
    spec = dict(synth.RAGGED_32, count=args.ragged)
    ns = synth.ragged_sizes(**spec)
    inst = synth.ragged_instances(ns, spec["seed"])
    ms = [torch.tensor(m, dtype=torch.float64, device=dev) for _, m, _ in inst]
    oms = [2 * math.pi * f for f, _, _ in inst]
    dirs = np.stack([d for _, _, d in inst])
    opts = GmresOptions(30, 1e-8, 300)
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
    for name, step in (("batch", step_batch), ("threaded", step_batch), ("sequential", step_seq)):
        if name == "threaded":
            os.environ["LSS_BATCH_THREADS"] = "1"
        ts, stats = timed(step, args.steps, 1, flush, stream)
        os.environ.pop("LSS_BATCH_THREADS", None)
        total, = max_over_ranks([sum(ts)], dev, world)
        flat = [x for st in stats for q in st for x in q]
        out[name] = {"value": len(ns) * args.steps * world / (total / 1e3), "ms_per_step": total / args.steps,
                     "iters_mean": float(np.mean([x["iters"] for x in flat])),
                     "relres_true_max": max(x["relres_true"] for x in flat),
                     "converged": all(x["relres_true"] <= 1e-8 for x in flat)}
    del batch, single
    return {"instances": len(ns), "unit": "instances solved/s",
            "step": "factor + plane-wave RHS + FGMRES solve of every instance (mixed precision)",
            "driver": "lockstep", **out["batch"], "threaded": out["threaded"], "sequential": out["sequential"],
            "batch_over_sequential": out["batch"]["value"] / out["sequential"]["value"]}


def traffic_record(group, workload):
    """DRAM bytes per launch of a kernel group from an ncu capture recorded in
    profiles/traffic.json, kept only while the kernel's source file still has
    the hash recorded with the capture (null once the kernel has changed)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        rec = json.load(open(p)).get(f"{group}:{workload}")
        if not rec:
            return None
        src = os.path.join(ROOT, "paper_1705_09443_gb300", "csrc", rec["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != rec["sha256_16"]:
            return None
        return rec
    except Exception:
        return None


# ---------------------------------------------------------------- oracle (CPU) legs
ORACLE_WORKER = r"""
import json, sys, time, math
sys.path.insert(0, {root!r})
import numpy as np
import synth
from oracle import lss_oracle as O
w = synth.WORKLOADS[{wl!r}]
m, dirs = synth.make_workload(w)
t0 = time.perf_counter()
pb = O.Problem2D(w.n, w.omega, m, O.Params(b_pml=w.b_pml, b_slab=w.b_slab, fronts={fronts}))
t_setup = time.perf_counter() - t0
g = O.ls_rhs(m, w.omega, pb.kw, dirs[{rhs}])
ts = []
V = [g / np.linalg.norm(g)]
for k in range({reps}):
    t0 = time.perf_counter()
    z = pb.precondition(V[-1])                     # one FGMRES/GMRES iteration:
    y = O.ls_apply(z, m, w.omega, pb.kw)           # P, A and MGS against the basis
    for v in V:
        y = y - np.vdot(v, y) * v
    ts.append(time.perf_counter() - t0)
    V.append(y / np.linalg.norm(y))
print(json.dumps(dict(t_setup=t_setup, t_iter=ts)))
"""


def oracle_sample(wl, reps, workers, rhs0=0):
    """`workers` spawned single-threaded processes, each building the oracle's
    set-up for the workload and timing `reps` GMRES iterations (P + A + MGS)
    on one right-hand side.  Returns their results (run concurrently)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs = []
    for q in range(workers):
        code = ORACLE_WORKER.format(root=ROOT, wl=wl, reps=reps, rhs=rhs0 + q, fronts=FRONTS)
        procs.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, env=env))
    out = []
    for p in procs:
        so, se = p.communicate(timeout=3600)
        if p.returncode != 0:
            raise RuntimeError(se[-2000:])
        out.append(json.loads(so.strip().splitlines()[-1]))
    return out


def oracle_rate(res, R, iters):
    """Solves/s of one single-threaded oracle process: the set-up amortised over
    the R right-hand sides of the medium, `iters` iterations per solve."""
    t_iter = float(np.mean(res["t_iter"]))
    return 1.0 / (res["t_setup"] / R + iters * t_iter), t_iter


def workload_text(w):
    med = (f"{w.n_gauss} Gaussians width {w.width}, c in {list(w.c_range)}" if w.medium == "gauss"
           else f"band-limited random medium (correlation length {w.width}, c in [0.8, 1.2])")
    return (f"{w.dim}D LS, n={w.n} (N={w.n ** w.dim}), omega/2pi={w.freq:g}, {med}, {w.n_rhs} plane wave(s)"
            f"{' in one solve call' if w.n_rhs > 1 else ''}, PML {w.b_pml}, slab {w.b_slab}, "
            f"{'two sweeping fronts' if FRONTS == 2 else 'one sweeping front'}, GMRES(30) tol 1e-8")


def reference_arm(args):
    """The oracle as it stands on the host cores (single thread): its set-up for
    the workload once, one full GMRES solve for its iteration count, and
    --steps samples of one GMRES iteration (P + A + MGS) each."""
    w = synth.WORKLOADS[args.workload]
    m, dirs = synth.make_workload(w)
    R = dirs.shape[0]
    from oracle import lss_oracle as O
    t0 = time.perf_counter()
    pb = O.Problem2D(w.n, w.omega, m, O.Params(b_pml=w.b_pml, b_slab=w.b_slab, fronts=FRONTS))
    t_setup = time.perf_counter() - t0
    g = O.ls_rhs(m, w.omega, pb.kw, dirs[0])
    t0 = time.perf_counter()
    res = O.gmres(lambda u: O.ls_apply(u, m, w.omega, pb.kw), pb.precondition, g, 30, 1e-8, 300)
    t_solve = time.perf_counter() - t0
    V = [g / np.linalg.norm(g)]
    ts = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        z = pb.precondition(V[-1])
        y = O.ls_apply(z, m, w.omega, pb.kw)
        for v in V:
            y = y - np.vdot(v, y) * v
        if k >= args.warmup:
            ts.append(time.perf_counter() - t0)
        V.append(y / np.linalg.norm(y))
    t_iter = float(np.mean(ts))
    per_rhs = t_setup / R + res.iters * t_iter
    v = 1.0 / per_rhs
    sample = (f"oracle set-up of the workload once ({t_setup:.1f} s, amortised over its {R} right-hand sides), "
              f"one full GMRES solve for the iteration count ({res.iters}, {t_solve:.1f} s), then "
              f"{args.steps} timed samples of one GMRES iteration (preconditioner, operator, MGS); "
              f"solves/s = 1 / (set-up / {R} + iterations x iteration time)")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_rhs * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_text(w)},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "oracle_iters": res.iters, "oracle_iteration_s": t_iter, "oracle_setup_s": t_setup}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--recursive", action="store_true",
                    help="3D workloads: the recursive approach of Sec. 3.1 for the headline solver")
    ap.add_argument("--fronts", type=int, default=2, choices=[1, 2],
                    help="sweeping fronts: 1 (Algorithm 2) or 2 (toward the middle slab, Sec. 2.4)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-workers", type=int, default=0, help="oracle worker processes (0: min(16, cores))")
    ap.add_argument("--fp64-sample", type=int, default=8, help="single-RHS FP64 solves timed (scaled to R)")
    ap.add_argument("--legs", default="2d_n256,3d_n64,3d_n64:rec",
                    help="further full-step legs (workload[:rec] for the 3D recursive approach; 'none' to skip)")
    ap.add_argument("--ragged", type=int, default=32, help="instances of the ragged batch line (0 to skip)")
    ap.add_argument("--only-ragged", action="store_true",
                    help="run the ragged batch line only and print it; not a bench line")
    ap.add_argument("--only-headline", action="store_true",
                    help="run the headline workload's steps only (warm-up, timed steps, the profiling pass) and "
                         "print its breakdown; for profiler launch lists, not a bench line")
    args = ap.parse_args()
    global FRONTS, RECURSIVE
    FRONTS = args.fronts
    RECURSIVE = args.recursive
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_arm(args)))
        return

    import torch
    from paper_1705_09443_gb300 import LSS_FP64, LSS_MIXED
    if world > 1:
        torch.distributed.init_process_group("nccl")
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2
    hbm, bf16, peak_src = peaks()
    if args.only_ragged:
        ragged = run_ragged(args, dev, world, flush)
        if rank == 0:
            print(json.dumps({"only_ragged": ragged}))
        return

    w, R, head = run_headline(args, dev, world, flush)
    if args.only_headline:
        if rank == 0:
            print(json.dumps({"only_headline": args.workload, "solves_per_s": head["value"],
                              "ms_per_step": head["ms_per_step"], "iters": head["iters"],
                              "breakdown_ms": head["prof_ms"], "launches_per_step": head["prof_launches"]}))
        return
    s64, plain = run_plain_fp64(args, dev, world, flush, w, R)
    groups = group_roofline(head["solver"], head, 4, R, head["iters"], hbm, bf16)
    fp64_groups = group_roofline(s64, {"prof_ms": plain["solve_breakdown_ms"],
                                       "prof_launches": plain["solve_launches"]}, 8, 1, plain["iters"], hbm, bf16)
    del head["solver"], s64
    legs = {}
    for wspec in [x for x in args.legs.split(",") if x and x != "none"]:
        wname, _, opt = wspec.partition(":")
        wl = synth.WORKLOADS[wname]
        if opt == "rec":   # the recursive approach (Sec. 3.1), mixed precision, against the non-recursive leg
            sv, leg = run_leg(args, dev, world, flush, wname, LSS_MIXED, 2, 1, recursive=True)
            base = legs.get(f"{wname}_mixed")
            if base:
                leg["relative_to_non_recursive"] = {
                    "setup_factor": leg["setup_factor_ms"] / base["setup_factor_ms"],
                    "solve": leg["solve_only"]["ms_per_solve_call"] / base["solve_only"]["ms_per_solve_call"],
                    "iters": [leg["iters"], base["iters"]]}
            legs[f"{wname}_recursive_mixed"] = leg
            del sv
            continue
        for pname, prec in (("mixed", LSS_MIXED), ("fp64", LSS_FP64)):
            heavy = wl.dim == 3 and prec == LSS_FP64
            steps = 1 if heavy else (2 if wl.dim == 3 else args.steps)
            warm = 0 if heavy else (1 if wl.dim == 3 else args.warmup)
            sv, leg = run_leg(args, dev, world, flush, wname, prec, steps, warm)
            leg["roofline_groups"] = group_roofline(sv, {"prof_ms": leg["breakdown_ms"],
                                                         "prof_launches": leg["launches_per_step"]},
                                                    4 if prec else 8, leg["R"], leg["iters"], hbm, bf16)
            legs[f"{wname}_{pname}"] = leg
            del sv
        if f"{wname}_fp64" in legs:
            legs[f"{wname}_mixed"]["mixed_over_fp64"] = legs[f"{wname}_mixed"]["value"] / legs[f"{wname}_fp64"]["value"]
    ragged = run_ragged(args, dev, world, flush) if args.ragged else None
    torch.cuda.synchronize()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        workers = args.cpu_workers or min(16, os.cpu_count() or 1)
        outs = oracle_sample(args.workload, 2, workers)
        iters = plain["iters"]
        rates = [oracle_rate(o, R, iters)[0] for o in outs]
        one = oracle_rate(outs[0], R, iters)
        cpu = {"value": float(sum(rates)), "unit": "solves/s", "cores": workers, "kind": "oracle",
               "one_core": {"value": float(np.mean(rates)), "cores": 1},
               "sample": (f"{workers} concurrent single-threaded oracle processes (numpy/scipy), each building "
                          f"the oracle's set-up of this workload and timing 2 GMRES iterations (P + A + MGS) on "
                          f"its own right-hand side; per process solves/s = 1 / (set-up / {R} + {iters:.1f} "
                          f"iterations x iteration time), the iteration count being the FP64 GPU path's (equal "
                          f"to the oracle's within one in the parity tests); value = sum over processes"),
               "setup_s": float(np.mean([o["t_setup"] for o in outs])), "iteration_s": one[1]}
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    dom = max(groups, key=lambda k: {"matvec": head["prof_ms"].get("matvec", 0),
                                     "sparsify": head["prof_ms"].get("sparsify", 0),
                                     "sweep": sum(head["prof_ms"].get(x, 0) for x in ("slab_a", "recur", "slab_e")),
                                     "factor": head["prof_ms"].get("factor", 0) + head["prof_ms"].get("iface", 0),
                                     "krylov": head["prof_ms"].get("krylov", 0)}.get(k, 0))
    roof = dict(groups[dom])
    tr = traffic_record(dom, args.workload)
    roof.update({"kernel_group": dom, "traffic": tr["dram_bytes_per_launch"] if tr else None,
                 "traffic_source": tr["note"] if tr else "no ncu capture of the current kernel source",
                 "peak_source": f"{peak_src} (HBM {hbm:.0f} GB/s); CUDA-core peaks derived (module constants)",
                 "groups": groups})
    line = {
        "metric": METRIC, "value": head["value"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64 preconditioner / c128 operator, Arnoldi, Givens, true residual",
        "data": "synthetic",
        "config": {"workload": workload_text(w), "precision": "mixed (FP32 slab factors and sweep)",
                   "slab_solver": ("block LU (bottom-up Schur complements along x2) on the 16-wide slabs, "
                                   "block cyclic reduction on the 32-wide ones") if R >= 16 and w.dim == 2 else
                                  "block cyclic reduction" if w.dim == 2 else "block elimination along x2",
                   "l2": "flushed (256 MB write) before every timed step; vectors exceed L2",
                   "per_omega_tables": "built once at solver creation (kernel FFT, alpha/beta, physical PML stencils)"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": head["e2e"],
        "gpu_launches": int(head["gpu_launches_per_step"] * args.steps), "clocks": head["clocks"],
        "iters": head["iters"], "relres_true_max": head["relres_true_max"], "converged": head["converged"],
        "error_vs_fp64": head["error_vs_fp64"], "solve_only": head["solve_only"], "autotune": head["autotune"],
        "step": "set_medium + factor + plane-wave RHS + FGMRES solve of all right-hand sides, per medium",
        "breakdown_ms": head["prof_ms"], "launches_per_step": head["prof_launches"],
        "plain_fp64": dict(plain, roofline_groups=fp64_groups),
        "mixed_batched_over_plain_fp64": head["value"] / plain["value"],
        "legs": legs, "ragged": ragged,
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
