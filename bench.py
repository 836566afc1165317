"""Benchmark: right-hand sides solved per second to ||b - D x|| / ||b|| < 1e-10.

Workload of one step (the default line): the 24^3x48 Wilson lattice with SU(3)
links U = exp(0.3 i H) (gauge seed 3) at the kappa where min|eig(gamma5 D)| = 1e-3;
Lan-DR(120,60) on D^dagger D for the first Gaussian right-hand side (seed 0), then
D-CG on 48 Gaussian right-hand sides (seeds 1..48) (arXiv:0901.3163, Sec. 2 method
on a synthetic stand-in for its quenched lattice): 49 right-hand sides per step.
A right-hand side counts only if its true residual was verified in FP64.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`value` is the chosen form: FP32 Lanczos and FP32 CG on the normal equations
(fused stencil kernels, 16 right-hand sides per launch) inside FP64 defect
correction, FP64 for x, the true residual, the deflation projection and the small
eigenproblem.  Beside it on the same operator:
  plain_fp64  the plain FP64 form (FP64 Lan-DR, then D-CG one right-hand side at a
              time, FP64 stencil), the first right-hand side in full and D-CG on a
              sample of right-hand sides, extrapolated to 48;
  evenodd     the same step through the even-odd (Schur complement) operator;
  c4          64 lattices of uneven size (8^4, 12^4, 16^4), D-MinRes on 8 RHS each,
              all lattices in one batched call, against lattice by lattice and FP64;
  c2          (with --c2) the 16^3x32 workload (MinRes-DR(100,40) + D-MinRes on 12
              point sources);
  dslash      the Wilson stencil alone (FP32 and bfloat16, 16 RHS per launch).

Prints one JSON line (rank 0).  Multi-GPU runs (torchrun) solve independent
replicas of the workload, one per rank, with no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "wilson_24x24x24x48"
C2 = "wilson_16x16x16x32"
C4 = "uneven_64"
# restart cycles of the 16^3x32 first right-hand side's MinRes-DR phase (both forms)
C2_DR_CYCLES = 150
# D-CG iterations per right-hand side of the FP64 form on the 24^3x48 workload, and
# the MVPs of its first right-hand side (FP64 Lan-DR(120,60) to its stopping rule, 229
# cycles at the tabulated kappa): the oracle runs the same FP64 algorithm but cannot
# finish this lattice in a bounded sample, so the reference arm extrapolates its seconds
# per iteration with these counts (taken from the FP64 form of the library on this
# workload, mean of 2 RHS; the default line reports the counts of its own FP64 run in
# plain_fp64)
REF_ITERS_PER_RHS = 2328
REF_FIRST_RHS_MVPS = 27830
# DRAM bytes (read + write) of one k_cg_k1 launch (16 RHS, 24^3x48), the dominant kernel,
# from one single-pass ncu capture of the kernel at this size (summarised under
# profiles/); None until taken for the current kernel
K1_TRAFFIC_BYTES = 8.30e9
METRIC = "RHS solved/s to |r|/|b|<1e-10 (Lan-DR(120,60) + D-CG, 49 Gaussian RHS, 24^3x48)"
UNIT = "RHS/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.proc = None
        self.lines = []
        self.dev = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return parse_clock_lines(self.lines)


def parse_clock_lines(lines):
    """Median SM clock, max clock and the throttle reasons seen in nvidia-smi CSV lines."""
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax = float(f[2])
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    sm.sort()
    med = sm[len(sm) // 2] if sm else None
    return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_ranks(ms, solved, world, device):
    """Replicas on N ranks: the job's time is the slowest rank's, its work the sum of
    every rank's solved right-hand sides (host-side reduction of two numbers; the data
    path has no collective)."""
    if world <= 1:
        return float(ms), float(solved)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms), float(solved)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(t[1])


def workload_rhs_count(name=WORKLOAD):
    """Right-hand sides in one step of a named workload."""
    import synth
    w = synth.WORKLOADS[name]
    return 12 if "point_sources" in w else 1 + len(w["rhs_seeds"])


def workload_inputs(kappa=None, name=WORKLOAD, rhs=None):
    """Links, kappa and right-hand sides of a named workload (synth.WORKLOADS).
    24^3x48: B[0] is the first RHS (seed 0), B[1:] the 48 D-CG RHS.
    16^3x32: the 12 spin-colour point sources at the origin.
    rhs: the indices (into that list) of the right-hand sides to make, in that order;
    None makes all of them (49 x 127 MB on 24^3x48)."""
    import numpy as np

    import synth
    w = synth.WORKLOADS[name]
    dims = w["dims"]
    U = synth.su3_links(dims, w["gauge_seed"])
    if kappa is None:
        kappa = synth.kappa_for(dims, w["gauge_seed"])
    V = synth.volume(dims)
    idx = list(range(workload_rhs_count(name))) if rhs is None else list(rhs)
    B = np.zeros((len(idx), V, 4, 3), dtype=np.complex128)
    if "point_sources" in w:
        for j, a in enumerate(idx):
            B[j] = synth.point_source(dims, a // 3, a % 3)
    else:
        seeds = (w["first_rhs_seed"],) + tuple(w["rhs_seeds"])
        for j, a in enumerate(idx):
            B[j] = synth.gaussian_spinor(dims, seeds[a])
    return w, dims, U, kappa, B


def workload_params(dlz, w, pr, name=WORKLOAD):
    """Solver parameters of one benchmark step (first RHS, then the others).

    24^3x48: Lan-DR(120,60) until the linear residual and the kept Ritz residuals
    converge (FP32 form: then D-CG from x over the 60 vectors), D-CG with FP64
    defect correction (inner reduction 1e-2).
    16^3x32: C2_DR_CYCLES MinRes-DR(100,40) restart cycles (run past linear
    convergence so that the 40 harmonic Ritz vectors converge), then D-MinRes from
    that x over the 40 vectors; re-orthogonalisation against the kept vectors every 30
    Lanczos steps (the paper gives no period)."""
    if name == C2:
        p_dr = dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_cycles=C2_DR_CYCLES, check_every=16,
                                  precision=pr, oversolve=1e9, finish=1, reorth_period=30)
    else:
        p_dr = dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_cycles=400, check_every=16,
                                  precision=pr, finish=1)
    p_d = dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_iter=200000, precision=pr,
                             check_every=16)
    return p_dr, p_d


def solve_step(dlz, op, b0, rest, pars, minres, host=None, profile=False):
    """One step: the first right-hand side by Lan-DR (MinRes-DR), the others by D-CG
    (D-MinRes) over its deflation set.  Returns (verified solves, stats of every RHS)."""
    p_dr, p_d = pars
    p_dr.profile = p_d.profile = int(profile)
    dr = dlz.minresdr if minres else dlz.landr
    ds = dlz.dminres if minres else dlz.dcg
    if host is None:
        x0, defl, st = dr(op, b0, p_dr)
        X, sts = ds(op, defl, rest, p_d)
    else:
        hb0, hrest, hx0, hX = host
        x0, defl, st = dr(op, hb0, p_dr, x=hx0)
        X, sts = ds(op, defl, hrest, p_d, X=hX)
    allst = [st] + list(sts)
    ok = sum(1 for s in allst if s.converged == 1 and s.true_residual <= 1e-10)
    return ok, allst


def kernel_roofline(stats, tag, peaks, src, name, traffic=None, traffic_src=None):
    """Roofline of one fused kernel kind from the profiled stats (CUDA events on the
    launching stream): algorithmic bytes per launch / average launch time."""
    ms = sum(s.kernel_ms[tag] for s in stats)
    nb = sum(s.kernel_bytes[tag] for s in stats)
    n = sum(s.kernel_launches[tag] for s in stats)
    if n == 0 or ms <= 0:
        return None
    avg = ms / n
    bpl = nb / n
    ach = bpl / (avg * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(ach / peaks["hbm_gbs"], 4), "peak_source": src, "kernel": name,
            "avg_launch_ms": round(avg, 5), "launches_timed": int(n), "bytes_per_launch": int(bpl),
            "traffic": traffic, "traffic_source": traffic_src}


def run_ours(args):
    import numpy as np
    import torch

    from paper_0901_3163_gb300 import dlz

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, dims, U, kappa, B = workload_inputs(args.kappa)
    nrhs = B.shape[0]
    op = dlz.create_operator(dims, torch.from_numpy(U).to(dev), kappa)
    Bd = torch.from_numpy(B).to(dev)
    b0, rest = Bd[0].contiguous(), Bd[1:].contiguous()
    pars = workload_params(dlz, w, dlz.F32)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # the last warm-up step carries the CUDA events of the kernel rooflines (every fused
    # stencil launch bracketed on the launching stream); the timed steps carry none
    pst = []
    for i in range(args.warmup):
        _, wst = solve_step(dlz, op, b0, rest, pars, False, profile=(i == args.warmup - 1))
        if i == args.warmup - 1:
            pst = wst[1:]
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    solved = 0
    stats = []
    for _ in range(args.steps):
        ok, allst = solve_step(dlz, op, b0, rest, pars, False)
        solved += ok
        stats.extend(allst)
    e1.record()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_max, solved_all = aggregate_ranks(ms, solved, world, dev)
    value = solved_all / (ms_max / 1e3)
    peaks, src = _peaks()
    roof = kernel_roofline(pst, 1, peaks, src,
                           "k_cg_k1 (fused FP32 CGNR: r gathered, t = D r + beta t, p = r + beta p, "
                           "e += alpha p_old; 16 RHS per launch)",
                           args.k1_traffic,
                           "ncu capture of the current kernel, one launch at this size "
                           "(summary under profiles/)" if args.k1_traffic else
                           "not captured for the current kernel")
    roof_k23 = kernel_roofline(pst, 2, peaks, src,
                               "k_cg_k23 (fused FP32 CGNR: t gathered, r -= alpha D^dag t; 16 RHS per launch)")
    it_ms = sum(s.kernel_ms[1] + s.kernel_ms[2] for s in pst)
    it_b = sum(s.kernel_bytes[1] + s.kernel_bytes[2] for s in pst)
    # end to end: host (pinned) buffers through the C ABI, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hb0 = torch.from_numpy(B[0].copy()).pin_memory()
        hrest = torch.from_numpy(B[1:].copy()).pin_memory()
        hx0 = torch.empty_like(hb0).pin_memory()
        hX = torch.empty_like(hrest).pin_memory()
        barrier()
        t0 = time.perf_counter()
        e2e_solved = 0
        for _ in range(max(1, args.e2e_steps)):
            ok, _ = solve_step(dlz, op, b0, rest, pars, False, host=(hb0, hrest, hx0, hX))
            e2e_solved += ok
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": round(e2e_solved / e2e_s * world, 4), "unit": UNIT,
               "h2d_bytes_per_step": int(B.nbytes), "d2h_bytes_per_step": int(B.nbytes),
               "steps": max(1, args.e2e_steps)}
        del hb0, hrest, hx0, hX
    dr_s = sum(s.seconds for s in stats[0::nrhs]) / max(args.steps, 1)
    d_s = sum(s.seconds for i, s in enumerate(stats) if i % nrhs) / max(args.steps, 1)
    launches = sum(s.gpu_launches for s in stats)
    mvps = sum(s.mvps for s in stats) // max(args.steps, 1)
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded SU(3) links exp(0.3iH), seeded complex Gaussian RHS)",
        "config": {"workload": WORKLOAD, "lattice": list(dims), "kappa": kappa, "m": w["m"], "k": w["k"],
                   "rhs": nrhs, "form": "chosen (FP32 inner, FP64 outer)", "tol": 1e-10,
                   "l2": "inputs and Krylov basis (121 x 63.7 MB FP32) larger than L2; no flush",
                   "first_rhs": "Lan-DR(120,60) on D^dag D to convergence, then D-CG from x",
                   "d_phase": "D-CG on 48 RHS, 16 per launch, FP64 defect correction",
                   "parallelism": f"replicas x{world}"},
        "e2e": e2e,
        "gpu_launches": int(launches), "gpu_launches_per_step": int(launches // max(args.steps, 1)),
        "library_kernels": "none: the restart V P and the projections run on the library's own tcgen05 kernels (counted above)",
        "mvps_per_step": int(mvps), "iterations_first_steps": [s.iterations for s in stats[:4]],
        "phase_seconds": {"first_rhs_dr": round(dr_s, 4), "deflated_48_rhs": round(d_s, 4)},
        "d_phase_rhs_per_s": round((nrhs - 1) / d_s, 4) if d_s > 0 else None,
        "roofline": roof, "roofline_k_cg_k23": roof_k23,
        "cg_iteration_hbm_gbs": round(it_b / (it_ms * 1e-3) / 1e9, 1) if it_ms > 0 else None,
        "clocks": clk,
    }
    if args.plain_rhs > 0:
        out["plain_fp64"] = plain_fp64(dlz, op, b0, rest, w, args.plain_rhs, nrhs, value)
        out["chosen_over_plain"] = out["plain_fp64"].pop("_ratio")
    out["dslash"] = dslash_lines(dlz, torch, op, dims, peaks)
    del op
    torch.cuda.empty_cache()
    if not args.no_evenodd:
        out["evenodd"] = run_evenodd(dlz, torch, w, dims, U, kappa, Bd, peaks, src, pars)
    del Bd, b0, rest
    torch.cuda.empty_cache()
    if not args.no_c4:
        out["c4"] = run_c4(dlz, torch, args.c4_lattices)
    if args.c2:
        out["c2"] = run_c2(dlz, torch, peaks, src)
    if rank == 0 and not args.no_cpu_baseline:
        pf = out.get("plain_fp64", {})
        out["cpu_baseline"] = cpu_baseline(pf.get("dcg_iterations_mean", REF_ITERS_PER_RHS),
                                           pf.get("first_rhs_mvps", REF_FIRST_RHS_MVPS),
                                           nrhs, budget_s=args.cpu_seconds,
                                           source="this run's FP64 form" if pf else "constants in bench.py")
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_evenodd(dlz, torch, w, dims, U, kappa, Bd, peaks, src, pars):
    """The same step through the even-odd operator (not in the paper; the standard Schur
    reduction the deflated methods apply to unchanged): b_e' = b_e + kappa H_eo b_o for
    all 49 RHS, Lan-DR(120,60) on Dhat^dag Dhat for the first, D-CG on Dhat^dag Dhat for
    the 48 others over its deflation set (FP32 inner, FP64 outer, as the chosen form),
    then x_o = b_o + kappa H_oe x_e.  The even-site system stops at 0.5e-10 relative
    residual: the odd rows of D x = b hold exactly, so ||b - D x|| = ||b_e' - Dhat x_e||,
    and ||b_e'|| / ||b|| (reported) stays below 2, which keeps the full relative
    residual below 1e-10.  One warm-up step (which also carries the CUDA events of
    the kernel rooflines), one timed step (CUDA events on the operator's stream,
    prepare and reconstruct included)."""
    op = dlz.create_operator_eo(dims, torch.from_numpy(U).cuda(), kappa)
    p_dr, p_d = pars
    p_dr = dlz.params_default(**{f: getattr(p_dr, f) for f, _ in p_dr._fields_})
    p_d = dlz.params_default(**{f: getattr(p_d, f) for f, _ in p_d._fields_})
    p_dr.tol = p_d.tol = 0.5e-10
    nrhs = Bd.shape[0]

    def step(profile=False):
        p_dr.profile = p_d.profile = int(profile)
        Be = dlz.eo_prepare(op, Bd)
        xe0, defl, st = dlz.landr(op, Be[0].contiguous(), p_dr)
        Xe, sts = dlz.dcg(op, defl, Be[1:].contiguous(), p_d)
        X = dlz.eo_reconstruct(op, torch.cat([xe0[None], Xe]).contiguous(), Bd)
        allst = [st] + list(sts)
        ok = sum(1 for s in allst if s.converged == 1 and s.true_residual <= 0.5e-10)
        return ok, allst, X, Be

    # the warm-up step carries the CUDA events of the kernel rooflines
    _, pst, X, Be = step(profile=True)
    bn = torch.linalg.vector_norm(Bd.reshape(nrhs, -1), dim=1)
    ben = torch.linalg.vector_norm(Be.reshape(nrhs, -1), dim=1)
    ratio = float((ben / bn).max())
    del X, Be
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    ok, allst, X, Be = step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    del X, Be
    roof = kernel_roofline(pst[1:], 2, peaks, src, "k_eo_hop<float> + k_cg_eo_k23b (even-odd fused CGNR, 16 RHS)")
    roof1 = kernel_roofline(pst[1:], 1, peaks, src, "k_eo_hop<float> + k_cg_eo_k1b (even-odd fused CGNR, 16 RHS)")
    out = {"workload": WORKLOAD + " (even-odd)", "value": round(ok / (ms / 1e3), 4), "unit": UNIT,
           "ms_per_step": round(ms, 1), "solved": ok, "even_rhs_norm_ratio_max": round(ratio, 4),
           "tol_even_system": 0.5e-10,
           "phase_seconds": {"first_rhs_dr": round(allst[0].seconds, 4),
                             "deflated_48_rhs": round(sum(s.seconds for s in allst[1:]), 4)},
           "iterations_first_steps": [s.iterations for s in allst[:4]],
           "roofline_k23_pair": roof, "roofline_k1_pair": roof1}
    del op
    return out


def plain_fp64(dlz, op, b0, rest, w, nsample, nrhs, chosen_value):
    """The plain FP64 form on the same operator: FP64 Lan-DR(120,60) on the first
    right-hand side (with its D-CG finish), then FP64 D-CG one right-hand side at a
    time on `nsample` of the 48, whose mean time is extrapolated to all 48."""
    import torch
    p_dr, p_d = workload_params(dlz, w, dlz.F64)
    # warm-up of the FP64 kernels: two restart cycles and a short D-CG
    wdr = dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_cycles=2, precision=dlz.F64)
    _, wd, _ = dlz.landr(op, b0, wdr)
    dlz.dcg(op, wd, rest[:1].contiguous(), dlz.params_default(max_iter=32, precision=dlz.F64))
    del wd
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x0, defl, st = dlz.landr(op, b0, p_dr)
    torch.cuda.synchronize()
    t_dr = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, sts = dlz.dcg(op, defl, rest[:nsample].contiguous(), p_d)
    torch.cuda.synchronize()
    t_d = time.perf_counter() - t0
    ok = [s.converged == 1 and s.true_residual <= 1e-10 for s in [st] + list(sts)]
    per_rhs = t_d / nsample
    step_s = t_dr + per_rhs * (nrhs - 1)
    value = nrhs / step_s if all(ok) else None
    return {"value": round(value, 5) if value else None, "unit": UNIT,
            "sample": f"first RHS in full + D-CG on {nsample} of {nrhs - 1} RHS, per-RHS time extrapolated",
            "first_rhs_seconds": round(t_dr, 3), "first_rhs_mvps": int(st.mvps), "first_rhs_cycles": st.cycles,
            "dcg_seconds_per_rhs": round(per_rhs, 3),
            "dcg_iterations_mean": float(sum(s.iterations for s in sts) / len(sts)),
            "all_verified": bool(all(ok)), "_ratio": round(chosen_value / value, 3) if value else None}


def dslash_lines(dlz, torch, op, dims, peaks):
    """The Wilson stencil alone as the solvers launch it, 16 RHS per launch."""
    import numpy as np
    V = int(np.prod(dims))
    ds = {}
    for name, dt, real in (("f32_batch16", dlz.F32, 4), ("bf16_batch16", dlz.BF16, 2)):
        xs = torch.randn((16, V, 4, 3), dtype=torch.complex64, device="cuda")
        ms = dlz.stencil_bench(op, xs, 30, dtype=dt)["ms"]
        nb = V * (48 * 16 * real + 48 * 4)
        ds[name] = {"avg_launch_ms": round(ms, 5), "gbs": round(nb / ms / 1e6, 1),
                    "frac_hbm": round(nb / ms / 1e6 / peaks["hbm_gbs"], 4), "bytes_per_launch": int(nb)}
        del xs
    xs = torch.randn((1, V, 4, 3), dtype=torch.complex128, device="cuda")
    ms = dlz.stencil_bench(op, xs, 20)["ms"]
    ds["f64_single"] = {"avg_launch_ms": round(ms, 5), "fp64_tflops": round(1368 * V / (ms * 1e-3) / 1e12, 3)}
    return ds


def c4_kappas(w):
    """kappa per lattice of the uneven batch: the sigma_min = 1e-3 rule computed by the
    oracle for the first lattice of each size (gauge seeds 3000, 3001, 3002) and used
    for every lattice of that size (the links of all lattices follow one recipe)."""
    import synth
    ks = []
    for i in range(w["lattices"]):
        dims = w["sizes"][i % 3]
        ks.append(synth.kappa_for(dims, w["gauge_seed0"] + i % 3))
    return ks


def run_c4(dlz, torch, nl=64):
    """64 lattices (i mod 3 -> 8^4, 12^4, 16^4) at the kappa of c4_kappas: FP32
    MinRes-DR(40,10) on one Gaussian RHS per lattice, then D-MinRes on 8 Gaussian RHS
    per lattice (512 solves) through one dlz_batch_dminres call (FP32, one launch per
    stage for all slots), against the same solves lattice by lattice (FP32, each
    lattice's RHS batched) and the plain FP64 form (one RHS at a time), both timed on
    one lattice of each size and counted for every lattice of that size."""
    import synth
    w = synth.WORKLOADS[C4]
    try:
        kap = c4_kappas(w)[:nl]
        ksrc = "sigma_min = 1e-3 rule per size class (oracle, first lattice of each size)"
    except KeyError as e:
        return {"unavailable": str(e)}
    ops, defls, Bs = [], [], []
    dr_s = 0.0
    for i in range(nl):
        dims = w["sizes"][i % 3]
        op = dlz.create_operator(dims, torch.from_numpy(synth.su3_links(dims, w["gauge_seed0"] + i)).cuda(),
                                 float(kap[i]))
        b0 = torch.from_numpy(synth.gaussian_spinor(dims, w["first_rhs_seed"])).cuda()
        ta = time.perf_counter()
        _, d, st = dlz.minresdr(op, b0, dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_cycles=400,
                                                           precision=dlz.F32))
        torch.cuda.synchronize()
        dr_s += time.perf_counter() - ta
        ops.append(op)
        defls.append(d)
        Bs.append(torch.from_numpy(synth.gaussian_spinors(dims, w["rhs_seeds"])).cuda())
    sites = sum(o.volume for o in ops)
    p32 = dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_iter=100000, precision=dlz.F32,
                             reliable_delta=1e-5)
    # one call, timed as a user makes it (its graph captures and the autotuner's trial
    # groups included: at the rule's kappa the solves run ~20k iterations)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    ta = time.perf_counter()
    Xs, sts = dlz.batch_dminres(ops, defls, Bs, p32)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - ta
    clk = clocks.stop()
    ok_batch = sum(1 for ss in sts for s in ss if s.converged == 1 and s.true_residual <= 1e-10)
    form, chunks, half = dlz.batch_last_choice(ops[0])
    choice = {"form": "persistent" if form == 1 else "graph", "chunks_per_block": chunks, "half_grid": bool(half)}
    # the lattice-by-lattice FP32 form and the plain FP64 form on one lattice of each size
    # (the first three), each lattice's time counted for every lattice of its size
    per_size = [sum(1 for i in range(nl) if i % 3 == j) for j in range(min(3, nl))]

    def sample(params):
        t_all, t_s, ok, n = 0.0, 0.0, 0, 0
        for j in range(min(3, nl)):
            torch.cuda.synchronize()
            ta = time.perf_counter()
            _, ss = dlz.dminres(ops[j], defls[j], Bs[j], params)
            torch.cuda.synchronize()
            dt = time.perf_counter() - ta
            t_s += dt
            t_all += dt * per_size[j]
            ok += sum(1 for s in ss if s.converged == 1 and s.true_residual <= 1e-10)
            n += len(ss)
        return t_all, t_s, ok, n

    t_seq, t_seq_sample, ok_seq, n_seq = sample(p32)
    p64 = dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_iter=100000)
    t64_all, t64, ok64, n64 = sample(p64)
    iters = [max(s.iterations for s in ss) for ss in sts]
    nsolve = sum(len(ss) for ss in sts)
    rate64 = (ok64 / n64) * nsolve / t64_all if n64 else None
    rate_seq = (ok_seq / n_seq) * nsolve / t_seq if n_seq else None
    out = {"workload": f"{nl} lattices 8^4/12^4/16^4, MinRes-DR(40,10) + D-MinRes x 8 RHS each",
           "kappa": sorted(set(round(k, 10) for k in kap)), "kappa_source": ksrc,
           "lattices": nl, "sites_total": int(sites), "rhs_total": int(sum(len(ss) for ss in sts)),
           "first_rhs_dr_seconds": round(dr_s, 3),
           "batched": {"seconds": round(t_batch, 3), "rhs_per_s": round(ok_batch / t_batch, 2), "solved": ok_batch,
                       "iterations_max": int(max(iters)), "autotuner_choice": choice},
           "lattice_by_lattice_f32": {"sample": "one lattice of each size, its 8 RHS batched; its time "
                                                 "counted for every lattice of that size",
                                      "seconds_sample": round(t_seq_sample, 3),
                                      "rhs_per_s": round(rate_seq, 2) if rate_seq else None},
           "plain_fp64": {"sample": "one lattice of each size, 8 RHS each, one RHS at a time; its time "
                                    "counted for every lattice of that size",
                          "seconds_sample": round(t64, 3), "rhs_per_s": round(rate64, 3) if rate64 else None},
           "batched_over_lattice_by_lattice": round((ok_batch / t_batch) / rate_seq, 3) if rate_seq else None,
           "chosen_over_plain": round((ok_batch / t_batch) / rate64, 3) if rate64 else None,
           "clocks": clk}
    return out


def run_c2(dlz, torch, peaks, src):
    """The 16^3x32 workload (MinRes-DR(100,40) on the point source at the origin, spin 0
    colour 0, then D-MinRes on the other 11 spin-colour point sources), chosen form:
    one warm-up step and one timed step (CUDA events), then a profiled step for the
    roofline of the fused MinRes kernel (k_minres_k1)."""
    w, dims, U, kappa, B = workload_inputs(name=C2)
    op = dlz.create_operator(dims, torch.from_numpy(U).cuda(), kappa)
    Bd = torch.from_numpy(B).cuda()
    b0, rest = Bd[0].contiguous(), Bd[1:].contiguous()
    pars = workload_params(dlz, w, dlz.F32, name=C2)
    solve_step(dlz, op, b0, rest, pars, True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    ok, allst = solve_step(dlz, op, b0, rest, pars, True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    _, pst = solve_step(dlz, op, b0, rest, pars, True, profile=True)
    roof = kernel_roofline(pst[1:], 1, peaks, src, "k_minres_k1 (fused FP32 Q stencil + MinRes update, 11 RHS)")
    return {"workload": C2, "kappa": kappa, "value": round(ok / (ms / 1e3), 4), "unit": UNIT,
            "ms_per_step": round(ms, 1), "solved": ok,
            "phase_seconds": {"first_rhs_dr": round(allst[0].seconds, 4),
                              "deflated_11_rhs": round(sum(s.seconds for s in allst[1:]), 4)},
            "roofline_k_minres_k1": roof}


def cpu_baseline(iters_per_rhs, first_rhs_mvps, nrhs, budget_s=20.0, source=""):
    """The FP64 oracle as it stands, on a bounded sample of the same workload: CG on
    the normal equations (oracle.krylov.cgnr with the plain-C Wilson operator) on the
    24^3x48 lattice for about `budget_s` seconds.  RHS/s extrapolates its seconds per
    MVP to one step of the FP64 algorithm: the first right-hand side's MVPs plus
    2 MVPs per D-CG iteration for each of the other right-hand sides."""
    import numpy as np

    from oracle import cwilson, krylov
    w, dims, U, kappa, B = workload_inputs(rhs=(1,))
    D = cwilson.operator(U, kappa, dims, "D")
    Dd = cwilson.operator(U, kappa, dims, "Ddag")
    b = B[0].reshape(-1)
    it = 2
    while True:
        t0 = time.perf_counter()
        x, info = krylov.cgnr(D, Dd, b, tol=1e-30, maxiter=it)
        el = time.perf_counter() - t0
        if el >= budget_s / 3 or it >= 4096:
            break
        it *= 2
    mv = 2 * it + 2
    s_per_mvp = el / mv
    step_mvps = first_rhs_mvps + (nrhs - 1) * (2 * iters_per_rhs + 2)
    threads = os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count())
    return {"value": round(nrhs / (s_per_mvp * step_mvps), 8), "unit": UNIT, "cores": int(threads),
            "kind": "oracle",
            "sample": (f"oracle CGNR, {it} iterations ({mv} MVPs) on 24^3x48 in {el:.1f} s on "
                       f"{platform.machine()}; RHS/s extrapolated to {step_mvps} MVPs per 49-RHS step "
                       f"(MVP counts of the FP64 algorithm from {source})")}


def run_reference(args):
    """The oracle timed as it stands on the host cores (rank 0 only): each step is a
    bounded sample of the workload (oracle CG on the normal equations, 24^3x48, a fixed
    number of iterations); RHS/s is extrapolated to the FP64 algorithm's MVPs per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import cwilson, krylov
    w, dims, U, kappa, B = workload_inputs(args.kappa, rhs=(1,))
    D = cwilson.operator(U, kappa, dims, "D")
    Dd = cwilson.operator(U, kappa, dims, "Ddag")
    b = B[0].reshape(-1)
    it = args.ref_iters
    for _ in range(args.warmup):
        krylov.cgnr(D, Dd, b, tol=1e-30, maxiter=2)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        krylov.cgnr(D, Dd, b, tol=1e-30, maxiter=it)
    el = time.perf_counter() - t0
    mv = args.steps * (2 * it + 2)
    nrhs = workload_rhs_count()
    step_mvps = REF_FIRST_RHS_MVPS + (nrhs - 1) * (2 * REF_ITERS_PER_RHS + 2)
    value = nrhs / (el / mv * step_mvps)
    threads = os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count())
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 8), "unit": UNIT,
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded SU(3) links exp(0.3iH), seeded complex Gaussian RHS)",
           "config": {"workload": WORKLOAD, "lattice": list(dims), "kappa": kappa, "m": w["m"], "k": w["k"],
                      "rhs": nrhs, "form": "oracle (FP64 CPU)", "tol": 1e-10,
                      "timed": f"per step {it} oracle CG iterations on the normal equations (one RHS)",
                      "parallelism": "rank 0 only"},
           "cpu_baseline": {"value": round(value, 8), "unit": UNIT, "cores": int(threads), "kind": "oracle",
                            "sample": (f"{args.steps} x {it} oracle CGNR iterations ({mv} MVPs) in {el:.1f} s; "
                                       f"RHS/s extrapolated to {step_mvps} MVPs per 49-RHS step (first RHS "
                                       f"{REF_FIRST_RHS_MVPS} MVPs + 48 x {REF_ITERS_PER_RHS} D-CG iterations, "
                                       f"counts of the FP64 algorithm taken from an FP64 run of the library)")},
           "e2e": {"value": round(value, 8), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_stencil_only(args):
    """The Wilson stencil alone, as the solvers launch it: FP32 batched over `nrhs`
    right-hand sides and FP64 single, on the benchmark lattice (or --lattice),
    timed with CUDA events over back-to-back launches.  Prints one JSON line."""
    import torch

    import synth
    from paper_0901_3163_gb300 import dlz
    dims = tuple(int(v) for v in args.lattice.split("x")) if args.lattice else synth.WORKLOADS[WORKLOAD]["dims"]
    V = synth.volume(dims)
    U = synth.su3_links(dims, 2)
    op = dlz.create_operator(dims, torch.from_numpy(U).cuda(), 0.25)
    out = {"mode": "stencil-only", "lattice": list(dims)}
    peaks, src = _peaks()
    for name, dt, nrhs in (("f32_batched", torch.complex64, args.nrhs), ("f64_single", torch.complex128, 1)):
        x = torch.randn((nrhs, V, 4, 3), dtype=dt, device="cuda")
        st = dlz.stencil_bench(op, x, args.stencil_iters)
        ms = st["ms"]
        real = 4 if dt == torch.complex64 else 8
        nbytes = V * (48 * nrhs + (48 if real == 4 else 72)) * real
        out[name] = {"nrhs": nrhs, "avg_launch_ms": round(ms, 5), "bytes_per_launch": nbytes,
                     "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                     "frac_hbm": round(nbytes / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                     "fp_tflops": round(1368 * V * nrhs / (ms * 1e-3) / 1e12, 3)}
    print(json.dumps(out), flush=True)


def run_ncu_case(args):
    """A short run of the benchmark's kernels for ncu captures.  cg (cg-eo): 48 fused
    FP32 CGNR iterations (full or even-odd operator) on 16 Gaussian RHS of the 16^3x32
    lattice, the launch shape of the 24^3x48 step on ~3 GB of device memory; cg24: the
    same on the 24^3x48 lattice (~7 GB).  minres: the 16^3x32 operator, MinRes-DR(100,40) for 2 cycles, then
    48 FP32 D-MinRes iterations on the 11 point sources.  ptc: one forward and
    backward of the learned-seed network on 16^4.  Prints the stats."""
    import torch

    import synth
    from paper_0901_3163_gb300 import dlz
    if args.ncu_case == "ptc":
        from paper_0901_3163_gb300 import ptc_train as T
        dims4 = (16, 16, 16, 16)
        op4 = dlz.create_operator(dims4, torch.from_numpy(synth.su3_links(dims4, 1000)).cuda(), 0.25)
        net = dlz.net_create(op4, T.default_widths(), T.init_weights(T.default_widths(), 1))
        gen = torch.Generator(device="cuda")
        gen.manual_seed(0)
        x = T.noise(torch, op4, 4, gen)
        f = dlz.net_forward(net, x)
        dlz.net_backward(net, f)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "ncu-case", "case": "ptc"}))
        return
    if args.ncu_case in ("cg", "cg-eo", "cg24"):
        # the fused CGNR kernels as the 24^3x48 step launches them (16 RHS per launch): on
        # the 16^3x32 lattice so that the device holds ~3 GB (cg, cg-eo), or on the
        # 24^3x48 lattice itself (cg24, ~7 GB); FP32 CG on the normal equations without
        # deflation, 48 iterations (inputs larger than L2)
        if args.ncu_case == "cg24":
            w2, dims, U, kappa, _ = workload_inputs(args.kappa, rhs=())
        else:
            w2, dims, U, kappa, _ = workload_inputs(name=C2, rhs=())
        mk = dlz.create_operator_eo if args.ncu_case == "cg-eo" else dlz.create_operator
        op = mk(dims, torch.from_numpy(U).cuda(), kappa)
        B = synth.gaussian_spinors(dims, list(range(1, 17)))
        if args.ncu_case == "cg-eo":
            B = B[:, ::2].copy()
        pd = dlz.params_default(m=100, k=40, tol=1e-10, max_iter=48, precision=dlz.F32)
        _, sts = dlz.dcg(op, None, torch.from_numpy(B).cuda(), pd)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "ncu-case", "case": args.ncu_case, "d_iterations": [s.iterations for s in sts]}))
        return
    w, dims, U, kappa, B = workload_inputs(name=C2)
    op = dlz.create_operator(dims, torch.from_numpy(U).cuda(), kappa)
    Bd = torch.from_numpy(B).cuda()
    p = dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_cycles=2, max_iter=12, precision=dlz.F32)
    _, d, st = dlz.minresdr(op, Bd[0].contiguous(), p)
    pd = dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_iter=48, precision=dlz.F32)
    _, sts = dlz.dminres(op, d, Bd[1:].contiguous(), pd)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "ncu-case", "dr": st.as_dict(), "d_iterations": [s.iterations for s in sts]}))


def run_learned_seed(args):
    """The learned deflation seed on the 16^4 lattice (kappa 0.25, the same link
    recipe): Lan-DR(100,40) eigenvectors of `--ls-train` training fields (gauge
    seeds 1000...), Adam training of the 1 -> 12 -> 16 -> 1 PTC network for
    `--ls-steps` steps of 4 noise vectors, then on `--ls-test` held-out fields
    (gauge seeds 2000...) the seeded Rayleigh-Ritz set against plain Lan-DR at an
    equal MVP budget and the untrained network: median Ritz residuals and D-CG
    iterations on 4 Gaussian right-hand sides.  Also times the network's forward
    and backward launches.  Prints one JSON line."""
    import numpy as np
    import torch

    import synth
    from paper_0901_3163_gb300 import dlz
    from paper_0901_3163_gb300 import ptc_train as T
    dims, kappa, m, k = (16, 16, 16, 16), 0.25, 100, 40
    V = synth.volume(dims)
    t0 = time.perf_counter()
    train_ops, train_defl, lan_s = [], [], []
    for i in range(args.ls_train):
        op = dlz.create_operator(dims, torch.from_numpy(synth.su3_links(dims, 1000 + i)).cuda(), kappa)
        b = torch.from_numpy(synth.gaussian_spinor(dims, 0)).cuda()
        ta = time.perf_counter()
        _, d, st = dlz.landr(op, b, dlz.params_default(m=m, k=k, tol=1e-10, max_cycles=400))
        torch.cuda.synchronize()
        lan_s.append(time.perf_counter() - ta)
        train_ops.append(op)
        train_defl.append(d)
    t_data = time.perf_counter() - t0
    widths = T.default_widths()
    W0 = T.init_weights(widths, 1)
    net = dlz.net_create(train_ops[0], widths, W0)
    net0 = dlz.net_create(train_ops[0], widths, W0)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    x = T.noise(torch, train_ops[0], 4, gen)
    f = dlz.net_forward(net, x)
    dlz.net_backward(net, f)
    dlz.net_zero_grad(net)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    torch.cuda.synchronize()
    e0.record()
    for _ in range(5):
        dlz.net_forward(net, x, out=f)
    e1.record()
    for _ in range(5):
        dlz.net_backward(net, f)
    e2.record()
    torch.cuda.synchronize()
    dlz.net_zero_grad(net)
    fw_ms, bw_ms = e0.elapsed_time(e1) / 5, e1.elapsed_time(e2) / 5
    fl = sum(9 * widths[i] * (widths[i + 1] * 48 + 36) * 8 for i in range(len(widths) - 1)) * V * 4
    t1 = time.perf_counter()
    hist = T.train(torch, net, train_ops, train_defl, steps=args.ls_steps, nvec=4, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    evals = []
    for j in range(args.ls_test):
        op = dlz.create_operator(dims, torch.from_numpy(synth.su3_links(dims, 2000 + j)).cuda(), kappa)
        bl = [torch.from_numpy(synth.gaussian_spinor(dims, s)).cuda() for s in (0, 1, 2, 3, 4)]
        evals.append(T.evaluate(torch, net, op, bl, m, k, seed=j, net_untrained=net0))
    med = lambda key: float(np.median([e[key] for e in evals]))  # noqa: E731
    mean_it = lambda key: float(np.mean([np.mean(e[key]) for e in evals]))  # noqa: E731
    out = {"mode": "learned-seed", "workload": "16^4 kappa 0.25, PTC 1-12-16-1, Lan-DR(100,40)",
           "train_fields": args.ls_train, "test_fields": args.ls_test, "steps": args.ls_steps,
           "data_seconds": round(t_data, 2), "lanczos_seconds_per_field": round(float(np.mean(lan_s)), 3),
           "train_seconds": round(t_train, 2), "loss_first20": round(float(np.mean(hist[:20])), 5),
           "loss_last20": round(float(np.mean(hist[-20:])), 5),
           "forward_ms_4vec": round(fw_ms, 3), "backward_ms_4vec": round(bw_ms, 3),
           "forward_tflops": round(fl / (fw_ms * 1e-3) / 1e12, 2),
           "backward_tflops": round(2 * fl / (bw_ms * 1e-3) / 1e12, 2),
           "per_field": evals,
           "ritz_median": {"seed": med("ritz_median_seed"), "untrained": med("ritz_median_untrained"),
                           "plain_equal_mvps": med("ritz_median_plain"),
                           "plain_one_m_cycle": med("ritz_median_plain_m_cycle")},
           "dcg_iterations_mean": {"seed": mean_it("dcg_iters_seed"), "plain_equal_mvps": mean_it("dcg_iters_plain_equal"),
                                   "plain_one_m_cycle": mean_it("dcg_iters_plain_cycle"),
                                   "undeflated": mean_it("cg_iters_undeflated")},
           "chosen": [e["chosen"] for e in evals], "all_converged": all(e["converged"] for e in evals)}
    print(json.dumps(out), flush=True)


def run_saturation(args):
    """Lan-DR(200, k) for k = 20, 60, 100, 150 (Sec. 2 runs m = 200 with k = 20, 60, 150)
    on the 16^3x32 lattice at its kappa, first Gaussian RHS (seed 0), FP64: the first
    right-hand side's MVPs, then D-CG on 4 Gaussian RHS (seeds 1..4) over each
    deflation set, and plain CG (no deflation) on the same RHS.  Saturation (Sec. 2):
    the D-CG iteration count stops falling once the deflated rate matches the rate CG
    reaches after its deflation knee.  Also Lan-DR(200,150) as a pure eigensolver
    (eig_only): cycles, MVPs and seconds until all 150 kept Ritz residuals converge.
    Prints one JSON line."""
    import torch

    import synth
    from paper_0901_3163_gb300 import dlz
    w, dims, U, kappa, _ = workload_inputs(name=C2, rhs=())
    op = dlz.create_operator(dims, torch.from_numpy(U).cuda(), kappa)
    b0 = torch.from_numpy(synth.gaussian_spinor(dims, 0)).cuda()
    B = torch.from_numpy(synth.gaussian_spinors(dims, (1, 2, 3, 4))).cuda()
    # FP64 throughout (the paper's study): an FP32 Lan-DR on D^dag D stalls with its lowest
    # Ritz residuals near 1e-5, above the smallest eigenvalues at this kappa, so the
    # deflation sets it hands on would not show what k alone does
    pd = dlz.params_default(m=200, k=20, tol=1e-10, max_iter=200000, precision=dlz.F64)
    rows = []
    t0 = time.perf_counter()
    _, sts = dlz.dcg(op, None, B, pd)
    torch.cuda.synchronize()
    rows.append({"k": 0, "dcg_iterations": [s.iterations for s in sts], "dcg_seconds": round(time.perf_counter() - t0, 3),
                 "verified": all(s.converged == 1 and s.true_residual <= 1e-10 for s in sts)})
    for k in args.sat_k:
        p = dlz.params_default(m=200, k=k, tol=1e-10, max_cycles=2000, precision=dlz.F64, finish=1)
        t0 = time.perf_counter()
        _, d, st = dlz.landr(op, b0, p)
        torch.cuda.synchronize()
        t_dr = time.perf_counter() - t0
        t0 = time.perf_counter()
        _, sts = dlz.dcg(op, d, B, pd)
        torch.cuda.synchronize()
        rows.append({"k": k, "first_rhs_mvps": int(st.mvps), "first_rhs_cycles": st.cycles,
                     "first_rhs_seconds": round(t_dr, 3), "first_rhs_verified": st.converged == 1,
                     "dcg_iterations": [s.iterations for s in sts], "dcg_seconds": round(time.perf_counter() - t0, 3),
                     "verified": all(s.converged == 1 and s.true_residual <= 1e-10 for s in sts)})
        del d
    p = dlz.params_default(m=200, k=150, tol=1e-10, max_cycles=4000, precision=dlz.F32, eig_only=1)
    # (the eigensolver row: FP32 form, kept residuals to 1e-5 ||A||)
    t0 = time.perf_counter()
    _, d, st = dlz.landr(op, b0, p)
    torch.cuda.synchronize()
    t_e = time.perf_counter() - t0
    kk, _ = dlz.defl_count(d)
    vals = [dlz.defl_get(d, i) for i in range(kk)]
    out = {"mode": "saturation", "workload": f"{C2} kappa {kappa}, Lan-DR(200,k) FP64, D-CG on 4 Gaussian RHS",
           "rows": rows,
           "eigensolver_k150": {"converged": st.converged == 1, "cycles": st.cycles, "mvps": int(st.mvps),
                                "seconds": round(t_e, 3), "lowest": vals[0][0], "highest_kept": vals[-1][0],
                                "max_ritz_residual": max(v[1] for v in vals)}}
    print(json.dumps(out), flush=True)


def run_gmresdr(args):
    """GMRES-DR(m,k) and D-GMRES(m) on D itself (FP64; the non-hermitian methods the
    paper contrasts with) beside MinRes-DR(m,k) + D-MinRes (FP64, the paper's hermitian
    method for the same D x = b) on one lattice: the first Gaussian RHS (seed 0) by the
    DR method, then 4 Gaussian RHS (seeds 1..4) by the deflated solver; MVPs, seconds
    and verified solves of each.  Lattice and kappa by --lattice / --kappa (default
    8^4 at kappa 0.25, gauge seed 3000).  Prints one JSON line."""
    import torch

    import synth
    from paper_0901_3163_gb300 import dlz
    dims = tuple(int(v) for v in args.lattice.split("x")) if args.lattice else (8, 8, 8, 8)
    kappa = args.kappa if args.kappa is not None else 0.25
    op = dlz.create_operator(dims, torch.from_numpy(synth.su3_links(dims, 3000)).cuda(), kappa)
    b0 = torch.from_numpy(synth.gaussian_spinor(dims, 0)).cuda()
    B = torch.from_numpy(synth.gaussian_spinors(dims, (1, 2, 3, 4))).cuda()
    m, k = args.gm_m, args.gm_k
    out = {"mode": "gmresdr", "lattice": list(dims), "kappa": kappa, "m": m, "k": k}
    for name, dr, ds in (("gmresdr_dgmres", dlz.gmresdr, dlz.dgmres), ("minresdr_dminres", dlz.minresdr, dlz.dminres)):
        p = dlz.params_default(m=m, k=k, tol=1e-10, max_cycles=2000, max_iter=200000)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, d, st = dr(op, b0, p)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        _, sts = ds(op, d, B, p)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out[name] = {"first_rhs": {"seconds": round(t1 - t0, 3), "mvps": int(st.mvps), "cycles": st.cycles,
                                   "verified": st.converged == 1},
                     "later_rhs": {"seconds": round(t2 - t1, 3), "mvps": [int(s.mvps) for s in sts],
                                   "verified": all(s.converged == 1 and s.true_residual <= 1e-10 for s in sts)}}
    _, stp = dlz.dgmres(op, None, B, dlz.params_default(m=m, k=k, tol=1e-10, max_iter=200000))
    out["plain_gmres_mvps"] = [int(s.mvps) for s in stp]
    print(json.dumps(out), flush=True)


def run_multi_lattice(args):
    """The uneven multi-lattice batch alone (the c4 key of the default line)."""
    import torch

    from paper_0901_3163_gb300 import dlz
    out = {"mode": "multi-lattice"}
    out.update(run_c4(dlz, torch, args.c4_lattices))
    print(json.dumps(out), flush=True)


def parser():
    """The command line of bench.py."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--plain-rhs", type=int, default=2,
                    help="D-CG right-hand sides of the plain FP64 form timed beside the chosen form")
    ap.add_argument("--k1-traffic", type=float, default=K1_TRAFFIC_BYTES,
                    help="ncu DRAM bytes per launch of the dominant kernel (None if not measured)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) leg")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-c4", action="store_true")
    ap.add_argument("--c2", action="store_true", help="add the 16^3x32 workload (c2 key)")
    ap.add_argument("--no-c2", action="store_true", help="(the default; kept for recorded command lines)")
    ap.add_argument("--no-evenodd", action="store_true")
    ap.add_argument("--c4-lattices", type=int, default=64)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-iters", type=int, default=16, help="oracle CGNR iterations per reference step")
    ap.add_argument("--stencil-only", action="store_true")
    ap.add_argument("--lattice", default=None)
    ap.add_argument("--nrhs", type=int, default=16)
    ap.add_argument("--stencil-iters", type=int, default=50)
    ap.add_argument("--ncu-case", nargs="?", const="minres", default=None,
                    choices=["minres", "cg", "cg-eo", "cg24", "ptc"])
    ap.add_argument("--learned-seed", action="store_true")
    ap.add_argument("--multi-lattice", action="store_true")
    ap.add_argument("--saturation", action="store_true")
    ap.add_argument("--gmresdr", action="store_true")
    ap.add_argument("--gm-m", type=int, default=40)
    ap.add_argument("--gm-k", type=int, default=10)
    ap.add_argument("--sat-k", type=int, nargs="+", default=[20, 60, 100, 150])
    ap.add_argument("--ls-train", type=int, default=32)
    ap.add_argument("--ls-test", type=int, default=8)
    ap.add_argument("--ls-steps", type=int, default=400)
    ap.add_argument("--kappa", type=float, default=None,
                    help="override the tabulated kappa (profiling and trial runs only)")
    return ap


def main():
    args = parser().parse_args()
    if args.stencil_only:
        run_stencil_only(args)
    elif args.ncu_case is not None:
        run_ncu_case(args)
    elif args.learned_seed:
        run_learned_seed(args)
    elif args.multi_lattice:
        run_multi_lattice(args)
    elif args.saturation:
        run_saturation(args)
    elif args.gmresdr:
        run_gmresdr(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
