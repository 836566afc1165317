"""Benchmark: right-hand sides solved per second to ||b - D x|| / ||b|| < 1e-10.

Workload (one step): the 16^3x32 Wilson lattice with SU(3) links
U = exp(0.3 i H) (gauge seed 2) at the kappa where min|eig(gamma5 D)| = 1e-3;
MinRes-DR(100,40) on the point source at the origin (spin 0, colour 0), then
D-MinRes on the other 11 spin-colour point sources (arXiv:0901.3163, Sec. 2
method on a synthetic stand-in for its quenched lattice).  Every right-hand
side counts only if its true residual was verified in FP64.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--form chosen|plain]
                    [--plain-steps P] [--impl ours|reference]

`value` is the chosen form (FP32 Lanczos/MinRes with FP64 defect correction,
right-hand sides batched); the plain FP64 form (one RHS at a time, FP64
stencil) is timed beside it on the same operator (`plain_fp64`).

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

WORKLOAD = "wilson_16x16x16x32"
# restart cycles of the first right-hand side's MinRes-DR phase (both forms)
DR_CYCLES = 150
# MVPs per right-hand side of the FP64 form of the workload (150 MinRes-DR(100,40)
# cycles + finish: 13968 MVPs; D-MinRes: 7648 each for the other 11), the unit the
# oracle's timing is extrapolated with when no FP64 GPU run is at hand
REF_MVPS_PER_RHS = 8175
# DRAM bytes (read + write) of one k_minres_k1 launch with 11 right-hand sides on the
# 16^3x32 lattice, from one ncu capture of the current kernel
# (ncu --set full -k regex:k_minres_k1 -s 24 -c 1 python bench.py --ncu-case)
K1_TRAFFIC_BYTES = 745467648 + 376429824
METRIC = "RHS solved/s to |r|/|b|<1e-10 (MinRes-DR(100,40) + D-MinRes, 12 point sources, 16^3x32)"
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


def workload_inputs(kappa=None):
    import numpy as np

    import synth
    w = synth.WORKLOADS[WORKLOAD]
    dims = w["dims"]
    U = synth.su3_links(dims, w["gauge_seed"])
    if kappa is None:
        kappa = synth.kappa_for(dims, w["gauge_seed"])
    V = synth.volume(dims)
    B = np.zeros((12, V, 4, 3), dtype=np.complex128)
    for a in range(12):
        B[a] = synth.point_source(dims, a // 3, a % 3)
    return w, dims, U, kappa, B


def workload_params(dlz, w, pr):
    """Solver parameters of one benchmark step (first RHS, then the other 11).

    First RHS: DR_CYCLES MinRes-DR(100,40) restart cycles (run past linear convergence
    so that the 40 harmonic Ritz vectors converge), then D-MinRes from that x over the
    40 vectors; the same schedule in both forms.  Re-orthogonalisation against the kept
    vectors every 30 Lanczos steps (the paper gives no period): 5% faster per step than
    every 10, same D-MinRes iterations."""
    p_dr = dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_cycles=DR_CYCLES, check_every=16,
                              precision=pr, oversolve=1e9, finish=1, reorth_period=30)
    p_d = dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_iter=200000, precision=pr,
                             check_every=16)
    return p_dr, p_d


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
    w, dims, U, kappa, B = workload_inputs()
    op = dlz.create_operator(dims, torch.from_numpy(U).to(dev), kappa)
    Bd = torch.from_numpy(B).to(dev)
    b0, rest = Bd[0].contiguous(), Bd[1:].contiguous()
    prec = dlz.F32 if args.form == "chosen" else dlz.F64

    def params(pr):
        return workload_params(dlz, w, pr)

    pars = params(prec)

    def step(profile=False, host=None, pp=None):
        p_dr, p_d = pp or pars
        p_dr.profile = p_d.profile = int(profile)
        if host is None:
            x0, defl, st = dlz.minresdr(op, b0, p_dr)
            X, sts = dlz.dminres(op, defl, rest, p_d)
        else:
            hb0, hrest, hx0, hX = host
            x0, defl, st = dlz.minresdr(op, hb0, p_dr, x=hx0)
            X, sts = dlz.dminres(op, defl, hrest, p_d, X=hX)
        allst = [st] + list(sts)
        ok = sum(1 for s in allst if s.converged == 1 and s.true_residual <= 1e-10)
        return ok, allst

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    solved = 0
    stats = []
    for _ in range(args.steps):
        ok, allst = step()
        solved += ok
        stats.extend(allst)
    e1.record()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    # one more step with every stencil launch timed by CUDA events (roofline only)
    _, pstats = step(profile=True)
    ms_max, solved_all = aggregate_ranks(ms, solved, world, dev)
    value = solved_all / (ms_max / 1e3)
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
        for _ in range(max(1, args.steps)):
            ok, _ = step(host=(hb0, hrest, hx0, hX))
            e2e_solved += ok
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e_value = e2e_solved / e2e_s * world
        e2e = {"value": round(e2e_value, 4), "unit": UNIT,
               "h2d_bytes_per_step": int(B.nbytes), "d2h_bytes_per_step": int(B.nbytes)}
    # roofline of the dominant kernel (the Wilson stencil), timed with events inside the steps
    # the dominant kernel is the stencil of the deflated phase (all 11 right-hand sides
    # batched into each launch in the mixed form); the first-RHS phase is reported apart
    dstats = pstats[1:]
    st_ms = sum(s.stencil_ms for s in dstats)
    st_n = sum(s.stencil_launches for s in dstats)
    st_bytes = sum(s.stencil_bytes for s in dstats)
    avg_ms = st_ms / max(st_n, 1)
    bytes_per_launch = st_bytes / max(st_n, 1)
    # flops: 1368 per site and right-hand side (bytes / reals-per-site gives site-RHS pairs)
    real = 8 if prec == dlz.F64 else 4
    peaks, src = _peaks()
    if prec == dlz.F64:
        # FP64 stencil, one right-hand side per launch: 1368 flops per 960 bytes is past
        # the ridge of GB300's FP64 pipe, so the roofline is the FP64 ALU rate
        nflops = bytes_per_launch / (120 * real) * 1368
        peak = 1.25
        roof = {"bound": "alu", "achieved": round(nflops / (avg_ms * 1e-3) / 1e12, 4),
                "peak": peak, "unit": "TFLOP/s FP64",
                "frac": round(nflops / (avg_ms * 1e-3) / 1e12 / peak, 4),
                "peak_source": "nominal GB300 FP64 (1.25 TFLOP/s); measured FMA probe 1.01 at 1987 MHz",
                "hbm_gbs": round(bytes_per_launch / (avg_ms * 1e-3) / 1e9, 1),
                "traffic": None, "kernel": "k_wilson<double>", "avg_launch_ms": round(avg_ms, 5),
                "bytes_per_launch": int(bytes_per_launch)}
    else:
        # the fused MinRes kernel K1 (Q stencil + update epilogue, 11 right-hand sides per
        # launch): 192 spinor reals per site and RHS + 48 link reals per site, FP32
        ach = bytes_per_launch / (avg_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(ach / peaks["hbm_gbs"], 4), "peak_source": src,
                "traffic": args.k1_traffic,
                "kernel": "k_minres_k1 (fused FP32 Q stencil + MinRes update, 11 RHS per launch)",
                "avg_launch_ms": round(avg_ms, 5), "launches_timed": int(st_n),
                "bytes_per_launch": int(bytes_per_launch)}
    dr_s = sum(s.seconds for s in stats[0::12]) / max(args.steps, 1)
    d_s = sum(s.seconds for i, s in enumerate(stats) if i % 12) / max(args.steps, 1)
    launches = sum(s.gpu_launches for s in stats)      # all timed steps (this library's kernels)
    mvps = sum(s.mvps for s in stats) // max(args.steps, 1)
    iters = [s.iterations for s in stats[:12]]
    extra = {}
    if args.form == "chosen" and args.plain_steps > 0:
        # the plain FP64 form on the same operator: one RHS at a time, FP64 stencil
        pp = params(dlz.F64)
        # warm-up of the FP64 kernels: two restart cycles and a short D-MinRes
        wdr = dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_cycles=2, precision=dlz.F64)
        _, wd, _ = dlz.minresdr(op, b0, wdr)
        dlz.dminres(op, wd, rest[:1].contiguous(), dlz.params_default(max_iter=32, precision=dlz.F64))
        del wd
        barrier()
        t0 = time.perf_counter()
        solved_p = 0
        pst = []
        for _ in range(args.plain_steps):
            ok, allst = step(pp=pp)
            solved_p += ok
            pst.extend(allst)
        barrier()
        el = time.perf_counter() - t0
        plain_mvps = sum(s.mvps for s in pst) // args.plain_steps
        extra["plain_fp64"] = {"value": round(solved_p / el, 4), "unit": UNIT, "steps": args.plain_steps,
                               "warmup": "2 restart cycles + 32 D-MinRes iterations",
                               "ms_per_step": round(el / args.plain_steps * 1e3, 1),
                               "mvps_per_step": int(plain_mvps),
                               "iterations_first_steps": [s.iterations for s in pst[:12]]}
        extra["chosen_over_plain"] = round(value / (solved_p / el), 3)
    # the Wilson stencil alone (Dslash), as the solvers launch it
    V = int(np.prod(dims))
    ds = {}
    for name, dt, nrhs in (("f32_batch11", torch.complex64, 11), ("f64_single", torch.complex128, 1)):
        xs = torch.randn((nrhs, V, 4, 3), dtype=dt, device=dev)
        ms_l = dlz.stencil_bench(op, xs, 50)["ms"]
        real = 4 if dt == torch.complex64 else 8
        nb = V * (48 * nrhs + (48 if real == 4 else 72)) * real
        ds[name] = {"avg_launch_ms": round(ms_l, 5), "gbs": round(nb / (ms_l * 1e-3) / 1e9, 1),
                    "frac_hbm": round(nb / (ms_l * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}
        del xs
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == dlz.F64 else "f32+f64",
        "data": "synthetic (seeded SU(3) links exp(0.3iH), point sources)",
        "config": {"workload": WORKLOAD, "lattice": list(dims), "kappa": kappa, "m": w["m"], "k": w["k"],
                   "rhs": 12, "form": args.form, "tol": 1e-10,
                   "l2": "inputs and Krylov basis (2.5 GB) larger than L2; no flush",
                   "first_rhs": f"{DR_CYCLES} MinRes-DR cycles, then D-MinRes from x",
                   "parallelism": f"replicas x{world}"},
        "e2e": e2e,
        "gpu_launches": int(launches), "gpu_launches_per_step": int(launches // max(args.steps, 1)),
        "library_kernels": "cuBLAS SGEMM for the restart V P (3 kernels per restart, not counted above)",
        "mvps_per_step": int(mvps), "iterations_first_steps": iters,
        "phase_seconds": {"first_rhs_dr": round(dr_s, 4), "deflated_11_rhs": round(d_s, 4)},
        "d_phase_rhs_per_s": round(11.0 / d_s, 4) if d_s > 0 else None,
        "roofline": roof, "dslash": ds, "clocks": clk,
    }
    out.update(extra)
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle runs the FP64 algorithm: extrapolate to the FP64 form's MVP count
        ref_mvps = extra.get("plain_fp64", {}).get("mvps_per_step", REF_MVPS_PER_RHS * 12)
        out["cpu_baseline"] = cpu_baseline(ref_mvps, budget_s=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline(mvps_per_step, budget_s=20.0):
    """The FP64 oracle as it stands, on a bounded sample of the same workload:
    MinRes-DR(100,40) cycles on the 16^3x32 lattice for about `budget_s` seconds;
    the RHS/s figure extrapolates its seconds per MVP (Lanczos steps, restarts and
    residual checks included) to the MVPs one step of the workload needs."""
    import numpy as np

    from oracle import cwilson, krylov, wilson
    w, dims, U, kappa, B = workload_inputs()
    Q = cwilson.operator(U, kappa, dims, "Q")
    b = wilson.apply_gamma5(B[0]).reshape(-1)
    t0 = time.perf_counter()
    cycles = 1
    while True:
        r = krylov.minresdr(Q, b, w["m"], w["k"], tol=1e-10, max_cycles=cycles)
        el = time.perf_counter() - t0
        if el >= budget_s or cycles >= 8:
            break
        cycles += 1
    # time the last run only
    t1 = time.perf_counter()
    r = krylov.minresdr(Q, b, w["m"], w["k"], tol=1e-10, max_cycles=max(1, cycles - 1))
    el = time.perf_counter() - t1
    s_per_mvp = el / max(r.info.mvps, 1)
    rhs_per_s = 12.0 / (s_per_mvp * max(mvps_per_step, 1))
    threads = os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count())
    return {"value": round(rhs_per_s, 6), "unit": UNIT, "cores": int(threads), "kind": "oracle",
            "sample": (f"oracle MinRes-DR(100,40), {r.cycles} cycle(s) = {r.info.mvps} MVPs in "
                       f"{el:.1f} s on {platform.machine()}; RHS/s extrapolated to "
                       f"{mvps_per_step} MVPs per 12-RHS step")}


def run_reference(args):
    """The oracle timed as it stands on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import cwilson, krylov, wilson
    w, dims, U, kappa, B = workload_inputs()
    Q = cwilson.operator(U, kappa, dims, "Q")
    b = wilson.apply_gamma5(B[0]).reshape(-1)
    # one bounded sample per step: one MinRes-DR(100,40) cycle (m Lanczos steps + restart)
    mvps_per_rhs = args.ref_mvps_per_rhs
    for _ in range(args.warmup):
        krylov.minresdr(Q, b, w["m"], w["k"], tol=1e-10, max_cycles=1)
    t0 = time.perf_counter()
    mv = 0
    for _ in range(args.steps):
        r = krylov.minresdr(Q, b, w["m"], w["k"], tol=1e-10, max_cycles=1)
        mv += r.info.mvps
    el = time.perf_counter() - t0
    value = 1.0 / (el / mv * mvps_per_rhs)
    threads = os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count())
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded SU(3) links exp(0.3iH), point sources)",
           "config": {"workload": WORKLOAD, "lattice": list(dims), "kappa": kappa, "m": w["m"], "k": w["k"],
                      "rhs": 12, "form": "oracle (FP64 CPU)", "tol": 1e-10,
                      "first_rhs": f"{DR_CYCLES} MinRes-DR cycles, then D-MinRes from x",
                      "parallelism": "rank 0 only"},
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": int(threads),
                            "kind": "oracle",
                            "sample": (f"per step one MinRes-DR(100,40) cycle ({mv // args.steps} MVPs); "
                                       f"RHS/s extrapolated at {mvps_per_rhs} MVPs per RHS")},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_stencil_only(args):
    """The Wilson stencil alone, as the solvers launch it: FP32 batched over `nrhs`
    right-hand sides and FP64 single, on the benchmark lattice (or --lattice),
    timed with CUDA events over back-to-back launches (inputs larger than L2
    when nrhs * 12.6 MB + links exceed 129 MB).  Prints one JSON line."""
    import numpy as np
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


def run_first_rhs_only(args):
    """One first-right-hand-side solve (MinRes-DR(100,40) on the point source) of
    the benchmark workload, for profiling the restart cycles; prints its stats.
    --kappa overrides the tabulated kappa (profiling runs only)."""
    import torch

    from paper_0901_3163_gb300 import dlz
    w, dims, U, kappa, B = workload_inputs(args.kappa)
    op = dlz.create_operator(dims, torch.from_numpy(U).cuda(), kappa)
    prec = dlz.F32 if args.form == "chosen" else dlz.F64
    p = dlz.params_default(m=w["m"], k=w["k"], tol=args.tol, max_cycles=args.max_cycles, precision=prec)
    x, d, st = dlz.minresdr(op, torch.from_numpy(B[0]).cuda(), p, deflate=True)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "first-rhs-only", "form": args.form, "kappa": kappa, "stats": st.as_dict()}))


def run_ncu_case(args):
    """A short run of the benchmark's kernels for ncu captures.  minres: the 16^3x32
    operator, a deflation set from 2 FP32 MinRes-DR(100,40) cycles (their
    finishing MinRes capped at 12 iterations), then 48 FP32 D-MinRes iterations
    on the 11 point sources batched (fused kernels with 11 right-hand sides per
    launch).  cg: the same with Lan-DR and D-CG on 11 Gaussian RHS.  ptc: one
    forward and backward of the learned-seed network on 16^4.  Prints the stats."""
    import torch

    import synth
    from paper_0901_3163_gb300 import dlz
    w, dims, U, kappa, B = workload_inputs()
    op = dlz.create_operator(dims, torch.from_numpy(U).cuda(), kappa)
    Bd = torch.from_numpy(B).cuda()
    if args.ncu_case == "ptc":
        # the learned-seed network on a 16^4 lattice: one forward and one backward of 4 vectors
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
    if args.ncu_case == "cg":
        # FP32 Lan-DR(100,40) for 2 cycles, then 48 fused CGNR iterations on 11 Gaussian RHS
        p = dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_cycles=2, max_iter=12, precision=dlz.F32)
        _, d, st = dlz.landr(op, Bd[0].contiguous(), p)
        G = torch.from_numpy(synth.gaussian_spinors(dims, list(range(1, 12)))).cuda()
        pd = dlz.params_default(m=w["m"], k=w["k"], tol=1e-10, max_iter=48, precision=dlz.F32)
        _, sts = dlz.dcg(op, d, G, pd)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "ncu-case", "case": "cg", "d_iterations": [s.iterations for s in sts]}))
        return
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
    (gauge seeds 2000...) the seeded Rayleigh-Ritz set (40 MVPs) against one
    Lan-DR(100,40) cycle (100 MVPs) and the untrained network: median Ritz
    residuals and D-CG iterations on 4 Gaussian right-hand sides.  Also times
    the network's forward and backward launches.  Prints one JSON line."""
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
    # kernel timing: one forward and one backward of 4 vectors (CUDA events)
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
    # algorithmic flops: per layer, site and vector 9 c_in c_out 48 complex FMAs (spin
    # mixing) + 9 c_in 36 (transport), 8 real flops each; backward twice that
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
    med = lambda key: float(np.median([e[key] for e in evals]))
    mean_it = lambda key: float(np.mean([np.mean(e[key]) for e in evals]))
    out = {"mode": "learned-seed", "workload": "16^4 kappa 0.25, PTC 1-12-16-1, Lan-DR(100,40)",
           "train_fields": args.ls_train, "test_fields": args.ls_test, "steps": args.ls_steps,
           "data_seconds": round(t_data, 2), "lanczos_seconds_per_field": round(float(np.mean(lan_s)), 3),
           "train_seconds": round(t_train, 2), "loss_first20": round(float(np.mean(hist[:20])), 5),
           "loss_last20": round(float(np.mean(hist[-20:])), 5),
           "forward_ms_4vec": round(fw_ms, 3), "backward_ms_4vec": round(bw_ms, 3),
           "forward_tflops": round(fl / (fw_ms * 1e-3) / 1e12, 2),
           "backward_tflops": round(2 * fl / (bw_ms * 1e-3) / 1e12, 2),
           "ritz_median": {"seed": med("ritz_median_seed"), "untrained": med("ritz_median_untrained"),
                           "plain_one_cycle": med("ritz_median_plain")},
           "dcg_iterations_mean": {"seed": mean_it("dcg_iters_seed"), "plain_one_cycle": mean_it("dcg_iters_plain_cycle"),
                                   "undeflated": mean_it("cg_iters_undeflated")},
           "chosen": [e["chosen"] for e in evals], "all_converged": all(e["converged"] for e in evals)}
    print(json.dumps(out), flush=True)


def run_multi_lattice(args):
    """Uneven multi-lattice batching: 64 lattices (i mod 3 -> 8^4, 12^4, 16^4), links
    by the same recipe (gauge seed 3000 + i), per-lattice kappa drawn uniformly in
    [0.21, 0.24] (numpy default_rng(4000)); MinRes-DR(40,10) (FP32 form) on one
    Gaussian RHS per lattice, then D-MinRes on 8 Gaussian RHS per lattice (512 solves):
    all lattices through one dlz_batch_dminres call (FP32, one launch per stage for
    all slots) against the same solves lattice by lattice (dlz_dminres, FP32 batched per
    lattice) and, on one lattice of each size, the plain FP64 form.  Prints one JSON line."""
    import numpy as np
    import torch

    import synth
    from paper_0901_3163_gb300 import dlz
    sizes = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16)]
    nl = args.ml_lattices
    kap = np.random.default_rng(4000).uniform(0.21, 0.24, nl)
    t0 = time.perf_counter()
    ops, defls, Bs = [], [], []
    dr_s = 0.0
    for i in range(nl):
        dims = sizes[i % 3]
        op = dlz.create_operator(dims, torch.from_numpy(synth.su3_links(dims, 3000 + i)).cuda(), float(kap[i]))
        b0 = torch.from_numpy(synth.gaussian_spinor(dims, 0)).cuda()
        ta = time.perf_counter()
        _, d, st = dlz.minresdr(op, b0, dlz.params_default(m=40, k=10, tol=1e-10, max_cycles=400, precision=dlz.F32))
        torch.cuda.synchronize()
        dr_s += time.perf_counter() - ta
        ops.append(op)
        defls.append(d)
        Bs.append(torch.from_numpy(synth.gaussian_spinors(dims, list(range(1, 9)))).cuda())
    t_setup = time.perf_counter() - t0
    sites = sum(o.volume for o in ops)
    # inner tolerance 1e-5: on these small, well-conditioned lattices the FP64 restarts
    # cost more than the re-projections save (278 against 309 RHS/s with 1e-2)
    p32 = dlz.params_default(m=40, k=10, tol=1e-10, max_iter=100000, precision=dlz.F32, reliable_delta=1e-5)
    dlz.batch_dminres(ops, defls, Bs, p32)          # warm-up (graph capture, scratch)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    ta = time.perf_counter()
    Xs, sts = dlz.batch_dminres(ops, defls, Bs, p32)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - ta
    clk = clocks.stop()
    ok_batch = sum(1 for ss in sts for s in ss if s.converged == 1 and s.true_residual <= 1e-10)
    ta = time.perf_counter()
    ok_seq = 0
    for o, d, B in zip(ops, defls, Bs):
        _, ss = dlz.dminres(o, d, B, p32)
        ok_seq += sum(1 for s in ss if s.converged == 1 and s.true_residual <= 1e-10)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - ta
    p64 = dlz.params_default(m=40, k=10, tol=1e-10, max_iter=100000)
    ta = time.perf_counter()
    ok64, n64 = 0, 0
    for j in range(min(3, nl)):            # one lattice of each size
        _, ss = dlz.dminres(ops[j], defls[j], Bs[j], p64)
        ok64 += sum(1 for s in ss if s.converged == 1 and s.true_residual <= 1e-10)
        n64 += len(ss)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - ta
    iters = [max(s.iterations for s in ss) for ss in sts]
    out = {"mode": "multi-lattice", "workload": f"{nl} lattices 8^4/12^4/16^4, kappa U[0.21,0.24], "
                                                f"MinRes-DR(40,10) + D-MinRes x 8 RHS each",
           "lattices": nl, "sites_total": int(sites), "rhs_total": int(sum(len(ss) for ss in sts)),
           "setup_seconds": round(t_setup, 2), "first_rhs_dr_seconds": round(dr_s, 3),
           "batched": {"seconds": round(t_batch, 3), "rhs_per_s": round(ok_batch / t_batch, 2), "solved": ok_batch,
                       "iterations_max": int(max(iters))},
           "lattice_by_lattice_f32": {"seconds": round(t_seq, 3), "rhs_per_s": round(ok_seq / t_seq, 2),
                                      "solved": ok_seq},
           "plain_fp64_sample": {"lattices": 3, "rhs": n64, "seconds": round(t64, 3),
                                 "rhs_per_s": round(ok64 / t64, 3) if t64 > 0 else None},
           "batched_over_lattice_by_lattice": round((ok_batch / t_batch) / (ok_seq / t_seq), 3),
           "clocks": clk}
    print(json.dumps(out), flush=True)


def run_c3(args):
    """Precision and batching on the 24^3x48 lattice (gauge seed 3, kappa by the
    sigma_min = 1e-3 rule from synth/kappa_table.json, or --kappa): FP32 Lan-DR(120,60)
    on D^dag D for the first Gaussian RHS (seed 0), then FP32 D-CG with FP64 defect
    correction on 48 Gaussian RHS (seeds 1..48) in batches of 16 per launch; the
    plain FP64 D-CG timed on 2 of them; the bare stencil in FP32 and bfloat16 with
    16 RHS per launch.  Prints one JSON line."""
    import numpy as np
    import torch

    import synth
    from paper_0901_3163_gb300 import dlz
    dims = (24, 24, 24, 48)
    V = synth.volume(dims)
    if args.kappa is not None:
        kappa, ksrc = args.kappa, "given on the command line (not the sigma_min rule)"
    else:
        try:
            kappa, ksrc = synth.kappa_for(dims, 3), "sigma_min(D) = 1e-3 rule (oracle)"
        except KeyError:
            print(json.dumps({"mode": "c3", "unavailable": "kappa of the 24^3x48 seed-3 lattice not in the table"}))
            return
    t0 = time.perf_counter()
    op = dlz.create_operator(dims, torch.from_numpy(synth.su3_links(dims, 3)).cuda(), kappa)
    t_links = time.perf_counter() - t0
    peaks, src = _peaks()
    ds = {}
    for name, dt, real in (("f32", dlz.F32, 4), ("bf16", dlz.BF16, 2)):
        xs = torch.randn((16, V, 4, 3), dtype=torch.complex64, device="cuda")
        ms = dlz.stencil_bench(op, xs, 20, dtype=dt)["ms"]
        nb = V * (48 * 16 * real + 48 * 4)
        ds[name] = {"avg_launch_ms": round(ms, 4), "gbs": round(nb / ms / 1e6, 1),
                    "frac_hbm": round(nb / ms / 1e6 / peaks["hbm_gbs"], 4)}
        del xs
    b0 = torch.from_numpy(synth.gaussian_spinor(dims, 0)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, d, st = dlz.landr(op, b0, dlz.params_default(m=120, k=60, tol=1e-10, max_cycles=args.max_cycles,
                                                     precision=dlz.F32))
    torch.cuda.synchronize()
    t_dr = time.perf_counter() - t0
    B = torch.from_numpy(synth.gaussian_spinors(dims, list(range(1, 49)))).cuda()
    pd = dlz.params_default(m=120, k=60, tol=1e-10, max_iter=200000, precision=dlz.F32, profile=1)
    t0 = time.perf_counter()
    _, sts = dlz.dcg(op, d, B, pd)
    torch.cuda.synchronize()
    t_d = time.perf_counter() - t0
    ok = sum(1 for s in sts if s.converged == 1 and s.true_residual <= 1e-10)
    st_ms = sum(s.stencil_ms for s in sts)
    st_b = sum(s.stencil_bytes for s in sts)
    p64 = dlz.params_default(m=120, k=60, tol=1e-10, max_iter=200000)
    t0 = time.perf_counter()
    _, s64 = dlz.dcg(op, d, B[:2].contiguous(), p64)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    ok64 = sum(1 for s in s64 if s.converged == 1 and s.true_residual <= 1e-10)
    out = {"mode": "c3", "workload": "24^3x48 Lan-DR(120,60) + D-CG on 48 Gaussian RHS",
           "kappa": kappa, "kappa_source": ksrc, "links_seconds": round(t_links, 1),
           "first_rhs": {"seconds": round(t_dr, 3), "cycles": st.cycles, "iterations": st.iterations,
                         "converged": st.converged},
           "dcg_f32_batched": {"seconds": round(t_d, 3), "rhs_per_s": round(ok / t_d, 4), "solved": ok,
                               "iterations": [s.iterations for s in sts[:3]],
                               "fused_kernel_gbs": round(st_b / max(st_ms, 1e-9) / 1e6, 1)},
           "dcg_plain_fp64_2rhs": {"seconds": round(t64, 3), "rhs_per_s": round(ok64 / t64, 4), "solved": ok64,
                                   "iterations": [s.iterations for s in s64]},
           "dslash_16rhs": ds, "peak_source": src}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["plain", "chosen"], default="chosen")
    ap.add_argument("--plain-steps", type=int, default=1,
                    help="timed steps of the plain FP64 form reported beside the chosen form")
    ap.add_argument("--k1-traffic", type=float, default=K1_TRAFFIC_BYTES,
                    help="ncu DRAM bytes per launch of the dominant kernel (None if not measured)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) leg")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--ref-mvps-per-rhs", type=int, default=REF_MVPS_PER_RHS)
    ap.add_argument("--stencil-only", action="store_true")
    ap.add_argument("--lattice", default=None)
    ap.add_argument("--nrhs", type=int, default=11)
    ap.add_argument("--stencil-iters", type=int, default=50)
    ap.add_argument("--first-rhs-only", action="store_true")
    ap.add_argument("--ncu-case", nargs="?", const="minres", default=None, choices=["minres", "cg", "ptc"])
    ap.add_argument("--learned-seed", action="store_true")
    ap.add_argument("--multi-lattice", action="store_true")
    ap.add_argument("--c3", action="store_true")
    ap.add_argument("--ml-lattices", type=int, default=64)
    ap.add_argument("--ls-train", type=int, default=32)
    ap.add_argument("--ls-test", type=int, default=8)
    ap.add_argument("--ls-steps", type=int, default=400)
    ap.add_argument("--max-cycles", type=int, default=4000)
    ap.add_argument("--kappa", type=float, default=None)
    ap.add_argument("--tol", type=float, default=1e-10)
    args = ap.parse_args()
    if args.stencil_only:
        run_stencil_only(args)
    elif args.first_rhs_only:
        run_first_rhs_only(args)
    elif args.ncu_case is not None:
        run_ncu_case(args)
    elif args.learned_seed:
        run_learned_seed(args)
    elif args.multi_lattice:
        run_multi_lattice(args)
    elif args.c3:
        run_c3(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
