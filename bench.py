"""Benchmark: Phi-applications per second (and the steady-state solve) on the 12-site open
transverse-field Ising chain, n = 4096, d = 12 dense decay jumps (J = 1, h = 1, gamma = 0.3).

One timed step = one application of the auxiliary map Phi~ = -K~ S~^{-1} in Schur
coordinates (the map Alg. 4 iterates), mixed precision: triangular Lyapunov solve + the jump
term as two tcgen05 split-FP16 GEMMs.  Inputs are synthetic (seeded), already resident in HBM;
the operands (L~ planes, 1.6 GB) exceed the 126 MB L2, so no flush is needed between steps.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--quick] [--no-fp64-solve]
    the default line also carries the set-up time, one FP64 application and the steady-state solve to
    ||L rho||_max <= 1e-10 in mixed precision and in FP64 (time, residual, iteration counts)
python bench.py --workload sweep      # the batched sweep: 1024 Kerr-cat steady states of uneven n
python bench.py --workload resolvent  # (lam - L) X = I/n, three shifts (Sec. 3.4)
python bench.py --workload euler      # implicit Euler on the stiff n = 32 family (Sec. 4.3)
python bench.py --workload gmres      # Alg. 3 steady state at n = 4096
python bench.py --workload cat        # memory-buffer cat: steady state + 3 slowest modes across n
python bench.py --workload spectrum   # k = 6 slowest modes of the 12-site TFIM by shift-invert Arnoldi (Alg. 5)
Multi-GPU: replicas only (each rank runs its own copy of the workload; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Phi-applies/s & steady-state solve time at n=4096, mixed vs FP64, resid<=1e-10"
WORKLOAD = dict(workload="tfim12_n4096_d12", N_sites=12, n=4096, d=12, J=1.0, h=1.0, gamma=0.3)


def max_over_ranks(values, world, device=None):
    """Element-wise maximum of per-rank timings over the process group (all_reduce MAX); the
    identity for a single process.  Replicas exchange nothing else."""
    if world == 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t]


def whole_job_rate(units_per_step, steps, world, ms):
    """Units processed by all ranks divided by the slowest rank's time (weak scaling)."""
    return units_per_step * steps * world / (ms / 1000.0)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return pk, "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # raw samples go to LB_CLOCKS_DIR (default: the system temp directory); the JSON line
        # carries their summary
        self.path = os.path.join(os.environ.get("LB_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"lindblad_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.f.close()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(n_sites=12, d_sample=1, repeats=1):
    """The oracle (oracle/krylov.py, NumPy/SciPy FP64) on a bounded sample of one Phi application:
    the jump term for d_sample of the 12 jump operators at n = 4096 and the Bartels-Stewart solve
    S^{-1} at n = 1024 (the 10-site chain), each timed `repeats` times; one application is estimated as
    (12 / d_sample) x the jump sample + (4096 / 1024)^3 x the Sylvester sample."""
    import numpy as np

    import lindblad_inputs as gi
    from oracle import krylov as K

    H, Ls = gi.tfim(n_sites, J=1.0, h=1.0, gamma=0.3)
    X = gi.random_hermitian(H.shape[0], seed=1)
    sysK = K.System(H, Ls[:d_sample])
    H10, L10 = gi.tfim(10, J=1.0, h=1.0, gamma=0.3)
    s10 = K.System(H10, L10)
    _ = s10.schur                                    # factorisation is set-up, not per apply
    X10 = gi.random_hermitian(H10.shape[0], seed=1)
    tk, ts = [], []
    for _ in range(repeats):
        t0 = time.perf_counter()
        sysK.K(X)
        tk.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        s10.S_inv(X10)
        ts.append(time.perf_counter() - t0)
    k_scale, s_scale = len(Ls) / d_sample, (H.shape[0] / H10.shape[0]) ** 3
    t_k, t_s = statistics.median(tk), statistics.median(ts)
    per_apply = t_k * k_scale + t_s * s_scale
    threads = len(os.sched_getaffinity(0))   # NumPy's BLAS uses every core it is given
    return {"value": 1.0 / per_apply, "unit": "Phi-applies/s", "cores": int(threads), "kind": "oracle",
            "sample": (f"oracle System.K with {d_sample}/12 jumps at n=4096 (x{k_scale:g}) plus Bartels-Stewart "
                       f"S^-1 (scipy Schur + ztrsyl) at n=1024 (x{s_scale:g}); est. {per_apply:.1f} s per apply"),
            "samples_run": repeats, "jump_sample_s": [round(v, 3) for v in tk],
            "sylvester_sample_s": [round(v, 3) for v in ts], "extrapolated": True,
            "extrapolation": {"jump_factor": k_scale, "sylvester_factor": s_scale}}


# DRAM bytes (read + write) per jump-term k_tc_gemm launch at n = 4096, d = 12: the two jump-term launches
# of one application captured on the 10-site chain (n = 1024, d = 10; dram__bytes_read.sum +
# dram__bytes_write.sum, profiles/tc_gemm_jump_tfim10_n1024.md): product (1) 99.6 + 53.4 MB, product (2)
# 177.3 + 0.06 MB, mean 165.2 MB per launch; the operand planes scale as d n^2, so x (12/10) x 16 = 19.2
# gives 3.17 GB per launch (the algorithmic bytes are 3.29 GB: L2 absorbs part of product (1)'s writes)
JUMP_GEMM_TRAFFIC_BYTES = 3.17e9
JUMP_GEMM_TRAFFIC_NOTE = ("ncu DRAM bytes of the current k_tc_gemm revision at n = 1024, d = 10, scaled by d n^2 to "
                          "n = 4096, d = 12 (the full-size capture needs more than one pass)")

SWEEP = dict(workload="kerr_cat_sweep_1024", count=1024, seed=0, n_range=[16, 160], d=2,
             eps2=[1.0, 8.0], K=[0.5, 2.0], kappa1=[1e-3, 1e-1], kappa2=1.0)


def fp32_alu_peak_tflops():
    """FP32 CUDA-core peak from the part's unit counts: 148 SMs x 128 FMA/clk x 2 flops x 2.032 GHz."""
    return 148 * 128 * 2 * 2.032e9 / 1e12


def sweep_cpu_baseline(params, sample=6):
    """The oracle's Alg. 4 (oracle/krylov.py, FP64) on `sample` instances of the sweep spread over n,
    scaled to the whole sweep by sum n^3."""
    import numpy as np

    import lindblad_inputs as gi
    from oracle import krylov as K

    order = np.argsort([p["n"] for p in params])
    picks = [int(order[int(i)]) for i in np.linspace(0, len(order) - 1, sample)]
    t_sum, w_sum = 0.0, 0.0
    for k in picks:
        p = params[k]
        H, Ls = gi.kerr_cat(p["n"], K=p["K"], eps2=p["eps2"], kappa2=p["kappa2"], kappa1=p["kappa1"])
        t0 = time.perf_counter()
        K.steady_state_phi_arnoldi(K.System(H, Ls), tol=1e-10, m=30, N=60)
        t_sum += time.perf_counter() - t0
        w_sum += p["n"] ** 3
    total = t_sum * sum(p["n"] ** 3 for p in params) / w_sum
    return {"value": len(params) / total, "unit": "steady-states/s", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle", "sample": (f"oracle Alg. 4 (m=30) on {sample} sweep instances "
                                         f"(n={sorted(params[k]['n'] for k in picks)}), {t_sum:.1f} s, scaled "
                                         f"by sum n^3 to the 1024-instance sweep ({total:.0f} s)")}


def run_sweep(args, world, device):
    import numpy as np
    import torch

    import lindblad_inputs as gi
    import paper_2608_30860_b300 as B

    torch.cuda.set_device(device)
    params = gi.kerr_cat_sweep(args.sweep_count, seed=SWEEP["seed"], nmin=args.sweep_n[0], nmax=args.sweep_n[1])
    systems = [gi.kerr_cat(p["n"], K=p["K"], eps2=p["eps2"], kappa2=p["kappa2"], kappa1=p["kappa1"])
               for p in params]
    ns = [p["n"] for p in params]
    d = 2
    Hh = torch.from_numpy(np.concatenate([H.reshape(-1) for H, _ in systems])).pin_memory()
    Lh = torch.from_numpy(np.concatenate([np.stack(L).reshape(-1) for _, L in systems])).pin_memory()
    Hd, Ld = Hh.to(device), Lh.to(device)
    rho = torch.empty_like(Hd)
    ws = torch.empty(B.lindblad_batched_workspace_bytes(ns, d), dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream()
    # tile shapes of the per-instance GEMMs from the library's autotuner (off the clock; a JSON cache is
    # reused when it matches the device, d and the largest size)
    tune = B.batched_tune(d, nmax=max(ns), cache=args.tile_cache) if args.tile_cache != "none" else None
    tiles = tune["tiles"] if tune else None
    for _ in range(args.warmup):
        B.steady_state_batched(ns, d, Hd, Ld, rho=rho, workspace=ws, tiles=tiles)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_launch0 = B.lb_launch_count()
    applies = 0
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.profiler.start()
        e0.record(stream)
        for _ in range(args.steps):
            _, infos, st = B.steady_state_batched(ns, d, Hd, Ld, rho=rho, workspace=ws, tiles=tiles)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    gpu_launches = B.lb_launch_count() - n_launch0
    worst = max(i["residual_max"] for i in infos)
    applies = [i["phi_applies"] for i in infos]
    anchors = [i["refine_steps"] for i in infos]
    flops32 = sum(a * (2 * d + 1) * n ** 3 * 8.0 for a, n in zip(applies, ns))
    # end to end: pinned host H, L in, rho out, inside the timed region
    rho_h = torch.empty_like(Hh).pin_memory()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        Hd.copy_(Hh, non_blocking=True)
        Ld.copy_(Lh, non_blocking=True)
        B.steady_state_batched(ns, d, Hd, Ld, rho=rho, workspace=ws, tiles=tiles)
        rho_h.copy_(rho, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1)
    return dict(ms=ms, e2e_ms=e2e_ms, clocks=clk.summary(), gpu_launches=gpu_launches, status=st,
                worst=worst, applies=applies, anchors=anchors, flops32=flops32, params=params,
                h2d=int(Hh.numel() + Lh.numel()) * 16, d2h=int(rho_h.numel()) * 16, ws_bytes=ws.numel(), tune=tune)


def sweep_line(args, r, world):
    count = args.sweep_count
    value = whole_job_rate(count, args.steps, world, r["ms"])
    per_sweep_s = r["ms"] / 1000.0 / args.steps
    achieved = r["flops32"] / per_sweep_s / 1e12
    peak = fp32_alu_peak_tflops()
    line = {
        "metric": "steady states/s of the batched Kerr-cat sweep (1024 instances, n in 16..160), resid<=1e-10",
        "value": value, "unit": "steady-states/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["ms"] / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64+f64", "data": "synthetic",
        "config": dict(SWEEP, count=count, n_range=list(args.sweep_n), parallelism="replicas" if world > 1 else "none",
                       l2=f"one step = the whole sweep ({r['ws_bytes'] / 1e9:.1f} GB of per-instance state) > L2; "
                          "no flush"),
        "roofline": {"bound": "alu", "kernel": "k_batched_solve (persistent, one CTA per instance)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None,
                     "peak_source": "FP32 CUDA-core peak from 148 SMs x 128 FMA/clk x 2 x 2.032 GHz",
                     "flops_per_step": r["flops32"],
                     "note": "algorithmic complex64 flops of the Phi applications (jump term + triangular solve); "
                             "the FP64 anchors and the set-up are not counted"},
        "e2e": {"value": whole_job_rate(count, args.steps, world, r["e2e_ms"]), "unit": "steady-states/s",
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": r["gpu_launches"],
        "clocks": r["clocks"],
        "status": r["status"], "worst_residual_max": r["worst"],
        "phi_applies_mean": sum(r["applies"]) / count, "fp64_anchors_mean": sum(r["anchors"]) / count,
    }
    if r.get("tune"):
        t = r["tune"]
        line["config"]["tiles"] = {b: t["shapes"][k] for b, k in zip(t["buckets"], t["tiles"])
                                   if int(b.split("<=")[1]) - 16 < max(args.sweep_n[1], 16)}
        line["config"]["tile_tuning"] = {"cached": t["cached"], "tune_s": round(t.get("tune_s", 0.0), 3),
                                         "cache": args.tile_cache}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = sweep_cpu_baseline(r["params"])
    return line


def measure_peaks(device):
    """Library-GEMM throughput of the units the batched and FP64 paths use (cuBLAS through torch,
    best of 5 after warm-up, CUDA events): FP64, FP32 (TF32 off), TF32, complex64, complex128."""
    import torch

    torch.cuda.set_device(device)
    out = {}
    cases = [("fp64", torch.float64, 4096, False, 2), ("fp32", torch.float32, 8192, False, 2),
             ("tf32", torch.float32, 8192, True, 2), ("c64", torch.complex64, 4096, False, 8),
             ("c128", torch.complex128, 2048, False, 8)]
    for name, dt, n, tf32, fl in cases:
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, dtype=dt, device=device)
        b = torch.randn(n, n, dtype=dt, device=device)
        for _ in range(2):
            a @ b
        torch.cuda.synchronize()
        best = None
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out[name + "_tflops"] = fl * n ** 3 / (best / 1000.0) / 1e12
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = False
    out["fp32_alu_peak_tflops_derived"] = fp32_alu_peak_tflops()
    return out


def _solve_record(info, st, seconds):
    return {"s": round(seconds, 3), "status": int(st), "residual_max": info["residual_max"],
            "restarts": info["restarts"], "phi_applies": info["phi_applies"], "gmres_steps": info["gmres_steps"],
            "refine_steps": info["refine_steps"]}


def run_ours(args, rank, world, device):
    import numpy as np
    import torch

    import lindblad_inputs as gi
    import paper_2608_30860_b300 as B

    torch.cuda.set_device(device)
    H, Ls = gi.tfim(args.sites, J=1.0, h=1.0, gamma=0.3)
    n, d = H.shape[0], len(Ls)
    Hd = torch.from_numpy(H).to(device)
    Ld = torch.from_numpy(np.stack(Ls)).to(device)
    del Ls
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    opts = B.default_opts(precision=B.LB_PREC_MIXED)
    h = B.lindblad_setup(Hd, Ld, opts)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    del Ld

    X = torch.from_numpy(gi.random_hermitian(n, seed=1)).to(device)
    X = X / torch.linalg.matrix_norm(X)
    Y = torch.empty_like(X)
    stream = torch.cuda.current_stream()

    def step(x, y, prec=B.LB_PREC_MIXED):
        # the map Alg. 4 iterates: Phi~ in Schur coordinates on a Hermitian Krylov vector
        B.phi_apply(h, x, y, schur=True, precision=prec, hermitian=True)

    for _ in range(args.warmup):
        step(X, Y)
    torch.cuda.synchronize()
    B.lb_set_profiling(h, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    n_launch0 = B.lb_launch_count()
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.profiler.start()   # profilers run with --profile-from-start off see the timed steps only
        e0.record(stream)
        for _ in range(args.steps):
            step(X, Y)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    gpu_launches = B.lb_launch_count() - n_launch0
    launches, kms, kflops = B.lb_kernel_stats(h, 0)
    B.lb_set_profiling(h, False)

    # end to end through the C ABI with host buffers: pinned H2D of the step's input, the
    # application, D2H of the result
    Xh = X.cpu().pin_memory()
    Yh = torch.empty_like(Xh).pin_memory()
    Xd = torch.empty_like(X)
    for _ in range(2):
        Xd.copy_(Xh, non_blocking=True)
        step(Xd, Y)
        Yh.copy_(Y, non_blocking=True)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        Xd.copy_(Xh, non_blocking=True)
        step(Xd, Y)
        Yh.copy_(Y, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1)

    extra = {"setup_s": round(setup_s, 2), "schur_backward_err": h.setup_info["schur_backward_err"]}
    if not args.quick:
        # the headline's other half: one FP64 application, and the steady-state solve to ||L rho||_max <= 1e-10
        # in both precisions (wall clock around the C-ABI call, which synchronises)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        step(X, Y, B.LB_PREC_FP64)
        g1.record(stream)
        torch.cuda.synchronize()
        extra["fp64_phi_apply_s"] = round(g0.elapsed_time(g1) / 1000.0, 3)
        o = B.default_opts(precision=B.LB_PREC_MIXED, tol=1e-10)
        t0 = time.perf_counter()
        rho, info, st = B.steady_state(h, o)
        extra["solve_mixed"] = _solve_record(info, st, time.perf_counter() - t0)
        extra["solve_mixed_s"] = extra["solve_mixed"]["s"]
        extra["solve_mixed_residual"] = info["residual_max"]
        if not args.no_fp64_solve:
            o = B.default_opts(precision=B.LB_PREC_FP64, tol=1e-10, max_restarts=args.fp64_restarts)
            t0 = time.perf_counter()
            rho64, info64, st64 = B.steady_state(h, o)
            extra["solve_fp64"] = _solve_record(info64, st64, time.perf_counter() - t0)
            extra["solve_fp64_s"] = extra["solve_fp64"]["s"]
            extra["solve_fp64_residual"] = info64["residual_max"]
            extra["mixed_vs_fp64_solve_speedup"] = round(extra["solve_fp64_s"] / max(extra["solve_mixed_s"], 1e-9), 2)
            extra["mixed_vs_fp64_state_rel_diff"] = float(torch.linalg.matrix_norm(rho - rho64) /
                                                          torch.linalg.matrix_norm(rho64))
        extra["end_to_end_mixed_s"] = round(setup_s + extra["solve_mixed_s"], 2)
    B.lindblad_destroy(h)
    return dict(ms=ms, e2e_ms=e2e_ms, launches=launches, kms=kms, kflops=kflops, clocks=clk.summary(),
                n=n, d=d, extra=extra, gpu_launches=gpu_launches)


def _setup_case(B, torch, device, H, Ls, **kw):
    import numpy as np
    Hd = torch.from_numpy(H).to(device)
    Ld = torch.from_numpy(np.stack(Ls)).to(device)
    o = B.default_opts(**kw)
    t0 = time.perf_counter()
    h = B.lindblad_setup(Hd, Ld, o)
    torch.cuda.synchronize()
    return h, time.perf_counter() - t0


def _kernel_roofline(B, h, pk, kid):
    """Algorithmic rate of the library's tensor-core (kid 0) or FP64 (kid 1) GEMM launches recorded while
    profiling was on, against the matching measured peak."""
    launches, kms, kfl = B.lb_kernel_stats(h, kid)
    if not launches:
        return None
    ach = kfl / (kms / 1000.0) / 1e12
    if kid == 0:
        peak, unit_src = pk["bf16_tflops"], "bf16_tflops burst (kind::f16 FP16 = BF16 rate)"
    else:
        peak, unit_src = 1.04, "cuBLAS DGEMM measured on this pool (bench.py --peaks)"
    return {"bound": "tensor" if kid == 0 else "fp64-alu", "kernel": "k_tc_gemm" if kid == 0 else "zgemm_f64_kernel",
            "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
            "peak_source": unit_src, "launches": launches, "ms_total": kms}


def run_workload(args, device):
    """Lines for the solvers built on the recycled preconditioned GMRES and for the cat qubit:
    resolvent (Sec. 3.4), implicit Euler (Sec. 4.3), Alg. 3 (Sec. 4.1) and the cat-qubit spectrum (Sec. 4.2)."""
    import numpy as np
    import torch

    import lindblad_inputs as gi
    import paper_2608_30860_b300 as B

    torch.cuda.set_device(device)
    pk, src = _peaks()
    stream = torch.cuda.current_stream()
    prec = B.LB_PREC_MIXED if args.precision == "mixed" else B.LB_PREC_FP64
    line = {"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic", "dtype": "f16x2-split/f32acc+f64" if prec else "f64"}
    n0 = B.lb_launch_count()
    with ClockSampler(torch.cuda.current_device()) as clk:
        if args.workload == "resolvent":
            # the paper's dense random family, (lam - L) X = I/n at lam = lam_max 10^{0,-1,-2}; lam_max from a
            # power iteration on L, off the clock
            n = args.n
            H, Ls = gi.paper_random_lindbladian(n, seed=0)
            h, setup_s = _setup_case(B, torch, device, H, Ls, precision=prec)
            v = torch.from_numpy(gi.random_operator(n, seed=3)).to(device)
            lmax = 0.0
            for _ in range(30):
                w = B.lindbladian_apply(h, v)
                lmax = float(torch.linalg.matrix_norm(w) / torch.linalg.matrix_norm(v))
                v = w / torch.linalg.matrix_norm(w)
            Bm = torch.eye(n, dtype=torch.complex128, device=device) / n
            per = {}
            for k in range(max(1, args.warmup // 3)):
                B.resolvent_solve(h, lmax, Bm, B.default_opts(precision=prec, tol=1e-8))
            B.lb_set_profiling(h, True)
            total = 0.0
            for lam_f in (1.0, 0.1, 0.01):
                lam = lmax * lam_f
                times = []
                for _ in range(args.steps):
                    t0 = time.perf_counter()
                    X, info, st = B.resolvent_solve(h, lam, Bm, B.default_opts(precision=prec, tol=1e-8, gmres_m=32,
                                                                              recycle_k=8))
                    times.append(time.perf_counter() - t0)
                per[f"lam_max*{lam_f:g}"] = {"s_median": statistics.median(times), "status": st,
                                             "residual_max": info["residual_max"], "gmres_steps": info["gmres_steps"]}
                total += statistics.median(times)
            line.update(metric="resolvent solves/s, (lam-L)X=I/n at lam=lam_max*10^{0,-1,-2}, resid<=1e-8",
                        value=3.0 / total, unit="solves/s", ms_per_step=1000.0 * total / 3.0,
                        config={"workload": f"paper_random_n{n}_d3_resolvent", "n": n, "d": 3, "gamma": 0.1,
                                "lam_max": lmax, "tol": 1e-8, "gmres_m": 32, "recycle_k": 8,
                                "l2": "operands exceed L2" if n >= 2048 else "operands fit L2"},
                        per_shift=per, setup_s=round(setup_s, 3))
        elif args.workload == "euler":
            # Sec. 4.3's stiff family: n = 32 dense random + K N^2, K in {0, 15}; fixed dt, steps/s
            n, dt, nsteps = 32, 0.01, 200
            per = {}
            tot_steps, tot_s = 0, 0.0
            for Kq in (0.0, 15.0):
                H, Ls = gi.stiff_random_lindbladian(n, K=Kq, seed=0)
                h, _ = _setup_case(B, torch, device, H, Ls)
                rho0 = torch.zeros((n, n), dtype=torch.complex128, device=device)
                rho0[0, 0] = 1.0
                B.implicit_euler(h, rho0, dt, 5, B.default_opts(tol=1e-8))
                t0 = time.perf_counter()
                rho, _, info, st = B.implicit_euler(h, rho0, dt, nsteps, B.default_opts(tol=1e-8, gmres_m=32, recycle_k=8))
                el = time.perf_counter() - t0
                per[f"K={Kq:g}"] = {"s": el, "steps_per_s": nsteps / el, "status": st,
                                    "gmres_steps_per_step": info["gmres_steps"] / nsteps,
                                    "worst_rel_step_residual": info["residual_max"]}
                tot_steps += nsteps
                tot_s += el
                B.lindblad_destroy(h)
            line.update(metric="implicit Euler steps/s (n=32 stiff random + K N^2, dt=0.01, step resid<=1e-8)",
                        value=tot_steps / tot_s, unit="steps/s", ms_per_step=1000.0 * tot_s / tot_steps,
                        config={"workload": "stiff_random_n32_euler", "n": n, "dt": dt, "steps": nsteps,
                                "K": [0.0, 15.0], "l2": "operands fit L2"}, per_K=per, dtype="f64")
            h = None
        elif args.workload == "gmres":
            # Alg. 3 (recycled preconditioned GMRES) at the benchmark's n = 4096 (or --sites)
            H, Ls = gi.tfim(args.sites, J=1.0, h=1.0, gamma=0.3)
            n = H.shape[0]
            h, setup_s = _setup_case(B, torch, device, H, Ls, precision=B.LB_PREC_MIXED)
            B.lb_set_profiling(h, True)
            t0 = time.perf_counter()
            rho, info, st = B.steady_state_gmres(h, B.default_opts(precision=prec, tol=1e-10, gmres_m=32, recycle_k=8))
            el = time.perf_counter() - t0
            line.update(metric="steady-state solve time, Alg. 3 (recycled preconditioned GMRES), resid<=1e-10",
                        value=el, unit="s", higher_is_better=False, ms_per_step=1000.0 * el,
                        config={"workload": f"tfim{args.sites}_n{n}_d{len(Ls)}_alg3", "n": n, "d": len(Ls),
                                "gmres_m": 32, "recycle_k": 8, "l2": "operands exceed L2"},
                        setup_s=round(setup_s, 2), solve=_solve_record(info, st, el), steps=1)
        elif args.workload == "spectrum":
            # the k = 6 slowest modes of the TFIM chain by shift-invert Arnoldi (Alg. 5, mu = 0, eta = 1) with
            # recycled, right-preconditioned inner solves; eigen-residuals ||L v - lam v||_max / ||v||_max
            H, Ls = gi.tfim(args.sites, J=1.0, h=1.0, gamma=0.3)
            n = H.shape[0]
            h, setup_s = _setup_case(B, torch, device, H, Ls, precision=prec)
            B.lb_set_profiling(h, True)
            t0 = time.perf_counter()
            ev, _, info, st = B.low_spectrum(h, args.k, opts=B.default_opts(precision=prec, tol=args.spectrum_tol,
                                                                          krylov_m=24, gmres_m=32, recycle_k=8))
            el = time.perf_counter() - t0
            line.update(metric=f"low spectrum (k={args.k}) by shift-invert Arnoldi, eigen-residual<={args.spectrum_tol:g}",
                        value=el, unit="s", higher_is_better=False, ms_per_step=1000.0 * el, steps=1,
                        config={"workload": f"tfim{args.sites}_n{n}_d{len(Ls)}_spectrum_k{args.k}", "n": n,
                                "d": len(Ls), "k": args.k, "mu": 0.0, "eta": 1.0, "krylov_m": 24, "gmres_m": 32,
                                "recycle_k": 8, "l2": "operands exceed L2" if n >= 2048 else "operands fit L2"},
                        setup_s=round(setup_s, 2), status=st, residual_max=info["residual_max"],
                        restarts=info["restarts"], op_applications=info["phi_applies"],
                        inner_gmres_steps=info["gmres_steps"], fp64_cycles=info["refine_steps"],
                        eigenvalues=[[float(x.real), float(x.imag)] for x in ev.numpy()])
        elif args.workload == "cat":
            # App. B memory-buffer cat: steady state (Alg. 4) and the 3 slowest modes (Alg. 5) across n
            per = {}
            tot = 0.0
            for ntarget in args.cat_n:
                na, nb = gi.memory_buffer_dims(ntarget)
                H, Ls = gi.memory_buffer_cat(na, nb)
                h, setup_s = _setup_case(B, torch, device, H, Ls, precision=prec)
                t0 = time.perf_counter()
                rho, info, st = B.steady_state(h, B.default_opts(precision=prec, tol=1e-10, max_restarts=200))
                t_ss = time.perf_counter() - t0
                t0 = time.perf_counter()
                ev, _, sinfo, sst = B.low_spectrum(h, 3, opts=B.default_opts(precision=prec, tol=1e-8, krylov_m=24))
                t_sp = time.perf_counter() - t0
                tot += t_ss + t_sp
                per[f"n={na * nb}"] = {"na": na, "nb": nb, "alpha2": na / 5.0, "setup_s": setup_s,
                                       "steady_state_s": t_ss, "steady_state_status": st,
                                       "residual_max": info["residual_max"], "spectrum_s": t_sp,
                                       "spectrum_status": sst, "decay_rates": [float(-x.real) for x in ev.numpy()],
                                       "eigenvalues": [[float(x.real), float(x.imag)] for x in ev.numpy()]}
                B.lindblad_destroy(h)
            line.update(metric="memory-buffer cat: steady state + 3 slowest modes, time per system",
                        value=len(args.cat_n) / tot, unit="systems/s", ms_per_step=1000.0 * tot / len(args.cat_n),
                        config={"workload": "memory_buffer_cat", "n_targets": args.cat_n,
                                "params": gi.MEMORY_BUFFER, "l2": "operands fit L2"}, per_n=per, steps=1)
            h = None
        else:
            raise ValueError(args.workload)
        torch.cuda.synchronize()
    line["clocks"] = clk.summary()
    line["gpu_launches"] = B.lb_launch_count() - n0
    if h is not None:
        line["roofline"] = _kernel_roofline(B, h, pk, 0 if prec else 1)
        B.lindblad_destroy(h)
    line["e2e"] = None
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true",
                    help="time the Phi applications only (skip the FP64 application and both steady-state solves)")
    ap.add_argument("--no-fp64-solve", action="store_true", help="skip the all-FP64 steady-state solve")
    ap.add_argument("--fp64-restarts", type=int, default=12, help="restart cap of the all-FP64 solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--peaks", action="store_true",
                    help="only measure library GEMM peaks (FP64, FP32, TF32, complex64/128) and print them")
    ap.add_argument("--workload", default="tfim12",
                    choices=["tfim12", "sweep", "resolvent", "euler", "gmres", "cat", "spectrum"],
                    help="tfim12: Phi applications + steady-state solves at n=4096 (default); sweep: the batched "
                         "Kerr-cat sweep; resolvent / euler / gmres / cat / spectrum: the GMRES-based solvers, the cat "
                         "qubit and the TFIM low spectrum")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"], help="precision of the extra workloads")
    ap.add_argument("--n", type=int, default=1024, help="size of the resolvent workload")
    ap.add_argument("--cat-n", type=int, nargs="+", default=[256, 512, 1024], help="target sizes of the cat workload")
    ap.add_argument("--k", type=int, default=6, help="eigenvalues of the spectrum workload")
    ap.add_argument("--spectrum-tol", type=float, default=1e-8, help="eigen-residual tolerance of the spectrum workload")
    ap.add_argument("--sweep-count", type=int, default=SWEEP["count"],
                    help="instances of the sweep (1024: the benchmark; small values give profiler cases)")
    ap.add_argument("--sweep-n", type=int, nargs=2, default=SWEEP["n_range"], metavar=("NMIN", "NMAX"))
    ap.add_argument("--tile-cache", default=os.path.join(os.path.expanduser("~"), ".cache", "lindblad_b300",
                                                        "batched_tiles.json"),
                    help="JSON cache of the batched engine's tile autotuner ('none': shape 0, no tuning)")
    ap.add_argument("--sites", type=int, default=12,
                    help="chain length (12: the n=4096 workload; smaller values give the small cases "
                         "used for profiler captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        # the oracle timed on the host cores, rank 0 only: every step times one bounded sample (one of the
        # 12 jump products at n = 4096 and one Bartels-Stewart solve at n = 1024) and extrapolates it to a
        # full application; the warm-up samples are not reported
        if rank != 0:
            return
        cpu_baseline(repeats=1)
        cb = cpu_baseline(repeats=max(1, min(args.steps, 10)))
        line = {"metric": METRIC, "value": cb["value"], "unit": "Phi-applies/s", "n_gpus": args.gpus,
                "steps": cb["samples_run"], "warmup": 1, "ms_per_step": 1000.0 / cb["value"],
                "ms_per_step_is_extrapolated": True,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "impl": "reference", "config": dict(WORKLOAD, parallelism="none"),
                "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": "Phi-applies/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    device = torch.device("cuda", local)
    if args.peaks:
        if rank == 0:
            with ClockSampler(torch.cuda.current_device()) as clk:
                pk = measure_peaks(device)
            print(json.dumps({"peaks": pk, "clocks": clk.summary()}))
        return
    if args.workload == "sweep":
        r = run_sweep(args, world, device)
        r["ms"], r["e2e_ms"] = max_over_ranks([r["ms"], r["e2e_ms"]], world, device)
        if rank == 0:
            print(json.dumps(sweep_line(args, r, world)))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if args.workload != "tfim12":
        if rank == 0:
            print(json.dumps(run_workload(args, device)))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    r = run_ours(args, rank, world, device)
    ms, e2e_ms = max_over_ranks([r["ms"], r["e2e_ms"]], world, device)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    pk, src = _peaks()
    value = whole_job_rate(1, args.steps, world, ms)
    e2e_value = whole_job_rate(1, args.steps, world, e2e_ms)
    n = r["n"]
    achieved = (r["kflops"] / (r["kms"] / 1000.0)) / 1e12 if r["launches"] else None
    peak = pk["bf16_tflops"]
    line = {
        "metric": METRIC, "value": value, "unit": "Phi-applies/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16x2-split/f32acc+f64", "data": "synthetic",
        "config": dict(WORKLOAD if args.sites == 12 else dict(workload=f"tfim{args.sites}_n{n}_d{r['d']}",
                                                              N_sites=args.sites, n=n, d=r["d"], J=1.0, h=1.0,
                                                              gamma=0.3),
                       parallelism="replicas" if world > 1 else "none",
                       step="Phi~ in Schur coordinates on a Hermitian Krylov vector (LB_APPLY_HERMITIAN)",
                       l2="operands (1.6 GB L~ planes) exceed L2; no flush"),
        "roofline": {"bound": "tensor", "kernel": "k_tc_gemm (tcgen05 split-FP16 complex GEMM, jump term)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": JUMP_GEMM_TRAFFIC_BYTES if args.sites == 12 else None,
                     "traffic_note": JUMP_GEMM_TRAFFIC_NOTE,
                     "peak_source": f"bf16_tflops burst of {src} MEASURED_PEAKS.json (kind::f16 FP16 = BF16 rate)",
                     "launches": r["launches"], "ms_per_launch": r["kms"] / max(r["launches"], 1),
                     "flops_per_launch": r["kflops"] / max(r["launches"], 1),
                     "flops_note": "algorithmic: 8 d n^3 for product (1), 4 d n^2 (n + 1) for the Hermitian "
                                   "product (2)"},
        "e2e": {"value": e2e_value, "unit": "Phi-applies/s", "h2d_bytes_per_step": 16 * n * n,
                "d2h_bytes_per_step": 16 * n * n},
        "gpu_launches": r["gpu_launches"],
        "clocks": r["clocks"],
    }
    line.update(r["extra"])
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
