"""Benchmark: Phi-applications per second (and the steady-state solve) on the 12-site open
transverse-field Ising chain, n = 4096, d = 12 dense decay jumps (J = 1, h = 1, gamma = 0.3).

One timed step = one application of the auxiliary map Phi~ = -K~ S~^{-1} in Schur
coordinates (the map Alg. 4 iterates), mixed precision: triangular Lyapunov solve + the jump
term as two tcgen05 split-FP16 GEMMs.  Inputs are synthetic (seeded), already resident in HBM;
the operands (L~ planes, 1.6 GB) exceed the 126 MB L2, so no flush is needed between steps.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--solve]
python bench.py --workload sweep   # the batched sweep: 1024 Kerr-cat steady states of uneven n
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


def cpu_baseline(n_sites=12, d_sample=1):
    """The oracle (oracle/krylov.py, NumPy/SciPy FP64) on a bounded sample of one Phi application:
    the jump term for d_sample of the 12 jump operators at n = 4096 (scaled by 12/d_sample) plus
    the Bartels-Stewart solve S^{-1} measured at n = 1024 (the 10-site chain, scaled by 4^3)."""
    import numpy as np

    import lindblad_inputs as gi
    from oracle import krylov as K

    H, Ls = gi.tfim(n_sites, J=1.0, h=1.0, gamma=0.3)
    X = gi.random_hermitian(H.shape[0], seed=1)
    sysK = K.System(H, Ls[:d_sample])
    t0 = time.perf_counter()
    sysK.K(X)
    t_k = (time.perf_counter() - t0) * (len(Ls) / d_sample)
    H10, L10 = gi.tfim(10, J=1.0, h=1.0, gamma=0.3)
    s10 = K.System(H10, L10)
    _ = s10.schur                                    # factorisation is set-up, not per apply
    X10 = gi.random_hermitian(H10.shape[0], seed=1)
    t0 = time.perf_counter()
    s10.S_inv(X10)
    t_s = (time.perf_counter() - t0) * (H.shape[0] / H10.shape[0]) ** 3
    threads = len(os.sched_getaffinity(0))   # NumPy's BLAS uses every core it is given
    per_apply = t_k + t_s
    return {"value": 1.0 / per_apply, "unit": "Phi-applies/s", "cores": int(threads), "kind": "oracle",
            "sample": (f"oracle System.K with {d_sample}/12 jumps at n=4096 scaled x{12 // d_sample}, plus "
                       "Bartels-Stewart S^-1 (scipy Schur + ztrsyl) at n=1024 scaled x64; "
                       f"est. {per_apply:.1f} s per apply")}


# DRAM bytes (read + write) per jump-term k_tc_gemm launch at n = 4096, d = 12, from one ncu capture
# of the current kernel (mean of the two launches of an application)
JUMP_GEMM_TRAFFIC_BYTES = (10165062144 + 3187236352 + 11702182656 + 238166528) / 2

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
    for _ in range(args.warmup):
        B.steady_state_batched(ns, d, Hd, Ld, rho=rho, workspace=ws)
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
            _, infos, st = B.steady_state_batched(ns, d, Hd, Ld, rho=rho, workspace=ws)
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
        B.steady_state_batched(ns, d, Hd, Ld, rho=rho, workspace=ws)
        rho_h.copy_(rho, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1)
    return dict(ms=ms, e2e_ms=e2e_ms, clocks=clk.summary(), gpu_launches=gpu_launches, status=st,
                worst=worst, applies=applies, anchors=anchors, flops32=flops32, params=params,
                h2d=int(Hh.numel() + Lh.numel()) * 16, d2h=int(rho_h.numel()) * 16, ws_bytes=ws.numel())


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
    for _ in range(args.warmup):
        B.phi_apply(h, X, Y, schur=True, precision=B.LB_PREC_MIXED)
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
            B.phi_apply(h, X, Y, schur=True, precision=B.LB_PREC_MIXED)
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
        B.phi_apply(h, Xd, Y, schur=True, precision=B.LB_PREC_MIXED)
        Yh.copy_(Y, non_blocking=True)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        Xd.copy_(Xh, non_blocking=True)
        B.phi_apply(h, Xd, Y, schur=True, precision=B.LB_PREC_MIXED)
        Yh.copy_(Y, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1)

    extra = {"setup_s": round(setup_s, 2), "schur_backward_err": h.setup_info["schur_backward_err"]}
    if args.fp64:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.phi_apply(h, X, Y, schur=True, precision=B.LB_PREC_FP64)
        torch.cuda.synchronize()
        extra["fp64_phi_apply_s"] = round(time.perf_counter() - t0, 3)
    if args.solve:
        o = B.default_opts(precision=B.LB_PREC_MIXED, tol=1e-10)
        t0 = time.perf_counter()
        rho, info, st = B.steady_state(h, o)
        torch.cuda.synchronize()
        extra["solve_mixed_s"] = round(time.perf_counter() - t0, 2)
        extra["solve_mixed_info"] = {k: info[k] for k in ("status", "restarts", "phi_applies", "gmres_steps",
                                                           "refine_steps", "residual_max")}
    B.lindblad_destroy(h)
    return dict(ms=ms, e2e_ms=e2e_ms, launches=launches, kms=kms, kflops=kflops, clocks=clk.summary(),
                n=n, d=d, extra=extra, gpu_launches=gpu_launches)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--solve", action="store_true", help="also time one mixed steady-state solve")
    ap.add_argument("--fp64", action="store_true", help="also time one all-FP64 Phi application")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--peaks", action="store_true",
                    help="only measure library GEMM peaks (FP64, FP32, TF32, complex64/128) and print them")
    ap.add_argument("--workload", default="tfim12", choices=["tfim12", "sweep"],
                    help="tfim12: Phi applications at n=4096 (default); sweep: the batched Kerr-cat sweep")
    ap.add_argument("--sweep-count", type=int, default=SWEEP["count"],
                    help="instances of the sweep (1024: the benchmark; small values give profiler cases)")
    ap.add_argument("--sweep-n", type=int, nargs=2, default=SWEEP["n_range"], metavar=("NMIN", "NMAX"))
    ap.add_argument("--sites", type=int, default=12,
                    help="chain length (12: the n=4096 workload; smaller values give the small cases "
                         "used for profiler captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        # the oracle timed on the host cores; rank 0 only
        if rank != 0:
            return
        cb = cpu_baseline()
        line = {"metric": METRIC, "value": cb["value"], "unit": "Phi-applies/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / cb["value"],
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
    r = run_ours(args, rank, world, device)
    ms, e2e_ms = max_over_ranks([r["ms"], r["e2e_ms"]], world, device)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    pk, src = _peaks()
    value = whole_job_rate(1, args.steps, world, ms)
    e2e_value = whole_job_rate(1, args.steps, world, e2e_ms)
    n = r["n"]
    per_launch_ms = r["kms"] / max(r["launches"], 1)
    achieved = (r["kflops"] / max(r["launches"], 1)) / (per_launch_ms / 1000.0) / 1e12 if r["launches"] else None
    peak = pk["bf16_tflops"]
    line = {
        "metric": METRIC, "value": value, "unit": "Phi-applies/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16x2-split/f32acc+f64", "data": "synthetic",
        "config": dict(WORKLOAD if args.sites == 12 else dict(workload=f"tfim{args.sites}_n{n}_d{r['d']}",
                                                              N_sites=args.sites, n=n, d=r["d"], J=1.0, h=1.0,
                                                              gamma=0.3),
                       parallelism="replicas" if world > 1 else "none",
                       l2="operands (1.6 GB L~ planes) exceed L2; no flush"),
        "roofline": {"bound": "tensor", "kernel": "k_tc_gemm (tcgen05 split-FP16 complex GEMM)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": JUMP_GEMM_TRAFFIC_BYTES if args.sites == 12 else None,
                     "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum per jump-term launch, "
                                       "profiles/tc_gemm_traffic_tfim12_n4096.md",
                     "peak_source": f"bf16_tflops burst of {src} MEASURED_PEAKS.json (kind::f16 FP16 = BF16 rate)",
                     "launches": r["launches"], "ms_per_launch": per_launch_ms,
                     "flops_per_launch": r["kflops"] / max(r["launches"], 1)},
        "e2e": {"value": e2e_value, "unit": "Phi-applies/s", "h2d_bytes_per_step": 16 * n * n,
                "d2h_bytes_per_step": 16 * n * n},
        "gpu_launches": None,
        "clocks": r["clocks"],
    }
    line.update(r["extra"])
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    # kernels the library launched inside the timed region (its own launch counter)
    line["gpu_launches"] = r["gpu_launches"]
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
