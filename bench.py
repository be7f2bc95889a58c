"""Throughput benchmark of the GB300 variational-MFG solver.

Headline workload: 2-D Neumann unit square 512 x 512, N_t = 128 (n =
33,554,432 space-time unknowns, 5n primal unknowns), nu = 1e-2, quadratic
Hamiltonian, f = m + V(x) with V a seeded cosine series, g = 0.1|x - (0.8,
0.8)|^2, m0 a Gaussian at (0.2, 0.2) -- the largest single-instance workload.

One step = one fixed-count solve: 300 accelerated Chambolle-Pock iterations
(each with its preconditioned AAt solve to relative tolerance 1e-10 against
||b||, and the per-cell prox) from the initial iterate, one CUDA-graph launch.
Metric: CP iterations per second (each CP iteration is one preconditioned AAt
solve).  Precision (default): the preconditioner in FP32 with its dense time
transforms on the tensor cores (tcgen05, split TF32), inside FP64 flexible
PCG with an FP64 AAt, FP64 residuals and dot products and the FP64 prox.

The JSON line also carries: the same metric through the host-buffer entry
point (e2e), the plain FP64 GPU path on the same workload, the dominant
kernel's roofline, each hot entry point on this workload, the 2-D periodic
128^2 x 64 four-viscosity batch and the 64-instance uneven batch at 300 CP
iterations, the exact-time-solve variant, one adjoint solve, the iterate's
error against the oracle on a short run, and the CPU oracle baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the reference arm of this
benchmark) on a bounded sample of the same workload.  Under torchrun each rank
solves its own copy (replicas; no data-path collective) and rank 0 prints the
aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

import mfg_inputs as mi

CP_PER_STEP = 300
CG_TOL = 1e-10
METRIC = "CP iterations/s (preconditioned AAt solves/s), 2-D Neumann 512^2 x 128"
WORKLOAD = ("2-D Neumann unit square 512x512, N_t=128 (n=33,554,432), nu=1e-2, "
            "300 CP iterations per step from the initial iterate")
# Precision of the timed solve and of the extras: FP32 preconditioner with the
# time transforms on the tensor cores (tcgen05, split TF32), FP64 elsewhere.
PRECISION = "mixed_tc"
# Algorithmic FP64 flops of one AAt apply per unknown in the factored form
# q = C (C^T p): K p (4 differences, 2 adds, 2 scalings, 1 add = 9),
# xm = nu Kp + (p - p')/dt (4), q = nu K xm + (xm - xm')/dt + 2 Kp (10 + 2 + 2)
# -> 27.  (The kernels issue 15 FP64 instructions per unknown, mostly FMAs.)
AAT_FLOPS_PER_UNKNOWN = 27
# Algorithmic bytes of one AAt apply: read p, write q (2 FP64 words per unknown).
AAT_BYTES_PER_UNKNOWN = 16
# GB300 FP64 rate (1.25 TFLOP/s, the profiling recipe's table; not in the
# measured-peaks file).  An FMA-chain probe on this machine measured 1.196.
FP64_PEAK_TFLOPS = 1.25


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value, world, backend_device=None):
    """Max of a float over ranks (identity for a single process)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as td
    t = torch.tensor([value], dtype=torch.float64, device=backend_device or "cpu")
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value, world, backend_device=None):
    if world <= 1:
        return value
    import torch
    import torch.distributed as td
    t = torch.tensor([value], dtype=torch.float64, device=backend_device or "cpu")
    td.all_reduce(t, op=td.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def profiled_traffic(name):
    """DRAM bytes per launch (read + write) recorded by the ncu summary in
    profiles/<name> ("dram_bytes_per_launch: X"), or None."""
    import re
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", open(path).read())
    return float(m.group(1)) if m else None


def _todev(dev):
    import torch
    return lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).reshape(-1).to(dev)


def _events(stream):
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


class Fixed:
    """A fixed-count solve of one plan from a fixed initial iterate; step() runs it once."""

    def __init__(self, L, dev, insts, probs, stream):
        import torch
        self.L, self.stream = L, stream
        self.plan = L.mfg_plan(probs)
        sz = L.mfg_sizes(self.plan)
        t = _todev(dev)
        cat = lambda key: np.concatenate([np.asarray(i[key], dtype=np.float64).reshape(-1) for i in insts])
        self.host = {k: cat(k) for k in ("m0", "V", "W", "y0")}
        self.m0, self.V, self.W, self.y0 = (t(self.host[k]) for k in ("m0", "V", "W", "y0"))
        self.y, self.ybar = torch.empty_like(self.y0), torch.empty_like(self.y0)
        self.z = torch.zeros(sz["dual"], dtype=torch.float64, device=dev)
        self.sizes = sz

    def step(self):
        self.y.copy_(self.y0)
        self.ybar.copy_(self.y0)
        self.z.zero_()
        rc, st = self.L.mfg_solve(self.plan, self.m0, self.V, self.W, self.y, self.ybar, self.z,
                                  stream=self.stream)
        if rc != 0:
            raise RuntimeError(f"solve failed: {rc} {self.L.mfg_last_error()}")
        return st

    def timed(self, steps=1, warmup=1):
        for _ in range(warmup):
            self.step()
        import torch
        torch.cuda.synchronize()
        a, b = _events(self.stream)
        a.record(self.stream)
        cp = cg = 0
        for _ in range(steps):
            st = self.step()
            cp += sum(s.cp_iters for s in st)
            cg += sum(s.cg_iters for s in st)
        b.record(self.stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 1e3
        return {"value": cp / t, "unit": "CP iterations/s", "ms_per_step": 1e3 * t / steps,
                "avg_pcg_per_cp": cg / max(cp, 1), "steps": steps}


def headline_problem(precision, cp=CP_PER_STEP, **kw):
    inst = mi.config3()
    p = dict(inst["problem"], max_cp=cp, cg_tol=CG_TOL, precision=precision, **kw)
    return inst, p


def config2_measure(L, dev, stream, precision, cp=CP_PER_STEP, steps=2):
    """The 2-D periodic 128^2 x 64 workload, four viscosities in one plan."""
    insts = [mi.config2(nu=nu) for nu in mi.CONFIG2_NU]
    probs = [dict(i["problem"], max_cp=cp, cg_tol=CG_TOL, precision=precision) for i in insts]
    fx = Fixed(L, dev, insts, probs, stream)
    L.mfg_autotune(fx.plan, stream=stream)
    out = fx.timed(steps=steps, warmup=1)
    out["workload"] = ("2-D periodic 128x128, N_t=64, nu in {1e-3,1e-2,1e-1,1} in one plan, "
                       f"{cp} CP iterations per instance per step")
    out["unknowns_cp_iters_per_s"] = out["value"] * 64 * 128 * 128
    return out


def batch_measure(L, dev, stream, precision, count=64, cp=CP_PER_STEP):
    """The uneven batch: `count` seeded instances (periodic or Neumann, N in
    {64,128,256}, N_t in {32,64,128}, nu log-uniform) in one plan and one graph
    launch; aggregate CP iterations/s."""
    insts = mi.config5(count=count)
    probs = [dict(i["problem"], max_cp=cp, cg_tol=CG_TOL, precision=precision) for i in insts]
    fx = Fixed(L, dev, insts, probs, stream)
    t0 = time.perf_counter()
    L.mfg_autotune(fx.plan, stream=stream)
    tune_s = time.perf_counter() - t0
    out = fx.timed(steps=1, warmup=1)
    out["autotune_seconds"] = tune_s
    nsum = sum(i["problem"]["nt"] * i["problem"]["n"][0] * i["problem"]["n"][1] for i in insts)
    out["workload"] = f"{count} uneven instances (seeds 100..{100 + count - 1}), {cp} CP iterations each"
    out["unknowns_total"] = nsum
    out["unknowns_cp_iters_per_s"] = nsum * out["value"] / count
    return out


def adjoint_measure(L, dev, cp_iters=300):
    """One forward solve (300 CP iterations) and one adjoint solve on the
    128^2 x 64 periodic workload with nu = 0.05 (loss on m(T))."""
    import torch
    inst = mi.config4()
    p = dict(inst["problem"], max_cp=cp_iters, cg_tol=CG_TOL, precision=PRECISION)
    plan = L.mfg_plan(p)
    n = p["nt"] * p["n"][0] * p["n"][1]
    S = p["n"][0] * p["n"][1]
    t = _todev(dev)
    y = t(inst["y0"])
    ybar = y.clone()
    z = torch.zeros(n, dtype=torch.float64, device=dev)
    L.mfg_solve(plan, t(inst["m0"]), t(inst["V"]), t(inst["W"]), y, ybar, z)
    dx = p["len"][0] / p["n"][0]
    gy = torch.zeros_like(y)
    gy[(p["nt"] - 1) * S: p["nt"] * S] = 2.0 * (y[(p["nt"] - 1) * S: p["nt"] * S] - t(inst["m_target"])) * dx * dx
    out = [torch.empty(S, dtype=torch.float64, device=dev) for _ in range(3)]
    dnu = torch.empty(1, dtype=torch.float64, device=dev)
    L.mfg_adjoint(plan, 0, y, z, gy, out[0], out[1], out[2], dnu, tol=1e-10)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, st = L.mfg_adjoint(plan, 0, y, z, gy, out[0], out[1], out[2], dnu, tol=1e-10)
    torch.cuda.synchronize()
    return {"workload": "2-D periodic 128x128, N_t=64, nu=0.05, loss ||m(T)-m_target||^2",
            "ms": 1e3 * (time.perf_counter() - t0), "adjoint_pcg_iters": int(st.cg_iters),
            "final_rel_residual": st.r_last, "status": int(rc), "dnu": float(dnu.item())}


def kernels_measure(L, dev, stream, peak_gbs):
    """Each hot entry point on the headline workload, timed with CUDA events on
    the launching stream.  `algorithmic_gbs` counts the bytes the step must
    move (operands read once, results written once); `kernel_gbs` counts what
    the kernels themselves read and write, intermediates included."""
    import torch
    inst, p = headline_problem("mixed", cp=1)
    n = p["nt"] * p["n"][0] * p["n"][1]
    t = _todev(dev)
    V, W = t(inst["V"]), t(inst["W"])
    g = torch.Generator(device=dev).manual_seed(3)
    r = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
    z = torch.empty_like(r)
    y = torch.randn(5 * n, dtype=torch.float64, device=dev, generator=g)
    y[:n] = y[:n].abs() + 0.5
    ybar = torch.empty_like(y)
    zd = 1e-2 * torch.randn(n, dtype=torch.float64, device=dev, generator=g)

    def timed(f, reps=5):
        for _ in range(2):
            f()
        torch.cuda.synchronize()
        a, b = _events(stream)
        a.record(stream)
        for _ in range(reps):
            f()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3 / reps

    def entry(sec, alg_bytes, kern_bytes, bound):
        return {"us": 1e6 * sec, "algorithmic_bytes": alg_bytes, "algorithmic_gbs": alg_bytes / sec / 1e9,
                "kernel_bytes": kern_bytes, "kernel_gbs": kern_bytes / sec / 1e9,
                "hbm_frac_algorithmic": alg_bytes / sec / 1e9 / peak_gbs, "bound": bound}

    out = {"workload": "2-D Neumann 512^2 x N_t 128, nu = 1e-2 (n = 33,554,432)"}
    plan = L.mfg_plan(dict(p, precision="mixed"))
    out["AAt apply (k_aat_x + k_aat_q)"] = entry(
        timed(lambda: L.mfg_apply_AAt(plan, 0, r, z, stream=stream)), 16 * n, 56 * n, "FP64 issue")
    out["C apply (k_apply_C)"] = entry(timed(lambda: L.mfg_apply_C(plan, 0, y, z, stream=stream)),
                                       48 * n, 48 * n, "FP64 issue")

    def prox_step():
        L.mfg_prox_step(plan, 0, 0.5, zd, y, ybar, V, W, stream=stream)
    # the in-solve primal step: reads z, y; writes y, ybar (y is overwritten in
    # place each repetition, which keeps the values in the same range)
    out["prox step (k_prox_cp, in-solve)"] = entry(timed(prox_step), 128 * n, 128 * n, "FP64 issue")
    # P^-1 in 3 passes' worth of algorithmic bytes (FP64 in, FP64 out, FP32 in between:
    # 8 + 4 + 4 + 4 + 4 + 8); the five passes move 48 B per unknown
    out["P^-1 apply, FP32, CUDA-core time pass"] = entry(
        timed(lambda: L.mfg_apply_precond(plan, 0, r, z, stream=stream)), 32 * n, 48 * n, "HBM / latency")
    plan_tc = L.mfg_plan(dict(p, precision="mixed_tc"))
    out["P^-1 apply, FP32, tensor-core time pass"] = entry(
        timed(lambda: L.mfg_apply_precond(plan_tc, 0, r, z, stream=stream)), 32 * n, 48 * n, "HBM / latency")
    return out


def exact_time_measure(L, dev, stream):
    """The headline step with l = 0 (time blocks solved exactly per spatial mode,
    P = AAt; not the paper's preconditioner), FP32 preconditioner."""
    inst, p = headline_problem("mixed", l=0)
    out = Fixed(L, dev, [inst], [p], stream).timed(steps=1, warmup=1)
    out["workload"] = "headline workload, l = 0 (exact time solve, P = AAt), precision mixed"
    return out


def varnu_measure(L, dev, stream, cp=100, reps=5):
    """A viscosity field nu(x) (smooth, 10:1 around 1e-2, seed 7) on the 2-D
    Neumann 128^2 x 64 grid, headline precision: plan build (host banded
    Cholesky per time frequency, the LU option of Alg. 1), one P^-1 apply next
    to the constant-nu apply of the same grid, and `cp` CP iterations per step."""
    import time

    import torch
    try:
        inst = mi.config_varnu(n=128, nt=64)
        p = dict(inst["problem"], max_cp=cp, cg_tol=CG_TOL, precision=PRECISION)
        t0 = time.perf_counter()
        fx = Fixed(L, dev, [inst], [p], stream)
        plan_s = time.perf_counter() - t0
        out = fx.timed(steps=1, warmup=1)
        n = fx.sizes["dual"]
        r = torch.randn(n, dtype=torch.float64, device=dev)
        z = torch.empty_like(r)
        pc = {k: v for k, v in p.items() if k != "nu_field"}
        const = L.mfg_plan(pc)

        def timed(plan):
            for _ in range(2):
                L.mfg_apply_precond(plan, 0, r, z, stream=stream)
            torch.cuda.synchronize()
            a, b = _events(stream)
            a.record(stream)
            for _ in range(reps):
                L.mfg_apply_precond(plan, 0, r, z, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            return 1e3 * a.elapsed_time(b) / reps

        out.update(workload=f"2-D Neumann 128^2 x 64, nu(x) smooth 10:1 around 1e-2, {cp} CP iterations per step, "
                            f"{PRECISION}", plan_build_s=plan_s, precond_apply_us=timed(fx.plan),
                   constant_nu_precond_apply_us=timed(const))
        return out
    except Exception as e:  # an extra line only: never let it break the benchmark line
        return {"unavailable": f"{type(e).__name__}: {e}"[:200]}


def cufft_compare(L, dev, reps=10):
    """cuFFT as a timed comparison only: torch.fft's 2-D real FFT forward and
    inverse over the 128 planes of the headline grid (FP32), next to one
    preconditioner apply of this library (FP64 in and out, spatial forward and
    inverse passes, time pass and division)."""
    import torch
    try:
        inst, p = headline_problem(PRECISION)
        x = torch.randn(p["nt"], p["n"][0], p["n"][1], dtype=torch.float32, device=dev)

        def timed(f):
            for _ in range(3):
                f()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                f()
            b.record()
            torch.cuda.synchronize()
            return 1e3 * a.elapsed_time(b) / reps

        t_fft = timed(lambda: torch.fft.irfft2(torch.fft.rfft2(x), s=tuple(p["n"])))
        plan = L.mfg_plan(p)
        r = torch.randn(x.numel(), dtype=torch.float64, device=dev)
        z = torch.empty_like(r)
        t_pre = timed(lambda: L.mfg_apply_precond(plan, 0, r, z))
        return {"workload": "128 planes of 512^2 (the headline grid; cuFFT does the periodic DFT, "
                            "the library the Neumann DCT-II)",
                "cufft_rfft2_irfft2_fp32_us": t_fft, "precond_apply_us": t_pre}
    except Exception as e:  # a comparison only: never let it break the benchmark line
        return {"unavailable": f"{type(e).__name__}: {e}"[:200]}


def oracle_parity(L, dev, stream, precision, iters=30):
    """The iterate after `iters` CP iterations on the stiffest 128^2 x 64
    instance (nu = 1, cond(AAt) ~ 7e9) against the FP64 oracle's exact-solve run
    (the full 300-iteration comparisons are in the GPU test-suite)."""
    import torch
    from oracle.cp import Solver
    inst = mi.config2(nu=1.0)
    p = dict(inst["problem"], max_cp=iters, cg_tol=CG_TOL, precision=precision)
    fx = Fixed(L, dev, [inst], [p], stream)
    fx.step()
    torch.cuda.synchronize()
    y = fx.y.cpu().numpy()
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal").run(inst["y0"], iters=iters)
    err = float(np.linalg.norm(y - ref["y"].reshape(-1)) / np.linalg.norm(ref["y"]))
    return {"workload": f"2-D periodic 128x128, N_t=64, nu=1, {iters} CP iterations, precision {precision}",
            "rel_l2_err_vs_oracle": err, "bar": 1e-8}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for key in ("Model name", "Vendor ID"):
            for ln in out.splitlines():
                if ln.startswith(key):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline_sample(iters=1, threads=None, which="headline", time_cap=None):
    """The oracle, as it stands, on a bounded sample: up to `iters` CP
    iterations (stopping early once `time_cap` seconds have passed) with its
    exact spatially-diagonalised AAt solve and bisection prox, on `threads`
    host threads (default all cores)."""
    import oracle
    from oracle.cp import Solver
    cores = oracle.set_threads(threads)
    try:
        if which == "headline":
            inst, p = headline_problem("fp64")
            label = "512^2 x 128 Neumann (the headline workload)"
        else:
            inst = mi.config2(nu=1e-2)
            p = dict(inst["problem"])
            label = "128^2 x 64 periodic, nu = 1e-2"
        s = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal")
        y, state, done = inst["y0"], {}, 0
        t0 = time.perf_counter()
        while done < iters:
            res = s.run(y, iters=1, ybar0=state.get("ybar"), x0=state.get("x"), tau0=state.get("tau"),
                        sigma0=state.get("sigma"))
            y = res["y"]
            state = {"ybar": res["ybar"], "x": res["x"], "tau": res["tau"], "sigma": res["sigma"]}
            done += 1
            if time_cap is not None and time.perf_counter() - t0 >= time_cap:
                break
        el = time.perf_counter() - t0
    finally:
        oracle.set_threads()
    return {"value": done / el, "unit": "CP iterations/s", "cores": cores, "kind": "oracle",
            "cpu": cpu_model(), "nproc": os.cpu_count(), "cp_iters": done,
            "sample": f"{done} CP iteration(s) of the {label} workload from the initial iterate (oracle: "
                      f"exact modal AAt solve, bisection prox), {el:.1f} s on {cores} thread(s)"}


def run_gpu(args):  # noqa: C901
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl", device_id=dev)
    import paper_2507_01958_gb300 as pkg
    L = pkg.lib()
    stream = torch.cuda.current_stream(dev)
    inst, p = headline_problem(args.precision, cp=args.cp_per_step)
    if args.small:
        if not args.quick:
            raise SystemExit("--small applies to --kernels-only and --quick runs only")
        inst = mi.config3(nt=32)  # 512^2 x 32: a profiling case, not a benchmark number
        p = dict(inst["problem"], max_cp=args.cp_per_step, cg_tol=CG_TOL, precision=args.precision)
    main = Fixed(L, dev, [inst], [p], stream)
    if not args.no_autotune:
        L.mfg_autotune(main.plan, stream=stream)
    schedule = L.mfg_get_schedule(main.plan, 0)
    if args.eager:
        L.mfg_set_launch_mode(main.plan, "eager")
    n_per = p["nt"] * p["n"][0] * p["n"][1]

    for _ in range(args.warmup):
        main.step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as td
        td.barrier()
    l0 = L.mfg_kernel_launches(main.plan)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = _events(stream)
    torch.cuda.synchronize()
    e0.record(stream)
    cg_total = cp_total = 0
    for _ in range(args.steps):
        st = main.step()
        cg_total += sum(s.cg_iters for s in st)
        cp_total += sum(s.cp_iters for s in st)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = L.mfg_kernel_launches(main.plan) - l0
    t_local = e0.elapsed_time(e1) / 1e3
    t = reduce_max(t_local, world, dev)
    cp_all = reduce_sum(float(cp_total), world, dev)
    cg_all = reduce_sum(float(cg_total), world, dev)
    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "value": cp_all / t, "unit": "CP iterations/s",
                              "ms_per_step": 1e3 * t / max(args.steps, 1), "pcg_iters": cg_all,
                              "cp_iters": cp_all, "gpu_launches": int(launches)}))
        return

    # End to end through the host-buffer entry point: every step copies the
    # inputs and the start iterate from pinned host memory and reads the
    # iterate back (copies inside the timed region).  Each timed step gets its
    # own pinned start iterate, filled before the timed region (the call
    # overwrites y, ybar, z with the result).
    pin = lambda a: torch.as_tensor(a).pin_memory()
    hm0, hV, hW = pin(main.host["m0"]), pin(main.host["V"]), pin(main.host["W"])
    e2e_steps = max(1, min(args.steps, 2))

    def start_iterate():
        return (pin(main.host["y0"].copy()), pin(main.host["y0"].copy()),
                torch.zeros(main.sizes["dual"], dtype=torch.float64).pin_memory())

    def host_step(bufs):
        hy, hyb, hz = bufs
        return L.mfg_solve_host(main.plan, hm0, hV, hW, hy, hyb, hz, stream=stream)[1]

    host_step(start_iterate())  # first call allocates the plan's staging buffers
    sets = [start_iterate() for _ in range(e2e_steps)]
    torch.cuda.synchronize()
    e2e_clocks = ClockSampler(local)
    e2e_clocks.start()
    h0 = time.perf_counter()
    for i in range(e2e_steps):
        st = host_step(sets[i])
    h1 = time.perf_counter()
    e2e_clk = e2e_clocks.stop()
    del sets
    t_e2e = reduce_max(h1 - h0, world, dev)
    cp_e2e = reduce_sum(float(sum(s.cp_iters for s in st) * e2e_steps), world, dev)
    sz = main.sizes
    h2d = 8 * (3 * sz["field"] + 2 * sz["primal"] + sz["dual"])
    d2h = 8 * (2 * sz["primal"] + sz["dual"])

    # Plain FP64 GPU path on the same workload, and the headline precision over
    # the same (shorter) count, for the mixed-vs-FP64 ratio and difference.
    cmp_iters = 30
    inst64, p64 = headline_problem("fp64", cp=cmp_iters)
    f64 = Fixed(L, dev, [inst64], [p64], stream)
    r64 = f64.timed(steps=1, warmup=1)
    instm, pm = headline_problem(args.precision, cp=cmp_iters)
    fm = Fixed(L, dev, [instm], [pm], stream)
    rm = fm.timed(steps=1, warmup=1)
    err_mixed = float(torch.linalg.norm(fm.y - f64.y) / torch.linalg.norm(f64.y))
    del f64, fm

    # Dominant kernel: the AAt apply (k_aat_x + k_aat_q, FP64 issue bound), timed
    # with CUDA events on the stream it is launched on, same launch shapes as in
    # the solve graph.
    p_in = torch.randn(n_per, dtype=torch.float64, device=dev)
    q_out = torch.empty_like(p_in)
    for _ in range(3):
        L.mfg_apply_AAt(main.plan, 0, p_in, q_out, stream=stream)
    reps = 20
    a0, a1 = _events(stream)
    a0.record(stream)
    for _ in range(reps):
        L.mfg_apply_AAt(main.plan, 0, p_in, q_out, stream=stream)
    a1.record(stream)
    torch.cuda.synchronize()
    t_aat = a0.elapsed_time(a1) / 1e3 / reps
    flops = AAT_FLOPS_PER_UNKNOWN * n_per
    achieved = flops / t_aat / 1e12
    traffic = profiled_traffic("k_aat_config3.md")
    del p_in, q_out

    peaks, src = load_peaks()
    extras = {}
    if not args.no_extras:
        extras["kernels_headline_workload"] = kernels_measure(L, dev, stream, peaks.get("hbm_gbs", 6800.0))
        extras["config2_four_viscosities"] = config2_measure(L, dev, stream, args.precision)
        extras["batch_uneven"] = batch_measure(L, dev, stream, args.precision)
        extras["exact_time_solve"] = exact_time_measure(L, dev, stream)
        extras["viscosity_field"] = varnu_measure(L, dev, stream)
        extras["adjoint"] = adjoint_measure(L, dev)
        extras["cufft_comparison"] = cufft_compare(L, dev)
        if rank == 0:
            extras["parity_vs_oracle"] = oracle_parity(L, dev, stream, args.precision)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(iters=1)
        cpu["one_core"] = cpu_baseline_sample(iters=2, threads=1, which="config2")

    if rank == 0:
        out = {
            "metric": METRIC,
            "value": cp_all / t,
            "unit": "CP iterations/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64+f32",
            "data": "synthetic (seeded fields shaped like the paper's experiments)",
            "config": {"workload": WORKLOAD, "instances": 1, "unknowns": n_per, "primal_unknowns": 5 * n_per,
                       "pcg_rel_tol": CG_TOL, "pcg_stop_reference": "||b|| of the system of eq. CC*",
                       "precision": args.precision, "parallelism": f"replicas x{world}",
                       "l2": "working set ~4 GB > 129 MB L2; no flush"},
            "pcg_iters_per_s": cg_all / t,
            "unknowns_cp_iters_per_s": cp_all * n_per / t,
            "avg_pcg_per_cp": cg_all / max(cp_all, 1.0),
            "fp64_path": {"value": r64["value"], "unit": "CP iterations/s", "cp_iters": cmp_iters,
                          "avg_pcg_per_cp": r64["avg_pcg_per_cp"],
                          "headline_precision_same_count": rm["value"]},
            "mixed_vs_fp64_speedup": rm["value"] / r64["value"],
            "mixed_rel_err_vs_fp64_path": err_mixed,
            "roofline": {"kernel": "AAt apply: k_aat_x + k_aat_q (C C^T stencil, FP64)", "bound": "alu",
                         "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                         "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch":
                             AAT_BYTES_PER_UNKNOWN * n_per, "avg_launch_us": 1e6 * t_aat,
                         "hbm_achieved_gbs": AAT_BYTES_PER_UNKNOWN * n_per / t_aat / 1e9,
                         "hbm_peak_gbs": peaks.get("hbm_gbs"), "peak_source": f"{src} (HBM); recipe table (FP64)"},
            "cpu_baseline": cpu,
            "e2e": {"value": cp_e2e / t_e2e, "unit": "CP iterations/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps, "clocks": e2e_clk},
            "gpu_launches": int(launches),
            "clocks": clk,
            "schedule": schedule,
        }
        out.update(extras)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as td
        td.barrier()
        td.destroy_process_group()


def run_kernels_only(args):
    """Three launches each of the standalone AAt, preconditioner and prox-step
    entry points (a short program for ncu captures).  --small takes the
    512^2 x 32 Neumann grid (vectors of 67 MB, still larger than L2 with the
    stencil intermediates) instead of the headline's 512^2 x 128.  --field
    takes the viscosity-field workload instead (128^2 x 64 Neumann, 10:1
    smooth field; --small: 64^2 x 32), whose preconditioner runs the banded
    per-frequency solves."""
    import torch
    import paper_2507_01958_gb300 as pkg
    L = pkg.lib()
    if args.field:
        inst = mi.config_varnu(n=64, nt=32) if args.small else mi.config_varnu()
    else:
        inst = mi.config3(nt=32) if args.small else mi.config3()
    p = dict(inst["problem"], max_cp=1, cg_tol=CG_TOL, precision=args.precision)
    plan = L.mfg_plan(p)
    n = p["nt"] * p["n"][0] * p["n"][1]
    g = torch.Generator(device="cuda").manual_seed(0)
    r = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    z = torch.empty_like(r)
    y = torch.randn(5 * n, dtype=torch.float64, device="cuda", generator=g)
    y[:n] = y[:n].abs() + 0.5
    ybar = torch.empty_like(y)
    V = torch.as_tensor(inst["V"]).reshape(-1).cuda()
    W = torch.as_tensor(inst["W"]).reshape(-1).cuda()
    for _ in range(3):
        L.mfg_apply_AAt(plan, 0, r, z)
        L.mfg_apply_precond(plan, 0, r, z)
        L.mfg_prox_step(plan, 0, 0.5, 1e-2 * r, y, ybar, V, W)
    torch.cuda.synchronize()
    print(json.dumps({"kernels_only": True, "unknowns": n, "launches": L.mfg_kernel_launches(plan)}))


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the host cores, one CP
    iteration of the headline workload per step."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    # a step is one CP iteration; the run stops after 150 s of oracle time (the
    # sample says how many of the requested steps it took).  The oracle has no
    # state worth warming up: every iteration does the same work.
    t0 = time.perf_counter()
    res = cpu_baseline_sample(iters=args.steps, time_cap=150.0)
    t = time.perf_counter() - t0
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": res["value"],
        "unit": "CP iterations/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t / res["cp_iters"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded fields shaped like the paper's experiments)",
        "config": {"workload": WORKLOAD, "instances": 1,
                   "sample": f"one CP iteration per step, {res['cp_iters']} of {args.steps} steps run (150 s cap)"},
        "cpu_baseline": {"value": res["value"], "unit": "CP iterations/s", "cores": res["cores"], "kind": "oracle",
                         "sample": res["sample"], "cpu": res["cpu"]},
        "e2e": {"value": res["value"], "unit": "CP iterations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cp-per-step", type=int, default=CP_PER_STEP)
    ap.add_argument("--precision", default=PRECISION, choices=["mixed", "mixed_tc", "mixed_df", "fp64"],
                    help="precision of the timed solve (default: FP32 preconditioner with the tensor-core time pass)")
    ap.add_argument("--quick", action="store_true", help="main timed loop only (profiling runs)")
    ap.add_argument("--no-extras", action="store_true", help="skip the extra measurements after the headline")
    ap.add_argument("--kernels-only", action="store_true",
                    help="three launches of each standalone hot kernel (for ncu captures)")
    ap.add_argument("--small", action="store_true",
                    help="--kernels-only or --quick on the 512^2 x 32 Neumann grid (profiling runs)")
    ap.add_argument("--field", action="store_true",
                    help="--kernels-only on the viscosity-field workload (banded preconditioner)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch choices instead of the autotuner's measured ones")
    ap.add_argument("--eager", action="store_true",
                    help="issue kernels one by one instead of one graph launch (per-kernel profiling)")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    elif args.kernels_only:
        run_kernels_only(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
