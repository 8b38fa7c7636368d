#!/usr/bin/env python3
"""Benchmark of the SEM Poisson hot path on GB300.

One step = one complete mixed-precision (FP32 operator / FP64 gather-scatter
sums, dots and refinement) Jacobi PCG solve to a relative residual of 1e-8 on
the deformed 32x32x32-element, N = 7 box (16.8 M local DOFs), right-hand side
uniform in [-1, 1) per global node (seed 0), inputs resident in HBM.
`value` = local DOFs x PCG iterations / step time (GDOF/s), summed over ranks.

Extra keys: time to solution (mixed and FP64), the FP32 and FP64 operator
throughput, the roofline of the dominant kernel (the FP32 element operator)
and of the plain FP32 and the FP64 operators,
the clocks seen during the timed region, the end-to-end number through the
C-ABI with host buffers, and the CPU oracle timed on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import tempfile
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Ax GDOF/s + PCG time-to-1e-8 residual, mixed/learned vs FP64, 1 GB300"
WORKLOAD = dict(kx=32, ky=32, kz=32, N=7, deform=True, rhs="uniform[-1,1) per global node, seed 0",
                tol=1e-8)
WORKLOAD_NAME = "deformed 32x32x32 hex, N=7 (16.8M local DOFs), Jacobi PCG to 1e-8, mixed FP32/FP64"
# the CPU oracle's sample: the benchmark workload itself (deformed 32^3, N = 7),
# a few FP64 Jacobi PCG iterations (1.4 to 4 s each on one core)
CPU_SAMPLE = dict(k=32, N=7, iters=4)
_ORACLE_PROBLEMS = {}
# DRAM bytes (read + write) per local DOF of one launch, from an ncu capture
# of the current kernels (the profile summaries under profiles/ give the
# commands); None until measured for the kernel as it stands.
TRAFFIC = {"operator_pcg": 42.65, "operator_plain": 31.11, "operator_fp64": 63.29}


class EnergyMeter:
    """Total energy counter of one GPU through the driver's NVML library
    (ctypes, read-only: nvmlDeviceGetTotalEnergyConsumption, millijoules
    since driver load).  None when the library or the counter is missing."""

    def __init__(self, index):
        import ctypes
        self.ok = False
        try:
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                return
            self.dev = ctypes.c_void_p()
            if self.lib.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.dev)) != 0:
                return
            self.ctypes = ctypes
            self.ok = self.read() is not None
        except OSError:
            pass

    def read(self):
        v = self.ctypes.c_ulonglong()
        if self.lib.nvmlDeviceGetTotalEnergyConsumption(self.dev, self.ctypes.byref(v)) != 0:
            return None
        return v.value / 1e3   # joules


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def fp64_peak(num_sms):
    """Nominal FP64 FMA rate in TFLOP/s, for context beside the measured one:
    SMs x 4 flop per clock (two FP64 FMAs per SM and clock, the rate behind
    GB300's nominal 1.25 TFLOP/s) x the maximum SM clock
    (MEASURED_PEAKS.json, else 2070 MHz)."""
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        mhz = float(json.load(open(p)).get("sm_max_mhz", mhz))
    return num_sms * 4 * mhz * 1e6 / 1e12, f"derived: {num_sms} SMs x 4 FP64 flop/clock x {mhz:.0f} MHz"


def fma_peaks(sem):
    """Measured FMA throughput of the CUDA cores (sem_fma_peak: 8 independent
    FMA chains per thread, 8 blocks of 256 threads per SM, CUDA events), in
    TFLOP/s: the roofline denominator of the compute-bound FP64 operator."""
    return {"fp64_tflops": sem.sem_fma_peak(True, 4096),
            "fp32_tflops": sem.sem_fma_peak(False, 262144),
            "method": "sem_fma_peak: 8 FMA chains per thread, 8 x 256 threads per SM, "
                      "one warm-up and one timed launch (CUDA events); no clock or power change"}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples go to a temporary file; the JSON line carries the summary
        self.path = os.path.join(tempfile.gettempdir(), f"sem_clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
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
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _single_thread_env():
    """Pool initializer: one BLAS/OpenMP thread per oracle process (set before
    the worker imports numpy)."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def _oracle_ax_worker(args):
    """One oracle process: builds a deformed k^3 box at order N (untimed),
    waits for the common start time, then times `reps` calls of the oracle's
    ax_local as it stands.  Returns (local DOFs, reps, seconds)."""
    N, k, reps, start_at = args
    import numpy as np
    from oracle import sem_oracle as so
    P = so.Problem(k, k, k, N, deform=True)
    u = np.random.default_rng(N).uniform(-1.0, 1.0, P.L)
    P.ax_local(u)   # first touch
    while time.time() < start_at:
        time.sleep(0.01)
    t0 = time.perf_counter()
    for _ in range(reps):
        P.ax_local(u)
    return P.L, reps, time.perf_counter() - t0


def cpu_legs(orders=(5, 7, 9, 11, 13, 15), k=8, reps=3):
    """The oracle (unchanged) on the host cores, beside the GPU numbers:
    config 1's full FP64 Jacobi PCG solve to 1e-10 (one core), and config 3's
    element operator per order on one core and on every core (one spawned
    process per core, each applying the oracle's ax_local to its own
    deformed k^3-element box, all started together; throughput = all local
    DOFs / the slowest process's time).  The oracle is single-threaded numpy
    (einsum contractions), so one process is one core."""
    import multiprocessing as mp
    from oracle import sem_oracle as so
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    out = {"cores_available": cores, "kind": "oracle"}
    P1 = so.Problem(4, 4, 4, 7)
    b1 = P1.rhs_sine()
    t0 = time.perf_counter()
    _, it1, hist1 = P1.pcg(b1, tol=1e-10, maxit=500)
    dt1 = time.perf_counter() - t0
    out["config1_fp64_pcg_to_1e-10"] = {"time_s": dt1, "iterations": it1, "relres": hist1[-1],
                                        "cores": 1, "local_dofs": P1.L}
    sweep = []
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_single_thread_env) as pool:
        for N in orders:
            L1, r1, t1 = _oracle_ax_worker((N, k, reps, 0.0))
            start = time.time() + 4.0 + 0.02 * N * N   # after every worker's (untimed) build
            res = pool.map(_oracle_ax_worker, [(N, k, reps, start)] * cores)
            tmax = max(r[2] for r in res)
            sweep.append({"N": N, "elements_per_process": k ** 3, "local_dofs_per_process": L1,
                          "gdofs_1core": L1 * r1 / t1 / 1e9,
                          "gdofs_all_cores": sum(r[0] * r[1] for r in res) / tmax / 1e9,
                          "cores": cores})
    out["config3_ax"] = sweep
    return out


def cpu_baseline(sample=CPU_SAMPLE):
    """The CPU oracle as it stands, on a bounded sample of the same work: the
    benchmark's problem (built once, untimed), a few FP64 Jacobi PCG
    iterations timed (the initial residual included)."""
    from oracle import sem_oracle as so
    key = (sample["k"], sample["N"])
    if key not in _ORACLE_PROBLEMS:
        P = so.Problem(sample["k"], sample["k"], sample["k"], sample["N"], deform=True)
        _ORACLE_PROBLEMS[key] = (P, P.rhs_uniform(0))
    P, b = _ORACLE_PROBLEMS[key]
    t0 = time.perf_counter()
    _, it, _ = P.pcg(b, fixed_iters=sample["iters"])
    dt = time.perf_counter() - t0
    value = P.L * it / dt / 1e9
    return {"value": value, "unit": "GDOF/s", "cores": 1, "kind": "oracle",
            "sample": f"{sample['iters']} FP64 Jacobi PCG iterations (initial residual included) "
                      f"of the numpy oracle on the benchmark problem, a deformed "
                      f"{sample['k']}^3-element N={sample['N']} box ({P.L} local DOFs), "
                      f"{dt:.1f} s; GDOF/s = local DOFs x iterations / time"}


def batched_leg(sem, torch):
    """64 independent deformed problems, k ~ U{8..24}, N ~ U{5,7,9} (seed 1),
    mixed precision to 1e-8: one batched solve (persistent launches, CUDA
    graph, autotuned) against the same problems solved one after another."""
    import sem_inputs
    cases = sem_inputs.batched_cases()
    meshes = [sem.box_mesh(k, k, k, deform=True) for k, _ in cases]
    t0 = time.perf_counter()
    b = sem.sem_batch_setup(meshes, [N for _, N in cases])
    setup_s = time.perf_counter() - t0
    fs, xs, hs = [], [], []
    for i in range(len(cases)):
        h = sem.sem_batch_problem(b, i)
        L = sem.sem_get_sizes(h).L
        f = torch.empty(L, dtype=torch.float64, device="cuda")
        sem.sem_rhs(h, sem.RHS_UNIFORM, 1000 + i, f)
        fs.append(f)
        xs.append(torch.zeros_like(f))
        hs.append(h)
    torch.cuda.synchronize()
    o = sem.sem_solve_opts()
    o.tol, o.maxit, o.precision = 1e-8, 5000, sem.SEM_MIXED_FP32
    sem.sem_batch_pcg_solve(b, fs, xs, o)   # warm-up (graph capture)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, infos = sem.sem_batch_pcg_solve(b, fs, xs, o)
    torch.cuda.synchronize()
    batched_s = time.perf_counter() - t0
    # the same problems, one standalone solve after another
    for i in range(len(cases)):
        sem.sem_pcg_solve_ex(hs[i], fs[i], None, xs[i], o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq_iters = 0
    seq_ok = True
    for i in range(len(cases)):
        rci, inf = sem.sem_pcg_solve_ex(hs[i], fs[i], None, xs[i], o)
        seq_iters += inf.iters
        seq_ok = seq_ok and rci == 0
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    Ls = [sem.sem_get_sizes(h).L for h in hs]
    total_L = sum(Ls)
    it = [i["iters"] for i in infos]
    dof_iters = sum(L_i * it_i for L_i, it_i in zip(Ls, it))
    out = {"problems": len(cases), "local_dofs": total_L, "orders": sorted(set(N for _, N in cases)),
           "k_range": [min(k for k, _ in cases), max(k for k, _ in cases)],
           "batched_ms": batched_s * 1e3, "sequential_ms": seq_s * 1e3,
           "speedup_vs_sequential": seq_s / batched_s, "setup_s": setup_s,
           "iterations_min_max": [min(it), max(it)], "all_converged": rc == 0 and seq_ok,
           "max_relres_true": max(i["relres_true"] for i in infos),
           "gdofs": dof_iters / batched_s / 1e9,
           "gdofs_sequential": dof_iters / seq_s / 1e9,
           "gdofs_definition": "sum over problems of local DOFs x iterations / time",
           "autotune": {f"n{N + 1}": {"variant": sem.sem_batch_get_option(b, f"variant_n{N + 1}"),
                                      "grid": sem.sem_batch_get_option(b, f"grid_n{N + 1}")}
                        for N in sorted(set(N for _, N in cases))},
           "launches_per_solve": infos[0]["launches"]}
    sem.sem_batch_destroy(b)
    return out


def order_sweep_leg(sem, torch, hbm_gbs, fp64_peak_tflops):
    """Deformed cubes of about 2^24 local DOFs at N = 5, 7, ..., 15: FP32 and
    FP64 operator (sem_ax_local) throughput with CUDA events, fraction of
    the HBM roofline (FP32: 32 B per DOF), FP64 flop rate (12 n^4 + 15 n^3
    per element), and the FP32 result's max-norm error relative to the FP64
    operator on the same input."""
    import sem_inputs
    out = []
    for N in (5, 7, 9, 11, 13, 15):
        c = sem_inputs.order_sweep_case(N)
        stream = torch.cuda.Stream()
        S = sem.Solver(c.kx, c.ky, c.kz, N, deform=True, stream=stream.cuda_stream)
        L = S.L
        with torch.cuda.stream(stream):
            gen = torch.Generator(device="cuda").manual_seed(N)
            u64 = torch.rand(L, dtype=torch.float64, device="cuda", generator=gen) * 2 - 1
            u32 = u64.float()
            w64 = torch.empty_like(u64)
            w32 = torch.empty_like(u32)
        stream.synchronize()

        def timed(fn, u, w, prec, reps):
            for _ in range(2):
                fn(S.h, u, w, prec)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn(S.h, u, w, prec)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        ms32 = timed(sem.sem_ax_local, u32, w32, sem.SEM_MIXED_FP32, 10)
        ms64 = timed(sem.sem_ax_local, u64, w64, sem.SEM_FP64, 3)
        err = float((w32.double() - w64).abs().max() / w64.abs().max())
        tc = {}
        for name, prec in (("tf32", sem.SEM_MIXED_TF32), ("bf16x3", sem.SEM_MIXED_BF16X3)):
            ms = timed(sem.sem_ax_local, u32, w32, prec, 5)
            tc[name] = {"gdofs": L / ms / 1e6,
                        "hbm_frac": L * 32 / (ms * 1e-3) / 1e9 / hbm_gbs,
                        "rel_err_vs_fp64": float((w32.double() - w64).abs().max() / w64.abs().max())}
        n = N + 1
        flops = S.E * (12 * n ** 4 + 15 * n ** 3)
        out.append({"N": N, "elements": S.E, "local_dofs": L,
                    "fp32_gdofs": L / ms32 / 1e6, "fp32_hbm_frac": L * 32 / (ms32 * 1e-3) / 1e9 / hbm_gbs,
                    "fp32_tflops": flops / (ms32 * 1e-3) / 1e12,
                    "fp64_gdofs": L / ms64 / 1e6, "fp64_tflops": flops / (ms64 * 1e-3) / 1e12,
                    "fp64_frac_of_measured_fma_peak": flops / (ms64 * 1e-3) / 1e12 / fp64_peak_tflops,
                    "fp32_rel_err_vs_fp64": err, "tensor_cores": tc,
                    "fp32_kernel": "bulk-copy staged" if n % 2 == 0 else "register/shared (unstaged)",
                    "fp32_variant": int(sem.sem_get_option(S.h, "ax_variant")),
                    "fp32_tune_ms": [sem.sem_get_option(S.h, f"ax_tune_ms_plain_{v}") for v in range(5)]})
        S.close()
        del u64, u32, w64, w32
    return out


def mg_leg(sem, torch, S, b, stream):
    """Multigrid-preconditioned solves of the benchmark problem (FP64 and
    mixed, to the same tolerance), the set-up time of the levels and the
    device time of one V-cycle in each precision."""
    out = {}
    with torch.cuda.stream(stream):
        x = torch.empty_like(b)
        r = b.clone()
        z = torch.empty_like(b)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sem.sem_mg_apply(S.h, r, z, sem.SEM_FP64)          # builds the levels
    torch.cuda.synchronize()
    out["setup_s"] = time.perf_counter() - t0
    levels = int(sem.sem_get_option(S.h, "mg_levels"))
    out["levels"] = levels
    out["omega"] = [sem.sem_get_option(S.h, f"mg_omega_{l}") for l in range(levels)]
    for name, prec, dt in (("fp64", sem.SEM_FP64, torch.float64),
                           ("mixed", sem.SEM_MIXED_FP32, torch.float32)):
        with torch.cuda.stream(stream):
            rr = r.to(dt)
            zz = torch.empty_like(rr)
        sem.sem_mg_apply(S.h, rr, zz, prec)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(5):
            sem.sem_mg_apply(S.h, rr, zz, prec)
        e1.record(stream)
        torch.cuda.synchronize()
        best = None
        for _ in range(2):
            _, inf = S.solve(b, tol=WORKLOAD["tol"], maxit=2000, precision=prec, x=x, precond="mg")
            if best is None or inf["solve_ms"] < best["solve_ms"]:
                best = inf
        out[name] = {"vcycle_ms": e0.elapsed_time(e1) / 5, "solve_ms": best["solve_ms"],
                     "iterations": best["iters"], "refinements": best["refinements"],
                     "relres_true": best["relres_true"], "converged": best["rc"] == 0}
    return out


def learned_leg(sem, torch, train_pairs=4096, pair_rows=1024, tests=32, epochs=8, batch=8192):
    """Config 5: deformed 16^3 elements, N = 7, random Fourier right-hand
    sides (modes |k| <= 8 per axis, amplitude 1/|k|^2).  Training pairs
    (b, x) come from the solver itself (zero x0, mixed, multigrid
    preconditioner, to 1e-8); each pair contributes `pair_rows` seeded
    random element rows.  Two networks: the element-local features, and the
    same plus a coarse approximation of the solution (two FP32
    multigrid-Richardson steps) at the element vertices.  On `tests`
    held-out right-hand sides, Jacobi PCG to 1e-8 from x0 = 0 and from each
    guess, FP64 and mixed; the learned times are CUDA events on the solver's
    stream around prediction + solve.  A control without the network (x0 =
    the same two multigrid steps) separates what the network adds."""
    stream = torch.cuda.Stream()
    S = sem.Solver(16, 16, 16, 7, deform=True, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        b = torch.empty(S.L, dtype=torch.float64, device="cuda")
        x0 = torch.empty_like(b)
        r = torch.empty_like(b)
        w = torch.empty_like(b)
    models = {}
    for name, coarse in (("local", 0), ("coarse", 2)):
        m = sem.sem_x0_create(S.h, 256, 7)
        sem.sem_x0_set_option(m, "pair_rows", pair_rows)
        sem.sem_x0_set_option(m, "reserve_rows", train_pairs * pair_rows)
        if coarse:
            sem.sem_x0_set_option(m, "coarse_cycles", coarse)
        models[name] = m
    t0 = time.perf_counter()
    gen_iters = []
    with torch.cuda.stream(stream):
        x = torch.empty_like(b)
    for sample in range(train_pairs):
        sem.sem_rhs_fourier(S.h, 5, sample, b)
        _, info = S.solve(b, tol=1e-8, maxit=500, precision=sem.SEM_MIXED_FP32, precond="mg", x=x)
        gen_iters.append(info["iters"])
        for m in models.values():
            sem.sem_x0_add_pair(m, b, x)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    rows = train_pairs * pair_rows
    steps = epochs * (rows // batch)
    flops_step = 2.0 * batch * (2 * 544 * 256 + 3 * 256 * 256 + 3 * 256 * 512)
    res = {"train_pairs": train_pairs, "rows_per_pair": pair_rows, "rows": rows, "epochs": epochs,
           "batch": batch, "steps": steps, "data_s": gen_s,
           "data_solver": "mixed, multigrid preconditioner, zero x0, to 1e-8",
           "data_iterations_max": max(gen_iters), "models": {}, "tests": []}
    for name, m in models.items():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loss = sem.sem_x0_train(m, epochs, batch, 1e-3, seed=0)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res["models"][name] = {"final_loss": loss, "train_ms": ms,
                               "train_tflops": flops_step * steps / (ms * 1e-3) / 1e12,
                               "flops": "GEMM flops of the 8 products per step (forward 3, backward 5)"}

    def timed(fn):
        ea = torch.cuda.Event(enable_timing=True)
        eb = torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        out = fn()
        eb.record(stream)
        torch.cuda.synchronize()
        return out, ea.elapsed_time(eb)

    def mg_steps(k):
        # the torch operations run on the solver's stream, in order with the
        # library's launches
        with torch.cuda.stream(stream):
            x0.zero_()
            for _ in range(k):
                sem.sem_ax(S.h, x0, w, sem.SEM_FP64)
                torch.sub(b, w, out=r)
                r32 = r.float()
                d32 = torch.empty_like(r32)
                sem.sem_mg_apply(S.h, r32, d32, sem.SEM_MIXED_FP32)
                x0.add_(d32.double())

    variants = (("local", 0), ("coarse", 0), ("coarse", 2))
    for sample in range(10001, 10001 + tests):
        sem.sem_rhs_fourier(S.h, 5, sample, b)
        row = {}
        for pname, prec in (("fp64", sem.SEM_FP64), ("mixed", sem.SEM_MIXED_FP32)):
            _, iz = S.solve(b, tol=1e-8, maxit=5000, precision=prec)
            entry = {"zero_iters": iz["iters"], "zero_ms": iz["solve_ms"]}
            (_, il), ms = timed(lambda: (mg_steps(2), S.solve(b, x0=x0, tol=1e-8, maxit=5000,
                                                                precision=prec))[1])
            entry["mg2_iters"], entry["mg2_ms"] = il["iters"], ms
            for mname, post in variants:
                m = models[mname]
                sem.sem_x0_set_option(m, "post_cycles", post)
                (_, il), ms = timed(lambda: (sem.sem_x0_predict(m, b, x0, True),
                                             S.solve(b, x0=x0, tol=1e-8, maxit=5000,
                                                     precision=prec))[1])
                key = f"{mname}_post{post}"
                entry[key + "_iters"], entry[key + "_ms"] = il["iters"], ms
                entry[key + "_converged"] = il["rc"] == 0
            row[pname] = entry
        res["tests"].append(row)
    summ = {}
    for pname in ("fp64", "mixed"):
        keys = ["zero", "mg2"] + [f"{m}_post{p}" for m, p in variants]
        summ[pname] = {k: {"iters_mean": statistics.mean(t[pname][k + "_iters"] for t in res["tests"]),
                           "ms_mean": statistics.mean(t[pname][k + "_ms"] for t in res["tests"])}
                       for k in keys}
    res["summary"] = summ
    for m in models.values():
        sem.sem_x0_destroy(m)
    S.close()
    return res


def reduce_over_ranks(ms_local, iters_local, world, dist, device):
    """Whole-job timing over the ranks: the slowest rank's time and the
    iterations all ranks did (each rank solves its own problem)."""
    if world == 1:
        return ms_local, iters_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(iters_local)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(float(u.item())))


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    steps = []
    for _ in range(min(max(args.warmup, 0), 1)):
        cpu_baseline(dict(CPU_SAMPLE, iters=1))
    for _ in range(args.steps):
        steps.append(cpu_baseline(dict(CPU_SAMPLE, iters=2)))
    vals = [s["value"] for s in steps]
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GDOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME,
                       "sample": "the benchmark problem, 2 FP64 Jacobi PCG iterations per step"},
            "cpu_baseline": {"value": v, "unit": "GDOF/s", "cores": 1, "kind": "oracle",
                             "sample": steps[-1]["sample"]},
            "e2e": {"value": v, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-problem batched leg")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-initial-guess leg")
    ap.add_argument("--no-sweep", action="store_true", help="skip the order sweep N = 5..15")
    ap.add_argument("--no-mg", action="store_true", help="skip the multigrid-preconditioner leg")
    ap.add_argument("--profile", action="store_true",
                    help="small run for ncu captures: 3 fixed mixed iterations, 2 FP32 operator calls, "
                         "1 FP64 operator call")
    ap.add_argument("--profile-mg", action="store_true",
                    help="ncu run of the multigrid preconditioner: one FP32 and one FP64 V-cycle "
                         "on the benchmark mesh inside the NVTX range mg_cycle")
    ap.add_argument("--profile-k", type=int, default=0,
                    help="with --profile: a k^3-element mesh instead of the benchmark's (smaller ncu captures)")
    ap.add_argument("--profile-sweep", type=int, default=0, metavar="N",
                    help="ncu run of the FP32 operator at order N (the order sweep's mesh, or a "
                         "k^3 mesh with --profile-k): two plain calls inside the NVTX range "
                         "bench_profile_sweep")
    ap.add_argument("--profile-variant", type=int, default=-1, metavar="V",
                    help="with --profile-sweep: run launch variant V of the staged operator instead "
                         "of the set-up autotuner's choice")
    ap.add_argument("--profile-learned", action="store_true",
                    help="ncu run of the learned guess's training: 16 pairs of the 16^3 N = 7 "
                         "problem, one epoch of batch 8192 (two steps) inside the NVTX range "
                         "bench_profile_learned; --profile-variant 0 runs the mma.sync products")
    ap.add_argument("--profile-batched", action="store_true",
                    help="ncu run of the 64-problem batch: one solve inside an NVTX range")
    ap.add_argument("--profile-batched-small", action="store_true",
                    help="as --profile-batched on 16 problems with k <= 14 (a few GB, for ncu --set full)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import paper_2503_02134_gb300 as sem

    if args.profile_learned:
        stream = torch.cuda.Stream()
        S = sem.Solver(16, 16, 16, 7, deform=True, stream=stream.cuda_stream)
        m = sem.sem_x0_create(S.h, 256, 7)
        sem.sem_x0_set_option(m, "umma", 0 if args.profile_variant == 0 else 1)
        sem.sem_x0_set_option(m, "pair_rows", 1024)
        with torch.cuda.stream(stream):
            b = torch.empty(S.L, dtype=torch.float64, device="cuda")
            x = torch.empty_like(b)
        for sample in range(16):
            sem.sem_rhs_fourier(S.h, 5, sample, b)
            S.solve(b, tol=1e-8, maxit=500, precision=sem.SEM_MIXED_FP32, precond="mg", x=x)
            sem.sem_x0_add_pair(m, b, x)
        sem.sem_x0_train(m, 1, 8192, 1e-3, seed=0)      # warm-up (first-use allocations)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("bench_profile_learned")
        loss = sem.sem_x0_train(m, 1, 8192, 1e-3, seed=1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_learned": "ok", "loss": loss}))
        sem.sem_x0_destroy(m)
        S.close()
        return 0

    if args.profile_sweep:
        import sem_inputs
        N = args.profile_sweep
        c = sem_inputs.order_sweep_case(N)
        k3 = (args.profile_k,) * 3 if args.profile_k > 0 else (c.kx, c.ky, c.kz)
        S = sem.Solver(*k3, N, deform=True)
        if args.profile_variant >= 0:
            sem.sem_set_option(S.h, "ax_variant", args.profile_variant)
        u = torch.rand(S.L, dtype=torch.float32, device="cuda",
                       generator=torch.Generator(device="cuda").manual_seed(N))
        w = torch.empty_like(u)
        sem.sem_ax_local(S.h, u, w, sem.SEM_MIXED_FP32)      # warm-up
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("bench_profile_sweep")
        for _ in range(2):
            sem.sem_ax_local(S.h, u, w, sem.SEM_MIXED_FP32)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_sweep": N, "elements": S.E,
                          "variant": int(sem.sem_get_option(S.h, "ax_variant"))}))
        S.close()
        return 0

    if args.profile_batched or args.profile_batched_small:
        import sem_inputs
        cases = (sem_inputs.batched_cases(count=16, kmax=14) if args.profile_batched_small
                 else sem_inputs.batched_cases())
        b = sem.sem_batch_setup([sem.box_mesh(k, k, k, deform=True) for k, _ in cases],
                                [N for _, N in cases])
        fs, xs = [], []
        for i in range(len(cases)):
            h = sem.sem_batch_problem(b, i)
            f = torch.empty(sem.sem_get_sizes(h).L, dtype=torch.float64, device="cuda")
            sem.sem_rhs(h, sem.RHS_UNIFORM, 1000 + i, f)
            fs.append(f)
            xs.append(torch.zeros_like(f))
        o = sem.sem_solve_opts()
        o.tol, o.maxit, o.precision = 1e-8, 5000, sem.SEM_MIXED_FP32
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("bench_profile_batched")
        sem.sem_batch_pcg_solve(b, fs, xs, o)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        sem.sem_batch_destroy(b)
        print(json.dumps({"profile_batched": "ok"}))
        return 0

    stream = torch.cuda.Stream()
    W = dict(WORKLOAD)
    if (args.profile or args.profile_mg) and args.profile_k > 0:
        W.update(kx=args.profile_k, ky=args.profile_k, kz=args.profile_k)
    S = sem.Solver(W["kx"], W["ky"], W["kz"], W["N"], deform=W["deform"], stream=stream.cuda_stream)
    L = S.L
    with torch.cuda.stream(stream):
        b = torch.empty(L, dtype=torch.float64, device="cuda")
        x = torch.empty(L, dtype=torch.float64, device="cuda")
    sem.sem_rhs(S.h, sem.RHS_UNIFORM, 0 + rank, b)
    stream.synchronize()

    def step(prec=sem.SEM_MIXED_FP32):
        _, info = S.solve(b, tol=W["tol"], maxit=5000, precision=prec, x=x)
        return info

    if args.profile_mg:
        with torch.cuda.stream(stream):
            z = torch.empty_like(b)
            b32 = b.float()
            z32 = torch.empty_like(b32)
        sem.sem_mg_apply(S.h, b, z, sem.SEM_FP64)            # set-up and warm-up
        sem.sem_mg_apply(S.h, b32, z32, sem.SEM_MIXED_FP32)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("mg_cycle")
        sem.sem_mg_apply(S.h, b32, z32, sem.SEM_MIXED_FP32)
        sem.sem_mg_apply(S.h, b, z, sem.SEM_FP64)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        S.close()
        print(json.dumps({"profile_mg": "ok"}))
        return 0

    if args.profile:
        with torch.cuda.stream(stream):
            u = torch.rand(L, dtype=torch.float32, device="cuda",
                           generator=torch.Generator(device="cuda").manual_seed(1))
            w = torch.empty_like(u)
            u64 = u.double()
            w64 = torch.empty_like(u64)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("bench_profile")
        S.solve(b, fixed_iters=3, precision=sem.SEM_MIXED_FP32, x=x, use_graph=False, chunk=3)
        for _ in range(2):
            sem.sem_ax_local(S.h, u, w, sem.SEM_MIXED_FP32)
        sem.sem_ax_local(S.h, u64, w64, sem.SEM_FP64)      # the FP64 operator, once
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        S.close()
        print(json.dumps({"profile_run": "ok"}))
        return 0

    for _ in range(max(args.warmup, 3)):
        info = step()
    # timed region
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    infos = []
    clocks = Clocks(local)
    with clocks:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("bench_timed_steps")
        ev0.record(stream)
        for _ in range(args.steps):
            infos.append(step())
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if world > 1:
            dist.barrier()
    ms_total = ev0.elapsed_time(ev1)
    iters = sum(i["iters"] for i in infos)
    ms_total, iters_all = reduce_over_ranks(ms_total, iters, world, dist, "cuda")
    ms = ms_total / args.steps
    units = L * iters_all
    value = units / (ms_total * 1e-3) / 1e9
    launches = sum(i["launches"] for i in infos)
    ok = all(i["rc"] == 0 and i["relres_true"] <= W["tol"] * 1.0000001 for i in infos)

    # FP64 time to solution on the same problem (untimed by the step loop),
    # and energy to solution of both (NVML counter around each solve)
    meter = EnergyMeter(local)
    energy = None
    if meter.ok:
        energy = {}
        for name, prec in (("fp64", sem.SEM_FP64), ("mixed", sem.SEM_MIXED_FP32)):
            torch.cuda.synchronize()
            j0 = meter.read()
            inf_e = step(prec)
            torch.cuda.synchronize()
            j1 = meter.read()
            energy[name] = {"joules": j1 - j0, "solve_ms": inf_e["solve_ms"]}
        energy["gain"] = energy["fp64"]["joules"] / max(energy["mixed"]["joules"], 1e-9)
        energy["note"] = "whole-GPU counter, includes idle and host-poll time"
    info64 = step(sem.SEM_FP64)
    info_mixed = infos[-1]

    # exactly 100 iterations without a convergence test: time per iteration
    def per_iter(prec, reps=2):
        best = None
        for _ in range(reps):
            _, inf = S.solve(b, fixed_iters=100, precision=prec, x=x)
            best = inf["solve_ms"] if best is None else min(best, inf["solve_ms"])
        return best / 100.0
    fixed = {"fp64_ms_per_iter": per_iter(sem.SEM_FP64),
             "mixed_ms_per_iter": per_iter(sem.SEM_MIXED_FP32)}
    fixed["speedup"] = fixed["fp64_ms_per_iter"] / fixed["mixed_ms_per_iter"]

    # accuracy of the mixed solve against the FP64 one: AE_k = | ||r_m,k|| -
    # ||r_d,k|| | per iteration (relative residual norms), MAE = mean |x_m - x_d|
    # over the unique interior nodes (c-weighted local mean)
    with torch.cuda.stream(stream):
        xm = torch.empty_like(b)
        xd = torch.empty_like(b)
    _, hm = S.solve(b, tol=W["tol"], maxit=5000, precision=sem.SEM_MIXED_FP32, x=xm, history=True)
    _, hd = S.solve(b, tol=W["tol"], maxit=5000, precision=sem.SEM_FP64, x=xd, history=True)
    cw = S.field(sem.FIELD_C)
    torch.cuda.synchronize()
    k = min(len(hm["history"]), len(hd["history"]))
    ae = np.abs(np.asarray(hm["history"][:k]) - np.asarray(hd["history"][:k]))
    mae = float((cw * (xm - xd).abs()).sum() / cw.sum())
    accuracy = {"ae_max": float(ae.max()), "ae_last_common": float(ae[-1]), "iterations_compared": k,
                "mae": mae, "max_abs_x_fp64": float(xd.abs().max()),
                "definition": "AE_k on relative residual norms, MAE c-weighted over unique nodes"}

    # operator throughput and the roofline of the FP32 element operator, timed
    # with CUDA events on the stream the library launches on
    def time_ax(prec, reps=20, local_only=True):
        dt = torch.float64 if prec == sem.SEM_FP64 else torch.float32
        with torch.cuda.stream(stream):
            u = torch.rand(L, dtype=dt, device="cuda",
                           generator=torch.Generator(device="cuda").manual_seed(2))
            w = torch.empty_like(u)
        fn = sem.sem_ax_local if local_only else sem.sem_ax
        for _ in range(3):
            fn(S.h, u, w, prec)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn(S.h, u, w, prec)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ax32_ms = time_ax(sem.SEM_MIXED_FP32)
    ax32_full_ms = time_ax(sem.SEM_MIXED_FP32, local_only=False)
    ax64_ms = time_ax(sem.SEM_FP64, reps=5)
    hbm, peak_kind = peaks()
    peak_source = (f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
                   else "fallback 6.8 TB/s")

    # per-kernel device times inside a mixed solve: the library records CUDA
    # events on its own stream around each launch of every iteration (graphs
    # off for this one untimed solve)
    sem.sem_set_option(S.h, "kernel_timing", 1)
    info_kt = step()
    kt = {k: sem.sem_get_option(S.h, k) for k in ("kt_iters", "kt_ms_ax", "kt_ms_gs", "kt_ms_update")}
    sem.sem_set_option(S.h, "kernel_timing", 0)
    it_step = info_mixed["iters"]
    shares = {name: kt[key] * it_step / ms for name, key in
              (("operator_pcg", "kt_ms_ax"), ("gather_scatter", "kt_ms_gs"), ("update", "kt_ms_update"))}

    # dominant kernel of the step: the PCG-mode FP32 operator (Jacobi +
    # p update prologue, Dot2 p.w epilogue)
    bytes_pcg = 44.0   # read r, J^-1, p_old, 6 G; write p, w (FP32)
    ax_pcg_ms = kt["kt_ms_ax"]
    ach = L * bytes_pcg / (ax_pcg_ms * 1e-3) / 1e9 if ax_pcg_ms > 0 else 0.0
    traffic = TRAFFIC.get("operator_pcg")
    roofline = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": traffic * L if traffic else None,
                "kernel": f"ax_tma_kernel<{W['N'] + 1},true> (FP32 operator, PCG mode)",
                "algorithmic_bytes_per_launch": L * bytes_pcg, "launch_ms": ax_pcg_ms,
                "timing": "CUDA events on the library stream around every launch of one mixed solve",
                "iterations_timed": kt["kt_iters"], "peak_source": peak_source}
    bytes_plain = 32.0   # FP32: read u + 6 G, write w
    ach_plain = L * bytes_plain / (ax32_ms * 1e-3) / 1e9
    traffic_plain = TRAFFIC.get("operator_plain")
    roofline_plain = {"bound": "hbm", "achieved": ach_plain, "peak": hbm, "unit": "GB/s",
                      "frac": ach_plain / hbm,
                      "traffic": traffic_plain * L if traffic_plain else None,
                      "kernel": f"ax_tma_kernel<{W['N'] + 1},false> (sem_ax_local, FP32 operator)",
                      "algorithmic_bytes_per_launch": L * bytes_plain, "launch_ms": ax32_ms,
                      "peak_source": peak_source}

    # the FP64 operator is bound by the FP64 pipe: 12 n^4 + 15 n^3 flop per
    # element (three derivative and three transposed contractions, the
    # symmetric 3x3 geometric product)
    n_gll = W["N"] + 1
    flops64 = S.E * (12 * n_gll ** 4 + 15 * n_gll ** 3)
    ach64 = flops64 / (ax64_ms * 1e-3) / 1e12
    fma = fma_peaks(sem)
    peak64 = fma["fp64_tflops"]
    nominal64, nominal64_how = fp64_peak(torch.cuda.get_device_properties(0).multi_processor_count)
    traffic64 = TRAFFIC.get("operator_fp64")
    roofline_fp64 = {"bound": "alu", "achieved": ach64, "peak": peak64, "unit": "TFLOP/s",
                     "frac": ach64 / peak64, "traffic": traffic64 * L if traffic64 else None,
                     "kernel": f"ax_kernel<{n_gll},double> (sem_ax_local, FP64 operator)",
                     "algorithmic_flops_per_launch": flops64, "launch_ms": ax64_ms,
                     "peak_source": "measured: " + fma["method"],
                     "nominal_peak": nominal64, "nominal_peak_source": nominal64_how}

    # end to end through the C-ABI with host (pinned) buffers
    fh = torch.empty(L, dtype=torch.float64, pin_memory=True)
    fh.copy_(b.cpu())
    xh = torch.empty(L, dtype=torch.float64, pin_memory=True)
    e2e_t, e2e_it = [], 0
    for _ in range(2):
        t0 = time.perf_counter()
        rc, inf = sem.sem_pcg_solve(S.h, fh, None, xh, W["tol"], 5000, sem.SEM_MIXED_FP32)
        e2e_t.append(time.perf_counter() - t0)
        e2e_it = inf.iters
    e2e_s = min(e2e_t)
    e2e = {"value": L * e2e_it * world / e2e_s / 1e9, "unit": "GDOF/s",
           "h2d_bytes_per_step": 8 * L, "d2h_bytes_per_step": 8 * L,
           "time_to_solution_ms": e2e_s * 1e3}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "elements": S.E, "N": S.N, "local_dofs": L,
                       "unique_dofs": S.U, "tol": W["tol"], "rhs": W["rhs"],
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (G alone is 403 MB FP32)"},
            "time_to_solution_ms": ms, "iterations": info_mixed["iters"],
            "refinements": info_mixed["refinements"], "relres_true": info_mixed["relres_true"],
            "converged": ok,
            "fp64": {"time_to_solution_ms": info64["solve_ms"], "iterations": info64["iters"],
                     "relres_true": info64["relres_true"]},
            "speedup_vs_fp64": info64["solve_ms"] / ms,
            "energy_to_solution": energy,
            "fixed_100_iterations": fixed,
            "accuracy_mixed_vs_fp64": accuracy,
            "ax_gdofs_fp32": L / (ax32_ms * 1e-3) / 1e9,
            "ax_gdofs_fp32_with_gs": L / (ax32_full_ms * 1e-3) / 1e9,
            "ax_gdofs_fp64": L / (ax64_ms * 1e-3) / 1e9,
            "roofline": roofline, "roofline_operator_plain": roofline_plain,
            "roofline_operator_fp64": roofline_fp64, "fma_peaks_measured": fma,
            "kernel_ms": {"operator_pcg": kt["kt_ms_ax"], "gather_scatter": kt["kt_ms_gs"],
                          "update": kt["kt_ms_update"]},
            "kernel_share_of_step": shares,
            "clocks": clocks.summary(), "e2e": e2e,
            "autotune": {k: sem.sem_get_option(S.h, k) for k in
                         ("ax_variant", "ax_variant_pcg", "ax_tune_ms_plain_0", "ax_tune_ms_plain_1",
                          "ax_tune_ms_plain_2", "ax_tune_ms_plain_3", "ax_tune_ms_pcg_0",
                          "ax_tune_ms_pcg_1", "ax_tune_ms_pcg_2", "ax_tune_ms_pcg_3")},
            "gpu_launches": launches,
        }
        if not args.no_mg:
            line["multigrid"] = mg_leg(sem, torch, S, b, stream)
        if not args.no_batched:
            line["batched"] = batched_leg(sem, torch)
        if not args.no_learned:
            line["learned_x0"] = learned_leg(sem, torch)
        if not args.no_sweep:
            line["order_sweep"] = order_sweep_leg(sem, torch, hbm, peak64)
        if not args.no_cpu and world >= 1:
            line["cpu_baseline"] = cpu_baseline()
            cb = line["cpu_baseline"]
            line["cpu_oracle_legs"] = cpu_legs()
            line["cpu_oracle_legs"]["config2_per_iteration_ms_1core"] = L / (cb["value"] * 1e9) * 1e3
        print(json.dumps(line))
    S.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
