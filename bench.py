#!/usr/bin/env python
"""Benchmark: AL-multigrid Stokes solves on one GB300 (mixed precision vs FP64).

One step = setup for the step's coefficients (vertex-star patch assembly and
FP64 factorisation on every level, coarse Cholesky, Schur blocks) followed by
an FGMRES solve of the augmented Stokes system to a 1e-8 relative residual,
preconditioned by the block-LDU preconditioner with a robust multigrid
V-cycle for A_gamma.  Default workload: the 3D multi-sinker problem on 32^3
hexes ([Q2]^3 x P1disc, 4 levels, 16 sinkers, DR = 1e8).

Printed JSON (one line, rank 0):
  value       solve DoF/s of the mixed path, inputs resident in HBM
              (free velocity + pressure DoFs per step / step time, all ranks)
  e2e         the same through the C ABI with host buffers (coefficients and
              force copied in, solution copied out inside the timed region)
  roofline    dominant kernel (finest-level vertex-star patch kernel): bytes
              per launch / CUDA-event launch time, measured during the timed steps
  cpu_baseline the FP64 oracle on a bounded sample of the same workload
Multi-GPU (torchrun): every rank solves its own replica (no communication on
the data path); the timed region is bracketed by barriers and the max over
ranks is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

# A batch runs its instances' FGMRES kernels on one stream per instance and its merged
# cycles on one stream per group; with the default 8 hardware work queues those streams
# share queues and wait behind one another's event waits.  Set before CUDA starts.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # 3D multi-sinker, 32^3 hexes, 4 levels (coarse 4^3), 16 sinkers, omega 0.15, delta 200, DR 1e8
    "sinker3d_32": dict(d=3, n=32, levels=4, count=16, omega=0.15, delta=200.0, dr=1e8, beta=10.0,
                        gamma=10.0, seed=0, sweeps=5),
    # the same 3D problem at the large gamma the AL method is built for, gamma 1e4, with the
    # P2 pairing (W = M_p(1/mu)): mixed mode refuses P1 there (2^-24 gamma / mu_min = 6e4)
    "sinker3d_32_g1e4": dict(d=3, n=32, levels=4, count=16, omega=0.15, delta=200.0, dr=1e8, beta=10.0,
                             gamma=1e4, seed=0, sweeps=5, schur="P2"),
    # 2D multi-sinker, 128^2 quads, 5 levels (coarse 8^2), 8 sinkers, omega 0.1, delta 200, DR 1e6;
    # gamma 1e2 of the set {1, 1e2, 1e4}: with the P1 pairing the FP32 cycle holds while
    # eps32 gamma / mu_min stays below about 0.1, and mu_min = 1e-3 here (1e4 would give 0.6)
    "sinker2d_128": dict(d=2, n=128, levels=5, count=8, omega=0.1, delta=200.0, dr=1e6, beta=10.0,
                         gamma=1e2, seed=0, sweeps=5),
    # 2D multi-sinker with the order-3 discretisation of Table k ([Q3]^2 x P2disc), 128^2 quads
    # (394,754 velocity + pressure DoFs: the size of Table exacttopleft), 5 levels, 8 sinkers,
    # DR 1e6, gamma 1e2, P1 pairing
    "sinker2d_q3_128": dict(d=2, n=128, levels=5, count=8, omega=0.1, delta=200.0, dr=1e6, beta=10.0,
                            gamma=1e2, seed=0, sweeps=5, order=3),
    # 3D multi-sinker with [Q3]^3 x P2disc, the element of the 3D runs of Table linear: 24^3
    # hexes (1,167,051 velocity + 138,240 pressure DoFs), 4 levels (coarse 3^3), 24 sinkers,
    # DR 1e8, gamma 1e3, P2 pairing (mixed mode refuses P1 there: 2^-24 gamma / mu_min = 0.6)
    "sinker3d_q3_24": dict(d=3, n=24, levels=4, count=24, omega=0.1, delta=200.0, dr=1e8, beta=10.0,
                           gamma=1e3, seed=0, sweeps=5, order=3, schur="P2"),
    # 3D anisotropic viscoplastic linearisation, 48^3 hexes, 4 levels (coarse 6^3): per-point
    # 4th-order tensor C (21 Mandel entries), mu_eff contrast ~1e10, gamma 1e3, P2 Schur pairing
    "viscoplastic3d_48": dict(kind="tensor", d=3, n=48, levels=4, gamma=1e3, seed=0, sweeps=5, schur="P2"),
}
# bounded samples of the same law for the oracle (CPU baseline / reference arm)
SAMPLES = {
    "sinker3d_32": dict(cpu_baseline=dict(n=12, levels=2), reference=dict(n=8, levels=3)),
    "sinker2d_128": dict(cpu_baseline=dict(n=64, levels=4), reference=dict(n=32, levels=3)),
    "sinker3d_32_g1e4": dict(cpu_baseline=dict(n=12, levels=2), reference=dict(n=8, levels=3)),
    "sinker2d_q3_128": dict(cpu_baseline=dict(n=32, levels=3), reference=dict(n=16, levels=3)),
    "sinker3d_q3_24": dict(cpu_baseline=dict(n=4, levels=2), reference=dict(n=4, levels=2)),
    "viscoplastic3d_48": dict(cpu_baseline=dict(n=8, levels=2), reference=dict(n=8, levels=2)),
}
RTOL = 1e-8
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def make_problem(spec, n=None, levels=None):
    from synthetic.problems import sinker_problem, sinker_problem_k, viscoplastic_problem
    if spec.get("order", 2) == 3:
        return sinker_problem_k(n or spec["n"], levels or spec["levels"], 3, spec["count"], spec["omega"],
                                spec["delta"], spec["dr"], spec["beta"], spec["gamma"], spec["seed"], d=spec["d"])
    if spec.get("kind") == "tensor":
        return viscoplastic_problem(spec["d"], n or spec["n"], levels or spec["levels"], spec["gamma"], spec["seed"])
    return sinker_problem(spec["d"], n or spec["n"], levels or spec["levels"], spec["count"], spec["omega"],
                          spec["delta"], spec["dr"], spec["beta"], spec["gamma"], spec["seed"])


def problem_dofs(pb):
    """Free velocity DoFs + pressure DoFs of the finest level."""
    k = pb.meta.get("order", 2)
    free_nodes = math.prod(k * v - 1 for v in pb.n)
    return pb.d * free_nodes + pressure_per_cell(pb.d, k) * math.prod(pb.n)


def pressure_per_cell(d, k):
    """Dimension of P_(k-1)^disc on a cell: C(k - 1 + d, d)."""
    return math.comb(k - 1 + d, d)


# --------------------------------------------------------------------------
# distributed plumbing (replicas only)
# --------------------------------------------------------------------------
class Dist:
    def __init__(self, gpus):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            backend = "nccl" if self._cuda() else "gloo"
            if backend == "nccl":
                import torch
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    @staticmethod
    def _cuda():
        try:
            import torch
            return torch.cuda.is_available()
        except Exception:
            return False

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v):
        if not self.pg:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device="cuda" if self._cuda() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


class ClockSampler:
    """nvidia-smi samples during the timed region (read only)."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
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
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBps", "hbm"):
                if k in d:
                    v = d[k]
                    return float(v["value"] if isinstance(v, dict) else v), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


def stored_traffic(kernel, workload):
    """Per-launch DRAM traffic from the committed ncu summary (profiles/traffic.txt),
    if it was taken on the current source of the kernel; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) != 5 or line.startswith("#") or parts[0] != kernel or parts[1] != workload:
            continue
        try:
            src = open(os.path.join(ROOT, parts[2]), "rb").read()
        except OSError:
            return None
        if hashlib.sha256(src).hexdigest()[:16] != parts[3]:
            return None
        return float(parts[4])
    return None


# --------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# --------------------------------------------------------------------------
def oracle_sample_step(spec, n, levels):
    import warnings
    warnings.simplefilter("ignore")
    from oracle.mg import Hierarchy
    from oracle.stokes import StokesSolver
    pb = make_problem(spec, n, levels)
    t0 = time.perf_counter()
    p2 = spec.get("schur") == "P2"
    if spec.get("order", 2) == 3:
        from oracle.qk import HierarchyK
        H = HierarchyK(pb.d, pb.n, 3, pb.mu, pb.gamma, steps=spec["sweeps"], W="Mp_mu" if p2 else "Mp")
    else:
        H = Hierarchy(pb.d, pb.n, pb.mu, pb.gamma, steps=spec["sweeps"], kind=spec.get("kind", "scalar"),
                      mu_eff=pb.meta.get("mu_eff"), W="Mp_mu" if p2 else "Mp")
    u, p, its, _ = StokesSolver(H, schur="P2" if p2 else "P1").solve(pb.f, pb.u_bc, rtol=RTOL)
    dt = time.perf_counter() - t0
    return problem_dofs(pb), dt, its


def cpu_worker(args):
    """Runs in a fresh single-threaded interpreter; prints one JSON line."""
    spec = WORKLOADS[args.workload]
    smp = SAMPLES[args.workload][args.sample_kind]
    out = []
    for _ in range(args.reps):
        dof, dt, its = oracle_sample_step(spec, smp["n"], smp["levels"])
        out.append((dof, dt, its))
    print(json.dumps({"runs": out}))


def host_cpu():
    """(logical cores, CPU model) of this host, read only."""
    cores = os.cpu_count() or 1
    model = "unknown"
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model == "unknown":
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:  # noqa: BLE001
            pass
    return cores, model


def run_oracle_subprocess(workload, kind, reps, threads=1):
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t,
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", "--workload", workload,
                        "--sample-kind", kind, "--reps", str(reps)], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])["runs"]


def cpu_baseline(workload):
    """The oracle on a bounded sample, on one thread and with BLAS on every core of the
    host (SciPy's sparse products stay single-threaded either way)."""
    smp = SAMPLES[workload]["cpu_baseline"]
    spec = WORKLOADS[workload]
    cores, model = host_cpu()
    dof, dt, its = run_oracle_subprocess(workload, "cpu_baseline", 1)[0]
    dof_a, dt_a, _ = run_oracle_subprocess(workload, "cpu_baseline", 1, threads=cores)[0]
    return {"value": dof / dt, "unit": "DoF/s", "cores": 1, "kind": "oracle",
            "sample": f"same law, {spec['d']}D {smp['n']}^{spec['d']} cells, {smp['levels']} levels, "
                      f"setup+solve to {RTOL:g} ({its} FGMRES its, {dt:.1f} s, {dof} DoFs), FP64 NumPy/SciPy, "
                      f"1 thread",
            "all_cores": {"value": dof_a / dt_a, "cores": cores, "s": dt_a,
                          "note": "BLAS threads = all cores; SciPy sparse products are single-threaded"},
            "host": {"logical_cores": cores, "cpu_model": model}}


def reference_arm(args, dist):
    """The oracle as it stands, on the host cores: each step one bounded sample."""
    if dist.rank != 0:
        return
    spec = WORKLOADS[args.workload]
    smp = SAMPLES[args.workload]["reference"]
    runs = run_oracle_subprocess(args.workload, "reference", args.warmup + args.steps)[args.warmup:]
    t = sum(r[1] for r in runs)
    dof = runs[0][0]
    value = dof * len(runs) / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(runs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "sample": f"{spec['d']}D {smp['n']}^{spec['d']}, "
                       f"{smp['levels']} levels, same law", "rtol": RTOL},
            "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": 1, "kind": "oracle",
                             "sample": f"{spec['d']}D {smp['n']}^{spec['d']} cells, {smp['levels']} levels"},
            "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "iterations": runs[0][2]}
    print(json.dumps(line))


METRIC = "AL-MG V-cycles/s & solve DoF/s to 1e-8 rel. residual, mixed vs FP64, 1xGB300"


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
# flops per cell of the sum-factorised A_gamma apply (scalar mu): forward
# gradients, point-wise stress and AL projection, transposed contractions
APPLY_FLOPS_PER_CELL = {2: 1100, 3: 8000}
# order 3 (scalar mu), as the kernels compute it: 2D, products over the 16 x 16 point-node
# pairs (gradient 1,024 + transposed 1,024 FMAs, pressure 228 FMAs, stress ~190 flops);
# 3D, sum-factorised (contractions 6,144 forward + 6,144 transposed FMAs, pressure 1,380
# FMAs, stress ~2,900 flops)
APPLY_FLOPS_PER_CELL_Q3 = {2: 4700, 3: 30200}


def ours(args, dist):
    import numpy as np
    import torch

    from paper_2107_00820_gb300 import Context, alstokes as A

    torch.cuda.set_device(dist.local)
    spec = WORKLOADS[args.workload]
    pb = make_problem(spec)
    dofs = problem_dofs(pb)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")  # noqa: E731
    mu_d = [dev(m) for m in pb.mu]
    tensor = spec.get("kind") == "tensor"
    mue_d = [dev(m) for m in pb.meta["mu_eff"]] if tensor else None
    schur = A.ALS_SCHUR_P2 if spec.get("schur") == "P2" else A.ALS_SCHUR_P1
    f_d, ubc_d = dev(pb.f), dev(pb.u_bc)
    order = spec.get("order", 2)
    nu = pb.d * math.prod(order * v + 1 for v in pb.n)
    npres = pressure_per_cell(pb.d, order) * math.prod(pb.n)
    u_d = torch.zeros(nu, dtype=torch.float64, device="cuda")
    p_d = torch.zeros(npres, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    ctx = Context(pb.d, pb.n, pb.levels, mu_d, pb.gamma, mu_eff=mue_d, stream=stream, mode=A.ALS_MODE_MIXED,
                  rtol=RTOL, maxit=200, sweeps=spec["sweeps"], schur=schur, order=order)

    def step():
        ctx.update_coefficients(mu_d, mue_d)
        return ctx.solve(f_d, ubc_d, None, u_d, p_d)[2]

    for _ in range(args.warmup):
        info = step()
    ctx.profile(True)
    step()                                  # capture the profiled V-cycle graph outside the timed region
    ctx.profile_read()
    clocks = ClockSampler(dist.local)
    clocks.start()
    launches0 = A.als_kernel_launches()
    dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    its = []
    for _ in range(args.steps):
        info = step()
        its.append(info.iterations)
    e1.record()
    torch.cuda.synchronize()
    dist.barrier()
    launches = A.als_kernel_launches() - launches0
    clk = clocks.stop()
    k4_ms, k4_n = ctx.profile_read()
    k1_ms, k1_n = ctx.profile_read_kernel(1)
    ctx.profile(False)

    # phases of one step: setup alone, solve alone (CUDA events on the stream); the
    # first solve after profiling recaptures the V-cycle graphs and is not timed
    ctx.solve(f_d, ubc_d, None, u_d, p_d)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    for _ in range(3):
        ctx.update_coefficients(mu_d, mue_d)
    p1.record()
    torch.cuda.synchronize()
    t_setup = p0.elapsed_time(p1) / 3 / 1e3
    solves = []
    for _ in range(3):
        p0.record()
        info_s = ctx.solve(f_d, ubc_d, None, u_d, p_d)[2]
        p1.record()
        torch.cuda.synchronize()
        solves.append(p0.elapsed_time(p1) / 1e3)
    t_solve = sorted(solves)[1]   # median of three
    fp32_peak, fp64_peak = A.als_measure_fma_peaks(stream)
    t_step = dist.max(e0.elapsed_time(e1) / args.steps) / 1e3
    value = dist.world * dofs / t_step

    # V-cycles/s of the mixed (FP32) cycle, replayed back to back
    b32 = torch.randn(nu, dtype=torch.float32, device="cuda")
    x32 = torch.zeros_like(b32)
    for _ in range(3):
        ctx.vcycle(b32, x32, A.ALS_PREC_FP32)
    torch.cuda.synchronize()
    nv = 20
    e0.record()
    for _ in range(nv):
        ctx.vcycle(b32, x32, A.ALS_PREC_FP32)
    e1.record()
    torch.cuda.synchronize()
    vcyc_s = nv / (e0.elapsed_time(e1) / 1e3)
    b64, x64 = b32.double(), torch.zeros(nu, dtype=torch.float64, device="cuda")
    ctx.vcycle(b64, x64, A.ALS_PREC_FP64)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(3):
        ctx.vcycle(b64, x64, A.ALS_PREC_FP64)
    e1.record()
    torch.cuda.synchronize()
    vcyc64_s = 3 / (e0.elapsed_time(e1) / 1e3)

    # all-FP64 GPU path on the same problem
    ctx64 = Context(pb.d, pb.n, pb.levels, mu_d, pb.gamma, mu_eff=mue_d, stream=stream, mode=A.ALS_MODE_FP64,
                    rtol=RTOL, maxit=200, sweeps=spec["sweeps"], schur=schur, order=order)
    u64 = torch.zeros_like(u_d)
    p64 = torch.zeros_like(p_d)
    ctx64.solve(f_d, ubc_d, None, u64, p64)
    torch.cuda.synchronize()
    e0.record()
    ctx64.update_coefficients(mu_d, mue_d)
    info64 = ctx64.solve(f_d, ubc_d, None, u64, p64)[2]
    e1.record()
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1) / 1e3
    e0.record()
    ctx64.solve(f_d, ubc_d, None, u64, p64)
    e1.record()
    torch.cuda.synchronize()
    t64_solve = e0.elapsed_time(e1) / 1e3
    err_u = float(torch.linalg.norm(u_d - u64) / torch.linalg.norm(u64))
    err_p = float(torch.linalg.norm(p_d - p64) / torch.linalg.norm(p64))
    ctx64.close()

    # the same mixed step with the patch and coarse inverses computed in FP64 instead of
    # double-float (options.setup = ALS_SETUP_FP64): setup time, iterations, solution
    # difference from the double-float setup's solution
    setup_fp64 = None
    if not args.quick and (order == 2 or pb.d == 3):   # 2D order 3 sets up in FP64 in both modes
        ctxf = Context(pb.d, pb.n, pb.levels, mu_d, pb.gamma, mu_eff=mue_d, stream=stream, mode=A.ALS_MODE_MIXED,
                       rtol=RTOL, maxit=200, sweeps=spec["sweeps"], schur=schur, setup=A.ALS_SETUP_FP64,
                       order=order)
        uf, pf = torch.zeros_like(u_d), torch.zeros_like(p_d)
        ctxf.solve(f_d, ubc_d, None, uf, pf)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(2):
            ctxf.update_coefficients(mu_d, mue_d)
        e1.record()
        torch.cuda.synchronize()
        t_setf = e0.elapsed_time(e1) / 2 / 1e3
        e0.record()
        info_f = ctxf.solve(f_d, ubc_d, None, uf, pf)[2]
        e1.record()
        torch.cuda.synchronize()
        setup_fp64 = {"setup_ms": t_setf * 1e3, "setup_ms_double_float": t_setup * 1e3,
                      "solve_ms": e0.elapsed_time(e1), "iterations": info_f.iterations,
                      "iterations_double_float": info_s.iterations,
                      "rel_diff_vs_double_float": {
                          "u": float(torch.linalg.norm(uf - u_d) / torch.linalg.norm(u_d)),
                          "p": float(torch.linalg.norm(pf - p_d) / torch.linalg.norm(p_d))}}
        ctxf.close()

    # the AL method at large gamma: the same workload at gamma 1e4 with the P2 pairing
    # (W = M_p(1/mu); mixed mode refuses P1 there), mixed against FP64: step time,
    # iterations, solution difference at rtol 1e-8, and the mixed solve run on to 1e-11
    # against the FP64 solve run to 1e-12 (the 1e-7 error bar)
    gamma_large = None
    if not tensor and not args.quick and order == 2:
        spec4 = dict(spec, gamma=1e4)
        pb4 = make_problem(spec4)
        mu4 = [dev(m) for m in pb4.mu]
        f4, ub4 = dev(pb4.f), dev(pb4.u_bc)
        res = {}
        for name, mode, rtol in (("mixed", A.ALS_MODE_MIXED, RTOL), ("fp64", A.ALS_MODE_FP64, RTOL),
                                 ("mixed_1e-11", A.ALS_MODE_MIXED, 1e-11), ("fp64_1e-12", A.ALS_MODE_FP64, 1e-12)):
            c4 = Context(pb4.d, pb4.n, pb4.levels, mu4, pb4.gamma, stream=stream, mode=mode, rtol=rtol, maxit=300,
                         sweeps=spec["sweeps"], schur=A.ALS_SCHUR_P2)
            u4, p4 = torch.zeros_like(u_d), torch.zeros_like(p_d)
            c4.solve(f4, ub4, None, u4, p4)
            torch.cuda.synchronize()
            e0.record()
            c4.update_coefficients(mu4)
            inf4 = c4.solve(f4, ub4, None, u4, p4)[2]
            e1.record()
            torch.cuda.synchronize()
            res[name] = (e0.elapsed_time(e1) / 1e3, inf4, u4, p4)
            c4.close()
        rd = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))  # noqa: E731
        gamma_large = {
            "gamma": 1e4, "schur": "P2", "value": dofs / res["mixed"][0], "unit": "DoF/s",
            "ms_per_step": res["mixed"][0] * 1e3, "iterations": res["mixed"][1].iterations,
            "fp64": {"solve_dof_per_s": dofs / res["fp64"][0], "ms_per_step": res["fp64"][0] * 1e3,
                     "iterations": res["fp64"][1].iterations},
            "mixed_vs_fp64_speedup": res["fp64"][0] / res["mixed"][0],
            "mixed_vs_fp64_rel_err": {"u": rd(res["mixed"][2], res["fp64"][2]), "p": rd(res["mixed"][3], res["fp64"][3])},
            "mixed_1e-11_vs_fp64_1e-12_rel_err": {"u": rd(res["mixed_1e-11"][2], res["fp64_1e-12"][2]),
                                                  "p": rd(res["mixed_1e-11"][3], res["fp64_1e-12"][3]),
                                                  "iterations": res["mixed_1e-11"][1].iterations}}

    # the optional bfloat16 storage of the FP32 cycle's star inverses (options.store) on the
    # same mesh at mild contrast (DR 1e4, gamma 10) with the P2 pairing, where it keeps the
    # FGMRES count (at the workload's DR 1e8 it does not converge, with either pairing):
    # solve time and iterations, FP32 V-cycles/s and the finest-level interior-star
    # kernel's live time, FP32 against bfloat16 storage
    # order 3: the same mixed step with the F-cycle, the cycle of the paper's 3D runs (Table
    # linear): iterations, solve time, FP32 F-cycles/s
    fcycle = None
    if not args.quick and order == 3:
        ctxc = Context(pb.d, pb.n, pb.levels, mu_d, pb.gamma, stream=stream, mode=A.ALS_MODE_MIXED,
                       rtol=RTOL, maxit=200, sweeps=spec["sweeps"], schur=schur, order=order, cycle=A.ALS_CYCLE_F)
        uc, pc = torch.zeros_like(u_d), torch.zeros_like(p_d)
        ctxc.solve(f_d, ubc_d, None, uc, pc)
        torch.cuda.synchronize()
        e0.record()
        info_c = ctxc.solve(f_d, ubc_d, None, uc, pc)[2]
        e1.record()
        torch.cuda.synchronize()
        t_fc = e0.elapsed_time(e1) / 1e3
        for _ in range(3):
            ctxc.vcycle(b32, x32, A.ALS_PREC_FP32)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(10):
            ctxc.vcycle(b32, x32, A.ALS_PREC_FP32)
        e1.record()
        torch.cuda.synchronize()
        fcycle = {"iterations": info_c.iterations, "converged": bool(info_c.converged), "solve_ms": t_fc * 1e3,
                  "fcycles_per_s": 10 / (e0.elapsed_time(e1) / 1e3),
                  "rel_diff_vs_vcycle": {"u": float(torch.linalg.norm(uc - u_d) / torch.linalg.norm(u_d)),
                                         "p": float(torch.linalg.norm(pc - p_d) / torch.linalg.norm(p_d))}}
        ctxc.close()

    bf16_storage = None
    if not tensor and not args.quick and (order == 2 or pb.d == 3):   # not built for order 3 in 2D
        specm = dict(spec, dr=1e4)
        pbm = make_problem(specm)
        mum = [dev(m) for m in pbm.mu]
        fm, ubm = dev(pbm.f), dev(pbm.u_bc)
        res = {}
        for name, store in (("fp32", A.ALS_STORE_FP32), ("bf16", A.ALS_STORE_BF16)):
            cm = Context(pbm.d, pbm.n, pbm.levels, mum, pbm.gamma, stream=stream, mode=A.ALS_MODE_MIXED, rtol=RTOL,
                         maxit=300, sweeps=spec["sweeps"], schur=A.ALS_SCHUR_P2, store=store, order=order)
            um, pm = torch.zeros_like(u_d), torch.zeros_like(p_d)
            cm.solve(fm, ubm, None, um, pm, check=False)
            torch.cuda.synchronize()
            e0.record()
            infm = cm.solve(fm, ubm, None, um, pm, check=False)[2]
            e1.record()
            torch.cuda.synchronize()
            t_sol = e0.elapsed_time(e1) / 1e3
            for _ in range(3):
                cm.vcycle(b32, x32, A.ALS_PREC_FP32)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(nv):
                cm.vcycle(b32, x32, A.ALS_PREC_FP32)
            e1.record()
            torch.cuda.synchronize()
            vc = nv / (e0.elapsed_time(e1) / 1e3)
            cm.profile(True)
            cm.vcycle(b32, x32, A.ALS_PREC_FP32)      # captures the timed graph
            torch.cuda.synchronize()
            cm.profile_read_kernel(0)
            for _ in range(16):
                cm.vcycle(b32, x32, A.ALS_PREC_FP32)
            torch.cuda.synchronize()
            k_ms, k_n = cm.profile_read_kernel(0)
            cm.profile(False)
            res[name] = {"solve_ms": t_sol * 1e3, "iterations": infm.iterations, "converged": bool(infm.converged),
                         "vcycles_per_s": vc, "star_kernel_us": 1e3 * k_ms / max(k_n, 1)}
            cm.close()
        bf16_storage = {"dr": specm.get("dr"), "gamma": pbm.gamma, "schur": "P2", **res,
                        "star_kernel_speedup": res["fp32"]["star_kernel_us"] / res["bf16"]["star_kernel_us"],
                        "vcycle_speedup": res["bf16"]["vcycles_per_s"] / res["fp32"]["vcycles_per_s"]}

    # end to end through the C ABI with host buffers
    mu_h = [np.ascontiguousarray(m) for m in pb.mu]
    mue_h = [np.ascontiguousarray(m) for m in pb.meta["mu_eff"]] if tensor else None
    f_h = np.ascontiguousarray(pb.f)
    ubc_h = np.ascontiguousarray(pb.u_bc)
    u_h = np.zeros(nu)
    p_h = np.zeros(npres)
    h2d = sum(m.nbytes for m in mu_h) + (sum(m.nbytes for m in mue_h) if tensor else 0) + f_h.nbytes + ubc_h.nbytes
    d2h = u_h.nbytes + p_h.nbytes
    ctx.update_coefficients(mu_h, mue_h)
    ctx.solve(f_h, ubc_h, None, u_h, p_h)
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record()
    for _ in range(args.steps):
        ctx.update_coefficients(mu_h, mue_h)
        ctx.solve(f_h, ubc_h, None, u_h, p_h)
    e1.record()
    torch.cuda.synchronize()
    t_e2e = dist.max(max(e0.elapsed_time(e1) / 1e3, time.perf_counter() - t0) / args.steps)
    ctx.close()

    # roofline of the dominant kernel: the finest-level interior-star patch kernel (the
    # boundary stars, with 1/3 .. 1/27 of the dofs, run in their own small kernel): per
    # interior vertex its packed FP32 inverse and its output row, plus r read once
    F = pb.n
    nverts = math.prod(v + 1 for v in F)
    # split star storage on levels of >= 32768 vertices at order 2 (interior stars only in the
    # interior-star kernel); order 3 streams every star's packed inverse in its one star kernel
    nint = math.prod(v - 1 for v in F) if (order == 2 and nverts >= 32768) else nverts
    npatch = pb.d * (2 * order - 1) ** pb.d
    packed = npatch * (npatch + 1) // 2
    if order == 2:
        bytes_per_launch = nint * (packed * 4 + npatch * 4) + nu * 4
    else:
        # order 3 times the star products and their node gather together: packed inverse
        # read, output rows written and read back, r read, z written
        bytes_per_launch = nint * (packed * 4 + 2 * npatch * 4) + 2 * nu * 4
    k4_launch_s = (k4_ms / max(k4_n, 1)) / 1e3
    achieved = bytes_per_launch / k4_launch_s / 1e9 if k4_n else None
    peak, peak_kind = measured_peak_hbm()
    # operator apply (K1 cell kernel) on the finest level, timed live inside the smoother
    ncells = math.prod(F)
    nq = (order + 1) ** pb.d
    ncq = (6 if pb.d == 2 else 21) if tensor else 1
    fused = pb.d == 3 and order == 2 and os.environ.get("ALS_FUSE_GATHER", "1") != "0"
    if fused:
        # the 3D smoother's cell kernel also forms Z_j from the star-patch outputs: read the
        # patch outputs, write Z_j and the staged cell outputs, read mu or C (FP32)
        k1_bytes = nverts * npatch * 4 + nu * 4 + ncells * nq * pb.d * 4 + ncells * nq * ncq * 4
    else:
        k1_bytes = nu * 4 * 2 + ncells * nq * ncq * 4      # read x, write y, read mu or C (FP32)
    if order == 3:   # the cell kernel reads x, mu and W^-1 and stages its outputs per cell (FP32)
        k1_bytes = nu * 4 + ncells * nq * 4 + ncells * pressure_per_cell(pb.d, 3) ** 2 * 4 + \
            ncells * nq * pb.d * 4
    k1_flops = ncells * ((APPLY_FLOPS_PER_CELL_Q3 if order == 3 else APPLY_FLOPS_PER_CELL)[pb.d] +
                         (nq * 2 * 2 * ncq if tensor else 0))
    k1_s = (k1_ms / max(k1_n, 1)) / 1e3
    roofline_apply = None
    if k1_n:
        alu = {"achieved": k1_flops / k1_s / 1e12, "peak": fp32_peak, "peak_kind": "measured FP32 FMA",
               "unit": "TFLOP/s", "frac": (k1_flops / k1_s / 1e12) / fp32_peak if fp32_peak else None}
        hbm = {"achieved": k1_bytes / k1_s / 1e9, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
               "frac": (k1_bytes / k1_s / 1e9) / peak}
        # scalar mu: about 27 flop/B against a machine balance of about 11 flop/B (ALU side);
        # tensor C: 21 FP32 coefficients per point make it about 3 flop/B (HBM side)
        roofline_apply = dict(hbm if tensor else alu)
        roofline_apply.update({
            "bound": "hbm" if tensor else "alu",
            "kernel": ("k_apply_lines (FP32 A_gamma cell kernel%s, finest level)"
                       % (" with the fused patch gather" if fused else "")) if order == 2 else
                      "k_qk%s_cells<float> (FP32 order-3 A_gamma cell kernel, finest level)" % ("3" if pb.d == 3 else ""),
            ("alu" if tensor else "hbm"): alu if tensor else hbm,
            "us_per_launch": k1_s * 1e6, "launches_timed": k1_n,
            "bytes_per_launch": k1_bytes, "flops_per_launch": k1_flops})
    out = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "dim": pb.d, "cells": list(pb.n), "levels": pb.levels, "order": order,
                   "gamma": pb.gamma, "dr": spec.get("dr", pb.meta.get("contrast")),
                   "sinkers": spec.get("count"), "coefficients": "tensor C (21 per point)" if tensor else "scalar mu",
                   "schur": spec.get("schur", "P1"), "dofs": dofs,
                   "smoother": f"GMRES({spec['sweeps']}) x vertex-star PSC", "rtol": RTOL,
                   "step": "setup (patch factorisation, coarse Cholesky, Schur) + mixed FGMRES solve",
                   "l2": "inputs larger than L2 (fine-level FP32+FP64 patch inverses %.1f GB)"
                         % (math.prod(v + 1 for v in pb.n) * 12 * npatch * (npatch + 1) / 2 / 1e9),
                   "parallelism": f"replicas x{dist.world}"},
        "iterations": its[-1] if its else None,
        "vcycles_per_s": vcyc_s,
        "fp64": {"solve_dof_per_s": dofs / t64, "ms_per_step": t64 * 1e3, "iterations": info64.iterations,
                 "vcycles_per_s": vcyc64_s},
        "mixed_vs_fp64_speedup": t64 / t_step,
        "mixed_vs_fp64_rel_err": {"u": err_u, "p": err_p},
        "setup_fp64": setup_fp64,
        "fcycle": fcycle,
        "gamma_1e4": gamma_large,
        "bf16_storage": bf16_storage,
        "e2e": {"value": dist.world * dofs / t_e2e, "unit": "DoF/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "hbm",
                     "kernel": ("k_patch_tma<%d> (FP32 interior-star smoother, finest level)" % pb.d) if order == 2
                     else "k_qk%s_star_apply_w + k_qk%s_star_gather<float> (FP32 order-3 star smoother, finest level)"
                     % (("3", "3") if pb.d == 3 else ("", "")),
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "bytes_per_launch": bytes_per_launch, "launches_timed": k4_n,
                     "units": {"stars_streamed": nint, "bytes_per_star": packed * 4 + npatch * 4,
                               "r_bytes": nu * 4},
                     "traffic": stored_traffic("k_patch_apply_f32_fine", args.workload)},
        "roofline_apply": roofline_apply,
        "phases": {"setup_ms": t_setup * 1e3, "solve_ms": t_solve * 1e3,
                   "solve_dof_per_s": dofs / t_solve, "solve_iterations": info_s.iterations,
                   "fp64_solve_ms": t64_solve * 1e3, "fp64_solve_dof_per_s": dofs / t64_solve},
        "measured_peaks": {"fp32_tflops": fp32_peak, "fp64_tflops": fp64_peak,
                           "how": "als_measure_fma_peaks: FMA chains on every SM, CUDA events"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if dist.rank == 0:
        if dist.world == 1 and not args.no_cpu_baseline:
            try:
                out["cpu_baseline"] = cpu_baseline(args.workload)
            except Exception as e:  # noqa: BLE001
                out["cpu_baseline"] = {"error": str(e)[:200]}
        print(json.dumps(out))


def ours_batch(args, dist):
    """Serving-style sweep: 64 independent multi-sinker instances (32 2D, 32 3D, uneven
    sizes, contrasts 1e4..1e8, gamma 1e2 / 1e4), mixed precision with the P2 Schur
    pairing.  Batched solves (interleaved FGMRES rounds, one wait per round) whose
    preconditioner cycles run as one merged launch per level operation for all live
    instances (the headline), against the same batch with the instances' own cycle
    graphs as concurrent branches, and against one-at-a-time calls on the same contexts;
    the same three forms for bare FP32 cycles."""
    import numpy as np
    import torch

    from paper_2107_00820_gb300 import Batch, alstokes as A
    from synthetic.problems import batch_instances

    torch.cuda.set_device(dist.local)
    pbs = batch_instances(32, 32, seed=64 * dist.rank)
    dofs = [problem_dofs(pb) for pb in pbs]
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")  # noqa: E731
    stream = torch.cuda.current_stream().cuda_stream
    opts = {"mode": A.ALS_MODE_MIXED, "schur": A.ALS_SCHUR_P2, "rtol": RTOL, "maxit": 300, "sweeps": 5}
    inst = [{"dim": pb.d, "n": pb.n, "levels": pb.levels, "coeffs": [dev(m) for m in pb.mu], "gamma": pb.gamma,
             "options": opts} for pb in pbs]
    t0 = time.perf_counter()
    batch = Batch(inst, stream)
    t_create = time.perf_counter() - t0
    f = [dev(pb.f) for pb in pbs]
    ubc = [dev(pb.u_bc) for pb in pbs]
    u = [torch.zeros(s[0], dtype=torch.float64, device="cuda") for s in batch.shapes]
    p = [torch.zeros(s[1], dtype=torch.float64, device="cuda") for s in batch.shapes]
    ctxs = [batch.instance(i) for i in range(len(pbs))]
    for _ in range(max(1, args.warmup - 2)):                   # captures every cycle graph
        _, _, infos = batch.solve(f, ubc, None, u, p)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        dist.barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return max(e0.elapsed_time(e1) / 1e3, time.perf_counter() - w0) / reps

    merged_mode = batch.mode == A.ALS_BATCH_MERGED
    clocks = ClockSampler(dist.local)
    clocks.start()
    launches0 = A.als_kernel_launches()
    t_batch = dist.max(timed(lambda: batch.solve(f, ubc, None, u, p), args.steps))
    launches = (A.als_kernel_launches() - launches0) // max(args.steps, 1)
    clk = clocks.stop()
    infos = batch.solve(f, ubc, None, u, p)[2]
    u_b = [x.clone() for x in u]

    # the same batch with the instances' own cycle graphs as concurrent branches
    batch.set_mode(A.ALS_BATCH_BRANCHES)
    batch.solve(f, ubc, None, u, p)                            # captures the instances' graphs
    t_branch = dist.max(timed(lambda: batch.solve(f, ubc, None, u, p), 1))
    same_branch = all(torch.equal(a, b) for a, b in zip(u_b, u))

    def one_at_a_time():
        for i, c in enumerate(ctxs):
            c.solve(f[i], ubc[i], None, u[i], p[i])
    t_seq = dist.max(timed(one_at_a_time, 1))
    same = all(torch.equal(a, b) for a, b in zip(u_b, u))

    # FP32 cycles: merged launches, the graph of the instances' cycle graphs, one at a time
    b32 = [torch.randn(s[0], dtype=torch.float32, device="cuda") for s in batch.shapes]
    x32 = [torch.zeros_like(t) for t in b32]
    batch.vcycle(b32, x32, A.ALS_PREC_FP32)
    t_bcyc = timed(lambda: batch.vcycle(b32, x32, A.ALS_PREC_FP32), 5)
    t_mcyc, merged_kernels, merged_tune = None, None, {}
    if merged_mode:
        batch.set_mode(A.ALS_BATCH_MERGED)
        batch.vcycle(b32, x32, A.ALS_PREC_FP32)
        t_mcyc = timed(lambda: batch.vcycle(b32, x32, A.ALS_PREC_FP32), 5)
        grouping, groups, gms, merged_kernels = batch.merged_plan()
        names = ("one group", "by dimension", "by dimension and levels", "by shape", "by shape, chunks of 4")
        merged_tune = {"grouping": names[grouping], "groups": groups,
                       "cycle_ms_per_grouping": {names[k]: (round(v, 3) if v >= 0 else None) for k, v in enumerate(gms)},
                       "variants": {}}
        vn = ("tma2", "tma3", "direct")
        for g in range(groups):
            members = batch.merged_tune(g, 1)[3]
            for lvl in range(1, max(pbs[i].levels for i in members)):
                pv, iv, ms, _ = batch.merged_tune(g, lvl)
                merged_tune["variants"][f"group{g}/level{lvl}"] = f"{vn[pv]}/{vn[iv]}"

    def seq_cycles():
        for i, c in enumerate(ctxs):
            c.vcycle(b32[i], x32[i], A.ALS_PREC_FP32)
    t_scyc = timed(seq_cycles, 3)
    its = [int(x.iterations) for x in infos]
    tuned = {}
    for i, pb in enumerate(pbs):
        for lvl in range(1, pb.levels):
            v = ctxs[i].autotune_info(lvl)[0]
            tuned[v] = tuned.get(v, 0) + 1
    total = sum(dofs)
    out = {
        "metric": "aggregate solve DoF/s, 64 independent instances (batched), mixed, 1e-8",
        "value": dist.world * total / t_batch, "unit": "DoF/s", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_batch * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "batch64", "instances": len(pbs), "dim_mix": "32 2D (16^2..256^2) + 32 3D (8^3..32^3)",
                   "dr": "10^U[4,8]", "gamma": "{1e2, 1e4}", "schur": "P2 (W = M_p(1/mu))", "rtol": RTOL,
                   "total_dofs": total, "step": "batched FGMRES solves of all instances (setup excluded)",
                   "cycle_form": "merged (one launch per level operation)" if merged_mode else "branches",
                   "l2": "inputs larger than L2 (all instances' patch inverses ~10^10 B)",
                   "parallelism": f"replicas x{dist.world}"},
        "branches": {"ms": t_branch * 1e3, "dof_per_s": total / t_branch, "bitwise_equal_to_merged": same_branch},
        "one_at_a_time": {"ms": t_seq * 1e3, "dof_per_s": total / t_seq, "bitwise_equal_to_batched": same},
        "batched_vs_one_at_a_time": t_seq / t_batch,
        "merged_vs_branches": t_branch / t_batch,
        "cycles": {"merged_ms": t_mcyc * 1e3 if t_mcyc else None, "branches_ms": t_bcyc * 1e3,
                   "one_at_a_time_ms": t_scyc * 1e3,
                   "merged_vs_one_at_a_time": t_scyc / t_mcyc if t_mcyc else None,
                   "branches_vs_one_at_a_time": t_scyc / t_bcyc,
                   "merged_kernels_per_cycle": merged_kernels, "prec": "fp32"},
        "iterations": {"min": min(its), "max": max(its), "mean": statistics.mean(its),
                       "all_converged": all(int(x.converged) == 1 for x in infos)},
        "merged_autotuner": merged_tune,
        "autotuner_choices": {("tma2", "tma3", "direct")[k]: v for k, v in sorted(tuned.items())},
        "create_s": t_create,
        "gpu_launches": launches,
        "clocks": clk,
    }
    batch.close()
    if dist.rank == 0:
        print(json.dumps(out))


def ours_exact(args, dist):
    """Table exacttopleft's study (Sec. 3) on the GPU: FGMRES iterations to a 1e6 residual
    reduction with the (1,1) block solved exactly (a one-level context: the dense inverse of
    A_gamma), P1 and P2, gamma 0 / 10 / 1e3, DR 1e4 / 1e6 / 1e8, 2D multi-sinker on 32^2."""
    import torch

    from paper_2107_00820_gb300 import Context, alstokes as A
    from synthetic.problems import sinker_problem

    torch.cuda.set_device(dist.local)
    n = 32
    table, t_setup, t_solve = {}, [], []
    for var in ("P1", "P2"):
        for g in (0.0, 10.0, 1e3):
            row = []
            for dr in (1e4, 1e6, 1e8):
                pb = sinker_problem(2, n, 1, 8, 0.1, 200.0, dr, 10.0, g, 0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ctx = Context(2, pb.n, 1, pb.mu, g, rtol=1e-6, maxit=300,
                              schur=A.ALS_SCHUR_P2 if var == "P2" else A.ALS_SCHUR_P1)
                t1 = time.perf_counter()
                info = ctx.solve(pb.f, pb.u_bc)[2]
                t2 = time.perf_counter()
                ctx.close()
                row.append(int(info.iterations))
                t_setup.append(t1 - t0)
                t_solve.append(t2 - t1)
            table[f"{var} gamma={g:g}"] = row
    dofs = 2 * (2 * n - 1) ** 2 + 3 * n * n
    out = {"metric": "FGMRES iterations with the exact (1,1) solve (Table exacttopleft), 2D 32^2, 1e6 reduction",
           "value": dofs / statistics.median(t_solve), "unit": "DoF/s (solve, median)", "n_gpus": 1,
           "steps": len(t_solve), "warmup": 0, "ms_per_step": 1e3 * statistics.median(t_solve),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "exact2d_32", "cells": [n, n], "dofs": dofs, "dr_columns": [1e4, 1e6, 1e8],
                      "solver": "one level: dense FP64 inverse of A_gamma (symmetric sweep), FGMRES rtol 1e-6"},
           "iterations": table,
           "paper_table_exacttopleft_394754_dofs": {"P1 gamma=0": [32, 48, 59], "P1 gamma=10": [7, 9, 10],
                                                    "P1 gamma=1000": [2, 3, 4], "P2 gamma=0": [32, 48, 59],
                                                    "P2 gamma=10": [10, 16, 20], "P2 gamma=1000": [2, 4, 5]},
           "setup_s_median": statistics.median(t_setup)}
    if dist.rank == 0:
        print(json.dumps(out))


def ours_newton(args, dist):
    """Newton's method for the viscoplastic rheology (Sec. 5.3.1) on the GPU: 3D 32^3, 4
    levels, tau_y 1, mu_ref 1, gamma 1e2, P2 pairing, mixed precision (FP32 cycle, FP64
    residuals and outer loop), Newton to a 1e-10 residual reduction; every step re-runs the
    setup for the linearised fourth-order coefficient at every level's Gauss points."""
    import numpy as np
    import torch

    from paper_2107_00820_gb300 import Context, alstokes as A

    torch.cuda.set_device(dist.local)
    d, n, L, gamma = 3, 32, 4, 1e2
    nn = 2 * n + 1
    g = np.arange(nn) / (nn - 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    X, Y, Z = (a.transpose(2, 1, 0).reshape(-1) for a in (X, Y, Z))
    uD = np.concatenate([np.sin(np.pi * X) * np.cos(np.pi * Y), -np.cos(np.pi * X) * np.sin(np.pi * Y),
                         np.zeros_like(X)])
    f = np.zeros((n ** 3, 27, 3))
    f[..., 2] = -1.0
    iu = np.triu_indices(6)
    C = (2.0 * np.eye(6))[iu]
    coeffs = [np.ascontiguousarray(np.broadcast_to(C, ((n >> (L - 1 - l)) ** 3, 27, 21))) for l in range(L)]
    mus = [np.ones(((n >> (L - 1 - l)) ** 3, 27)) for l in range(L)]
    ctx = Context(d, n, L, coeffs, gamma, mu_eff=mus, schur=A.ALS_SCHUR_P2, maxit=300, mode=A.ALS_MODE_MIXED)
    fd = torch.as_tensor(f, device="cuda")
    ud = torch.as_tensor(uD, device="cuda")
    u = torch.zeros(ctx.nu(), dtype=torch.float64, device="cuda")
    p = torch.zeros(ctx.npres(), dtype=torch.float64, device="cuda")
    ctx.newton_solve(fd, ud, u, p, mu_ref=1.0, tau_y=1.0, rtol=1e-10)     # warm-up (graphs, tuning)
    torch.cuda.synchronize()
    ts = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        info = ctx.newton_solve(fd, ud, u, p, mu_ref=1.0, tau_y=1.0, rtol=1e-10)[2]
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    hist, lin = ctx.newton_history()
    dofs = d * (2 * n - 1) ** 3 + (d + 1) * n ** 3
    t = statistics.median(ts)
    out = {"metric": "Newton solve DoF/s to 1e-10 (viscoplastic rheology), mixed, 1xGB300",
           "value": dofs / t, "unit": "DoF/s", "n_gpus": 1, "steps": len(ts), "warmup": 1, "ms_per_step": 1e3 * t,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "newton3d_32", "cells": [n] * 3, "levels": L, "gamma": gamma, "schur": "P2",
                      "mu_ref": 1.0, "tau_y": 1.0, "dofs": dofs},
           "newton_steps": info.iterations, "linear_iterations": lin[1:],
           "residual_history": [float(v) for v in hist]}
    ctx.close()
    if dist.rank == 0:
        print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sinker3d_32",
                    choices=sorted(WORKLOADS) + ["batch64", "exact2d_32", "newton3d_32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the FP64-setup and gamma 1e4 side measurements")
    ap.add_argument("--cpu-worker", action="store_true")
    ap.add_argument("--sample-kind", default="cpu_baseline")
    ap.add_argument("--reps", type=int, default=1)
    args = ap.parse_args()
    if args.cpu_worker:
        cpu_worker(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        # the oracle arm needs no process group: rank 0 runs it, the other ranks exit
        reference_arm(args, _RankOnly())
        return
    dist = Dist(args.gpus)
    try:
        if args.workload == "batch64":
            ours_batch(args, dist)
        elif args.workload == "exact2d_32":
            ours_exact(args, dist)
        elif args.workload == "newton3d_32":
            ours_newton(args, dist)
        else:
            ours(args, dist)
    finally:
        dist.close()


class _RankOnly:
    def __init__(self):
        self.rank = int(os.environ.get("RANK", "0"))


if __name__ == "__main__":
    main()
