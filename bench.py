#!/usr/bin/env python
"""Benchmark of the matrix-free DG operator (one JSON line on rank 0).

A step is one FP64 residual evaluation r = A u - F (Algorithm 1 of Sec. 3.6 plus
the right hand side) on the 32^3-cell, Q_7 unit-cube workload with per-cell
log-normal diffusion (16.8 M DOF), inputs resident in HBM.  The vectors (u, r:
134 MB each) and the work buffers (335 MB) are larger than the 129 MB L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (direct quadrature, single thread)
on a bounded sample of the same workload's cells on the host cores.
Multi-GPU runs are independent replicas (one problem per rank, weak scaling):
the operator application needs no data-path collective.
"""

from __future__ import annotations

import argparse
import hashlib
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

# Unit-count peaks: SMs x FMA per clock per SM (2 FP64, 128 FP32) x 2 flop x maximum SM clock.  The values below
# are those of a GB300 (152 SMs, 2070 MHz); set_unit_peaks() replaces them with the running device's SM count and
# the maximum SM clock nvidia-smi reports, before anything is measured.
UNIT_SMS, UNIT_MHZ = 152, 2070.0
FP64_PEAK_TFLOPS = UNIT_SMS * 2 * 2 * UNIT_MHZ * 1e6 / 1e12
FP32_PEAK_TFLOPS = UNIT_SMS * 128 * 2 * UNIT_MHZ * 1e6 / 1e12


def set_unit_peaks(device_index=0):
    """The unit-count peaks of the device in use (SM count from CUDA, maximum SM clock from nvidia-smi)."""
    global UNIT_SMS, UNIT_MHZ, FP64_PEAK_TFLOPS, FP32_PEAK_TFLOPS
    import torch
    if not torch.cuda.is_available():
        return
    UNIT_SMS = torch.cuda.get_device_properties(device_index).multi_processor_count
    try:
        out = subprocess.run(["nvidia-smi", f"--id={device_index}", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        UNIT_MHZ = float(out.stdout.strip().splitlines()[0])
    except Exception:
        pass
    FP64_PEAK_TFLOPS = UNIT_SMS * 2 * 2 * UNIT_MHZ * 1e6 / 1e12
    FP32_PEAK_TFLOPS = UNIT_SMS * 128 * 2 * UNIT_MHZ * 1e6 / 1e12

# DRAM traffic per launch measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum) for the
# kernels as they were when profiled, keyed by the sha256 of the kernel source at that time.
NCU_TRAFFIC = {
    ("dg_cell_kernel", "f1e344aa4d41ba1e"): 135631360 + 271920128,  # 135.63 MB read + 271.92 MB write
    ("dg_face_kernel", "f1e344aa4d41ba1e"): 474571776 + 113187328,  # 474.57 MB read + 113.19 MB write
}


# FP32 lane instructions (FADD + FFMA + FMUL) per cell of the double-float kernels at k = 7, from the ncu
# counters smsp__sass_thread_inst_executed_op_{fadd,ffma,fmul}_pred_on.sum of one launch / 32768 cells
F64X_FP32_INST_PER_CELL = {"cell": (9747562496 + 2602565632 + 878706688) / 32768,
                           "face": (5093392384 + 1496776704 + 499712000) / 32768}


def kernel_source_hash():
    p = os.path.join(ROOT, "paper_1711_10885_gb300", "csrc", "dg_kernels.cuh")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_max(values):
    """Element-wise max over ranks of a list of floats (the timing rule: slowest rank counts)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return [float(v) for v in values]
    dev = torch.device("cuda", torch.cuda.current_device()) if tdist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_mdofs(world_size, dofs_per_rank, steps, ms):
    """Whole-job throughput of independent replicas: all ranks' DOF-applications over the slowest rank's time."""
    return world_size * dofs_per_rank * steps / (ms * 1e-3) / 1e6


def run_reference(args):
    """CPU oracle on bounded samples of the workload's cells (rank 0 only)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1711_10885_gb300 import inputs
    oracle.build()
    w = inputs.unit_cube_q7_32()
    pr = oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c)
    # size one step's sample so that warmup + steps take about two minutes
    t0 = time.perf_counter()
    oracle.apply(pr, w.u, cells=list(range(8)))
    per_cell = (time.perf_counter() - t0) / 8
    budget_s = 120.0 / max(1, args.steps + args.warmup)
    cells_per_step = int(max(8, min(w.ncell, budget_s / per_cell)))
    rng = np.random.default_rng(99)
    for _ in range(args.warmup):
        oracle.apply(pr, w.u, cells=rng.choice(w.ncell, cells_per_step, replace=False))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.apply(pr, w.u, cells=rng.choice(w.ncell, cells_per_step, replace=False))
    dt = time.perf_counter() - t0
    mdofs = args.steps * cells_per_step * w.nb / dt / 1e6
    sample = f"{cells_per_step} random cells of the 32^3 Q7 workload per step (A u on those cells)"
    line = {"metric": "DG FP64 residual apply throughput, 32^3 cells Q7 (16.8M DOF)", "value": mdofs,
            "unit": "MDOF/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "unit_cube_q7_32", "cells": [32, 32, 32], "k": 7, "dofs": w.ndof},
            "impl": "reference",
            "cpu_baseline": {"value": mdofs, "unit": "MDOF/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": mdofs, "unit": "MDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(w, seconds=15.0):
    """Oracle (single thread, direct quadrature) on a bounded sample of the same workload's cells."""
    import numpy as np

    import oracle
    oracle.build()
    pr = oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c)
    t0 = time.perf_counter()
    oracle.apply(pr, w.u, cells=list(range(8)))
    per_cell = (time.perf_counter() - t0) / 8
    count = int(max(16, min(w.ncell, seconds / per_cell)))
    cells = np.random.default_rng(7).choice(w.ncell, count, replace=False)
    t0 = time.perf_counter()
    oracle.apply(pr, w.u, cells=cells)
    dt = time.perf_counter() - t0
    return {"value": count * w.nb / dt / 1e6, "unit": "MDOF/s", "cores": 1, "kind": "oracle",
            "sample": f"A u on {count} random cells of the 32^3 Q7 workload ({dt:.1f} s, one thread)",
            "host": host_cpu()}


def host_cpu():
    """The host the oracle ran on: logical CPUs and the CPU model (from /proc/cpuinfo or lscpu, where present)."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu": model or platform.processor() or platform.machine()}


def run_profile_solver(args):
    """Minimal launch sequence for profilers of the solver kernels: at 48^3 Q5 (fast diagonalisation only, under
    1 GB on the device) W + K FP32 and FP64 block-Jacobi applications and learned-preconditioner applications
    (untrained network); then one outer iteration of the mixed solve (one inner FGMRES(30) cycle) at 32^3 Q5 for
    the basis passes (about 3 GB), and one inner FGMRES(20) cycle with the FP16 basis at 48^3 Q5 (about 4 GB), with
    block-Jacobi and with red-black Gauss-Seidel."""
    import torch

    from paper_1711_10885_gb300 import dg, inputs
    torch.cuda.set_device(0)
    w = inputs.unit_cube_q5_48(with_u=False)
    op = dg.operator_for(w)
    op.precond_setup(dg.DG_BJ_FAST_DIAG)
    mlp = dg.MLP(w.k, seed=0)
    r = torch.randn(w.ndof, dtype=torch.float32, device="cuda")
    z = torch.empty_like(r)
    r64, z64 = r.double(), torch.empty(w.ndof, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for _ in range(args.warmup + args.steps):
        op.precond_apply(r, z)
    for _ in range(args.warmup + args.steps):
        op.precond_apply(r64, z64)
    for _ in range(args.warmup + args.steps):
        mlp.apply(op, r, z)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(10):
        mlp.apply(op, r, z)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / 10
    flops = 2.0 * w.ncell * (256 * mlp.kinp + 256 * 256 + mlp.outp * 256)
    mlp.close()
    op.close()
    del r, z, r64, z64
    ws = inputs.Workload("unit_cube_q5_32", (32, 32, 32), 5, inputs.log_normal_D(32 ** 3, 1.0, 3), f_kind="sines",
                         f_params=inputs.sine_modes(4))
    ops = dg.operator_for(ws)
    ops.precond_setup(dg.DG_BJ_FAST_DIAG)
    x = torch.zeros(ws.ndof, dtype=torch.float64, device="cuda")
    st = ops.solve(x, mode=dg.DG_SOLVE_MIXED, preconditioner=dg.DG_PRECOND_BLOCK_JACOBI, rtol=1e-10, restart=30,
                   outer_restart=20, inner_rtol=1e-3, max_iterations=1, raise_on_error=False)
    ops.close()
    del x
    # one inner FGMRES(20) cycle with the FP16 basis at 48^3 Q5 (outer restart 1: about 4 GB on the device)
    op = dg.operator_for(w)
    op.precond_setup(dg.DG_BJ_FAST_DIAG)
    x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    st48 = op.solve(x, mode=dg.DG_SOLVE_MIXED, preconditioner=dg.DG_PRECOND_BLOCK_JACOBI, rtol=1e-10, restart=20,
                    outer_restart=1, inner_rtol=1e-3, max_iterations=1, inner_basis_precision=1, raise_on_error=False)
    # the same cycle with red-black Gauss-Seidel (one-colour operator, Krylov step in Eisenstat's form)
    x.zero_()
    st48g = op.solve(x, mode=dg.DG_SOLVE_MIXED, preconditioner=dg.DG_PRECOND_RB_GS, rtol=1e-10, restart=20,
                     outer_restart=1, inner_rtol=1e-3, max_iterations=1, inner_basis_precision=1, raise_on_error=False)
    op.close()
    print(json.dumps({"profile": "solver", "mlp_apply_ms": ms, "mlp_tflops": flops / (ms * 1e-3) / 1e12,
                      "cells": w.ncell, "solve_32": {k: st[k] for k in ("iterations", "inner_iterations")},
                      "solve_48_fp16_basis": {k: st48[k] for k in ("iterations", "inner_iterations")},
                      "solve_48_fp16_basis_rbgs": {k: st48g[k] for k in ("iterations", "inner_iterations")}}))


def run_profile(args):
    """Minimal launch sequence for profilers: W + K residual applies on the bench workload."""
    import torch

    from paper_1711_10885_gb300 import dg, inputs
    if args.profile_solver:
        return run_profile_solver(args)
    torch.cuda.set_device(0)
    if args.tensor:
        # tensor diffusion on the 32^3 Q7 workload: W + K residual applies
        import numpy as np
        w = inputs.unit_cube_q7_32()
        op = dg.Operator(w.n, w.k, 1.0, b=w.b, c=w.c, D_tensor=inputs.log_normal_tensors(w.ncell, 1.0, 60),
                         f_qp=np.ones(w.ncell * (w.k + 1) ** 3))
        u = torch.tensor(w.u, device="cuda")
        r = torch.empty_like(u)
        prec = dg.DG_F64X if args.precision == "f64x" else dg.DG_F64
        for _ in range(args.warmup + args.steps):
            op.apply_residual(u, r, precision=prec)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "ok", "applies": args.warmup + args.steps, "r_norm": float(r.abs().max())}))
        op.close()
        return
    if args.f32:
        # the FP32 operator of the mixed solve's inner FGMRES: 48^3 cells, Q5 (23.9 M DOF), W + K Jacobian applies
        w = inputs.Workload("unit_cube_q5_48", (48, 48, 48), 5, inputs.log_normal_D(48 ** 3, 1.0, 3))
        op = dg.Operator(w.n, w.k, w.D, b=w.b, c=w.c)
        u = torch.tensor(inputs.uniform_u(w.ndof, 5), dtype=torch.float32, device="cuda")
        y = torch.empty_like(u)
        for _ in range(args.warmup + args.steps):
            op.apply_jacobian(u, y)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "ok", "applies": args.warmup + args.steps, "y_max": float(y.abs().max())}))
        op.close()
        return
    if args.small:
        # the 8^3-cell Q3 unit-cube workload: W + K residual applies
        w = inputs.unit_cube_q3_8()
        op = dg.operator_for(w)
        u = torch.tensor(w.u, device="cuda")
        r = torch.empty_like(u)
        for _ in range(args.warmup + args.steps):
            op.apply_residual(u, r)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "ok", "applies": args.warmup + args.steps, "r_max": float(r.abs().max())}))
        op.close()
        return
    if args.mlp_forward:
        # network inference on 262144 feature rows (k = 4): W + K forward passes
        mlp = dg.MLP(4, seed=7)
        X = torch.randn(262144, mlp.kinp, device="cuda").to(torch.bfloat16)
        for _ in range(args.warmup + args.steps):
            Y = mlp.forward(X)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "ok", "forwards": args.warmup + args.steps, "y_max": float(Y.abs().max())}))
        mlp.close()
        return
    if args.problem_b:
        # Problem B (point-wise coefficients, k = 7, m = 10) on problem_b^3 sheared cells: W + K residual applies
        import numpy as np
        n, k = args.problem_b, 7
        m = k + 3
        J = inputs.sheared_jacobian(np.full(3, 1.0 / n), 70)
        fields = inputs.PolynomialFields(70, np.zeros(3), J @ np.full(3, float(n)))
        xv, xf = affine_grid_points((n, n, n), m, np.zeros(3), J)
        op = dg.Operator((n, n, n), k, 1.0, b=(0.0, 0.0, 0.0), c=0.0, m=m, jacobian=J, D_qp=fields.D(xv),
                         D_face=fields.D(xf), c_qp=fields.c(xv), velocity="points", b_qp=fields.b(xv),
                         b_face=inputs.face_normal_velocity_affine(fields.b, xf, J), f_qp=np.ones(n ** 3 * m ** 3))
        u = torch.tensor(inputs.uniform_u(op.ndof, 71), device="cuda")
        r = torch.empty_like(u)
        prec = dg.DG_F64X if args.precision == "f64x" else dg.DG_F64
        for _ in range(args.warmup + args.steps):
            op.apply_residual(u, r, precision=prec)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "ok", "applies": args.warmup + args.steps, "r_norm": float(r.abs().max())}))
        op.close()
        return
    if args.matrix:
        # matrix-based comparison: assemble on matrix_n^3 cells of degree matrix_k, then W + K products
        w = inputs.small_case(n=(args.matrix_n,) * 3, k=args.matrix_k, seed=200 + args.matrix_k)
        op = dg.operator_for(w)
        A = dg.Matrix(op)
        x = torch.tensor(w.u, device="cuda")
        y = torch.empty_like(x)
        for _ in range(args.warmup + args.steps):
            A.spmv(x, y)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "ok", "spmv": args.warmup + args.steps, "nnzb": A.nnzb, "y_max": float(y.abs().max())}))
        A.close()
        op.close()
        return
    if args.transport:
        # Taylor-Green transport (k = 5, m = 8): W + K Heun steps, 4 launches each
        import numpy as np
        w = inputs.taylor_green(args.transport, 5)
        op = dg.operator_for(w)
        xi = (np.polynomial.legendre.leggauss(w.m)[0] + 1.0) / 2.0
        z = op.project(inputs.gaussian_bump_grid(w, xi, xp=torch, device="cuda").contiguous())
        prec = dg.DG_F64X if args.precision == "f64x" else dg.DG_F64
        op.ssprk2(z, 0.3 * 2 * np.pi / args.transport / 11, args.warmup + args.steps, precision=prec)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "ok", "heun_steps": args.warmup + args.steps, "z_max": float(z.abs().max())}))
        op.close()
        return
    w = inputs.unit_cube_q7_32()
    op = dg.operator_for(w)
    u = torch.tensor(w.u, device="cuda")
    prec = {"f64": dg.DG_F64, "f64x": dg.DG_F64X, "f32": dg.DG_F32}[args.precision]
    if prec == dg.DG_F32:
        u = u.float()
    r = torch.empty_like(u)
    torch.cuda.synchronize()
    for _ in range(args.warmup + args.steps):
        op.apply_residual(u, r, precision=prec)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "ok", "applies": args.warmup + args.steps, "r_norm": float(r.abs().max())}))
    op.close()


def solve_benchmark(rtol=1e-10, inner_rtol=1e-3, restart=30, outer_restart=20, with_fp64=True):
    """Mixed-precision vs plain FP64 block-Jacobi FGMRES on the 48^3 Q5 workload (sine source, log-normal D).
    The mixed solve runs with its default inner block inverse (fast diagonalisation) and with the FP32 dense
    blocks; with_fp64=False skips the two-minute plain FP64 solve."""
    import torch

    from paper_1711_10885_gb300 import dg, flops, inputs
    w = inputs.unit_cube_q5_48(with_u=False)
    op = dg.operator_for(w)
    # the fast diagonalisation alone (what the default mixed solve needs), then the dense blocks too
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    op_fd = dg.operator_for(w)
    op_fd.precond_setup(dg.DG_BJ_FAST_DIAG)
    torch.cuda.synchronize()
    setup_fd_s = time.perf_counter() - t0
    x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st_fd = op_fd.solve(x, mode=dg.DG_SOLVE_MIXED, preconditioner=dg.DG_PRECOND_BLOCK_JACOBI, rtol=rtol,
                        restart=restart, outer_restart=outer_restart, inner_rtol=inner_rtol, raise_on_error=False)
    torch.cuda.synchronize()
    st_fd["wall_s"] = time.perf_counter() - t0
    op_fd.close()
    del x
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    op.precond_setup()
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    out = {"workload": "unit_cube_q5_48", "dofs": w.ndof, "rtol": rtol, "precond_setup_s": setup_s,
           "mixed_fast_diag_only": dict(st_fd, setup_s=setup_fd_s,
                                        time_to_solution_s=setup_fd_s + st_fd["wall_s"])}
    xs = {}
    runs = [("mixed", dg.DG_SOLVE_MIXED, 0), ("mixed_fp32_blocks", dg.DG_SOLVE_MIXED, 1)]
    if with_fp64:
        runs.insert(0, ("fp64", dg.DG_SOLVE_FP64, 0))
    for name, mode, ibp in runs:
        x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = op.solve(x, mode=mode, preconditioner=dg.DG_PRECOND_BLOCK_JACOBI, rtol=rtol, restart=restart,
                      outer_restart=outer_restart, inner_rtol=inner_rtol, raise_on_error=False,
                      inner_block_precision=ibp)
        torch.cuda.synchronize()
        st["wall_s"] = time.perf_counter() - t0
        out[name] = st
        xs[name] = x
    if with_fp64:
        out["field_diff_mixed_vs_fp64"] = float((xs["mixed"] - xs["fp64"]).abs().max() / xs["fp64"].abs().max())
        out["speedup_mixed_vs_fp64"] = out["fp64"]["wall_s"] / out["mixed"]["wall_s"]
    out["field_diff_default_vs_fp32_blocks"] = float((xs["mixed"] - xs["mixed_fp32_blocks"]).abs().max()
                                                     / xs["mixed_fp32_blocks"].abs().max())
    # operator throughput at this size
    for prec, dt in (("f32", torch.float32), ("f64", torch.float64)):
        u = torch.rand(w.ndof, dtype=dt, device="cuda")
        y = torch.empty_like(u)
        for _ in range(3):
            op.apply_jacobian(u, y)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(20):
            op.apply_jacobian(u, y)
        b.record()
        b.synchronize()
        out[f"apply_{prec}_mdofs"] = w.ndof * 20 / (a.elapsed_time(b) * 1e-3) / 1e6
        # executed flops of the cell and face kernels (flops.py model) against the unit-count peak
        tflops = out[f"apply_{prec}_mdofs"] * 1e6 * flops.apply_flops_per_dof(w.k, w.n, residual=False) / 1e12
        out[f"apply_{prec}_tflops"] = tflops
        out[f"apply_{prec}_frac_of_peak"] = tflops / (FP32_PEAK_TFLOPS if prec == "f32" else FP64_PEAK_TFLOPS)
        r = torch.empty_like(u)
        a.record()
        for _ in range(20):
            op.precond_apply(u, r)
        b.record()
        b.synchronize()
        out[f"block_jacobi_{prec}_ms"] = a.elapsed_time(b) / 20
    op.close()
    return out


def _timed_solve(op, n, clock_dev=0, **kw):
    """One dg_solve from x = 0 with wall time and the SM clock sampled during it; returns (stats, x)."""
    import torch

    from paper_1711_10885_gb300 import dg
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    sampler = ClockSampler(clock_dev)
    sampler.start()
    t0 = time.perf_counter()
    st = op.solve(x, raise_on_error=False, **kw)
    torch.cuda.synchronize()
    st["wall_s"] = time.perf_counter() - t0
    st["clocks"] = sampler.stop()
    st["converged"] = st["status"] == dg.DG_OK
    return st, x


def _precond_timing(op, n, reps=20):
    """The block inverse of a set-up handle: what was built (dg_precond_info), the FP32 and FP64 application times
    and the FP32 red-black Gauss-Seidel application time (CUDA events on the current stream, after three
    warm-ups)."""
    import torch

    info, ncx = op.precond_info()
    out = {"info": info, "complex_cells": ncx}
    r = torch.rand(n, dtype=torch.float32, device="cuda") - 0.5
    work = torch.empty_like(r)
    cases = (("fp32_us", r, op.precond_apply), ("fp64_us", r.double(), op.precond_apply),
             ("rbgs_fp32_us", r, lambda v, z: op.precond_apply_rbgs(v, z, work)))
    for name, v, fn in cases:
        z = torch.empty_like(v)
        for _ in range(3):
            fn(v, z)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn(v, z)
        b.record()
        b.synchronize()
        out[name] = a.elapsed_time(b) / reps * 1e3
    return out


def _f32_apply_timing(op, w, reps=20):
    """The FP32 Jacobian apply of the inner solve on this mesh: time per apply (CUDA events, after five warm-ups),
    MDOF/s and the executed-flop rate against the FP32 unit-count peak."""
    import torch

    from paper_1711_10885_gb300 import flops, inputs
    u = torch.tensor(inputs.uniform_u(w.ndof, 2), dtype=torch.float32, device="cuda")
    y = torch.empty_like(u)
    for _ in range(5):
        op.apply_jacobian(u, y)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        op.apply_jacobian(u, y)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    tf = flops.apply_flops_per_dof(w.k, w.n, residual=False) * w.ndof / (ms * 1e-3) / 1e12
    return {"apply_us": ms * 1e3, "mdofs": w.ndof / ms / 1e3, "tflops": tf, "frac_of_fp32_peak": tf / FP32_PEAK_TFLOPS}


def solve_section(fp64_cap_s=100.0, fp64_cap_s_q4=20.0, learned=True):
    """The solve half of the headline metric, in the default line (one GPU):

    q5_48: 48^3 Q5 (23.9 M DOF), log-normal D, 8 sine modes, to 1e-10 relative residual: the mixed-precision
      solve (FP64 outer FGMRES(20), FGMRES(30) with red-black Gauss-Seidel, with the true residual, defect
      update and orthogonalisation in FP64; FP32 inner FGMRES(30) on the FP32 operator) with the FP64 outer operator (the conforming variant) and with the
      double-float outer operator, each with the inner Krylov basis stored in FP32 and in scaled FP16, each with
      block-Jacobi (exact block inverse by fast diagonalisation) and with red-black block Gauss-Seidel; against
      plain FP64 FGMRES(30) with the same preconditioner in FP64, each capped at fp64_cap_s seconds.
    q4_64: 64^3 Q4 (32.8 M DOF), sigma 1.5, to 1e-8: mixed + block-Jacobi and mixed + red-black Gauss-Seidel
      (FP32 and FP16 inner basis), mixed + block-Jacobi + the learned first direction, the network alone in every
      inner application (capped), and plain FP64 with either preconditioner (capped at fp64_cap_s_q4 seconds).
      The network is trained on the solver's own pairs first (timed)."""
    import torch

    from paper_1711_10885_gb300 import dg, inputs, learned as learned_mod
    out = {}
    w = inputs.unit_cube_q5_48(with_u=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    op = dg.operator_for(w)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    op.precond_setup(dg.DG_BJ_FAST_DIAG)
    torch.cuda.synchronize()
    q5 = {"workload": "unit_cube_q5_48", "dofs": w.ndof, "rtol": 1e-10, "operator_setup_s": t1 - t0,
          "precond_setup_s": time.perf_counter() - t1,
          "precond": "block-Jacobi (exact block inverse by fast diagonalisation) or red-black block Gauss-Seidel "
                     "(suffix _rbgs); FP32 in the inner solve, FP64 in the plain solve",
          "block_inverse": _precond_timing(op, w.ndof), "fp32_apply": _f32_apply_timing(op, w)}
    xs = {}
    # each outer operator with the inner Krylov basis stored in FP32 (the default) and in scaled FP16
    variants = (("mixed_fp64_outer", 1, 0), ("mixed_df_outer", 0, 0), ("mixed_fp64_outer_fp16_basis", 1, 1),
                ("mixed_df_outer_fp16_basis", 0, 1))
    # outer restart: 20 with block-Jacobi, 30 with red-black Gauss-Seidel (the faster one for each in
    # --restart-sweep)
    pcs = (("", dg.DG_PRECOND_BLOCK_JACOBI), ("_rbgs", dg.DG_PRECOND_RB_GS))
    for sfx, pc in pcs:
        mo = 30 if pc == dg.DG_PRECOND_RB_GS else 20
        for name, outer, basis in variants:
            st, xs[name + sfx] = _timed_solve(op, w.ndof, mode=dg.DG_SOLVE_MIXED, preconditioner=pc, rtol=1e-10,
                                              inner_rtol=1e-3, restart=30, outer_restart=mo, outer_precision=outer,
                                              inner_basis_precision=basis)
            st["outer_restart"] = mo
            q5[name + sfx] = st
        # plain FP64: its iteration rate first, to turn the time cap into an iteration cap
        st, _ = _timed_solve(op, w.ndof, mode=dg.DG_SOLVE_FP64, preconditioner=pc, rtol=1e-10, max_iterations=60)
        cap = max(60, int(fp64_cap_s / (st["wall_s"] / max(1, st["iterations"]))))
        st, xs["fp64" + sfx] = _timed_solve(op, w.ndof, mode=dg.DG_SOLVE_FP64, preconditioner=pc, rtol=1e-10,
                                            max_iterations=cap)
        st["iteration_cap"] = cap
        q5["fp64" + sfx] = st
        ref = xs["fp64" + sfx]
        for name, _, _ in variants:
            if st["converged"]:
                q5[name + sfx]["field_diff_vs_fp64"] = float((xs[name + sfx] - ref).abs().max() / ref.abs().max())
                q5["speedup_" + name + sfx] = st["wall_s"] / q5[name + sfx]["wall_s"]
            else:
                q5["speedup_lower_bound_" + name + sfx] = st["wall_s"] / q5[name + sfx]["wall_s"]
    conv = [q5["fp64" + sfx]["wall_s"] for sfx, _ in pcs if q5["fp64" + sfx]["converged"]]
    best_mixed = min((q5[name + sfx]["wall_s"], name + sfx) for sfx, _ in pcs for name, _, _ in variants)
    q5["fastest_mixed"] = best_mixed[1]
    if conv:
        q5["speedup_fastest_mixed_vs_fastest_fp64"] = min(conv) / best_mixed[0]
    op.close()
    del xs
    out["q5_48"] = q5
    if not learned:
        return out

    train = [inputs.Workload(f"train{s_}", (32, 32, 32), 4, inputs.log_normal_D(32 ** 3, 1.5, s_))
             for s_ in (10, 11, 12, 13)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mlp, info = learned_mod.train_preconditioner(train, 4, pairs=20000, epochs=60, batch=256, lr=1e-3, seed=0,
                                                 minus_block_jacobi=False)
    torch.cuda.synchronize()
    info["train_s"] = time.perf_counter() - t0
    ev = inputs.Workload("eval", (64, 64, 64), 4, inputs.log_normal_D(64 ** 3, 1.5, 20))
    t0 = time.perf_counter()
    op = dg.operator_for(ev)
    op.precond_setup(dg.DG_BJ_FAST_DIAG)
    torch.cuda.synchronize()
    q4 = {"workload": "64^3 Q4, D log-normal sigma 1.5 (seed 20)", "dofs": ev.ndof, "rtol": 1e-8, "mlp": info,
          "setup_s": time.perf_counter() - t0, "block_inverse": _precond_timing(op, ev.ndof),
          "fp32_apply": _f32_apply_timing(op, ev)}
    common = dict(rtol=1e-8, inner_rtol=1e-2, mlp=mlp)
    for sfx, pc in (("bj", dg.DG_PRECOND_BLOCK_JACOBI), ("rbgs", dg.DG_PRECOND_RB_GS)):
        mo = 30 if pc == dg.DG_PRECOND_RB_GS else 20
        q4["mixed_" + sfx], _ = _timed_solve(op, ev.ndof, mode=dg.DG_SOLVE_MIXED, preconditioner=pc,
                                             outer_restart=mo, **common)
        q4["mixed_" + sfx + "_fp16_basis"], _ = _timed_solve(op, ev.ndof, mode=dg.DG_SOLVE_MIXED, preconditioner=pc,
                                                             outer_restart=mo, inner_basis_precision=1, **common)
        q4["mixed_" + sfx]["outer_restart"] = q4["mixed_" + sfx + "_fp16_basis"]["outer_restart"] = mo
    q4["mixed_bj_learned"], _ = _timed_solve(op, ev.ndof, mode=dg.DG_SOLVE_MIXED,
                                             preconditioner=dg.DG_PRECOND_BJ_MLP, mlp_placement=1, **common)
    q4["mixed_learned_only"], _ = _timed_solve(op, ev.ndof, mode=dg.DG_SOLVE_MIXED,
                                               preconditioner=dg.DG_PRECOND_MLP, max_iterations=30, **common)
    for sfx, pc in (("bj", dg.DG_PRECOND_BLOCK_JACOBI), ("rbgs", dg.DG_PRECOND_RB_GS)):
        st, _ = _timed_solve(op, ev.ndof, mode=dg.DG_SOLVE_FP64, preconditioner=pc, rtol=1e-8, max_iterations=30)
        cap = max(30, int(fp64_cap_s_q4 / (st["wall_s"] / max(1, st["iterations"]))))
        q4["fp64_" + sfx], _ = _timed_solve(op, ev.ndof, mode=dg.DG_SOLVE_FP64, preconditioner=pc, rtol=1e-8,
                                            max_iterations=cap)
        q4["fp64_" + sfx]["iteration_cap"] = cap
    mlp.close()
    op.close()
    out["q4_64"] = q4
    return out


def restart_sweep():
    """Outer restart length of the mixed solve (double-float outer operator, inner FGMRES(30) with the FP16 basis;
    block-Jacobi and red-black Gauss-Seidel, suffix _rbgs): 48^3 Q5 to 1e-10 for 10, 20, 30, 60 and 64^3 Q4
    (sigma 1.5) to 1e-8 for 10, 20, 30; and the plain FP64 FGMRES(60) with block-Jacobi at 48^3 Q5 (the reference
    solve of the bench uses FGMRES(30))."""
    from paper_1711_10885_gb300 import dg, inputs
    out = {}
    cases = (("q5_48", inputs.unit_cube_q5_48(with_u=False), 1e-10, 1e-3, (10, 20, 30, 60)),
             ("q4_64", inputs.Workload("eval", (64, 64, 64), 4, inputs.log_normal_D(64 ** 3, 1.5, 20)), 1e-8, 1e-2,
              (10, 20, 30)))
    for name, w, rtol, itol, restarts in cases:
        op = dg.operator_for(w)
        op.precond_setup(dg.DG_BJ_FAST_DIAG)
        out[name] = {}
        for sfx, pc in (("", dg.DG_PRECOND_BLOCK_JACOBI), ("_rbgs", dg.DG_PRECOND_RB_GS)):
            for mo in restarts:
                st, _ = _timed_solve(op, w.ndof, mode=dg.DG_SOLVE_MIXED, preconditioner=pc, rtol=rtol,
                                     inner_rtol=itol, restart=30, outer_restart=mo, inner_basis_precision=1)
                key = str(mo) + sfx
                out[name][key] = {k: st[k] for k in ("iterations", "inner_iterations", "rel_residual", "wall_s",
                                                     "converged")}
                out[name][key]["sm_mhz"] = st["clocks"].get("sm_mhz")
        if name == "q5_48":  # the plain FP64 reference with a restart of 60 instead of 30
            st, _ = _timed_solve(op, w.ndof, mode=dg.DG_SOLVE_FP64, preconditioner=dg.DG_PRECOND_BLOCK_JACOBI,
                                 rtol=rtol, restart=60, max_iterations=6000)
            out[name]["fp64_restart_60"] = {k: st[k] for k in ("iterations", "rel_residual", "wall_s", "converged")}
        op.close()
    return out


def peak_probes():
    """FP64 FMA, FP64 tensor-core (mma.sync m8n8k4) and FP32 FMA throughput of this GPU (dg_peak_probe), each
    timed with events on the launching stream after a warm-up launch, best of three, with the SM clock."""
    import torch

    from paper_1711_10885_gb300 import dg
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    out = {}
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.2)
    for name, kind, iters in (("dfma", dg.DG_PROBE_DFMA, 25000), ("dmma", dg.DG_PROBE_DMMA, 6000),
                              ("ffma", dg.DG_PROBE_FFMA, 1500000)):
        dg.peak_probe(kind, iters // 10, sink)
        best = None
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fl = dg.peak_probe(kind, iters, sink)
            b.record(stream)
            b.synchronize()
            t = fl / (a.elapsed_time(b) * 1e-3) / 1e12
            best = t if best is None else max(best, t)
        out[name + "_tflops"] = best
    out["clocks"] = sampler.stop()
    out["unit_count_fp64_tflops"] = FP64_PEAK_TFLOPS
    out["unit_count_fp32_tflops"] = FP32_PEAK_TFLOPS
    out["dmma_over_dfma"] = out["dmma_tflops"] / out["dfma_tflops"]
    return out


def f32_degrees(reps=50):
    """FP32 Jacobian apply (the inner operator of the mixed solve) per degree 1..7 at about 24 M DOF: time per apply
    (CUDA events, after five warm-ups), GDOF/s and the executed-flop rate against the FP32 unit-count peak."""
    import torch

    from paper_1711_10885_gb300 import dg, flops, inputs
    out = {}
    for k, n in ((1, 144), (2, 96), (3, 72), (4, 58), (5, 48), (6, 42), (7, 36)):
        w = inputs.Workload("f32", (n, n, n), k, inputs.log_normal_D(n ** 3, 1.0, 1))
        op = dg.Operator(w.n, w.k, w.D, b=w.b, c=w.c)
        u = torch.tensor(inputs.uniform_u(w.ndof, 2), dtype=torch.float32, device="cuda")
        y = torch.empty_like(u)
        for _ in range(5):
            op.apply_jacobian(u, y)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            op.apply_jacobian(u, y)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / reps
        tf = flops.apply_flops_per_dof(k, w.n, residual=False) * w.ndof / (ms * 1e-3) / 1e12
        out[k] = {"cells": n ** 3, "dofs": w.ndof, "apply_us": ms * 1e3, "gdofs": w.ndof / ms / 1e6,
                  "tflops": tf, "frac_of_fp32_peak": tf / FP32_PEAK_TFLOPS}
        op.close()
    return out


def tensor_benchmark(reps=20):
    """The paper's Problem A coefficients (Sec. 5.1: tensor-valued diffusion, constant per cell) on the
    32^3 Q7 workload: per-cell SPD tensors R diag(l) R^T with log-normal eigenvalues (seed 60), b, c, f
    as in the scalar workload; the same mesh with affine (sheared and rotated) cells.  FP64 and
    double-float residual applications."""
    import numpy as np
    import torch

    from paper_1711_10885_gb300 import dg, flops, inputs
    w = inputs.unit_cube_q7_32()
    Dt = inputs.log_normal_tensors(w.ncell, 1.0, 60)
    th = 0.35
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    S = np.array([[1.0, 0.25, -0.15], [0.0, 1.1, 0.3], [0.05, 0.0, 0.9]])
    J = R @ S @ np.diag([1.0 / 32] * 3)
    N = w.k + 1
    cell_fl = flops.cell_kernel_flops_td(N) * w.ncell
    face_fl = flops.face_kernel_flops_td(N) * w.ncell
    stream = torch.cuda.current_stream()
    out = {"workload": "unit_cube_q7_32 with per-cell tensors", "dofs": w.ndof,
           "executed_flops_per_dof": (cell_fl + face_fl) / w.ndof, "paper_flopdof": flops.paper_flopdof(w.k)}
    for name, jac in (("axis_parallel", None), ("affine", J)):
        op = dg.Operator(w.n, w.k, 1.0, b=w.b, c=w.c, D_tensor=Dt, jacobian=jac,
                         f_qp=np.ones(w.ncell * N ** 3))
        u = torch.tensor(w.u, device="cuda")
        r = torch.empty_like(u)
        rec = {}
        for pname, prec in (("f64", dg.DG_F64), ("f64x", dg.DG_F64X)):
            for _ in range(3):
                op.apply_residual(u, r, precision=prec)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * reps)]
            for i in range(reps):
                ev[3 * i].record(stream)
                op.apply_stage(0, u, r, residual=True, precision=prec)
                ev[3 * i + 1].record(stream)
                op.apply_stage(1, u, r, residual=True, precision=prec)
                ev[3 * i + 2].record(stream)
            torch.cuda.synchronize()
            cms = sum(ev[3 * i].elapsed_time(ev[3 * i + 1]) for i in range(reps)) / reps
            fms = sum(ev[3 * i + 1].elapsed_time(ev[3 * i + 2]) for i in range(reps)) / reps
            rec[pname] = {"mdofs": w.ndof / ((cms + fms) * 1e-3) / 1e6,
                          "kernels_ms": {"dg_cell_kernel_td": cms, "dg_face_kernel<td>": fms},
                          "fp64_equivalent_tflops": (cell_fl + face_fl) / ((cms + fms) * 1e-3) / 1e12}
        ach = cell_fl / (rec["f64"]["kernels_ms"]["dg_cell_kernel_td"] * 1e-3) / 1e12
        rec["roofline_f64"] = {"bound": "alu", "kernel": "dg_cell_kernel_td<8, double>", "achieved": ach,
                               "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS}
        out[name] = rec
        op.close()
    return out


def affine_grid_points(n, m, lo, J):
    """Gauss points of the cells lo + J (ic + [0,1]^3): volume [ncell, m^3, 3] (point q = i1 + m (i2 + m i3)) and
    every cell's faces [ncell, 6, m^2, 3] (face 2 dir + side, point pa + m pb over the tangential axes)."""
    import numpy as np
    xi = (np.polynomial.legendre.leggauss(m)[0] + 1.0) / 2.0
    nx, ny, nz = n
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ic = np.stack([ix, iy, iz], axis=-1).reshape(-1, 3).astype(np.float64)
    p3, p2, p1 = np.meshgrid(xi, xi, xi, indexing="ij")
    pts = np.stack([p1, p2, p3], axis=-1).reshape(-1, 3)
    J = np.asarray(J, dtype=np.float64)
    vol = np.asarray(lo) + (ic[:, None, :] + pts[None, :, :]) @ J.T
    pb, pa = np.meshgrid(xi, xi, indexing="ij")
    face_ref = np.empty((6, m * m, 3))
    for face in range(6):
        d, side = face // 2, face % 2
        ta, tb = (1, 2) if d == 0 else ((0, 2) if d == 1 else (0, 1))
        face_ref[face, :, d] = side
        face_ref[face, :, ta] = pa.ravel()
        face_ref[face, :, tb] = pb.ravel()
    faces = np.asarray(lo) + (ic[:, None, None, :] + face_ref[None]) @ J.T
    return vol, faces


def problem_b_benchmark(reps=20, n=32, k=7, seed=70):
    """Problem B of Sec. 5.1 on one GPU: n^3 sheared affine cells of the unit cube's image, Q_k, q = 2p+4
    (m = k+3 Gauss points per direction), D(x) quadratic SPD, b(x) affine, c(x) affine (inputs.PolynomialFields,
    seeded), f = 1, g = 0.  FP64 and double-float residual applications, per-kernel event times."""
    import numpy as np
    import torch

    from paper_1711_10885_gb300 import dg, flops, inputs
    m, N = k + 3, k + 1
    h = np.full(3, 1.0 / n)
    J = inputs.sheared_jacobian(h, seed)
    lo = np.zeros(3)
    fields = inputs.PolynomialFields(seed, lo, J @ np.full(3, float(n)))
    t0 = time.time()
    xv, xf = affine_grid_points((n, n, n), m, lo, J)
    kw = dict(D_qp=fields.D(xv), D_face=fields.D(xf), c_qp=fields.c(xv), velocity="points", b_qp=fields.b(xv),
              b_face=inputs.face_normal_velocity_affine(fields.b, xf, J))
    del xf
    ncell = n ** 3
    op = dg.Operator((n, n, n), k, 1.0, b=(0.0, 0.0, 0.0), c=0.0, m=m, jacobian=J, f_qp=np.ones(ncell * m ** 3),
                     **kw)
    setup_s = time.time() - t0
    del kw, xv
    u = torch.tensor(inputs.uniform_u(op.ndof, seed + 1), device="cuda")
    r = torch.empty_like(u)
    stream = torch.cuda.current_stream()
    cell_fl = flops.cell_kernel_flops_pw(N, m) * ncell
    face_fl = flops.face_kernel_flops_pw(N, m) * ncell
    by = flops.bytes_per_cell_pw(N, m)
    out = {"workload": f"problem_b_q{k}_{n}: {n}^3 sheared cells, k = {k}, m = {m}, polynomial D(x), b(x), c(x)",
           "dofs": op.ndof, "setup_s": setup_s, "executed_flops_per_dof": (cell_fl + face_fl) / op.ndof,
           "algorithmic_bytes_per_dof": (by["cell"] + by["face"]) / N ** 3,
           "paper_problem_b_p7_mdofs_32_cores": 398.0}
    hbm, hbm_src = hbm_peak_gbs()
    for pname, prec in (("f64", dg.DG_F64), ("f64x", dg.DG_F64X)):
        for _ in range(3):
            op.apply_residual(u, r, precision=prec)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * reps)]
        for i in range(reps):
            ev[3 * i].record(stream)
            op.apply_stage(0, u, r, residual=True, precision=prec)
            ev[3 * i + 1].record(stream)
            op.apply_stage(1, u, r, residual=True, precision=prec)
            ev[3 * i + 2].record(stream)
        torch.cuda.synchronize()
        cms = sum(ev[3 * i].elapsed_time(ev[3 * i + 1]) for i in range(reps)) / reps
        fms = sum(ev[3 * i + 1].elapsed_time(ev[3 * i + 2]) for i in range(reps)) / reps
        out[pname] = {"mdofs": op.ndof / ((cms + fms) * 1e-3) / 1e6,
                      "kernels_ms": {"dg_cell_kernel_td<pw>": cms, "dg_face_kernel<td, pw>": fms},
                      "fp64_equivalent_tflops": (cell_fl + face_fl) / ((cms + fms) * 1e-3) / 1e12,
                      "algorithmic_gbs": {"cell": by["cell"] * ncell / (cms * 1e-3) / 1e9,
                                          "face": by["face"] * ncell / (fms * 1e-3) / 1e9,
                                          "peak": hbm, "peak_source": hbm_src}}
    ach = cell_fl / (out["f64"]["kernels_ms"]["dg_cell_kernel_td<pw>"] * 1e-3) / 1e12
    out["roofline_f64"] = {"bound": "alu", "kernel": f"dg_cell_kernel_td<{N}, double, M={m}, pw>", "achieved": ach,
                           "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS}
    op.close()
    return out


def multilinear_grid_points(n, m, verts):
    """Gauss points of the trilinear cells of a vertex grid: volume [ncell, m^3, 3] and every cell's faces
    [ncell, 6, m^2, 3] (the layouts of dg_quadrature_points 0 and 7)."""
    import numpy as np
    xi = (np.polynomial.legendre.leggauss(m)[0] + 1.0) / 2.0
    nx, ny, nz = n
    V = np.asarray(verts, dtype=np.float64).reshape(nz + 1, ny + 1, nx + 1, 3)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    C = np.stack([V[iz + c, iy + b, ix + a] for c in range(2) for b in range(2) for a in range(2)], axis=1)

    def shape(loc):  # [p, 3] local coordinates -> trilinear weights [p, 8] (corner a + 2 b + 4 c)
        return np.stack([(loc[:, 0] if a else 1 - loc[:, 0]) * (loc[:, 1] if b else 1 - loc[:, 1]) *
                         (loc[:, 2] if c else 1 - loc[:, 2]) for c in range(2) for b in range(2) for a in range(2)],
                        axis=1)

    p3, p2, p1 = np.meshgrid(xi, xi, xi, indexing="ij")
    vol = np.einsum("qv,cvd->cqd", shape(np.stack([p1.ravel(), p2.ravel(), p3.ravel()], axis=1)), C)
    pb, pa = np.meshgrid(xi, xi, indexing="ij")
    faces = np.empty((C.shape[0], 6, m * m, 3))
    for face in range(6):
        d, side = face // 2, face % 2
        ta, tb = (1, 2) if d == 0 else ((0, 2) if d == 1 else (0, 1))
        loc = np.empty((m * m, 3))
        loc[:, d], loc[:, ta], loc[:, tb] = side, pa.ravel(), pb.ravel()
        faces[:, face] = np.einsum("pv,cvd->cpd", shape(loc), C)
    return vol, faces


def problem_c_benchmark(reps=20, n=32, k=7, seed=80):
    """Problem C of Sec. 5.1 on one GPU: n^3 multilinear cells of the unit cube (vertices moved by up to 0.2 h,
    inputs.multilinear_vertices), Q_k, m = k+3 Gauss points per direction, D(x) quadratic SPD and c(x) affine
    (inputs.PolynomialFields), constant b, f = 1, g = 0.  FP64 and double-float residual applications."""
    import numpy as np
    import torch

    from paper_1711_10885_gb300 import dg, flops, inputs
    m, N = k + 3, k + 1
    verts = inputs.multilinear_vertices((n, n, n), seed=seed, amplitude=0.2)
    fields = inputs.PolynomialFields(seed, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    t0 = time.time()
    xv, xf = multilinear_grid_points((n, n, n), m, verts)
    kw = dict(D_qp=fields.D(xv), D_face=fields.D(xf), c_qp=fields.c(xv))
    del xv, xf
    ncell = n ** 3
    op = dg.Operator((n, n, n), k, 1.0, b=tuple(fields.b0), c=0.0, m=m, vertices=verts,
                     f_qp=np.ones(ncell * m ** 3), **kw)
    setup_s = time.time() - t0
    del kw
    u = torch.tensor(inputs.uniform_u(op.ndof, seed + 1), device="cuda")
    r = torch.empty_like(u)
    stream = torch.cuda.current_stream()
    cell_fl = flops.cell_kernel_flops_pw(N, m) * ncell
    face_fl = flops.face_kernel_flops_pw(N, m) * ncell
    out = {"workload": f"problem_c_q{k}_{n}: {n}^3 multilinear cells, k = {k}, m = {m}, polynomial D(x), c(x)",
           "dofs": op.ndof, "setup_s": setup_s, "executed_flops_per_dof": (cell_fl + face_fl) / op.ndof}
    for pname, prec in (("f64", dg.DG_F64), ("f64x", dg.DG_F64X)):
        for _ in range(3):
            op.apply_residual(u, r, precision=prec)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * reps)]
        for i in range(reps):
            ev[3 * i].record(stream)
            op.apply_stage(0, u, r, residual=True, precision=prec)
            ev[3 * i + 1].record(stream)
            op.apply_stage(1, u, r, residual=True, precision=prec)
            ev[3 * i + 2].record(stream)
        torch.cuda.synchronize()
        cms = sum(ev[3 * i].elapsed_time(ev[3 * i + 1]) for i in range(reps)) / reps
        fms = sum(ev[3 * i + 1].elapsed_time(ev[3 * i + 2]) for i in range(reps)) / reps
        out[pname] = {"mdofs": op.ndof / ((cms + fms) * 1e-3) / 1e6,
                      "kernels_ms": {"dg_cell_kernel_td<pw>": cms, "dg_face_kernel<td, pw>": fms},
                      "fp64_equivalent_tflops": (cell_fl + face_fl) / ((cms + fms) * 1e-3) / 1e12}
    ach = cell_fl / (out["f64"]["kernels_ms"]["dg_cell_kernel_td<pw>"] * 1e-3) / 1e12
    out["roofline_f64"] = {"bound": "alu", "kernel": f"dg_cell_kernel_td<{N}, double, M={m}, pw>", "achieved": ach,
                           "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS}
    op.close()
    return out


def small_case_latency(replays=1000):
    """The 8^3-cell Q3 unit-cube workload (32 768 DOF; the problem the oracle finishes in milliseconds):
    latency of one FP64 residual apply, launched directly and replayed from a captured CUDA graph (the two
    kernels of the apply); median over `replays` single-apply timings with CUDA events."""
    import statistics as st

    import torch

    from paper_1711_10885_gb300 import dg, inputs
    w = inputs.unit_cube_q3_8()
    op = dg.operator_for(w)
    u = torch.tensor(w.u, device="cuda")
    r = torch.empty_like(u)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            op.apply_residual(u, r, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        op.apply_residual(u, r)
    stream = torch.cuda.current_stream()
    out = {"workload": "unit_cube_q3_8", "dofs": w.ndof}
    for name, fn in (("direct", lambda: op.apply_residual(u, r)), ("graph", graph.replay)):
        for _ in range(10):
            fn()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * replays)]
        for i in range(replays):
            ev[2 * i].record(stream)
            fn()
            ev[2 * i + 1].record(stream)
        torch.cuda.synchronize()
        lat = st.median(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(replays))
        out[name] = {"median_us": lat * 1e3, "mdofs": w.ndof / (lat * 1e-3) / 1e6}
    op.close()
    return out


def mlp_forward_benchmark(rows=262144, k=4, reps=20):
    """Inference of the learned preconditioner's network (132 -> 256 -> 256 -> 125 at k = 4, BF16 operands,
    FP32 accumulation) on `rows` feature rows (64^3 cells): the tcgen05 kernel (tensor memory accumulators)
    against the mma.sync kernel, with the dense flops 2 (kinp 256 + 256^2 + 256 outp) per row."""
    import numpy as np
    import torch

    from paper_1711_10885_gb300 import dg
    mlp = dg.MLP(k, seed=7)
    X = torch.randn(rows, mlp.kinp, device="cuda").to(torch.bfloat16)
    Y = torch.empty(rows, mlp.outp, device="cuda")
    flop = 2.0 * rows * (mlp.kinp * 256 + 256 * 256 + 256 * mlp.outp)
    stream = torch.cuda.current_stream()
    peak = 1937.5
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
    except Exception:
        pass
    out = {"rows": rows, "k": k, "gflop_per_forward": flop / 1e9}
    for name, env in (("tcgen05", None), ("mma_sync", "1")):
        if env:
            os.environ["DG_MLP_NO_TCGEN05"] = env
        try:
            for _ in range(3):
                mlp.forward(X)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                mlp.forward(X)
            b.record(stream)
            b.synchronize()
        finally:
            os.environ.pop("DG_MLP_NO_TCGEN05", None)
        ms = a.elapsed_time(b) / reps
        out[name] = {"ms": ms, "tflops": flop / (ms * 1e-3) / 1e12, "frac_of_bf16_peak": flop / (ms * 1e-3) / 1e12 / peak}
    out["peak_bf16_tflops"] = peak
    mlp.close()
    return out


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of this GPU pool (MEASURED_PEAKS.json), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def matrix_benchmark(reps=20, degrees=(1, 3, 5, 7)):
    """Matrix-free vs matrix-based application (Sec. 5.2 table): per degree, the operator's block-sparse
    matrix is assembled on a mesh whose matrix takes 3-40 GB of HBM, and its product is timed next
    to the matrix-free FP64 (and double-float) application on a ~17-24 M DOF mesh of the same workload
    family (per-cell log-normal D, b = (1, .5, .25), c = 1).  The matrix-based meshes are smaller, as in
    the paper, because the matrix has 7 (k+1)^6 entries per cell."""
    import torch

    from paper_1711_10885_gb300 import dg, inputs
    peak, peak_src = hbm_peak_gbs()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps

    n_mat = {1: 96, 2: 64, 3: 48, 4: 32, 5: 24, 6: 18, 7: 14}  # matrices of 3-40 GB, >= 2744 block rows
    n_free = {1: 128, 2: 96, 3: 64, 4: 56, 5: 48, 6: 40, 7: 32}
    out = {"hbm_peak_gbs": peak, "hbm_peak_source": peak_src, "degrees": {}}
    for k in degrees:
        nb = (k + 1) ** 3
        wm = inputs.small_case(n=(n_mat[k],) * 3, k=k, seed=200 + k)
        op = dg.operator_for(wm)
        A = dg.Matrix(op)
        x = torch.tensor(wm.u, device="cuda")
        y = torch.empty_like(x)
        ms_spmv = timed(lambda: A.spmv(x, y))
        bytes_spmv = A.nnzb * nb * nb * 8 + A.nnzb * nb * 8 + wm.ndof * 8 + (A.nrows + 1 + A.nnzb) * 4
        check = float((y - op.apply_jacobian(x)).abs().max() / op.apply_jacobian(x).abs().max())
        rec = {"matrix_mesh": [n_mat[k]] * 3, "matrix_dofs": wm.ndof, "matrix_gb": A.nnzb * nb * nb * 8 / 1e9,
               "assembly_s": A.assemble_seconds, "assembly_mdofs": wm.ndof / A.assemble_seconds / 1e6,
               "spmv_ms": ms_spmv, "spmv_mdofs": wm.ndof / (ms_spmv * 1e-3) / 1e6,
               "spmv_gbs": bytes_spmv / (ms_spmv * 1e-3) / 1e9, "spmv_hbm_frac": bytes_spmv / (ms_spmv * 1e-3) / 1e9 / peak,
               "spmv_vs_apply_rel": check}
        A.close()
        op.close()
        del x, y
        wf = inputs.small_case(n=(n_free[k],) * 3, k=k, seed=300 + k)
        op = dg.operator_for(wf)
        x = torch.tensor(wf.u, device="cuda")
        y = torch.empty_like(x)
        ms64 = timed(lambda: op.apply_jacobian(x, y))
        msx = timed(lambda: op.apply_jacobian(x, y, precision=dg.DG_F64X))
        rec.update({"free_mesh": [n_free[k]] * 3, "free_dofs": wf.ndof,
                    "free_f64_mdofs": wf.ndof / (ms64 * 1e-3) / 1e6, "free_f64x_mdofs": wf.ndof / (msx * 1e-3) / 1e6})
        rec["speedup_f64_over_matrix"] = rec["free_f64_mdofs"] / rec["spmv_mdofs"]
        rec["speedup_f64x_over_matrix"] = rec["free_f64x_mdofs"] / rec["spmv_mdofs"]
        out["degrees"][k] = rec
        op.close()
    out["paper_context"] = ("2x Xeon E5-2698v3, 32 cores (Sec. 5.2 table): p=7 matrix-free A 570 MDOF/s, "
                            "matrix-based 1.46 MDOF/s (x390), assembly 0.66 MDOF/s; p=1: 170 vs 206 MDOF/s")
    return out


def batch_benchmark(reps=20):
    """64 uneven problems (n ~ U{4..24}, k ~ U{2..8}, seed 5): one graph launch vs the standalone applies."""
    import torch

    from paper_1711_10885_gb300 import dg, inputs
    ws = inputs.batch_problems(64, seed=5)
    ops = [dg.operator_for(w) for w in ws]
    xs = [torch.tensor(w.u, device="cuda") for w in ws]
    ys = [torch.empty_like(x) for x in xs]
    t0 = time.perf_counter()
    batch = dg.Batch(ops)
    tune_s = time.perf_counter() - t0
    dofs = sum(w.ndof for w in ws)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps

    def standalone():
        for op, x, y in zip(ops, xs, ys):
            op.apply_jacobian(x, y)

    ms_batch = timed(lambda: batch.apply(xs, ys))
    ms_alone = timed(standalone)
    out = {"problems": len(ws), "dofs": dofs, "graph_launch_ms": ms_batch, "standalone_sum_ms": ms_alone,
           "batch_mdofs": dofs / (ms_batch * 1e-3) / 1e6, "standalone_mdofs": dofs / (ms_alone * 1e-3) / 1e6,
           "speedup": ms_alone / ms_batch, "autotune_s": tune_s,
           "tuning": {k: batch.tuning(k) for k in sorted({w.k for w in ws})},
           "candidates": "0: F cells/CTA x 1 line/thread (standalone layout), 1: F/2 x 1, 2: F x 2, 3: 2F x 2; "
                         "F = floor(256 / (k+1)^2)"}
    batch.close()
    for op in ops:
        op.close()
    return out


def learned_benchmark(rtol=1e-8, fp64_cap_s=60.0, pairs=20000, epochs=60):
    """Learned preconditioner at 64^3 Q4 (32.8M DOF, sigma 1.5, seed 20), trained on four 32^3 Q4 meshes
    (seeds 10..13): time to rtol for plain FP64 block-Jacobi FGMRES(30) (capped), the same with the learned
    first direction per cycle, and the mixed-precision solve with and without it."""
    import torch

    from paper_1711_10885_gb300 import dg, inputs, learned
    train = [inputs.Workload(f"train{s}", (32, 32, 32), 4, inputs.log_normal_D(32 ** 3, 1.5, s)) for s in
             (10, 11, 12, 13)]
    t0 = time.perf_counter()
    mlp, info = learned.train_preconditioner(train, 4, pairs=pairs, epochs=epochs, batch=256, lr=1e-3, seed=0,
                                             minus_block_jacobi=False)
    torch.cuda.synchronize()
    info["train_s"] = time.perf_counter() - t0
    ev = inputs.Workload("eval", (64, 64, 64), 4, inputs.log_normal_D(64 ** 3, 1.5, 20))
    op = dg.operator_for(ev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    op.precond_setup()
    torch.cuda.synchronize()
    out = {"workload": "64^3 Q4, D log-normal sigma 1.5", "dofs": ev.ndof, "rtol": rtol, "mlp": info,
           "precond_setup_s": time.perf_counter() - t0}
    # FP64 iteration rate, to cap the plain FP64 solve at about fp64_cap_s seconds
    x = torch.zeros(ev.ndof, dtype=torch.float64, device="cuda")
    st = op.solve(x, mode=dg.DG_SOLVE_FP64, preconditioner=dg.DG_PRECOND_BLOCK_JACOBI, rtol=rtol, max_iterations=30,
                  raise_on_error=False)
    cap = max(30, int(fp64_cap_s / (st["seconds"] / 30)))
    runs = (("fp64_bj", dg.DG_SOLVE_FP64, dg.DG_PRECOND_BLOCK_JACOBI, cap),
            ("fp64_bj_learned", dg.DG_SOLVE_FP64, dg.DG_PRECOND_BJ_MLP, cap),
            ("mixed_bj", dg.DG_SOLVE_MIXED, dg.DG_PRECOND_BLOCK_JACOBI, 0),
            ("mixed_bj_learned", dg.DG_SOLVE_MIXED, dg.DG_PRECOND_BJ_MLP, 0))
    for name, mode, pc, maxit in runs:
        x = torch.zeros(ev.ndof, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = op.solve(x, mode=mode, preconditioner=pc, mlp=mlp, mlp_placement=1, rtol=rtol, inner_rtol=1e-2,
                      max_iterations=maxit, raise_on_error=False)
        torch.cuda.synchronize()
        st["wall_s"] = time.perf_counter() - t0
        out[name] = st
    mlp.close()
    op.close()
    return out


def transport_benchmark(n=64, k=5, steps=10, warmup=3):
    """The transport example of Sec. 5.3 at single-GPU scale: Taylor-Green flow on the periodic cube
    (-pi, pi)^3, D = 5e-6, c = f = 0, q = 2p+4 (m = k+3 Gauss points), Heun's method from the projected
    Gaussian bump.  One step = two Runge-Kutta stages = two operator applications with the stage update
    fused into the face kernel (dg_ssprk2).  Timed with the FP64 operator and with the double-float one
    (FP64 vectors and FP64 stage updates, operator on the FP32 pipes)."""
    import numpy as np
    import torch

    from paper_1711_10885_gb300 import dg, flops, inputs
    w = inputs.taylor_green(n, k)
    t0 = time.time()
    op = dg.operator_for(w)
    setup_s = time.time() - t0
    xi = (np.polynomial.legendre.leggauss(w.m)[0] + 1.0) / 2.0
    u0 = inputs.gaussian_bump_grid(w, xi, xp=torch, device="cuda")
    z0 = op.project(u0.contiguous())
    del u0
    stream = torch.cuda.current_stream()
    h = 2 * np.pi / n
    dt = 0.3 * h / (2 * k + 1)  # CFL with max |b| = 1
    mass0 = z0.view(w.ncell, -1)[:, 0].sum().item()
    N, M = k + 1, w.m
    cell_fl = flops.cell_kernel_flops(N, M, vb=True) * w.ncell
    face_fl = flops.face_kernel_flops(N, M=M, stage=True) * w.ncell
    out = {"workload": w.name, "cells": [n, n, n], "k": k, "m": M, "dofs": w.ndof, "dt": dt,
           "executed_flops_per_dof_stage": (cell_fl + face_fl) / w.ndof}
    finals = {}
    for name, prec in (("f64", dg.DG_F64), ("f64x", dg.DG_F64X)):
        z = z0.clone()
        op.ssprk2(z, dt, warmup, precision=prec)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        op.ssprk2(z, dt, steps, precision=prec)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        mass1 = z.view(w.ncell, -1)[:, 0].sum().item()
        # per-kernel times of one operator application (cell kernel; face kernel with the residual epilogue)
        r = torch.empty_like(z)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * steps)]
        for i in range(steps):
            ev[3 * i].record(stream)
            op.apply_stage(0, z, r, residual=True, precision=prec)
            ev[3 * i + 1].record(stream)
            op.apply_stage(1, z, r, residual=True, precision=prec)
            ev[3 * i + 2].record(stream)
        torch.cuda.synchronize()
        cell_ms = sum(ev[3 * i].elapsed_time(ev[3 * i + 1]) for i in range(steps)) / steps
        face_ms = sum(ev[3 * i + 1].elapsed_time(ev[3 * i + 2]) for i in range(steps)) / steps
        finals[name] = z
        out[name] = {"ms_per_heun_step": ms, "heun_steps_per_s": 1e3 / ms,
                     "mdofs_per_stage": 2 * w.ndof / (ms * 1e-3) / 1e6,
                     "mdof_steps_per_s": w.ndof / (ms * 1e-3) / 1e6,
                     "kernels_ms": {"dg_cell_kernel<vb>": cell_ms, "dg_face_kernel<vb>": face_ms},
                     "fp64_equivalent_tflops": 2 * (cell_fl + face_fl) / (ms * 1e-3) / 1e12,
                     "mass_drift_rel": abs(mass1 - mass0) / abs(mass0),
                     "finite": bool(torch.isfinite(z).all().item())}
    cms = out["f64"]["kernels_ms"]["dg_cell_kernel<vb>"]
    achieved = cell_fl / (cms * 1e-3) / 1e12
    out["roofline_f64"] = {"bound": "alu", "kernel": "dg_cell_kernel<double, M=8, VB>", "achieved": achieved,
                           "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                           "flops_per_launch": cell_fl}
    out["f64x_vs_f64_after_steps"] = float(((finals["f64x"] - finals["f64"]).abs().max()
                                            / finals["f64"].abs().max()).item())
    out["setup_s"] = setup_s
    out["paper_context"] = ("240^3 p=5 (3e9 DOF), 165000 steps in 143000 core-h on 6144 cores incl. I/O "
                            "(Sec. 5.3): about 5.9e3 MDOF-steps/s for that machine")
    op.close()
    return out


def run_ours(args):
    import numpy as np
    import torch

    from paper_1711_10885_gb300 import dg, flops, inputs

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    w = inputs.unit_cube_q7_32()
    op = dg.operator_for(w)
    u = torch.tensor(w.u, device=dev)
    r = torch.empty_like(u)
    N = w.k + 1

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        op.apply_residual(u, r)
    barrier()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        op.apply_residual(u, r)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    # per-kernel durations on the launching stream (same kernels, same launch configuration)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * args.steps)]
    for i in range(args.steps):
        ev[3 * i].record(stream)
        op.apply_stage(0, u, r, residual=True)
        ev[3 * i + 1].record(stream)
        op.apply_stage(1, u, r, residual=True)
        ev[3 * i + 2].record(stream)
    barrier()
    cell_ms = sum(ev[3 * i].elapsed_time(ev[3 * i + 1]) for i in range(args.steps)) / args.steps
    face_ms = sum(ev[3 * i + 1].elapsed_time(ev[3 * i + 2]) for i in range(args.steps)) / args.steps
    clocks = sampler.stop() if sampler else None

    # end to end through the C ABI with host buffers: every step copies its input u from pinned host memory,
    # applies the operator and copies its result r back.  Serial: one stream.  Pipelined (the "e2e" figure):
    # two device buffer sets and three streams, so that step i+1's H2D copy and step i-1's D2H copy overlap
    # step i's apply.
    u_h = torch.tensor(w.u).pin_memory()
    r_hs = [torch.empty_like(u_h).pin_memory() for _ in range(2)]
    for _ in range(2):
        u.copy_(u_h, non_blocking=True)
        op.apply_residual(u, r)
        r_hs[0].copy_(r, non_blocking=True)
    barrier()
    e2e_steps = max(3, min(args.steps, 50))
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(e2e_steps):
        u.copy_(u_h, non_blocking=True)
        op.apply_residual(u, r)
        r_hs[0].copy_(r, non_blocking=True)
    e3.record(stream)
    barrier()
    e2e_serial_ms = e2.elapsed_time(e3) / e2e_steps
    u_ds, r_ds = [u, torch.empty_like(u)], [r, torch.empty_like(r)]
    s_in, s_op, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

    def pipelined(nsteps):
        done = [torch.cuda.Event() for _ in range(2)]      # apply of the buffer set finished
        copied = [torch.cuda.Event() for _ in range(2)]    # its input is on the device
        fetched = [torch.cuda.Event() for _ in range(2)]   # its result is on the host
        for i in range(nsteps):
            b = i % 2
            if i >= 2:
                s_in.wait_event(done[b])
            with torch.cuda.stream(s_in):
                u_ds[b].copy_(u_h, non_blocking=True)
            copied[b].record(s_in)
            s_op.wait_event(copied[b])
            if i >= 2:
                s_op.wait_event(fetched[b])
            op.apply_residual(u_ds[b], r_ds[b], stream=s_op)
            done[b].record(s_op)
            s_out.wait_event(done[b])
            with torch.cuda.stream(s_out):
                r_hs[b].copy_(r_ds[b], non_blocking=True)
            fetched[b].record(s_out)
        return fetched

    for st_ in (s_in, s_op, s_out):
        st_.wait_stream(stream)
    pipelined(4)
    barrier()
    e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e4.record(stream)
    for st_ in (s_in, s_op, s_out):
        st_.wait_stream(stream)
    last = pipelined(e2e_steps)
    for ev_ in last:
        stream.wait_event(ev_)
    e5.record(stream)
    barrier()
    e2e_ms = e4.elapsed_time(e5) / e2e_steps

    # other precisions / operations of the same path, reported alongside
    extra = {}
    for name, fn, x in (("jacobian_f64", op.apply_jacobian, u), ("residual_f32", op.apply_residual, u.float()),
                        ("residual_f64x", lambda a_, b_: op.apply_residual(a_, b_, precision=dg.DG_F64X), u)):
        y = torch.empty_like(x)
        for _ in range(3):
            fn(x, y)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(20):
            fn(x, y)
        b.record(stream)
        b.synchronize()
        extra[name + "_mdofs"] = w.ndof * 20 / (a.elapsed_time(b) * 1e-3) / 1e6

    # double-float (DG_F64X) per-kernel times on the launching stream
    evx = [torch.cuda.Event(enable_timing=True) for _ in range(3 * args.steps)]
    for i in range(args.steps):
        evx[3 * i].record(stream)
        op.apply_stage(0, u, r, residual=True, precision=dg.DG_F64X)
        evx[3 * i + 1].record(stream)
        op.apply_stage(1, u, r, residual=True, precision=dg.DG_F64X)
        evx[3 * i + 2].record(stream)
    barrier()
    xcell_ms = sum(evx[3 * i].elapsed_time(evx[3 * i + 1]) for i in range(args.steps)) / args.steps
    xface_ms = sum(evx[3 * i + 1].elapsed_time(evx[3 * i + 2]) for i in range(args.steps)) / args.steps

    ms, e2e_ms, e2e_serial_ms = dist_max([ms, e2e_ms, e2e_serial_ms])
    if rank != 0:
        torch.distributed.destroy_process_group()
        return

    mdofs = job_mdofs(ws, w.ndof, args.steps, ms)
    cell_fl = flops.cell_kernel_flops(N) * w.ncell
    face_fl = flops.face_kernel_flops(N, w.n, residual=True) * w.ncell
    dominant = ("dg_cell_kernel", cell_fl, cell_ms) if cell_ms >= face_ms else ("dg_face_kernel", face_fl, face_ms)
    achieved = dominant[1] / (dominant[2] * 1e-3) / 1e12
    src_hash = kernel_source_hash()
    traffic = NCU_TRAFFIC.get((dominant[0], src_hash))
    line = {
        "metric": "DG FP64 residual apply throughput, 32^3 cells Q7 (16.8M DOF)",
        "value": mdofs, "unit": "MDOF/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "unit_cube_q7_32", "cells": [32, 32, 32], "k": 7, "dofs": w.ndof,
                   "D": "log-normal sigma 1 per cell", "b": list(w.b), "c": w.c, "penalty": "2k(k+1)/h",
                   "l2": "inputs larger than L2 (u, r 134 MB; work 335 MB), no flush",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "alu", "kernel": dominant[0], "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                     "peak_source": f"{UNIT_SMS} SMs x 2 FP64 FMA/clk x 2 x {UNIT_MHZ:.0f} MHz (unit counts and "
                                    "max clock)",
                     "flops_per_launch": dominant[1]},
        "kernels_ms": {"dg_cell_kernel": cell_ms, "dg_face_kernel": face_ms},
        "executed_flops_per_dof": (cell_fl + face_fl) / w.ndof,
        "paper_flopdof": flops.paper_flopdof(w.k),
        "fp64_tflops_executed": (cell_fl + face_fl) / (ms / args.steps * 1e-3) / 1e12,
        "e2e": {"value": job_mdofs(ws, w.ndof, 1, e2e_ms), "unit": "MDOF/s", "h2d_bytes_per_step": 8 * w.ndof,
                "d2h_bytes_per_step": 8 * w.ndof,
                "how": "pipelined: step i+1's H2D and step i-1's D2H overlap step i's apply (3 streams, 2 buffer "
                       "sets)", "serial_value": job_mdofs(ws, w.ndof, 1, e2e_serial_ms)},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
        "extra": extra,
        "f64x": {
            "what": "FP64 vectors, operator in double-float (FP32 pairs) arithmetic; parity <= 1e-12 vs the FP64 oracle",
            "mdofs": extra["residual_f64x_mdofs"],
            "kernels_ms": {"dg_cell_kernel<dfl>": xcell_ms, "dg_face_kernel<dfl>": xface_ms},
            "fp64_equivalent_tflops": (cell_fl + face_fl) / ((xcell_ms + xface_ms) * 1e-3) / 1e12,
            # FP32 lane instructions per cell (FADD + FFMA + FMUL, ncu counters of the current kernels)
            "fp32_issue_frac_cell_kernel": F64X_FP32_INST_PER_CELL["cell"] * w.ncell / (xcell_ms * 1e-3)
                                           / (FP32_PEAK_TFLOPS * 1e12 / 2),
            "fp32_issue_frac_face_kernel": F64X_FP32_INST_PER_CELL["face"] * w.ncell / (xface_ms * 1e-3)
                                           / (FP32_PEAK_TFLOPS * 1e12 / 2),
        },
    }
    if ws == 1:
        line["peaks"] = peak_probes()
        line["roofline"]["peak_measured_dfma"] = line["peaks"]["dfma_tflops"]
        line["roofline"]["frac_of_measured_dfma"] = achieved / line["peaks"]["dfma_tflops"]
    if ws == 1:
        line["small_case_latency"] = small_case_latency()
    if ws == 1:
        line["mlp_forward"] = mlp_forward_benchmark()
    if ws == 1 and not args.no_batch:
        line["batch"] = batch_benchmark()
    if ws == 1 and not args.no_transport:
        line["transport"] = transport_benchmark()
    if ws == 1 and not args.no_matrix:
        line["matrix_based"] = matrix_benchmark(degrees=(3, 7))
    if ws == 1 and not args.no_tensor:
        line["tensor_diffusion"] = tensor_benchmark()
    if ws == 1 and not args.no_problem_b:
        line["problem_b"] = problem_b_benchmark()
        line["problem_c"] = problem_c_benchmark()
    if ws == 1 and not args.no_solve:
        line["solve"] = solve_section(learned=not args.no_learned)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)
    op.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="skip the solve comparisons of the default line")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner part of them")
    ap.add_argument("--solve-section", action="store_true", help="print only the default line's solve section")
    ap.add_argument("--restart-sweep", action="store_true",
                    help="print only the mixed solves (double-float outer operator, FP16 inner basis) at 48^3 Q5 and "
                         "64^3 Q4 for several outer restart lengths")
    ap.add_argument("--peaks", action="store_true", help="print only the arithmetic throughput probes")
    ap.add_argument("--f32", action="store_true", help="with --profile: W + K FP32 applies at 48^3 Q5")
    ap.add_argument("--f32-degrees", action="store_true", help="print only the FP32 apply per degree")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-problem batched-apply comparison")
    ap.add_argument("--no-transport", action="store_true", help="skip the Taylor-Green transport section")
    ap.add_argument("--no-matrix", action="store_true", help="skip the matrix-based comparison section")
    ap.add_argument("--no-tensor", action="store_true", help="skip the tensor-diffusion / affine section")
    ap.add_argument("--tensor", action="store_true", help="print only the tensor-diffusion / affine section")
    ap.add_argument("--no-problem-b", action="store_true",
                    help="skip the Problem B (point-wise coefficients) and Problem C (multilinear cells) sections")
    ap.add_argument("--mlp-forward", action="store_true", help="print only the network inference timing")
    ap.add_argument("--small", action="store_true", help="with --profile: W + K applies of the 8^3 Q3 workload")
    ap.add_argument("--problem-c", type=int, default=None, metavar="N",
                    help="print only the Problem C section on N^3 multilinear cells (k = 7, m = 10)")
    ap.add_argument("--problem-b", type=int, default=None, metavar="N",
                    help="print only the Problem B section on N^3 cells (k = 7, m = 10); with --profile: only "
                         "W + K residual applies of it")
    ap.add_argument("--matrix", action="store_true",
                    help="print only the matrix-free vs matrix-based comparison for k = 1, 3, 5, 7; with --profile: "
                         "assemble on --matrix-n^3 cells of degree --matrix-k and run W + K products")
    ap.add_argument("--matrix-k", type=int, default=7)
    ap.add_argument("--matrix-n", type=int, default=8)
    ap.add_argument("--transport", type=int, default=None, metavar="N",
                    help="print only the Taylor-Green transport benchmark on N^3 cells (k = 5, m = 8); with "
                         "--profile: only W + K Heun steps of it")
    ap.add_argument("--solve-only", nargs="?", const="all", default=None, choices=["all", "mixed", "learned"],
                    help="print the solver comparisons only (mixed precision at 48^3 Q5, learned at 64^3 Q4)")
    ap.add_argument("--no-fp64-solve", action="store_true",
                    help="with --solve-only mixed: skip the plain FP64 reference solve (about two minutes)")
    ap.add_argument("--profile-solver", action="store_true",
                    help="with --profile: block-Jacobi and network applications at 48^3 Q5 instead")
    ap.add_argument("--precision", default="f64", choices=["f64", "f64x", "f32"],
                    help="precision of the --profile applies")
    ap.add_argument("--profile", action="store_true",
                    help="only run warmup + steps residual applies (for ncu launch lists and captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl != "reference":
        set_unit_peaks(int(os.environ.get("LOCAL_RANK", "0")))
    if args.impl == "reference":
        run_reference(args)
    elif args.profile:
        run_profile(args)
    elif args.matrix:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"matrix_based": matrix_benchmark()}), flush=True)
    elif args.tensor:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"tensor_diffusion": tensor_benchmark()}), flush=True)
    elif args.problem_b:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"problem_b": problem_b_benchmark(n=args.problem_b)}), flush=True)
    elif args.mlp_forward:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"mlp_forward": mlp_forward_benchmark()}), flush=True)
    elif args.problem_c:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"problem_c": problem_c_benchmark(n=args.problem_c)}), flush=True)
    elif args.transport:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"transport": transport_benchmark(n=args.transport, steps=args.steps,
                                                           warmup=args.warmup)}), flush=True)
    elif args.restart_sweep:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"restart_sweep": restart_sweep()}), flush=True)
    elif args.solve_section:
        import torch
        torch.cuda.set_device(0)
        t0 = time.perf_counter()
        out = solve_section(learned=not args.no_learned)
        print(json.dumps({"solve": out, "section_s": time.perf_counter() - t0}), flush=True)
    elif args.peaks:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"peaks": peak_probes()}), flush=True)
    elif args.f32_degrees:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"f32_degrees": f32_degrees()}), flush=True)
    elif args.solve_only:
        import torch
        torch.cuda.set_device(0)
        if args.solve_only in ("all", "mixed"):
            print(json.dumps({"mixed_precision_q5_48": solve_benchmark(with_fp64=not args.no_fp64_solve)}),
                  flush=True)
        if args.solve_only in ("all", "learned"):
            print(json.dumps({"learned_q4_64": learned_benchmark()}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
