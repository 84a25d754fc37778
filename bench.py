#!/usr/bin/env python
"""Benchmark of the block r1-sparse Jacobian hot path; prints ONE JSON line.

One step is one pass of the whole path over the 128 x 128, N = 60 (b = 63)
workload, FP64, inputs resident in HBM:
  update_values (repack S, U, V)  -> SMW block-Jacobi setup
  -> OPS x matvec y = J x         -> OPS x block-Jacobi apply z = M x
  -> one J^T x and one M^T x      -> GMRES(30) to 1e-10 (FP64)
  -> flexible GMRES(30) to 1e-10 with FP32 operators (mixed)
  -> adjoint GMRES on J^T and the gradient outer products.
``value`` = FP64 matvecs + FP64 block-Jacobi applies executed in a step (the
explicit loops plus those inside the FP64 and adjoint solves) / step time.
FP32 operator calls of the mixed solve are not counted.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
With N > 1 (torchrun) every rank runs an independent replica of the same
workload on its own GPU (no data-path collective): weak scaling.
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
sys.path.insert(0, ROOT)

METRIC = "Jacobian matvecs/s + block-Jacobi applies/s (HBM % peak) vs dense BSR, same GPU"
UNIT = "ops/s"
WORKLOAD = "grid128_N60"
N_SMS = 152
FP64_FMA_PER_CLK_PER_SM = 2          # GB300: measured 0.594 T FMA/s at 1.98 GHz on 152 SMs
L2_BYTES = 135528448


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


def _traffic_record():
    """ncu DRAM bytes per sts_jac_matvec call, valid only for the kernel source it was taken on."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic_grid128_N60.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            rec[k.strip()] = v.strip()
    src = open(os.path.join(ROOT, "paper_2403_09198_gb300", "csrc", "kernels_matvec.cu"), "rb").read()
    if rec.get("kernels_matvec_sha256") != hashlib.sha256(src).hexdigest():
        return None
    try:
        return float(rec["dram_bytes_per_matvec"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for name, val in zip(names, r[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_elapsed(elapsed: float, device) -> float:
    """Max over ranks of a per-rank elapsed time; unchanged in a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return elapsed
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(w, seconds: float, max_pairs: int = 2000):
    """Time the FP64 oracle (as it stands) on the host cores: (matvec, block-Jacobi
    apply) pairs of the same workload until about ``seconds`` have elapsed;
    the block factors are set up once, untimed."""
    import numpy as np
    import oracle
    J = oracle.Jacobian.from_workload(w)
    F = oracle.bj_setup(J)
    x = np.random.default_rng(0).standard_normal(w.n)
    t0 = time.perf_counter()
    pairs = 0
    while pairs < max_pairs and (pairs == 0 or time.perf_counter() - t0 < seconds):
        oracle.matvec(J, x)
        oracle.bj_apply(F, x)
        pairs += 1
    dt = time.perf_counter() - t0
    return 2 * pairs / dt, dt, oracle.max_threads(), pairs


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores, same metric and unit."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_2403_09198_gb300 import inputs
    oracle.build()
    w = inputs.named_workload(WORKLOAD)
    import numpy as np
    J = oracle.Jacobian.from_workload(w)
    F = oracle.bj_setup(J)
    x = np.random.default_rng(0).standard_normal(w.n)

    def step():
        oracle.matvec(J, x)
        oracle.bj_apply(F, x)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = 2 * args.steps / dt
    sample = (f"per step 1 dense-block matvec + 1 dense-LU block-Jacobi apply of {WORKLOAD} "
              f"(factors set up once, untimed)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(w):
    return {"workload": f"{WORKLOAD}: 128x128 cells, N=60 levels, b=63, band +-2, "
                        f"2 pairs per diagonal block, 1 per neighbour block, seed 1",
            "n_cells": w.n_cells, "N": w.N, "b": w.b, "nnz_S": int(w.S.shape[0]),
            "n_pairs": w.n_pairs, "l2": "inputs larger than L2 (425 MB per matvec, 137 MB per apply)"}


def run_ours(args):
    import numpy as np
    import torch
    import __graft_entry__
    from paper_2403_09198_gb300 import binding, inputs
    from paper_2403_09198_gb300.binding import StsJacobian

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    __graft_entry__.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    w = inputs.named_workload(WORKLOAD)
    n = w.n
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    S, U, V, b, Wd = t(w.S), t(w.U), t(w.V), t(w.rhs), t(w.W)
    # component-major vectors for the explicit loops (the kernels' own layout)
    jac = StsJacobian(w, S, U, V, layout="component", transpose=True, mixed=True)
    stream = torch.cuda.current_stream()
    xv = torch.randn(n, dtype=torch.float64, device=dev)
    y = torch.empty_like(xv)
    z = torch.empty_like(xv)
    ops = args.ops
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    per = {"mv": [], "ap": []}
    counted = {}

    def step(record=False, values=None):
        # the step's Jacobian values: device-resident, or host arrays in the
        # end-to-end leg (copied in by update_values)
        jac.update_values(*(values if values is not None else (S, U, V)))
        jac.bjacobi_setup()
        ev[0].record(stream)
        for _ in range(ops):
            jac.matvec(xv, out=y)
        ev[1].record(stream)
        for _ in range(ops):
            jac.bjacobi_apply(xv, out=z)
        ev[2].record(stream)
        jac.matvec(xv, out=y, trans=True)
        jac.bjacobi_apply(xv, out=z, trans=True)
        xs, i64 = jac.gmres(b, rtol=1e-10, restart=30)
        xm, imx = jac.gmres(b, rtol=1e-10, restart=30, mixed=True)
        lam, iad = jac.gmres(Wd * Wd * xs, rtol=1e-10, restart=30, trans=True)
        g = jac.grad(lam, xs)
        if record:
            torch.cuda.synchronize()
            per["mv"].append(ev[0].elapsed_time(ev[1]) / ops)
            per["ap"].append(ev[1].elapsed_time(ev[2]) / ops)
        # FP64 operator calls of the step: explicit loops, one J^T and one M^T,
        # and the FP64 products and applies each solve reports (the mixed solve's
        # FP32 operators are not counted)
        mv = ops + 1 + i64.matvecs + iad.matvecs + imx.matvecs
        ap = ops + 1 + i64.applies + iad.applies + imx.applies
        counted.update(mv=mv, ap=ap, gmres=i64, mixed=imx, adjoint=iad)
        return xs, xm, lam, g

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    l0 = binding.launch_count()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ops_done = 0
    for k in range(args.steps):
        step(record=True)
        ops_done += counted["mv"] + counted["ap"]
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches = binding.launch_count() - l0
    ck = clocks.stop()
    elapsed = aggregate_elapsed(e0.elapsed_time(e1) / 1e3, dev)
    value = ops_done * ws / elapsed
    mv_ms = statistics.median(per["mv"])
    ap_ms = statistics.median(per["ap"])
    # handle memory of the device-resident step, before the end-to-end leg adds the
    # staging buffer for values updated from host memory
    fact_mem = jac.memory_bytes()

    # roofline of the dominant operation (one sts_jac_matvec = pair-dot pass + main pass)
    hbm_peak, sm_max_mhz, peak_kind = _peaks()
    mv_bytes = 8 * (w.S.shape[0] + 2 * w.n_pairs * w.b + 2 * n) + 4 * w.nnzb
    mv_flops = 2 * (w.S.shape[0] + 2 * w.n_pairs * w.b)
    fp64_peak = N_SMS * FP64_FMA_PER_CLK_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12   # TFLOP/s
    ach_tflops = mv_flops / (mv_ms * 1e-3) / 1e12
    ap_bytes = 8 * (w.n_cells * (w.nnz_d + 2 * w.r_diag * w.b + w.r_diag ** 2) + 2 * n)

    # end to end through the public API: values and vectors from pinned host memory
    e2e = None
    if not args.no_e2e:
        hS = torch.from_numpy(w.S).pin_memory()
        hU = torch.from_numpy(np.ascontiguousarray(w.U)).pin_memory()
        hV = torch.from_numpy(np.ascontiguousarray(w.V)).pin_memory()
        hx = xv.cpu().pin_memory()
        hb = torch.from_numpy(w.rhs).pin_memory()
        hW = torch.from_numpy(w.W).pin_memory()
        outs = None            # pinned host buffers for the step's results, made on first use

        def e2e_step():
            nonlocal outs
            xv.copy_(hx, non_blocking=True)
            b.copy_(hb, non_blocking=True)
            Wd.copy_(hW, non_blocking=True)
            xs, xm, lam, g = step(values=(hS.numpy(), hU.numpy(), hV.numpy()))
            res = [y, z, xs, xm, lam] + list(g)
            if outs is None:
                outs = [torch.empty(a.shape, dtype=a.dtype, pin_memory=True) for a in res]
            for o, a in zip(outs, res):
                o.copy_(a, non_blocking=True)
            return outs

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_ops = 0
        n_e2e = max(1, args.steps)
        for _ in range(n_e2e):
            e2e_step()
            e2e_ops += counted["mv"] + counted["ap"]
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        h2d = 8 * (w.S.shape[0] + 2 * w.n_pairs * w.b + 3 * n)
        d2h = sum(a.numel() * a.element_size() for a in outs)
        e2e = {"value": e2e_ops * ws / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * t_e2e / n_e2e}

    # dense-BSR baseline on the same GPU (outside the timed step)
    dense = None
    if not args.no_dense:
        jd = StsJacobian(w, S, U, V, layout="component", dense=True)

        def avg(fn, reps):
            for _ in range(2):
                fn()
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            c.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(c) / reps

        dmv = avg(lambda: jd.matvec(xv, out=y), 10)
        t0 = time.perf_counter()
        jd.bjacobi_setup()
        dsetup = time.perf_counter() - t0
        dap = avg(lambda: jd.bjacobi_apply(xv, out=z), 10)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, dinfo = jd.gmres(b, rtol=1e-10, restart=30)
        dgm = time.perf_counter() - t0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        jac.bjacobi_setup()
        fsetup = time.perf_counter() - t0
        t0 = time.perf_counter()
        _, finfo = jac.gmres(b, rtol=1e-10, restart=30)
        fgm = time.perf_counter() - t0
        dense_bytes = 8 * (w.nnzb * w.b * w.b + 2 * n)
        dense = {"matvec_ms": dmv, "apply_ms": dap, "setup_ms": 1e3 * dsetup,
                 "gmres_ms": 1e3 * dgm, "gmres_iterations": dinfo.iterations,
                 "gmres_true_rel_residual": dinfo.true_rel_residual,
                 "matvec_GBps": dense_bytes / (dmv * 1e-3) / 1e9,
                 "memory_GB": jd.memory_bytes() / 1e9,
                 "speedup_matvec": dmv / mv_ms, "speedup_apply": dap / ap_ms,
                 "factored_setup_ms": 1e3 * fsetup, "factored_gmres_ms": 1e3 * fgm,
                 "factored_gmres_true_rel_residual": finfo.true_rel_residual,
                 "speedup_gmres_time_to_tolerance": dgm / fgm,
                 "factored_memory_GB": fact_mem / 1e9}
        jd.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        v, dt, cores, pairs = oracle_sample(w, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{pairs} dense-block matvecs + {pairs} dense-LU block-Jacobi "
                         f"applies of {WORKLOAD} on the host cores ({dt:.1f} s)"}

    traffic = _traffic_record()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": _config(w),
        "run": {"ops_per_step": {"matvec_fp64": counted["mv"], "bj_apply_fp64": counted["ap"],
                                 "explicit_loops": ops},
                "parallelism": "replicas" if ws > 1 else "single GPU", "vec_layout": "component-major"},
        "roofline": {"bound": "alu", "kernel": "sts_jac_matvec FP64 (k_dots + k_mv_struct)",
                     "achieved": ach_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": ach_tflops / fp64_peak,
                     "peak_source": f"152 SMs x 2 FP64 FMA/clk x 2 flop x {sm_max_mhz:.0f} MHz",
                     "traffic": traffic, "algorithmic_bytes": mv_bytes,
                     "hbm": {"achieved": mv_bytes / (mv_ms * 1e-3) / 1e9, "peak": hbm_peak,
                             "unit": "GB/s", "frac": mv_bytes / (mv_ms * 1e-3) / 1e9 / hbm_peak,
                             "peak_kind": peak_kind}},
        "breakdown": {"matvec_ms": mv_ms, "bj_apply_ms": ap_ms,
                      "bj_apply_GBps": ap_bytes / (ap_ms * 1e-3) / 1e9,
                      "gmres_iterations": counted["gmres"].iterations,
                      "gmres_true_rel_residual": counted["gmres"].true_rel_residual,
                      "mixed_iterations": counted["mixed"].iterations,
                      "mixed_restarts": counted["mixed"].restarts,
                      "mixed_true_rel_residual": counted["mixed"].true_rel_residual,
                      "adjoint_iterations": counted["adjoint"].iterations},
        "dense_bsr": dense,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": ck,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    jac.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def _timer(stream):
    import torch

    def avg(fn, reps):
        for _ in range(2):
            fn()
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        c.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(c) / reps
    return avg


def _oracle_ops(w, with_apply: bool):
    """One FP64 oracle matvec (and block-Jacobi apply) of the workload on the host
    cores, timed as it stands: the CPU baseline beside a report."""
    import numpy as np
    import oracle
    oracle.build()
    J = oracle.Jacobian.from_workload(w)
    x = np.random.default_rng(0).standard_normal(w.n)
    t0 = time.perf_counter()
    oracle.matvec(J, x)
    out = {"matvec_ms": 1e3 * (time.perf_counter() - t0), "cores": oracle.max_threads(),
           "kind": "oracle (dense blocks assembled on the fly)"}
    if with_apply:
        F = oracle.bj_setup(J)
        t0 = time.perf_counter()
        oracle.bj_apply(F, x)
        out["apply_ms"] = 1e3 * (time.perf_counter() - t0)
    return out


def run_report(args):
    """Extra measurements beyond the default line (one JSON line each):
    nsweep  matvec time and handle memory vs N, factored vs dense, fitted exponents;
    large   256x256, N=200: factored vs dense matvec, apply, setup, GMRES time to 1e-10;
    mixed   512x512, N=60: FP64 GMRES vs FP32/FP64 flexible GMRES, error vs the oracle;
    pairs   128x128, N=60 with the paper's pair counts (1 + 2 per face, 2 per neighbour
            block): factored vs dense matvec, apply, setup, GMRES, roofline fractions;
    newton  128x128, N=60 HLL-flux model: residual, Jacobian generation, values update,
            setup, GMRES, and one Newton pseudo-time step, factored vs dense;
    kernels 128x128, N=60: three rounds of FP64 and FP32 matvec and apply, a short
            fixed launch sequence for kernel profilers (no timing);
    dd      128x128, N=60 cut into 1, 2 (strips) and 4 (2 x 2 tiles) parts held by this
            process: matvec with its halo exchange, block-Jacobi, GMRES to 1e-10,
            against the single handle."""
    import numpy as np
    import torch
    import __graft_entry__
    from paper_2403_09198_gb300 import inputs
    from paper_2403_09198_gb300.binding import StsJacobian
    __graft_entry__.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    avg = _timer(stream)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()

    if args.report == "dd":
        from paper_2403_09198_gb300.dd import DdPlan, DdSolver, grid_partition
        w = inputs.named_workload("grid128_N60")
        S, U, V = t(w.S), t(w.U), t(w.V)
        ref = StsJacobian(w, S, U, V, layout="component")
        ref.bjacobi_setup()
        xv = torch.randn(w.n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(xv)
        b = t(w.rhs.reshape(w.n_cells, w.b).T.ravel())
        out = {"report": "dd", "workload": "grid128_N60: 128x128 cells, N=60, b=63, 2/1 pairs",
               "single": {"matvec_ms": avg(lambda: ref.matvec(xv, out=y), 50),
                          "apply_ms": avg(lambda: ref.bjacobi_apply(xv, out=y), 50)}}
        ref.gmres(b, rtol=1e-10)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = ref.gmres(b, rtol=1e-10)
        out["single"].update(gmres_ms=1e3 * (time.perf_counter() - t0), iterations=info.iterations)
        for name, (px, py) in (("1 part", (1, 1)), ("2 strips", (1, 2)), ("2x2 tiles", (2, 2))):
            part = grid_partition(128, 128, px, py)
            plans, jacs = [], []
            for p in range(px * py):
                P = DdPlan(w.block_indptr, w.block_indices, part, px * py, p)
                L, (Sl, Ul, Vl) = P.gather(w, S, U, V)
                j = StsJacobian(L, Sl, Ul, Vl, layout="component")
                j.bjacobi_setup()
                plans.append(P)
                jacs.append(j)
            solver = DdSolver(jacs, plans)
            xs = [torch.randn(P.n_local * w.b, dtype=torch.float64, device="cuda") for P in plans]
            bs = []
            for P in plans:
                loc = w.rhs.reshape(w.n_cells, w.b)[P.local_to_global]
                bs.append(t(np.ascontiguousarray(loc.T).ravel()))
            r = {"parts": px * py, "ghost_cells": int(sum(P.n_ghost for P in plans)),
                 "matvec_ms": avg(lambda: solver.matvec(xs), 50),
                 "apply_ms": avg(lambda: solver.bjacobi_apply(xs), 50)}
            solver.gmres(bs, rtol=1e-10)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = solver.gmres(bs, rtol=1e-10)
            r.update(gmres_ms=1e3 * (time.perf_counter() - t0), iterations=info.iterations,
                     true_rel_residual=info.true_rel_residual)
            out[name] = r
            solver.close()
            for j in jacs:
                j.close()
        ref.close()
        print(json.dumps(out), flush=True)
        return

    if args.report == "kernels":
        w = inputs.named_workload("grid128_N60")
        j = StsJacobian(w, t(w.S), t(w.U), t(w.V), layout="component", mixed=True)
        j.bjacobi_setup()
        x = torch.randn(w.n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        x32 = x.float()
        y32 = torch.empty_like(x32)
        for _ in range(3):
            j.matvec(x, out=y)
            j.bjacobi_apply(x, out=y)
            j.matvec(x32, out=y32)
            j.bjacobi_apply(x32, out=y32)
        torch.cuda.synchronize()
        j.close()
        print(json.dumps({"report": "kernels", "workload": "grid128_N60", "rounds": 3}), flush=True)
        return

    if args.report == "nsweep":
        for L in (40, 128):
            rows = []
            for N in (10, 20, 40, 60, 100, 150, 200):
                if L == 128 and N > 100:
                    continue            # dense 128x128 blocks above N=100 exceed a minute of setup
                w = inputs.make_workload(L, L, N=N, w=2, r_diag=2, r_off=1, seed=N)
                S, U, V = t(w.S), t(w.U), t(w.V)
                x = torch.randn(w.n, dtype=torch.float64, device="cuda")
                y = torch.empty_like(x)
                f = StsJacobian(w, S, U, V, layout="component")
                tf = avg(lambda: f.matvec(x, out=y), 20)
                mf = f.memory_bytes()
                f.close()
                d = StsJacobian(w, S, U, V, layout="component", dense=True)
                td = avg(lambda: d.matvec(x, out=y), 10)
                md = d.memory_bytes()
                d.close()
                rows.append(dict(N=N, b=w.b, factored_ms=tf, dense_ms=td, factored_bytes=mf, dense_bytes=md,
                                 S_values=int(w.S.shape[0])))
                del S, U, V
                torch.cuda.empty_cache()
            Ns = np.log([r["b"] for r in rows])
            fit = lambda key: float(np.polyfit(Ns, np.log([r[key] for r in rows]), 1)[0])
            print(json.dumps({"report": "nsweep", "grid": f"{L}x{L}", "rows": rows,
                              "slope_vs_b": {k: fit(k) for k in ("factored_ms", "dense_ms", "factored_bytes",
                                                                 "dense_bytes")}}), flush=True)
        return

    if args.report == "large":
        w = inputs.named_workload("grid256_N200")
        S, U, V, b = t(w.S), t(w.U), t(w.V), t(w.rhs)
        x = torch.randn(w.n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        out = {"report": "large", "workload": "grid256_N200: 256x256 cells, N=200, b=203, band +-4, 3/1 pairs"}
        for name, kw in (("factored", {}), ("dense", {"dense": True})):
            j = StsJacobian(w, S, U, V, layout="component", **kw)
            r = {"matvec_ms": avg(lambda: j.matvec(x, out=y), 5 if kw else 20),
                 "memory_GB": j.memory_bytes() / 1e9}
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            j.bjacobi_setup()
            r["setup_ms"] = 1e3 * (time.perf_counter() - t0)
            r["apply_ms"] = avg(lambda: j.bjacobi_apply(x, out=y), 5 if kw else 20)
            j.gmres(b, rtol=1e-10, restart=30)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = j.gmres(b, rtol=1e-10, restart=30)
            r["gmres_ms"] = 1e3 * (time.perf_counter() - t0)
            r["gmres_iterations"] = info.iterations
            r["gmres_true_rel_residual"] = info.true_rel_residual
            out[name] = r
            j.close()
            torch.cuda.empty_cache()
        out["speedup"] = {k: out["dense"][k] / out["factored"][k] for k in ("matvec_ms", "apply_ms", "setup_ms",
                                                                             "gmres_ms")}
        out["oracle"] = _oracle_ops(w, with_apply=False)
        out["oracle"]["factored_matvec_speedup"] = out["oracle"]["matvec_ms"] / out["factored"]["matvec_ms"]
        print(json.dumps(out), flush=True)
        return

    if args.report == "pairs":
        # the paper's pair counts (Section 4.3): 1 + 2 per face on diagonal blocks,
        # 2 per neighbour block; algorithmic bytes count each block's own pairs
        w = inputs.named_workload("grid128_N60_pairs9")
        S, U, V, b = t(w.S), t(w.U), t(w.V), t(w.rhs)
        x = torch.randn(w.n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        counts = np.diff(w.pair_indptr)
        rd = counts[w.is_diag_block()]
        mv_bytes = 8 * (w.S.shape[0] + 2 * w.n_pairs * w.b + 2 * w.n) + 4 * w.nnzb
        mv_flops = 2 * (w.S.shape[0] + 2 * w.n_pairs * w.b)
        ap_bytes = 8 * (int(np.sum(w.nnz_d + 2 * rd * w.b + rd * rd)) + 2 * w.n)
        hbm_peak, sm_mhz, src = _peaks()
        fp64_peak = N_SMS * FP64_FMA_PER_CLK_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        out = {"report": "pairs",
               "workload": "grid128_N60_pairs9: 128x128 cells, N=60, b=63, band +-2, diagonal blocks "
                           "1 + 2 pairs per face (9 inside, 7 on edges, 5 at corners), 2 per neighbour block",
               "n_pairs": w.n_pairs, "diag_pair_counts": {str(k): int(np.sum(rd == k)) for k in np.unique(rd)},
               "matvec_algorithmic_bytes": mv_bytes, "matvec_flops": mv_flops, "apply_algorithmic_bytes": ap_bytes}
        for name, kw in (("factored", {}), ("dense", {"dense": True})):
            j = StsJacobian(w, S, U, V, layout="component", **kw)
            r = {"matvec_ms": avg(lambda: j.matvec(x, out=y), 10 if kw else 200),
                 "memory_GB": j.memory_bytes() / 1e9}
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            j.bjacobi_setup()
            r["setup_ms"] = 1e3 * (time.perf_counter() - t0)
            r["apply_ms"] = avg(lambda: j.bjacobi_apply(x, out=y), 10 if kw else 200)
            j.gmres(b, rtol=1e-10, restart=30)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = j.gmres(b, rtol=1e-10, restart=30)
            r["gmres_ms"] = 1e3 * (time.perf_counter() - t0)
            r["gmres_iterations"] = info.iterations
            r["gmres_true_rel_residual"] = info.true_rel_residual
            out[name] = r
            j.close()
            torch.cuda.empty_cache()
        f = out["factored"]
        f["matvec_TFLOPs"] = mv_flops / (f["matvec_ms"] * 1e-3) / 1e12
        f["matvec_frac_fp64_peak"] = f["matvec_TFLOPs"] / fp64_peak
        f["matvec_GBps"] = mv_bytes / (f["matvec_ms"] * 1e-3) / 1e9
        f["apply_GBps"] = ap_bytes / (f["apply_ms"] * 1e-3) / 1e9
        f["matvec_frac_hbm"] = f["matvec_GBps"] / hbm_peak
        f["apply_frac_hbm"] = f["apply_GBps"] / hbm_peak
        out["peaks"] = {"hbm_GBps": hbm_peak, "fp64_TFLOPs": fp64_peak, "source": src}
        out["speedup"] = {k: out["dense"][k] / f[k] for k in ("matvec_ms", "apply_ms", "setup_ms", "gmres_ms")}
        out["oracle"] = _oracle_ops(w, with_apply=True)
        print(json.dumps(out), flush=True)
        return

    if args.report == "newton":
        # one implicit pseudo-time step (Newton from Q^0 = Q^n) of the HLL-flux
        # model, its parts timed alone, factored storage against dense BSR
        from paper_2403_09198_gb300.binding import StsFlow
        c = inputs.make_flow_case(128, 128, N=60, w=2, seed=13, dt=0.5)
        f = StsFlow(c)
        L, z = f.layout, f.sizes
        Q, Qn = t(c.Q), t(c.Qn)
        R = torch.empty_like(Q)
        S, U, V = f.jacobian(Q)
        gen_bytes = 8 * (z.nnz_S + 2 * z.n_pairs * z.block_size + 6 * z.n_cells * z.block_size)
        out = {"report": "newton",
               "workload": "flow128_N60: 128x128 cells, N=60 species, b=63, band +-2, dt=0.5, "
                           "1 + 2 pairs per face on diagonal blocks, 2 per neighbour block",
               "residual_ms": avg(lambda: f.residual(Q, Qn, out=R), 50),
               "jacobian_ms": avg(lambda: f.jacobian(Q, S, U, V), 20),
               "jacobian_written_bytes": gen_bytes}
        out["jacobian_GBps"] = gen_bytes / (out["jacobian_ms"] * 1e-3) / 1e9
        rhs = -f.residual(Q, Qn).reshape(-1)
        for name, kw in (("factored", {}), ("dense", {"dense": True})):
            jac = f.jacobian_handle(Q=Q, **kw)
            r = {"update_values_ms": avg(lambda: jac.update_values(S, U, V), 3 if kw else 10)}
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            jac.bjacobi_setup()
            r["setup_ms"] = 1e3 * (time.perf_counter() - t0)
            jac.gmres(rhs, rtol=1e-10)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, gi = jac.gmres(rhs, rtol=1e-10)
            r["gmres_ms"] = 1e3 * (time.perf_counter() - t0)
            r["gmres_iterations"] = gi.iterations
            Qs = Qn.clone()
            f.newton(jac, Qs, Qn, rtol=1e-10)           # warm-up of the whole step
            Qs = Qn.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info, hist = f.newton(jac, Qs, Qn, rtol=1e-10)
            r["newton_step_ms"] = 1e3 * (time.perf_counter() - t0)
            r["newton"] = {k: info[k] for k in ("iterations", "linear_iterations", "halvings", "res0", "res")}
            r["residual_history"] = hist.tolist()
            r["memory_GB"] = jac.memory_bytes() / 1e9
            if not kw:
                # inexact Newton: each linear solve to the Eisenstat-Walker forcing term
                Qs = Qn.clone()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info_f, hist_f = f.newton(jac, Qs, Qn, rtol=1e-10, forcing=True)
                r["forcing"] = {"newton_step_ms": 1e3 * (time.perf_counter() - t0),
                                "newton": {k: info_f[k] for k in ("iterations", "linear_iterations", "halvings",
                                                                   "res0", "res")},
                                "residual_history": hist_f.tolist()}
            out[name] = r
            jac.close()
            torch.cuda.empty_cache()
        out["speedup_newton_step"] = out["dense"]["newton_step_ms"] / out["factored"]["newton_step_ms"]
        f.close()
        print(json.dumps(out), flush=True)
        return

    if args.report == "mixed":
        import oracle
        oracle.build()
        w = inputs.named_workload("grid512_N60")
        S, U, V, b = t(w.S), t(w.U), t(w.V), t(w.rhs)
        j = StsJacobian(w, S, U, V, mixed=True)
        j.bjacobi_setup()
        res = {"report": "mixed", "workload": "grid512_N60: 512x512 cells, N=60, b=63, 2/1 pairs"}
        for mode in ("fp64", "mixed"):
            j.gmres(b, rtol=1e-10, restart=30, mixed=(mode == "mixed"))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            xs, info = j.gmres(b, rtol=1e-10, restart=30, mixed=(mode == "mixed"))
            res[mode] = {"ms": 1e3 * (time.perf_counter() - t0), "iterations": info.iterations,
                         "restarts": info.restarts, "true_rel_residual": info.true_rel_residual,
                         "x": xs.cpu().numpy()}
        x32 = torch.randn(w.n, dtype=torch.float32, device="cuda")
        res["fp32_matvec_ms"] = avg(lambda: j.matvec(x32, out=torch.empty_like(x32)), 20)
        res["fp32_apply_ms"] = avg(lambda: j.bjacobi_apply(x32, out=torch.empty_like(x32)), 20)
        x64 = x32.double()
        res["fp64_matvec_ms"] = avg(lambda: j.matvec(x64, out=torch.empty_like(x64)), 20)
        res["fp64_apply_ms"] = avg(lambda: j.bjacobi_apply(x64, out=torch.empty_like(x64)), 20)
        j.close()
        # the FP64 oracle solves the same system on the host cores
        J = oracle.Jacobian.from_workload(w)
        t0 = time.perf_counter()
        xo, io = oracle.gmres(J, w.rhs, restart=30, rtol=1e-12)
        res["oracle"] = {"s": time.perf_counter() - t0, "iterations": io["iterations"],
                         "true_rel_residual": io["true_rel"], "cores": oracle.max_threads()}
        for mode in ("fp64", "mixed"):
            xm = res[mode].pop("x")
            res[mode]["rel_error_vs_oracle"] = float(np.linalg.norm(xm - xo) / np.linalg.norm(xo))
        # kappa estimate of J: power iterations on J^T J and on (J^T J)^-1 via the oracle
        rng = np.random.default_rng(0)
        v = rng.standard_normal(w.n)
        for _ in range(8):
            v = oracle.matvec(J, oracle.matvec(J, v), trans=True)
            v /= np.linalg.norm(v)
        smax = np.sqrt(np.linalg.norm(oracle.matvec(J, oracle.matvec(J, v), trans=True)))
        u = rng.standard_normal(w.n)
        F = oracle.bj_setup(J)
        for _ in range(4):
            u, _ = oracle.gmres(J, u, restart=30, rtol=1e-12, factors=F)
            u, _ = oracle.gmres(J, u, restart=30, rtol=1e-12, trans=True, factors=F)
            u /= np.linalg.norm(u)
        z, _ = oracle.gmres(J, u, restart=30, rtol=1e-12, factors=F)
        z, _ = oracle.gmres(J, z, restart=30, rtol=1e-12, trans=True, factors=F)
        smin = 1.0 / np.sqrt(np.linalg.norm(z))
        res["kappa_estimate"] = float(smax / smin)
        res["bound_kappa_x_1e-10"] = res["kappa_estimate"] * 1e-10
        print(json.dumps(res), flush=True)
        return


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--ops", type=int, default=1000, help="explicit matvec / apply loop length per step")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample length")
    p.add_argument("--no-dense", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--report", choices=["nsweep", "large", "mixed", "kernels", "pairs", "newton", "dd"], default=None,
                   help="print an extra measurement instead of the benchmark line")
    args = p.parse_args()
    if args.report:
        run_report(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
