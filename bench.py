#!/usr/bin/env python
"""Benchmark: Nys-IP-PMM QP solves per second on GB300 (one JSON line).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

A step is one whole Nys-IP-PMM solve of a synthetic separable QP (every
Newton system through the Nystrom sketch, core factorisation, PCG, back
substitution and step lengths), inputs resident in HBM.  Multi-GPU runs are
independent replicas (one QP per rank, no collective on the data path):
`value` = solves of all ranks / max-over-ranks time.

Extra keys: `roofline` (normal-equations operator, the dominant kernel pair,
timed with CUDA events on the solver's stream), `cpu_baseline` (the CPU
oracle on a bounded sample, rank 0), `e2e` (the same solves through the C ABI
with pinned host buffers, copies inside the timed region), `clocks`
(nvidia-smi samples taken during the timed region) and `gpu_launches`
(kernels of libnys.so launched inside the timed region).
`--impl reference` times the CPU oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# name -> (generator kwargs, ell, tol, description)
WORKLOADS = {
    "small-fp64": dict(gen=("workload_small", {}), ell=20, tol=1e-6,
                       desc="m=200, n=500, sigma_i=1/i, q~U[0,1], ell=20, tol 1e-6, FP64"),
    "fp64-5000x20000": dict(gen=("workload_fp64", {}), ell=100, tol=1e-8,
                            desc="m=5000, n=20000, sigma_i=i^-0.8, q 50% zero, ell=100, tol 1e-8, FP64"),
    "fp64-2000x10000-exp": dict(gen=("workload_precision_scaled", {}), ell=40, tol=1e-6,
                                desc="m=2000, n=10000, sigma_i=exp(-i/200)+1e-3, q~U[0,1], ell=40, tol 1e-6, FP64"),
}
DEFAULT_WORKLOAD = "fp64-2000x10000-exp"

# FP64 ALU peak: 152 SMs x 2 DFMA/clk/SM x 2 flop at the 2070 MHz maximum SM
# clock (the nominal 1.25 TFLOP/s FP64 of GB300 expressed in unit counts).
DFMA_PER_CLK_PER_SM = 2
SMS = 152
SM_MAX_MHZ = 2070.0


def fp64_alu_peak_tflops(mhz: float = SM_MAX_MHZ) -> float:
    return SMS * DFMA_PER_CLK_PER_SM * 2 * mhz * 1e6 / 1e12


def make_qp(name: str, rank: int):
    from paper_2404_14524_gb300 import synth
    w = WORKLOADS[name]
    fn, kw = w["gen"]
    kw = dict(kw)
    base = {"workload_small": 1235, "workload_fp64": 1236, "workload_precision_scaled": 1237}[fn]
    kw["seed"] = base + 1000 * rank          # replicas solve different QPs
    return getattr(synth, fn)(**kw)


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == 7:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        smax = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def traffic_record(kernel_file: str):
    """dram bytes per launch of the operator from the committed ncu summary,
    or None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    src = open(os.path.join(ROOT, "paper_2404_14524_gb300", "csrc", kernel_file), "rb").read()
    if rec.get("source_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return rec


def cpu_baseline(qp, w, gpu_ipm: int, gpu_pcg: int, seed: int):
    """The oracle as it stands on this host.  Whole solve when that is short;
    otherwise timed components extrapolated with the GPU run's counts."""
    from oracle import nys_oracle as O
    threads = os.cpu_count()
    m, n = qp.A.shape
    # components: one IPM iteration with PCG forced to zero, and PCG iterations
    t0 = time.perf_counter()
    O.solve_qp(qp, O.Options(tol=w["tol"], ell=w["ell"], seed=seed, forced_ipm=1, forced_pcg=[0, 0]))
    t_ipm = time.perf_counter() - t0
    D = O.scaling_D(qp.x0, qp.z0, qp.q, 1.0)
    F = O.nystrom(qp.A, D, O.gaussian_omega(seed, 0, m, min(w["ell"], m)))
    xi = np.random.default_rng(0).standard_normal(m)
    k_pcg = 20
    t0 = time.perf_counter()
    O.pcg(lambda v: O.normal_matvec(qp.A, D, 1e-3, v), lambda v: O.precond_inv_apply(F, 1e-3, v),
          xi, 0.0, k_pcg, forced_iters=k_pcg)
    t_pcg = (time.perf_counter() - t0) / k_pcg
    est = gpu_ipm * t_ipm + gpu_pcg * t_pcg
    sample = (f"1 oracle IPM iteration with PCG forced to 0 ({t_ipm:.3f} s) + {k_pcg} oracle PCG "
              f"iterations ({t_pcg * 1e3:.2f} ms each) on the same {m}x{n} workload, extrapolated with "
              f"the GPU run's counts ({gpu_ipm} IPM, {gpu_pcg} PCG iterations per solve)")
    if est <= 30.0:
        t0 = time.perf_counter()
        r = O.solve_qp(qp, O.Options(tol=w["tol"], ell=w["ell"], seed=seed))
        full = time.perf_counter() - t0
        return {"value": 1.0 / full, "unit": "QP solves/s", "cores": threads, "kind": "oracle",
                "sample": f"one whole oracle solve of the same workload ({r.ipm_iters} IPM, "
                          f"{sum(r.pcg_iters)} PCG iterations, {full:.2f} s)"}
    return {"value": 1.0 / est, "unit": "QP solves/s", "cores": threads, "kind": "oracle",
            "sample": sample}


def run_reference(args, w, rank, world):
    """Reference arm: the CPU oracle, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    from oracle import nys_oracle as O
    qp = make_qp(args.workload, 0)
    seed = 7
    m, n = qp.A.shape
    # bounded sample per step: at most `budget` seconds of oracle work
    t0 = time.perf_counter()
    r = O.solve_qp(qp, O.Options(tol=w["tol"], ell=w["ell"], seed=seed, max_ipm_iter=3))
    probe = time.perf_counter() - t0
    whole = probe < 20.0 / max(1, args.steps + args.warmup)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        if whole:
            r = O.solve_qp(qp, O.Options(tol=w["tol"], ell=w["ell"], seed=seed))
        else:
            r = O.solve_qp(qp, O.Options(tol=w["tol"], ell=w["ell"], seed=seed, max_ipm_iter=3))
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    per = statistics.mean(times)
    if whole:
        value, sample = 1.0 / per, f"whole oracle solve ({r.ipm_iters} IPM iterations) per step"
    else:
        value, sample = None, "first 3 oracle IPM iterations per step (whole solve exceeds the step budget)"
    line = {"metric": "QP solves/s to KKT tol", "value": value, "unit": "QP solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "desc": w["desc"], "m": m, "n": n},
            "cpu_baseline": {"value": value, "unit": "QP solves/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "QP solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2404_14524_gb300 import build
    build.build()
    from paper_2404_14524_gb300 import nys

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    qp = make_qp(args.workload, rank)
    m, n = qp.A.shape
    seed = 7
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    A, b, c, q, x0, y0, z0 = (T(v) for v in (qp.A, qp.b, qp.c, qp.q, qp.x0, qp.y0, qp.z0))
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        h = nys.Handle(m, n, ell=w["ell"], tol=w["tol"], seed=seed, max_pcg_iter=1000, stream=stream)
        for _ in range(args.warmup):
            x, y, z, info = nys.nys_solve(h, A, b, c, q, x0, y0, z0)
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        l0 = nys.nys_kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        with ClockSampler(local) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                x, y, z, info = nys.nys_solve(h, A, b, c, q, x0, y0, z0)
                infos.append(info)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        launches = nys.nys_kernel_launches() - l0
        ms = e0.elapsed_time(e1)
        clocks = clk.summary()
        t = torch.tensor([ms, float(launches)], dtype=torch.float64, device=dev)
        if world > 1:
            tmax = t.clone()
            dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
            tsum = t.clone()
            dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
            ms, launches = float(tmax[0]), int(tsum[1])
        value = args.steps * world / (ms / 1e3)

        # Roofline of the dominant kernel pair: (N + delta I) v, A^T pass + A pass.
        D = torch.rand(n, dtype=torch.float64, device=dev) + 0.5
        v = torch.randn(m, dtype=torch.float64, device=dev)
        out = torch.empty_like(v)
        for _ in range(3):
            nys.nys_normal_matvec(h, A, D, 1e-3, v, out)
        reps = 20
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(reps):
            nys.nys_normal_matvec(h, A, D, 1e-3, v, out)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        op_s = f0.elapsed_time(f1) / reps / 1e3
        flops = 4.0 * m * n                      # 2 FMA per element of A per operator application
        bytes_alg = 2.0 * m * n * 8 + 8.0 * (3 * m + 2 * n)
        peak = fp64_alu_peak_tflops()
        tr = traffic_record("gemv_f64.cu")
        roofline = {"bound": "alu", "achieved": flops / op_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "frac": flops / op_s / 1e12 / peak,
                    "traffic": (tr["bytes_per_launch"] * (m * n) / tr["elements"]) if tr else None,
                    "kernel": "normal-equations operator (k_atv_partial + k_atv_reduce + k_av), FP64",
                    "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (nominal FP64 1.25 TFLOP/s)",
                    "hbm_gbs": bytes_alg / op_s / 1e9, "op_ms": op_s * 1e3,
                    "algorithmic_flops": flops, "algorithmic_bytes": bytes_alg}

        # e2e through the C ABI with pinned host buffers
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hA, hb, hc, hq, hx0, hy0, hz0 = (pin(vv) for vv in (qp.A, qp.b, qp.c, qp.q, qp.x0, qp.y0, qp.z0))
        nys.nys_solve(h, hA, hb, hc, hq, hx0, hy0, hz0)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            nys.nys_solve(h, hA, hb, hc, hq, hx0, hy0, hz0)
        torch.cuda.synchronize(dev)
        e2e_s = time.perf_counter() - t0
        if world > 1:
            te = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
            e2e_s = float(te[0])
        h2d = 8 * (m * n + m + 3 * n + n + m + n)
        d2h = 8 * (2 * n + m)

    last = infos[-1]
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(qp, w, last["ipm_iters"], last["pcg_iters_total"], seed)
        line = {
            "metric": "QP solves/s to KKT tol", "value": value, "unit": "QP solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"], "m": m, "n": n, "ell": w["ell"],
                       "tol": w["tol"], "form": "fp64", "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 (A = {m * n * 8 / 1e6:.0f} MB)" if m * n * 8 > 129e6
                       else "A fits in L2 (no flush)"},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": args.steps * world / e2e_s, "unit": "QP solves/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "clocks": clocks, "gpu_launches": launches,
            "solve": {"status": last["status"], "ipm_iters": last["ipm_iters"],
                      "pcg_iters": last["pcg_iters_total"], "rel_primal": last["rel_primal"],
                      "rel_dual": last["rel_dual"], "mu": last["mu"], "rel_gap": last["rel_gap"]},
        }
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
