#!/usr/bin/env python
"""Benchmark: Nys-IP-PMM QP solves per second on GB300 (one JSON line).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

A step is one whole Nys-IP-PMM solve of the workload (every Newton system
through the Nystrom sketch, the core factorisation, PCG, back substitution
and the step lengths; for the batch workload all of its QPs; for the
differentiation workload the forward solves plus the adjoint solves), with
the inputs resident in HBM.  Multi-GPU runs are independent replicas (one
workload per rank, no collective on the data path): `value` = solves of all
ranks / max-over-ranks time.

Extra keys: `roofline` (the dominant kernel, timed with CUDA events on the
solver's stream), `cpu_baseline` (the CPU oracle on a bounded sample, rank 0,
N=1), `e2e` (the same solves through the C ABI with pinned host buffers,
copies inside the timed region), `clocks` (nvidia-smi samples taken during the
timed region), `gpu_launches` (kernels of libnys.so launched inside the
timed region) and, on one GPU, `config3`: one whole solve of the m=20000,
n=100000, ell=400 workload in the precision form (BF16 + refinement) and in
the FP64 form on the same QP (QP/s, counts, KKT measures, the precision form's
distance from the FP64 form's answer; about 15 minutes, `--no-config3` skips
it).  `--impl reference` times the CPU oracle instead.
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
# the batching form runs one stream per problem in flight: let up to 32 of
# them reach the GPU through separate hardware queues (the default is 8);
# read when the CUDA context is created, so set before torch is imported
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np  # noqa: E402

# name -> workload description
WORKLOADS = {
    "small-fp64": dict(form="fp64", m=200, n=500, ell=20, tol=1e-6, gen="small",
                       desc="m=200, n=500, sigma_i=1/i, q~U[0,1], ell=20, tol 1e-6, FP64 form"),
    "box-200x500": dict(form="box", m=200, n=500, ell=20, tol=1e-6, gen="box",
                        desc="m=200, n=500, sigma_i=1/i, q~U[0,1], 10% free and 30% box-constrained variables "
                             "(problem (P~)), ell=20, tol 1e-6, FP64 form"),
    "svm-100x98528": dict(form="box", m=101, n=98628, ell=50, tol=1e-6, gen="svm", start="practical",
                          desc="dual linear SVM (supplement formulation, (P~): d=100 free, 98528 box variables "
                               "0<=p<=1), synthetic dense features of the SensIT shape, ell=50, tol 1e-6, "
                               "practical initial point, FP64 form"),
    "portfolio-1600x1000x20": dict(form="box", m=1021, n=2620, ell=20, tol=1e-8, gen="portfolio", start="practical",
                                   desc="factor-model portfolio (supplement formulation, (P~)): 1600 assets, "
                                        "1000 correlation rows, 20 factors, ell=20, tol 1e-8, practical initial "
                                        "point, FP64 form"),
    "fp64-5000x20000": dict(form="fp64", m=5000, n=20000, ell=100, tol=1e-8, gen="fp64",
                            desc="m=5000, n=20000, sigma_i=i^-0.8, q 50% zero, ell=100, tol 1e-8, FP64 form"),
    "precision-20000x100000": dict(form="bf16", m=20000, n=100000, ell=400, tol=1e-6, gen="device-exp200",
                                   desc="m=20000, n=100000, sigma_i=exp(-i/200)+1e-3, q~U[0,1], FP32 A stored "
                                        "BF16, FP32/float-float refinement, ell=400, tol 1e-6"),
    "precision-4000x20000": dict(form="bf16", m=4000, n=20000, ell=80, tol=1e-6, gen="device-exp200",
                                 desc="m=4000, n=20000 (scaled precision workload), ell=80, tol 1e-6"),
    "precision-fp8-4000x20000": dict(form="fp8", m=4000, n=20000, ell=80, tol=1e-6, gen="device-exp200",
                                     desc="m=4000, n=20000 (scaled precision workload), FP32 A stored FP8 "
                                          "E4M3 with per-row scales for the inner PCG, ell=80, tol 1e-6"),
    "precision-fp8-20000x100000": dict(form="fp8", m=20000, n=100000, ell=400, tol=1e-6, gen="device-exp200",
                                       desc="m=20000, n=100000, sigma_i=exp(-i/200)+1e-3, FP32 A stored FP8 "
                                            "E4M3 + row scales (inner PCG), BF16 sketch, ell=400, tol 1e-6"),
    "batch-256": dict(form="batch", count=256, ell=32, tol=1e-6, gen="batch",
                      desc="256 QPs, m~U{64..1024}, n~U{4m..8m}, sigma_i=1/i, q~U[0,1], "
                           "ell=min(32, m/4), tol 1e-6, FP64 form, nys_solve_batched"),
    "diff-64x512x2048": dict(form="diff", count=64, m=512, n=2048, ell=32, tol=1e-8, gen="diff",
                             desc="64 Gaussian QPs 512x2048, q~U[0.1,1], forward tol 1e-8 + adjoint "
                                  "(dL/d(c,b,q,A), L=||x*-x_t||^2)"),
}
DEFAULT_WORKLOAD = "small-fp64"

SMS = 152
SM_MAX_MHZ = 2070.0
DFMA_PER_CLK_PER_SM = 2        # GB300: 1.25 TFLOP/s FP64 nominal = 152 x 2 x 2 x 2.07 GHz


def fp64_alu_peak_tflops(mhz: float = SM_MAX_MHZ) -> float:
    return SMS * DFMA_PER_CLK_PER_SM * 2 * mhz * 1e6 / 1e12


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6681.5), d.get("bf16_tflops", 1873.8), "measured"
    return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.path = index, None, None

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
        num = lambda v: v.replace(".", "", 1).isdigit()
        sm = [float(r[0]) for r in rows if num(r[0])]
        smax = [float(r[1]) for r in rows if num(r[1])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def traffic_record(kernel_file: str, key: str):
    """dram bytes per unit of work of a kernel from the committed ncu summary,
    or None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(key)
    if not rec:
        return None
    src = open(os.path.join(ROOT, "paper_2404_14524_gb300", "csrc", kernel_file), "rb").read()
    if rec.get("source_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return rec


# ------------------------------------------------------------------ workloads

def host_workload(w, rank):
    """numpy problems (list) for the host-generated workloads."""
    from paper_2404_14524_gb300 import synth
    g = w["gen"]
    off = 1000 * rank
    if g == "small":
        return [synth.workload_small(1235 + off)]
    if g == "box":
        return [synth.workload_box(1240 + off)]
    if g == "svm":
        return [synth.svm_qp(1241 + off, 100, 98528)]
    if g == "portfolio":
        return [synth.portfolio_qp(1242 + off, 1600, 1000, 20)]
    if g == "fp64":
        return [synth.workload_fp64(1236 + off)]
    if g == "batch":
        return synth.workload_batch(1238 + off, count=w["count"])
    if g == "diff":
        qps, targets = synth.workload_diff(1239 + off, count=w["count"], m=w["m"], n=w["n"])
        for qp, t in zip(qps, targets):
            qp.target = t
        return qps
    return None


def device_workload(w, rank, dev, host_gen=False):
    from paper_2404_14524_gb300 import synth
    import torch
    if host_gen:
        # the same spectrum generated with numpy (no device QR), FP32 A the problem
        qp = synth.spectral_qp(1237 + 1000 * rank, w["m"], w["n"], "exp200", "uniform")
        A32 = qp.A.astype(np.float32)
        A64 = A32.astype(np.float64)
        b = A64 @ qp.x0
        c = A64.T @ qp.y0 + qp.z0 - qp.q * qp.x0
        T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        return (T(A32), T(b), T(c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))
    A, b, c, q, x0, y0, z0 = synth.spectral_qp_device(1237 + 1000 * rank, w["m"], w["n"], "exp200", "uniform",
                                                      device=dev, dtype=torch.float32)
    torch.cuda.synchronize(dev)
    return A, b, c, q, x0, y0, z0


# ------------------------------------------------------------------ CPU oracle legs

def oracle_component_times(A64, b, c, q, x0, y0, z0, ell, tol, seed, box=None):
    from oracle import nys_oracle as O
    m, n = A64.shape
    t0 = time.perf_counter()
    O.solve(A64, b, c, q, x0, y0, z0, O.Options(tol=tol, ell=ell, seed=seed, forced_ipm=1, forced_pcg=[0, 0]),
            **(box or {}))
    t_ipm = time.perf_counter() - t0
    D = O.scaling_D(x0, z0, q, 1.0)
    F = O.nystrom(A64, D, O.gaussian_omega(seed, 0, m, min(ell, m)))
    xi = np.random.default_rng(0).standard_normal(m)
    k = 10
    t0 = time.perf_counter()
    O.pcg(lambda v: O.normal_matvec(A64, D, 1e-3, v), lambda v: O.precond_inv_apply(F, 1e-3, v), xi, 0.0, k,
          forced_iters=k)
    return t_ipm, (time.perf_counter() - t0) / k


_SINGLE_CORE_SOLVE = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, sys.argv[1])
from oracle import nys_oracle as O
d = np.load(sys.argv[2])
cfg = json.loads(sys.argv[3])
opt = O.Options(tol=cfg["tol"], ell=cfg["ell"], seed=cfg["seed"], reuse_pcg=cfg["reuse"])
box = {k: d[k] for k in ("kind", "u", "s0") if k in d.files}
t0 = time.perf_counter()
if cfg["practical"]:
    O.solve_from_practical_start(d["A"], d["b"], d["c"], d["q"], opt, box.get("kind"), box.get("u"))
else:
    O.solve(d["A"], d["b"], d["c"], d["q"], d["x0"], d["y0"], d["z0"], opt, **box)
print(time.perf_counter() - t0)
"""


def oracle_single_core(p, w, seed, practical=False, reuse=0):
    """Seconds of one whole oracle solve of problem `p` in a child process whose
    BLAS and OpenMP pools are limited to one thread (None if it fails)."""
    import subprocess
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
              "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "qp.npz")
        arrays = dict(A=p["A64"], b=p["b"], c=p["c"], q=p["q"], x0=p["x0"], y0=p["y0"], z0=p["z0"])
        if p.get("box"):
            arrays.update(p["box"])
        np.savez(path, **arrays)
        cfg = json.dumps(dict(tol=w["tol"], ell=int(p["ell"]), seed=seed, reuse=reuse, practical=practical))
        try:
            res = subprocess.run([sys.executable, "-c", _SINGLE_CORE_SOLVE, ROOT, path, cfg], env=env,
                                 capture_output=True, text=True, timeout=120)
            return float(res.stdout.strip().splitlines()[-1]) if res.returncode == 0 else None
        except (subprocess.TimeoutExpired, ValueError, IndexError):
            return None


def cpu_baseline(problems, w, runs, seed, practical=False, reuse=0):
    """The oracle as it stands on this host's cores: a whole solve when one
    takes at most ~30 s (else timed components extrapolated with the GPU
    run's iteration counts)."""
    from oracle import nys_oracle as O
    cores = os.cpu_count()
    qp = problems[0]
    A64 = qp["A64"]
    t_ipm, t_pcg = oracle_component_times(A64, qp["b"], qp["c"], qp["q"], qp["x0"], qp["y0"], qp["z0"],
                                          qp["ell"], w["tol"], seed, qp.get("box"))
    ipm, pcg = runs[0]["ipm_iters"], runs[0]["pcg_iters_total"]
    est = ipm * t_ipm + pcg * t_pcg
    per_step = len(problems)
    if est * per_step <= 30.0:
        t0 = time.perf_counter()
        for p in problems:
            opt = O.Options(tol=w["tol"], ell=p["ell"], seed=seed, reuse_pcg=reuse)
            if practical:
                bx = p.get("box") or {}
                O.solve_from_practical_start(p["A64"], p["b"], p["c"], p["q"], opt, bx.get("kind"), bx.get("u"))
            else:
                O.solve(p["A64"], p["b"], p["c"], p["q"], p["x0"], p["y0"], p["z0"], opt, **(p.get("box") or {}))
        full = time.perf_counter() - t0
        out = {"value": per_step / full, "unit": "QP solves/s", "cores": cores, "kind": "oracle",
               "sample": f"whole oracle solve(s) of the same workload ({per_step} QP, {full:.2f} s)"}
        one = oracle_single_core(problems[0], w, seed, practical, reuse) if est <= 15.0 else None
        if one is not None:
            out["single_core"] = {"value": 1.0 / one, "unit": "QP solves/s", "cores": 1,
                                  "sample": f"one whole oracle solve with BLAS/OpenMP limited to one thread "
                                            f"({one:.2f} s)"}
        return out
    m, n = A64.shape
    return {"value": 1.0 / est, "unit": "QP solves/s", "cores": cores, "kind": "oracle",
            "sample": f"1 oracle IPM iteration with PCG forced to 0 ({t_ipm:.3f} s) + 10 oracle PCG iterations "
                      f"({t_pcg * 1e3:.2f} ms each) on the first {m}x{n} QP, extrapolated with the GPU run's "
                      f"counts ({ipm} IPM, {pcg} PCG iterations per solve)"}


def run_reference(args, w, rank, world):
    """Reference arm: the CPU oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    from oracle import nys_oracle as O
    probs = host_workload(w, 0)
    if probs is None:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm runs the host-generated "
                          "workloads; this workload is generated on the GPU"}), flush=True)
        return
    seed = 7
    times, sample = [], ""
    budget = 150.0 / max(1, args.steps + args.warmup)
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        done = 0
        for qp in probs:
            ell = min(w["ell"], max(1, qp.m // 4)) if w["form"] == "batch" else w["ell"]
            opt = O.Options(tol=w["tol"], ell=ell, seed=seed, reuse_pcg=args.reuse_pcg)
            if args.practical_start:
                O.solve_from_practical_start(qp.A, qp.b, qp.c, qp.q, opt, qp.kind, qp.u)
            else:
                O.solve_qp(qp, opt)
            done += 1
            if time.perf_counter() - t0 > budget:
                break
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt / done)
        sample = f"{done} of {len(probs)} QP(s) solved whole per step"
    per = statistics.mean(times)
    value = 1.0 / per
    line = {"metric": "QP solves/s to KKT tol", "value": value, "unit": "QP solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3 * len(probs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "desc": w["desc"]},
            "cpu_baseline": {"value": value, "unit": "QP solves/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "QP solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ranks

def reduce_over_ranks(ms: float, launches: int, device):
    """Replica runs (one independent workload per rank, no data-path
    collective): the job's time is the slowest rank's, its launches the sum."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, float(launches)], dtype=torch.float64, device=device)
    tmax, tsum = t.clone(), t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), int(tsum[1])


def job_throughput(steps: int, per_step: int, world: int, ms: float) -> float:
    """Whole-job units per second: every rank solves `per_step` problems per
    step (weak scaling), over the slowest rank's time."""
    return steps * per_step * world / (ms / 1e3)


# ------------------------------------------------------------------ GPU arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--host-gen", action="store_true",
                    help="generate the large precision workloads with numpy instead of on the GPU")
    ap.add_argument("--no-gemv", action="store_true",
                    help="skip the operator GEMV measurement at the large workload shapes")
    ap.add_argument("--practical-start", action="store_true",
                    help="start every solve at the practical initial point (start_mode=1) instead of the "
                         "workload's interior point")
    ap.add_argument("--max-batch", type=int, default=None,
                    help="batch workloads: solves in flight at once (worker solvers of nys_solve_batched; "
                         "default: the whole batch)")
    ap.add_argument("--reuse-pcg", type=int, default=0,
                    help="keep the Nystrom factor while both PCG solves of an IPM iteration take at most this "
                         "many iterations (0: a fresh sketch every iteration, Algorithm 6 as written)")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="precision workloads: also time one FP64-form solve of the same QP")
    ap.add_argument("--no-config3", action="store_true",
                    help="skip the record of one whole m=20000, n=100000 solve in the precision and FP64 forms "
                         "(run by default on one GPU, about 15 minutes)")
    ap.add_argument("--profile-kernel", choices=["f64_operator", "bf16_operator", "sketch_gemm", "ff_pcg", "bf16_pcg"],
                    help="run only this kernel --reps times on an m x n (x ell) case (for ncu captures)")
    ap.add_argument("--m", type=int, default=5000)
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--ell", type=int, default=400)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    if args.profile_kernel:
        profile_kernel(args)
        return
    w = WORKLOADS[args.workload]
    if args.max_batch is None:
        args.max_batch = w.get("count", 32)
    if w.get("start") == "practical":
        args.practical_start = True
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
    barrier = (lambda: dist.barrier()) if world > 1 else (lambda: None)
    seed = 7
    form = w["form"]
    stream = torch.cuda.Stream(device=dev)

    # ---- problems resident in HBM
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    host_probs = host_workload(w, rank)
    if host_probs is not None:
        dev_probs = []
        for qp in host_probs:
            ell = min(w["ell"], max(1, qp.m // 4)) if form == "batch" else w["ell"]
            pr = tuple(T(v) for v in (qp.A, qp.b, qp.c, qp.q, qp.x0, qp.y0, qp.z0)) + (ell,)
            if qp.kind is not None:      # problem (P~): kinds, upper bounds, start of s
                pr = pr + (dict(kind=T(qp.kind), u=T(qp.u), s0=T(qp.s0)),)
            dev_probs.append(pr)
    else:
        dev_probs = [device_workload(w, rank, dev, args.host_gen) + (w["ell"],)]
    mmax = max(p[0].shape[0] for p in dev_probs)
    nmax = max(p[0].shape[1] for p in dev_probs)
    a_bytes = sum(p[0].numel() * p[0].element_size() for p in dev_probs)

    with torch.cuda.stream(stream):
        if form in ("batch", "diff"):
            h = nys.Handle(mmax, nmax, ell=w["ell"], tol=w["tol"], seed=seed, max_batch=args.max_batch,
                           stream=stream, reuse_pcg=args.reuse_pcg)
        else:
            h = nys.Handle(mmax, nmax, ell=w["ell"], tol=w["tol"], seed=seed, stream=stream,
                           precision_mode={"bf16": 1, "fp8": 2}.get(form, 0),
                           start_mode=1 if args.practical_start else 0, reuse_pcg=args.reuse_pcg)
        last_sol = {}      # the last solve's iterate (compared with the FP64 form)
        # the start point the solves receive (None: the practical start computes it)
        start = (lambda pr: pr[4:7]) if not args.practical_start else (lambda pr: (None, None, None))

        def step():
            if form == "batch":
                return [r[3] for r in nys.nys_solve_batched(h, dev_probs)]
            if form == "diff":
                # forward solves of the whole batch in one call, then the adjoints
                out = []
                for k, (x, y, z, info) in enumerate(nys.nys_solve_batched(h, dev_probs)):
                    pr = dev_probs[k]
                    g = 2.0 * (x - T(host_probs[k].target))
                    nys.nys_adjoint(h, pr[0], pr[3], x, y, z, info, g, eta=1e-10)
                    out.append(info)
                return out
            out = []
            for pr in dev_probs:
                x, y, z, info = nys.nys_solve(h, *pr[:4], *start(pr), **(pr[8] if len(pr) > 8 else {}))
                last_sol["xyz"] = (x, y, z)
                if form == "diff":
                    g = 2.0 * (x - T(host_probs[len(out)].target))
                    nys.nys_adjoint(h, pr[0], pr[3], x, y, z, info, g, eta=1e-10)
                out.append(info)
            return out

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        l0 = nys.nys_kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        runs, timed = [], []
        t_wall = time.perf_counter()
        with ClockSampler(local) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                runs = step()
                timed.extend(runs)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall
        barrier()
        torch.cuda.synchronize(dev)
        launches = nys.nys_kernel_launches() - l0
        # worker streams of the batched solves are not ordered with `stream`: use the wall clock there
        ms = t_wall * 1e3 if form in ("batch", "diff") else e0.elapsed_time(e1)
        clocks = clk.summary()
        if world > 1:
            ms, launches = reduce_over_ranks(ms, launches, dev)
        per_step = len(dev_probs)
        value = job_throughput(args.steps, per_step, world, ms)

        # ---- roofline of the dominant kernel
        A0 = dev_probs[0][0]
        m0, n0 = A0.shape
        hbm_peak, bf16_peak, peak_src = measured_peaks()
        if form in ("batch", "diff"):
            # nys_solve_batched: the PCG solves of each Newton phase share cluster launches
            routes = ["cluster (shared batch launches)"]
        else:
            routes = sorted({nys.ROUTE_NAMES[nys.nys_pcg_route(h, pr[0].shape[0], pr[0].shape[1], pr[7])]
                             for pr in dev_probs}) if form not in ("bf16", "fp8") else ["graph"]
        pcg_iters = sum(i["pcg_iters_total"] for i in timed)
        pcg_s = sum(i["pcg_seconds"] for i in timed)
        pcg = {"routes": routes, "iters": pcg_iters, "device_s": pcg_s,
               "us_per_iter": 1e6 * pcg_s / max(pcg_iters, 1)}
        if form not in ("bf16", "fp8") and "graph" not in routes and pcg_s > 0:
            # one launch per PCG solve (thread-block cluster or cooperative grid):
            # that kernel dominates; its algorithmic FP64 work per iteration is
            # the operator (4 m n), the preconditioner (4 m ell) and the CG
            # vector updates and dots (12 m)
            fl = sum(pcg_flops_per_iter(pr[0].shape[0], pr[0].shape[1], pr[7]) * i["pcg_iters_total"]
                     for pr, i in zip(dev_probs * args.steps, timed))
            peak = fp64_alu_peak_tflops()
            # DRAM bytes of one launch from the committed ncu capture of this
            # workload's cluster kernel (None when the kernel changed since)
            tr = traffic_record("pcg_cluster.cu", "pcg_cluster_small-fp64") \
                if args.workload == "small-fp64" and routes == ["cluster-smem"] else None
            roofline = {"bound": "alu", "achieved": fl / pcg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "frac": fl / pcg_s / 1e12 / peak, "traffic": tr["bytes_per_launch"] if tr else None,
                        "kernel": "whole-PCG kernel (" + ", ".join(routes) + "), one launch per Newton solve",
                        "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (nominal FP64 1.25 TFLOP/s)",
                        "launch_avg_ms": 1e3 * pcg_s / max(1, 2 * sum(i["ipm_iters"] for i in timed)),
                        "algorithmic_flops": fl}
        elif form == "bf16":
            # BF16 operator: A^T pass over the BF16 transpose + A pass, FP32 accumulation
            bytes_alg = 2.0 * m0 * n0 * 2 + 4.0 * (3 * m0 + 2 * n0)
            op_s = time_lp_operator(nys, h, A0, stream)
            roofline = {"bound": "hbm", "achieved": bytes_alg / op_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                        "frac": bytes_alg / op_s / 1e9 / hbm_peak, "traffic": None,
                        "kernel": "BF16 normal-equations operator (k_rows<bf16> over A^T and A)",
                        "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})", "op_ms": op_s * 1e3,
                        "algorithmic_bytes": bytes_alg}
        elif form == "fp8":
            # FP8 operator: E4M3 A^T pass + A pass with row scales, FP32 accumulation
            bytes_alg = 2.0 * m0 * n0 * 1 + 4.0 * (4 * m0 + 2 * n0)
            op_s = time_fp8_operator(nys, h, A0, stream)
            roofline = {"bound": "hbm", "achieved": bytes_alg / op_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                        "frac": bytes_alg / op_s / 1e9 / hbm_peak, "traffic": None,
                        "kernel": "FP8 normal-equations operator (k_rows<e4m3> over Q^T and Q, row scales)",
                        "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})", "op_ms": op_s * 1e3,
                        "algorithmic_bytes": bytes_alg}
        else:
            roofline = fp64_operator_roofline(nys, h, A0, stream)
        # ---- e2e: the same solves through the C ABI from pinned host buffers
        e2e = None
        if form in ("fp64", "box", "bf16", "fp8"):
            pin = lambda t: t.detach().cpu().pin_memory()
            hp = [tuple(pin(t) for t in pr[:4]) + tuple(None if t is None else pin(t) for t in start(pr))
                  for pr in dev_probs]
            hbox = [{k: pin(t) for k, t in pr[8].items() if not (args.practical_start and k in ("s0", "w0"))}
                    if len(pr) > 8 else {} for pr in dev_probs]
            nys.nys_solve(h, *hp[0], **hbox[0])
            barrier()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                for pr, bx in zip(hp, hbox):
                    nys.nys_solve(h, *pr, **bx)
            e2e_s = time.perf_counter() - t0
            if world > 1:
                e2e_s, _ = reduce_over_ranks(e2e_s, 0, dev)
            h2d = sum(sum(t.numel() * t.element_size() for t in pr if t is not None) for pr in hp) + \
                sum(sum(t.numel() * t.element_size() for t in bx.values()) for bx in hbox)
            d2h = sum(8 * (2 * pr[0].shape[1] + pr[0].shape[0]) for pr in hp) + \
                sum(8 * 2 * pr[0].shape[1] for pr, bx in zip(hp, hbox) if bx)
            e2e = {"value": args.steps * per_step * world / e2e_s, "unit": "QP solves/s",
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        else:
            e2e = {"value": None, "unit": "QP solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                   "note": "batch/diff workloads take device tensors only"}

        # the GEMV pairs at the large workload shapes (the metric's GEMV GB/s)
        gemv = operator_rooflines(nys, dev, stream) if (rank == 0 and not args.no_gemv) else None
        # the precision form against the FP64 form on the 20000 x 100000 workload
        cfg3 = config3_record(nys, dev, stream, seed, cpu=not args.no_cpu_baseline) \
            if (world == 1 and not args.no_config3 and form not in ("bf16", "fp8")) else None

        fp64_cmp = None
        if form in ("bf16", "fp8") and args.compare_fp64:
            A64 = dev_probs[0][0].double()
            h64 = nys.Handle(m0, n0, ell=w["ell"], tol=w["tol"], seed=seed, stream=stream)
            t0 = time.perf_counter()
            x64, y64, z64, i64 = nys.nys_solve(h64, A64, *dev_probs[0][1:7], check=False)
            torch.cuda.synchronize(dev)
            t64 = time.perf_counter() - t0
            rel = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
            xl, yl, zl = last_sol["xyz"]
            fp64_cmp = {"value": 1.0 / t64, "unit": "QP solves/s", "status": i64["status"],
                        "ipm_iters": i64["ipm_iters"], "pcg_iters": i64["pcg_iters_total"],
                        "rel_primal": i64["rel_primal"], "rel_dual": i64["rel_dual"], "mu": i64["mu"],
                        # the precision form's answer against the FP64 form's (both stop at tol)
                        "precision_vs_fp64": {"x": rel(xl, x64), "y": rel(yl, y64), "z": rel(zl, z64)}}
            h64.close()
            del A64

    last = runs[0]
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            probs = []
            if host_probs is not None:
                for qp, pr in zip(host_probs[:4], dev_probs[:4]):
                    box = dict(kind=qp.kind, u=qp.u, s0=qp.s0) if qp.kind is not None else None
                    probs.append(dict(A64=qp.A, b=qp.b, c=qp.c, q=qp.q, x0=qp.x0, y0=qp.y0, z0=qp.z0, ell=pr[7],
                                      box=box))
            else:
                pr = dev_probs[0]
                probs.append(dict(A64=pr[0].double().cpu().numpy(), b=pr[1].cpu().numpy(), c=pr[2].cpu().numpy(),
                                  q=pr[3].cpu().numpy(), x0=pr[4].cpu().numpy(), y0=pr[5].cpu().numpy(),
                                  z0=pr[6].cpu().numpy(), ell=pr[7]))
            cpu = cpu_baseline(probs, w, runs, seed, args.practical_start, args.reuse_pcg)
        line = {
            "metric": "QP solves/s to KKT tol", "value": value, "unit": "QP solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "box": "f64", "bf16": "bf16", "fp8": "fp8e4m3", "batch": "f64",
                      "diff": "f64"}[form],
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"], "form": form, "qps_per_step": per_step,
                       "start": "practical initial point" if args.practical_start else "workload interior point",
                       "max_batch": args.max_batch if form in ("batch", "diff") else None,
                       "inflight_tuned": nys.nys_batch_inflight(h) if form in ("batch", "diff") else None,
                       "reuse_pcg": args.reuse_pcg,
                       "m_max": mmax, "n_max": nmax, "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 (A = {a_bytes / 1e6:.0f} MB)" if a_bytes > 129e6
                       else f"A = {a_bytes / 1e6:.1f} MB fits in L2 (no flush; latency-bound)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
            "solve": {"status": max(r["status"] for r in runs), "ipm_iters": last["ipm_iters"],
                      "sketches": last.get("sketches"),
                      "pcg_iters": last["pcg_iters_total"], "refine_steps": last["refine_steps"],
                      "rel_primal": max(r["rel_primal"] for r in runs), "rel_dual": max(r["rel_dual"] for r in runs),
                      "mu": max(r["mu"] for r in runs)},
        }
        if fp64_cmp is not None:
            line["fp64_form_same_qp"] = fp64_cmp
        line["pcg"] = pcg
        if gemv is not None:
            line["gemv"] = gemv
        if cfg3 is not None:
            line["config3"] = cfg3
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


def profile_kernel(args):
    """A few launches of one kernel on a bounded case, CUDA-event timed."""
    import torch
    from paper_2404_14524_gb300 import build
    build.build()
    from paper_2404_14524_gb300 import nys
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(0)
    m, n, reps = args.m, args.n, args.reps
    if args.profile_kernel == "f64_operator":
        A = torch.randn(m, n, generator=g, device=dev, dtype=torch.float64)
        h = nys.Handle(m, n, ell=8)
        D = torch.rand(n, generator=g, device=dev, dtype=torch.float64) + 0.5
        v = torch.randn(m, generator=g, device=dev, dtype=torch.float64)
        run = lambda: nys.nys_normal_matvec(h, A, D, 1e-3, v)
        work = {"bytes": 16.0 * m * n, "flops": 4.0 * m * n}
    elif args.profile_kernel == "bf16_operator":
        A = (torch.randn(m, n, generator=g, device=dev) / 100).to(torch.bfloat16)
        AT = A.T.contiguous()
        h = nys.Handle(m, n, ell=8, precision_mode=1)
        D = torch.rand(n, generator=g, device=dev, dtype=torch.float64) + 0.5
        v = torch.randn(m, generator=g, device=dev, dtype=torch.float64)
        run = lambda: nys.nys_normal_matvec_lp(h, A, AT, D, 1e-3, v)
        work = {"bytes": 4.0 * m * n, "flops": 4.0 * m * n}
    elif args.profile_kernel in ("ff_pcg", "bf16_pcg"):
        # forced PCG iterations on the precision form's operator (graph route)
        ell = min(args.ell, 64)
        A32 = torch.randn(m, n, generator=g, device=dev) / n ** 0.5
        h = nys.Handle(m, n, ell=ell, precision_mode=1)
        D = torch.rand(n, generator=g, device=dev, dtype=torch.float64) + 0.5
        U = torch.zeros(ell, m, device=dev, dtype=torch.float64)     # orthonormal columns e_0 .. e_{ell-1}
        U[torch.arange(ell, device=dev), torch.arange(ell, device=dev)] = 1.0
        lam = torch.linspace(10.0, 1.0, ell, device=dev, dtype=torch.float64)
        xi = torch.randn(m, generator=g, device=dev, dtype=torch.float64)
        opk = "ff" if args.profile_kernel == "ff_pcg" else "bf16"
        iters = 40
        run = lambda: nys.nys_pcg_lp(h, A32, opk, D, 1e-3, U, lam, xi, 0.0, iters, forced=iters)
        per = 8.0 if opk == "ff" else 4.0
        work = {"bytes": per * m * n * iters, "flops": 4.0 * m * n * iters}
    else:
        ell = args.ell
        A = (torch.randn(m, n, generator=g, device=dev) / 100).to(torch.bfloat16)
        B = (torch.randn(ell, n, generator=g, device=dev) / 100).to(torch.bfloat16)
        h = nys.Handle(m, n, ell=ell, precision_mode=1)   # workspace sized for K=n: split-K is not capped
        run = lambda: nys.nys_gemm_bf16(h, A, B)
        work = {"bytes": 2.0 * m * n, "flops": 2.0 * m * n * ell}
    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / reps / 1e3
    print(json.dumps({"kernel": args.profile_kernel, "m": m, "n": n, "reps": reps, "ms": sec * 1e3,
                      "GB/s": work["bytes"] / sec / 1e9, "TFLOP/s": work["flops"] / sec / 1e12}), flush=True)


def pcg_flops_per_iter(m, n, ell):
    """Algorithmic FP64 flops of one PCG iteration: A^T p and A t (4 m n),
    U^T r and U s (4 m ell), and the CG dots and updates (12 m)."""
    return 4.0 * m * n + 4.0 * m * ell + 12.0 * m


def fp64_operator_roofline(nys, h, A0, stream, reps=50):
    """FP64 operator (A^T pass, reduction, A pass) timed with CUDA events on
    `stream`: DFMA-bound, reported against the nominal FP64 rate."""
    import torch
    dev = A0.device
    m0, n0 = A0.shape
    flops = 4.0 * m0 * n0
    bytes_alg = 2.0 * m0 * n0 * 8 + 8.0 * (3 * m0 + 2 * n0)
    D = torch.rand(n0, dtype=torch.float64, device=dev) + 0.5
    v = torch.randn(m0, dtype=torch.float64, device=dev)
    out = torch.empty_like(v)
    for _ in range(3):
        nys.nys_normal_matvec(h, A0, D, 1e-3, v, out)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(reps):
        nys.nys_normal_matvec(h, A0, D, 1e-3, v, out)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    op_s = f0.elapsed_time(f1) / reps / 1e3
    peak = fp64_alu_peak_tflops()
    tr = traffic_record("gemv_f64.cu", "fp64_operator")
    return {"bound": "alu", "achieved": flops / op_s / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": flops / op_s / 1e12 / peak,
            "traffic": (tr["bytes_per_element"] * m0 * n0) if tr else None,
            "kernel": "FP64 normal-equations operator (k_atv_partial + k_atv_reduce + k_av)",
            "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (nominal FP64 1.25 TFLOP/s)",
            "hbm_gbs": bytes_alg / op_s / 1e9, "op_ms": op_s * 1e3,
            "algorithmic_flops": flops, "algorithmic_bytes": bytes_alg}


def config3_record(nys, dev, stream, seed, cpu=True):
    """The metric's "BF16+refine vs FP64 form" on its own configuration: one
    whole solve of the m=20000, n=100000, ell=400, tol 1e-6 workload in the
    precision form (BF16 inner PCG + FP32 / float-float refinement) and one in
    the FP64 form on the same QP (the FP32 matrix defines the problem), each
    timed from the call to its return; the precision form's answer relative to
    the FP64 form's (the oracle cannot solve this size in bench time: its
    per-component times on this QP, extrapolated with the GPU's counts, are
    reported instead)."""
    import torch
    w = WORKLOADS["precision-20000x100000"]
    t_all = time.perf_counter()
    rec = {"workload": "precision-20000x100000", "desc": w["desc"]}
    with torch.cuda.stream(stream):
        A, b, c, q, x0, y0, z0 = device_workload(w, 0, dev)
        m, n = A.shape
        forms = {}
        sols = {}
        for name, mode in (("bf16_refine", 1), ("fp64", 0)):
            Ause = A if mode else A.double()
            h = nys.Handle(m, n, ell=w["ell"], tol=w["tol"], seed=seed, stream=stream, precision_mode=mode)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            x, y, z, info = nys.nys_solve(h, Ause, b, c, q, x0, y0, z0, check=False)
            torch.cuda.synchronize(dev)
            t = time.perf_counter() - t0
            h.close()
            del Ause
            sols[name] = (x, y, z)
            forms[name] = {"value": 1.0 / t, "unit": "QP solves/s", "seconds": t, "status": info["status"],
                           "ipm_iters": info["ipm_iters"], "pcg_iters": info["pcg_iters_total"],
                           "refine_steps": info["refine_steps"], "pcg_device_s": info["pcg_seconds"],
                           "rel_primal": info["rel_primal"], "rel_dual": info["rel_dual"], "mu": info["mu"],
                           "rel_gap": info["rel_gap"],
                           "kkt_met": max(info["rel_primal"], info["rel_dual"], info["mu"]) <= w["tol"]}
        rel = lambda a, b_: float(torch.linalg.norm(a - b_) / torch.linalg.norm(b_))
        (xb, yb, zb), (xf, yf, zf) = sols["bf16_refine"], sols["fp64"]
        rec["forms"] = forms
        rec["precision_vs_fp64"] = {"x": rel(xb, xf), "y": rel(yb, yf), "z": rel(zb, zf)}
        rec["speedup_bf16_refine_over_fp64"] = forms["fp64"]["seconds"] / forms["bf16_refine"]["seconds"]
        if cpu:
            A64 = A.double().cpu().numpy()
            t_ipm, t_pcg = oracle_component_times(A64, b.cpu().numpy(), c.cpu().numpy(), q.cpu().numpy(),
                                                  x0.cpu().numpy(), y0.cpu().numpy(), z0.cpu().numpy(),
                                                  w["ell"], w["tol"], seed)
            del A64
            ipm, pcg = forms["fp64"]["ipm_iters"], forms["fp64"]["pcg_iters"]
            est = ipm * t_ipm + pcg * t_pcg
            rec["cpu_baseline"] = {"value": 1.0 / est, "unit": "QP solves/s", "cores": os.cpu_count(),
                                   "kind": "oracle",
                                   "sample": f"1 oracle IPM iteration with PCG forced to 0 ({t_ipm:.1f} s) + 10 "
                                             f"oracle PCG iterations ({t_pcg:.3f} s each) on this QP, "
                                             f"extrapolated with the FP64 form's counts ({ipm} IPM, {pcg} PCG)"}
        del A, b, c, q, x0, y0, z0, sols, xb, yb, zb, xf, yf, zf
        torch.cuda.empty_cache()
    rec["wall_s"] = time.perf_counter() - t_all
    return rec


def operator_rooflines(nys, dev, stream):
    """The operator GEMV pairs at the large workload shapes (inputs far larger
    than L2, random entries): FP64 at m=5000, n=20000, BF16 and FP8 (E4M3,
    row scales) at m=20000, n=100000; and the sketch's two tensor-core
    products at m=20000, n=100000, ell=400."""
    import torch
    out = {}
    g = torch.Generator(device=dev).manual_seed(0)
    with torch.cuda.stream(stream):
        A = torch.randn(5000, 20000, generator=g, device=dev, dtype=torch.float64)
        h = nys.Handle(5000, 20000, ell=8, stream=stream)
        out["fp64_5000x20000"] = fp64_operator_roofline(nys, h, A, stream, reps=20)
        h.close()
        del A
        m, n = 20000, 100000
        A32 = torch.randn(m, n, generator=g, device=dev, dtype=torch.float32)
        h8 = nys.Handle(m, n, ell=8, precision_mode=2, stream=stream)
        op8_s = time_fp8_operator(nys, h8, A32, stream)
        h8.close()
        A = A32.to(torch.bfloat16)
        AT = A32.T.contiguous().to(torch.bfloat16)
        del A32
        h = nys.Handle(m, n, ell=8, precision_mode=1, stream=stream)
        D = torch.rand(n, dtype=torch.float64, device=dev) + 0.5
        v = torch.randn(m, dtype=torch.float64, device=dev)
        o = torch.empty_like(v)
        for _ in range(3):
            nys.nys_normal_matvec_lp(h, A, AT, D, 1e-3, v, o)
        reps = 20
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(reps):
            nys.nys_normal_matvec_lp(h, A, AT, D, 1e-3, v, o)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        op_s = f0.elapsed_time(f1) / reps / 1e3
        h.close()
        hs = nys.Handle(m, n, ell=400, precision_mode=1, stream=stream)
        out["sketch_gemm_20000x100000x400"] = sketch_gemm_record(nys, hs, A, AT, stream)
        hs.close()
        del A, AT
    hbm_peak, _, src = measured_peaks()
    bytes_alg = 2.0 * m * n * 2 + 4.0 * (3 * m + 2 * n)
    out["bf16_20000x100000"] = {"bound": "hbm", "achieved": bytes_alg / op_s / 1e9, "peak": hbm_peak,
                                "unit": "GB/s", "frac": bytes_alg / op_s / 1e9 / hbm_peak, "op_ms": op_s * 1e3,
                                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src})"}
    b8 = 2.0 * m * n + 4.0 * (4 * m + 2 * n)
    out["fp8_20000x100000"] = {"bound": "hbm", "achieved": b8 / op8_s / 1e9, "peak": hbm_peak,
                               "unit": "GB/s", "frac": b8 / op8_s / 1e9 / hbm_peak, "op_ms": op8_s * 1e3,
                               "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src})"}
    torch.cuda.empty_cache()
    return out


def sketch_gemm_record(nys, h, A, AT, stream, ell=400, reps=10):
    """The precision form's two sketch products (Algorithm 1, second step) at
    m=20000, n=100000, ell=400: T = A^T Omega (M = n, K = m) and Y = A T'
    (M = m, K = n), 2 m n ell flop each, BF16 operands with FP32
    accumulation, inputs far larger than L2.  Each product is timed alone with
    CUDA events on `stream` over `reps` calls of nys_gemm_bf16 (the product
    and, where tiles are split across CTA pairs, the fixed-order sum of their
    partials; one host synchronisation per call is inside the timed region)."""
    import torch
    dev = A.device
    m, n = A.shape
    g = torch.Generator(device=dev).manual_seed(1)
    Om = torch.randn(ell, m, generator=g, device=dev).to(torch.bfloat16)
    Tt = (torch.randn(ell, n, generator=g, device=dev) / 100).to(torch.bfloat16)
    _, peak, src = measured_peaks()
    prods = {}
    for key, X, B in (("T = A^T Omega", AT, Om), ("Y = A T'", A, Tt)):
        out = torch.empty((ell, X.shape[0]), dtype=torch.float32, device=dev)
        for _ in range(3):
            nys.nys_gemm_bf16(h, X, B, out=out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            nys.nys_gemm_bf16(h, X, B, out=out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        sec = e0.elapsed_time(e1) / reps / 1e3
        fl = 2.0 * X.shape[0] * X.shape[1] * ell
        prods[key] = {"M": X.shape[0], "K": X.shape[1], "N": ell, "ms": sec * 1e3, "achieved": fl / sec / 1e12,
                      "frac": fl / sec / 1e12 / peak}
        del out
    tot_fl = sum(2.0 * v["M"] * v["K"] * ell for v in prods.values())
    tot_s = sum(v["ms"] for v in prods.values()) / 1e3
    tr = traffic_record("umma_bf16.cu", "sketch_gemm_pair_8000x40000")
    return {"bound": "tensor", "achieved": tot_fl / tot_s / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": tot_fl / tot_s / 1e12 / peak, "products": prods,
            "traffic_ncu_8000x40000x400": None if tr is None else {
                "bytes_per_launch": tr["bytes_per_launch"], "algorithmic_bytes": tr["algorithmic_bytes"]},
            "kernel": "k_umma_gemm_pair (tcgen05.mma.cta_group::2) + k_pair_reduce",
            "peak_source": f"MEASURED_PEAKS.json bf16_tflops, burst ({src})"}


def time_fp8_operator(nys, h, A32, stream, reps=20):
    """Average duration of the FP8 operator pair (E4M3 copies with row scales
    made by the library from the FP32 A), CUDA events on `stream`."""
    import torch
    dev = A32.device
    m, n = A32.shape
    Q, QT, sc = nys.nys_quantize_fp8(h, A32)
    D = torch.rand(n, dtype=torch.float64, device=dev) + 0.5
    v = torch.randn(m, dtype=torch.float64, device=dev)
    out = torch.empty_like(v)
    for _ in range(3):
        nys.nys_normal_matvec_fp8(h, m, n, Q, QT, sc, D, 1e-3, v, out)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(reps):
        nys.nys_normal_matvec_fp8(h, m, n, Q, QT, sc, D, 1e-3, v, out)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    del Q, QT
    return f0.elapsed_time(f1) / reps / 1e3


def time_lp_operator(nys, h, A32, stream):
    """Average duration of the precision form's BF16 operator pair (A^T pass
    over the BF16 transpose, then the A pass), CUDA events on `stream`."""
    import torch
    dev = A32.device
    m, n = A32.shape
    Ab = A32.to(torch.bfloat16)
    AbT = A32.T.contiguous().to(torch.bfloat16)
    D = torch.rand(n, dtype=torch.float64, device=dev) + 0.5
    v = torch.randn(m, dtype=torch.float64, device=dev)
    out = torch.empty_like(v)
    for _ in range(3):
        nys.nys_normal_matvec_lp(h, Ab, AbT, D, 1e-3, v, out)
    reps = 20
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(reps):
        nys.nys_normal_matvec_lp(h, Ab, AbT, D, 1e-3, v, out)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    del Ab, AbT
    return f0.elapsed_time(f1) / reps / 1e3


if __name__ == "__main__":
    main()
