"""bench.py on the CPU: the reference arm (the oracle on the host cores)
prints one JSON line with the contract's keys, and the CPU-baseline helpers
report rates in QP solves per second."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "small-fp64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_cpu_baseline_rates_count_every_sampled_problem():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2404_14524_gb300 import synth
    w = dict(bench.WORKLOADS["small-fp64"])
    qps = [synth.spectral_qp(60 + i, 40, 100, "inv") for i in range(3)]
    probs = [dict(A64=q.A, b=q.b, c=q.c, q=q.q, x0=q.x0, y0=q.y0, z0=q.z0, ell=8, box=None) for q in qps]
    out = bench.cpu_baseline(probs, w, [{"ipm_iters": 20, "pcg_iters_total": 200}], 7)
    # three QPs in `full` seconds: the rate is 3 / full, i.e. the sample says so
    # (the sample prints the time rounded to 0.01 s)
    full = float(out["sample"].split(",")[-1].split("s)")[0])
    assert 3 / (full + 0.006) <= out["value"] <= 3 / max(full - 0.006, 1e-9)
    assert out["single_core"]["cores"] == 1 and out["single_core"]["value"] > 0
