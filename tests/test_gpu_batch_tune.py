"""The batching form's PCG cluster-plan autotuner (the project's autotuner for
cluster size and tile shape; NYS_BATCH_PLAN_TUNE=0 turns it off): a batch of
128 QPs of uneven shapes tunes each shape bucket once before any problem
starts (nys_batch_plan reports the choice), every QP meets the KKT tolerance
of (P)/(D), and a second call, running the cached plans, reproduces every
result bit for bit."""
import numpy as np
import pytest
import torch

from oracle import nys_oracle as O
from paper_2404_14524_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def nys():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_14524_gb300 import build
    build.build()
    from paper_2404_14524_gb300 import nys as N
    N.lib()
    return N


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def test_plan_autotuner_tunes_buckets_and_keeps_results(nys, monkeypatch):
    monkeypatch.setenv("NYS_BATCH_TUNE", "1")
    monkeypatch.setenv("NYS_BATCH_PLAN_TUNE", "1")
    qps = synth.workload_batch(seed=21, count=128, m_lo=64, m_hi=200)
    mx, nx = max(q.m for q in qps), max(q.n for q in qps)
    ell = 16
    h = nys.Handle(mx, nx, ell=ell, tol=1e-6, seed=3, max_batch=16)
    probs = [tuple(T(v) for v in (q.A, q.b, q.c, q.q, q.x0, q.y0, q.z0)) for q in qps]
    # nothing is tuned before the first large batch
    assert nys.nys_batch_plan(h, qps[0].m, qps[0].n, min(ell, qps[0].m))[0] is False
    res = nys.nys_solve_batched(h, probs)
    for q, (x, y, z, info) in zip(qps, res):
        assert info["status"] == 0 and info["device_iteration"] == 1
        rp, rd, mu = O.kkt_measures(q.A, q.b, q.c, q.q, *(t.cpu().numpy() for t in (x, y, z)))
        assert max(rp, rd, mu) <= 1e-6
    for q in qps:
        tuned, ctas, a_smem = nys.nys_batch_plan(h, q.m, q.n, min(ell, q.m))
        assert tuned and ctas in (4, 8, 16) and a_smem in (0, 1)
        assert a_smem == 1 or ctas in (4, 8)
    res2 = nys.nys_solve_batched(h, probs)
    for (x, y, z, i1), (x2, y2, z2, i2) in zip(res, res2):
        assert torch.equal(x, x2) and torch.equal(y, y2) and torch.equal(z, z2)
        assert i1["ipm_iters"] == i2["ipm_iters"] and i1["pcg_log"] == i2["pcg_log"]
