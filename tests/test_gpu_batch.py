"""The batching form: many uneven QPs in one nys_solve_batched call give the
same iterates as the same QPs submitted one per call and as plain nys_solve
(bit for bit: every reduction is deterministic and every launch shape depends
on the problem alone, not on what else runs), and meet the KKT tolerance."""
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
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_batched_equals_sequential_and_meets_kkt(nys):
    qps = synth.workload_batch(seed=42, count=10, m_lo=64, m_hi=200)
    mx, nx = max(q.m for q in qps), max(q.n for q in qps)
    probs = [tuple(T(v) for v in (q.A, q.b, q.c, q.q, q.x0, q.y0, q.z0)) for q in qps]
    hb = nys.Handle(mx, nx, ell=16, tol=1e-6, seed=9, max_batch=4)
    res = nys.nys_solve_batched(hb, probs)
    h1 = nys.Handle(mx, nx, ell=16, tol=1e-6, seed=9, max_batch=1)
    hs = nys.Handle(mx, nx, ell=16, tol=1e-6, seed=9)
    for qp, pr, (x, y, z, info) in zip(qps, probs, res):
        assert info["status"] == 0
        (x1, y1, z1, inf1), = nys.nys_solve_batched(h1, [pr])
        assert torch.equal(x, x1) and torch.equal(y, y1) and torch.equal(z, z1)
        assert info["ipm_iters"] == inf1["ipm_iters"] and info["pcg_iters_total"] == inf1["pcg_iters_total"]
        rp, rd, mu = O.kkt_measures(qp.A, qp.b, qp.c, qp.q, *(t.cpu().numpy() for t in (x, y, z)))
        assert rp <= 1e-6 and rd <= 1e-6 and mu <= 1e-6
        xs, ys, zs, inf2 = nys.nys_solve(hs, *pr)
        assert torch.equal(x, xs) and torch.equal(y, ys) and torch.equal(z, zs)


def test_batched_requires_a_batch_handle(nys):
    h = nys.Handle(16, 100, ell=4)
    qp = synth.workload_batch(seed=1, count=1, m_lo=8, m_hi=10)[0]
    with pytest.raises(nys.NysError) as e:
        nys.nys_solve_batched(h, [tuple(T(v) for v in (qp.A, qp.b, qp.c, qp.q, qp.x0, qp.y0, qp.z0))])
    assert "max_batch" in str(e.value)
