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


def _omega_response(qp, opt, rec):
    """How far the oracle's own final iterate moves when every Omega_k is
    perturbed by 2e-16 relative, with the iteration counts held: the rounding
    noise floor of a whole solve on this problem."""
    import dataclasses
    orig = O.gaussian_omega

    def pert(seed, kk, m, ell):
        om = orig(seed, kk, m, ell)
        return om * (1 + 2e-16 * np.sign(np.sin(np.arange(om.size))).reshape(om.shape))
    O.gaussian_omega = pert
    try:
        b = O.solve_qp(qp, dataclasses.replace(opt, forced_pcg=rec.pcg_iters, forced_ipm=rec.ipm_iters))
    finally:
        O.gaussian_omega = orig
    rel = lambda u, v: np.linalg.norm(u - v) / np.linalg.norm(v)
    return max(rel(b.x, rec.x), rel(b.y, rec.y), rel(b.z, rec.z))


def test_batched_matches_oracle_with_forced_counts(nys):
    """QPs shaped like the 256-QP batching workload (m up to 1024, n in
    [4m, 8m], sigma_i = 1/i, ell = min(32, m/4)) solved in one batched call,
    each with its own recorded oracle PCG and IPM counts: every iterate
    matches the oracle's element by element, to 1e-9 relative or 100x the
    oracle's own rounding response where that floor is higher.  The largest
    systems run on thread-block clusters that read A from L2."""
    shapes = [(1024, 6144), (700, 3500), (300, 1800), (96, 500)]
    qps = [synth.spectral_qp(5000 + m, m, n, "inv", "uniform") for m, n in shapes]
    ells = [min(32, m // 4) for m, _ in shapes]
    recs, floors = [], []
    for qp, ell in zip(qps, ells):
        opt = O.Options(ell=ell, tol=1e-6, seed=9)
        rec = O.solve_qp(qp, opt)
        assert rec.status == "converged"
        recs.append(rec)
        floors.append(_omega_response(qp, opt, rec))
    mx, nx = max(q.m for q in qps), max(q.n for q in qps)
    hb = nys.Handle(mx, nx, ell=32, tol=1e-6, seed=9, max_batch=len(qps))
    probs = [tuple(T(v) for v in (q.A, q.b, q.c, q.q, q.x0, q.y0, q.z0)) + (ell,) for q, ell in zip(qps, ells)]
    res = nys.nys_solve_batched(hb, probs, forced=[(r.pcg_iters, r.ipm_iters) for r in recs])
    for qp, rec, fl, (x, y, z, info) in zip(qps, recs, floors, res):
        assert info["ipm_iters"] == rec.ipm_iters and info["pcg_log"] == rec.pcg_iters
        tol = max(1e-9, 100 * fl)
        errs = [float(np.linalg.norm(g.cpu().numpy() - w) / np.linalg.norm(w))
                for g, w in ((x, rec.x), (y, rec.y), (z, rec.z))]
        print(f"m={qp.m} n={qp.n} errs={errs} floor={fl:.1e}")
        assert max(errs) <= tol
        assert info["rel_primal"] <= 1e-6 and info["rel_dual"] <= 1e-6 and info["mu"] <= 1e-6
        rtol = max(1e-6, 10 * tol)
        assert info["rho"] == pytest.approx(rec.rho, rel=rtol) and info["delta"] == pytest.approx(rec.delta, rel=rtol)
