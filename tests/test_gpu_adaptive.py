"""The adaptive sketch size on the GPU against the oracle: with the oracle's
PCG counts forced, the library builds its factors with the same sequence of
sketch sizes and reaches the same iterates (well-conditioned trajectory:
1e-9, or 100x the oracle's own rounding response where that is higher); a
free-running adaptive solve meets the KKT tolerance; the option is rejected
with preconditioner reuse and in the batching form."""
import dataclasses

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


def relerr(got, want):
    got = got.detach().cpu().numpy() if isinstance(got, torch.Tensor) else got
    return np.linalg.norm(got - want) / np.linalg.norm(want)


def _response(qp, opt, rec):
    orig = O.gaussian_omega

    def pert(seed, kk, m, ell):
        om = orig(seed, kk, m, ell)
        return om * (1 + 2e-16 * np.sign(np.sin(np.arange(om.size))).reshape(om.shape))
    O.gaussian_omega = pert
    try:
        b = O.solve_qp(qp, dataclasses.replace(opt, forced_pcg=rec.pcg_iters, forced_ipm=rec.ipm_iters))
    finally:
        O.gaussian_omega = orig
    return max(relerr(b.x, rec.x), relerr(b.y, rec.y), relerr(b.z, rec.z))


@pytest.mark.parametrize("cost", [10, 40])
def test_adaptive_sketch_sizes_and_iterates_match_oracle(nys, cost):
    qp = synth.gaussian_qp(11, 512, 2048)
    opt = O.Options(tol=1e-8, ell=32, seed=7, adapt_cost=cost)
    rec = O.solve_qp(qp, opt)
    assert rec.status == "converged"
    ells = [e.ell for e in rec.trace]
    assert len(set(ells)) > 1, ells                  # the size did change
    floor = _response(qp, opt, rec)
    h = nys.Handle(qp.m, qp.n, ell=32, tol=1e-8, seed=7, adapt_cost=cost, forced_pcg=rec.pcg_iters,
                   forced_ipm=rec.ipm_iters)
    x, y, z, info = nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))
    assert info["ell_log"] == ells
    assert info["pcg_log"] == rec.pcg_iters and info["sketches"] == len(ells)
    errs = [relerr(g, w) for g, w in ((x, rec.x), (y, rec.y), (z, rec.z))]
    print(f"cost={cost} ells={ells} errs={errs} floor={floor:.1e}")
    assert max(errs) <= max(1e-9, 100 * floor)


def test_free_running_adaptive_solve_meets_kkt(nys):
    qp = synth.workload_small()
    h = nys.Handle(qp.m, qp.n, ell=20, tol=1e-6, seed=3, adapt_cost=40)
    x, y, z, info = nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))
    assert info["status"] == 0 and info["ell_log"][0] == 2 and max(info["ell_log"]) <= 20
    rp, rd, mu = O.kkt_measures(qp.A, qp.b, qp.c, qp.q, *(t.cpu().numpy() for t in (x, y, z)))
    assert max(rp, rd, mu) <= 1e-6


def test_adaptive_rejected_with_reuse_and_in_batches(nys):
    qp = synth.workload_small()
    args = [T(v) for v in (qp.A, qp.b, qp.c, qp.q, qp.x0, qp.y0, qp.z0)]
    h = nys.Handle(qp.m, qp.n, ell=20, adapt_cost=40, reuse_pcg=10)
    with pytest.raises(nys.NysError) as e:
        nys.nys_solve(h, *args)
    assert e.value.code == nys.NYS_ERR_ARG
    hb = nys.Handle(qp.m, qp.n, ell=20, adapt_cost=40, max_batch=2)
    with pytest.raises(nys.NysError) as e:
        nys.nys_solve_batched(hb, [tuple(args)])
    assert e.value.code == nys.NYS_ERR_ARG
