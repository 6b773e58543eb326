"""The device-resident IPM iteration (every scalar decision of Algorithm 6 on
the GPU, one CUDA-graph launch per IPM iteration) against the host-driven
phases and against the oracle: the same iterates bit for bit (both paths
round alike), the oracle's iterates where its trajectory is insensitive to
rounding, the termination variants (forced and maximum iteration counts),
the PMM update's state for a resumed solve, the batching form with
per-problem counts, and a non-finite input reported as an error status."""
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


def _handle(nys, monkeypatch, device, m, n, **kw):
    monkeypatch.setenv("NYS_DEVICE_IPM", "1" if device else "0")
    h = nys.Handle(m, n, **kw)
    monkeypatch.delenv("NYS_DEVICE_IPM")
    return h


def _args(qp):
    return [T(v) for v in (qp.A, qp.b, qp.c, qp.q, qp.x0, qp.y0, qp.z0)]


@pytest.mark.parametrize("seed,tol", [(1235, 1e-6), (77, 1e-8)])
def test_device_iteration_equals_host_phases(nys, monkeypatch, seed, tol):
    qp = synth.workload_small(seed=seed)
    args = _args(qp)
    hd = _handle(nys, monkeypatch, True, qp.m, qp.n, ell=20, tol=tol, seed=3)
    hh = _handle(nys, monkeypatch, False, qp.m, qp.n, ell=20, tol=tol, seed=3)
    xd, yd, zd, idv = nys.nys_solve(hd, *args, want_pmm=True)
    xh, yh, zh, ih = nys.nys_solve(hh, *args, want_pmm=True)
    assert idv["device_iteration"] == 1 and ih["device_iteration"] == 0
    for a, b in ((xd, xh), (yd, yh), (zd, zh), (idv["lam"], ih["lam"]), (idv["zeta"], ih["zeta"])):
        assert torch.equal(a, b)
    for k in ("status", "ipm_iters", "pcg_iters_total", "sketches", "rho", "delta", "mu", "rel_primal",
              "rel_dual", "peu_ref_p", "peu_ref_d"):
        assert idv[k] == ih[k], k
    assert idv["pcg_log"] == ih["pcg_log"]
    assert idv["pcg_seconds"] > 0.0


def test_device_iteration_follows_the_oracle(nys, monkeypatch):
    """512 x 2048 Gaussian QP to tol 1e-8 with the oracle's counts: the
    oracle's trajectory is insensitive to rounding there (final iterate
    moves ~1e-15 under a 2e-16 change of Omega), so the device-resident
    solve must match it to 1e-9, and reach the same PMM parameters.  A is
    8 MB, beyond a cluster's shared memory: the cluster route that reads A
    from L2 is selected (the batching form's route) so that this single
    solve takes the device-resident path."""
    qp = synth.gaussian_qp(11, 512, 2048)
    rec = O.solve_qp(qp, O.Options(tol=1e-8, ell=32, seed=7))
    monkeypatch.setenv("NYS_PCG_PATH", "cluster")
    h = _handle(nys, monkeypatch, True, qp.m, qp.n, ell=32, tol=1e-8, seed=7, forced_pcg=rec.pcg_iters,
                forced_ipm=rec.ipm_iters)
    monkeypatch.delenv("NYS_PCG_PATH")
    assert nys.nys_pcg_route(h, qp.m, qp.n, 32) == nys.NYS_ROUTE_CLUSTER_L2
    x, y, z, info = nys.nys_solve(h, *_args(qp))
    assert info["device_iteration"] == 1
    assert info["ipm_iters"] == rec.ipm_iters and info["pcg_log"] == rec.pcg_iters
    assert max(relerr(x, rec.x), relerr(y, rec.y), relerr(z, rec.z)) <= 1e-9
    assert info["rho"] == pytest.approx(rec.rho, rel=1e-9) and info["delta"] == pytest.approx(rec.delta, rel=1e-9)


@pytest.mark.parametrize("max_ipm,forced_ipm,status", [(3, -1, 1), (200, 4, 1), (200, 0, 1)])
def test_device_iteration_termination_variants(nys, monkeypatch, max_ipm, forced_ipm, status):
    qp = synth.workload_small(seed=5)
    args = _args(qp)
    res = []
    for device in (True, False):
        h = _handle(nys, monkeypatch, device, qp.m, qp.n, ell=20, tol=1e-6, seed=1, max_ipm_iter=max_ipm,
                    forced_ipm=forced_ipm)
        res.append(nys.nys_solve(h, *args, check=False))
    (xd, _, _, idv), (xh, _, _, ih) = res
    want_iters = forced_ipm if forced_ipm >= 0 else max_ipm
    assert idv["ipm_iters"] == ih["ipm_iters"] == want_iters
    assert idv["status"] == ih["status"] == status
    assert torch.equal(xd, xh)


def test_device_iteration_resumes_from_a_saved_state(nys, monkeypatch):
    """One oracle state resumed on the device path (lambda, zeta, rho, delta,
    the PMM references and k0) gives the oracle's next iterate."""
    qp = synth.workload_small()
    ref = O.solve_qp(qp, O.Options(tol=1e-6, ell=20, seed=7), record=True)
    k = 4
    t, nxt = ref.trace[k], ref.trace[k + 1]
    x, y, z, lam, zeta = t.state
    h = _handle(nys, monkeypatch, True, qp.m, qp.n, ell=20, tol=1e-6, seed=7, forced_pcg=[t.pcg_pred, t.pcg_corr],
                forced_ipm=1, rho0=t.rho, delta0=t.delta)
    gx, gy, gz, info = nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), T(x), T(y), T(z), lam0=T(lam),
                                     zeta0=T(zeta), k0=k, peu_ref=t.ref, want_pmm=True)
    assert info["device_iteration"] == 1
    assert max(relerr(gx, nxt.state[0]), relerr(gy, nxt.state[1]), relerr(gz, nxt.state[2])) <= 1e-9
    assert info["rho"] == pytest.approx(nxt.rho, rel=1e-9) and info["delta"] == pytest.approx(nxt.delta, rel=1e-9)
    assert relerr(info["lam"], nxt.state[3]) <= 1e-9 and relerr(info["zeta"], nxt.state[4]) <= 1e-9


def test_batched_device_iterations_equal_single_solves(nys, monkeypatch):
    """Problems of the batching workload's shapes in one nys_solve_batched
    call (no lock step: each advances at its own pace) give the same bits
    as the same problems solved one per call on the same path."""
    qps = synth.workload_batch(seed=43, count=6, m_lo=64, m_hi=240)
    mx, nx = max(q.m for q in qps), max(q.n for q in qps)
    hb = _handle(nys, monkeypatch, True, mx, nx, ell=16, tol=1e-6, seed=9, max_batch=3)
    probs = [tuple(_args(q)) for q in qps]
    res = nys.nys_solve_batched(hb, probs)
    h1 = _handle(nys, monkeypatch, True, mx, nx, ell=16, tol=1e-6, seed=9, max_batch=1)
    for qp, pr, (x, y, z, info) in zip(qps, probs, res):
        assert info["status"] == 0 and info["device_iteration"] == 1
        (x1, y1, z1, i1), = nys.nys_solve_batched(h1, [pr])
        assert torch.equal(x, x1) and torch.equal(y, y1) and torch.equal(z, z1)
        rp, rd, mu = O.kkt_measures(qp.A, qp.b, qp.c, qp.q, *(t.cpu().numpy() for t in (x, y, z)))
        assert max(rp, rd, mu) <= 1e-6


def test_non_finite_input_on_the_device_path(nys, monkeypatch):
    qp = synth.workload_small(seed=9)
    A = qp.A.copy()
    A[3, 7] = np.nan
    args = _args(qp)
    h = _handle(nys, monkeypatch, True, qp.m, qp.n, ell=20, tol=1e-6, seed=1)
    with pytest.raises(nys.NysError) as e:
        nys.nys_solve(h, T(A), *args[1:])
    assert e.value.code == nys.NYS_ERR_NUMERIC
    x, y, z, info = nys.nys_solve(h, *args)
    assert info["status"] == 0 and info["device_iteration"] == 1 and torch.isfinite(x).all()
