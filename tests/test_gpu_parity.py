"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Element-by-element comparisons on the same seeded inputs, at sizes that span
several tiles with ragged tails, plus the edge cases of each step.
Tolerances: the FP64 form is compared at 1e-9 relative for whole-solve
iterates (the stated target) and tighter for single steps, where only the
summation order differs (bounds derived from n * 2^-53 growth).
"""
import numpy as np
import pytest
import torch

from oracle import nys_oracle as O
from paper_2404_14524_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nys():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_14524_gb300 import build
    build.build()
    from paper_2404_14524_gb300 import nys as N
    N.lib()
    return N


DEV = torch.device("cuda", 0)


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def P(a):
    """m x ell numpy panel -> (ell, m) tensor (column-major panel)."""
    return T(np.asarray(a).T)


def relerr(got, want):
    got = got.detach().cpu().numpy() if isinstance(got, torch.Tensor) else got
    d = np.linalg.norm(want)
    return np.linalg.norm(got - want) / (d if d > 0 else 1.0)


# ----------------------------------------------------------------- generators

@pytest.mark.parametrize("m,ell,k", [(200, 20, 0), (517, 33, 5), (1, 1, 0)])
def test_gaussian_matches_oracle(nys, m, ell, k):
    h = nys.Handle(max(m, 2), 4, ell=ell)
    got = nys.nys_gaussian(h, 12345, k, m, ell).cpu().numpy().T
    want = O.gaussian_omega(12345, k, m, ell)
    # same uniform bits; log/cos of two libraries may differ in the last ulps
    assert np.allclose(got, want, rtol=1e-14, atol=1e-14)


# -------------------------------------------------------------- a1, a2

@pytest.mark.parametrize("m,n", [(203, 517), (1, 1), (64, 1025), (777, 129), (101, 98628), (37, 70001), (9, 4097)])
def test_scaling_and_normal_matvec(nys, m, n):
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((m, n))
    x, z, q = rng.uniform(0.1, 2, n), rng.uniform(0.01, 2, n), rng.uniform(0, 1, n)
    q[::4] = 0
    v = rng.standard_normal(m)
    h = nys.Handle(m, n, ell=1)
    D = nys.nys_scaling(h, T(x), T(z), T(q), 0.37)
    Dw = O.scaling_D(x, z, q, 0.37)
    assert relerr(D, Dw) <= 1e-15
    out = nys.nys_normal_matvec(h, T(A), D, 1e-3, T(v))
    want = O.normal_matvec(A, Dw, 1e-3, v)
    tol = 4 * (m + n) * 2.0 ** -53 * np.linalg.norm(np.abs(A) @ (Dw * (np.abs(A).T @ np.abs(v))))
    assert np.linalg.norm(out.cpu().numpy() - want) <= tol + 1e-300


def test_normal_matvec_padded_leading_dimension(nys):
    rng = np.random.default_rng(5)
    m, n, lda = 130, 301, 320
    Abig = rng.standard_normal((m, lda))
    D, v = rng.uniform(0.1, 1, n), rng.standard_normal(m)
    h = nys.Handle(m, n, ell=1)
    At = T(Abig)[:, :n]                           # strided view, lda = 320
    Dt, vt = T(D), T(v)                           # keep the tensors alive across the call
    out = torch.empty(m, dtype=torch.float64, device=DEV)
    lib = nys.lib()
    rc = lib.nys_normal_matvec(h.h, m, n, 0, nys._ptr(At), lda, nys._ptr(Dt), 0.5, nys._ptr(vt),
                               nys._ptr(out))
    assert rc == 0
    assert relerr(out, O.normal_matvec(Abig[:, :n], D, 0.5, v)) <= 1e-13


# ------------------------------------------------------------------ a3, a4

@pytest.mark.parametrize("m,n,ell", [(200, 500, 20), (333, 700, 65), (70, 90, 70)])
def test_sketch_matches_oracle(nys, m, n, ell):
    rng = np.random.default_rng(m + n + ell)
    A = rng.standard_normal((m, n)) / np.sqrt(n)
    D = rng.uniform(0.05, 3, n)
    Om = O.gaussian_omega(3, 1, m, ell)
    h = nys.Handle(m, n, ell=ell)
    Y = nys.nys_sketch(h, T(A), T(D), P(Om)).cpu().numpy().T
    Yw = O.sketch(A, D, Om)
    assert np.abs(Y - Yw).max() <= 1e-12 * np.abs(Yw).max()


def _factor_pair(nys, m, n, ell, seed, rank=None, dscale=1.0):
    rng = np.random.default_rng(seed)
    if rank is None:
        A = rng.standard_normal((m, n)) * (np.arange(1, m + 1) ** -1.0)[:, None]
    else:
        A = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n)) / np.sqrt(n)
    D = rng.uniform(0.1, 3, n) * dscale
    Om = O.gaussian_omega(seed, 0, m, ell)
    Y = O.sketch(A, D, Om)
    Fw = O.nystrom_from_sketch(Y, Om)
    h = nys.Handle(m, n, ell=ell)
    U, lam, nu = nys.nys_nystrom(h, P(Y), P(Om))
    return h, A, D, Om, Fw, U.cpu().numpy().T, lam.cpu().numpy(), nu


@pytest.mark.parametrize("m,n,ell", [(200, 500, 20), (301, 450, 47), (64, 64, 64), (5, 9, 1), (7, 12, 7),
                                     (1024, 1500, 32), (6200, 6300, 20), (600, 900, 120), (1000, 1500, 201)])
def test_nystrom_factor_matches_oracle(nys, m, n, ell):
    """2 <= ell <= 32 and m <= 6144: one-sided Jacobi on B by a thread-block
    cluster (one CTA per column pair); B nearly square and small: Jacobi on
    B in one CTA's shared memory; otherwise QR of B first (shifted Cholesky
    QR3) and Jacobi on the ell x ell factor (cluster for ell <= 32, one CTA
    up to ell = 160, else the cooperative kernel)."""
    h, A, D, Om, Fw, U, lam, nu = _factor_pair(nys, m, n, ell, seed=m + ell)
    assert nu == Fw.nu
    assert np.all(np.diff(lam) <= 0) and np.all(lam >= 0)
    assert np.allclose(lam, Fw.lam, rtol=1e-10, atol=1e-12 * Fw.lam[0])
    assert np.abs(U.T @ U - np.eye(ell)).max() < 1e-12
    Nh, Nhw = U @ np.diag(lam) @ U.T, Fw.U @ np.diag(Fw.lam) @ Fw.U.T
    assert np.linalg.norm(Nh - Nhw, 2) <= 1e-10 * np.linalg.norm(Nhw, 2)


@pytest.mark.parametrize("f32_start,gram", [("1", "1"), ("1", "0"), ("0", "1")])
@pytest.mark.parametrize("m,ell,dspan", [(200, 20, 0.0), (150, 30, 12.0), (1024, 32, 6.0), (120, 12, 16.0)])
def test_nystrom_factor_with_and_without_the_fp32_jacobi_start(nys, monkeypatch, f32_start, gram, m, ell, dspan):
    """The small direct route starts the FP64 Jacobi from an FP32 Jacobi
    rotation V (made orthogonal in FP64), then runs the FP64 sweeps either on
    the Gram matrix of B V (one CTA; gram "1") or on B V itself (cluster);
    every way the factor matches the oracle's (D spanning up to 16 orders of
    magnitude, as in late IPM iterations)."""
    rng = np.random.default_rng(m + ell)
    n = 3 * m
    A = rng.standard_normal((m, n)) / np.sqrt(n)
    D = 10.0 ** rng.uniform(-dspan / 2, dspan / 2, n)
    Om = O.gaussian_omega(5, 1, m, ell)
    Y = O.sketch(A, D, Om)
    Fw = O.nystrom_from_sketch(Y, Om)
    monkeypatch.setenv("NYS_JACOBI_F32", f32_start)
    monkeypatch.setenv("NYS_JACOBI_GRAM", gram)
    h = nys.Handle(m, n, ell=ell)
    U, lam, nu = nys.nys_nystrom(h, P(Y), P(Om))
    U, lam = U.cpu().numpy().T, lam.cpu().numpy()
    assert nu == Fw.nu
    assert np.allclose(lam, Fw.lam, rtol=1e-10, atol=1e-12 * Fw.lam[0])
    assert np.abs(U.T @ U - np.eye(ell)).max() < 1e-12
    Nh, Nhw = U @ np.diag(lam) @ U.T, Fw.U @ np.diag(Fw.lam) @ Fw.U.T
    assert np.linalg.norm(Nh - Nhw, 2) <= 1e-10 * np.linalg.norm(Nhw, 2)


def test_nystrom_exact_for_low_rank(nys):
    h, A, D, Om, Fw, U, lam, nu = _factor_pair(nys, 120, 300, 12, seed=9, rank=6)
    N = A @ (D[:, None] * A.T)
    assert np.linalg.norm(U @ np.diag(lam) @ U.T - N, 2) <= 1e-9 * np.linalg.norm(N, 2)


def test_nystrom_ill_conditioned_scaling(nys):
    """D spanning 12 orders of magnitude (late IPM iterations)."""
    rng = np.random.default_rng(4)
    m, n, ell = 150, 400, 30
    A = rng.standard_normal((m, n)) / np.sqrt(n)
    D = 10.0 ** rng.uniform(-6, 6, n)
    Om = O.gaussian_omega(4, 2, m, ell)
    Y = O.sketch(A, D, Om)
    Fw = O.nystrom_from_sketch(Y, Om)
    h = nys.Handle(m, n, ell=ell)
    U, lam, nu = nys.nys_nystrom(h, P(Y), P(Om))
    U, lam = U.cpu().numpy().T, lam.cpu().numpy()
    assert np.allclose(lam, Fw.lam, rtol=1e-8, atol=1e-13 * Fw.lam[0])
    delta = 1e-6
    r = rng.standard_normal(m)
    got = nys.nys_precond_apply(h, P(U), T(lam), delta, T(r))
    want = O.precond_inv_apply(Fw, delta, r)
    assert relerr(got, want) <= 1e-8


# -------------------------------------------------------------------- a6, a5

@pytest.mark.parametrize("m,ell", [(200, 20), (513, 1), (1000, 100)])
def test_precond_apply_matches_oracle(nys, m, ell):
    rng = np.random.default_rng(m)
    Uq, _ = np.linalg.qr(rng.standard_normal((m, ell)))
    lam = np.sort(rng.uniform(0, 5, ell))[::-1].copy()
    lam[-1] = 0.0
    F = O.NystromFactor(U=Uq, lam=lam, nu=0.0)
    r = rng.standard_normal(m)
    h = nys.Handle(m, 4, ell=ell)
    for delta in (1e-9, 1e-2, 4.0):
        got = nys.nys_precond_apply(h, P(Uq), T(lam), delta, T(r))
        assert relerr(got, O.precond_inv_apply(F, delta, r)) <= 1e-13


@pytest.mark.parametrize("m,n,ell,delta", [(200, 500, 20, 1e-3), (257, 611, 31, 1e-6)])
def test_pcg_matches_oracle(nys, m, n, ell, delta):
    h, A, D, Om, Fw, U, lam, nu = _factor_pair(nys, m, n, ell, seed=11 + m)
    rng = np.random.default_rng(1)
    xi = rng.standard_normal(m)
    eta = 1e-8
    want = O.pcg(lambda v: O.normal_matvec(A, D, delta, v), lambda v: O.precond_inv_apply(Fw, delta, v),
                 xi, eta, 1000)
    dy, it, res, rc = nys.nys_pcg(h, T(A), T(D), delta, P(U), T(lam), T(xi), eta, 1000)
    # Free-running CG decides its exit on a residual that crosses eta; on an
    # ill-conditioned system rounding shifts that crossing by a few percent of
    # the iterations.  Both solutions satisfy the residual test, so each lies
    # within eta ||xi|| / lambda_min(M) of the exact solution of the dense system.
    assert abs(it - want.iters) <= max(2, 0.05 * want.iters) and rc == 0
    M = A @ (D[:, None] * A.T) + delta * np.eye(m)
    exact = np.linalg.solve(M, xi)
    g = dy.cpu().numpy()
    assert np.linalg.norm(xi - M @ g) <= 1.001 * eta * np.linalg.norm(xi)
    bound = eta * np.linalg.norm(xi) / np.linalg.eigvalsh(M)[0]
    assert np.linalg.norm(g - exact) <= 1.001 * bound
    # forced count and a zero right-hand side
    dy, it, res, rc = nys.nys_pcg(h, T(A), T(D), delta, P(U), T(lam), T(xi), eta, 1000, forced=3)
    w3 = O.pcg(lambda v: O.normal_matvec(A, D, delta, v), lambda v: O.precond_inv_apply(Fw, delta, v),
               xi, eta, 1000, forced_iters=3)
    assert it == 3 and relerr(dy, w3.x) <= 1e-11
    dy, it, res, rc = nys.nys_pcg(h, T(A), T(D), delta, P(U), T(lam), T(np.zeros(m)), eta, 1000)
    assert it == 0 and float(dy.abs().max()) == 0.0


def test_pcg_max_iter_warning(nys):
    h, A, D, Om, Fw, U, lam, nu = _factor_pair(nys, 150, 300, 5, seed=3)
    xi = np.random.default_rng(2).standard_normal(150)
    dy, it, res, rc = nys.nys_pcg(h, T(A), T(D), 1e-9, P(U), T(lam), T(xi), 1e-14, 4)
    assert it == 4 and rc == nys.NYS_WARN_PCG_MAXITER


# ----------------------------------------------------------------- a7, a8

def test_newton_direction_matches_oracle(nys):
    rng = np.random.default_rng(8)
    m, n, ell = 150, 420, 15
    A = rng.standard_normal((m, n)) / np.sqrt(n)
    x, z = rng.uniform(0.1, 2, n), rng.uniform(0.1, 2, n)
    q = rng.uniform(0, 1, n)
    rho, delta = 0.2, 0.05
    D = O.scaling_D(x, z, q, rho)
    Om = O.gaussian_omega(1, 0, m, ell)
    F = O.nystrom(A, D, Om)
    r_d, r_p, r_xz = rng.standard_normal(n), rng.standard_normal(m), -x * z
    want = O.newton_direction(A, x, z, D, delta, r_d, r_p, r_xz, F, 1e-10, 500)
    h = nys.Handle(m, n, ell=ell)
    dx, dy, dz, it = nys.nys_newton(h, T(A), T(x), T(z), T(D), delta, T(r_d), T(r_p), T(r_xz),
                                    P(F.U), T(F.lam), 1e-10, 500)
    assert it == want.pcg_iters
    for g, w in ((dx, want.dx), (dy, want.dy), (dz, want.dz)):
        assert relerr(g, w) <= 1e-10


def test_step_length_bit_exact(nys):
    rng = np.random.default_rng(9)
    h = nys.Handle(4, 5000, ell=1)
    for n in (1, 7, 5000):
        v = rng.uniform(0.01, 2, n)
        dv = rng.standard_normal(n) * 3
        assert nys.nys_step_length(h, T(v), T(dv)) == O.step_length(v, dv)
    v = np.ones(10)
    assert nys.nys_step_length(h, T(v), T(np.ones(10))) == 0.995     # no negative component


# ------------------------------------------------------------------ whole solve

def _omega_sensitivity(qp, opt, state, k, lam, zeta, ref):
    """How far one oracle IPM step moves when Omega_k is perturbed by 2e-16
    relative: the rounding-level noise floor of that step (late IPM steps run
    many CG iterations on ill-conditioned systems, which amplify rounding)."""
    orig = O.gaussian_omega

    def pert(seed, kk, m, ell):
        om = orig(seed, kk, m, ell)
        return om * (1 + 2e-16 * np.sign(np.sin(np.arange(om.size))).reshape(om.shape))
    x, y, z = state
    kw = dict(lam0=lam, zeta0=zeta, k0=k, ref_p0=ref[0], ref_d0=ref[1])
    a = O.solve(qp.A, qp.b, qp.c, qp.q, x, y, z, opt, **kw)
    O.gaussian_omega = pert
    try:
        b = O.solve(qp.A, qp.b, qp.c, qp.q, x, y, z, opt, **kw)
    finally:
        O.gaussian_omega = orig
    return max(relerr(u, v) for u, v in ((a.x, b.x), (a.y, b.y), (a.z, b.z)))


@pytest.fixture(scope="module")
def small_run():
    qp = synth.workload_small()
    ref = O.solve_qp(qp, O.Options(tol=1e-6, ell=20, seed=7), record=True)
    return qp, ref


@pytest.mark.parametrize("k", [0, 1, 2, 5, 9, 13, -4, -3, -2, -1])
def test_single_ipm_step_matches_oracle(nys, small_run, k):
    """One IPM iteration (sketch, core, two PCG solves, steps, PEU) resumed on
    the GPU from the oracle's state k, with the oracle's PCG counts: the next
    iterate must agree to 1e-9 relative, or to 100x the oracle's own response
    to a 2e-16 perturbation of Omega_k where that floor is higher."""
    qp, ref = small_run
    k = k % len(ref.trace)
    t = ref.trace[k]
    x, y, z, lam, zeta = t.state
    forced = [t.pcg_pred, t.pcg_corr]
    opt = O.Options(tol=1e-6, ell=20, seed=7, rho0=t.rho, delta0=t.delta, forced_ipm=1, forced_pcg=forced)
    nxt = ref.trace[k + 1] if k + 1 < len(ref.trace) else None
    want = nxt.state[:3] if nxt is not None else (ref.x, ref.y, ref.z)
    floor = _omega_sensitivity(qp, opt, (x, y, z), k, lam, zeta, t.ref)
    tol = max(1e-9, 100 * floor)
    h = nys.Handle(qp.m, qp.n, ell=20, tol=1e-6, seed=7, forced_pcg=forced, forced_ipm=1,
                   rho0=t.rho, delta0=t.delta)
    gx, gy, gz, info = nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), T(x), T(y), T(z),
                                     lam0=T(lam), zeta0=T(zeta), k0=k, peu_ref=t.ref, want_pmm=True)
    errs = [relerr(g, w) for g, w in ((gx, want[0]), (gy, want[1]), (gz, want[2]))]
    print(f"k={k} errs={errs} floor={floor:.2e}")
    assert max(errs) <= tol
    if nxt is not None:
        # PMM update after the step: each parameter shrinks by 1 - r or
        # 1 - (2/3) r with r = |mu' - mu| / max(mu', mu); mu' = x'^T z' / n
        # carries up to twice the iterate's relative error, which moves r by
        # as much in absolute terms and a parameter by that over its factor.
        # Each estimate took the oracle's branch: it was re-centred (equal to
        # the new iterate) exactly when the oracle's was, and the references
        # moved with it.
        for got, old, new in ((info["rho"], t.rho, nxt.rho), (info["delta"], t.delta, nxt.delta)):
            tol_reg = 2 * tol / (new / old)
            assert abs(got - new) <= tol_reg * new
        # the references are residual norms of the new iterate (differences of
        # O(1) terms): they carry the iterate's error in absolute terms
        assert (info["peu_ref_p"], info["peu_ref_d"]) == pytest.approx(nxt.ref, rel=2 * tol, abs=10 * tol)
        assert relerr(info["lam"], nxt.state[3]) <= tol and relerr(info["zeta"], nxt.state[4]) <= tol


def test_small_workload_solution_matches_oracle(nys, small_run):
    """Whole m=200, n=500 solve with the oracle's PCG and IPM counts: same KKT
    quality, and the final iterates agree far below the 1e-6 tolerance (the
    oracle itself moves ~1e-7 under a 2e-16 perturbation of Omega)."""
    qp, ref = small_run
    h = nys.Handle(qp.m, qp.n, ell=20, tol=1e-6, seed=7, forced_pcg=ref.pcg_iters, forced_ipm=ref.ipm_iters)
    x, y, z, info = nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))
    assert info["ipm_iters"] == ref.ipm_iters and info["pcg_log"] == ref.pcg_iters
    for g, w in ((x, ref.x), (y, ref.y), (z, ref.z)):
        assert relerr(g, w) <= 1e-5
    assert info["rel_primal"] <= 1e-6 and info["rel_dual"] <= 1e-6 and info["mu"] <= 1e-6


def _trajectory_response(qp, opt, rec):
    """Per IPM iteration, how far the oracle's own state at the top of that
    iteration moves when every Omega_k is perturbed by 2e-16 relative (the
    counts held): the rounding noise floor of the trajectory up to there."""
    import dataclasses
    orig = O.gaussian_omega

    def pert(seed, kk, m, ell):
        om = orig(seed, kk, m, ell)
        return om * (1 + 2e-16 * np.sign(np.sin(np.arange(om.size))).reshape(om.shape))
    O.gaussian_omega = pert
    try:
        b = O.solve_qp(qp, dataclasses.replace(opt, forced_pcg=rec.pcg_iters, forced_ipm=rec.ipm_iters),
                       record=True)
    finally:
        O.gaussian_omega = orig
    per = [max(relerr(eb.state[i], ea.state[i]) for i in range(3)) for ea, eb in zip(rec.trace, b.trace)]
    final = max(relerr(b.x, rec.x), relerr(b.y, rec.y), relerr(b.z, rec.z))
    return per, final


def test_whole_solve_within_1e9_on_a_well_conditioned_trajectory(nys):
    """Differentiation-shaped QP (512 x 2048 Gaussian A, q ~ U[0.1, 1], tol
    1e-8): the oracle's own trajectory is insensitive to rounding (its final
    iterate moves ~1e-15 under a 2e-16 change of Omega), so the GPU's whole
    solve, with the oracle's counts, must match the oracle's iterate to 1e-9."""
    qp = synth.gaussian_qp(11, 512, 2048)
    opt = O.Options(tol=1e-8, ell=32, seed=7)
    rec = O.solve_qp(qp, opt, record=True)
    assert rec.status == "converged"
    per, final = _trajectory_response(qp, opt, rec)
    assert final <= 1e-12
    h = nys.Handle(qp.m, qp.n, ell=32, tol=1e-8, seed=7, forced_pcg=rec.pcg_iters, forced_ipm=rec.ipm_iters)
    x, y, z, info = nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))
    assert info["ipm_iters"] == rec.ipm_iters and info["pcg_log"] == rec.pcg_iters
    errs = [relerr(g, w) for g, w in ((x, rec.x), (y, rec.y), (z, rec.z))]
    print(f"whole solve errs={errs} oracle response={final:.1e}")
    assert max(errs) <= 1e-9
    assert info["rho"] == pytest.approx(rec.rho, rel=1e-9) and info["delta"] == pytest.approx(rec.delta, rel=1e-9)


def test_small_workload_trajectory_within_1e9_while_the_oracle_is_stable(nys, small_run):
    """m=200, n=500: the oracle's trajectory stays insensitive to rounding
    (response <= 1e-11) for its first K iterations and then amplifies it by
    orders of magnitude (ill-conditioned late Newton systems with forced CG
    counts).  The GPU's first K iterations, run as one solve from the
    workload's start with the oracle's counts, must match the oracle's state
    at the top of iteration K to 1e-9."""
    qp, ref = small_run
    opt = O.Options(tol=1e-6, ell=20, seed=7)
    per, _ = _trajectory_response(qp, opt, ref)
    # the last top-of-iteration state whose response is still <= 1e-11
    K = next((k for k, p in enumerate(per) if p > 1e-11), len(per)) - 1
    assert K >= 8, per
    h = nys.Handle(qp.m, qp.n, ell=20, tol=1e-6, seed=7, forced_pcg=ref.pcg_iters[:2 * K], forced_ipm=K)
    x, y, z, info = nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))
    want = ref.trace[K].state if K < len(ref.trace) else (ref.x, ref.y, ref.z)
    errs = [relerr(g, w) for g, w in zip((x, y, z), want[:3])]
    print(f"K={K} errs={errs}")
    assert info["ipm_iters"] == K and max(errs) <= 1e-9


def test_free_running_solve_meets_kkt(nys):
    """Without forced counts the GPU decides its own PCG exits and stops by its
    own KKT test; it must converge to the same point within the tolerance."""
    qp = synth.workload_small(seed=77)
    ref = O.solve_qp(qp, O.Options(tol=1e-8, ell=20, seed=3))
    h = nys.Handle(qp.m, qp.n, ell=20, tol=1e-8, seed=3)
    x, y, z, info = nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))
    assert info["status"] == 0
    rp, rd, mu = O.kkt_measures(qp.A, qp.b, qp.c, qp.q, *(t.cpu().numpy() for t in (x, y, z)))
    assert rp <= 1e-8 and rd <= 1e-8 and mu <= 1e-8
    assert relerr(x, ref.x) <= 1e-5


def test_host_buffers_give_identical_results(nys):
    qp = synth.workload_small(seed=5)
    h = nys.Handle(qp.m, qp.n, ell=20, tol=1e-6, seed=1)
    dev = nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))
    cpu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    host = nys.nys_solve(h, cpu(qp.A), cpu(qp.b), cpu(qp.c), cpu(qp.q), cpu(qp.x0), cpu(qp.y0), cpu(qp.z0))
    for a, b in zip(dev[:3], host[:3]):
        assert torch.equal(a.cpu(), b)


def test_tiny_and_degenerate_problems(nys):
    """m = 1 with ell = 1, and an LP (q = 0), against hand-derived KKT points."""
    h = nys.Handle(1, 3, ell=1, tol=1e-9)
    A, b = np.array([[1.0, 1.0, 1.0]]), np.array([1.0])
    c, q = np.array([1.0, 2.0, 3.0]), np.zeros(3)
    x, y, z, info = nys.nys_solve(h, T(A), T(b), T(c), T(q), T(np.ones(3)), T(np.zeros(1)), T(np.ones(3)))
    assert info["status"] == 0
    assert np.allclose(x.cpu().numpy(), [1, 0, 0], atol=1e-7) and abs(float(y[0]) - 1.0) < 1e-6


def test_bad_arguments_are_rejected(nys):
    h = nys.Handle(10, 20, ell=5)
    lib = nys.lib()
    out = torch.empty(10, dtype=torch.float64, device=DEV)
    A = torch.zeros(10, 20, dtype=torch.float64, device=DEV)
    # m larger than the handle, wrong dtype, lda < n
    assert lib.nys_normal_matvec(h.h, 11, 20, 0, nys._ptr(A), 20, nys._ptr(out), 0.0, nys._ptr(out), nys._ptr(A)) == -1
    assert lib.nys_normal_matvec(h.h, 10, 20, 2, nys._ptr(A), 20, nys._ptr(out), 0.0, nys._ptr(out), nys._ptr(A)) == -1
    assert lib.nys_normal_matvec(h.h, 10, 20, 0, nys._ptr(A), 19, nys._ptr(out), 0.0, nys._ptr(out), nys._ptr(A)) == -1
    assert "bad argument" in nys.nys_last_error(h)


def test_non_finite_input_is_reported_not_faulted(nys):
    """A NaN in A reaches the residuals of the first iteration: the solve stops
    with NYS_ERR_NUMERIC (arithmetic on NaN, no device fault), and the same
    handle then solves a clean problem normally."""
    qp = synth.workload_small(seed=9)
    A = qp.A.copy()
    A[3, 7] = np.nan
    h = nys.Handle(qp.m, qp.n, ell=20, tol=1e-6, seed=1)
    rest = [T(v) for v in (qp.b, qp.c, qp.q, qp.x0, qp.y0, qp.z0)]
    with pytest.raises(nys.NysError) as e:
        nys.nys_solve(h, T(A), *rest)
    assert e.value.code == nys.NYS_ERR_NUMERIC
    x, y, z, info = nys.nys_solve(h, T(qp.A), *rest)
    assert info["status"] == 0 and torch.isfinite(x).all()


def test_core_breakdown_is_reported_not_trapped(nys):
    """Omega = 0 makes Omega^T Y_nu singular: the Cholesky must report a
    breakdown status (no trap) and the handle must stay usable."""
    m, ell = 50, 5
    h = nys.Handle(m, 10, ell=ell)
    Y = P(np.random.default_rng(0).standard_normal((m, ell)))
    Z = torch.zeros_like(Y)
    with pytest.raises(nys.NysError) as e:
        nys.nys_nystrom(h, Y, Z)
    assert e.value.code == nys.NYS_ERR_CORE_BREAKDOWN
    # still usable
    out = nys.nys_precond_apply(h, P(np.eye(m)[:, :ell]), T(np.ones(ell)), 1.0, T(np.ones(m)))
    assert torch.isfinite(out).all()


@pytest.mark.parametrize("m,n,ell,path,route", [
    (300, 900, 24, "cluster", 0),       # A's column bands in shared memory
    (7, 41, 3, "cluster", 0),           # fewer rows and columns than CTAs
    (700, 1400, 16, "cluster", 1),      # A read from L2 by the cluster
    (300, 900, 24, "cooperative", 2),   # grid-wide cooperative launch
])
def test_one_launch_pcg_routes_match_the_graph_pcg(nys, monkeypatch, m, n, ell, path, route):
    """Small systems run the whole PCG in one launch (a thread-block cluster,
    or one cooperative grid); each route must give the multi-kernel (CUDA
    graph) path's solution up to summation order."""
    h1, A, D, Om, Fw, U, lam, nu = _factor_pair(nys, m, n, ell, seed=21)
    xi = np.random.default_rng(4).standard_normal(m)
    monkeypatch.setenv("NYS_PCG_PATH", path)
    hr = nys.Handle(m, n, ell=ell)
    monkeypatch.setenv("NYS_PCG_PATH", "graph")
    h0 = nys.Handle(m, n, ell=ell)
    monkeypatch.delenv("NYS_PCG_PATH")
    assert nys.nys_pcg_route(hr, m, n, ell) == route
    assert nys.nys_pcg_route(h0, m, n, ell) == nys.NYS_ROUTE_GRAPH
    delta, eta, maxit = 1e-4, 1e-9, 4000
    for forced in (5, -1):
        a, ia, ra, _ = nys.nys_pcg(hr, T(A), T(D), delta, P(U), T(lam), T(xi), eta, maxit, forced=forced)
        b, ib, rb, _ = nys.nys_pcg(h0, T(A), T(D), delta, P(U), T(lam), T(xi), eta, maxit, forced=forced)
        if forced >= 0:      # same iterations: rounding only
            assert ia == ib and relerr(a, b.cpu().numpy()) <= 1e-11
            continue
        # at the tolerance crossing the count moves with the summation order
        # (as for the oracle comparison above): within max(2, 5%)
        assert ia < maxit and ib < maxit
        assert abs(ia - ib) <= max(2, int(0.05 * ib))
        # both meet the residual test (true FP64 residual, with room for the
        # drift of the recursive one), and two such solutions differ by at
        # most (|r_a| + |r_b|) / lambda_min(N + delta I) <= (|r_a| + |r_b|) / delta
        an, bn = a.cpu().numpy(), b.cpu().numpy()
        res = lambda v: np.linalg.norm(xi - O.normal_matvec(A, D, delta, v))
        assert res(an) <= 10 * eta * np.linalg.norm(xi) and res(bn) <= 10 * eta * np.linalg.norm(xi)
        assert np.linalg.norm(an - bn) <= (res(an) + res(bn)) / delta * (1 + 1e-6)