"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself:
library routines it does not use, assembled block systems, closed forms,
invariants and brute force.  All run on the CPU (no GPU marker).
"""
import itertools
import os

import numpy as np
import pytest
import scipy.optimize
import scipy.stats

from oracle import nys_oracle as O
from paper_2404_14524_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- generators

def test_eps_is_float64_spacing():
    """Algorithm 1, step 3: eps(x) is the float64 spacing at x (numpy.spacing)."""
    rng = np.random.default_rng(0)
    xs = np.concatenate([10.0 ** rng.uniform(-300, 300, 2000), [1.0, 2.0, 3.0, 0.5, 1e-300, 1e300]])
    for x in xs:
        assert O.eps_of(float(x)) == float(np.spacing(x))


def _splitmix_sequential(seed: int, count: int):
    """SplitMix64 in its sequential form (state += gamma; output = mix(state))."""
    mask = (1 << 64) - 1
    state = seed & mask
    out = []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


@pytest.mark.parametrize("seed", [0, 1, 0xDEADBEEFCAFEBABE, 2**64 - 1])
def test_splitmix_counter_access_matches_sequential_stream(seed):
    seq = _splitmix_sequential(seed, 300)
    ctr = O.splitmix64_at(seed, np.arange(300, dtype=np.uint64))
    assert [int(v) for v in ctr] == seq


def test_omega_is_standard_gaussian_and_fresh_per_iteration():
    """Algorithm 1, step 1: i.i.d. N(0, 1) entries; a new draw per IPM iteration."""
    om0 = O.gaussian_omega(11, 0, 400, 50)
    om1 = O.gaussian_omega(11, 1, 400, 50)
    assert om0.shape == (400, 50)
    ks = scipy.stats.kstest(om0.ravel(), "norm")
    assert ks.pvalue > 1e-3
    assert abs(om0.mean()) < 0.03 and abs(om0.std() - 1.0) < 0.03
    assert abs(np.corrcoef(om0.ravel(), om1.ravel())[0, 1]) < 0.03
    # entries are addressed by (k, i, j): a sub-block of a larger draw agrees
    big = O.gaussian_omega(11, 0, 400, 60)
    assert np.array_equal(big[:, :50], om0)


# ------------------------------------------------------- Newton system (Alg. 4)

def _tiny_state(seed, m=7, n=15):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    x = rng.uniform(0.1, 2.0, n)
    z = rng.uniform(0.1, 2.0, n)
    q = rng.uniform(0.0, 1.0, n)
    q[::3] = 0.0
    return rng, A, x, z, q


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_newton_direction_solves_the_block_newton_system(seed):
    """Algorithm 4 must reproduce the solution of the 3x3-block Newton system of
    Eq. Newton, assembled densely and solved by LAPACK."""
    rng, A, x, z, q = _tiny_state(seed)
    m, n = A.shape
    rho, delta = 0.3, 0.05
    r_d, r_p, r_xz = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(n)
    D = O.scaling_D(x, z, q, rho)
    F = O.nystrom(A, D, O.gaussian_omega(5, 0, m, 3))
    d = O.newton_direction(A, x, z, D, delta, r_d, r_p, r_xz, F, eta=1e-14, maxit=500)
    K = np.block([
        [-(np.diag(q) + rho * np.eye(n)), A.T, np.eye(n)],
        [A, delta * np.eye(m), np.zeros((m, n))],
        [np.diag(z), np.zeros((n, m)), np.diag(x)],
    ])
    sol = np.linalg.solve(K, np.concatenate([r_d, r_p, r_xz]))
    got = np.concatenate([d.dx, d.dy, d.dz])
    assert np.allclose(got, sol, rtol=1e-9, atol=1e-9 * np.abs(sol).max())


def test_inexact_solve_leaves_residual_only_in_the_second_block():
    """Prop. 3.2: with an inexact dy, blocks 1 and 3 of Eq. Newton stay exact
    and block 2 carries the normal-equations residual."""
    rng, A, x, z, q = _tiny_state(7, m=9, n=20)
    m, n = A.shape
    rho, delta = 0.2, 0.1
    r_d, r_p, r_xz = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(n)
    D = O.scaling_D(x, z, q, rho)
    F = O.nystrom(A, D, O.gaussian_omega(5, 0, m, 2))
    d = O.newton_direction(A, x, z, D, delta, r_d, r_p, r_xz, F, eta=1e-30, maxit=500, forced_iters=2)
    b1 = -(q + rho) * d.dx + A.T @ d.dy + d.dz - r_d
    b2 = A @ d.dx + delta * d.dy - r_p
    b3 = z * d.dx + x * d.dz - r_xz
    assert np.abs(b1).max() < 1e-12 and np.abs(b3).max() < 1e-12
    assert np.linalg.norm(b2) > 1e-6          # two iterations are far from exact


# ------------------------------------------------------ Nystrom (Alg. 1, 2)

def _psd_operator(seed, m, n, rank=None):
    rng = np.random.default_rng(seed)
    if rank is None:
        A = rng.standard_normal((m, n)) * (np.arange(1, m + 1) ** -1.0)[:, None]
    else:
        A = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n))
    D = rng.uniform(0.1, 3.0, n)
    return A, D, A @ (D[:, None] * A.T)


def test_nystrom_factor_invariants():
    """Alg. 1 output: orthonormal U, lambda >= 0 descending; N_hat PSD and
    N - N_hat >= -nu I (Nystrom of N + nu I is dominated by N + nu I)."""
    A, D, N = _psd_operator(3, 60, 90)
    F = O.nystrom(A, D, O.gaussian_omega(9, 0, 60, 12))
    assert np.abs(F.U.T @ F.U - np.eye(12)).max() < 1e-12
    assert np.all(F.lam >= 0) and np.all(np.diff(F.lam) <= 0)
    Nh = F.U @ np.diag(F.lam) @ F.U.T
    ev = np.linalg.eigvalsh(N - Nh)
    assert ev.min() >= -F.nu - 1e-13 * np.linalg.norm(N, 2)
    assert np.linalg.eigvalsh(Nh).min() >= -1e-13 * np.linalg.norm(N, 2)


def test_nystrom_matches_the_pseudoinverse_formula():
    """Eq. Nystrom-approx: N_hat = Y (Omega^T Y)^+ Y^T (up to the nu shift)."""
    A, D, N = _psd_operator(4, 50, 80)
    Om = O.gaussian_omega(2, 3, 50, 10)
    F = O.nystrom(A, D, Om)
    Y = N @ Om
    ref = Y @ np.linalg.pinv(Om.T @ Y) @ Y.T
    Nh = F.U @ np.diag(F.lam) @ F.U.T
    assert np.linalg.norm(Nh - ref, 2) <= 1e-9 * np.linalg.norm(ref, 2)


def test_nystrom_is_exact_when_rank_is_at_most_ell():
    A, D, N = _psd_operator(5, 40, 70, rank=6)
    F = O.nystrom(A, D, O.gaussian_omega(1, 0, 40, 8))
    Nh = F.U @ np.diag(F.lam) @ F.U.T
    assert np.linalg.norm(Nh - N, 2) <= 1e-10 * np.linalg.norm(N, 2)
    assert np.all(F.lam[6:] <= 1e-10 * F.lam[0])


def test_preconditioner_inverse_inverts_the_preconditioner():
    """Eq. Nys_precond_inv is the inverse of Eq. Nys_precond."""
    A, D, N = _psd_operator(6, 45, 60)
    F = O.nystrom(A, D, O.gaussian_omega(4, 0, 45, 9))
    v = np.random.default_rng(0).standard_normal(45)
    for delta in (1e-6, 1e-2, 3.0):
        assert np.allclose(O.precond_apply(F, delta, O.precond_inv_apply(F, delta, v)), v, atol=1e-11)


def test_preconditioned_spectrum_bounds():
    """Spectrum of P^{-1}(N + delta I) lies in [delta - nu, lam_ell + delta + ||N - N_hat||];
    with an exact N_hat it has exactly the two values {delta, lam_ell + delta}."""
    A, D, N = _psd_operator(8, 40, 60)
    m = 40
    for delta in (1e-3, 1e-1):
        F = O.nystrom(A, D, O.gaussian_omega(2, 0, m, 10))
        Pinv = np.column_stack([O.precond_inv_apply(F, delta, e) for e in np.eye(m)])
        ev = np.sort(np.linalg.eigvals(Pinv @ (N + delta * np.eye(m))).real)
        err = np.linalg.norm(N - F.U @ np.diag(F.lam) @ F.U.T, 2)
        assert ev[0] >= delta - F.nu - 1e-12 and ev[-1] <= F.lam[-1] + delta + err + 1e-10
    A, D, N = _psd_operator(9, 30, 50, rank=5)
    F = O.nystrom(A, D, O.gaussian_omega(3, 0, 30, 7))
    delta = 0.05
    Pinv = np.column_stack([O.precond_inv_apply(F, delta, e) for e in np.eye(30)])
    ev = np.sort(np.linalg.eigvals(Pinv @ (N + delta * np.eye(30))).real)
    lam_ell = F.lam[-1]
    assert np.all(np.minimum(np.abs(ev - delta), np.abs(ev - (lam_ell + delta))) < 1e-8)


# -------------------------------------------------------------------- PCG

def test_pcg_matches_dense_direct_solve():
    A, D, N = _psd_operator(10, 60, 100)
    delta = 1e-3
    F = O.nystrom(A, D, O.gaussian_omega(1, 0, 60, 10))
    rhs = np.random.default_rng(1).standard_normal(60)
    res = O.pcg(lambda v: O.normal_matvec(A, D, delta, v), lambda v: O.precond_inv_apply(F, delta, v),
                rhs, eta=1e-13, maxit=1000)
    ref = np.linalg.solve(N + delta * np.eye(60), rhs)
    assert res.converged
    assert np.linalg.norm(res.x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_pcg_with_exact_nystrom_converges_in_two_iterations():
    """Two distinct preconditioned eigenvalues => CG terminates in two steps."""
    A, D, N = _psd_operator(11, 50, 70, rank=6)
    delta = 1e-2
    F = O.nystrom(A, D, O.gaussian_omega(5, 0, 50, 8))
    rhs = np.random.default_rng(2).standard_normal(50)
    res = O.pcg(lambda v: O.normal_matvec(A, D, delta, v), lambda v: O.precond_inv_apply(F, delta, v),
                rhs, eta=1e-10, maxit=50)
    assert res.iters <= 2 and res.converged


def test_unpreconditioned_cg_terminates_in_distinct_eigenvalue_count():
    """Textbook CG property on a diagonal system with 4 distinct eigenvalues."""
    diag = np.repeat([1.0, 2.0, 5.0, 9.0], 10)
    rhs = np.random.default_rng(3).standard_normal(40)
    res = O.pcg(lambda v: diag * v, lambda v: v, rhs, eta=1e-12, maxit=100)
    assert res.iters == 4 and np.allclose(res.x, rhs / diag, atol=1e-12)


def test_pcg_error_decreases_in_the_operator_norm():
    """A textbook property of (preconditioned) CG: the error's M-norm,
    M = N + delta I, decreases strictly at every iteration, and the iterates
    with k forced steps are the same whatever the stopping tolerance."""
    A, D, N = _psd_operator(12, 80, 120)
    delta = 1e-4
    M = N + delta * np.eye(80)
    F = O.nystrom(A, D, O.gaussian_omega(3, 0, 80, 6))
    rhs = np.random.default_rng(4).standard_normal(80)
    xs = np.linalg.solve(M, rhs)
    errs = []
    for k in range(0, 25):
        res = O.pcg(lambda v: O.normal_matvec(A, D, delta, v), lambda v: O.precond_inv_apply(F, delta, v),
                    rhs, eta=0.0, maxit=1000, forced_iters=k)
        e = res.x - xs
        errs.append(float(np.sqrt(e @ M @ e)))
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_pcg_zero_rhs():
    res = O.pcg(lambda v: 2 * v, lambda v: v, np.zeros(5), eta=1e-8, maxit=10)
    assert res.iters == 0 and np.all(res.x == 0)


# ------------------------------------------------------------ step lengths

def test_step_length_by_brute_force():
    rng = np.random.default_rng(4)
    for _ in range(50):
        v = rng.uniform(0.01, 2.0, 12)
        dv = rng.standard_normal(12) * rng.uniform(0.1, 10)
        a = O.step_length(v, dv)
        lo, hi = 0.0, 1.0          # largest alpha in [0, 1] keeping v + alpha dv >= 0
        if np.all(v + dv >= 0):
            lo = 1.0
        else:
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if np.all(v + mid * dv >= 0):
                    lo = mid
                else:
                    hi = mid
        assert abs(a - 0.995 * lo) <= 1e-12
    assert O.step_length(np.ones(3), np.ones(3)) == 0.995


# ------------------------------------------------------------- whole solve

def _read_golden():
    recs = []
    with open(os.path.join(GOLDEN, "kkt_points.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = [p.strip() for p in line.split("|")]
            vec = lambda s: np.array([float(t) for t in s.split()])
            A = np.array([[float(t) for t in row.split()] for row in parts[1].split(";")])
            recs.append((parts[0], A, vec(parts[2]), vec(parts[3]), vec(parts[4]),
                         vec(parts[5]), vec(parts[6]), vec(parts[7])))
    return recs


@pytest.mark.parametrize("rec", _read_golden(), ids=lambda r: r[0])
def test_solve_reaches_hand_derived_kkt_points(rec):
    name, A, b, c, q, xs, ys, zs = rec
    m, n = A.shape
    r = O.solve(A, b, c, q, np.ones(n), np.zeros(m), np.ones(n),
                O.Options(tol=1e-10, ell=m, seed=3, max_pcg_iter=200))
    assert r.status == "converged", (name, r.ipm_iters)
    assert np.allclose(r.x, xs, atol=1e-7)
    assert np.allclose(r.y, ys, atol=1e-6)
    assert np.allclose(r.z, zs, atol=1e-6)


def _active_set_brute_force(A, b, c, q):
    """Exact optimum of a strictly convex separable QP by enumerating supports."""
    m, n = A.shape
    for size in range(m, n + 1):
        for S in itertools.combinations(range(n), size):
            S = list(S)
            K = np.block([[np.diag(q[S]), -A[:, S].T], [A[:, S], np.zeros((m, m))]])
            if abs(np.linalg.det(K)) < 1e-12:
                continue
            sol = np.linalg.solve(K, np.concatenate([-c[S], b]))
            xS, y = sol[:len(S)], sol[len(S):]
            x = np.zeros(n)
            x[S] = xS
            zz = c + q * x - A.T @ y
            if np.all(xS >= -1e-12) and np.all(zz >= -1e-12):
                return x, y, zz
    raise AssertionError("no KKT point found")


@pytest.mark.parametrize("seed", range(6))
def test_solve_matches_active_set_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = 2, 6
    A = rng.standard_normal((m, n))
    x0 = rng.uniform(0.5, 1.5, n)
    b = A @ x0
    c = rng.standard_normal(n)
    q = rng.uniform(0.2, 1.0, n)
    xs, ys, zs = _active_set_brute_force(A, b, c, q)
    r = O.solve(A, b, c, q, np.ones(n), np.zeros(m), np.ones(n), O.Options(tol=1e-10, ell=2, seed=seed))
    assert r.status == "converged"
    assert np.allclose(r.x, xs, atol=1e-6)
    assert np.allclose(r.y, ys, atol=1e-5)


@pytest.mark.parametrize("seed", range(3))
def test_lp_matches_scipy_highs(seed):
    """Q = 0 (an LP): the objective value must agree with scipy's HiGHS."""
    rng = np.random.default_rng(200 + seed)
    m, n = 4, 12
    A = rng.standard_normal((m, n))
    b = A @ rng.uniform(0.5, 1.5, n)
    c = rng.uniform(0.1, 2.0, n)
    ref = scipy.optimize.linprog(c, A_eq=A, b_eq=b, bounds=[(0, None)] * n, method="highs")
    r = O.solve(A, b, c, np.zeros(n), np.ones(n), np.zeros(m), np.ones(n),
                O.Options(tol=1e-9, ell=m, seed=seed))
    assert r.status == "converged"
    assert abs(c @ r.x - ref.fun) <= 1e-6 * (1 + abs(ref.fun))


def test_small_workload_meets_kkt_and_gap():
    """The m=200, n=500 workload reaches the relative KKT tolerance and a small
    duality gap; iteration count in the range the paper reports (well under 50)."""
    qp = synth.workload_small()
    r = O.solve_qp(qp, O.Options(tol=1e-6, ell=20, seed=7))
    assert r.status == "converged" and r.ipm_iters < 50
    rp, rd, mu = O.kkt_measures(qp.A, qp.b, qp.c, qp.q, r.x, r.y, r.z)
    assert rp <= 1e-6 and rd <= 1e-6 and mu <= 1e-6
    assert r.rel_gap <= 1e-4
    assert np.all(r.x > 0) and np.all(r.z > 0)


def test_regularisation_trace_shape():
    """Algorithm 6 starts at rho = delta = 8 and both decrease to the floor
    region as mu falls (qualitatively as in Tables 7-8)."""
    qp = synth.workload_small()
    r = O.solve_qp(qp, O.Options(tol=1e-6, ell=20, seed=7))
    assert r.trace[0].rho == 8.0 and r.trace[0].delta == 8.0
    rhos = [t.rho for t in r.trace]
    assert all(b <= a for a, b in zip(rhos, rhos[1:]))
    assert rhos[-1] < 1e-6


# ---------------------------------------------------------------- FP8 storage

def test_e4m3_rounding_follows_the_format_definition():
    """E4M3 (sign, 4-bit exponent with bias 7, 3-bit mantissa, no infinities,
    largest finite 1.75 * 2^8 = 448, subnormal spacing 2^-9): values worked
    out from the definition, including ties to the even mantissa and
    saturation."""
    cases = {
        448.0: 448.0, 500.0: 448.0, 1e6: 448.0, 1.0: 1.0,
        1.0625: 1.0,            # halfway between 1.000 and 1.125: even mantissa 000
        1.1875: 1.25,           # halfway between 1.125 and 1.250: even mantissa 010
        -3.3: -3.25,            # spacing 0.25 in [2, 4)
        2.0 ** -7: 2.0 ** -7,   # subnormal 4 * 2^-9
        2.0 ** -10: 0.0,        # half a subnormal step: ties to 0
        3 * 2.0 ** -10: 2.0 ** -8,  # 1.5 steps: ties to the even 2 steps
        2.0 ** -6 * 1.0625: 2.0 ** -6,
        240.0: 240.0, 248.0: 256.0,  # spacing 16 in [128, 256): 248 ties to even 256
    }
    got = O.e4m3_round(np.array(list(cases)))
    assert np.array_equal(got, np.array(list(cases.values())))


def test_e4m3_codes_decode_and_round_to_themselves():
    """Every finite E4M3 code decodes to a value that rounds to itself;
    the codes 0x7E, 0x08, 0x01 are 448, 2^-6 and 2^-9; 0x7F is NaN."""
    vals = O.e4m3_decode(np.arange(256))
    fin = np.isfinite(vals)
    assert fin.sum() == 254                       # 0x7F and 0xFF are NaN
    assert np.array_equal(O.e4m3_round(vals[fin]), vals[fin])
    assert vals[0x7E] == 448.0 and vals[0x08] == 2.0 ** -6 and vals[0x01] == 2.0 ** -9
    pos = np.sort(vals[1:0x7F])
    assert np.all(np.diff(pos) > 0)               # 126 distinct positive values


def test_fp8_rowscale_quantisation_bounds():
    """Each nonzero row reaches +-448 after scaling; every element is within
    half a quantum: |A - s Q| <= 2^-4 |A| in the normal range, <= s 2^-10
    below it."""
    rng = np.random.default_rng(3)
    A = (rng.standard_normal((17, 40)) * np.exp(rng.uniform(-8, 8, (17, 1)))).astype(np.float32)
    A[5] = 0.0
    Q, s = O.fp8_rowscale_quantize(A)
    assert s[5] == 1.0 and np.all(Q[5] == 0)
    nz = np.arange(17) != 5
    assert np.allclose(np.max(np.abs(Q[nz]), axis=1), 448.0)
    err = np.abs(A.astype(np.float64) - s[:, None].astype(np.float64) * Q)
    bound = np.maximum(2.0 ** -4 * np.abs(A), s[:, None] * 2.0 ** -10) * (1 + 1e-6)
    assert np.all(err <= bound)
