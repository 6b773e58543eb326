"""Pins of the oracle's free and box-constrained variables (problems (P~)/(D~),
Algorithm 4 with w and s, Eq. predictor-RHS / corrector-RHS, Eq. stepsize-p /
stepsize-d) against what the paper and the mathematics fix: the 5x5-block
Newton system of Eq. Newton-free-box assembled densely, scipy's HiGHS on
bounded LPs, brute-force active-set enumeration of tiny QPs, hand-derived KKT
points (tests/golden/kkt_points_box.txt) and brute-force step-length scans.
CPU only."""
import itertools
import os

import numpy as np
import pytest
import scipy.optimize

from oracle import nys_oracle as O
from paper_2404_14524_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KI, KF, KJ = O.KIND_I, O.KIND_F, O.KIND_J


def _box_state(seed, m=6, n=14):
    """Random interior iterate with every kind present (w, s zero outside J, z zero on F)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    kind = np.array([KI, KF, KJ] * (n // 3) + [KI] * (n % 3), dtype=np.int8)
    rng.shuffle(kind)
    jj, ff = kind == KJ, kind == KF
    x = np.where(ff, rng.standard_normal(n), rng.uniform(0.1, 2.0, n))
    z = np.where(ff, 0.0, rng.uniform(0.1, 2.0, n))
    w = np.where(jj, rng.uniform(0.1, 2.0, n), 0.0)
    s = np.where(jj, rng.uniform(0.1, 2.0, n), 0.0)
    q = rng.uniform(0.0, 1.0, n)
    q[::4] = 0.0
    return rng, A, kind, x, z, w, s, q


def _newton_matrix(A, kind, x, z, w, s, q, rho, delta):
    """Eq. Newton-free-box with unknowns (dx, dy, dw_J, dz_IJ, ds_J), E_S the
    row selections of the index sets."""
    m, n = A.shape
    ij, jj = np.flatnonzero(kind != KF), np.flatnonzero(kind == KJ)
    E = np.eye(n)
    EJ, EIJ = E[jj], E[ij]
    nj, nij = len(jj), len(ij)
    Z = lambda r, c: np.zeros((r, c))
    return np.block([
        [-(np.diag(q) + rho * E), A.T, Z(n, nj), EIJ.T, -EJ.T],
        [A, delta * np.eye(m), Z(m, nj), Z(m, nij), Z(m, nj)],
        [EJ, Z(nj, m), np.eye(nj), Z(nj, nij), Z(nj, nj)],
        [np.diag(z[ij]) @ EIJ, Z(nij, m), Z(nij, nj), np.diag(x[ij]), Z(nij, nj)],
        [Z(nj, n), Z(nj, m), np.diag(s[jj]), Z(nj, nij), np.diag(w[jj])],
    ])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_box_newton_direction_solves_the_block_system(seed):
    """Algorithm 4 with w, s reproduces the dense solution of Eq. Newton-free-box
    (signs and blocks as printed; E_S selections of I u J and J)."""
    rng, A, kind, x, z, w, s, q = _box_state(seed)
    m, n = A.shape
    rho, delta = 0.3, 0.05
    ij, jj = kind != KF, kind == KJ
    r_d, r_p = rng.standard_normal(n), rng.standard_normal(m)
    r_u = np.where(jj, rng.standard_normal(n), 0.0)
    r_xz = np.where(ij, rng.standard_normal(n), 0.0)
    r_ws = np.where(jj, rng.standard_normal(n), 0.0)
    D = O.scaling_D(x, z, q, rho, kind, w, s)
    F = O.nystrom(A, D, O.gaussian_omega(5, 0, m, 3))
    d = O.newton_direction(A, x, z, D, delta, r_d, r_p, r_xz, F, eta=1e-14, maxit=500,
                           kind=kind, w=w, s=s, r_u=r_u, r_ws=r_ws)
    K = _newton_matrix(A, kind, x, z, w, s, q, rho, delta)
    sol = np.linalg.solve(K, np.concatenate([r_d, r_p, r_u[jj], r_xz[ij], r_ws[jj]]))
    nj, nij = int(jj.sum()), int(ij.sum())
    dx, dy = sol[:n], sol[n:n + m]
    dwJ = sol[n + m:n + m + nj]
    dzIJ = sol[n + m + nj:n + m + nj + nij]
    dsJ = sol[n + m + nj + nij:]
    tol = 1e-9 * np.abs(sol).max()
    assert np.allclose(d.dx, dx, atol=tol) and np.allclose(d.dy, dy, atol=tol)
    assert np.allclose(d.dw[jj], dwJ, atol=tol) and np.allclose(d.dz[ij], dzIJ, atol=tol)
    assert np.allclose(d.ds[jj], dsJ, atol=tol)
    # the variables a kind does not have stay exactly zero
    assert np.all(d.dz[~ij] == 0.0) and np.all(d.dw[~jj] == 0.0) and np.all(d.ds[~jj] == 0.0)


def test_box_inexact_solve_leaves_residual_only_in_the_second_block():
    """Prop. 3.2 carried to Eq. Newton-free-box: with an inexact dy every block
    row but the second (A dx + delta dy = r_p) holds to rounding."""
    rng, A, kind, x, z, w, s, q = _box_state(9, m=8, n=21)
    m, n = A.shape
    rho, delta = 0.2, 0.1
    ij, jj = kind != KF, kind == KJ
    r_d, r_p = rng.standard_normal(n), rng.standard_normal(m)
    r_u = np.where(jj, rng.standard_normal(n), 0.0)
    r_xz = np.where(ij, rng.standard_normal(n), 0.0)
    r_ws = np.where(jj, rng.standard_normal(n), 0.0)
    D = O.scaling_D(x, z, q, rho, kind, w, s)
    F = O.nystrom(A, D, O.gaussian_omega(5, 0, m, 2))
    d = O.newton_direction(A, x, z, D, delta, r_d, r_p, r_xz, F, eta=1e-30, maxit=500, forced_iters=2,
                           kind=kind, w=w, s=s, r_u=r_u, r_ws=r_ws)
    b1 = -(q + rho) * d.dx + A.T @ d.dy + d.dz - d.ds - r_d
    b2 = A @ d.dx + delta * d.dy - r_p
    b3 = (d.dx + d.dw - r_u)[jj]
    b4 = (z * d.dx + x * d.dz - r_xz)[ij]
    b5 = (s * d.dw + w * d.ds - r_ws)[jj]
    for b in (b1, b3, b4, b5):
        assert np.abs(b).max() < 1e-11
    assert np.linalg.norm(b2) > 1e-6


def test_box_scaling_reduces_to_the_non_negative_case():
    """With every variable in I the general Theta^{-1} is Z X^{-1}; a free
    variable keeps only q + rho; a box one adds S W^{-1}."""
    rng, A, kind, x, z, w, s, q = _box_state(4)
    rho = 0.7
    allI = np.zeros_like(kind)
    assert np.array_equal(O.scaling_D(x, z, q, rho, allI, w * 0, s * 0), O.scaling_D(x, z, q, rho))
    D = O.scaling_D(x, z, q, rho, kind, w, s)
    ff, jj = kind == KF, kind == KJ
    assert np.allclose(D[ff], 1.0 / (q[ff] + rho), rtol=1e-15)
    assert np.allclose(D[jj], 1.0 / (q[jj] + z[jj] / x[jj] + s[jj] / w[jj] + rho), rtol=1e-15)


def test_box_step_lengths_by_brute_force():
    """alpha_p is the largest step in [0, 1] keeping x_IJ and w_J non-negative
    (free x unbounded), alpha_d likewise for z_IJ and s_J, both times 0.995."""
    rng = np.random.default_rng(11)
    for trial in range(40):
        _, _, kind, x, z, w, s, _ = _box_state(100 + trial, m=2, n=12)
        ij, jj = kind != KF, kind == KJ
        dx, dz = rng.standard_normal(12) * 3, np.where(ij, rng.standard_normal(12) * 3, 0.0)
        dw, ds = np.where(jj, rng.standard_normal(12) * 3, 0.0), np.where(jj, rng.standard_normal(12) * 3, 0.0)
        ap, ad = O.step_lengths(x, dx, z, dz, kind, w, dw, s, ds)

        def largest(ok):
            if ok(1.0):
                return 1.0
            lo, hi = 0.0, 1.0
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                lo, hi = (mid, hi) if ok(mid) else (lo, mid)
            return lo
        okp = lambda a: np.all((x + a * dx)[ij] >= 0) and np.all((w + a * dw)[jj] >= 0)
        okd = lambda a: np.all((z + a * dz)[ij] >= 0) and np.all((s + a * ds)[jj] >= 0)
        assert abs(ap - 0.995 * largest(okp)) <= 1e-12
        assert abs(ad - 0.995 * largest(okd)) <= 1e-12


# ------------------------------------------------------------- whole solves

def _kinds(tokens):
    return np.array([{"I": KI, "F": KF, "J": KJ}[t] for t in tokens.split()], dtype=np.int8)


def _read_golden():
    recs = []
    with open(os.path.join(GOLDEN, "kkt_points_box.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = [p.strip() for p in line.split("|")]
            vec = lambda t: np.array([float(v) for v in t.split()])
            A = np.array([[float(v) for v in row.split()] for row in parts[3].split(";")])
            recs.append(dict(name=parts[0], kind=_kinds(parts[1]), u=vec(parts[2]), A=A, b=vec(parts[4]),
                             c=vec(parts[5]), q=vec(parts[6]), x=vec(parts[7]), y=vec(parts[8]),
                             z=vec(parts[9]), s=vec(parts[10])))
    return recs


def _interior_start(kind, u, m):
    n = len(kind)
    x0 = np.where(kind == KJ, 0.5 * u, np.where(kind == KF, 0.0, 1.0))
    return x0, np.zeros(m), np.ones(n), np.where(kind == KJ, 1.0, 0.0)


@pytest.mark.parametrize("rec", _read_golden(), ids=lambda r: r["name"])
def test_box_solve_reaches_hand_derived_kkt_points(rec):
    A, kind, u = rec["A"], rec["kind"], rec["u"]
    m, n = A.shape
    x0, y0, z0, s0 = _interior_start(kind, u, m)
    r = O.solve(A, rec["b"], rec["c"], rec["q"], x0, y0, z0,
                O.Options(tol=1e-10, ell=m, seed=3, max_pcg_iter=200), kind=kind, u=u, s0=s0)
    assert r.status == "converged", (rec["name"], r.ipm_iters)
    assert np.allclose(r.x, rec["x"], atol=1e-7)
    assert np.allclose(r.y, rec["y"], atol=1e-6)
    assert np.allclose(r.z, rec["z"], atol=1e-6)
    assert np.allclose(r.s, rec["s"], atol=1e-6)
    jj = kind == KJ
    assert np.allclose(r.w[jj], u[jj] - r.x[jj], atol=1e-9)


def _box_active_set_brute_force(A, b, c, q, kind, u):
    """Exact optimum of a strictly convex separable QP with free (F), non-negative
    (I) and box (J) variables: enumerate which variables sit at a bound (0, or u
    on J), solve the equality-constrained QP in the others, keep the point whose
    x stays within its bounds and whose multipliers have the right signs."""
    m, n = A.shape
    choices = [("B",) if k == KF else ("B", "L") if k == KI else ("B", "L", "U") for k in kind]
    for pick in itertools.product(*choices):
        S = [j for j in range(n) if pick[j] == "B"]
        x = np.zeros(n)
        for j in range(n):
            if pick[j] == "U":
                x[j] = u[j]
        K = np.block([[np.diag(q[S]), -A[:, S].T], [A[:, S], np.zeros((m, m))]])
        if abs(np.linalg.det(K)) < 1e-12:
            continue
        rhs = np.concatenate([-c[S], b - A @ x])
        sol = np.linalg.solve(K, rhs)
        x[S] = sol[:len(S)]
        y = sol[len(S):]
        g = c + q * x - A.T @ y          # = z - s
        ok = True
        for j in range(n):
            if kind[j] != KF and x[j] < -1e-12:
                ok = False
            if kind[j] == KJ and x[j] > u[j] + 1e-12:
                ok = False
            if pick[j] == "L" and g[j] < -1e-12:
                ok = False
            if pick[j] == "U" and g[j] > 1e-12:
                ok = False
        if ok:
            z = np.where((np.array(pick) == "L"), g, 0.0)
            s = np.where((np.array(pick) == "U"), -g, 0.0)
            return x, y, z, s
    raise AssertionError("no KKT point found")


@pytest.mark.parametrize("seed", range(6))
def test_box_solve_matches_active_set_enumeration(seed):
    rng = np.random.default_rng(300 + seed)
    m, n = 2, 7
    A = rng.standard_normal((m, n))
    kind = np.array([KF, KI, KI, KJ, KJ, KJ, KI], dtype=np.int8)
    x0 = np.where(kind == KF, rng.standard_normal(n), rng.uniform(0.5, 1.5, n))
    u = np.where(kind == KJ, x0 + rng.uniform(0.1, 0.6, n), 0.0)
    b = A @ x0
    c = 2.0 * rng.standard_normal(n)
    q = rng.uniform(0.2, 1.0, n)
    xs, ys, zs, ss = _box_active_set_brute_force(A, b, c, q, kind, u)
    x_start, y_start, z_start, s_start = _interior_start(kind, u, m)
    r = O.solve(A, b, c, q, x_start, y_start, z_start, O.Options(tol=1e-10, ell=2, seed=seed),
                kind=kind, u=u, s0=s_start)
    assert r.status == "converged"
    assert np.allclose(r.x, xs, atol=1e-6)
    assert np.allclose(r.y, ys, atol=1e-5)
    assert np.allclose(r.s, ss, atol=1e-5) and np.allclose(r.z, zs, atol=1e-5)


@pytest.mark.parametrize("seed", range(3))
def test_bounded_lp_matches_scipy_highs(seed):
    """Q = 0 with free, non-negative and box variables: the optimal value agrees
    with scipy's HiGHS on the same bounds."""
    rng = np.random.default_rng(400 + seed)
    m, n = 4, 15
    A = rng.standard_normal((m, n))
    kind = np.array([KF] * 2 + [KI] * 7 + [KJ] * 6, dtype=np.int8)
    x0 = np.where(kind == KF, rng.standard_normal(n), rng.uniform(0.5, 1.5, n))
    u = np.where(kind == KJ, x0 + rng.uniform(0.2, 1.0, n), 0.0)
    b = A @ x0
    # c = A^T y + z - s with z, s >= 0 on their sets and z_F = s_F = 0 keeps the LP bounded
    y = rng.standard_normal(m)
    c = A.T @ y + np.where(kind == KF, 0.0, rng.uniform(0.1, 1.0, n)) - np.where(kind == KJ, rng.uniform(0, 2, n), 0.0)
    bounds = [(None, None) if k == KF else (0, None) if k == KI else (0, uj) for k, uj in zip(kind, u)]
    ref = scipy.optimize.linprog(c, A_eq=A, b_eq=b, bounds=bounds, method="highs")
    assert ref.status == 0
    x_start, y_start, z_start, s_start = _interior_start(kind, u, m)
    r = O.solve(A, b, c, np.zeros(n), x_start, y_start, z_start, O.Options(tol=1e-9, ell=m, seed=seed),
                kind=kind, u=u, s0=s_start)
    assert r.status == "converged"
    assert abs(c @ r.x - ref.fun) <= 1e-6 * (1 + abs(ref.fun))


def test_box_workload_meets_kkt_and_bounds():
    """The 200 x 500 workload with 10% free and 30% box variables reaches the
    tolerance with a small duality gap, keeps every bound strictly, and uses
    the upper bounds (some x_J end at u_J)."""
    qp = synth.workload_box()
    r = O.solve_qp(qp, O.Options(tol=1e-6, ell=20, seed=7))
    assert r.status == "converged" and r.ipm_iters < 60
    rp, rd, mu = O.kkt_measures(qp.A, qp.b, qp.c, qp.q, r.x, r.y, r.z, qp.kind, qp.u, r.w, r.s)
    assert rp <= 1e-6 and rd <= 1e-6 and mu <= 1e-6
    assert r.rel_gap <= 1e-4
    ij, jj = qp.kind != KF, qp.kind == KJ
    assert np.all(r.x[ij] > 0) and np.all(r.z[ij] > 0) and np.all(r.w[jj] > 0) and np.all(r.s[jj] > 0)
    assert np.all(r.z[~ij] == 0) and np.all(r.s[~jj] == 0) and np.all(r.w[~jj] == 0)
    assert np.sum(r.x[jj] > qp.u[jj] - 1e-4) > 0


def test_all_non_negative_kinds_reproduce_the_plain_solve():
    """Every variable in I (kind all zeros, no box) is problem (P)/(D): the
    general code path adds exact zeros only, so the iterates agree to rounding."""
    qp = synth.spectral_qp(77, 30, 80, "inv")
    opt = O.Options(tol=1e-8, ell=10, seed=2)
    a = O.solve_qp(qp, opt)
    b = O.solve(qp.A, qp.b, qp.c, qp.q, qp.x0, qp.y0, qp.z0, opt, kind=np.zeros(80, dtype=np.int8),
                u=np.zeros(80), s0=np.zeros(80))
    assert a.ipm_iters == b.ipm_iters and a.pcg_iters == b.pcg_iters
    assert np.allclose(a.x, b.x, rtol=0, atol=1e-12) and np.allclose(a.y, b.y, rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_box_iteration_equals_standard_form_with_explicit_slacks(seed):
    """Without regularisation (rho = delta = 0) an IP-PMM iteration on (P~) with
    I and J variables is the iteration of problem (P) on the standard form that
    makes the slack explicit: variables (x, w_J) >= 0, constraints
    [[A, 0], [E_J, I]] (x, w_J) = (b, u_J), whose duals are (y, -s_J) for the
    rows and (z, s_J) for the columns.  Mehrotra's corrector of that (P)
    carries the products dw ds and the combined mu of Algorithm 5, so the two
    iterates agree when both Newton systems are solved exactly (sketch size
    equal to the system size: the Nystrom preconditioner is then exact)."""
    rng = np.random.default_rng(500 + seed)
    m, n = 3, 10
    A = rng.standard_normal((m, n))
    kind = np.array([KI, KJ] * (n // 2), dtype=np.int8)
    rng.shuffle(kind)
    J = np.flatnonzero(kind == KJ)
    nj = len(J)
    x0 = rng.uniform(0.5, 1.5, n)
    u = np.where(kind == KJ, x0 + rng.uniform(0.5, 1.5, n), 0.0)
    w0 = np.where(kind == KJ, u - x0 + rng.uniform(-0.2, 0.2, n), 0.0)   # r_u != 0 at the start
    z0 = rng.uniform(0.2, 1.5, n)
    s0 = np.where(kind == KJ, rng.uniform(0.2, 1.5, n), 0.0)
    y0 = rng.standard_normal(m)
    b = A @ rng.uniform(0.5, 1.5, n)
    c = rng.standard_normal(n)
    q = rng.uniform(0.0, 1.0, n)
    kw = dict(tol=1e-14, seed=1, rho0=0.0, delta0=0.0, reg_floor=0.0, forced_ipm=1, max_pcg_iter=200)
    rb = O.solve(A, b, c, q, x0, y0, z0, O.Options(ell=m, **kw), kind=kind, u=u, s0=s0, w0=w0)
    EJ = np.eye(n)[J]
    A2 = np.block([[A, np.zeros((m, nj))], [EJ, np.eye(nj)]])
    re = O.solve(A2, np.concatenate([b, u[J]]), np.concatenate([c, np.zeros(nj)]),
                 np.concatenate([q, np.zeros(nj)]), np.concatenate([x0, w0[J]]),
                 np.concatenate([y0, -s0[J]]), np.concatenate([z0, s0[J]]), O.Options(ell=m + nj, **kw))
    close = lambda a, e: np.allclose(a, e, rtol=1e-8, atol=1e-8 * (1 + np.abs(e).max()))
    assert close(rb.x, re.x[:n]) and close(rb.w[J], re.x[n:])
    assert close(rb.y, re.y[:m]) and close(rb.s[J], -re.y[m:])
    assert close(rb.z, re.z[:n]) and close(rb.s[J], re.z[n:])
    assert abs(rb.trace[0].alpha_p - re.trace[0].alpha_p) < 1e-10
    assert abs(rb.trace[0].alpha_d - re.trace[0].alpha_d) < 1e-10


# ------------------------------------------------------------ practical start

def _read_start_golden():
    recs = []
    with open(os.path.join(GOLDEN, "start_points.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p = [t.strip() for t in line.split("|")]
            vec = lambda t: np.array([float(v) for v in t.split()])
            A = np.array([[float(v) for v in row.split()] for row in p[3].split(";")])
            recs.append(dict(name=p[0], kind=_kinds(p[1]), u=vec(p[2]), A=A, b=vec(p[4]), c=vec(p[5]),
                             q=vec(p[6]), x=vec(p[7]), y=vec(p[8]), z=vec(p[9]), w=vec(p[10]), s=vec(p[11])))
    return recs


@pytest.mark.parametrize("rec", _read_start_golden(), ids=lambda r: r["name"])
def test_practical_start_matches_hand_derived_points(rec):
    st = O.practical_start(rec["A"], rec["b"], rec["c"], rec["q"], O.Options(ell=1, seed=0), rec["kind"], rec["u"])
    for got, nm in ((st.x, "x"), (st.y, "y"), (st.z, "z"), (st.w, "w"), (st.s, "s")):
        assert np.allclose(got, rec[nm], rtol=1e-12, atol=1e-12), nm


@pytest.mark.parametrize("seed", range(4))
def test_practical_start_is_strictly_interior(seed):
    """Whatever the candidate's signs, the shifted start has x_IJ, z_IJ, w_J,
    s_J > 0, z_F = 0 and w = s = 0 outside J (the purpose of the shifts)."""
    qp = synth.box_qp(900 + seed, 30, 90, 0.2, 0.4)
    c = qp.c + 3.0 * np.random.default_rng(seed).standard_normal(qp.n)     # far from dual feasible
    st = O.practical_start(qp.A, qp.b, c, qp.q, O.Options(ell=8, seed=seed), qp.kind, qp.u)
    ij, jj = qp.kind != KF, qp.kind == KJ
    assert np.all(st.x[ij] > 0) and np.all(st.z[ij] > 0) and np.all(st.w[jj] > 0) and np.all(st.s[jj] > 0)
    assert np.all(st.z[~ij] == 0) and np.all(st.w[~jj] == 0) and np.all(st.s[~jj] == 0)


@pytest.mark.parametrize("seed", range(4))
def test_solve_from_practical_start_matches_active_set_enumeration(seed):
    """From the practical start (no interior point supplied) the solve reaches
    the brute-force optimum of a tiny QP with free, non-negative and box
    variables."""
    rng = np.random.default_rng(700 + seed)
    m, n = 2, 7
    A = rng.standard_normal((m, n))
    kind = np.array([KF, KI, KI, KJ, KJ, KJ, KI], dtype=np.int8)
    x0 = np.where(kind == KF, rng.standard_normal(n), rng.uniform(0.5, 1.5, n))
    u = np.where(kind == KJ, x0 + rng.uniform(0.1, 0.6, n), 0.0)
    b = A @ x0
    c = 2.0 * rng.standard_normal(n)
    q = rng.uniform(0.2, 1.0, n)
    xs, ys, _, _ = _box_active_set_brute_force(A, b, c, q, kind, u)
    r = O.solve_from_practical_start(A, b, c, q, O.Options(tol=1e-10, ell=2, seed=seed), kind, u)
    assert r.status == "converged"
    assert np.allclose(r.x, xs, atol=1e-6) and np.allclose(r.y, ys, atol=1e-5)


def test_solve_from_practical_start_reaches_the_same_solution():
    """The 200 x 500 workloads, (P) and (P~), from the practical start instead
    of the generator's interior point: converged, and the same optimum (the
    QPs are strictly convex where q > 0 and have a unique solution)."""
    for qp in (synth.workload_small(), synth.workload_box()):
        opt = O.Options(tol=1e-8, ell=20, seed=7)
        a = O.solve_qp(qp, opt)
        b = O.solve_from_practical_start(qp.A, qp.b, qp.c, qp.q, opt, qp.kind, qp.u)
        assert a.status == "converged" and b.status == "converged" and b.ipm_iters < 60
        assert np.linalg.norm(a.x - b.x) <= 1e-5 * np.linalg.norm(a.x)


# ------------------------------------------ SVM- and portfolio-shaped problems

def test_svm_formulation_matches_a_library_svm():
    """The supplement's dual-SVM (P~) (free v, 0 <= p <= tau, A = [[I, -X diag(lab)],
    [0, lab^T]]) solved by the oracle from the practical start gives the
    separating hyperplane of scikit-learn's linear C-SVM (libsvm) with
    C = tau; the (P~) multipliers reproduce the SVM margin conditions
    (lab_i (x_i^T v + b0) >= 1 where p_i = 0, = 1 inside the box, <= 1 at tau)."""
    svm = pytest.importorskip("sklearn.svm")
    d, ns, tau = 6, 120, 1.0
    qp = synth.svm_qp(11, d, ns, tau=tau, sep=0.8)
    r = O.solve_from_practical_start(qp.A, qp.b, qp.c, qp.q, O.Options(tol=1e-10, ell=d + 1, seed=1),
                                     qp.kind, qp.u)
    assert r.status == "converged"
    v, p = r.x[:d], r.x[d:]
    Xs = -qp.A[:d, d:] * qp.A[d, d:][None, :]          # recover X from -X diag(lab) and lab^T
    lab = qp.A[d, d:]
    ref = svm.SVC(kernel="linear", C=tau, tol=1e-12).fit(Xs.T, lab)
    assert np.allclose(v, ref.coef_[0], atol=1e-5)
    b0 = -r.y[d]
    margin = lab * (Xs.T @ v + b0)
    assert abs(b0 - ref.intercept_[0]) < 1e-4
    assert np.all(margin[p < 1e-8] >= 1 - 1e-6)
    inside = (p > 1e-6) & (p < tau - 1e-6)
    assert np.allclose(margin[inside], 1.0, atol=1e-5)
    assert np.all(margin[p > tau - 1e-8] <= 1 + 1e-6)


def test_portfolio_formulation_matches_the_original_problem():
    """The factor-model (P~) (variables x, y = F^T x, slack t) reaches the same
    optimum as scipy's SLSQP on the original problem
    min -r^T x / gamma + x^T (F F^T + Dg) x s.t. M x <= u, 1^T x = 1, x >= 0."""
    na, dd, s = 12, 5, 3
    qp = synth.portfolio_qp(13, na, dd, s)
    r = O.solve_from_practical_start(qp.A, qp.b, qp.c, qp.q, O.Options(tol=1e-10, ell=dd + s + 1, seed=2),
                                     qp.kind, qp.u)
    assert r.status == "converged"
    F = qp.A[:s, :na].T
    M = qp.A[s:s + dd, :na]
    u = qp.b[s:s + dd]
    Dg = 0.5 * qp.q[:na]
    rr = -qp.c[:na]
    Sig = F @ F.T + np.diag(Dg)
    f = lambda x: -rr @ x + x @ Sig @ x
    cons = [{"type": "ineq", "fun": lambda x: u - M @ x, "jac": lambda x: -M},
            {"type": "eq", "fun": lambda x: np.sum(x) - 1.0, "jac": lambda x: np.ones((1, na))}]
    ref = scipy.optimize.minimize(f, np.full(na, 1.0 / na), jac=lambda x: -rr + 2 * Sig @ x, method="SLSQP",
                                  bounds=[(0, None)] * na, constraints=cons, options={"ftol": 1e-14, "maxiter": 500})
    assert ref.success
    x = r.x[:na]
    assert abs(f(x) - ref.fun) <= 1e-7 * (1 + abs(ref.fun))
    assert np.allclose(x, ref.x, atol=1e-5)
    assert np.allclose(r.x[na:na + s], F.T @ x, atol=1e-8)          # y = F^T x


# ------------------------------------------------------- preconditioner reuse

def test_preconditioner_reuse_reaches_the_same_optimum():
    """Keeping the previous Nystrom factor while PCG stays cheap (reuse_pcg = R)
    changes only the preconditioner, never the Newton systems: the solve
    still meets the KKT tolerance at the same optimum, with fewer sketches;
    R = 0 is Algorithm 6 as written (a factor in every iteration)."""
    qp = synth.workload_small()
    base = O.solve_qp(qp, O.Options(tol=1e-8, ell=20, seed=7))
    assert all(not t.reused for t in base.trace)
    r = O.solve_qp(qp, O.Options(tol=1e-8, ell=20, seed=7, reuse_pcg=60))
    assert r.status == "converged"
    reused = [t.reused for t in r.trace]
    assert 0 < sum(reused) < len(reused) and not reused[0]
    # the rule: a factor is kept exactly when both previous solves took <= R iterations
    for k in range(1, len(r.trace)):
        prev = r.trace[k - 1]
        assert reused[k] == (prev.pcg_pred <= 60 and prev.pcg_corr <= 60)
    assert np.linalg.norm(r.x - base.x) <= 1e-6 * np.linalg.norm(base.x)
