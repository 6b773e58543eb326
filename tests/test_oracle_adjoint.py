"""Pins of the oracle's transposed-KKT gradients (the differentiation form).

Pinned against finite differences of the exact solution map of tiny QPs
(brute-force active-set solutions, which are exact linear algebra for a fixed
active set) and against a closed form."""
import itertools

import numpy as np
import pytest

from oracle import nys_oracle as O


def _exact_solution(A, b, c, q):
    m, n = A.shape
    for size in range(m, n + 1):
        for S in itertools.combinations(range(n), size):
            S = list(S)
            K = np.block([[np.diag(q[S]), -A[:, S].T], [A[:, S], np.zeros((m, m))]])
            if abs(np.linalg.det(K)) < 1e-12:
                continue
            sol = np.linalg.solve(K, np.concatenate([-c[S], b]))
            x = np.zeros(n)
            x[S] = sol[:len(S)]
            y = sol[len(S):]
            zz = c + q * x - A.T @ y
            if np.all(sol[:len(S)] >= -1e-13) and np.all(zz >= -1e-13):
                return x, y
    raise AssertionError("no KKT point")


@pytest.mark.parametrize("seed", range(4))
def test_adjoint_matches_finite_differences_of_the_exact_solution(seed):
    rng = np.random.default_rng(300 + seed)
    m, n = 2, 5
    A = rng.standard_normal((m, n))
    b = A @ rng.uniform(0.5, 1.5, n)
    c = rng.standard_normal(n)
    q = rng.uniform(0.3, 1.0, n)
    xt = rng.uniform(0, 1, n)
    loss = lambda x: float(np.sum((x - xt) ** 2))
    r = O.solve(A, b, c, q, np.ones(n), np.zeros(m), np.ones(n), O.Options(tol=1e-12, ell=m, seed=1))
    assert r.status == "converged"
    x_ex, _ = _exact_solution(A, b, c, q)
    assert np.allclose(r.x, x_ex, atol=1e-9)
    # strict complementarity keeps the active set fixed under small perturbations
    G = O.kkt_adjoint(A, r.x, r.y, r.z, q, r.rho, r.delta, 2 * (r.x - xt))
    h = 1e-6

    def fd(perturb):
        xp, _ = _exact_solution(*perturb(+h))
        xm, _ = _exact_solution(*perturb(-h))
        return (loss(xp) - loss(xm)) / (2 * h)
    for j in range(n):
        e = np.eye(n)[j]
        assert abs(fd(lambda s: (A, b, c + s * e, q)) - G.c[j]) <= 1e-5 * (1 + abs(G.c[j]))
        assert abs(fd(lambda s: (A, b, c, q + s * e)) - G.q[j]) <= 1e-5 * (1 + abs(G.q[j]))
    for i in range(m):
        e = np.eye(m)[i]
        assert abs(fd(lambda s: (A, b + s * e, c, q)) - G.b[i]) <= 1e-5 * (1 + abs(G.b[i]))
    for i, j in [(0, 0), (1, 3), (0, 4)]:
        E = np.zeros((m, n))
        E[i, j] = 1.0
        assert abs(fd(lambda s: (A + s * E, b, c, q)) - G.A[i, j]) <= 1e-5 * (1 + abs(G.A[i, j]))


def test_adjoint_one_variable_closed_form():
    """n = m = 1, A = a: x* = b/a; with L = (x - t)^2: dL/db = 2(x-t)/a,
    dL/dA = -2(x-t) b / a^2, dL/dc = dL/dq = 0."""
    a, b, t = 2.0, 3.0, 0.25
    A = np.array([[a]])
    r = O.solve(A, np.array([b]), np.array([0.5]), np.array([1.0]), np.ones(1), np.zeros(1), np.ones(1),
                O.Options(tol=1e-12, ell=1, seed=0))
    x = r.x[0]
    assert abs(x - b / a) < 1e-9
    G = O.kkt_adjoint(A, r.x, r.y, r.z, np.array([1.0]), r.rho, r.delta, np.array([2 * (x - t)]))
    assert abs(G.b[0] - 2 * (x - t) / a) < 1e-6
    assert abs(G.A[0, 0] + 2 * (x - t) * b / a ** 2) < 1e-6
    assert abs(G.c[0]) < 1e-6 and abs(G.q[0]) < 1e-6


def test_adjoint_normal_equation_form_equals_dense_form():
    """Eliminating lam3 and lam1 gives (A D A^T + delta I) lam2 = A D g and
    lam1 = D (g - A^T lam2) with the D of Eq. normal-eq (same matrix as the
    Newton systems, so the Nystrom preconditioner applies unchanged)."""
    rng = np.random.default_rng(7)
    m, n = 6, 15
    A = rng.standard_normal((m, n))
    x, z = rng.uniform(0.1, 2, n), rng.uniform(0.1, 2, n)
    y = rng.standard_normal(m)
    q = rng.uniform(0, 1, n)
    rho, delta = 1e-3, 1e-4
    g = rng.standard_normal(n)
    G = O.kkt_adjoint(A, x, y, z, q, rho, delta, g)
    D = O.scaling_D(x, z, q, rho)
    l2 = np.linalg.solve(A @ (D[:, None] * A.T) + delta * np.eye(m), A @ (D * g))
    l1 = D * (g - A.T @ l2)
    assert np.allclose(G.b, l2, rtol=1e-9, atol=1e-12) and np.allclose(G.c, -l1, rtol=1e-9, atol=1e-12)
