"""The differentiation form: GPU transposed-KKT gradients (nys_adjoint and the
autograd Function) against the oracle's dense KKT adjoint at the same final
iterate, and against finite differences of the oracle's solution map."""
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


@pytest.mark.parametrize("m,n", [(40, 160), (128, 512)])
def test_adjoint_matches_dense_kkt_at_the_gpu_solution(nys, m, n):
    qp = synth.gaussian_qp(500 + m, m, n)
    rng = np.random.default_rng(m)
    xt = rng.uniform(0, 1, n)
    h = nys.Handle(m, n, ell=min(32, m // 4), tol=1e-8, seed=3)
    x, y, z, info = nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))
    assert info["status"] == 0
    xs, ys, zs = (t.cpu().numpy() for t in (x, y, z))
    g = 2 * (xs - xt)
    G = nys.nys_adjoint(h, T(qp.A), T(qp.q), x, y, z, info, T(g), eta=1e-13)
    W = O.kkt_adjoint(qp.A, xs, ys, zs, qp.q, info["rho"], info["delta"], g)
    for k, want in (("c", W.c), ("b", W.b), ("q", W.q), ("A", W.A)):
        got = G[k].cpu().numpy()
        err = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)
        assert err <= 1e-6, (k, err)


def _exact_solution(A, b, c, q):
    """Exact optimum of a tiny strictly convex QP by enumerating supports."""
    import itertools
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
            zz = c + q * x - A.T @ sol[len(S):]
            if np.all(sol[:len(S)] >= -1e-13) and np.all(zz >= -1e-13):
                return x
    raise AssertionError("no KKT point")


@pytest.mark.parametrize("seed", range(3))
def test_autograd_function_matches_finite_differences(nys, seed):
    """d/d(A, b, c, q) of L = ||x* - x_t||^2 through backward() (nys_adjoint on
    the GPU) against central differences (h = 1e-6) of the exact solution map
    of tiny QPs (brute-force active sets), on random directions: 1e-5 rel."""
    rng = np.random.default_rng(900 + seed)
    m, n = 3, 9
    A0 = rng.standard_normal((m, n))
    b0 = A0 @ rng.uniform(0.5, 1.5, n)
    c0 = rng.standard_normal(n)
    q0 = rng.uniform(0.2, 1.0, n)
    xt = rng.uniform(0, 1, n)
    h = nys.Handle(m, n, ell=m, tol=1e-10, seed=2)
    A, b, c, q = (T(v).requires_grad_(True) for v in (A0, b0, c0, q0))
    x, y, z = nys.qp_solve(A, b, c, q, T(np.ones(n)), T(np.zeros(m)), T(np.ones(n)), h)
    assert np.allclose(x.detach().cpu().numpy(), _exact_solution(A0, b0, c0, q0), atol=1e-8)
    ((x - T(xt)) ** 2).sum().backward()
    loss = lambda AA, bb, cc, qq: float(np.sum((_exact_solution(AA, bb, cc, qq) - xt) ** 2))
    hs = 1e-6
    for _ in range(4):
        dA, db, dc, dq = rng.standard_normal((m, n)), rng.standard_normal(m), rng.standard_normal(n), \
            0.1 * rng.standard_normal(n)
        fd = (loss(A0 + hs * dA, b0 + hs * db, c0 + hs * dc, q0 + hs * dq) -
              loss(A0 - hs * dA, b0 - hs * db, c0 - hs * dc, q0 - hs * dq)) / (2 * hs)
        an = float((A.grad.cpu().numpy() * dA).sum() + b.grad.cpu().numpy() @ db +
                   c.grad.cpu().numpy() @ dc + q.grad.cpu().numpy() @ dq)
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (fd, an)


def test_adjoint_reuses_the_last_factor_of_the_solve(nys):
    """When the handle (or the batch worker that solved the problem) still
    holds the solve's last Nystrom factor for the same A, the adjoint takes it
    instead of sketching N again (fewer kernel launches); the gradients agree
    with the re-sketched path and with the dense KKT solve."""
    m, n = 128, 512
    qp = synth.gaussian_qp(777, m, n)
    xt = np.random.default_rng(1).uniform(0, 1, n)
    A = T(qp.A)
    h = nys.Handle(m, n, ell=32, tol=1e-8, seed=3)
    x, y, z, info = nys.nys_solve(h, A, T(qp.b), T(qp.c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))
    g = T(2 * (x.cpu().numpy() - xt))
    l0 = nys.nys_kernel_launches()
    G1 = nys.nys_adjoint(h, A, T(qp.q), x, y, z, info, g, eta=1e-13)          # same A: reuse
    l1 = nys.nys_kernel_launches()
    G2 = nys.nys_adjoint(h, A.clone(), T(qp.q), x, y, z, info, g, eta=1e-13)  # other pointer: re-sketch
    l2 = nys.nys_kernel_launches()
    assert l1 - l0 < l2 - l1
    xs, ys, zs = (t.cpu().numpy() for t in (x, y, z))
    W = O.kkt_adjoint(qp.A, xs, ys, zs, qp.q, info["rho"], info["delta"], g.cpu().numpy())
    for k, want in (("c", W.c), ("b", W.b), ("q", W.q), ("A", W.A)):
        a, b = G1[k].cpu().numpy(), G2[k].cpu().numpy()
        assert np.linalg.norm(a - want) <= 1e-6 * np.linalg.norm(want)
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(want)
    # forward through the batching form: the worker's factor is found
    hb = nys.Handle(m, n, ell=32, tol=1e-8, seed=3, max_batch=2)
    (xb, yb, zb, ib), = nys.nys_solve_batched(hb, [(A, T(qp.b), T(qp.c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))])
    l3 = nys.nys_kernel_launches()
    G3 = nys.nys_adjoint(hb, A, T(qp.q), xb, yb, zb, ib, g, eta=1e-13)
    l4 = nys.nys_kernel_launches()
    assert l4 - l3 < l2 - l1
    assert np.linalg.norm(G3["A"].cpu().numpy() - W.A) <= 1e-6 * np.linalg.norm(W.A)
