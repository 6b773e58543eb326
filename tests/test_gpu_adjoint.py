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


def test_autograd_function_matches_finite_differences(nys):
    """d/d(b, c, q) of L = ||x* - x_t||^2 via backward(), against central
    differences of the oracle's tight solve on random directions (1e-5 rel.)."""
    m, n = 20, 60
    qp = synth.gaussian_qp(77, m, n)
    rng = np.random.default_rng(1)
    xt = rng.uniform(0, 1, n)
    h = nys.Handle(m, n, ell=m, tol=1e-10, seed=2)
    A, b, c, q = (T(v).requires_grad_(True) for v in (qp.A, qp.b, qp.c, qp.q))
    x, y, z = nys.qp_solve(A, b, c, q, T(qp.x0), T(qp.y0), T(qp.z0), h)
    L = ((x - T(xt)) ** 2).sum()
    L.backward()

    def loss(bb, cc, qq):
        r = O.solve(qp.A, bb, cc, qq, qp.x0, qp.y0, qp.z0, O.Options(tol=1e-12, ell=m, seed=2))
        return float(np.sum((r.x - xt) ** 2))
    hstep = 1e-6
    for _ in range(4):
        db, dc, dq = rng.standard_normal(m), rng.standard_normal(n), rng.standard_normal(n) * 0.1
        fd = (loss(qp.b + hstep * db, qp.c + hstep * dc, qp.q + hstep * dq) -
              loss(qp.b - hstep * db, qp.c - hstep * dc, qp.q - hstep * dq)) / (2 * hstep)
        an = float(b.grad.cpu().numpy() @ db + c.grad.cpu().numpy() @ dc + q.grad.cpu().numpy() @ dq)
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (fd, an)
