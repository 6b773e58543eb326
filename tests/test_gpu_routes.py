"""Each PCG route against the oracle at sizes where the route is the one the
library picks by itself for a single solve (no NYS_PCG_PATH override): a
thread-block cluster with A in shared memory, one cooperative grid (A up to
2^23 entries), and the per-step kernels of the CUDA-graph route (A above
2^23 entries).  The cluster that reads A from L2 is the batching form's
route; tests/test_gpu_batch.py runs it on its natural sizes.

Forced iteration counts compare iterates element by element (rounding order
only); free-running solves must meet the residual test on the dense system
and stay within eta ||xi|| / lambda_min of its exact solution; the Newton
direction of Algorithm 4 is compared on the graph route's natural size."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

from oracle import nys_oracle as O

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)

# (m, n, ell) chosen to land on each single-solve route (two shapes each for
# the cooperative grid); the test below checks the library's own choice.
SIZES = [(200, 500, 20), (900, 2600, 24), (4000, 2048, 16), (1024, 6144, 32), (1500, 6000, 40)]


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


def P(a):
    return T(np.asarray(a).T)


def relerr(got, want):
    got = got.detach().cpu().numpy() if isinstance(got, torch.Tensor) else got
    return np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)


def _system(nys, m, n, ell, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) * (np.arange(1, m + 1) ** -0.8)[:, None] / np.sqrt(n)
    D = 10.0 ** rng.uniform(-2, 2, n)
    Om = O.gaussian_omega(seed, 0, m, ell)
    Fw = O.nystrom(A, D, Om)
    h = nys.Handle(m, n, ell=ell)
    U, lam, _ = nys.nys_nystrom(h, P(O.sketch(A, D, Om)), P(Om))
    return h, A, D, Fw, U, lam


def test_sizes_cover_every_route(nys):
    routes = set()
    for m, n, ell in SIZES:
        h = nys.Handle(m, n, ell=ell)
        routes.add(nys.nys_pcg_route(h, m, n, ell))
        h.close()
    assert routes == {nys.NYS_ROUTE_CLUSTER_SMEM, nys.NYS_ROUTE_COOPERATIVE, nys.NYS_ROUTE_GRAPH}, routes


@pytest.mark.parametrize("m,n,ell", SIZES)
def test_natural_route_pcg_matches_oracle(nys, m, n, ell):
    h, A, D, Fw, U, lam = _system(nys, m, n, ell, seed=m + n)
    delta, eta = 1e-5, 1e-9
    xi = np.random.default_rng(m).standard_normal(m)
    Mv = lambda v: O.normal_matvec(A, D, delta, v)
    Pv = lambda v: O.precond_inv_apply(Fw, delta, v)
    # forced count: the same Krylov iterates up to summation order
    for forced in (1, 12):
        want = O.pcg(Mv, Pv, xi, eta, 1000, forced_iters=forced)
        dy, it, res, rc = nys.nys_pcg(h, T(A), T(D), delta, U, lam, T(xi), eta, 1000, forced=forced)
        assert it == forced and relerr(dy, want.x) <= 1e-10, (forced, relerr(dy, want.x))
    # free running: both meet the test; at the crossing the count moves with
    # the summation order by a few percent
    want = O.pcg(Mv, Pv, xi, eta, 4000)
    dy, it, res, rc = nys.nys_pcg(h, T(A), T(D), delta, U, lam, T(xi), eta, 4000)
    assert rc == 0 and want.converged
    assert abs(it - want.iters) <= max(2, 0.05 * want.iters)
    g = dy.cpu().numpy()
    M = A @ (D[:, None] * A.T) + delta * np.eye(m)
    assert np.linalg.norm(xi - M @ g) <= 1.01 * eta * np.linalg.norm(xi)
    exact = np.linalg.solve(M, xi)
    bound = 2.02 * eta * np.linalg.norm(xi) / sla.eigh(M, eigvals_only=True, subset_by_index=[0, 0])[0]
    assert np.linalg.norm(g - exact) <= bound
    assert np.linalg.norm(g - want.x) <= bound


@pytest.mark.parametrize("m,n,ell", [SIZES[3], SIZES[4]])
def test_natural_route_newton_direction_matches_oracle(nys, m, n, ell):
    """Algorithm 4 (RHS, PCG with a forced count, back-substitution) on the
    cooperative and graph routes' natural sizes: to 1e-10, or 100x the
    oracle's own rounding response where that floor is higher."""
    rng = np.random.default_rng(n)
    A = rng.standard_normal((m, n)) * (np.arange(1, m + 1) ** -1.0)[:, None]
    x, z = rng.uniform(0.1, 2, n), rng.uniform(0.01, 2, n)
    q = rng.uniform(0, 1, n)
    q[::3] = 0.0
    rho, delta = 1e-3, 1e-4
    D = O.scaling_D(x, z, q, rho)
    F = O.nystrom(A, D, O.gaussian_omega(2, 1, m, ell))
    r_d, r_p, r_xz = rng.standard_normal(n), rng.standard_normal(m), -x * z
    # rounding floor: the oracle's own response to a 2e-16 relative change of A
    # with the count held (CG on this system amplifies summation-order noise)
    a0 = O.newton_direction(A, x, z, D, delta, r_d, r_p, r_xz, F, 1e-8, 1000, 20)
    A2 = A * (1 + 2e-16 * np.sign(np.sin(np.arange(A.size)))).reshape(A.shape)
    a1 = O.newton_direction(A2, x, z, D, delta, r_d, r_p, r_xz, F, 1e-8, 1000, 20)
    floor = max(relerr(a1.dx, a0.dx), relerr(a1.dy, a0.dy), relerr(a1.dz, a0.dz))
    tol = max(1e-10, 100 * floor)
    h = nys.Handle(m, n, ell=ell)
    for forced in (20, None):
        want = O.newton_direction(A, x, z, D, delta, r_d, r_p, r_xz, F, 1e-8, 1000, forced)
        dx, dy, dz, it = nys.nys_newton(h, T(A), T(x), T(z), T(D), delta, T(r_d), T(r_p), T(r_xz),
                                        P(F.U), T(F.lam), 1e-8, 1000, **({} if forced is None else
                                                                        {"forced": forced}))
        if forced is not None:
            assert it == forced
            errs = [relerr(g, w) for g, w in ((dx, want.dx), (dy, want.dy), (dz, want.dz))]
            print(f"errs={errs} floor={floor:.1e}")
            assert max(errs) <= tol
        else:
            assert abs(it - want.pcg_iters) <= max(2, 0.05 * want.pcg_iters)
