"""Seeded synthetic separable-QP workloads.

This module only builds problem data: it holds none of the solver's arithmetic,
so both the CUDA path and the CPU oracle can take their inputs from it.

Every workload is a primal-dual pair (P)/(D) of Section 1 with diagonal
Q = diag(q) >= 0 and x >= 0.  The paper's own workloads (SVM datasets of
Table 3, the portfolio generator of Section 5.1) are not reproducible here,
so these generators stand in for them with dense constraint matrices of a
prescribed singular-value spectrum:

    A = U diag(sigma) V^T,  U = Haar m x m orthogonal,  V = Haar n x m
    (orthonormal columns), built as the sign-fixed Q factor of a Gaussian.

The feasible start is built so that the start point is strictly interior and
primal/dual feasible: x0 ~ U[0.5, 1.5], b = A x0, y0 ~ N(0, 1),
z0 ~ U[0, 1] clamped to >= 1e-3, c = A^T y0 + z0 - Q x0.

Problems with free and box-constrained variables, (P~)/(D~), carry a kind per
variable (KIND_I: x_j >= 0, KIND_F: free, KIND_J: 0 <= x_j <= u_j), the upper
bounds u and the start s0 of the bound multipliers; see `box_qp`.
"""
from __future__ import annotations

import dataclasses
import numpy as np

Z0_FLOOR = 1e-3
KIND_I, KIND_F, KIND_J = 0, 1, 2


@dataclasses.dataclass
class QP:
    """One separable QP (P)/(D) with a feasible interior start point (all float64,
    A row-major m x n)."""
    A: np.ndarray
    b: np.ndarray
    c: np.ndarray
    q: np.ndarray
    x0: np.ndarray
    y0: np.ndarray
    z0: np.ndarray
    name: str = ""
    kind: np.ndarray | None = None    # int8 per variable (None: every x_j >= 0)
    u: np.ndarray | None = None       # upper bounds (0 outside KIND_J)
    s0: np.ndarray | None = None      # start of the bound multipliers (0 outside KIND_J)

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.shape[1]


def haar_columns(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """rows x cols matrix with orthonormal columns, Haar-distributed (QR of a
    Gaussian with the signs of R's diagonal folded into Q)."""
    g = rng.standard_normal((rows, cols))
    qf, r = np.linalg.qr(g, mode="reduced")
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return qf * s[None, :]


def spectrum_matrix(rng: np.random.Generator, m: int, n: int, sigma: np.ndarray) -> np.ndarray:
    """A = U diag(sigma) V^T with Haar factors; requires m <= n, len(sigma) == m."""
    assert m <= n and sigma.shape == (m,)
    u = haar_columns(rng, m, m)
    v = haar_columns(rng, n, m)
    return np.ascontiguousarray((u * sigma[None, :]) @ v.T)


def feasible_qp(rng: np.random.Generator, A: np.ndarray, q: np.ndarray, name: str = "") -> QP:
    """Attach the feasible-start generator to a constraint matrix and diag(Q)."""
    m, n = A.shape
    x0 = rng.uniform(0.5, 1.5, n)
    y0 = rng.standard_normal(m)
    z0 = np.maximum(rng.uniform(0.0, 1.0, n), Z0_FLOOR)
    b = A @ x0
    c = A.T @ y0 + z0 - q * x0
    return QP(A=A, b=b, c=c, q=q, x0=x0, y0=y0, z0=z0, name=name)


def feasible_box_qp(rng: np.random.Generator, A: np.ndarray, q: np.ndarray, frac_free: float,
                    frac_box: float, name: str = "") -> QP:
    """Feasible interior start for (P~)/(D~): a random floor(frac_free n)
    variables are free, floor(frac_box n) box-constrained, the rest
    non-negative.  x0 ~ U[0.5, 1.5] on I and J, N(0, 1) on F;
    u_J = x0_J + U[0.5, 1.5] (so the slack u - x0 lies in [0.5, 1.5]);
    z0 ~ U[0, 1] clamped to >= 1e-3 on I and J, 0 on F; s0 likewise on J,
    0 elsewhere; y0 ~ N(0, 1); b = A x0 and c = A^T y0 + z0 - s0 - Q x0, so
    the start satisfies both equality constraints."""
    m, n = A.shape
    perm = rng.permutation(n)
    nf, nb = int(frac_free * n), int(frac_box * n)
    kind = np.full(n, KIND_I, dtype=np.int8)
    kind[perm[:nf]] = KIND_F
    kind[perm[nf:nf + nb]] = KIND_J
    free, box = kind == KIND_F, kind == KIND_J
    x0 = np.where(free, rng.standard_normal(n), rng.uniform(0.5, 1.5, n))
    u = np.where(box, x0 + rng.uniform(0.5, 1.5, n), 0.0)
    y0 = rng.standard_normal(m)
    z0 = np.where(free, 0.0, np.maximum(rng.uniform(0.0, 1.0, n), Z0_FLOOR))
    s0 = np.where(box, np.maximum(rng.uniform(0.0, 1.0, n), Z0_FLOOR), 0.0)
    b = A @ x0
    c = A.T @ y0 + z0 - s0 - q * x0
    return QP(A=A, b=b, c=c, q=q, x0=x0, y0=y0, z0=z0, name=name, kind=kind, u=u, s0=s0)


def box_qp(seed: int, m: int, n: int, frac_free: float = 0.1, frac_box: float = 0.3,
           sigma_kind: str = "inv", q_kind: str = "uniform") -> QP:
    """Dense QP with free and box-constrained variables (problems (P~)/(D~)):
    the spectral constraint matrix of `spectral_qp` with the start of
    `feasible_box_qp`."""
    rng = np.random.default_rng(seed)
    i = np.arange(1, m + 1, dtype=np.float64)
    sigma = {"inv": 1.0 / i, "pow0.8": i ** -0.8, "exp200": np.exp(-i / 200.0) + 1e-3}[sigma_kind]
    A = spectrum_matrix(rng, m, n, sigma)
    q = make_q(rng, n, q_kind)
    return feasible_box_qp(rng, A, q, frac_free, frac_box,
                           name=f"box-{sigma_kind}-{m}x{n}-f{frac_free}-b{frac_box}-s{seed}")


def svm_qp(seed: int, d: int, n_samples: int, tau: float = 1.0, sep: float = 1.0) -> QP:
    """Dual linear SVM with l1 slack penalty, written as (P~) (the supplement's
    SVM formulation): x = (v, p), v in R^d free, 0 <= p_i <= tau;
    A = [[I_d, -X diag(lab)], [0, lab^T]], b = 0, Q = diag(1_d, 0_n),
    c = (0_d, -1_n) (the objective 1/2 v^T v - sum p_i).
    Synthetic dense features stand in for the SVM datasets: balanced labels
    lab = +-1, samples X_i = (lab_i * mu + g_i) / sqrt(d) with mu ~ sep * N(0, I_d)
    and g_i ~ N(0, I_d) (every entry non-zero).  Start (interior; primal
    feasible when n_samples is even): p0 = tau/2, v0 = X diag(lab) p0,
    y0 = 0, z0 = s0 = 1 on J."""
    rng = np.random.default_rng(seed)
    lab = np.where(rng.permutation(n_samples) < n_samples // 2, 1.0, -1.0)
    mu = sep * rng.standard_normal(d)
    X = (lab[None, :] * mu[:, None] + rng.standard_normal((d, n_samples))) / np.sqrt(d)
    m, n = d + 1, d + n_samples
    A = np.zeros((m, n))
    A[:d, :d] = np.eye(d)
    A[:d, d:] = -X * lab[None, :]
    A[d, d:] = lab
    q = np.concatenate([np.ones(d), np.zeros(n_samples)])
    c = np.concatenate([np.zeros(d), -np.ones(n_samples)])
    kind = np.concatenate([np.full(d, KIND_F), np.full(n_samples, KIND_J)]).astype(np.int8)
    u = np.concatenate([np.zeros(d), np.full(n_samples, tau)])
    p0 = np.full(n_samples, 0.5 * tau)
    x0 = np.concatenate([(X * lab[None, :]) @ p0, p0])
    z0 = np.concatenate([np.zeros(d), np.ones(n_samples)])
    s0 = np.concatenate([np.zeros(d), np.ones(n_samples)])
    return QP(A=np.ascontiguousarray(A), b=np.zeros(m), c=c, q=q, x0=x0, y0=np.zeros(m), z0=z0,
              name=f"svm-{d}x{n_samples}-s{seed}", kind=kind, u=u, s0=s0)


def portfolio_qp(seed: int, n_assets: int, d: int, s: int, gamma: float = 1.0) -> QP:
    """Factor-model portfolio problem of the supplement, written as (P~):
    minimise -r^T x / gamma + x^T Dg x + y^T y subject to y = F^T x, M x <= u,
    1^T x = 1, x >= 0, y free.  Variables (x, y, t) with the slack t >= 0 of
    M x + t = u: A = [[F^T, -I_s, 0], [M, 0, I_d], [1^T, 0, 0]],
    b = (0_s, u, 1), Q = diag(2 Dg, 2 1_s, 0_d), c = (-r / gamma, 0, 0).
    Risk model: Sigma = U diag(lam) U^T + 0.01 I with U Haar (n x 2s) and a
    spectrum that decays fast over the first s and slowly after
    (lam_i = exp(-8 i / s) for i <= s, then 0.01 (s / i)^0.5); F = the top-s
    eigenpairs U_s diag(lam_s)^{1/2} and Dg = diag(Sigma - F F^T) (exact
    eigenpairs stand in for the paper's randomized Nystrom risk model).
    M rows ~ N(0, I_n); r ~ N(0, 1); u ~ U[0, 1], raised where needed to
    M 1/n + 1e-3 so that the equal-weight portfolio is feasible.  Start
    (interior): x0 = 1/n, y0' = F^T x0, t0 = u - M x0; dual y0 = 0, z0 = 1
    on x and t, 0 on the free y."""
    rng = np.random.default_rng(seed)
    k = 2 * s
    U = haar_columns(rng, n_assets, k)
    i = np.arange(1, k + 1, dtype=np.float64)
    lam = np.where(i <= s, np.exp(-8.0 * i / s), 0.01 * np.sqrt(s / i))
    F = U[:, :s] * np.sqrt(lam[:s])[None, :]
    Dg = (U[:, s:] ** 2) @ lam[s:] + 0.01
    M = rng.standard_normal((d, n_assets))
    r = rng.standard_normal(n_assets)
    xe = np.full(n_assets, 1.0 / n_assets)
    u = np.maximum(rng.uniform(0.0, 1.0, d), M @ xe + 1e-3)
    m, n = s + d + 1, n_assets + s + d
    A = np.zeros((m, n))
    A[:s, :n_assets] = F.T
    A[:s, n_assets:n_assets + s] = -np.eye(s)
    A[s:s + d, :n_assets] = M
    A[s:s + d, n_assets + s:] = np.eye(d)
    A[s + d, :n_assets] = 1.0
    b = np.concatenate([np.zeros(s), u, [1.0]])
    q = np.concatenate([2.0 * Dg, np.full(s, 2.0), np.zeros(d)])
    c = np.concatenate([-r / gamma, np.zeros(s + d)])
    kind = np.concatenate([np.full(n_assets, KIND_I), np.full(s, KIND_F), np.full(d, KIND_I)]).astype(np.int8)
    x0 = np.concatenate([xe, F.T @ xe, u - M @ xe])
    z0 = np.concatenate([np.ones(n_assets), np.zeros(s), np.ones(d)])
    return QP(A=np.ascontiguousarray(A), b=b, c=c, q=q, x0=x0, y0=np.zeros(m), z0=z0,
              name=f"portfolio-{n_assets}x{d}x{s}-s{seed}", kind=kind, u=np.zeros(n), s0=np.zeros(n))


def spectral_qp(seed: int, m: int, n: int, sigma_kind: str, q_kind: str = "uniform") -> QP:
    """Single dense QP with a prescribed spectrum.

    sigma_kind: "inv" (sigma_i = 1/i), "pow0.8" (sigma_i = i^-0.8),
                "exp200" (sigma_i = exp(-i/200) + 1e-3).
    q_kind:     "uniform" (q ~ U[0,1]), "half_zero" (50% zeros, rest U[0,1]),
                "uniform_0.1" (q ~ U[0.1, 1]), "zero" (an LP).
    """
    rng = np.random.default_rng(seed)
    i = np.arange(1, m + 1, dtype=np.float64)
    if sigma_kind == "inv":
        sigma = 1.0 / i
    elif sigma_kind == "pow0.8":
        sigma = i ** -0.8
    elif sigma_kind == "exp200":
        sigma = np.exp(-i / 200.0) + 1e-3
    else:
        raise ValueError(sigma_kind)
    A = spectrum_matrix(rng, m, n, sigma)
    q = make_q(rng, n, q_kind)
    return feasible_qp(rng, A, q, name=f"spectral-{sigma_kind}-{m}x{n}-s{seed}")


def make_q(rng: np.random.Generator, n: int, q_kind: str) -> np.ndarray:
    if q_kind == "uniform":
        return rng.uniform(0.0, 1.0, n)
    if q_kind == "half_zero":
        q = rng.uniform(0.0, 1.0, n)
        q[rng.permutation(n)[: n // 2]] = 0.0
        return q
    if q_kind == "uniform_0.1":
        return rng.uniform(0.1, 1.0, n)
    if q_kind == "zero":
        return np.zeros(n)
    raise ValueError(q_kind)


def gaussian_qp(seed: int, m: int, n: int, q_kind: str = "uniform_0.1") -> QP:
    """Dense QP with i.i.d. N(0, 1/n) constraint entries (the differentiation
    workload: 64 QPs of 512 x 2048 with q ~ U[0.1, 1])."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) / np.sqrt(n)
    q = make_q(rng, n, q_kind)
    return feasible_qp(rng, A, q, name=f"gaussian-{m}x{n}-s{seed}")


def low_rank_qp(seed: int, m: int, n: int, rank: int, q_kind: str = "uniform") -> QP:
    """QP whose A has exact rank `rank` < m (A A^T singular); b is still
    consistent because b = A x0.  Used where N = A D A^T must have rank <= ell."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n)) / np.sqrt(n)
    q = make_q(rng, n, q_kind)
    return feasible_qp(rng, A, q, name=f"lowrank{rank}-{m}x{n}-s{seed}")


# ---------------------------------------------------------------------------
# Named workloads with the shapes of the five benchmark configurations.
# ---------------------------------------------------------------------------

def workload_small(seed: int = 1235) -> QP:
    """m=200, n=500, sigma_i = 1/i, q ~ U[0,1]; solved with ell=20, tol 1e-6."""
    return spectral_qp(seed, 200, 500, "inv", "uniform")


def workload_box(seed: int = 1240, m: int = 200, n: int = 500) -> QP:
    """The m=200, n=500 shape (sigma_i = 1/i, q ~ U[0,1]) with 10% free and
    30% box-constrained variables; solved with ell=20, tol 1e-6."""
    return box_qp(seed, m, n, 0.1, 0.3, "inv", "uniform")


def workload_fp64(seed: int = 1236) -> QP:
    """m=5000, n=20000, sigma_i = i^-0.8, q half zeros; ell=100, tol 1e-8."""
    return spectral_qp(seed, 5000, 20000, "pow0.8", "half_zero")


def workload_fp64_scaled(seed: int = 1236, m: int = 1000, n: int = 4000) -> QP:
    """Scaled-down shape of the m=5000, n=20000 workload (same recipe)."""
    return spectral_qp(seed, m, n, "pow0.8", "half_zero")


def workload_precision_scaled(seed: int = 1237, m: int = 2000, n: int = 10000) -> QP:
    """Scaled-down shape of the m=20000, n=100000 precision workload
    (sigma_i = exp(-i/200) + 1e-3, q ~ U[0,1])."""
    return spectral_qp(seed, m, n, "exp200", "uniform")


def workload_batch(seed: int = 1238, count: int = 256, m_lo: int = 64, m_hi: int = 1024):
    """`count` QPs with m ~ U{m_lo..m_hi}, n ~ U{4m..8m}, sigma_i = 1/i,
    q ~ U[0,1]; per-QP ell = min(32, m // 4)."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        m = int(rng.integers(m_lo, m_hi + 1))
        n = int(rng.integers(4 * m, 8 * m + 1))
        out.append(spectral_qp(seed * 1000 + t, m, n, "inv", "uniform"))
    return out


def workload_diff(seed: int = 1239, count: int = 64, m: int = 512, n: int = 2048):
    """`count` Gaussian QPs (m x n) with q ~ U[0.1, 1] and targets x_t ~ U[0,1]
    for the loss L = ||x* - x_t||^2."""
    rng = np.random.default_rng(seed)
    qps = [gaussian_qp(seed * 1000 + t, m, n, "uniform_0.1") for t in range(count)]
    targets = [rng.uniform(0.0, 1.0, n) for _ in range(count)]
    return qps, targets


def spectral_qp_device(seed: int, m: int, n: int, sigma_kind: str, q_kind: str = "uniform",
                       device="cuda", dtype=None):
    """Large-scale variant of `spectral_qp` generated on the GPU with torch
    (Haar factors from a QR of a Gaussian on the device).  A is returned in
    `dtype` (float32 by default: the FP32 matrix then defines the problem) and
    the feasible start is built from that stored A in FP64.  Returns torch
    tensors on `device`: A, b, c, q, x0, y0, z0."""
    import torch
    dtype = dtype or torch.float32
    g = torch.Generator(device=device).manual_seed(seed)
    i = torch.arange(1, m + 1, dtype=torch.float64, device=device)
    sigma = {"inv": 1.0 / i, "pow0.8": i ** -0.8, "exp200": torch.exp(-i / 200.0) + 1e-3}[sigma_kind]
    work = torch.float32
    u, ru = torch.linalg.qr(torch.randn(m, m, generator=g, device=device, dtype=work))
    u = u * torch.where(torch.diagonal(ru) < 0, -1.0, 1.0)
    v, rv = torch.linalg.qr(torch.randn(n, m, generator=g, device=device, dtype=work))
    v = v * torch.where(torch.diagonal(rv) < 0, -1.0, 1.0)
    A = ((u * sigma.to(work)) @ v.T).to(dtype).contiguous()
    del u, v, ru, rv
    gq = torch.rand(n, generator=g, device=device, dtype=torch.float64)
    if q_kind == "half_zero":
        gq[torch.randperm(n, generator=g, device=device)[: n // 2]] = 0.0
    elif q_kind == "uniform_0.1":
        gq = 0.1 + 0.9 * gq
    elif q_kind == "zero":
        gq = torch.zeros_like(gq)
    x0 = 0.5 + torch.rand(n, generator=g, device=device, dtype=torch.float64)
    y0 = torch.randn(m, generator=g, device=device, dtype=torch.float64)
    z0 = torch.rand(n, generator=g, device=device, dtype=torch.float64).clamp(min=Z0_FLOOR)
    A64 = A.double()
    b = A64 @ x0
    c = A64.T @ y0 + z0 - gq * x0
    del A64
    return A, b, c, gq, x0, y0, z0
