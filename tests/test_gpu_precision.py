"""The precision form: tcgen05 BF16 sketch products and the BF16 + refinement
Newton solve, against the FP64 CPU oracle on the FP32 problem matrix."""
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


GEMM_SHAPES = [(128, 16, 64), (300, 40, 1000), (777, 256, 2048), (1000, 416, 5000), (129, 400, 4100),
               (2000, 100, 20001), (513, 96, 256), (3000, 416, 3000), (256, 512, 64)]


@pytest.mark.parametrize("kernel", ["0", "1"])
@pytest.mark.parametrize("M,N,K", GEMM_SHAPES)
def test_tensor_core_gemm_matches_fp64(nys, monkeypatch, kernel, M, N, K):
    """tcgen05 kind::f16 BF16 products (FP32 accumulation) against an FP64
    product of the same BF16 values; bound: K * 2^-24 growth on sum |a b|.
    kernel "0": one CTA per 128-row stripe (cta_group::1) with split-K;
    "1": a CTA pair per 256-row stripe (cta_group::2), k-blocks spread over
    the resident pairs -- shapes with whole tiles written directly (513 x 96
    x 256, 256 x 512 x 64) and with tiles summed from several pairs."""
    monkeypatch.setenv("NYS_UMMA_PAIR", kernel)
    g = torch.Generator().manual_seed(M + N + K)
    ldk = (K + 7) // 8 * 8
    A = torch.zeros(M, ldk, dtype=torch.bfloat16)
    B = torch.zeros(N, ldk, dtype=torch.bfloat16)
    A[:, :K] = (torch.rand(M, K, generator=g) - 0.5).to(torch.bfloat16)
    B[:, :K] = (torch.rand(N, K, generator=g) - 0.5).to(torch.bfloat16)
    h = nys.Handle(16384, 4096, ell=128)   # workspace for the pair kernel's partial tiles
    Ad, Bd = A.to(DEV), B.to(DEV)
    Av = Ad[:, :K] if ldk == K else Ad.narrow(1, 0, K)
    C = nys.nys_gemm_bf16(h, Av, Bd.narrow(1, 0, K)).cpu().double()
    ref = (A[:, :K].double() @ B[:, :K].double().T).T
    bound = (A[:, :K].double().abs() @ B[:, :K].double().abs().T).T
    err = (C - ref).abs()
    assert float((err - 4 * K * 2.0 ** -24 * bound).max()) <= 1e-6
    # deterministic: the same bits on a second call
    C2 = nys.nys_gemm_bf16(h, Av, Bd.narrow(1, 0, K)).cpu().double()
    assert torch.equal(C, C2)


@pytest.mark.parametrize("kernel", ["0", "1"])
@pytest.mark.parametrize("m,n,ell", [(300, 1200, 40), (2000, 600, 100), (500, 1200, 400), (1000, 3000, 400)])
def test_precision_sketch_matches_fp64(nys, monkeypatch, kernel, m, n, ell):
    """The precision form's sketch (Algorithm 1, second step, on the tensor
    cores): T = A_b^T Omega_b, T' = BF16(D .* T), Y = A_b T' against the FP64
    product A_b (D .* (A_b^T Omega_b)) of the same BF16 values.  Bound: the
    FP32 accumulation of each product (4 K 2^-24 on sums of |a b|) and one
    BF16 rounding of D .* T (2^-8).  The shapes put the D-scaled BF16 output
    of the first product on the direct path (300 x 1200, 500 x 1200: whole tiles) and on
    the summed-partials path (2000 x 600, 1000 x 3000), with one and two MMA
    chunks (ell 40 / 100 and 400)."""
    monkeypatch.setenv("NYS_UMMA_PAIR", kernel)
    rng = np.random.default_rng(m + n + ell)
    A32 = (rng.standard_normal((m, n)) / np.sqrt(n)).astype(np.float32)
    D = 10.0 ** rng.uniform(-2, 2, n)
    Om = rng.standard_normal((m, ell))
    h = nys.Handle(m, n, ell=ell, precision_mode=1)
    Y = nys.nys_sketch(h, torch.from_numpy(A32).to(DEV), torch.from_numpy(D).to(DEV),
                       torch.from_numpy(np.ascontiguousarray(Om.T)).to(DEV)).cpu().numpy().T
    Ab = torch.from_numpy(A32).bfloat16().double().numpy()
    Omb = torch.from_numpy(Om).float().bfloat16().double().numpy()
    T = Ab.T @ Omb
    Yref = Ab @ (D[:, None] * T)
    errT = 4 * m * 2.0 ** -24 * (np.abs(Ab.T) @ np.abs(Omb))
    Tmag = D[:, None] * (np.abs(T) + errT)
    bound = (np.abs(Ab) @ (2.0 ** -8 * Tmag + D[:, None] * errT)
             + 4 * n * 2.0 ** -24 * (np.abs(Ab) @ Tmag) * (1 + 2.0 ** -8))
    assert np.all(np.abs(Y - Yref) <= bound), float(np.max(np.abs(Y - Yref) / bound))
    assert np.linalg.norm(Y - Yref) <= 1e-2 * np.linalg.norm(Yref)


def _qp32(seed, m, n):
    qp = synth.workload_precision_scaled(seed=seed, m=m, n=n)
    A32 = qp.A.astype(np.float32)                 # the FP32 matrix defines the problem
    A64 = A32.astype(np.float64)
    b = A64 @ qp.x0                               # keep the start feasible for the FP32 matrix
    c = A64.T @ qp.y0 + qp.z0 - qp.q * qp.x0
    return A32, A64, b, c, qp


def test_precision_form_meets_kkt_and_tracks_the_fp64_oracle(nys):
    """BF16 inner PCG + FP32/float-float refinement: KKT <= 1e-6 on the FP32
    problem, and the solution agrees with the FP64 oracle's to the tolerance
    level (both stop at tol 1e-6 on different iterates)."""
    m, n, ell, tol = 600, 3000, 30, 1e-6
    A32, A64, b, c, qp = _qp32(31, m, n)
    ref = O.solve(A64, b, c, qp.q, qp.x0, qp.y0, qp.z0, O.Options(tol=tol, ell=ell, seed=5))
    assert ref.status == "converged"
    h = nys.Handle(m, n, ell=ell, tol=tol, seed=5, precision_mode=1)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    x, y, z, info = nys.nys_solve(h, T(A32), T(b), T(c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))
    assert info["status"] == 0, info
    xs, ys, zs = (t.cpu().numpy() for t in (x, y, z))
    rp, rd, mu = O.kkt_measures(A64, b, c, qp.q, xs, ys, zs)
    assert rp <= tol and rd <= tol and mu <= tol
    err = np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x)
    print(f"precision form: {info['ipm_iters']} IPM, {info['pcg_iters_total']} PCG, "
          f"{info['refine_steps']} refinement steps; |x - x_oracle| / |x| = {err:.2e}")
    assert err <= 1e-3
    assert info["refine_steps"] >= 2 * info["ipm_iters"]


def test_precision_form_with_a_large_sketch(nys):
    """ell = 128 takes the QR route of the Nystrom core and a 128-column
    tensor-core sketch; the solve must still meet KKT <= 1e-6 (checked in
    FP64 on the FP32 problem)."""
    m, n, ell, tol = 1200, 5000, 128, 1e-6
    A32, A64, b, c, qp = _qp32(44, m, n)
    h = nys.Handle(m, n, ell=ell, tol=tol, seed=6, precision_mode=1)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    x, y, z, info = nys.nys_solve(h, T(A32), T(b), T(c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))
    assert info["status"] in (0, 2), info
    rp, rd, mu = O.kkt_measures(A64, b, c, qp.q, *(t.cpu().numpy() for t in (x, y, z)))
    assert rp <= tol and rd <= tol and mu <= tol


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_fp8_quantisation_matches_the_definition(nys):
    """Per-row scales and E4M3 codes against the definition (FP32 division,
    round to nearest even, saturation), bit for bit; the transposed copy
    holds the same codes; padding is zero."""
    m, n = 37, 53
    rng = np.random.default_rng(8)
    A = (rng.standard_normal((m, n)) * np.exp(rng.uniform(-6, 6, (m, 1)))).astype(np.float32)
    A[4] = 0.0
    A[7, 3] = 1e-30
    h = nys.Handle(m, n, ell=4, precision_mode=2)
    Q, QT, s = nys.nys_quantize_fp8(h, T(A))
    Qref, sref = O.fp8_rowscale_quantize(A)
    assert np.array_equal(s.cpu().numpy(), sref)
    q = Q.cpu().numpy()
    assert np.array_equal(O.e4m3_decode(q[:, :n]), Qref)
    assert np.all(q[:, n:] == 0) and np.all(QT.cpu().numpy()[:, m:] == 0)
    assert np.array_equal(QT.cpu().numpy()[:, :m], q[:, :n].T)


@pytest.mark.parametrize("m,n", [(300, 1000), (1001, 4099)])
def test_fp8_operator_matches_the_definition(nys, m, n):
    """diag(s) Q (D .* (Q^T (s .* v))) + delta v with FP32 products and sums
    against the same expression in FP64 on the decoded codes: FP32 rounding
    of the inputs and of sums of up to max(m, n) terms."""
    rng = np.random.default_rng(m + n)
    A = (rng.standard_normal((m, n)) / np.sqrt(n)).astype(np.float32)
    h = nys.Handle(m, n, ell=4, precision_mode=2)
    Q, QT, s = nys.nys_quantize_fp8(h, T(A))
    Qd = O.e4m3_decode(Q.cpu().numpy()[:, :n])
    sv = s.cpu().numpy()
    D = rng.uniform(0.1, 3.0, n)
    v = rng.standard_normal(m)
    out = nys.nys_normal_matvec_fp8(h, m, n, Q, QT, s, T(D), 1e-3, T(v)).cpu().numpy()
    ref = O.fp8_normal_matvec(Qd, sv, D, 1e-3, v)
    # elementwise bound: (max(m, n) + 4) * 2^-24 on the sums of |terms|
    absref = np.abs(sv) * (np.abs(Qd) @ (D * (np.abs(Qd).T @ np.abs(sv * v)))) + 1e-3 * np.abs(v)
    assert np.all(np.abs(out - ref) <= (max(m, n) + 4) * 2.0 ** -24 * absref * 2)


def test_fp8_precision_form_meets_kkt(nys):
    """precision_mode 2: FP8 inner PCG (E4M3 A and A^T with row scales),
    FP32 float-float refinement: KKT <= 1e-6 on the FP32 problem, and the
    solution agrees with the FP64 oracle's to the tolerance level."""
    m, n, ell, tol = 600, 3000, 30, 1e-6
    A32, A64, b, c, qp = _qp32(31, m, n)
    ref = O.solve(A64, b, c, qp.q, qp.x0, qp.y0, qp.z0, O.Options(tol=tol, ell=ell, seed=5))
    h = nys.Handle(m, n, ell=ell, tol=tol, seed=5, precision_mode=2)
    x, y, z, info = nys.nys_solve(h, T(A32), T(b), T(c), T(qp.q), T(qp.x0), T(qp.y0), T(qp.z0))
    assert info["status"] in (0, 2), info
    xs, ys, zs = (t.cpu().numpy() for t in (x, y, z))
    rp, rd, mu = O.kkt_measures(A64, b, c, qp.q, xs, ys, zs)
    assert rp <= tol and rd <= tol and mu <= tol
    err = np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x)
    print(f"FP8 precision form: {info['ipm_iters']} IPM, {info['pcg_iters_total']} PCG, "
          f"{info['refine_steps']} refinement steps; |x - x_oracle| / |x| = {err:.2e}")
    assert err <= 1e-3


@pytest.mark.parametrize("op", ["ff", "bf16", "fp8"])
def test_precision_operator_pcg(nys, op):
    """PCG on the precision form's operators: with the float-float FP32
    operator it solves the FP32 matrix's system (true FP64 residual at the
    tolerance); with BF16 / FP8 storage it solves the system of the rounded
    matrix (residual measured with the rounded values)."""
    m, n, ell = 400, 1600, 16
    rng = np.random.default_rng(12)
    A32 = (rng.standard_normal((m, n)) * (np.arange(1, m + 1) ** -0.5)[:, None] / np.sqrt(n)).astype(np.float32)
    A64 = A32.astype(np.float64)
    D = rng.uniform(0.1, 3.0, n)
    Om = O.gaussian_omega(3, 0, m, ell)
    F = O.nystrom_from_sketch(O.sketch(A64, D, Om), Om)
    xi = rng.standard_normal(m)
    delta, eta = 1e-3, 1e-8
    h = nys.Handle(m, n, ell=ell, precision_mode=2 if op == "fp8" else 1)
    U = T(np.ascontiguousarray(F.U.T))
    dy, it, res, rc = nys.nys_pcg_lp(h, T(A32), op, T(D), delta, U, T(F.lam), T(xi), eta, 2000)
    assert rc == 0 and it < 2000
    y = dy.cpu().numpy()
    if op == "ff":
        Ar = A64
    elif op == "bf16":
        Ar = torch.from_numpy(A32).to(torch.bfloat16).double().numpy()
    else:
        Q, s = O.fp8_rowscale_quantize(A32)
        Ar = s[:, None].astype(np.float64) * Q
    r = np.linalg.norm(xi - O.normal_matvec(Ar, D, delta, y)) / np.linalg.norm(xi)
    # FP32 products: the recursive residual meets eta; the true one within the
    # operator's rounding (n 2^-24 relative for the FP32 sums, 2^-44 for float-float)
    assert r <= (10 * eta if op == "ff" else 10 * eta + 1e-5)
