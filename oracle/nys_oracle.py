"""Plain FP64 CPU oracle of Nys-IP-PMM (arxiv 2404.14524) for separable QPs.

TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU-baseline
leg of the benchmark import this module.  The product (the CUDA library and its
Python binding) never imports, calls or links it, and it shares no code with
the CUDA path: the two meet only through the seeded workload generators.

The oracle is deliberately slow and literal.  Each function follows one passage
of the paper, step by step and in the paper's notation, with library routines
(matrix products, Cholesky, triangular solve, SVD) as the only building blocks.
Readings taken where the paper is silent or garbled are marked READING.

Scope: the practical method (Algorithm 6 driving the Mehrotra predictor-corrector
of Algorithm 5 and the Newton solve of Algorithm 4) for problem (P)/(D), where
every variable is non-negative (I = {1..n}), and for its generalisation
(P~)/(D~) with free variables (set F) and box-constrained variables
0 <= x_j <= u_j (set J) of the section on free and box-constrained variables.
The all-non-negative case is the general code with F = J = {}: it only adds
exact zeros, so both cases share one implementation.

Pinning (tests/test_oracle_*.py): every function is checked against something
other than itself -- the assembled 3x3-block Newton system (Eq. Newton) and
the 5x5-block system with free and box-constrained variables
(Eq. Newton-free-box), scipy's HiGHS on bounded LPs, hand-derived practical
starting points (tests/golden/start_points.txt),
P_Nys from Eq. Nys_precond against P_Nys^{-1} from Eq. Nys_precond_inv, the
Nystrom invariants of Section 2.3.2, a dense direct solve of the normal
equations, brute-force active-set solutions of tiny QPs, hand-derived KKT
points (tests/golden/), brute-force step-length scans, and numpy's spacing()
for eps().  The PEU rule, the termination rule and the PCG tolerance are
builder's readings of passages that only cite another paper; their constants
are "parity unpinned" (they are made identical on both sides, not checked
against the paper).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg as sla

# ---------------------------------------------------------------------------
# Counter-based Gaussian test matrices (Algorithm 1, first step).
#
# READING: Algorithm 1 draws a fresh Gaussian Omega in every call.  Both the
# oracle and the CUDA path draw entry (i, j) of Omega_k (IPM iteration k,
# m x ell) from the SplitMix64 stream of Steele, Lea and Flood (OOPSLA 2014),
# seeded with `seed`, at stream positions 2c and 2c+1 with
# c = (k*ell + j)*m + i, turned into uniforms u = ((bits >> 11) + 1/2) 2^-53
# and into one normal deviate by Box-Muller: sqrt(-2 ln u1) cos(2 pi u2).
# ---------------------------------------------------------------------------

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_at(seed: int, pos: np.ndarray) -> np.ndarray:
    """Output number `pos` (0-based) of the SplitMix64 stream whose state
    starts at `seed`: the state after pos+1 increments by the golden gamma,
    passed through the SplitMix64 finaliser."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (pos.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def gaussian_omega(seed: int, k: int, m: int, ell: int) -> np.ndarray:
    """Omega_k, m x ell, float64 (row i, column j)."""
    i = np.arange(m, dtype=np.uint64)[:, None]
    j = np.arange(ell, dtype=np.uint64)[None, :]
    c = (np.uint64(k) * np.uint64(ell) + j) * np.uint64(m) + i
    b1 = splitmix64_at(seed, np.uint64(2) * c)
    b2 = splitmix64_at(seed, np.uint64(2) * c + np.uint64(1))
    u1 = ((b1 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    u2 = ((b2 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def eps_of(x: float) -> float:
    """eps(x) of Algorithm 1, third step: the spacing of float64 numbers at x > 0,
    2^(floor(log2 x) - 52).  READING: exactly Julia/MATLAB eps()."""
    if not (x > 0.0) or not math.isfinite(x):
        raise ValueError("eps_of needs a positive finite argument")
    _, e = math.frexp(x)          # x = f 2^e, f in [0.5, 1)
    return math.ldexp(1.0, e - 53)


# ---------------------------------------------------------------------------
# Normal-equations operator (Section 2.1.2, Eq. normal-eq).
# ---------------------------------------------------------------------------

# Variable kinds of (P~)/(D~): x_j >= 0 (I), free (F), 0 <= x_j <= u_j (J).
KIND_I, KIND_F, KIND_J = 0, 1, 2


def scaling_D(x: np.ndarray, z: np.ndarray, q: np.ndarray, rho: float,
              kind: np.ndarray | None = None, w: np.ndarray | None = None,
              s: np.ndarray | None = None) -> np.ndarray:
    """Diagonal of (Q + Theta^{-1} + rho I)^{-1} with Theta = X Z^{-1}
    (Section 2.1.2, below Eq. delta_z).

    With free and box-constrained variables (Eq. normal-eq-free-box),
    eliminating dz, dw and ds from Eq. Newton-free-box leaves
    Theta^{-1}_j = z_j / x_j on I, z_j / x_j + s_j / w_j on J and 0 on F."""
    if kind is None:
        return 1.0 / (q + z / x + rho)
    theta_inv = np.zeros_like(x)
    ij = kind != KIND_F
    theta_inv[ij] = z[ij] / x[ij]
    jj = kind == KIND_J
    theta_inv[jj] += s[jj] / w[jj]
    return 1.0 / (q + theta_inv + rho)


def normal_matvec(A: np.ndarray, D: np.ndarray, delta: float, v: np.ndarray) -> np.ndarray:
    """(N_k + delta I) v with N_k = A D A^T (Eq. normal-eq)."""
    return A @ (D * (A.T @ v)) + delta * v


def sketch(A: np.ndarray, D: np.ndarray, Omega: np.ndarray) -> np.ndarray:
    """Y = N Omega with N = A D A^T (Algorithm 1, second step)."""
    return A @ (D[:, None] * (A.T @ Omega))


# ---------------------------------------------------------------------------
# FP8 storage of the precision form (a per-row-scaled variant of the
# operator of Eq. normal-eq): E4M3 = 1 sign, 4 exponent (bias 7), 3 mantissa
# bits, no infinities, largest finite 448, subnormal spacing 2^-9.
# ---------------------------------------------------------------------------

E4M3_MAX = 448.0


def e4m3_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest E4M3 value (ties to even mantissa), saturating at
    +-448.  Works on the exact values of x (FP64 holds every input exactly)."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.clip(e, -6.0, 8.0)                  # below 2^-6: the subnormal spacing 2^-9
    quantum = np.exp2(e - 3.0)                 # 3 mantissa bits
    q = np.round(a / quantum) * quantum        # numpy rounds halves to even
    q = np.minimum(q, E4M3_MAX)
    return np.copysign(q, x)


def e4m3_decode(bits: np.ndarray) -> np.ndarray:
    """Values of E4M3 bit patterns (uint8)."""
    b = np.asarray(bits, dtype=np.int64)
    sgn = np.where(b >> 7, -1.0, 1.0)
    ex = (b >> 3) & 15
    man = b & 7
    val = np.where(ex == 0, man / 8.0 * 2.0 ** -6, (1.0 + man / 8.0) * np.exp2(ex - 7.0))
    val = np.where((ex == 15) & (man == 7), np.nan, val)
    return sgn * val


def fp8_rowscale_quantize(A32: np.ndarray):
    """Per-row scales s_r = max_c |A_rc| / 448 (1 for a zero row), computed in
    FP32 as stored, and the E4M3 values of A_rc / s_r (the division in FP32).
    Returns (Qvalues FP64, s FP32) with A ~ diag(s) Q."""
    A32 = np.asarray(A32, dtype=np.float32)
    mx = np.max(np.abs(A32), axis=1)
    s = np.where(mx > 0, mx / np.float32(E4M3_MAX), np.float32(1.0)).astype(np.float32)
    ratio = (A32 / s[:, None]).astype(np.float32)
    return e4m3_round(ratio.astype(np.float64)), s


def fp8_normal_matvec(Q: np.ndarray, s: np.ndarray, D: np.ndarray, delta: float, v: np.ndarray) -> np.ndarray:
    """The FP8 operator diag(s) Q (D .* (Q^T (s .* v))) + delta v in FP64."""
    s = np.asarray(s, dtype=np.float64)
    t = D * (Q.T @ (s * v))
    return s * (Q @ t) + delta * v


# ---------------------------------------------------------------------------
# Randomized Nystrom approximation (Algorithm 1) and preconditioner
# (Algorithm 2, Eq. Nys_precond_inv).
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class NystromFactor:
    U: np.ndarray       # m x ell, orthonormal columns
    lam: np.ndarray     # ell, descending, >= 0
    nu: float           # the shift of Algorithm 1


def nystrom_from_sketch(Y: np.ndarray, Omega: np.ndarray) -> NystromFactor:
    """Algorithm 1, steps 3-8, given the sketch Y = N Omega."""
    nu = eps_of(float(np.linalg.norm(Y, "fro")))          # step 3
    Ynu = Y + nu * Omega                                  # step 4
    G = Omega.T @ Ynu
    G = 0.5 * (G + G.T)                                   # READING: symmetrise before chol
    C = np.linalg.cholesky(G).T                           # step 5: upper C, G = C^T C
    B = sla.solve_triangular(C, Ynu.T, trans="T", lower=False).T   # step 6: B = Ynu C^{-1}
    Uh, S, _ = np.linalg.svd(B, full_matrices=False)      # step 7: thin SVD
    lam = np.maximum(0.0, S * S - nu)                     # step 8
    return NystromFactor(U=Uh, lam=lam, nu=nu)


def nystrom(A: np.ndarray, D: np.ndarray, Omega: np.ndarray) -> NystromFactor:
    """Algorithm 1 for N = A D A^T with a given Gaussian test matrix."""
    return nystrom_from_sketch(sketch(A, D, Omega), Omega)


def precond_inv_apply(F: NystromFactor, delta: float, r: np.ndarray) -> np.ndarray:
    """P_Nys^{-1} r (Eq. Nys_precond_inv):
    (lam_ell + delta) U (Lam + delta I)^{-1} U^T r + (I - U U^T) r.
    READING: lam_ell is the last diagonal entry of the clipped, descending Lambda."""
    lam_ell = F.lam[-1]
    Utr = F.U.T @ r
    return (lam_ell + delta) * (F.U @ (Utr / (F.lam + delta))) + r - F.U @ Utr


def precond_apply(F: NystromFactor, delta: float, v: np.ndarray) -> np.ndarray:
    """P_Nys v (Eq. Nys_precond): U (Lam + delta I) U^T v / (lam_ell + delta) + (I - U U^T) v."""
    lam_ell = F.lam[-1]
    Utv = F.U.T @ v
    return (F.U @ ((F.lam + delta) * Utv)) / (lam_ell + delta) + v - F.U @ Utv


# ---------------------------------------------------------------------------
# Preconditioned CG on (N + delta I) dy = xi (Section 2.2).
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    res_norm: float       # recursive residual norm at exit
    converged: bool


def pcg(apply_M, apply_Pinv, rhs: np.ndarray, eta: float, maxit: int,
        forced_iters: int | None = None) -> PCGResult:
    """Textbook preconditioned CG from x0 = 0 (Golub & Van Loan, Alg. 11.5.1).

    READING: stop at the top of an iteration once the recursive residual
    satisfies ||r||_2 <= eta ||rhs||_2; `forced_iters` instead runs exactly that
    many iterations (used to align iteration counts with another solver)."""
    x = np.zeros_like(rhs)
    r = rhs.copy()
    bnorm = float(np.linalg.norm(rhs))
    if bnorm == 0.0:
        return PCGResult(x=x, iters=0, res_norm=0.0, converged=True)
    zv = apply_Pinv(r)
    p = zv.copy()
    rz = float(r @ zv)
    it = 0
    limit = forced_iters if forced_iters is not None else maxit
    while it < limit:
        if forced_iters is None and float(np.linalg.norm(r)) <= eta * bnorm:
            break
        w = apply_M(p)
        alpha = rz / float(p @ w)
        x = x + alpha * p
        r = r - alpha * w
        zv = apply_Pinv(r)
        rz_new = float(r @ zv)
        beta = rz_new / rz
        p = zv + beta * p
        rz = rz_new
        it += 1
    rn = float(np.linalg.norm(r))
    return PCGResult(x=x, iters=it, res_norm=rn, converged=rn <= eta * bnorm)


def pcg_tolerance(mu: float) -> float:
    """READING (the theory only asks for a residual of order mu_k, Prop. 3.2):
    eta_k = max(1e-10, min(1e-2, 0.1 mu_k)), relative to ||xi||."""
    return max(1e-10, min(1e-2, 0.1 * mu))


# ---------------------------------------------------------------------------
# Newton direction through the normal equations (Algorithm 4 with I = all).
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Direction:
    dx: np.ndarray
    dy: np.ndarray
    dz: np.ndarray
    pcg_iters: int
    pcg_res: float
    dw: np.ndarray | None = None      # box-constrained variables only
    ds: np.ndarray | None = None


def newton_direction(A, x, z, D, delta, r_d, r_p, r_xz, F, eta, maxit,
                     forced_iters=None, kind=None, w=None, s=None, r_u=None,
                     r_ws=None) -> Direction:
    """Algorithm 4.  For I = {1..n} (kind None):
    xi_au = -X^{-1} r_xz;  xi = r_p + A D (r_d + xi_au);
    (A D A^T + delta I) dy = xi by Nystrom PCG;
    dx = D (A^T dy - r_d - xi_au);
    dz = X^{-1} (r_xz - Z dx).
    With free (F) and box-constrained (J) variables, `kind` marks each index
    and w, s, r_u, r_ws are the slack, its dual and their right-hand sides
    (zero outside J):
    xi_au = 0 on F, -r_xz / x on I, -r_xz / x + r_ws / w - s r_u / w on J;
    dw = r_u - dx on J (0 elsewhere); dz = X^{-1}(r_xz - Z dx) on I and J
    (0 on F); ds = W^{-1}(r_ws - S dw) on J (0 elsewhere).
    READING: Algorithm 4 prints dz = X^{-1} r_xz - Z dx (and ds = W^{-1} r_ws
    - S dw); the corresponding block rows of Eq. Newton / Eq. Newton-free-box
    give X^{-1}(r_xz - Z dx) and W^{-1}(r_ws - S dw), which are used."""
    if kind is None:
        xi_au = -r_xz / x
    else:
        xi_au = np.zeros_like(x)
        ij = kind != KIND_F
        jj = kind == KIND_J
        xi_au[ij] = -r_xz[ij] / x[ij]
        xi_au[jj] += r_ws[jj] / w[jj] - s[jj] * r_u[jj] / w[jj]
    xi = r_p + A @ (D * (r_d + xi_au))
    res = pcg(lambda v: normal_matvec(A, D, delta, v),
              lambda v: precond_inv_apply(F, delta, v),
              xi, eta, maxit, forced_iters)
    dy = res.x
    dx = D * (A.T @ dy - r_d - xi_au)
    if kind is None:
        dz = (r_xz - z * dx) / x
        return Direction(dx=dx, dy=dy, dz=dz, pcg_iters=res.iters, pcg_res=res.res_norm)
    dz = np.zeros_like(x)
    dz[ij] = (r_xz[ij] - z[ij] * dx[ij]) / x[ij]
    dw = np.zeros_like(x)
    dw[jj] = r_u[jj] - dx[jj]
    ds = np.zeros_like(x)
    ds[jj] = (r_ws[jj] - s[jj] * dw[jj]) / w[jj]
    return Direction(dx=dx, dy=dy, dz=dz, pcg_iters=res.iters, pcg_res=res.res_norm, dw=dw, ds=ds)


def step_length(v: np.ndarray, dv: np.ndarray) -> float:
    """Fraction-to-boundary step (Eq. stepsize-p / stepsize-d):
    0.995 min{1, min over dv_i < 0 of -v_i / dv_i}."""
    neg = dv < 0.0
    a = 1.0
    if np.any(neg):
        a = min(1.0, float(np.min(-v[neg] / dv[neg])))
    return 0.995 * a


def step_lengths(x, dx, z, dz, kind=None, w=None, dw=None, s=None, ds=None):
    """(alpha_p, alpha_d) of Eq. stepsize-p / stepsize-d.  alpha_p covers x on
    I and J (free x_F are unbounded) and the slack w on J; alpha_d covers z on
    I and J and s on J.  For I = {1..n} these are the steps of x and z."""
    if kind is None:
        return step_length(x, dx), step_length(z, dz)
    ij, jj = kind != KIND_F, kind == KIND_J
    ap = step_length(np.concatenate([x[ij], w[jj]]), np.concatenate([dx[ij], dw[jj]]))
    ad = step_length(np.concatenate([z[ij], s[jj]]), np.concatenate([dz[ij], ds[jj]]))
    return ap, ad


def duality_measure(x, z, kind=None, w=None, s=None) -> float:
    """mu = (x_IJ^T z_IJ + w_J^T s_J) / (|IJ| + |J|) (Algorithm 5, fourth step);
    x^T z / n for I = {1..n}.  With no bounded variable at all (every x_j
    free) there is no complementarity and mu = 0."""
    if kind is None:
        return float(x @ z) / x.shape[0]
    ij, jj = kind != KIND_F, kind == KIND_J
    count = int(ij.sum()) + int(jj.sum())
    if count == 0:
        return 0.0
    return (float(x[ij] @ z[ij]) + float(w[jj] @ s[jj])) / count


# ---------------------------------------------------------------------------
# Nys-IP-PMM driver (Algorithm 6 with Algorithm 5).
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Options:
    tol: float = 1e-6
    ell: int = 20
    max_ipm_iter: int = 200
    max_pcg_iter: int = 1000
    seed: int = 0
    rho0: float = 8.0            # Algorithm 6, second step
    delta0: float = 8.0
    reg_floor: float = 5e-10     # floor seen in Tables 7-8
    forced_pcg: list | None = None   # per Newton solve: predictor, corrector, ...
    forced_ipm: int | None = None
    reuse_pcg: int = 0           # > 0: keep the Nystrom factor while PCG stays at or under this many iterations
    adapt_cost: int = 0          # > 0: adaptive sketch size (sketch_size_next); the cost of a factor at
                                 #   the largest size, in PCG iterations
    ell_min: int = 0             # smallest adaptive sketch size (0: max(1, ell // 8))


@dataclasses.dataclass
class IterRecord:
    k: int
    mu: float
    rel_p: float
    rel_d: float
    rho: float
    delta: float
    nu: float
    lam_max: float
    lam_min: float
    alpha_p: float
    alpha_d: float
    pcg_pred: int
    pcg_corr: int
    state: tuple | None = None
    reused: bool = False         # the Nystrom factor of the previous iteration was kept
    ref: tuple | None = None     # (ref_p, ref_d) of the PEU at the top of this iteration (record=True)
    ell: int = 0                 # sketch size of this iteration's factor


@dataclasses.dataclass
class Result:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    status: str               # "converged" | "max_iter"
    ipm_iters: int
    pcg_iters: list           # per Newton solve, in order
    rel_p: float
    rel_d: float
    mu: float
    rel_gap: float
    rho: float
    delta: float
    trace: list
    w: np.ndarray | None = None     # slack u - x and its dual (box-constrained
    s: np.ndarray | None = None     #   variables; zero outside J)
    lam: np.ndarray | None = None   # PMM estimates and PEU references after the last update
    zeta: np.ndarray | None = None
    ref_p: float = float("nan")
    ref_d: float = float("nan")


# ---------------------------------------------------------------------------
# Sketch size per IPM iteration (Algorithm 6, "choose sketch size l_k").
#
# The paper leaves the choice open and shows its trade-off (the rank-versus-
# time experiment of the SVM section): a larger sketch makes the factor
# dearer and the PCG solves cheaper, and the total time has a U-shape in l.
# READING (builder's rule): with a factor costing about c(l) = cost * l /
# l_max PCG iterations and PCG work that falls roughly like 1/l, the total is
# smallest where the two are equal, so after iteration k, with P_k PCG
# iterations in its two solves, the next sketch doubles when P_k > 2 c(l_k)
# and halves when P_k < c(l_k) / 2, within [l_min, l_max]; l_0 = l_min.
# Integer comparisons only, so both implementations take the same decision.
# Omega_k of size l_k is the first l_k columns of the l_max-wide Omega_k (the
# test matrices of different iterations stay disjoint draws).
# ---------------------------------------------------------------------------

def sketch_size_bounds(ell_max: int, ell_min: int) -> int:
    """The smallest adaptive sketch size: ell_min when given, else l_max / 8."""
    lo = ell_min if ell_min > 0 else ell_max // 8
    return max(1, min(lo, ell_max))


def sketch_size_next(ell: int, pcg_total: int, ell_min: int, ell_max: int, cost: int) -> int:
    """The next sketch size from this iteration's PCG count (see above)."""
    if pcg_total * ell_max > 2 * cost * ell and ell < ell_max:
        return min(ell_max, 2 * ell)
    if 2 * pcg_total * ell_max < cost * ell and ell > ell_min:
        return max(ell_min, (ell + 1) // 2)
    return ell


# ---------------------------------------------------------------------------
# PMM parameter update (Algorithm 6, last step).
#
# The paper takes this step from Pougkakiotis-Gondzio's PEU without restating
# it; what it does fix is the outcome: rho_0 = delta_0 = 8, the two parameters
# move independently of each other, and neither goes below 5e-10 (the traces
# of Tables 7-8).  Between two consecutive rows of those tables each
# parameter shrinks by one of two factors, 1 - r or 1 - (2/3) r, with r the
# same for both (tests/golden/peu_tables.txt checks every row pair).
# READING, in the spirit of the method of multipliers: the multiplier
# estimate lambda and its penalty delta belong to the primal constraint
# Ax = b, the proximal centre zeta and its weight rho to the dual one.  An
# estimate is re-centred on the new iterate (lambda <- y, zeta <- x) when its
# infeasibility made enough progress, and then its parameter takes the larger
# cut (1 - r); otherwise the estimate stays and the parameter takes the
# smaller cut (1 - (2/3) r).  r = |mu_{k+1} - mu_k| / max(mu_k, mu_{k+1}).
# ---------------------------------------------------------------------------

PEU_PROGRESS = 0.95      # READING: an infeasibility made progress when it fell to 95% of its reference
PEU_SLOW_CUT = 2.0 / 3.0  # Tables 7-8: the other parameter shrinks by 1 - (2/3) r


@dataclasses.dataclass
class PMM:
    """PMM subproblem parameters lambda^k, zeta^k, rho_k, delta_k with the
    relative primal / dual infeasibility recorded at the last re-centring of
    lambda / zeta (ref_p / ref_d)."""
    lam: np.ndarray
    zeta: np.ndarray
    rho: float
    delta: float
    ref_p: float
    ref_d: float


def peu_progress(rel_new: float, ref: float, tol: float) -> bool:
    """READING: progress means the relative infeasibility fell to
    PEU_PROGRESS times its reference or meets the termination tolerance.  An
    estimate whose reference already met the tolerance (a feasible start,
    where it is zero) always counts as progressing: without that clause it
    could not be re-centred before the solve ends."""
    return ref <= tol or rel_new <= max(PEU_PROGRESS * ref, tol)


def peu_update(pmm: PMM, x: np.ndarray, y: np.ndarray, mu_old: float, mu_new: float,
               rel_p: float, rel_d: float, tol: float, floor: float) -> PMM:
    """One PMM parameter update (see the block comment above): rel_p, rel_d
    are the relative infeasibilities (kkt_measures) of the new iterate x, y."""
    den = max(mu_old, mu_new)
    r = abs(mu_new - mu_old) / den if den > 0.0 else 0.0
    if peu_progress(rel_p, pmm.ref_p, tol):
        lam, ref_p, delta = y.copy(), rel_p, (1.0 - r) * pmm.delta
    else:
        lam, ref_p, delta = pmm.lam, pmm.ref_p, (1.0 - PEU_SLOW_CUT * r) * pmm.delta
    if peu_progress(rel_d, pmm.ref_d, tol):
        zeta, ref_d, rho = x.copy(), rel_d, (1.0 - r) * pmm.rho
    else:
        zeta, ref_d, rho = pmm.zeta, pmm.ref_d, (1.0 - PEU_SLOW_CUT * r) * pmm.rho
    return PMM(lam=lam, zeta=zeta, rho=max(floor, rho), delta=max(floor, delta),
               ref_p=ref_p, ref_d=ref_d)


def kkt_measures(A, b, c, q, x, y, z, kind=None, u=None, w=None, s=None):
    """READING of the termination test (Algorithm 3 tests absolute norms; the
    experiments speak of relative infeasibilities): relative primal and dual
    infeasibility and the duality measure mu = x^T z / n.
    With free and box-constrained variables the primal residual stacks
    Ax - b with the slack equation x_J + w_J - u_J (third block row of the
    system behind Eq. Newton-free-box), relative to 1 + ||(b, u_J)||; the dual
    residual is c + Qx - A^T y - z + s (dual constraint of (D~)); mu is
    duality_measure()."""
    if kind is None:
        rel_p = float(np.linalg.norm(A @ x - b)) / (1.0 + float(np.linalg.norm(b)))
        rel_d = float(np.linalg.norm(c + q * x - A.T @ y - z)) / (1.0 + float(np.linalg.norm(c)))
        mu = float(x @ z) / x.shape[0]
        return rel_p, rel_d, mu
    jj = kind == KIND_J
    rp = np.concatenate([A @ x - b, x[jj] + w[jj] - u[jj]])
    rel_p = float(np.linalg.norm(rp)) / (1.0 + float(np.linalg.norm(np.concatenate([b, u[jj]]))))
    rel_d = float(np.linalg.norm(c + q * x - A.T @ y - z + s)) / (1.0 + float(np.linalg.norm(c)))
    return rel_p, rel_d, duality_measure(x, z, kind, w, s)


def duality_gap(b, c, q, x, y, kind=None, u=None, s=None):
    """|pobj - dobj| / (1 + |pobj|) with the objectives of (P) and (D), or of
    (P~) and (D~), whose dual objective also subtracts u^T s."""
    pobj = 0.5 * float(x @ (q * x)) + float(c @ x)
    dobj = float(b @ y) - 0.5 * float(x @ (q * x))
    if kind is not None:
        jj = kind == KIND_J
        dobj -= float(u[jj] @ s[jj])
    return abs(pobj - dobj) / (1.0 + abs(pobj))


def solve(A, b, c, q, x0, y0, z0, opt: Options, lam0=None, zeta0=None, k0: int = 0,
          record: bool = False, kind=None, u=None, s0=None, w0=None,
          ref_p0: float | None = None, ref_d0: float | None = None) -> Result:
    """Nys-IP-PMM from a given strictly interior start (Algorithm 6).

    READING (start): the workloads supply a strictly feasible interior point
    (x0, y0, z0); it is used as (x^0, y^0, z^0), with lambda^0 = y^0,
    zeta^0 = x^0, rho_0 = delta_0 = 8 (Algorithm 6, second step).
    Warm start (resume): lam0, zeta0 replace lambda^0, zeta^0, opt.rho0 and
    opt.delta0 carry the PMM parameters, and k0 is the index of the first IPM
    iteration (it selects Omega_k).  With record=True every trace entry also
    holds the state (x, y, z, lambda, zeta) at the top of its iteration
    (followed by w, s for problems with box-constrained variables) and
    `ref` the pair (ref_p, ref_d) in force there.
    The PMM parameters follow peu_update() after every iteration.  A resumed
    solve also takes ref_p0, ref_d0: the relative infeasibilities at the last
    re-centring of lambda and zeta (default: those of the start point).

    Free and box-constrained variables (problems (P~)/(D~)): `kind` holds
    KIND_I, KIND_F or KIND_J per variable, u the upper bounds (read on J
    only), s0 the start of the bound multipliers s (read on J only, > 0) and
    w0 the start of the slack w (default u - x0 on J).  z0 is ignored on F
    (z_F = 0).  The iteration follows Algorithm 5 with the predictor
    right-hand sides of Eq. predictor-RHS and the corrector right-hand sides
    of Eq. corrector-RHS; w moves with the primal step, s with the dual one."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    x, y, z = x0.astype(np.float64).copy(), y0.astype(np.float64).copy(), z0.astype(np.float64).copy()
    w = s = None
    box = kind is not None
    if box:
        kind = np.asarray(kind, dtype=np.int8)
        ij, jj = kind != KIND_F, kind == KIND_J
        u = np.where(jj, np.asarray(u, dtype=np.float64), 0.0)       # u_{I u F} = 0
        z[~ij] = 0.0                                                 # z_F = 0
        w = np.where(jj, (u - x) if w0 is None else np.asarray(w0, dtype=np.float64), 0.0)
        s = np.where(jj, np.asarray(s0, dtype=np.float64), 0.0)
    lam_pmm = y.copy() if lam0 is None else np.asarray(lam0, dtype=np.float64).copy()
    zeta = x.copy() if zeta0 is None else np.asarray(zeta0, dtype=np.float64).copy()
    rho, delta = opt.rho0, opt.delta0
    rel_p0, rel_d0, _ = kkt_measures(A, b, c, q, x, y, z, kind, u, w, s)
    pmm = PMM(lam=lam_pmm, zeta=zeta, rho=rho, delta=delta,
              ref_p=rel_p0 if ref_p0 is None else float(ref_p0),
              ref_d=rel_d0 if ref_d0 is None else float(ref_d0))
    ell_max = min(opt.ell, m)
    adaptive = opt.adapt_cost > 0
    if adaptive and opt.reuse_pcg > 0:
        raise ValueError("adaptive sketch size and preconditioner reuse are exclusive")
    ell_lo = sketch_size_bounds(ell_max, opt.ell_min)
    ell = ell_lo if adaptive else ell_max
    trace, pcg_counts = [], []
    status = "max_iter"
    forced = list(opt.forced_pcg) if opt.forced_pcg is not None else None
    k = 0
    rel_p = rel_d = mu = float("nan")
    while True:
        rel_p, rel_d, mu = kkt_measures(A, b, c, q, x, y, z, kind, u, w, s)
        if opt.forced_ipm is not None:
            if k >= opt.forced_ipm:
                status = "converged" if (rel_p <= opt.tol and rel_d <= opt.tol and mu <= opt.tol) else "forced"
                break
        elif rel_p <= opt.tol and rel_d <= opt.tol and mu <= opt.tol:
            status = "converged"
            break
        if k >= opt.max_ipm_iter:
            break
        lam_pmm, zeta, rho, delta = pmm.lam, pmm.zeta, pmm.rho, pmm.delta
        state_lam, state_zeta, state_ref = lam_pmm.copy(), zeta.copy(), (pmm.ref_p, pmm.ref_d)
        x_top, y_top, z_top = x.copy(), y.copy(), z.copy()
        w_top, s_top = (w.copy(), s.copy()) if box else (None, None)
        D = scaling_D(x, z, q, rho, kind, w, s)
        # READING (preconditioner reuse, which the paper only suggests): with
        # opt.reuse_pcg = R > 0 the factor of the previous iteration is kept
        # when both of its PCG solves took at most R iterations; otherwise (and
        # always with R = 0, Algorithm 6 as written) N_k is sketched afresh.
        reuse = (opt.reuse_pcg > 0 and k > 0 and pcg_counts[-2] <= opt.reuse_pcg
                 and pcg_counts[-1] <= opt.reuse_pcg)
        if adaptive and k > 0:
            ell = sketch_size_next(ell, pcg_counts[-2] + pcg_counts[-1], ell_lo, ell_max, opt.adapt_cost)
        if not reuse:
            Omega = gaussian_omega(opt.seed, k0 + k, m, ell_max)[:, :ell]
            F = nystrom(A, D, Omega)
        eta = pcg_tolerance(mu)
        # Predictor (Algorithm 5, first step; Eq. predictor-RHS).
        Ax, Aty = A @ x, A.T @ y
        r_p = b - Ax - delta * (y - lam_pmm)
        if box:
            r_d = c + q * x - Aty - z + s + rho * (x - zeta)
            r_u = np.where(jj, u - x - w, 0.0)
            r_xz = np.where(ij, -x * z, 0.0)
            r_ws = np.where(jj, -w * s, 0.0)
        else:
            r_d = c + q * x - Aty - z + rho * (x - zeta)
            r_u = r_ws = None
            r_xz = -x * z
        fp = forced.pop(0) if forced else None
        pred = newton_direction(A, x, z, D, delta, r_d, r_p, r_xz, F, eta, opt.max_pcg_iter, fp,
                                kind, w, s, r_u, r_ws)
        ap_bar, ad_bar = step_lengths(x, pred.dx, z, pred.dz, kind, w, pred.dw, s, pred.ds)
        if box:                                                               # Eq. mu-aff
            mu_aff = duality_measure(x + ap_bar * pred.dx, z + ad_bar * pred.dz, kind,
                                     w + ap_bar * pred.dw, s + ad_bar * pred.ds)
        else:
            mu_aff = float((x + ap_bar * pred.dx) @ (z + ad_bar * pred.dz)) / n
        mu_tilde = mu_aff ** 3 / mu ** 2 if mu > 0.0 else 0.0
        # Corrector (Eq. corrector-RHS).
        zero_n, zero_m = np.zeros(n), np.zeros(m)
        if box:
            r_xz_c = np.where(ij, mu_tilde - pred.dx * pred.dz, 0.0)
            r_ws_c = np.where(jj, mu_tilde - pred.dw * pred.ds, 0.0)
        else:
            r_xz_c = mu_tilde - pred.dx * pred.dz
            r_ws_c = None
        fc = forced.pop(0) if forced else None
        corr = newton_direction(A, x, z, D, delta, zero_n, zero_m, r_xz_c, F, eta, opt.max_pcg_iter, fc,
                                kind, w, s, zero_n if box else None, r_ws_c)
        dx, dy, dz = pred.dx + corr.dx, pred.dy + corr.dy, pred.dz + corr.dz
        dw = ds = None
        if box:
            dw, ds = pred.dw + corr.dw, pred.ds + corr.ds
        alpha_p, alpha_d = step_lengths(x, dx, z, dz, kind, w, dw, s, ds)
        x = x + alpha_p * dx
        y = y + alpha_d * dy
        z = z + alpha_d * dz
        if box:
            w = w + alpha_p * dw
            s = s + alpha_d * ds
        mu_new = duality_measure(x, z, kind, w, s)
        pcg_counts += [pred.pcg_iters, corr.pcg_iters]
        rec = IterRecord(k=k0 + k, mu=mu, rel_p=rel_p, rel_d=rel_d, rho=rho, delta=delta, nu=F.nu,
                         lam_max=float(F.lam[0]), lam_min=float(F.lam[-1]),
                         alpha_p=alpha_p, alpha_d=alpha_d,
                         pcg_pred=pred.pcg_iters, pcg_corr=corr.pcg_iters, reused=reuse, ell=ell)
        if record:
            rec.state = (x_top, y_top, z_top, state_lam, state_zeta)
            if box:
                rec.state += (w_top, s_top)
            rec.ref = state_ref
        trace.append(rec)
        # Algorithm 6, last step: PMM parameters of the next subproblem.
        rel_p_new, rel_d_new, _ = kkt_measures(A, b, c, q, x, y, z, kind, u, w, s)
        pmm = peu_update(pmm, x, y, mu, mu_new, rel_p_new, rel_d_new, opt.tol, opt.reg_floor)
        mu = mu_new
        k += 1
    return Result(x=x, y=y, z=z, status=status, ipm_iters=k, pcg_iters=pcg_counts,
                  rel_p=rel_p, rel_d=rel_d, mu=mu, rel_gap=duality_gap(b, c, q, x, y, kind, u, s),
                  rho=pmm.rho, delta=pmm.delta, trace=trace, w=w, s=s,
                  lam=pmm.lam, zeta=pmm.zeta, ref_p=pmm.ref_p, ref_d=pmm.ref_d)


# ---------------------------------------------------------------------------
# Practical initial point (the supplement's construction for the initial point,
# after Mehrotra and Pougkakiotis-Gondzio).
# ---------------------------------------------------------------------------

START_DELTA = 10.0       # regularisation of A A^T in both candidate solves (supplement)
START_PCG_TOL = 1e-10    # READING: relative residual of those two Nystrom PCG solves


@dataclasses.dataclass
class StartPoint:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    w: np.ndarray        # zero outside J
    s: np.ndarray        # zero outside J
    pcg_iters: tuple     # iterations of the two candidate solves


def practical_start(A, b, c, q, opt: Options, kind=None, u=None, k: int = 0) -> StartPoint:
    """Initial point of the supplement for (P~)/(D~) (problem (P) when kind is None).

    Candidate: x~ = u/2 + A^T (A A^T)^{-1} (b - A u/2), y~ = (A A^T)^{-1} A (c + Q x~),
    with A A^T regularised as A A^T + 10 I and both systems solved by Nystrom
    PCG (Algorithm 1 on N = A A^T, i.e. D = I, with Omega_k; Algorithm 2 with
    delta = 10); g = c - A^T y~ + Q x~; z~ = g/2 on J and g elsewhere;
    s~_J = -z~_J; w~_J = u_J - x~_J.  Shifts: delta_p = max(-1.5 min over
    x~_IJ and w~_J, 0), delta_d likewise over z~_IJ and s~_J;
    gamma = (x~_IJ + delta_p)^T (z~_IJ + delta_d) + (w~_J + delta_p)^T (s~_J + delta_d);
    delta_p~ = delta_p + gamma / 2 / (sum_IJ (z~ + delta_d) + sum_J (s~ + delta_d));
    delta_d~ = delta_d + gamma / 2 / (sum_IJ (x~ + delta_p) + sum_J (w~ + delta_p)).
    Start: x_IJ, w_J shifted by delta_p~ (x_F unshifted), z_IJ, s_J by
    delta_d~, z_F = 0, y = y~.
    READING: the supplement prints x~ + delta_d in the denominator of
    delta_d~; the primal sums shifted by delta_p (the primal shift, as in
    Mehrotra's heuristic) are used.  READING: Omega_k is the test matrix of
    the first IPM iteration's index, and both PCG solves stop at the relative
    residual START_PCG_TOL (or max_pcg_iter).  A shift whose denominator is 0
    (no bounded variable) is 0."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    kind = np.zeros(n, dtype=np.int8) if kind is None else np.asarray(kind, dtype=np.int8)
    ij, jj = kind != KIND_F, kind == KIND_J
    uu = np.zeros(n) if u is None else np.where(jj, np.asarray(u, dtype=np.float64), 0.0)
    ones = np.ones(n)
    F = nystrom(A, ones, gaussian_omega(opt.seed, k, m, min(opt.ell, m)))
    apply_M = lambda v: normal_matvec(A, ones, START_DELTA, v)
    apply_P = lambda v: precond_inv_apply(F, START_DELTA, v)
    r1 = pcg(apply_M, apply_P, b - A @ (0.5 * uu), START_PCG_TOL, opt.max_pcg_iter)
    xt = 0.5 * uu + A.T @ r1.x
    r2 = pcg(apply_M, apply_P, A @ (c + q * xt), START_PCG_TOL, opt.max_pcg_iter)
    yt = r2.x
    g = c - A.T @ yt + q * xt
    zt = np.where(jj, 0.5 * g, g)
    st = np.where(jj, -zt, 0.0)
    wt = np.where(jj, uu - xt, 0.0)
    prim = np.concatenate([xt[ij], wt[jj]])
    dual = np.concatenate([zt[ij], st[jj]])
    dp = max(-1.5 * float(np.min(prim)), 0.0) if prim.size else 0.0
    dd = max(-1.5 * float(np.min(dual)), 0.0) if dual.size else 0.0
    gamma = float((xt[ij] + dp) @ (zt[ij] + dd)) + float((wt[jj] + dp) @ (st[jj] + dd))
    den_p = float(np.sum(zt[ij] + dd)) + float(np.sum(st[jj] + dd))
    den_d = float(np.sum(xt[ij] + dp)) + float(np.sum(wt[jj] + dp))
    dpt = dp + (0.5 * gamma / den_p if den_p != 0.0 else 0.0)
    ddt = dd + (0.5 * gamma / den_d if den_d != 0.0 else 0.0)
    return StartPoint(x=np.where(ij, xt + dpt, xt), y=yt, z=np.where(ij, zt + ddt, 0.0),
                      w=np.where(jj, wt + dpt, 0.0), s=np.where(jj, st + ddt, 0.0),
                      pcg_iters=(r1.iters, r2.iters))


def solve_from_practical_start(A, b, c, q, opt: Options, kind=None, u=None, k0: int = 0, **kw) -> Result:
    """Algorithm 6 started at practical_start() (Omega_{k0} for its sketch)."""
    st = practical_start(A, b, c, q, opt, kind, u, k0)
    if kind is None:
        return solve(A, b, c, q, st.x, st.y, st.z, opt, k0=k0, **kw)
    return solve(A, b, c, q, st.x, st.y, st.z, opt, k0=k0, kind=kind, u=u, s0=st.s, w0=st.w, **kw)


def solve_qp(qp, opt: Options, **kw) -> Result:
    """Convenience wrapper over a workload record with fields A, b, c, q, x0, y0, z0
    (and kind, u, s0 when the record has box-constrained or free variables)."""
    if getattr(qp, "kind", None) is not None:
        kw.setdefault("kind", qp.kind)
        kw.setdefault("u", qp.u)
        kw.setdefault("s0", qp.s0)
    return solve(qp.A, qp.b, qp.c, qp.q, qp.x0, qp.y0, qp.z0, opt, **kw)


# ---------------------------------------------------------------------------
# Differentiation through the solution (transposed KKT system).
#
# At the final iterate the regularised Newton matrix of Eq. Newton,
#   J = [[Q + rho I, -A^T, -I], [A, delta I, 0], [Z, 0, X]],
# is the Jacobian of the (perturbed) optimality conditions of (P)/(D) with
# respect to (x, y, z).  For a loss L(x*) with g = dL/dx*, the implicit
# function theorem gives dL/dtheta = -lam^T dF/dtheta with J^T lam = (g, 0, 0).
# READING: the adjoint uses the final rho, delta and (x, z) of the solve.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Gradients:
    c: np.ndarray
    b: np.ndarray
    q: np.ndarray
    A: np.ndarray


def kkt_adjoint(A, x, y, z, q, rho, delta, g) -> Gradients:
    """Dense transposed-KKT solve (LU) for the gradients of L(x*):
    dL/dc = -lam1, dL/db = lam2, dL/dq = -lam1 .* x, dL/dA = y lam1^T - lam2 x^T."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    J = np.block([
        [np.diag(q + rho), -A.T, -np.eye(n)],
        [A, delta * np.eye(m), np.zeros((m, n))],
        [np.diag(z), np.zeros((n, m)), np.diag(x)],
    ])
    lam = np.linalg.solve(J.T, np.concatenate([g, np.zeros(m), np.zeros(n)]))
    l1, l2 = lam[:n], lam[n:n + m]
    return Gradients(c=-l1, b=l2, q=-l1 * x, A=np.outer(y, l1) - np.outer(l2, x))
