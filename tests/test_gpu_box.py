"""Parity of the CUDA path with the CPU oracle on problems with free and
box-constrained variables, (P~)/(D~): Algorithm 4 with w and s, the
right-hand sides of Eq. predictor-RHS / corrector-RHS and the step lengths of
Eq. stepsize-p / stepsize-d, through nys_solve's var_kind, u, w0, s0 fields.

Tolerances follow the all-non-negative parity tests: one IPM step resumed
from the oracle's state at 1e-9 relative (or 100x the oracle's own response
to a 2e-16 perturbation of Omega_k), whole solves with the oracle's PCG and
IPM counts at 1e-5, KKT measures at the solve's tolerance."""
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


def K8(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int8)).to(DEV)


def relerr(got, want):
    got = got.detach().cpu().numpy() if isinstance(got, torch.Tensor) else got
    d = np.linalg.norm(want)
    return np.linalg.norm(got - want) / (d if d > 0 else 1.0)


def _np(*ts):
    return [t.cpu().numpy() for t in ts]


def _solve(nys, h, qp, x0=None, y0=None, z0=None, s0=None, w0=None, **kw):
    x0 = qp.x0 if x0 is None else x0
    y0 = qp.y0 if y0 is None else y0
    z0 = qp.z0 if z0 is None else z0
    s0 = qp.s0 if s0 is None else s0
    return nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), T(x0), T(y0), T(z0), kind=K8(qp.kind),
                         u=T(qp.u), s0=T(s0), w0=None if w0 is None else T(w0), **kw)


@pytest.fixture(scope="module")
def box_run():
    qp = synth.workload_box()
    ref = O.solve_qp(qp, O.Options(tol=1e-6, ell=20, seed=7), record=True)
    return qp, ref


def _omega_sensitivity(qp, opt, state, k, ref):
    """Relative move of one oracle IPM step under a 2e-16 relative perturbation
    of Omega_k (the rounding-level noise floor of that step)."""
    orig = O.gaussian_omega

    def pert(seed, kk, m, ell):
        om = orig(seed, kk, m, ell)
        return om * (1 + 2e-16 * np.sign(np.sin(np.arange(om.size))).reshape(om.shape))
    x, y, z, lam, zeta, w, s = state
    kw = dict(lam0=lam, zeta0=zeta, k0=k, kind=qp.kind, u=qp.u, s0=s, w0=w, ref_p0=ref[0], ref_d0=ref[1])
    a = O.solve(qp.A, qp.b, qp.c, qp.q, x, y, z, opt, **kw)
    O.gaussian_omega = pert
    try:
        b = O.solve(qp.A, qp.b, qp.c, qp.q, x, y, z, opt, **kw)
    finally:
        O.gaussian_omega = orig
    return max(relerr(u, v) for u, v in ((a.x, b.x), (a.y, b.y), (a.z, b.z), (a.w, b.w), (a.s, b.s)))


@pytest.mark.parametrize("k", [0, 1, 2, 6, 12, 20, -3, -2, -1])
def test_box_single_ipm_step_matches_oracle(nys, box_run, k):
    """One IPM iteration on (P~) resumed on the GPU from the oracle's state k
    (x, y, z, w, s, lambda, zeta, rho, delta), with the oracle's PCG counts:
    the next x, y, z, w, s agree to 1e-9 relative, or to 100x the oracle's
    own rounding response where that floor is higher."""
    qp, ref = box_run
    k = k % len(ref.trace)
    t = ref.trace[k]
    x, y, z, lam, zeta, w, s = t.state
    forced = [t.pcg_pred, t.pcg_corr]
    opt = O.Options(tol=1e-6, ell=20, seed=7, rho0=t.rho, delta0=t.delta, forced_ipm=1, forced_pcg=forced)
    nxt = ref.trace[k + 1] if k + 1 < len(ref.trace) else None
    want = (nxt.state[0], nxt.state[1], nxt.state[2], nxt.state[5], nxt.state[6]) if nxt is not None \
        else (ref.x, ref.y, ref.z, ref.w, ref.s)
    floor = _omega_sensitivity(qp, opt, t.state, k, t.ref)
    tol = max(1e-9, 100 * floor)
    h = nys.Handle(qp.m, qp.n, ell=20, tol=1e-6, seed=7, forced_pcg=forced, forced_ipm=1,
                   rho0=t.rho, delta0=t.delta)
    gx, gy, gz, info = _solve(nys, h, qp, x, y, z, s0=s, w0=w, lam0=T(lam), zeta0=T(zeta), k0=k,
                              peu_ref=t.ref, want_pmm=True)
    errs = [relerr(g, v) for g, v in zip((gx, gy, gz, info["w"], info["s"]), want)]
    print(f"k={k} errs={errs} floor={floor:.2e}")
    assert max(errs) <= tol
    if nxt is not None:
        for got, old, new in ((info["rho"], t.rho, nxt.rho), (info["delta"], t.delta, nxt.delta)):
            tol_reg = 2 * tol / (new / old)
            assert abs(got - new) <= tol_reg * new
        # the references are residual norms of the new iterate (differences of
        # O(1) terms): they carry the iterate's error in absolute terms
        assert (info["peu_ref_p"], info["peu_ref_d"]) == pytest.approx(nxt.ref, rel=2 * tol, abs=10 * tol)
        assert relerr(info["lam"], nxt.state[3]) <= tol and relerr(info["zeta"], nxt.state[4]) <= tol


def test_box_whole_solve_matches_oracle(nys, box_run):
    """The 200 x 500 workload with 10% free and 30% box variables, with the
    oracle's PCG and IPM counts: same KKT quality, iterates agree far below
    the 1e-6 tolerance, the invariants z_F = 0 and w = s = 0 outside J hold
    exactly, and w = u - x on J to rounding."""
    qp, ref = box_run
    h = nys.Handle(qp.m, qp.n, ell=20, tol=1e-6, seed=7, forced_pcg=ref.pcg_iters, forced_ipm=ref.ipm_iters)
    x, y, z, info = _solve(nys, h, qp)
    assert info["ipm_iters"] == ref.ipm_iters and info["pcg_log"] == ref.pcg_iters
    w, s = info["w"], info["s"]
    for g, v in ((x, ref.x), (y, ref.y), (z, ref.z), (w, ref.w), (s, ref.s)):
        assert relerr(g, v) <= 1e-5
    assert info["rel_primal"] <= 1e-6 and info["rel_dual"] <= 1e-6 and info["mu"] <= 1e-6
    xn, yn, zn, wn, sn = _np(x, y, z, w, s)
    rp, rd, mu = O.kkt_measures(qp.A, qp.b, qp.c, qp.q, xn, yn, zn, qp.kind, qp.u, wn, sn)
    assert rp <= 1e-6 and rd <= 1e-6 and mu <= 1e-6
    assert abs(info["rel_primal"] - rp) <= 1e-9 and abs(info["mu"] - mu) <= 1e-12
    ff, jj = qp.kind == O.KIND_F, qp.kind == O.KIND_J
    assert np.all(zn[ff] == 0) and np.all(wn[~jj] == 0) and np.all(sn[~jj] == 0)
    assert np.abs(wn[jj] - (qp.u[jj] - xn[jj])).max() <= 1e-12 * np.abs(qp.u).max()
    assert abs(info["rel_gap"] - ref.rel_gap) <= 1e-6


def test_box_free_running_solve_meets_kkt(nys):
    """Without forced counts, tol 1e-8, another seed and mix (20% free, 40%
    box): the (P~) KKT measures of the GPU's answer are within tolerance and
    the solution matches the oracle's to the tolerance level."""
    qp = synth.box_qp(2024, 150, 600, 0.2, 0.4)
    ref = O.solve_qp(qp, O.Options(tol=1e-8, ell=20, seed=3))
    assert ref.status == "converged"
    h = nys.Handle(qp.m, qp.n, ell=20, tol=1e-8, seed=3)
    x, y, z, info = _solve(nys, h, qp)
    assert info["status"] == 0
    rp, rd, mu = O.kkt_measures(qp.A, qp.b, qp.c, qp.q, *_np(x, y, z), qp.kind, qp.u, *_np(info["w"], info["s"]))
    assert rp <= 1e-8 and rd <= 1e-8 and mu <= 1e-8
    assert relerr(x, ref.x) <= 1e-5


def test_all_non_negative_kinds_take_the_plain_iteration_bit_for_bit(nys):
    """Every kind 0 (x >= 0) through the (P~) kernels: they add exact zeros only,
    so the iterates equal the plain (P) solve's bit for bit."""
    qp = synth.workload_small(seed=12)
    n = qp.n
    h = nys.Handle(qp.m, n, ell=20, tol=1e-6, seed=2)
    args = [T(v) for v in (qp.A, qp.b, qp.c, qp.q, qp.x0, qp.y0, qp.z0)]
    x1, y1, z1, i1 = nys.nys_solve(h, *args)
    x2, y2, z2, i2 = nys.nys_solve(h, *args, kind=K8(np.zeros(n)), u=T(np.zeros(n)), s0=T(np.zeros(n)))
    assert torch.equal(x1, x2) and torch.equal(y1, y2) and torch.equal(z1, z2)
    assert i1["pcg_log"] == i2["pcg_log"] and i1["rel_gap"] == i2["rel_gap"]
    assert torch.count_nonzero(i2["w"]) == 0 and torch.count_nonzero(i2["s"]) == 0


def test_box_host_buffers_give_identical_results(nys):
    qp = synth.box_qp(31, 120, 400)
    h = nys.Handle(qp.m, qp.n, ell=16, tol=1e-6, seed=1)
    dev = _solve(nys, h, qp)
    cpu = lambda a, dt=np.float64: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory()
    host = nys.nys_solve(h, cpu(qp.A), cpu(qp.b), cpu(qp.c), cpu(qp.q), cpu(qp.x0), cpu(qp.y0), cpu(qp.z0),
                         kind=cpu(qp.kind, np.int8), u=cpu(qp.u), s0=cpu(qp.s0))
    for a, b in zip(dev[:3], host[:3]):
        assert torch.equal(a.cpu(), b)
    assert torch.equal(dev[3]["w"].cpu(), host[3]["w"]) and torch.equal(dev[3]["s"].cpu(), host[3]["s"])


def _read_golden():
    import os
    recs = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "kkt_points_box.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p = [t.strip() for t in line.split("|")]
            vec = lambda t: np.array([float(v) for v in t.split()])
            kind = np.array([{"I": 0, "F": 1, "J": 2}[t] for t in p[1].split()], dtype=np.int8)
            A = np.array([[float(v) for v in row.split()] for row in p[3].split(";")])
            recs.append((p[0], kind, vec(p[2]), A, vec(p[4]), vec(p[5]), vec(p[6]), vec(p[7]), vec(p[8]),
                         vec(p[9]), vec(p[10])))
    return recs


@pytest.mark.parametrize("rec", _read_golden(), ids=lambda r: r[0])
def test_box_hand_derived_kkt_points(nys, rec):
    name, kind, u, A, b, c, q, xs, ys, zs, ss = rec
    m, n = A.shape
    x0 = np.where(kind == 2, 0.5 * u, np.where(kind == 1, 0.0, 1.0))
    s0 = np.where(kind == 2, 1.0, 0.0)
    h = nys.Handle(m, n, ell=m, tol=1e-10, seed=3, max_pcg_iter=200)
    x, y, z, info = nys.nys_solve(h, T(A), T(b), T(c), T(q), T(x0), T(np.zeros(m)), T(np.ones(n)),
                                  kind=K8(kind), u=T(u), s0=T(s0))
    assert info["status"] == 0, (name, info)
    assert np.allclose(x.cpu().numpy(), xs, atol=1e-7)
    assert np.allclose(y.cpu().numpy(), ys, atol=1e-6)
    assert np.allclose(z.cpu().numpy(), zs, atol=1e-6)
    assert np.allclose(info["s"].cpu().numpy(), ss, atol=1e-6)


def test_box_invalid_entries_are_rejected(nys):
    """Invalid kinds and J entries are counted on the device before the first
    iteration and reported as NYS_ERR_ARG (no device fault, no partial solve)."""
    qp = synth.box_qp(5, 40, 100)
    h = nys.Handle(qp.m, qp.n, ell=8)
    bad_kind = qp.kind.copy()
    bad_kind[3] = 3
    bad_w = np.where(qp.kind == 2, qp.u - qp.x0, 0.0)
    bad_w[np.flatnonzero(qp.kind == 2)[0]] = -1.0
    bad_s = qp.s0.copy()
    bad_s[np.flatnonzero(qp.kind == 2)[1]] = 0.0
    args = [T(v) for v in (qp.A, qp.b, qp.c, qp.q, qp.x0, qp.y0, qp.z0)]
    cases = [dict(kind=K8(bad_kind), u=T(qp.u), s0=T(qp.s0)),
             dict(kind=K8(qp.kind), u=T(qp.u), s0=T(qp.s0), w0=T(bad_w)),
             dict(kind=K8(qp.kind), u=T(qp.u), s0=T(bad_s)),
             dict(kind=K8(qp.kind), s0=T(qp.s0))]                       # u missing with J entries
    for kw in cases:
        with pytest.raises(nys.NysError) as e:
            nys.nys_solve(h, *args, **kw)
        assert e.value.code == nys.NYS_ERR_ARG
    # the handle stays usable
    x, y, z, info = nys.nys_solve(h, *args, kind=K8(qp.kind), u=T(qp.u), s0=T(qp.s0))
    assert info["status"] == 0


def test_box_batch_equals_plain_solves(nys):
    """A batch mixing (P~) and (P) problems of uneven sizes: each result equals
    the plain nys_solve of the same problem bit for bit."""
    qps = [synth.box_qp(60 + i, m, 4 * m, 0.1, 0.3) for i, m in enumerate((64, 150, 90))] + \
        synth.workload_batch(seed=8, count=2, m_lo=64, m_hi=120)
    mx, nx = max(q.m for q in qps), max(q.n for q in qps)
    hb = nys.Handle(mx, nx, ell=16, tol=1e-6, seed=4, max_batch=3)
    hs = nys.Handle(mx, nx, ell=16, tol=1e-6, seed=4)
    probs = []
    for q in qps:
        pr = tuple(T(v) for v in (q.A, q.b, q.c, q.q, q.x0, q.y0, q.z0))
        if q.kind is not None:
            pr = pr + (0, dict(kind=K8(q.kind), u=T(q.u), s0=T(q.s0)))
        probs.append(pr)
    res = nys.nys_solve_batched(hb, probs)
    for q, pr, (x, y, z, info) in zip(qps, probs, res):
        assert info["status"] == 0
        if q.kind is not None:
            xs, ys, zs, i2 = nys.nys_solve(hs, *pr[:7], kind=pr[8]["kind"], u=pr[8]["u"], s0=pr[8]["s0"])
            assert torch.equal(info["w"], i2["w"]) and torch.equal(info["s"], i2["s"])
            rp, rd, mu = O.kkt_measures(q.A, q.b, q.c, q.q, *_np(x, y, z), q.kind, q.u, *_np(info["w"], info["s"]))
        else:
            xs, ys, zs, i2 = nys.nys_solve(hs, *pr)
            rp, rd, mu = O.kkt_measures(q.A, q.b, q.c, q.q, *_np(x, y, z))
        assert torch.equal(x, xs) and torch.equal(y, ys) and torch.equal(z, zs)
        assert rp <= 1e-6 and rd <= 1e-6 and mu <= 1e-6


def test_box_precision_form_meets_kkt(nys):
    """The precision form (BF16 inner PCG, float-float refinement) on a (P~)
    problem whose FP32 matrix defines it: KKT <= 1e-6 on that problem and the
    solution agrees with the FP64 oracle's to the tolerance level."""
    qp = synth.box_qp(77, 500, 2500, 0.1, 0.3, "exp200")
    A32 = qp.A.astype(np.float32)
    A64 = A32.astype(np.float64)
    b = A64 @ qp.x0
    c = A64.T @ qp.y0 + qp.z0 - qp.s0 - qp.q * qp.x0
    ref = O.solve(A64, b, c, qp.q, qp.x0, qp.y0, qp.z0, O.Options(tol=1e-6, ell=30, seed=5),
                  kind=qp.kind, u=qp.u, s0=qp.s0)
    assert ref.status == "converged"
    h = nys.Handle(qp.m, qp.n, ell=30, tol=1e-6, seed=5, precision_mode=1)
    x, y, z, info = nys.nys_solve(h, torch.from_numpy(A32).to(DEV), T(b), T(c), T(qp.q), T(qp.x0), T(qp.y0),
                                  T(qp.z0), kind=K8(qp.kind), u=T(qp.u), s0=T(qp.s0))
    assert info["status"] in (0, 2)
    rp, rd, mu = O.kkt_measures(A64, b, c, qp.q, *_np(x, y, z), qp.kind, qp.u, *_np(info["w"], info["s"]))
    assert rp <= 1e-6 and rd <= 1e-6 and mu <= 1e-6
    assert relerr(x, ref.x) <= 1e-3


# ------------------------------------------------------------ practical start

@pytest.mark.parametrize("which", ["plain", "box"])
def test_practical_start_matches_oracle(nys, which):
    """start_mode=1 with zero IPM iterations returns the practical initial
    point: it matches the oracle's to the level of its two PCG solves
    (relative residual 1e-10)."""
    qp = synth.workload_small() if which == "plain" else synth.workload_box()
    opt = O.Options(tol=1e-6, ell=20, seed=7)
    st = O.practical_start(qp.A, qp.b, qp.c, qp.q, opt, qp.kind, qp.u)
    h = nys.Handle(qp.m, qp.n, ell=20, tol=1e-6, seed=7, forced_ipm=0, start_mode=1)
    box = dict(kind=K8(qp.kind), u=T(qp.u)) if qp.kind is not None else {}
    x, y, z, info = nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), None, None, None, **box)
    got = [x, y, z] + ([info["w"], info["s"]] if box else [])
    want = [st.x, st.y, st.z] + ([st.w, st.s] if box else [])
    errs = [relerr(g, v) for g, v in zip(got, want)]
    print(which, errs)
    assert max(errs) <= 1e-8
    assert info["pcg_iters_total"] == 0 and info["ipm_iters"] == 0


@pytest.mark.parametrize("which", ["plain", "box"])
def test_solve_from_practical_start_matches_oracle(nys, which):
    """A whole solve from the practical start with the oracle's PCG and IPM
    counts: KKT within tolerance and the iterates agree with the oracle's far
    below it."""
    qp = synth.workload_small() if which == "plain" else synth.workload_box()
    opt = O.Options(tol=1e-6, ell=20, seed=7)
    ref = O.solve_from_practical_start(qp.A, qp.b, qp.c, qp.q, opt, qp.kind, qp.u)
    assert ref.status == "converged"
    h = nys.Handle(qp.m, qp.n, ell=20, tol=1e-6, seed=7, forced_pcg=ref.pcg_iters, forced_ipm=ref.ipm_iters,
                   start_mode=1)
    box = dict(kind=K8(qp.kind), u=T(qp.u)) if qp.kind is not None else {}
    x, y, z, info = nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), None, None, None, **box)
    assert info["ipm_iters"] == ref.ipm_iters and info["pcg_log"] == ref.pcg_iters
    for g, v in ((x, ref.x), (y, ref.y), (z, ref.z)):
        assert relerr(g, v) <= 1e-5
    assert info["rel_primal"] <= 1e-6 and info["rel_dual"] <= 1e-6 and info["mu"] <= 1e-6


def test_practical_start_in_the_precision_form(nys):
    """start_mode=1 with the precision form (float-float FP32 operator for the
    two start solves): converges to KKT <= 1e-6 on the FP32 problem."""
    qp = synth.box_qp(78, 400, 2000, 0.1, 0.3, "exp200")
    A32 = qp.A.astype(np.float32)
    A64 = A32.astype(np.float64)
    b = A64 @ qp.x0
    c = A64.T @ qp.y0 + qp.z0 - qp.s0 - qp.q * qp.x0
    h = nys.Handle(qp.m, qp.n, ell=30, tol=1e-6, seed=5, precision_mode=1, start_mode=1)
    x, y, z, info = nys.nys_solve(h, torch.from_numpy(A32).to(DEV), T(b), T(c), T(qp.q), None, None, None,
                                  kind=K8(qp.kind), u=T(qp.u))
    assert info["status"] in (0, 2)
    rp, rd, mu = O.kkt_measures(A64, b, c, qp.q, *_np(x, y, z), qp.kind, qp.u, *_np(info["w"], info["s"]))
    assert rp <= 1e-6 and rd <= 1e-6 and mu <= 1e-6


# ------------------------------------------------ SVM- and portfolio-shaped problems

@pytest.mark.parametrize("which", ["svm", "portfolio"])
def test_svm_and_portfolio_problems_match_oracle(nys, which):
    """The supplement's two (P~) formulations on small synthetic instances
    (dual SVM: free v, box-constrained p; factor-model portfolio: free factor
    exposures, non-negative weights and slacks), solved from the practical
    start with the oracle's PCG and IPM counts: iterates agree to 1e-6 (the
    oracle's own response to a 2e-16 change of Omega is 1e-11 / 3e-10 here)
    and the KKT measures meet the tolerance."""
    if which == "svm":
        qp, tol, ell = synth.svm_qp(5, 20, 800), 1e-6, 10
    else:
        qp, tol, ell = synth.portfolio_qp(6, 400, 250, 10), 1e-8, 20
    opt = O.Options(tol=tol, ell=ell, seed=3)
    ref = O.solve_from_practical_start(qp.A, qp.b, qp.c, qp.q, opt, qp.kind, qp.u)
    assert ref.status == "converged"
    h = nys.Handle(qp.m, qp.n, ell=ell, tol=tol, seed=3, forced_pcg=ref.pcg_iters, forced_ipm=ref.ipm_iters,
                   start_mode=1)
    x, y, z, info = nys.nys_solve(h, T(qp.A), T(qp.b), T(qp.c), T(qp.q), None, None, None, kind=K8(qp.kind),
                                  u=T(qp.u))
    assert info["ipm_iters"] == ref.ipm_iters and info["pcg_log"] == ref.pcg_iters
    for g, v in ((x, ref.x), (y, ref.y), (z, ref.z), (info["w"], ref.w), (info["s"], ref.s)):
        assert relerr(g, v) <= 1e-6
    rp, rd, mu = O.kkt_measures(qp.A, qp.b, qp.c, qp.q, *_np(x, y, z), qp.kind, qp.u, *_np(info["w"], info["s"]))
    assert rp <= tol and rd <= tol and mu <= tol


# ------------------------------------------------------- preconditioner reuse

@pytest.mark.parametrize("which", ["plain", "box"])
def test_preconditioner_reuse_matches_oracle(nys, which):
    """reuse_pcg = 40: the GPU keeps the factor in the same iterations as the
    oracle (its decisions follow the PCG counts, here forced to the oracle's)
    and reaches the same iterates."""
    qp = synth.workload_small() if which == "plain" else synth.workload_box()
    opt = O.Options(tol=1e-6, ell=20, seed=7, reuse_pcg=40)
    ref = O.solve_qp(qp, opt)
    n_sketch = sum(1 for t in ref.trace if not t.reused)
    assert n_sketch < ref.ipm_iters
    h = nys.Handle(qp.m, qp.n, ell=20, tol=1e-6, seed=7, forced_pcg=ref.pcg_iters, forced_ipm=ref.ipm_iters,
                   reuse_pcg=40)
    if which == "plain":
        x, y, z, info = nys.nys_solve(h, *(T(v) for v in (qp.A, qp.b, qp.c, qp.q, qp.x0, qp.y0, qp.z0)))
    else:
        x, y, z, info = _solve(nys, h, qp)
    assert info["sketches"] == n_sketch and info["pcg_log"] == ref.pcg_iters
    for g, v in ((x, ref.x), (y, ref.y), (z, ref.z)):
        assert relerr(g, v) <= 1e-5
    assert info["rel_primal"] <= 1e-6 and info["rel_dual"] <= 1e-6 and info["mu"] <= 1e-6
