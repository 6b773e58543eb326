"""Pins of the oracle's PMM parameter update (Algorithm 6, last step).

The paper delegates the update of rho_k, delta_k, lambda^k, zeta^k to
Pougkakiotis-Gondzio's PEU, but prints its outcome on nine problems: the
supplement's Tables 7 and 8 (tests/golden/peu_tables.txt).  Those traces fix
(i) rho_0 = delta_0 = 8, (ii) the floor 5e-10, and (iii) that between two
rows each parameter shrinks by either 1 - r or 1 - (2/3) r with one r shared
by both -- the two parameters move independently.  These tests check the
oracle's peu_update against the tables with interval arithmetic on the
printed digits, and check that a plausible wrong constant does not fit.
"""
from __future__ import annotations

import math
import pathlib

import numpy as np
import pytest

import oracle.nys_oracle as O
from paper_2404_14524_gb300 import synth as S

GOLDEN = pathlib.Path(__file__).parent / "golden" / "peu_tables.txt"
FLOOR = 5e-10


def load_tables():
    blocks, cur = {}, None
    for ln in GOLDEN.read_text().splitlines():
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        if ln.startswith("["):
            cur = ln[1:-1]
            blocks[cur] = []
            continue
        k, r, d = ln.split()
        blocks[cur].append((int(k), r, d))
    return blocks


def printed_interval(tok: str):
    """The interval of reals that round to the printed 3-significant-digit token."""
    v = float(tok)
    mant, ex = tok.lower().split("e")
    half = 0.5 * 10.0 ** (int(ex) - (len(mant.split(".")[1]) if "." in mant else 0))
    return v - half, v + half


def factor_interval(a_tok, b_tok):
    """Interval of b / a for the printed values a -> b."""
    a0, a1 = printed_interval(a_tok)
    b0, b1 = printed_interval(b_tok)
    return b0 / a1, b1 / a0


def r_interval(f_iv, cut):
    """r with 1 - cut * r inside the factor interval f_iv."""
    return (1.0 - f_iv[1]) / cut, (1.0 - f_iv[0]) / cut


def transition_fits(rho_pair, delta_pair, slow_cut):
    """Is there one r in [0, 1] and one branch per parameter (cut 1 or slow_cut)
    that reproduces both printed factors?"""
    fr = factor_interval(*rho_pair)
    fd = factor_interval(*delta_pair)
    for cr in (1.0, slow_cut):
        for cd in (1.0, slow_cut):
            a = r_interval(fr, cr)
            b = r_interval(fd, cd)
            lo, hi = max(a[0], b[0], 0.0), min(a[1], b[1], 1.0)
            if lo <= hi:
                return True
    return False


def unclamped_transitions(blocks):
    for name, rows in blocks.items():
        for (k, r0, d0), (k1, r1, d1) in zip(rows, rows[1:]):
            if float(r1) <= FLOOR or float(d1) <= FLOOR:
                continue
            yield name, k, (r0, r1), (d0, d1)


def test_tables_start_at_eight_and_respect_the_floor():
    blocks = load_tables()
    assert len(blocks) == 9
    for name, rows in blocks.items():
        assert rows[0][0] == 0 and float(rows[0][1]) == 8.0 and float(rows[0][2]) == 8.0, name
        for _, r, d in rows:
            assert float(r) >= FLOOR and float(d) >= FLOOR
        floored = False
        for _, r, d in rows:            # once a parameter is on the floor it stays there
            if float(r) == FLOOR and float(d) == FLOOR:
                floored = True
            elif floored:
                pytest.fail(f"{name}: a parameter left the floor")
    assert O.Options().rho0 == 8.0 and O.Options().delta0 == 8.0
    assert O.Options().reg_floor == FLOOR


def test_every_table_row_pair_fits_the_two_cut_rule():
    blocks = load_tables()
    trans = list(unclamped_transitions(blocks))
    assert len(trans) > 80
    bad = [t[:2] for t in trans if not transition_fits(t[2], t[3], O.PEU_SLOW_CUT)]
    assert not bad, bad


@pytest.mark.parametrize("wrong", [0.5, 1.0 / 3.0, 0.75, 0.6])
def test_a_wrong_slow_cut_does_not_fit_the_tables(wrong):
    blocks = load_tables()
    misses = [t[:2] for t in unclamped_transitions(blocks) if not transition_fits(t[2], t[3], wrong)]
    assert misses, f"slow cut {wrong} would also fit every row"


def test_tables_show_independent_parameters():
    """In at least one row pair per problem family the two factors differ
    beyond rounding: rho and delta are not one parameter."""
    blocks = load_tables()
    split = 0
    for name, k, rp, dp in unclamped_transitions(blocks):
        fr, fd = factor_interval(*rp), factor_interval(*dp)
        if fr[1] < fd[0] or fd[1] < fr[0]:
            split += 1
    assert split >= 10


def _pmm(rho=8.0, delta=8.0, ref_p=1.0, ref_d=1.0, m=3, n=4):
    return O.PMM(lam=np.zeros(m), zeta=np.zeros(n), rho=rho, delta=delta, ref_p=ref_p, ref_d=ref_d)


def test_peu_update_reproduces_a_split_row_of_the_tables():
    """CIFAR10 (Table 8), k = 0 -> 1: delta 8 -> 2.27 (the full cut gives r),
    rho then takes the slow cut: 8 (1 - (2/3) r) must print as 4.18."""
    r = 1.0 - 2.27 / 8.0
    mu_old, mu_new = 1.0, 1.0 - r                       # |mu_new - mu_old| / max = r
    x, y = np.arange(4.0), np.arange(3.0)
    out = O.peu_update(_pmm(ref_p=1.0, ref_d=1.0), x, y, mu_old, mu_new,
                       rel_p=0.5, rel_d=0.99, tol=1e-6, floor=FLOOR)
    assert out.delta == pytest.approx(2.27, rel=1e-12)
    assert f"{out.rho:.2e}" == "4.18e+00"
    # the primal estimate followed the iterate, the dual one stayed
    assert np.array_equal(out.lam, y) and out.ref_p == 0.5
    assert np.array_equal(out.zeta, np.zeros(4)) and out.ref_d == 1.0


def test_peu_update_branches_floor_and_feasible_start():
    x, y = np.ones(4), np.ones(3)
    # no progress on either side: both take the slow cut, nothing re-centres
    out = O.peu_update(_pmm(), x, y, 1.0, 0.4, rel_p=0.97, rel_d=0.96, tol=1e-6, floor=FLOOR)
    assert out.rho == pytest.approx(8.0 * (1.0 - 0.4)) and out.delta == pytest.approx(8.0 * (1.0 - 0.4))
    assert out.ref_p == 1.0 and out.ref_d == 1.0 and not out.lam.any() and not out.zeta.any()
    # exactly 95% counts as progress
    out = O.peu_update(_pmm(), x, y, 1.0, 0.4, rel_p=0.95, rel_d=0.2, tol=1e-6, floor=FLOOR)
    assert out.delta == pytest.approx(8.0 * 0.4) and out.rho == pytest.approx(8.0 * 0.4)
    # mu growing: r is taken relative to the larger of the two
    out = O.peu_update(_pmm(), x, y, 0.5, 2.0, rel_p=0.1, rel_d=2.0, tol=1e-6, floor=FLOOR)
    assert out.delta == pytest.approx(8.0 * 0.25) and out.rho == pytest.approx(8.0 * (1.0 - 0.5))
    # floor
    out = O.peu_update(_pmm(rho=1e-9, delta=1e-9), x, y, 1.0, 1e-3, rel_p=0.1, rel_d=0.1, tol=1e-6,
                       floor=FLOOR)
    assert out.rho == FLOOR and out.delta == FLOOR
    # a reference that already met the tolerance (feasible start) re-centres at once
    out = O.peu_update(_pmm(ref_p=0.0, ref_d=3e-7), x, y, 1.0, 0.5, rel_p=0.03, rel_d=0.8, tol=1e-6,
                       floor=FLOOR)
    assert out.delta == pytest.approx(4.0) and out.rho == pytest.approx(4.0)
    assert out.ref_p == 0.03 and out.ref_d == 0.8 and out.lam.all() and out.zeta.all()
    # reaching the tolerance is progress even from a reference just above it
    out = O.peu_update(_pmm(ref_p=1.02e-6), x, y, 1.0, 0.5, rel_p=1e-6, rel_d=2.0, tol=1e-6, floor=FLOOR)
    assert out.delta == pytest.approx(4.0) and out.rho == pytest.approx(8.0 * (1.0 - 0.5 * 2.0 / 3.0))


def _check_trace_follows_rule(res, mu_end):
    tr = res.trace
    mus = [e.mu for e in tr] + [mu_end]
    rhos = [e.rho for e in tr] + [res.rho]
    dels = [e.delta for e in tr] + [res.delta]
    for k in range(len(tr)):
        den = max(mus[k], mus[k + 1])
        r = abs(mus[k + 1] - mus[k]) / den
        for old, new in ((rhos[k], rhos[k + 1]), (dels[k], dels[k + 1])):
            cands = [max(FLOOR, (1.0 - r) * old), max(FLOOR, (1.0 - 2.0 / 3.0 * r) * old)]
            assert min(abs(new - c) for c in cands) <= 1e-12 * old, (k, old, new, cands)


def test_solve_trace_has_independent_rho_and_delta():
    """m=200, n=500 workload from its feasible start: rho_0 = delta_0 = 8, the
    two parameters part after the first updates, both stay >= 5e-10, and every
    update is one of the two cuts of the shared r."""
    qp = S.workload_small()
    res = O.solve_qp(qp, O.Options(ell=20, tol=1e-6))
    assert res.status == "converged"
    tr = res.trace
    assert tr[0].rho == 8.0 and tr[0].delta == 8.0
    assert any(abs(e.rho - e.delta) > 1e-3 * max(e.rho, e.delta) for e in tr)
    assert all(e.rho >= FLOOR and e.delta >= FLOOR for e in tr)
    _check_trace_follows_rule(res, res.mu)


def test_practical_start_trace_parts_at_once():
    """From the supplement's practical start (infeasible) the first update
    already treats the two infeasibilities differently, as in Tables 7-8."""
    qp = S.workload_small()
    res = O.solve_from_practical_start(qp.A, qp.b, qp.c, qp.q, O.Options(ell=20, tol=1e-6))
    assert res.status == "converged"
    assert res.trace[1].rho != res.trace[1].delta
    _check_trace_follows_rule(res, res.mu)


def test_resume_with_references_reproduces_the_solve():
    """A solve resumed from a recorded top-of-iteration state (x, y, z,
    lambda, zeta, rho, delta and the two PEU references) follows the
    uninterrupted trajectory."""
    qp = S.workload_small()
    opt = O.Options(ell=20, tol=1e-6)
    full = O.solve_qp(qp, opt, record=True)
    k = 6
    e = full.trace[k]
    x, y, z, lam, zeta = e.state
    o2 = O.Options(ell=20, tol=1e-6, rho0=e.rho, delta0=e.delta)
    part = O.solve(qp.A, qp.b, qp.c, qp.q, x, y, z, o2, lam0=lam, zeta0=zeta, k0=k,
                   ref_p0=e.ref[0], ref_d0=e.ref[1])
    assert part.ipm_iters == full.ipm_iters - k
    assert np.array_equal(part.x, full.x) and np.array_equal(part.y, full.y)
    assert part.rho == full.rho and part.delta == full.delta
