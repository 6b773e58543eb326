"""The adaptive sketch size of the oracle (Algorithm 6, "choose sketch size
l_k").  The rule is a reading (the paper shows the rank/time trade-off but no
rule), so its constants are "parity unpinned"; these tests pin what it must
do: the decision table, the bounds, Omega_k of size l_k being the first l_k
columns of the l_max-wide Omega_k, a fixed size when it is off, and a solve
that still reaches the KKT point with every step following the rule."""
import numpy as np
import pytest

import oracle.nys_oracle as O
from paper_2404_14524_gb300 import synth as S


def test_bounds():
    assert O.sketch_size_bounds(20, 0) == 2
    assert O.sketch_size_bounds(7, 0) == 1
    assert O.sketch_size_bounds(400, 0) == 50
    assert O.sketch_size_bounds(20, 5) == 5
    assert O.sketch_size_bounds(20, 50) == 20


@pytest.mark.parametrize("ell,pcg,want", [
    (4, 17, 8),      # 17 * 20 = 340 > 2 * 40 * 4 = 320: grow
    (4, 16, 4),      # 320 is not > 320: keep
    (16, 70, 20),    # 70 * 20 = 1400 > 1280: grows to l_max, not beyond
    (20, 200, 20),   # at l_max already
    (16, 7, 8),      # 2 * 7 * 20 = 280 < 40 * 16 = 640: shrink
    (16, 16, 16),    # 640 is not < 640: keep
    (3, 0, 2),       # shrinks to ceil(3 / 2) = 2 = l_min
    (2, 0, 2),       # at l_min already
])
def test_decision_table(ell, pcg, want):
    assert O.sketch_size_next(ell, pcg, 2, 20, 40) == want


def test_omega_of_a_smaller_sketch_is_a_column_prefix():
    full = O.gaussian_omega(9, 3, 50, 16)
    part = O.gaussian_omega(9, 3, 50, 16)[:, :5]
    assert np.array_equal(full[:, :5], part)
    # and Omega_k of consecutive iterations are disjoint draws of the stream
    nxt = O.gaussian_omega(9, 4, 50, 16)
    assert not np.any(np.isin(full, nxt))


def test_off_means_a_fixed_sketch_size():
    qp = S.workload_small()
    r = O.solve_qp(qp, O.Options(ell=20, tol=1e-6))
    assert all(e.ell == 20 for e in r.trace)


@pytest.mark.parametrize("cost", [10, 40, 160])
def test_adaptive_solve_follows_the_rule_and_meets_kkt(cost):
    qp = S.workload_small()
    r = O.solve_qp(qp, O.Options(ell=20, tol=1e-6, adapt_cost=cost))
    assert r.status == "converged"
    rp, rd, mu = O.kkt_measures(qp.A, qp.b, qp.c, qp.q, r.x, r.y, r.z)
    assert max(rp, rd, mu) <= 1e-6
    tr = r.trace
    assert tr[0].ell == O.sketch_size_bounds(20, 0)
    for a, b in zip(tr, tr[1:]):
        assert b.ell == O.sketch_size_next(a.ell, a.pcg_pred + a.pcg_corr, 2, 20, cost)
    # the same KKT point as the fixed-size solve, to the tolerance
    f = O.solve_qp(qp, O.Options(ell=20, tol=1e-6))
    assert np.linalg.norm(r.x - f.x) / np.linalg.norm(f.x) <= 1e-3


def test_adaptive_with_reuse_is_rejected():
    qp = S.workload_small()
    with pytest.raises(ValueError):
        O.solve_qp(qp, O.Options(ell=20, adapt_cost=40, reuse_pcg=10))
