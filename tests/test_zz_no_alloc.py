"""The allocation-free operator entry point (for callers that cannot allocate
device memory, e.g. inside a stream capture or under a fixed memory pool)
gives the same (N + delta I) v as the handle-based nys_normal_matvec and as
the CPU oracle's operator, on two calls in a row through the C ABI, including
the largest n the fixed scratch holds (where no room is left for split
partial sums).  Collected last on purpose."""
import numpy as np
import pytest
import torch

from oracle import nys_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nys():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_14524_gb300 import build
    build.build()
    from paper_2404_14524_gb300 import nys as N
    N.lib()
    return N


def test_noalloc_operator_matches_the_handle_operator_twice(nys):
    dev = torch.device("cuda", 0)
    g = torch.Generator(device="cpu").manual_seed(3)
    m, n = 1500, 7001
    A = torch.randn(m, n, generator=g, dtype=torch.float64).to(dev)
    h = nys.Handle(m, n, ell=1)
    out = torch.empty(m, dtype=torch.float64, device=dev)
    for call in range(2):                       # the shared scratch keeps the previous call's data
        D = (torch.rand(n, generator=g, dtype=torch.float64) + 0.1).to(dev)
        v = torch.randn(m, generator=g, dtype=torch.float64).to(dev)
        delta = 10.0 ** (-3 - call)
        rc = nys.nys_normal_matvec_noalloc(A, D, delta, v, out)
        assert rc == 0
        ref = nys.nys_normal_matvec(h, A, D, delta, v)
        torch.cuda.synchronize()
        err = float((out - ref).abs().max() / ref.abs().max())
        assert err <= 1e-13, (call, err)
        _check_against_oracle(A, D, delta, v, out)


def _check_against_oracle(A, D, delta, v, out):
    """Element by element against the oracle's FP64 operator, within the
    rounding bound of two length-(m + n) dot-product chains."""
    An, Dn, vn = (t.cpu().numpy() for t in (A, D, v))
    want = O.normal_matvec(An, Dn, delta, vn)
    m, n = An.shape
    bound = 4 * (m + n) * 2.0 ** -53 * (np.abs(An) @ (Dn * (np.abs(An).T @ np.abs(vn))) + abs(delta) * np.abs(vn))
    assert np.all(np.abs(out.cpu().numpy() - want) <= bound + 1e-300)


def test_noalloc_operator_at_the_largest_n_matches_the_oracle_twice(nys):
    """n = 2^20 fills the scratch with t alone: the entry point must fall back
    to the unsplit A^T v pass and still agree with the oracle."""
    dev = torch.device("cuda", 0)
    g = torch.Generator(device="cpu").manual_seed(11)
    m, n = 3, 1 << 20
    A = torch.randn(m, n, generator=g, dtype=torch.float64).to(dev)
    out = torch.empty(m, dtype=torch.float64, device=dev)
    for call in range(2):
        D = (torch.rand(n, generator=g, dtype=torch.float64) + 0.1).to(dev)
        v = torch.randn(m, generator=g, dtype=torch.float64).to(dev)
        assert nys.nys_normal_matvec_noalloc(A, D, 0.25 * (call + 1), v, out) == 0
        torch.cuda.synchronize()
        _check_against_oracle(A, D, 0.25 * (call + 1), v, out)


def test_noalloc_rejects_sizes_beyond_the_scratch(nys):
    dev = torch.device("cuda", 0)
    m, n = 2, (1 << 20) + 8
    A = torch.zeros(m, n, dtype=torch.float64, device=dev)
    D = torch.ones(n, dtype=torch.float64, device=dev)
    v = torch.ones(m, dtype=torch.float64, device=dev)
    out = torch.empty(m, dtype=torch.float64, device=dev)
    assert nys.nys_normal_matvec_noalloc(A, D, 0.0, v, out) == nys.NYS_ERR_NOMEM
