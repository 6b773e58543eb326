"""The allocation-free operator entry point (for callers that cannot allocate
device memory, e.g. inside a stream capture or under a fixed memory pool)
gives the same (N + delta I) v as the handle-based nys_normal_matvec, on two
calls in a row through the C ABI.  Collected last on purpose."""
import numpy as np
import pytest
import torch

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


def test_noalloc_rejects_sizes_beyond_the_scratch(nys):
    dev = torch.device("cuda", 0)
    m, n = 2, (1 << 20) + 8
    A = torch.zeros(m, n, dtype=torch.float64, device=dev)
    D = torch.ones(n, dtype=torch.float64, device=dev)
    v = torch.ones(m, dtype=torch.float64, device=dev)
    out = torch.empty(m, dtype=torch.float64, device=dev)
    assert nys.nys_normal_matvec_noalloc(A, D, 0.0, v, out) == nys.NYS_ERR_NOMEM
