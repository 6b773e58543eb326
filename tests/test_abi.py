"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/nys.h (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2404_14524_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "nys.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nys_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_the_solver_api():
    names = _declared()
    for n in ("nys_create", "nys_solve", "nys_destroy", "nys_last_error", "nys_normal_matvec",
              "nys_sketch", "nys_nystrom", "nys_pcg", "nys_precond_apply", "nys_step_length"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_2404_14524_gb300 import nys
    assert sorted(nys.exported_symbols()) == _declared()
    nys.lib()


def test_struct_layouts_match_the_header(libpath):
    """Sizes of the ctypes mirrors equal the C structs (compiled probe)."""
    import subprocess
    import tempfile
    from paper_2404_14524_gb300 import nys
    src = ('#include "nys.h"\n#include <stdio.h>\n#include <stddef.h>\n'
           'int main(){printf("%zu %zu %zu\\n", sizeof(nys_options), sizeof(nys_problem), sizeof(nys_result));return 0;}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "p")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == [ctypes.sizeof(nys.Options), ctypes.sizeof(nys.Problem),
                                     ctypes.sizeof(nys.Result)]


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2404_14524_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "from oracle" not in txt and "import oracle" not in txt, f


def test_box_fields_are_checked_before_the_library_is_called():
    """The binding rejects kinds that are not a contiguous int8 vector of
    length n and float64 bounds of the wrong placement, without touching
    libnys.so (marshalling only)."""
    import torch
    from paper_2404_14524_gb300 import nys
    cpu = torch.device("cpu")
    n = 5
    kind = torch.tensor([0, 1, 2, 0, 2], dtype=torch.int8)
    u = torch.ones(n, dtype=torch.float64)
    f, keep = nys._box_fields(kind, u, u, None, n, cpu, True)
    assert set(f) == {"var_kind", "u", "s0"} and len(keep) == 3
    assert nys._box_fields(None, None, None, None, n, cpu, True) == ({}, [])
    with pytest.raises(TypeError):
        nys._box_fields(kind.to(torch.int32), u, u, None, n, cpu, True)
    with pytest.raises(TypeError):
        nys._box_fields(kind[:4], u, u, None, n, cpu, True)
    with pytest.raises(TypeError):
        nys._box_fields(kind, u.float(), u, None, n, cpu, True)


def test_one_call_solve_sizes_a_handle_and_releases_it(monkeypatch):
    """nys.solve: a handle of A's size, the practical start when no x0 is given,
    nys_solve with the same tensors, and the handle closed afterwards (the
    library itself is replaced by fakes: marshalling only)."""
    import torch
    from paper_2404_14524_gb300 import nys
    made, calls = [], []

    class FakeHandle:
        def __init__(self, m, n, **kw):
            self.m, self.n, self.kw, self.closed = m, n, kw, False
            made.append(self)

        def close(self):
            self.closed = True

    def fake_solve(h, A, b, c, q, x0, y0, z0, **kw):
        calls.append((h, x0, kw))
        return "x", "y", "z", {"status": 0}

    monkeypatch.setattr(nys, "Handle", FakeHandle)
    monkeypatch.setattr(nys, "nys_solve", fake_solve)
    A = torch.zeros(3, 7, dtype=torch.float64)
    v = torch.zeros(7, dtype=torch.float64)
    out = nys.solve(A, torch.zeros(3, dtype=torch.float64), v, v, ell=2, tol=1e-8, reuse_pcg=5)
    assert out[3]["status"] == 0
    h = made[0]
    assert (h.m, h.n) == (3, 7) and h.closed
    assert h.kw == {"ell": 2, "tol": 1e-8, "reuse_pcg": 5, "start_mode": 1}
    assert calls[0][1] is None and calls[0][2]["kind"] is None
    nys.solve(A, torch.zeros(3, dtype=torch.float64), v, v, x0=v, y0=torch.zeros(3, dtype=torch.float64), z0=v)
    assert "start_mode" not in made[1].kw and made[1].closed


def test_plain_c_program_links_and_gets_argument_errors(libpath):
    """A C program built against include/nys.h and linked with libnys.so:
    defaults as documented, invalid arguments rejected with NYS_ERR_ARG before
    any device work, and nys_create either succeeds (a GPU is present: the
    handle is destroyed again) or reports NYS_ERR_CUDA (no GPU) -- never a crash."""
    import subprocess
    import tempfile
    src = r'''
#include "nys.h"
#include <stdio.h>
int main(void) {
  nys_options o;
  nys_default_options(&o);
  printf("%g %d %d %d %g %g %d %d %d %d %d\n", o.tol, o.ell, o.max_ipm_iter, o.max_pcg_iter, o.rho0, o.reg_floor,
         o.forced_ipm_iters, o.start_mode, o.reuse_pcg, o.adapt_cost, o.ell_min);
  nys_handle h = 0;
  printf("%d %d %d\n", nys_create(0, &o, 10, 20, 0, 0), nys_create(&h, &o, 0, 20, 0, 0),
         nys_create(&h, 0, 10, 20, 0, 0));
  o.precision_mode = 3;
  printf("%d\n", nys_create(&h, &o, 10, 20, 0, 0));
  o.precision_mode = 0;
  int rc = nys_create(&h, &o, 10, 20, 0, 0);
  printf("%d\n", rc);
  if (rc == NYS_OK) {
    nys_problem p = {0};
    nys_result r = {0};
    printf("%d\n", nys_solve(h, &p, &r));    /* m = n = 0: rejected */
    nys_destroy(h);
  } else {
    printf("%d\n", NYS_ERR_ARG);
  }
  return 0;
}
'''
    libdir = os.path.dirname(libpath)
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(B.nvcc())), "lib64")
    env = dict(os.environ, LD_LIBRARY_PATH=os.pathsep.join([libdir, cuda_lib, os.environ.get("LD_LIBRARY_PATH", "")]))
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe, "-L", libdir, "-lnys",
                        "-Wl,-rpath," + libdir], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True, env=env, timeout=120).stdout
    lines = out.split("\n")
    assert lines[0].split() == ["1e-06", "20", "200", "1000", "8", "5e-10", "-1", "0", "0", "0", "0"]
    assert lines[1].split() == ["-1", "-1", "-1"]
    assert lines[2] == "-1"
    assert lines[3] in ("0", "-2")
    assert lines[4] == "-1"
