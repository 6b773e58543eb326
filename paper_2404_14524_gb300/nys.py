"""Thin ctypes binding of the C ABI in include/nys.h.

Argument marshalling only: every step runs in libnys.so's CUDA kernels.
Functions keep the C names (nys_create, nys_solve, ...).  Tensors are
torch tensors on the handle's CUDA device (float64, contiguous); tall
m x ell panels are passed as (ell, m) row-major tensors, i.e. column-major
m x ell with leading dimension m.  The binding raises NysError when the
library reports an error and fails loudly (ImportError) when libnys.so has
not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnys.so")

NYS_OK = 0
NYS_ERR_ARG = -1
NYS_ERR_CUDA = -2
NYS_ERR_NUMERIC = -3
NYS_ERR_CORE_BREAKDOWN = -4
NYS_ERR_TIMEOUT = -5
NYS_ERR_NOMEM = -6
NYS_WARN_MAXITER = 1
NYS_WARN_PCG_MAXITER = 2
NYS_F64, NYS_F32, NYS_BF16, NYS_FP8E4M3 = 0, 1, 2, 3

STATUS_NAMES = {0: "ok", -1: "bad argument", -2: "CUDA error", -3: "numeric error",
                -4: "core breakdown", -5: "device wait timed out", -6: "out of memory",
                1: "IPM max iterations", 2: "PCG max iterations"}


class NysError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)} ({code}): {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("ell", ctypes.c_int), ("max_ipm_iter", ctypes.c_int),
                ("max_pcg_iter", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("precision_mode", ctypes.c_int), ("rho0", ctypes.c_double),
                ("delta0", ctypes.c_double), ("reg_floor", ctypes.c_double),
                ("forced_pcg_iters", ctypes.POINTER(ctypes.c_int)), ("n_forced_pcg", ctypes.c_int),
                ("forced_ipm_iters", ctypes.c_int), ("start_mode", ctypes.c_int), ("reuse_pcg", ctypes.c_int),
                ("adapt_cost", ctypes.c_int), ("ell_min", ctypes.c_int)]


class Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("a_dtype", ctypes.c_int),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_longlong),
                ("b", ctypes.c_void_p), ("c", ctypes.c_void_p), ("q", ctypes.c_void_p),
                ("x0", ctypes.c_void_p), ("y0", ctypes.c_void_p), ("z0", ctypes.c_void_p),
                ("host", ctypes.c_int), ("lam0", ctypes.c_void_p), ("zeta0", ctypes.c_void_p),
                ("k0", ctypes.c_int), ("ell", ctypes.c_int),
                ("var_kind", ctypes.c_void_p), ("u", ctypes.c_void_p), ("w0", ctypes.c_void_p),
                ("s0", ctypes.c_void_p), ("has_peu_ref", ctypes.c_int), ("peu_ref_p", ctypes.c_double),
                ("peu_ref_d", ctypes.c_double), ("forced_override", ctypes.c_int),
                ("forced_pcg_iters", ctypes.POINTER(ctypes.c_int)), ("n_forced_pcg", ctypes.c_int),
                ("forced_ipm_iters", ctypes.c_int)]

# variable kinds of problems (P~)/(D~) (Problem.var_kind)
KIND_I, KIND_F, KIND_J = 0, 1, 2


class Result(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("lam", ctypes.c_void_p), ("zeta", ctypes.c_void_p),
                ("status", ctypes.c_int), ("ipm_iters", ctypes.c_int),
                ("pcg_iters_total", ctypes.c_int), ("refine_steps", ctypes.c_int),
                ("rel_primal", ctypes.c_double), ("rel_dual", ctypes.c_double),
                ("mu", ctypes.c_double), ("rel_gap", ctypes.c_double), ("rho", ctypes.c_double),
                ("delta", ctypes.c_double), ("seconds", ctypes.c_double),
                ("pcg_seconds", ctypes.c_double), ("pcg_log", ctypes.POINTER(ctypes.c_int)), ("pcg_log_cap", ctypes.c_int),
                ("pcg_log_len", ctypes.c_int), ("w", ctypes.c_void_p), ("s", ctypes.c_void_p),
                ("sketches", ctypes.c_int), ("peu_ref_p", ctypes.c_double), ("peu_ref_d", ctypes.c_double),
                ("ell_log", ctypes.POINTER(ctypes.c_int)), ("ell_log_cap", ctypes.c_int), ("ell_log_len", ctypes.c_int),
                ("device_iteration", ctypes.c_int)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_LL = ctypes.c_longlong

_SIGS = {
    "nys_default_options": (None, [ctypes.POINTER(Options)]),
    "nys_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(Options), _I, _I, _I, _P]),
    "nys_solve": (_I, [_P, ctypes.POINTER(Problem), ctypes.POINTER(Result)]),
    "nys_destroy": (_I, [_P]),
    "nys_last_error": (ctypes.c_char_p, [_P]),
    "nys_kernel_launches": (ctypes.c_ulonglong, []),
    "nys_pcg_route": (_I, [_P, _I, _I, _I]),
    "nys_scaling": (_I, [_P, _I, _P, _P, _P, _D, _P]),
    "nys_normal_matvec": (_I, [_P, _I, _I, _I, _P, _LL, _P, _D, _P, _P]),
    "nys_normal_matvec_lp": (_I, [_P, _I, _I, _I, _P, _LL, _P, _LL, _P, _D, _P, _P]),
    "nys_normal_matvec_noalloc": (_I, [_I, _I, _P, _LL, _P, _D, _P, _P, _P]),
    "nys_quantize_fp8": (_I, [_P, _I, _I, _P, _LL, _P, _LL, _P, _LL, _P]),
    "nys_normal_matvec_fp8": (_I, [_P, _I, _I, _P, _LL, _P, _LL, _P, _P, _D, _P, _P]),
    "nys_gaussian": (_I, [_P, ctypes.c_ulonglong, _I, _I, _I, _P, _I]),
    "nys_sketch": (_I, [_P, _I, _I, _I, _P, _LL, _P, _I, _P, _P, _I]),
    "nys_nystrom": (_I, [_P, _I, _I, _P, _P, _I, _P, _P, ctypes.POINTER(_D)]),
    "nys_precond_apply": (_I, [_P, _I, _I, _P, _I, _P, _D, _P, _P]),
    "nys_pcg": (_I, [_P, _I, _I, _I, _P, _LL, _P, _D, _I, _P, _I, _P, _P, _P, _D, _I, _I,
                     ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "nys_pcg_lp": (_I, [_P, _I, _I, _P, _LL, _I, _P, _D, _I, _P, _I, _P, _P, _P, _D, _I, _I,
                        ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "nys_newton": (_I, [_P, _I, _I, _I, _P, _LL, _P, _P, _P, _D, _P, _P, _P, _I, _P, _I, _P, _D,
                        _I, _I, _P, _P, _P, ctypes.POINTER(_I)]),
    "nys_step_length": (_I, [_P, _I, _P, _P, ctypes.POINTER(_D)]),
    "nys_gemm_bf16": (_I, [_P, _I, _I, _I, _P, _LL, _P, _LL, _P, _LL]),
    "nys_solve_batched": (_I, [_P, _I, ctypes.POINTER(Problem), ctypes.POINTER(Result)]),
    "nys_batch_inflight": (_I, [_P]),
    "nys_batch_plan": (_I, [_P, _I, _I, _I, _P, _P]),
    "nys_adjoint": (_I, [_P, _I, ctypes.POINTER(Problem), ctypes.POINTER(Result), _P, _D, _P, _P, _P, _P]),
}


def lib():
    """Load libnys.so (built by paper_2404_14524_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2404_14524_gb300.build` "
                              "(the solver has no non-CUDA fallback)")
        l = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(l, name)
            f.restype = res
            f.argtypes = args
        _lib = l
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _f64(t, name, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device is not None and t.device != device:
        raise ValueError(f"{name} must be on {device}")
    return t


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Handle:
    """Owner of one nys_handle (workspace on the current CUDA device, bound to a stream)."""

    def __init__(self, max_m: int, max_n: int, ell: int = 20, tol: float = 1e-6, seed: int = 0,
                 max_ipm_iter: int = 200, max_pcg_iter: int = 1000, forced_pcg=None,
                 forced_ipm: int = -1, stream=None, max_batch: int = 0, **kw):
        l = lib()
        o = Options()
        l.nys_default_options(ctypes.byref(o))
        o.tol, o.ell, o.seed = tol, ell, seed
        o.max_ipm_iter, o.max_pcg_iter = max_ipm_iter, max_pcg_iter
        for k, v in kw.items():
            setattr(o, k, v)
        self._forced = None
        if forced_pcg is not None:
            self._forced = (ctypes.c_int * len(forced_pcg))(*[int(v) for v in forced_pcg])
            o.forced_pcg_iters = self._forced
            o.n_forced_pcg = len(forced_pcg)
        o.forced_ipm_iters = forced_ipm
        self.options = o
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        rc = l.nys_create(ctypes.byref(h), ctypes.byref(o), max_m, max_n, max_batch,
                          ctypes.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise NysError(rc, "nys_create failed")
        self.h = h
        self.max_m, self.max_n, self.ell = max_m, max_n, min(ell, max_m)

    def close(self):
        if getattr(self, "h", None):
            lib().nys_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc: int, allow_warn: bool = True):
        if rc < 0 or (rc > 0 and not allow_warn):
            raise NysError(rc, lib().nys_last_error(self.h).decode())
        return rc


# ------------------------------------------------------------------ entry points

def nys_create(max_m, max_n, **kw) -> Handle:
    return Handle(max_m, max_n, **kw)


def nys_destroy(h: Handle):
    h.close()


def nys_last_error(h: Handle) -> str:
    return lib().nys_last_error(h.h).decode()


def nys_kernel_launches() -> int:
    return int(lib().nys_kernel_launches())


NYS_ROUTE_CLUSTER_SMEM, NYS_ROUTE_CLUSTER_L2, NYS_ROUTE_COOPERATIVE, NYS_ROUTE_GRAPH = 0, 1, 2, 3
ROUTE_NAMES = {0: "cluster-smem", 1: "cluster-l2", 2: "cooperative", 3: "graph"}


def nys_pcg_route(h, m: int, n: int, ell: int) -> int:
    """Route (NYS_ROUTE_*) an FP64 PCG solve of this size takes on this handle."""
    rc = int(lib().nys_pcg_route(h.h, m, n, ell))
    if rc < 0:
        raise NysError(rc, "nys_pcg_route: bad argument")
    return rc


def nys_scaling(h: Handle, x, z, q, rho: float, D=None):
    n = x.numel()
    D = torch.empty_like(x) if D is None else D
    h.check(lib().nys_scaling(h.h, n, _ptr(_f64(x, "x")), _ptr(_f64(z, "z")), _ptr(_f64(q, "q")),
                              float(rho), _ptr(_f64(D, "D"))))
    return D


def nys_normal_matvec(h: Handle, A, D, delta: float, v, out=None):
    m, n = A.shape
    out = torch.empty_like(v) if out is None else out
    h.check(lib().nys_normal_matvec(h.h, m, n, NYS_F64, _ptr(_f64(A, "A")), A.stride(0),
                                    _ptr(_f64(D, "D")), float(delta), _ptr(_f64(v, "v")),
                                    _ptr(_f64(out, "out"))))
    return out


def nys_normal_matvec_lp(h: Handle, A, AT, D, delta: float, v, out=None):
    """Precision-form operator with reduced-precision copies A (m x n) and
    AT (n x m), torch.bfloat16 or float32, row-major."""
    m, n = A.shape
    dt = {torch.bfloat16: NYS_BF16, torch.float32: NYS_F32}[A.dtype]
    out = torch.empty_like(v) if out is None else out
    h.check(lib().nys_normal_matvec_lp(h.h, m, n, dt, _ptr(A), A.stride(0), _ptr(AT), AT.stride(0),
                                       _ptr(_f64(D, "D")), float(delta), _ptr(_f64(v, "v")), _ptr(_f64(out, "out"))))
    return out


def nys_quantize_fp8(h: Handle, A32):
    """E4M3 copies of an FP32 row-major A (m x n) with per-row scales:
    returns (Q, QT, row_scale); Q is m x round16(n) and QT n x round16(m)
    uint8 tensors holding the E4M3 bits (padding zero), row_scale FP32."""
    m, n = A32.shape
    if A32.dtype != torch.float32:
        raise TypeError("A must be float32")
    ldq, ldqt = (n + 15) // 16 * 16, (m + 15) // 16 * 16
    Q = torch.empty(m, ldq, dtype=torch.uint8, device=A32.device)
    QT = torch.empty(n, ldqt, dtype=torch.uint8, device=A32.device)
    s = torch.empty(m, dtype=torch.float32, device=A32.device)
    h.check(lib().nys_quantize_fp8(h.h, m, n, _ptr(A32), A32.stride(0), _ptr(Q), ldq, _ptr(QT), ldqt, _ptr(s)))
    return Q, QT, s


def nys_normal_matvec_fp8(h: Handle, m: int, n: int, Q, QT, row_scale, D, delta: float, v, out=None):
    """FP8 operator diag(s) Q (D .* (Q^T (s .* v))) + delta v (precision_mode 2 handle)."""
    out = torch.empty_like(v) if out is None else out
    h.check(lib().nys_normal_matvec_fp8(h.h, m, n, _ptr(Q), Q.stride(0), _ptr(QT), QT.stride(0), _ptr(row_scale),
                                        _ptr(_f64(D, "D")), float(delta), _ptr(_f64(v, "v")), _ptr(_f64(out, "out"))))
    return out


def nys_normal_matvec_noalloc(A, D, delta: float, v, out, stream=None) -> int:
    """(N + delta I) v with no handle and no allocation (fixed library scratch;
    see include/nys.h).  `out` must be preallocated; returns the status code."""
    m, n = A.shape
    st = stream if stream is not None else torch.cuda.current_stream()
    return int(lib().nys_normal_matvec_noalloc(m, n, _ptr(_f64(A, "A")), A.stride(0), _ptr(_f64(D, "D")),
                                               float(delta), _ptr(_f64(v, "v")), _ptr(_f64(out, "out")),
                                               ctypes.c_void_p(st.cuda_stream)))


def nys_gaussian(h: Handle, seed: int, k: int, m: int, ell: int, out=None):
    out = torch.empty((ell, m), dtype=torch.float64, device=h.device) if out is None else out
    h.check(lib().nys_gaussian(h.h, seed, k, m, ell, _ptr(_f64(out, "Omega")), out.shape[1]))
    return out


def nys_sketch(h: Handle, A, D, Omega, out=None):
    """Y = A (D .* (A^T Omega)); A float64 (FP64 sketch) or float32 (the
    precision form's BF16 tensor-core sketch, precision-form handle)."""
    m, n = A.shape
    ell = Omega.shape[0]
    out = torch.empty_like(Omega) if out is None else out
    if A.dtype == torch.float32:
        if A.stride(1) != 1 or not A.is_cuda:
            raise TypeError("A must be a row-major CUDA tensor")
        dt, pa = NYS_F32, _ptr(A)
    else:
        dt, pa = NYS_F64, _ptr(_f64(A, "A"))
    h.check(lib().nys_sketch(h.h, m, n, dt, pa, A.stride(0), _ptr(_f64(D, "D")),
                             ell, _ptr(_f64(Omega, "Omega")), _ptr(_f64(out, "Y")), Omega.shape[1]))
    return out


def nys_nystrom(h: Handle, Y, Omega):
    ell, ld = Y.shape
    m = ld
    U = torch.empty_like(Y)
    lam = torch.empty(ell, dtype=torch.float64, device=Y.device)
    nu = ctypes.c_double()
    h.check(lib().nys_nystrom(h.h, m, ell, _ptr(_f64(Y, "Y")), _ptr(_f64(Omega, "Omega")), ld,
                              _ptr(U), _ptr(lam), ctypes.byref(nu)))
    return U, lam, nu.value


def nys_precond_apply(h: Handle, U, lam, delta: float, r, out=None):
    ell, m = U.shape
    out = torch.empty_like(r) if out is None else out
    h.check(lib().nys_precond_apply(h.h, m, ell, _ptr(_f64(U, "U")), m, _ptr(_f64(lam, "lam")),
                                    float(delta), _ptr(_f64(r, "r")), _ptr(_f64(out, "out"))))
    return out


def nys_pcg(h: Handle, A, D, delta: float, U, lam, xi, eta: float, max_iter: int, forced: int = -1,
            out=None):
    m, n = A.shape
    ell = U.shape[0]
    out = torch.empty_like(xi) if out is None else out
    it = ctypes.c_int()
    res = ctypes.c_double()
    rc = lib().nys_pcg(h.h, m, n, NYS_F64, _ptr(_f64(A, "A")), A.stride(0), _ptr(_f64(D, "D")),
                       float(delta), ell, _ptr(_f64(U, "U")), U.shape[1], _ptr(_f64(lam, "lam")),
                       _ptr(_f64(xi, "xi")), _ptr(_f64(out, "dy")), float(eta), int(max_iter),
                       int(forced), ctypes.byref(it), ctypes.byref(res))
    h.check(rc)
    return out, it.value, res.value, rc


def nys_pcg_lp(h: Handle, A32, op: str, D, delta: float, U, lam, xi, eta: float, max_iter: int, forced: int = -1,
               out=None):
    """PCG on the precision form's operator built from the FP32 matrix A32:
    op "bf16", "fp8" or "ff" (FP32 with float-float sums).  Returns
    (dy, iters, |r|, status)."""
    m, n = A32.shape
    ell = U.shape[0]
    dt = {"bf16": NYS_BF16, "fp8": NYS_FP8E4M3, "ff": NYS_F32}[op]
    out = torch.empty_like(xi) if out is None else out
    it = ctypes.c_int()
    res = ctypes.c_double()
    if A32.dtype != torch.float32 or A32.stride(1) != 1:
        raise TypeError("A must be row-major float32")
    rc = lib().nys_pcg_lp(h.h, m, n, _ptr(A32), A32.stride(0), dt, _ptr(_f64(D, "D")), float(delta), ell,
                          _ptr(_f64(U, "U")), U.shape[1], _ptr(_f64(lam, "lam")), _ptr(_f64(xi, "xi")),
                          _ptr(_f64(out, "out")),
                          float(eta), int(max_iter), int(forced), ctypes.byref(it), ctypes.byref(res))
    if rc < 0:
        h.check(rc)
    return out, it.value, res.value, rc


def nys_newton(h: Handle, A, x, z, D, delta, r_d, r_p, r_xz, U, lam, eta, max_iter, forced=-1):
    m, n = A.shape
    ell = U.shape[0]
    dx, dz = torch.empty_like(x), torch.empty_like(x)
    dy = torch.empty_like(r_p)
    it = ctypes.c_int()
    rc = lib().nys_newton(h.h, m, n, NYS_F64, _ptr(_f64(A, "A")), A.stride(0), _ptr(_f64(x, "x")),
                          _ptr(_f64(z, "z")), _ptr(_f64(D, "D")), float(delta), _ptr(_f64(r_d, "r_d")),
                          _ptr(_f64(r_p, "r_p")), _ptr(_f64(r_xz, "r_xz")), ell, _ptr(_f64(U, "U")),
                          U.shape[1], _ptr(_f64(lam, "lam")), float(eta), int(max_iter), int(forced),
                          _ptr(dx), _ptr(dy), _ptr(dz), ctypes.byref(it))
    h.check(rc)
    return dx, dy, dz, it.value


def nys_gemm_bf16(h: Handle, A, B, out=None):
    """C = A B^T (A: M x K, B: N x K, torch.bfloat16 row-major) on the tensor
    cores; returns C as an (N, M) float32 tensor (column-major M x N)."""
    M, K = A.shape
    N = B.shape[0]
    for t, nm in ((A, "A"), (B, "B")):
        if t.dtype != torch.bfloat16 or t.stride(1) != 1:
            raise TypeError(f"{nm} must be a row-major bfloat16 tensor")
    out = torch.empty((N, M), dtype=torch.float32, device=A.device) if out is None else out
    h.check(lib().nys_gemm_bf16(h.h, M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(out), M))
    return out


def nys_step_length(h: Handle, v, dv) -> float:
    a = ctypes.c_double()
    h.check(lib().nys_step_length(h.h, v.numel(), _ptr(_f64(v, "v")), _ptr(_f64(dv, "dv")),
                                  ctypes.byref(a)))
    return a.value


def _box_fields(kind, u, s0, w0, n, dev, host):
    """Problem fields of (P~)/(D~): int8 kinds, float64 u, s0 and optional w0 (n each)."""
    if kind is None:
        return {}, []
    where = torch.device("cpu") if host else dev
    if not isinstance(kind, torch.Tensor) or kind.dtype != torch.int8 or kind.shape != (n,) \
            or not kind.is_contiguous() or kind.device != where:
        raise TypeError(f"var_kind must be a contiguous int8 tensor of length {n} on {where}")
    keep = [kind]
    f = {"var_kind": kind.data_ptr()}
    for t, nm in ((u, "u"), (s0, "s0"), (w0, "w0")):
        if t is not None:
            _f64(t, nm, where)
            keep.append(t)
            f[nm] = t.data_ptr()
    return f, keep


def nys_solve(h: Handle, A, b, c, q, x0, y0, z0, pcg_log_cap: int = 4096, check: bool = True,
              lam0=None, zeta0=None, k0: int = 0, want_pmm: bool = False, kind=None, u=None,
              s0=None, w0=None, peu_ref=None):
    """Solve one QP.  CUDA tensors -> device problem; CPU tensors -> host
    problem (the library stages the data; pin the tensors for fast copies).
    lam0/zeta0/k0 resume from a saved state (rho/delta come from the handle's
    options; peu_ref = (ref_p, ref_d) are the PMM update's references,
    None = those of the start point).  kind (int8: KIND_I, KIND_F, KIND_J per variable), u, s0 and
    optionally w0 make it problem (P~) with free and box-constrained
    variables; info then also holds the final w and s.  With a handle
    created with start_mode=1 (the practical initial point) x0, y0, z0, s0
    and w0 may be None.  Returns
    (x, y, z, info); with want_pmm, info also holds the final lam and zeta."""
    m, n = A.shape
    host = not A.is_cuda
    dev = None if host else A.device
    if A.dtype == torch.float32:          # precision form: FP32 A defines the problem
        a_dtype = NYS_F32
        if A.stride(1) != 1:
            raise ValueError("A must be row-major")
    else:
        a_dtype = NYS_F64
        _f64(A, "A", dev if not host else torch.device("cpu"))
    for t, nm in ((b, "b"), (c, "c"), (q, "q"), (x0, "x0"), (y0, "y0"), (z0, "z0")):
        if t is not None or nm in ("b", "c", "q"):       # x0, y0, z0 may be None with start_mode=1
            _f64(t, nm, dev if not host else torch.device("cpu"))
    mk = (lambda k: torch.empty(k, dtype=torch.float64, pin_memory=True)) if host else \
        (lambda k: torch.empty(k, dtype=torch.float64, device=dev))
    x, y, z = mk(n), mk(m), mk(n)
    lam, zeta = (mk(m), mk(n)) if want_pmm else (None, None)
    for t, nm in ((lam0, "lam0"), (zeta0, "zeta0")):
        if t is not None:
            _f64(t, nm, dev if not host else torch.device("cpu"))
    bf, _keep = _box_fields(kind, u, s0, w0, n, dev, host)
    opt_ptr = lambda t: t.data_ptr() if t is not None else None
    p = Problem(m=m, n=n, a_dtype=a_dtype, A=A.data_ptr(), lda=A.stride(0), b=b.data_ptr(),
                c=c.data_ptr(), q=q.data_ptr(), x0=opt_ptr(x0), y0=opt_ptr(y0),
                z0=opt_ptr(z0), host=1 if host else 0,
                lam0=lam0.data_ptr() if lam0 is not None else None,
                zeta0=zeta0.data_ptr() if zeta0 is not None else None, k0=k0, **bf)
    if peu_ref is not None:
        p.has_peu_ref, p.peu_ref_p, p.peu_ref_d = 1, float(peu_ref[0]), float(peu_ref[1])
    log = (ctypes.c_int * pcg_log_cap)()
    elog = (ctypes.c_int * pcg_log_cap)()
    w, s = (mk(n), mk(n)) if kind is not None else (None, None)
    r = Result(x=x.data_ptr(), y=y.data_ptr(), z=z.data_ptr(),
               lam=lam.data_ptr() if lam is not None else None,
               zeta=zeta.data_ptr() if zeta is not None else None,
               pcg_log=log, pcg_log_cap=pcg_log_cap, ell_log=elog, ell_log_cap=pcg_log_cap,
               w=w.data_ptr() if w is not None else None, s=s.data_ptr() if s is not None else None)
    rc = lib().nys_solve(h.h, ctypes.byref(p), ctypes.byref(r))
    if check:
        h.check(rc)
    info = {k: getattr(r, k) for k in ("status", "ipm_iters", "pcg_iters_total", "refine_steps",
                                       "rel_primal", "rel_dual", "mu", "rel_gap", "rho", "delta",
                                       "seconds", "pcg_seconds", "sketches", "peu_ref_p",
                                       "peu_ref_d", "device_iteration")}
    info["pcg_log"] = list(log[: r.pcg_log_len])
    info["ell_log"] = list(elog[: r.ell_log_len])
    if want_pmm:
        info["lam"], info["zeta"] = lam, zeta
    if kind is not None:
        info["w"], info["s"] = w, s
    return x, y, z, info


def solve(A, b, c, q, x0=None, y0=None, z0=None, ell: int = 20, tol: float = 1e-6, kind=None, u=None,
          s0=None, w0=None, **options):
    """One call: a handle sized for A (start_mode 1, the practical initial
    point, when no x0 is given), nys_solve, and the handle released again.
    Tensors as for nys_solve; other keyword arguments are nys_options fields
    (seed, max_ipm_iter, max_pcg_iter, precision_mode, reuse_pcg, ...).
    x0, y0, z0 are given together or not at all; under start_mode=1 any
    given start is ignored.  Returns (x, y, z, info)."""
    m, n = A.shape
    given = [t is not None for t in (x0, y0, z0)]
    if any(given) and not all(given):
        raise ValueError("x0, y0 and z0 must be given together (or all None for the practical start)")
    if x0 is None:
        options.setdefault("start_mode", 1)
    h = Handle(m, n, ell=ell, tol=tol, **options)
    try:
        return nys_solve(h, A, b, c, q, x0, y0, z0, kind=kind, u=u, s0=s0, w0=w0)
    finally:
        h.close()


def nys_adjoint(h: Handle, A, q, x, y, z, info, dL_dx, eta: float = 1e-12):
    """Gradients of L(x*) for one solved QP (device FP64 tensors; `info` is the
    dict returned by nys_solve).  Returns dict(c=..., b=..., q=..., A=...)."""
    m, n = A.shape
    _f64(A, "A", A.device)
    p = Problem(m=m, n=n, a_dtype=NYS_F64, A=A.data_ptr(), lda=A.stride(0), q=_f64(q, "q").data_ptr(), host=0)
    r = Result(x=_f64(x, "x").data_ptr(), y=_f64(y, "y").data_ptr(), z=_f64(z, "z").data_ptr(),
               rho=info["rho"], delta=info["delta"], ipm_iters=info["ipm_iters"])
    gc, gq = torch.empty(n, dtype=torch.float64, device=A.device), torch.empty(n, dtype=torch.float64, device=A.device)
    gb = torch.empty(m, dtype=torch.float64, device=A.device)
    gA = torch.empty(m, n, dtype=torch.float64, device=A.device)
    rc = lib().nys_adjoint(h.h, 1, ctypes.byref(p), ctypes.byref(r), _ptr(_f64(dL_dx, "dL_dx")), float(eta),
                           _ptr(gc), _ptr(gb), _ptr(gq), _ptr(gA))
    h.check(rc)
    return {"c": gc, "b": gb, "q": gq, "A": gA}


class NysQPFunction(torch.autograd.Function):
    """x* = argmin of the separable QP (P) as a differentiable function of
    (A, b, c, q).  Forward: nys_solve; backward: nys_adjoint (transposed-KKT
    solve by Nystrom PCG).  A FP32 input is solved in FP64 and its gradient
    returned in FP32."""

    @staticmethod
    def forward(ctx, A, b, c, q, x0, y0, z0, handle, eta):
        A64 = A.double().contiguous()
        x, y, z, info = nys_solve(handle, A64, b, c, q, x0, y0, z0)
        ctx.save_for_backward(A64, q, x, y, z)
        ctx.info, ctx.handle, ctx.eta, ctx.a_dtype = info, handle, eta, A.dtype
        ctx.mark_non_differentiable(y, z)
        return x, y, z

    @staticmethod
    def backward(ctx, gx, gy, gz):
        A64, q, x, y, z = ctx.saved_tensors
        g = nys_adjoint(ctx.handle, A64, q, x, y, z, ctx.info, gx.contiguous(), ctx.eta)
        return g["A"].to(ctx.a_dtype), g["b"], g["c"], g["q"], None, None, None, None, None


def qp_solve(A, b, c, q, x0, y0, z0, handle, eta: float = 1e-12):
    """Differentiable solve: returns (x, y, z); gradients flow to A, b, c, q through x."""
    return NysQPFunction.apply(A, b, c, q, x0, y0, z0, handle, eta)


def nys_batch_inflight(h: Handle) -> int:
    """Problems in flight the handle's batch autotuner chose (0: not tuned yet)."""
    return int(lib().nys_batch_inflight(h.h))


def nys_batch_plan(h: Handle, m: int, n: int, ell: int):
    """(tuned, ctas, a_smem): the PCG cluster plan the handle's batch
    autotuner chose for the shape bucket of (m, n, ell)."""
    c, a = ctypes.c_int(), ctypes.c_int()
    rc = lib().nys_batch_plan(h.h, m, n, ell, ctypes.byref(c), ctypes.byref(a))
    h.check(rc)
    return rc == 1, c.value, a.value


def nys_solve_batched(h: Handle, problems, check: bool = True, forced=None, pcg_log_cap: int = 4096):
    """Solve a list of QPs [(A, b, c, q, x0, y0, z0[, ell[, box]]), ...]
    (device tensors; optional per-problem sketch size, 0 = the handle's; box
    = dict(kind=, u=, s0=[, w0=]) for a problem (P~)) in one call; the handle
    must have max_batch >= 1.  forced: optional per-problem parity counts,
    a list of (pcg_counts, ipm_iters) or None entries.  Returns a list of
    (x, y, z, info); info holds the PCG log, and w and s for the (P~)
    problems."""
    k = len(problems)
    P = (Problem * k)()
    R = (Result * k)()
    outs, keep = [], []
    logs = [(ctypes.c_int * pcg_log_cap)() for _ in range(k)]
    for i, pr in enumerate(problems):
        A, b, c, q, x0, y0, z0 = pr[:7]
        ell_i = int(pr[7]) if len(pr) > 7 else 0
        bx = pr[8] if len(pr) > 8 else None
        m, n = A.shape
        a_dtype = NYS_F32 if A.dtype == torch.float32 else NYS_F64
        x = torch.empty(n, dtype=torch.float64, device=A.device)
        y = torch.empty(m, dtype=torch.float64, device=A.device)
        z = torch.empty(n, dtype=torch.float64, device=A.device)
        bf, kp = _box_fields(bx.get("kind"), bx.get("u"), bx.get("s0"), bx.get("w0"), n, A.device, False) \
            if bx else ({}, [])
        keep += kp
        w = torch.empty(n, dtype=torch.float64, device=A.device) if bx else None
        s = torch.empty(n, dtype=torch.float64, device=A.device) if bx else None
        P[i] = Problem(m=m, n=n, a_dtype=a_dtype, A=A.data_ptr(), lda=A.stride(0), b=b.data_ptr(), c=c.data_ptr(),
                       q=q.data_ptr(), x0=x0.data_ptr(), y0=y0.data_ptr(), z0=z0.data_ptr(), host=0, ell=ell_i, **bf)
        if forced is not None and forced[i] is not None:
            fp, fi = forced[i]
            arr = (ctypes.c_int * max(1, len(fp)))(*fp)
            keep.append(arr)
            P[i].forced_override, P[i].forced_pcg_iters, P[i].n_forced_pcg = 1, arr, len(fp)
            P[i].forced_ipm_iters = -1 if fi is None else int(fi)
        R[i] = Result(x=x.data_ptr(), y=y.data_ptr(), z=z.data_ptr(),
                      w=w.data_ptr() if w is not None else None, s=s.data_ptr() if s is not None else None,
                      pcg_log=logs[i], pcg_log_cap=pcg_log_cap)
        outs.append((x, y, z, w, s))
    rc = lib().nys_solve_batched(h.h, k, P, R)
    if check:
        h.check(rc)
    res = []
    for i, (x, y, z, w, s) in enumerate(outs):
        info = {f: getattr(R[i], f) for f in ("status", "ipm_iters", "pcg_iters_total", "refine_steps", "rel_primal",
                                              "rel_dual", "mu", "rel_gap", "rho", "delta", "seconds",
                                              "pcg_seconds", "sketches", "device_iteration")}
        info["pcg_log"] = list(logs[i][: R[i].pcg_log_len])
        if w is not None:
            info["w"], info["s"] = w, s
        res.append((x, y, z, info))
    return res
