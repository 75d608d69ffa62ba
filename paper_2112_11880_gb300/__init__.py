"""Python binding of libhelm (complex Krylov solvers for Helmholtz FEM on GB300).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libhelm.so, reached through its C ABI (include/helm.h) with
ctypes.  PyTorch provides device memory and streams.  There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.

The functions keep the C names (helm_csr_create, helm_spmv, helm_dot,
helm_nrm2, helm_axpby, helm_bicgstab_solve, helm_adjoint, ...); `CsrMatrix`
and `solve` are thin conveniences over them.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libhelm.so")

HELM_OK = 0
HELM_ERR_INVALID = 1
HELM_ERR_CUDA = 2
HELM_ERR_NOMEM = 3
HELM_ERR_NOT_CONVERGED = 4
HELM_ERR_BREAKDOWN = 5
HELM_ERR_TIMEOUT = 6
HELM_ERR_NONFINITE = 7
STATUS_NAMES = {0: "ok", 1: "invalid", 2: "cuda", 3: "nomem", 4: "not_converged", 5: "breakdown",
                6: "timeout", 7: "nonfinite"}

HELM_C128 = 0
HELM_C64 = 1
HELM_CSR_VALIDATE = 1
HELM_CSR_SLICED_ONLY = 2
HELM_DDM_IMPEDANCE = 1

HELM_BICGSTAB = 0
HELM_TFQMR = 1
HELM_BICGSTABL = 2
HELM_PREC_FP64 = 0
HELM_PREC_MIXED = 1
HELM_LAUNCH_AUTO = 0
HELM_LAUNCH_GRAPH = 1
HELM_LAUNCH_PERSISTENT = 2
HELM_LAUNCH_HOST = 3
HELM_PRECOND_NONE = 0
HELM_PRECOND_JACOBI = 1


class helm_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int32), ("use_x0", ctypes.c_int32),
                ("method", ctypes.c_int32), ("precision", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("deadline_s", ctypes.c_double), ("ell", ctypes.c_int32), ("launch", ctypes.c_int32),
                ("precond", ctypes.c_int32)]


class helm_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32), ("relres_recur", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("status", ctypes.c_int32), ("spmv_count", ctypes.c_int32)]

    def as_dict(self):
        return {"status": STATUS_NAMES.get(self.status, self.status), "iters": self.iters,
                "restarts": self.restarts, "relres_recur": self.relres_recur,
                "relres_true": self.relres_true, "spmv_count": self.spmv_count}


class HelmError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")


_P = ctypes.c_void_p
# name -> (restype, argtypes); the declarations of include/helm.h
SIGNATURES = {
    "helm_csr_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int64, _P, _P, _P,
                                       ctypes.c_int, ctypes.c_uint32, _P]),
    "helm_csr_destroy": (ctypes.c_int, [_P]),
    "helm_csr_diagonals": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "helm_spmv": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "helm_dot": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, _P, _P, ctypes.c_int, _P, _P]),
    "helm_dot_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, _P, _P, ctypes.c_int, _P, _P]),
    "helm_nrm2": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, _P, _P, _P]),
    "helm_axpby": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, _P, _P, _P, _P, _P]),
    "helm_opts_default": (None, [ctypes.POINTER(helm_opts)]),
    "helm_bicgstab_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(helm_opts), ctypes.POINTER(helm_info), _P]),
    "helm_adjoint": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(helm_opts), _P, _P, ctypes.POINTER(helm_info), _P]),
    "helm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "helm_grad_sound_speed": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _P, _P, ctypes.c_double, _P, _P]),
    "helm_assemble_helmholtz": (ctypes.c_int, [ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P, ctypes.c_double, _P,
                                               _P]),
    "helm_conj_scale": (ctypes.c_int, [ctypes.c_int64, _P, _P, _P, _P]),
    "helm_sweep_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int64, _P, _P, _P, _P, _P, _P]),
    "helm_sweep_destroy": (ctypes.c_int, [_P]),
    "helm_sweep_solve": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, ctypes.c_int32,
                                        ctypes.POINTER(helm_opts), _P, _P]),
    "helm_sweep_spmv": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, ctypes.c_int32, _P]),
    "helm_ddm_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_uint32, _P]),
    "helm_ddm_destroy": (ctypes.c_int, [_P]),
    "helm_ddm_subdomains": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]),
    "helm_ddm_apply": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, _P]),
    "helm_ddm_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(helm_opts), ctypes.POINTER(helm_info), _P]),
}

_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhelm.so (built by build.py / __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libhelm.so not built ({path}); run paper_2112_11880_gb300/build.py")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int, what: str):
    if status != HELM_OK:
        raise HelmError(status, what)


def _stream(stream=None) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(getattr(stream, "cuda_stream", stream) or 0)


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


def _c2(z) -> ctypes.Array:
    z = complex(z)
    return (ctypes.c_double * 2)(z.real, z.imag)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.complex128:
        return HELM_C128
    if t.dtype == torch.complex64:
        return HELM_C64
    raise TypeError(f"expected complex128 or complex64, got {t.dtype}")


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("tensors must be on a CUDA device")
        if t is not None and not t.is_contiguous():
            raise ValueError("tensors must be contiguous")


# ---------------------------------------------------------------- C-named wrappers

def helm_csr_create(n, nnz, d_rowptr, d_colind, d_vals, dt, flags=0, stream=None) -> int:
    lib = load_library()
    h = _P()
    _check(lib.helm_csr_create(ctypes.byref(h), int(n), int(nnz), d_rowptr, d_colind, d_vals, int(dt),
                               int(flags), _stream(stream)), "helm_csr_create")
    return h.value


def helm_csr_destroy(handle) -> None:
    _check(load_library().helm_csr_destroy(handle), "helm_csr_destroy")


def helm_csr_diagonals(handle) -> int:
    """Diagonals of the handle's diagonal copy (0: complex64 products read the sliced copy)."""
    out = ctypes.c_int32(0)
    _check(load_library().helm_csr_diagonals(handle, ctypes.byref(out)), "helm_csr_diagonals")
    return out.value


def helm_spmv(handle, alpha, x, beta, y, stream=None) -> None:
    _require_cuda(x, y)
    _check(load_library().helm_spmv(handle, _c2(alpha), _ptr(x), _c2(beta), _ptr(y), _stream(stream)), "helm_spmv")


def helm_dot(x, y, out, conj_x: bool = True, stream=None) -> None:
    """out (device complex128 scalar) = (x, y)."""
    _require_cuda(x, y, out)
    if x.numel() != y.numel() or x.dtype != y.dtype:
        raise ValueError("x and y must have the same length and dtype")
    import torch
    if out.dtype != torch.complex128 or out.numel() < 1:
        raise ValueError("out must be a complex128 device tensor")
    _check(load_library().helm_dot(x.numel(), _dtype_code(x), _ptr(x), _ptr(y), 1 if conj_x else 0, _ptr(out),
                                   _stream(stream)), "helm_dot")


def helm_dot_noalloc(x, y, out, conj_x: bool = True, stream=None) -> None:
    """out (device complex128 scalar) = (x, y), computed with the library's
    fixed scratch array instead of allocated memory (for callers that cannot
    allocate; see include/helm.h)."""
    _require_cuda(x, y, out)
    if x.numel() != y.numel() or x.dtype != y.dtype:
        raise ValueError("x and y must have the same length and dtype")
    import torch
    if out.dtype != torch.complex128 or out.numel() < 1:
        raise ValueError("out must be a complex128 device tensor")
    _check(load_library().helm_dot_noalloc(x.numel(), _dtype_code(x), _ptr(x), _ptr(y), 1 if conj_x else 0,
                                           _ptr(out), _stream(stream)), "helm_dot_noalloc")


def helm_nrm2(x, out, stream=None) -> None:
    """out (device float64 scalar) = ||x||_2."""
    _require_cuda(x, out)
    import torch
    if out.dtype != torch.float64 or out.numel() < 1:
        raise ValueError("out must be a float64 device tensor")
    _check(load_library().helm_nrm2(x.numel(), _dtype_code(x), _ptr(x), _ptr(out), _stream(stream)), "helm_nrm2")


def helm_axpby(alpha, x, beta, y, stream=None) -> None:
    """y = alpha x + beta y."""
    _require_cuda(x, y)
    if x is not None and (x.numel() != y.numel() or x.dtype != y.dtype):
        raise ValueError("x and y must have the same length and dtype")
    _check(load_library().helm_axpby(y.numel(), _dtype_code(y), _c2(alpha), _ptr(x), _c2(beta), _ptr(y),
                                     _stream(stream)), "helm_axpby")


def default_opts(**kw) -> helm_opts:
    o = helm_opts()
    load_library().helm_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def helm_bicgstab_solve(handle, b, x, opts: Optional[helm_opts] = None, stream=None) -> dict:
    """Solve A x = b; returns the info dict (status is reported, not raised,
    for solver outcomes; argument and CUDA errors raise)."""
    _require_cuda(b, x)
    info = helm_info()
    o = opts if opts is not None else default_opts()
    st = load_library().helm_bicgstab_solve(handle, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(info),
                                            _stream(stream))
    if st in (HELM_ERR_INVALID, HELM_ERR_CUDA, HELM_ERR_NOMEM):
        raise HelmError(st, "helm_bicgstab_solve")
    return info.as_dict()


def helm_adjoint(handle, u, dLdu, mu, dLdvals=None, opts: Optional[helm_opts] = None, stream=None) -> dict:
    _require_cuda(u, dLdu, mu, dLdvals)
    info = helm_info()
    o = opts if opts is not None else default_opts()
    st = load_library().helm_adjoint(handle, _ptr(u), _ptr(dLdu), ctypes.byref(o), _ptr(mu), _ptr(dLdvals),
                                     ctypes.byref(info), _stream(stream))
    if st in (HELM_ERR_INVALID, HELM_ERR_CUDA, HELM_ERR_NOMEM):
        raise HelmError(st, "helm_adjoint")
    return info.as_dict()


def _host_f64(a):
    import numpy as np
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


def helm_grad_sound_speed(dLdvals, elem_map, Me, Bf, top, c, omega, grad, stream=None) -> None:
    _require_cuda(dLdvals, elem_map, top, c, grad)
    me, pme = _host_f64(Me)
    bf, pbf = _host_f64(Bf)
    if me.size != 64 or bf.size != 64:
        raise ValueError("Me and Bf must have 64 entries")
    _check(load_library().helm_grad_sound_speed(c.numel(), _ptr(dLdvals), _ptr(elem_map), pme, pbf, _ptr(top),
                                                _ptr(c), float(omega), _ptr(grad), _stream(stream)),
           "helm_grad_sound_speed")


def helm_assemble_helmholtz(K, slot_elem, slot_pair, Me, Bf, top, c, omega, vals, stream=None) -> None:
    _require_cuda(K, slot_elem, slot_pair, top, c, vals)
    me, pme = _host_f64(Me)
    bf, pbf = _host_f64(Bf)
    _check(load_library().helm_assemble_helmholtz(K.numel(), _ptr(K), _ptr(slot_elem), _ptr(slot_pair), pme, pbf,
                                                  _ptr(top), _ptr(c), float(omega), _ptr(vals), _stream(stream)),
           "helm_assemble_helmholtz")


def helm_conj_scale(alpha, x, y, stream=None) -> None:
    """y = alpha conj(x) (complex128)."""
    _require_cuda(x, y)
    _check(load_library().helm_conj_scale(x.numel(), _c2(alpha), _ptr(x), _ptr(y), _stream(stream)),
           "helm_conj_scale")


def helm_sweep_create(n, nnz, d_rowptr, d_colind, d_K, d_M, d_B, stream=None) -> int:
    h = _P()
    _check(load_library().helm_sweep_create(ctypes.byref(h), int(n), int(nnz), d_rowptr, d_colind, d_K, d_M, d_B,
                                            _stream(stream)), "helm_sweep_create")
    return h.value


def helm_sweep_destroy(handle) -> None:
    _check(load_library().helm_sweep_destroy(handle), "helm_sweep_destroy")


def helm_sweep_spmv(handle, omegas, X, Y, stream=None) -> None:
    """Y[:, j] = A_j X[:, j] for the frequencies `omegas` (X, Y: n x F
    complex128, row-major, device)."""
    import numpy as np
    for t in (X, Y):
        if not t.is_cuda or t.dim() != 2 or t.stride(1) != 1:
            raise ValueError("X, Y: 2-D CUDA tensors with unit column stride")
    w = np.ascontiguousarray(np.asarray(omegas, dtype=np.float64))
    F = int(w.size)
    _check(load_library().helm_sweep_spmv(handle, F, w.ctypes.data_as(ctypes.c_void_p), _ptr(X), int(X.stride(0)),
                                          _ptr(Y), int(Y.stride(0)), _stream(stream)), "helm_sweep_spmv")


def helm_sweep_solve(handle, omegas, b, X, opts: Optional[helm_opts] = None, stream=None):
    """Solve all frequencies; b is [n] (shared) or [n, F]; X is [n, F]
    complex128 (row-major).  Returns a list of per-frequency info dicts."""
    import numpy as np
    _require_cuda(b, X)
    w = np.ascontiguousarray(omegas, dtype=np.float64)
    F = int(w.size)
    b_ld = 0 if b.dim() == 1 else int(b.shape[1])
    infos = (helm_info * F)()
    o = opts if opts is not None else default_opts()
    st = load_library().helm_sweep_solve(handle, F, w.ctypes.data_as(ctypes.c_void_p), _ptr(b), b_ld, _ptr(X),
                                         int(X.shape[1]), ctypes.byref(o), ctypes.cast(infos, ctypes.c_void_p),
                                         _stream(stream))
    if st in (HELM_ERR_INVALID, HELM_ERR_CUDA, HELM_ERR_NOMEM):
        raise HelmError(st, "helm_sweep_solve")
    return [infos[j].as_dict() for j in range(F)]


class Ddm:
    """Schwarz decomposition of a CsrMatrix into `nsub` overlapping row
    blocks, the subdomain solves batched (see helm_ddm_create)."""

    def __init__(self, A, nsub: int, overlap: int, window: int = 256, impedance: bool = True, stream=None):
        self.A = A  # the handle borrows A
        h = _P()
        _check(load_library().helm_ddm_create(ctypes.byref(h), A.handle, int(nsub), int(overlap), int(window),
                                              HELM_DDM_IMPEDANCE if impedance else 0, _stream(stream)),
               "helm_ddm_create")
        self.handle = h.value
        self.n = A.n

    def subdomains(self):
        rows, nnz = ctypes.c_int32(0), ctypes.c_int64(0)
        _check(load_library().helm_ddm_subdomains(self.handle, ctypes.byref(rows), ctypes.byref(nnz)),
               "helm_ddm_subdomains")
        return rows.value, nnz.value

    def apply(self, r, z=None, inner_tol: float = 1e-3, stream=None):
        """z = M r, the restricted additive Schwarz preconditioner."""
        import torch
        _check_vector(r, self.n, torch.complex128, "r")
        if z is None:
            z = torch.empty_like(r)
        _check_vector(z, self.n, torch.complex128, "z")
        _require_cuda(r, z)
        _check(load_library().helm_ddm_apply(self.handle, _ptr(r), _ptr(z), float(inner_tol), _stream(stream)),
               "helm_ddm_apply")
        return z

    def solve(self, b, x=None, stream=None, **opts):
        import torch
        _check_vector(b, self.n, torch.complex128, "b")
        if x is None:
            x = torch.zeros_like(b)
        _check_vector(x, self.n, torch.complex128, "x")
        _require_cuda(b, x)
        info = helm_info()
        o = default_opts(**opts)
        st = load_library().helm_ddm_solve(self.handle, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(info),
                                           _stream(stream))
        if st in (HELM_ERR_INVALID, HELM_ERR_CUDA, HELM_ERR_NOMEM):
            raise HelmError(st, "helm_ddm_solve")
        return x, info.as_dict()

    def close(self):
        if getattr(self, "handle", None):
            load_library().helm_ddm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sweep:
    """Frequency sweep on one pattern: A_j = K - w_j^2 M + i w_j B."""

    def __init__(self, rowptr, colind, K, M, B, device="cuda"):
        import torch
        dev = torch.device(device)
        self.rowptr = torch.as_tensor(rowptr, dtype=torch.int32).to(dev).contiguous()
        self.colind = torch.as_tensor(colind, dtype=torch.int32).to(dev).contiguous()
        self.K = torch.as_tensor(K, dtype=torch.float64).to(dev).contiguous()
        self.M = torch.as_tensor(M, dtype=torch.float64).to(dev).contiguous()
        self.B = torch.as_tensor(B, dtype=torch.float64).to(dev).contiguous()
        self.n = self.rowptr.numel() - 1
        self.nnz = self.colind.numel()
        self.handle = helm_sweep_create(self.n, self.nnz, _ptr(self.rowptr), _ptr(self.colind), _ptr(self.K),
                                        _ptr(self.M), _ptr(self.B))

    def solve(self, omegas, b, X=None, **opts):
        import torch
        F = len(omegas)
        _check_vector(b, self.n, torch.complex128, "b", None if b.dim() == 1 else F)
        if X is None:
            X = torch.zeros((self.n, F), dtype=torch.complex128, device=b.device)
        _check_vector(X, self.n, torch.complex128, "X", F)
        infos = helm_sweep_solve(self.handle, omegas, b, X, default_opts(**opts))
        return X, infos

    def matvec(self, omegas, X, Y=None):
        """Y[:, j] = A_j X[:, j], the sweep's own on-the-fly product."""
        import torch
        F = len(omegas)
        _check_vector(X, self.n, torch.complex128, "X", F)
        if Y is None:
            Y = torch.empty_like(X)
        _check_vector(Y, self.n, torch.complex128, "Y", F)
        helm_sweep_spmv(self.handle, omegas, X, Y)
        return Y

    def close(self):
        if getattr(self, "handle", None):
            helm_sweep_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def helm_status_string(status: int) -> str:
    return load_library().helm_status_string(int(status)).decode()


# ---------------------------------------------------------------- conveniences

def _check_vector(t, n: int, dtype, name: str, cols: Optional[int] = None) -> None:
    """Dtype and shape of a vector (cols None: n entries) or a row-major n x cols
    block against the matrix it meets.  The C ABI takes bare device pointers and
    cannot see a buffer that is too short, so the convenience layer checks."""
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if cols is None:
        if t.numel() != n:
            raise ValueError(f"{name}: expected {n} entries, got {t.numel()}")
    elif tuple(t.shape) != (n, cols):
        raise ValueError(f"{name}: expected shape ({n}, {cols}), got {tuple(t.shape)}")


class CsrMatrix:
    """A CSR matrix on the GPU with its libhelm handle.  Holds references to
    the index and value tensors so they outlive the handle."""

    def __init__(self, rowptr, colind, vals, validate: bool = False, stream=None, sliced_only: bool = False):
        import torch
        _require_cuda(rowptr, colind, vals)
        if rowptr.dtype != torch.int32 or colind.dtype != torch.int32:
            raise TypeError("rowptr and colind must be int32")
        self.rowptr, self.colind, self.vals = rowptr, colind, vals
        self.n = rowptr.numel() - 1
        self.nnz = colind.numel()
        self.dtype = vals.dtype
        flags = (HELM_CSR_VALIDATE if validate else 0) | (HELM_CSR_SLICED_ONLY if sliced_only else 0)
        self.handle = helm_csr_create(self.n, self.nnz, _ptr(rowptr), _ptr(colind), _ptr(vals), _dtype_code(vals),
                                      flags, stream)

    @classmethod
    def from_host(cls, rowptr, colind, vals, device="cuda", validate: bool = False, sliced_only: bool = False):
        import torch
        return cls(torch.as_tensor(rowptr, dtype=torch.int32).to(device).contiguous(),
                   torch.as_tensor(colind, dtype=torch.int32).to(device).contiguous(),
                   torch.as_tensor(vals).to(device).contiguous(), validate=validate, sliced_only=sliced_only)

    def matvec(self, x, y=None, alpha=1.0, beta=0.0, stream=None):
        import torch
        _check_vector(x, self.n, self.dtype, "x")
        if y is None:
            y = torch.empty_like(x)
        _check_vector(y, self.n, self.dtype, "y")
        helm_spmv(self.handle, alpha, x, beta, y, stream)
        return y

    def diagonals(self) -> int:
        return helm_csr_diagonals(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            helm_csr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(A: CsrMatrix, b, x=None, stream=None, **opts):
    """x = A^{-1} b with BiCGStab (default options of helm_opts_default)."""
    import torch
    _check_vector(b, A.n, torch.complex128, "b")
    if x is None:
        x = torch.empty_like(b)
    _check_vector(x, A.n, torch.complex128, "x")
    info = helm_bicgstab_solve(A.handle, b, x, default_opts(**opts), stream)
    return x, info
