"""CPU oracle for the Helmholtz Krylov hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package.  The product library (paper_2112_11880_gb300) never
imports it, and this package never imports the product library: the two share
no code.  Inputs come from `helmgen`, the seeded generator both sides use.

The compiled part (helm_oracle.cpp) holds the sequential C++ SpMV, zdotc,
norm and BiCGStab.  This module adds the numpy-level pieces that are plain
definitions: forming A(w) = K - w^2 M_c + i w B_c for a frequency, dense
solves on tiny meshes, and the adjoint sound-speed gradient chain.

Parity pins for every function here are in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "helm_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "libhelm_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", 1: "invalid", 4: "not_converged", 5: "breakdown", 7: "nonfinite"}


_OMP_PATH = os.path.join(_HERE, "_build", "libhelm_oracle_omp.so")
_omp_lib = None


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with g++ -O2 (no fast-math) if it is missing or stale.
    openmp: the all-core build of the same source for the benchmark's CPU
    baseline (-fopenmp; the tests use the sequential build only)."""
    path = _OMP_PATH if openmp else _LIB_PATH
    os.makedirs(os.path.dirname(path), exist_ok=True)
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared"] + (["-fopenmp"] if openmp else [])
                          + ["-o", tmp, _SRC])
    os.replace(tmp, path)
    return path


def _load(openmp: bool = False):
    global _lib, _omp_lib
    with _lock:
        if (_omp_lib if openmp else _lib) is None:
            lib = ctypes.CDLL(build(openmp=openmp))
            P = ctypes.c_void_p
            lib.oracle_spmv.argtypes = [ctypes.c_int32, P, P, P, P, P]
            lib.oracle_spmv.restype = None
            lib.oracle_zdotc.argtypes = [ctypes.c_int64, P, P, P]
            lib.oracle_zdotc.restype = None
            lib.oracle_dznrm2.argtypes = [ctypes.c_int64, P]
            lib.oracle_dznrm2.restype = ctypes.c_double
            lib.oracle_bicgstab.argtypes = [ctypes.c_int32, P, P, P, P, P, ctypes.c_double,
                                            ctypes.c_int32, ctypes.c_int, P, P, P]
            lib.oracle_bicgstab.restype = ctypes.c_int
            lib.oracle_tfqmr.argtypes = lib.oracle_bicgstab.argtypes
            lib.oracle_tfqmr.restype = ctypes.c_int
            lib.oracle_bicgstabl.argtypes = [ctypes.c_int32, P, P, P, P, P, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int32, ctypes.c_int, P, P, P]
            lib.oracle_bicgstabl.restype = ctypes.c_int
            if openmp:
                _omp_lib = lib
            else:
                _lib = lib
    return _omp_lib if openmp else _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def spmv(rowptr, colind, vals, x) -> np.ndarray:
    """y = A x for complex128 CSR (sequential, CSR order)."""
    lib = _load()
    n = len(rowptr) - 1
    rp, prp = _c(rowptr, np.int32)
    ci, pci = _c(colind, np.int32)
    v, pv = _c(vals, np.complex128)
    xx, px = _c(x, np.complex128)
    y = np.empty(n, dtype=np.complex128)
    lib.oracle_spmv(n, prp, pci, pv, px, y.ctypes.data_as(ctypes.c_void_p))
    return y


def zdotc(x, y) -> complex:
    """(x, y) = sum conj(x_i) y_i with Neumaier-compensated sums."""
    lib = _load()
    xx, px = _c(x, np.complex128)
    yy, py = _c(y, np.complex128)
    if xx.size != yy.size:
        raise ValueError("length mismatch")
    out = np.zeros(2)
    lib.oracle_zdotc(xx.size, px, py, out.ctypes.data_as(ctypes.c_void_p))
    return complex(out[0], out[1])


def dznrm2(x) -> float:
    lib = _load()
    xx, px = _c(x, np.complex128)
    return float(lib.oracle_dznrm2(xx.size, px))


def bicgstab(rowptr, colind, vals, b, tol=1e-8, maxit=20000, x0=None, openmp=False):
    """Textbook BiCGStab; returns (x, info dict).  openmp: run the all-core
    build (benchmark baseline only)."""
    return _krylov("oracle_bicgstab", rowptr, colind, vals, b, tol, maxit, x0, openmp=openmp)


def tfqmr(rowptr, colind, vals, b, tol=1e-8, maxit=20000, x0=None):
    """Transpose-free QMR (Saad 2003, Algorithm 7.8); returns (x, info dict)."""
    return _krylov("oracle_tfqmr", rowptr, colind, vals, b, tol, maxit, x0)


def bicgstabl(rowptr, colind, vals, b, ell=2, tol=1e-8, maxit=20000, x0=None):
    """BiCGStab(l) (Sleijpen & Fokkema 1993); one iteration = one outer cycle."""
    return _krylov("oracle_bicgstabl", rowptr, colind, vals, b, tol, maxit, x0, ell=ell)


def _krylov(fname, rowptr, colind, vals, b, tol, maxit, x0, ell=None, openmp=False):
    lib = _load(openmp)
    n = len(rowptr) - 1
    rp, prp = _c(rowptr, np.int32)
    ci, pci = _c(colind, np.int32)
    v, pv = _c(vals, np.complex128)
    bb, pb = _c(b, np.complex128)
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    rt = ctypes.c_double(0.0)
    head = (n, prp, pci, pv, pb, x.ctypes.data_as(ctypes.c_void_p))
    if ell is not None:
        head = head + (int(ell),)
    st = getattr(lib, fname)(*head, float(tol), int(maxit), 0 if x0 is None else 1, ctypes.byref(it),
                             ctypes.byref(rr), ctypes.byref(rt))
    return x, {"status": STATUS.get(st, st), "iters": it.value, "relres_recur": rr.value,
               "relres_true": rt.value}


# ---------------------------------------------------------------------------
# numpy-level definitions
# ---------------------------------------------------------------------------

def jacobi_scale(rowptr, colind, vals):
    """Right Jacobi preconditioning written out (the paper's P- solvers, Section 4,
    with the diagonal as the preconditioner): D = diag(A), a row without a stored
    nonzero diagonal taking 1; returns (values of A D^-1, d, 1/d).  Solving
    (A D^-1) y = b and setting x = D^-1 y solves A x = b."""
    rowptr = np.asarray(rowptr)
    colind = np.asarray(colind)
    vals = np.asarray(vals, dtype=np.complex128)
    n = len(rowptr) - 1
    d = np.ones(n, dtype=np.complex128)
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            if colind[k] == i:
                if vals[k] != 0 and np.isfinite(vals[k]):
                    d[i] = vals[k]
                break
    dinv = 1.0 / d
    return vals * dinv[colind], d, dinv


def jacobi_solve(method, rowptr, colind, vals, b, **kw):
    """x = D^-1 y with y from `method` (bicgstab, tfqmr, bicgstabl) on A D^-1."""
    vs, d, dinv = jacobi_scale(rowptr, colind, vals)
    x0 = kw.pop("x0", None)
    y0 = None if x0 is None else d * np.asarray(x0, dtype=np.complex128)
    y, info = method(rowptr, colind, vs, b, x0=y0, **kw)
    return dinv * y, info


def ddm_blocks(n: int, nsub: int, overlap: int):
    """The decomposition of helm_ddm_create written out: owned blocks
    [p n / nsub, (p + 1) n / nsub) and their extensions by `overlap` rows on
    both sides, clamped to [0, n).  Returns [(s, e, a, b)]."""
    out = []
    for p in range(nsub):
        s, e = p * n // nsub, (p + 1) * n // nsub
        out.append((s, e, max(0, s - overlap), min(n, e + overlap)))
    return out


def ras_apply(rowptr, colind, vals, r, nsub: int, overlap: int, impedance: bool = False) -> np.ndarray:
    """Restricted additive Schwarz (Cai & Sarkis 1999) by its definition,
    z = sum_p Rt_p^T A_p^{-1} R_p r, with A_p the principal submatrix of A on
    the extended block p (dense LAPACK solves; small matrices only) and Rt_p^T
    keeping the rows block p owns.  impedance: A_p's rows that couple to rows
    outside the block get i sum_{j outside} |a_ij| on their diagonal (an
    absorbing condition on the artificial boundary)."""
    Ad = densify(rowptr, colind, vals)
    n = Ad.shape[0]
    r = np.asarray(r, dtype=np.complex128)
    z = np.zeros(n, dtype=np.complex128)
    for s, e, a, b in ddm_blocks(n, nsub, overlap):
        Ap = Ad[a:b, a:b].copy()
        if impedance:
            lost = np.abs(Ad[a:b, :a]).sum(axis=1) + np.abs(Ad[a:b, b:]).sum(axis=1)
            Ap[np.arange(b - a), np.arange(b - a)] += 1j * lost
        y = np.linalg.solve(Ap, r[a:b])
        z[s:e] = y[s - a:e - a]
    return z


def helmholtz_values(K, Mc, Bc, w: float) -> np.ndarray:
    """A(w) = K - w^2 M_c + i w B_c entry by entry (the frequency-dependent
    system of the Helmholtz problem of Section 1 with the impedance term)."""
    K = np.asarray(K, dtype=np.float64)
    return (K - (w * w) * np.asarray(Mc)) + 1j * (w * np.asarray(Bc))


def densify(rowptr, colind, vals, ncols=None) -> np.ndarray:
    n = len(rowptr) - 1
    D = np.zeros((n, n if ncols is None else ncols), dtype=np.complex128)
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            D[i, colind[k]] += vals[k]
    return D


def dense_solve(rowptr, colind, vals, b) -> np.ndarray:
    """LAPACK zgesv on the densified matrix (tiny meshes only)."""
    return np.linalg.solve(densify(rowptr, colind, vals), np.asarray(b, dtype=np.complex128))


def loss(u, receivers, d) -> float:
    """L = sum over receivers of |u_r - d_r|^2."""
    e = np.asarray(u)[receivers] - np.asarray(d)
    return float(np.sum(e.real ** 2 + e.imag ** 2))


def adjoint_rhs(n, u, receivers, d) -> np.ndarray:
    """w = dL/du in the holomorphic sense: w_r = conj(u_r - d_r) on receivers."""
    w = np.zeros(n, dtype=np.complex128)
    w[receivers] = np.conj(np.asarray(u)[receivers] - np.asarray(d))
    return w


def nnz_gradient(rowptr, colind, mu, u) -> np.ndarray:
    """G_k = -mu_i u_j for CSR slot k = (i, j): dL/dA_ij for L real, u = A^-1 b
    and A^T mu = dL/du (A = A^T here)."""
    rows = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    return -np.asarray(mu)[rows] * np.asarray(u)[np.asarray(colind)]


def sound_speed_gradient(G, elem_map, Me, Bf, c, w, top) -> np.ndarray:
    """dL/dc_e = 2 Re sum_{a,b} G[map[e,a,b]] dA_ab/dc_e with
    dA/dc_e = (2 w^2 / c_e^3) M_e - i (w / c_e^2) B_f (B_f only on top elements).
    Slots eliminated by the Dirichlet condition (map = -1) do not depend on c."""
    E = elem_map.shape[0]
    grad = np.zeros(E)
    Gm = np.where(elem_map >= 0, np.asarray(G)[np.maximum(elem_map, 0)], 0.0)   # [E, 64]
    c = np.asarray(c, dtype=np.float64)
    dM = (2.0 * w * w / c ** 3)[:, None] * Me.reshape(1, 64)
    dB = np.where(np.asarray(top)[:, None], (w / c ** 2)[:, None] * Bf.reshape(1, 64), 0.0)
    dA = dM - 1j * dB
    grad = 2.0 * np.real(np.sum(Gm * dA, axis=1))
    return grad
