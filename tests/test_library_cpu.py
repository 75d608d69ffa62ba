"""CPU-side checks of the C-ABI library: it builds, loads without a GPU and
exports every function include/helm.h declares.  No compute calls."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(helm_\w+)\s*\(", txt, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2112_11880_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["helm_csr_create", "helm_csr_destroy", "helm_spmv", "helm_dot", "helm_axpby",
                     "helm_bicgstab_solve", "helm_adjoint", "helm_status_string"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    cdll, path = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (helm_\w+)", out))
    missing = _declared() - exported
    assert not missing, missing
    for name in _declared():
        getattr(cdll, name)   # resolvable through dlsym


def test_binding_signatures_cover_header():
    import paper_2112_11880_gb300 as h
    assert _declared() <= set(h.SIGNATURES)


def test_host_only_entry_points(lib):
    import paper_2112_11880_gb300 as h
    assert h.helm_status_string(h.HELM_ERR_NOT_CONVERGED).startswith("iteration cap")
    assert h.helm_status_string(99) == "unknown status"
    o = h.default_opts()
    assert o.tol == 1e-8 and o.maxit == 20000 and o.method == h.HELM_BICGSTAB


def test_product_package_does_not_reach_the_oracle():
    pkg = os.path.join(ROOT, "paper_2112_11880_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".hpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", txt).lower() or f.endswith(".md"), f


def test_convenience_layer_checks_vectors_before_the_call():
    """The C ABI takes bare device pointers, so a short or mistyped vector
    would be read or written out of bounds on the device: the Python
    convenience layer rejects it before anything reaches the library."""
    torch = pytest.importorskip("torch")
    import paper_2112_11880_gb300 as h
    A = object.__new__(h.CsrMatrix)
    A.n, A.dtype, A.handle = 5, torch.complex128, None
    ok = torch.zeros(5, dtype=torch.complex128)
    with pytest.raises(ValueError, match="expected 5 entries"):
        h.solve(A, torch.zeros(4, dtype=torch.complex128))
    with pytest.raises(TypeError, match="complex128"):
        h.solve(A, torch.zeros(5, dtype=torch.complex64))
    with pytest.raises(ValueError, match="x: expected 5 entries"):
        h.solve(A, ok, x=torch.zeros(6, dtype=torch.complex128))
    with pytest.raises(TypeError):
        A.matvec(torch.zeros(5, dtype=torch.complex64))
    with pytest.raises(ValueError, match="y: expected 5 entries"):
        A.matvec(ok, torch.zeros(3, dtype=torch.complex128))
    S = object.__new__(h.Sweep)
    S.n, S.handle = 5, None
    with pytest.raises(ValueError, match=r"b: expected shape \(5, 2\)"):
        S.solve([1.0, 2.0], torch.zeros(5, 3, dtype=torch.complex128))
    with pytest.raises(ValueError, match=r"X: expected shape \(5, 2\)"):
        S.solve([1.0, 2.0], ok, X=torch.zeros(5, 3, dtype=torch.complex128))
    with pytest.raises(ValueError, match="b: expected 5 entries"):
        S.solve([1.0, 2.0], torch.zeros(4, dtype=torch.complex128))
    h._check_vector(torch.zeros(5, 2, dtype=torch.complex128), 5, torch.complex128, "X", 2)
