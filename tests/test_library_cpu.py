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
