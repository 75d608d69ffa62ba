"""GPU parity of TFQMR (method = HELM_TFQMR) against dense LU, the oracle's
TFQMR and its degenerate cases."""
import numpy as np
import pytest

import helmgen as g
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2112_11880_gb300 as helm  # noqa: E402

DEV = torch.device("cuda:0")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


@pytest.mark.parametrize("dims,F", [((2, 2, 2), 300.0), ((5, 4, 3), 450.0), ((9, 7, 6), 900.0)])
def test_tfqmr_vs_dense_lu(dims, F):
    cfg = g.tiny_config(*dims, h=0.1, F=F, seed=3)
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, F)
    b = g.source(p) + 0.2 * g.complex_vector(p.n, 4) * (~p.dirichlet)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x, info = helm.solve(A, _dev(b), tol=1e-12, maxit=10000, method=helm.HELM_TFQMR)
    assert info["status"] == "ok", info
    xg = x.cpu().numpy()
    res = np.linalg.norm(b - oracle.spmv(p.rowptr, p.colind, vals, xg)) / np.linalg.norm(b)
    assert res <= 1e-12 * (1 + 1e-6)
    xs = oracle.dense_solve(p.rowptr, p.colind, vals, b)
    xo, _ = oracle.tfqmr(p.rowptr, p.colind, vals, b, tol=1e-12, maxit=10000)
    e_g = np.linalg.norm(xg - xs) / np.linalg.norm(xs)
    e_o = np.linalg.norm(xo - xs) / np.linalg.norm(xs)
    assert e_g <= max(1e-8, 2 * e_o)
    A.close()


def test_tfqmr_box20_parity():
    cfg = g.CONFIGS["box20"]
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    b = g.source(p)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x, info = helm.solve(A, _dev(b), tol=1e-8, maxit=20000, method=helm.HELM_TFQMR)
    assert info["status"] == "ok", info
    xg = x.cpu().numpy()
    res = np.linalg.norm(b - oracle.spmv(p.rowptr, p.colind, vals, xg)) / np.linalg.norm(b)
    assert res <= 1e-8 * (1 + 1e-6)
    xo, io = oracle.tfqmr(p.rowptr, p.colind, vals, b, tol=1e-8, maxit=20000)
    x_t, _ = oracle.bicgstab(p.rowptr, p.colind, vals, b, tol=1e-13, maxit=60000)
    nt = np.linalg.norm(x_t)
    e_g = np.linalg.norm(xg - x_t) / nt
    e_o = np.linalg.norm(xo - x_t) / nt
    print(f"box20 TFQMR: gpu iters {info['iters']} oracle iters {io['iters']}, err {e_g:.2e} vs {e_o:.2e}")
    assert e_g <= max(1e-8, 2 * e_o)
    assert abs(info["iters"] - io["iters"]) <= 0.05 * io["iters"] + 2
    A.close()


def test_tfqmr_degenerate_cases():
    cfg = g.tiny_config(3, 3, 3, h=0.1, F=450.0, seed=5)
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    b = g.source(p) + 0.2 * g.complex_vector(p.n, 6) * (~p.dirichlet)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    o = dict(method=helm.HELM_TFQMR)
    x, info = helm.solve(A, torch.zeros(p.n, dtype=torch.complex128, device=DEV), **o)
    assert info["status"] == "ok" and info["iters"] == 0 and torch.all(x == 0)
    x, info = helm.solve(A, _dev(b), tol=1e-30, maxit=1, **o)
    assert info["status"] == "not_converged" and info["iters"] == 1
    bad = b.copy()
    bad[3] = np.nan
    assert helm.solve(A, _dev(bad), **o)[1]["status"] == "nonfinite"
    x, info = helm.solve(A, _dev(b), tol=1e-12, maxit=20000, deadline_s=1e-9, **o)
    assert info["status"] == "timeout"
    A.close()
