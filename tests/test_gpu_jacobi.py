"""GPU parity of the right-Jacobi preconditioned solvers (the paper's P-
solvers with the diagonal as preconditioner) against dense LU and the
oracle's Jacobi solve: same iteration counts within the rounding-order
spread, solutions at the FP64 solver gates, the reported residual that of
A x = b itself, warm starts, and the argument checks."""
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
METHODS = {"bicgstab": (helm.HELM_BICGSTAB, oracle.bicgstab), "tfqmr": (helm.HELM_TFQMR, oracle.tfqmr),
           "bicgstabl": (helm.HELM_BICGSTABL, oracle.bicgstabl)}


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def _relres(p, vals, b, x):
    return np.linalg.norm(b - oracle.spmv(p.rowptr, p.colind, vals, x)) / np.linalg.norm(b)


@pytest.mark.parametrize("method", list(METHODS))
@pytest.mark.parametrize("dims,F", [((3, 3, 3), 300.0), ((8, 6, 5), 700.0)])
def test_jacobi_vs_dense_lu(method, dims, F):
    cfg = g.tiny_config(*dims, h=0.1, F=F, seed=2)
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, F)
    b = g.source(p) + 0.1 * g.complex_vector(p.n, 4) * (~p.dirichlet)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x, info = helm.solve(A, _dev(b), tol=1e-11, maxit=20000, method=METHODS[method][0],
                         precond=helm.HELM_PRECOND_JACOBI)
    assert info["status"] == "ok", info
    xg = x.cpu().numpy()
    r = _relres(p, vals, b, xg)
    assert r <= 1e-11 * (1 + 1e-6) and abs(r - info["relres_true"]) <= 1e-3 * r + 1e-16
    xs = oracle.dense_solve(p.rowptr, p.colind, vals, b)
    cond = np.linalg.cond(oracle.densify(p.rowptr, p.colind, vals))
    assert np.linalg.norm(xg - xs) / np.linalg.norm(xs) <= max(1e-8, 10 * cond * 1e-11)
    A.close()


def test_jacobi_box20_10ppw_against_oracle():
    cfg = g.CONFIGS["box20_10ppw"]
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    b = g.source(p)
    x_o, i_o = oracle.jacobi_solve(oracle.bicgstab, p.rowptr, p.colind, vals, b, tol=cfg.tol, maxit=20000)
    x_t, _ = oracle.bicgstab(p.rowptr, p.colind, vals, b, tol=1e-13, maxit=60000)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x, info = helm.solve(A, _dev(b), tol=cfg.tol, maxit=20000, precond=helm.HELM_PRECOND_JACOBI)
    assert info["status"] == "ok", info
    xg = x.cpu().numpy()
    print(f"box20_10ppw Jacobi: gpu iters {info['iters']} oracle iters {i_o['iters']}")
    assert abs(info["iters"] - i_o["iters"]) <= max(5, 0.1 * i_o["iters"])
    assert _relres(p, vals, b, xg) <= cfg.tol * (1 + 1e-6)
    e_g = np.linalg.norm(xg - x_t) / np.linalg.norm(x_t)
    e_o = np.linalg.norm(x_o - x_t) / np.linalg.norm(x_t)
    assert e_g <= max(1e-8, 2 * e_o)
    A.close()


def test_jacobi_warm_start_and_missing_diagonal():
    # warm start: x0 near the solution converges in few iterations to the same answer
    cfg = g.tiny_config(8, 6, 5, h=0.1, F=700.0, seed=2)
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    b = g.source(p)
    xs = oracle.dense_solve(p.rowptr, p.colind, vals, b)
    x0 = xs + 1e-4 * np.linalg.norm(xs) / np.sqrt(p.n) * g.complex_vector(p.n, 9) * (~p.dirichlet)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x = _dev(x0)
    info = helm.helm_bicgstab_solve(A.handle, _dev(b), x,
                                    helm.default_opts(tol=1e-11, use_x0=1, precond=helm.HELM_PRECOND_JACOBI))
    assert info["status"] == "ok"
    assert np.linalg.norm(x.cpu().numpy() - xs) <= 1e-8 * np.linalg.norm(xs)
    cold = helm.solve(A, _dev(b), tol=1e-11, precond=helm.HELM_PRECOND_JACOBI)[1]
    assert info["iters"] < cold["iters"]
    A.close()
    # a row that stores no diagonal keeps scale 1
    rowptr = np.array([0, 2, 4, 6], np.int32)
    colind = np.array([0, 2, 0, 2, 1, 2], np.int32)
    v = np.array([2.0, 1.0, 1.0, 3.0, 4.0, 5.0 + 1j], np.complex128)
    bb = np.array([1.0, 2.0, 3.0 - 1j])
    A = helm.CsrMatrix.from_host(rowptr, colind, v, device=DEV)
    x, info = helm.solve(A, _dev(bb), tol=1e-13, maxit=100, precond=helm.HELM_PRECOND_JACOBI)
    assert info["status"] == "ok"
    assert np.allclose(x.cpu().numpy(), np.linalg.solve(oracle.densify(rowptr, colind, v), bb), rtol=1e-11)
    A.close()


def test_jacobi_argument_checks():
    p = g.assemble(g.tiny_config(3, 3, 3))
    vals = g.helmholtz_values(p, 200.0)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    b = _dev(g.source(p))
    with pytest.raises(helm.HelmError):
        helm.solve(A, b, precision=helm.HELM_PREC_MIXED, precond=helm.HELM_PRECOND_JACOBI)
    with pytest.raises(helm.HelmError):
        helm.solve(A, b, precond=7)
    A.close()
