"""GPU parity of the mixed-precision solve (complex64 inner BiCGStab inside
FP64 iterative refinement): the final residual is an FP64 true residual,
checked here again with the oracle's SpMV, and the solution meets the same
gate as the FP64 solver against a tight oracle / dense LU solution."""
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


def _true_relres(p, vals, b, x):
    return np.linalg.norm(b - oracle.spmv(p.rowptr, p.colind, vals, x)) / np.linalg.norm(b)


@pytest.mark.parametrize("dims,F", [((3, 3, 3), 300.0), ((8, 6, 5), 700.0)])
def test_mixed_vs_dense_lu(dims, F):
    cfg = g.tiny_config(*dims, h=0.1, F=F, seed=2)
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, F)
    b = g.source(p) + 0.1 * g.complex_vector(p.n, 4) * (~p.dirichlet)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x, info = helm.solve(A, _dev(b), tol=1e-10, precision=helm.HELM_PREC_MIXED, inner_tol=1e-4)
    assert info["status"] == "ok", info
    xg = x.cpu().numpy()
    r = _true_relres(p, vals, b, xg)
    assert r <= 1e-10 and abs(r - info["relres_true"]) <= 1e-3 * r + 1e-16
    xs = oracle.dense_solve(p.rowptr, p.colind, vals, b)
    assert np.linalg.norm(xg - xs) / np.linalg.norm(xs) <= 1e-8
    A.close()


def test_mixed_box20_against_tight_oracle():
    cfg = g.CONFIGS["box20"]
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    b = g.source(p)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x, info = helm.solve(A, _dev(b), tol=1e-10, maxit=200000, precision=helm.HELM_PREC_MIXED, inner_tol=1e-4)
    assert info["status"] == "ok", info
    xg = x.cpu().numpy()
    assert _true_relres(p, vals, b, xg) <= 1e-10
    x_t, _ = oracle.bicgstab(p.rowptr, p.colind, vals, b, tol=1e-13, maxit=60000)
    err = np.linalg.norm(xg - x_t) / np.linalg.norm(x_t)
    print(f"box20 mixed: inner iters {info['iters']}, refinement steps {info['restarts']}, error vs tight {err:.2e}")
    assert err <= 1e-8
    A.close()


def test_mixed_zero_rhs_and_bad_input():
    cfg = g.tiny_config(3, 3, 3)
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x, info = helm.solve(A, torch.zeros(p.n, dtype=torch.complex128, device=DEV), precision=helm.HELM_PREC_MIXED)
    assert info["status"] == "ok" and torch.all(x == 0)
    bad = g.source(p)
    bad[5] = np.inf
    x, info = helm.solve(A, _dev(bad), precision=helm.HELM_PREC_MIXED)
    assert info["status"] == "nonfinite"
    A.close()
