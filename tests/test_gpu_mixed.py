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


@pytest.mark.parametrize("e", [-100, 100])
def test_mixed_is_scale_invariant(e):
    """A right-hand side scaled by 2^e (exact in FP64) gives the solution scaled
    by 2^e.  Run in the problem's own scale, the complex64 recurrence would
    underflow (2^-100: squared entries ~1e-68) or overflow (2^100: ~1e52)."""
    cfg = g.CONFIGS["box20"]
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    b = g.source(p)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x1, i1 = helm.solve(A, _dev(b), tol=1e-10, maxit=200000, precision=helm.HELM_PREC_MIXED)
    xs, i2 = helm.solve(A, _dev(np.ldexp(b.real, e) + 1j * np.ldexp(b.imag, e)), tol=1e-10, maxit=200000,
                        precision=helm.HELM_PREC_MIXED)
    assert i1["status"] == "ok" and i2["status"] == "ok", (i1, i2)
    x1, xs = x1.cpu().numpy(), xs.cpu().numpy()
    xs = np.ldexp(xs.real, -e) + 1j * np.ldexp(xs.imag, -e)
    assert np.linalg.norm(xs - x1) <= 1e-8 * np.linalg.norm(x1)
    A.close()


def test_mixed_warm_start():
    """x0 = a perturbed solution: the residual replacement starts from b - A x0."""
    cfg = g.tiny_config(8, 6, 5, h=0.1, F=700.0, seed=2)
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    b = g.source(p)
    xs = oracle.dense_solve(p.rowptr, p.colind, vals, b)
    x0 = xs + 1e-3 * np.linalg.norm(xs) / np.sqrt(p.n) * g.complex_vector(p.n, 9) * (~p.dirichlet)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x = _dev(x0)
    opts = helm.default_opts(tol=1e-11, maxit=20000, precision=helm.HELM_PREC_MIXED, use_x0=1)
    info = helm.helm_bicgstab_solve(A.handle, _dev(b), x, opts)
    assert info["status"] == "ok", info
    assert np.linalg.norm(x.cpu().numpy() - xs) <= 1e-9 * np.linalg.norm(xs)
    A.close()


@pytest.mark.parametrize("name", ["cavity120", "cavity200"])
def test_mixed_full_size_to_1e10(name):
    """The full-size cavities (376,431 and 1,644,381 unknowns) to 1e-10 with
    the default inner tolerance: status ok, the FP64 true residual recomputed
    on the host (scipy, from the generator's matrix) at most 1e-10 and equal
    to the reported one, and the solution gate against a tight FP64 solve
    (1e-12): ||x_mixed - x_tight|| <= max(1e-8, 2 ||x_fp64 - x_tight||) with
    x_fp64 the FP64 solve at the same 1e-10.  The error of the mixed solution
    against the FP64 one is printed."""
    import scipy.sparse as sp
    cfg = g.CONFIGS[name]
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    b = g.source(p)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    bd = _dev(b)
    x32, i32 = helm.solve(A, bd, tol=1e-10, maxit=400000, precision=helm.HELM_PREC_MIXED, deadline_s=400.0)
    assert i32["status"] == "ok", i32
    x64, i64 = helm.solve(A, bd, tol=1e-10, maxit=300000, deadline_s=400.0)
    assert i64["status"] == "ok", i64
    xt, it = helm.solve(A, bd, tol=1e-12, maxit=400000, deadline_s=400.0)
    assert it["status"] == "ok", it
    A.close()
    Ah = sp.csr_matrix((vals, p.colind, p.rowptr), shape=(p.n, p.n))
    xm = x32.cpu().numpy()
    r = float(np.linalg.norm(b - Ah @ xm) / np.linalg.norm(b))
    assert r <= 1e-10 * (1 + 1e-6) and abs(r - i32["relres_true"]) <= 1e-3 * r
    xt = xt.cpu().numpy()
    nt = np.linalg.norm(xt)
    e_m = np.linalg.norm(xm - xt) / nt
    e_f = np.linalg.norm(x64.cpu().numpy() - xt) / nt
    e_mf = np.linalg.norm(xm - x64.cpu().numpy()) / np.linalg.norm(x64.cpu().numpy())
    print(f"{name} mixed: {i32['iters']} complex64 iterations in {i32['restarts']} refinement steps; FP64 "
          f"{i64['iters']} iterations; error vs tight {e_m:.2e} (FP64 at 1e-10: {e_f:.2e}); vs FP64 {e_mf:.2e}")
    assert e_m <= max(1e-8, 2 * e_f), (e_m, e_f)
