"""Schwarz domain decomposition with the subdomain solves batched on one GPU
(helm_ddm_*): the block-diagonal matrix of the principal submatrices, the
restricted additive Schwarz operator against the oracle's definition of it
(dense solves of the same blocks), and the preconditioned GCR solve against
the oracle's BiCGStab under the solution gate (true residual <= tol;
||x - x_tight|| <= max(1e-8, 2 ||x_oracle - x_tight||))."""
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


def _problem(dims, F, seed):
    p = g.assemble(g.tiny_config(*dims, h=0.1, F=F, seed=seed))
    vals = g.helmholtz_values(p, F)
    return p, vals


@pytest.mark.parametrize("impedance", [False, True])
@pytest.mark.parametrize("nsub,planes", [(1, 0), (2, 1), (3, 2), (5, 1)])
def test_ddm_blocks_and_ras_against_the_oracle(nsub, planes, impedance):
    """D holds exactly the entries of the principal submatrices of the
    extended blocks (rows and entries counted from the oracle's
    decomposition), and M r with a tight inner solve equals the oracle's
    sum_p Rt_p^T A_p^-1 R_p r, with and without the impedance term."""
    dims = (6, 5, 7)
    p, vals = _problem(dims, 650.0, 3)
    plane = (dims[0] + 1) * (dims[1] + 1)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    S = helm.Ddm(A, nsub, planes * plane, impedance=impedance)
    rows, nnz = S.subdomains()
    blocks = oracle.ddm_blocks(p.n, nsub, planes * plane)
    Ad = oracle.densify(p.rowptr, p.colind, vals)
    assert rows == sum(b - a for _, _, a, b in blocks)
    rowof = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    assert nnz == sum(int(np.count_nonzero((rowof >= a) & (rowof < b) & (p.colind >= a) & (p.colind < b)))
                      for _, _, a, b in blocks)
    r = g.complex_vector(p.n, 17) * (~p.dirichlet)
    z = S.apply(_dev(r), inner_tol=1e-13).cpu().numpy()
    ref = oracle.ras_apply(p.rowptr, p.colind, vals, r, nsub, planes * plane, impedance=impedance)
    # the batched inner solve ends at ||R r - D y|| <= 1e-13 ||R r||: each block's
    # error is A_p^-1 times its share of that residual
    def block(a, b):
        Ap = Ad[a:b, a:b].copy()
        if impedance:
            lost = np.abs(Ad[a:b, :a]).sum(axis=1) + np.abs(Ad[a:b, b:]).sum(axis=1)
            Ap[np.arange(b - a), np.arange(b - a)] += 1j * lost
        return Ap
    inv_norm = max(1.0 / np.linalg.svd(block(a, b), compute_uv=False)[-1] for _, _, a, b in blocks)
    rd = np.sqrt(sum(np.linalg.norm(r[a:b]) ** 2 for _, _, a, b in blocks))
    assert np.linalg.norm(z - ref) <= 10 * 1e-13 * inv_norm * rd
    if nsub == 1:
        xs = oracle.dense_solve(p.rowptr, p.colind, vals, r)
        assert np.linalg.norm(z - xs) <= 10 * 1e-13 * inv_norm * rd
    S.close()
    A.close()


@pytest.mark.parametrize("name,nsub,planes,inner_tol", [("box20", 2, 2, 1e-3), ("box20", 4, 1, 1e-3),
                                                         ("box20_10ppw", 4, 2, 1e-2)])
def test_ddm_solve_box20(name, nsub, planes, inner_tol):
    """The 20^3 box (4.5 and 10 points per wavelength) in 2 or 4 slabs with
    the impedance term, GCR over 256 directions, to 1e-8."""
    cfg = g.CONFIGS[name]
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    b = g.source(p)
    plane = (cfg.nx + 1) * (cfg.ny + 1)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    S = helm.Ddm(A, nsub, planes * plane, window=256)
    x, info = S.solve(_dev(b), tol=1e-8, maxit=1000, inner_tol=inner_tol)
    assert info["status"] == "ok", info
    xg = x.cpu().numpy()
    r = np.linalg.norm(b - oracle.spmv(p.rowptr, p.colind, vals, xg)) / np.linalg.norm(b)
    assert r <= 1e-8 * (1 + 1e-6) and abs(r - info["relres_true"]) <= 1e-3 * r
    xo, _ = oracle.bicgstab(p.rowptr, p.colind, vals, b, tol=1e-8, maxit=20000)
    xt, _ = oracle.bicgstab(p.rowptr, p.colind, vals, b, tol=1e-13, maxit=60000)
    nt = np.linalg.norm(xt)
    e_g, e_o = np.linalg.norm(xg - xt) / nt, np.linalg.norm(xo - xt) / nt
    print(f"{name} ddm nsub={nsub} overlap={planes} planes: {info['iters']} outer steps, "
          f"{(info['spmv_count'] - info['iters']) // 2} inner iterations; error {e_g:.2e} (oracle {e_o:.2e})")
    assert e_g <= max(1e-8, 2 * e_o)
    # a warm start from the solution ends at once
    x2, info2 = S.solve(_dev(b), x=x.clone(), tol=1e-8, maxit=1000, inner_tol=inner_tol, use_x0=1)
    assert info2["status"] == "ok" and info2["iters"] == 0
    S.close()
    A.close()


def test_ddm_degenerate_cases():
    p, vals = _problem((4, 3, 5), 400.0, 5)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    for nsub, ov, w in ((0, 1, 8), (p.n + 1, 0, 8), (2, -1, 8), (2, 1, 0), (2, 1, 513)):
        with pytest.raises(helm.HelmError):
            helm.Ddm(A, nsub, ov, window=w)
    S = helm.Ddm(A, 3, 10, window=64)
    zero = torch.zeros(p.n, dtype=torch.complex128, device=DEV)
    x, info = S.solve(zero, x=_dev(g.complex_vector(p.n, 1)))
    assert info["status"] == "ok" and torch.all(x == 0)
    b = _dev(g.source(p) + 0.2 * g.complex_vector(p.n, 6) * (~p.dirichlet))
    x, info = S.solve(b, tol=1e-14, maxit=1)
    assert info["status"] == "not_converged" and info["iters"] == 1
    bad = b.clone()
    bad[3] = complex("nan")
    x, info = S.solve(bad)
    assert info["status"] == "nonfinite"
    x, info = S.solve(b, tol=1e-12, maxit=100)
    assert info["status"] == "ok" and info["relres_true"] <= 1e-12
    S.close()
    A.close()
