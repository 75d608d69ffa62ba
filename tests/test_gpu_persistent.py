"""The persistent form of the BiCGStab solve (one cooperative kernel, grid
barriers between the phases) against the graph form: both run the same
phases on the same rows of the same threads and add the same partial sums in
the same order, so every solve must agree bit for bit -- iterations,
restarts, statuses and x -- including restarts near rounding level, right
Jacobi, a warm start, ragged rows and the degenerate cases.  A deadline that
expires inside the kernel ends it with a timeout and leaves the context
usable."""
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


def _both(A, b, x0=None, **kw):
    """Solve with the graph and with the persistent kernel; return both."""
    out = []
    for launch in (helm.HELM_LAUNCH_GRAPH, helm.HELM_LAUNCH_PERSISTENT):
        x = torch.empty_like(b) if x0 is None else x0.clone()
        info = helm.helm_bicgstab_solve(A.handle, b, x, helm.default_opts(launch=launch, **kw))
        out.append((x, info))
    return out


def _assert_same(res):
    (xg, ig), (xp, ip) = res
    for k in ("status", "iters", "restarts", "spmv_count"):
        assert ig[k] == ip[k], (k, ig, ip)
    assert ig["relres_true"] == ip["relres_true"] and ig["relres_recur"] == ip["relres_recur"]
    assert torch.equal(torch.view_as_real(xg), torch.view_as_real(xp))


@pytest.mark.parametrize("name,kw", [
    ("box20", dict(tol=1e-8)),
    ("box20", dict(tol=1e-8, precond=helm.HELM_PRECOND_JACOBI)),
    ("box20_10ppw", dict(tol=1e-10)),
])
def test_persistent_matches_graph_bit_for_bit(name, kw):
    cfg = g.CONFIGS[name]
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    res = _both(A, _dev(g.source(p)), maxit=20000, **kw)
    assert res[0][1]["status"] == "ok", res[0][1]
    _assert_same(res)
    # the persistent result meets the oracle's gate on its own
    xg = res[1][0].cpu().numpy()
    r = np.linalg.norm(g.source(p) - oracle.spmv(p.rowptr, p.colind, vals, xg)) / np.linalg.norm(g.source(p))
    assert r <= kw["tol"] * (1 + 1e-6)
    A.close()


def test_persistent_warm_start_ragged_rows_and_restarts():
    """A random complex CSR with ragged rows (1 to 41 entries, a partial last
    slice), made diagonally dominant, with a warm start, and a tiny Helmholtz system at a tolerance near rounding level
    where the recurrence converges before the true residual does, so the
    solve restarts from x inside the kernel (the graph path restarts from the
    host)."""
    rp, ci, v = g.random_csr(1000, 40, seed=21, empty_row_frac=0.05)
    n = rp.size - 1
    d = np.zeros(n, complex)
    rows = np.repeat(np.arange(n), np.diff(rp))
    np.add.at(d, rows, np.abs(v))
    Ad = np.zeros((n, n), complex)
    Ad[rows, ci] += v
    Ad[np.arange(n), np.arange(n)] += d + 1.0
    rp2, ci2, v2 = _dense_to_csr(Ad)
    A = helm.CsrMatrix.from_host(rp2, ci2, v2, device=DEV)
    b = _dev(g.complex_vector(n, 22))
    x0 = _dev(0.01 * g.complex_vector(n, 23))
    res = _both(A, b, x0=x0, tol=1e-12, maxit=2000, use_x0=1)
    assert res[0][1]["status"] == "ok"
    _assert_same(res)
    A.close()

    restarted = 0
    for dims, F in (((8, 6, 5), 700.0), ((9, 7, 6), 900.0)):
        p = g.assemble(g.tiny_config(*dims, h=0.1, F=F, seed=2))
        vals = g.helmholtz_values(p, F)
        b = g.source(p) + 0.1 * g.complex_vector(p.n, 4) * (~p.dirichlet)
        A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
        for tol in (1e-13, 1e-15):
            res = _both(A, _dev(b), tol=tol, maxit=3000)
            _assert_same(res)
            info = res[1][1]
            if info["status"] == "ok":
                assert info["relres_true"] <= tol
            restarted += info["restarts"]
        A.close()
    assert restarted >= 1


def _dense_to_csr(D):
    rp = [0]
    ci, v = [], []
    for i in range(D.shape[0]):
        nz = np.nonzero(D[i])[0]
        ci.extend(nz.tolist())
        v.extend(D[i, nz].tolist())
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32), np.array(v, np.complex128)


def test_persistent_degenerate_cases():
    p = g.assemble(g.tiny_config(3, 3, 3, h=0.1, F=450.0, seed=5))
    vals = g.helmholtz_values(p, 450.0)
    b = g.source(p) + 0.2 * g.complex_vector(p.n, 6) * (~p.dirichlet)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    pers = dict(launch=helm.HELM_LAUNCH_PERSISTENT)
    zero = torch.zeros(p.n, dtype=torch.complex128, device=DEV)
    x = _dev(g.complex_vector(p.n, 1))
    info = helm.helm_bicgstab_solve(A.handle, zero, x, helm.default_opts(**pers))
    assert info["status"] == "ok" and info["iters"] == 0 and torch.all(x == 0)
    x, info = helm.solve(A, _dev(b), tol=1e-30, maxit=1, **pers)
    assert info["status"] == "not_converged" and info["iters"] == 1
    bad = b.copy()
    bad[4] = np.nan
    x, info = helm.solve(A, _dev(bad), **pers)
    assert info["status"] == "nonfinite"
    Z = helm.CsrMatrix.from_host(p.rowptr, p.colind, np.zeros_like(vals), device=DEV)
    x, info = helm.solve(Z, _dev(b), **pers)
    assert info["status"] == "breakdown"
    Z.close()
    for kw in (dict(tol=1e-30, maxit=7), dict(tol=1e-10, maxit=5000)):
        _assert_same(_both(A, _dev(b), **kw))
    A.close()


def test_persistent_deadline_returns_timeout():
    """Failure detection without a fault: the deadline is read by one block
    and carried to every block in the reduction that ends an iteration, so
    the whole grid stops together with a timeout; the next solve works."""
    p = g.assemble(g.CONFIGS["box20"])
    vals = g.helmholtz_values(p, 1500.0)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    pers = dict(launch=helm.HELM_LAUNCH_PERSISTENT)
    x, info = helm.solve(A, _dev(g.source(p)), tol=1e-12, maxit=20000, deadline_s=1e-9, **pers)
    assert info["status"] == "timeout" and info["iters"] == 1
    x, info = helm.solve(A, _dev(g.source(p)), tol=1e-6, maxit=20000, **pers)
    assert info["status"] == "ok"
    A.close()
