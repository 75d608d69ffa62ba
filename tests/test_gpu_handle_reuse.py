"""One CSR handle serving many solves: the handle caches a CUDA graph per
(b, x, variant) and grows its vector workspace on demand (dropping the
graphs that captured the old buffers).  Every variant must keep its own graph,
and a repeated solve must return the same bits as the first one, whatever
ran on the handle in between."""
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


def _relres(p, vals, b, x):
    return np.linalg.norm(b - oracle.spmv(p.rowptr, p.colind, vals, x)) / np.linalg.norm(b)


def _problem():
    cfg = g.tiny_config(8, 6, 5, h=0.1, F=700.0, seed=4)
    p = g.assemble(cfg)
    return p, g.helmholtz_values(p, cfg.F)


def test_graph_cache_keeps_variants_apart_on_neighbouring_vectors():
    """b1 = buf[0:n] and b2 = buf[1:n+1] are 16 bytes apart.  A Jacobi solve on
    b1 and a plain solve on b2 into the same x are different graphs: the plain
    one must solve A x = b2 (oracle residual), and repeating either returns
    its first bits."""
    p, vals = _problem()
    n = p.n
    buf_h = np.concatenate([g.source(p), [0.0]]) + 0.1 * g.complex_vector(n + 1, 5)
    buf = torch.as_tensor(buf_h, device=DEV)
    b1, b2 = buf[0:n], buf[1:n + 1]
    assert b2.data_ptr() - b1.data_ptr() == 16
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x = torch.empty(n, dtype=torch.complex128, device=DEV)
    runs = [(b1, buf_h[0:n], dict(precond=helm.HELM_PRECOND_JACOBI)), (b2, buf_h[1:n + 1], dict())]
    first = []
    for rep in range(2):
        for k, (bt, bh, kw) in enumerate(runs):
            _, info = helm.solve(A, bt, x=x, tol=1e-10, maxit=5000, **kw)
            assert info["status"] == "ok", (k, info)
            xh = x.cpu().numpy()
            assert _relres(p, vals, bh, xh) <= 1e-10 * (1 + 1e-6), (rep, k)
            if rep == 0:
                first.append((xh.copy(), info["iters"]))
            else:
                assert np.array_equal(xh, first[k][0]) and info["iters"] == first[k][1], (k, info)
    A.close()


def test_methods_interleaved_on_one_handle():
    """BiCGStab, TFQMR, BiCGStab(l) (l = 2 and 8: the workspace grows), the
    Jacobi variants, mixed precision, the persistent kernel and the host
    loop in turn on one handle with the same b and x, twice: the second pass
    gives the first pass's bits and iteration counts, and every result meets
    tol in the oracle's residual."""
    p, vals = _problem()
    b_h = g.source(p) + 0.2 * g.complex_vector(p.n, 7) * (~p.dirichlet)
    b = torch.as_tensor(b_h, device=DEV)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x = torch.empty_like(b)
    variants = [
        ("bicgstab", dict()),
        ("tfqmr", dict(method=helm.HELM_TFQMR)),
        ("bicgstabl2", dict(method=helm.HELM_BICGSTABL, ell=2)),
        ("bicgstab_jacobi", dict(precond=helm.HELM_PRECOND_JACOBI)),
        ("bicgstabl8", dict(method=helm.HELM_BICGSTABL, ell=8)),
        ("mixed", dict(precision=helm.HELM_PREC_MIXED, inner_tol=1e-2)),
        ("tfqmr_jacobi", dict(method=helm.HELM_TFQMR, precond=helm.HELM_PRECOND_JACOBI)),
        ("persistent", dict(launch=helm.HELM_LAUNCH_PERSISTENT)),
        ("host", dict(launch=helm.HELM_LAUNCH_HOST)),
    ]
    first = {}
    for rep in range(2):
        for name, kw in variants:
            _, info = helm.solve(A, b, x=x, tol=1e-10, maxit=20000, **kw)
            assert info["status"] == "ok", (name, info)
            xh = x.cpu().numpy()
            assert _relres(p, vals, b_h, xh) <= 1e-10 * (1 + 1e-6), name
            if rep == 0:
                first[name] = (xh.copy(), info["iters"])
            else:
                assert np.array_equal(xh, first[name][0]) and info["iters"] == first[name][1], (name, info)
    # the three launch forms of BiCGStab give the same bits
    assert np.array_equal(first["bicgstab"][0], first["persistent"][0])
    assert np.array_equal(first["bicgstab"][0], first["host"][0])
    A.close()
