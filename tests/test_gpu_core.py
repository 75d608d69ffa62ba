"""GPU parity of the C-ABI kernels against the CPU oracle (complex128 SpMV,
complex64 SpMV, zdotc/zdotu, norm, axpby) and of the BiCGStab solver against
dense LU and the oracle's BiCGStab.  Gates:
  SpMV  |y_gpu - y_ref|_i <= 1e-13 * sum_j |a_ij| |x_j|       (complex128)
  dot   |d_gpu - d_ref|   <= 1e-13 * sum_i |x_i| |y_i|         (complex128)
  solve true residual <= tol and
        |u_gpu - u_tight| / |u_tight| <= max(1e-8, 2 |u_oracle - u_tight| / |u_tight|)
Complex64 gates come from FP32 rounding: (len + 2) * 2^-23 * sum |a||x|."""
import math

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
U32 = 2.0 ** -23


def _abs_scale(rowptr, colind, vals, x):
    rows = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    return np.bincount(rows, weights=np.abs(vals) * np.abs(x[colind]), minlength=len(rowptr) - 1)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_11880_gb300 import build
    build.build()
    helm.load_library()


def _matrices():
    out = {}
    p = g.assemble(g.CONFIGS["box20"])
    out["box20"] = (p.rowptr, p.colind, g.helmholtz_values(p, 1500.0))
    # ragged: empty rows, n not a multiple of the tile, nnz not a multiple of 4
    rp, ci, v = g.random_csr(1000, 60, seed=5)
    if rp[-1] % 4 == 0:
        rp, ci, v = g.random_csr(1001, 60, seed=6)
    out["ragged"] = (rp, ci, v)
    # long rows: one tile holds more entries than a staged tile can take
    rng = np.random.default_rng(7)
    n = 300
    lens = np.full(n, 3)
    lens[5:40] = 250
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=rowptr[1:])
    cols = np.concatenate([np.sort(rng.choice(n, size=l, replace=False)) for l in lens]).astype(np.int32)
    out["longrows"] = (rowptr.astype(np.int32), cols, g.complex_vector(int(rowptr[-1]), 8))
    # tiny
    p = g.assemble(g.tiny_config(2, 2, 2))
    out["tiny"] = (p.rowptr, p.colind, g.helmholtz_values(p, 200.0))
    return out


MATS = _matrices()


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("ab", [(1.0, 0.0), (0.5 - 2j, 0.0), (1.0 + 1j, -0.25 + 3j)])
def test_spmv_c128(name, ab):
    rp, ci, v = MATS[name]
    n = len(rp) - 1
    alpha, beta = ab
    A = helm.CsrMatrix.from_host(rp, ci, v, device=DEV, validate=True)
    x = g.complex_vector(n, 1)
    y0 = g.complex_vector(n, 2)
    yd = _dev(y0.copy())
    A.matvec(_dev(x), yd, alpha=alpha, beta=beta)
    y = yd.cpu().numpy()
    ax = oracle.spmv(rp, ci, v, x)
    ref = alpha * ax + beta * y0
    scale = abs(alpha) * _abs_scale(rp, ci, v, x) + abs(beta) * np.abs(y0)
    assert np.all(np.abs(y - ref) <= 1e-13 * scale + 1e-300)
    A.close()


@pytest.mark.parametrize("name", ["box20", "ragged", "longrows"])
def test_spmv_c64(name):
    rp, ci, v = MATS[name]
    n = len(rp) - 1
    v32 = v.astype(np.complex64)
    A = helm.CsrMatrix.from_host(rp, ci, v32, device=DEV)
    x32 = g.complex_vector(n, 3).astype(np.complex64)
    y = A.matvec(_dev(x32)).cpu().numpy().astype(np.complex128)
    ref = oracle.spmv(rp, ci, v32.astype(np.complex128), x32.astype(np.complex128))
    lens = np.diff(rp)
    scale = _abs_scale(rp, ci, v32.astype(np.complex128), x32.astype(np.complex128))
    assert np.all(np.abs(y - ref) <= (lens + 2) * 2 * U32 * scale + 1e-30)
    A.close()


def test_spmv_full_size_sampled_rows():
    """120x60x50 cavity at full size: sampled rows recomputed by the oracle."""
    cfg = g.CONFIGS["cavity120"]
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x = g.complex_vector(p.n, 9)
    y = A.matvec(_dev(x)).cpu().numpy()
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([rng.choice(p.n, 4000, replace=False), [0, p.n - 1]]))
    for i in rows:
        k0, k1 = p.rowptr[i], p.rowptr[i + 1]
        sub_rp = np.array([0, k1 - k0], np.int32)
        ref = oracle.spmv(sub_rp, p.colind[k0:k1], vals[k0:k1], x)[0]
        scale = np.sum(np.abs(vals[k0:k1]) * np.abs(x[p.colind[k0:k1]]))
        assert abs(y[i] - ref) <= 1e-13 * scale
    A.close()


@pytest.mark.parametrize("n", [0, 1, 257, 1_000_003])
@pytest.mark.parametrize("conj", [True, False])
def test_dot_c128(n, conj):
    x = g.complex_vector(n, 11)
    y = g.complex_vector(n, 12)
    out = torch.zeros(1, dtype=torch.complex128, device=DEV)
    helm.helm_dot(_dev(x), _dev(y), out, conj_x=conj)
    d = complex(out.cpu().numpy()[0])
    ref = oracle.zdotc(x if conj else np.conj(x), y)
    assert abs(d - ref) <= 1e-13 * np.sum(np.abs(x) * np.abs(y)) + 1e-300
    # reproducible bit for bit
    out2 = torch.zeros(1, dtype=torch.complex128, device=DEV)
    helm.helm_dot(_dev(x), _dev(y), out2, conj_x=conj)
    assert complex(out2.cpu().numpy()[0]) == d


def test_dot_correlated_and_norm():
    x = g.complex_vector(500_000, 13)
    y = x + 1e-6 * g.complex_vector(500_000, 14)
    out = torch.zeros(1, dtype=torch.complex128, device=DEV)
    helm.helm_dot(_dev(x), _dev(y), out)
    d = complex(out.cpu().numpy()[0])
    assert abs(d - oracle.zdotc(x, y)) <= 1e-13 * np.sum(np.abs(x) * np.abs(y))
    nrm = torch.zeros(1, dtype=torch.float64, device=DEV)
    helm.helm_nrm2(_dev(x), nrm)
    assert abs(float(nrm.cpu()[0]) - oracle.dznrm2(x)) <= 1e-13 * oracle.dznrm2(x)


def test_dot_c64():
    n = 300_001
    x = g.complex_vector(n, 15).astype(np.complex64)
    y = g.complex_vector(n, 16).astype(np.complex64)
    out = torch.zeros(1, dtype=torch.complex128, device=DEV)
    helm.helm_dot(_dev(x), _dev(y), out)
    d = complex(out.cpu().numpy()[0])
    ref = oracle.zdotc(x.astype(np.complex128), y.astype(np.complex128))
    per_thread = math.ceil(n / (torch.cuda.get_device_properties(0).multi_processor_count * 8 * 256))
    assert abs(d - ref) <= (per_thread + 2) * 2 * U32 * np.sum(np.abs(x) * np.abs(y))


AXPBY_CASES = [(2 - 1j, 0.5 + 0.5j), (0.0, 3.0), (1.5, 0.0), (1j, 1.0), (0.0, 0.0), (1.0, 0.0), (0.0, 1.0),
               (0.7, 1.0), (1.0, -2.5), (1.0, 1.0), (0.0, 0.6 + 0.8j), (-0.3, 0.5 - 2j), (1.0, 1j)]


@pytest.mark.parametrize("alpha,beta", AXPBY_CASES)
def test_axpby(alpha, beta):
    n = 100_003
    x = g.complex_vector(n, 17)
    y = g.complex_vector(n, 18)
    yd = _dev(y.copy())
    helm.helm_axpby(alpha, _dev(x), beta, yd)
    ref = alpha * x + beta * y
    scale = abs(alpha) * np.abs(x) + abs(beta) * np.abs(y)
    assert np.all(np.abs(yd.cpu().numpy() - ref) <= 4e-16 * scale + 1e-300)


@pytest.mark.parametrize("alpha,beta", AXPBY_CASES[:6] + [(0.7, 1.0), (1.0, -2.5)])
def test_axpby_complex64_and_aliased(alpha, beta):
    """complex64 vectors (FP32 products: at most 4 roundings of 2^-24 each
    relative to |alpha||x| + |beta||y|), and x equal to y (y = (alpha + beta) y
    element by element)."""
    n = 70_001
    x = g.complex_vector(n, 27).astype(np.complex64)
    y = g.complex_vector(n, 28).astype(np.complex64)
    yd = _dev(y.copy())
    helm.helm_axpby(alpha, _dev(x), beta, yd)
    a32, b32 = complex(np.complex64(alpha)), complex(np.complex64(beta))
    xe, ye = x.astype(np.complex128), y.astype(np.complex128)
    ref = a32 * xe + b32 * ye
    scale = abs(a32) * np.abs(xe) + abs(b32) * np.abs(ye)
    assert np.all(np.abs(yd.cpu().numpy().astype(np.complex128) - ref) <= 4 * 2.0 ** -24 * scale + 1e-38)
    z = g.complex_vector(n, 29)
    zd = _dev(z.copy())
    helm.helm_axpby(alpha, zd, beta, zd)
    ref = alpha * z + beta * z
    scale = (abs(alpha) + abs(beta)) * np.abs(z)
    assert np.all(np.abs(zd.cpu().numpy() - ref) <= 4e-16 * scale + 1e-300)


def _banded_csr(n, offsets, drop, seed):
    """A matrix on the given diagonals with a fraction `drop` of the
    off-diagonal slots left out (empty slots of the diagonal copy)."""
    rng = np.random.default_rng(seed)
    rp, ci, vv = [0], [], []
    for i in range(n):
        for d in offsets:
            j = i + d
            if 0 <= j < n and (d == 0 or rng.random() >= drop):
                ci.append(j)
                vv.append(complex(rng.uniform(-1, 1), rng.uniform(-1, 1) if rng.random() < 0.2 else 0.0))
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32), np.array(vv, np.complex128)


def _dia_cases():
    out = {"box20": MATS["box20"]}  # n = 9261: a partial last slice of 13 rows
    p = g.assemble(g.tiny_config(20, 16, 12, h=0.05, seed=3))  # n = 4641: a last slice of one row
    out["mesh4641"] = (p.rowptr, p.colind, g.helmholtz_values(p, 600.0))
    out["banded"] = _banded_csr(1003, [-40, -3, -1, 0, 1, 2, 17, 333], 0.1, 9)
    return out


DIA = _dia_cases()


@pytest.mark.parametrize("name", list(DIA))
def test_spmv_c64_diagonal_copy_matches_sliced(name):
    """complex64 matrices on few diagonals get a diagonal copy: the product
    equals the sliced copy's bit for bit (same FP32 operations in column
    order, empty slots skipped; also with an Inf in x next to a row that has
    no entry there) and meets the complex64 gate against the oracle."""
    rp, ci, v = DIA[name]
    n = len(rp) - 1
    v32 = v.astype(np.complex64)
    A = helm.CsrMatrix.from_host(rp, ci, v32, device=DEV)
    B = helm.CsrMatrix.from_host(rp, ci, v32, device=DEV, sliced_only=True)
    assert A.diagonals() > 0 and B.diagonals() == 0
    x32 = g.complex_vector(n, 13).astype(np.complex64)
    ya = A.matvec(_dev(x32))
    yb = B.matvec(_dev(x32))
    assert torch.equal(torch.view_as_real(ya), torch.view_as_real(yb))
    y = ya.cpu().numpy().astype(np.complex128)
    ref = oracle.spmv(rp, ci, v32.astype(np.complex128), x32.astype(np.complex128))
    scale = _abs_scale(rp, ci, v32.astype(np.complex128), x32.astype(np.complex128))
    assert np.all(np.abs(y - ref) <= (np.diff(rp) + 2) * 2 * U32 * scale + 1e-30)
    y0 = g.complex_vector(n, 14).astype(np.complex64)
    ya, yb = _dev(y0.copy()), _dev(y0.copy())
    A.matvec(_dev(x32), ya, alpha=0.5 - 2j, beta=1 + 1j)
    B.matvec(_dev(x32), yb, alpha=0.5 - 2j, beta=1 + 1j)
    assert torch.equal(torch.view_as_real(ya), torch.view_as_real(yb))
    # an Inf in x at a column that some row's diagonal slot covers without an entry
    rows_with = set(np.repeat(np.arange(n), np.diff(rp))[ci == 1].tolist())
    if len(rows_with) < n:
        xi = x32.copy()
        xi[1] = np.inf
        ya, yb = A.matvec(_dev(xi)).cpu().numpy(), B.matvec(_dev(xi)).cpu().numpy()
        assert np.array_equal(ya, yb, equal_nan=True)
        assert np.all(np.isfinite(ya[[i for i in range(n) if i not in rows_with]]))
    A.close()
    B.close()


def test_diagonal_copy_only_where_it_fits():
    """No diagonal copy for a pattern off its longest row's diagonals, or one
    whose diagonals would hold more than 1.5 slots per entry (a small mesh,
    mostly boundary; a band with half its slots empty)."""
    rp, ci, v = MATS["ragged"]
    A = helm.CsrMatrix.from_host(rp, ci, v.astype(np.complex64), device=DEV)
    assert A.diagonals() == 0
    A.close()
    for rp, ci, v in (_banded_csr(500, [-7, -1, 0, 1, 7], 0.6, 4), MATS["tiny"]):
        A = helm.CsrMatrix.from_host(rp, ci, v.astype(np.complex64), device=DEV)
        assert A.diagonals() == 0
        A.close()


def test_mixed_solve_same_with_and_without_diagonal_copy():
    """The complex64 inner solves of mixed precision read the diagonal copy
    of the handle's complex64 values; the whole solve matches a handle
    without it bit for bit."""
    p = g.assemble(g.CONFIGS["box20"])
    vals = g.helmholtz_values(p, 1500.0)
    b = _dev(g.source(p))
    out = []
    for sliced in (False, True):
        A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV, sliced_only=sliced)
        assert (A.diagonals() > 0) != sliced
        x, info = helm.solve(A, b, tol=1e-8, maxit=20000, precision=helm.HELM_PREC_MIXED)
        assert info["status"] == "ok", info
        out.append((x, info))
        A.close()
    (xa, ia), (xb, ib) = out
    assert torch.equal(torch.view_as_real(xa), torch.view_as_real(xb))
    assert ia["iters"] == ib["iters"] and ia["relres_true"] == ib["relres_true"]


def test_invalid_arguments_rejected():
    rp, ci, v = MATS["tiny"]
    bad = ci.copy()
    bad[3] = len(rp) + 5
    with pytest.raises(helm.HelmError):
        helm.CsrMatrix.from_host(rp, bad, v, device=DEV, validate=True)
    A = helm.CsrMatrix.from_host(rp, ci, v, device=DEV)
    x = _dev(g.complex_vector(len(rp) - 1, 1))
    with pytest.raises(helm.HelmError):
        helm.helm_spmv(A.handle, 1.0, x, 0.0, x)   # aliasing x and y
    A.close()


def test_overlapping_vectors_rejected():
    """Input and output vectors that share memory (the same buffer, or views
    one element apart) are rejected by the product, the solve, the sweep and
    the Schwarz preconditioner; disjoint neighbours are accepted."""
    p, vals = _tiny_problem((4, 3, 3), 400.0, 2)[:2]
    n = p.n
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    buf = _dev(g.complex_vector(2 * n + 1, 3))
    lo, hi, apart = buf[0:n], buf[1:n + 1], buf[n:2 * n]
    for y in (lo, hi):
        with pytest.raises(helm.HelmError):
            helm.helm_spmv(A.handle, 1.0, lo, 0.0, y)
        with pytest.raises(helm.HelmError):
            helm.helm_bicgstab_solve(A.handle, lo, y)
    helm.helm_spmv(A.handle, 1.0, lo, 0.0, apart)
    info = helm.helm_bicgstab_solve(A.handle, lo, apart, helm.default_opts(tol=1e-10))
    assert info["status"] == "ok"
    D = helm.Ddm(A, 2, 4)
    with pytest.raises(helm.HelmError):
        D.apply(lo, hi)
    with pytest.raises(helm.HelmError):
        D.solve(lo, hi)
    D.close()
    S = helm.Sweep(p.rowptr, p.colind, p.K, p.Mc, p.Bc, device=DEV)
    w = [g.omega(f) for f in (200.0, 300.0)]
    X = torch.zeros((n, 2), dtype=torch.complex128, device=DEV)
    B2 = torch.zeros((n + 1, 2), dtype=torch.complex128, device=DEV)
    with pytest.raises(helm.HelmError):
        helm.helm_sweep_solve(S.handle, w, B2[0:n], B2[1:n + 1])
    with pytest.raises(helm.HelmError):
        helm.helm_sweep_spmv(S.handle, w, B2[0:n], B2[1:n + 1])
    helm.helm_sweep_spmv(S.handle, w, B2[0:n], X)
    S.close()
    A.close()


# ---------------------------------------------------------------- BiCGStab

def _tiny_problem(dims, F, seed):
    cfg = g.tiny_config(*dims, h=0.1, F=F, seed=seed)
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, F)
    b = g.source(p) + 0.2 * g.complex_vector(p.n, seed + 1) * (~p.dirichlet)
    return p, vals, b


@pytest.mark.parametrize("dims,F", [((2, 2, 2), 300.0), ((5, 4, 3), 450.0), ((9, 7, 6), 900.0)])
def test_bicgstab_vs_dense_lu(dims, F):
    p, vals, b = _tiny_problem(dims, F, 3)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x, info = helm.solve(A, _dev(b), tol=1e-12, maxit=10000)
    assert info["status"] == "ok"
    xs = oracle.dense_solve(p.rowptr, p.colind, vals, b)
    xr, rinfo = oracle.bicgstab(p.rowptr, p.colind, vals, b, tol=1e-12, maxit=10000)
    xg = x.cpu().numpy()
    res = np.linalg.norm(b - oracle.spmv(p.rowptr, p.colind, vals, xg)) / np.linalg.norm(b)
    assert res <= 1e-12 * (1 + 1e-6)
    e_g = np.linalg.norm(xg - xs) / np.linalg.norm(xs)
    e_o = np.linalg.norm(xr - xs) / np.linalg.norm(xs)
    assert e_g <= max(1e-8, 2 * e_o)
    A.close()


@pytest.fixture(scope="module")
def box20():
    cfg = g.CONFIGS["box20"]
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    b = g.source(p)
    x_o, info_o = oracle.bicgstab(p.rowptr, p.colind, vals, b, tol=cfg.tol, maxit=20000)
    x_t, info_t = oracle.bicgstab(p.rowptr, p.colind, vals, b, tol=1e-13, maxit=60000)
    return p, vals, b, x_o, info_o, x_t


def test_bicgstab_box20_parity(box20):
    p, vals, b, x_o, info_o, x_t = box20
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x, info = helm.solve(A, _dev(b), tol=1e-8, maxit=20000)
    assert info["status"] == "ok", info
    xg = x.cpu().numpy()
    res = np.linalg.norm(b - oracle.spmv(p.rowptr, p.colind, vals, xg)) / np.linalg.norm(b)
    assert res <= 1e-8 * (1 + 1e-6) and abs(res - info["relres_true"]) <= 1e-3 * res
    nt = np.linalg.norm(x_t)
    e_g = np.linalg.norm(xg - x_t) / nt
    e_o = np.linalg.norm(x_o - x_t) / nt
    assert e_g <= max(1e-8, 2 * e_o), (e_g, e_o)
    print(f"box20: gpu iters {info['iters']} oracle iters {info_o['iters']}")
    assert abs(info["iters"] - info_o["iters"]) <= 0.05 * info_o["iters"] + 2
    A.close()


def test_bicgstab_degenerate_cases():
    p, vals, b = _tiny_problem((3, 3, 3), 450.0, 5)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    zero = torch.zeros(p.n, dtype=torch.complex128, device=DEV)
    x = _dev(g.complex_vector(p.n, 1))
    info = helm.helm_bicgstab_solve(A.handle, zero, x, helm.default_opts())
    assert info["status"] == "ok" and info["iters"] == 0 and torch.all(x == 0)
    x, info = helm.solve(A, _dev(b), tol=1e-30, maxit=1)
    assert info["status"] == "not_converged" and info["iters"] == 1
    xs = _dev(oracle.dense_solve(p.rowptr, p.colind, vals, b))
    info = helm.helm_bicgstab_solve(A.handle, _dev(b), xs, helm.default_opts(use_x0=1))
    assert info["status"] == "ok" and info["iters"] == 0
    bad = b.copy()
    bad[4] = np.nan
    x, info = helm.solve(A, _dev(bad))
    assert info["status"] == "nonfinite"
    Z = helm.CsrMatrix.from_host(p.rowptr, p.colind, np.zeros_like(vals), device=DEV)
    x, info = helm.solve(Z, _dev(b))
    assert info["status"] == "breakdown"
    Z.close()
    A.close()


def test_bicgstab_deadline_returns_timeout():
    """Failure detection without a fault: a deadline that expires during the
    first iteration makes the device loop stop and report a timeout."""
    p = g.assemble(g.CONFIGS["box20"])
    vals = g.helmholtz_values(p, 1500.0)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    x, info = helm.solve(A, _dev(g.source(p)), tol=1e-12, maxit=20000, deadline_s=1e-9)
    assert info["status"] == "timeout" and 1 <= info["iters"] <= 2
    # the context stays usable
    x, info = helm.solve(A, _dev(g.source(p)), tol=1e-6, maxit=20000)
    assert info["status"] == "ok"
    A.close()


def test_bicgstab_repeated_solves_reuse_graph(box20):
    p, vals, b, *_ = box20
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    bd = _dev(b)
    x = torch.empty_like(bd)
    infos = [helm.helm_bicgstab_solve(A.handle, bd, x, helm.default_opts(tol=1e-6)) for _ in range(3)]
    assert all(i["status"] == "ok" for i in infos)
    assert len({i["iters"] for i in infos}) == 1      # deterministic
    A.close()


@pytest.mark.parametrize("method,prec", [("bicgstab", "fp64"), ("tfqmr", "fp64"), ("bicgstabl", "fp64"),
                                         ("bicgstab", "mixed")])
def test_graph_and_host_loops_agree_bit_for_bit(box20, method, prec):
    """The graph (device-driven while node, dependent launches) and the
    host-driven loop run the same kernels on the same grids with fixed-order
    reductions: same iterations, same x to the last bit.  An explicit graph
    request must not fall back to the host loop."""
    p, vals, b, *_ = box20
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    bd = _dev(b)
    kw = dict(tol=1e-9, maxit=20000, method={"bicgstab": helm.HELM_BICGSTAB, "tfqmr": helm.HELM_TFQMR,
                                              "bicgstabl": helm.HELM_BICGSTABL}[method],
              precision=helm.HELM_PREC_MIXED if prec == "mixed" else helm.HELM_PREC_FP64)
    xg, xh = torch.empty_like(bd), torch.empty_like(bd)
    ig = helm.helm_bicgstab_solve(A.handle, bd, xg, helm.default_opts(launch=helm.HELM_LAUNCH_GRAPH, **kw))
    ih = helm.helm_bicgstab_solve(A.handle, bd, xh, helm.default_opts(launch=helm.HELM_LAUNCH_HOST, **kw))
    assert ig["status"] == "ok" and ih["status"] == "ok", (ig, ih)
    assert ig["iters"] == ih["iters"] and ig["restarts"] == ih["restarts"]
    assert torch.equal(torch.view_as_real(xg), torch.view_as_real(xh))
    A.close()
