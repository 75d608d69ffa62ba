"""Pins of the CPU oracle and the input generator against facts that do not
come from the oracle itself: exact rational arithmetic, dense LAPACK solves,
closed forms of the Q1 discretisation, a manufactured plane wave, special
cases of BiCGStab, and central finite differences.  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest

import helmgen as g
import oracle

EPS = np.finfo(np.float64).eps


# ---------------------------------------------------------------- generator

@pytest.mark.parametrize("h", [0.05, 0.0375, 1.0])
def test_element_matrix_identities(h):
    Ke, Me, Bf = g.element_matrices(h)
    ones = np.ones(8)
    assert np.allclose(Ke @ ones, 0.0, atol=1e-14 / h)        # constants in the kernel of K_e
    assert math.isclose(ones @ Me @ ones, h ** 3, rel_tol=1e-14)  # integral of 1 over the cube
    assert math.isclose(ones @ Bf @ ones, h ** 2, rel_tol=1e-14)  # area of the top face
    assert np.array_equal(Ke, Ke.T) and np.array_equal(Me, Me.T) and np.array_equal(Bf, Bf.T)
    assert np.all(np.linalg.eigvalsh(Me) > 0)
    ev = np.linalg.eigvalsh(Ke)
    assert abs(ev[0]) < 1e-12 / h and np.all(ev[1:] > 0)      # one-dimensional kernel
    # only the four top nodes (az = 1) carry the face matrix
    top = [a for a in range(8) if (a >> 2) & 1]
    mask = np.zeros((8, 8), bool)
    mask[np.ix_(top, top)] = True
    assert np.all(Bf[~mask] == 0)


def _golden_q1():
    import os
    from fractions import Fraction as Fr
    path = os.path.join(os.path.dirname(__file__), "golden", "q1_element_h1.txt")
    mats, cur = {}, None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line in ("K", "M", "B"):
            cur = mats.setdefault(line, [])
        else:
            cur.append([float(Fr(t)) for t in line.split()])
    return {k: np.array(v) for k, v in mats.items()}


@pytest.mark.parametrize("h", [1.0, 0.5, 0.0375])
def test_element_matrices_match_exact_fixture(h):
    """The generator's element matrices equal the exact unit-cube rationals of
    tests/golden/q1_element_h1.txt scaled by h, h^3, h^2 (a few ulps)."""
    gold = _golden_q1()
    Ke, Me, Bf = g.element_matrices(h)
    for got, ref, sc in ((Ke, gold["K"], h), (Me, gold["M"], h ** 3), (Bf, gold["B"], h ** 2)):
        assert np.allclose(got, ref * sc, rtol=8 * EPS, atol=8 * EPS * sc)


def test_global_mass_and_area():
    cfg = g.tiny_config(4, 3, 5, h=0.2)
    p = g.assemble(cfg, c=np.ones(cfg.n_elem), dirichlet=False)
    L = (cfg.nx * cfg.h, cfg.ny * cfg.h, cfg.nz * cfg.h)
    assert math.isclose(p.Mc.sum(), L[0] * L[1] * L[2], rel_tol=1e-13)
    assert math.isclose(p.Bc.sum(), L[0] * L[1], rel_tol=1e-13)
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    rowsum = np.bincount(rows, weights=p.K, minlength=p.n)
    assert np.allclose(rowsum, 0.0, atol=1e-12)


@pytest.mark.parametrize("name", ["box20", "sweep60"])
def test_pattern_size_and_exact_symmetry(name):
    cfg = g.CONFIGS[name]
    p = g.assemble(cfg)
    assert p.nnz == cfg.nnz and p.n == cfg.n
    assert np.all(np.diff(p.rowptr) <= 27) and np.diff(p.rowptr).max() == 27
    for i in range(0, p.n, max(1, p.n // 500)):
        cols = p.colind[p.rowptr[i]:p.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
    import scipy.sparse as sp
    for F in cfg.freqs[:2]:
        A = sp.csr_matrix((g.helmholtz_values(p, F), p.colind, p.rowptr), shape=(p.n, p.n))
        D = (A - A.T).tocoo()
        assert D.nnz == 0 or np.all(D.data == 0)    # A == A^T bit for bit
    # Dirichlet rows are identity rows
    d = np.flatnonzero(p.dirichlet)
    assert np.all(np.diff(p.rowptr)[d] == 1)
    assert np.all(p.colind[p.rowptr[d]] == d) and np.all(p.K[p.rowptr[d]] == 1.0)


def test_source_and_receivers():
    p = g.assemble(g.CONFIGS["box20"])
    b = g.source(p)
    assert np.all(b[p.dirichlet] == 0) and np.all(b.imag == 0)
    i = int(np.argmax(np.abs(b)))
    c = np.array([10, 10, 10]) * 0.05
    assert np.allclose(p.coords[i], c)
    assert math.isclose(b[i].real, 0.05 ** 3)
    r = g.receivers(p, 64, seed=1)
    assert len(set(r.tolist())) == 64 and not p.dirichlet[r].any()


def test_element_nnz_map():
    cfg = g.tiny_config(3, 2, 3)
    p = g.assemble(cfg)
    m = g.element_nnz_map(p)
    en = g.element_nodes(cfg)
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    for e in range(cfg.n_elem):
        for a in range(8):
            for b in range(8):
                k = m[e, 8 * a + b]
                if p.dirichlet[en[e, a]] or p.dirichlet[en[e, b]]:
                    assert k == -1
                else:
                    assert rows[k] == en[e, a] and p.colind[k] == en[e, b]


# ---------------------------------------------------------------- SpMV

def _tiny_problems():
    out = []
    for dims, F, seed in [((2, 2, 2), 300.0, 0), ((3, 3, 3), 450.0, 5), ((4, 2, 3), 700.0, 7)]:
        cfg = g.tiny_config(*dims, h=0.1, F=F, seed=seed)
        p = g.assemble(cfg)
        out.append((p, g.helmholtz_values(p, F)))
    return out


def _abs_scale(rowptr, colind, vals, x):
    rows = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    return np.bincount(rows, weights=np.abs(vals) * np.abs(x[colind]), minlength=len(rowptr) - 1)


def test_spmv_equals_dense_matvec():
    for p, vals in _tiny_problems():
        x = g.complex_vector(p.n, 11)
        y = oracle.spmv(p.rowptr, p.colind, vals, x)
        yd = oracle.densify(p.rowptr, p.colind, vals) @ x
        scale = _abs_scale(p.rowptr, p.colind, vals, x)
        assert np.all(np.abs(y - yd) <= 4 * 27 * EPS * scale + 1e-300)
    # ragged random CSR with empty rows and a non-square column space
    rp, ci, v = g.random_csr(300, 40, seed=3, ncols=500)
    x = g.complex_vector(500, 4)
    y = oracle.spmv(rp, ci, v, x)
    yd = oracle.densify(rp, ci, v, ncols=500) @ x
    assert np.all(np.abs(y - yd) <= 4 * 40 * EPS * _abs_scale(rp, ci, v, x) + 1e-300)
    assert np.all(y[np.diff(rp) == 0] == 0)


def test_spmv_exact_small_integers():
    # integer-valued entries: every product and partial sum is exact
    rp, ci, v = g.random_csr(200, 30, seed=9)
    v = np.round(v * 8) + 1j * np.round(v.imag * 8)
    x = np.round(g.complex_vector(200, 10) * 16)
    y = oracle.spmv(rp, ci, v, x)
    for i in range(200):
        acc_r = acc_i = 0
        for k in range(rp[i], rp[i + 1]):
            a, b = v[k], x[ci[k]]
            acc_r += int(a.real) * int(b.real) - int(a.imag) * int(b.imag)
            acc_i += int(a.real) * int(b.imag) + int(a.imag) * int(b.real)
        assert y[i] == complex(acc_r, acc_i)


def test_spmv_bilinear_symmetry():
    p = g.assemble(g.CONFIGS["box20"])
    vals = g.helmholtz_values(p, 1500.0)
    x = g.complex_vector(p.n, 1)
    y = g.complex_vector(p.n, 2)
    lhs = np.sum(x * oracle.spmv(p.rowptr, p.colind, vals, y))
    rhs = np.sum(y * oracle.spmv(p.rowptr, p.colind, vals, x))
    scale = np.sum(np.abs(x) * _abs_scale(p.rowptr, p.colind, vals, np.abs(y)))
    assert abs(lhs - rhs) <= 1e-14 * scale


# ---------------------------------------------------------------- dots

def _exact_dot(x, y, conj=True):
    re = Fraction(0)
    im = Fraction(0)
    for a, b in zip(x, y):
        ar, ai = Fraction(a.real), Fraction(a.imag)
        if conj:
            ai = -ai
        br, bi = Fraction(b.real), Fraction(b.imag)
        re += ar * br - ai * bi
        im += ar * bi + ai * br
    return re, im


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_zdotc_against_exact_rationals(seed):
    n = 257
    x = g.complex_vector(n, seed)
    y = g.complex_vector(n, seed + 100)
    if seed == 2:   # strongly correlated: |(x,y)| close to sum |x||y|
        y = x + 1e-3 * y
    d = oracle.zdotc(x, y)
    er, ei = _exact_dot(x, y)
    bound = 3 * EPS * float(np.sum(np.abs(x) * np.abs(y)))
    assert abs(Fraction(d.real) - er) <= bound
    assert abs(Fraction(d.imag) - ei) <= bound
    # a dropped conjugate is caught: the unconjugated sum differs
    ur, ui = _exact_dot(x, y, conj=False)
    assert abs(float(ur - er)) + abs(float(ui - ei)) > 1e3 * bound


def test_zdotc_symmetries_and_norm():
    x = g.complex_vector(1000, 5)
    y = g.complex_vector(1000, 6)
    a = oracle.zdotc(x, y)
    b = oracle.zdotc(y, x)
    assert a == b.conjugate()                     # (x, y) = conj((y, x)) exactly
    xx = oracle.zdotc(x, x)
    assert xx.imag == 0.0 and xx.real > 0
    nrm = oracle.dznrm2(x)
    exact = sum(Fraction(v.real) ** 2 + Fraction(v.imag) ** 2 for v in x)
    assert abs(nrm - math.sqrt(float(exact))) <= 2 * EPS * nrm
    assert abs(nrm * nrm - xx.real) <= 4 * EPS * xx.real
    assert oracle.zdotc(np.zeros(0), np.zeros(0)) == 0 and oracle.dznrm2(np.zeros(0)) == 0


# ---------------------------------------------------------------- BiCGStab

def _csr_diag(d):
    n = len(d)
    return np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.asarray(d, np.complex128)


def test_bicgstab_scaled_identity_one_iteration():
    rp, ci, v = _csr_diag(np.full(10, 2.5 + 2.5j))
    b = g.complex_vector(10, 3)
    x, info = oracle.bicgstab(rp, ci, v, b, tol=1e-12)
    assert info["status"] == "ok" and info["iters"] == 1
    assert np.allclose(x, b / (2.5 + 2.5j), rtol=1e-15, atol=0)


def test_bicgstab_diagonal_converges_in_distinct_eigenvalues():
    # Krylov space of a diagonal matrix with 3 distinct values has dimension 3
    d = np.array([1.0, 2.0 + 1j, 3.0 - 2j] * 5)
    rp, ci, v = _csr_diag(d)
    b = g.complex_vector(15, 8)
    x, info = oracle.bicgstab(rp, ci, v, b, tol=1e-12)
    assert info["status"] == "ok" and info["iters"] <= 3
    assert np.allclose(x, b / d, rtol=1e-10)


def test_bicgstab_degenerate_cases():
    p, vals = _tiny_problems()[0]
    b = np.zeros(p.n, np.complex128)
    x, info = oracle.bicgstab(p.rowptr, p.colind, vals, b)
    assert info["status"] == "ok" and info["iters"] == 0 and np.all(x == 0)
    b = g.source(p) + g.complex_vector(p.n, 1) * (~p.dirichlet)
    x, info = oracle.bicgstab(p.rowptr, p.colind, vals, b, tol=1e-30, maxit=1)
    assert info["status"] == "not_converged" and info["iters"] == 1
    xs = oracle.dense_solve(p.rowptr, p.colind, vals, b)
    x, info = oracle.bicgstab(p.rowptr, p.colind, vals, b, tol=1e-8, x0=xs)
    assert info["status"] == "ok" and info["iters"] == 0
    bad = b.copy()
    bad[3] = np.nan
    x, info = oracle.bicgstab(p.rowptr, p.colind, vals, bad)
    assert info["status"] == "nonfinite"
    # singular: a zero matrix breaks down at the first denominator
    z = np.zeros_like(vals)
    x, info = oracle.bicgstab(p.rowptr, p.colind, z, b)
    assert info["status"] == "breakdown"


def test_bicgstab_matches_dense_lu():
    for p, vals in _tiny_problems():
        b = g.complex_vector(p.n, 21) * (~p.dirichlet)
        xs = oracle.dense_solve(p.rowptr, p.colind, vals, b)
        x, info = oracle.bicgstab(p.rowptr, p.colind, vals, b, tol=1e-12)
        assert info["status"] == "ok"
        assert info["relres_true"] <= 1.5e-12
        cond = np.linalg.cond(oracle.densify(p.rowptr, p.colind, vals))
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 10 * cond * 1e-12


def _column_problem(nz, k_target=6.0, nxy=2, c=340.0):
    """Thin column of height 1 m: constant speed, u = 1 lifted on z = 0."""
    h = 1.0 / nz
    F = k_target * c / (2 * math.pi)
    cfg = g.tiny_config(nxy, nxy, nz, h=h, F=F)
    cc = np.full(cfg.n_elem, c)
    full = g.assemble(cfg, c=cc, dirichlet=False)
    elim = g.assemble(cfg, c=cc, dirichlet=True)
    Af = g.helmholtz_values(full, F)
    # lift: b_i = -sum_{j on z=0} A_ij for free rows i
    rows = np.repeat(np.arange(full.n), np.diff(full.rowptr))
    on_d = elim.dirichlet[full.colind]
    b = -np.bincount(rows[on_d], weights=Af[on_d].real, minlength=full.n) \
        - 1j * np.bincount(rows[on_d], weights=Af[on_d].imag, minlength=full.n)
    b[elim.dirichlet] = 0.0
    vals = g.helmholtz_values(elim, F)
    x, info = oracle.bicgstab(elim.rowptr, elim.colind, vals, b, tol=1e-13, maxit=100000)
    assert info["status"] == "ok"
    u = x.copy()
    u[elim.dirichlet] = 1.0
    k = 2 * math.pi * F / c
    return elim, u, k, h


def test_manufactured_plane_wave_q1_rate():
    """u = exp(-i k z) solves -u'' - k^2 u = 0 with u(0) = 1 and the impedance
    condition du/dn = -i k u on the top face; Q1 nodal error falls as h^2."""
    errs = []
    for nz in (16, 32, 64):
        p, u, k, h = _column_problem(nz)
        exact = np.exp(-1j * k * p.coords[:, 2])
        errs.append(np.max(np.abs(u - exact)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.7 < r2 < 4.3, errs
    assert errs[-1] < 5e-3


def test_one_dimensional_closed_form():
    """Constant-in-(x, y) solutions of the 3-D Q1 system are exactly the 1-D
    linear-element solution (tensor-product structure); its interior obeys the
    discrete dispersion relation cos(k_h h) = (6 - 2 (kh)^2) / (6 + (kh)^2)."""
    nz = 24
    p, u, k, h = _column_problem(nz, k_target=9.0, nxy=3)
    # 1-D linear elements on [0, 1]: stiffness/mass/impedance, u_0 = 1
    N = nz + 1
    K = np.zeros((N, N)); M = np.zeros((N, N))
    for e in range(nz):
        K[e:e + 2, e:e + 2] += np.array([[1, -1], [-1, 1]]) / h
        M[e:e + 2, e:e + 2] += np.array([[2, 1], [1, 2]]) * h / 6
    A = K - k * k * M + 0j
    A[N - 1, N - 1] += 1j * k
    rhs = -A[1:, 0]
    U = np.concatenate([[1.0], np.linalg.solve(A[1:, 1:], rhs)])
    zk = np.rint(p.coords[:, 2] / h).astype(int)
    assert np.max(np.abs(u - U[zk])) < 1e-10
    # discrete dispersion in the interior (no source)
    ch = (6 - 2 * (k * h) ** 2) / (6 + (k * h) ** 2)
    for j in range(1, nz):
        assert abs(U[j + 1] + U[j - 1] - 2 * ch * U[j]) < 1e-12


# ---------------------------------------------------------------- adjoint

def _loss_of_c(cfg, c, b, rec, d):
    p = g.assemble(cfg, c=c)
    u = oracle.dense_solve(p.rowptr, p.colind, g.helmholtz_values(p, cfg.F), b)
    return oracle.loss(u, rec, d)


def test_sound_speed_gradient_against_finite_differences():
    cfg = g.tiny_config(3, 2, 3, h=0.1, F=450.0, seed=4)
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    b = g.source(p) + 0.3 * g.complex_vector(p.n, 2) * (~p.dirichlet)
    rec = g.receivers(p, 6, seed=1)
    c_true = g.sound_speed(cfg, seed=2)
    pt = g.assemble(cfg, c=c_true)
    d = oracle.dense_solve(pt.rowptr, pt.colind, g.helmholtz_values(pt, cfg.F), b)[rec]
    u = oracle.dense_solve(p.rowptr, p.colind, vals, b)
    w = oracle.adjoint_rhs(p.n, u, rec, d)
    mu = oracle.dense_solve(p.rowptr, p.colind, vals, w)       # A^T = A
    G = oracle.nnz_gradient(p.rowptr, p.colind, mu, u)
    Ke, Me, Bf = g.element_matrices(cfg.h)
    top = (np.arange(cfg.n_elem) // (cfg.nx * cfg.ny)) == cfg.nz - 1
    grad = oracle.sound_speed_gradient(G, g.element_nnz_map(p), Me, Bf, p.c,
                                       g.omega(cfg.F), top)
    eps = 1e-3
    fd = np.empty(cfg.n_elem)
    for e in range(cfg.n_elem):
        cp = p.c.copy(); cp[e] += eps
        cm = p.c.copy(); cm[e] -= eps
        fd[e] = (_loss_of_c(cfg, cp, b, rec, d) - _loss_of_c(cfg, cm, b, rec, d)) / (2 * eps)
    assert np.max(np.abs(grad - fd)) <= 1e-6 * np.max(np.abs(fd))
    # gradient with respect to b (PyTorch convention 2 conj(mu)) by finite differences
    gb = 2 * np.conj(mu)
    for i in rec[:3]:
        for unit in (1.0, 1j):
            bp = b.copy(); bp[i] += eps * unit
            bm = b.copy(); bm[i] -= eps * unit
            f = (oracle.loss(oracle.dense_solve(p.rowptr, p.colind, vals, bp), rec, d)
                 - oracle.loss(oracle.dense_solve(p.rowptr, p.colind, vals, bm), rec, d)) / (2 * eps)
            ref = gb[i].real if unit == 1.0 else gb[i].imag
            assert abs(f - ref) <= 1e-6 * max(1.0, abs(ref)) + 1e-9


def test_helmholtz_values_against_element_assembly():
    """The oracle's A(w) = K - w^2 M_c + i w B_c on the assembled arrays equals
    the Helmholtz operator's definition summed element by element here,
    sum_e K_e - (w / c_e)^2 M_e + i (w / c_e) B_f (B_f on the elements with a
    face on the impedance plane), with the Dirichlet rows as identity rows and
    their columns dropped.  The two routes share only the element matrices
    (pinned by the exact fixture): a wrong power of w or of c_e, a sign or a
    dropped term fails here.  A varying sound speed, two frequencies."""
    cfg = g.tiny_config(3, 2, 3, h=0.1, seed=5)
    p = g.assemble(cfg)
    assert np.ptp(p.c) > 0
    Ke, Me, Bf = g.element_matrices(cfg.h)
    en = g.element_nodes(cfg)
    top = g.top_elements(cfg).astype(bool)
    D = p.dirichlet
    for F in (150.0, 900.0):
        w = g.omega(F)
        E = np.zeros((p.n, p.n), dtype=np.complex128)
        for e in range(cfg.n_elem):
            k = w / p.c[e]
            Ae = Ke - k * k * Me + (1j * k * Bf if top[e] else 0.0)
            for a in range(8):
                for b in range(8):
                    E[en[e, a], en[e, b]] += Ae[a, b]
        E[D, :] = 0.0
        E[:, D] = 0.0
        E[D, D] = 1.0
        A = oracle.densify(p.rowptr, p.colind, oracle.helmholtz_values(p.K, p.Mc, p.Bc, w))
        scale = np.abs(Ke).max() + (w / p.c.min()) ** 2 * np.abs(Me).max() + (w / p.c.min()) * np.abs(Bf).max()
        assert np.max(np.abs(A - E)) <= 1e-14 * scale
        # the impedance term is present exactly on the top plane's couplings
        assert np.any(A.imag != 0) and np.all(A.imag[~np.isin(np.arange(p.n), en[top].ravel()), :] == 0)
    assert np.array_equal(oracle.helmholtz_values(p.K, p.Mc, p.Bc, 0.0).real, p.K)


# ---------------------------------------------------------------- TFQMR

def test_tfqmr_scaled_identity_one_iteration():
    rp, ci, v = _csr_diag(np.full(12, 3.0 - 1.0j))
    b = g.complex_vector(12, 5)
    x, info = oracle.tfqmr(rp, ci, v, b, tol=1e-12)
    assert info["status"] == "ok" and info["iters"] == 1
    assert np.allclose(x, b / (3.0 - 1.0j), rtol=1e-14, atol=0)


def test_tfqmr_matches_dense_lu_and_degenerate_cases():
    for p, vals in _tiny_problems():
        b = g.complex_vector(p.n, 22) * (~p.dirichlet)
        xs = oracle.dense_solve(p.rowptr, p.colind, vals, b)
        x, info = oracle.tfqmr(p.rowptr, p.colind, vals, b, tol=1e-12, maxit=10000)
        assert info["status"] == "ok" and info["relres_true"] <= 1e-12
        cond = np.linalg.cond(oracle.densify(p.rowptr, p.colind, vals))
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 10 * cond * 1e-12
    p, vals = _tiny_problems()[1]
    x, info = oracle.tfqmr(p.rowptr, p.colind, vals, np.zeros(p.n, np.complex128))
    assert info["status"] == "ok" and info["iters"] == 0 and np.all(x == 0)
    b = g.complex_vector(p.n, 23) * (~p.dirichlet)
    x, info = oracle.tfqmr(p.rowptr, p.colind, vals, b, tol=1e-30, maxit=1)
    assert info["status"] == "not_converged" and info["iters"] == 1
    bad = b.copy()
    bad[2] = np.nan
    assert oracle.tfqmr(p.rowptr, p.colind, vals, bad)[1]["status"] == "nonfinite"


@pytest.mark.parametrize("k", [2, 3, 4])
def test_krylov_methods_terminate_in_the_number_of_distinct_eigenvalues(k):
    """With k distinct eigenvalues the Krylov space of b has dimension k, so
    the BiCG process underneath all three methods ends after k steps: TFQMR
    (k CGS steps, two quasi-minimal-residual half-steps each) within k
    iterations, BiCGStab(l) (l BiCG steps per cycle) within ceil(k/l) cycles.
    A wrong coefficient or index in either recurrence delays that."""
    d = np.array([1.0, 2.0 + 1j, 3.0 - 2j, 0.5 + 0.5j][:k] * 5)
    rp, ci, v = _csr_diag(d)
    b = g.complex_vector(d.size, 8)
    x, info = oracle.tfqmr(rp, ci, v, b, tol=1e-12)
    assert info["status"] == "ok" and info["iters"] <= k
    assert np.allclose(x, b / d, rtol=1e-12, atol=0)
    for ell in (1, 2, 4):
        x, info = oracle.bicgstabl(rp, ci, v, b, ell=ell, tol=1e-12)
        assert info["status"] == "ok" and info["iters"] <= -(-k // ell), ell
        assert np.allclose(x, b / d, rtol=1e-12, atol=0)


def test_tfqmr_reports_ok_only_with_the_true_residual_below_tol():
    """TFQMR's stop test is a bound on the residual; near rounding level the
    recurrence drifts from b - A x, so the bound can pass while the true
    residual has not.  The oracle then checks the true residual and restarts
    from the current x: ok is reported only when b - A x itself meets tol
    (on these meshes the bound passes first from tol = 1e-15 down)."""
    cases = 0
    for dims, F in (((8, 6, 5), 700.0), ((9, 7, 6), 900.0)):
        p = g.assemble(g.tiny_config(*dims, h=0.1, F=F, seed=2))
        vals = g.helmholtz_values(p, F)
        b = g.source(p) + 0.1 * g.complex_vector(p.n, 4) * (~p.dirichlet)
        for tol in (1e-13, 1e-15, 3e-16):
            x, info = oracle.tfqmr(p.rowptr, p.colind, vals, b, tol=tol, maxit=3000)
            r = np.linalg.norm(b - oracle.spmv(p.rowptr, p.colind, vals, x)) / np.linalg.norm(b)
            assert abs(r - info["relres_true"]) <= 1e-3 * r
            if info["status"] == "ok":
                assert info["relres_true"] <= tol, (p.n, tol, info)
                cases += 1
    assert cases >= 5


@pytest.mark.parametrize("method", ["bicgstab", "bicgstabl"])
def test_bicgstab_reports_ok_only_with_the_true_residual_below_tol(method):
    """One acceptance rule for every method: near rounding level the
    BiCGStab recurrence drifts from b - A x, so its residual can pass tol
    while the true residual has not; the oracle then restarts from the current
    x, and reports ok only when b - A x itself, recomputed here with the plain
    SpMV, meets tol.  An oracle that accepted up to 1.5 tol (or took the
    recurrence's word) fails the assertion on these meshes."""
    cases = 0
    for dims, F in (((8, 6, 5), 700.0), ((9, 7, 6), 900.0)):
        p = g.assemble(g.tiny_config(*dims, h=0.1, F=F, seed=2))
        vals = g.helmholtz_values(p, F)
        b = g.source(p) + 0.1 * g.complex_vector(p.n, 4) * (~p.dirichlet)
        for tol in (1e-13, 1e-15, 3e-16):
            if method == "bicgstab":
                x, info = oracle.bicgstab(p.rowptr, p.colind, vals, b, tol=tol, maxit=3000)
            else:
                x, info = oracle.bicgstabl(p.rowptr, p.colind, vals, b, ell=2, tol=tol, maxit=1500)
            r = np.linalg.norm(b - oracle.spmv(p.rowptr, p.colind, vals, x)) / np.linalg.norm(b)
            assert abs(r - info["relres_true"]) <= 1e-3 * r
            if info["status"] == "ok":
                assert r <= tol * (1 + 1e-3), (p.n, tol, info)
                cases += 1
            else:
                assert info["status"] == "not_converged" and info["relres_true"] > tol
    assert cases >= 3


# ---------------------------------------------------------------- BiCGStab(l)

@pytest.mark.parametrize("ell", [1, 2, 4, 8])
def test_bicgstabl_matches_dense_lu(ell):
    for p, vals in _tiny_problems():
        b = g.complex_vector(p.n, 24) * (~p.dirichlet)
        xs = oracle.dense_solve(p.rowptr, p.colind, vals, b)
        x, info = oracle.bicgstabl(p.rowptr, p.colind, vals, b, ell=ell, tol=1e-12, maxit=10000)
        assert info["status"] == "ok" and info["relres_true"] <= 1.5e-12
        cond = np.linalg.cond(oracle.densify(p.rowptr, p.colind, vals))
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 10 * cond * 1e-12


def test_bicgstabl_one_is_bicgstab_and_special_cases():
    # l = 1 is mathematically BiCGStab: same iteration count on small systems
    for p, vals in _tiny_problems()[1:]:
        b = g.complex_vector(p.n, 25) * (~p.dirichlet)
        _, i1 = oracle.bicgstabl(p.rowptr, p.colind, vals, b, ell=1, tol=1e-12)
        _, ib = oracle.bicgstab(p.rowptr, p.colind, vals, b, tol=1e-12)
        assert abs(i1["iters"] - ib["iters"]) <= 1
    rp, ci, v = _csr_diag(np.full(9, 1.5 + 0.5j))
    b = g.complex_vector(9, 6)
    x, info = oracle.bicgstabl(rp, ci, v, b, ell=4, tol=1e-12)
    assert info["status"] == "ok" and info["iters"] == 1 and np.allclose(x, b / (1.5 + 0.5j), rtol=1e-13)
    p, vals = _tiny_problems()[1]
    x, info = oracle.bicgstabl(p.rowptr, p.colind, vals, np.zeros(p.n, np.complex128), ell=2)
    assert info["status"] == "ok" and info["iters"] == 0 and np.all(x == 0)


# ---------------------------------------------------------------- right Jacobi

def test_jacobi_scale_is_column_scaling_by_the_diagonal():
    """A D^-1 equals the dense product with diag(1/a_ii); its diagonal is 1; a
    row without a stored diagonal keeps scale 1 (pins against dense algebra)."""
    for p, vals in _tiny_problems():
        vs, d, dinv = oracle.jacobi_scale(p.rowptr, p.colind, vals)
        A = oracle.densify(p.rowptr, p.colind, vals)
        assert np.array_equal(d, np.diag(A))
        As = oracle.densify(p.rowptr, p.colind, vs)
        assert np.allclose(As, A @ np.diag(1.0 / np.diag(A)), rtol=0, atol=4 * EPS * np.abs(As).max())
        assert np.allclose(np.diag(As), 1.0, rtol=0, atol=4 * EPS)
    # row 1 stores no diagonal
    rowptr = np.array([0, 2, 4, 6], np.int32)
    colind = np.array([0, 2, 0, 2, 1, 2], np.int32)
    vals = np.array([2.0, 1.0, 1.0, 3.0, 4.0, 5.0 + 1j], np.complex128)
    vs, d, dinv = oracle.jacobi_scale(rowptr, colind, vals)
    assert np.array_equal(d, [2.0, 1.0, 5.0 + 1j])
    b = np.array([1.0, 2.0, 3.0 - 1j])
    x, info = oracle.jacobi_solve(oracle.bicgstab, rowptr, colind, vals, b, tol=1e-14, maxit=100)
    assert info["status"] == "ok"
    assert np.allclose(x, np.linalg.solve(oracle.densify(rowptr, colind, vals), b), rtol=1e-12)


@pytest.mark.parametrize("method", ["bicgstab", "tfqmr", "bicgstabl"])
def test_jacobi_solve_matches_dense_lu(method):
    fn = getattr(oracle, method)
    for p, vals in _tiny_problems():
        b = g.complex_vector(p.n, 26) * (~p.dirichlet)
        xs = oracle.dense_solve(p.rowptr, p.colind, vals, b)
        x, info = oracle.jacobi_solve(fn, p.rowptr, p.colind, vals, b, tol=1e-12, maxit=10000)
        assert info["status"] == "ok"
        # the true residual it reports is that of A D^-1 y = b, i.e. of A x = b
        r = np.linalg.norm(b - oracle.spmv(p.rowptr, p.colind, vals, x)) / np.linalg.norm(b)
        assert r <= 2e-12
        cond = np.linalg.cond(oracle.densify(p.rowptr, p.colind, vals))
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 10 * cond * 1e-12


# ---------------------------------------------------------------- restricted additive Schwarz

def _csr_of_dense(D):
    rp, ci, vv = [0], [], []
    for i in range(D.shape[0]):
        nz = np.nonzero(D[i])[0]
        ci.extend(nz.tolist())
        vv.extend(D[i, nz].tolist())
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32), np.array(vv, np.complex128)


def test_ras_closed_form_on_a_tridiagonal_matrix():
    """tridiag(-1, 2, -1) of order 4, two blocks, overlap 1: the extended
    blocks are rows 0-2 and 1-3, each the 3x3 matrix whose inverse is
    [[3, 2, 1], [2, 4, 2], [1, 2, 3]] / 4.  For r = e_1 block 0 keeps rows 0, 1
    of (2, 4, 2) / 4 and block 1 rows 1, 2 (its rows 2, 3 of A) of
    (3, 2, 1) / 4: z = (1/2, 1, 1/2, 1/4)."""
    T = 2 * np.eye(4) - np.eye(4, k=1) - np.eye(4, k=-1)
    rp, ci, vv = _csr_of_dense(T.astype(np.complex128))
    z = oracle.ras_apply(rp, ci, vv, np.array([0, 1, 0, 0], np.complex128), nsub=2, overlap=1)
    assert np.allclose(z, [0.5, 1.0, 0.5, 0.25], rtol=0, atol=1e-15)
    assert oracle.ddm_blocks(4, 2, 1) == [(0, 2, 0, 3), (2, 4, 1, 4)]
    # with the impedance term: block 0's row 2 loses |a_23| = 1, block 1's
    # first row (row 1 of A) loses |a_10| = 1, so the blocks are
    # [[2,-1,0],[-1,2,-1],[0,-1,2+i]] and [[2+i,-1,0],[-1,2,-1],[0,-1,2]];
    # solving them by hand gives y = (11-2i, 22-4i, .)/25 and (., 8-6i, 4-3i)/25
    z = oracle.ras_apply(rp, ci, vv, np.array([0, 1, 0, 0], np.complex128), nsub=2, overlap=1, impedance=True)
    assert np.allclose(z, np.array([11 - 2j, 22 - 4j, 8 - 6j, 4 - 3j]) / 25, rtol=0, atol=1e-15)
    assert oracle.ddm_blocks(10, 3, 2) == [(0, 3, 0, 5), (3, 6, 1, 8), (6, 10, 4, 10)]


def test_ras_is_the_inverse_where_the_blocks_do_not_couple():
    """One block (any overlap), or a block-diagonal matrix split along its
    blocks (any overlap): the restricted additive Schwarz operator is A^-1
    itself, with or without the impedance term (no row loses a coupling).
    And it is linear in r."""
    p = g.assemble(g.tiny_config(3, 3, 2, h=0.1, seed=4))
    vals = g.helmholtz_values(p, 500.0)
    r = g.complex_vector(p.n, 30)
    xs = oracle.dense_solve(p.rowptr, p.colind, vals, r)
    for ov in (0, 3, 100):
        assert np.allclose(oracle.ras_apply(p.rowptr, p.colind, vals, r, 1, ov), xs, rtol=1e-12, atol=0)
    A = oracle.densify(p.rowptr, p.colind, vals)
    B = np.zeros((2 * p.n, 2 * p.n), np.complex128)
    B[:p.n, :p.n] = A
    B[p.n:, p.n:] = 2.0 * A
    rp, ci, vv = _csr_of_dense(B)
    r2 = g.complex_vector(2 * p.n, 31)
    exact = np.linalg.solve(B, r2)
    for ov in (0, 5):
        assert np.allclose(oracle.ras_apply(rp, ci, vv, r2, 2, 0), exact, rtol=1e-12, atol=0)
        assert np.allclose(oracle.ras_apply(rp, ci, vv, r2, 2, 0, impedance=True), exact, rtol=1e-12, atol=0)
        assert np.allclose(oracle.ras_apply(rp, ci, vv, r2, 2, ov), exact, rtol=1e-12, atol=0)
    ra = oracle.ras_apply(p.rowptr, p.colind, vals, r, 3, 4)
    rb = oracle.ras_apply(p.rowptr, p.colind, vals, 2j * r + xs, 3, 4)
    rc = oracle.ras_apply(p.rowptr, p.colind, vals, xs, 3, 4)
    assert np.allclose(rb, 2j * ra + rc, rtol=1e-12, atol=1e-14 * np.abs(rb).max())
