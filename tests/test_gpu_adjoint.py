"""GPU parity of the adjoint path: assembly of A(c), the adjoint solve and the
scatter onto stored entries, the chain onto per-element sound speed, and the
torch.autograd.Function end to end -- against the oracle, a dense reference
gradient, and central finite differences along random directions on the
80x40x32 cavity (gate 1e-6)."""
import numpy as np
import pytest

import helmgen as g
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2112_11880_gb300 as helm  # noqa: E402
from paper_2112_11880_gb300 import autograd as hgrad  # noqa: E402

DEV = torch.device("cuda:0")


def _fem(p, F):
    m = g.element_nnz_map(p)
    se, sp = g.slot_elements(p, m)
    _, Me, Bf = g.element_matrices(p.cfg.h)
    return hgrad.HelmholtzFEM(p.rowptr, p.colind, p.K, se, sp, m, Me, Bf, g.top_elements(p.cfg), g.omega(F), DEV)


def _setup(cfg, nrec=6):
    p = g.assemble(cfg)
    b = g.source(p) + 0.3 * g.complex_vector(p.n, 2) * (~p.dirichlet)
    rec = g.receivers(p, nrec, seed=1)
    pt = g.assemble(cfg, c=g.sound_speed(cfg, seed=2))
    return p, b, rec, pt


@pytest.mark.parametrize("name", ["tiny", "adjoint80"])
def test_assembly_matches_generator_bit_for_bit(name):
    cfg = g.tiny_config(3, 2, 3, h=0.1, F=450.0, seed=4) if name == "tiny" else g.CONFIGS[name]
    p = g.assemble(cfg)
    fem = _fem(p, cfg.F)
    vals = fem.assemble(torch.as_tensor(p.c, device=DEV)).cpu().numpy()
    ref = g.helmholtz_values(p, cfg.F)
    assert np.array_equal(vals.view(np.float64), ref.view(np.float64))


def test_adjoint_scatter_and_chain_vs_oracle():
    cfg = g.tiny_config(4, 3, 3, h=0.1, F=450.0, seed=4)
    p, b, rec, pt = _setup(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    d = oracle.dense_solve(pt.rowptr, pt.colind, g.helmholtz_values(pt, cfg.F), b)[rec]
    u = oracle.dense_solve(p.rowptr, p.colind, vals, b)
    w = oracle.adjoint_rhs(p.n, u, rec, d)
    mu_ref = oracle.dense_solve(p.rowptr, p.colind, vals, w)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    mu = torch.empty(p.n, dtype=torch.complex128, device=DEV)
    G = torch.empty(p.nnz, dtype=torch.complex128, device=DEV)
    info = helm.helm_adjoint(A.handle, torch.as_tensor(u, device=DEV), torch.as_tensor(w, device=DEV), mu, G,
                             helm.default_opts(tol=1e-13, maxit=50000))
    assert info["status"] == "ok"
    mu_h = mu.cpu().numpy()
    assert np.linalg.norm(mu_h - mu_ref) <= 1e-9 * np.linalg.norm(mu_ref)
    G_ref = oracle.nnz_gradient(p.rowptr, p.colind, mu_h, u)
    assert np.array_equal(G.cpu().numpy(), G_ref) or np.max(np.abs(G.cpu().numpy() - G_ref)) <= 1e-15 * np.max(np.abs(G_ref))
    fem = _fem(p, cfg.F)
    grad = torch.empty(cfg.n_elem, dtype=torch.float64, device=DEV)
    helm.helm_grad_sound_speed(G, fem.elem_map, fem.Me, fem.Bf, fem.top, torch.as_tensor(p.c, device=DEV),
                               fem.omega, grad)
    _, Me, Bf = g.element_matrices(cfg.h)
    ref = oracle.sound_speed_gradient(G_ref, g.element_nnz_map(p), Me, Bf, p.c, g.omega(cfg.F),
                                      g.top_elements(cfg).astype(bool))
    assert np.max(np.abs(grad.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    A.close()


def test_adjoint_rejects_overlapping_outputs():
    """mu and dL/dA may not share memory with u, dL/du or each other."""
    cfg = g.tiny_config(3, 3, 3, h=0.1, F=400.0, seed=4)
    p = g.assemble(cfg)
    vals = g.helmholtz_values(p, cfg.F)
    A = helm.CsrMatrix.from_host(p.rowptr, p.colind, vals, device=DEV)
    n = p.n
    buf = torch.as_tensor(g.complex_vector(3 * n + 1, 2), device=DEV)
    u, w = buf[0:n], buf[n:2 * n]
    G = torch.empty(p.nnz, dtype=torch.complex128, device=DEV)
    for mu in (buf[1:n + 1], buf[n + 1:2 * n + 1]):
        with pytest.raises(helm.HelmError):
            helm.helm_adjoint(A.handle, u, w, mu, G)
    mu = buf[2 * n:3 * n]
    Gb = torch.empty(p.nnz + n, dtype=torch.complex128, device=DEV)
    with pytest.raises(helm.HelmError):
        helm.helm_adjoint(A.handle, u, w, Gb[0:n], Gb[1:p.nnz + 1])
    info = helm.helm_adjoint(A.handle, u, w, mu, G, helm.default_opts(tol=1e-10))
    assert info["status"] == "ok"
    A.close()


def _loss_gpu(c, b, fem, rec, d, opts):
    with torch.no_grad():
        u = hgrad.solve_sound_speed(c, b, fem, opts)
    e = u[rec] - d
    return float(torch.sum(e.real ** 2 + e.imag ** 2))


def test_autograd_matches_dense_reference_gradient():
    cfg = g.tiny_config(3, 2, 3, h=0.1, F=450.0, seed=4)
    p, b, rec, pt = _setup(cfg)
    d = oracle.dense_solve(pt.rowptr, pt.colind, g.helmholtz_values(pt, cfg.F), b)[rec]
    # dense reference gradient (oracle chain with dense solves)
    vals = g.helmholtz_values(p, cfg.F)
    u = oracle.dense_solve(p.rowptr, p.colind, vals, b)
    mu = oracle.dense_solve(p.rowptr, p.colind, vals, oracle.adjoint_rhs(p.n, u, rec, d))
    _, Me, Bf = g.element_matrices(cfg.h)
    ref = oracle.sound_speed_gradient(oracle.nnz_gradient(p.rowptr, p.colind, mu, u), g.element_nnz_map(p), Me, Bf,
                                      p.c, g.omega(cfg.F), g.top_elements(cfg).astype(bool))
    fem = _fem(p, cfg.F)
    c = torch.as_tensor(p.c, device=DEV).requires_grad_(True)
    bt = torch.as_tensor(b, device=DEV).requires_grad_(True)
    u_t = hgrad.solve_sound_speed(c, bt, fem, helm.default_opts(tol=1e-13, maxit=50000))
    dt = torch.as_tensor(d, device=DEV)
    e = u_t[torch.as_tensor(rec, device=DEV)] - dt
    L = torch.sum(e.real ** 2 + e.imag ** 2)
    L.backward()
    assert np.max(np.abs(c.grad.cpu().numpy() - ref)) <= 1e-8 * np.max(np.abs(ref))
    gb_ref = 2 * np.conj(mu)
    assert np.max(np.abs(bt.grad.cpu().numpy() - gb_ref)) <= 1e-8 * np.max(np.abs(gb_ref))


def test_adjoint80_gradient_against_central_differences():
    """80x40x32 cavity, 64 receivers, loss sum |u_r - d_r|^2: the adjoint
    gradient along 20 random unit directions matches central differences to
    1e-6, and likewise for the source.  The difference quotient is only as
    good as the solves behind it: its noise is about kappa * tol * L / eps, so
    the solves run to 1e-13 and the step is eps = 1 m/s (3e-3 of c) with the
    fourth-order central stencil, whose O(eps^4) truncation stays below 1e-8
    (measured worst case 2.6e-7; second order at 0.1 m/s gave 7.9e-7)."""
    cfg = g.CONFIGS["adjoint80"]
    p = g.assemble(cfg)
    b = torch.as_tensor(g.source(p), device=DEV)
    rec_np = g.receivers(p, 64, seed=1)
    rec = torch.as_tensor(rec_np, device=DEV)
    fem = _fem(p, cfg.F)
    opts = helm.default_opts(tol=1e-13, maxit=300000)
    c_true = torch.as_tensor(g.sound_speed(cfg, seed=2), device=DEV)
    with torch.no_grad():
        d = hgrad.solve_sound_speed(c_true, b, fem, opts)[rec]
    c0 = torch.as_tensor(p.c, device=DEV)
    c = c0.clone().requires_grad_(True)
    bt = b.clone().requires_grad_(True)
    u = hgrad.solve_sound_speed(c, bt, fem, opts)
    e = u[rec] - d
    L = torch.sum(e.real ** 2 + e.imag ** 2)
    L.backward()
    grad = c.grad.detach()
    rng = np.random.default_rng(3)
    eps = 1.0
    worst = 0.0
    for _ in range(20):
        v = rng.standard_normal(cfg.n_elem)
        v /= np.linalg.norm(v)
        vt = torch.as_tensor(v, device=DEV)
        f = {k: _loss_gpu(c0 + k * eps * vt, b, fem, rec, d, opts) for k in (-2, -1, 1, 2)}
        fd = (-f[2] + 8 * f[1] - 8 * f[-1] + f[-2]) / (12 * eps)
        ad = float(torch.dot(grad, vt))
        worst = max(worst, abs(fd - ad) / max(abs(ad), 1e-300))
    print(f"adjoint80: max relative FD mismatch over 20 directions {worst:.2e}")
    assert worst <= 1e-6
    # source: one complex direction on the receivers' neighbourhood
    vb = torch.as_tensor(g.complex_vector(p.n, 5) * (~p.dirichlet), device=DEV)
    vb = vb / torch.linalg.vector_norm(vb)
    eps_b = 1e-4 * float(torch.linalg.vector_norm(b))
    fd = (_loss_gpu(c0, b + eps_b * vb, fem, rec, d, opts) - _loss_gpu(c0, b - eps_b * vb, fem, rec, d, opts)) / (2 * eps_b)
    ad = float(torch.sum(bt.grad.real * vb.real + bt.grad.imag * vb.imag))
    assert abs(fd - ad) <= 1e-6 * abs(ad)
