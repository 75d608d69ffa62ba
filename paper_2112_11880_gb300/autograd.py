"""Differentiable Helmholtz solve for PyTorch: the adjoint of u = A(c)^{-1} b.

Two torch.autograd.Functions, each a thin shell over libhelm kernels:

  AssembleHelmholtz.apply(c, fem) -> vals
      forward : helm_assemble_helmholtz, A(c) = K - w^2 M_c(c) + i w B_c(c)
      backward: helm_conj_scale (PyTorch -> holomorphic convention) and
                helm_grad_sound_speed (chain onto per-element c)
  SolveHelmholtz.apply(vals, b, fem, opts) -> u
      forward : helm_csr_create + helm_bicgstab_solve
      backward: helm_conj_scale, helm_adjoint (A^T mu = dL/du, dL/dA = -mu u^T
                on the stored entries), helm_conj_scale back to PyTorch's
                convention for dL/db and dL/dvals

PyTorch's gradient of a real loss with respect to a complex tensor z is
2 conj(dL/dz) with dL/dz the holomorphic (Wirtinger) derivative; the library
works with dL/dz and the conversions are the helm_conj_scale calls.
"""
from __future__ import annotations

import torch

from . import (CsrMatrix, HelmError, _check_vector, default_opts, helm_adjoint, helm_assemble_helmholtz,
               helm_bicgstab_solve, helm_conj_scale, helm_grad_sound_speed)


class HelmholtzFEM:
    """GPU-resident data of one Helmholtz FEM problem at angular frequency w:
    CSR pattern, the c-independent K values, the slot -> (element, pair) table
    for assembly, the element -> slot map for the gradient, the element mass
    and impedance-face matrices and the top-element flags."""

    def __init__(self, rowptr, colind, K, slot_elem, slot_pair, elem_map, Me, Bf, top, omega, device="cuda"):
        dev = torch.device(device)
        t = lambda a, dt: torch.as_tensor(a).to(device=dev, dtype=dt).contiguous()  # noqa: E731
        self.device = dev
        self.rowptr = t(rowptr, torch.int32)
        self.colind = t(colind, torch.int32)
        self.K = t(K, torch.float64)
        self.slot_elem = t(slot_elem, torch.int32)
        self.slot_pair = t(slot_pair, torch.uint8)
        self.elem_map = t(elem_map, torch.int32)
        self.top = t(top, torch.uint8)
        self.Me = torch.as_tensor(Me, dtype=torch.float64).reshape(64).cpu().numpy()
        self.Bf = torch.as_tensor(Bf, dtype=torch.float64).reshape(64).cpu().numpy()
        self.omega = float(omega)
        self.n = self.rowptr.numel() - 1
        self.nnz = self.colind.numel()
        self.n_elem = self.top.numel()

    def assemble(self, c: torch.Tensor) -> torch.Tensor:
        vals = torch.empty(self.nnz, dtype=torch.complex128, device=self.device)
        helm_assemble_helmholtz(self.K, self.slot_elem, self.slot_pair, self.Me, self.Bf, self.top,
                                c.detach().contiguous(), self.omega, vals)
        return vals


class AssembleHelmholtz(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, fem: HelmholtzFEM):
        if c.dtype != torch.float64 or c.numel() != fem.n_elem:
            raise ValueError("c must be float64 with one entry per element")
        ctx.fem = fem
        ctx.save_for_backward(c)
        return fem.assemble(c)

    @staticmethod
    def backward(ctx, grad_vals):
        (c,) = ctx.saved_tensors
        fem = ctx.fem
        G = torch.empty_like(grad_vals)
        helm_conj_scale(0.5, grad_vals.contiguous(), G)          # holomorphic dL/dA
        grad_c = torch.empty_like(c)
        helm_grad_sound_speed(G, fem.elem_map, fem.Me, fem.Bf, fem.top, c.contiguous(), fem.omega, grad_c)
        return grad_c, None


class SolveHelmholtz(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, b, fem: HelmholtzFEM, opts=None):
        _check_vector(b, fem.n, torch.complex128, "b")
        A = CsrMatrix(fem.rowptr, fem.colind, vals.detach().contiguous())
        u = torch.empty_like(b)
        o = opts if opts is not None else default_opts()
        info = helm_bicgstab_solve(A.handle, b.detach().contiguous(), u, o)
        if info["status"] != "ok":
            A.close()
            raise HelmError(4, f"forward solve: {info}")
        ctx.A = A
        ctx.opts = o
        ctx.info = info
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        A = ctx.A
        w = torch.empty_like(u)
        helm_conj_scale(0.5, grad_u.contiguous(), w)             # holomorphic dL/du
        mu = torch.empty_like(u)
        G = torch.empty(A.nnz, dtype=torch.complex128, device=u.device)
        info = helm_adjoint(A.handle, u, w, mu, G, ctx.opts)
        A.close()
        if info["status"] != "ok":
            raise HelmError(4, f"adjoint solve: {info}")
        grad_b = torch.empty_like(mu)
        helm_conj_scale(2.0, mu, grad_b)
        grad_vals = torch.empty_like(G)
        helm_conj_scale(2.0, G, grad_vals)
        return grad_vals, grad_b, None, None


def solve_sound_speed(c, b, fem: HelmholtzFEM, opts=None):
    """u = A(c)^{-1} b, differentiable in c (float64 per element) and b."""
    return SolveHelmholtz.apply(AssembleHelmholtz.apply(c, fem), b, fem, opts)
