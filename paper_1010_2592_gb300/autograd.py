"""torch.autograd.Function around f(A) b and its adjoint (argument marshalling only).

    y = FAFunction.apply(U, mu, b, ctx, mass, t_bc, scale, solver_kwargs)

forward: loads U and mu into the library context and returns y = f(A) b
(fa_apply_f, any mode/precision in solver_kwargs).  backward: with
eta = dL/dy (torch's convention for a real loss of a complex tensor; for
L = Re <eta, y> it is eta itself) it calls fa_grad, which recomputes the
shift solutions by a single-pass FP64 solve, solves the adjoint systems with
A^H = A(-mu) and runs the link-force kernel; it returns dL/dU, dL/dmu and
dL/db.  The scale c of A is held fixed.  Nothing is stored between forward
and backward except the inputs: the recomputation replaces storing the
N_s shift solutions.
"""
from __future__ import annotations

import torch


class FAFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, U, mu, b, ctx, mass, t_bc, scale, solver_kwargs):
        ctx.set_gauge(U.detach().contiguous())
        ctx.set_params(mass, float(mu), t_bc, scale)
        y = ctx.apply_f(b.detach().contiguous(), **solver_kwargs).y
        fctx.save_for_backward(U, mu, b)
        fctx.fa = (ctx, mass, t_bc, scale, solver_kwargs)
        return y

    @staticmethod
    def backward(fctx, gy):
        U, mu, b = fctx.saved_tensors
        ctx, mass, t_bc, scale, kw = fctx.fa
        ctx.set_gauge(U.detach().contiguous())
        ctx.set_params(mass, float(mu), t_bc, scale)
        _, gU, gmu, gb, _ = ctx.grad(b.detach().contiguous(), gy.contiguous(),
                                     ell=kw.get("ell", 2), tol=min(kw.get("tol", 1e-10), 1e-12))
        gmu_t = torch.tensor(gmu, dtype=mu.dtype, device=mu.device)
        return gU, gmu_t, gb, None, None, None, None, None
