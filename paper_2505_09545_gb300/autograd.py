"""torch.autograd.Function wrappers around the C ABI (argument marshalling only).

`scatter(pos, eps, wavelength, ...)` -> (F, sigma) runs gdm_assemble + gdm_solve + gdm_cross_sections;
its backward calls gdm_backward (adjoint solve with the same LU factors). `nearfield(...)` runs
gdm_nearfield; its backward calls gdm_nearfield_backward. Complex gradients follow PyTorch's
convention (dL/dRe + i dL/dIm = 2 dL/dz^*); the C ABI takes and returns conjugate Wirtinger
derivatives dL/dz^*, hence the factors of 2 below.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class _Scatter(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, eps, wavelength, gctx, step, e0, khat, precision):
        lam = float(wavelength.detach().cpu())
        prob = B.GDMProblem(pos.detach().contiguous(), lam, 3, eps=eps.detach().contiguous(), step=step)
        F0 = B.incident_planewave(gctx, prob.pos, lam, e0, khat)
        A = B.assemble(gctx, prob, precision)
        F, ipiv, _ = B.solve(gctx, prob, A, F0, precision)
        e2 = np.sum(np.abs(np.atleast_2d(e0)) ** 2, axis=1)
        ext, sca, ab = B.cross_sections(gctx, prob, F0, F, e2)
        ctx.gctx, ctx.prob, ctx.A, ctx.ipiv, ctx.F = gctx, prob, A, ipiv, F
        ctx.e0, ctx.khat, ctx.precision = e0, khat, precision
        return F, torch.stack([ext, sca, ab], dim=-1)

    @staticmethod
    def backward(ctx, gF, gsig):
        gF_w = None if gF is None else (0.5 * gF).contiguous()
        g_sigma = None if gsig is None else gsig.detach().double().cpu().numpy()
        gp, ge, gl, _ = B.backward(ctx.gctx, ctx.prob, ctx.A, ctx.ipiv, ctx.F, ctx.e0, ctx.khat, gF=gF_w,
                                   g_sigma=g_sigma, precision=ctx.precision)
        return gp, ge, gl.reshape(()), None, None, None, None, None


class _Nearfield(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, eps, wavelength, F, r_eval, gctx, step, e0, khat):
        lam = float(wavelength.detach().cpu())
        prob = B.GDMProblem(pos.detach().contiguous(), lam, 3, eps=eps.detach().contiguous(), step=step)
        F0e = B.incident_planewave(gctx, r_eval, lam, e0, khat, kind_out=6)
        E, _ = B.nearfield(gctx, prob, F.detach().contiguous(), r_eval.contiguous(), F0e, with_h=False)
        ctx.gctx, ctx.prob, ctx.F, ctx.r_eval, ctx.e0, ctx.khat = gctx, prob, F.detach(), r_eval, e0, khat
        return E

    @staticmethod
    def backward(ctx, gE):
        p = ctx.prob
        dev = gE.device
        gF = torch.zeros_like(ctx.F)
        gp = torch.zeros((p.n, 3), dtype=torch.float64, device=dev)
        ge = torch.zeros(p.n, dtype=torch.complex128, device=dev)
        gl = torch.zeros(1, dtype=torch.float64, device=dev)
        B.nearfield_backward(ctx.gctx, p, ctx.F, ctx.r_eval, ctx.e0, (0.5 * gE).contiguous(), ctx.khat,
                             gF_accum=gF, grad_pos=gp, grad_eps=ge, grad_wavelength=gl)
        return gp, ge, gl.reshape(()), 2.0 * gF, None, None, None, None, None


def scatter(pos, eps, wavelength, gctx, step, e0, khat=(0.0, 0.0, 1.0), precision="fp32"):
    """Differentiable solve: returns F ((n_rhs, 3N) complex128) and sigma ((n_rhs, 3): ext, sca, abs)."""
    return _Scatter.apply(pos, eps, wavelength, gctx, step, e0, khat, precision)


def nearfield(pos, eps, wavelength, F, r_eval, gctx, step, e0, khat=(0.0, 0.0, 1.0)):
    """Differentiable near field E ((n_rhs, 3m) complex128) at r_eval from the solved fields F."""
    return _Nearfield.apply(pos, eps, wavelength, F, r_eval, gctx, step, e0, khat)
