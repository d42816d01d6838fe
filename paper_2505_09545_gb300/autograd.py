"""torch.autograd.Function wrappers around the C ABI (argument marshalling only).

`scatter(pos, eps, wavelength, ...)` -> (F, sigma) runs gdm_assemble + gdm_solve + gdm_cross_sections;
its backward calls gdm_backward (adjoint solve with the same LU factors). `scatter_spectrum` does the same
for many wavelengths at once through gdm_solve_batched / gdm_backward_batched. `nearfield(...)` runs
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


class _ScatterSpectrum(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, eps, wavelengths, gctx, step, e0, khat, precision, n_streams):
        lams = [float(v) for v in wavelengths.detach().cpu().tolist()]
        pos_d, eps_d = pos.detach().contiguous(), eps.detach().contiguous()
        probs = [B.GDMProblem(pos_d, lam, 3, eps=eps_d, step=step) for lam in lams]
        Fs, sigs, _, As, ipivs = B.solve_batched(gctx, probs, [e0] * len(lams), precision=precision, khat=khat,
                                                 n_streams=n_streams, return_factors=True)
        ctx.gctx, ctx.probs, ctx.As, ctx.ipivs, ctx.Fs = gctx, probs, As, ipivs, Fs
        ctx.e0, ctx.khat, ctx.precision, ctx.n_streams = e0, khat, precision, n_streams
        return torch.stack(Fs), torch.stack([s.t() for s in sigs])

    @staticmethod
    def backward(ctx, gF, gsig):
        L = len(ctx.probs)
        gFs = None if gF is None else [(0.5 * gF[i]).contiguous() for i in range(L)]
        gs = None if gsig is None else [gsig[i].detach().double().cpu().numpy() for i in range(L)]
        gp, ge, gl, _ = B.backward_batched(ctx.gctx, ctx.probs, ctx.As, ctx.ipivs, ctx.Fs, ctx.e0,
                                           precision=ctx.precision, khat=ctx.khat, gFs=gFs, g_sigmas=gs,
                                           n_streams=ctx.n_streams)
        return gp, ge, gl, None, None, None, None, None, None


def scatter_spectrum(pos, eps, wavelengths, gctx, step, e0, khat=(0.0, 0.0, 1.0), precision="fp32", n_streams=0):
    """Differentiable solves of one structure at several wavelengths (a 1-D tensor): returns F
    ((L, n_rhs, 3N) complex128) and sigma ((L, n_rhs, 3): ext, sca, abs). The wavelengths run concurrently
    (gdm_solve_batched forward, gdm_backward_batched backward); the gradients with respect to pos and eps
    are summed over the wavelengths, the one with respect to each wavelength is its own."""
    return _ScatterSpectrum.apply(pos, eps, wavelengths, gctx, step, e0, khat, precision, n_streams)


def scatter(pos, eps, wavelength, gctx, step, e0, khat=(0.0, 0.0, 1.0), precision="fp32"):
    """Differentiable solve: returns F ((n_rhs, 3N) complex128) and sigma ((n_rhs, 3): ext, sca, abs)."""
    return _Scatter.apply(pos, eps, wavelength, gctx, step, e0, khat, precision)


def nearfield(pos, eps, wavelength, F, r_eval, gctx, step, e0, khat=(0.0, 0.0, 1.0)):
    """Differentiable near field E ((n_rhs, 3m) complex128) at r_eval from the solved fields F."""
    return _Nearfield.apply(pos, eps, wavelength, F, r_eval, gctx, step, e0, khat)
