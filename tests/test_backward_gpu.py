"""GPU adjoint gradients (gdm_backward, gdm_nearfield_backward, autograd wrappers) against the
oracle's FP64 adjoint (1e-8 normwise) and against central finite differences of the GPU forward
(h = 1e-4, 1e-5 relative per directional derivative)."""
import numpy as np
import pytest
import torch

import gdm_workloads as W
import oracle as O

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


@pytest.fixture(scope="module")
def G():
    import paper_2505_09545_gb300 as G
    return G


@pytest.fixture(scope="module")
def ctx(G):
    c = G.Context(0)
    yield c
    c.close()


def small_cylinder():
    cyl = W.cylinder_diff(radius=30.0, height=40.0, step=10.0)
    rng = np.random.default_rng(11)
    cyl.eps = cyl.eps + rng.uniform(-0.5, 0.5, cyl.n)
    return cyl


def gpu_loss_and_grads(G, ctx, cyl, lam, precision):
    from paper_2505_09545_gb300 import autograd as AG
    pos = torch.tensor(cyl.pos, device=DEV, requires_grad=True)
    eps = torch.tensor(cyl.eps, device=DEV, requires_grad=True)
    wl = torch.tensor(lam, dtype=torch.float64, device=DEV, requires_grad=True)
    rp = torch.tensor(cyl.r_eval, device=DEV)
    F, sig = AG.scatter(pos, eps, wl, ctx, cyl.step, cyl.e0, precision=precision)
    E = AG.nearfield(pos, eps, wl, F, rp, ctx, cyl.step, cyl.e0)
    L = (E.abs() ** 2).sum() + sig[:, 1].sum()
    L.backward()
    return float(L.detach()), pos.grad.cpu().numpy(), eps.grad.cpu().numpy(), float(wl.grad)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32"])
def test_backward_matches_oracle_adjoint(G, ctx, precision):
    cyl = small_cylinder()
    for lam in (450.0, 700.0):
        L, gp, ge, gl = gpu_loss_and_grads(G, ctx, cyl, lam, precision)
        pr = O.Problem(cyl.pos, lam, 3, eps=cyl.eps, step=cyl.step)
        Lo, gpo, geo, glo = O.loss_and_grad_probe_sca(pr, cyl.e0, cyl.r_eval[0])
        assert abs(L - Lo) <= 1e-9 * abs(Lo)
        assert np.linalg.norm(gp - gpo) <= 1e-8 * np.linalg.norm(gpo)
        assert np.linalg.norm(ge - geo) <= 1e-8 * np.linalg.norm(geo)
        assert abs(gl - glo) <= 1e-8 * abs(glo) + 1e-14


def test_backward_matches_finite_differences(G, ctx):
    """Adjoint directional derivatives vs central differences of the GPU forward (FP64 path)."""
    from paper_2505_09545_gb300 import autograd as AG
    cyl = small_cylinder()
    lam = 600.0
    L0, gp, ge, gl = gpu_loss_and_grads(G, ctx, cyl, lam, "fp64")
    rp = torch.tensor(cyl.r_eval, device=DEV)

    def L(pos=cyl.pos, eps=cyl.eps, lm=lam):
        with torch.no_grad():
            F, sig = AG.scatter(torch.tensor(pos, device=DEV), torch.tensor(eps, device=DEV),
                                torch.tensor(lm, dtype=torch.float64, device=DEV), ctx, cyl.step, cyl.e0,
                                precision="fp64")
            E = AG.nearfield(torch.tensor(pos, device=DEV), torch.tensor(eps, device=DEV),
                             torch.tensor(lm, dtype=torch.float64, device=DEV), F, rp, ctx, cyl.step, cyl.e0)
            return float((E.abs() ** 2).sum() + sig[:, 1].sum())

    rng = np.random.default_rng(3)
    h = 1e-4
    for _ in range(4):
        v = rng.standard_normal(cyl.pos.shape)
        fd = (L(pos=cyl.pos + h * v) - L(pos=cyl.pos - h * v)) / (2 * h)
        np.testing.assert_allclose(np.sum(gp * v), fd, rtol=1e-5)
        w = rng.standard_normal(cyl.n) + 1j * rng.standard_normal(cyl.n)
        fd = (L(eps=cyl.eps + h * w) - L(eps=cyl.eps - h * w)) / (2 * h)
        np.testing.assert_allclose(np.sum(np.real(np.conj(ge) * w)), fd, rtol=1e-5)
    for (l, c) in [(0, 0), (cyl.n // 2, 2), (cyl.n - 1, 1)]:
        pp = cyl.pos.copy(); pp[l, c] += h
        pm = cyl.pos.copy(); pm[l, c] -= h
        fd = (L(pos=pp) - L(pos=pm)) / (2 * h)
        np.testing.assert_allclose(gp[l, c], fd, rtol=1e-5, atol=1e-7 * np.abs(gp).max())
    fd = (L(lm=lam + h) - L(lm=lam - h)) / (2 * h)
    np.testing.assert_allclose(gl, fd, rtol=1e-5)


def spectrum_loss_and_grads(G, ctx, cyl, lams, precision, n_streams):
    from paper_2505_09545_gb300 import autograd as AG
    pos = torch.tensor(cyl.pos, device=DEV, requires_grad=True)
    eps = torch.tensor(cyl.eps, device=DEV, requires_grad=True)
    wls = torch.tensor(lams, dtype=torch.float64, device=DEV, requires_grad=True)
    rp = torch.tensor(cyl.r_eval, device=DEV)
    F, sig = AG.scatter_spectrum(pos, eps, wls, ctx, cyl.step, cyl.e0, precision=precision, n_streams=n_streams)
    L = 0.0
    for i in range(len(lams)):
        E = AG.nearfield(pos, eps, wls[i], F[i], rp, ctx, cyl.step, cyl.e0)
        L = L + (E.abs() ** 2).sum() + sig[i, :, 1].sum()
    L.backward()
    return float(L.detach()), pos.grad.cpu().numpy(), eps.grad.cpu().numpy(), wls.grad.cpu().numpy()


@pytest.mark.parametrize("precision,n_streams", [("tf32", 3), ("fp64", 2)])
def test_spectrum_backward_matches_oracle(G, ctx, precision, n_streams):
    """Loss summed over three wavelengths through scatter_spectrum (concurrent forward solves and adjoint
    solves, gradients summed on the GPU): the loss and every gradient against the oracle's adjoint summed
    over the same wavelengths (1e-8 normwise), and each wavelength's own gradient."""
    cyl = small_cylinder()
    lams = [455.0, 610.0, 780.0]
    L, gp, ge, gl = spectrum_loss_and_grads(G, ctx, cyl, lams, precision, n_streams)
    Lo, gpo, geo, glo = 0.0, 0.0, 0.0, []
    for lam in lams:
        pr = O.Problem(cyl.pos, lam, 3, eps=cyl.eps, step=cyl.step)
        a, b, c, d = O.loss_and_grad_probe_sca(pr, cyl.e0, cyl.r_eval[0])
        Lo, gpo, geo = Lo + a, gpo + b, geo + c
        glo.append(d)
    assert abs(L - Lo) <= 1e-9 * abs(Lo)
    assert np.linalg.norm(gp - gpo) <= 1e-8 * np.linalg.norm(gpo)
    assert np.linalg.norm(ge - geo) <= 1e-8 * np.linalg.norm(geo)
    np.testing.assert_allclose(gl, np.array(glo), rtol=1e-8, atol=1e-14)
