"""Far-field amplitudes (gdm_farfield) and the far-field scattering cross section (gdm_sigma_farfield)
against the oracle: amplitudes to 1e-12 of the largest, the quadrature to 1e-10 relative at the same grid;
and the optical theorem on the GPU for radiatively dressed ED/MD dipoles (sigma_ext - sigma_abs =
sigma_sca,ff to quadrature accuracy)."""
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


def t(x):
    return torch.tensor(np.ascontiguousarray(x), device=DEV)


def cases():
    s3 = W.random_cells(140, seed=6)
    s6 = W.metasurface_edmd(nx=7, ny=5, seed=2)
    return [(s3, 560.0), (s6, 610.0)]


def problems(G, s, lam):
    if s.kind == 3:
        return (G.GDMProblem(t(s.pos), lam, 3, eps=t(s.eps), step=s.step),
                O.Problem(s.pos, lam, 3, eps=s.eps, step=s.step))
    al = O.lorentz_alpha6(s.omega0_e, s.omega0_m, s.gamma_ev, s.amp_nm, lam)
    return G.GDMProblem(t(s.pos), lam, 6, alpha6=t(al)), O.Problem(s.pos, lam, 6, alpha6=al)


@pytest.mark.parametrize("case", [0, 1])
def test_farfield_matches_oracle(G, ctx, case):
    s, lam = cases()[case]
    prob, pr = problems(G, s, lam)
    Fo = pr.solve(pr.plane_wave(s.e0))
    F = t(Fo.T)
    dirs = W.sphere_points(301, 1.0, seed=9)
    f = G.farfield(ctx, prob, F, t(dirs)).cpu().numpy()               # (n_rhs, 3q)
    fo = pr.farfield_amplitude(Fo, dirs)                              # (q, 3, n_rhs)
    np.testing.assert_allclose(f.T.reshape(fo.shape), fo, atol=1e-12 * np.abs(fo).max())
    sig = G.sigma_farfield(ctx, prob, F, np.ones(s.n_rhs), n_theta=24, n_phi=48).cpu().numpy()
    so = pr.farfield_scattering(Fo, s.e0, n_theta=24, n_phi=48)
    np.testing.assert_allclose(sig, so, rtol=1e-10)


def test_optical_theorem_on_the_gpu(G, ctx):
    """Radiatively dressed ED/MD dipoles: sigma_ext - sigma_abs (gdm_cross_sections of a refined TF32 solve)
    equals the far-field integral of the scattered intensity (gdm_sigma_farfield)."""
    s, lam = cases()[1]
    prob, _ = problems(G, s, lam)
    F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0, kind_out=6)
    A = G.assemble(ctx, prob, "fp32")
    F, _, _ = G.solve(ctx, prob, A, F0, "tf32")
    ext, sca, ab = G.cross_sections(ctx, prob, F0, F, np.ones(s.n_rhs))
    ff = G.sigma_farfield(ctx, prob, F, np.ones(s.n_rhs), n_theta=96, n_phi=192)
    np.testing.assert_allclose((ext - ab).cpu().numpy(), ff.cpu().numpy(), rtol=1e-6)
