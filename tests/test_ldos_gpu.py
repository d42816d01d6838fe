"""Point-dipole illumination (gdm_incident_dipole) and the electric / magnetic LDOS (gdm_ldos) against the
oracle: fields to 1e-12 of the largest, LDOS to 1e-9 (refined solves)."""
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


@pytest.mark.parametrize("kind_out", [3, 6])
def test_incident_dipole_matches_oracle(G, ctx, kind_out):
    s = W.random_cells(50, seed=3)
    lam = 590.0
    pr = O.Problem(s.pos, lam, 3, eps=s.eps, step=s.step)
    rng = np.random.default_rng(4)
    src = W.sphere_points(5, 120.0, seed=6)
    mom = rng.standard_normal((5, 6)) + 1j * rng.standard_normal((5, 6))
    F0 = G.incident_dipole(ctx, t(s.pos), lam, t(src), t(mom), kind_out=kind_out).cpu().numpy().T
    F0o = O.dipole_illumination(pr, s.pos, src, mom, kind_out)
    np.testing.assert_allclose(F0, F0o, atol=1e-12 * np.abs(F0o).max())


@pytest.mark.parametrize("magnetic,precision", [(False, "tf32"), (True, "tf32"), (False, "fp64")])
def test_ldos_matches_oracle(G, ctx, magnetic, precision):
    """Emitters around and between the cells of a 120-cell structure."""
    s = W.random_cells(120, seed=14)
    lam = 620.0
    pr = O.Problem(s.pos, lam, 3, eps=s.eps, step=s.step)
    r0 = np.concatenate([W.sphere_points(6, 70.0, seed=2), [[5.0, 5.0, 60.0]]])
    prob = G.GDMProblem(t(s.pos), lam, 3, eps=t(s.eps), step=s.step)
    got = G.ldos(ctx, prob, t(r0), magnetic=magnetic, precision=precision).cpu().numpy()
    want = O.ldos(pr, r0, magnetic=magnetic)
    np.testing.assert_allclose(got, want, rtol=1e-9)


@pytest.mark.parametrize("theta,kind_out", [(0.0, 3), (0.35, 6)])
def test_incident_gaussian_matches_oracle(G, ctx, theta, kind_out):
    """Paraxial Gaussian beam (tight focus, oblique) against the oracle at 1e-13 of the largest entry."""
    r = W.sphere_points(500, 400.0, seed=8) * np.random.default_rng(1).uniform(0, 1, (500, 1))
    e0 = np.array([[1.0, 0.5j, 0.0], [0.2, 1.0, 0.0]])
    lam, w0, focus = 610.0, 450.0, (20.0, -10.0, 35.0)
    got = G.incident_gaussian(ctx, t(r), lam, e0, w0, focus=focus, theta=theta, kind_out=kind_out).cpu().numpy().T
    want = O.gaussian_paraxial(r, 2 * np.pi / lam, 1.0, e0, w0, focus=focus, theta=theta, kind_out=kind_out)
    np.testing.assert_allclose(got, want, atol=1e-13 * np.abs(want).max())
