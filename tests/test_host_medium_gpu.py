"""ED/MD point dipoles, dipole sources, LDOS and GPM extraction in a homogeneous host medium
(eps_env != 1) on the GPU, against the oracle.

In a non-magnetic host the 6x6 dyad is [[G^Ep, -G^Hp], [G^Hp, eps_env G^Ep]] at k = n_env k0, and the
radiation terms of the cross sections and of the Lorentzian dressing carry the host factors; the oracle's
forms are pinned (Maxwell curls, Mie dipole terms in a host, optical theorem, LDOS power balance) on the
CPU. Tolerances as for the vacuum parity tests: assembly 1e-6 (complex64) and 1e-12 (complex128) per
block, refined fields 1e-9, cross sections and near fields 1e-9 relative, residual 1e-13 of the largest
term, far-field amplitudes 1e-12 of the largest.
"""
import numpy as np
import pytest
import torch

import gdm_workloads as W
import oracle as O

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
WATER = 1.77
GLASS = 2.25


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


def edmd(G, s, lam, eps_env):
    al = O.lorentz_alpha6(s.omega0_e, s.omega0_m, s.gamma_ev, s.amp_nm, lam, eps_env=eps_env)
    return (G.GDMProblem(t(s.pos), lam, 6, alpha6=t(al), eps_env=eps_env),
            O.Problem(s.pos, lam, 6, alpha6=al, eps_env=eps_env))


def block_errors(Ag, Ao, kind):
    n = Ao.shape[0] // kind
    d = np.abs(Ag - Ao).reshape(n, kind, n, kind).max(axis=(1, 3))
    m = np.abs(Ao).reshape(n, kind, n, kind).max(axis=(1, 3))
    return (d / m).max()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("fp64", 1e-12)])
@pytest.mark.parametrize("eps_env", [WATER, GLASS])
def test_assembly_edmd_in_host(G, ctx, prec, tol, eps_env):
    s = W.metasurface_edmd(nx=7, ny=5, pitch=400.0, seed=3)
    prob, pr = edmd(G, s, 640.0, eps_env)
    A = G.assemble(ctx, prob, prec)
    Ag = A.cpu().numpy()[:, :6 * s.n].T
    assert block_errors(Ag, pr.matrix(), 6) < tol


def test_alpha6_lorentz_in_host(G, ctx):
    s = W.metasurface_edmd(nx=9, ny=8, seed=7)
    w0e, w0m = t(s.omega0_e), t(s.omega0_m)
    for lam in (450.0, 560.0, 800.0):
        ag = G.alpha6_lorentz(ctx, w0e, w0m, s.gamma_ev, s.amp_nm, lam, eps_env=WATER).cpu().numpy()
        ao = O.lorentz_alpha6(s.omega0_e, s.omega0_m, s.gamma_ev, s.amp_nm, lam, eps_env=WATER)
        np.testing.assert_allclose(ag, ao, rtol=1e-13, atol=1e-13 * np.abs(ao).max())


@pytest.mark.parametrize("subset", [False, True])
def test_residual_edmd_in_host(G, ctx, subset):
    """The double-float matrix-free residual F0 - A F of ED/MD dipoles in water, three right-hand sides;
    the subset case spreads 150 dipoles over the 64 x 64 array (phases k R up to ~600 rad in water)."""
    if subset:
        s = W.metasurface_edmd(nx=64, ny=64, pitch=400.0, seed=4)
        sub = np.sort(np.random.default_rng(8).choice(s.n, 150, replace=False))
        s.pos, s.omega0_e, s.omega0_m = s.pos[sub], s.omega0_e[sub], s.omega0_m[sub]
    else:
        s = W.metasurface_edmd(nx=14, ny=12, pitch=400.0, seed=6)
    lam = 505.0
    prob, pr = edmd(G, s, lam, WATER)
    rng = np.random.default_rng(3)
    e0 = np.array([[1, 0, 0], [0, 1, 0], [1, 1j, 0]], complex) / np.array([[1.0], [1.0], [np.sqrt(2.0)]])
    F = rng.standard_normal((3, 6 * s.n)) + 1j * rng.standard_normal((3, 6 * s.n))
    F0 = G.incident_planewave(ctx, prob.pos, lam, e0, eps_env=WATER, kind_out=6)
    r, n2 = G.residual(ctx, prob, F0, t(F))
    ro = O.residual_rows(pr, F0.cpu().numpy().T, F.T, np.arange(s.n)).reshape(6 * s.n, 3)
    scale = np.abs(pr.matrix()).max() * np.abs(F).max()
    assert np.abs(r.cpu().numpy().T - ro).max() <= 1e-13 * scale
    np.testing.assert_allclose(n2.cpu().numpy(), np.sum(np.abs(ro) ** 2, axis=0), rtol=1e-10)


@pytest.mark.parametrize("prec", ["tf32", "fp32", "fp64"])
def test_solve_nearfield_crosssections_edmd_in_host(G, ctx, prec):
    """6N = 1920 ED/MD array in water at two wavelengths: refined fields, cross sections, and the near
    field (E and H with the incident wave) at points above the array, against the oracle."""
    s = W.metasurface_edmd(nx=20, ny=16, pitch=400.0, seed=4)
    r_eval = np.stack(np.meshgrid(np.linspace(-3000, 3000, 9), np.linspace(-2500, 2500, 7), [350.0, 900.0],
                                  indexing="ij"), -1).reshape(-1, 3)
    for lam in (520.0, 700.0):
        prob, pr = edmd(G, s, lam, WATER)
        F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0, eps_env=WATER, kind_out=6)
        A = G.assemble(ctx, prob, "fp64" if prec == "fp64" else "fp32")
        F, _, info = G.solve(ctx, prob, A, F0, prec)
        F0o = pr.plane_wave(s.e0)
        np.testing.assert_allclose(F0.cpu().numpy().T, F0o, rtol=0, atol=1e-13)
        Fo = pr.solve(F0o)
        err = np.linalg.norm(F.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
        assert np.all(err < 1e-9), (lam, err, info)
        ext, sca, ab = G.cross_sections(ctx, prob, F0, F, np.ones(s.n_rhs))
        xo = pr.cross_sections(F0o, Fo, s.e0)
        for g, o in zip((ext, sca, ab), xo):
            np.testing.assert_allclose(g.cpu().numpy(), o, rtol=1e-9, atol=1e-9 * abs(xo[0]).max())
        inc = G.incident_planewave(ctx, t(r_eval), lam, s.e0, eps_env=WATER, kind_out=6)
        E, H = G.nearfield(ctx, prob, t(Fo.T), t(r_eval), F0_eval=inc)
        Eo, Ho = pr.nearfield(Fo, r_eval, s.e0)
        for g, o in ((E, Eo), (H, Ho)):
            g = g.cpu().numpy().reshape(s.n_rhs, -1, 3).transpose(1, 2, 0)
            np.testing.assert_allclose(g, o, rtol=0, atol=1e-9 * np.abs(o).max())


def test_farfield_and_optical_theorem_in_host(G, ctx):
    """Far-field amplitudes (n_env on the magnetic term) and the far-field cross section against the
    oracle, and the optical theorem on the GPU for the dressed dipoles in glass."""
    s = W.metasurface_edmd(nx=7, ny=5, seed=2)
    lam = 610.0
    prob, pr = edmd(G, s, lam, GLASS)
    Fo = pr.solve(pr.plane_wave(s.e0))
    F = t(Fo.T)
    dirs = W.sphere_points(301, 1.0, seed=9)
    f = G.farfield(ctx, prob, F, t(dirs)).cpu().numpy()
    fo = pr.farfield_amplitude(Fo, dirs)
    np.testing.assert_allclose(f.T.reshape(fo.shape), fo, atol=1e-12 * np.abs(fo).max())
    sig = G.sigma_farfield(ctx, prob, F, np.ones(s.n_rhs), n_theta=24, n_phi=48).cpu().numpy()
    np.testing.assert_allclose(sig, pr.farfield_scattering(Fo, s.e0, n_theta=24, n_phi=48), rtol=1e-10)
    F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0, eps_env=GLASS, kind_out=6)
    A = G.assemble(ctx, prob, "fp32")
    Fg, _, _ = G.solve(ctx, prob, A, F0, "tf32")
    ext, sca, ab = G.cross_sections(ctx, prob, F0, Fg, np.ones(s.n_rhs))
    ff = G.sigma_farfield(ctx, prob, Fg, np.ones(s.n_rhs), n_theta=96, n_phi=192)
    np.testing.assert_allclose((ext - ab).cpu().numpy(), ff.cpu().numpy(), rtol=1e-6)


@pytest.mark.parametrize("kind_out", [3, 6])
def test_incident_dipole_in_host(G, ctx, kind_out):
    s = W.random_cells(50, seed=3)
    lam = 590.0
    pr = O.Problem(s.pos, lam, 3, eps=s.eps, step=s.step, eps_env=WATER)
    rng = np.random.default_rng(4)
    src = W.sphere_points(5, 120.0, seed=6)
    mom = rng.standard_normal((5, 6)) + 1j * rng.standard_normal((5, 6))
    F0 = G.incident_dipole(ctx, t(s.pos), lam, t(src), t(mom), kind_out=kind_out, eps_env=WATER).cpu().numpy().T
    F0o = O.dipole_illumination(pr, s.pos, src, mom, kind_out)
    np.testing.assert_allclose(F0, F0o, atol=1e-12 * np.abs(F0o).max())


@pytest.mark.parametrize("magnetic", [False, True])
def test_ldos_in_host(G, ctx, magnetic):
    s = W.random_cells(120, seed=14)
    lam = 620.0
    pr = O.Problem(s.pos, lam, 3, eps=s.eps, step=s.step, eps_env=WATER)
    r0 = np.concatenate([W.sphere_points(6, 70.0, seed=2), [[5.0, 5.0, 60.0]]])
    prob = G.GDMProblem(t(s.pos), lam, 3, eps=t(s.eps), step=s.step, eps_env=WATER)
    got = G.ldos(ctx, prob, t(r0), magnetic=magnetic, precision="tf32").cpu().numpy()
    np.testing.assert_allclose(got, O.ldos(pr, r0, magnetic=magnetic), rtol=1e-9)


def test_gpm_in_host(G, ctx):
    """GPM of a 40-cell structure in water: 4 sites, 12 plane waves (6 angles x 2 polarisations) + 12
    dipole sources, 60 probes."""
    s = W.random_cells(40, seed=21)
    lam = 580.0
    r_gpm = W.farthest_points(s.pos, 4, 21)
    khat, e0, ds_pos, ds_mom = W.gpm_illumination_set(n_angles=6, n_sources=12, source_radius=150.0, seed=21)
    r_probe = W.sphere_points(60, 90.0, seed=28)
    prob = G.GDMProblem(t(s.pos), lam, 3, eps=t(s.eps), step=s.step, eps_env=WATER)
    a, P, rel = G.gpm_extract(ctx, prob, t(r_gpm), t(r_probe), khat, e0, t(ds_pos), t(ds_mom), precision="tf32")
    pr = O.Problem(s.pos, lam, 3, eps=s.eps, step=s.step, eps_env=WATER)
    ao, Po, _, relo = O.gpm_extract(pr, r_gpm, r_probe, khat, e0, ds_pos, ds_mom)
    np.testing.assert_allclose(P.cpu().numpy(), Po, atol=1e-8 * np.abs(Po).max())
    np.testing.assert_allclose(a.cpu().numpy(), ao, atol=1e-8 * np.abs(ao).max())
    assert abs(rel - relo) <= 1e-6 * relo + 1e-12
