"""GPU parity: the CUDA library (through its C ABI) against the CPU FP64 oracle.

Tolerances (stated by the method's target accuracy):
* assembled matrix, complex64: |dA| <= 1e-6 * max|entry of the 3x3 (6x6) block| per block;
* assembled matrix, complex128: 1e-12 relative per block;
* refined fields: ||dF_q|| / ||F_q|| <= 1e-9 per illumination;
* near fields and cross sections: 1e-9 relative (absolute floor 1e-9 * max value).
Sizes span several tiles with ragged tails (3N not a multiple of any tile size).
"""
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


def gpu_problem(G, s, lam):
    if s.kind == 3:
        return G.GDMProblem(t(s.pos), lam, 3, eps=t(s.eps), step=s.step)
    al = O.lorentz_alpha6(s.omega0_e, s.omega0_m, s.gamma_ev, s.amp_nm, lam)
    return G.GDMProblem(t(s.pos), lam, 6, alpha6=t(al))


def oracle_problem(s, lam):
    if s.kind == 3:
        return O.Problem(s.pos, lam, 3, eps=s.eps, step=s.step)
    return O.Problem(s.pos, lam, 6, alpha6=O.lorentz_alpha6(s.omega0_e, s.omega0_m, s.gamma_ev, s.amp_nm, lam))


def block_errors(Ag, Ao, kind):
    """max over blocks of max|dA_block| / max|A_block|."""
    n = Ao.shape[0] // kind
    d = np.abs(Ag - Ao).reshape(n, kind, n, kind).max(axis=(1, 3))
    m = np.abs(Ao).reshape(n, kind, n, kind).max(axis=(1, 3))
    return (d / m).max()


def structures():
    return [W.random_cells(150, seed=1), W.random_cells(61, seed=2, lossy=False)]


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("fp64", 1e-12)])
def test_assembly_cells(G, ctx, prec, tol):
    for s in structures():
        lam = float(s.wavelengths[0])
        A = G.assemble(ctx, gpu_problem(G, s, lam), prec)
        ns = 3 * s.n
        Ag = A.cpu().numpy()[:, :ns].T
        Ao = oracle_problem(s, lam).matrix()
        assert block_errors(Ag, Ao, 3) < tol


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("fp64", 1e-12)])
def test_assembly_edmd(G, ctx, prec, tol):
    s = W.metasurface_edmd(nx=7, ny=5, pitch=400.0)
    lam = 640.0
    A = G.assemble(ctx, gpu_problem(G, s, lam), prec)
    Ag = A.cpu().numpy()[:, :6 * s.n].T
    Ao = oracle_problem(s, lam).matrix()
    assert block_errors(Ag, Ao, 6) < tol



@pytest.mark.parametrize("eps_env", [1.0, 1.77])
def test_assembly_edmd_several_tiles(G, ctx, eps_env):
    """ED/MD assembly across several 64-target x 4-source tiles with ragged tails in both directions
    (143 dipoles: 2 full target tiles + 15, 35 full source tiles + 3), in vacuum and in a host."""
    s = W.metasurface_edmd(nx=13, ny=11, pitch=400.0, seed=9)
    lam = 610.0
    al = O.lorentz_alpha6(s.omega0_e, s.omega0_m, s.gamma_ev, s.amp_nm, lam, eps_env=eps_env)
    A = G.assemble(ctx, G.GDMProblem(t(s.pos), lam, 6, alpha6=t(al), eps_env=eps_env), "fp32")
    Ag = A.cpu().numpy()[:, :6 * s.n].T
    Ao = O.Problem(s.pos, lam, 6, alpha6=al, eps_env=eps_env).matrix()
    assert block_errors(Ag, Ao, 6) < 1e-6

def test_assembly_large_phase(G, ctx):
    """The 64 x 64 metasurface's extent (25.6 um): kR up to ~450 rad needs the double-float phase."""
    s = W.metasurface_edmd(nx=64, ny=64, pitch=400.0)
    rng = np.random.default_rng(0)
    sub = np.sort(rng.choice(s.n, 40, replace=False))
    s.pos = s.pos[sub]
    s.omega0_e, s.omega0_m = s.omega0_e[sub], s.omega0_m[sub]
    lam = 500.0
    A = G.assemble(ctx, gpu_problem(G, s, lam), "fp32")
    Ag = A.cpu().numpy()[:, :6 * s.n].T
    Ao = oracle_problem(s, lam).matrix()
    assert block_errors(Ag, Ao, 6) < 1e-6


def test_planewave(G, ctx):
    s = W.random_cells(70, seed=4)
    F0 = G.incident_planewave(ctx, t(s.pos), 530.0, W.XYPOL, kind_out=6)
    ref = O.plane_wave(s.pos, 2 * np.pi / 530.0, 1.0, W.XYPOL, (0, 0, 1.0), 6)
    np.testing.assert_allclose(F0.cpu().numpy().T, ref, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_solve_cells(G, ctx, prec):
    for s in structures():
        lam = float(s.wavelengths[0])
        prob = gpu_problem(G, s, lam)
        F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0)
        A = G.assemble(ctx, prob, prec)
        F, ipiv, info = G.solve(ctx, prob, A, F0, prec)
        pr = oracle_problem(s, lam)
        Fo = pr.solve(pr.plane_wave(s.e0))
        err = np.linalg.norm(F.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
        assert np.all(err < 1e-9), (prec, err, info)



@pytest.mark.parametrize("prec", ["fp32", "tf32"])
@pytest.mark.parametrize("scale", [1e-30, 1e30])
def test_solve_illumination_far_outside_fp32_range(G, ctx, prec, scale):
    """The solution is linear in F0: an illumination scaled by 1e-30 (or 1e30) gives the scaled fields to the
    same accuracy. Unscaled, the FP32 refinement residuals of the weak illumination (~1e-40) would flush to
    zero and the refinement would stop on a zero correction with an unrefined solution."""
    s = W.random_cells(150, seed=1)
    lam = float(s.wavelengths[0])
    prob = gpu_problem(G, s, lam)
    F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0)
    A = G.assemble(ctx, prob, prec)
    F, ipiv, info = G.solve(ctx, prob, A, F0, prec)
    Fs, _, info_s = G.solve(ctx, prob, A, F0 * scale, prec, ipiv=ipiv, factored=True)
    d = (Fs / scale - F).norm(dim=1) / F.norm(dim=1)
    assert float(d.max()) < 1e-9, (d, info, info_s)
    assert info_s["rel_residual"] < 1e-10, info_s


def test_solve_sphere_config(G, ctx):
    """The plain-FP64 sphere workload (N = 925, 3N = 2775): fields, near field on the 968-point grid,
    cross sections."""
    s = W.sphere_plain_fp64()
    lam = float(s.wavelengths[0])
    prob = gpu_problem(G, s, lam)
    F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0)
    A = G.assemble(ctx, prob, "fp64")
    F, ipiv, info = G.solve(ctx, prob, A, F0, "fp64")
    r_eval = t(s.r_eval)
    F0e = G.incident_planewave(ctx, r_eval, lam, s.e0, kind_out=6)
    E, H = G.nearfield(ctx, prob, F, r_eval, F0e)
    ext, sca, ab = G.cross_sections(ctx, prob, F0, F, np.ones(s.n_rhs))
    pr = oracle_problem(s, lam)
    F0o = pr.plane_wave(s.e0)
    Fo = pr.solve(F0o)
    err = np.linalg.norm(F.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
    assert np.all(err < 1e-9), err
    Eo, Ho = pr.nearfield(Fo, s.r_eval, s.e0)
    for g, o in ((E, Eo), (H, Ho)):
        go = g.cpu().numpy().T.reshape(-1, 3, s.n_rhs)
        np.testing.assert_allclose(go.reshape(o.shape), o, rtol=1e-9, atol=1e-9 * np.abs(o).max())
    xo = pr.cross_sections(F0o, Fo, s.e0)
    for g, o in zip((ext, sca, ab), xo):
        np.testing.assert_allclose(g.cpu().numpy(), o, rtol=1e-9, atol=1e-9 * abs(xo[0]).max())


def test_nearfield_kernel_isolated(G, ctx):
    """Near field from the oracle's own fields (isolates the repropagation kernel), kinds 3 and 6."""
    for s, lam in ((W.random_cells(90, seed=8), 555.0), (W.metasurface_edmd(nx=6, ny=6), 700.0)):
        pr = oracle_problem(s, lam)
        Fo = pr.solve(pr.plane_wave(s.e0))
        rng = np.random.default_rng(1)
        r_eval = rng.uniform(-2000, 2000, (300, 3)) + np.array([0, 0, 3000.0])
        E, H = G.nearfield(ctx, gpu_problem(G, s, lam), t(Fo.T), t(r_eval), None)
        Eo, Ho = pr.nearfield(Fo, r_eval, s.e0, with_incident=False)
        np.testing.assert_allclose(E.cpu().numpy().T.reshape(Eo.shape[0], 3, -1), Eo, rtol=1e-10,
                                   atol=1e-10 * np.abs(Eo).max())
        np.testing.assert_allclose(H.cpu().numpy().T.reshape(Ho.shape[0], 3, -1), Ho, rtol=1e-10,
                                   atol=1e-10 * np.abs(Ho).max())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solve_edmd(G, ctx, prec):
    s = W.metasurface_edmd(nx=9, ny=7, pitch=400.0)
    lam = 610.0
    prob = gpu_problem(G, s, lam)
    F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0, kind_out=6)
    A = G.assemble(ctx, prob, prec)
    F, ipiv, info = G.solve(ctx, prob, A, F0, prec)
    pr = oracle_problem(s, lam)
    F0o = pr.plane_wave(s.e0)
    Fo = pr.solve(F0o)
    err = np.linalg.norm(F.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
    assert np.all(err < 1e-9), err
    ext, sca, ab = G.cross_sections(ctx, prob, F0, F, np.ones(s.n_rhs))
    xo = pr.cross_sections(F0o, Fo, s.e0)
    for g, o in zip((ext, sca, ab), xo):
        np.testing.assert_allclose(g.cpu().numpy(), o, rtol=1e-9, atol=1e-9 * abs(xo[0]).max())


def test_single_dipole_and_single_cell(G, ctx):
    """Degenerate sizes: one cell (N = 1) and one effective dipole."""
    s = W.Structure(name="one", kind=3, pos=np.zeros((1, 3)), step=7.0, eps=np.array([4.0 + 1.0j]),
                    wavelengths=np.array([500.0]), e0=W.XYPOL.copy())
    prob = gpu_problem(G, s, 500.0)
    F0 = G.incident_planewave(ctx, prob.pos, 500.0, s.e0)
    for prec in ("fp64", "fp32"):
        A = G.assemble(ctx, prob, prec)
        F, _, _ = G.solve(ctx, prob, A, F0, prec)
        np.testing.assert_allclose(F.cpu().numpy(), F0.cpu().numpy() * 3 / (4.0 + 1.0j + 2), rtol=1e-12)


def test_invalid_arguments(G, ctx):
    s = W.random_cells(10, seed=3)
    prob = gpu_problem(G, s, 500.0)
    with pytest.raises(G.GDMError):
        G.assemble(ctx, prob, "fp32", lda=29)        # odd / too small leading dimension
    bad = G.GDMProblem(prob.pos, -1.0, 3, eps=prob.eps, step=10.0)
    with pytest.raises(G.GDMError):
        G.assemble(ctx, bad, "fp32")


@pytest.mark.parametrize("prec,tol_plain,max_iters", [("tf32", 5e-2, 16), ("bf16", 2e-1, 30), ("fp32", 1e-4, 5),
                                                        ("fp64", 1e-11, 2)])
def test_lu_factor_quality(G, ctx, prec, tol_plain, max_iters):
    """The factors themselves (no refinement) solve the system to the precision's level, so a wrong
    trailing update cannot hide behind the FP64 refinement. 3N = 2100: eight outer blocks, the
    tensor-core update runs with trailing sizes 1844 ... 52 (ragged tiles; with BF16 the updates of at
    least 512 columns run on the BF16 pair kernel, 256-row tiles with ragged ends in both directions)."""
    s = W.random_cells(700, seed=12)
    lam = float(s.wavelengths[0])
    prob = gpu_problem(G, s, lam)
    F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0)
    A = G.assemble(ctx, prob, prec)
    F1, ipiv, _ = G.solve(ctx, prob, A, F0, prec, no_refine=True)
    pr = oracle_problem(s, lam)
    Fo = pr.solve(pr.plane_wave(s.e0))
    e1 = np.linalg.norm(F1.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
    assert np.all(e1 < tol_plain), e1
    F2, _, info = G.solve(ctx, prob, A, F0, prec, ipiv=ipiv, factored=True)
    e2 = np.linalg.norm(F2.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
    assert np.all(e2 < 1e-9) and info["iterations"] <= max_iters, (e1, e2, info)


@pytest.mark.parametrize("prec,switch", [("tf32", None), ("tf32", "GDM_LU_PREP_L"), ("tf32", "GDM_PANEL_SINGLE"),
                                         ("tf32", "GDM_U12_ACCUMULATE"), ("fp32", None), ("fp32", "GDM_PANEL_SINGLE")])
def test_recursive_block_factorisation(G, ctx, prec, switch, monkeypatch):
    """The recursive in-block factorisation (used from n = 8192 on; forced here at 3N = 2100: four full
    512-column blocks split 256/128/64 down to pairs of 32-column panels, and a ragged 52-column last
    block) gives factors of the precision's quality and refined fields at 1e-9, like the panel-by-panel
    path. Each 64-column leaf runs as one two-panel launch (its K = 32 update in FP32 inside the kernel);
    GDM_PANEL_SINGLE takes the one-panel launches with the interchange pass and the tensor-core update
    between them. At TF32 the panels write L's embedding for the updates and U is rounded in storage;
    GDM_LU_PREP_L takes the path that prepares both operands before each update instead. U12 is written by
    a store-only tensor-core product (rounded to TF32 in its epilogue) where the CTA-pair kernel applies
    (the first three blocks here) and by zeroing plus an accumulating product elsewhere (the last one);
    GDM_U12_ACCUMULATE takes the second form for every block."""
    monkeypatch.setenv("GDM_LU_RECURSIVE", "1")
    if switch:
        monkeypatch.setenv(switch, "1")
    s = W.random_cells(700, seed=12)
    lam = float(s.wavelengths[0])
    prob = gpu_problem(G, s, lam)
    F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0)
    pr = oracle_problem(s, lam)
    Fo = pr.solve(pr.plane_wave(s.e0))
    A = G.assemble(ctx, prob, prec)
    F1, ipiv, _ = G.solve(ctx, prob, A, F0, prec, no_refine=True)
    e1 = np.linalg.norm(F1.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
    assert np.all(e1 < (5e-2 if prec == "tf32" else 1e-4)), e1
    F2, _, info = G.solve(ctx, prob, A, F0, prec, ipiv=ipiv, factored=True)
    e2 = np.linalg.norm(F2.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
    assert np.all(e2 < 1e-9), (e1, e2, info)


@pytest.mark.parametrize("eps,expect_refactor", [(12.25 + 0.0j, False), (-8.0 + 0.5j, False), (-2.2 + 0.3j, True)])
def test_pivoting_certificate_and_fallback(G, ctx, eps, expect_refactor):
    """Pivots are searched inside each 32 x 32 diagonal block and certified against the rows below.
    Dielectric cells: certificate <= 1 (identical to partial pivoting). Metallic cells near the plasmon
    resonance: the certificate exceeds the limit and the solve refactors with whole-column pivoting.
    Either way the refined fields match the oracle."""
    s = W.random_cells(120, seed=3)
    s.eps = np.full(s.n, eps, complex)
    lam = 500.0
    prob = gpu_problem(G, s, lam)
    F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0)
    pr = oracle_problem(s, lam)
    Fo = pr.solve(pr.plane_wave(s.e0))
    for prec in ("fp32", "fp64"):
        A = G.assemble(ctx, prob, prec)
        F, _, info = G.solve(ctx, prob, A, F0, prec)
        err = np.linalg.norm(F.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
        assert np.all(err < 1e-9), (err, info)
        assert bool(info["refactored"]) == expect_refactor, info
        if eps.real > 0:
            assert info["pivot_growth"] <= 1.0
        A = G.assemble(ctx, prob, prec)
        F, _, info = G.solve(ctx, prob, A, F0, prec, global_pivot=True)
        err = np.linalg.norm(F.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
        assert np.all(err < 1e-9) and not info["refactored"]


@pytest.mark.parametrize("lossy", [True, False])
def test_residual_matches_oracle(G, ctx, lossy):
    """gdm_residual (double-float pair sums for cells) = the oracle's F0 - A F, row by row, for arbitrary
    (not solved) fields, to 1e-13 of the largest term."""
    s = W.random_cells(300, seed=31, lossy=lossy)
    lam = 530.0
    prob = gpu_problem(G, s, lam)
    rng = np.random.default_rng(2)
    F = rng.standard_normal((2, 3 * s.n)) + 1j * rng.standard_normal((2, 3 * s.n))
    F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0)
    r, n2 = G.residual(ctx, prob, F0, t(F))
    pr = oracle_problem(s, lam)
    ro = O.residual_rows(pr, F0.cpu().numpy().T, F.T, np.arange(s.n)).reshape(3 * s.n, 2)
    scale = np.abs(pr.matrix()).max() * np.abs(F).max()
    assert np.abs(r.cpu().numpy().T - ro).max() <= 1e-13 * scale
    np.testing.assert_allclose(n2.cpu().numpy(), np.sum(np.abs(ro) ** 2, axis=0), rtol=1e-10)


@pytest.mark.parametrize("subset", [False, True])
def test_residual_matches_oracle_edmd(G, ctx, subset):
    """gdm_residual for ED/MD dipoles (double-float 6x6 dyads with the electric-magnetic cross blocks) =
    the oracle's F0 - A F for arbitrary fields and three right-hand sides (a two-RHS and a one-RHS pass),
    to 1e-13 of the largest term; the subset case scatters 150 dipoles over the full 64 x 64 array, so
    the phases k R reach ~450 rad."""
    if subset:
        s = W.metasurface_edmd(nx=64, ny=64, pitch=400.0, seed=4)
        sub = np.sort(np.random.default_rng(8).choice(s.n, 150, replace=False))
        s.pos, s.omega0_e, s.omega0_m = s.pos[sub], s.omega0_e[sub], s.omega0_m[sub]
    else:
        s = W.metasurface_edmd(nx=14, ny=12, pitch=400.0, seed=6)
    lam = 505.0
    prob = gpu_problem(G, s, lam)
    rng = np.random.default_rng(3)
    e0 = np.array([[1, 0, 0], [0, 1, 0], [1, 1j, 0]], complex) / np.array([[1.0], [1.0], [np.sqrt(2.0)]])
    F = rng.standard_normal((3, 6 * s.n)) + 1j * rng.standard_normal((3, 6 * s.n))
    F0 = G.incident_planewave(ctx, prob.pos, lam, e0, kind_out=6)
    r, n2 = G.residual(ctx, prob, F0, t(F))
    pr = oracle_problem(s, lam)
    ro = O.residual_rows(pr, F0.cpu().numpy().T, F.T, np.arange(s.n)).reshape(6 * s.n, 3)
    scale = np.abs(pr.matrix()).max() * np.abs(F).max()
    assert np.abs(r.cpu().numpy().T - ro).max() <= 1e-13 * scale
    np.testing.assert_allclose(n2.cpu().numpy(), np.sum(np.abs(ro) ** 2, axis=0), rtol=1e-10)


@pytest.mark.parametrize("prec", ["tf32", "fp32", "fp64"])
def test_metasurface_medium_several_wavelengths(G, ctx, prec):
    """ED/MD point-dipole array with electric-magnetic cross Green blocks, 6N = 1920 (four 512-column
    blocks, ragged tail), three wavelengths across the resonance band: refined fields and cross
    sections against the oracle's dense solve."""
    s = W.metasurface_edmd(nx=20, ny=16, pitch=400.0, seed=4)
    for lam in (505.0, 620.0, 790.0):
        prob = gpu_problem(G, s, lam)
        F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0, kind_out=6)
        A = G.assemble(ctx, prob, "fp64" if prec == "fp64" else "fp32")
        F, _, info = G.solve(ctx, prob, A, F0, prec)
        pr = oracle_problem(s, lam)
        F0o = pr.plane_wave(s.e0)
        Fo = pr.solve(F0o)
        err = np.linalg.norm(F.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
        assert np.all(err < 1e-9), (lam, err, info)
        ext, sca, ab = G.cross_sections(ctx, prob, F0, F, np.ones(s.n_rhs))
        xo = pr.cross_sections(F0o, Fo, s.e0)
        for g, o in zip((ext, sca, ab), xo):
            np.testing.assert_allclose(g.cpu().numpy(), o, rtol=1e-9, atol=1e-9 * abs(xo[0]).max())


def test_metasurface_full_size_sampled_residual(G, ctx):
    """The full 64 x 64 metasurface (6N = 24,576) in TF32 + refinement at the shortest wavelength
    (largest phase range): the oracle evaluates F0 - A F exactly for a seeded sample of 48 dipoles,
    which must be at the level of the FP64 refinement (1e-11 of |F0|)."""
    s = W.metasurface_edmd(nx=64, ny=64, pitch=400.0, seed=4)
    lam = 500.0
    prob = gpu_problem(G, s, lam)
    F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0, kind_out=6)
    A = G.assemble(ctx, prob, "fp32")
    F, _, info = G.solve(ctx, prob, A, F0, "tf32")
    del A
    pr = oracle_problem(s, lam)
    rows = np.sort(np.random.default_rng(5).choice(s.n, 48, replace=False))
    Fh = F.cpu().numpy().T
    F0h = F0.cpu().numpy().T
    r = O.residual_rows(pr, F0h, Fh, rows)
    F0s = F0h.reshape(s.n, 6, -1)[rows]
    rel = np.linalg.norm(r.reshape(-1, r.shape[-1]), axis=0) / np.linalg.norm(F0s.reshape(-1, r.shape[-1]), axis=0)
    assert np.all(rel < 1e-11), (rel, info)
    assert info["rel_residual"] < 1e-11, info


def test_alpha6_lorentz(G, ctx):
    """Lorentzian ED/MD polarisabilities on the GPU against the oracle's, across the resonance band."""
    s = W.metasurface_edmd(nx=13, ny=11, seed=7)
    w0e, w0m = t(s.omega0_e), t(s.omega0_m)
    for lam in (450.0, 496.0, 620.0, 800.0):
        ag = G.alpha6_lorentz(ctx, w0e, w0m, s.gamma_ev, s.amp_nm, lam).cpu().numpy()
        ao = O.lorentz_alpha6(s.omega0_e, s.omega0_m, s.gamma_ev, s.amp_nm, lam)
        np.testing.assert_allclose(ag, ao, rtol=1e-13, atol=1e-13 * np.abs(ao).max())
