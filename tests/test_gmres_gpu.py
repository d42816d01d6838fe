"""Matrix-free preconditioned GMRES (gdm_solve_gmres) against the oracle.

The iterative solve must reach the same fields as the oracle's dense solve (1e-9 relative per
illumination, the field tolerance of the dense path) for cuboids and irregular blobs whose blocks and
coarse cells are ragged, in vacuum and in a host, with every preconditioner variant; at a size beyond the
dense tests (24,000 cells, 3N = 72,000) the oracle evaluates F0 - A F exactly on a seeded sample of cells,
which must sit at the solver's tolerance.
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


def cuboid(nx, ny, nz, seed, step=10.0):
    pos = W.cuboid_cells(nx, ny, nz, step)
    rng = np.random.default_rng(seed)
    eps = rng.uniform(2.0, 16.0, len(pos)) + 1j * rng.uniform(0.0, 0.5, len(pos))
    return pos, eps, step


def blob(n, seed, step=15.0):
    rng = np.random.default_rng(seed)
    pos = W.eden_blob(n, step, rng)
    eps = rng.uniform(2.0, 16.0, n) + 1j * rng.uniform(0.0, 0.3, n)
    return pos, eps, step


def check(G, ctx, pos, eps, step, lam, eps_env=1.0, tol_f=1e-9, **kw):
    prob = G.GDMProblem(t(pos), lam, 3, eps=t(eps), step=step, eps_env=eps_env)
    F0 = G.incident_planewave(ctx, prob.pos, lam, W.XYPOL, eps_env=eps_env)
    F, info = G.solve_gmres(ctx, prob, F0, **kw)
    pr = O.Problem(pos, lam, 3, eps=eps, step=step, eps_env=eps_env)
    Fo = pr.solve(pr.plane_wave(W.XYPOL))
    err = np.linalg.norm(F.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
    assert np.all(err < tol_f), (err, info)
    assert info["rel_residual"] <= 1e-12 and info["status"] == 0, info
    return info


@pytest.mark.parametrize("precision,fast", [("tf32", True), ("fp32", True), ("tf32", False)])
def test_gmres_cuboid_matches_oracle(G, ctx, precision, fast):
    """14 x 12 x 9 cells (N = 1,512), eps ~ U[2,16] + i U[0,0.5]: blocks of 256 cells (six, the last
    ragged), coarse cells of 8 children and, on the odd face, of 4; Arnoldi steps on the FP32 operator
    (cycles refined by the double-float residual) or on the double-float operator throughout."""
    pos, eps, step = cuboid(14, 12, 9, seed=2)
    info = check(G, ctx, pos, eps, step, 500.0, precision=precision, block_cells=256, fast_operator=fast)
    assert info["iterations"] < 100, info


def test_gmres_blob_matches_oracle_all_variants(G, ctx):
    """An Eden blob of 1,100 cells (irregular surface: coarse cells with 1 to 8 children, blocks of 200):
    the full two-level preconditioner, each part alone, and plain GMRES all reach the oracle's fields,
    and the preconditioners with the block part take fewer steps than plain GMRES."""
    pos, eps, step = blob(1100, seed=7)
    its = {}
    for name, kw in (("full", {}), ("coarse", {"blocks": False}), ("blocks", {"coarse": False}),
                     ("plain", {"coarse": False, "blocks": False})):
        its[name] = check(G, ctx, pos, eps, step, 620.0, block_cells=200, restart=40, **kw)["iterations"]
    assert its["full"] < its["plain"] and its["blocks"] < its["plain"], its


def test_gmres_in_host_medium(G, ctx):
    pos, eps, step = blob(700, seed=3)
    check(G, ctx, pos, eps, step, 560.0, eps_env=1.77, block_cells=128)


def test_gmres_small_and_single_block(G, ctx):
    """Fewer cells than one block (the block part is the whole TF32 inverse), and a single cell."""
    pos, eps, step = cuboid(5, 4, 3, seed=9)
    info = check(G, ctx, pos, eps, step, 480.0)
    assert info["iterations"] <= 12, info
    check(G, ctx, np.zeros((1, 3)), np.array([9.0 + 0.5j]), 10.0, 480.0)


@pytest.mark.parametrize("n_rhs,block_cells", [(3, 300), (8, 1024)])
def test_gmres_many_rhs_and_largest_blocks(G, ctx, n_rhs, block_cells):
    """Right-hand sides in lockstep (an odd count; the maximum of 8 with the largest blocks, whose block
    solve keeps 3,072 rows x 8 right-hand sides in shared memory): plane waves along seeded directions
    with seeded polarisations, each against the oracle's dense solve."""
    pos, eps, step = blob(1300, seed=17)
    lam = 540.0
    rng = np.random.default_rng(n_rhs)
    prob = G.GDMProblem(t(pos), lam, 3, eps=t(eps), step=step)
    pr = O.Problem(pos, lam, 3, eps=eps, step=step)
    F0s, F0o = [], []
    for q in range(n_rhs):
        kh = rng.standard_normal(3)
        kh /= np.linalg.norm(kh)
        e0 = np.cross(kh, rng.standard_normal(3)).astype(complex)
        e0 /= np.linalg.norm(e0)
        F0s.append(G.incident_planewave(ctx, prob.pos, lam, e0[None, :], khat=tuple(kh)))
        F0o.append(pr.plane_wave(e0[None, :], khat=kh))
    F0 = torch.cat(F0s, 0)
    F, info = G.solve_gmres(ctx, prob, F0, block_cells=block_cells)
    Fo = pr.solve(np.concatenate(F0o, axis=1))
    err = np.linalg.norm(F.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
    assert np.all(err < 1e-9), (err, info)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-12, info


def test_gmres_large_sampled_residual(G, ctx):
    """24,000 cells (3N = 72,000, beyond the dense tests): the oracle's exact residual rows on 48 seeded
    cells relative to |F0| there, at the solver's tolerance."""
    pos, eps, step = cuboid(40, 30, 20, seed=5)
    lam = 500.0
    prob = G.GDMProblem(t(pos), lam, 3, eps=t(eps), step=step)
    F0 = G.incident_planewave(ctx, prob.pos, lam, W.XYPOL)
    F, info = G.solve_gmres(ctx, prob, F0)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-12, info
    pr = O.Problem(pos, lam, 3, eps=eps, step=step)
    rows = np.sort(np.random.default_rng(11).choice(len(pos), 48, replace=False))
    r = O.residual_rows(pr, F0.cpu().numpy().T, F.cpu().numpy().T, rows)
    f0 = F0.cpu().numpy().T.reshape(len(pos), 3, -1)[rows]
    rel = np.linalg.norm(r.reshape(-1, r.shape[-1]), axis=0) / np.linalg.norm(f0.reshape(-1, r.shape[-1]), axis=0)
    assert np.all(rel < 1e-10), (rel, info)


def test_gmres_errors(G, ctx):
    pos, eps, step = cuboid(6, 5, 4, seed=1)
    prob = G.GDMProblem(t(pos), 500.0, 3, eps=t(eps), step=step)
    F0 = G.incident_planewave(ctx, prob.pos, 500.0, W.XYPOL)
    with pytest.raises(G.GDMError) as e:
        G.solve_gmres(ctx, prob, F0, max_iter=2, coarse=False, blocks=False)
    assert e.value.status == 5  # GDM_ERR_NOT_CONVERGED
    with pytest.raises(G.GDMError):
        G.solve_gmres(ctx, prob, F0.repeat(5, 1))             # 10 right-hand sides > 8
    with pytest.raises(G.GDMError):
        G.solve_gmres(ctx, prob, F0, precision="fp64")         # the preconditioner factors in TF32 / FP32
    s = W.metasurface_edmd(nx=3, ny=3, n_lambda=1)
    al = O.lorentz_alpha6(s.omega0_e, s.omega0_m, s.gamma_ev, s.amp_nm, 600.0)
    p6 = G.GDMProblem(t(s.pos), 600.0, 6, alpha6=t(al))
    with pytest.raises(G.GDMError):
        G.solve_gmres(ctx, p6, G.incident_planewave(ctx, p6.pos, 600.0, W.XYPOL, kind_out=6))
    # the context stays usable
    check(G, ctx, pos, eps, step, 500.0)
