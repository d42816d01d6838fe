"""Batched solves (gdm_solve_batched) and the LU block-width autotuner (gdm_autotune) against the oracle.

A batch mixes uneven cell structures (3N from 120 to 1860, spanning several outer LU blocks with ragged
tails), Eden blobs on the 15 nm mesh, a metallic structure whose in-block pivots fail the certificate
(refactored with whole-column pivoting inside the batch) and an ED/MD dipole array, each at its own
wavelength with two illuminations. Every item's refined fields must match the oracle's dense solve to
1e-9 and its cross sections to 1e-9 relative (absolute floor 1e-9 x sigma_ext), whatever the number of
streams the batch runs on.
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


def t(x):
    return torch.tensor(np.ascontiguousarray(x), device=DEV)


def structures():
    out = []
    rng = np.random.default_rng(21)
    for i, n in enumerate((40, 90, 180, 400, 620)):
        s = W.random_cells(n, seed=40 + i)
        s.wavelengths = np.array([rng.uniform(400.0, 1000.0)])
        out.append(s)
    metal = W.random_cells(120, seed=3)
    metal.eps = np.full(metal.n, -2.2 + 0.3j)
    metal.wavelengths = np.array([500.0])
    out.append(metal)
    out += W.blob_batch(n_struct=3, n_min=50, n_max=300, seed=9)
    out.append(W.metasurface_edmd(nx=8, ny=6, seed=5, n_lambda=1))
    out[-1].wavelengths = np.array([640.0])
    return out


def gpu_problem(G, s):
    lam = float(s.wavelengths[0])
    if s.kind == 3:
        return G.GDMProblem(t(s.pos), lam, 3, eps=t(s.eps), step=s.step)
    al = O.lorentz_alpha6(s.omega0_e, s.omega0_m, s.gamma_ev, s.amp_nm, lam)
    return G.GDMProblem(t(s.pos), lam, 6, alpha6=t(al))


def check_against_oracle(s, F, sig):
    lam = float(s.wavelengths[0])
    if s.kind == 3:
        pr = O.Problem(s.pos, lam, 3, eps=s.eps, step=s.step)
    else:
        pr = O.Problem(s.pos, lam, 6, alpha6=O.lorentz_alpha6(s.omega0_e, s.omega0_m, s.gamma_ev, s.amp_nm, lam))
    F0o = pr.plane_wave(s.e0)
    Fo = pr.solve(F0o)
    err = np.linalg.norm(F.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
    assert np.all(err < 1e-9), (s.name, err)
    xo = pr.cross_sections(F0o, Fo, s.e0)
    g = sig.cpu().numpy()
    for r in range(3):
        np.testing.assert_allclose(g[r], xo[r], rtol=1e-9, atol=1e-9 * abs(xo[0]).max())


@pytest.mark.parametrize("n_streams,precision", [(1, "tf32"), (4, "tf32"), (3, "fp32"), (2, "fp64")])
def test_batched_matches_oracle(G, n_streams, precision):
    ctx = G.Context(0)
    try:
        ss = structures()
        probs = [gpu_problem(G, s) for s in ss]
        Fs, sigs, infos = G.solve_batched(ctx, probs, [s.e0 for s in ss], precision=precision, n_streams=n_streams)
        torch.cuda.synchronize()
        for s, F, sig, info in zip(ss, Fs, sigs, infos):
            assert info["status"] == 0, (s.name, info)
            check_against_oracle(s, F, sig)
        assert infos[5]["refactored"] == 1  # the metallic structure
        assert sum(i["refactored"] for i in infos) == 1
    finally:
        ctx.close()


def test_batch_follows_the_context_stream(G):
    """Work queued on the caller's stream before the batch is visible to it (the positions below are
    written by a copy on that stream just before the call)."""
    ctx = G.Context(0)
    try:
        s = W.random_cells(150, seed=77)
        pos = torch.zeros((s.n, 3), dtype=torch.float64, device=DEV)
        host = torch.tensor(s.pos).pin_memory()
        pos.copy_(host, non_blocking=True)
        prob = G.GDMProblem(pos, float(s.wavelengths[0]), 3, eps=t(s.eps), step=s.step)
        Fs, sigs, infos = G.solve_batched(ctx, [prob], [s.e0], precision="tf32", n_streams=2)
        out = sigs[0].clone()  # on the caller's stream, after the batch
        torch.cuda.synchronize()
        check_against_oracle(s, Fs[0], out)
    finally:
        ctx.close()


def test_autotune_table_and_tuned_solves(G):
    ctx = G.Context(0)
    try:
        table = G.autotune(ctx, [600, 1800, 3000], precision="tf32")
        assert len(table) == 8
        for cls in (1, 2, 3):  # 600 -> <= 1024, 1800 -> <= 2048, 3000 -> <= 4096
            assert table[cls] in (128, 256, 512), table
        assert table[0] == 0 and all(v == 0 for v in table[4:]), table
        ss = [W.random_cells(n, seed=60 + n) for n in (200, 600, 1000)]
        probs = [gpu_problem(G, s) for s in ss]
        Fs, sigs, infos = G.solve_batched(ctx, probs, [s.e0 for s in ss], precision="tf32", n_streams=3)
        for s, F, sig in zip(ss, Fs, sigs):
            check_against_oracle(s, F, sig)
    finally:
        ctx.close()
