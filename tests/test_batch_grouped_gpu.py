"""The grouped factorisation and refinement of a batch: gdm_solve_batched at TF32 factors all its problems
together, one lock-step launch per panel step of the largest problem (panels, interchanges with the U rows,
tensor-core updates over the tiles of every problem), captured once into a CUDA graph and replayed; then
refines all of them together (residuals, scaling, both triangular solves and the update as one launch each
per step, one host check of every problem's norms per step).

The sizes sit on and around the panel (32 rows) and outer block (128/256/512 rows) boundaries, from a
single cell (3N = 3) up to 3N = 1,029, with ragged tails, so that problems drop out of the lock step at
every kind of step: inside a block, at a block edge, and with a partial last panel. Every problem's
refined fields must match the oracle's dense solve to 1e-9 and its cross sections to 1e-9, for each outer
block width, on the first call (capture) and on a second call with new buffers (replay through a
rewritten table), and the per-problem path (GDM_BATCH_POOL) must agree with the oracle on the same batch.
"""
import os

import numpy as np
import pytest
import torch

import gdm_workloads as W
import oracle as O

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None

# cells -> 3N: 1 -> 3, 11 -> 33, 21 -> 63, 32 -> 96, 43 -> 129, 86 -> 258, 171 -> 513, 192 -> 576, 343 -> 1029
CELLS = (1, 11, 21, 32, 43, 86, 171, 192, 343)


@pytest.fixture(scope="module")
def G():
    import paper_2505_09545_gb300 as G
    return G


def t(x):
    return torch.tensor(np.ascontiguousarray(x), device=DEV)


def structures():
    ss = [W.random_cells(n, seed=200 + n) for n in CELLS]
    ss += W.blob_batch(n_struct=2, n_min=120, n_max=260, seed=13)
    return ss


def oracle_solution(s):
    pr = O.Problem(s.pos, float(s.wavelengths[0]), 3, eps=s.eps, step=s.step)
    F0 = pr.plane_wave(s.e0)
    F = pr.solve(F0)
    return F, pr.cross_sections(F0, F, s.e0)


@pytest.fixture(scope="module")
def reference():
    ss = structures()
    return ss, [oracle_solution(s) for s in ss]


def check(ss, ref, Fs, sigs, infos):
    for s, (Fo, xo), F, sig, info in zip(ss, ref, Fs, sigs, infos):
        assert info["status"] == 0, (s.name, info)
        err = np.linalg.norm(F.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
        assert np.all(err < 1e-9), (s.name, err)
        g = sig.cpu().numpy()
        for r in range(3):
            np.testing.assert_allclose(g[r], xo[r], rtol=1e-9, atol=1e-9 * abs(xo[0]).max())


@pytest.mark.parametrize("nb", [128, 256, 512])
def test_grouped_factorisation_matches_oracle(G, reference, nb, monkeypatch):
    ss, ref = reference
    monkeypatch.setenv("GDM_BATCH_NB", str(nb))
    monkeypatch.delenv("GDM_BATCH_POOL", raising=False)
    ctx = G.Context(0)
    try:
        for call in range(2):  # capture, then replay with new buffers
            probs = [G.GDMProblem(t(s.pos), float(s.wavelengths[0]), 3, eps=t(s.eps), step=s.step) for s in ss]
            l0 = ctx.launches
            Fs, sigs, infos = G.solve_batched(ctx, probs, [s.e0 for s in ss], precision="tf32", n_streams=3)
            torch.cuda.synchronize()
            check(ss, ref, Fs, sigs, infos)
            assert sum(i["refactored"] for i in infos) == 0
            assert ctx.launches > l0
    finally:
        ctx.close()


@pytest.mark.parametrize("switch", ["GDM_BATCH_POOL", "GDM_BATCH_REFINE_POOL"])
def test_per_problem_path_agrees(G, reference, monkeypatch, switch):
    """The per-problem factorisations (GDM_BATCH_POOL) and the per-problem refinements on the stream pool
    (GDM_BATCH_REFINE_POOL) reach the oracle too."""
    ss, ref = reference
    monkeypatch.setenv(switch, "1")
    ctx = G.Context(0)
    try:
        probs = [G.GDMProblem(t(s.pos), float(s.wavelengths[0]), 3, eps=t(s.eps), step=s.step) for s in ss]
        Fs, sigs, infos = G.solve_batched(ctx, probs, [s.e0 for s in ss], precision="tf32", n_streams=3)
        torch.cuda.synchronize()
        check(ss, ref, Fs, sigs, infos)
    finally:
        ctx.close()


def test_autotuned_grouped_width(G, reference, monkeypatch):
    """gdm_autotune_batched picks one of the candidate widths for these sizes, keeps it in the context, and
    the batch factored with it still matches the oracle; a width fixed by GDM_BATCH_NB makes it refuse."""
    ss, ref = reference
    monkeypatch.delenv("GDM_BATCH_NB", raising=False)
    monkeypatch.delenv("GDM_BATCH_POOL", raising=False)
    ctx = G.Context(0)
    try:
        probs = [G.GDMProblem(t(s.pos), float(s.wavelengths[0]), 3, eps=t(s.eps), step=s.step) for s in ss]
        nb = G.autotune_batched(ctx, [p.size for p in probs])
        assert nb in (128, 256, 512)
        Fs, sigs, infos = G.solve_batched(ctx, probs, [s.e0 for s in ss], precision="tf32", n_streams=2)
        torch.cuda.synchronize()
        check(ss, ref, Fs, sigs, infos)
        monkeypatch.setenv("GDM_BATCH_NB", "256")
        with pytest.raises(G.GDMError):
            G.autotune_batched(ctx, [p.size for p in probs])
    finally:
        ctx.close()


def test_grouped_refinement_reports_non_convergence(G, reference):
    """A refinement cap of one step with an unreachable tolerance: every problem of the grouped refinement
    reports GDM_ERR_NOT_CONVERGED in its record and the call fails with it; the context still solves the
    batch correctly afterwards."""
    ss, ref = reference
    ctx = G.Context(0)
    try:
        probs = [G.GDMProblem(t(s.pos), float(s.wavelengths[0]), 3, eps=t(s.eps), step=s.step) for s in ss]
        with pytest.raises(G.GDMError) as e:
            G.solve_batched(ctx, probs, [s.e0 for s in ss], precision="tf32", n_streams=2, max_iter=1, tol=1e-30)
        assert "NOT_CONVERGED" in str(e.value)
        Fs, sigs, infos = G.solve_batched(ctx, probs, [s.e0 for s in ss], precision="tf32", n_streams=2)
        torch.cuda.synchronize()
        check(ss, ref, Fs, sigs, infos)
    finally:
        ctx.close()
