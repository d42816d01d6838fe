"""Effective-model (GPM) extraction on the GPU (gdm_gpm_extract) against the oracle.

Tolerances: the extraction chains refined solves (1e-12), near-field sums (FP64) and two FP64
least-squares fits, so alpha_eff agrees with the oracle's (LAPACK least squares) to 1e-8 of its
largest entry; the exact case (effective dipoles on the cells) to the same level against the
closed form alpha A^{-1}.
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


def run_both(G, s, lam, r_gpm, n_angles, n_sources, n_probe, seed, precision):
    khat, e0, ds_pos, ds_mom = W.gpm_illumination_set(n_angles=n_angles, n_sources=n_sources,
                                                      source_radius=150.0, seed=seed)
    r_probe = W.sphere_points(n_probe, 90.0, seed=seed + 7)
    ctx = G.Context(0)
    try:
        prob = G.GDMProblem(t(s.pos), lam, 3, eps=t(s.eps), step=s.step)
        a, P, rel = G.gpm_extract(ctx, prob, t(r_gpm), t(r_probe), khat, e0, t(ds_pos), t(ds_mom),
                                  precision=precision)
        a, P = a.cpu().numpy(), P.cpu().numpy()
    finally:
        ctx.close()
    pr = O.Problem(s.pos, lam, 3, eps=s.eps, step=s.step)
    ao, Po, F0g, relo = O.gpm_extract(pr, r_gpm, r_probe, khat, e0, ds_pos, ds_mom)
    return a, P, rel, ao, Po, relo, pr


@pytest.mark.parametrize("precision", ["tf32", "fp64"])
def test_gpm_matches_oracle(G, precision):
    """60 cells, 6 effective dipole pairs, 28 plane waves + 10 dipole sources, 80 probes."""
    s = W.random_cells(60, seed=21)
    r_gpm = W.farthest_points(s.pos, 6, 21)
    a, P, rel, ao, Po, relo, _ = run_both(G, s, 580.0, r_gpm, 14, 10, 80, 21, precision)
    np.testing.assert_allclose(P, Po, atol=1e-8 * np.abs(Po).max())
    np.testing.assert_allclose(a, ao, atol=1e-8 * np.abs(ao).max())
    assert abs(rel - relo) <= 1e-6 * relo + 1e-12


def test_gpm_sites_on_cells_is_exact(G):
    """Effective dipoles on the cells of a 5-cell structure: alpha_eff = alpha A^{-1} in the electric blocks
    and zero elsewhere (the same closed form as the oracle's pin)."""
    s = W.random_cells(5, seed=8)
    lam = 560.0
    a, P, rel, ao, Po, relo, pr = run_both(G, s, lam, s.pos, 16, 10, 60, 8, "fp32")
    alpha = np.repeat(O.cell_polarizability(s.eps, 1.0, s.step), 3)
    ee = alpha[:, None] * np.linalg.inv(pr.matrix())
    want = np.zeros((30, 30), complex)
    for j in range(5):
        for l in range(5):
            want[6 * j:6 * j + 3, 6 * l:6 * l + 3] = ee[3 * j:3 * j + 3, 3 * l:3 * l + 3]
    assert rel < 1e-9
    np.testing.assert_allclose(a, want, atol=1e-8 * np.abs(want).max())


def test_gpm_rejects_too_few_illuminations(G):
    s = W.random_cells(20, seed=2)
    khat, e0, ds_pos, ds_mom = W.gpm_illumination_set(n_angles=2, n_sources=1, seed=2)
    ctx = G.Context(0)
    try:
        prob = G.GDMProblem(t(s.pos), 500.0, 3, eps=t(s.eps), step=s.step)
        with pytest.raises(G.GDMError):
            G.gpm_extract(ctx, prob, t(W.farthest_points(s.pos, 2, 2)), t(W.sphere_points(20, 90.0)), khat, e0,
                          t(ds_pos), t(ds_mom))
    finally:
        ctx.close()
