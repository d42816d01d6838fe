"""Failure detection on the GPU without faulting it: every error comes back as a status code and the
context stays usable.

* a bounded device wait on a flag that nothing sets gives up (50 ms) and reports GDM_ERR_TIMEOUT;
* a NaN permittivity is reported (singular pivot or non-finite refinement), not propagated silently;
* an exactly singular system (one cell at eps = -2, where 1 - S alpha = 0, FP32 assembly) reports
  GDM_ERR_SINGULAR;
* a refinement capped at one step reports GDM_ERR_NOT_CONVERGED with the step count in its info.
After each, a regular solve on the same context matches the oracle.
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


def solve_ok(G, ctx):
    s = W.random_cells(80, seed=9)
    lam = float(s.wavelengths[0])
    prob = G.GDMProblem(t(s.pos), lam, 3, eps=t(s.eps), step=s.step)
    F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0)
    A = G.assemble(ctx, prob, "tf32")
    F, _, _ = G.solve(ctx, prob, A, F0, "tf32")
    pr = O.Problem(s.pos, lam, 3, eps=s.eps, step=s.step)
    Fo = pr.solve(pr.plane_wave(s.e0))
    err = np.linalg.norm(F.cpu().numpy().T - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
    assert np.all(err < 1e-9)


def test_bounded_wait_times_out(G, ctx):
    st = G.lib().gdm_diag_wait_timeout(ctx.h, 50.0)
    assert st == 8, G.lib().gdm_status_string(st)   # GDM_ERR_TIMEOUT
    solve_ok(G, ctx)


def test_nan_input_is_reported(G, ctx):
    s = W.random_cells(60, seed=5)
    eps = s.eps.copy()
    eps[17] = np.nan
    prob = G.GDMProblem(t(s.pos), 550.0, 3, eps=t(eps), step=s.step)
    F0 = G.incident_planewave(ctx, prob.pos, 550.0, s.e0)
    A = G.assemble(ctx, prob, "tf32")
    with pytest.raises(G.GDMError) as e:
        G.solve(ctx, prob, A, F0, "tf32")
    assert e.value.status in (3, 4)                  # GDM_ERR_NONFINITE or GDM_ERR_SINGULAR
    solve_ok(G, ctx)


@pytest.mark.parametrize("prec", ["tf32", "fp32"])
def test_exactly_singular_system(G, ctx, prec):
    """The FP32 assembly forms the cell diagonal as 1 + (eps - 1)/3, exactly 0 at eps = -2 (the FP64 one,
    1 - S alpha with S = -4 pi/(3 d^3), rounds to ~1e-16: nearly, not exactly, singular)."""
    prob = G.GDMProblem(t(np.zeros((1, 3))), 500.0, 3, eps=t(np.array([-2.0 + 0.0j])), step=10.0)
    F0 = G.incident_planewave(ctx, prob.pos, 500.0, W.XPOL)
    A = G.assemble(ctx, prob, prec)
    with pytest.raises(G.GDMError) as e:
        G.solve(ctx, prob, A, F0, prec)
    assert e.value.status == 4                       # GDM_ERR_SINGULAR
    solve_ok(G, ctx)


def test_refinement_cap(G, ctx):
    s = W.random_cells(200, seed=6)
    lam = float(s.wavelengths[0])
    prob = G.GDMProblem(t(s.pos), lam, 3, eps=t(s.eps), step=s.step)
    F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0)
    A = G.assemble(ctx, prob, "tf32")
    with pytest.raises(G.GDMError) as e:
        G.solve(ctx, prob, A, F0, "tf32", max_iter=1, tol=1e-15)
    assert e.value.status == 5                       # GDM_ERR_NOT_CONVERGED
    solve_ok(G, ctx)
