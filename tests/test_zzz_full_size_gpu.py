"""Parity at the benchmark's full sizes, in the configurations bench.py times. The 40 x 30 x 10 cuboid
(3N = 36,000) with TF32 factors refined to an estimated relative error of 1e-10 (the contraction of the
last two corrections), as bench.py runs it, and to a last relative correction of 1e-10: every
field element against the oracle's dense FP64 solution of the same system (stored once under
tests/golden/ by oracle/make_golden_cuboid.py, which calls only the oracle), the cross sections against
the oracle's, the exact FP64 residual rows F0 - A F of a seeded sample of cells (relative to |F0|
there) and the incident field at those cells; the 256 Eden blobs (50 to 1,500 cells each) in one
gdm_solve_batched call (estimated error 1e-10, as bench.py runs it), every item's cross sections, and three sampled items (the smallest, the largest,
one seeded) against the oracle's dense solve; the 1,970-cell cylinder's gradients at one wavelength
against the oracle's adjoint. The file sorts after the quick ones so that its long cases run late.
"""
import os

import numpy as np
import pytest
import torch

import gdm_workloads as W
import oracle as O

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cuboid40x30x10_oracle.npz")


@pytest.fixture(scope="module")
def G():
    import paper_2505_09545_gb300 as G
    return G


def t(x):
    return torch.tensor(np.ascontiguousarray(x), device=DEV)


def sampled_residual(pr, F0h, Fh, n_rows, seed):
    """max over right-hand sides of ||(F0 - A F)[rows]|| / ||F0[rows]|| for seeded rows (oracle, FP64)."""
    rows = np.sort(np.random.default_rng(seed).choice(pr.n, n_rows, replace=False))
    r = O.residual_rows(pr, F0h, Fh, rows)
    f0 = F0h.reshape(pr.n, 3, -1)[rows]
    nr = F0h.shape[1]
    return float(np.max(np.linalg.norm(r.reshape(-1, nr), axis=0) / np.linalg.norm(f0.reshape(-1, nr), axis=0))), rows


@pytest.mark.parametrize("err_estimate", [False, True])
def test_cuboid_40x30x10_full_size(G, err_estimate):
    """Both refinement stops: the last relative correction <= 1e-10, and the error estimated from the
    contraction of the last two corrections <= 1e-10 (GDM_SOLVE_ERR_ESTIMATE, which stops a step earlier
    when the corrections contract fast)."""
    s = W.cuboid_precision()
    lam = float(s.wavelengths[0])
    ctx = G.Context(0)
    try:
        prob = G.GDMProblem(t(s.pos), lam, 3, eps=t(s.eps), step=s.step)
        F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0)
        A = G.assemble(ctx, prob, "tf32")
        F, _, info = G.solve(ctx, prob, A, F0, "tf32", tol=1e-10, err_estimate=err_estimate)
        del A
        ext, sca, ab = (x.cpu().numpy() for x in G.cross_sections(ctx, prob, F0, F, np.ones(2)))
        F0h, Fh = F0.cpu().numpy().T, F.cpu().numpy().T
    finally:
        ctx.close()
    assert info["status"] == 0 and info["rel_correction"] <= (1e-7 if err_estimate else 1e-10), info
    # every element of both fields against the oracle's dense FP64 solve: ||dF_q|| / ||F_q|| <= 1e-9
    gold = np.load(GOLDEN)
    Fo = gold["F"]
    assert Fo.shape == Fh.shape
    err = np.linalg.norm(Fh - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
    assert np.all(err < 1e-9), (err, info)
    for g, o in zip((ext, sca, ab), gold["sigma"]):
        np.testing.assert_allclose(g, o, rtol=1e-9, atol=1e-9 * np.abs(gold["sigma"][0]).max())
    pr = O.Problem(s.pos, lam, 3, eps=s.eps, step=s.step)
    rel, rows = sampled_residual(pr, F0h, Fh, 48, seed=5)
    assert rel < 1e-10, (rel, info)
    # the incident field at the sampled cells
    f0o = pr.plane_wave(s.e0).reshape(pr.n, 3, -1)[rows]
    np.testing.assert_allclose(F0h.reshape(pr.n, 3, -1)[rows], f0o, rtol=0, atol=1e-14)
    # cross sections: the oracle's formula on the GPU fields
    xo = pr.cross_sections(F0h, Fh, s.e0)
    for g, o in zip((ext, sca, ab), xo):
        np.testing.assert_allclose(g, o, rtol=1e-9, atol=1e-9 * np.abs(xo[0]).max())



def test_cuboid_40x30x10_full_size_bf16(G):
    """The headline system with BF16 trailing updates (GDM_BF16_REFINE) refined to a relative correction of
    1e-10: every field element against the oracle's stored dense FP64 solution at 1e-9."""
    s = W.cuboid_precision()
    lam = float(s.wavelengths[0])
    ctx = G.Context(0)
    try:
        prob = G.GDMProblem(t(s.pos), lam, 3, eps=t(s.eps), step=s.step)
        F0 = G.incident_planewave(ctx, prob.pos, lam, s.e0)
        A = G.assemble(ctx, prob, "bf16")
        F, _, info = G.solve(ctx, prob, A, F0, "bf16", tol=1e-10)
        del A
        Fh = F.cpu().numpy().T
    finally:
        ctx.close()
    assert info["status"] == 0 and info["rel_correction"] <= 1e-10, info
    Fo = np.load(GOLDEN)["F"]
    err = np.linalg.norm(Fh - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
    assert np.all(err < 1e-9), (err, info)

def test_cuboid_nearfield_map_full_size(G):
    """The near-field leg of bench.py at its size: the 320 x 320 map 50 nm above the 40 x 30 x 10 cuboid (102,400
    points x 12,000 dipoles, E and H, both illuminations) from the oracle's stored fields, so that the kernel alone
    is compared: 64 seeded points against the oracle's repropagation, 1e-10 relative to the largest field value."""
    gold = np.load(GOLDEN)
    Fo = gold["F"]
    s = W.cuboid_precision()
    lam = float(s.wavelengths[0])
    r = W.nearfield_plane(320, 400.0, 100.0)
    ctx = G.Context(0)
    try:
        prob = G.GDMProblem(t(s.pos), lam, 3, eps=t(s.eps), step=s.step)
        E, H = G.nearfield(ctx, prob, t(Fo.T), t(r))
        pick = np.sort(np.random.default_rng(11).choice(r.shape[0], 64, replace=False))
        Eg = E.cpu().numpy().reshape(2, -1, 3)[:, pick]
        Hg = H.cpu().numpy().reshape(2, -1, 3)[:, pick]
    finally:
        ctx.close()
    pr = O.Problem(s.pos, lam, 3, eps=s.eps, step=s.step)
    Eo, Ho = pr.nearfield(Fo, r[pick], s.e0, with_incident=False)   # (64, 3, n_rhs)
    Eo, Ho = Eo.transpose(2, 0, 1), Ho.transpose(2, 0, 1)
    assert np.abs(Eg - Eo).max() <= 1e-10 * np.abs(Eo).max()
    assert np.abs(Hg - Ho).max() <= 1e-10 * np.abs(Ho).max()

def test_blob_batch_256_full_size(G):
    ss = W.blob_batch()
    ctx = G.Context(0)
    try:
        probs = [G.GDMProblem(t(s.pos), float(s.wavelengths[0]), 3, eps=t(s.eps), step=s.step) for s in ss]
        Fs, sigs, infos = G.solve_batched(ctx, probs, [s.e0 for s in ss], precision="tf32", tol=1e-10,
                                          err_estimate=True)
        torch.cuda.synchronize()
        Fh = [F.cpu().numpy().T for F in Fs]
        sig = [x.cpu().numpy() for x in sigs]
    finally:
        ctx.close()
    assert all(i["status"] == 0 for i in infos), [i for i in infos if i["status"] != 0][:3]
    sizes = np.array([s.n for s in ss])
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes)), int(np.random.default_rng(7).integers(len(ss)))}
    for k, s in enumerate(ss):
        lam = float(s.wavelengths[0])
        pr = O.Problem(s.pos, lam, 3, eps=s.eps, step=s.step)
        F0o = pr.plane_wave(s.e0)
        xo = pr.cross_sections(F0o, Fh[k], s.e0)
        for r in range(3):
            np.testing.assert_allclose(sig[k][r], xo[r], rtol=1e-9, atol=1e-9 * np.abs(xo[0]).max())
        if k in pick:
            Fo = pr.solve(F0o)
            err = np.linalg.norm(Fh[k] - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
            assert np.all(err < 1e-9), (s.name, s.n, err)


def test_cylinder_1970_cells_full_size_gradients(G):
    """The differentiation workload's full cylinder (r 80, h 100, d 10: N = 1,970, eps = 12.25 + 0.05i) at
    its first wavelength, through the autograd wrappers with TF32 factors: L = |E(probe)|^2 + sigma_sca and
    its gradients with respect to every position, every eps and the wavelength, against the oracle's FP64
    adjoint (1e-9 on L, 1e-8 normwise on the gradients)."""
    from paper_2505_09545_gb300 import autograd as AG
    cyl = W.cylinder_diff()
    lam = float(cyl.wavelengths[0])
    ctx = G.Context(0)
    try:
        pos = torch.tensor(cyl.pos, device=DEV, requires_grad=True)
        eps = torch.tensor(cyl.eps, device=DEV, requires_grad=True)
        wl = torch.tensor(lam, dtype=torch.float64, device=DEV, requires_grad=True)
        rp = torch.tensor(cyl.r_eval, device=DEV)
        F, sig = AG.scatter(pos, eps, wl, ctx, cyl.step, cyl.e0, precision="tf32")
        E = AG.nearfield(pos, eps, wl, F, rp, ctx, cyl.step, cyl.e0)
        L = (E.abs() ** 2).sum() + sig[:, 1].sum()
        L.backward()
        L, gp, ge, gl = float(L.detach()), pos.grad.cpu().numpy(), eps.grad.cpu().numpy(), float(wl.grad)
    finally:
        ctx.close()
    pr = O.Problem(cyl.pos, lam, 3, eps=cyl.eps, step=cyl.step)
    Lo, gpo, geo, glo = O.loss_and_grad_probe_sca(pr, cyl.e0, cyl.r_eval[0])
    assert abs(L - Lo) <= 1e-9 * abs(Lo), (L, Lo)
    assert np.linalg.norm(gp - gpo) <= 1e-8 * np.linalg.norm(gpo)
    assert np.linalg.norm(ge - geo) <= 1e-8 * np.linalg.norm(geo)
    assert abs(gl - glo) <= 1e-8 * abs(glo) + 1e-14
