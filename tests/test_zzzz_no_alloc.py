"""gdm_cross_sections_noalloc against gdm_cross_sections, through the C ABI.

The no-allocation variant keeps its partial sums in one fixed device buffer per device, so two calls
in a row with different problems (cells, then ED/MD dipoles, with ragged sizes) must each match the
allocating entry point; the tolerance is the cross-section parity tolerance of the GPU tests
(1e-9 relative, absolute floor 1e-9 x max value). The file sorts last so that it also runs after
every other GPU test has used the library on the same device.
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


def close(a, b):
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    return np.allclose(a, b, rtol=1e-9, atol=1e-9 * np.abs(b).max())


def random_fields(n_sys, n_rhs, seed):
    rng = np.random.default_rng(seed)
    F0 = rng.standard_normal((n_rhs, n_sys)) + 1j * rng.standard_normal((n_rhs, n_sys))
    F = rng.standard_normal((n_rhs, n_sys)) + 1j * rng.standard_normal((n_rhs, n_sys))
    return t(F0), t(F)


def test_noalloc_matches_allocating_entry_point_over_two_calls(G):
    ctx = G.Context(0)
    try:
        s1 = W.random_cells(1000, seed=11)  # 4 blocks of 256 with a ragged tail
        p1 = G.GDMProblem(t(s1.pos), 532.0, 3, eps=t(s1.eps), step=s1.step)
        F0a, Fa = random_fields(3 * s1.n, 3, seed=5)
        e2a = [1.0, 2.5, 0.7]
        s2 = W.metasurface_edmd(nx=9, ny=7, pitch=400.0)
        al = O.lorentz_alpha6(s2.omega0_e, s2.omega0_m, s2.gamma_ev, s2.amp_nm, 640.0)
        p2 = G.GDMProblem(t(s2.pos), 640.0, 6, alpha6=t(al))
        F0b, Fb = random_fields(6 * s2.n, 2, seed=6)
        e2b = [1.0, 1.0]

        out1 = torch.full((3, 3), float("nan"), dtype=torch.float64, device=DEV)
        out2 = torch.full((3, 2), float("nan"), dtype=torch.float64, device=DEV)
        G.binding.cross_sections_noalloc(ctx, p1, F0a, Fa, e2a, out1)
        G.binding.cross_sections_noalloc(ctx, p2, F0b, Fb, e2b, out2)
        torch.cuda.synchronize()
        ref1 = torch.stack(G.cross_sections(ctx, p1, F0a, Fa, e2a))
        ref2 = torch.stack(G.cross_sections(ctx, p2, F0b, Fb, e2b))
        assert torch.isfinite(out1).all() and torch.isfinite(out2).all()
        assert close(out1, ref1)
        assert close(out2, ref2)
        # the first problem again, after the second one has overwritten the shared scratch
        out3 = torch.empty((3, 3), dtype=torch.float64, device=DEV)
        G.binding.cross_sections_noalloc(ctx, p1, F0a, Fa, e2a, out3)
        assert close(out3, ref1)
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(G):
    ctx = G.Context(0)
    try:
        # ceil(n/256) * n_rhs = 1025 * 64 > 65536: refused on the host before anything is launched,
        # so the tiny buffers below are never read
        n = 256 * 1025
        tiny = torch.zeros(8, dtype=torch.complex128, device=DEV)
        pos = torch.zeros((1, 3), dtype=torch.float64, device=DEV)
        p = G.GDMProblem(pos, 500.0, 3, eps=tiny, step=10.0)
        p.n = n
        out = torch.zeros((3, 64), dtype=torch.float64, device=DEV)
        F = torch.zeros((64, 8), dtype=torch.complex128, device=DEV)
        with pytest.raises(G.GDMError) as e:
            G.binding.cross_sections_noalloc(ctx, p, F, F, [1.0] * 64, out)
        assert e.value.status == 2 and "fixed scratch" in str(e.value)
        # the context stays usable
        s = W.random_cells(40, seed=3)
        p1 = G.GDMProblem(t(s.pos), 500.0, 3, eps=t(s.eps), step=s.step)
        F0, F1 = random_fields(3 * s.n, 1, seed=7)
        out1 = torch.empty((3, 1), dtype=torch.float64, device=DEV)
        G.binding.cross_sections_noalloc(ctx, p1, F0, F1, [1.0], out1)
        assert close(out1, torch.stack(G.cross_sections(ctx, p1, F0, F1, [1.0])))
    finally:
        ctx.close()


def test_noalloc_allocates_no_device_memory(G):
    """The defining property: a call takes no device memory. The first call on a device looks up the fixed
    buffer (and, in a fresh process, loads the module that holds it), so the check runs on a context created
    afterwards, whose own workspace has never been allocated: free device memory must not move across the
    call."""
    s = W.random_cells(300, seed=21)
    F0, F = random_fields(3 * s.n, 2, seed=8)
    pos, eps = t(s.pos), t(s.eps)
    out = torch.empty((3, 2), dtype=torch.float64, device=DEV)
    warm = G.Context(0)
    try:
        G.binding.cross_sections_noalloc(warm, G.GDMProblem(pos, 600.0, 3, eps=eps, step=s.step), F0, F,
                                         [1.0, 1.0], out)
        torch.cuda.synchronize()
    finally:
        warm.close()
    ctx = G.Context(0)
    try:
        p = G.GDMProblem(pos, 600.0, 3, eps=eps, step=s.step)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(DEV)[0]
        G.binding.cross_sections_noalloc(ctx, p, F0, F, [1.0, 1.0], out)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info(DEV)[0]
        assert free1 == free0
        assert torch.isfinite(out).all()
    finally:
        ctx.close()
