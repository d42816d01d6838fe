"""Seeded synthetic inputs for the Green's Dyadic Method (GDM) hot path.

This module is shared by the CPU oracle, the tests and the benchmark. It only
*draws* inputs (cell positions on cubic meshes, per-cell permittivities,
wavelengths, illumination polarisations, Lorentzian resonance parameters,
near-field probe grids). It contains none of the method's arithmetic: no Green
tensor, no polarisability, no linear algebra. Each side (oracle and CUDA
library) turns these raw inputs into the physics on its own.

Workloads follow the shapes of the paper's examples and benchmarks:
discretised dielectric particles on a cubic mesh (paper Sec. "Volume
discretization polarizabilities", minimum example and runtime benchmark) and
arrays of effective electric/magnetic point dipoles (Sec. "Hybrid
discretization GDM", quasi-BIC array example).

Units: nanometres for lengths and wavelengths, electron-volts for Lorentzian
resonance energies. All arrays are numpy float64 / complex128.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

HC_EV_NM = 1239.84198  # h*c in eV*nm: converts a photon energy in eV to a vacuum wavelength in nm


@dataclass
class Structure:
    """One scattering problem's raw inputs.

    kind == 3: discretised cells (electric response only), `eps` per cell and
    mesh `step`. kind == 6: effective point dipoles with Lorentzian electric and
    magnetic resonances (`omega0_e`, `omega0_m`, `gamma_ev`, `amp_nm`).
    """
    name: str
    kind: int
    pos: np.ndarray                     # (n, 3) float64, nm
    step: float = 0.0                   # cubic mesh step d (nm); 0 for point dipoles
    eps: Optional[np.ndarray] = None    # (n,) complex128 cell permittivity (kind 3)
    omega0_e: Optional[np.ndarray] = None  # (n,) eV, electric resonance (kind 6)
    omega0_m: Optional[np.ndarray] = None  # (n,) eV, magnetic resonance (kind 6)
    gamma_ev: float = 0.0               # Lorentzian width (eV) (kind 6)
    amp_nm: float = 0.0                 # Lorentzian amplitude radius a (nm): static alpha = a^3 (kind 6)
    eps_env: float = 1.0
    wavelengths: np.ndarray = field(default_factory=lambda: np.array([500.0]))
    e0: np.ndarray = field(default_factory=lambda: np.array([[1, 0, 0]], complex))  # (n_rhs, 3) E amplitudes
    khat: np.ndarray = field(default_factory=lambda: np.array([0.0, 0.0, 1.0]))     # propagation direction
    r_eval: Optional[np.ndarray] = None  # (m, 3) near-field evaluation points

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_rhs(self) -> int:
        return int(self.e0.shape[0])


def _lattice(ix, iy, iz, step, offset=(0.0, 0.0, 0.0)):
    g = np.stack(np.meshgrid(ix, iy, iz, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    return (g + np.asarray(offset, np.float64)) * step


def sphere_cells(radius, step):
    """Cubic-mesh cells d*(i,j,l) with |r| <= radius (origin on a cell centre)."""
    m = int(np.ceil(radius / step)) + 1
    r = np.arange(-m, m + 1)
    g = _lattice(r, r, r, step)
    keep = np.einsum("ij,ij->i", g, g) <= radius * radius * (1 + 1e-12)
    return g[keep]


def cuboid_cells(nx, ny, nz, step):
    """nx*ny*nz cells centred on the origin (half-step offsets for even counts)."""
    return _lattice(np.arange(nx) - (nx - 1) / 2, np.arange(ny) - (ny - 1) / 2,
                    np.arange(nz) - (nz - 1) / 2, step)


def cylinder_cells(radius, height, step):
    """Cylinder along z: columns d*(i,j) with i^2+j^2 <= (radius/d)^2, layers (l+1/2)*d in [0, height]."""
    m = int(np.ceil(radius / step)) + 1
    r = np.arange(-m, m + 1)
    nz = int(round(height / step))
    g = _lattice(r, r, np.arange(nz), step, offset=(0.0, 0.0, 0.5))
    keep = g[:, 0] ** 2 + g[:, 1] ** 2 <= radius * radius * (1 + 1e-12)
    return g[keep]


def eden_blob(n_cells, step, rng):
    """Random connected blob grown from the origin: repeatedly add a uniformly
    chosen empty face-neighbour of the current set (Eden growth)."""
    occupied = {(0, 0, 0)}
    order = [(0, 0, 0)]
    frontier = []
    frontier_set = set()
    nbrs = ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))

    def push(c):
        for d in nbrs:
            q = (c[0] + d[0], c[1] + d[1], c[2] + d[2])
            if q not in occupied and q not in frontier_set:
                frontier_set.add(q)
                frontier.append(q)

    push((0, 0, 0))
    while len(order) < n_cells:
        k = int(rng.integers(len(frontier)))
        q = frontier[k]
        frontier[k] = frontier[-1]
        frontier.pop()
        frontier_set.discard(q)
        occupied.add(q)
        order.append(q)
        push(q)
    return np.asarray(order, np.float64) * step


def nearfield_grid_outside_sphere(half_width, n_per_axis, exclude_radius):
    """linspace(-w, w, n)^3 probe grid with points at |r| <= exclude_radius removed."""
    a = np.linspace(-half_width, half_width, n_per_axis)
    g = np.stack(np.meshgrid(a, a, a, indexing="ij"), -1).reshape(-1, 3)
    keep = np.einsum("ij,ij->i", g, g) > exclude_radius * exclude_radius
    return np.ascontiguousarray(g[keep])


def nearfield_plane(n_side, half_width, z):
    """n_side x n_side near-field map on the plane at height z: linspace(-w, w, n_side)^2 (a field map above
    a structure, the paper's near-field example in 2D)."""
    a = np.linspace(-half_width, half_width, n_side)
    g = np.stack(np.meshgrid(a, a, indexing="ij"), -1).reshape(-1, 2)
    return np.ascontiguousarray(np.concatenate([g, np.full((g.shape[0], 1), float(z))], 1))


XPOL = np.array([[1.0, 0.0, 0.0]], complex)
XYPOL = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]], complex)


def sphere_plain_fp64():
    """Dielectric sphere R = 60 nm, step 10 nm (N = 925), eps = 12.25, lambda = 600 nm,
    x-polarised plane wave along +z, near field on a 10^3 grid spanning +-150 nm
    outside the sphere (points within R + d/2 removed)."""
    pos = sphere_cells(60.0, 10.0)
    return Structure(name="sphere_r60_d10", kind=3, pos=pos, step=10.0,
                     eps=np.full(pos.shape[0], 12.25 + 0.0j), wavelengths=np.array([600.0]),
                     e0=XPOL.copy(), r_eval=nearfield_grid_outside_sphere(150.0, 10, 65.0))


def cuboid_precision(nx=40, ny=30, nz=10, step=10.0, seed=2):
    """Cuboid nx*ny*nz cells (40x30x10 -> N = 12,000, 3N = 36,000), per-cell
    eps ~ U[2,16] + i U[0,0.5], lambda = 500 nm, x- and y-polarised plane waves along +z."""
    rng = np.random.default_rng(seed)
    pos = cuboid_cells(nx, ny, nz, step)
    n = pos.shape[0]
    eps = rng.uniform(2.0, 16.0, n) + 1j * rng.uniform(0.0, 0.5, n)
    return Structure(name=f"cuboid_{nx}x{ny}x{nz}_d{step:g}", kind=3, pos=pos, step=step, eps=eps,
                     wavelengths=np.array([500.0]), e0=XYPOL.copy())


def blob_batch(n_struct=256, n_min=50, n_max=1500, step=15.0, seed=3):
    """n_struct independent Eden blobs with N ~ U{n_min..n_max}, eps ~ U[2,16] (real),
    own lambda ~ U[400,1000] nm, x- and y-polarised plane waves along +z."""
    rng = np.random.default_rng(seed)
    out: List[Structure] = []
    for s in range(n_struct):
        n = int(rng.integers(n_min, n_max + 1))
        pos = eden_blob(n, step, rng)
        eps = rng.uniform(2.0, 16.0, n) + 0.0j
        lam = float(rng.uniform(400.0, 1000.0))
        out.append(Structure(name=f"blob{s}", kind=3, pos=pos, step=step, eps=eps,
                             wavelengths=np.array([lam]), e0=XYPOL.copy()))
    return out


def metasurface_edmd(nx=64, ny=64, pitch=400.0, seed=4, n_lambda=32):
    """nx*ny square array (z = 0) of point scatterers with Lorentzian electric and
    magnetic resonances omega0 ~ U[2,3] eV (drawn separately), width 0.1 eV,
    amplitude radius 80 nm; lambdas linspace(500, 800, n_lambda); x- and y-polarised
    normal-incidence plane waves."""
    rng = np.random.default_rng(seed)
    pos = _lattice(np.arange(nx) - (nx - 1) / 2, np.arange(ny) - (ny - 1) / 2, np.array([0.0]), pitch)
    n = pos.shape[0]
    w_e = rng.uniform(2.0, 3.0, n)
    w_m = rng.uniform(2.0, 3.0, n)
    return Structure(name=f"metasurface_{nx}x{ny}_p{pitch:g}", kind=6, pos=pos, omega0_e=w_e,
                     omega0_m=w_m, gamma_ev=0.1, amp_nm=80.0,
                     wavelengths=np.linspace(500.0, 800.0, n_lambda), e0=XYPOL.copy())


def cylinder_diff(radius=80.0, height=100.0, step=10.0, n_lambda=8):
    """Cylinder r = 80 nm, h = 100 nm, step 10 nm, eps = 12.25 + 0.05i, lambdas
    linspace(450, 800, 8), x-polarised plane wave along +z; one probe point 50 nm
    above the top face (top cell centre + d/2 + 50 nm)."""
    pos = cylinder_cells(radius, height, step)
    ztop = pos[:, 2].max() + step / 2 + 50.0
    return Structure(name=f"cylinder_r{radius:g}_h{height:g}_d{step:g}", kind=3, pos=pos, step=step,
                     eps=np.full(pos.shape[0], 12.25 + 0.05j),
                     wavelengths=np.linspace(450.0, 800.0, n_lambda), e0=XPOL.copy(),
                     r_eval=np.array([[0.0, 0.0, ztop]]))


def random_cells(n, step=10.0, seed=0, box=None, lossy=True):
    """Small random structure for parity tests: n distinct cells drawn from a box of
    the cubic mesh, eps ~ U[2,16] + i U[0,0.5]."""
    rng = np.random.default_rng(seed)
    if box is None:
        box = max(2, int(np.ceil(n ** (1 / 3) * 1.6)))
    flat = rng.choice(box ** 3, size=n, replace=False)
    ijk = np.stack(np.unravel_index(flat, (box, box, box)), -1).astype(np.float64)
    pos = (ijk - (box - 1) / 2) * step
    eps = rng.uniform(2.0, 16.0, n) + 1j * (rng.uniform(0.0, 0.5, n) if lossy else 0.0)
    return Structure(name=f"random{n}_s{seed}", kind=3, pos=pos, step=step, eps=eps,
                     wavelengths=np.array([rng.uniform(400.0, 900.0)]), e0=XYPOL.copy())


def omega_ev_to_wavelength_nm(w_ev):
    return HC_EV_NM / np.asarray(w_ev, np.float64)


def sphere_points(n, radius, center=(0.0, 0.0, 0.0), seed=0):
    """n seeded points uniformly distributed on a sphere (probe and source positions around a structure)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return np.asarray(center, np.float64) + radius * v


def farthest_points(pos, m, seed=0):
    """m positions picked from pos by farthest-point sampling from a seeded start (effective-dipole sites
    spread through a structure)."""
    pos = np.asarray(pos, np.float64)
    rng = np.random.default_rng(seed)
    idx = [int(rng.integers(len(pos)))]
    d = np.linalg.norm(pos - pos[idx[0]], axis=1)
    while len(idx) < m:
        j = int(np.argmax(d))
        idx.append(j)
        d = np.minimum(d, np.linalg.norm(pos - pos[j], axis=1))
    return pos[np.sort(idx)]


def gpm_illumination_set(n_angles=8, n_sources=8, source_radius=200.0, center=(0.0, 0.0, 0.0), seed=0):
    """Illuminations for an effective-model extraction: plane waves along n_angles seeded directions with
    two orthogonal polarisations each (khat, e0 lists), and n_sources electric dipole sources of seeded
    orientation on a sphere of radius source_radius (positions (s, 3), moments (s, 6)); the source moments
    have magnitude source_radius^3 so that their near fields at the centre are of order one, like the
    plane waves'."""
    rng = np.random.default_rng(seed)
    khat, e0 = [], []
    for _ in range(n_angles):
        k = rng.standard_normal(3)
        k /= np.linalg.norm(k)
        a = np.cross(k, [1.0, 0.0, 0.0] if abs(k[0]) < 0.9 else [0.0, 1.0, 0.0])
        a /= np.linalg.norm(a)
        b = np.cross(k, a)
        for pol in (a, b):
            khat.append(k)
            e0.append(pol.astype(np.complex128))
    ds_pos = sphere_points(n_sources, source_radius, center, seed + 1)
    mom = np.zeros((n_sources, 6), np.complex128)
    d = rng.standard_normal((n_sources, 3))
    mom[:, :3] = source_radius ** 3 * d / np.linalg.norm(d, axis=1, keepdims=True)
    return khat, e0, ds_pos, mom
