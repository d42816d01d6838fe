"""CPU FP64 oracle for the Green's Dyadic Method (GDM) hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this module:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it. It shares no code with the CUDA library.

Plain, slow, obviously-correct numpy float64/complex128 code that follows the
paper (Wiecha et al., "TorchGDM", arXiv:2505.09545) in its own notation:

* Sec. "Formalism and implementation", Eq. (LPS_6by6) and Eq. (superprop_G):
  the 6x6 Green dyad G = [[G^Ep, G^Em], [G^Hp, G^Hm]] that propagates the
  fields of electric (p) and magnetic (m) point dipoles.  The paper defers the
  explicit tensors to its pyGDM reference; here they are the standard
  Gaussian-unit fields of an oscillating point dipole in a non-magnetic host of
  permittivity eps_env (time factor exp(-i w t), outgoing exp(+ikR)), see
  `green_ep` / `green_hp` / `green6`.
* Eq. (LPS_6by6_discrete): F_i = F0_i + sum_j G(r_i, r_j) alpha_j F_j.
* Eq. (GDM_system_of_equations) read as  sum_j [delta_ij I - G_ij alpha_j] F_j = F0_i
  (the printed equation carries a stray F(r_j) inside the bracket; this reading
  is the one consistent with Eq. LPS_6by6_discrete).
* Sec. "Volume discretization polarizabilities": alpha_pE = chi_ee d^3 / (4 pi)
  with chi_ee read as eps - eps_env, and the cubic self-term
  S^Ep = -I 4 pi / (3 eps_env d^3) (Eq. selfterm_SEp_cubic); effective point
  polarisabilities have a zero self-term.
* Sec. "Effective polarizabilities ...": k0 = 2 pi / lambda0, Mie dipole
  polarisabilities alpha_pE = (3i/2) a1 / (k0^3 n_env), alpha_mH = (3i/2) b1 / (k0^3 n_env^3).
* Sec. "Observables": near fields by repropagation of the dipole moments through
  Eq. (LPS_6by6_discrete); extinction / absorption / scattering cross sections
  (the paper cites Markel 2019 for them without printing them; the forms used
  are the standard coupled-dipole ones stated in `cross_sections`).
* Sec. "Numerical solution" / "Automatic differentiation": gradients of a real
  loss through the linear solve by the adjoint method (`loss_and_grad_probe_sca`).

Layout conventions shared with the library's C interface (a contract, not code):
dipole-interleaved unknowns (index k*i + c, k = 3 or 6), plane-wave right-hand
sides stored one column per illumination.
"""
from __future__ import annotations

import numpy as np

FOUR_PI = 4.0 * np.pi


# ----------------------------------------------------------------------------- basics
def wavenumbers(wavelength, eps_env=1.0):
    """k0 = 2 pi / lambda0 (Sec. "Effective polarizabilities ..."); k = n_env k0."""
    k0 = 2.0 * np.pi / float(wavelength)
    return k0, np.sqrt(float(eps_env)) * k0


def cell_polarizability(eps, eps_env, step):
    """alpha_pE = chi_ee d^3 / (4 pi), chi_ee = eps - eps_env (Sec. "Volume discretization polarizabilities")."""
    return (np.asarray(eps, np.complex128) - eps_env) * step ** 3 / FOUR_PI


def cubic_selfterm(eps_env, step):
    """S^Ep = -I 4 pi / (3 eps_env d^3) (Eq. selfterm_SEp_cubic); returned as the scalar factor of I."""
    return -FOUR_PI / (3.0 * eps_env * step ** 3)


def lorentz_alpha6(omega0_e, omega0_m, gamma_ev, amp_nm, wavelength, hc_ev_nm=1239.84198, eps_env=1.0):
    """Effective ED/MD point polarisabilities from Lorentzian lines (Sec. "Effective
    polarizabilities ...": manual Lorentzian lineshapes) in a host of permittivity eps_env.

    alpha0(w) = a^3 w0^2 / (w0^2 - w^2 - i gamma w); dressed with the radiative reaction of the
    host, Im G^Ep(0) = (2/3) k^3/eps_env for the electric and Im G^Hm(0) = (2/3) k^3 for the
    magnetic line (k = n_env k0): alpha_e = 1/(1/alpha0 - i (2/3) k^3/eps_env), alpha_m =
    1/(1/alpha0 - i (2/3) k^3), so that a lone lossless scatterer obeys the optical theorem.
    Returns (n, 6, 6) complex: diag(alpha_e I3, alpha_m I3)."""
    w = hc_ev_nm / float(wavelength)
    k = np.sqrt(float(eps_env)) * 2.0 * np.pi / float(wavelength)
    out = np.zeros((len(omega0_e), 6, 6), np.complex128)
    for blk, w0 in ((0, np.asarray(omega0_e)), (3, np.asarray(omega0_m))):
        a0 = amp_nm ** 3 * w0 ** 2 / (w0 ** 2 - w ** 2 - 1j * gamma_ev * w)
        rr = (2.0 / 3.0) * k ** 3 / (float(eps_env) if blk == 0 else 1.0)
        a = 1.0 / (1.0 / a0 - 1j * rr)
        for c in range(3):
            out[:, blk + c, blk + c] = a
    return out


# ----------------------------------------------------------------------------- Green dyads
def green_ep(R, k, eps_env=1.0):
    """G^Ep(R): electric field at r of an electric point dipole at r' (R = r - r' != 0).

    E = exp(ikR)/eps_env [ (k^2/R + ik/R^2 - 1/R^3) I + (-k^2/R - 3ik/R^2 + 3/R^3) u u^T ] p,
    u = R/|R|: the textbook (Gaussian units) radiating-dipole field, near, intermediate and
    far zone terms. Block G^Ep of Eq. (superprop_G). R: (..., 3) -> (..., 3, 3)."""
    R = np.asarray(R, np.float64)
    r = np.sqrt(np.sum(R * R, axis=-1))
    u = R / r[..., None]
    ph = np.exp(1j * k * r) / eps_env
    a = ph * (k * k / r + 1j * k / r ** 2 - 1.0 / r ** 3)
    b = ph * (-k * k / r - 3j * k / r ** 2 + 3.0 / r ** 3)
    return a[..., None, None] * np.eye(3) + b[..., None, None] * (u[..., :, None] * u[..., None, :])


def cross_matrix(u):
    """[u]_x with [u]_x v = u x v. u: (..., 3) -> (..., 3, 3)."""
    u = np.asarray(u)
    z = np.zeros(u.shape[:-1])
    return np.stack([np.stack([z, -u[..., 2], u[..., 1]], -1),
                     np.stack([u[..., 2], z, -u[..., 0]], -1),
                     np.stack([-u[..., 1], u[..., 0], z], -1)], -2)


def green_hp(R, k0, k):
    """G^Hp(R): magnetic field of an electric point dipole, H = k0 k exp(ikR) (1/R + i/(k R^2)) (u x p).

    Curl of the vector potential A = -i k0 p exp(ikR)/R; block G^Hp of Eq. (superprop_G)."""
    R = np.asarray(R, np.float64)
    r = np.sqrt(np.sum(R * R, axis=-1))
    c = k0 * k * np.exp(1j * k * r) * (1.0 / r + 1j / (k * r * r))
    return c[..., None, None] * cross_matrix(R / r[..., None])


def green6(R, k0, k, eps_env=1.0):
    """Full 6x6 dyad of Eq. (superprop_G) in a non-magnetic host of permittivity eps_env (k = n_env k0).

    The fields of a magnetic dipole follow from those of an electric one by duality: its magnetic field
    is the electric-dipole kernel without the 1/eps_env of G^Ep (the host is non-magnetic), G^Hm =
    eps_env G^Ep, and its electric field is E = (i/(k0 eps_env)) curl H (Ampere, exp(-i w t)), which
    gives G^Em = -G^Hp. In vacuum: G^Hm = G^Ep, G^Em = -G^Hp."""
    gep = green_ep(R, k, eps_env)
    ghp = green_hp(R, k0, k)
    top = np.concatenate([gep, -ghp], -1)
    bot = np.concatenate([ghp, eps_env * gep], -1)
    return np.concatenate([top, bot], -2)


# ----------------------------------------------------------------------------- problem
class Problem:
    """Physics of one (structure, wavelength): positions, polarisabilities, wavenumbers.

    kind 3: discretised cells, isotropic alpha_i = (eps_i - eps_env) d^3/(4 pi), self-term S.
    kind 6: effective point dipoles with full 6x6 alpha_i, zero self-term."""

    def __init__(self, pos, wavelength, kind=3, eps=None, step=0.0, alpha6=None, eps_env=1.0):
        self.pos = np.ascontiguousarray(pos, np.float64)
        self.n = self.pos.shape[0]
        self.kind = int(kind)
        self.wavelength = float(wavelength)
        self.eps_env = float(eps_env)
        self.k0, self.k = wavenumbers(wavelength, eps_env)
        self.step = float(step)
        if self.kind == 3:
            self.eps = np.asarray(eps, np.complex128)
            self.alpha = cell_polarizability(self.eps, self.eps_env, self.step)
            self.selfterm = cubic_selfterm(self.eps_env, self.step)
        elif self.kind == 6:
            self.alpha6 = np.asarray(alpha6, np.complex128).reshape(self.n, 6, 6)
        else:
            raise ValueError("kind must be 3 or 6")

    @property
    def size(self):
        return self.kind * self.n

    # Eq. (LPS_6by6_discrete): the coupling dyads G(r_i, r_j), self-terms on the diagonal
    def coupling_blocks(self, rows=None):
        """(len(rows), n, k, k) blocks G(r_i, r_j); G_ii = S (cells) or 0 (effective dipoles)."""
        rows = np.arange(self.n) if rows is None else np.asarray(rows)
        R = self.pos[rows, None, :] - self.pos[None, :, :]
        same = np.all(R == 0.0, axis=-1)
        Rs = np.where(same[..., None], 1.0, R)
        if self.kind == 3:
            G = green_ep(Rs, self.k, self.eps_env)
            G[same] = self.selfterm * np.eye(3)
        else:
            G = green6(Rs, self.k0, self.k, self.eps_env)
            G[same] = 0.0
        return G

    def alpha_blocks(self):
        if self.kind == 3:
            return self.alpha[:, None, None] * np.eye(3)
        return self.alpha6

    def matrix_blocks(self, rows=None):
        """A_ij = delta_ij I - G_ij alpha_j (Eq. GDM_system_of_equations, reading above)."""
        rows = np.arange(self.n) if rows is None else np.asarray(rows)
        G = self.coupling_blocks(rows)
        Ga = np.einsum("ijab,jbc->ijac", G, self.alpha_blocks())
        A = -Ga
        for t, i in enumerate(rows):
            A[t, i] += np.eye(self.kind)
        return A

    def matrix(self):
        """Dense kN x kN system matrix, dipole-interleaved rows/columns (k*i + c)."""
        A = self.matrix_blocks()
        kk = self.kind
        return A.transpose(0, 2, 1, 3).reshape(self.n * kk, self.n * kk)

    # plane-wave illumination (Sec. "Observables", illumination fields)
    def plane_wave(self, e0, khat=(0.0, 0.0, 1.0), r=None):
        """E0(r) = e0 exp(i k khat.r), H0 = n_env khat x E0. Returns (m*kind_out, n_rhs)
        with kind_out = self.kind (E only for cells, E and H interleaved per point for ED/MD)."""
        return plane_wave(self.pos if r is None else r, self.k, np.sqrt(self.eps_env), e0, khat, self.kind)

    def solve(self, F0):
        """F = A^{-1} F0 (Eq. GDM_system_of_equations; LAPACK zgesv as the solve step)."""
        return np.linalg.solve(self.matrix(), F0)

    def moments(self, F):
        """(p, m)_i = alpha_i F_i (dipole-moment relation). F: (kN, n_rhs) -> same shape."""
        nr = F.shape[1]
        Fi = F.reshape(self.n, self.kind, nr)
        P = np.einsum("iab,ibr->iar", self.alpha_blocks(), Fi)
        return P.reshape(self.n * self.kind, nr)

    def nearfield(self, F, r_eval, e0, khat=(0.0, 0.0, 1.0), with_incident=True):
        """Repropagated fields at r_eval (Sec. "Observables"): E(r) = E0(r) + sum_j [G^Ep p_j + G^Em m_j],
        H(r) = H0(r) + sum_j [G^Hp p_j + G^Hm m_j]. Returns (E, H): each (m, 3, n_rhs)."""
        r_eval = np.asarray(r_eval, np.float64)
        m = r_eval.shape[0]
        nr = F.shape[1]
        P = self.moments(F).reshape(self.n, self.kind, nr)
        R = r_eval[:, None, :] - self.pos[None, :, :]
        if self.kind == 3:
            E = np.einsum("ijab,jbr->iar", green_ep(R, self.k, self.eps_env), P)
            H = np.einsum("ijab,jbr->iar", green_hp(R, self.k0, self.k), P)
        else:
            G6 = green6(R, self.k0, self.k, self.eps_env)
            EH = np.einsum("ijab,jbr->iar", G6, P)
            E, H = EH[:, :3], EH[:, 3:]
        if with_incident:
            inc = plane_wave(r_eval, self.k, np.sqrt(self.eps_env), e0, khat, 6).reshape(m, 6, nr)
            E = E + inc[:, :3]
            H = H + inc[:, 3:]
        return E, H

    def cross_sections(self, F0, F, e0):
        """Extinction, absorption and scattering cross sections (nm^2), one per illumination.

        sigma_ext = 4 pi k / (eps_env |E0|^2) sum_i Im(E0_i^* . p_i + H0_i^* . m_i)
        sigma_abs (cells)   = 4 pi k / (eps_env |E0|^2) sum_i Im(E_i^* . p_i)
        sigma_abs (ED/MD)   = 4 pi k / (eps_env |E0|^2) sum_i [Im(E_i^*.p_i) - 2/3 k^3/eps_env |p_i|^2
                                                           + Im(H_i^*.m_i) - 2/3 k^3 |m_i|^2]
        sigma_sca = sigma_ext - sigma_abs.
        (Standard coupled-dipole forms; the paper cites them, Sec. "Observables". The radiated powers of
        the electric and magnetic dipoles in the host, c k0 k^3 |p|^2/(3 eps_env) and c k0 k^3 |m|^2/3,
        give the two radiation terms; the incident intensity is c n_env |E0|^2/(8 pi).)"""
        e0 = np.atleast_2d(np.asarray(e0, np.complex128))
        e2 = np.sum(np.abs(e0) ** 2, axis=1)
        P = self.moments(F)
        pref = FOUR_PI * self.k / (self.eps_env * e2)
        ext = pref * np.sum(np.imag(np.conj(F0) * P), axis=0)
        ab = np.sum(np.imag(np.conj(F) * P), axis=0)
        if self.kind == 6:
            Pi = P.reshape(self.n, 6, -1)
            ab = ab - (2.0 / 3.0) * self.k ** 3 * (np.sum(np.abs(Pi[:, :3]) ** 2, axis=(0, 1)) / self.eps_env
                                                   + np.sum(np.abs(Pi[:, 3:]) ** 2, axis=(0, 1)))
        ab = pref * ab
        return ext, ext - ab, ab

    def farfield_amplitude(self, F, dirs):
        """Far-field amplitude f(rhat) at unit directions dirs (q, 3) (Sec. "Observables", repropagation to
        infinity): the scattered field along rhat is f exp(ikr)/r, f = k^2/eps_env sum_j exp(-ik rhat.r_j)
        [p_j - rhat (rhat.p_j) - n_env rhat x m_j] (far zone of G^Ep and of G^Em = -G^Hp, k0 k = k^2/n_env).
        Returns (q, 3, n_rhs)."""
        rh = np.asarray(dirs, np.float64)
        nr = F.shape[1]
        P = self.moments(F).reshape(self.n, self.kind, nr)
        phase = np.exp(-1j * self.k * (rh @ self.pos.T))
        p = np.einsum("qj,jar->qar", phase, P[:, :3])
        f = p - rh[:, :, None] * np.einsum("qa,qar->qr", rh, p)[:, None, :]
        if self.kind == 6:
            mm = np.einsum("qj,jar->qar", phase, P[:, 3:])
            f = f - np.sqrt(self.eps_env) * np.cross(rh[:, :, None], mm, axisa=1, axisb=1, axisc=1)
        return f * self.k ** 2 / self.eps_env

    def farfield_scattering(self, F, e0, n_theta=64, n_phi=128):
        """sigma_sca by integrating the far-field intensity over the unit sphere
        (Sec. "Observables", scattered intensity via repropagation). Gauss-Legendre in
        cos(theta) times uniform phi. Far field: f(rhat) = k^2/eps_env sum_j exp(-ik rhat.r_j)
        [p_j - rhat (rhat.p_j) - n_env rhat x m_j]; the scattered intensity c n_env |f|^2/(8 pi r^2) over
        the incident c n_env |E0|^2/(8 pi)."""
        e0 = np.atleast_2d(np.asarray(e0, np.complex128))
        e2 = np.sum(np.abs(e0) ** 2, axis=1)
        x, w = np.polynomial.legendre.leggauss(n_theta)
        phi = np.arange(n_phi) * (2 * np.pi / n_phi)
        ct = np.repeat(x, n_phi)
        wt = np.repeat(w, n_phi) * (2 * np.pi / n_phi)
        st = np.sqrt(1 - ct ** 2)
        ph = np.tile(phi, n_theta)
        rh = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1)     # (q, 3)
        nr = F.shape[1]
        P = self.moments(F).reshape(self.n, self.kind, nr)
        phase = np.exp(-1j * self.k * (rh @ self.pos.T))                # (q, n)
        p = np.einsum("qj,jar->qar", phase, P[:, :3])
        f = p - rh[:, :, None] * np.einsum("qa,qar->qr", rh, p)[:, None, :]
        if self.kind == 6:
            mm = np.einsum("qj,jar->qar", phase, P[:, 3:])
            f = f - np.sqrt(self.eps_env) * np.cross(rh[:, :, None], mm, axisa=1, axisb=1, axisc=1)
        f = f * self.k ** 2 / self.eps_env
        return np.einsum("q,qr->r", wt, np.sum(np.abs(f) ** 2, axis=1)) / e2


def plane_wave(r, k, n_env, e0, khat, kind_out):
    """Plane wave E0 = e0 exp(i k khat.r), H0 = n_env khat x E0 at points r.
    Returns (m*kind_out, n_rhs): per point 3 (E) or 6 (E, H) components."""
    r = np.asarray(r, np.float64)
    e0 = np.atleast_2d(np.asarray(e0, np.complex128))
    khat = np.asarray(khat, np.float64)
    ph = np.exp(1j * k * (r @ khat))                          # (m,)
    E = ph[:, None, None] * e0.T[None, :, :]                  # (m, 3, n_rhs)
    if kind_out == 3:
        return E.reshape(-1, e0.shape[0])
    H = n_env * np.cross(khat[None, :, None], E, axisa=1, axisb=1, axisc=1)
    return np.concatenate([E, H], axis=1).reshape(-1, e0.shape[0])


def gaussian_paraxial(r, k, n_env, e0, w0, focus=(0.0, 0.0, 0.0), theta=0.0, kind_out=3):
    """Paraxial focused Gaussian beam (Sec. "Illuminations": GaussianParaxial, after the cited nano-optics
    textbook), with the longitudinal field from the divergence condition (the paper's correction for tight
    focus). Beam frame: propagation along z', focus at `focus`, incidence angle theta in the XZ plane
    (z' = (sin theta, 0, cos theta) in the lab). With z0 = k w0^2 / 2 and g = 1 + i z'/z0:
      E_t  = e0 exp(i k z') exp(-(x'^2 + y'^2) / (w0^2 g)) / g          (e0 transverse: x', y' components)
      E_z' = (i/k) (dE_x'/dx' + dE_y'/dy'),  H_t = n_env z' x E_t,  H_z' = (i/k) (dH_x'/dx' + dH_y'/dy').
    e0: (n_rhs, 3) complex in the beam frame (z' component ignored). Returns (m kind_out, n_rhs)."""
    r = np.asarray(r, np.float64) - np.asarray(focus, np.float64)
    e0 = np.atleast_2d(np.asarray(e0, np.complex128))
    ct, st = np.cos(theta), np.sin(theta)
    ex, ey, ez = np.array([ct, 0.0, -st]), np.array([0.0, 1.0, 0.0]), np.array([st, 0.0, ct])
    xp, yp, zp = r @ ex, r @ ey, r @ ez
    z0 = k * w0 * w0 / 2.0
    g = 1.0 + 1j * zp / z0
    u = np.exp(1j * k * zp) * np.exp(-(xp * xp + yp * yp) / (w0 * w0 * g)) / g      # (m,)
    d = -2.0 / (w0 * w0 * g)                                                         # d/dx' of the envelope: d x' u
    out = []
    for q in range(e0.shape[0]):
        a, b = e0[q, 0], e0[q, 1]
        Ex, Ey = a * u, b * u
        Ez = (1j / k) * d * (xp * a + yp * b) * u
        Hx, Hy = -n_env * b * u, n_env * a * u
        Hz = (1j / k) * d * (xp * (-n_env * b) + yp * (n_env * a)) * u
        E = Ex[:, None] * ex + Ey[:, None] * ey + Ez[:, None] * ez
        H = Hx[:, None] * ex + Hy[:, None] * ey + Hz[:, None] * ez
        out.append(np.concatenate([E, H], 1) if kind_out == 6 else E)
    return np.stack(out, -1).reshape(-1, e0.shape[0])


# ----------------------------------------------------------------------------- sampled forms
def residual_rows(prob: Problem, F0, F, rows):
    """r_i = F0_i - sum_j A_ij F_j for the dipoles in `rows` (O(N) per row): the
    definition of the linear system, evaluated one row at a time for large N."""
    rows = np.asarray(rows)
    A = prob.matrix_blocks(rows)                       # (r, n, k, k)
    nr = F.shape[1]
    Fi = F.reshape(prob.n, prob.kind, nr)
    AF = np.einsum("ijab,jbr->iar", A, Fi)
    F0i = F0.reshape(prob.n, prob.kind, nr)[rows]
    return F0i - AF


# ----------------------------------------------------------------------------- gradients
def _dgreen_ep(R, k, eps_env=1.0):
    """Derivatives of G^Ep: returns (G, dG/dR_c for c=0..2 stacked on axis -3, dG/dk)."""
    R = np.asarray(R, np.float64)
    r = np.sqrt(np.sum(R * R, axis=-1))
    u = R / r[..., None]
    e = np.exp(1j * k * r) / eps_env
    a = e * (k * k / r + 1j * k / r ** 2 - 1.0 / r ** 3)
    b = e * (-k * k / r - 3j * k / r ** 2 + 3.0 / r ** 3)
    da = 1j * k * a + e * (-k * k / r ** 2 - 2j * k / r ** 3 + 3.0 / r ** 4)
    db = 1j * k * b + e * (k * k / r ** 2 + 6j * k / r ** 3 - 9.0 / r ** 4)
    dka = 1j * r * a + e * (2 * k / r + 1j / r ** 2)
    dkb = 1j * r * b + e * (-2 * k / r - 3j / r ** 2)
    I3 = np.eye(3)
    uu = u[..., :, None] * u[..., None, :]
    G = a[..., None, None] * I3 + b[..., None, None] * uu
    dG = []
    for c in range(3):
        du = (I3[c] - u[..., c:c + 1] * u) / r[..., None]          # d u / d R_c
        duu = du[..., :, None] * u[..., None, :] + u[..., :, None] * du[..., None, :]
        dG.append((da * u[..., c])[..., None, None] * I3 + (db * u[..., c])[..., None, None] * uu
                  + b[..., None, None] * duu)
    dGk = dka[..., None, None] * I3 + dkb[..., None, None] * uu
    return G, np.stack(dG, axis=-3), dGk


def probe_sca_loss(prob: Problem, e0, r_probe, khat=(0.0, 0.0, 1.0)):
    """Loss of one wavelength: L = |E_tot(r_probe)|^2 + sum over illuminations of sigma_sca
    (cells, kind 3). Forward only (used for finite differences)."""
    F0 = prob.plane_wave(e0, khat)
    F = prob.solve(F0)
    E, _ = prob.nearfield(F, np.atleast_2d(r_probe), e0, khat)
    ext, sca, ab = prob.cross_sections(F0, F, e0)
    return float(np.sum(np.abs(E) ** 2) + np.sum(sca))


def loss_and_grad_probe_sca(prob: Problem, e0, r_probe, khat=(0.0, 0.0, 1.0)):
    """Adjoint gradient of `probe_sca_loss` (kind 3) w.r.t. cell positions (n, 3),
    cell permittivities (n, complex; dL/dRe eps + i dL/dIm eps) and the vacuum wavelength.

    With A F = F0 and g = dL/dF* (conjugate Wirtinger derivative), solve A^H mu = g;
    then dL = 2 Re[mu^H (dF0 - dA F)] + explicit terms (Sec. "Numerical solution": the
    derivative of the LU-solved system)."""
    assert prob.kind == 3
    e0 = np.atleast_2d(np.asarray(e0, np.complex128))
    khat = np.asarray(khat, np.float64)
    n, nr, k = prob.n, e0.shape[0], prob.k
    rp = np.asarray(r_probe, np.float64).reshape(3)
    F0 = prob.plane_wave(e0, khat)
    A = prob.matrix()
    F = np.linalg.solve(A, F0)
    P = prob.moments(F)
    al = prob.alpha
    e2 = np.sum(np.abs(e0) ** 2, axis=1)
    c = FOUR_PI * k / (prob.eps_env * e2)                           # (nr,)
    # forward observables
    Rp = rp[None, :] - prob.pos                                      # (n, 3)
    Gp, dGp, dGpk = _dgreen_ep(Rp, k, prob.eps_env)                  # (n,3,3), (n,3,3,3), (n,3,3)
    E0p = plane_wave(rp[None, :], k, np.sqrt(prob.eps_env), e0, khat, 3)   # (3, nr)
    Pi = P.reshape(n, 3, nr)
    Fi = F.reshape(n, 3, nr)
    F0i = F0.reshape(n, 3, nr)
    Ep = E0p + np.einsum("jab,jbr->ar", Gp, Pi)                      # (3, nr)
    ext = c * np.sum(np.imag(np.conj(F0) * P), axis=0)
    ab = c * np.sum(np.imag(np.conj(F) * P), axis=0)
    L = float(np.sum(np.abs(Ep) ** 2) + np.sum(ext - ab))
    # g = dL/dF*
    g = np.einsum("jba,br->jar", np.conj(Gp), Ep) * np.conj(al)[:, None, None]      # probe
    g = g + (0.5j * c)[None, None, :] * np.conj(al)[:, None, None] * F0i             # sigma_ext
    g = g - c[None, None, :] * np.imag(al)[:, None, None] * Fi                        # -sigma_abs
    mu = np.linalg.solve(A.conj().T, g.reshape(3 * n, nr))
    mub = np.conj(mu).reshape(n, 3, nr)
    # pair sums (i != j) of dG/dR and dG/dk; G mu-bar including the self-term
    R = prob.pos[:, None, :] - prob.pos[None, :, :]
    same = np.all(R == 0.0, axis=-1)
    Rs = np.where(same[..., None], 1.0, R)
    G, dG, dGk = _dgreen_ep(Rs, k, prob.eps_env)
    G[same] = prob.selfterm * np.eye(3)
    dG[same] = 0.0
    dGk[same] = 0.0
    Gmu = np.einsum("ijab,jbr->iar", G, mub)
    dGP = np.einsum("ijcab,jbr->icar", dG, Pi)                       # (n, 3c, 3a, nr)
    dGmu = np.einsum("ijcab,jbr->icar", dG, mub)
    dGkP = np.einsum("ijab,jbr->iar", dGk, Pi)
    # --- permittivity: dL = Re(C_j dalpha_j), dalpha = d^3/(4pi) deps
    C = 2.0 * np.einsum("jar,jar->j", Fi, Gmu)
    C = C + 2.0 * np.einsum("ar,jab,jbr->j", np.conj(Ep), Gp, Fi)
    C = C - 1j * np.einsum("r,jar,jar->j", c, np.conj(F0i), Fi)
    C = C + 1j * np.einsum("r,jar->j", c, np.abs(Fi) ** 2)
    grad_eps = np.conj(C * prob.step ** 3 / FOUR_PI)
    # --- positions
    gpos = 2.0 * np.real(np.einsum("lar,lcar->lc", mub, dGP) + np.einsum("lar,lcar->lc", Pi, dGmu))
    gpos += 2.0 * np.real(np.einsum("lar,c,lar->lc", mub, 1j * k * khat, F0i))            # dF0/dr
    gpos += -2.0 * np.real(np.einsum("ar,lcab,lbr->lc", np.conj(Ep), dGp, Pi))          # probe, via r_l
    # sigma_ext explicit: c * Im(dE0_l^H p_l), dE0_l/dr_c = i k khat_c E0_l
    gpos += np.einsum("r,lcr->lc", c,
                      np.imag(np.einsum("c,lar,lar->lcr", -1j * k * khat, np.conj(F0i), Pi)))
    # --- wavenumber (then wavelength)
    zdot = (prob.pos @ khat)                                                              # (n,)
    dF0k = 1j * zdot[:, None, None] * F0i
    dLdk = 2.0 * np.real(np.einsum("jar,jar->", mub, dF0k))
    dLdk += 2.0 * np.real(np.einsum("jar,jar->", mub, dGkP))
    dE0pk = 1j * float(rp @ khat) * E0p
    dEpk = dE0pk + np.einsum("jab,jbr->ar", dGpk, Pi)
    dLdk += 2.0 * np.real(np.sum(np.conj(Ep) * dEpk))
    dLdk += float(np.sum((ext - ab) / k))
    dLdk += float(np.sum(c * np.sum(np.imag(np.conj(dF0k) * Pi), axis=(0, 1))))
    dkdlam = -k / prob.wavelength
    return L, gpos, grad_eps, dLdk * dkdlam


# ----------------------------------------------------------------------------- effective models (GPM)
def dipole_source_fields(r_eval, r_src, moments, k0, k, eps_env=1.0):
    """Fields of local point-dipole sources in the host, used as illuminations for the effective-model
    extraction (Sec. "Effective polarizabilities ..."): [E; H](r) = G6(r - r_s) [p_s; m_s] with the 6x6
    dyad of Eq. (superprop_G). r_src (s, 3), moments (s, 6) complex. Returns (6 m, s): column q holds the
    (E, H) of source q at every point."""
    r_eval = np.asarray(r_eval, np.float64)
    R = r_eval[:, None, :] - np.asarray(r_src, np.float64)[None, :, :]
    EH = np.einsum("iqab,qb->iaq", green6(R, k0, k, eps_env), np.asarray(moments, np.complex128))
    return EH.reshape(-1, len(r_src))


def dipole_illumination(prob: Problem, r_eval, src_pos, src_mom, kind_out=3):
    """Incident field of point-dipole sources (Sec. "Illuminations": electric and magnetic dipole sources)
    in the problem's host: column q = fields of source q at r_eval, (kind_out m, n_src)."""
    EH = dipole_source_fields(r_eval, src_pos, src_mom, prob.k0, prob.k, prob.eps_env)
    m = len(r_eval)
    if kind_out == 6:
        return EH
    return EH.reshape(m, 6, -1)[:, :3].reshape(3 * m, -1)


def ldos(prob: Problem, r0, magnetic=False):
    """Partial local density of states of the structured environment, normalised to the bare host (Sec.
    "Observables": electric and magnetic LDOS): for a unit dipole u (x, y, z) at r0, the structure is solved
    under its field and the emitter's decay rate relative to the homogeneous host is its total emitted power
    over the host's, (w/2) Im(u . E_sca(r0)) over c k0 k^3/(3 eps_env):
    rho_u / rho_0 = 1 + 3 eps_env/(2 k^3) Im(u . E_sca(r0)), and for a magnetic emitter (host power
    c k0 k^3/3) rho_u / rho_0 = 1 + 3/(2 k^3) Im(u . H_sca(r0)). Cells. Returns (n_pos, 3)."""
    assert prob.kind == 3
    r0 = np.asarray(r0, np.float64)
    out = np.zeros((len(r0), 3))
    for e, r in enumerate(r0):
        mom = np.zeros((3, 6), np.complex128)
        for u in range(3):
            mom[u, u + (3 if magnetic else 0)] = 1.0
        F0 = dipole_illumination(prob, prob.pos, np.repeat(r[None], 3, 0), mom, 3)
        F = prob.solve(F0)
        E, H = prob.nearfield(F, r[None], None, with_incident=False)
        field = H if magnetic else E
        for u in range(3):
            out[e, u] = 1.0 + 1.5 * (1.0 if magnetic else prob.eps_env) / prob.k ** 3 * field[0, u, u].imag
    return out


def gpm_illuminations(prob: Problem, r_eval, pw_khat, pw_e0, ds_pos, ds_mom):
    """The extraction's illumination set at r_eval: plane waves (one per (khat, e0) pair, unit-free
    amplitudes e0), then local dipole sources. Returns (6 m, n_ill) incident (E, H) per point."""
    cols = [plane_wave(r_eval, prob.k, np.sqrt(prob.eps_env), e0, kh, 6) for kh, e0 in zip(pw_khat, pw_e0)]
    if len(ds_pos):
        cols.append(dipole_source_fields(r_eval, ds_pos, ds_mom, prob.k0, prob.k, prob.eps_env))
    return np.concatenate(cols, axis=1)


def gpm_extract(prob: Problem, r_gpm, r_probe, pw_khat, pw_e0, ds_pos, ds_mom):
    """Global polarizability matrix of a discretised structure (Sec. "Effective polarizabilities",
    GPM extraction), in the paper's order:
      1. full simulations of the structure for every illumination of the set;
      2. its scattered fields (E, H) at the probe positions;
      3. the effective electric and magnetic dipole moments at the M positions r_gpm that reproduce
         those fields best in the L2 sense (least squares through the 6x6 dyads);
      4. alpha_eff (6M x 6M) minimising || alpha_eff F0 - P || over the illuminations, F0 the incident
         (E, H) at the M positions and P the fitted moments: alpha_eff = P F0^+.
    The 6x6 dyads are those of the problem's host. LAPACK least squares (numpy lstsq) as the
    library step. Returns (alpha_eff, P, F0g, rel_fit) with rel_fit the relative residual of step 3."""
    assert prob.kind == 3
    n = prob.n
    F0c = gpm_illuminations(prob, prob.pos, pw_khat, pw_e0, ds_pos, ds_mom)
    nill = F0c.shape[1]
    F0c = F0c.reshape(n, 6, nill)[:, :3].reshape(3 * n, nill)
    F = prob.solve(F0c)
    E, H = prob.nearfield(F, r_probe, None, with_incident=False)
    S = np.concatenate([E, H], axis=1).reshape(-1, nill)
    R = np.asarray(r_probe, np.float64)[:, None, :] - np.asarray(r_gpm, np.float64)[None, :, :]
    G6 = green6(R, prob.k0, prob.k, prob.eps_env)                     # (P, M, 6, 6)
    Gp = G6.transpose(0, 2, 1, 3).reshape(6 * len(r_probe), 6 * len(r_gpm))
    P = np.linalg.lstsq(Gp, S, rcond=None)[0]
    rel_fit = np.linalg.norm(Gp @ P - S) / np.linalg.norm(S)
    F0g = gpm_illuminations(prob, r_gpm, pw_khat, pw_e0, ds_pos, ds_mom)
    alpha_t = np.linalg.lstsq(F0g.T, P.T, rcond=None)[0]
    return alpha_t.T, P, F0g, rel_fit


# ----------------------------------------------------------------------------- Mie theory
def mie_coefficients(m, x, n_max=None):
    """Bohren & Huffman sphere coefficients a_n, b_n (n = 1..n_max) for relative index m
    and size parameter x = k a, with Riccati-Bessel functions psi_n(z) = z j_n(z),
    xi_n(z) = z h_n^(1)(z) (scipy spherical Bessel functions as the library step)."""
    from scipy.special import spherical_jn, spherical_yn
    if n_max is None:
        n_max = int(np.ceil(x + 4.05 * x ** (1 / 3) + 2))
    n = np.arange(1, n_max + 1)
    mx = m * x

    def psi(z):
        return z * spherical_jn(n, z)

    def dpsi(z):
        return spherical_jn(n, z) + z * spherical_jn(n, z, derivative=True)

    def xi(z):
        return z * (spherical_jn(n, z) + 1j * spherical_yn(n, z))

    def dxi(z):
        return (spherical_jn(n, z) + 1j * spherical_yn(n, z)) + z * (
            spherical_jn(n, z, derivative=True) + 1j * spherical_yn(n, z, derivative=True))

    a = (m * psi(mx) * dpsi(x) - psi(x) * dpsi(mx)) / (m * psi(mx) * dxi(x) - xi(x) * dpsi(mx))
    b = (psi(mx) * dpsi(x) - m * psi(x) * dpsi(mx)) / (psi(mx) * dxi(x) - m * xi(x) * dpsi(mx))
    return a, b


def mie_cross_sections(radius, eps_sphere, wavelength, eps_env=1.0):
    """sigma_ext, sigma_sca (nm^2) of a homogeneous sphere (Bohren & Huffman series)."""
    n_env = np.sqrt(eps_env)
    k = 2 * np.pi * n_env / wavelength
    m = np.sqrt(complex(eps_sphere)) / n_env
    x = k * radius
    a, b = mie_coefficients(m, x)
    nn = np.arange(1, len(a) + 1)
    qe = 2.0 / x ** 2 * np.sum((2 * nn + 1) * np.real(a + b))
    qs = 2.0 / x ** 2 * np.sum((2 * nn + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    area = np.pi * radius ** 2
    return qe * area, qs * area


def mie_dipole_alpha(radius, eps_sphere, wavelength, eps_env=1.0):
    """alpha_pE = (3i/2) a1 / (k0^3 n_env), alpha_mH = (3i/2) b1 / (k0^3 n_env^3)
    (Sec. "Effective polarizabilities of spherical ... particles", 3D case)."""
    n_env = np.sqrt(eps_env)
    k0 = 2 * np.pi / wavelength
    m = np.sqrt(complex(eps_sphere)) / n_env
    a, b = mie_coefficients(m, k0 * n_env * radius)
    return 1.5j * a[0] / (k0 ** 3 * n_env), 1.5j * b[0] / (k0 ** 3 * n_env ** 3)
