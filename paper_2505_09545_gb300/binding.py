"""Thin ctypes binding of the GDM C ABI (include/gdm.h).

Argument marshalling only: every step of the hot path runs in the CUDA library.
PyTorch provides device memory and the current CUDA stream. The functions keep
the C names (without the ``gdm_`` prefix) and raise ``GDMError`` on a non-OK status.

Tensor layouts (column-major C arrays seen from torch):
* fields / right-hand sides: torch tensor (n_rhs, kind*m) complex128 -- row q is
  column q of the C array;
* system matrix: torch tensor (n_cols, lda) complex64/complex128 -- row j is column j.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

from . import _build

GDM_OK = 0
STATUS = {0: "GDM_OK", 1: "GDM_ERR_INVALID_ARG", 2: "GDM_ERR_SHAPE", 3: "GDM_ERR_NONFINITE", 4: "GDM_ERR_SINGULAR",
          5: "GDM_ERR_NOT_CONVERGED", 6: "GDM_ERR_OOM", 7: "GDM_ERR_CUDA", 8: "GDM_ERR_TIMEOUT",
          9: "GDM_ERR_UNSUPPORTED"}
PRECISION = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
SOLVE_FACTORED = 1
SOLVE_NO_REFINE = 2
SOLVE_GLOBAL_PIVOT = 4
SOLVE_ERR_ESTIMATE = 8


class GDMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Problem(C.Structure):
    _fields_ = [("n", C.c_int64), ("kind", C.c_int32), ("reserved", C.c_int32), ("pos", C.c_void_p),
                ("eps", C.c_void_p), ("alpha6", C.c_void_p), ("step", C.c_double), ("eps_env", C.c_double),
                ("wavelength", C.c_double)]


class BackwardItem(C.Structure):
    _fields_ = [("prob", Problem), ("A", C.c_void_p), ("lda", C.c_int64), ("ipiv", C.c_void_p), ("F", C.c_void_p),
                ("gF", C.c_void_p), ("g_sigma", C.c_void_p), ("e0", C.c_void_p), ("khat", C.c_void_p),
                ("grad_wavelength", C.c_void_p), ("n_rhs", C.c_int32), ("reserved", C.c_int32)]


class BatchItem(C.Structure):
    _fields_ = [("prob", Problem), ("A", C.c_void_p), ("lda", C.c_int64), ("ipiv", C.c_void_p), ("F0", C.c_void_p),
                ("F", C.c_void_p), ("sigma", C.c_void_p), ("e0", C.c_void_p), ("khat", C.c_void_p),
                ("e0_norm2", C.c_void_p), ("n_rhs", C.c_int32), ("reserved", C.c_int32)]


class SolveOpts(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("flags", C.c_int32), ("tol", C.c_double)]


class GmresOpts(C.Structure):
    _fields_ = [("restart", C.c_int32), ("max_iter", C.c_int32), ("tol", C.c_double), ("block_cells", C.c_int32),
                ("flags", C.c_int32)]


GMRES_NO_COARSE = 1
GMRES_NO_BLOCKS = 2
GMRES_EXACT_OPERATOR = 4


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("status", C.c_int32), ("rel_correction", C.c_double),
                ("rel_residual", C.c_double), ("factor_ms", C.c_double), ("refine_ms", C.c_double),
                ("pivot_growth", C.c_double), ("refactored", C.c_int32), ("cycles", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_lock = threading.Lock()
P = C.c_void_p
I64 = C.c_int64
D = C.c_double
PD = C.POINTER(C.c_double)
_SIGS = {
    "gdm_create": ([C.POINTER(C.c_void_p), C.c_int, P], C.c_int),
    "gdm_destroy": ([P], C.c_int),
    "gdm_set_stream": ([P, P], C.c_int),
    "gdm_ctx_check": ([P], C.c_int),
    "gdm_status_string": ([C.c_int], C.c_char_p),
    "gdm_last_error": ([P], C.c_char_p),
    "gdm_launch_count": ([P], I64),
    "gdm_workspace_size": ([C.POINTER(Problem), C.c_int, C.c_int, C.POINTER(C.c_size_t)], C.c_int),
    "gdm_refine_stop_measure": ([C.c_double, C.c_double, C.c_int32], C.c_double),
    "gdm_incident_planewave": ([P, P, I64, D, D, PD, PD, C.c_int, C.c_int, P], C.c_int),
    "gdm_assemble": ([P, C.POINTER(Problem), C.c_int, P, I64], C.c_int),
    "gdm_solve": ([P, C.POINTER(Problem), C.c_int, P, I64, P, P, P, C.c_int, C.POINTER(SolveOpts),
                   C.POINTER(SolveInfo)], C.c_int),
    "gdm_nearfield": ([P, C.POINTER(Problem), P, P, I64, P, C.c_int, P, P], C.c_int),
    "gdm_residual": ([P, C.POINTER(Problem), P, P, C.c_int, P, P], C.c_int),
    "gdm_cross_sections": ([P, C.POINTER(Problem), P, P, C.c_int, PD, P, P, P], C.c_int),
    "gdm_alpha6_lorentz": ([P, I64, P, P, C.c_double, C.c_double, C.c_double, C.c_double, P], C.c_int),
    "gdm_solve_batched": ([P, C.c_int, P, C.c_int, P, C.c_int, P], C.c_int),
    "gdm_autotune": ([P, C.c_int, P, C.c_int, P], C.c_int),
    "gdm_autotune_batched": ([P, P, C.c_int, P], C.c_int),
    "gdm_diag_wait_timeout": ([P, C.c_double], C.c_int),
    "gdm_incident_gaussian": ([P, P, I64, C.c_double, C.c_double, PD, C.c_double, PD, C.c_double, C.c_int, C.c_int,
                               P], C.c_int),
    "gdm_incident_dipole": ([P, P, I64, C.c_double, C.c_double, P, P, C.c_int, C.c_int, P], C.c_int),
    "gdm_ldos": ([P, C.c_int, C.POINTER(Problem), P, I64, P, P, C.c_int, C.c_int, P], C.c_int),
    "gdm_farfield": ([P, C.POINTER(Problem), P, C.c_int, P, I64, P], C.c_int),
    "gdm_sigma_farfield": ([P, C.POINTER(Problem), P, C.c_int, PD, C.c_int, C.c_int, P], C.c_int),
    "gdm_gpm_extract": ([P, C.c_int, C.POINTER(Problem), P, I64, P, P, C.c_int, P, C.c_int, C.c_int, P, P, C.c_int,
                         P, P, P, P, PD], C.c_int),
    "gdm_backward_batched": ([P, C.c_int, P, C.c_int, C.c_int, P, P, P], C.c_int),
    "gdm_cross_sections_noalloc": ([P, C.POINTER(Problem), P, P, C.c_int, PD, P, P, P], C.c_int),
    "gdm_backward": ([P, C.POINTER(Problem), C.c_int, P, I64, P, P, C.c_int, PD, PD, P, PD, P, P, P,
                      C.POINTER(SolveInfo)], C.c_int),
    "gdm_nearfield_backward": ([P, C.POINTER(Problem), P, P, I64, C.c_int, PD, PD, P, P, P, P, P], C.c_int),
    "gdm_solve_gmres": ([P, C.c_int, C.POINTER(Problem), P, P, C.c_int, C.POINTER(GmresOpts),
                         C.POINTER(SolveInfo)], C.c_int),
    "gdm_lattice_partition": ([P, I64, C.c_double, C.c_int, P, P, P, C.POINTER(I64)], C.c_int),
    "gdm_profile_enable": ([P, C.c_int], C.c_int),
    "gdm_profile_read": ([P, C.POINTER(I64), PD, PD, PD], C.c_int),
    "gdm_profile_phases": ([P, C.c_int, PD], C.c_int),
}
PHASES = ["panel", "laswp", "trsm_small", "inblock_update", "u12_update", "trailing_update", "correction_solves",
          "residual", "other", "operator_f32", "gradient"]


def lib():
    """Load libgdm.so (building it first if the sources are newer). Raises if it cannot be loaded:
    there is no fallback path."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not _build.up_to_date():
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"GDM CUDA library missing at {path}")
            L = C.CDLL(path)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _ptr(t):
    return C.c_void_p(0) if t is None else C.c_void_p(t.data_ptr())


def _dbl_array(x):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a, a.ctypes.data_as(PD)


class Context:
    """A library context bound to one CUDA device; calls run on torch's current stream."""

    def __init__(self, device=None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = lib().gdm_create(C.byref(h), self.device.index or 0,
                                  C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))
        if st != GDM_OK:
            raise GDMError(st, "gdm_create failed")
        self.h = h

    def _sync_stream(self):
        lib().gdm_set_stream(self.h, C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))

    def _check(self, st, what):
        if st != GDM_OK:
            raise GDMError(st, f"{what}: {lib().gdm_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            lib().gdm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self):
        """Synchronise and raise on device-side errors recorded since the last check."""
        self._check(lib().gdm_ctx_check(self.h), "device check")

    @property
    def launches(self):
        return int(lib().gdm_launch_count(self.h))

    def profile(self, enable=True):
        """Start (or stop) CUDA-event timing of the LU trailing-update kernel launches."""
        self._check(lib().gdm_profile_enable(self.h, 1 if enable else 0), "gdm_profile_enable")

    def phases(self, enable=True):
        """Read (and reset) the per-phase device times, then enable/disable phase accounting."""
        out = (C.c_double * len(PHASES))()
        self._check(lib().gdm_profile_phases(self.h, 1 if enable else 0, out), "gdm_profile_phases")
        return {k: out[i] for i, k in enumerate(PHASES)}

    def profile_read(self):
        n = I64(0)
        ms, fl, by = D(0), D(0), D(0)
        self._check(lib().gdm_profile_read(self.h, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)),
                    "gdm_profile_read")
        return {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}


class GDMProblem:
    """Device-resident description of one problem (keeps its tensors alive)."""

    def __init__(self, pos, wavelength, kind=3, eps=None, step=0.0, alpha6=None, eps_env=1.0):
        self.pos = pos.contiguous()
        assert self.pos.dtype == torch.float64 and self.pos.is_cuda and self.pos.shape[-1] == 3
        self.kind = int(kind)
        self.eps = None if eps is None else eps.contiguous()
        self.alpha6 = None if alpha6 is None else alpha6.contiguous()
        if self.eps is not None:
            assert self.eps.dtype == torch.complex128 and self.eps.is_cuda
        if self.alpha6 is not None:
            assert self.alpha6.dtype == torch.complex128 and self.alpha6.is_cuda
        self.step = float(step)
        self.eps_env = float(eps_env)
        self.wavelength = float(wavelength)
        self.n = int(self.pos.shape[0])

    @property
    def size(self):
        return self.kind * self.n

    def struct(self):
        return Problem(self.n, self.kind, 0, self.pos.data_ptr(), 0 if self.eps is None else self.eps.data_ptr(),
                       0 if self.alpha6 is None else self.alpha6.data_ptr(), self.step, self.eps_env,
                       self.wavelength)


def padded_lda(n_sys):
    return (n_sys + 31) // 32 * 32


def alpha6_lorentz(ctx: Context, omega0_e, omega0_m, gamma_ev, amp_nm, wavelength, out=None, eps_env=1.0):
    """Lorentzian ED/MD polarisabilities on the GPU, dressed for a host of permittivity eps_env:
    (n, 6, 6) complex128 device tensor."""
    w0e = omega0_e.contiguous()
    w0m = omega0_m.contiguous()
    n = w0e.shape[0]
    if out is None:
        out = torch.empty((n, 6, 6), dtype=torch.complex128, device=w0e.device)
    ctx._sync_stream()
    ctx._check(lib().gdm_alpha6_lorentz(ctx.h, n, _ptr(w0e), _ptr(w0m), float(gamma_ev), float(amp_nm),
                                        float(wavelength), float(eps_env), _ptr(out)), "gdm_alpha6_lorentz")
    return out


def incident_planewave(ctx: Context, r, wavelength, e0, khat=(0.0, 0.0, 1.0), eps_env=1.0, kind_out=3):
    """F0 at points r (device (m,3) f64): returns (n_rhs, kind_out*m) complex128."""
    e0 = np.atleast_2d(np.asarray(e0, np.complex128))
    n_rhs = e0.shape[0]
    ea, ep = _dbl_array(e0.view(np.float64).reshape(-1))
    ka, kp = _dbl_array(khat)
    r = r.contiguous()
    out = torch.empty((n_rhs, kind_out * r.shape[0]), dtype=torch.complex128, device=r.device)
    ctx._sync_stream()
    ctx._check(lib().gdm_incident_planewave(ctx.h, _ptr(r), r.shape[0], float(wavelength), float(eps_env), ep, kp,
                                            n_rhs, kind_out, _ptr(out)), "gdm_incident_planewave")
    return out


def assemble(ctx: Context, prob: GDMProblem, precision="fp32", lda=None, out=None):
    """A = I - G alpha, column-major: returns torch (n_sys, lda) complex64 (complex128 for fp64)."""
    ns = prob.size
    lda = padded_lda(ns) if lda is None else lda
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    if out is None:
        out = torch.empty((ns, lda), dtype=dt, device=prob.pos.device)
    s = prob.struct()
    ctx._sync_stream()
    ctx._check(lib().gdm_assemble(ctx.h, C.byref(s), PRECISION[precision], _ptr(out), lda), "gdm_assemble")
    return out


def solve(ctx: Context, prob: GDMProblem, A, F0, precision="fp32", ipiv=None, factored=False, max_iter=0, tol=0.0,
          no_refine=False, info=True, F=None, global_pivot=False, err_estimate=False):
    """Factor A in place (unless factored) and solve A F = F0 with FP64 refinement.
    F0: (n_rhs, n_sys) complex128. err_estimate: stop when the error estimated from the contraction of the
    last two corrections is <= tol (GDM_SOLVE_ERR_ESTIMATE) instead of the last correction.
    Returns (F, ipiv, info dict or None)."""
    ns = prob.size
    lda = A.shape[1]
    if ipiv is None:
        ipiv = torch.empty(ns, dtype=torch.int32, device=A.device)
    if F is None:
        F = torch.empty_like(F0)
    n_rhs = F0.shape[0]
    flags = ((SOLVE_FACTORED if factored else 0) | (SOLVE_NO_REFINE if no_refine else 0)
             | (SOLVE_GLOBAL_PIVOT if global_pivot else 0) | (SOLVE_ERR_ESTIMATE if err_estimate else 0))
    opts = SolveOpts(int(max_iter), flags, float(tol))
    inf = SolveInfo() if info else None
    s = prob.struct()
    ctx._sync_stream()
    ctx._check(lib().gdm_solve(ctx.h, C.byref(s), PRECISION[precision], _ptr(A), lda, _ptr(ipiv), _ptr(F0.contiguous()),
                               _ptr(F), n_rhs, C.byref(opts), C.byref(inf) if info else None), "gdm_solve")
    return F, ipiv, (inf.as_dict() if info else None)


def solve_gmres(ctx: Context, prob: GDMProblem, F0, precision="tf32", restart=0, max_iter=0, tol=0.0,
                block_cells=0, coarse=True, blocks=True, fast_operator=True, F=None):
    """gdm_solve_gmres: matrix-free preconditioned GMRES for cells. F0: (n_rhs, 3n) complex128 device.
    Returns (F, info dict)."""
    if F is None:
        F = torch.empty_like(F0)
    flags = ((0 if coarse else GMRES_NO_COARSE) | (0 if blocks else GMRES_NO_BLOCKS)
             | (0 if fast_operator else GMRES_EXACT_OPERATOR))
    opts = GmresOpts(int(restart), int(max_iter), float(tol), int(block_cells), flags)
    inf = SolveInfo()
    s = prob.struct()
    ctx._sync_stream()
    ctx._check(lib().gdm_solve_gmres(ctx.h, PRECISION[precision], C.byref(s), _ptr(F0.contiguous()), _ptr(F),
                                     F0.shape[0], C.byref(opts), C.byref(inf)), "gdm_solve_gmres")
    return F, inf.as_dict()


def lattice_partition(pos, step, block_cells=512):
    """gdm_lattice_partition (host only): (perm, parent, coarse_offsets) as numpy int32 arrays for host
    positions pos ((n, 3) float64)."""
    pos = np.ascontiguousarray(np.asarray(pos, np.float64))
    n = pos.shape[0]
    perm = np.empty(n, np.int32)
    parent = np.empty(n, np.int32)
    coff = np.empty(n + 1, np.int32)
    nc = I64(0)
    st = lib().gdm_lattice_partition(pos.ctypes.data, n, float(step), int(block_cells), perm.ctypes.data,
                                     parent.ctypes.data, coff.ctypes.data, C.byref(nc))
    if st != GDM_OK:
        raise GDMError(st, "gdm_lattice_partition")
    return perm, parent, coff[:nc.value + 1].copy()


def residual(ctx: Context, prob: GDMProblem, F0, F):
    """FP64 matrix-free residual F0 - A F: returns (r, ||r_q||^2) with r shaped like F."""
    r = torch.empty_like(F)
    n2 = torch.zeros(F.shape[0], dtype=torch.float64, device=F.device)
    s = prob.struct()
    ctx._sync_stream()
    ctx._check(lib().gdm_residual(ctx.h, C.byref(s), _ptr(F0.contiguous()), _ptr(F.contiguous()), F.shape[0], _ptr(r),
                                  _ptr(n2)), "gdm_residual")
    return r, n2


def nearfield(ctx: Context, prob: GDMProblem, F, r_eval, F0_eval=None, with_h=True):
    """E (and H) at r_eval: returns (E, H) each (n_rhs, 3*m) complex128 (H None if not requested)."""
    n_rhs = F.shape[0]
    m = r_eval.shape[0]
    E = torch.empty((n_rhs, 3 * m), dtype=torch.complex128, device=F.device)
    H = torch.empty_like(E) if with_h else None
    s = prob.struct()
    ctx._sync_stream()
    ctx._check(lib().gdm_nearfield(ctx.h, C.byref(s), _ptr(F.contiguous()), _ptr(r_eval.contiguous()), m,
                                   _ptr(None if F0_eval is None else F0_eval.contiguous()), n_rhs, _ptr(E), _ptr(H)),
               "gdm_nearfield")
    return E, H


def cross_sections(ctx: Context, prob: GDMProblem, F0, F, e0_norm2):
    """(ext, sca, abs) device tensors of n_rhs doubles (nm^2)."""
    n_rhs = F.shape[0]
    na, npp = _dbl_array(e0_norm2)
    out = torch.empty((3, n_rhs), dtype=torch.float64, device=F.device)
    s = prob.struct()
    ctx._sync_stream()
    ctx._check(lib().gdm_cross_sections(ctx.h, C.byref(s), _ptr(F0.contiguous()), _ptr(F.contiguous()), n_rhs, npp,
                                        _ptr(out[0]), _ptr(out[1]), _ptr(out[2])), "gdm_cross_sections")
    return out[0], out[1], out[2]


def cross_sections_noalloc(ctx: Context, prob: GDMProblem, F0, F, e0_norm2, out):
    """gdm_cross_sections_noalloc: writes (ext, sca, abs) into the caller's (3, n_rhs) float64 device tensor
    `out`; the library allocates nothing."""
    n_rhs = F.shape[0]
    if out.shape != (3, n_rhs) or out.dtype != torch.float64 or not out.is_contiguous():
        raise ValueError("out must be a contiguous (3, n_rhs) float64 tensor")
    if not (F0.is_contiguous() and F.is_contiguous()):
        raise ValueError("F0 and F must be contiguous")
    na, npp = _dbl_array(e0_norm2)
    s = prob.struct()
    ctx._sync_stream()
    ctx._check(lib().gdm_cross_sections_noalloc(ctx.h, C.byref(s), _ptr(F0), _ptr(F), n_rhs, npp, _ptr(out[0]),
                                                _ptr(out[1]), _ptr(out[2])), "gdm_cross_sections_noalloc")
    return out[0], out[1], out[2]


def solve_batched(ctx: Context, probs, e0s, precision="tf32", khat=(0.0, 0.0, 1.0), n_streams=0, with_sigma=True,
                  max_iter=0, tol=0.0, return_factors=False, err_estimate=False):
    """gdm_solve_batched over independent problems: probs is a list of GDMProblem, e0s a list of (n_rhs, 3)
    complex plane-wave amplitudes (one per problem). Allocates the items' matrices, pivots, fields and
    cross sections (one device buffer of each kind, sliced per item); err_estimate as for solve; returns
    (F list of (n_rhs, kind*n)
    complex128, sigma list of (3, n_rhs) or None, info list of dicts)."""
    prec = PRECISION[precision]
    n = len(probs)
    items = (BatchItem * n)()
    e0l = [np.atleast_2d(np.asarray(e0, np.complex128)) for e0 in e0s]
    nrhs = [e.shape[0] for e in e0l]
    sizes = [pb.size for pb in probs]
    ldas = [padded_lda(ns) for ns in sizes]
    dev = probs[0].pos.device if n else torch.device("cuda")
    cdt = torch.complex128 if precision == "fp64" else torch.complex64

    def offsets(counts, align):
        off, acc = [], 0
        for c in counts:
            off.append(acc)
            acc += (c + align - 1) // align * align
        return off, max(acc, 1)

    # element offsets aligned to 256 bytes (32 complex64, 16 complex128 elements)
    a_off, a_tot = offsets([ns * lda for ns, lda in zip(sizes, ldas)], 32)
    p_off, p_tot = offsets(sizes, 64)
    f_off, f_tot = offsets([r * ns for r, ns in zip(nrhs, sizes)], 16)
    s_off, s_tot = offsets([3 * r for r in nrhs], 32)
    Abuf = torch.empty(a_tot, dtype=cdt, device=dev)
    Pbuf = torch.empty(p_tot, dtype=torch.int32, device=dev)
    F0buf = torch.empty(f_tot, dtype=torch.complex128, device=dev)
    Fbuf = torch.empty(f_tot, dtype=torch.complex128, device=dev)
    Sbuf = torch.empty(s_tot, dtype=torch.float64, device=dev) if with_sigma else None
    e0all = np.ascontiguousarray(np.concatenate([e.reshape(-1) for e in e0l]).view(np.float64)) if n else None
    e0_off = np.cumsum([0] + [6 * r for r in nrhs])
    ka, kp = _dbl_array(khat)
    keep = [Abuf, Pbuf, F0buf, Fbuf, Sbuf, e0all, ka]
    Fs, sigs, As, ipivs = [], [], [], []
    a_ptr, p_ptr, f0_ptr, f_ptr = Abuf.data_ptr(), Pbuf.data_ptr(), F0buf.data_ptr(), Fbuf.data_ptr()
    e_ptr = e0all.ctypes.data if n else 0
    for i, pb in enumerate(probs):
        ns, lda, r = sizes[i], ldas[i], nrhs[i]
        it = items[i]
        it.prob = pb.struct()
        it.A, it.lda = a_ptr + a_off[i] * Abuf.element_size(), lda
        it.ipiv = p_ptr + p_off[i] * 4
        it.F0, it.F = f0_ptr + f_off[i] * 16, f_ptr + f_off[i] * 16
        it.sigma = Sbuf.data_ptr() + s_off[i] * 8 if with_sigma else 0
        it.e0 = e_ptr + int(e0_off[i]) * 8
        it.khat = ka.ctypes.data
        it.e0_norm2 = 0
        it.n_rhs = r
        Fs.append(Fbuf[f_off[i]:f_off[i] + r * ns].view(r, ns))
        sigs.append(Sbuf[s_off[i]:s_off[i] + 3 * r].view(3, r) if with_sigma else None)
        if return_factors:
            As.append(Abuf[a_off[i]:a_off[i] + ns * lda].view(ns, lda))
            ipivs.append(Pbuf[p_off[i]:p_off[i] + ns])
    opts = SolveOpts(int(max_iter), SOLVE_ERR_ESTIMATE if err_estimate else 0, float(tol))
    infos = (SolveInfo * n)()
    ctx._sync_stream()
    ctx._check(lib().gdm_solve_batched(ctx.h, prec, items, n, C.byref(opts), int(n_streams), infos),
               "gdm_solve_batched")
    del keep
    out = (Fs, sigs, [infos[i].as_dict() for i in range(n)])
    return out + (As, ipivs) if return_factors else out


def backward_batched(ctx: Context, probs, As, ipivs, Fs, e0, precision="tf32", khat=(0.0, 0.0, 1.0), gFs=None,
                     g_sigmas=None, grad_pos=None, grad_eps=None, grad_wavelengths=None, n_streams=0):
    """gdm_backward_batched for one structure at several wavelengths (probs share pos and eps): the position
    and eps gradients of all items summed into grad_pos / grad_eps, dL/dlambda per item into
    grad_wavelengths (len(probs) doubles). gFs: list of dL/dF^* tensors (or None), g_sigmas: list of host
    (n_rhs, 3) arrays (or None)."""
    n = len(probs)
    dev = Fs[0].device
    nc = probs[0].n
    if grad_pos is None:
        grad_pos = torch.zeros((nc, 3), dtype=torch.float64, device=dev)
    if grad_eps is None:
        grad_eps = torch.zeros(nc, dtype=torch.complex128, device=dev)
    if grad_wavelengths is None:
        grad_wavelengths = torch.zeros(n, dtype=torch.float64, device=dev)
    e0 = np.atleast_2d(np.asarray(e0, np.complex128))
    ea, ep = _dbl_array(e0.view(np.float64).reshape(-1))
    ka, kp = _dbl_array(khat)
    keep = [ea, ka]
    items = (BackwardItem * n)()
    for i in range(n):
        it = items[i]
        it.prob = probs[i].struct()
        it.A, it.lda, it.ipiv = As[i].data_ptr(), As[i].shape[1], ipivs[i].data_ptr()
        F = Fs[i].contiguous()
        keep.append(F)
        it.F = F.data_ptr()
        if gFs is not None and gFs[i] is not None:
            g = gFs[i].contiguous()
            keep.append(g)
            it.gF = g.data_ptr()
        if g_sigmas is not None and g_sigmas[i] is not None:
            ga, gp = _dbl_array(np.asarray(g_sigmas[i], np.float64).reshape(-1))
            keep.append(ga)
            it.g_sigma = ga.ctypes.data
        it.e0 = ea.ctypes.data
        it.khat = ka.ctypes.data
        it.grad_wavelength = grad_wavelengths.data_ptr() + 8 * i
        it.n_rhs = e0.shape[0]
    infos = (SolveInfo * n)()
    ctx._sync_stream()
    ctx._check(lib().gdm_backward_batched(ctx.h, PRECISION[precision], items, n, int(n_streams), _ptr(grad_pos),
                                          _ptr(grad_eps), infos), "gdm_backward_batched")
    return grad_pos, grad_eps, grad_wavelengths, [infos[i].as_dict() for i in range(n)]


def gpm_extract(ctx: Context, prob: GDMProblem, r_gpm, r_probe, pw_khat, pw_e0, ds_pos, ds_mom, precision="tf32"):
    """gdm_gpm_extract: effective (E, H) -> (p, m) polarizability matrix of the structure at the sites r_gpm
    ((M, 3) device), fitted to its scattered fields at r_probe ((P, 3) device) for plane waves (host lists
    khat, e0) and dipole sources (device (s, 3) positions, (s, 6) moments). Returns (alpha_eff (6M, 6M),
    moments (6M, n_ill), relative residual of the moment fit)."""
    M = r_gpm.shape[0]
    kh = np.ascontiguousarray(np.asarray(pw_khat, np.float64).reshape(-1, 3))
    e0 = np.ascontiguousarray(np.asarray(pw_e0, np.complex128).reshape(-1, 3))
    n_pw, n_ds = kh.shape[0], (0 if ds_pos is None else ds_pos.shape[0])
    dev = r_gpm.device
    ns = prob.size
    A = torch.empty((ns, padded_lda(ns)), dtype=torch.complex128 if precision == "fp64" else torch.complex64,
                    device=dev)
    ipiv = torch.empty(ns, dtype=torch.int32, device=dev)
    alpha = torch.empty((6 * M, 6 * M), dtype=torch.complex128, device=dev)
    mom = torch.empty((n_pw + n_ds, 6 * M), dtype=torch.complex128, device=dev)
    rel = D(0.0)
    s = prob.struct()
    ctx._sync_stream()
    ctx._check(lib().gdm_gpm_extract(ctx.h, PRECISION[precision], C.byref(s), _ptr(A), A.shape[1], _ptr(ipiv),
                                     _ptr(r_gpm.contiguous()), M, _ptr(r_probe.contiguous()), r_probe.shape[0], n_pw,
                                     kh.ctypes.data, e0.ctypes.data, n_ds,
                                     _ptr(None if ds_pos is None else ds_pos.contiguous()),
                                     _ptr(None if ds_mom is None else ds_mom.contiguous()), _ptr(alpha), _ptr(mom),
                                     C.byref(rel)), "gdm_gpm_extract")
    # the library writes column-major matrices
    return alpha.t(), mom.t(), rel.value


def farfield(ctx: Context, prob: GDMProblem, F, dirs):
    """Far-field amplitudes f(rhat) at the unit directions dirs ((q, 3) device): (n_rhs, 3q) complex128."""
    n_rhs = F.shape[0]
    q = dirs.shape[0]
    out = torch.empty((n_rhs, 3 * q), dtype=torch.complex128, device=F.device)
    s = prob.struct()
    ctx._sync_stream()
    ctx._check(lib().gdm_farfield(ctx.h, C.byref(s), _ptr(F.contiguous()), n_rhs, _ptr(dirs.contiguous()), q,
                                  _ptr(out)), "gdm_farfield")
    return out


def sigma_farfield(ctx: Context, prob: GDMProblem, F, e0_norm2, n_theta=64, n_phi=128):
    """sigma_sca from the far-field integral (device (n_rhs,) float64, nm^2)."""
    n_rhs = F.shape[0]
    na, npp = _dbl_array(e0_norm2)
    out = torch.empty(n_rhs, dtype=torch.float64, device=F.device)
    s = prob.struct()
    ctx._sync_stream()
    ctx._check(lib().gdm_sigma_farfield(ctx.h, C.byref(s), _ptr(F.contiguous()), n_rhs, npp, int(n_theta),
                                        int(n_phi), _ptr(out)), "gdm_sigma_farfield")
    return out


def incident_gaussian(ctx: Context, r, wavelength, e0, w0, focus=(0.0, 0.0, 0.0), theta=0.0, eps_env=1.0,
                      kind_out=3):
    """Paraxial Gaussian beam at r ((m, 3) device): (n_rhs, kind_out*m) complex128; e0 (n_rhs, 3) in the beam
    frame, waist w0, focus, incidence angle theta in the XZ plane."""
    e0 = np.atleast_2d(np.asarray(e0, np.complex128))
    n_rhs = e0.shape[0]
    ea, ep = _dbl_array(e0.view(np.float64).reshape(-1))
    fa, fp = _dbl_array(focus)
    r = r.contiguous()
    out = torch.empty((n_rhs, kind_out * r.shape[0]), dtype=torch.complex128, device=r.device)
    ctx._sync_stream()
    ctx._check(lib().gdm_incident_gaussian(ctx.h, _ptr(r), r.shape[0], float(wavelength), float(eps_env), ep,
                                           float(w0), fp, float(theta), n_rhs, kind_out, _ptr(out)),
               "gdm_incident_gaussian")
    return out


def incident_dipole(ctx: Context, r, wavelength, src_pos, src_mom, kind_out=3, eps_env=1.0):
    """Fields of point dipoles (device (s, 3) positions, (s, 6) complex moments) at r ((m, 3) device), in a
    host of permittivity eps_env: (s, kind_out*m) complex128, one row per source."""
    n_src = src_pos.shape[0]
    out = torch.empty((n_src, kind_out * r.shape[0]), dtype=torch.complex128, device=r.device)
    ctx._sync_stream()
    ctx._check(lib().gdm_incident_dipole(ctx.h, _ptr(r.contiguous()), r.shape[0], float(wavelength),
                                         float(eps_env), _ptr(src_pos.contiguous()), _ptr(src_mom.contiguous()), n_src, kind_out,
                                         _ptr(out)), "gdm_incident_dipole")
    return out


def ldos(ctx: Context, prob: GDMProblem, r0, magnetic=False, precision="tf32"):
    """Electric (or magnetic) partial LDOS rho_u/rho_0 for u = x, y, z at r0 ((n, 3) device): (n, 3) float64."""
    ns = prob.size
    dev = r0.device
    A = torch.empty((ns, padded_lda(ns)), dtype=torch.complex128 if precision == "fp64" else torch.complex64,
                    device=dev)
    ipiv = torch.empty(ns, dtype=torch.int32, device=dev)
    out = torch.empty((r0.shape[0], 3), dtype=torch.float64, device=dev)
    s = prob.struct()
    ctx._sync_stream()
    ctx._check(lib().gdm_ldos(ctx.h, PRECISION[precision], C.byref(s), _ptr(A), A.shape[1], _ptr(ipiv),
                              _ptr(r0.contiguous()), r0.shape[0], 1 if magnetic else 0, _ptr(out)), "gdm_ldos")
    return out


def autotune(ctx: Context, sizes, precision="tf32"):
    """gdm_autotune: LU block width per size class for this context; returns the 8-entry table."""
    sz = np.ascontiguousarray(np.asarray(sizes, np.int64))
    out = (C.c_int * 8)()
    ctx._sync_stream()
    ctx._check(lib().gdm_autotune(ctx.h, PRECISION[precision], sz.ctypes.data_as(C.c_void_p), len(sz), out),
               "gdm_autotune")
    return list(out)


def autotune_batched(ctx: Context, sizes):
    """gdm_autotune_batched: outer block width of the grouped (lock-step) factorisation of a TF32 batch with
    these system sizes, kept in the context; returns it."""
    sz = np.ascontiguousarray(np.asarray(sizes, np.int64))
    out = C.c_int(0)
    ctx._sync_stream()
    ctx._check(lib().gdm_autotune_batched(ctx.h, sz.ctypes.data_as(C.c_void_p), len(sz), C.byref(out)),
               "gdm_autotune_batched")
    return out.value


def backward(ctx: Context, prob: GDMProblem, A, ipiv, F, e0, khat=(0.0, 0.0, 1.0), gF=None, g_sigma=None,
             precision="fp32", grad_pos=None, grad_eps=None, grad_wavelength=None):
    """Adjoint backward (kind 3): adds dL/dr, dL/deps, dL/dlambda into the given (or new zero) tensors."""
    n_rhs = F.shape[0]
    dev = F.device
    if grad_pos is None:
        grad_pos = torch.zeros((prob.n, 3), dtype=torch.float64, device=dev)
    if grad_eps is None:
        grad_eps = torch.zeros(prob.n, dtype=torch.complex128, device=dev)
    if grad_wavelength is None:
        grad_wavelength = torch.zeros(1, dtype=torch.float64, device=dev)
    e0 = np.atleast_2d(np.asarray(e0, np.complex128))
    ea, ep = _dbl_array(e0.view(np.float64).reshape(-1))
    ka, kp = _dbl_array(khat)
    if g_sigma is not None:
        ga, gp = _dbl_array(np.asarray(g_sigma, np.float64).reshape(-1))
    else:
        gp = None
    inf = SolveInfo()
    s = prob.struct()
    ctx._sync_stream()
    ctx._check(lib().gdm_backward(ctx.h, C.byref(s), PRECISION[precision], _ptr(A), A.shape[1], _ptr(ipiv),
                                  _ptr(F.contiguous()), n_rhs, ep, kp, _ptr(None if gF is None else gF.contiguous()),
                                  gp, _ptr(grad_pos), _ptr(grad_eps), _ptr(grad_wavelength), C.byref(inf)),
               "gdm_backward")
    return grad_pos, grad_eps, grad_wavelength, inf.as_dict()


def nearfield_backward(ctx: Context, prob: GDMProblem, F, r_eval, e0, gE, khat=(0.0, 0.0, 1.0), gF_accum=None,
                       grad_pos=None, grad_eps=None, grad_wavelength=None):
    n_rhs = F.shape[0]
    dev = F.device
    e0 = np.atleast_2d(np.asarray(e0, np.complex128))
    ea, ep = _dbl_array(e0.view(np.float64).reshape(-1))
    ka, kp = _dbl_array(khat)
    s = prob.struct()
    ctx._sync_stream()
    ctx._check(lib().gdm_nearfield_backward(ctx.h, C.byref(s), _ptr(F.contiguous()), _ptr(r_eval.contiguous()),
                                            r_eval.shape[0], n_rhs, ep, kp, _ptr(gE.contiguous()), _ptr(gF_accum),
                                            _ptr(grad_pos), _ptr(grad_eps), _ptr(grad_wavelength)),
               "gdm_nearfield_backward")
    return gF_accum, grad_pos, grad_eps, grad_wavelength
