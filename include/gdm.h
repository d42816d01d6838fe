/*
 * gdm.h -- C ABI of the GB300 (sm_103a) Green's Dyadic Method hot path.
 *
 * The library solves the discretised Lippmann-Schwinger equation of the
 * coupled-dipole / Green's Dyadic Method (Wiecha et al., "TorchGDM",
 * arXiv:2505.09545, Sec. "Formalism and implementation"):
 *
 *     F_i = F0_i + sum_j G(r_i, r_j) alpha_j F_j          (Eq. LPS_6by6_discrete)
 *     sum_j [delta_ij I - G(r_i, r_j) alpha_j] F_j = F0_i  (Eq. GDM_system_of_equations,
 *                                                         read without the stray F(r_j))
 *
 * for every illumination, then evaluates near fields and cross sections from
 * the self-consistent dipoles (Sec. "Observables") and gradients through the
 * solve (Sec. "Numerical solution", automatic differentiation of the LU solve).
 *
 * Conventions used by every call
 * ------------------------------
 * Units: Gaussian (cgs) as in the paper, lengths and wavelengths in nm. Time
 *   factor exp(-i w t): outgoing waves are exp(+ikR), lossy media have Im(eps) > 0.
 * Complex numbers are stored interleaved (re, im): complex128 = 2 doubles,
 *   complex64 = 2 floats.
 * Unknowns are dipole-interleaved: index kind*i + c, with kind = 3 (E of cell i,
 *   c = x,y,z) or kind = 6 (E then H of effective dipole i). The paper orders all
 *   E before all H (Sec. "Hybrid discretization GDM"); this is a permutation of it.
 * Matrices are column-major with a leading dimension `lda` (complex elements):
 *   entry (row, col) at A[col*lda + row]. Right-hand sides / fields are
 *   (kind*n) x n_rhs column-major with leading dimension kind*n.
 * Memory: every pointer documented as "device" is caller-owned device memory on
 *   the context's device; "host" pointers are ordinary host memory. The library
 *   never frees caller memory. The context owns only its scratch space.
 * Streams: every call is enqueued on the context's stream and returns without
 *   waiting for the GPU, unless documented otherwise. The returned status covers
 *   argument validation and launch errors; errors found on the device (a zero
 *   pivot, a refinement that did not converge, a bounded device wait that ran
 *   out) are reported through gdm_solve_info and gdm_ctx_check().
 * Errors: no call aborts or exits. On failure the call returns a non-zero
 *   gdm_status and gdm_last_error() holds a one-line message.
 */
#ifndef GDM_H
#define GDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GDM_OK = 0,
    GDM_ERR_INVALID_ARG = 1,   /* null pointer, bad kind/precision, non-positive size */
    GDM_ERR_SHAPE = 2,         /* lda too small, misaligned leading dimension */
    GDM_ERR_NONFINITE = 3,     /* NaN/Inf found in an input or produced by the solve */
    GDM_ERR_SINGULAR = 4,      /* exactly zero pivot in the LU factorisation */
    GDM_ERR_NOT_CONVERGED = 5, /* iterative refinement did not reach the tolerance */
    GDM_ERR_OOM = 6,           /* scratch allocation failed (device memory, or host memory / threads) */
    GDM_ERR_CUDA = 7,          /* CUDA runtime / driver error */
    GDM_ERR_TIMEOUT = 8,       /* a bounded device-side wait gave up */
    GDM_ERR_UNSUPPORTED = 9    /* valid request that this build does not implement */
} gdm_status;

/* Arithmetic of the factorisation. All modes return FP64 fields.
 * GDM_FP64        : complex128 matrix, FP64 LU and triangular solves (the plain path).
 * GDM_FP32        : complex64 matrix, LU with FP32-accurate tensor-core trailing
 *                   updates (TF32 hi/lo split, three products), FP64 refinement.
 * GDM_TF32_REFINE : complex64 matrix, LU with single-pass TF32 tensor-core
 *                   trailing updates, FP64 refinement.
 * GDM_BF16_REFINE : complex64 matrix, LU whose trailing updates A22 -= A21 U12 run
 *                   with BF16 operands (rounded to nearest even) and FP32 accumulation
 *                   on the tensor cores, the rest as GDM_TF32_REFINE; FP64 refinement,
 *                   which takes more steps than with TF32 factors (8 significand bits
 *                   against 11). The paper's solve is a plain LU (Sec. "Numerical
 *                   solution"); lower-precision factors with refinement are this
 *                   library's own. BF16 has FP32's exponent range, so no scaling is
 *                   needed beyond the refinement's own right-hand-side scaling. */
typedef enum { GDM_FP64 = 0, GDM_FP32 = 1, GDM_TF32_REFINE = 2, GDM_BF16_REFINE = 3 } gdm_precision;

typedef struct gdm_ctx gdm_ctx;

/* One scattering problem at one wavelength.
 * kind 3: discretised cubic cells, electric response only. alpha_i =
 *   (eps_i - eps_env) d^3 / (4 pi) (Sec. "Volume discretization polarizabilities"),
 *   self-term S = -I 4 pi / (3 eps_env d^3) (Eq. selfterm_SEp_cubic).
 * kind 6: effective electric/magnetic point dipoles with full 6x6 polarisability
 *   alpha_i (dipole-moment relation (p, m) = alpha F), zero self-term. In a host of
 *   permittivity eps_env (non-magnetic) the 6x6 dyad is [[G^Ep, -G^Hp], [G^Hp, eps_env G^Ep]]
 *   with k = n_env 2 pi / lambda0 (Gaussian units, exp(-i w t)). */
typedef struct {
    int64_t n;              /* number of dipoles (cells or effective dipoles), >= 1 */
    int32_t kind;           /* 3 or 6 */
    int32_t reserved;
    const double *pos;      /* device, n x 3 row-major (x, y, z), nm */
    const double *eps;      /* kind 3: device, n complex128 cell permittivities; else NULL */
    const double *alpha6;   /* kind 6: device, n x 6 x 6 complex128, row-major per dipole; else NULL */
    double step;            /* kind 3: cubic mesh step d (nm), > 0; ignored for kind 6 */
    double eps_env;         /* real host permittivity, > 0 */
    double wavelength;      /* vacuum wavelength lambda0 (nm), > 0 */
} gdm_problem;

/* Refinement controls for gdm_solve. Zero-initialised => defaults. */
typedef struct {
    int32_t max_iter;       /* refinement steps allowed (default 40; FP64: default 3) */
    int32_t flags;          /* GDM_SOLVE_* bit flags */
    double tol;             /* stop when max_r ||dF_r|| / ||F_r|| <= tol (default 1e-12) */
} gdm_solve_opts;

#define GDM_SOLVE_FACTORED 1      /* A already holds this problem's factors and ipiv its pivots */
#define GDM_SOLVE_NO_REFINE 2     /* return the plain triangular-solve result */
#define GDM_SOLVE_GLOBAL_PIVOT 4  /* always search pivots over the whole column (partial pivoting) */
/* Stop on the estimated error instead of the last correction: when the last two relative corrections
 * c_prev, c of a right-hand side contract by rho = c / c_prev <= 1/4, the corrections that would follow sum
 * to about rho c / (1 - rho) (a geometric tail), which is the relative error left in the returned F; the
 * refinement stops once that estimate (else c itself) is <= tol for every right-hand side. Iterative
 * refinement with an error estimate from the contraction of successive corrections, as in Demmel et al.,
 * "Error bounds from extra-precise iterative refinement", ACM TOMS 32 (2006). rel_correction still reports
 * the last correction. */
#define GDM_SOLVE_ERR_ESTIMATE 8
/* Pivoting: by default each 32-column panel searches its pivots among the rows of its 32 x 32
 * diagonal block and certifies the choice against all rows below. If some row below exceeds its
 * pivot by more than GDM_PIVOT_GROWTH_LIMIT, gdm_solve re-assembles A from the problem and factors
 * again with partial pivoting over whole columns; a certificate <= 1 means the factors are exactly
 * those of partial pivoting. */
#define GDM_PIVOT_GROWTH_LIMIT 4.0

typedef struct {
    int32_t iterations;          /* refinement steps taken */
    int32_t status;              /* gdm_status of the device-side checks */
    double rel_correction;       /* last max_r ||dF_r|| / ||F_r|| */
    double rel_residual;         /* last max_r ||F0_r - A F_r|| / ||F0_r|| (FP64, matrix-free) */
    double factor_ms;            /* device time of the factorisation (0 if skipped) */
    double refine_ms;            /* device time of solves + refinement */
    double pivot_growth;         /* largest |entry below| / |pivot| seen by the panels (<= 1: partial pivoting) */
    int32_t refactored;          /* 1 if the factorisation was redone with whole-column pivoting */
    int32_t cycles;              /* gdm_solve_gmres: restart cycles (the double-float true residual is
                                    evaluated cycles times: before every cycle but the first, whose
                                    iterate is 0, and at the end); 0 for the direct solves */
} gdm_solve_info;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`; `stream` is a cudaStream_t (NULL =
 * the legacy default stream). Allocates nothing until a call needs scratch. */
gdm_status gdm_create(gdm_ctx **ctx, int device, void *stream);
gdm_status gdm_destroy(gdm_ctx *ctx);
gdm_status gdm_set_stream(gdm_ctx *ctx, void *stream);
/* Waits for the context's stream, then returns the first device-side error
 * recorded since the last check (GDM_OK if none) and clears it. */
gdm_status gdm_ctx_check(gdm_ctx *ctx);

/* Failure-detection check (no paper counterpart): launches one thread that waits for a device
 * flag which nothing sets, giving up after limit_ms (<= 2000) like every bounded wait of the
 * library's persistent kernels, records GDM_ERR_TIMEOUT in the context's device error record
 * and returns what gdm_ctx_check reads back: GDM_ERR_TIMEOUT, with the context usable
 * afterwards (the record is cleared by the read). Synchronous. */
gdm_status gdm_diag_wait_timeout(gdm_ctx *ctx, double limit_ms);
const char *gdm_status_string(gdm_status s);
const char *gdm_last_error(gdm_ctx *ctx);
/* Number of kernel launches this context has issued so far. */
int64_t gdm_launch_count(gdm_ctx *ctx);

/* Scratch bytes a gdm_solve / gdm_backward of this problem will hold in the
 * context (pivot-independent panel buffers, tensor-core operand buffers and the
 * embedding of L, the U12 block operator, refinement vectors; the factorisation and
 * the refinement share one arena, so this is the larger of the two), for the default
 * outer block width. */
gdm_status gdm_workspace_size(const gdm_problem *p, int n_rhs, gdm_precision prec, size_t *bytes);

/* The quantity a refinement compares with tol after a step whose largest relative correction over the
 * right-hand sides was c, the step before having had c_prev (<= 0: no step before): c itself, or, with
 * GDM_SOLVE_ERR_ESTIMATE in flags and a clear contraction rho = c / c_prev <= 1/4, the estimated relative
 * error left after the step, rho c / (1 - rho). Host-only (the rule gdm_solve and gdm_solve_batched apply). */
double gdm_refine_stop_measure(double c, double c_prev, int32_t flags);

/* ---------------------------------------------------------------- polarisabilities */

/* Effective electric/magnetic dipole polarisabilities from Lorentzian lines (Sec.
 * "Effective polarizabilities", manually set lineshapes) in a host of permittivity eps_env, for
 * the kind 6 problem's alpha6: with w = hc/lambda (eV) and k = n_env 2 pi / lambda,
 *   alpha0   = a^3 w0^2 / (w0^2 - w^2 - i gamma w),
 *   alpha_e  = 1 / (1/alpha0 - i (2/3) k^3 / eps_env),  alpha_m = 1 / (1/alpha0 - i (2/3) k^3)
 * (radiative reaction of the host, so that a lone lossless dipole obeys the optical theorem),
 * alpha6_i = diag(alpha_e I3, alpha_m I3). omega0_e, omega0_m: device n resonance energies
 * (eV). alpha6_out: device n x 6 x 6 complex128 (row-major 6x6 per dipole), overwritten. */
gdm_status gdm_alpha6_lorentz(gdm_ctx *ctx, int64_t n, const double *omega0_e, const double *omega0_m,
                              double gamma_ev, double amp_nm, double wavelength, double eps_env,
                              double *alpha6_out);

/* ---------------------------------------------------------------- illumination */

/* Plane wave E0(r) = e0 exp(i k khat.r), H0 = n_env khat x E0, k = n_env 2 pi / lambda0,
 * at m points. r: device m x 3. e0: host n_rhs x 3 complex128 amplitudes.
 * khat: host 3 doubles, unit propagation direction. kind_out = 3 writes E only,
 * 6 writes (E, H) per point. F0: device (kind_out*m) x n_rhs complex128. */
gdm_status gdm_incident_planewave(gdm_ctx *ctx, const double *r, int64_t m, double wavelength,
                                  double eps_env, const double *e0, const double *khat, int n_rhs,
                                  int kind_out, double *F0);

/* Paraxial focused Gaussian beam (Sec. "Illuminations": GaussianParaxial, with the longitudinal
 * field that keeps it divergence-free for tight focus). Beam frame: propagation along
 * z' = (sin theta, 0, cos theta), focus at focus (host 3 doubles, nm), waist w0 (nm); with
 * z0 = k w0^2/2 and g = 1 + i z'/z0 the transverse field is e0 exp(i k z')
 * exp(-(x'^2 + y'^2)/(w0^2 g))/g, E_z' = (i/k) div_t E_t, H_t = n_env z' x E_t, H_z' likewise.
 * e0: host n_rhs x 3 complex128 in the beam frame (x', y' used). r: device m x 3.
 * F0: device (kind_out*m) x n_rhs complex128. */
gdm_status gdm_incident_gaussian(gdm_ctx *ctx, const double *r, int64_t m, double wavelength, double eps_env,
                                 const double *e0, double w0, const double *focus, double theta, int n_rhs,
                                 int kind_out, double *F0);

/* Incident field of point-dipole sources (Sec. "Illuminations": electric and magnetic dipole
 * sources) in a host of permittivity eps_env: column q is [E; H](r) = G6(r - r_q) [p_q; m_q] at
 * the m points r_eval, G6 the host's 6x6 dyad (see gdm_problem).
 * src_pos: device n_src x 3; src_mom: device n_src x 6 complex128 (p, m); 1 <= n_src <= 1024.
 * kind_out 3 writes E only, 6 writes (E, H) per point. F0: device (kind_out*m) x n_src complex128. */
gdm_status gdm_incident_dipole(gdm_ctx *ctx, const double *r_eval, int64_t m, double wavelength, double eps_env,
                               const double *src_pos, const double *src_mom, int n_src, int kind_out, double *F0);

/* ---------------------------------------------------------------- hot path */

/* Assemble the dense system matrix A = I - G alpha (Eq. GDM_system_of_equations):
 * block (i, j) = delta_ij I - G(r_i, r_j) alpha_j, with G(r_i, r_i) the self-term.
 * prec GDM_FP64 writes complex128, otherwise complex64. A: device, column-major,
 * (kind*n) x (kind*n), lda >= kind*n complex elements, lda even. */
gdm_status gdm_assemble(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, void *A, int64_t lda);

/* Factor A in place (blocked LU with partial pivoting; complex128 for GDM_FP64,
 * complex64 otherwise) unless opts->flags has GDM_SOLVE_FACTORED, then solve
 * A F = F0 for n_rhs right-hand sides and refine in FP64 with the residual
 * F0 - A F computed matrix-free from the Green dyads (no stored FP64 matrix).
 * A: device matrix from gdm_assemble (overwritten by its LU factors).
 * ipiv: device int32 array of kind*n pivots (written, or read when FACTORED).
 * F0: device (kind*n) x n_rhs complex128. F: device output, same shape.
 * info: host, may be NULL. Synchronises the stream when info != NULL. */
gdm_status gdm_solve(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, void *A, int64_t lda,
                     int32_t *ipiv, const double *F0, double *F, int n_rhs, const gdm_solve_opts *opts,
                     gdm_solve_info *info);

/* One independent problem of a batch (a structure at one wavelength with its illuminations).
 * All pointers except e0, khat and e0_norm2 are device memory owned by the caller. */
typedef struct {
    gdm_problem prob;        /* structure, wavelength (device pos / eps / alpha6) */
    void *A;                 /* (kind*n) x lda matrix storage: complex64, complex128 for GDM_FP64 */
    int64_t lda;             /* as for gdm_assemble */
    int32_t *ipiv;           /* kind*n pivots (written) */
    double *F0;              /* (kind*n) x n_rhs complex128 incident field: read, or written when e0 != NULL */
    double *F;               /* (kind*n) x n_rhs complex128 solved fields (written) */
    double *sigma;           /* 3 x n_rhs doubles (ext row, sca row, abs row) written, or NULL */
    const double *e0;        /* host n_rhs x 3 complex128 plane-wave amplitudes, or NULL when F0 is given */
    const double *khat;      /* host 3 doubles, unit propagation direction (NULL: +z), used with e0 */
    const double *e0_norm2;  /* host n_rhs |E0|^2 for sigma when e0 is NULL */
    int32_t n_rhs;           /* 1..64 */
    int32_t reserved;
} gdm_batch_item;

/* The per-problem path of gdm_incident_planewave (when e0 is given), gdm_assemble,
 * gdm_solve and gdm_cross_sections (when sigma is given) for n_items independent
 * problems of any sizes, e.g. many structures each at its own wavelength (the paper's
 * workloads sweep wavelengths, polarisations and geometries). The items run concurrently:
 * the context keeps up to n_streams child contexts (own stream and scratch; 0 = 8, at most
 * 16), each driven by a host thread that takes the largest remaining item next. Work
 * already queued on the context stream comes first and later work on it waits for the
 * batch. Synchronous. infos: host n_items records (may be NULL), status per item.
 * Returns GDM_OK, or the first error; a numerical failure of one item (NOT_CONVERGED,
 * NONFINITE, SINGULAR) is recorded in its info and the other items still run, any other
 * error stops the batch. */
gdm_status gdm_solve_batched(gdm_ctx *ctx, gdm_precision prec, const gdm_batch_item *items, int n_items,
                             const gdm_solve_opts *opts, int n_streams, gdm_solve_info *infos);

/* One wavelength of a spectrum for gdm_backward_batched: the factors, pivots and fields of
 * that wavelength's solve, and the upstream gradients. Pointers are device memory unless
 * marked host. */
typedef struct {
    gdm_problem prob;          /* kind 3; n, pos, eps, step and eps_env shared by all items */
    const void *A;             /* factors from gdm_solve / gdm_solve_batched */
    int64_t lda;
    const int32_t *ipiv;
    const double *F;           /* (3n) x n_rhs complex128 solved fields */
    const double *gF;          /* (3n) x n_rhs dL/dF^* (conjugate Wirtinger), or NULL */
    const double *g_sigma;     /* host n_rhs x 3 dL/d(ext, sca, abs), or NULL */
    const double *e0;          /* host n_rhs x 3 complex128 plane-wave amplitudes */
    const double *khat;        /* host 3 doubles (NULL: +z) */
    double *grad_wavelength;   /* one double: dL/dlambda of this item ADDED here, or NULL */
    int32_t n_rhs;
    int32_t reserved;
} gdm_backward_item;

/* gdm_backward for a loss summed over the wavelengths of one structure (the paper's spectral
 * inverse-design losses, e.g. a target response over a band): every item's adjoint solve
 * and gradient kernels, run concurrently on up to n_streams child contexts (0 = 8, at most
 * 16) like gdm_solve_batched, with the position and permittivity gradients of all items
 * summed and ADDED to grad_pos (n x 3) and grad_eps (n complex128; either may be NULL). The
 * items must share the structure (same n, pos and eps pointers, step, eps_env). Synchronous;
 * infos: host n_items records or NULL. Errors as gdm_solve_batched. */
gdm_status gdm_backward_batched(gdm_ctx *ctx, gdm_precision prec, const gdm_backward_item *items, int n_items,
                                int n_streams, double *grad_pos, double *grad_eps, gdm_solve_info *infos);

/* ---------------------------------------------------------------- iterative solver */

typedef struct {
    int32_t restart;      /* Krylov vectors per cycle m (default 60 when <= 0; at most 120) */
    int32_t max_iter;     /* operator applications allowed in total (default 1000 when <= 0) */
    double tol;           /* stop when max_r ||F0_r - A F_r|| / ||F0_r|| <= tol (default 1e-12 when <= 0) */
    int32_t block_cells;  /* cells per block of the block-Jacobi part (default 512 when <= 0; at most 1024) */
    int32_t flags;        /* GDM_GMRES_* bit flags */
} gdm_gmres_opts;

#define GDM_GMRES_NO_COARSE 1  /* leave out the coarse-model correction of the preconditioner */
#define GDM_GMRES_NO_BLOCKS 2  /* leave out its block-Jacobi part (both flags: plain GMRES) */
#define GDM_GMRES_EXACT_OPERATOR 4  /* Arnoldi steps on the double-float operator, not the FP32 one */

/* Solve A F = F0 for a discretised structure (kind 3) without forming A, for structures beyond the
 * dense path's memory (no paper counterpart: the paper bounds its full inversion to about 10^4
 * dipoles and names iterative schemes as the way past it, Sec. "Conclusions" and "Benchmarks").
 * Flexible GMRES(m) in FP64 on the matrix-free operator, right-preconditioned by
 *   M^-1 v = P A_c^-1 R v + B^-1 (v - P R v),
 * A_c the coarser model (cells merged 2 x 2 x 2 on the lattice: centroid position, summed
 * polarisability in the couplings, and the self-term block 1 + chi/(3 eps_env) of a cube filled
 * with the merged cells' mean susceptibility chi), R the mean over the merged cells, P the copy
 * back, B the exact diagonal blocks of A over runs of block_cells cells in Morton order of the
 * lattice; A_c and the blocks are assembled and factored by the mixed-precision LU in `prec`
 * (GDM_TF32_REFINE or GDM_FP32). A structure of at most block_cells cells is preconditioned by its
 * whole LU alone (the coarse term is left out).
 * Each restart cycle starts from the true residual F0 - A F in double-float arithmetic (the
 * refinement residual of gdm_solve, ~1e-13 relative). Unless GDM_GMRES_EXACT_OPERATOR is set, its
 * Arnoldi steps use FP32 Green sums (double-float phase, ~1e-6 relative) and the cycle ends once it
 * has reduced its residual by 1e-4: the cycles are the outer steps of an iterative refinement, and a
 * cycle that fails to halve the true residual switches the rest of the solve to the double-float
 * operator. Cells are assumed on a cubic lattice of step p->step (positions are rounded to it for
 * the grouping only). F0, F: device (3n) x n_rhs complex128, 1 <= n_rhs <= 8 (all right-hand sides
 * iterate in lockstep). Device memory: about (2m + 6) 3n n_rhs complex128 vectors, the block factors
 * (3 block_cells x 8 bytes per row of A) and the coarse factors ((3n/8)^2 x 8 bytes); allocated and
 * freed inside the call. info (nullable): iterations = operator applications, rel_residual = final
 * max_r ||F0_r - A F_r|| / ||F0_r||, rel_correction = last GMRES residual estimate, factor_ms =
 * preconditioner set-up, refine_ms = iterations, pivot_growth / refactored over all factorisations.
 * GDM_ERR_NOT_CONVERGED when max_iter is reached first (F then holds the last iterate). Synchronous. */
gdm_status gdm_solve_gmres(gdm_ctx *ctx, gdm_precision prec, const gdm_problem *p, const double *F0, double *F,
                           int n_rhs, const gdm_gmres_opts *opts, gdm_solve_info *info);

/* The host-side grouping gdm_solve_gmres applies (exposed for inspection and tests; host memory only,
 * no context, no GPU). Cells are put on the cubic lattice of step `step` (coordinates rounded relative
 * to the minimum corner) and sorted by the 3D Morton key of their lattice indices. perm (n int32):
 * permuted position -> original cell. parent (n int32): permuted cell -> coarse cell, the coarse cells
 * being the 2 x 2 x 2 lattice cubes in the same order; coarse_offsets (n + 1 int32, first *n_coarse + 1
 * used): first permuted cell of every coarse cell, then n. The block-Jacobi blocks are the runs
 * [b block_cells, (b + 1) block_cells) of the permuted order. GDM_ERR_INVALID_ARG on null pointers,
 * n outside [1, 2^26], a non-positive step or non-finite positions. */
gdm_status gdm_lattice_partition(const double *pos, int64_t n, double step, int block_cells, int32_t *perm,
                                 int32_t *parent, int32_t *coarse_offsets, int64_t *n_coarse);

/* ---------------------------------------------------------------- effective models */

/* Global polarizability matrix (GPM) of a discretised structure (Sec. "Effective
 * polarizabilities", GPM extraction; kind 3, in the problem's host): the structure is assembled into A
 * (as gdm_assemble), factored once and solved (FP64-refined) for n_pw plane waves and n_ds
 * local dipole sources; its scattered (E, H) at the n_probe probe positions are fitted in the
 * least-squares sense by electric and magnetic dipoles at the n_sites positions r_gpm (one
 * moment set per illumination); then alpha_eff (6M x 6M, M = n_sites) minimises
 * || alpha_eff F0 - P || over the illuminations, F0 the incident (E, H) at the sites and P the
 * fitted moments, i.e. alpha_eff = P F0^+.
 * A, lda, ipiv: matrix storage and pivots as for gdm_solve (overwritten).
 * r_gpm: device M x 3 (1 <= M <= 64). r_probe: device n_probe x 3 (n_probe >= M).
 * pw_khat: host n_pw x 3 unit directions; pw_e0: host n_pw x 3 complex128 amplitudes.
 * ds_pos: device n_ds x 3; ds_mom: device n_ds x 6 complex128 (p, m) source moments.
 * n_pw + n_ds <= 512 and >= 6 M. alpha_eff: device (6M) x (6M) complex128, column-major,
 * per site (E, H) -> (p, m) ordering. moments: device (6M) x (n_pw + n_ds) complex128 or NULL.
 * rel_fit: host, relative L2 residual of the moment fit, or NULL. Synchronous.
 * GDM_ERR_SINGULAR when the fit's normal matrix is not positive definite (too few or badly
 * placed probes or illuminations for the number of sites). */
gdm_status gdm_gpm_extract(gdm_ctx *ctx, gdm_precision prec, const gdm_problem *p, void *A, int64_t lda,
                           int32_t *ipiv, const double *r_gpm, int n_sites, const double *r_probe, int n_probe,
                           int n_pw, const double *pw_khat, const double *pw_e0, int n_ds, const double *ds_pos,
                           const double *ds_mom, double *alpha_eff, double *moments, double *rel_fit);

/* LU block-width autotuner (no paper counterpart). For each size class present in sizes
 * (system dimensions kind*n; classes <= 512, 1024, ..., 32768, larger), times the
 * factorisation of a synthetic well-conditioned complex64 matrix of the class's largest
 * size with outer block widths 128, 256 and 512, and keeps the fastest in the context
 * (used by gdm_solve, gdm_solve_batched and gdm_backward on this context). prec:
 * GDM_FP32 or GDM_TF32_REFINE. Allocates one scratch matrix of the largest size for the
 * duration of the call; synchronous. nb_out: host 8 ints (chosen width per class, 0 =
 * untouched), may be NULL. GDM_ERR_UNSUPPORTED when the GDM_LU_NB environment variable
 * fixes the width. */
gdm_status gdm_autotune(gdm_ctx *ctx, gdm_precision prec, const int64_t *sizes, int n_sizes, int *nb_out);

/* Outer block width of the grouped factorisation that gdm_solve_batched uses for a whole TF32
 * batch (no paper counterpart): times that factorisation (all problems in lock step, one
 * CUDA graph) on synthetic well-conditioned complex64 matrices of exactly the given system
 * dimensions sizes[0..n_sizes) (kind*n each, n_sizes >= 2) with widths 128, 256 and 512, and
 * keeps the fastest in the context. Allocates the matrices (sum of sizes^2 complex64) for the
 * duration of the call; synchronous. nb_out: host int, the chosen width, may be NULL.
 * GDM_ERR_UNSUPPORTED when the GDM_BATCH_NB environment variable fixes the width. */
gdm_status gdm_autotune_batched(gdm_ctx *ctx, const int64_t *sizes, int n_sizes, int *nb_out);

/* Residual r = F0 - A F of problem p for given fields F (FP64 result), computed matrix-free: the
 * Green dyads are regenerated for every pair (double-float arithmetic for cells, FP64 for ED/MD dipoles),
 * no stored matrix. This is the residual that drives gdm_solve's refinement (Eq. GDM_system_of_equations).
 * F0, F, r: device (kind*n) x n_rhs complex128; norms2: device n_rhs doubles receiving ||r_q||^2, or NULL. */
gdm_status gdm_residual(gdm_ctx *ctx, const gdm_problem *p, const double *F0, const double *F, int n_rhs, double *r,
                        double *norms2);

/* Near field by repropagation (Sec. "Observables"): at m points r_eval (device,
 * m x 3, none on a dipole), E = E0 + sum_j [G^Ep p_j + G^Em m_j] and
 * H = H0 + sum_j [G^Hp p_j + G^Hm m_j] with (p, m)_j = alpha_j F_j.
 * F: device solved fields (kind*n) x n_rhs complex128. F0_eval: device (6*m) x n_rhs
 * incident (E, H) at r_eval, or NULL for scattered fields only. E_out, H_out:
 * device (3*m) x n_rhs complex128; H_out may be NULL. */
gdm_status gdm_nearfield(gdm_ctx *ctx, const gdm_problem *p, const double *F, const double *r_eval,
                         int64_t m, const double *F0_eval, int n_rhs, double *E_out, double *H_out);

/* Cross sections (nm^2) per illumination, FP64:
 *   ext = 4 pi k / (eps_env |E0|^2) sum_i Im(E0_i^* . p_i + H0_i^* . m_i)
 *   abs = 4 pi k / (eps_env |E0|^2) sum_i Im(E_i^* . p_i)                      (kind 3)
 *   abs = 4 pi k / (eps_env |E0|^2) sum_i [Im(E_i^*.p_i) - 2/3 k^3/eps_env |p_i|^2
 *                                          + Im(H_i^*.m_i) - 2/3 k^3 |m_i|^2]  (kind 6)
 *   sca = ext - abs.
 * F0, F: device (kind*n) x n_rhs complex128. e0_norm2: host n_rhs values |E0|^2.
 * ext, sca, abs: device n_rhs doubles each (any may be NULL). */
gdm_status gdm_cross_sections(gdm_ctx *ctx, const gdm_problem *p, const double *F0, const double *F,
                              int n_rhs, const double *e0_norm2, double *ext, double *sca, double *abs);

/* Far-field scattering amplitudes (Sec. "Observables", scattering by repropagation of the dipoles
 * to infinity): the scattered field along rhat is f(rhat) exp(ikr)/r with
 *   f(rhat) = k^2/eps_env sum_j exp(-i k rhat.r_j) [p_j - rhat (rhat.p_j) - n_env rhat x m_j].
 * F: device (kind*n) x n_rhs solved fields. dirs: device q x 3 unit vectors. f_out: device
 * (3q) x n_rhs complex128. FP64. */
gdm_status gdm_farfield(gdm_ctx *ctx, const gdm_problem *p, const double *F, int n_rhs, const double *dirs,
                        int64_t q, double *f_out);

/* Scattering cross section from the far field: sigma_sca,ff = integral of |f|^2 over the unit
 * sphere / |E0|^2, with n_theta Gauss-Legendre nodes in cos(theta) times n_phi uniform azimuths
 * (the library builds the grid). For radiatively consistent models it equals sigma_ext -
 * sigma_abs; for cells it is the far-field value that gdm_cross_sections' sigma_sca (a
 * difference) approximates. e0_norm2: host n_rhs |E0|^2; sigma: device n_rhs doubles (nm^2). */
gdm_status gdm_sigma_farfield(gdm_ctx *ctx, const gdm_problem *p, const double *F, int n_rhs, const double *e0_norm2,
                              int n_theta, int n_phi, double *sigma);

/* Partial local density of states of the structured environment, normalised to the bare host
 * (Sec. "Observables": electric and magnetic LDOS; the decay-rate enhancement of a dipole
 * emitter): for unit dipoles along x, y, z at each of the n_pos positions r0, the structure
 * (kind 3) is solved under the emitter's field (one factorisation for all, FP64-refined) and
 * rho_u / rho_0 = 1 + 3 eps_env/(2 k^3) Im(u . E_sca(r0)), or 1 + 3/(2 k^3) Im(u . H_sca(r0))
 * when magnetic != 0 (emitted power over the host's c k0 k^3/(3 eps_env), resp. c k0 k^3/3).
 * A, lda, ipiv: storage as for gdm_solve (assembled and factored here). r0: device n_pos x 3
 * (1 <= n_pos <= 340, not on a cell). ldos: device n_pos x 3 doubles. Synchronous. */
gdm_status gdm_ldos(gdm_ctx *ctx, gdm_precision prec, const gdm_problem *p, void *A, int64_t lda, int32_t *ipiv,
                    const double *r0, int n_pos, int magnetic, double *ldos);

/* Largest ceil(n/256) * n_rhs that gdm_cross_sections_noalloc accepts: its fixed device
 * scratch holds this many (ext, abs) partial-sum pairs, 1 MiB per device. */
#define GDM_XSEC_NOALLOC_MAX_PARTS 65536

/* gdm_cross_sections without any device allocation. The paper has no counterpart: this is a
 * deployment variant with the same arguments and results as gdm_cross_sections (same
 * partial-sum kernel, same summation order). It is for callers that must not allocate device
 * memory: a step running while another allocator (a PyTorch caching allocator at its limit,
 * say) holds the free memory, or a latency-bound loop that cannot afford cudaMalloc/cudaFree,
 * which may synchronise the whole device. The partial sums live in one fixed file-scope device
 * buffer per device (GDM_XSEC_NOALLOC_MAX_PARTS pairs), and the prefactors are passed as a
 * kernel argument. The first call on each device looks up that buffer's address
 * (cudaGetSymbolAddress, with the context's device current); make it before any stream capture.
 * Nothing in the buffer needs to start at zero: every slot read is written earlier in the same
 * call. The buffer is shared by every context and stream of a device, so calls that overlap on
 * the GPU race on it: order them on one stream or synchronise in between.
 * Errors: as gdm_cross_sections, plus GDM_ERR_SHAPE when ceil(n/256) * n_rhs exceeds
 * GDM_XSEC_NOALLOC_MAX_PARTS (nothing is launched), and GDM_ERR_CUDA if the address lookup fails. */
gdm_status gdm_cross_sections_noalloc(gdm_ctx *ctx, const gdm_problem *p, const double *F0, const double *F,
                                      int n_rhs, const double *e0_norm2, double *ext, double *sca,
                                      double *abs);

/* Adjoint backward of gdm_solve + gdm_cross_sections for plane-wave illumination
 * (kind 3). Given the upstream gradient gF = dL/dF^* (device (3n) x n_rhs
 * complex128, conjugate Wirtinger derivative, may be NULL) and g_sigma (host
 * n_rhs x 3: dL/d(ext, sca, abs), may be NULL), solves A^H mu = g with the
 * factors held in A/ipiv (FP64-refined, matrix-free A^H residual), then ADDS to
 *   grad_pos  (device n x 3)        dL/dr
 *   grad_eps  (device n complex128) dL/dRe(eps) + i dL/dIm(eps)
 *   grad_wavelength (device 1 double) dL/dlambda0
 * (each may be NULL). e0: host n_rhs x 3 complex128, khat: host 3 doubles, the
 * plane waves that produced F0. info: host, may be NULL. */
gdm_status gdm_backward(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, const void *A, int64_t lda,
                        const int32_t *ipiv, const double *F, int n_rhs, const double *e0, const double *khat,
                        const double *gF, const double *g_sigma, double *grad_pos, double *grad_eps,
                        double *grad_wavelength, gdm_solve_info *info);

/* Backward of gdm_nearfield for plane-wave illumination (kind 3): given
 * gE = dL/dE_out^* (device (3m) x n_rhs complex128), ADDS the explicit
 * contributions to grad_pos, grad_eps, grad_wavelength (as in gdm_backward) and
 * ADDS dL/dF^* to gF_accum (device (3n) x n_rhs complex128), to be passed on to
 * gdm_backward. Any output may be NULL. */
gdm_status gdm_nearfield_backward(gdm_ctx *ctx, const gdm_problem *p, const double *F, const double *r_eval,
                                  int64_t m, int n_rhs, const double *e0, const double *khat, const double *gE,
                                  double *gF_accum, double *grad_pos, double *grad_eps, double *grad_wavelength);

/* ---------------------------------------------------------------- diagnostics */

/* Time every launch of the dominant kernel of the factorisation (the trailing update
 * A22 -= A21 U12 of the LU) with CUDA events on the context stream. enable = 1 clears the
 * record and starts recording; enable = 0 stops. Adds no synchronisation. */
gdm_status gdm_profile_enable(gdm_ctx *ctx, int enable);
/* Number of recorded launches, their summed device time (ms), summed algorithmic flops
 * (8 M N K per complex M x N x K update) and algorithmic bytes (read A21, U12, C; write C).
 * Synchronises the context stream. Any output pointer may be NULL. */
gdm_status gdm_profile_read(gdm_ctx *ctx, int64_t *launches, double *total_ms, double *flops, double *bytes);

/* Phase accounting: with enable = 1 subsequent calls record device time per phase of the solve
 * (CUDA events around each phase; adds host overhead, for diagnostics only). ms_out (host, 11 doubles,
 * nullable) receives the times recorded since the previous call, in the order: panel factorisation,
 * row interchanges, small triangular solves, in-block updates, U12 updates, trailing update,
 * correction solves (gdm_solve_gmres: its preconditioner), refinement residual (double-float
 * operator), other (gdm_solve_gmres: orthogonalisation), FP32 operator of gdm_solve_gmres, gradient
 * pair sums of gdm_backward (dG/dr, dG/dk).
 * Synchronises the stream when ms_out != NULL. */
gdm_status gdm_profile_phases(gdm_ctx *ctx, int enable, double *ms_out);

#ifdef __cplusplus
}
#endif
#endif /* GDM_H */
