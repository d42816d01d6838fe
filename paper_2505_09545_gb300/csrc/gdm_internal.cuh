// Internal declarations shared by the library's translation units.
// Nothing here is part of the public C ABI (include/gdm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "../../include/gdm.h"

// ------------------------------------------------------------------ context
#define GDM_NB_CLASSES 8  // system size classes: <= 512, 1024, 2048, ..., 32768, larger
#define GDM_POOL_MAX 16
struct gdm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    int max_smem_optin = 0;
    char err[512] = {0};
    int64_t launches = 0;
    // grow-only scratch arena owned by the context
    void *ws = nullptr;
    size_t ws_bytes = 0;
    // device-side error record: [0] first gdm_status, [1] detail, [2..3] grid-barrier counters
    int *dflags = nullptr;
    // pinned host mirror for synchronous reads of small device results
    void *hpinned = nullptr;
    size_t hpinned_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    // small parameter arrays copied from the host (stream-ordered); offset reset per API call
    char *dparams = nullptr;
    size_t param_off = 0;
    // optional event timing of the dominant kernel (gdm_profile_enable)
    int prof_on = 0;
    int prof_n = 0;
    cudaEvent_t *prof_ev = nullptr;  // 2 * GDM_PROF_MAX events, created lazily
    double prof_flops = 0.0, prof_bytes = 0.0;
    // phase accounting
    int ph_on = 0;
    int ph_n = 0;
    cudaEvent_t *ph_ev = nullptr;  // 2 * GDM_PH_MAX events
    int *ph_id = nullptr;
    // LU block width per size class (0 = built-in default), set by gdm_autotune
    int nb_table[GDM_NB_CLASSES] = {0};
    // child contexts of gdm_solve_batched (each owns its stream)
    gdm_ctx *pool[GDM_POOL_MAX] = {nullptr};
    int npool = 0;
    bool owns_stream = false;
    // schedule, tables and captured graph of the last grouped factorisation (batch_lu.cu), and its outer
    // block width (0 = built-in default), set by gdm_autotune_batched
    void *glu = nullptr;
    int glu_nb = 0;
    // tables and scratch of the last grouped refinement (batch_refine.cu)
    void *grf = nullptr;
    // SMs a Green-sum launch sizes its source split for (0: all): a child of the pool shares the GPU with
    // the other children running at the same time
    int share_sms = 0;
};
#define GDM_PH_MAX 32768
#define GDM_PROF_MAX 4096
// phase accounting (diagnostics): device time per phase, summed over bracketed regions
enum { GDM_PH_PANEL = 0, GDM_PH_LASWP, GDM_PH_TRSM, GDM_PH_INBLOCK, GDM_PH_U12, GDM_PH_TRAILING, GDM_PH_TRSV,
       GDM_PH_RESIDUAL, GDM_PH_OTHER, GDM_PH_OPERATOR_F32, GDM_PH_GRADIENT, GDM_NPHASES };
struct gdm_phase_rec;
gdm_status gdm_phase_begin(gdm_ctx *ctx, int phase);
gdm_status gdm_phase_end(gdm_ctx *ctx, int phase);
// bracket one launch of the profiled kernel (no-ops unless profiling is on)
gdm_status gdm_prof_begin(gdm_ctx *ctx, int *slot);
gdm_status gdm_prof_end(gdm_ctx *ctx, int slot, double flops, double bytes);
#define GDM_PARAM_BYTES (1 << 16)

// set the context error string, return the status
gdm_status gdm_fail(gdm_ctx *ctx, gdm_status s, const char *fmt, ...);

#define GDM_CUDA_TRY(ctx, call)                                                                       \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return gdm_fail((ctx), (e_ == cudaErrorMemoryAllocation) ? GDM_ERR_OOM : GDM_ERR_CUDA,    \
                            "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));      \
    } while (0)

// C++ exceptions (host containers, worker threads) must not cross the C ABI: entry points that use them
// wrap their body in GDM_GUARD_BEGIN ... GDM_GUARD_END(ctx), which turns an escaping exception into
// GDM_ERR_OOM with its message in the context
gdm_status gdm_host_exception(gdm_ctx *ctx);
#define GDM_GUARD_BEGIN try {
#define GDM_GUARD_END(ctx)                 \
    }                                      \
    catch (...) {                          \
        return gdm_host_exception(ctx);    \
    }

#define GDM_TRY(...)                       \
    do {                                   \
        gdm_status s_ = (__VA_ARGS__);     \
        if (s_ != GDM_OK) return s_;       \
    } while (0)

// check the last kernel launch, count it
gdm_status gdm_after_launch(gdm_ctx *ctx, const char *what);
#define GDM_LAUNCHED(ctx, what) GDM_TRY(gdm_after_launch((ctx), (what)))

// scratch arena: returns a pointer to >= bytes of device memory (256-B aligned),
// invalidating earlier pointers if it has to grow (it synchronises first).
gdm_status gdm_scratch(gdm_ctx *ctx, size_t bytes, void **ptr);
gdm_status gdm_pinned(gdm_ctx *ctx, size_t bytes, void **ptr);
// copy a small host array into the context's parameter buffer (stream-ordered); call
// gdm_params_reset at the start of each API call.
gdm_status gdm_upload(gdm_ctx *ctx, const void *host, size_t bytes, void **dev);
static inline void gdm_params_reset(gdm_ctx *ctx) { ctx->param_off = 0; }

// carve sub-buffers out of one scratch block
struct ScratchCarver {
    char *base;
    size_t off = 0;
    explicit ScratchCarver(void *b) : base((char *)b) {}
    template <class T> T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = (T *)(base + off);
        off += count * sizeof(T);
        return p;
    }
    static size_t round(size_t b) { return (b + 255) & ~size_t(255); }
};

// ------------------------------------------------------------------ device error flags
#define GDM_FLAG_STATUS 0
#define GDM_FLAG_DETAIL 1
#define GDM_FLAG_BAR_COUNT 2
#define GDM_FLAG_BAR_GEN 3
#define GDM_FLAG_GROWTH 4
#define GDM_FLAG_PANEL_TICKET 5  // finish counter of the panel kernels (returns to 0 after each launch)
#define GDM_FLAG_DIAG 6          // never written: the wait of gdm_diag_wait_timeout
#define GDM_NFLAGS 8

__device__ __forceinline__ void gdm_dev_error(int *flags, int status, int detail) {
    if (atomicCAS(&flags[GDM_FLAG_STATUS], 0, status) == 0) flags[GDM_FLAG_DETAIL] = detail;
}

// bounded spin limit for device waits (~ a second with nanosleep backoff)
#define GDM_SPIN_LIMIT (1 << 24)

// ------------------------------------------------------------------ complex helpers
struct cd {
    double x, y;
};
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {  // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }
// a += b * c
__host__ __device__ __forceinline__ void cfma(double2 &a, double2 b, double2 c) {
    a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
    a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}
__host__ __device__ __forceinline__ void cfma(float2 &a, float2 b, float2 c) {
    a.x = fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x));
    a.y = fmaf(b.x, c.y, fmaf(b.y, c.x, a.y));
}
// a -= b * c
__host__ __device__ __forceinline__ void cfms(double2 &a, double2 b, double2 c) {
    a.x = fma(-b.x, c.x, fma(b.y, c.y, a.x));
    a.y = fma(-b.x, c.y, fma(-b.y, c.x, a.y));
}
__host__ __device__ __forceinline__ void cfms(float2 &a, float2 b, float2 c) {
    a.x = fmaf(-b.x, c.x, fmaf(b.y, c.y, a.x));
    a.y = fmaf(-b.x, c.y, fmaf(-b.y, c.x, a.y));
}
__host__ __device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__host__ __device__ __forceinline__ float cabs1(float2 a) { return fabsf(a.x) + fabsf(a.y); }
__host__ __device__ __forceinline__ double2 crecip(double2 a) {
    double d = a.x * a.x + a.y * a.y;
    return make_double2(a.x / d, -a.y / d);
}
__host__ __device__ __forceinline__ float2 crecip(float2 a) {
    // scaled to avoid overflow of |a|^2 for large entries
    float s = fmaxf(fabsf(a.x), fabsf(a.y));
    float ax = a.x / s, ay = a.y / s;
    float d = ax * ax + ay * ay;
    return make_float2(ax / (d * s), -ay / (d * s));
}

template <class T> struct cplx;
template <> struct cplx<float> { typedef float2 t; };
template <> struct cplx<double> { typedef double2 t; };

// ------------------------------------------------------------------ internal launchers (defined per .cu)
// green.cu
gdm_status gdm_launch_planewave(gdm_ctx *ctx, const double *r, int64_t m, double k, double n_env, const double *e0,
                                const double *khat, int n_rhs, int kind_out, double *F0);
gdm_status gdm_launch_assemble(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, void *A, int64_t lda);
// residual r = F0 - A F (mode 0) or the adjoint residual r = g - A^H mu (mode 1), FP64 matrix-free.
// Writes r (kN x n_rhs) and, if norms != NULL, per-RHS ||r||^2 into norms[0..n_rhs).
gdm_status gdm_launch_residual(gdm_ctx *ctx, const gdm_problem *p, const double *rhs, const double *X, int n_rhs,
                               int adjoint, double *r, double *norms2);
gdm_status gdm_launch_nearfield(gdm_ctx *ctx, const gdm_problem *p, const double *F, const double *r_eval, int64_t m,
                                const double *F0_eval, int n_rhs, double *E_out, double *H_out);
gdm_status gdm_launch_cross_sections(gdm_ctx *ctx, const gdm_problem *p, const double *F0, const double *F, int n_rhs,
                                     const double *e0_norm2, double *ext, double *sca, double *abs);
gdm_status gdm_launch_farfield(gdm_ctx *ctx, const gdm_problem *p, const double *F, int n_rhs, const double *dirs,
                               int64_t q, double *f_out, const double *wts, const double *inv_e2, double *sigma);
gdm_status gdm_launch_gaussian(gdm_ctx *ctx, const double *r, int64_t m, double k, double n_env, double w0,
                               const double *focus, double theta, const double *e0, int n_rhs, int kind_out,
                               double *F0);
gdm_status gdm_launch_alpha6_lorentz(gdm_ctx *ctx, int64_t n, const double *w0e, const double *w0m, double gamma_ev,
                                     double amp_nm, double wavelength, double eps_env, double *out);
gdm_status gdm_launch_cross_sections_noalloc(gdm_ctx *ctx, const gdm_problem *p, const double *F0, const double *F,
                                             int n_rhs, const double *e0_norm2, double *ext, double *sca,
                                             double *abs);
// linear algebra (lu.cu)
// Factor A in place. global_pivot = 0: pivots searched inside each 32 x 32 diagonal block, with the
// largest |row below| / |pivot| ratio returned in *growth_out (<= 1: identical to partial pivoting);
// global_pivot = 1: partial pivoting over the whole column (cooperative panel kernel).
gdm_status gdm_lu_factor(gdm_ctx *ctx, gdm_precision prec, void *A, int64_t n, int64_t lda, int32_t *ipiv,
                         int global_pivot, float *growth_out);
// solve op(A) X = B in place on B (complex of the factor precision, n x n_rhs, ldb);
// conj_trans = 0: A X = B using P, L, U; conj_trans = 1: A^H X = B.
gdm_status gdm_lu_solve(gdm_ctx *ctx, gdm_precision prec, const void *A, int64_t n, int64_t lda, const int32_t *ipiv,
                        void *B, int64_t ldb, int n_rhs, int conj_trans);
// trsv.cu: persistent blocked solves (pivots must stay inside their row blocks) and the check for that
size_t gdm_trsv_sync_bytes(int64_t n);
gdm_status gdm_pivots_local(gdm_ctx *ctx, const int32_t *ipiv, int64_t n, int nbs, int *sync_buf, int *local);
gdm_status gdm_trsv_persistent(gdm_ctx *ctx, gdm_precision prec, const void *A, int64_t n, int64_t lda,
                               const int32_t *ipiv, void *B, int64_t ldb, int n_rhs, int conj_trans, int *sync_buf,
                               const void *dinv);
size_t gdm_trsv_inv_bytes(int64_t n);
gdm_status gdm_trsv_prepare(gdm_ctx *ctx, gdm_precision prec, const void *A, int64_t n, int64_t lda,
                            const int32_t *ipiv, void *dinv, int conj_trans);
int gdm_lu_block(const gdm_ctx *ctx, gdm_precision prec, int64_t n);
int gdm_size_class(int64_t n);
// refine.cu
gdm_status gdm_refined_solve(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, const void *A, int64_t lda,
                             const int32_t *ipiv, const double *rhs, double *X, int n_rhs, int adjoint,
                             const gdm_solve_opts *opts, gdm_solve_info *info);
// backward.cu
gdm_status gdm_launch_backward(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, const void *A, int64_t lda,
                               const int32_t *ipiv, const double *F, int n_rhs, const double *e0, const double *khat,
                               const double *gF, const double *g_sigma, double *grad_pos, double *grad_eps,
                               double *grad_wavelength, gdm_solve_info *info);
gdm_status gdm_launch_nearfield_backward(gdm_ctx *ctx, const gdm_problem *p, const double *F, const double *r_eval,
                                         int64_t m, int n_rhs, const double *e0, const double *khat, const double *gE,
                                         double *gF_accum, double *grad_pos, double *grad_eps,
                                         double *grad_wavelength);

// ------------------------------------------------------------------ grouped LU of a batch (batch_lu.cu)
// The problems of a batch are factored in lock step: every launch covers one step (a panel, or the trailing
// update of an outer block) of all problems that still have it, through a table sorted by decreasing size,
// so that the problems of a launch are a prefix of the table and the launch's work is split by a prefix sum
// of per-problem counts (CTA b belongs to problem i when prefix[i] <= b < prefix[i + 1]).
struct GluItem {
    float2 *A;
    int64_t lda, n;
    int32_t *ipiv;
    unsigned *growth;  // pivot certificate (float bits), as gdm_lu_factor's growth record
    int *status;       // [0] first error status, [1] detail (the layout of the context flags)
    int *ticket;       // finish counter of the panel kernels
    float *lx;         // TF32 embedding of the current outer block's L (rows from the block's first row on):
                       // real rows 2 (r - b0) and 2 (r - b0) + 1 of 2 nbo floats each
    void *pdiag;       // the current panel's factored diagonal block (U, reciprocal pivots) for its rows
};
struct alignas(64) GluMap {  // an encoded TMA descriptor (CUtensorMap)
    unsigned char bytes[128];
};
struct GluMaps {
    GluMap lx, b, c;  // A operand (the embedding of L), B operand and C chunks (both on the matrix)
};
enum { GLU_PANEL = 0, GLU_TRAIL = 1 };
#define GLU_SWAP_COLS 128  // columns per CTA of the grouped interchange and solve

// problem owning work unit b: the largest i in [0, na) with prefix[i] <= b (called by a whole warp; two rounds
// of 32 parallel probes cover 1024 problems, more rounds beyond)
__device__ __forceinline__ int glu_find_item(const int *__restrict__ prefix, int na, int b) {
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = na;
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) / 32;
        const int idx = lo + lane * step;
        const bool ok = idx < hi && __ldg(&prefix[idx]) <= b;
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        lo += (31 - __clz(m)) * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// Regions of C updated by one grouped GEMM launch for a problem of order n (complex rows x columns):
//   GLU_PANEL after the 32-column panel at c0 of the block [b0, b0 + nbo): the block's columns right of the
//     panel, all rows below it (A: Ma x Na), and the block's rows below the panel, columns right of the block
//     (B: Mb x Nb); both with K = 32 (the panel). The C block right of and below the outer block waits for
//   GLU_TRAIL after the block: rows and columns right of it (A: Ma x Na, K = nbo).
__host__ __device__ inline void glu_regions(int kind, int64_t n, int64_t b0, int64_t c0, int nbo, int64_t &Ma,
                                            int64_t &Na, int64_t &Mb, int64_t &Nb) {
    if (kind == GLU_PANEL) {
        const int64_t be = (b0 + nbo < n) ? b0 + nbo : n, base = c0 + 32;
        Ma = n - base;
        Na = be - base;
        Mb = Na;
        Nb = n - be;
    } else {
        Ma = Na = n - (b0 + nbo);
        Mb = Nb = 0;
    }
    if (Ma <= 0 || Na <= 0) Ma = Na = 0;
    if (Mb <= 0 || Nb <= 0) Mb = Nb = 0;
}
// 128 x 256 tiles of the real embedding (2M real rows) of a region
__host__ __device__ inline int glu_region_tiles(int64_t M, int64_t N) {
    return (M > 0 && N > 0) ? (int)((2 * M + 127) / 128) * (int)((N + 255) / 256) : 0;
}
__host__ __device__ inline int glu_tiles(int kind, int64_t n, int64_t b0, int64_t c0, int nbo) {
    int64_t Ma, Na, Mb, Nb;
    glu_regions(kind, n, b0, c0, nbo, Ma, Na, Mb, Nb);
    return glu_region_tiles(Ma, Na) + glu_region_tiles(Mb, Nb);
}
// tile t of a problem: real-row tile mt, first column col0 (relative to the region origin, which is the
// launch's base row and column) and width ncols, real rows below mlim updated. Inside a region, groups of 8
// column tiles with the row tile varying slowest across a group's columns (operand tiles shared in L2).
struct GluTile {
    int mt, col0, ncols, mlim;
};
__host__ __device__ inline GluTile glu_tile(int kind, int64_t n, int64_t b0, int64_t c0, int nbo, int t) {
    int64_t Ma, Na, Mb, Nb;
    glu_regions(kind, n, b0, c0, nbo, Ma, Na, Mb, Nb);
    const int tA = glu_region_tiles(Ma, Na);
    int64_t M = Ma, N = Na, off = 0;
    if (t >= tA) {
        t -= tA;
        M = Mb;
        N = Nb;
        off = Na;
    }
    const int num_m = (int)((2 * M + 127) / 128), num_n = (int)((N + 255) / 256);
    const int per_group = num_m * 8, g = t / per_group, idx = t - g * per_group;
    const int gn = (num_n - g * 8) < 8 ? (num_n - g * 8) : 8;
    const int nt = g * 8 + idx % gn;
    GluTile r;
    r.mt = idx / gn;
    r.col0 = (int)(off + (int64_t)nt * 256);
    r.ncols = (int)((N - (int64_t)nt * 256) < 256 ? (N - (int64_t)nt * 256) : 256);
    r.mlim = (int)(2 * M);
    return r;
}
// launches of the grouped LU (lu.cu, lu_tc.cu)
gdm_status gdm_glu_panel(gdm_ctx *ctx, const GluItem *items, const int *prefix, int na, int nblocks, int64_t b0,
                         int64_t c0, int nbo);
gdm_status gdm_glu_swap_trsm(gdm_ctx *ctx, const GluItem *items, const int *prefix, int na, int nblocks,
                             int64_t c0);
gdm_status gdm_glu_gemm(gdm_ctx *ctx, const GluItem *items, const GluMaps *maps, const int *prefix, int na,
                        int ntiles, int kind, int64_t b0, int64_t c0, int nbo);
gdm_status gdm_glu_gemm_init(gdm_ctx *ctx);
gdm_status gdm_glu_panel_init(gdm_ctx *ctx);
gdm_status gdm_glu_diag(gdm_ctx *ctx, const GluItem *items, int na, int64_t b0, int64_t c0, int nbo);
gdm_status gdm_glu_rows(gdm_ctx *ctx, const GluItem *items, const int *prefix, int na, int nblocks, int64_t b0,
                        int64_t c0, int nbo);
size_t gdm_glu_pdiag_bytes();
// encodes the tensor maps of every problem (host); false if the driver's encoder is unavailable or refuses
bool gdm_glu_encode(const GluItem *items, int n_items, int nbo, GluMaps *maps);
// the grouped factorisation of a batch (batch_lu.cu) and the release of its cached schedule
gdm_status gdm_glu_factor(gdm_ctx *ctx, int n_items, float2 *const *A, const int64_t *lda, const int64_t *n,
                          int32_t *const *ipiv, int nbo, float *growth, int *status, float *ms);
void gdm_glu_release(gdm_ctx *ctx);

// ------------------------------------------------------------------ grouped refinement of a batch (batch_refine.cu)
// Cells (kind 3) with at most two right-hand sides, factored by the grouped LU: every refinement step of
// all problems still refining runs as one launch per kernel, the problems' work units split by a prefix
// sum over a list of problem indices (CTA b works for problem list[k] when prefix[k] <= b < prefix[k + 1]).
struct GrItem {
    int64_t n;        // cells; the system has 3n rows
    int nr;           // right-hand sides (1 or 2)
    int nblk;         // 128-row blocks of the system
    const double *pos;
    const double2 *eps;
    double eps_env, d3_4pi, self_S;
    float kk[6];                // k, k^2 and 1/eps_env as FP32 (hi, lo) pairs (double-float sums)
    float khi, klo, inv_eps;    // the FP32 sums' wavenumber pair and 1/eps_env
    const float2 *A;            // factors
    int64_t lda;
    const int32_t *ipiv;        // their pivots (inside 32-row panels)
    const double2 *rhs;         // (3n) x nr
    double2 *X;                 // (3n) x nr solution
    double2 *r, *P, *partial;   // residual, moments, Green-sum partials (nc x 2 x n x 3)
    float2 *w;                  // work vector of the triangular solves, (3n) x nr
    void *dip;                  // FP32-pair positions (48-byte records)
    float *rec;                 // double-float source records of the residual
    float2 *ops;                // block operators, 4 planes of 128 x 128 per block
    int *sync;                  // triangular-solve flags (nblk + 2)
    double *norms;              // [2q] ||d_q||^2, [2q + 1] ||X_q||^2, [4 + q] ||r_q||^2, [6 + q] ||rhs_q||^2
    int64_t chunk;              // sources per Green-sum chunk
    int nc;                     // chunks
    // inputs and observables (batches of cells solved wholly in lock step)
    double k, n_env;            // host wavenumber and refractive index
    double e0[12];              // plane-wave amplitudes (x, y, z complex per right-hand side)
    double khat[3];             // propagation direction
    int has_e0;                 // 1: F0 is the plane wave (written), 0: F0 is given
    int has_sigma;
    void *dipa;                 // FP32 assembly records (positions, alpha, diagonal block)
    double *sigma;              // 3 x nr cross sections (ext row, sca row, abs row), device, or unused
    double pref[2];             // 4 pi k / (eps_env |E0_q|^2)
    double *xs;                 // [2q] sum Im(E0* . p), [2q + 1] sum Im(E* . p)
};
#define TRSV_OPS_CTAS 4  // CTAs per 128-row block of the block-operator kernel (both triangles)
// problem of work unit b of a grouped launch: k with prefix[k] <= b < prefix[k + 1] (whole CTA; uses a warp)
__device__ __forceinline__ int gr_unit(const int *__restrict__ list, const int *__restrict__ prefix, int na, int b,
                                       int *local) {
    __shared__ int s_k;
    if (threadIdx.x < 32) {
        const int k = glu_find_item(prefix, na, b);
        if (threadIdx.x == 0) s_k = k;
    }
    __syncthreads();
    const int k = s_k;
    *local = b - __ldg(&prefix[k]);
    return __ldg(&list[k]);
}
// grouped launches (green.cu, green_ff.cu, trsv.cu, refine.cu); units per problem as their comments say
gdm_status gdm_gr_prep_dip(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units);
gdm_status gdm_gr_moments(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units);
gdm_status gdm_gr_green_f32(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units);
gdm_status gdm_gr_prep_src(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units);
gdm_status gdm_gr_green_ff(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units,
                           const void *tab);
gdm_status gdm_gr_finalize(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units);
gdm_status gdm_gr_block_ops(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units);
gdm_status gdm_gr_trsv(gdm_ctx *ctx, const GrItem *it, const void *maps, const int *list, const int *jprefix,
                       int nj, int units, int mode, int *ticket);
gdm_status gdm_gr_norm2(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units);
gdm_status gdm_gr_to_work(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units,
                          int from_r);
gdm_status gdm_gr_update(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units,
                         int accumulate);
// one problem of a grouped refinement (host view) and the refinement itself (batch_refine.cu): solves
// A F = F0 for every problem with the factors in A, ipiv, refined to max_q ||dF_q|| / ||F_q|| <= tol within
// max_iter steps; fills infos (iterations, rel_correction, rel_residual, refine_ms, status per problem:
// GDM_OK, GDM_ERR_NOT_CONVERGED or GDM_ERR_NONFINITE). Returns a failure of the call itself only.
struct GrProblem {
    const gdm_problem *p;
    float2 *A;
    int64_t lda;
    const int32_t *ipiv;
    double *F0;
    double *F;
    int n_rhs;
    const double *e0;        // host plane-wave amplitudes (n_rhs x 3 complex), or NULL when F0 is given
    const double *khat;      // host direction (NULL: +z)
    const double *e0_norm2;  // host |E0_q|^2 when e0 is NULL (for the cross sections)
    double *sigma;           // device 3 x n_rhs cross sections, or NULL
};
// gdm_gr_prepare: the table of this call's problems (kept with its scratch while the sizes stay the same);
// gdm_gr_inputs: plane waves (problems with e0) and the FP32 assembly of every problem of the table;
// gdm_gr_refine: the refinement of the problems with use[i] != 0 (caller's order; A holds their factors);
// gdm_gr_xsec: their cross sections (problems with sigma)
gdm_status gdm_gr_prepare(gdm_ctx *ctx, int n_items, const GrProblem *pb);
gdm_status gdm_gr_inputs(gdm_ctx *ctx);
gdm_status gdm_gr_refine(gdm_ctx *ctx, const unsigned char *use, double tol, int max_iter, int flags,
                         gdm_solve_info *infos);
gdm_status gdm_gr_xsec(gdm_ctx *ctx, const unsigned char *use);
gdm_status gdm_gr_planewave(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units);
gdm_status gdm_gr_prep_dipa(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units);
gdm_status gdm_gr_assemble(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units);
gdm_status gdm_gr_xsec_partial(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na,
                               int units);
gdm_status gdm_gr_xsec_final(gdm_ctx *ctx, const GrItem *it, const int *list, int na);
void gdm_gr_release(gdm_ctx *ctx);
// host: the TMA descriptor of a problem's factors for the triangular solves (128 bytes into map); false if
// the encoder refuses
bool gdm_trsv_encode_map(const float2 *A, int64_t n, int64_t lda, void *map);
// fills dev_tab (257 x 16 bytes, device) with the phase-reduction table of the double-float sums
gdm_status gdm_ff_table_fill(gdm_ctx *ctx, void *dev_tab);

// problem helpers
static inline double gdm_k0(const gdm_problem *p) { return 2.0 * 3.14159265358979323846 / p->wavelength; }

// shared by gdm_solve and gdm_solve_batched (defined in the C-ABI translation unit)
extern "C" __attribute__((visibility("hidden"))) gdm_status gdm_check_solve_args(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, const void *A, int64_t lda,
                                const int32_t *ipiv, const double *F0, const double *F, int n_rhs);
extern "C" __attribute__((visibility("hidden"))) gdm_status gdm_solve_core(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, void *A, int64_t lda,
                                     int32_t *ipiv, const double *F0, double *F, int n_rhs,
                                     const gdm_solve_opts *opts, gdm_solve_info *info);
