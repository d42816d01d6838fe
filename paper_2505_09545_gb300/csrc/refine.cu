// Mixed-precision iterative refinement of the GDM solve.
//
// X_0 = LU^{-1} b in the factor precision; then repeat
//   r = b - A X          (matrix-free: the Green dyads are regenerated per pair, never stored)
//   d = LU^{-1} r        (factor precision)
//   X = X + d            (FP64)
// until max_q ||d_q|| / ||X_q|| <= tol (or, with GDM_SOLVE_ERR_ESTIMATE, until the error estimate from the
// contraction of the last two corrections is). The adjoint variant solves A^H X = b with the same factors
// (conjugate-transposed triangular solves) and the matrix-free residual b - A^H X.
// Residual arithmetic: double-float (pairs of FP32 on the FP32 pipes, about 48 significand bits; the
// GB300 FP64 pipe runs at ~1/64 of the FP32 rate), which matches the oracle's FP64 residual to ~1e-13 of
// its largest term, four orders inside the 1e-9 field tolerance. GDM_RESIDUAL_FP64 selects FP64 Green sums
// instead (and the adjoint of ED/MD dipoles always uses them). For cells with TF32 factors the residuals of
// the first steps, while the last relative correction is above 1e-3, are FP32 Green sums (double-float
// phase, ~1e-6 relative, ~1/6 of the double-float work): the correction they yield is then accurate to
// ~1e-2 relative, below the factorisation's own contraction (~0.03 per step), so they cost no extra step;
// every later residual, which decides the accuracy and the stop, is double-float.
// Scaling: each right-hand side of a low-precision triangular solve (b, then every r) is multiplied by the
// power of two that brings its largest column norm near 1, and the correction is scaled back in FP64, so
// that a residual far below the FP32 range (a weak illumination, a late refinement step) is not flushed to
// zero. The scale is computed on the device from the norms the previous kernels accumulated.
#include <math.h>
#include <stdlib.h>

#include "gdm_internal.cuh"

gdm_status gdm_launch_residual_ws(gdm_ctx *ctx, const gdm_problem *p, const double *rhs, const double *X, int n_rhs,
                                  int adjoint, double *r, double *norms2, double2 *Pbuf, double2 *partial, void *ffws,
                                  int ff_prepare);
size_t gdm_ff_scratch_bytes(int64_t n);
size_t gdm_green_partial_bytes(gdm_ctx *ctx, int64_t m, int64_t n, int out);
gdm_status gdm_ff_prepare(gdm_ctx *ctx, const gdm_problem *p, void *ffws);
const void *gdm_ff_positions(void *ffws);
gdm_status gdm_launch_residual_f32(gdm_ctx *ctx, const gdm_problem *p, const double *rhs, const double *X, int n_rhs,
                                   double *r, double *norms2, double2 *Pbuf, double2 *partial, const void *dipf);

// power of two that brings the largest of the n_rhs column norms (given squared) near 1; 1 if they are
// all zero or not finite. Exact in every precision, so scaling by it loses nothing.
__device__ __forceinline__ double work_scale(const double *__restrict__ norms2, int n_rhs) {
    double m = 0.0;
    for (int q = 0; q < n_rhs; q++) m = fmax(m, norms2[q]);
    if (!(m > 0.0) || !isfinite(m)) return 1.0;
    return ldexp(1.0, -ilogb(sqrt(m)));
}

template <class C>
__global__ void k_to_work(const double2 *__restrict__ src, C *__restrict__ dst, int64_t count,
                          const double *__restrict__ norms2, int n_rhs) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double scale = work_scale(norms2, n_rhs);
    C v;
    v.x = src[i].x * scale;
    v.y = src[i].y * scale;
    dst[i] = v;
}

// X (+)= d/scale ; accumulate ||d||^2 and ||X||^2 per RHS; flag non-finite values
template <class C>
__global__ void k_update(double2 *__restrict__ X, const C *__restrict__ d, int64_t ld, int n_rhs, int accumulate,
                         const double *__restrict__ scale_norms2, double *__restrict__ norms, int *flags) {
    int q = blockIdx.y;
    const double inv_scale = 1.0 / work_scale(scale_norms2, n_rhs);
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double dn = 0.0, xn = 0.0;
    if (i < ld) {
        C dv = d[q * ld + i];
        double dx = dv.x * inv_scale, dy = dv.y * inv_scale;
        double2 x = accumulate ? X[q * ld + i] : make_double2(0.0, 0.0);
        x.x += dx;
        x.y += dy;
        X[q * ld + i] = x;
        dn = dx * dx + dy * dy;
        xn = x.x * x.x + x.y * x.y;
        if (!isfinite(xn)) gdm_dev_error(flags, GDM_ERR_NONFINITE, (int)i);
    }
    for (int o = 16; o > 0; o >>= 1) {
        dn += __shfl_down_sync(0xffffffffu, dn, o);
        xn += __shfl_down_sync(0xffffffffu, xn, o);
    }
    __shared__ double rd[32], rx[32];
    if ((threadIdx.x & 31) == 0) {
        rd[threadIdx.x >> 5] = dn;
        rx[threadIdx.x >> 5] = xn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            dn += rd[w];
            xn += rx[w];
        }
        atomicAdd(&norms[2 * q], dn);
        atomicAdd(&norms[2 * q + 1], xn);
    }
}

__global__ void k_norm2(const double2 *__restrict__ v, int64_t ld, double *__restrict__ out) {
    int q = blockIdx.y;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < ld) {
        double2 x = v[q * ld + i];
        s = x.x * x.x + x.y * x.y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double r[32];
    if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) s += r[w];
        atomicAdd(&out[q], s);
    }
}

// ---------------------------------------------------------------- grouped refinement steps of a batch
// (every kernel: ceil(3n nr / 256) CTAs of 256 per listed problem, element e = q (3n) + row)
namespace {
__device__ __forceinline__ void block_sum2(double &a, double &b, double *red) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[2 * w] = a;
        red[2 * w + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 1; k < (int)(blockDim.x >> 5); k++) {
            a += red[2 * k];
            b += red[2 * k + 1];
        }
}

// ||rhs_q||^2 into norms[6 + q]
__global__ void __launch_bounds__(256) k_gr_norm2(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                  const int *__restrict__ prefix, int na) {
    __shared__ double red[16];
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const GrItem &g = items[i];
    const int64_t ld = 3 * g.n, e0 = (int64_t)local * 256;
    const int64_t e = e0 + threadIdx.x;
    const int q = (int)(e0 / ld);  // a CTA spans at most one column boundary: split its sum by column
    double a = 0.0, b = 0.0;
    if (e < ld * g.nr) {
        const double2 v = g.rhs[e];
        const double s2 = v.x * v.x + v.y * v.y;
        if (e / ld == q) a = s2;
        else b = s2;
    }
    block_sum2(a, b, red);
    if (threadIdx.x == 0) {
        atomicAdd(&g.norms[6 + q], a);
        if (b != 0.0) atomicAdd(&g.norms[6 + q + 1], b);
    }
}

// w = (r or rhs) x the power of two that brings the largest column norm near 1
__global__ void __launch_bounds__(256) k_gr_to_work(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                    const int *__restrict__ prefix, int na, int from_r) {
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const GrItem &g = items[i];
    const int64_t e = (int64_t)local * 256 + threadIdx.x;
    if (e >= 3 * g.n * g.nr) return;
    const double scale = work_scale(g.norms + (from_r ? 4 : 6), g.nr);
    const double2 v = from_r ? g.r[e] : g.rhs[e];
    g.w[e] = make_float2((float)(v.x * scale), (float)(v.y * scale));
}

// X (+)= w / scale; ||d_q||^2 into norms[2q], ||X_q||^2 into norms[2q + 1]
__global__ void __launch_bounds__(256) k_gr_update(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                   const int *__restrict__ prefix, int na, int accumulate) {
    __shared__ double red[16];
    __shared__ double red2[16];
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const GrItem &g = items[i];
    const int64_t ld = 3 * g.n, e0 = (int64_t)local * 256;
    const int64_t e = e0 + threadIdx.x;
    const int q = (int)(e0 / ld);
    const double inv_scale = 1.0 / work_scale(g.norms + (accumulate ? 4 : 6), g.nr);
    double dn0 = 0.0, dn1 = 0.0, xn0 = 0.0, xn1 = 0.0;
    if (e < ld * g.nr) {
        const float2 dv = g.w[e];
        const double dx = dv.x * inv_scale, dy = dv.y * inv_scale;
        double2 x = accumulate ? g.X[e] : make_double2(0.0, 0.0);
        x.x += dx;
        x.y += dy;
        g.X[e] = x;
        const double d2 = dx * dx + dy * dy, x2 = x.x * x.x + x.y * x.y;
        if (e / ld == q) {
            dn0 = d2;
            xn0 = x2;
        } else {
            dn1 = d2;
            xn1 = x2;
        }
    }
    block_sum2(dn0, dn1, red);
    block_sum2(xn0, xn1, red2);
    if (threadIdx.x == 0) {
        atomicAdd(&g.norms[2 * q], dn0);
        atomicAdd(&g.norms[2 * q + 1], xn0);
        if (dn1 != 0.0 || xn1 != 0.0) {
            atomicAdd(&g.norms[2 * q + 2], dn1);
            atomicAdd(&g.norms[2 * q + 3], xn1);
        }
    }
}
}  // namespace

gdm_status gdm_gr_norm2(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units) {
    if (units <= 0) return GDM_OK;
    k_gr_norm2<<<(unsigned)units, 256, 0, ctx->stream>>>(it, list, prefix, na);
    GDM_LAUNCHED(ctx, "gr_norm2");
    return GDM_OK;
}

gdm_status gdm_gr_to_work(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units,
                          int from_r) {
    if (units <= 0) return GDM_OK;
    k_gr_to_work<<<(unsigned)units, 256, 0, ctx->stream>>>(it, list, prefix, na, from_r);
    GDM_LAUNCHED(ctx, "gr_to_work");
    return GDM_OK;
}

gdm_status gdm_gr_update(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units,
                         int accumulate) {
    if (units <= 0) return GDM_OK;
    k_gr_update<<<(unsigned)units, 256, 0, ctx->stream>>>(it, list, prefix, na, accumulate);
    GDM_LAUNCHED(ctx, "gr_update");
    return GDM_OK;
}

template <class C>
static gdm_status refined_t(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, const void *A, int64_t lda,
                            const int32_t *ipiv, const double *rhs, double *X, int n_rhs, int adjoint,
                            const gdm_solve_opts *opts, gdm_solve_info *info) {
    const int64_t ns = p->n * p->kind;
    const int64_t cnt = ns * n_rhs;
    size_t need = ScratchCarver::round(cnt * sizeof(double2)) * 2 + ScratchCarver::round(cnt * sizeof(C)) +
                  ScratchCarver::round(gdm_green_partial_bytes(ctx, p->n, p->n, p->kind)) +
                  ScratchCarver::round(sizeof(double) * 4 * n_rhs) + ScratchCarver::round(gdm_trsv_sync_bytes(ns)) +
                  ScratchCarver::round(gdm_trsv_inv_bytes(ns)) + ScratchCarver::round(gdm_ff_scratch_bytes(p->n)) +
                  4096;
    // the LU scratch is not needed any more: the refinement reuses the arena
    void *ws;
    GDM_TRY(gdm_scratch(ctx, need, &ws));
    ScratchCarver sc(ws);
    double2 *r = sc.take<double2>(cnt);
    double2 *Pbuf = sc.take<double2>(cnt);
    C *w = sc.take<C>(cnt);
    double2 *partial = sc.take<double2>(gdm_green_partial_bytes(ctx, p->n, p->n, p->kind) / sizeof(double2));
    double *dnorm = sc.take<double>(4 * n_rhs);
    int *tsync = sc.take<int>(gdm_trsv_sync_bytes(ns) / sizeof(int));
    void *dinv = sc.take<char>(gdm_trsv_inv_bytes(ns));
    // double-float residual unless GDM_RESIDUAL_FP64 is set (the adjoint residual of ED/MD dipoles is not built)
    void *ffws = (!getenv("GDM_RESIDUAL_FP64") && (p->kind == 3 || !adjoint)) ? sc.take<char>(gdm_ff_scratch_bytes(p->n))
                                                                               : nullptr;
    double *hn;
    GDM_TRY(gdm_pinned(ctx, sizeof(double) * 4 * n_rhs, (void **)&hn));
    // TF32 and BF16 factors only: their first solution is off by ~1e-2; FP32 (3-product) and FP64 factors start
    // closer than the FP32 residual resolves
    const bool fast_ok = ffws && p->kind == 3 && !adjoint && (prec == GDM_TF32_REFINE || prec == GDM_BF16_REFINE) &&
                         !getenv("GDM_REFINE_EXACT");
    bool ff_prepared = false;
    const unsigned nb = (unsigned)((ns + 255) / 256);
    const dim3 gq(nb, (unsigned)n_rhs);
    // ||b||^2 for the relative residual
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(dnorm, 0, sizeof(double) * 4 * n_rhs, ctx->stream));
    k_norm2<<<gq, 256, 0, ctx->stream>>>((const double2 *)rhs, ns, dnorm + 3 * n_rhs);
    GDM_LAUNCHED(ctx, "norm2");
    // persistent block solves when every pivot stays inside its row block
    int local = 0;
    if (prec != GDM_FP64 && !getenv("GDM_TRSV_LAUNCHES")) GDM_TRY(gdm_pivots_local(ctx, ipiv, ns, 32, tsync, &local));
    if (local) GDM_TRY(gdm_trsv_prepare(ctx, prec, A, ns, lda, ipiv, dinv, adjoint));
    auto lu_solve = [&](void *w) -> gdm_status {
        GDM_TRY(gdm_phase_begin(ctx, GDM_PH_TRSV));
        gdm_status st = local ? gdm_trsv_persistent(ctx, prec, A, ns, lda, ipiv, w, ns, n_rhs, adjoint, tsync, dinv)
                              : gdm_lu_solve(ctx, prec, A, ns, lda, ipiv, w, ns, n_rhs, adjoint);
        GDM_TRY(st);
        return gdm_phase_end(ctx, GDM_PH_TRSV);
    };
    if (info) GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
    // initial solve
    k_to_work<C><<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>((const double2 *)rhs, w, cnt,
                                                                         dnorm + 3 * n_rhs, n_rhs);
    GDM_LAUNCHED(ctx, "to_work");
    GDM_TRY(lu_solve(w));
    k_update<C><<<gq, 256, 0, ctx->stream>>>((double2 *)X, w, ns, n_rhs, 0, dnorm + 3 * n_rhs, dnorm, ctx->dflags);
    GDM_LAUNCHED(ctx, "update");
    int it = 0;
    double relc = 1.0, relr = -1.0, prev = -1.0, stop = 1.0;
    if (!(opts->flags & GDM_SOLVE_NO_REFINE)) {
        for (it = 1; it <= opts->max_iter; it++) {
            GDM_CUDA_TRY(ctx, cudaMemsetAsync(dnorm, 0, sizeof(double) * 3 * n_rhs, ctx->stream));
            GDM_TRY(gdm_phase_begin(ctx, GDM_PH_RESIDUAL));
            if (fast_ok && relc > 1e-3) {
                if (!ff_prepared) GDM_TRY(gdm_ff_prepare(ctx, p, ffws));
                ff_prepared = true;
                GDM_TRY(gdm_launch_residual_f32(ctx, p, rhs, X, n_rhs, (double *)r, dnorm + 2 * n_rhs, Pbuf, partial,
                                                gdm_ff_positions(ffws)));
            } else {
                GDM_TRY(gdm_launch_residual_ws(ctx, p, rhs, X, n_rhs, adjoint, (double *)r, dnorm + 2 * n_rhs, Pbuf,
                                               partial, ffws, ffws && !ff_prepared));
                ff_prepared = ffws != nullptr;
            }
            GDM_TRY(gdm_phase_end(ctx, GDM_PH_RESIDUAL));
            // scale the residual into a safe FP32 range before the low-precision solve (by its own norms,
            // accumulated by the residual kernel), and the correction back
            k_to_work<C><<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(r, w, cnt, dnorm + 2 * n_rhs, n_rhs);
            GDM_LAUNCHED(ctx, "to_work");
            GDM_TRY(lu_solve(w));
            k_update<C><<<gq, 256, 0, ctx->stream>>>((double2 *)X, w, ns, n_rhs, 1, dnorm + 2 * n_rhs, dnorm,
                                                     ctx->dflags);
            GDM_LAUNCHED(ctx, "update");
            GDM_CUDA_TRY(ctx, cudaMemcpyAsync(hn, dnorm, sizeof(double) * 4 * n_rhs, cudaMemcpyDeviceToHost,
                                              ctx->stream));
            GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            prev = it > 1 ? relc : -1.0;
            relc = 0.0;
            relr = 0.0;
            bool finite = true;
            for (int q = 0; q < n_rhs; q++) {
                double dq = hn[2 * q], xq = hn[2 * q + 1], rq = hn[2 * n_rhs + q], bq = hn[3 * n_rhs + q];
                if (!isfinite(dq) || !isfinite(xq) || !isfinite(rq)) finite = false;
                double c = xq > 0 ? sqrt(dq / xq) : (dq > 0 ? INFINITY : 0.0);
                double rr = bq > 0 ? sqrt(rq / bq) : 0.0;
                if (c > relc) relc = c;
                if (rr > relr) relr = rr;
            }
            if (!finite) {
                // collect (and clear) the device record too: a singular pivot found by the factorisation is
                // the cause to report, and must not surface in the context's next call
                gdm_status dev = gdm_ctx_check(ctx);
                gdm_status st = dev != GDM_OK ? dev : GDM_ERR_NONFINITE;
                if (info) {
                    info->iterations = it;
                    info->status = st;
                }
                return gdm_fail(ctx, st, "non-finite values in the refined solution (%s)", gdm_status_string(st));
            }
            stop = gdm_refine_stop_measure(relc, prev, opts->flags);
            if (stop <= opts->tol) break;
        }
        if (it > opts->max_iter) it = opts->max_iter;
    }
    if (info) {
        GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev2, ctx->stream));
        GDM_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev2));
        float ms = 0.f;
        GDM_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev1, ctx->ev2));
        info->refine_ms = ms;
        info->iterations = (opts->flags & GDM_SOLVE_NO_REFINE) ? 0 : it;
        info->rel_correction = relc;
        info->rel_residual = relr;
    }
    if (!(opts->flags & GDM_SOLVE_NO_REFINE)) {
        // the loop synchronised the stream already: collect device-side errors of the whole solve
        gdm_status dev = gdm_ctx_check(ctx);
        if (info) info->status = dev;
        if (dev != GDM_OK) return dev;
        if (stop > opts->tol) {
            if (info) info->status = GDM_ERR_NOT_CONVERGED;
            return gdm_fail(ctx, GDM_ERR_NOT_CONVERGED, "refinement stopped at relative correction %.3e > tol %.3e",
                            relc, opts->tol);
        }
    }
    return GDM_OK;
}

gdm_status gdm_refined_solve(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, const void *A, int64_t lda,
                             const int32_t *ipiv, const double *rhs, double *X, int n_rhs, int adjoint,
                             const gdm_solve_opts *opts, gdm_solve_info *info) {
    if (prec == GDM_FP64) return refined_t<double2>(ctx, p, prec, A, lda, ipiv, rhs, X, n_rhs, adjoint, opts, info);
    return refined_t<float2>(ctx, p, prec, A, lda, ipiv, rhs, X, n_rhs, adjoint, opts, info);
}
