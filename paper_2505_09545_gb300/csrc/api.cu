// C-ABI entry points: context management, argument validation, dispatch.
#include <math.h>
#include <stdarg.h>

#include <exception>
#include <new>
#include <vector>

#include "gdm_internal.cuh"

#include <stdlib.h>

size_t gdm_ff_scratch_bytes(int64_t n);
size_t gdm_green_partial_bytes(gdm_ctx *ctx, int64_t m, int64_t n, int out);
gdm_status gdm_launch_residual_ws(gdm_ctx *ctx, const gdm_problem *p, const double *rhs, const double *X, int n_rhs,
                                  int adjoint, double *r, double *norms2, double2 *Pbuf, double2 *partial, void *ffws,
                                  int ff_prepare);

gdm_status gdm_fail(gdm_ctx *ctx, gdm_status s, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

gdm_status gdm_host_exception(gdm_ctx *ctx) {
    try {
        throw;
    } catch (const std::exception &e) {
        return gdm_fail(ctx, GDM_ERR_OOM, "host allocation or thread creation failed: %s", e.what());
    } catch (...) {
        return gdm_fail(ctx, GDM_ERR_OOM, "host allocation or thread creation failed");
    }
}

gdm_status gdm_after_launch(gdm_ctx *ctx, const char *what) {
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gdm_fail(ctx, GDM_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    return GDM_OK;
}

gdm_status gdm_scratch(gdm_ctx *ctx, size_t bytes, void **ptr) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes > ctx->ws_bytes) {
        if (ctx->ws) {
            GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            GDM_CUDA_TRY(ctx, cudaFree(ctx->ws));
            ctx->ws = nullptr;
            ctx->ws_bytes = 0;
        }
        GDM_CUDA_TRY(ctx, cudaMalloc(&ctx->ws, bytes));
        ctx->ws_bytes = bytes;
    }
    *ptr = ctx->ws;
    return GDM_OK;
}

gdm_status gdm_pinned(gdm_ctx *ctx, size_t bytes, void **ptr) {
    if (bytes > ctx->hpinned_bytes) {
        if (ctx->hpinned) {
            GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            cudaFreeHost(ctx->hpinned);
            ctx->hpinned = nullptr;
            ctx->hpinned_bytes = 0;
        }
        GDM_CUDA_TRY(ctx, cudaMallocHost(&ctx->hpinned, bytes));
        ctx->hpinned_bytes = bytes;
    }
    *ptr = ctx->hpinned;
    return GDM_OK;
}

gdm_status gdm_upload(gdm_ctx *ctx, const void *host, size_t bytes, void **dev) {
    size_t off = (ctx->param_off + 255) & ~size_t(255);
    if (off + bytes > GDM_PARAM_BYTES) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "parameter block too large");
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->dparams + off, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    ctx->param_off = off + bytes;
    *dev = ctx->dparams + off;
    return GDM_OK;
}

gdm_status gdm_prof_begin(gdm_ctx *ctx, int *slot) {
    *slot = -1;
    if (!ctx->prof_on || ctx->prof_n >= GDM_PROF_MAX) return GDM_OK;
    if (!ctx->prof_ev) {
        ctx->prof_ev = new (std::nothrow) cudaEvent_t[2 * GDM_PROF_MAX];
        if (!ctx->prof_ev) return gdm_fail(ctx, GDM_ERR_OOM, "profile events");
        for (int i = 0; i < 2 * GDM_PROF_MAX; i++) GDM_CUDA_TRY(ctx, cudaEventCreate(&ctx->prof_ev[i]));
    }
    *slot = ctx->prof_n;
    GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->prof_ev[2 * *slot], ctx->stream));
    return GDM_OK;
}

gdm_status gdm_prof_end(gdm_ctx *ctx, int slot, double flops, double bytes) {
    if (slot < 0) return GDM_OK;
    GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->prof_ev[2 * slot + 1], ctx->stream));
    ctx->prof_n = slot + 1;
    ctx->prof_flops += flops;
    ctx->prof_bytes += bytes;
    return GDM_OK;
}

gdm_status gdm_phase_begin(gdm_ctx *ctx, int phase) {
    if (!ctx->ph_on || ctx->ph_n >= GDM_PH_MAX) return GDM_OK;
    if (!ctx->ph_ev) {
        ctx->ph_ev = new (std::nothrow) cudaEvent_t[2 * GDM_PH_MAX];
        ctx->ph_id = new (std::nothrow) int[GDM_PH_MAX];
        if (!ctx->ph_ev || !ctx->ph_id) return gdm_fail(ctx, GDM_ERR_OOM, "phase events");
        for (int i = 0; i < 2 * GDM_PH_MAX; i++) GDM_CUDA_TRY(ctx, cudaEventCreate(&ctx->ph_ev[i]));
    }
    ctx->ph_id[ctx->ph_n] = phase;
    GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ph_ev[2 * ctx->ph_n], ctx->stream));
    return GDM_OK;
}

gdm_status gdm_phase_end(gdm_ctx *ctx, int phase) {
    if (!ctx->ph_on || ctx->ph_n >= GDM_PH_MAX) return GDM_OK;
    (void)phase;
    GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ph_ev[2 * ctx->ph_n + 1], ctx->stream));
    ctx->ph_n++;
    return GDM_OK;
}

extern "C" {

gdm_status gdm_profile_phases(gdm_ctx *ctx, int enable, double *ms_out) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    if (ms_out) {
        GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
        GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        for (int p = 0; p < GDM_NPHASES; p++) ms_out[p] = 0.0;
        for (int i = 0; i < ctx->ph_n; i++) {
            float t = 0.f;
            GDM_CUDA_TRY(ctx, cudaEventElapsedTime(&t, ctx->ph_ev[2 * i], ctx->ph_ev[2 * i + 1]));
            ms_out[ctx->ph_id[i]] += t;
        }
    }
    ctx->ph_on = enable ? 1 : 0;
    ctx->ph_n = 0;
    return GDM_OK;
}

gdm_status gdm_profile_enable(gdm_ctx *ctx, int enable) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    ctx->prof_on = enable ? 1 : 0;
    if (enable) {
        ctx->prof_n = 0;
        ctx->prof_flops = 0.0;
        ctx->prof_bytes = 0.0;
    }
    return GDM_OK;
}

gdm_status gdm_profile_read(gdm_ctx *ctx, int64_t *launches, double *total_ms, double *flops, double *bytes) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    double ms = 0.0;
    for (int i = 0; i < ctx->prof_n; i++) {
        float t = 0.f;
        GDM_CUDA_TRY(ctx, cudaEventElapsedTime(&t, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]));
        ms += t;
    }
    if (launches) *launches = ctx->prof_n;
    if (total_ms) *total_ms = ms;
    if (flops) *flops = ctx->prof_flops;
    if (bytes) *bytes = ctx->prof_bytes;
    return GDM_OK;
}

const char *gdm_status_string(gdm_status s) {
    switch (s) {
        case GDM_OK: return "GDM_OK";
        case GDM_ERR_INVALID_ARG: return "GDM_ERR_INVALID_ARG";
        case GDM_ERR_SHAPE: return "GDM_ERR_SHAPE";
        case GDM_ERR_NONFINITE: return "GDM_ERR_NONFINITE";
        case GDM_ERR_SINGULAR: return "GDM_ERR_SINGULAR";
        case GDM_ERR_NOT_CONVERGED: return "GDM_ERR_NOT_CONVERGED";
        case GDM_ERR_OOM: return "GDM_ERR_OOM";
        case GDM_ERR_CUDA: return "GDM_ERR_CUDA";
        case GDM_ERR_TIMEOUT: return "GDM_ERR_TIMEOUT";
        case GDM_ERR_UNSUPPORTED: return "GDM_ERR_UNSUPPORTED";
    }
    return "GDM_ERR_UNKNOWN";
}

const char *gdm_last_error(gdm_ctx *ctx) { return ctx ? ctx->err : "null context"; }

int64_t gdm_launch_count(gdm_ctx *ctx) { return ctx ? ctx->launches : 0; }

gdm_status gdm_create(gdm_ctx **out, int device, void *stream) {
    if (!out) return GDM_ERR_INVALID_ARG;
    *out = nullptr;
    gdm_ctx *ctx = new (std::nothrow) gdm_ctx();
    if (!ctx) return GDM_ERR_OOM;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete ctx;
        return GDM_ERR_CUDA;
    }
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    e = cudaMalloc(&ctx->dflags, GDM_NFLAGS * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->dflags, 0, GDM_NFLAGS * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->dparams, GDM_PARAM_BYTES);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev2);
    if (e != cudaSuccess) {
        gdm_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? GDM_ERR_OOM : GDM_ERR_CUDA;
    }
    *out = ctx;
    return GDM_OK;
}

gdm_status gdm_destroy(gdm_ctx *ctx) {
    if (!ctx) return GDM_OK;
    cudaSetDevice(ctx->device);
    for (int i = 0; i < ctx->npool; i++) gdm_destroy(ctx->pool[i]);
    ctx->npool = 0;
    if (ctx->stream || ctx->ws) cudaStreamSynchronize(ctx->stream);
    gdm_glu_release(ctx);
    gdm_gr_release(ctx);
    if (ctx->owns_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->dflags) cudaFree(ctx->dflags);
    if (ctx->dparams) cudaFree(ctx->dparams);
    if (ctx->hpinned) cudaFreeHost(ctx->hpinned);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->ev2) cudaEventDestroy(ctx->ev2);
    if (ctx->prof_ev) {
        for (int i = 0; i < 2 * GDM_PROF_MAX; i++) cudaEventDestroy(ctx->prof_ev[i]);
        delete[] ctx->prof_ev;
    }
    if (ctx->ph_ev) {
        for (int i = 0; i < 2 * GDM_PH_MAX; i++) cudaEventDestroy(ctx->ph_ev[i]);
        delete[] ctx->ph_ev;
        delete[] ctx->ph_id;
    }
    delete ctx;
    return GDM_OK;
}

gdm_status gdm_set_stream(gdm_ctx *ctx, void *stream) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    ctx->stream = (cudaStream_t)stream;
    return GDM_OK;
}

}  // extern "C"

// one thread waits (bounded by the global timer) for a device flag that nothing sets, then records a timeout
static __global__ void k_wait_unset_flag(volatile int *never_set, long long limit_ns, int *flags) {
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (*never_set) return;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if ((long long)(t - t0) > limit_ns) {
            gdm_dev_error(flags, GDM_ERR_TIMEOUT, 99);
            return;
        }
        __nanosleep(1000);
    }
}

extern "C" {

gdm_status gdm_diag_wait_timeout(gdm_ctx *ctx, double limit_ms) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    if (!(limit_ms > 0) || limit_ms > 2000) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "limit must be in (0, 2000] ms");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    // a flag slot that no kernel of this call sets (zeroed at context creation, never written)
    k_wait_unset_flag<<<1, 1, 0, ctx->stream>>>(ctx->dflags + GDM_FLAG_DIAG, (long long)(limit_ms * 1e6), ctx->dflags);
    GDM_LAUNCHED(ctx, "wait_unset_flag");
    return gdm_ctx_check(ctx);
}

gdm_status gdm_ctx_check(gdm_ctx *ctx) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    int h[2] = {0, 0};
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(h, ctx->dflags, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dflags, 0, 2 * sizeof(int), ctx->stream));
    if (h[0] != 0)
        return gdm_fail(ctx, (gdm_status)h[0], "device reported %s (detail %d)", gdm_status_string((gdm_status)h[0]),
                        h[1]);
    return GDM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ validation
static gdm_status check_problem(gdm_ctx *ctx, const gdm_problem *p) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    if (!p) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "problem is NULL");
    if (p->n < 1) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "n must be >= 1 (got %lld)", (long long)p->n);
    if (p->kind != 3 && p->kind != 6) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "kind must be 3 or 6");
    if (!p->pos) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "pos is NULL");
    if (!(p->wavelength > 0.0) || !isfinite(p->wavelength))
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "wavelength must be finite and > 0");
    if (!(p->eps_env > 0.0) || !isfinite(p->eps_env))
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "eps_env must be finite and > 0");
    if (p->kind == 3) {
        if (!p->eps) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "kind 3 needs eps");
        if (!(p->step > 0.0) || !isfinite(p->step))
            return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "kind 3 needs a finite mesh step > 0");
    } else {
        if (!p->alpha6) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "kind 6 needs alpha6");
    }
    if (p->n * p->kind > (int64_t)1 << 30) return gdm_fail(ctx, GDM_ERR_SHAPE, "system too large");
    return GDM_OK;
}

static gdm_status check_prec(gdm_ctx *ctx, gdm_precision prec) {
    if (prec != GDM_FP64 && prec != GDM_FP32 && prec != GDM_TF32_REFINE && prec != GDM_BF16_REFINE)
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    return GDM_OK;
}

static gdm_status check_lda(gdm_ctx *ctx, int64_t n_sys, int64_t lda) {
    if (lda < n_sys) return gdm_fail(ctx, GDM_ERR_SHAPE, "lda %lld < system size %lld", (long long)lda, (long long)n_sys);
    if (lda % 2) return gdm_fail(ctx, GDM_ERR_SHAPE, "lda must be even (16-byte aligned columns)");
    return GDM_OK;
}

extern "C" {

// c itself, or with GDM_SOLVE_ERR_ESTIMATE and a clear contraction (rho = c / c_prev <= 1/4) the geometric
// tail rho c / (1 - rho) of the corrections still to come, i.e. the relative error left after this step
double gdm_refine_stop_measure(double c, double c_prev, int32_t flags) {
    if ((flags & GDM_SOLVE_ERR_ESTIMATE) && c_prev > 0.0 && c >= 0.0) {
        const double rho = c / c_prev;
        if (rho <= 0.25) return rho * c / (1.0 - rho);
    }
    return c;
}

gdm_status gdm_workspace_size(const gdm_problem *p, int n_rhs, gdm_precision prec, size_t *bytes) {
    if (!p || !bytes || n_rhs < 1) return GDM_ERR_INVALID_ARG;
    int64_t ns = p->n * p->kind;
    // refinement: vectors, Green-sum partials, solve operators and flags (the arena the factorisation used)
    size_t vec = (size_t)ns * n_rhs * 16;
    size_t b = 6 * vec + 64 * 1024;
    if (prec != GDM_FP64) b += (size_t)ns * n_rhs * 8;
    b += (size_t)ns * 64 * 16;
    if (prec != GDM_FP64) {
        // factorisation at the default outer block width (an upper bound for the size-class widths): panel
        // candidates, the tensor-core operand buffers (embedded L panel and a U12 copy; the FP32 split
        // doubles both), the U12 block operator and row block, and for the recursive TF32 factorisation
        // (3N >= 8192) the embedding of L that its panels write
        const int64_t nb = gdm_lu_block(nullptr, prec, ns);
        const size_t lx = (size_t)2 * ns * 2 * nb * 4, u = (size_t)ns * 2 * nb * 4;
        size_t f = (size_t)2 * 256 * (16 + 32 * 8) + 64 * 1024;
        f += (prec == GDM_FP32 ? 2 * lx + 2 * u : lx + u) + 4096;
        if (nb <= 512) f += (size_t)nb * nb * 8 + (size_t)nb * ns * 8;
        if (prec == GDM_TF32_REFINE && ns >= 8192 && nb <= 512) f += lx;
        if (f > b) b = f;
    }
    *bytes = b;
    return GDM_OK;
}

gdm_status gdm_alpha6_lorentz(gdm_ctx *ctx, int64_t n, const double *omega0_e, const double *omega0_m,
                              double gamma_ev, double amp_nm, double wavelength, double eps_env,
                              double *alpha6_out) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    if (!omega0_e || !omega0_m || !alpha6_out) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (n < 1) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "n must be >= 1");
    if (!(wavelength > 0) || !isfinite(wavelength) || !(amp_nm > 0) || !(gamma_ev >= 0) || !(eps_env > 0) ||
        !isfinite(eps_env))
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "need wavelength > 0, amp_nm > 0, gamma_ev >= 0, eps_env > 0");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return gdm_launch_alpha6_lorentz(ctx, n, omega0_e, omega0_m, gamma_ev, amp_nm, wavelength, eps_env, alpha6_out);
}

gdm_status gdm_incident_planewave(gdm_ctx *ctx, const double *r, int64_t m, double wavelength, double eps_env,
                                  const double *e0, const double *khat, int n_rhs, int kind_out, double *F0) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    if (!r || !e0 || !khat || !F0) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (m < 1 || n_rhs < 1) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "m and n_rhs must be >= 1");
    if (kind_out != 3 && kind_out != 6) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "kind_out must be 3 or 6");
    if (!(wavelength > 0) || !(eps_env > 0)) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "bad wavelength/eps_env");
    double kn = 0;
    for (int c = 0; c < 3; c++) kn += khat[c] * khat[c];
    if (fabs(kn - 1.0) > 1e-9) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "khat must be a unit vector");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    double n_env = sqrt(eps_env);
    double k = n_env * 2.0 * 3.14159265358979323846 / wavelength;
    return gdm_launch_planewave(ctx, r, m, k, n_env, e0, khat, n_rhs, kind_out, F0);
}

gdm_status gdm_incident_gaussian(gdm_ctx *ctx, const double *r, int64_t m, double wavelength, double eps_env,
                                 const double *e0, double w0, const double *focus, double theta, int n_rhs,
                                 int kind_out, double *F0) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    if (!r || !e0 || !focus || !F0) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (m < 1 || n_rhs < 1 || n_rhs > 64) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "need m >= 1, n_rhs in [1, 64]");
    if (kind_out != 3 && kind_out != 6) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "kind_out must be 3 or 6");
    if (!(wavelength > 0) || !(eps_env > 0) || !(w0 > 0) || !isfinite(theta))
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "need wavelength, eps_env, w0 > 0 and a finite angle");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    gdm_params_reset(ctx);
    const double n_env = sqrt(eps_env);
    const double k = n_env * 2.0 * 3.14159265358979323846 / wavelength;
    return gdm_launch_gaussian(ctx, r, m, k, n_env, w0, focus, theta, e0, n_rhs, kind_out, F0);
}

gdm_status gdm_assemble(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, void *A, int64_t lda) {
    GDM_TRY(check_problem(ctx, p));
    GDM_TRY(check_prec(ctx, prec));
    if (!A) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "A is NULL");
    GDM_TRY(check_lda(ctx, p->n * p->kind, lda));
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return gdm_launch_assemble(ctx, p, prec, A, lda);
}

// factor (local pivots, certificate, whole-column refactor if needed) and refine; arguments validated
gdm_status gdm_solve_core(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, void *A, int64_t lda, int32_t *ipiv,
                          const double *F0, double *F, int n_rhs, const gdm_solve_opts *opts, gdm_solve_info *info) {
    const int64_t ns = p->n * p->kind;
    gdm_solve_opts o = {0, 0, 0.0};
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = (prec == GDM_FP64) ? 3 : 40;
    if (!(o.tol > 0)) o.tol = 1e-12;
    if (info) memset(info, 0, sizeof(*info));
    float fms = 0.f;
    float growth = 1.f;
    int refactored = 0;
    if (!(o.flags & GDM_SOLVE_FACTORED)) {
        if (info) GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
        int global = (o.flags & GDM_SOLVE_GLOBAL_PIVOT) ? 1 : 0;
        GDM_TRY(gdm_lu_factor(ctx, prec, A, ns, lda, ipiv, global, &growth));
        if (!global && !(growth <= (float)GDM_PIVOT_GROWTH_LIMIT)) {
            // the in-block pivots are not safe for this matrix: rebuild A and pivot over whole columns
            GDM_TRY(gdm_launch_assemble(ctx, p, prec, A, lda));
            GDM_TRY(gdm_lu_factor(ctx, prec, A, ns, lda, ipiv, 1, &growth));
            refactored = 1;
        }
        if (info) {
            GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
            GDM_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev1));
            GDM_CUDA_TRY(ctx, cudaEventElapsedTime(&fms, ctx->ev0, ctx->ev1));
        }
    }
    gdm_status s = gdm_refined_solve(ctx, p, prec, A, lda, ipiv, F0, F, n_rhs, 0, &o, info);
    if (info) {
        info->factor_ms = fms;
        info->pivot_growth = growth;
        info->refactored = refactored;
    }
    return s;
}

gdm_status gdm_check_solve_args(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, const void *A, int64_t lda,
                                const int32_t *ipiv, const double *F0, const double *F, int n_rhs) {
    GDM_TRY(check_problem(ctx, p));
    GDM_TRY(check_prec(ctx, prec));
    if (!A || !ipiv || !F0 || !F) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (n_rhs < 1 || n_rhs > 64) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "n_rhs must be in [1, 64]");
    return check_lda(ctx, p->n * p->kind, lda);
}

gdm_status gdm_solve(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, void *A, int64_t lda, int32_t *ipiv,
                     const double *F0, double *F, int n_rhs, const gdm_solve_opts *opts, gdm_solve_info *info) {
    GDM_TRY(gdm_check_solve_args(ctx, p, prec, A, lda, ipiv, F0, F, n_rhs));
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return gdm_solve_core(ctx, p, prec, A, lda, ipiv, F0, F, n_rhs, opts, info);
}

gdm_status gdm_residual(gdm_ctx *ctx, const gdm_problem *p, const double *F0, const double *F, int n_rhs, double *r,
                        double *norms2) {
    GDM_TRY(check_problem(ctx, p));
    if (!F0 || !F || !r) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (n_rhs < 1 || n_rhs > 64) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "n_rhs must be in [1, 64]");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    gdm_params_reset(ctx);
    const int64_t cnt = p->n * p->kind * n_rhs;
    const bool ff = !getenv("GDM_RESIDUAL_FP64");
    size_t pb = gdm_green_partial_bytes(ctx, p->n, p->n, p->kind);
    size_t need = ScratchCarver::round(cnt * sizeof(double2)) + ScratchCarver::round(pb) +
                  ScratchCarver::round(gdm_ff_scratch_bytes(p->n)) + 1024;
    void *ws;
    GDM_TRY(gdm_scratch(ctx, need, &ws));
    ScratchCarver sc(ws);
    double2 *Pbuf = sc.take<double2>(cnt);
    double2 *partial = sc.take<double2>(pb / sizeof(double2));
    void *ffws = ff ? sc.take<char>(gdm_ff_scratch_bytes(p->n)) : nullptr;
    return gdm_launch_residual_ws(ctx, p, F0, F, n_rhs, 0, r, norms2, Pbuf, partial, ffws, 1);
}

gdm_status gdm_nearfield(gdm_ctx *ctx, const gdm_problem *p, const double *F, const double *r_eval, int64_t m,
                         const double *F0_eval, int n_rhs, double *E_out, double *H_out) {
    GDM_TRY(check_problem(ctx, p));
    if (!F || !r_eval || !E_out) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (m < 1 || n_rhs < 1) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "m and n_rhs must be >= 1");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return gdm_launch_nearfield(ctx, p, F, r_eval, m, F0_eval, n_rhs, E_out, H_out);
}

gdm_status gdm_cross_sections(gdm_ctx *ctx, const gdm_problem *p, const double *F0, const double *F, int n_rhs,
                              const double *e0_norm2, double *ext, double *sca, double *abs) {
    GDM_TRY(check_problem(ctx, p));
    if (!F0 || !F || !e0_norm2) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (n_rhs < 1 || n_rhs > 64) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "n_rhs must be in [1, 64]");
    for (int r = 0; r < n_rhs; r++)
        if (!(e0_norm2[r] > 0)) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "|E0|^2 must be > 0");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return gdm_launch_cross_sections(ctx, p, F0, F, n_rhs, e0_norm2, ext, sca, abs);
}

gdm_status gdm_farfield(gdm_ctx *ctx, const gdm_problem *p, const double *F, int n_rhs, const double *dirs, int64_t q,
                        double *f_out) {
    GDM_TRY(check_problem(ctx, p));
    if (!F || !dirs || !f_out) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (q < 1 || n_rhs < 1 || n_rhs > 64) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "need q >= 1, n_rhs in [1, 64]");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return gdm_launch_farfield(ctx, p, F, n_rhs, dirs, q, f_out, nullptr, nullptr, nullptr);
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n from the Chebyshev-like guess)
static void gauss_legendre(int n, double *x, double *w) {
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; i++) {
        double z = cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int l = 2; l <= n; l++) {
                const double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) {
                p1 = z;
                p0 = 1.0;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int l = 2; l <= n; l++) {
            const double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) p0 = 1.0;
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

gdm_status gdm_sigma_farfield(gdm_ctx *ctx, const gdm_problem *p, const double *F, int n_rhs, const double *e0_norm2,
                              int n_theta, int n_phi, double *sigma) {
    GDM_TRY(check_problem(ctx, p));
    if (!F || !e0_norm2 || !sigma) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (n_rhs < 1 || n_rhs > 64) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "n_rhs must be in [1, 64]");
    if (n_theta < 2 || n_theta > 4096 || n_phi < 1 || n_phi > 8192)
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "need 2 <= n_theta <= 4096 and 1 <= n_phi <= 8192");
    for (int r = 0; r < n_rhs; r++)
        if (!(e0_norm2[r] > 0)) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "|E0|^2 must be > 0");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    GDM_GUARD_BEGIN
    const int64_t q = (int64_t)n_theta * n_phi;
    std::vector<double> x(n_theta), w(n_theta), h((size_t)4 * q + n_rhs);
    gauss_legendre(n_theta, x.data(), w.data());
    const double pi = 3.14159265358979323846, dphi = 2.0 * pi / n_phi;
    for (int i = 0; i < n_theta; i++) {
        const double ct = x[i], st = sqrt(fmax(0.0, 1.0 - ct * ct));
        for (int j = 0; j < n_phi; j++) {
            const int64_t t = (int64_t)i * n_phi + j;
            h[3 * t] = st * cos(j * dphi);
            h[3 * t + 1] = st * sin(j * dphi);
            h[3 * t + 2] = ct;
            h[3 * q + t] = w[i] * dphi;
        }
    }
    for (int r = 0; r < n_rhs; r++) h[4 * q + r] = 1.0 / e0_norm2[r];
    double *d = nullptr;
    GDM_CUDA_TRY(ctx, cudaMallocAsync((void **)&d, h.size() * sizeof(double), ctx->stream));
    gdm_status st = GDM_OK;
    if (cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        st = gdm_fail(ctx, GDM_ERR_CUDA, "far-field grid upload");
    if (st == GDM_OK) st = gdm_launch_farfield(ctx, p, F, n_rhs, d, q, nullptr, d + 3 * q, d + 4 * q, sigma);
    // the host grid must stay alive until the copy has been consumed
    cudaStreamSynchronize(ctx->stream);
    cudaFreeAsync(d, ctx->stream);
    return st;
    GDM_GUARD_END(ctx)
}

gdm_status gdm_cross_sections_noalloc(gdm_ctx *ctx, const gdm_problem *p, const double *F0, const double *F,
                                      int n_rhs, const double *e0_norm2, double *ext, double *sca, double *abs) {
    GDM_TRY(check_problem(ctx, p));
    if (!F0 || !F || !e0_norm2) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (n_rhs < 1 || n_rhs > 64) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "n_rhs must be in [1, 64]");
    for (int r = 0; r < n_rhs; r++)
        if (!(e0_norm2[r] > 0)) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "|E0|^2 must be > 0");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    GDM_GUARD_BEGIN
    return gdm_launch_cross_sections_noalloc(ctx, p, F0, F, n_rhs, e0_norm2, ext, sca, abs);
    GDM_GUARD_END(ctx)
}

gdm_status gdm_backward(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, const void *A, int64_t lda,
                        const int32_t *ipiv, const double *F, int n_rhs, const double *e0, const double *khat,
                        const double *gF, const double *g_sigma, double *grad_pos, double *grad_eps,
                        double *grad_wavelength, gdm_solve_info *info) {
    GDM_TRY(check_problem(ctx, p));
    GDM_TRY(check_prec(ctx, prec));
    if (p->kind != 3) return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "gdm_backward is implemented for kind 3");
    if (!A || !ipiv || !F || !e0 || !khat) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (n_rhs < 1 || n_rhs > 64) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "n_rhs must be in [1, 64]");
    GDM_TRY(check_lda(ctx, p->n * p->kind, lda));
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return gdm_launch_backward(ctx, p, prec, A, lda, ipiv, F, n_rhs, e0, khat, gF, g_sigma, grad_pos, grad_eps,
                               grad_wavelength, info);
}

gdm_status gdm_nearfield_backward(gdm_ctx *ctx, const gdm_problem *p, const double *F, const double *r_eval,
                                  int64_t m, int n_rhs, const double *e0, const double *khat, const double *gE,
                                  double *gF_accum, double *grad_pos, double *grad_eps, double *grad_wavelength) {
    GDM_TRY(check_problem(ctx, p));
    if (p->kind != 3) return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "gdm_nearfield_backward is implemented for kind 3");
    if (!F || !r_eval || !e0 || !khat || !gE) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (m < 1 || n_rhs < 1 || n_rhs > 64) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "bad m or n_rhs");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return gdm_launch_nearfield_backward(ctx, p, F, r_eval, m, n_rhs, e0, khat, gE, gF_accum, grad_pos, grad_eps,
                                         grad_wavelength);
}

}  // extern "C"
