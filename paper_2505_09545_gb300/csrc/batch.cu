// Batched solves of many independent problems of uneven size (structures, wavelengths, illuminations),
// and the LU block-width autotuner.
//
// gdm_solve_batched keeps a pool of child contexts inside the caller's context, each with its own stream,
// scratch arena, flags and pinned buffers. One host worker thread per child takes items largest first
// (longest-processing-time order) from a shared counter and runs the whole per-item path on its child's
// stream: plane wave, assembly, LU (in-block pivots with certificate, whole-column refactor when needed),
// FP64-refined solve, cross sections. The small launches of many problems therefore overlap on the GPU
// instead of running one problem at a time; the refinement's per-iteration host check of one item blocks
// only its own worker. Events order the pool after the work already queued on the caller's stream, and
// the caller's stream after the pool.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "gdm_internal.cuh"
#include "pool.cuh"

#define PI_D 3.14159265358979323846

// child contexts of the pool runner (pool.cuh), created on first use and owned by the context
gdm_status gdm_ensure_pool(gdm_ctx *ctx, int want) {
    while (ctx->npool < want) {
        cudaStream_t st = nullptr;
        GDM_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        gdm_ctx *c = nullptr;
        gdm_status s = gdm_create(&c, ctx->device, st);
        if (s != GDM_OK) {
            cudaStreamDestroy(st);
            return gdm_fail(ctx, s, "could not create a child context for the pool");
        }
        c->owns_stream = true;
        ctx->pool[ctx->npool++] = c;
    }
    return GDM_OK;
}


namespace {

// plane wave (when e0 is given) and, unless the item is factored already, assembly
gdm_status item_inputs(gdm_ctx *c, gdm_precision prec, const gdm_batch_item *it, bool assemble) {
    const gdm_problem *p = &it->prob;
    gdm_params_reset(c);
    if (it->e0) {
        const double n_env = sqrt(p->eps_env);
        const double k = n_env * 2.0 * PI_D / p->wavelength;
        static const double zhat[3] = {0.0, 0.0, 1.0};
        GDM_TRY(gdm_launch_planewave(c, p->pos, p->n, k, n_env, it->e0, it->khat ? it->khat : zhat, it->n_rhs,
                                     p->kind, it->F0));
    }
    if (assemble) GDM_TRY(gdm_launch_assemble(c, p, prec, it->A, it->lda));
    return GDM_OK;
}

gdm_status item_xsec(gdm_ctx *c, const gdm_batch_item *it);

// factorisation (unless FACTORED), refined solve and cross sections of one item
gdm_status item_solve(gdm_ctx *c, gdm_precision prec, const gdm_batch_item *it, const gdm_solve_opts *opts,
                      gdm_solve_info *info) {
    const gdm_problem *p = &it->prob;
    gdm_status s = gdm_solve_core(c, p, prec, it->A, it->lda, it->ipiv, it->F0, it->F, it->n_rhs, opts, info);
    if (s != GDM_OK) return s;
    return item_xsec(c, it);
}

// cross sections of one solved item, if asked for
gdm_status item_xsec(gdm_ctx *c, const gdm_batch_item *it) {
    const gdm_problem *p = &it->prob;
    if (it->sigma) {
        double e2[64];
        for (int q = 0; q < it->n_rhs; q++) {
            if (it->e0) {
                e2[q] = 0.0;
                for (int c3 = 0; c3 < 6; c3++) e2[q] += it->e0[6 * q + c3] * it->e0[6 * q + c3];
            } else {
                e2[q] = it->e0_norm2[q];
            }
        }
        GDM_TRY(gdm_launch_cross_sections(c, p, it->F0, it->F, it->n_rhs, e2, it->sigma, it->sigma + it->n_rhs,
                                          it->sigma + 2 * it->n_rhs));
    }
    return GDM_OK;
}

// the full per-item path on one child context
gdm_status run_item(gdm_ctx *c, gdm_precision prec, const gdm_batch_item *it, const gdm_solve_opts *opts,
                    gdm_solve_info *info) {
    GDM_TRY(item_inputs(c, prec, it, !(opts && (opts->flags & GDM_SOLVE_FACTORED))));
    return item_solve(c, prec, it, opts, info);
}

// Items factored together by the grouped LU (batch_lu.cu): TF32 factors with in-panel pivots, matrices
// whose storage the tensor maps accept (16-byte aligned, even leading dimension); GDM_BATCH_POOL keeps the
// per-item factorisations (diagnostics)
bool grouped_ok(gdm_precision prec, const gdm_batch_item *items, int n_items, const gdm_solve_opts *opts) {
    if (prec != GDM_TF32_REFINE || n_items < 2 || getenv("GDM_BATCH_POOL")) return false;
    if (opts && (opts->flags & (GDM_SOLVE_FACTORED | GDM_SOLVE_GLOBAL_PIVOT))) return false;
    for (int i = 0; i < n_items; i++)
        if (((uintptr_t)items[i].A & 15) || (items[i].lda & 1)) return false;
    return true;
}

// outer block width of the grouped LU: GDM_BATCH_NB if set, else the tuned width, else 256
int grouped_nb(const gdm_ctx *ctx) {
    const char *e = getenv("GDM_BATCH_NB");
    int nb = e ? atoi(e) : ctx->glu_nb;
    if (nb < 64 || nb > 512 || nb % 32) nb = 256;
    return nb;
}

// plane waves and assembly on the pool, one grouped factorisation on the context stream, then refined
// solves and cross sections on the pool. An item whose in-panel pivots fail the certificate (or that met
// a zero pivot) is re-assembled and factored alone with pivots over whole columns.
gdm_status solve_grouped(gdm_ctx *ctx, gdm_precision prec, const gdm_batch_item *items, int n_items,
                         const gdm_solve_opts *opts, int n_streams, gdm_solve_info *infos,
                         const std::vector<int64_t> &size) {
    gdm_solve_opts fo = {0, 0, 0.0};
    if (opts) fo = *opts;
    gdm_solve_opts go = fo;
    fo.flags |= GDM_SOLVE_FACTORED;
    go.flags |= GDM_SOLVE_GLOBAL_PIVOT;
    std::vector<float2 *> A((size_t)n_items);
    std::vector<int64_t> lda((size_t)n_items);
    std::vector<int32_t *> ipiv((size_t)n_items);
    for (int i = 0; i < n_items; i++) {
        A[i] = (float2 *)items[i].A;
        lda[i] = items[i].lda;
        ipiv[i] = items[i].ipiv;
    }
    // cells with one or two illuminations are refined (and their cross sections summed) all together
    // (batch_refine.cu), unless GDM_BATCH_REFINE_POOL keeps them per item on the pool (diagnostics); when
    // every item is such a problem, their plane waves and assembly run together too
    std::vector<int> gpos((size_t)n_items, -1);
    std::vector<GrProblem> gp;
    const bool grouped_refine = !getenv("GDM_BATCH_REFINE_POOL") && !(fo.flags & GDM_SOLVE_NO_REFINE);
    for (int i = 0; i < n_items; i++) {
        const gdm_batch_item *it = &items[i];
        if (grouped_refine && it->prob.kind == 3 && it->n_rhs <= 2) {
            gpos[i] = (int)gp.size();
            gp.push_back(GrProblem{&it->prob, A[i], lda[i], ipiv[i], it->F0, it->F, it->n_rhs, it->e0, it->khat,
                                   it->e0_norm2, it->sigma});
        }
    }
    const bool all_grouped = (int)gp.size() == n_items;
    if (!gp.empty()) GDM_TRY(gdm_gr_prepare(ctx, (int)gp.size(), gp.data()));
    if (all_grouped) {
        GDM_TRY(gdm_gr_inputs(ctx));
    } else {
        GDM_TRY(gdm_run_pool(
            ctx, n_items, size.data(), n_streams, infos,
            [&](gdm_ctx *c, int, int i, gdm_solve_info *) { return item_inputs(c, prec, &items[i], true); }, nullptr));
    }
    std::vector<float> growth((size_t)n_items, 0.f);
    std::vector<int> st((size_t)n_items, 0);
    float ms = 0.f;
    GDM_TRY(gdm_glu_factor(ctx, n_items, A.data(), lda.data(), size.data(), ipiv.data(), grouped_nb(ctx),
                           growth.data(), st.data(), &ms));
    auto cert_ok = [&](int i) { return st[i] == GDM_OK && growth[i] <= (float)GDM_PIVOT_GROWTH_LIMIT; };
    std::vector<unsigned char> use(gp.size(), 0);
    std::vector<gdm_solve_info> ginf(gp.size());
    int n_pool = 0;
    for (int i = 0; i < n_items; i++) {
        if (gpos[i] >= 0 && cert_ok(i)) use[gpos[i]] = 1;
        else n_pool++;
    }
    if (!gp.empty()) {
        memset(ginf.data(), 0, sizeof(gdm_solve_info) * gp.size());
        GDM_TRY(gdm_gr_refine(ctx, use.data(), fo.tol > 0 ? fo.tol : 1e-12, fo.max_iter > 0 ? fo.max_iter : 40,
                              fo.flags, ginf.data()));
        GDM_TRY(gdm_gr_xsec(ctx, use.data()));
    }
    auto grouped_info = [&](int i, gdm_solve_info *inf) {
        *inf = ginf[gpos[i]];
        inf->factor_ms = ms;
        inf->pivot_growth = growth[i];
        return (gdm_status)inf->status;
    };
    if (n_pool == 0) {
        // every item was refined together: records, and the first numerical failure as the call's status
        gdm_status first = GDM_OK;
        int first_item = -1;
        for (int i = 0; i < n_items; i++) {
            gdm_solve_info tmp;
            const gdm_status s = grouped_info(i, infos ? &infos[i] : &tmp);
            if (s != GDM_OK && first == GDM_OK) {
                first = s;
                first_item = i;
            }
        }
        if (first != GDM_OK)
            return gdm_fail(ctx, first, "item %d: refinement: %s", first_item, gdm_status_string(first));
        return GDM_OK;
    }
    return gdm_run_pool(
        ctx, n_items, size.data(), n_streams, infos,
        [&](gdm_ctx *c, int, int i, gdm_solve_info *inf) {
            const gdm_batch_item *it = &items[i];
            if (gpos[i] >= 0 && use[gpos[i]]) {
                const gdm_status s = grouped_info(i, inf);
                if (s != GDM_OK) return gdm_fail(c, s, "refinement of the item: %s", gdm_status_string(s));
                return GDM_OK;
            }
            if (!cert_ok(i)) {
                GDM_TRY(item_inputs(c, prec, it, true));
                gdm_status s = item_solve(c, prec, it, &go, inf);
                inf->refactored = 1;
                return s;
            }
            gdm_status s = item_solve(c, prec, it, &fo, inf);
            inf->factor_ms = ms;
            inf->pivot_growth = growth[i];
            return s;
        },
        nullptr);
}

// grad[i] += sum_w acc[w][i] over the children's gradient accumulators (5 doubles per cell: 3 position,
// then 2 for the complex eps gradient)
__global__ void k_sum_children(const double *__restrict__ acc, int nw, int64_t n, double *grad_pos, double *grad_eps) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 5 * n) return;
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += acc[(int64_t)w * 5 * n + i];
    if (i < 3 * n) {
        if (grad_pos) grad_pos[i] += s;
    } else if (grad_eps) {
        grad_eps[i - 3 * n] += s;
    }
}

struct BackwardSum {
    double *acc;
    int64_t n;
    double *grad_pos, *grad_eps;
};
gdm_status backward_sum(gdm_ctx *ctx, int nw, void *arg) {
    BackwardSum *b = (BackwardSum *)arg;
    k_sum_children<<<(unsigned)((5 * b->n + 255) / 256), 256, 0, ctx->stream>>>(b->acc, nw, b->n, b->grad_pos,
                                                                              b->grad_eps);
    GDM_LAUNCHED(ctx, "sum_children");
    return GDM_OK;
}

// prefixes the item index to the message the argument check left in ctx->err (formatted from a copy:
// the message buffer is also the destination)
gdm_status fail_item(gdm_ctx *ctx, gdm_status s, int i) {
    char msg[sizeof(ctx->err)];
    memcpy(msg, ctx->err, sizeof(msg));
    msg[sizeof(msg) - 1] = 0;
    return gdm_fail(ctx, s, "item %d: %s", i, msg);
}

}  // namespace

extern "C" {

gdm_status gdm_solve_batched(gdm_ctx *ctx, gdm_precision prec, const gdm_batch_item *items, int n_items,
                             const gdm_solve_opts *opts, int n_streams, gdm_solve_info *infos) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    if (n_items < 0 || (n_items > 0 && !items)) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "bad item list");
    if (n_items == 0) return GDM_OK;
    for (int i = 0; i < n_items; i++) {
        const gdm_batch_item *it = &items[i];
        gdm_status s = gdm_check_solve_args(ctx, &it->prob, prec, it->A, it->lda, it->ipiv, it->F0, it->F, it->n_rhs);
        if (s != GDM_OK) return fail_item(ctx, s, i);
        if (it->sigma && !it->e0 && !it->e0_norm2)
            return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "item %d: cross sections need e0 or e0_norm2", i);
        if (it->sigma && !it->e0)
            for (int q = 0; q < it->n_rhs; q++)
                if (!(it->e0_norm2[q] > 0)) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "item %d: |E0|^2 <= 0", i);
    }
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    GDM_GUARD_BEGIN
    std::vector<int64_t> size((size_t)n_items);
    for (int i = 0; i < n_items; i++) size[i] = items[i].prob.n * items[i].prob.kind;
    if (grouped_ok(prec, items, n_items, opts))
        return solve_grouped(ctx, prec, items, n_items, opts, n_streams, infos, size);
    return gdm_run_pool(ctx, n_items, size.data(), n_streams, infos,
                    [&](gdm_ctx *c, int, int i, gdm_solve_info *inf) { return run_item(c, prec, &items[i], opts, inf); },
                    nullptr);
    GDM_GUARD_END(ctx)
}

gdm_status gdm_backward_batched(gdm_ctx *ctx, gdm_precision prec, const gdm_backward_item *items, int n_items,
                                int n_streams, double *grad_pos, double *grad_eps, gdm_solve_info *infos) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    if (n_items < 0 || (n_items > 0 && !items)) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "bad item list");
    if (n_items == 0) return GDM_OK;
    const gdm_problem *p0 = &items[0].prob;
    for (int i = 0; i < n_items; i++) {
        const gdm_backward_item *it = &items[i];
        const gdm_problem *p = &it->prob;
        if (p->kind != 3) return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "item %d: the adjoint is implemented for kind 3", i);
        if (p->n != p0->n || p->pos != p0->pos || p->eps != p0->eps || p->step != p0->step ||
            p->eps_env != p0->eps_env)
            return gdm_fail(ctx, GDM_ERR_INVALID_ARG,
                            "item %d: the items must share one structure (n, pos, eps, step, eps_env); only the "
                            "wavelength may differ",
                            i);
        gdm_status s = gdm_check_solve_args(ctx, p, prec, it->A, it->lda, it->ipiv, it->F, it->F, it->n_rhs);
        if (s != GDM_OK) return fail_item(ctx, s, i);
        if (!it->e0) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "item %d: e0 is NULL", i);
    }
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const int64_t n = p0->n;
    int ns = n_streams > 0 ? n_streams : 8;
    if (ns > GDM_POOL_MAX) ns = GDM_POOL_MAX;
    if (ns > n_items) ns = n_items;
    // one gradient accumulator per child: a child runs its items one after another on its own stream
    double *acc = nullptr;
    GDM_CUDA_TRY(ctx, cudaMallocAsync((void **)&acc, sizeof(double) * 5 * n * ns, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(acc, 0, sizeof(double) * 5 * n * ns, ctx->stream));
    static const double zhat[3] = {0.0, 0.0, 1.0};
    BackwardSum bs = {acc, n, grad_pos, grad_eps};
    gdm_status st;
    try {
        std::vector<int64_t> size((size_t)n_items, n);
        st = gdm_run_pool(
            ctx, n_items, size.data(), ns, infos,
            [&](gdm_ctx *c, int w, int i, gdm_solve_info *inf) {
                const gdm_backward_item *it = &items[i];
                double *a = acc + (int64_t)w * 5 * n;
                return gdm_launch_backward(c, &it->prob, prec, it->A, it->lda, it->ipiv, it->F, it->n_rhs, it->e0,
                                           it->khat ? it->khat : zhat, it->gF, it->g_sigma, a, a + 3 * n,
                                           it->grad_wavelength, inf);
            },
            backward_sum, &bs);
    } catch (...) {
        st = gdm_host_exception(ctx);
    }
    cudaFreeAsync(acc, ctx->stream);
    return st;
}

}  // extern "C"

// ------------------------------------------------------------------ autotuner
namespace {
// deterministic well-conditioned test matrix: diagonal 4 + hashed entries in [-0.5, 0.5]^2 / sqrt(n)
__global__ void k_tune_matrix(float2 *A, int64_t n, int64_t lda, float scale) {
    const int64_t total = n * lda;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / lda, r = e % lda;
        uint64_t h = (uint64_t)e * 0x9E3779B97F4A7C15ull;
        h ^= h >> 31;
        h *= 0xBF58476D1CE4E5B9ull;
        h ^= h >> 29;
        float re = ((float)(h & 0xffffff) / 16777216.0f - 0.5f) * scale;
        float im = ((float)((h >> 24) & 0xffffff) / 16777216.0f - 0.5f) * scale;
        if (r == c) re += 4.0f;
        A[e] = (r < n) ? make_float2(re, im) : make_float2(0.f, 0.f);
    }
}
}  // namespace

extern "C" gdm_status gdm_autotune(gdm_ctx *ctx, gdm_precision prec, const int64_t *sizes, int n_sizes,
                                   int *nb_out) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    if (!sizes || n_sizes < 1) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "no sizes");
    if (prec != GDM_FP32 && prec != GDM_TF32_REFINE)
        return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "the block width is tuned for the FP32 precisions only");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    int64_t cls_max[GDM_NB_CLASSES] = {0};
    for (int i = 0; i < n_sizes; i++) {
        if (sizes[i] < 1) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "sizes must be >= 1");
        const int c = gdm_size_class(sizes[i]);
        cls_max[c] = std::max(cls_max[c], sizes[i]);
    }
    int64_t nmax = 0;
    for (int c = 0; c < GDM_NB_CLASSES; c++) nmax = std::max(nmax, cls_max[c]);
    const int64_t ldmax = (nmax + 31) / 32 * 32;
    float2 *A = nullptr;
    int32_t *ipiv = nullptr;
    GDM_CUDA_TRY(ctx, cudaMalloc(&A, sizeof(float2) * nmax * ldmax));
    cudaError_t e = cudaMalloc(&ipiv, sizeof(int32_t) * nmax);
    if (e != cudaSuccess) {
        cudaFree(A);
        return gdm_fail(ctx, GDM_ERR_OOM, "autotune buffers");
    }
    gdm_status st = GDM_OK;
    const int cand[3] = {128, 256, 512};
    const char *env = getenv("GDM_LU_NB");
    if (env) st = gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "GDM_LU_NB is set: it overrides any tuned width");
    for (int c = 0; c < GDM_NB_CLASSES && st == GDM_OK; c++) {
        const int64_t n = cls_max[c];
        if (!n) continue;
        const int64_t lda = (n + 31) / 32 * 32;
        float best = 1e30f;
        int best_nb = 512;
        for (int j = 0; j < 3 && st == GDM_OK; j++) {
            if (cand[j] > 2 * n && j > 0) break;
            ctx->nb_table[c] = cand[j];
            float ms = 0.f;
            for (int rep = 0; rep < 2 && st == GDM_OK; rep++) {
                k_tune_matrix<<<4 * ctx->sm_count, 256, 0, ctx->stream>>>(A, n, lda, 1.0f / sqrtf((float)n));
                if (cudaGetLastError() != cudaSuccess) {
                    st = gdm_fail(ctx, GDM_ERR_CUDA, "autotune matrix");
                    break;
                }
                if (cudaEventRecord(ctx->ev0, ctx->stream) != cudaSuccess) st = GDM_ERR_CUDA;
                if (st == GDM_OK) st = gdm_lu_factor(ctx, prec, A, n, lda, ipiv, 0, nullptr);
                if (st == GDM_OK && cudaEventRecord(ctx->ev1, ctx->stream) != cudaSuccess) st = GDM_ERR_CUDA;
                if (st == GDM_OK && cudaEventSynchronize(ctx->ev1) != cudaSuccess) st = GDM_ERR_CUDA;
                if (st == GDM_OK) cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
            }
            if (st == GDM_OK && ms < best) {
                best = ms;
                best_nb = cand[j];
            }
        }
        ctx->nb_table[c] = best_nb;
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(A);
    cudaFree(ipiv);
    if (st != GDM_OK) return st;
    if (nb_out)
        for (int c = 0; c < GDM_NB_CLASSES; c++) nb_out[c] = ctx->nb_table[c];
    return GDM_OK;
}

// Grouped-factorisation width for one batch's sizes: the lock-step LU of synthetic matrices of those sizes,
// timed per candidate width (the second of two runs: the first captures the schedule's graph)
extern "C" gdm_status gdm_autotune_batched(gdm_ctx *ctx, const int64_t *sizes, int n_sizes, int *nb_out) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    if (!sizes || n_sizes < 2) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "need at least two sizes");
    if (getenv("GDM_BATCH_NB"))
        return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "GDM_BATCH_NB is set: it overrides any tuned width");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    GDM_GUARD_BEGIN
    std::vector<int64_t> lda((size_t)n_sizes), n(sizes, sizes + n_sizes);
    std::vector<size_t> off((size_t)n_sizes), poff((size_t)n_sizes);
    size_t elems = 0, pv = 0;
    for (int i = 0; i < n_sizes; i++) {
        if (sizes[i] < 1) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "sizes must be >= 1");
        lda[i] = (sizes[i] + 31) / 32 * 32;
        off[i] = elems;
        elems += (size_t)sizes[i] * lda[i];
        poff[i] = pv;
        pv += (size_t)(sizes[i] + 63) / 64 * 64;
    }
    float2 *M = nullptr;
    int32_t *piv = nullptr;
    GDM_CUDA_TRY(ctx, cudaMalloc(&M, sizeof(float2) * elems));
    if (cudaMalloc(&piv, sizeof(int32_t) * pv) != cudaSuccess) {
        cudaFree(M);
        return gdm_fail(ctx, GDM_ERR_OOM, "autotune buffers");
    }
    std::vector<float2 *> Ap((size_t)n_sizes);
    std::vector<int32_t *> pp((size_t)n_sizes);
    for (int i = 0; i < n_sizes; i++) {
        Ap[i] = M + off[i];
        pp[i] = piv + poff[i];
    }
    const int cand[3] = {128, 256, 512};
    int best_nb = 256;
    float best = 1e30f;
    gdm_status st = GDM_OK;
    for (int c = 0; c < 3 && st == GDM_OK; c++) {
        float ms = 0.f;
        for (int rep = 0; rep < 2 && st == GDM_OK; rep++) {
            for (int i = 0; i < n_sizes; i++) {
                k_tune_matrix<<<2 * ctx->sm_count, 256, 0, ctx->stream>>>(Ap[i], n[i], lda[i],
                                                                          1.0f / sqrtf((float)n[i]));
                if (cudaGetLastError() != cudaSuccess) st = gdm_fail(ctx, GDM_ERR_CUDA, "autotune matrix");
            }
            if (st == GDM_OK)
                st = gdm_glu_factor(ctx, n_sizes, Ap.data(), lda.data(), n.data(), pp.data(), cand[c], nullptr,
                                    nullptr, &ms);
        }
        if (st == GDM_OK && ms < best) {
            best = ms;
            best_nb = cand[c];
        }
    }
    cudaStreamSynchronize(ctx->stream);
    gdm_glu_release(ctx);  // the synthetic matrices' table goes with them
    cudaFree(M);
    cudaFree(piv);
    if (st != GDM_OK) return st;
    ctx->glu_nb = best_nb;
    if (nb_out) *nb_out = best_nb;
    return GDM_OK;
    GDM_GUARD_END(ctx)
}
