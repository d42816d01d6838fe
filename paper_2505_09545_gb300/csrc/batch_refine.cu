// Grouped refinement of a batch: the mixed-precision iterative refinement of refine.cu for all the
// problems of a batch at once (cells with TF32 factors from the grouped LU, at most two right-hand sides).
//
// Every step is one launch per kernel over all problems still refining: the residual r = b - A X
// (moments, then the FP32 Green sums while a problem's last relative correction is above 1e-3, the
// double-float ones after, then the finalize with the self-term and the norms), the power-of-two scaling
// into the work vector, the two triangular solves (one persistent launch per triangle over every
// problem's row blocks, tickets ordered by position in solve order so that all problems' chains advance
// together) and the FP64 update with its norms. One device-to-host copy of all problems' norms per step
// decides which problems have converged (max_q ||d_q|| / ||X_q|| <= tol) and which residual each of the
// others takes next; the converged ones leave the lists of the following launches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gdm_internal.cuh"

namespace {

constexpr int GR_CHUNK = 256;  // sources per Green-sum chunk

struct RPlan {
    std::vector<int64_t> n;  // signature: cells per problem (sorted, decreasing)
    std::vector<int> nr;
    std::vector<int> order;  // table position -> caller's index (of the prepared call)
    char *dmem = nullptr;    // tables, scratch and flags
    GrItem *d_items = nullptr;
    void *d_maps = nullptr;  // one 128-byte descriptor per problem
    int *d_lists = nullptr;  // list and prefix sums of a step's launches
    size_t lists_cap = 0;
    int *d_tickets = nullptr;
    int *d_sync = nullptr;   // all problems' solve flags, contiguous
    size_t sync_ints = 0;
    double *d_norms = nullptr;
    void *d_tab = nullptr;
    std::vector<GrItem> h_items;
    char *h_pinned = nullptr;  // descriptors, then list staging, then the norms read back
    size_t maps_bytes = 0, stage_bytes = 0;
    ~RPlan() {
        if (dmem) cudaFree(dmem);
        if (h_pinned) cudaFreeHost(h_pinned);
    }
};

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// the work units per problem of each kind of launch
inline int units_elem(const GrItem &g) { return (int)((3 * g.n * g.nr + 255) / 256); }
inline int units_cell(const GrItem &g) { return (int)((g.n + 255) / 256); }
inline int units_green(const GrItem &g) { return (int)((g.n + 127) / 128) * g.nc; }
inline int units_ops(const GrItem &g) { return g.nblk * TRSV_OPS_CTAS; }
inline int units_asm(const GrItem &g) { return (int)((g.n + 127) / 128) * (int)((g.n + 7) / 8); }

}  // namespace

namespace {

// scratch of every problem (kept while the batch's sizes stay the same)
gdm_status alloc_rplan(gdm_ctx *ctx, RPlan &R) {
    const int N = (int)R.n.size();
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = up256(off + bytes);
        return o;
    };
    const size_t o_items = take(sizeof(GrItem) * N);
    const size_t o_maps = take((size_t)128 * N);
    const size_t o_tab = take(257 * 16);
    const size_t o_tickets = take(sizeof(int) * 8);
    const size_t o_norms = take(sizeof(double) * 8 * N);
    const size_t o_xs = take(sizeof(double) * 4 * N);
    std::vector<size_t> o_r(N), o_P(N), o_w(N), o_part(N), o_dip(N), o_dipa(N), o_rec(N), o_ops(N), o_sync(N);
    size_t sync_ints = 0;
    for (int i = 0; i < N; i++) {
        const int64_t n = R.n[i], ns = 3 * n;
        const int64_t nc = (n + GR_CHUNK - 1) / GR_CHUNK;
        const int64_t nblk = (ns + 127) / 128;
        o_r[i] = take(sizeof(double2) * ns * 2);
        o_P[i] = take(sizeof(double2) * ns * 2);
        o_w[i] = take(sizeof(float2) * ns * 2);
        o_part[i] = take(sizeof(double2) * nc * 2 * ns);
        o_dip[i] = take((size_t)48 * n);
        o_dipa[i] = take((size_t)48 * n);
        o_rec[i] = take((size_t)4 * (8 + 4 * 3 * 2) * n);
        o_ops[i] = take(sizeof(float2) * 4 * nblk * 128 * 128);
        o_sync[i] = sync_ints;
        sync_ints += (size_t)nblk + 8;
    }
    const size_t o_sync0 = take(sizeof(int) * sync_ints);
    // lists and prefix sums of one step: the problem lists (N each) and prefix sums (N + 1 each) of up to 12
    // launches, plus the per-position prefix of the solves
    R.lists_cap = (size_t)12 * (2 * N + 1) + 512;
    const size_t o_lists = take(sizeof(int) * R.lists_cap);
    GDM_CUDA_TRY(ctx, cudaMalloc((void **)&R.dmem, off));
    char *b = R.dmem;
    R.d_items = (GrItem *)(b + o_items);
    R.d_maps = b + o_maps;
    R.d_tab = b + o_tab;
    R.d_tickets = (int *)(b + o_tickets);
    R.d_norms = (double *)(b + o_norms);
    R.d_sync = (int *)(b + o_sync0);
    R.sync_ints = sync_ints;
    R.d_lists = (int *)(b + o_lists);
    R.h_items.assign(N, GrItem());
    for (int i = 0; i < N; i++) {
        GrItem &g = R.h_items[i];
        memset(&g, 0, sizeof(g));
        g.n = R.n[i];
        g.nr = R.nr[i];
        g.nblk = (int)((3 * g.n + 127) / 128);
        g.r = (double2 *)(b + o_r[i]);
        g.P = (double2 *)(b + o_P[i]);
        g.w = (float2 *)(b + o_w[i]);
        g.partial = (double2 *)(b + o_part[i]);
        g.dip = b + o_dip[i];
        g.dipa = b + o_dipa[i];
        g.xs = (double *)(b + o_xs) + 4 * i;
        g.rec = (float *)(b + o_rec[i]);
        g.ops = (float2 *)(b + o_ops[i]);
        g.sync = R.d_sync + o_sync[i];
        g.norms = R.d_norms + 8 * i;
        g.chunk = GR_CHUNK;
        g.nc = (int)((g.n + GR_CHUNK - 1) / GR_CHUNK);
    }
    R.maps_bytes = up256((size_t)128 * N);
    R.stage_bytes = up256(sizeof(int) * R.lists_cap);
    GDM_CUDA_TRY(ctx, cudaMallocHost((void **)&R.h_pinned,
                                     R.maps_bytes + up256(sizeof(GrItem) * N) + R.stage_bytes +
                                         up256(sizeof(double) * 8 * N)));
    GDM_TRY(gdm_ff_table_fill(ctx, R.d_tab));
    return GDM_OK;
}

// list and prefix sums of one launch over the problems `act` (positions in the table, decreasing size):
// appended to the staging vector; returns the offsets and the total units
struct LaunchLists {
    int list_off, prefix_off, na, units;
};
template <class F>
LaunchLists add_launch(std::vector<int> &stage, const std::vector<int> &act, const std::vector<GrItem> &items, F units) {
    LaunchLists L;
    L.na = (int)act.size();
    L.list_off = (int)stage.size();
    for (int k : act) stage.push_back(k);
    L.prefix_off = (int)stage.size();
    int acc = 0;
    for (int k : act) {
        stage.push_back(acc);
        acc += units(items[k]);
    }
    stage.push_back(acc);
    L.units = acc;
    return L;
}

}  // namespace

void gdm_gr_release(gdm_ctx *ctx) {
    delete (RPlan *)ctx->grf;
    ctx->grf = nullptr;
}

namespace {
// host staging areas of the pinned block: descriptors, the table, the lists of one step, the norms
struct Staging {
    char *maps;
    GrItem *items;
    int *lists;
    double *norms;
};
Staging staging(RPlan &R) {
    const int N = (int)R.n.size();
    Staging st;
    st.maps = R.h_pinned;
    st.items = (GrItem *)(R.h_pinned + R.maps_bytes);
    st.lists = (int *)((char *)st.items + up256(sizeof(GrItem) * N));
    st.norms = (double *)((char *)st.lists + R.stage_bytes);
    return st;
}

// copies a step's lists to the device (the previous step's copy has completed: every step ends with a
// synchronisation)
gdm_status upload_lists(gdm_ctx *ctx, RPlan &R, const std::vector<int> &stage) {
    if (stage.size() > R.lists_cap) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "grouped lists");
    int *h = staging(R).lists;
    memcpy(h, stage.data(), sizeof(int) * stage.size());
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(R.d_lists, h, sizeof(int) * stage.size(), cudaMemcpyHostToDevice, ctx->stream));
    return GDM_OK;
}
}  // namespace

gdm_status gdm_gr_prepare(gdm_ctx *ctx, int n_items, const GrProblem *pb) {
    if (n_items < 1) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "grouped batch: no problems");
    for (int i = 0; i < n_items; i++)
        if (pb[i].p->kind != 3 || pb[i].n_rhs < 1 || pb[i].n_rhs > 2)
            return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "grouped batch: cells with one or two right-hand sides");
    // table order: decreasing size (the solves' tickets need it)
    std::vector<int> order(n_items);
    for (int i = 0; i < n_items; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pb[a].p->n > pb[b].p->n; });
    RPlan *R = (RPlan *)ctx->grf;
    bool same = R && (int)R->n.size() == n_items;
    for (int k = 0; same && k < n_items; k++)
        same = R->n[k] == pb[order[k]].p->n && R->nr[k] == pb[order[k]].n_rhs;
    if (!same) {
        gdm_gr_release(ctx);
        R = new RPlan();
        ctx->grf = R;
        for (int k = 0; k < n_items; k++) {
            R->n.push_back(pb[order[k]].p->n);
            R->nr.push_back(pb[order[k]].n_rhs);
        }
        gdm_status s = alloc_rplan(ctx, *R);
        if (s != GDM_OK) {
            gdm_gr_release(ctx);
            return s;
        }
    }
    R->order = order;
    // this call's problems: pointers, scalars, amplitudes and descriptors of the factors' storage
    const double PI = 3.14159265358979323846;
    const Staging st = staging(*R);
    GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));  // the staging buffers are free
    for (int k = 0; k < n_items; k++) {
        const GrProblem &q = pb[order[k]];
        GrItem &g = R->h_items[k];
        const gdm_problem *p = q.p;
        g.n_env = sqrt(p->eps_env);
        g.k = g.n_env * 2.0 * PI / p->wavelength;
        g.pos = p->pos;
        g.eps = (const double2 *)p->eps;
        g.eps_env = p->eps_env;
        g.d3_4pi = p->step * p->step * p->step / (4.0 * PI);
        g.self_S = -4.0 * PI / (3.0 * p->eps_env * p->step * p->step * p->step);
        const double v[3] = {g.k, g.k * g.k, 1.0 / p->eps_env};
        for (int t = 0; t < 3; t++) {
            g.kk[2 * t] = (float)v[t];
            g.kk[2 * t + 1] = (float)(v[t] - (double)g.kk[2 * t]);
        }
        g.khi = (float)g.k;
        g.klo = (float)(g.k - (double)g.khi);
        g.inv_eps = (float)(1.0 / p->eps_env);
        g.A = q.A;
        g.lda = q.lda;
        g.ipiv = q.ipiv;
        g.rhs = (const double2 *)q.F0;
        g.X = (double2 *)q.F;
        g.has_e0 = q.e0 != nullptr;
        memset(g.e0, 0, sizeof(g.e0));
        static const double zhat[3] = {0.0, 0.0, 1.0};
        const double *kh = q.khat ? q.khat : zhat;
        for (int t = 0; t < 3; t++) g.khat[t] = kh[t];
        for (int r = 0; r < q.n_rhs; r++) {
            double e2 = 0.0;
            if (q.e0) {
                for (int c = 0; c < 6; c++) {
                    g.e0[6 * r + c] = q.e0[6 * r + c];
                    e2 += q.e0[6 * r + c] * q.e0[6 * r + c];
                }
            } else if (q.e0_norm2) {
                e2 = q.e0_norm2[r];
            }
            g.pref[r] = e2 > 0 ? 4.0 * PI * g.k / (p->eps_env * e2) : 0.0;
        }
        g.has_sigma = q.sigma != nullptr;
        g.sigma = q.sigma;
        st.items[k] = g;
        if (!gdm_trsv_encode_map(q.A, 3 * p->n, q.lda, st.maps + (size_t)128 * k))
            return gdm_fail(ctx, GDM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the grouped solves");
    }
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(R->d_items, st.items, sizeof(GrItem) * n_items, cudaMemcpyHostToDevice,
                                      ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(R->d_maps, st.maps, (size_t)128 * n_items, cudaMemcpyHostToDevice,
                                      ctx->stream));
    return GDM_OK;
}

gdm_status gdm_gr_inputs(gdm_ctx *ctx) {
    RPlan *R = (RPlan *)ctx->grf;
    if (!R) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "grouped batch not prepared");
    const int N = (int)R->n.size();
    std::vector<int> all(N), stage;
    for (int k = 0; k < N; k++) all[k] = k;
    const LaunchLists Lc = add_launch(stage, all, R->h_items, units_cell);
    const LaunchLists La = add_launch(stage, all, R->h_items, units_asm);
    GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));  // the lists' staging buffer is free
    GDM_TRY(upload_lists(ctx, *R, stage));
    const int *dl = R->d_lists;
    GDM_TRY(gdm_gr_planewave(ctx, R->d_items, dl + Lc.list_off, dl + Lc.prefix_off, Lc.na, Lc.units));
    GDM_TRY(gdm_gr_prep_dipa(ctx, R->d_items, dl + Lc.list_off, dl + Lc.prefix_off, Lc.na, Lc.units));
    return gdm_gr_assemble(ctx, R->d_items, dl + La.list_off, dl + La.prefix_off, La.na, La.units);
}

gdm_status gdm_gr_refine(gdm_ctx *ctx, const unsigned char *use, double tol, int max_iter, int flags,
                         gdm_solve_info *infos) {
    RPlan *R = (RPlan *)ctx->grf;
    if (!R) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "grouped batch not prepared");
    const int N = (int)R->n.size();
    const std::vector<GrItem> &items = R->h_items;
    const Staging sg = staging(*R);
    std::vector<int> sel;
    for (int k = 0; k < N; k++)
        if (use[R->order[k]]) sel.push_back(k);
    if (sel.empty()) return GDM_OK;
    GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));  // the lists' staging buffer is free
    std::vector<int> stage;
    const int *dl = R->d_lists;
    struct Solve {
        int list_off, jp_off, nj, units;
    };
    // tickets of the solves: position tk in solve order slowest; the problems with more than tk blocks are
    // a prefix of the list (decreasing size)
    auto add_solve = [&](const std::vector<int> &act) {
        Solve t;
        t.list_off = (int)stage.size();
        for (int k : act) stage.push_back(k);
        t.jp_off = (int)stage.size();
        t.nj = act.empty() ? 0 : items[act[0]].nblk;
        int acc = 0;
        for (int tk = 0; tk < t.nj; tk++) {
            stage.push_back(acc);
            for (int k : act)
                if (items[k].nblk > tk) acc++;
        }
        stage.push_back(acc);
        t.units = acc;
        return t;
    };
    auto solve = [&](const Solve &t) -> gdm_status {
        for (int mode = 0; mode < 2; mode++) {
            GDM_CUDA_TRY(ctx, cudaMemsetAsync(R->d_sync, 0, sizeof(int) * R->sync_ints, ctx->stream));
            GDM_CUDA_TRY(ctx, cudaMemsetAsync(R->d_tickets + mode, 0, sizeof(int), ctx->stream));
            GDM_TRY(gdm_gr_trsv(ctx, R->d_items, R->d_maps, dl + t.list_off, dl + t.jp_off, t.nj, t.units, mode,
                                R->d_tickets + mode));
        }
        return GDM_OK;
    };
#define GR_ARGS(L) R->d_items, dl + (L).list_off, dl + (L).prefix_off, (L).na, (L).units
    GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
    // set-up and the first solve: X = LU^{-1} F0
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(R->d_norms, 0, sizeof(double) * 8 * N, ctx->stream));
    {
        stage.clear();
        const LaunchLists Lc = add_launch(stage, sel, items, units_cell);
        const LaunchLists Lo = add_launch(stage, sel, items, units_ops);
        const LaunchLists Le = add_launch(stage, sel, items, units_elem);
        const Solve T = add_solve(sel);
        GDM_TRY(upload_lists(ctx, *R, stage));
        GDM_TRY(gdm_gr_prep_dip(ctx, GR_ARGS(Lc)));
        GDM_TRY(gdm_gr_block_ops(ctx, GR_ARGS(Lo)));
        GDM_TRY(gdm_gr_norm2(ctx, GR_ARGS(Le)));
        GDM_TRY(gdm_gr_to_work(ctx, GR_ARGS(Le), 0));
        GDM_TRY(solve(T));
        GDM_TRY(gdm_gr_update(ctx, GR_ARGS(Le), 0));
    }
    std::vector<double> relc(N, 1.0), relr(N, -1.0);
    std::vector<int> done(N, 0), iters(N, 0), stat(N, GDM_OK);
    for (int it = 1; it <= max_iter; it++) {
        std::vector<int> act, f32, ff;
        for (int k : sel)
            if (!done[k]) {
                act.push_back(k);
                // FP32 residuals while the last relative correction is above 1e-3 (as refine.cu)
                (relc[k] > 1e-3 ? f32 : ff).push_back(k);
            }
        if (act.empty()) break;
        // ||d||, ||X||, ||r|| of every problem start from zero; ||F0|| stays
        GDM_CUDA_TRY(ctx, cudaMemset2DAsync(R->d_norms, 8 * sizeof(double), 0, 6 * sizeof(double), N, ctx->stream));
        stage.clear();
        const LaunchLists Le = add_launch(stage, act, items, units_elem);
        const LaunchLists Lf = add_launch(stage, f32, items, units_green);
        const LaunchLists Ls = add_launch(stage, ff, items, units_cell);
        const LaunchLists Lg = add_launch(stage, ff, items, units_green);
        const LaunchLists Lc = add_launch(stage, act, items, units_cell);
        const Solve T = add_solve(act);
        GDM_TRY(upload_lists(ctx, *R, stage));
        GDM_TRY(gdm_gr_moments(ctx, GR_ARGS(Le)));
        GDM_TRY(gdm_gr_green_f32(ctx, GR_ARGS(Lf)));
        GDM_TRY(gdm_gr_prep_src(ctx, GR_ARGS(Ls)));
        GDM_TRY(gdm_gr_green_ff(ctx, GR_ARGS(Lg), R->d_tab));
        GDM_TRY(gdm_gr_finalize(ctx, GR_ARGS(Lc)));
        GDM_TRY(gdm_gr_to_work(ctx, GR_ARGS(Le), 1));
        GDM_TRY(solve(T));
        GDM_TRY(gdm_gr_update(ctx, GR_ARGS(Le), 1));
        GDM_CUDA_TRY(ctx, cudaMemcpyAsync(sg.norms, R->d_norms, sizeof(double) * 8 * N, cudaMemcpyDeviceToHost,
                                          ctx->stream));
        GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        for (int k : act) {
            const double *h = sg.norms + 8 * k;
            double c = 0.0, rr = 0.0;
            bool finite = true;
            for (int q = 0; q < items[k].nr; q++) {
                const double dq = h[2 * q], xq = h[2 * q + 1], rq = h[4 + q], bq = h[6 + q];
                if (!std::isfinite(dq) || !std::isfinite(xq) || !std::isfinite(rq)) finite = false;
                c = std::max(c, xq > 0 ? std::sqrt(dq / xq) : (dq > 0 ? INFINITY : 0.0));
                rr = std::max(rr, bq > 0 ? std::sqrt(rq / bq) : 0.0);
            }
            const double stop = gdm_refine_stop_measure(c, it > 1 ? relc[k] : -1.0, flags);
            relc[k] = c;
            relr[k] = rr;
            iters[k] = it;
            if (!finite) {
                stat[k] = GDM_ERR_NONFINITE;
                done[k] = 1;
            } else if (stop <= tol) {
                done[k] = 1;
            }
        }
    }
#undef GR_ARGS
    GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev2, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev2));
    // a timed-out wait in a kernel is the whole call's failure
    GDM_TRY(gdm_ctx_check(ctx));
    float ms = 0.f;
    GDM_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev1, ctx->ev2));
    for (int k : sel) {
        if (!done[k]) stat[k] = GDM_ERR_NOT_CONVERGED;
        gdm_solve_info &inf = infos[R->order[k]];
        inf.iterations = iters[k];
        inf.rel_correction = relc[k];
        inf.rel_residual = relr[k];
        inf.refine_ms = ms;
        inf.status = stat[k];
    }
    return GDM_OK;
}

gdm_status gdm_gr_xsec(gdm_ctx *ctx, const unsigned char *use) {
    RPlan *R = (RPlan *)ctx->grf;
    if (!R) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "grouped batch not prepared");
    const int N = (int)R->n.size();
    std::vector<int> sel, stage;
    for (int k = 0; k < N; k++)
        if (use[R->order[k]] && R->h_items[k].has_sigma) sel.push_back(k);
    if (sel.empty()) return GDM_OK;
    const LaunchLists L = add_launch(stage, sel, R->h_items, units_cell);
    GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));  // the lists' staging buffer is free
    GDM_TRY(upload_lists(ctx, *R, stage));
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(R->h_items[0].xs, 0, sizeof(double) * 4 * N, ctx->stream));
    const int *dl = R->d_lists;
    GDM_TRY(gdm_gr_xsec_partial(ctx, R->d_items, dl + L.list_off, dl + L.prefix_off, L.na, L.units));
    return gdm_gr_xsec_final(ctx, R->d_items, dl + L.list_off, L.na);
}
