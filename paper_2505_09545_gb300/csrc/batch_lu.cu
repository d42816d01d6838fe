// Grouped LU of a batch of independent problems of uneven size (TF32 factors, pivots inside 32-row
// panels with certificate), in lock step: one launch per step covers every problem that still has that
// step, so the ~(n / 32) x 3 launches of the largest problem factor the whole batch instead of that many
// launches per problem.
//
// Per outer block [b0, b0 + nbo) and per 32-column panel c0 inside it:
//   k_glu_diag        the panel's 32 x 32 diagonal block of every problem with n > c0 (one warp each:
//                     pivots, the factored block, U and reciprocal pivots for the rows),
//   k_glu_rows        the rows below it (certificate, L, and the TF32 embedding of L that the updates read),
//   k_glu_swap_trsm   the panel's interchanges and L11^{-1} on its rows right of the panel (U, rounded to
//                     TF32),
//   k_glu_gemm        C -= L U with K = 32 on the block's columns right of the panel and the block's rows
//                     below it (tcgen05, tiles of all problems in one persistent launch);
// then per block k_glu_gemm with K = nbo on the trailing matrix. Problems are kept in a table sorted by
// decreasing n, so each launch covers a prefix of it, and its work units (CTAs or tiles) are split by a
// prefix sum of per-problem counts computed here on the host. The factors have the layout gdm_lu_factor
// produces (row interchanges applied to the columns right of each panel only, L in product form), so the
// refined solve takes them as they are.
//
// The schedule depends only on the sorted sizes and the block width; it is captured once into a CUDA graph
// and replayed while those stay the same. The problems' pointers live in a device table that the graph's
// kernels read, so a new set of buffers of the same sizes only rewrites that table and its tensor maps.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gdm_internal.cuh"

namespace {

enum { L_PANEL = 0, L_SWAP = 1, L_GEMM_PANEL = 2, L_GEMM_TRAIL = 3, L_DIAG = 4 };
struct Launch {
    int type;
    int64_t b0, c0;
    int na;     // problems covered (a prefix of the sorted table)
    int off;    // offset of the launch's prefix sum (na + 1 entries) in the prefix array
    int count;  // total work units
};

struct Plan {
    // signature: the problems' sizes in the caller's order and the block width
    std::vector<int64_t> n_caller;
    int nbo = 0;
    std::vector<int> order;  // table position -> caller's index
    std::vector<Launch> launches;
    std::vector<int> prefix;
    // device buffers: one allocation for the tables and records, one for the L embeddings
    char *dmem = nullptr;
    float *dlx = nullptr;
    GluItem *d_items = nullptr;
    GluMaps *d_maps = nullptr;
    int *d_prefix = nullptr;
    unsigned *d_growth = nullptr;
    int *d_status = nullptr;
    int *d_ticket = nullptr;
    char *d_pdiag = nullptr;  // one GluPanelDiag record per problem
    size_t pdiag_stride = 0;
    std::vector<size_t> lx_off;
    // host copies of the table (pinned staging for the uploads)
    GluItem *h_items = nullptr;
    GluMaps *h_maps = nullptr;
    unsigned *h_growth = nullptr;
    int *h_status = nullptr;
    bool table_valid = false;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;  // kernel launches per replay

    ~Plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (dmem) cudaFree(dmem);
        if (dlx) cudaFree(dlx);
        if (h_maps) cudaFreeHost(h_maps);  // the pinned block starts with the maps
    }
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// the lock-step schedule of sizes n_sorted (decreasing) with outer block nbo; the CTAs of a panel's rows
// sized so that a launch fills about one wave of the rows kernel's resident CTAs (four per SM)
void build_schedule(Plan &P, const std::vector<int64_t> &ns, int nbo, int sm_count) {
    const int N = (int)ns.size();
    const int64_t nmax = ns[0];
    std::vector<int> cnt;
    auto add = [&](int type, int64_t b0, int64_t c0, int na, const std::vector<int> &c) {
        int tot = 0;
        for (int i = 0; i < na; i++) tot += c[i];
        if (tot == 0) return;
        Launch L{type, b0, c0, na, (int)P.prefix.size(), tot};
        int acc = 0;
        for (int i = 0; i < na; i++) {
            P.prefix.push_back(acc);
            acc += c[i];
        }
        P.prefix.push_back(acc);
        P.launches.push_back(L);
    };
    const int64_t target_ctas = 4 * (int64_t)sm_count;
    for (int64_t b0 = 0; b0 < nmax; b0 += nbo) {
        for (int64_t c0 = b0; c0 < b0 + nbo && c0 < nmax; c0 += 32) {
            int na = 0;
            while (na < N && ns[na] > c0) na++;
            cnt.assign(na, 0);
            // panel
            int64_t rows_total = 0;
            std::vector<int64_t> rows(na);
            for (int i = 0; i < na; i++) {
                const int64_t be = std::min(b0 + nbo, ns[i]);
                const int64_t w = std::min<int64_t>(32, be - c0);
                rows[i] = ns[i] - c0 - w;
                rows_total += rows[i];
            }
            int64_t R = (rows_total + target_ctas - 1) / target_ctas;
            R = std::max<int64_t>(128, (R + 127) / 128 * 128);
            // the diagonal blocks (one warp per problem), then the rows below
            P.launches.push_back(Launch{L_DIAG, b0, c0, na, 0, na});
            for (int i = 0; i < na; i++) cnt[i] = (int)((rows[i] + R - 1) / R);
            add(L_PANEL, b0, c0, na, cnt);
            // interchanges and U rows right of full panels
            for (int i = 0; i < na; i++) {
                const int64_t be = std::min(b0 + nbo, ns[i]);
                const bool full = be - c0 >= 32;
                cnt[i] = full ? (int)((ns[i] - c0 - 32 + GLU_SWAP_COLS - 1) / GLU_SWAP_COLS) : 0;
            }
            add(L_SWAP, b0, c0, na, cnt);
            for (int i = 0; i < na; i++) cnt[i] = glu_tiles(GLU_PANEL, ns[i], b0, c0, nbo);
            add(L_GEMM_PANEL, b0, c0, na, cnt);
        }
        int na = 0;
        while (na < N && ns[na] > b0 + nbo) na++;
        cnt.assign(na, 0);
        for (int i = 0; i < na; i++) cnt[i] = glu_tiles(GLU_TRAIL, ns[i], b0, 0, nbo);
        add(L_GEMM_TRAIL, b0, 0, na, cnt);
    }
}

gdm_status alloc_plan(gdm_ctx *ctx, Plan &P, const std::vector<int64_t> &ns) {
    const int N = (int)ns.size();
    size_t off = 0;
    const size_t o_items = off;
    off = align_up(off + sizeof(GluItem) * N, 256);
    const size_t o_maps = off;
    off = align_up(off + sizeof(GluMaps) * N, 256);
    const size_t o_prefix = off;
    off = align_up(off + sizeof(int) * P.prefix.size(), 256);
    const size_t o_growth = off;
    off = align_up(off + sizeof(unsigned) * N, 256);
    const size_t o_status = off;
    off = align_up(off + sizeof(int) * 2 * N, 256);
    const size_t o_ticket = off;
    off = align_up(off + sizeof(int) * N, 256);
    const size_t o_pdiag = off;
    const size_t pdiag = align_up(gdm_glu_pdiag_bytes(), 256);
    off += pdiag * N;
    GDM_CUDA_TRY(ctx, cudaMalloc((void **)&P.dmem, off));
    P.d_items = (GluItem *)(P.dmem + o_items);
    P.d_maps = (GluMaps *)(P.dmem + o_maps);
    P.d_prefix = (int *)(P.dmem + o_prefix);
    P.d_growth = (unsigned *)(P.dmem + o_growth);
    P.d_status = (int *)(P.dmem + o_status);
    P.d_ticket = (int *)(P.dmem + o_ticket);
    P.d_pdiag = P.dmem + o_pdiag;
    P.pdiag_stride = pdiag;
    // L embeddings: (2n) x (2 nbo) floats per problem
    size_t lx = 0;
    P.lx_off.resize(N);
    for (int i = 0; i < N; i++) {
        P.lx_off[i] = lx;
        lx = align_up(lx + sizeof(float) * 2 * ns[i] * 2 * P.nbo, 256);
    }
    GDM_CUDA_TRY(ctx, cudaMalloc((void **)&P.dlx, lx));
    const size_t hbytes = align_up(sizeof(GluMaps) * N, 256) + align_up(sizeof(GluItem) * N, 256) +
                          align_up(sizeof(unsigned) * N, 256) + align_up(sizeof(int) * 2 * N, 256);
    char *h = nullptr;
    GDM_CUDA_TRY(ctx, cudaMallocHost((void **)&h, hbytes));
    P.h_maps = (GluMaps *)h;  // first: 64-byte alignment of the maps
    P.h_items = (GluItem *)(h + align_up(sizeof(GluMaps) * N, 256));
    P.h_growth = (unsigned *)((char *)P.h_items + align_up(sizeof(GluItem) * N, 256));
    P.h_status = (int *)((char *)P.h_growth + align_up(sizeof(unsigned) * N, 256));
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(P.d_prefix, P.prefix.data(), sizeof(int) * P.prefix.size(),
                                      cudaMemcpyHostToDevice, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(P.d_ticket, 0, sizeof(int) * N, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return GDM_OK;
}

gdm_status issue(gdm_ctx *ctx, Plan &P) {
    const int N = (int)P.n_caller.size();
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(P.d_growth, 0, sizeof(unsigned) * N, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(P.d_status, 0, sizeof(int) * 2 * N, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(P.d_ticket, 0, sizeof(int) * N, ctx->stream));
    for (const Launch &L : P.launches) {
        const int *pre = P.d_prefix + L.off;
        switch (L.type) {
        case L_DIAG: GDM_TRY(gdm_glu_diag(ctx, P.d_items, L.na, L.b0, L.c0, P.nbo)); break;
        case L_PANEL: GDM_TRY(gdm_glu_rows(ctx, P.d_items, pre, L.na, L.count, L.b0, L.c0, P.nbo)); break;
        case L_SWAP: GDM_TRY(gdm_glu_swap_trsm(ctx, P.d_items, pre, L.na, L.count, L.c0)); break;
        case L_GEMM_PANEL:
            GDM_TRY(gdm_glu_gemm(ctx, P.d_items, P.d_maps, pre, L.na, L.count, GLU_PANEL, L.b0, L.c0, P.nbo));
            break;
        default:
            GDM_TRY(gdm_glu_gemm(ctx, P.d_items, P.d_maps, pre, L.na, L.count, GLU_TRAIL, L.b0, 0, P.nbo));
            break;
        }
    }
    return GDM_OK;
}

}  // namespace

void gdm_glu_release(gdm_ctx *ctx) {
    delete (Plan *)ctx->glu;
    ctx->glu = nullptr;
}

// Factor problems i = 0 .. n_items-1 (complex64 A[i], n[i] x n[i] with leading dimension lda[i], pivots
// ipiv[i]) together with outer block width nbo (a multiple of 32, at most 512). growth[i] receives the pivot
// certificate of problem i (as gdm_lu_factor's growth_out) and status[i] its device status (GDM_OK, or
// GDM_ERR_SINGULAR for a zero pivot). *ms: device time of the factorisation.
gdm_status gdm_glu_factor(gdm_ctx *ctx, int n_items, float2 *const *A, const int64_t *lda, const int64_t *n,
                          int32_t *const *ipiv, int nbo, float *growth, int *status, float *ms) {
    if (n_items < 1) return GDM_OK;
    if (nbo < 64 || nbo > 512 || nbo % 32) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "grouped LU block width");
    for (int i = 0; i < n_items; i++)
        if (n[i] < 1 || ((uintptr_t)A[i] & 15) || (lda[i] & 1) || lda[i] < n[i] || 2 * n[i] >= (int64_t)1 << 30)
            return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "problem %d does not fit the grouped factorisation", i);
    Plan *P = (Plan *)ctx->glu;
    const bool same = P && P->nbo == nbo && (int)P->n_caller.size() == n_items &&
                      std::equal(P->n_caller.begin(), P->n_caller.end(), n);
    if (!same) {
        gdm_glu_release(ctx);
        P = new Plan();
        ctx->glu = P;
        P->n_caller.assign(n, n + n_items);
        P->nbo = nbo;
        P->order.resize(n_items);
        for (int i = 0; i < n_items; i++) P->order[i] = i;
        std::stable_sort(P->order.begin(), P->order.end(), [&](int a, int b) { return n[a] > n[b]; });
        std::vector<int64_t> ns(n_items);
        for (int k = 0; k < n_items; k++) ns[k] = n[P->order[k]];
        build_schedule(*P, ns, nbo, ctx->sm_count);
        gdm_status s = alloc_plan(ctx, *P, ns);
        if (s != GDM_OK) {
            gdm_glu_release(ctx);
            return s;
        }
    }
    // the table of this call's buffers (rewritten, with its tensor maps, only when a pointer changed)
    bool changed = !P->table_valid;
    for (int k = 0; k < n_items; k++) {
        const int i = P->order[k];
        GluItem g;
        g.A = A[i];
        g.lda = lda[i];
        g.n = n[i];
        g.ipiv = ipiv[i];
        g.growth = P->d_growth + k;
        g.status = P->d_status + 2 * k;
        g.ticket = P->d_ticket + k;
        g.lx = P->dlx + P->lx_off[k] / sizeof(float);
        g.pdiag = P->d_pdiag + P->pdiag_stride * k;
        if (changed || memcmp(&g, &P->h_items[k], sizeof(g)) != 0) {
            changed = true;
            P->h_items[k] = g;
        }
    }
    if (changed) {
        // the previous call's copies out of the staging buffers have completed (its results were read)
        GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        if (!gdm_glu_encode(P->h_items, n_items, nbo, P->h_maps))
            return gdm_fail(ctx, GDM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the grouped factorisation");
        GDM_CUDA_TRY(ctx, cudaMemcpyAsync(P->d_items, P->h_items, sizeof(GluItem) * n_items, cudaMemcpyHostToDevice,
                                          ctx->stream));
        GDM_CUDA_TRY(ctx, cudaMemcpyAsync(P->d_maps, P->h_maps, sizeof(GluMaps) * n_items, cudaMemcpyHostToDevice,
                                          ctx->stream));
        P->table_valid = true;
    }
    if (!P->exec) {
        // capture the schedule once (kernel attributes are set before the capture starts)
        // on a stream of its own: the context's stream may be the legacy default stream, which cannot be
        // captured (the graph is then launched on the context's stream)
        GDM_TRY(gdm_glu_gemm_init(ctx));
        GDM_TRY(gdm_glu_panel_init(ctx));
        const int64_t l0 = ctx->launches;
        cudaStream_t cs = nullptr, user = ctx->stream;
        GDM_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            return gdm_fail(ctx, GDM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        }
        ctx->stream = cs;
        gdm_status s = issue(ctx, *P);
        ctx->stream = user;
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        cudaStreamDestroy(cs);
        if (s != GDM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return gdm_fail(ctx, GDM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&P->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            P->exec = nullptr;
            return gdm_fail(ctx, GDM_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(e));
        }
        P->kernels = ctx->launches - l0;
        ctx->launches = l0;
    }
    GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaGraphLaunch(P->exec, ctx->stream));
    ctx->launches += P->kernels;
    GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(P->h_growth, P->d_growth, sizeof(unsigned) * n_items, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(P->h_status, P->d_status, sizeof(int) * 2 * n_items, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    // a kernel-level failure (a timed-out wait) is the whole batch's
    GDM_TRY(gdm_ctx_check(ctx));
    if (ms) GDM_CUDA_TRY(ctx, cudaEventElapsedTime(ms, ctx->ev0, ctx->ev1));
    for (int k = 0; k < n_items; k++) {
        const int i = P->order[k];
        float g;
        memcpy(&g, &P->h_growth[k], sizeof(float));
        if (growth) growth[i] = g;
        if (status) status[i] = P->h_status[2 * k];
    }
    return GDM_OK;
}
