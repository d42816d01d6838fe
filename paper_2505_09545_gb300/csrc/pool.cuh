// Pool runner shared by the batched solves and the iterative solver: independent work items run on the
// child contexts of a context (each with its own stream, scratch arena, flags and pinned buffers), one
// host worker thread per child. Internal to the library.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <thread>
#include <vector>

#include "gdm_internal.cuh"

// create child contexts until the context has `want` of them (at most GDM_POOL_MAX)
gdm_status gdm_ensure_pool(gdm_ctx *ctx, int want);

// GDM_POOL_FULL_GRIDS: children size their Green sums for the whole GPU (diagnostics)
inline bool share_env() { return getenv("GDM_POOL_FULL_GRIDS") != nullptr; }

inline bool gdm_per_item_numeric(gdm_status s) {
    return s == GDM_ERR_NOT_CONVERGED || s == GDM_ERR_NONFINITE || s == GDM_ERR_SINGULAR;
}

// Runs fn(child, item, info) for every item on up to n_streams child contexts, largest first. The pool
// starts after the work queued on the caller's stream; once the children have finished and the caller's
// stream waits for them, after(ctx, children used, after_arg) may queue follow-up work on that stream.
// Numerical failures stay with their item; any other error stops the remaining items.
template <class Fn>
gdm_status gdm_run_pool(gdm_ctx *ctx, int n_items, const int64_t *size, int n_streams, gdm_solve_info *infos,
                        Fn fn, gdm_status (*after)(gdm_ctx *, int, void *), void *after_arg = nullptr) {
    int ns = n_streams > 0 ? n_streams : 8;
    if (ns > GDM_POOL_MAX) ns = GDM_POOL_MAX;
    if (ns > n_items) ns = n_items;
    GDM_TRY(gdm_ensure_pool(ctx, ns));
    std::vector<int> order(n_items);
    for (int i = 0; i < n_items; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return size[a] > size[b]; });
    std::vector<gdm_solve_info> local((size_t)n_items);
    gdm_solve_info *inf = infos ? infos : local.data();
    memset(inf, 0, sizeof(gdm_solve_info) * (size_t)n_items);

    GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev2, ctx->stream));
    int64_t launches0[GDM_POOL_MAX];
    for (int w = 0; w < ns; w++) {
        gdm_ctx *c = ctx->pool[w];
        memcpy(c->nb_table, ctx->nb_table, sizeof(ctx->nb_table));
        c->share_sms = share_env() ? 0 : std::max(16, ctx->sm_count / ns);
        c->err[0] = 0;
        launches0[w] = c->launches;
        GDM_CUDA_TRY(ctx, cudaStreamWaitEvent(c->stream, ctx->ev2, 0));
    }
    std::atomic<int> next(0);
    std::atomic<bool> stop(false);
    std::mutex mu;
    gdm_status first = GDM_OK;
    int first_item = -1;
    char first_msg[sizeof(ctx->err)] = {0};
    auto worker = [&](int w) {
        gdm_ctx *c = ctx->pool[w];
        if (cudaSetDevice(ctx->device) != cudaSuccess) {
            stop = true;
            return;
        }
        for (;;) {
            if (stop.load()) break;
            const int k = next.fetch_add(1);
            if (k >= n_items) break;
            const int i = order[k];
            gdm_status s;
            try {
                s = fn(c, w, i, &inf[i]);
            } catch (...) {  // an exception must not leave the worker thread
                s = gdm_host_exception(c);
            }
            inf[i].status = s;
            if (s != GDM_OK) {
                std::lock_guard<std::mutex> lock(mu);
                if (first == GDM_OK || (gdm_per_item_numeric(first) && !gdm_per_item_numeric(s))) {
                    first = s;
                    first_item = i;
                    memcpy(first_msg, c->err, sizeof(first_msg));
                }
                if (!gdm_per_item_numeric(s)) stop = true;
            }
        }
    };
    std::vector<std::thread> threads;
    threads.reserve(ns);
    for (int w = 0; w < ns; w++) threads.emplace_back(worker, w);
    for (auto &t : threads) t.join();
    for (int w = 0; w < ns; w++) {
        gdm_ctx *c = ctx->pool[w];
        ctx->launches += c->launches - launches0[w];
        GDM_CUDA_TRY(ctx, cudaEventRecord(c->ev2, c->stream));
        GDM_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, c->ev2, 0));
    }
    if (after) GDM_TRY(after(ctx, ns, after_arg));
    if (first != GDM_OK) return gdm_fail(ctx, first, "item %d: %s", first_item, first_msg);
    return GDM_OK;
}

