// Persistent blocked triangular solves with the LU factors (right-hand sides of the refinement and
// of the adjoint). One CTA per row block of NBS rows (NBS = the factorisation's outer block). A CTA
// takes a ticket in dependency order, subtracts the contributions of the already solved blocks as
// they are published (bounded waits on per-block flags; a CTA only ever waits for lower tickets, which
// are already running), solves its diagonal block and publishes its rows.
//
//   mode 0  L   : y_j = L_jj^{-1} P_j (b_j - sum_{k<j} L_jk y_k)       (forward, pivots inside block j)
//   mode 1  U   : y_j = U_jj^{-1} (b_j - sum_{k>j} U_jk y_k)           (backward)
//   mode 2  U^H : y_j = U_jj^{-H} (b_j - sum_{k<j} U_kj^H y_k)         (forward)
//   mode 3  L^H : y_j = P_j^T L_jj^{-H} (b_j - sum_{k>j} L_kj^H y_k)   (backward)
//
// Valid when every pivot stays inside its own row block (the factorisation with pivots searched inside
// the diagonal blocks); otherwise the launch-per-panel solver of lu.cu is used.
#include "gdm_internal.cuh"

namespace {

__device__ __forceinline__ uint64_t gtimer_t() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <class C> __device__ __forceinline__ C cz() {
    C v;
    v.x = 0;
    v.y = 0;
    return v;
}
template <class C> __device__ __forceinline__ C conjc(C a) {
    a.y = -a.y;
    return a;
}

// thread 0 waits for flag[k] (or a global abort); returns false on abort/timeout
__device__ bool wait_flag(volatile int *flag, volatile int *abort_flag, int *gflags) {
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        if (*flag == 0) {
            uint64_t t0 = gtimer_t();
            unsigned it = 0;
            while (*flag == 0) {
                __nanosleep(64);
                if ((++it & 255) == 0) {
                    if (*abort_flag) {
                        ok = 0;
                        break;
                    }
                    if (gtimer_t() - t0 > 2000000000ull) {
                        gdm_dev_error(gflags, GDM_ERR_TIMEOUT, 3);
                        *abort_flag = 1;
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <class C, int NBS, int NR>
__global__ void __launch_bounds__(2 * NBS) k_trsv_persistent(const C *__restrict__ A, int64_t lda, int64_t n,
                                                             const int32_t *__restrict__ ipiv, C *__restrict__ B,
                                                             int64_t ldb, int rhs0, int nr_here, int mode,
                                                             int *sync_buf, int *gflags) {
    constexpr int NT = 2 * NBS;
    constexpr int NW = NT / 32;
    __shared__ C acc[NBS][NR];
    __shared__ C yk[NBS][NR];
    __shared__ C part[NBS][NR];
    __shared__ int s_ticket;
    const int nblk = (int)((n + NBS - 1) / NBS);
    int *ticket = sync_buf;
    volatile int *abort_flag = (volatile int *)(sync_buf + 1);
    volatile int *flags = (volatile int *)(sync_buf + 2);
    if (threadIdx.x == 0) s_ticket = atomicAdd(ticket, 1);
    __syncthreads();
    const int tk = s_ticket;
    if (tk >= nblk) return;
    const bool fwd = (mode == 0 || mode == 2);
    const int j = fwd ? tk : nblk - 1 - tk;
    const int64_t r0 = (int64_t)j * NBS;
    const int nr = (int)min((int64_t)NBS, n - r0);
    const int tid = threadIdx.x;
    // initial acc = b_j
    for (int e = tid; e < NBS * NR; e += NT) {
        int r = e / NR, q = e % NR;
        acc[r][q] = (r < nr && q < nr_here) ? B[(int64_t)(rhs0 + q) * ldb + r0 + r] : cz<C>();
    }
    __syncthreads();
    // -------- contributions of the solved blocks
    for (int s = 0; s < tk; s++) {
        const int k = fwd ? s : nblk - 1 - s;
        if (!wait_flag(flags + k, abort_flag, gflags)) return;
        const int64_t k0 = (int64_t)k * NBS;
        const int nk = (int)min((int64_t)NBS, n - k0);
        for (int e = tid; e < NBS * NR; e += NT) {
            int r = e / NR, q = e % NR;
            yk[r][q] = (r < nk && q < nr_here) ? __ldcg(B + (int64_t)(rhs0 + q) * ldb + k0 + r) : cz<C>();
        }
        __syncthreads();
        if (mode <= 1) {
            // acc[r] -= sum_c M[r0+r][k0+c] yk[c]; two threads per row, each half the columns
            const int r = tid % NBS, h = tid / NBS;
            C sum[NR];
#pragma unroll
            for (int q = 0; q < NR; q++) sum[q] = cz<C>();
            if (r < nr) {
                const C *col = A + (k0 + h * (NBS / 2)) * lda + r0 + r;
                const int cend = min(NBS / 2, nk - h * (NBS / 2));
#pragma unroll 8
                for (int c = 0; c < cend; c++) {
                    C m = col[(int64_t)c * lda];
#pragma unroll
                    for (int q = 0; q < NR; q++) cfma(sum[q], m, yk[h * (NBS / 2) + c][q]);
                }
            }
            if (h == 1)
#pragma unroll
                for (int q = 0; q < NR; q++) part[r][q] = sum[q];
            __syncthreads();
            if (h == 0 && r < nr)
#pragma unroll
                for (int q = 0; q < NR; q++) acc[r][q] = csub(acc[r][q], cadd(sum[q], part[r][q]));
        } else {
            // acc[c] -= sum_rr conj(M[k0+rr][r0+c]) yk[rr]; one warp per column (rows across lanes)
            const int w = tid / 32, lane = tid % 32;
            for (int c = w; c < nr; c += NW) {
                const C *col = A + (r0 + c) * lda + k0;
                C sum[NR];
#pragma unroll
                for (int q = 0; q < NR; q++) sum[q] = cz<C>();
                for (int rr = lane; rr < nk; rr += 32) {
                    C m = conjc(col[rr]);
#pragma unroll
                    for (int q = 0; q < NR; q++) cfma(sum[q], m, yk[rr][q]);
                }
#pragma unroll
                for (int q = 0; q < NR; q++)
                    for (int o = 16; o > 0; o >>= 1) {
                        sum[q].x += __shfl_down_sync(0xffffffffu, sum[q].x, o);
                        sum[q].y += __shfl_down_sync(0xffffffffu, sum[q].y, o);
                    }
                if (lane == 0)
#pragma unroll
                    for (int q = 0; q < NR; q++) acc[c][q] = csub(acc[c][q], sum[q]);
            }
        }
        __syncthreads();
    }
    // -------- diagonal block
    const C *D = A + r0 * lda + r0;  // D[r + c*lda]
    if (mode == 0 && tid < NR) {
        // apply the block's row interchanges in order (partners are inside the block)
        for (int t = 0; t < nr; t++) {
            int p = ipiv[r0 + t] - (int)r0;
            if (p != t) {
                C a = acc[t][tid];
                acc[t][tid] = acc[p][tid];
                acc[p][tid] = a;
            }
        }
    }
    __syncthreads();
    // column-oriented substitution in sub-blocks of 32: solve the 32 x 32 diagonal piece with one warp per
    // right-hand side (shuffles), then update the remaining rows of the block
    const bool lower_like = (mode == 0 || mode == 2);
    const int nsub = (nr + 31) / 32;
    for (int si = 0; si < nsub; si++) {
        const int sb = lower_like ? si : nsub - 1 - si;
        const int c0 = sb * 32;
        const int w = min(32, nr - c0);
        const int wi = tid / 32, lane = tid % 32;
        if (wi < NR && wi < nr_here) {
            // T[lane][i]: entry (c0+lane, c0+i) of the effective triangle
            C T[32];
#pragma unroll
            for (int i = 0; i < 32; i++) {
                C v = cz<C>();
                if (lane < w && i < w) {
                    if (mode <= 1) v = D[(int64_t)(c0 + i) * lda + c0 + lane];
                    else v = conjc(D[(int64_t)(c0 + lane) * lda + c0 + i]);
                }
                T[i] = v;
            }
            C v = lane < w ? acc[c0 + lane][wi] : cz<C>();
            const bool unit = (mode == 0 || mode == 3);
            if (lower_like) {
#pragma unroll
                for (int i = 0; i < 32; i++) {
                    if (i < w) {
                        if (!unit && lane == i) v = cmul(v, crecip(T[i]));
                        C xi;
                        xi.x = __shfl_sync(0xffffffffu, v.x, i);
                        xi.y = __shfl_sync(0xffffffffu, v.y, i);
                        if (lane > i && lane < w) cfms(v, T[i], xi);
                    }
                }
            } else {
#pragma unroll
                for (int i = 31; i >= 0; i--) {
                    if (i < w) {
                        if (!unit && lane == i) v = cmul(v, crecip(T[i]));
                        C xi;
                        xi.x = __shfl_sync(0xffffffffu, v.x, i);
                        xi.y = __shfl_sync(0xffffffffu, v.y, i);
                        if (lane < i) cfms(v, T[i], xi);
                    }
                }
            }
            if (lane < w) acc[c0 + lane][wi] = v;
        }
        __syncthreads();
        // update rows of the block not yet solved with the 32 solved values
        const int ub = lower_like ? c0 + w : 0;
        const int ue = lower_like ? nr : c0;
        for (int r = ub + tid; r < ue; r += NT) {
            C sum[NR];
#pragma unroll
            for (int q = 0; q < NR; q++) sum[q] = cz<C>();
            for (int i = 0; i < w; i++) {
                C m;
                if (mode <= 1) m = D[(int64_t)(c0 + i) * lda + r];
                else m = conjc(D[(int64_t)r * lda + c0 + i]);
#pragma unroll
                for (int q = 0; q < NR; q++) cfma(sum[q], m, acc[c0 + i][q]);
            }
#pragma unroll
            for (int q = 0; q < NR; q++) acc[r][q] = csub(acc[r][q], sum[q]);
        }
        __syncthreads();
    }
    if (mode == 3 && tid < NR) {
        for (int t = nr - 1; t >= 0; t--) {
            int p = ipiv[r0 + t] - (int)r0;
            if (p != t) {
                C a = acc[t][tid];
                acc[t][tid] = acc[p][tid];
                acc[p][tid] = a;
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < nr * NR; e += NT) {
        int r = e / NR, q = e % NR;
        if (q < nr_here) B[(int64_t)(rhs0 + q) * ldb + r0 + r] = acc[r][q];
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicExch((int *)(flags + j), 1);
}

// every pivot inside its own block of NBS rows?
__global__ void k_pivots_local(const int32_t *__restrict__ ipiv, int64_t n, int nbs, int *bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (ipiv[i] / nbs != i / nbs) atomicExch(bad, 1);
}

template <class C, int NBS>
gdm_status launch_modes(gdm_ctx *ctx, const C *A, int64_t lda, int64_t n, const int32_t *ipiv, C *B, int64_t ldb,
                        int n_rhs, const int *modes, int nmodes, int *sync_buf) {
    const int nblk = (int)((n + NBS - 1) / NBS);
    for (int mi = 0; mi < nmodes; mi++) {
        for (int q0 = 0; q0 < n_rhs; q0 += 2) {
            int nr = n_rhs - q0 < 2 ? n_rhs - q0 : 2;
            GDM_CUDA_TRY(ctx, cudaMemsetAsync(sync_buf, 0, sizeof(int) * (nblk + 2), ctx->stream));
            k_trsv_persistent<C, NBS, 2><<<nblk, 2 * NBS, 0, ctx->stream>>>(A, lda, n, ipiv, B, ldb, q0, nr, modes[mi],
                                                                            sync_buf, ctx->dflags);
            GDM_LAUNCHED(ctx, "trsv_persistent");
        }
    }
    return GDM_OK;
}

}  // namespace

size_t gdm_trsv_sync_bytes(int64_t n) { return sizeof(int) * ((n + 127) / 128 + 8); }

// 1 if all pivots stay inside their NBS-row block (synchronises)
gdm_status gdm_pivots_local(gdm_ctx *ctx, const int32_t *ipiv, int64_t n, int nbs, int *sync_buf, int *local) {
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(sync_buf, 0, sizeof(int), ctx->stream));
    k_pivots_local<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(ipiv, n, nbs, sync_buf);
    GDM_LAUNCHED(ctx, "pivots_local");
    int *h;
    GDM_TRY(gdm_pinned(ctx, 64, (void **)&h));
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(h, sync_buf, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    *local = (*h == 0);
    return GDM_OK;
}

// solve with the factors: conj_trans = 0: U^{-1} L^{-1} P b; conj_trans = 1: P^T L^{-H} U^{-H} b
gdm_status gdm_trsv_persistent(gdm_ctx *ctx, gdm_precision prec, const void *A, int64_t n, int64_t lda,
                               const int32_t *ipiv, void *B, int64_t ldb, int n_rhs, int conj_trans, int *sync_buf) {
    static const int fwd[2] = {0, 1}, adj[2] = {2, 3};
    const int *modes = conj_trans ? adj : fwd;
    if (prec == GDM_FP64)
        return launch_modes<double2, 128>(ctx, (const double2 *)A, lda, n, ipiv, (double2 *)B, ldb, n_rhs, modes, 2,
                                          sync_buf);
    return launch_modes<float2, 256>(ctx, (const float2 *)A, lda, n, ipiv, (float2 *)B, ldb, n_rhs, modes, 2, sync_buf);
}
