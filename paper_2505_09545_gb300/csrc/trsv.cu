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
                                                             const C *__restrict__ dinv, int *sync_buf, int *gflags) {
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
        const int64_t k0 = (int64_t)k * NBS;
        const int nk = (int)min((int64_t)NBS, n - k0);
        {
            // pull this dependency block into L2 while (possibly) waiting for its solution
            const int64_t cb = (mode <= 1) ? k0 : r0;  // first column of the block read below
            const int64_t rb = (mode <= 1) ? r0 : k0;  // first row
            const int ncol = (mode <= 1) ? nk : nr, nrow = (mode <= 1) ? nr : nk;
            const int lines_per_col = (int)((nrow * sizeof(C) + 127) / 128);
            for (int e = tid; e < ncol * lines_per_col; e += NT) {
                const char *ptr = (const char *)(A + (cb + e / lines_per_col) * lda + rb) + (e % lines_per_col) * 128;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
            }
        }
        if (!wait_flag(flags + k, abort_flag, gflags)) return;
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
#pragma unroll 16
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
    // diagonal block in pieces of 32: x_s = inv(T_ss) acc_s with the precomputed 32 x 32 inverses of the
    // factors' diagonal pieces (conjugate-transposed for the adjoint modes), then update the remaining rows
    const bool lower_like = (mode == 0 || mode == 2);
    const int nsub = (nr + 31) / 32;
    const int use_u = (mode == 1 || mode == 2);
    const bool herm = (mode >= 2);
    for (int si = 0; si < nsub; si++) {
        const int sb = lower_like ? si : nsub - 1 - si;
        const int c0 = sb * 32;
        const int w = min(32, nr - c0);
        const C *Ti = dinv + ((int64_t)2 * ((r0 + c0) / 32) + use_u) * 1024;
        __syncthreads();
        // x[row][q] = sum_i Tinv_eff[row][i] acc[c0+i][q]; one thread per (row, q)
        C xv = cz<C>();
        const int row = tid % 32, q = tid / 32;
        if (q < NR && row < w) {
            C m[32];
#pragma unroll
            for (int i = 0; i < 32; i++) m[i] = herm ? conjc(Ti[i * 32 + row]) : Ti[row * 32 + i];
#pragma unroll
            for (int i = 0; i < 32; i++)
                if (i < w) cfma(xv, m[i], acc[c0 + i][q]);
        }
        __syncthreads();
        if (q < NR && row < w) acc[c0 + row][q] = xv;
        __syncthreads();
        const int ub = lower_like ? c0 + w : 0;
        const int ue = lower_like ? nr : c0;
        for (int r = ub + tid; r < ue; r += NT) {
            C sum[NR];
#pragma unroll
            for (int qq = 0; qq < NR; qq++) sum[qq] = cz<C>();
            C m[32];
#pragma unroll
            for (int i = 0; i < 32; i++) {
                if (i < w) m[i] = (mode <= 1) ? D[(int64_t)(c0 + i) * lda + r] : conjc(D[(int64_t)r * lda + c0 + i]);
            }
#pragma unroll
            for (int i = 0; i < 32; i++)
                if (i < w)
#pragma unroll
                    for (int qq = 0; qq < NR; qq++) cfma(sum[qq], m[i], acc[c0 + i][qq]);
#pragma unroll
            for (int qq = 0; qq < NR; qq++) acc[r][qq] = csub(acc[r][qq], sum[qq]);
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

// Inverses of the 32 x 32 diagonal pieces of L (unit lower) and U (upper) of every panel:
// inv[(2*p + 0)*1024 + r*32 + c] = (L_pp^{-1})[r][c], inv[(2*p + 1)*1024 + r*32 + c] = (U_pp^{-1})[r][c].
// One warp per triangle; lane c computes column c of the inverse by substitution on e_c.
template <class C>
__global__ void k_diag_inverses(const C *__restrict__ A, int64_t lda, int64_t n, C *__restrict__ inv) {
    // one warp (block) per triangle
    const int warp = blockIdx.x, lane = threadIdx.x & 31;
    const int np = (int)((n + 31) / 32);
    if (warp >= 2 * np) return;
    const int p = warp / 2, up = warp & 1;
    const int64_t c0 = (int64_t)p * 32;
    const int w = (int)min((int64_t)32, n - c0);
    __shared__ C t[32][33];
    for (int r = 0; r < 32; r++) {
        C v = cz<C>();
        if (r < w && lane < w) v = A[(c0 + lane) * lda + c0 + r];
        t[r][lane] = v;  // t[row][col]
    }
    __syncwarp();
    C x[32];
#pragma unroll
    for (int r = 0; r < 32; r++) x[r] = cz<C>();
    if (lane < w) {
        if (!up) {
            // L x = e_lane, unit lower: forward
#pragma unroll
            for (int r = 0; r < 32; r++) {
                if (r < w) {
                    C v = (r == lane) ? C{1, 0} : cz<C>();
#pragma unroll
                    for (int j = 0; j < 32; j++)
                        if (j < r) cfms(v, t[r][j], x[j]);
                    x[r] = v;
                }
            }
        } else {
            // U x = e_lane: backward with division by the diagonal
#pragma unroll
            for (int r = 31; r >= 0; r--) {
                if (r < w) {
                    C v = (r == lane) ? C{1, 0} : cz<C>();
#pragma unroll
                    for (int j = 0; j < 32; j++)
                        if (j > r && j < w) cfms(v, t[r][j], x[j]);
                    x[r] = cmul(v, crecip(t[r][r]));
                }
            }
        }
    }
    C *o = inv + ((int64_t)2 * p + up) * 1024;
#pragma unroll
    for (int r = 0; r < 32; r++) o[r * 32 + lane] = x[r];
}

// every pivot inside its own block of NBS rows?
__global__ void k_pivots_local(const int32_t *__restrict__ ipiv, int64_t n, int nbs, int *bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (ipiv[i] / nbs != i / nbs) atomicExch(bad, 1);
}

template <class C, int NBS>
gdm_status launch_modes(gdm_ctx *ctx, const C *A, int64_t lda, int64_t n, const int32_t *ipiv, C *B, int64_t ldb,
                        int n_rhs, const int *modes, int nmodes, int *sync_buf, C *dinv) {
    const int nblk = (int)((n + NBS - 1) / NBS);
    for (int mi = 0; mi < nmodes; mi++) {
        for (int q0 = 0; q0 < n_rhs; q0 += 2) {
            int nr = n_rhs - q0 < 2 ? n_rhs - q0 : 2;
            GDM_CUDA_TRY(ctx, cudaMemsetAsync(sync_buf, 0, sizeof(int) * (nblk + 2), ctx->stream));
            k_trsv_persistent<C, NBS, 2><<<nblk, 2 * NBS, 0, ctx->stream>>>(A, lda, n, ipiv, B, ldb, q0, nr, modes[mi],
                                                                            dinv, sync_buf, ctx->dflags);
            GDM_LAUNCHED(ctx, "trsv_persistent");
        }
    }
    return GDM_OK;
}

}  // namespace

size_t gdm_trsv_sync_bytes(int64_t n) { return sizeof(int) * ((n + 127) / 128 + 8); }

// bytes of the diagonal-piece inverses (complex128 size, enough for both precisions)
size_t gdm_trsv_inv_bytes(int64_t n) { return (size_t)2 * ((n + 31) / 32) * 1024 * sizeof(double2); }

gdm_status gdm_trsv_prepare(gdm_ctx *ctx, gdm_precision prec, const void *A, int64_t n, int64_t lda, void *dinv) {
    const int np = (int)((n + 31) / 32);
    const unsigned blocks = (unsigned)(2 * np);
    if (prec == GDM_FP64)
        k_diag_inverses<double2><<<blocks, 32, 0, ctx->stream>>>((const double2 *)A, lda, n, (double2 *)dinv);
    else
        k_diag_inverses<float2><<<blocks, 32, 0, ctx->stream>>>((const float2 *)A, lda, n, (float2 *)dinv);
    GDM_LAUNCHED(ctx, "diag_inverses");
    return GDM_OK;
}

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
                               const int32_t *ipiv, void *B, int64_t ldb, int n_rhs, int conj_trans, int *sync_buf,
                               const void *dinv) {
    static const int fwd[2] = {0, 1}, adj[2] = {2, 3};
    const int *modes = conj_trans ? adj : fwd;
    if (prec == GDM_FP64)
        return launch_modes<double2, 128>(ctx, (const double2 *)A, lda, n, ipiv, (double2 *)B, ldb, n_rhs, modes, 2,
                                          sync_buf, (double2 *)dinv);
    return launch_modes<float2, 256>(ctx, (const float2 *)A, lda, n, ipiv, (float2 *)B, ldb, n_rhs, modes, 2, sync_buf,
                                     (float2 *)dinv);
}
