// Blocked complex LU factorisation with partial pivoting and blocked triangular solves
// (Sec. "Numerical solution": the GDM system is solved by LU decomposition).
//
// Storage: column-major complex (float2 or double2), leading dimension lda.
// Algorithm: right-looking blocked LU with outer block NB and panels of width NBP:
//   for each outer block [b0, b0+nb):
//     for each panel [c0, c0+w) inside the block:
//       factor the tall panel rows [c0, n) with partial pivoting (cooperative kernel: the panel rows
//         live in the shared memory of up to one CTA per SM, one bounded grid barrier per column);
//       swap the same rows in the other columns of the block; triangular solve + GEMM update of the
//         block's remaining columns;
//     swap the block's pivot rows in the trailing columns, U12 = L11^{-1} A12, A22 -= A21 U12.
// Columns to the left of a panel are never swapped: L is kept in the row order of the step that produced
// it, and the forward solve applies each panel's row swaps to the right-hand side just before using that
// panel's columns of L (the product form y = L_S^{-1} P_S ... L_1^{-1} P_1 b at panel granularity).
// For the FP32 precisions the trailing update A22 -= A21 U12 runs on the tcgen05 tensor cores
// (lu_tc.cu); everything else uses the SIMT kernels of this file.
#include <cooperative_groups.h>
#include <nvtx3/nvToolsExt.h>
#include <stdlib.h>

#include "gdm_internal.cuh"

#define NBP 32        // panel width (columns per cooperative panel factorisation)
#define PANEL_THREADS 256

// tensor-core trailing update (lu_tc.cu); returns GDM_ERR_UNSUPPORTED when not applicable
gdm_status gdm_tc_trailing_update(gdm_ctx *ctx, gdm_precision prec, float2 *A, int64_t lda, int64_t n, int64_t b0,
                                  int64_t nb, void *ws, size_t ws_bytes);
size_t gdm_tc_workspace_bytes(int64_t n, int64_t nb, gdm_precision prec);
gdm_status gdm_tc_update_ext(gdm_ctx *ctx, gdm_precision prec, float2 *C, int64_t ldc, int64_t r0, int64_t c0,
                             const float2 *L, int64_t ldl, const float2 *U, int64_t ldu, int64_t u_r0, int64_t u_c0,
                             int64_t Mc, int64_t Nc, int64_t Kc, void *ws, size_t ws_bytes, int prof,
                             int u_is_tf32, int out_mode = 0);
gdm_status gdm_tc_update(gdm_ctx *ctx, gdm_precision prec, float2 *A, int64_t lda, int64_t n, int64_t r0, int64_t c0,
                         int64_t k0, int64_t Mc, int64_t Nc, int64_t Kc, void *ws, size_t ws_bytes, int prof);
gdm_status gdm_tc_update_lx(gdm_ctx *ctx, float2 *C, int64_t ldc, int64_t r0, int64_t c0, const float *Lx,
                            int64_t lx_pitch, const float2 *U, int64_t ldu, int64_t u_r0, int64_t u_c0, int64_t Mc,
                            int64_t Nc, int64_t Kc, int prof);

// ------------------------------------------------------------------ bounded grid barrier
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// All CTAs of a cooperative launch meet here. Gives up after ~2 s (sets GDM_ERR_TIMEOUT and
// returns false) instead of spinning forever.
__device__ bool grid_barrier(int *flags, unsigned nblocks) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile int *vgen = flags + GDM_FLAG_BAR_GEN;
        int g = *vgen;
        __threadfence();
        int arrived = atomicAdd(flags + GDM_FLAG_BAR_COUNT, 1);
        if (arrived == (int)nblocks - 1) {
            atomicExch(flags + GDM_FLAG_BAR_COUNT, 0);
            __threadfence();
            atomicAdd(flags + GDM_FLAG_BAR_GEN, 1);
        } else {
            uint64_t t0 = globaltimer_ns();
            unsigned it = 0;
            while (*vgen == g) {
                __nanosleep(32);
                if ((++it & 1023) == 0 && (globaltimer_ns() - t0 > 2000000000ull || it > (1u << 26))) {
                    gdm_dev_error(flags, GDM_ERR_TIMEOUT, 1);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// ------------------------------------------------------------------ panel factorisation
template <class C> struct PanelScratch {
    double *cand_val;  // [2][P]
    int64_t *cand_row; // [2][P]
    C *cand_vals;      // [2][P][NBP]
    C *top_row;        // [2][NBP]
};

template <class T> __device__ __forceinline__ T ld_cg(const T *p);
template <> __device__ __forceinline__ float2 ld_cg<float2>(const float2 *p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 ld_cg<double2>(const double2 *p) { return __ldcg(p); }

// Factor rows [c0, n) x cols [c0, c0+w) in place. CTA b owns rows [c0 + b*rpc, c0 + (b+1)*rpc).
template <class C>
__global__ void __launch_bounds__(PANEL_THREADS) k_panel(C *__restrict__ A, int64_t lda, int64_t n, int64_t c0, int w,
                                                         int rpc, int32_t *__restrict__ ipiv, PanelScratch<C> ps,
                                                         int *flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tile = (C *)smem_raw;  // [NBP][rpc], column-major
    __shared__ C prow[NBP];
    __shared__ double wv[PANEL_THREADS / 32];
    __shared__ int64_t wr[PANEL_THREADS / 32];
    __shared__ int64_t s_wrow;
    __shared__ double s_wval;
    __shared__ int s_wcta;
    const unsigned P = gridDim.x;
    const int b = blockIdx.x;
    const int64_t r0 = c0 + (int64_t)b * rpc;
    const int nr = (int)max((int64_t)0, min((int64_t)rpc, n - r0));
    // load
    for (int c = 0; c < w; c++)
        for (int lr = threadIdx.x; lr < nr; lr += PANEL_THREADS) tile[c * rpc + lr] = A[(c0 + c) * lda + r0 + lr];
    __syncthreads();
    for (int t = 0; t < w; t++) {
        const int par = t & 1;
        // 1. local argmax of |re| + |im| over eligible rows (global row >= c0 + t)
        int lstart = (b == 0) ? t : 0;
        double best = -1.0;
        int64_t brow = INT64_MAX;
        for (int lr = lstart + threadIdx.x; lr < nr; lr += PANEL_THREADS) {
            double v = (double)cabs1(tile[t * rpc + lr]);
            if (v > best) {
                best = v;
                brow = r0 + lr;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_down_sync(0xffffffffu, best, o);
            int64_t orow = __shfl_down_sync(0xffffffffu, brow, o);
            if (ov > best || (ov == best && orow < brow)) {
                best = ov;
                brow = orow;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            wv[threadIdx.x >> 5] = best;
            wr[threadIdx.x >> 5] = brow;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < PANEL_THREADS / 32; k++)
                if (wv[k] > best || (wv[k] == best && wr[k] < brow)) {
                    best = wv[k];
                    brow = wr[k];
                }
            s_wval = best;
            s_wrow = brow;
        }
        __syncthreads();
        best = s_wval;
        brow = s_wrow;
        if (P > 1) {
            // 2. publish candidate (and the current top row from CTA 0)
            if (threadIdx.x == 0) {
                ps.cand_val[par * P + b] = best;
                ps.cand_row[par * P + b] = (best >= 0.0) ? brow : INT64_MAX;
            }
            if (threadIdx.x < w) {
                if (best >= 0.0) ps.cand_vals[((size_t)par * P + b) * NBP + threadIdx.x] = tile[threadIdx.x * rpc + (brow - r0)];
                if (b == 0) ps.top_row[par * NBP + threadIdx.x] = tile[threadIdx.x * rpc + t];
            }
            // 3. all CTAs meet
            if (!grid_barrier(flags, P)) return;
            // 4. global winner (max value, lowest row on ties)
            if (threadIdx.x < 32) {
                double v = -2.0;
                int64_t rr = INT64_MAX;
                int cb = 0;
                for (int k = threadIdx.x; k < (int)P; k += 32) {
                    double kv = __ldcg(ps.cand_val + par * P + k);
                    int64_t kr = __ldcg((const long long *)(ps.cand_row + par * P + k));
                    if (kv > v || (kv == v && kr < rr)) {
                        v = kv;
                        rr = kr;
                        cb = k;
                    }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    double ov = __shfl_down_sync(0xffffffffu, v, o);
                    int64_t orr = __shfl_down_sync(0xffffffffu, rr, o);
                    int ocb = __shfl_down_sync(0xffffffffu, cb, o);
                    if (ov > v || (ov == v && orr < rr)) {
                        v = ov;
                        rr = orr;
                        cb = ocb;
                    }
                }
                if (threadIdx.x == 0) {
                    s_wval = v;
                    s_wrow = rr;
                    s_wcta = cb;
                }
            }
            __syncthreads();
            if (threadIdx.x < w) prow[threadIdx.x] = ld_cg(ps.cand_vals + ((size_t)par * P + s_wcta) * NBP + threadIdx.x);
        } else {
            if (threadIdx.x < w) prow[threadIdx.x] = tile[threadIdx.x * rpc + (brow - r0)];
        }
        __syncthreads();
        const int64_t wrow = s_wrow;
        const double wval = s_wval;
        const int64_t prow_g = c0 + t;
        if (b == 0 && threadIdx.x == 0) {
            ipiv[prow_g] = (int32_t)wrow;
            if (!(wval > 0.0)) gdm_dev_error(flags, GDM_ERR_SINGULAR, (int)prow_g);
        }
        // 5. swap rows prow_g <-> wrow inside the panel
        if (wrow != prow_g) {
            int64_t owner = (wrow - c0) / rpc;
            if (owner == b && threadIdx.x < w) {
                C old = (P > 1) ? ld_cg(ps.top_row + par * NBP + threadIdx.x) : tile[threadIdx.x * rpc + t];
                tile[threadIdx.x * rpc + (wrow - r0)] = old;
            }
            __syncthreads();
            if (b == 0 && threadIdx.x < w) tile[threadIdx.x * rpc + t] = prow[threadIdx.x];
        }
        __syncthreads();
        // 6. scale the pivot column and update the rest of the panel
        C pv = prow[t];
        C inv;
        if (cabs1(pv) > 0) inv = crecip(pv);
        else {
            inv.x = 0;
            inv.y = 0;
        }
        int ustart = (b == 0) ? t + 1 : 0;
        for (int lr = ustart + threadIdx.x; lr < nr; lr += PANEL_THREADS) {
            C l = cmul(tile[t * rpc + lr], inv);
            tile[t * rpc + lr] = l;
            for (int c = t + 1; c < w; c++) cfms(tile[c * rpc + lr], l, prow[c]);
        }
        __syncthreads();
    }
    for (int c = 0; c < w; c++)
        for (int lr = threadIdx.x; lr < nr; lr += PANEL_THREADS) A[(c0 + c) * lda + r0 + lr] = tile[c * rpc + lr];
}

// ------------------------------------------------------------------ panel with pivoting inside the diagonal block
// Factor rows [c0, n) x cols [c0, c0+w): every CTA factors the w x w diagonal block D with partial pivoting
// among D's own rows (so the rows below never move), then solves its share of the rows below:
// L21 = A21 U11^{-1}. No grid-wide synchronisation. Certificate: for every row below and column k the
// updated entry (before division by the pivot) is compared with the pivot in |re|+|im|; the largest ratio
// is recorded in growth[0] (as float bits). A ratio <= 1 means the pivots are exactly those of partial
// pivoting over the whole column (rows of D win ties, as they have the lower index).
// Every CTA of a panel launch reads the unfactored diagonal block from A at its start, so the factored
// block may only be stored once no CTA can still read it: the last CTA to finish (ticket in the flags)
// stores its own copy and returns the ticket to 0 for the next launch.
// (ticket: the finish counter; nblk: the CTAs that factor this panel)
template <class C>
__device__ void panel_store_diag_last(C *A, int64_t lda, int64_t c0, int w, const C *D, int ldd, int *ticket,
                                      int nblk) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1) == nblk - 1;
    }
    __syncthreads();
    if (!s_last) return;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
        int r = e % w, c = e / w;
        A[(c0 + c) * lda + c0 + r] = D[r * ldd + c];
    }
    if (threadIdx.x == 0) atomicExch(ticket, 0);
}
template <class C>
__device__ void panel_store_diag_last(C *A, int64_t lda, int64_t c0, int w, const C *D, int ldd, int *flags) {
    panel_store_diag_last(A, lda, c0, w, D, ldd, &flags[GDM_FLAG_PANEL_TICKET], (int)gridDim.x);
}

template <class C>
__global__ void __launch_bounds__(256) k_panel_local(C *__restrict__ A, int64_t lda, int64_t n, int64_t c0, int w,
                                                     int32_t *__restrict__ ipiv, unsigned *growth, int *flags) {
    typedef decltype(C().x) T;
    __shared__ C D[NBP][NBP + 1];   // diagonal block, factored in place (L strictly below, U on and above)
    __shared__ C Ui[NBP][NBP + 1];  // U^{-1}
    for (int e = threadIdx.x; e < NBP * NBP; e += blockDim.x) {
        int r = e % NBP, c = e / NBP;
        C v;
        v.x = 0;
        v.y = 0;
        if (r < w && c < w) v = A[(c0 + c) * lda + c0 + r];
        D[r][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // one warp: partial pivoting among the block's rows; lane = row for the search, column for the swap
        const int lane = threadIdx.x;
        for (int t = 0; t < w; t++) {
            double v = (lane >= t && lane < w) ? (double)cabs1(D[lane][t]) : -1.0;
            int idx = lane;
            for (int o = 16; o > 0; o >>= 1) {
                double ov = __shfl_down_sync(0xffffffffu, v, o);
                int oi = __shfl_down_sync(0xffffffffu, idx, o);
                if (ov > v || (ov == v && oi < idx)) {
                    v = ov;
                    idx = oi;
                }
            }
            const int p = __shfl_sync(0xffffffffu, idx, 0);
            const double pv = __shfl_sync(0xffffffffu, v, 0);
            if (blockIdx.x == 0 && lane == 0) {
                ipiv[c0 + t] = (int32_t)(c0 + p);
                if (!(pv > 0.0)) gdm_dev_error(flags, GDM_ERR_SINGULAR, (int)(c0 + t));
            }
            if (p != t && lane < w) {
                C a = D[t][lane];
                D[t][lane] = D[p][lane];
                D[p][lane] = a;
            }
            __syncwarp();
            C piv = D[t][t];
            C inv;
            if (cabs1(piv) > 0) inv = crecip(piv);
            else {
                inv.x = 0;
                inv.y = 0;
            }
            if (lane > t && lane < w) {
                C l = cmul(D[lane][t], inv);
                D[lane][t] = l;
                for (int c = t + 1; c < w; c++) cfms(D[lane][c], l, D[t][c]);
            }
            __syncwarp();
        }
        // U^{-1}, one column per lane (back substitution)
        if (lane < w) {
            for (int r = w - 1; r >= 0; r--) {
                C sacc;
                sacc.x = (r == lane) ? 1 : 0;
                sacc.y = 0;
                for (int j = r + 1; j < w; j++) cfms(sacc, D[r][j], Ui[j][lane]);
                C d = D[r][r];
                Ui[r][lane] = cabs1(d) > 0 ? cmul(sacc, crecip(d)) : sacc;
            }
        }
    }
    __syncthreads();
    // rows below the diagonal block: L21 = A21 U^{-1}; certificate from l_k U_kk (the updated entry that
    // partial pivoting would have compared with the pivot U_kk)
    float worst = 0.f;
    for (int64_t r = c0 + w + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        C x[NBP];
#pragma unroll
        for (int j = 0; j < NBP; j++)
            if (j < w) x[j] = A[(c0 + j) * lda + r];
        for (int k = 0; k < w; k++) {
            C l;
            l.x = 0;
            l.y = 0;
#pragma unroll
            for (int j = 0; j < NBP; j++)
                if (j <= k) cfma(l, x[j], Ui[j][k]);
            T pa = cabs1(D[k][k]);
            if (pa > 0) worst = fmaxf(worst, (float)(cabs1(cmul(l, D[k][k])) / pa));
            A[(c0 + k) * lda + r] = l;
        }
    }
    for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_down_sync(0xffffffffu, worst, o));
    if ((threadIdx.x & 31) == 0 && worst > 0.f) atomicMax(growth, __float_as_uint(worst));
    panel_store_diag_last(A, lda, c0, w, &D[0][0], NBP + 1, flags);
}

// 1/x for normal positive x: approximate reciprocal + one Newton step (relative error ~1 ulp)
__device__ __forceinline__ float rcp_nr(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r * fmaf(-x, r, 2.0f);
}

// FP32 version of the same panel, written as compact loops: every CTA factors the 32 x 32 diagonal block in
// warp 0 and then solves its rows below, and straight-line code for either part (the 32 steps unrolled) runs
// once per warp and stalls on instruction fetch, so both parts are runtime loops over the step k whose bodies
// touch registers at fixed indices only. A lane keeps the not yet eliminated part of its row shifted to the
// front of a register window, x[i] = column k + i, so that column k is always x[0]; each step removes x[0]
// and shifts the window by one while it subtracts the multiple of the pivot row. U is kept in shared memory
// in position order, zero-padded to 64 columns, so the window's reads past column 31 see zeros.
// Pivoting as in k_panel_local: lane q of warp 0 holds row q of the diagonal block and tracks the position
// its row occupies in the LAPACK-style swap sequence (pos); the pivot of step t is the largest |re|+|im| in
// column t among the rows not yet chosen, ties going to the lowest current position (two warp reductions:
// the maximum of the magnitudes' bit patterns, then the lowest position attaining it); ipiv[t] is the
// position the chosen row occupied. The rows below solve x U = a by forward substitution, in four phases
// whose windows shrink with the remaining columns (32, 24, 16, 8), with the growth certificate of
// k_panel_local.
__device__ __forceinline__ float2 cmul_inv_piv(float2 a, float2 piv) {
    // a / piv with 1/piv = conj(piv/sc) / (|piv/sc|^2 sc) (scaled against overflow), reciprocals from the
    // hardware approximation refined by one Newton step
    const float sc = fmaxf(fabsf(piv.x), fabsf(piv.y));
    if (!(sc > 0.f)) return make_float2(0.f, 0.f);
    const float is = rcp_nr(sc);
    const float ax = piv.x * is, ay = piv.y * is;
    const float rr = rcp_nr(fmaf(ax, ax, ay * ay) * sc);
    return cmul(a, make_float2(ax * rr, -ay * rr));
}

// one forward-substitution step on a window of W unknowns (x[0] = column k): returns the multiplier and
// shifts the window, x[i] <- x[i + 1] - l U[k][k + 1 + i]
template <int W>
__device__ __forceinline__ float2 subst_step(float2 *x, const float2 *__restrict__ Urow, float2 invd_k) {
    const float2 l = cmul(x[0], invd_k);
#pragma unroll
    for (int i = 0; i < W - 1; i++) {
        x[i] = x[i + 1];
        cfms(x[i], l, Urow[1 + i]);
    }
    x[W - 1] = make_float2(0.f, 0.f);
    return l;
}

// one elimination step of the diagonal block on a window of W columns (r[0] = column t). (m, key) is the
// pivot of column t, found by the previous step: the chosen row publishes itself into U, the others take
// their multiplier and the shifted update. Column t + 1 is updated first and its pivot search (two warp
// reductions: the maximum of the magnitudes' bit patterns among the rows not yet chosen, then the lowest
// position attaining it) is issued before the rest of the update, which hides the reductions' latency. The
// update is unconditional (multiplier 0 for rows already chosen, whose registers are not read again).
template <int W>
__device__ __forceinline__ void diag_step(float2 *r, int t, int lane, int &pos, bool &done, unsigned &m,
                                          unsigned &key, float2 (*Uz)[2 * NBP], float2 (*Lr)[NBP + 1], int64_t c0,
                                          int32_t *__restrict__ ipiv, int *flags, bool first) {
    if (first && lane == 0) {
        ipiv[c0 + t] = (int32_t)(c0 + key);
        if (!(__uint_as_float(m) > 0.f)) gdm_dev_error(flags, GDM_ERR_SINGULAR, (int)(c0 + t));
    }
    const bool is_p = !done && pos == (int)key;
    if (is_p) {
#pragma unroll
        for (int i = 0; i < W; i++) Uz[t][t + i] = r[i];
    }
    // the row at position t moves to the pivot's old position
    if (pos == t) pos = (int)key;
    if (is_p) {
        pos = t;
        done = true;
    }
    __syncwarp();
    const float2 l = done ? make_float2(0.f, 0.f) : cmul_inv_piv(r[0], Uz[t][t]);
    Lr[lane][t] = l;
    float2 n0 = r[1];
    cfms(n0, l, Uz[t][t + 1]);
    // |re|+|im| >= 0, so its bit pattern orders like the value
    const unsigned vb = done ? 0u : __float_as_uint(fabsf(n0.x) + fabsf(n0.y));
    m = __reduce_max_sync(0xffffffffu, vb);
    key = __reduce_min_sync(0xffffffffu, (!done && vb == m) ? (unsigned)pos : 0xffffffffu);
#pragma unroll
    for (int i = 1; i < W - 1; i++) {
        r[i] = r[i + 1];
        cfms(r[i], l, Uz[t][t + 1 + i]);
    }
    r[0] = n0;
    r[W - 1] = make_float2(0.f, 0.f);
}

// Warp-wide factorisation of a w x w diagonal block at (c0, c0) whose row `lane` is in r (zero beyond w,
// destroyed): the pivots to ipiv (first: this CTA records them and a zero pivot), U in position order into
// Uz (zero-padded beyond the block by the caller), every row's multipliers by step into Lr[lane], and each
// row's final position into posof.
__device__ __forceinline__ void diag_factor_warp(float2 *r, int w, int lane, float2 (*Uz)[2 * NBP],
                                                 float2 (*Lr)[NBP + 1], int *posof, int64_t c0,
                                                 int32_t *__restrict__ ipiv, int *flags, bool first) {
    int pos = lane;         // current position of this lane's row
    bool done = lane >= w;  // chosen as a pivot row already (or outside the block)
    // pivot of column 0; every step then finds the next one
    const unsigned vb0 = done ? 0u : __float_as_uint(fabsf(r[0].x) + fabsf(r[0].y));
    unsigned m = __reduce_max_sync(0xffffffffu, vb0);
    unsigned key = __reduce_min_sync(0xffffffffu, (!done && vb0 == m) ? (unsigned)pos : 0xffffffffu);
    // windows shrink with the columns left: 32 - t <= W
    int t = 0;
#pragma unroll 1
    for (; t < w && t < 8; t++) diag_step<32>(r, t, lane, pos, done, m, key, Uz, Lr, c0, ipiv, flags, first);
#pragma unroll 1
    for (; t < w && t < 16; t++) diag_step<24>(r, t, lane, pos, done, m, key, Uz, Lr, c0, ipiv, flags, first);
#pragma unroll 1
    for (; t < w && t < 24; t++) diag_step<16>(r, t, lane, pos, done, m, key, Uz, Lr, c0, ipiv, flags, first);
#pragma unroll 1
    for (; t < w; t++) diag_step<8>(r, t, lane, pos, done, m, key, Uz, Lr, c0, ipiv, flags, first);
    if (lane < w) posof[lane] = pos;
}

// Forward substitution of one row x (its 32 entries in a full panel's columns, destroyed) against the
// panel's factored diagonal block (U in position order Uz, reciprocal pivots invd, 1 / |pivot| inv_pa): the
// multipliers to lout[k] and, unless acol is null, to acol[k lda] (column k of the panel in this row);
// the certificate's largest ratio into worst. Four phases whose windows shrink with the columns left.
__device__ __forceinline__ void subst_row32(float2 *x, float2 (*Uz)[2 * NBP], const float2 *invd,
                                            const float *inv_pa, float2 *lout, float2 *acol, int64_t lda,
                                            float &worst) {
#define SUBST_PHASE(W_, KEND)                                                                      \
    for (; k < (KEND); k++) {                                                                      \
        worst = fmaxf(worst, (fabsf(x[0].x) + fabsf(x[0].y)) * inv_pa[k]);                        \
        const float2 l_ = subst_step<W_>(x, &Uz[k][k], invd[k]);                                   \
        lout[k] = l_;                                                                              \
        if (acol) acol[k * lda] = l_;                                                              \
    }
    int k = 0;
#pragma unroll 1
    SUBST_PHASE(32, 8)
#pragma unroll 1
    SUBST_PHASE(24, 16)
#pragma unroll 1
    SUBST_PHASE(16, 24)
#pragma unroll 1
    SUBST_PHASE(8, 32)
#undef SUBST_PHASE
}

// The body is shared with the grouped panel of a batch (GROUPED): CTA bid of nblk factoring this panel, the
// finish counter in *ticket, and the multipliers of every full panel also written, rounded to TF32, into the
// real embedding that the batch's tensor-core updates read (Lx: real rows 2 (r - b0) and 2 (r - b0) + 1,
// columns lx_col .. lx_col + 64 of rows of lx_pitch floats), so that no separate pass reads L again. There
// the rows run in CTA-wide rounds whose multipliers pass through shared memory (Ls, dynamic), so that the
// embedding goes out in coalesced 16-byte stores.
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
template <bool GROUPED>
__device__ __forceinline__ void panel_f32_body(float2 *__restrict__ A, int64_t lda, int64_t n, int64_t c0, int w,
                                               int32_t *__restrict__ ipiv, unsigned *growth, int *ticket,
                                               int *flags, int bid, int nblk, float *__restrict__ Lx,
                                               int64_t b0, int lx_col, int lx_pitch, float2 (*Ls)[NBP + 1]) {
    __shared__ float2 Uz[NBP][2 * NBP];   // U in position order, row t = columns t.. ; zero elsewhere
    __shared__ float2 Lr[NBP][NBP + 1];   // multipliers of lane q's row, by step
    __shared__ float2 F[NBP][NBP + 1];    // factored diagonal block in position order (for the final store)
    __shared__ float2 invd[NBP];
    __shared__ float inv_pa[NBP];
    __shared__ int posof[NBP];
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t r_first = c0 + w + bid * (int64_t)blockDim.x + tid;
    const int64_t r_step = (int64_t)nblk * blockDim.x;
    for (int e = tid; e < NBP * 2 * NBP; e += blockDim.x) (&Uz[0][0])[e] = make_float2(0.f, 0.f);
    // the first row below is loaded while warp 0 factors the diagonal block
    float2 x[NBP];
#pragma unroll
    for (int c = 0; c < NBP; c++)
        x[c] = (c < w && r_first < n) ? A[(c0 + c) * lda + r_first] : make_float2(0.f, 0.f);
    __syncthreads();
    if (tid < 32) {
        float2 r[NBP];
#pragma unroll
        for (int c = 0; c < NBP; c++) {
            r[c] = make_float2(0.f, 0.f);
            if (c < w && lane < w) r[c] = A[(c0 + c) * lda + c0 + lane];
        }
        diag_factor_warp(r, w, lane, Uz, Lr, posof, c0, ipiv, flags, bid == 0);
    }
    __syncthreads();
    if (tid < w) {
        const float2 d = Uz[tid][tid];
        const float pa = fabsf(d.x) + fabsf(d.y);
        invd[tid] = pa > 0.f ? crecip(d) : make_float2(0.f, 0.f);
        inv_pa[tid] = pa > 0.f ? 1.0f / pa : 0.f;
        const int p = posof[tid];
        for (int c = 0; c < w; c++) F[p][c] = c < p ? Lr[tid][c] : Uz[p][c];
    }
    __syncthreads();
    float worst = 0.f;
#define PANEL_PHASE(W_, KEND)                                                                      \
    for (; k < w && k < (KEND); k++) {                                                             \
        worst = fmaxf(worst, (fabsf(x[0].x) + fabsf(x[0].y)) * inv_pa[k]);                         \
        const float2 l_ = subst_step<W_>(x, &Uz[k][k], invd[k]);                                   \
        A[(c0 + k) * lda + r] = l_;                                                                \
        if (GROUPED) Ls[tid][k] = l_;                                                              \
    }
#define PANEL_ROW()                                                                                \
    {                                                                                              \
        int k = 0;                                                                                 \
        _Pragma("unroll 1") PANEL_PHASE(32, 8)                                                     \
        _Pragma("unroll 1") PANEL_PHASE(24, 16)                                                    \
        _Pragma("unroll 1") PANEL_PHASE(16, 24)                                                    \
        _Pragma("unroll 1") PANEL_PHASE(8, 32)                                                     \
    }
    if (!GROUPED) {
        for (int64_t r = r_first; r < n; r += r_step) {
            if (r != r_first) {
#pragma unroll
                for (int c = 0; c < NBP; c++) x[c] = (c < w) ? A[(c0 + c) * lda + r] : make_float2(0.f, 0.f);
            }
            PANEL_ROW()
        }
    } else {
        for (int64_t rb = r_first - tid; rb < n; rb += r_step) {
            const int64_t r = rb + tid;
            if (r < n) {
                if (rb != r_first - tid) {
#pragma unroll
                    for (int c = 0; c < NBP; c++) x[c] = (c < w) ? A[(c0 + c) * lda + r] : make_float2(0.f, 0.f);
                }
                PANEL_ROW()
            }
            __syncthreads();
            if (w == NBP) {
                // real rows 2 (r - b0) + h, floats lx_col + 4 q .. + 4 (the column pairs k = 2q, 2q + 1)
                const int nrow = (int)min((int64_t)blockDim.x, n - rb);
                for (int e = tid; e < nrow * 32; e += blockDim.x) {
                    const int i = e >> 5, h = (e >> 4) & 1, q = e & 15;
                    const float2 a = Ls[i][2 * q], b = Ls[i][2 * q + 1];
                    const float4 v = h ? make_float4(tf32_rna(a.y), tf32_rna(a.x), tf32_rna(b.y), tf32_rna(b.x))
                                       : make_float4(tf32_rna(a.x), tf32_rna(-a.y), tf32_rna(b.x), tf32_rna(-b.y));
                    *(float4 *)(Lx + (2 * (rb + i - b0) + h) * (int64_t)lx_pitch + lx_col + 4 * q) = v;
                }
            }
            __syncthreads();
        }
    }
#undef PANEL_ROW
#undef PANEL_PHASE
    for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_down_sync(0xffffffffu, worst, o));
    if (lane == 0 && worst > 0.f) atomicMax(growth, __float_as_uint(worst));
    panel_store_diag_last(A, lda, c0, w, &F[0][0], NBP + 1, ticket, nblk);
}

__global__ void __launch_bounds__(128) k_panel_local_f32(float2 *__restrict__ A, int64_t lda, int64_t n, int64_t c0,
                                                         int w, int32_t *__restrict__ ipiv, unsigned *growth,
                                                         int *flags) {
    panel_f32_body<false>(A, lda, n, c0, w, ipiv, growth, &flags[GDM_FLAG_PANEL_TICKET], flags, blockIdx.x,
                          gridDim.x, nullptr, 0, 0, 0, nullptr);
}
// the same, also writing the TF32 embedding of the multipliers into Lx (rows relative to b0, pitch lx_pitch
// floats) for the updates of the recursive factorisation
__global__ void __launch_bounds__(128) k_panel_local_f32_lx(float2 *__restrict__ A, int64_t lda, int64_t n,
                                                            int64_t c0, int w, int32_t *__restrict__ ipiv,
                                                            unsigned *growth, int *flags, float *__restrict__ Lx,
                                                            int64_t b0, int lx_pitch) {
    extern __shared__ float2 pl_ls[];  // 128 x (NBP + 1) multipliers of a round of rows
    panel_f32_body<true>(A, lda, n, c0, w, ipiv, growth, &flags[GDM_FLAG_PANEL_TICKET], flags, blockIdx.x,
                         gridDim.x, Lx, b0, (int)(2 * (c0 - b0)), lx_pitch, (float2(*)[NBP + 1])pl_ls);
}

// Two full panels in one launch, columns [c0, c0 + 64): the bottom level of the recursive block
// factorisation, in place of panel, interchange-and-solve of the next panel's top rows, K = 32 update of its
// columns, and panel. Every CTA
//   1. factors the first 32 x 32 diagonal block (warp 0),
//   2. forms the U block right of it, U12 = L11^{-1} P1 A12 (rows in position order; warps 1-3, eleven
//      columns each, lane = row), while warp 0 finds the first panel's multipliers of the second diagonal
//      block's rows,
//   3. brings those rows up to date, A22 - L21 U12 in FP32 (all four warps, eight columns each), and factors
//      the second diagonal block (warp 0),
// and then takes its share of the rows below: the first panel's multipliers, the row's next 32 columns
// updated by them and U12 (FP32 products, in place of the K = 32 tensor-core update), and the second panel's
// multipliers. Pivots, certificate and errors as in the one-panel kernel; the second panel's interchanges
// stay inside its block (product form: the first panel's multipliers of those rows keep their order). The
// last CTA to finish stores the 64 x 64 diagonal region. With Lx, the multipliers of both panels of the
// rows below c0 + 64 also go out as their TF32 embedding (rows from b0, lx_pitch floats a real row),
// staged through shared memory in CTA-wide rounds.
constexpr int PANEL2_SMEM = (2 * NBP * 2 * NBP + 128 * (NBP + 1)) * (int)sizeof(float2);
__global__ void __launch_bounds__(128, 2) k_panel2_f32(float2 *__restrict__ A, int64_t lda, int64_t n, int64_t c0,
                                                      int32_t *__restrict__ ipiv, unsigned *growth, int *flags,
                                                      float *__restrict__ Lx, int64_t b0, int lx_pitch) {
    extern __shared__ __align__(16) float2 p2_dyn[];
    float2(*Uz1)[2 * NBP] = (float2(*)[2 * NBP])p2_dyn;  // U of the first block, position order, zero-padded
    float2(*Uz2)[2 * NBP] = Uz1 + NBP;                   // and of the second
    float2(*Ls)[NBP + 1] = (float2(*)[NBP + 1])(Uz2 + NBP);  // multipliers of a round of rows
    __shared__ float2 Lr[NBP][NBP + 1];   // multipliers of lane q's row by step (either block)
    __shared__ float2 F1[NBP][NBP + 1];   // first diagonal block factored, position order
    __shared__ float2 F2[NBP][NBP + 1];   // second
    __shared__ float2 Ub[NBP][NBP + 2];   // U12: rows in the first block's position order
    __shared__ float2 L2[NBP][NBP + 1];   // first panel's multipliers of the second block's rows
    __shared__ float2 invd1[NBP], invd2[NBP];
    __shared__ float inv_pa1[NBP], inv_pa2[NBP];
    __shared__ int posof[NBP];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool first = blockIdx.x == 0;
    const int64_t r_first = c0 + 2 * NBP + blockIdx.x * (int64_t)blockDim.x + tid;
    const int64_t r_step = (int64_t)gridDim.x * blockDim.x;
    for (int e = tid; e < 2 * NBP * 2 * NBP; e += blockDim.x) (&Uz1[0][0])[e] = make_float2(0.f, 0.f);
    // the first row below is loaded while warp 0 factors the diagonal blocks
    float2 x[NBP];
#pragma unroll
    for (int c = 0; c < NBP; c++) x[c] = r_first < n ? A[(c0 + c) * lda + r_first] : make_float2(0.f, 0.f);
    __syncthreads();
    float worst = 0.f;
    // 1. first diagonal block
    if (tid < 32) {
        float2 r[NBP];
#pragma unroll
        for (int c = 0; c < NBP; c++) r[c] = A[(c0 + c) * lda + c0 + lane];
        diag_factor_warp(r, NBP, lane, Uz1, Lr, posof, c0, ipiv, flags, first);
    }
    __syncthreads();
    if (tid < NBP) {
        const float2 d = Uz1[tid][tid];
        const float pa = fabsf(d.x) + fabsf(d.y);
        invd1[tid] = pa > 0.f ? crecip(d) : make_float2(0.f, 0.f);
        inv_pa1[tid] = pa > 0.f ? 1.0f / pa : 0.f;
        const int p = posof[tid];
        for (int c = 0; c < NBP; c++) F1[p][c] = c < p ? Lr[tid][c] : Uz1[p][c];
    }
    __syncthreads();
    // 2. U12 = L11^{-1} P1 A12 on warps 1-3 (columns 11 (w - 1) .. + 11, lane = row: first the interchanges,
    // row q of the block to its position posof[q], then the unit-lower solve by position); meanwhile warp 0
    // takes the second block's rows through the first panel (their multipliers into L2)
    if (warp > 0) {
        constexpr int UC = 11;
        const int cb = UC * (warp - 1), nc = min(UC, NBP - cb);
        float2 v[UC];
#pragma unroll
        for (int j = 0; j < UC; j++) v[j] = j < nc ? A[(c0 + NBP + cb + j) * lda + c0 + lane] : make_float2(0.f, 0.f);
        const int p = posof[lane];
#pragma unroll
        for (int j = 0; j < UC; j++)
            if (j < nc) Ub[p][cb + j] = v[j];
        __syncwarp();
#pragma unroll
        for (int j = 0; j < UC; j++) v[j] = j < nc ? Ub[lane][cb + j] : make_float2(0.f, 0.f);
#pragma unroll 1
        for (int t = 0; t < NBP - 1; t++) {
            const float2 lt = F1[lane][t];
#pragma unroll
            for (int j = 0; j < UC; j++) {
                const float2 xt = make_float2(__shfl_sync(0xffffffffu, v[j].x, t), __shfl_sync(0xffffffffu, v[j].y, t));
                if (lane > t) cfms(v[j], lt, xt);
            }
        }
#pragma unroll
        for (int j = 0; j < UC; j++)
            if (j < nc) Ub[lane][cb + j] = v[j];
    } else {
        float2 r[NBP];
#pragma unroll
        for (int c = 0; c < NBP; c++) r[c] = A[(c0 + c) * lda + c0 + NBP + lane];
        subst_row32(r, Uz1, invd1, inv_pa1, L2[lane], nullptr, lda, worst);
    }
    __syncthreads();
    // 3. A22 - L21 U12 for the second block's rows (warp w: columns 8w .. 8w + 8, lane = row) into Lr, then its
    // factorisation from there (warp 0; the factorisation's multipliers overwrite Lr after the row is read)
    {
        float2 v[8];
#pragma unroll
        for (int j = 0; j < 8; j++) v[j] = A[(c0 + NBP + 8 * warp + j) * lda + c0 + NBP + lane];
#pragma unroll 4
        for (int k = 0; k < NBP; k++) {
            const float2 l = L2[lane][k];
#pragma unroll
            for (int j = 0; j < 8; j++) cfms(v[j], l, Ub[k][8 * warp + j]);
        }
#pragma unroll
        for (int j = 0; j < 8; j++) Lr[lane][8 * warp + j] = v[j];
    }
    __syncthreads();
    if (tid < 32) {
        float2 r[NBP];
#pragma unroll
        for (int c = 0; c < NBP; c++) r[c] = Lr[lane][c];
        __syncwarp();
        diag_factor_warp(r, NBP, lane, Uz2, Lr, posof, c0 + NBP, ipiv, flags, first);
    }
    __syncthreads();
    if (tid < NBP) {
        const float2 d = Uz2[tid][tid];
        const float pa = fabsf(d.x) + fabsf(d.y);
        invd2[tid] = pa > 0.f ? crecip(d) : make_float2(0.f, 0.f);
        inv_pa2[tid] = pa > 0.f ? 1.0f / pa : 0.f;
        const int p = posof[tid];
        for (int c = 0; c < NBP; c++) F2[p][c] = c < p ? Lr[tid][c] : Uz2[p][c];
    }
    __syncthreads();
    // the rows below, in CTA-wide rounds (uniform trip count, for the barriers of the embedding stores)
    auto store_lx = [&](int64_t rb, int col) {
        // real rows 2 (r - b0) + h, floats col + 4 q .. + 4 (the column pairs k = 2q, 2q + 1)
        const int nrow = (int)min((int64_t)blockDim.x, n - rb);
        for (int e = tid; e < nrow * 32; e += blockDim.x) {
            const int i = e >> 5, h = (e >> 4) & 1, q = e & 15;
            const float2 a = Ls[i][2 * q], b = Ls[i][2 * q + 1];
            const float4 v = h ? make_float4(tf32_rna(a.y), tf32_rna(a.x), tf32_rna(b.y), tf32_rna(b.x))
                               : make_float4(tf32_rna(a.x), tf32_rna(-a.y), tf32_rna(b.x), tf32_rna(-b.y));
            *(float4 *)(Lx + (2 * (rb + i - b0) + h) * (int64_t)lx_pitch + col + 4 * q) = v;
        }
    };
    for (int64_t rb = r_first - tid; rb < n; rb += r_step) {
        const int64_t r = rb + tid;
        float2 y[NBP];
        if (r < n) {
            if (rb != r_first - tid) {
#pragma unroll
                for (int c = 0; c < NBP; c++) x[c] = A[(c0 + c) * lda + r];
            }
            subst_row32(x, Uz1, invd1, inv_pa1, Ls[tid], A + c0 * lda + r, lda, worst);
#pragma unroll
            for (int c = 0; c < NBP; c++) y[c] = A[(c0 + NBP + c) * lda + r];
#pragma unroll 2
            for (int k = 0; k < NBP; k++) {
                const float2 l = Ls[tid][k];
#pragma unroll
                for (int c = 0; c < NBP; c++) cfms(y[c], l, Ub[k][c]);
            }
        }
        if (Lx) {
            __syncthreads();
            store_lx(rb, (int)(2 * (c0 - b0)));
            __syncthreads();
        }
        if (r < n) subst_row32(y, Uz2, invd2, inv_pa2, Ls[tid], A + (c0 + NBP) * lda + r, lda, worst);
        if (Lx) {
            __syncthreads();
            store_lx(rb, (int)(2 * (c0 + NBP - b0)));
            __syncthreads();
        }
    }
    for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_down_sync(0xffffffffu, worst, o));
    if (lane == 0 && worst > 0.f) atomicMax(growth, __float_as_uint(worst));
    // the 64 x 64 diagonal region, once no CTA can still read it
    int *ticket = &flags[GDM_FLAG_PANEL_TICKET];
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    for (int e = tid; e < 4 * NBP * NBP; e += blockDim.x) {
        const int rr = e & (2 * NBP - 1), cc = e >> 6;
        float2 v;
        if (rr < NBP) v = cc < NBP ? F1[rr][cc] : Ub[rr][cc - NBP];
        else v = cc < NBP ? L2[rr - NBP][cc] : F2[rr - NBP][cc - NBP];
        A[(c0 + cc) * lda + c0 + rr] = v;
    }
    if (tid == 0) atomicExch(ticket, 0);
}

// Grouped panel of a batch (lock-step over the problems of a decreasing-size table): CTA b works for the
// problem whose CTA range [prefix[i], prefix[i+1]) holds b, on its panel [c0, c0 + w) of the outer block
// [b0, b0 + nbo); pivots, certificate and errors go to the problem's own records.
__global__ void __launch_bounds__(128) k_glu_panel(const GluItem *__restrict__ items, const int *__restrict__ prefix,
                                                   int na, int64_t b0, int64_t c0, int nbo) {
    extern __shared__ float2 glu_ls[];  // 128 x (NBP + 1) multipliers of a round of rows
    __shared__ int s_item;
    if (threadIdx.x < 32) {
        const int i = glu_find_item(prefix, na, (int)blockIdx.x);
        if (threadIdx.x == 0) s_item = i;
    }
    __syncthreads();
    const int i = s_item;
    const GluItem g = items[i];
    const int64_t be = min(b0 + nbo, g.n);
    const int w = (int)min((int64_t)NBP, be - c0);
    panel_f32_body<true>(g.A, g.lda, g.n, c0, w, g.ipiv, g.growth, g.ticket, g.status, (int)blockIdx.x - prefix[i],
                         prefix[i + 1] - prefix[i], g.lx, b0, (int)(2 * (c0 - b0)), 2 * nbo,
                         (float2(*)[NBP + 1])glu_ls);
}
constexpr int GLU_PANEL_SMEM = 128 * (NBP + 1) * (int)sizeof(float2);

// The grouped panel in two launches, so that the diagonal block of a panel is factored once per problem
// instead of once per CTA: k_glu_diag (one warp per problem) factors it (pivots, certificate base, the
// factored block stored to A) and leaves U in position order (zero-padded to 64 columns) with the
// reciprocal pivots in the problem's GluPanelDiag record; k_glu_rows then solves the rows below in every
// CTA from that record, with no serial prefix.
struct GluPanelDiag {
    float2 Uz[NBP][2 * NBP];
    float2 invd[NBP];
    float inv_pa[NBP];
};
__global__ void __launch_bounds__(32) k_glu_diag(const GluItem *__restrict__ items, int64_t b0, int64_t c0, int nbo) {
    __shared__ float2 Uz[NBP][2 * NBP];
    __shared__ float2 Lr[NBP][NBP + 1];
    const int lane = threadIdx.x;
    const GluItem g = items[blockIdx.x];
    const int64_t be = min(b0 + nbo, g.n);
    const int w = (int)min((int64_t)NBP, be - c0);
    float2 *__restrict__ A = g.A;
    const int64_t lda = g.lda;
    for (int e = lane; e < NBP * 2 * NBP; e += 32) (&Uz[0][0])[e] = make_float2(0.f, 0.f);
    float2 r[NBP];
#pragma unroll
    for (int c = 0; c < NBP; c++) {
        r[c] = make_float2(0.f, 0.f);
        if (c < w && lane < w) r[c] = A[(c0 + c) * lda + c0 + lane];
    }
    __syncwarp();
    int pos = lane;
    bool done = lane >= w;
    const unsigned vb0 = done ? 0u : __float_as_uint(fabsf(r[0].x) + fabsf(r[0].y));
    unsigned m = __reduce_max_sync(0xffffffffu, vb0);
    unsigned key = __reduce_min_sync(0xffffffffu, (!done && vb0 == m) ? (unsigned)pos : 0xffffffffu);
    int t = 0;
#pragma unroll 1
    for (; t < w && t < 8; t++) diag_step<32>(r, t, lane, pos, done, m, key, Uz, Lr, c0, g.ipiv, g.status, true);
#pragma unroll 1
    for (; t < w && t < 16; t++) diag_step<24>(r, t, lane, pos, done, m, key, Uz, Lr, c0, g.ipiv, g.status, true);
#pragma unroll 1
    for (; t < w && t < 24; t++) diag_step<16>(r, t, lane, pos, done, m, key, Uz, Lr, c0, g.ipiv, g.status, true);
#pragma unroll 1
    for (; t < w; t++) diag_step<8>(r, t, lane, pos, done, m, key, Uz, Lr, c0, g.ipiv, g.status, true);
    __syncwarp();
    GluPanelDiag *pd = (GluPanelDiag *)g.pdiag;
    if (lane < w) {
        const float2 d = Uz[lane][lane];
        const float pa = fabsf(d.x) + fabsf(d.y);
        pd->invd[lane] = pa > 0.f ? crecip(d) : make_float2(0.f, 0.f);
        pd->inv_pa[lane] = pa > 0.f ? 1.0f / pa : 0.f;
        // this lane's row of the factored block sits at its final position pos: multipliers left of it, U
        // from it on
        for (int c = 0; c < w; c++) A[(c0 + c) * lda + c0 + pos] = c < pos ? Lr[lane][c] : Uz[pos][c];
    } else {
        pd->invd[lane] = make_float2(0.f, 0.f);
        pd->inv_pa[lane] = 0.f;
    }
    for (int e = lane; e < NBP * 2 * NBP; e += 32) (&pd->Uz[0][0])[e] = (&Uz[0][0])[e];
}

// rows below the panel of every problem from its GluPanelDiag record: CTA b works for the problem whose
// range of the prefix sum holds b (the rows of a problem are split over its CTAs in rounds of 128)
__global__ void __launch_bounds__(128) k_glu_rows(const GluItem *__restrict__ items, const int *__restrict__ prefix,
                                                  int na, int64_t b0, int64_t c0, int nbo) {
    extern __shared__ float2 glu_ls2[];  // 128 x (NBP + 1) multipliers of a round of rows
    float2(*Ls)[NBP + 1] = (float2(*)[NBP + 1])glu_ls2;
    __shared__ float2 Uz[NBP][2 * NBP];
    __shared__ float2 invd[NBP];
    __shared__ float inv_pa[NBP];
    __shared__ int s_item;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        const int i = glu_find_item(prefix, na, (int)blockIdx.x);
        if (tid == 0) s_item = i;
    }
    __syncthreads();
    const int ii = s_item;
    const GluItem g = items[ii];
    const int bid = (int)blockIdx.x - prefix[ii], nblk = prefix[ii + 1] - prefix[ii];
    const int64_t be = min(b0 + nbo, g.n), n = g.n, lda = g.lda;
    const int w = (int)min((int64_t)NBP, be - c0);
    float2 *__restrict__ A = g.A;
    const GluPanelDiag *pd = (const GluPanelDiag *)g.pdiag;
    for (int e = tid; e < NBP * 2 * NBP; e += blockDim.x) (&Uz[0][0])[e] = (&pd->Uz[0][0])[e];
    if (tid < NBP) {
        invd[tid] = pd->invd[tid];
        inv_pa[tid] = pd->inv_pa[tid];
    }
    __syncthreads();
    const int lx_col = (int)(2 * (c0 - b0)), lx_pitch = 2 * nbo;
    const int64_t r_step = (int64_t)nblk * blockDim.x;
    float worst = 0.f;
    float2 x[NBP];
    for (int64_t rb = c0 + w + bid * (int64_t)blockDim.x; rb < n; rb += r_step) {
        const int64_t r = rb + tid;
        if (r < n) {
#pragma unroll
            for (int c = 0; c < NBP; c++) x[c] = (c < w) ? A[(c0 + c) * lda + r] : make_float2(0.f, 0.f);
            int k = 0;
#define ROWS_PHASE(W_, KEND)                                                                       \
    for (; k < w && k < (KEND); k++) {                                                             \
        worst = fmaxf(worst, (fabsf(x[0].x) + fabsf(x[0].y)) * inv_pa[k]);                         \
        const float2 l_ = subst_step<W_>(x, &Uz[k][k], invd[k]);                                   \
        A[(c0 + k) * lda + r] = l_;                                                                \
        Ls[tid][k] = l_;                                                                           \
    }
#pragma unroll 1
            ROWS_PHASE(32, 8)
#pragma unroll 1
            ROWS_PHASE(24, 16)
#pragma unroll 1
            ROWS_PHASE(16, 24)
#pragma unroll 1
            ROWS_PHASE(8, 32)
#undef ROWS_PHASE
        }
        __syncthreads();
        if (w == NBP) {
            const int nrow = (int)min((int64_t)blockDim.x, n - rb);
            for (int e = tid; e < nrow * 32; e += blockDim.x) {
                const int i = e >> 5, h = (e >> 4) & 1, q = e & 15;
                const float2 a = Ls[i][2 * q], b = Ls[i][2 * q + 1];
                const float4 v = h ? make_float4(tf32_rna(a.y), tf32_rna(a.x), tf32_rna(b.y), tf32_rna(b.x))
                                   : make_float4(tf32_rna(a.x), tf32_rna(-a.y), tf32_rna(b.x), tf32_rna(-b.y));
                *(float4 *)(g.lx + (2 * (rb + i - b0) + h) * (int64_t)lx_pitch + lx_col + 4 * q) = v;
            }
        }
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_down_sync(0xffffffffu, worst, o));
    if (lane == 0 && worst > 0.f) atomicMax(g.growth, __float_as_uint(worst));
}

// ------------------------------------------------------------------ block operator for the U12 row block
// Applies the panels q_begin, q_begin + 32, ... < nr of a factored block (view D, row and column 0 at the
// block's first row; pivots of each 32-row panel inside that panel, global row indices in ipiv, base = the
// block's first row) to CPB columns held in shared memory, X[c nr + r]: the product form the factorisation
// produced, each panel's L below its diagonal block stored in the row order before the later panels'
// interchanges. Per panel: the interchanges (each lane tracks where its row's content moves in the swap
// sequence, then one scatter), the unit-lower solve with the diagonal block (warp c takes column c, lane =
// row), and the rows of the later panels, x_r -= L[r, panel] x_panel (one thread per row).
template <int CPB>
__device__ __forceinline__ void apply_panels_smem(float2 *X, int nr, int q_begin, const float2 *__restrict__ D,
                                                  int64_t lda, const int32_t *__restrict__ ipiv, int64_t base,
                                                  float2 (*Lpp)[33]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int q0 = q_begin; q0 < nr; q0 += 32) {
        for (int e = tid; e < 32 * 32; e += blockDim.x) {
            const int i = e & 31, j = e >> 5;
            Lpp[i][j] = (i > j) ? D[(int64_t)(q0 + j) * lda + q0 + i] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (warp < CPB) {
            // lane t holds the panel-local row that step t swaps with; pos follows the content of row lane
            const int piv = (int)(ipiv[base + q0 + lane] - base) - q0;
            int pos = lane;
#pragma unroll 4
            for (int t = 0; t < 32; t++) {
                const int r2 = __shfl_sync(0xffffffffu, piv, t);
                if (r2 != t && r2 >= 0 && r2 < 32) {
                    if (pos == t) pos = r2;
                    else if (pos == r2) pos = t;
                }
            }
            float2 *x = X + warp * nr + q0;
            float2 v = x[lane];
            __syncwarp();
            x[pos] = v;
            __syncwarp();
            v = x[lane];
            for (int t = 0; t < 31; t++) {
                const float2 xt = make_float2(__shfl_sync(0xffffffffu, v.x, t), __shfl_sync(0xffffffffu, v.y, t));
                if (lane > t) cfms(v, Lpp[lane][t], xt);
            }
            x[lane] = v;
        }
        __syncthreads();
        for (int r = q0 + 32 + tid; r < nr; r += blockDim.x) {
            float2 l[32];
#pragma unroll
            for (int j = 0; j < 32; j++) l[j] = D[(int64_t)(q0 + j) * lda + r];
#pragma unroll
            for (int c = 0; c < CPB; c++) {
                float2 acc = X[c * nr + r];
                const float2 *xp = X + c * nr + q0;
#pragma unroll
                for (int j = 0; j < 32; j++) cfms(acc, l[j], xp[j]);
                X[c * nr + r] = acc;
            }
        }
        __syncthreads();
    }
}

// For the outer block [b0, b0+nb) (nb a multiple of 32), form negM = -(L_S^{-1} P_S ... L_1^{-1} P_1)
// restricted to the block's rows; then U12 = -negM A12 for the block's rows of the trailing columns. CTA b
// forms columns CPB b .. + CPB of the operator by applying the panels to those columns of I; panels before
// the one holding column CPB b leave them untouched (their rows are zero there).
template <int CPB>
__global__ void __launch_bounds__(512) k_block_linv(const float2 *__restrict__ A, int64_t lda, int64_t b0, int nb,
                                                    const int32_t *__restrict__ ipiv, float2 *__restrict__ negM) {
    extern __shared__ __align__(16) float2 X[];  // X[c * nb + r], CPB columns
    __shared__ float2 Lpp[32][33];
    const int col0 = CPB * blockIdx.x;
    for (int e = threadIdx.x; e < CPB * nb; e += blockDim.x) {
        const int c = e / nb, r = e % nb;
        X[e] = make_float2(r == col0 + c ? 1.f : 0.f, 0.f);
    }
    apply_panels_smem<CPB>(X, nb, 32 * (col0 / 32), A + b0 * lda + b0, lda, ipiv, b0, Lpp);
    for (int e = threadIdx.x; e < CPB * nb; e += blockDim.x) {
        const int c = e / nb, r = e % nb;
        const float2 v = X[e];
        negM[(int64_t)(col0 + c) * nb + r] = make_float2(-v.x, -v.y);
    }
}

// In-place triangular step of the recursive block factorisation: rows [lo, lo + nr) (nr a multiple of 32, the
// factored left part, pivots of each 32-row panel inside that panel) of columns [col0, col0 + ncols) become
// U = L_S^{-1} P_S ... L_1^{-1} P_1 A (the product form of the left part's panels). CTA b takes CPB columns
// into shared memory and applies the panels in order. round_tf32: the result is stored rounded to TF32.
template <int CPB>
__global__ void __launch_bounds__(512) k_panels_apply(float2 *__restrict__ A, int64_t lda, int64_t lo, int nr,
                                                      int64_t col0, int ncols, const int32_t *__restrict__ ipiv,
                                                      int round_tf32) {
    extern __shared__ __align__(16) float2 X[];  // X[c * nr + r], CPB columns
    __shared__ float2 Lpp[32][33];
    const int c_first = CPB * blockIdx.x;
    const int nc = min(CPB, ncols - c_first);
    for (int e = threadIdx.x; e < CPB * nr; e += blockDim.x) {
        const int c = e / nr, r = e % nr;
        X[e] = (c < nc) ? A[(col0 + c_first + c) * lda + lo + r] : make_float2(0.f, 0.f);
    }
    apply_panels_smem<CPB>(X, nr, 0, A + lo * lda + lo, lda, ipiv, lo, Lpp);
    for (int e = threadIdx.x; e < CPB * nr; e += blockDim.x) {
        const int c = e / nr, r = e % nr;
        if (c < nc) A[(col0 + c_first + c) * lda + lo + r] =
            round_tf32 ? make_float2(tf32_rna(X[e].x), tf32_rna(X[e].y)) : X[e];
    }
}

// columns per CTA of the two kernels above: about 128 CTAs for the widths met here (a CTA's panel chain is
// serial; fewer columns per CTA shorten each of its steps)
static int apply_cpb(int64_t cols) { return cols >= 1024 ? 8 : cols >= 512 ? 4 : cols >= 256 ? 2 : 1; }

template <int CPB>
static gdm_status launch_block_linv_t(gdm_ctx *ctx, const float2 *A, int64_t lda, int64_t b0, int nb,
                                      const int32_t *ipiv, float2 *negM) {
    static bool attr = false;
    if (!attr) {
        GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_block_linv<CPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)((size_t)CPB * 1024 * sizeof(float2))));
        attr = true;
    }
    const int bthreads = nb < 256 ? 256 : (nb > 512 ? 512 : nb);  // one thread per row up to 512
    k_block_linv<CPB><<<(unsigned)(nb / CPB), bthreads, (size_t)CPB * nb * sizeof(float2), ctx->stream>>>(
        A, lda, b0, nb, ipiv, negM);
    GDM_LAUNCHED(ctx, "block_linv");
    return GDM_OK;
}
static gdm_status launch_block_linv(gdm_ctx *ctx, const float2 *A, int64_t lda, int64_t b0, int nb,
                                    const int32_t *ipiv, float2 *negM) {
    if (nb > 1024 || (nb & 31)) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "block operator width %d", nb);
    switch (apply_cpb(nb)) {
        case 8: return launch_block_linv_t<8>(ctx, A, lda, b0, nb, ipiv, negM);
        case 4: return launch_block_linv_t<4>(ctx, A, lda, b0, nb, ipiv, negM);
        case 2: return launch_block_linv_t<2>(ctx, A, lda, b0, nb, ipiv, negM);
        default: return launch_block_linv_t<1>(ctx, A, lda, b0, nb, ipiv, negM);
    }
}

template <int CPB>
static gdm_status launch_panels_apply_t(gdm_ctx *ctx, float2 *A, int64_t lda, int64_t lo, int nr, int64_t col0,
                                        int ncols, const int32_t *ipiv, int round_tf32) {
    static bool attr = false;
    if (!attr) {
        GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_panels_apply<CPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)((size_t)CPB * 1024 * sizeof(float2))));
        attr = true;
    }
    const int bthreads = nr < 256 ? 256 : (nr > 512 ? 512 : nr);
    k_panels_apply<CPB><<<(unsigned)((ncols + CPB - 1) / CPB), bthreads, (size_t)CPB * nr * sizeof(float2),
                          ctx->stream>>>(A, lda, lo, nr, col0, ncols, ipiv, round_tf32);
    GDM_LAUNCHED(ctx, "panels_apply");
    return GDM_OK;
}
static gdm_status launch_panels_apply(gdm_ctx *ctx, float2 *A, int64_t lda, int64_t lo, int nr, int64_t col0,
                                      int ncols, const int32_t *ipiv, int round_tf32) {
    if (nr > 1024 || (nr & 31)) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "panel application over %d rows", nr);
    switch (apply_cpb(ncols)) {
        case 8: return launch_panels_apply_t<8>(ctx, A, lda, lo, nr, col0, ncols, ipiv, round_tf32);
        case 4: return launch_panels_apply_t<4>(ctx, A, lda, lo, nr, col0, ncols, ipiv, round_tf32);
        case 2: return launch_panels_apply_t<2>(ctx, A, lda, lo, nr, col0, ncols, ipiv, round_tf32);
        default: return launch_panels_apply_t<1>(ctx, A, lda, lo, nr, col0, ncols, ipiv, round_tf32);
    }
}

// A[r0 + i, c0 + c] rounded to TF32 (nearest) in place, i < nr, c < nc: U12 once its GEMM is done, so that
// the trailing update reads it straight from storage
__global__ void k_round_tf32_block(float2 *__restrict__ A, int64_t lda, int64_t r0, int nr, int64_t c0, int64_t nc) {
    const int64_t total = (int64_t)nr * nc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / nr, i = e % nr;
        float2 *a = A + (c0 + c) * lda + r0 + i;
        const float2 v = *a;
        *a = make_float2(tf32_rna(v.x), tf32_rna(v.y));
    }
}

// T[i + c * nb] = A[b0 + i, c0 + c], and with zero_src the source zeroed (for a U12 GEMM that accumulates
// into it; the store-only one overwrites it). round_tf32: T rounded to TF32 (nearest), for the single-product
// updates whose tensor cores would otherwise truncate it
__global__ void k_gather_zero(float2 *__restrict__ A, int64_t lda, int64_t b0, int64_t c0, int nb, int64_t nc,
                              float2 *__restrict__ T, int round_tf32, int zero_src) {
    const int64_t total = (int64_t)nb * nc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / nb, i = e % nb;
        float2 *a = A + (c0 + c) * lda + b0 + i;
        const float2 v = *a;
        T[e] = round_tf32 ? make_float2(tf32_rna(v.x), tf32_rna(v.y)) : v;
        if (zero_src) *a = make_float2(0.f, 0.f);
    }
}

// ------------------------------------------------------------------ row interchanges
// Apply pivots ipiv[k_begin..k_end) in order to columns [cb, ce) (one thread per column).
template <class C>
__global__ void k_laswp(C *__restrict__ A, int64_t lda, int64_t cb, int64_t ce, const int32_t *__restrict__ ipiv,
                        int64_t k_begin, int64_t k_end) {
    __shared__ int32_t sp[1024];
    int64_t col = cb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int nk = (int)(k_end - k_begin);
    for (int t = threadIdx.x; t < nk; t += blockDim.x) sp[t] = ipiv[k_begin + t];
    __syncthreads();
    if (col >= ce) return;
    C *a = A + col * lda;
    for (int t = 0; t < nk; t++) {
        int64_t r1 = k_begin + t, r2 = sp[t];
        if (r2 != r1) {
            C x = a[r1], y = a[r2];
            a[r1] = y;
            a[r2] = x;
        }
    }
}

// Same for a right-hand-side block B (ldb) with n_rhs columns; reverse order for the transpose.
template <class C>
__global__ void k_laswp_rhs(C *__restrict__ B, int64_t ldb, int n_rhs, const int32_t *__restrict__ ipiv,
                            int64_t k_begin, int64_t k_end, int reverse) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_rhs) return;
    C *b = B + q * ldb;
    int nk = (int)(k_end - k_begin);
    for (int s = 0; s < nk; s++) {
        int t = reverse ? nk - 1 - s : s;
        int64_t r1 = k_begin + t, r2 = ipiv[k_begin + t];
        if (r2 != r1) {
            C x = b[r1], y = b[r2];
            b[r1] = y;
            b[r2] = x;
        }
    }
}

// ------------------------------------------------------------------ small triangular solves
// X = L^{-1} B in place, L unit lower w x w at A[c0, c0]; B = A[c0 .. c0+w, cb .. ce) (one warp per column).
template <class C>
__global__ void k_trsm_small(C *__restrict__ A, int64_t lda, int64_t c0, int w, int64_t cb, int64_t ce) {
    __shared__ C L[NBP][NBP + 1];
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
        int r = e % w, c = e / w;
        L[r][c] = A[(c0 + c) * lda + c0 + r];
    }
    __syncthreads();
    int lane = threadIdx.x & 31;
    int64_t col = cb + (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (col >= ce) return;
    C *bcol = A + col * lda + c0;
    C v;
    v.x = 0;
    v.y = 0;
    if (lane < w) v = bcol[lane];
    for (int i = 0; i < w; i++) {
        C xi;
        xi.x = __shfl_sync(0xffffffffu, v.x, i);
        xi.y = __shfl_sync(0xffffffffu, v.y, i);
        if (lane > i && lane < w) cfms(v, L[lane][i], xi);
    }
    if (lane < w) bcol[lane] = v;
}

// Grouped interchanges and triangular solve of a batch, after the panel at c0 (32 columns, its pivots inside
// its own 32 rows) of every problem that has columns right of it: rows c0 .. c0 + 32 of those columns get
// the panel's interchanges in order, then L11^{-1} (unit lower), and are stored rounded to TF32 (nearest),
// the value the tensor-core updates read as their B operand. One warp solves 4 columns side by side (lane =
// row), GLU_SWAP_COLS columns per CTA; CTA b works for the problem whose range of the prefix sum holds b.
__global__ void __launch_bounds__(256) k_glu_swap_trsm(const GluItem *__restrict__ items,
                                                       const int *__restrict__ prefix, int na, int64_t c0) {
    __shared__ float2 L[NBP][NBP + 1];
    __shared__ int src[NBP], piv[NBP];
    __shared__ int s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        const int i = glu_find_item(prefix, na, (int)blockIdx.x);
        if (lane == 0) s_item = i;
    }
    __syncthreads();
    const int i = s_item;
    float2 *__restrict__ A = items[i].A;
    const int64_t lda = items[i].lda, n = items[i].n;
    for (int e = threadIdx.x; e < NBP * NBP; e += blockDim.x) {
        const int r = e % NBP, c = e / NBP;
        L[r][c] = A[(c0 + c) * lda + c0 + r];
    }
    if (warp == 0) {
        // final position -> source row of the interchange sequence (position t swapped with ipiv[t])
        piv[lane] = items[i].ipiv[c0 + lane] - (int)c0;
        src[lane] = lane;
        __syncwarp();
        if (lane == 0) {
            for (int t = 0; t < NBP; t++) {
                const int qt = piv[t];
                if (qt > t && qt < NBP) {
                    const int a = src[t];
                    src[t] = src[qt];
                    src[qt] = a;
                }
            }
        }
    }
    __syncthreads();
    const int sr = src[lane];
#pragma unroll 1
    for (int grp = 0; grp < GLU_SWAP_COLS / 32; grp++) {
        const int64_t col0 = c0 + NBP + (int64_t)(blockIdx.x - prefix[i]) * GLU_SWAP_COLS + grp * 32 + warp * 4;
        if (col0 >= n) break;
        float2 v[4];
#pragma unroll
        for (int j = 0; j < 4; j++)
            v[j] = col0 + j < n ? A[(col0 + j) * lda + c0 + sr] : make_float2(0.f, 0.f);
#pragma unroll 4
        for (int k = 0; k < NBP; k++) {
            const float2 lk = L[lane][k];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                float2 xk;
                xk.x = __shfl_sync(0xffffffffu, v[j].x, k);
                xk.y = __shfl_sync(0xffffffffu, v[j].y, k);
                if (lane > k) cfms(v[j], lk, xk);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (col0 + j < n) A[(col0 + j) * lda + c0 + lane] = make_float2(tf32_rna(v[j].x), tf32_rna(v[j].y));
    }
}

// raises the grouped panel's dynamic shared-memory limit (once, before any launch is captured into a graph)
gdm_status gdm_glu_panel_init(gdm_ctx *ctx) {
    static bool attr = false;
    if (!attr) {
        GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_glu_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               GLU_PANEL_SMEM));
        GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_glu_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               GLU_PANEL_SMEM));
        attr = true;
    }
    return GDM_OK;
}

size_t gdm_glu_pdiag_bytes() { return sizeof(GluPanelDiag); }

gdm_status gdm_glu_diag(gdm_ctx *ctx, const GluItem *items, int na, int64_t b0, int64_t c0, int nbo) {
    if (na <= 0) return GDM_OK;
    k_glu_diag<<<(unsigned)na, 32, 0, ctx->stream>>>(items, b0, c0, nbo);
    GDM_LAUNCHED(ctx, "glu_diag");
    return GDM_OK;
}

gdm_status gdm_glu_rows(gdm_ctx *ctx, const GluItem *items, const int *prefix, int na, int nblocks, int64_t b0,
                        int64_t c0, int nbo) {
    if (nblocks <= 0) return GDM_OK;
    GDM_TRY(gdm_glu_panel_init(ctx));
    k_glu_rows<<<(unsigned)nblocks, 128, GLU_PANEL_SMEM, ctx->stream>>>(items, prefix, na, b0, c0, nbo);
    GDM_LAUNCHED(ctx, "glu_rows");
    return GDM_OK;
}

gdm_status gdm_glu_panel(gdm_ctx *ctx, const GluItem *items, const int *prefix, int na, int nblocks, int64_t b0,
                         int64_t c0, int nbo) {
    if (nblocks <= 0) return GDM_OK;
    GDM_TRY(gdm_glu_panel_init(ctx));
    k_glu_panel<<<(unsigned)nblocks, 128, GLU_PANEL_SMEM, ctx->stream>>>(items, prefix, na, b0, c0, nbo);
    GDM_LAUNCHED(ctx, "glu_panel");
    return GDM_OK;
}

gdm_status gdm_glu_swap_trsm(gdm_ctx *ctx, const GluItem *items, const int *prefix, int na, int nblocks,
                             int64_t c0) {
    if (nblocks <= 0) return GDM_OK;
    k_glu_swap_trsm<<<(unsigned)nblocks, 256, 0, ctx->stream>>>(items, prefix, na, c0);
    GDM_LAUNCHED(ctx, "glu_swap_trsm");
    return GDM_OK;
}

// ------------------------------------------------------------------ SIMT complex GEMM  C -= A * B
#define GM_BM 64
#define GM_BN 64
#define GM_BK 16
// C: M x N at Cp (ldc); A: M x K at Ap (lda); B: K x N at Bp (ldb); all column-major complex.
template <class C>
__global__ void __launch_bounds__(256) k_gemm_sub(C *__restrict__ Cp, int64_t ldc, const C *__restrict__ Ap,
                                                  int64_t lda, const C *__restrict__ Bp, int64_t ldb, int64_t M,
                                                  int64_t N, int64_t K) {
    __shared__ C As[GM_BK][GM_BM + 1];
    __shared__ C Bs[GM_BK][GM_BN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t m0 = (int64_t)blockIdx.x * GM_BM, n0 = (int64_t)blockIdx.y * GM_BN;
    C acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            acc[i][j].x = 0;
            acc[i][j].y = 0;
        }
    for (int64_t k0 = 0; k0 < K; k0 += GM_BK) {
        for (int e = threadIdx.x; e < GM_BK * GM_BM; e += 256) {
            int mm = e % GM_BM, kk = e / GM_BM;
            C v;
            v.x = 0;
            v.y = 0;
            if (m0 + mm < M && k0 + kk < K) v = Ap[(k0 + kk) * lda + m0 + mm];
            As[kk][mm] = v;
        }
        for (int e = threadIdx.x; e < GM_BK * GM_BN; e += 256) {
            int kk = e % GM_BK, nn = e / GM_BK;
            C v;
            v.x = 0;
            v.y = 0;
            if (n0 + nn < N && k0 + kk < K) v = Bp[(n0 + nn) * ldb + k0 + kk];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GM_BK; kk++) {
            C a[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) bv[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) cfma(acc[i][j], a[i], bv[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        int64_t nn = n0 + ty + 16 * j;
        if (nn >= N) continue;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            int64_t mm = m0 + tx + 16 * i;
            if (mm >= M) continue;
            C *c = Cp + nn * ldc + mm;
            *c = csub(*c, acc[i][j]);
        }
    }
}

template <class C>
static gdm_status gemm_sub(gdm_ctx *ctx, C *Cp, int64_t ldc, const C *Ap, int64_t lda, const C *Bp, int64_t ldb,
                           int64_t M, int64_t N, int64_t K) {
    if (M <= 0 || N <= 0 || K <= 0) return GDM_OK;
    dim3 grid((unsigned)((M + GM_BM - 1) / GM_BM), (unsigned)((N + GM_BN - 1) / GM_BN));
    if (grid.y > 65535) return gdm_fail(ctx, GDM_ERR_SHAPE, "gemm grid too large");
    k_gemm_sub<C><<<grid, 256, 0, ctx->stream>>>(Cp, ldc, Ap, lda, Bp, ldb, M, N, K);
    GDM_LAUNCHED(ctx, "gemm_sub");
    return GDM_OK;
}

// ------------------------------------------------------------------ factorisation driver
template <class C>
static gdm_status panel_factor(gdm_ctx *ctx, C *A, int64_t lda, int64_t n, int64_t c0, int w, int32_t *ipiv,
                               PanelScratch<C> ps, int pmax) {
    int64_t m = n - c0;
    int P = (int)((m + 255) / 256);
    if (P > pmax) P = pmax;
    if (P < 1) P = 1;
    int rpc = (int)((m + P - 1) / P);
    if (rpc < w) rpc = w;
    P = (int)((m + rpc - 1) / rpc);
    size_t smem = (size_t)NBP * rpc * sizeof(C);
    if (smem > (size_t)ctx->max_smem_optin - 4096)
        return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "panel of %lld rows does not fit the cooperative panel kernel",
                        (long long)m);
    static bool attr_set[2] = {false, false};
    int slot = sizeof(C) == 8 ? 0 : 1;
    if (!attr_set[slot]) {
        GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_panel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               ctx->max_smem_optin - 4096));
        attr_set[slot] = true;
    }
    if (P > 1) GDM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dflags + GDM_FLAG_BAR_COUNT, 0, sizeof(int), ctx->stream));
    int *flags = ctx->dflags;
    void *args[] = {&A, &lda, &n, &c0, &w, &rpc, &ipiv, &ps, &flags};
    if (P > 1) {
        GDM_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((void *)k_panel<C>, dim3(P), dim3(PANEL_THREADS), args, smem,
                                                      ctx->stream));
    } else {
        k_panel<C><<<1, PANEL_THREADS, smem, ctx->stream>>>(A, lda, n, c0, w, rpc, ipiv, ps, flags);
    }
    GDM_LAUNCHED(ctx, "panel");
    return GDM_OK;
}

template <class C>
static gdm_status laswp(gdm_ctx *ctx, C *A, int64_t lda, int64_t cb, int64_t ce, const int32_t *ipiv, int64_t kb,
                        int64_t ke) {
    if (ce <= cb || ke <= kb) return GDM_OK;
    if (ke - kb > 1024) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "laswp block too large");
    unsigned nb = (unsigned)((ce - cb + 127) / 128);
    k_laswp<C><<<nb, 128, 0, ctx->stream>>>(A, lda, cb, ce, ipiv, kb, ke);
    GDM_LAUNCHED(ctx, "laswp");
    return GDM_OK;
}

template <class C>
static gdm_status trsm_small(gdm_ctx *ctx, C *A, int64_t lda, int64_t c0, int w, int64_t cb, int64_t ce) {
    if (ce <= cb) return GDM_OK;
    const int wpb = 8;
    unsigned nb = (unsigned)((ce - cb + wpb - 1) / wpb);
    k_trsm_small<C><<<nb, wpb * 32, 0, ctx->stream>>>(A, lda, c0, w, cb, ce);
    GDM_LAUNCHED(ctx, "trsm_small");
    return GDM_OK;
}

int gdm_size_class(int64_t n) {
    int c = 0;
    while (c < GDM_NB_CLASSES - 1 && n > ((int64_t)512 << c)) c++;
    return c;
}

// outer block width of the LU: FP64 128 (SIMT updates); otherwise GDM_LU_NB if set, else the context's
// autotuned width for this size class, else 512
int gdm_lu_block(const gdm_ctx *ctx, gdm_precision prec, int64_t n) {
    if (prec == GDM_FP64) return 128;
    const char *e = getenv("GDM_LU_NB");
    int nb = e ? atoi(e) : 0;
    if (!nb && ctx) nb = ctx->nb_table[gdm_size_class(n)];
    if (nb < 64 || nb > 1024 || nb % 32) nb = 512;
    return nb;
}

// sub-block update C -= L U inside the matrix: tensor cores for the FP32 precisions, SIMT otherwise
template <class C>
static gdm_status update(gdm_ctx *ctx, gdm_precision prec, C *A, int64_t lda, int64_t n, int64_t r0, int64_t c0,
                         int64_t k0, int64_t Mc, int64_t Nc, int64_t Kc, void *tcws, size_t tcbytes) {
    if (Mc <= 0 || Nc <= 0 || Kc <= 0) return GDM_OK;
    gdm_status s = GDM_ERR_UNSUPPORTED;
    if (sizeof(C) == 8 && tcws)
        s = gdm_tc_update(ctx, prec, (float2 *)A, lda, n, r0, c0, k0, Mc, Nc, Kc, tcws, tcbytes, 0);
    if (s == GDM_ERR_UNSUPPORTED)
        s = gemm_sub<C>(ctx, A + c0 * lda + r0, lda, A + k0 * lda + r0, lda, A + c0 * lda + k0, lda, Mc, Nc, Kc);
    return s;
}

// the TF32 embedding of the current outer block's L that the recursive factorisation's updates read (rows
// from b0, pitch floats per real row); Lx == nullptr: the updates prepare their operands themselves
struct LxBuf {
    float *Lx = nullptr;
    int64_t b0 = 0;
    int pitch = 0;
};

template <class C>
static gdm_status panel_local(gdm_ctx *ctx, C *A, int64_t lda, int64_t n, int64_t c0, int w, int32_t *ipiv,
                              unsigned *growth, const LxBuf &lx = LxBuf()) {
    int64_t below = n - c0 - w;
    if (sizeof(C) == 8 && !getenv("GDM_PANEL_SMEM")) {
        int blocks = (int)((below + 127) / 128);
        if (blocks < 1) blocks = 1;
        if (blocks > 4 * ctx->sm_count) blocks = 4 * ctx->sm_count;
        if (lx.Lx) {
            static bool attr = false;
            if (!attr) {
                GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_panel_local_f32_lx,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, GLU_PANEL_SMEM));
                attr = true;
            }
            k_panel_local_f32_lx<<<blocks, 128, GLU_PANEL_SMEM, ctx->stream>>>(
                (float2 *)A, lda, n, c0, w, ipiv, growth, ctx->dflags, lx.Lx, lx.b0, lx.pitch);
            GDM_LAUNCHED(ctx, "panel_local_f32_lx");
            return GDM_OK;
        }
        k_panel_local_f32<<<blocks, 128, 0, ctx->stream>>>((float2 *)A, lda, n, c0, w, ipiv, growth, ctx->dflags);
        GDM_LAUNCHED(ctx, "panel_local_f32");
        return GDM_OK;
    }
    int blocks = (int)((below + 255) / 256);
    if (blocks < 1) blocks = 1;
    if (blocks > 4 * ctx->sm_count) blocks = 4 * ctx->sm_count;
    k_panel_local<C><<<blocks, 256, 0, ctx->stream>>>(A, lda, n, c0, w, ipiv, growth, ctx->dflags);
    GDM_LAUNCHED(ctx, "panel_local");
    return GDM_OK;
}

// Recursive factorisation of the columns [lo, hi) of one outer block (rows [lo, n)), FP32 factors on tensor
// cores: factor the left part (a multiple of 32 columns), turn the right part's top rows into U with the
// left part's panels, update the right part's rows below with one GEMM (K = width of the left part), then
// factor the right part. Same arithmetic as panel-by-panel right-looking updates, but the GEMMs have
// K = 256, 128, 64, 32 instead of fifteen K = 32 updates of the full remaining block width.
// With an embedding buffer (lx.Lx) the panels write L's TF32 embedding as they go, the panel applications
// store U rounded to TF32, and the updates read both straight from there (no preparation pass).
static gdm_status factor_rec(gdm_ctx *ctx, gdm_precision prec, float2 *A, int64_t lda, int64_t n, int64_t lo,
                             int64_t hi, int32_t *ipiv, unsigned *growth, void *tcws, size_t tcbytes,
                             const LxBuf &lx) {
    const int64_t w = hi - lo;
    if (w <= NBP) {
        GDM_TRY(gdm_phase_begin(ctx, GDM_PH_PANEL));
        GDM_TRY(panel_local<float2>(ctx, A, lda, n, lo, (int)w, ipiv, growth, lx));
        return gdm_phase_end(ctx, GDM_PH_PANEL);
    }
    if (w == 2 * NBP && !getenv("GDM_PANEL_SINGLE") && !getenv("GDM_PANEL_SMEM")) {
        // both panels of a 64-column block in one launch
        GDM_TRY(gdm_phase_begin(ctx, GDM_PH_PANEL));
        static bool attr = false;
        if (!attr) {
            GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_panel2_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   PANEL2_SMEM));
            attr = true;
        }
        int blocks = (int)((n - hi + 127) / 128);
        if (blocks < 1) blocks = 1;
        if (blocks > 2 * ctx->sm_count) blocks = 2 * ctx->sm_count;  // one wave (two CTAs an SM)
        k_panel2_f32<<<blocks, 128, PANEL2_SMEM, ctx->stream>>>(A, lda, n, lo, ipiv, growth, ctx->dflags, lx.Lx,
                                                                 lx.b0, lx.pitch);
        GDM_LAUNCHED(ctx, "panel2_f32");
        return gdm_phase_end(ctx, GDM_PH_PANEL);
    }
    const int64_t mid = lo + NBP * ((w + 2 * NBP - 1) / (2 * NBP));
    GDM_TRY(factor_rec(ctx, prec, A, lda, n, lo, mid, ipiv, growth, tcws, tcbytes, lx));
    const int nr = (int)(mid - lo), ncols = (int)(hi - mid);
    GDM_TRY(gdm_phase_begin(ctx, GDM_PH_TRSM));
    GDM_TRY(launch_panels_apply(ctx, A, lda, lo, nr, mid, ncols, ipiv, lx.Lx != nullptr));
    GDM_TRY(gdm_phase_end(ctx, GDM_PH_TRSM));
    GDM_TRY(gdm_phase_begin(ctx, GDM_PH_INBLOCK));
    if (lx.Lx) {
        // rows [mid, n) of L's columns [lo, mid) in the embedding; U = rows [lo, mid) of columns [mid, hi)
        const float *lp = lx.Lx + 2 * (mid - lx.b0) * (int64_t)lx.pitch + 2 * (lo - lx.b0);
        gdm_status s = gdm_tc_update_lx(ctx, A, lda, mid, mid, lp, lx.pitch, A, lda, lo, mid, n - mid, hi - mid,
                                        mid - lo, 0);
        if (s == GDM_ERR_UNSUPPORTED)
            s = update<float2>(ctx, prec, A, lda, n, mid, mid, lo, n - mid, hi - mid, mid - lo, tcws, tcbytes);
        GDM_TRY(s);
    } else {
        GDM_TRY(update<float2>(ctx, prec, A, lda, n, mid, mid, lo, n - mid, hi - mid, mid - lo, tcws, tcbytes));
    }
    GDM_TRY(gdm_phase_end(ctx, GDM_PH_INBLOCK));
    return factor_rec(ctx, prec, A, lda, n, mid, hi, ipiv, growth, tcws, tcbytes, lx);
}

template <class C>
static gdm_status lu_factor_t(gdm_ctx *ctx, gdm_precision prec, C *A, int64_t n, int64_t lda, int32_t *ipiv,
                              int global_pivot, unsigned *growth) {
    // whole-column pivoting moves rows below the block, so it factors one 32-column panel per block
    const int NB = global_pivot ? NBP : gdm_lu_block(ctx, prec, n);
    int pmax = ctx->sm_count;
    // scratch: panel candidates + tensor-core operand buffers
    size_t pbytes = ScratchCarver::round(2 * pmax * sizeof(double)) + ScratchCarver::round(2 * pmax * sizeof(int64_t)) +
                    ScratchCarver::round((size_t)2 * pmax * NBP * sizeof(C)) +
                    ScratchCarver::round(2 * NBP * sizeof(C));
    size_t tcbytes = (sizeof(C) == 8) ? gdm_tc_workspace_bytes(n, NB, prec) : 0;
    // U12 through the block operator (tensor cores, local pivots): operator and gathered row block
    const bool u12_op = sizeof(C) == 8 && tcbytes && !global_pivot && NB <= 512 && !getenv("GDM_U12_PANELS");
    size_t opbytes = u12_op ? ScratchCarver::round((size_t)NB * NB * sizeof(C)) +
                                  ScratchCarver::round((size_t)NB * n * sizeof(C))
                            : 0;
    // recursive blocks pay off on large systems; small ones (the batched workloads) keep the panel-by-panel
    // updates, whose per-problem latency is lower
    const bool recursive =
        u12_op && NB <= 1024 && (n >= 8192 || getenv("GDM_LU_RECURSIVE")) && !getenv("GDM_INBLOCK_PANELS");
    // TF32: the panels write L's embedding for the updates as they go (rows from the outer block's first row,
    // 2 NB floats a real row) and U is rounded in storage, so the updates need no operand preparation
    const bool lx_path = recursive && prec == GDM_TF32_REFINE && !(lda & 1) && !((uintptr_t)A & 15) &&
                         !getenv("GDM_LU_PREP_L") && !getenv("GDM_TC_TRUNCATE");
    const size_t lxbytes = lx_path ? ScratchCarver::round((size_t)2 * n * 2 * NB * sizeof(float)) : 0;
    void *ws;
    GDM_TRY(gdm_scratch(ctx, pbytes + tcbytes + opbytes + lxbytes + 1024, &ws));
    ScratchCarver sc(ws);
    PanelScratch<C> ps;
    ps.cand_val = sc.take<double>(2 * pmax);
    ps.cand_row = sc.take<int64_t>(2 * pmax);
    ps.cand_vals = sc.take<C>((size_t)2 * pmax * NBP);
    ps.top_row = sc.take<C>(2 * NBP);
    void *tcws = tcbytes ? sc.take<char>(tcbytes) : nullptr;
    float2 *negM = u12_op ? sc.take<float2>((size_t)NB * NB) : nullptr;
    float2 *T12 = u12_op ? sc.take<float2>((size_t)NB * n) : nullptr;
    LxBuf lx;
    if (lx_path) {
        lx.Lx = sc.take<float>((size_t)2 * n * 2 * NB);
        lx.pitch = 2 * NB;
    }
    for (int64_t b0 = 0; b0 < n; b0 += NB) {
        int64_t nb = n - b0 < NB ? n - b0 : NB;
        int64_t be = b0 + nb;
        lx.b0 = b0;
        if (recursive)
            GDM_TRY(factor_rec(ctx, prec, (float2 *)A, lda, n, b0, be, ipiv, growth, tcws, tcbytes, lx));
        else
        for (int64_t c0 = b0; c0 < be; c0 += NBP) {
            int w = (int)(be - c0 < NBP ? be - c0 : NBP);
            GDM_TRY(gdm_phase_begin(ctx, GDM_PH_PANEL));
            if (global_pivot) GDM_TRY(panel_factor<C>(ctx, A, lda, n, c0, w, ipiv, ps, pmax));
            else GDM_TRY(panel_local<C>(ctx, A, lda, n, c0, w, ipiv, growth));
            GDM_TRY(gdm_phase_end(ctx, GDM_PH_PANEL));
            GDM_TRY(gdm_phase_begin(ctx, GDM_PH_LASWP));
            GDM_TRY(laswp<C>(ctx, A, lda, c0 + w, be, ipiv, c0, c0 + w));
            GDM_TRY(gdm_phase_end(ctx, GDM_PH_LASWP));
            if (c0 + w < be) {
                GDM_TRY(gdm_phase_begin(ctx, GDM_PH_TRSM));
                GDM_TRY(trsm_small<C>(ctx, A, lda, c0, w, c0 + w, be));
                GDM_TRY(gdm_phase_end(ctx, GDM_PH_TRSM));
                GDM_TRY(gdm_phase_begin(ctx, GDM_PH_INBLOCK));
                GDM_TRY(update<C>(ctx, prec, A, lda, n, c0 + w, c0 + w, c0, n - c0 - w, be - c0 - w, w, tcws, tcbytes));
                GDM_TRY(gdm_phase_end(ctx, GDM_PH_INBLOCK));
            }
        }
        if (be < n && u12_op) {
            // U12 = M A12 with the block operator M = L_S^{-1} P_S ... L_1^{-1} P_1 (one tensor-core GEMM)
            GDM_TRY(gdm_phase_begin(ctx, GDM_PH_U12));
            const int nbi = (int)nb;
            GDM_TRY(launch_block_linv(ctx, (const float2 *)A, lda, b0, nbi, ipiv, negM));
            const int64_t nc = n - be;
            const int64_t tot = (int64_t)nbi * nc;
            unsigned gb = (unsigned)((tot + 255) / 256);
            if (gb > (unsigned)(8 * ctx->sm_count)) gb = 8 * ctx->sm_count;
            const int tf32_in = prec != GDM_FP32 && !getenv("GDM_TC_TRUNCATE");
            // the store-only product writes U12 over the block's rows (rounded to TF32 for the trailing update
            // on the embedding path); where it does not apply, the rows are zeroed and the product accumulated
            const bool store = tf32_in && !getenv("GDM_U12_ACCUMULATE");
            k_gather_zero<<<gb, 256, 0, ctx->stream>>>((float2 *)A, lda, b0, be, nbi, nc, T12, tf32_in, !store);
            GDM_LAUNCHED(ctx, "gather_zero");
            gdm_status s = GDM_ERR_UNSUPPORTED;
            if (store)
                s = gdm_tc_update_ext(ctx, prec, (float2 *)A, lda, b0, be, negM, nbi, T12, nbi, 0, 0, nbi, nc, nbi,
                                      tcws, tcbytes, 0, tf32_in, lx.Lx ? 2 : 1);
            if (s == GDM_ERR_UNSUPPORTED) {
                if (store)
                    GDM_CUDA_TRY(ctx, cudaMemset2DAsync((float2 *)A + be * lda + b0, (size_t)lda * sizeof(float2), 0,
                                                        (size_t)nbi * sizeof(float2), (size_t)nc, ctx->stream));
                GDM_TRY(gdm_tc_update_ext(ctx, prec, (float2 *)A, lda, b0, be, negM, nbi, T12, nbi, 0, 0, nbi, nc,
                                          nbi, tcws, tcbytes, 0, tf32_in));
                if (lx.Lx) {
                    k_round_tf32_block<<<gb, 256, 0, ctx->stream>>>((float2 *)A, lda, b0, nbi, be, nc);
                    GDM_LAUNCHED(ctx, "round_tf32_block");
                }
            } else {
                GDM_TRY(s);
            }
            GDM_TRY(gdm_phase_end(ctx, GDM_PH_U12));
        } else if (be < n) {
            // U12 = L11^{-1} A12 panel by panel; each panel's interchanges reach the trailing columns just
            // before its triangular solve (L rows of later panels are still in their pre-interchange order)
            for (int64_t c0 = b0; c0 < be; c0 += NBP) {
                int w = (int)(be - c0 < NBP ? be - c0 : NBP);
                GDM_TRY(gdm_phase_begin(ctx, GDM_PH_LASWP));
                GDM_TRY(laswp<C>(ctx, A, lda, be, n, ipiv, c0, c0 + w));
                GDM_TRY(gdm_phase_end(ctx, GDM_PH_LASWP));
                GDM_TRY(gdm_phase_begin(ctx, GDM_PH_TRSM));
                GDM_TRY(trsm_small<C>(ctx, A, lda, c0, w, be, n));
                GDM_TRY(gdm_phase_end(ctx, GDM_PH_TRSM));
                if (c0 + w < be) {
                    GDM_TRY(gdm_phase_begin(ctx, GDM_PH_U12));
                    GDM_TRY(update<C>(ctx, prec, A, lda, n, c0 + w, be, c0, be - c0 - w, n - be, w, tcws, tcbytes));
                    GDM_TRY(gdm_phase_end(ctx, GDM_PH_U12));
                }
            }
        }
        if (be < n) {
            // A22 -= A21 U12
            GDM_TRY(gdm_phase_begin(ctx, GDM_PH_TRAILING));
            gdm_status s = GDM_ERR_UNSUPPORTED;
            if (lx.Lx && n - be >= 64) {
                // rows [be, n) of the block's L embedding against the rounded U12 in place
                nvtxRangePushA("gdm_trailing_update");
                s = gdm_tc_update_lx(ctx, (float2 *)A, lda, be, be, lx.Lx + 2 * (be - b0) * (int64_t)lx.pitch,
                                     lx.pitch, (const float2 *)A, lda, b0, be, n - be, n - be, nb, 1);
                nvtxRangePop();
            }
            if (s == GDM_ERR_UNSUPPORTED && sizeof(C) == 8 && tcws)
                s = gdm_tc_trailing_update(ctx, prec, (float2 *)A, lda, n, b0, nb, tcws, tcbytes);
            if (s == GDM_ERR_UNSUPPORTED) {
                int slot;
                GDM_TRY(gdm_prof_begin(ctx, &slot));
                s = gemm_sub<C>(ctx, A + be * lda + be, lda, A + b0 * lda + be, lda, A + be * lda + b0, lda, n - be,
                                n - be, nb);
                double mm = (double)(n - be);
                GDM_TRY(gdm_prof_end(ctx, slot, 8.0 * mm * mm * nb,
                                     sizeof(C) * (2.0 * mm * mm + 2.0 * mm * nb)));
            }
            GDM_TRY(s);
            GDM_TRY(gdm_phase_end(ctx, GDM_PH_TRAILING));
        }
    }
    return GDM_OK;
}

gdm_status gdm_lu_factor(gdm_ctx *ctx, gdm_precision prec, void *A, int64_t n, int64_t lda, int32_t *ipiv,
                         int global_pivot, float *growth_out) {
    // the growth record lives in the flags allocation (slot GDM_FLAG_GROWTH)
    unsigned *growth = (unsigned *)(ctx->dflags + GDM_FLAG_GROWTH);
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(growth, 0, sizeof(unsigned), ctx->stream));
    gdm_status s = (prec == GDM_FP64) ? lu_factor_t<double2>(ctx, prec, (double2 *)A, n, lda, ipiv, global_pivot, growth)
                                      : lu_factor_t<float2>(ctx, prec, (float2 *)A, n, lda, ipiv, global_pivot, growth);
    if (s != GDM_OK) return s;
    if (growth_out) {
        unsigned *h;
        GDM_TRY(gdm_pinned(ctx, 64, (void **)&h));
        GDM_CUDA_TRY(ctx, cudaMemcpyAsync(h, growth, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
        GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        float g;
        memcpy(&g, h, sizeof(float));
        *growth_out = global_pivot ? 1.0f : g;
    }
    return GDM_OK;
}

// ------------------------------------------------------------------ triangular solves on right-hand sides
// Diagonal-block solve for one panel (w <= NBP): lower unit (forward) or upper non-unit (backward);
// conj = 1 solves with the conjugate transpose of the stored triangle. One warp per RHS column.
template <class C>
__global__ void k_trsv_diag(const C *__restrict__ A, int64_t lda, int64_t c0, int w, C *__restrict__ B, int64_t ldb,
                            int n_rhs, int upper, int conj) {
    __shared__ C T[NBP][NBP + 1];
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
        int r = e % w, c = e / w;
        C v = A[(c0 + c) * lda + c0 + r];
        if (conj) {
            v.y = -v.y;
            T[c][r] = v;  // transpose
        } else
            T[r][c] = v;
    }
    __syncthreads();
    int lane = threadIdx.x & 31;
    int q = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (q >= n_rhs) return;
    C *b = B + q * ldb + c0;
    C v;
    v.x = 0;
    v.y = 0;
    if (lane < w) v = b[lane];
    // effective triangle after the optional conjugate transpose
    bool eff_upper = conj ? !upper : upper;
    bool unit = !upper;  // L is unit diagonal, U is not (transpose keeps the diagonal)
    if (!eff_upper) {
        for (int i = 0; i < w; i++) {
            if (!unit && lane == i) v = cmul(v, crecip(T[i][i]));
            C xi;
            xi.x = __shfl_sync(0xffffffffu, v.x, i);
            xi.y = __shfl_sync(0xffffffffu, v.y, i);
            if (lane > i && lane < w) cfms(v, T[lane][i], xi);
        }
    } else {
        for (int i = w - 1; i >= 0; i--) {
            if (!unit && lane == i) v = cmul(v, crecip(T[i][i]));
            C xi;
            xi.x = __shfl_sync(0xffffffffu, v.x, i);
            xi.y = __shfl_sync(0xffffffffu, v.y, i);
            if (lane < i) cfms(v, T[lane][i], xi);
        }
    }
    if (lane < w) b[lane] = v;
}

// y[r0:r1] -= M[r0:r1, c0:c0+w] * y[c0:c0+w]   (thread per row, loop over RHS)
template <class C>
__global__ void k_gemv_sub(const C *__restrict__ A, int64_t lda, int64_t r0, int64_t r1, int64_t c0, int w,
                           C *__restrict__ B, int64_t ldb, int n_rhs) {
    __shared__ C xs[NBP][8];
    int64_t r = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int q0 = 0; q0 < n_rhs; q0 += 8) {
        int nq = n_rhs - q0 < 8 ? n_rhs - q0 : 8;
        __syncthreads();
        for (int e = threadIdx.x; e < w * nq; e += blockDim.x) xs[e % w][e / w] = B[(q0 + e / w) * ldb + c0 + e % w];
        __syncthreads();
        if (r < r1) {
            C acc[8];
            for (int q = 0; q < 8; q++) {
                acc[q].x = 0;
                acc[q].y = 0;
            }
            for (int c = 0; c < w; c++) {
                C a = A[(c0 + c) * lda + r];
                for (int q = 0; q < nq; q++) cfma(acc[q], a, xs[c][q]);
            }
            for (int q = 0; q < nq; q++) {
                C *y = B + (q0 + q) * ldb + r;
                *y = csub(*y, acc[q]);
            }
        }
    }
}

// y[c0:c0+w] -= M[r0:r1, c0:c0+w]^H * y[r0:r1]   (block per column of M, reduction over rows)
template <class C>
__global__ void k_gemv_h_sub(const C *__restrict__ A, int64_t lda, int64_t r0, int64_t r1, int64_t c0,
                             C *__restrict__ B, int64_t ldb, int n_rhs) {
    int c = blockIdx.x;
    int q = blockIdx.y;
    const C *a = A + (c0 + c) * lda;
    const C *y = B + q * ldb;
    double sx = 0, sy = 0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        C m = a[r], v = y[r];
        // conj(m) * v
        sx += (double)m.x * v.x + (double)m.y * v.y;
        sy += (double)m.x * v.y - (double)m.y * v.x;
    }
    __shared__ double rx[32], ry[32];
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
    }
    if ((threadIdx.x & 31) == 0) {
        rx[threadIdx.x >> 5] = sx;
        ry[threadIdx.x >> 5] = sy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); k++) {
            sx += rx[k];
            sy += ry[k];
        }
        C *o = B + q * ldb + c0 + c;
        o->x -= sx;
        o->y -= sy;
    }
}

template <class C>
static gdm_status lu_solve_t(gdm_ctx *ctx, gdm_precision prec, const C *A, int64_t n, int64_t lda,
                             const int32_t *ipiv, C *B, int64_t ldb, int n_rhs, int conj_trans) {
    const int wpb = 4;
    unsigned nbq = (unsigned)((n_rhs + wpb - 1) / wpb);
    if (!conj_trans) {
        for (int64_t b0 = 0; b0 < n; b0 += NBP) {
            int64_t be = b0 + NBP < n ? b0 + NBP : n;
            k_laswp_rhs<C><<<(n_rhs + 31) / 32, 32, 0, ctx->stream>>>(B, ldb, n_rhs, ipiv, b0, be, 0);
            GDM_LAUNCHED(ctx, "laswp_rhs");
            for (int64_t c0 = b0; c0 < be; c0 += NBP) {
                int w = (int)(be - c0 < NBP ? be - c0 : NBP);
                k_trsv_diag<C><<<nbq, wpb * 32, 0, ctx->stream>>>(A, lda, c0, w, B, ldb, n_rhs, 0, 0);
                GDM_LAUNCHED(ctx, "trsv_diag");
                if (c0 + w < n) {
                    k_gemv_sub<C><<<(unsigned)((n - c0 - w + 255) / 256), 256, 0, ctx->stream>>>(A, lda, c0 + w, n, c0,
                                                                                                w, B, ldb, n_rhs);
                    GDM_LAUNCHED(ctx, "gemv_sub");
                }
            }
        }
        for (int64_t c0 = ((n - 1) / NBP) * NBP; c0 >= 0; c0 -= NBP) {
            int w = (int)(n - c0 < NBP ? n - c0 : NBP);
            k_trsv_diag<C><<<nbq, wpb * 32, 0, ctx->stream>>>(A, lda, c0, w, B, ldb, n_rhs, 1, 0);
            GDM_LAUNCHED(ctx, "trsv_diag");
            if (c0 > 0) {
                k_gemv_sub<C><<<(unsigned)((c0 + 255) / 256), 256, 0, ctx->stream>>>(A, lda, 0, c0, c0, w, B, ldb,
                                                                                     n_rhs);
                GDM_LAUNCHED(ctx, "gemv_sub");
            }
        }
    } else {
        // A^{-H} = P_1^T L_1^{-H} ... P_S^T L_S^{-H} U^{-H}: first U^H z = b (forward), then per block
        // (last to first): z_b -= L21^H z_rest; z_b = L_bb^{-H} z_b; undo the block's row swaps.
        for (int64_t c0 = 0; c0 < n; c0 += NBP) {
            int w = (int)(n - c0 < NBP ? n - c0 : NBP);
            if (c0 > 0) {
                k_gemv_h_sub<C><<<dim3(w, n_rhs), 256, 0, ctx->stream>>>(A, lda, 0, c0, c0, B, ldb, n_rhs);
                GDM_LAUNCHED(ctx, "gemv_h_sub");
            }
            k_trsv_diag<C><<<nbq, wpb * 32, 0, ctx->stream>>>(A, lda, c0, w, B, ldb, n_rhs, 1, 1);
            GDM_LAUNCHED(ctx, "trsv_diag");
        }
        int64_t last_b0 = ((n - 1) / NBP) * NBP;
        for (int64_t b0 = last_b0; b0 >= 0; b0 -= NBP) {
            int64_t be = b0 + NBP < n ? b0 + NBP : n;
            int64_t last_c0 = b0 + ((be - 1 - b0) / NBP) * NBP;
            for (int64_t c0 = last_c0; c0 >= b0; c0 -= NBP) {
                int w = (int)(be - c0 < NBP ? be - c0 : NBP);
                if (c0 + w < n) {
                    k_gemv_h_sub<C><<<dim3(w, n_rhs), 256, 0, ctx->stream>>>(A, lda, c0 + w, n, c0, B, ldb, n_rhs);
                    GDM_LAUNCHED(ctx, "gemv_h_sub");
                }
                k_trsv_diag<C><<<nbq, wpb * 32, 0, ctx->stream>>>(A, lda, c0, w, B, ldb, n_rhs, 0, 1);
                GDM_LAUNCHED(ctx, "trsv_diag");
            }
            k_laswp_rhs<C><<<(n_rhs + 31) / 32, 32, 0, ctx->stream>>>(B, ldb, n_rhs, ipiv, b0, be, 1);
            GDM_LAUNCHED(ctx, "laswp_rhs");
        }
    }
    return GDM_OK;
}

gdm_status gdm_lu_solve(gdm_ctx *ctx, gdm_precision prec, const void *A, int64_t n, int64_t lda, const int32_t *ipiv,
                        void *B, int64_t ldb, int n_rhs, int conj_trans) {
    if (prec == GDM_FP64)
        return lu_solve_t<double2>(ctx, prec, (const double2 *)A, n, lda, ipiv, (double2 *)B, ldb, n_rhs, conj_trans);
    return lu_solve_t<float2>(ctx, prec, (const float2 *)A, n, lda, ipiv, (float2 *)B, ldb, n_rhs, conj_trans);
}
