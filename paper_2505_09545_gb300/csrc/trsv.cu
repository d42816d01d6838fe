// Persistent blocked triangular solves with the FP32 LU factors (correction solves of the refinement and
// the adjoint solve). The rows are cut into blocks of 128 rows. Once per factorisation, the solve operator
// of every diagonal block is formed explicitly:
//   M_j  = L_pK^{-1} P_pK ... L_p1^{-1} P_p1 restricted to block j  (its 32-row panels p1..pK, with their
//          row interchanges, in the product form the factorisation produced),
//   Ui_j = U_jj^{-1}.
// A solve is then one kernel per triangle: one CTA per row block takes a ticket in dependency order,
// subtracts the contributions of the already published blocks (bounded waits on per-block flags; a CTA
// only waits for lower tickets, which are already running), applies its block operator and publishes its
// rows:
//   mode 0  L   : y_j = M_j (b_j - sum_{k<j} L_jk y_k)             (forward)
//   mode 1  U   : y_j = Ui_j (b_j - sum_{k>j} U_jk y_k)            (backward)
//   mode 2  U^H : y_j = Ui_j^H (b_j - sum_{k<j} U_kj^H y_k)        (forward)
//   mode 3  L^H : y_j = M_j^H (b_j - sum_{k>j} L_kj^H y_k)         (backward)
// The matrix blocks and operators reach shared memory through the TMA engine (a producer warp and a ring
// of stages), which is what keeps one CTA's stream of 128 KB blocks at bandwidth: ordinary loads from
// 256 threads capped it near 17 GB/s per SM. Valid when every pivot stays inside its own 32-row panel
// (pivots searched inside the diagonal blocks); otherwise, and for the FP64 factors, the launch-per-panel
// solver of lu.cu is used.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "gdm_internal.cuh"

#define TRSV_NBS_F32 128
#define TRSV_W_MIN_BLOCKS 32  // row blocks from which the last dependency is folded into W_j (3N >= 3,969)
// the threshold, or GDM_TRSV_W_MIN when set (diagnostics: W_j for shorter systems too)
static int trsv_w_min() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("GDM_TRSV_W_MIN");
        v = e ? atoi(e) : TRSV_W_MIN_BLOCKS;
        if (v < 2) v = 2;
    }
    return v;
}

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

// ------------------------------------------------------------------ block operators
// Per (row block j, triangle) the explicit operator of the block's diagonal part: M_j = L_S^{-1} P_S ...
// L_1^{-1} P_1 (the block's 32-row panels, pivots inside each panel) or Ui_j = U_jj^{-1}, applied to the
// columns of I and stored column-major (coalesced for y = X acc) and row-major (for y = X^H acc).
// A warp solves eight columns of X side by side (lane = row within each 32-row group, 4 groups in registers);
// a CTA of 8 warps covers 64 columns, so that a triangle takes 2 CTAs. The block's factor columns are staged in shared
// memory one 32-column panel at a time: L forward (interchanges of the panel across lanes, then unit lower
// substitution into its own and the later row groups), U backward (division by the diagonal, then the
// column's multiple subtracted from the rows above).
constexpr int OPS_CPW = 8;  // columns per warp
static_assert(2 * TRSV_NBS_F32 / (8 * OPS_CPW) == TRSV_OPS_CTAS, "CTAs per row block of the operators");
__device__ __forceinline__ void block_ops_body(const float2 *__restrict__ A, int64_t lda, int64_t n,
                                               const int32_t *__restrict__ ipiv, float2 *__restrict__ ops, int bid) {
    constexpr int NBS = TRSV_NBS_F32, R = NBS / 32, CGS = NBS / (8 * OPS_CPW);
    __shared__ float2 Ds[32][NBS + 1];
    __shared__ int piv[NBS];
    const int cg = bid % CGS, tri = (bid / CGS) & 1, j = bid / (2 * CGS);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r0 = (int64_t)j * NBS;
    if (r0 >= n) return;
    const int nr = (int)min((int64_t)NBS, n - r0);
    const float2 *D = A + r0 * lda + r0;  // D[r + k*lda]
    const int cb = cg * 8 * OPS_CPW + warp * OPS_CPW;
    float2 x[OPS_CPW][R];
#pragma unroll
    for (int u = 0; u < OPS_CPW; u++)
#pragma unroll
        for (int q = 0; q < R; q++)
            x[u][q] = make_float2((q * 32 + lane == cb + u && cb + u < nr) ? 1.f : 0.f, 0.f);
    if (tri == 0) {
        for (int t = tid; t < nr; t += blockDim.x) piv[t] = (int)(ipiv[r0 + t] - r0);
#pragma unroll
        for (int p = 0; p < R; p++) {
            const int p0 = 32 * p;
            if (p0 >= nr) break;
            const int w = min(32, nr - p0);
            __syncthreads();
            for (int e = tid; e < 32 * NBS; e += blockDim.x) {
                const int t = e / NBS, row = e % NBS;
                Ds[t][row] = (t < w && row < nr) ? D[(int64_t)(p0 + t) * lda + row] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            // the panel's interchanges, in order: rows p0 + t and p0 + q exchange (lanes t and q)
            for (int t = 0; t < w; t++) {
                const int q = piv[p0 + t] - p0;
                if (q > t && q < w) {
#pragma unroll
                    for (int u = 0; u < OPS_CPW; u++) {
                        const float2 vt = make_float2(__shfl_sync(0xffffffffu, x[u][p].x, t),
                                                      __shfl_sync(0xffffffffu, x[u][p].y, t));
                        const float2 vq = make_float2(__shfl_sync(0xffffffffu, x[u][p].x, q),
                                                      __shfl_sync(0xffffffffu, x[u][p].y, q));
                        if (lane == t) x[u][p] = vq;
                        else if (lane == q) x[u][p] = vt;
                    }
                }
            }
            for (int t = 0; t < w; t++) {
                float2 xt[OPS_CPW];
#pragma unroll
                for (int u = 0; u < OPS_CPW; u++)
                    xt[u] = make_float2(__shfl_sync(0xffffffffu, x[u][p].x, t), __shfl_sync(0xffffffffu, x[u][p].y, t));
#pragma unroll
                for (int q2 = p; q2 < R; q2++) {
                    if (q2 > p || lane > t) {
                        const float2 l = Ds[t][q2 * 32 + lane];
#pragma unroll
                        for (int u = 0; u < OPS_CPW; u++) cfms(x[u][q2], l, xt[u]);
                    }
                }
            }
        }
    } else {
#pragma unroll
        for (int p = R - 1; p >= 0; p--) {
            const int p0 = 32 * p;
            if (p0 >= nr) continue;
            const int w = min(32, nr - p0);
            __syncthreads();
            for (int e = tid; e < 32 * NBS; e += blockDim.x) {
                const int t = e / NBS, row = e % NBS;
                Ds[t][row] = (t < w && row < p0 + w) ? D[(int64_t)(p0 + t) * lda + row] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            for (int t = w - 1; t >= 0; t--) {
                const float2 d = Ds[t][p0 + t];
                float2 xr[OPS_CPW];
#pragma unroll
                for (int u = 0; u < OPS_CPW; u++) {
                    float2 v = make_float2(__shfl_sync(0xffffffffu, x[u][p].x, t), __shfl_sync(0xffffffffu, x[u][p].y, t));
                    v = cabs1(d) > 0 ? cmul(v, crecip(d)) : v;
                    if (lane == t) x[u][p] = v;
                    xr[u] = v;
                }
#pragma unroll
                for (int q2 = 0; q2 <= p; q2++) {
                    if (q2 < p || lane < t) {
                        const float2 uk = Ds[t][q2 * 32 + lane];
#pragma unroll
                        for (int u = 0; u < OPS_CPW; u++) cfms(x[u][q2], uk, xr[u]);
                    }
                }
            }
        }
    }
    float2 *ocm = ops + (int64_t)(4 * j + 2 * tri) * NBS * NBS;
    float2 *orm = ocm + (int64_t)NBS * NBS;
#pragma unroll
    for (int u = 0; u < OPS_CPW; u++)
#pragma unroll
        for (int q = 0; q < R; q++) {
            const int row = q * 32 + lane, col = cb + u;
            ocm[col * NBS + row] = x[u][q];
            orm[row * NBS + col] = x[u][q];
        }
}
__global__ void __launch_bounds__(256, 2) k_block_ops(const float2 *__restrict__ A, int64_t lda, int64_t n,
                                                      const int32_t *__restrict__ ipiv, float2 *__restrict__ ops) {
    block_ops_body(A, lda, n, ipiv, ops, blockIdx.x);
}
// the same for every listed problem of a batch: nblk x TRSV_OPS_CTAS CTAs per problem
__global__ void __launch_bounds__(256, 2) k_gr_block_ops(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                         const int *__restrict__ prefix, int na) {
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const GrItem &g = items[i];
    block_ops_body(g.A, g.lda, 3 * g.n, g.ipiv, g.ops, local);
}

// ------------------------------------------------------------------ last-dependency operators
// W_j folds block j's last dependency into its operator, so that once y of the preceding block (in solve order)
// is published, y_j = z_j - W_j y_pred needs one 128 x 128 product instead of two:
//   mode 0 (L):   W = M_j D_{j,j-1},            mode 1 (U):   W = Ui_j D_{j,j+1},
//   mode 2 (U^H): W = Ui_j^H D_{j-1,j}^H,       mode 3 (L^H): W = M_j^H D_{j+1,j}^H,
// with D_{i,k} the 128 x 128 block of the factors (rows of block i, columns of block k, zero past n), and
// z_j = Op_j (b_j - all other dependencies), computed before y_pred is available. CTA (j, mode) forms W in 16-wide
// K chunks staged in shared memory, each thread an 8 x 8 tile of it; W is stored column-major.
__global__ void __launch_bounds__(256) k_block_w(const float2 *__restrict__ A, int64_t lda, int64_t n,
                                                 const float2 *__restrict__ ops, float2 *__restrict__ wops,
                                                 int mode0) {
    constexpr int NBS = TRSV_NBS_F32;
    constexpr int KC = 16;               // K chunk
    __shared__ float2 Op[NBS][KC + 1];   // Op[r][kk]
    __shared__ float2 Dk[KC][NBS + 1];   // D[kk][c]
    const int j = blockIdx.x, mode = mode0 + (int)blockIdx.y;
    const int nblk = (int)((n + NBS - 1) / NBS);
    const int pred = (mode == 0 || mode == 2) ? j - 1 : j + 1;
    float2 *W = wops + (size_t)(4 * j + mode) * NBS * NBS;
    const int tid = threadIdx.x;
    if (pred < 0 || pred >= nblk) {
        for (int e = tid; e < NBS * NBS; e += blockDim.x) W[e] = make_float2(0.f, 0.f);
        return;
    }
    // operator planes: 4j + 2 tri + layout (tri 0: M_j, tri 1: Ui_j; layout 0 column-, 1 row-major)
    const bool herm = mode >= 2;
    const int tri = (mode == 1 || mode == 2) ? 1 : 0;
    const float2 *X = ops + (size_t)(4 * j + 2 * tri + (herm ? 1 : 0)) * NBS * NBS;
    const int64_t rj = (int64_t)j * NBS, rp = (int64_t)pred * NBS;
    const int tr = tid >> 4, tc = tid & 15;  // rows 8 tr .. +8, columns 8 tc .. +8
    float2 acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; a++)
#pragma unroll
        for (int b = 0; b < 8; b++) acc[a][b] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < NBS; k0 += KC) {
        __syncthreads();
        // Op[r][k0 + kk]: plain operator X[r][k] = X_cm[k NBS + r]; hermitian conj(X[k][r]) = conj(X_rm[k NBS + r])
        for (int e = tid; e < NBS * KC; e += blockDim.x) {
            const int r = e % NBS, kk = e / NBS;
            float2 v = X[(size_t)(k0 + kk) * NBS + r];
            if (herm) v.y = -v.y;
            Op[r][kk] = v;
        }
        // D_eff[k0 + kk][c]: modes 0/1: A[rj + k, rp + c]; modes 2/3: conj(A[rp + c, rj + k])
        for (int e = tid; e < KC * NBS; e += blockDim.x) {
            float2 v = make_float2(0.f, 0.f);
            if (!herm) {
                const int kk = e % KC, c = e / KC;
                const int64_t row = rj + k0 + kk, col = rp + c;
                if (row < n && col < n) v = A[col * lda + row];
                Dk[kk][c] = v;
            } else {
                const int c = e % NBS, kk = e / NBS;
                const int64_t row = rp + c, col = rj + k0 + kk;
                if (row < n && col < n) {
                    v = A[col * lda + row];
                    v.y = -v.y;
                }
                Dk[kk][c] = v;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < KC; kk++) {
            float2 o[8], d[8];
#pragma unroll
            for (int a = 0; a < 8; a++) o[a] = Op[8 * tr + a][kk];
#pragma unroll
            for (int b = 0; b < 8; b++) d[b] = Dk[kk][8 * tc + b];
#pragma unroll
            for (int a = 0; a < 8; a++)
#pragma unroll
                for (int b = 0; b < 8; b++) cfma(acc[a][b], o[a], d[b]);
        }
    }
#pragma unroll
    for (int b = 0; b < 8; b++)
#pragma unroll
        for (int a = 0; a < 8; a++) W[(size_t)(8 * tc + b) * NBS + 8 * tr + a] = acc[a][b];
}

// ------------------------------------------------------------------ TMA-fed persistent solve
// Per CTA (row block j): warps 0..7 compute, warp 8 streams data with the TMA engine into a ring of
// NSTAGE shared-memory stages of HALF = NBS/2 columns x NBS rows (one half of a 128 x 128 block):
// first the dependency blocks in processing order, then the block operator. When a dependency is already
// published as its stage is issued, the producer also brings its solution vector y_k into that stage (one
// bulk copy per right-hand side; B's columns 16-byte aligned, a full block), so that the consumers do not
// stall on a load of y_k between two blocks; a dependency published later (the recent ones, on the chain
// of the solve) is waited for and loaded by the consumers, so that its blocks are still prefetched. A
// block is published only after all blocks before it in solve order, so one acquire of a flag covers
// every earlier dependency too.
#define TS_NBS 128
#define TS_HALF 64
#define TS_NSTAGE 3
#define TS_STAGE_BYTES (TS_HALF * TS_NBS * 8)  // 64 KB of complex64

__device__ __forceinline__ uint32_t smem_u32t(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void tmbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32t(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void tmbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32t(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tmbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32t(bar)) : "memory");
}
__device__ __forceinline__ bool tmbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32t(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// bounded wait (~2 s) on an mbarrier phase; false on timeout or when the CTA is aborting
__device__ bool tmbar_wait(uint64_t *bar, uint32_t parity, volatile int *cta_abort, int *gflags) {
    if (tmbar_try(bar, parity)) return true;
    uint64_t t0 = gtimer_t();
    for (uint32_t it = 1;; ++it) {
        if (tmbar_try(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*cta_abort) return false;
            if (gtimer_t() - t0 > 2000000000ull) {
                gdm_dev_error(gflags, GDM_ERR_TIMEOUT, 4);
                *cta_abort = 1;
                return false;
            }
        }
    }
}
__device__ __forceinline__ void tma2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32t(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32t(bar))
        : "memory");
}
__device__ __forceinline__ void bulk1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32t(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32t(bar))
                 : "memory");
}

// (the body takes the descriptor by address and, for the grouped solves of a batch, the block's position in
// solve order tk_given; tk_given < 0 takes a ticket from sync_buf[0])
template <int NR>
__device__ __forceinline__ void trsv_tma_body(const CUtensorMap *tmAp, int64_t n, float2 *__restrict__ B,
                                              int64_t ldb, int rhs0, int nr_here, int mode,
                                              const float2 *__restrict__ ops, const float2 *__restrict__ wops,
                                              int *sync_buf, int *gflags, int tk_given) {
    constexpr int NBS = TS_NBS, HALF = TS_HALF;
    extern __shared__ __align__(1024) unsigned char tsm[];
    float2 *ring = (float2 *)tsm;  // [NSTAGE][HALF][NBS]
    __shared__ __align__(8) uint64_t full[TS_NSTAGE], empty[TS_NSTAGE];
    __shared__ float2 acc[NBS][NR], yk[NBS][NR], part[NBS][NR];
    __shared__ __align__(16) float2 ybuf[TS_NSTAGE][NR][NBS];  // y_k of the dependency in each stage
    __shared__ int ymode[TS_NSTAGE];  // 1: the stage's y_k is in ybuf (set by the producer before its arrive)
    __shared__ int s_ticket, s_dec[2];
    __shared__ volatile int cta_abort;
    const int nblk = (int)((n + NBS - 1) / NBS);
    int *ticket = sync_buf;
    volatile int *gabort = (volatile int *)(sync_buf + 1);
    volatile int *flags = (volatile int *)(sync_buf + 2);
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    // y_k by bulk copies: every column of B 16-byte aligned (and, per block, a full block)
    const bool ytma = (((uintptr_t)B & 15) == 0) && ((ldb & 1) == 0);
    // right-hand sides the bulk copies do not fill stay zero (the copies never write these, so no proxy fence)
    for (int e = tid; e < TS_NSTAGE * NR * NBS; e += blockDim.x)
        if ((e / NBS) % NR >= nr_here) (&ybuf[0][0][0])[e] = make_float2(0.f, 0.f);
    if (tid == 0) {
        s_ticket = tk_given >= 0 ? tk_given : atomicAdd(ticket, 1);
        for (int st = 0; st < TS_NSTAGE; st++) {
            tmbar_init(&full[st], 1);
            tmbar_init(&empty[st], 8);
        }
        cta_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int tk = s_ticket;
    if (tk >= nblk) return;
    const bool fwd = (mode == 0 || mode == 2);
    const int j = fwd ? tk : nblk - 1 - tk;
    const int64_t r0 = (int64_t)j * NBS;
    const int nr = (int)min((int64_t)NBS, n - r0);
    // items: halves of the dependency blocks (with W: all but the last), the two halves of the operator, then (with
    // W, tk >= 1) the two halves of W_j, which applies the last dependency y_pred once it is published
    const bool has_w = wops != nullptr && tk >= 1;
    const int ndep = has_w ? tk - 1 : tk;
    const int nitems = 2 * ndep + 2 + (has_w ? 2 : 0);
    const float2 *opm = ops + (int64_t)(4 * j + 2 * ((mode == 1 || mode == 2) ? 1 : 0) + (mode >= 2 ? 1 : 0)) * NBS * NBS;
    const float2 *wopm = has_w ? wops + (int64_t)(4 * j + mode) * NBS * NBS : nullptr;

    if (warp == 8) {
        // ---------------- producer
        if (lane == 0) {
            int issued = 0;
            int ypub = -1;  // dependencies known published: solve-order positions <= ypub
            for (int it = 0; it < nitems; it++) {
                const int st = it % TS_NSTAGE;
                const uint32_t ph = (uint32_t)((it / TS_NSTAGE) & 1);
                if (!tmbar_wait(&empty[st], ph ^ 1, &cta_abort, gflags)) break;
                issued = it + 1;
                float2 *dst = ring + (size_t)st * HALF * NBS;
                const int half = it & 1;
                // the dependency this item belongs to (position sk in solve order, block kd), or -1
                int sk = -1;
                if (it < 2 * ndep) sk = it / 2;
                else if (it >= 2 * ndep + 2) sk = tk - 1;
                const int kd = sk < 0 ? -1 : (fwd ? sk : nblk - 1 - sk);
                bool ycopy = false;
                if (kd >= 0 && ytma && (int64_t)(kd + 1) * NBS <= n) {
                    if (sk <= ypub) {
                        ycopy = true;
                    } else {
                        int f;
                        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(f) : "l"(flags + kd) : "memory");
                        if (f != 0) {
                            // order the published data (generic proxy) before the bulk copies' reads
                            asm volatile("fence.proxy.async.global;" ::: "memory");
                            ypub = sk;
                            ycopy = true;
                        }
                    }
                }
                ymode[st] = ycopy ? 1 : 0;
                if (ycopy) {
                    tmbar_expect_tx(&full[st], TS_STAGE_BYTES + (uint32_t)(nr_here * NBS * 8));
                    for (int q = 0; q < nr_here; q++)
                        bulk1d(&ybuf[st][q][0], B + (int64_t)(rhs0 + q) * ldb + (int64_t)kd * NBS, NBS * 8,
                               &full[st]);
                } else {
                    tmbar_expect_tx(&full[st], TS_STAGE_BYTES);
                }
                if (it < 2 * ndep) {
                    const int s = it / 2;
                    const int k = fwd ? s : nblk - 1 - s;
                    const int64_t k0 = (int64_t)k * NBS;
                    // no-trans: columns of block k, rows of block j; conj-trans: columns of block j, rows of block k
                    const int x = (int)(2 * ((mode <= 1) ? r0 : k0));
                    const int y = (int)(((mode <= 1) ? k0 : r0) + half * HALF);
                    tma2d(dst, tmAp, x, y, &full[st]);
                } else if (it < 2 * ndep + 2) {
                    bulk1d(dst, opm + (size_t)half * HALF * NBS, TS_STAGE_BYTES, &full[st]);
                } else {
                    bulk1d(dst, wopm + (size_t)half * HALF * NBS, TS_STAGE_BYTES, &full[st]);
                }
            }
            // on an abort, let the copies still in flight land before the CTA (and its shared memory) goes away;
            // the most recent NSTAGE items are the latest phase of each stage
            if (cta_abort) {
                for (int it = max(0, issued - TS_NSTAGE); it < issued; it++) {
                    uint64_t *bar = &full[it % TS_NSTAGE];
                    const uint32_t ph = (uint32_t)((it / TS_NSTAGE) & 1);
                    uint64_t t0 = gtimer_t();
                    while (!tmbar_try(bar, ph) && gtimer_t() - t0 < 2000000000ull) {
                    }
                }
            }
        }
        return;
    }
    // ---------------- consumers (warps 0..7, 256 threads); thread 0 takes every wait and publishes the
    // outcome before a named barrier so all consumer warps branch alike
    int dc = 0;
    auto agree = [&](bool ok0) -> bool {
        if (tid == 0) s_dec[dc & 1] = ok0 ? 1 : 0;
        asm volatile("bar.sync 1, 256;" ::: "memory");
        bool r = s_dec[dc & 1] != 0;
        dc++;
        return r;
    };
    for (int e = tid; e < NBS * NR; e += 256) {
        int r = e / NR, q = e % NR;
        acc[r][q] = (r < nr && q < nr_here) ? B[(int64_t)(rhs0 + q) * ldb + r0 + r] : make_float2(0.f, 0.f);
    }
    const int r = tid % NBS, hh = tid / NBS;  // row and which 32-column quarter pair (no-trans)
    float2 zr[NR];                            // z_j = Op_j acc of row r (threads hh == 0), before W_j y_pred
    int it = 0;
    // stage s: 0 .. ndep-1 dependencies, ndep the operator, ndep + 1 (has_w) the last dependency through W_j
    const int nstage = ndep + 1 + (has_w ? 1 : 0);
    for (int s = 0; s < nstage; s++) {
        const bool is_op = (s == ndep);
        const bool is_w = (s == ndep + 1);
        // y_k loaded by the consumers (for a half whose stage did not bring it), once per dependency
        bool have_yk = false;
        auto load_yk = [&]() -> bool {
            // dependency s, or for is_w (s = tk) the preceding block in solve order, dependency tk - 1
            const int sk = is_w ? s - 1 : s;
            const int k = fwd ? sk : nblk - 1 - sk;
            const int64_t k0 = (int64_t)k * NBS;
            const int nk = (int)min((int64_t)NBS, n - k0);
            bool ok0 = true;
            if (tid == 0) {
                if (flags[k] == 0) {
                    uint64_t t0 = gtimer_t();
                    unsigned w = 0;
                    while (flags[k] == 0) {
                        if ((++w & 255) == 0) {
                            if (*gabort || cta_abort) {
                                ok0 = false;
                                break;
                            }
                            if (gtimer_t() - t0 > 2000000000ull) {
                                gdm_dev_error(gflags, GDM_ERR_TIMEOUT, 3);
                                *gabort = 1;
                                ok0 = false;
                                break;
                            }
                        }
                    }
                }
                __threadfence();
            }
            if (!agree(ok0)) {
                cta_abort = 1;
                return false;
            }
            for (int e = tid; e < NBS * NR; e += 256) {
                int rr = e / NR, q = e % NR;
                yk[rr][q] = (rr < nk && q < nr_here) ? __ldcg(B + (int64_t)(rhs0 + q) * ldb + k0 + rr)
                                                     : make_float2(0.f, 0.f);
            }
            asm volatile("bar.sync 1, 256;" ::: "memory");
            return true;
        };
        float2 sum[NR];
#pragma unroll
        for (int q = 0; q < NR; q++) sum[q] = make_float2(0.f, 0.f);
        for (int half = 0; half < 2; half++, it++) {
            const int st = it % TS_NSTAGE;
            bool ok0 = true;
            if (tid == 0) ok0 = tmbar_wait(&full[st], (uint32_t)((it / TS_NSTAGE) & 1), &cta_abort, gflags);
            if (!agree(ok0)) {
                cta_abort = 1;
                return;
            }
            const bool yt = !is_op && ymode[st] != 0;
            if (!is_op && !yt && !have_yk) {
                if (!load_yk()) return;
                have_yk = true;
            }
            const float2 *sb = ring + (size_t)st * HALF * NBS;  // sb[c * NBS + row]
            // the vector the block multiplies: element (row cc, right-hand side q) at src[cc * srs + q * sqs]
            const float2 *src = is_op ? &acc[0][0] : (yt ? &ybuf[st][0][0] : &yk[0][0]);
            const int srs = yt ? 1 : NR, sqs = yt ? NBS : 1;
            if (mode <= 1 || is_op || is_w) {
                // y_r -= sum_c M[r][c] v[c] (operator: y_r = sum_c Op[r][c] acc[c]; W: sum_c W[r][c] y_pred[c]);
                // thread (r, hh) takes 32 columns
                const bool herm = is_op && mode >= 2;
#pragma unroll 8
                for (int c = hh * 32; c < hh * 32 + 32; c++) {
                    float2 m = sb[c * NBS + r];
                    if (herm) m.y = -m.y;
                    const int cc = half * HALF + c;
#pragma unroll
                    for (int q = 0; q < NR; q++) cfma(sum[q], m, src[cc * srs + q * sqs]);
                }
            } else {
                // acc[c] -= sum_rr conj(M[k0+rr][r0+c]) yk[rr]: 4 threads per column of this half, rows rotated
                const int c = tid / 4, p = tid % 4;
                float2 cs[NR];
#pragma unroll
                for (int q = 0; q < NR; q++) cs[q] = make_float2(0.f, 0.f);
#pragma unroll 8
                for (int i = 0; i < NBS / 4; i++) {
                    const int rr = (p + 4 * i + 4 * c) & (NBS - 1);
                    float2 m = sb[c * NBS + rr];
                    m.y = -m.y;
#pragma unroll
                    for (int q = 0; q < NR; q++) cfma(cs[q], m, src[rr * srs + q * sqs]);
                }
#pragma unroll
                for (int q = 0; q < NR; q++)
                    for (int o = 1; o < 4; o <<= 1) {
                        cs[q].x += __shfl_xor_sync(0xffffffffu, cs[q].x, o);
                        cs[q].y += __shfl_xor_sync(0xffffffffu, cs[q].y, o);
                    }
                if (p == 0 && half * HALF + c < nr)
#pragma unroll
                    for (int q = 0; q < NR; q++) acc[half * HALF + c][q] = csub(acc[half * HALF + c][q], cs[q]);
            }
            __syncwarp();
            if (lane == 0) tmbar_arrive(&empty[st]);
        }
        if (mode <= 1 || is_op || is_w) {
            if (hh == 1)
#pragma unroll
                for (int q = 0; q < NR; q++) part[r][q] = sum[q];
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (hh == 0 && r < nr) {
                if (is_op && !has_w) {
                    for (int q = 0; q < NR; q++)
                        if (q < nr_here) B[(int64_t)(rhs0 + q) * ldb + r0 + r] = cadd(sum[q], part[r][q]);
                } else if (is_op) {
#pragma unroll
                    for (int q = 0; q < NR; q++) zr[q] = cadd(sum[q], part[r][q]);
                } else if (is_w) {
                    for (int q = 0; q < NR; q++)
                        if (q < nr_here) B[(int64_t)(rhs0 + q) * ldb + r0 + r] = csub(zr[q], cadd(sum[q], part[r][q]));
                } else {
#pragma unroll
                    for (int q = 0; q < NR; q++) acc[r][q] = csub(acc[r][q], cadd(sum[q], part[r][q]));
                }
            }
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");
    }
    __threadfence();
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (tid == 0) atomicExch((int *)(flags + j), 1);
}
template <int NR>
__global__ void __launch_bounds__(288, 1) k_trsv_tma(const __grid_constant__ CUtensorMap tmA, int64_t n,
                                                   float2 *__restrict__ B, int64_t ldb, int rhs0, int nr_here,
                                                   int mode, const float2 *__restrict__ ops,
                                                   const float2 *__restrict__ wops, int *sync_buf, int *gflags) {
    trsv_tma_body<NR>(&tmA, n, B, ldb, rhs0, nr_here, mode, ops, wops, sync_buf, gflags, -1);
}
// The solves of every listed problem of a batch in one launch: a global ticket T (taken in launch order)
// enumerates (position tk in solve order, problem) with tk slowest, so that every problem's blocks come in
// dependency order and the first blocks of all problems come first; jprefix[tk] counts the tickets before
// position tk (the problems with more than tk blocks are a prefix of the list, which is sorted by
// decreasing size). Each problem has its own flags (GrItem sync) and descriptor (maps).
__global__ void __launch_bounds__(288, 1) k_gr_trsv(const GrItem *__restrict__ items, const CUtensorMap *maps,
                                                    const int *__restrict__ list, const int *__restrict__ jprefix,
                                                    int nj, int mode, int *ticket, int *gflags) {
    __shared__ int s_t[2];
    if (threadIdx.x == 0) {
        const int T = atomicAdd(ticket, 1);
        int tk = 0;
        while (tk + 1 < nj && jprefix[tk + 1] <= T) tk++;
        s_t[0] = tk;
        s_t[1] = list[T - jprefix[tk]];
    }
    __syncthreads();
    const int tk = s_t[0], i = s_t[1];
    const GrItem &g = items[i];
    // the descriptor was written by the host before the launch: order that write before the copies
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)&maps[i]) : "memory");
    trsv_tma_body<2>(&maps[i], 3 * g.n, g.w, 3 * g.n, 0, g.nr, mode, g.ops, nullptr, g.sync, gflags, tk);
}

// every pivot inside its own block of nbs rows?
__global__ void k_pivots_local(const int32_t *__restrict__ ipiv, int64_t n, int nbs, int *bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (ipiv[i] / nbs != i / nbs) atomicExch(bad, 1);
}

PFN_cuTensorMapEncodeTiled_v12000 trsv_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

gdm_status launch_modes_f32(gdm_ctx *ctx, const float2 *A, int64_t lda, int64_t n, float2 *B, int64_t ldb, int n_rhs,
                            const int *modes, int nmodes, int *sync_buf, const float2 *ops) {
    const int nblk = (int)((n + TS_NBS - 1) / TS_NBS);
    auto fn = trsv_encode_fn();
    if (!fn) return gdm_fail(ctx, GDM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)(2 * n), (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)(2 * lda * 4)};
    cuuint32_t box[2] = {2 * TS_NBS, TS_HALF};
    cuuint32_t es[2] = {1, 1};
    if (fn(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)A, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return gdm_fail(ctx, GDM_ERR_CUDA, "cuTensorMapEncodeTiled failed (solve)");
    const int smem = TS_NSTAGE * TS_STAGE_BYTES;
    static bool attr = false;
    if (!attr) {
        GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_trsv_tma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = true;
    }
    for (int mi = 0; mi < nmodes; mi++) {
        for (int q0 = 0; q0 < n_rhs; q0 += 2) {
            int nr = n_rhs - q0 < 2 ? n_rhs - q0 : 2;
            GDM_CUDA_TRY(ctx, cudaMemsetAsync(sync_buf, 0, sizeof(int) * (nblk + 2), ctx->stream));
            const float2 *wops = nblk >= trsv_w_min() ? ops + (size_t)4 * nblk * TS_NBS * TS_NBS : nullptr;
            k_trsv_tma<2><<<nblk, 288, smem, ctx->stream>>>(map, n, B, ldb, q0, nr, modes[mi], ops, wops, sync_buf,
                                                            ctx->dflags);
            GDM_LAUNCHED(ctx, "trsv_tma");
        }
    }
    return GDM_OK;
}

template <class C, int NBS> gdm_status launch_ops(gdm_ctx *ctx, const C *A, int64_t lda, int64_t n, const int32_t *ipiv,
                                                  C *ops, int conj_trans) {
    static_assert(NBS == TRSV_NBS_F32, "block operators of 128-row blocks");
    const int nblk = (int)((n + NBS - 1) / NBS);
    k_block_ops<<<(unsigned)(2 * nblk * (NBS / (8 * OPS_CPW))), 256, 0, ctx->stream>>>(
        (const float2 *)A, lda, n, ipiv, (float2 *)ops);
    GDM_LAUNCHED(ctx, "block_ops");
    // the last-dependency operators W of the two modes of this solve direction (after all operator planes), for
    // systems long enough that the shorter dependency chain repays forming them
    if (nblk >= trsv_w_min()) {
        k_block_w<<<dim3((unsigned)nblk, 2), 256, 0, ctx->stream>>>((const float2 *)A, lda, n, (const float2 *)ops,
                                                                    (float2 *)ops + (size_t)4 * nblk * NBS * NBS,
                                                                    conj_trans ? 2 : 0);
        GDM_LAUNCHED(ctx, "block_w");
    }
    return GDM_OK;
}

}  // namespace

bool gdm_trsv_encode_map(const float2 *A, int64_t n, int64_t lda, void *map) {
    auto fn = trsv_encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)(2 * n), (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)(2 * lda * 4)};
    cuuint32_t box[2] = {2 * TS_NBS, TS_HALF};
    cuuint32_t es[2] = {1, 1};
    return fn((CUtensorMap *)map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)A, dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

gdm_status gdm_gr_block_ops(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units) {
    if (units <= 0) return GDM_OK;
    k_gr_block_ops<<<(unsigned)units, 256, 0, ctx->stream>>>(it, list, prefix, na);
    GDM_LAUNCHED(ctx, "gr_block_ops");
    return GDM_OK;
}

// one triangle (mode 0: L, mode 1: U) of every listed problem; the flags of those problems and *ticket must
// be zero at the launch
gdm_status gdm_gr_trsv(gdm_ctx *ctx, const GrItem *it, const void *maps, const int *list, const int *jprefix,
                       int nj, int units, int mode, int *ticket) {
    if (units <= 0) return GDM_OK;
    const int smem = TS_NSTAGE * TS_STAGE_BYTES;
    static bool attr = false;
    if (!attr) {
        GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_gr_trsv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = true;
    }
    k_gr_trsv<<<(unsigned)units, 288, smem, ctx->stream>>>(it, (const CUtensorMap *)maps, list, jprefix, nj, mode,
                                                          ticket, ctx->dflags);
    GDM_LAUNCHED(ctx, "gr_trsv");
    return GDM_OK;
}

size_t gdm_trsv_sync_bytes(int64_t n) { return sizeof(int) * ((n + 31) / 32 + 8); }

// bytes of the FP32 block operators (4 planes of 128 x 128 per row block) and the last-dependency operators W
// (one plane per solve mode and row block)
size_t gdm_trsv_inv_bytes(int64_t n) {
    const int64_t nb32 = (n + TRSV_NBS_F32 - 1) / TRSV_NBS_F32;
    return (size_t)8 * nb32 * TRSV_NBS_F32 * TRSV_NBS_F32 * sizeof(float2);
}

// 1 if all pivots stay inside their nbs-row block (synchronises)
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

gdm_status gdm_trsv_prepare(gdm_ctx *ctx, gdm_precision prec, const void *A, int64_t n, int64_t lda,
                            const int32_t *ipiv, void *ops, int conj_trans) {
    if (prec == GDM_FP64) return GDM_ERR_UNSUPPORTED;  // the FP64 path uses the launch-per-panel solver
    return launch_ops<float2, TRSV_NBS_F32>(ctx, (const float2 *)A, lda, n, ipiv, (float2 *)ops, conj_trans);
}

// solve with the factors: conj_trans = 0: U^{-1} L^{-1} P b; conj_trans = 1: P^T L^{-H} U^{-H} b
gdm_status gdm_trsv_persistent(gdm_ctx *ctx, gdm_precision prec, const void *A, int64_t n, int64_t lda,
                               const int32_t *ipiv, void *B, int64_t ldb, int n_rhs, int conj_trans, int *sync_buf,
                               const void *ops) {
    (void)ipiv;
    static const int fwd[2] = {0, 1}, adj[2] = {2, 3};
    const int *modes = conj_trans ? adj : fwd;
    if (prec == GDM_FP64) return GDM_ERR_UNSUPPORTED;  // the FP64 path uses the launch-per-panel solver
    return launch_modes_f32(ctx, (const float2 *)A, lda, n, (float2 *)B, ldb, n_rhs, modes, 2, sync_buf,
                            (const float2 *)ops);
}
