// Iterative solver for discretised structures beyond the dense path.
//
// The paper stores and inverts the dense coupling matrix, which bounds it to about 10^4 dipoles, and
// names iterative schemes as the way past that bound (Sec. "Conclusions", Sec. "Benchmarks"). This file
// solves A F = F0 for cells (kind 3) without forming A:
//
//   * flexible GMRES(m) in FP64 (right preconditioning, the preconditioned basis Z kept explicitly so
//     that an inexact, FP32 preconditioner is allowed), classical Gram-Schmidt with one
//     re-orthogonalisation, Givens rotations on the host, all right-hand sides in lockstep;
//   * the operator A z is matrix-free (O(N^2) pair evaluations per step, O(N) memory). Every cycle
//     starts from the true residual b - A x in double-float arithmetic (the refinement residual), and
//     its Arnoldi steps apply an FP32 operator (FP32 Green sums with a double-float phase, about 1e-6
//     relative, ~1/9 of the double-float work) until the cycle has reduced its residual by 1e-4: the
//     cycles are the outer steps of an iterative refinement whose inner solver is FGMRES on the
//     low-precision operator, so the solution still reaches the double-float accuracy. A cycle that
//     fails to halve the true residual switches the rest of the solve to the double-float operator;
//     GDM_GMRES_EXACT_OPERATOR uses it throughout;
//   * a two-level mixed-precision preconditioner
//         M^-1 v = P A_c^-1 R v + B^-1 (v - P R v)
//     A_c: a coarser model of the structure, its cells merged 2 x 2 x 2 on the lattice (position = the
//          children's centroid, polarisability = the sum of the children's), factored by the TF32
//          tensor-core LU. A coarse cell with k children stands for a cube of volume k d^3 filled with
//          their mean susceptibility chi = mean(eps_i - eps_env): its self-term block is that of such a
//          cube, 1 - S alpha = 1 + chi/(3 eps_env) whatever k, while its coupling to the other coarse
//          cells carries the summed polarisability. (Diluting chi over the full (2 d)^3 cube instead
//          makes the partly filled coarse cells at a surface respond far too weakly, and the coarse
//          correction then slows GMRES down several-fold on irregular structures.)
//     R:   average over the children; P: copy to the children;
//     B:   block Jacobi, the exact diagonal blocks of A over runs of consecutive cells in Morton
//          (Z-curve) order of the lattice, each factored by the TF32 LU and applied by one CTA per
//          block (forward and backward substitution through shared memory).
// Cells are sorted by their Morton key once; in that order the children of a coarse cell and the cells
// of a block are contiguous (the coarse key is the fine key shifted by three bits), and the solver runs
// on the permuted system.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <complex>
#include <utility>
#include <vector>

#include "gdm_internal.cuh"
#include "pool.cuh"

gdm_status gdm_launch_residual_ws(gdm_ctx *ctx, const gdm_problem *p, const double *rhs, const double *X, int n_rhs,
                                  int adjoint, double *r, double *norms2, double2 *Pbuf, double2 *partial, void *ffws,
                                  int ff_prepare);
size_t gdm_ff_scratch_bytes(int64_t n);
size_t gdm_green_partial_bytes(gdm_ctx *ctx, int64_t m, int64_t n, int out);
gdm_status gdm_launch_residual_f32(gdm_ctx *ctx, const gdm_problem *p, const double *rhs, const double *X, int n_rhs,
                                   double *r, double *norms2, double2 *Pbuf, double2 *partial, const void *dipf);
const void *gdm_ff_positions(void *ffws);
gdm_status gdm_ff_prepare(gdm_ctx *ctx, const gdm_problem *p, void *ffws);

namespace {

constexpr int GM_MAX_RHS = 8;
constexpr int GM_MAX_RESTART = 120;
constexpr int GM_MAX_BLOCK_CELLS = 1024;
constexpr int GM_T = 256;              // threads of the vector kernels
constexpr int GM_ROWS = 4 * GM_T;      // rows per CTA of the reductions
constexpr int BJ_T = 512;              // threads of the block solve
constexpr int BJ_W = 32;               // panel width of the block solve (the LU's pivot panel)
constexpr double GM_INNER = 1e-4;      // residual reduction per cycle with the FP32 operator

inline unsigned nblk(int64_t n, int t = GM_T) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------ partition (host)
uint64_t spread3(uint64_t v) {
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}

struct Partition {
    std::vector<int> perm;    // permuted position -> original cell
    std::vector<int> parent;  // permuted cell -> coarse cell
    std::vector<int> coff;    // coarse cell -> first permuted child (nc + 1)
    std::vector<int> boff;    // block -> first permuted cell (nb + 1)
};

void make_partition(const std::vector<double> &pos, int64_t n, double d, int block_cells, Partition &P) {
    double mn[3] = {pos[0], pos[1], pos[2]};
    for (int64_t i = 1; i < n; i++)
        for (int a = 0; a < 3; a++) mn[a] = std::min(mn[a], pos[3 * i + a]);
    std::vector<std::pair<uint64_t, int>> key(n);
    for (int64_t i = 0; i < n; i++) {
        uint64_t k = 0;
        for (int a = 0; a < 3; a++) {
            double t = floor((pos[3 * i + a] - mn[a]) / d + 0.5);
            uint64_t c = t < 0 ? 0 : (t > 2097151.0 ? 2097151 : (uint64_t)t);
            k |= spread3(c) << a;
        }
        key[i] = {k, (int)i};
    }
    std::sort(key.begin(), key.end());
    P.perm.resize(n);
    P.parent.resize(n);
    P.coff.clear();
    for (int64_t i = 0; i < n; i++) {
        P.perm[i] = key[i].second;
        if (i == 0 || (key[i].first >> 3) != (key[i - 1].first >> 3)) P.coff.push_back((int)i);
        P.parent[i] = (int)P.coff.size() - 1;
    }
    P.coff.push_back((int)n);
    P.boff.clear();
    for (int64_t s = 0; s < n; s += block_cells) P.boff.push_back((int)s);
    P.boff.push_back((int)n);
}

// ------------------------------------------------------------------ set-up kernels
__global__ void k_gather_cells(const double *__restrict__ pos, const double2 *__restrict__ eps,
                               const int *__restrict__ perm, int64_t n, double *__restrict__ pos_p,
                               double2 *__restrict__ eps_p) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = perm[i];
    for (int a = 0; a < 3; a++) pos_p[3 * i + a] = pos[3 * o + a];
    eps_p[i] = eps[o];
}

// coarse cell: centroid of its children; eps_c - eps_env = (1/8) sum (eps_i - eps_env), i.e. alpha_c =
// sum alpha_i at the mesh step 2 d; chi_c = mean (eps_i - eps_env) for its self-term block
__global__ void k_coarse_cells(const double *__restrict__ pos_p, const double2 *__restrict__ eps_p,
                               const int *__restrict__ coff, int64_t nc, double eps_env, double *__restrict__ pos_c,
                               double2 *__restrict__ eps_c, double2 *__restrict__ chi_c) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int b = coff[c], e = coff[c + 1];
    double s[3] = {0.0, 0.0, 0.0};
    double2 x = make_double2(0.0, 0.0);
    for (int i = b; i < e; i++) {
        for (int a = 0; a < 3; a++) s[a] += pos_p[3 * i + a];
        x.x += eps_p[i].x - eps_env;
        x.y += eps_p[i].y;
    }
    const double inv = 1.0 / (e - b);
    for (int a = 0; a < 3; a++) pos_c[3 * c + a] = s[a] * inv;
    eps_c[c] = make_double2(eps_env + 0.125 * x.x, 0.125 * x.y);
    chi_c[c] = make_double2(x.x * inv, x.y * inv);
}

// self-term blocks of the coarse model: 1 + chi_c/(3 eps_env) on the diagonal of each 3 x 3 block
__global__ void k_coarse_diag(float2 *__restrict__ Ac, int64_t lda, const double2 *__restrict__ chi_c, int64_t nc,
                              double inv3eps) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 3 * nc) return;
    const double2 chi = chi_c[e / 3];
    Ac[e * lda + e] = make_float2((float)(1.0 + chi.x * inv3eps), (float)(chi.y * inv3eps));
}

// rows of a (3 n) x n_rhs block, permuted: dst[3 i + a] = src[3 perm[i] + a] (or the inverse)
__global__ void k_permute_rows(const double2 *__restrict__ src, double2 *__restrict__ dst, const int *__restrict__ perm,
                               int64_t n, int nr, int inverse) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 3 * n * nr) return;
    const int64_t ns = 3 * n, q = e / ns, r = e % ns, i = r / 3, a = r % 3;
    const int64_t o = 3 * (int64_t)perm[i] + a;
    if (inverse) dst[q * ns + o] = src[q * ns + r];
    else dst[q * ns + r] = src[q * ns + o];
}

// ------------------------------------------------------------------ preconditioner kernels
// rc = R v (mean over the children), FP32 for the coarse solve; yc = rc (solved in place afterwards)
__global__ void k_restrict(const double2 *__restrict__ v, int64_t ns, int nr, const int *__restrict__ coff,
                           int64_t nc, float2 *__restrict__ rc, float2 *__restrict__ yc) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 3 * nc * nr) return;
    const int64_t nc3 = 3 * nc, q = e / nc3, r = e % nc3, c = r / 3, a = r % 3;
    const int b = coff[c], en = coff[c + 1];
    double sx = 0.0, sy = 0.0;
    for (int i = b; i < en; i++) {
        const double2 x = v[q * ns + 3 * (int64_t)i + a];
        sx += x.x;
        sy += x.y;
    }
    const double inv = 1.0 / (en - b);
    const float2 o = make_float2((float)(sx * inv), (float)(sy * inv));
    rc[e] = o;
    yc[e] = o;
}

// z = B^-1 (v - P rc) + P yc over one block per CTA. fac: the block's LU factors (complex64,
// column-major, leading dimension ld), pivots in the LU's product form: per 32-row panel the row
// interchanges of that panel, then the unit-lower elimination; backward substitution with the upper
// factor (diagonal included) panel by panel from the last. The block's right-hand sides stay in shared
// memory; the factors are streamed once per substitution.
template <int NR>
__global__ void __launch_bounds__(BJ_T) k_bj_solve(const float2 *__restrict__ fac, const int64_t *__restrict__ fac_off,
                                                   const int *__restrict__ fac_ld, const int32_t *__restrict__ piv,
                                                   const int *__restrict__ boff, const double2 *__restrict__ v,
                                                   int64_t ns, const int *__restrict__ parent,
                                                   const float2 *__restrict__ rc, const float2 *__restrict__ yc,
                                                   int64_t nc3, int use_coarse, double2 *__restrict__ z) {
    extern __shared__ float2 ysm[];  // [NR][m]
    constexpr int nr = NR;
    const int b = blockIdx.x;
    const int s = boff[b];
    const int m = 3 * (boff[b + 1] - s);
    const int64_t r0 = 3 * (int64_t)s;
    const float2 *A = fac + fac_off[b];
    const int64_t ld = fac_ld[b];
    const int32_t *ip = piv + r0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < m * nr; e += BJ_T) {
        const int q = e / m, r = e % m;
        const double2 x = v[q * ns + r0 + r];
        float2 y = make_float2((float)x.x, (float)x.y);
        if (use_coarse) y = csub(y, rc[q * nc3 + 3 * (int64_t)parent[s + r / 3] + r % 3]);
        ysm[q * m + r] = y;
    }
    __syncthreads();
    // the panel's 32 x 32 diagonal block, staged so that the warp-serial solve reads shared memory only
    __shared__ float2 D[BJ_W][BJ_W + 1];
    __shared__ int spiv[BJ_W];  // the panel's row interchanges
    // y[r] -= sum_{i < w} A[r, c0 + i] y[c0 + i] for the rows r of [rb, re) (16 independent loads in flight)
    auto update = [&](int c0, int w, int rb, int re) {
        for (int r = rb + tid; r < re; r += BJ_T) {
            float2 acc[NR];
#pragma unroll
            for (int q = 0; q < NR; q++) acc[q] = make_float2(0.f, 0.f);
            for (int i0 = 0; i0 < w; i0 += 16) {
                float2 a[16];
#pragma unroll
                for (int k = 0; k < 16; k++) a[k] = i0 + k < w ? A[(c0 + i0 + k) * ld + r] : make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < 16; k++)
                    if (i0 + k < w) {
#pragma unroll
                        for (int q = 0; q < NR; q++) cfma(acc[q], a[k], ysm[q * m + c0 + i0 + k]);
                    }
            }
#pragma unroll
            for (int q = 0; q < NR; q++) ysm[q * m + r] = csub(ysm[q * m + r], acc[q]);
        }
    };
    auto stage_diag = [&](int c0, int w) {
        for (int e = tid; e < BJ_W * BJ_W; e += BJ_T) {
            const int r = e % BJ_W, c = e / BJ_W;
            D[r][c] = (r < w && c < w) ? A[(c0 + c) * ld + c0 + r] : make_float2(0.f, 0.f);
        }
        if (tid < w) spiv[tid] = ip[c0 + tid];
    };
    // forward: P, then L^-1 (unit diagonal), panel by panel
    for (int c0 = 0; c0 < m; c0 += BJ_W) {
        const int w = min(BJ_W, m - c0);
        stage_diag(c0, w);
        __syncthreads();
        if (tid < nr) {
            float2 *y = ysm + tid * m;
            for (int k = 0; k < w; k++) {
                const int r1 = c0 + k, r2 = spiv[k];
                if (r2 != r1) {
                    const float2 t = y[r1];
                    y[r1] = y[r2];
                    y[r2] = t;
                }
            }
        }
        __syncthreads();
        if (warp < nr) {
            float2 *y = ysm + warp * m;
            float2 x = lane < w ? y[c0 + lane] : make_float2(0.f, 0.f);
            for (int i = 0; i < w; i++) {
                float2 xi;
                xi.x = __shfl_sync(0xffffffffu, x.x, i);
                xi.y = __shfl_sync(0xffffffffu, x.y, i);
                if (lane > i && lane < w) cfms(x, D[lane][i], xi);
            }
            if (lane < w) y[c0 + lane] = x;
        }
        __syncthreads();
        update(c0, w, c0 + w, m);
        __syncthreads();
    }
    // backward: U^-1, last panel first
    for (int c0 = ((m - 1) / BJ_W) * BJ_W; c0 >= 0; c0 -= BJ_W) {
        const int w = min(BJ_W, m - c0);
        stage_diag(c0, w);
        __syncthreads();
        if (warp < nr) {
            float2 *y = ysm + warp * m;
            float2 x = lane < w ? y[c0 + lane] : make_float2(0.f, 0.f);
            for (int i = w - 1; i >= 0; i--) {
                if (lane == i) {
                    const float2 u = D[i][i];
                    const float dd = 1.0f / (u.x * u.x + u.y * u.y);
                    x = cmul(x, make_float2(u.x * dd, -u.y * dd));
                }
                float2 xi;
                xi.x = __shfl_sync(0xffffffffu, x.x, i);
                xi.y = __shfl_sync(0xffffffffu, x.y, i);
                if (lane < i) cfms(x, D[lane][i], xi);
            }
            if (lane < w) y[c0 + lane] = x;
        }
        __syncthreads();
        update(c0, w, 0, c0);
        __syncthreads();
    }
    for (int e = tid; e < m * nr; e += BJ_T) {
        const int q = e / m, r = e % m;
        float2 y = ysm[q * m + r];
        double2 o = make_double2((double)y.x, (double)y.y);
        if (use_coarse) {
            const float2 c = yc[q * nc3 + 3 * (int64_t)parent[s + r / 3] + r % 3];
            o.x += (double)c.x;
            o.y += (double)c.y;
        }
        z[q * ns + r0 + r] = o;
    }
}

template <int NR>
gdm_status launch_bj(gdm_ctx *ctx, int nb, int smem, const float2 *fac, const int64_t *foff, const int *fld,
                     const int32_t *piv, const int *boff, const double2 *v, int64_t ns, const int *parent,
                     const float2 *rc, const float2 *yc, int64_t nc3, int use_coarse, double2 *z, bool set_attr) {
    if (set_attr)
        GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_bj_solve<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    else {
        k_bj_solve<NR><<<nb, BJ_T, smem, ctx->stream>>>(fac, foff, fld, piv, boff, v, ns, parent, rc, yc, nc3,
                                                        use_coarse, z);
        GDM_LAUNCHED(ctx, "gmres_block_solve");
    }
    return GDM_OK;
}

gdm_status launch_bj_nr(gdm_ctx *ctx, int nr, int nb, int smem, const float2 *fac, const int64_t *foff,
                        const int *fld, const int32_t *piv, const int *boff, const double2 *v, int64_t ns,
                        const int *parent, const float2 *rc, const float2 *yc, int64_t nc3, int use_coarse,
                        double2 *z, bool set_attr) {
#define GM_BJ_CASE(K)                                                                                          \
    case K:                                                                                                    \
        return launch_bj<K>(ctx, nb, smem, fac, foff, fld, piv, boff, v, ns, parent, rc, yc, nc3, use_coarse, z, \
                            set_attr);
    switch (nr) {
        GM_BJ_CASE(1)
        GM_BJ_CASE(2)
        GM_BJ_CASE(3)
        GM_BJ_CASE(4)
        GM_BJ_CASE(5)
        GM_BJ_CASE(6)
        GM_BJ_CASE(7)
        GM_BJ_CASE(8)
    }
#undef GM_BJ_CASE
    return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "block solve: n_rhs %d", nr);
}

// z = P yc + (v - P rc): the coarse correction alone (no block part)
__global__ void k_coarse_only(const double2 *__restrict__ v, int64_t ns, int nr, const int *__restrict__ parent,
                              const float2 *__restrict__ rc, const float2 *__restrict__ yc, int64_t nc3,
                              double2 *__restrict__ z) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ns * nr) return;
    const int64_t q = e / ns, r = e % ns;
    const int64_t c = q * nc3 + 3 * (int64_t)parent[r / 3] + r % 3;
    const double2 x = v[e];
    z[e] = make_double2(x.x - (double)rc[c].x + (double)yc[c].x, x.y - (double)rc[c].y + (double)yc[c].y);
}

// ------------------------------------------------------------------ Krylov kernels
// part[(q * J + i) * nct + cta] = sum over the CTA's rows of conj(V_i[r, q]) w[r, q], i < J; eight basis
// vectors per reduction round
__global__ void __launch_bounds__(GM_T) k_gm_dots(const double2 *__restrict__ V, int64_t ns, int nr, int J,
                                                  const double2 *__restrict__ w, double2 *__restrict__ part) {
    const int cta = blockIdx.x, q = blockIdx.y, nct = gridDim.x;
    const int64_t rb = (int64_t)cta * GM_ROWS;
    double2 wl[4];
    for (int k = 0; k < 4; k++) {
        const int64_t r = rb + threadIdx.x + k * GM_T;
        wl[k] = r < ns ? w[q * ns + r] : make_double2(0.0, 0.0);
    }
    __shared__ double2 red[8][GM_T / 32];
    for (int i0 = 0; i0 < J; i0 += 8) {
        double2 s[8];
#pragma unroll
        for (int t = 0; t < 8; t++) {
            s[t] = make_double2(0.0, 0.0);
            if (i0 + t < J) {
                const double2 *vi = V + ((int64_t)(i0 + t) * nr + q) * ns;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int64_t r = rb + threadIdx.x + k * GM_T;
                    if (r < ns) s[t] = cadd(s[t], cconjmul(vi[r], wl[k]));
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s[t].x += __shfl_down_sync(0xffffffffu, s[t].x, o);
                s[t].y += __shfl_down_sync(0xffffffffu, s[t].y, o);
            }
            if ((threadIdx.x & 31) == 0) red[t][threadIdx.x >> 5] = s[t];
        }
        __syncthreads();
        if (threadIdx.x < 8 && i0 + (int)threadIdx.x < J) {
            double2 tt = red[threadIdx.x][0];
            for (int k = 1; k < GM_T / 32; k++) tt = cadd(tt, red[threadIdx.x][k]);
            part[((int64_t)q * J + i0 + threadIdx.x) * nct + cta] = tt;
        }
        __syncthreads();
    }
}

// h[q * J + i] = sum over CTAs of the partial dot products (fixed order)
__global__ void k_gm_dots_final(const double2 *__restrict__ part, int nct, int J, double2 *__restrict__ h) {
    const int i = blockIdx.x, q = blockIdx.y;
    const double2 *p = part + ((int64_t)q * J + i) * nct;
    double2 s = make_double2(0.0, 0.0);
    for (int c = threadIdx.x; c < nct; c += 32) s = cadd(s, p[c]);
    for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_down_sync(0xffffffffu, s.x, o);
        s.y += __shfl_down_sync(0xffffffffu, s.y, o);
    }
    if (threadIdx.x == 0) h[(int64_t)q * J + i] = s;
}

// w[r, q] -= sum_i V_i[r, q] h[q * J + i]; with norm partials != NULL also ||w||^2 per CTA after the update
__global__ void __launch_bounds__(GM_T) k_gm_orth(const double2 *__restrict__ V, int64_t ns, int nr, int J,
                                                  const double2 *__restrict__ h, double2 *__restrict__ w,
                                                  double *__restrict__ npart) {
    const int cta = blockIdx.x, q = blockIdx.y, nct = gridDim.x;
    const int64_t rb = (int64_t)cta * GM_ROWS;
    __shared__ double2 hs[GM_MAX_RESTART + 1];
    for (int i = threadIdx.x; i < J; i += GM_T) hs[i] = h[(int64_t)q * J + i];
    __syncthreads();
    double nn = 0.0;
    for (int k = 0; k < 4; k++) {
        const int64_t r = rb + threadIdx.x + k * GM_T;
        if (r >= ns) break;
        double2 x = w[q * ns + r];
        for (int i = 0; i < J; i++) cfms(x, V[((int64_t)i * nr + q) * ns + r], hs[i]);
        w[q * ns + r] = x;
        nn += x.x * x.x + x.y * x.y;
    }
    if (!npart) return;
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_down_sync(0xffffffffu, nn, o);
    __shared__ double red[GM_T / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = red[0];
        for (int k = 1; k < GM_T / 32; k++) t += red[k];
        npart[(int64_t)q * nct + cta] = t;
    }
}

__global__ void k_gm_norm_final(const double *__restrict__ npart, int nct, double *__restrict__ out) {
    const int q = blockIdx.x;
    double s = 0.0;
    for (int c = threadIdx.x; c < nct; c += 32) s += npart[(int64_t)q * nct + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[q] = s;
}

struct Scales {
    double s[GM_MAX_RHS];
};

// dst[r, q] = src[r, q] * s[q]
__global__ void k_gm_scale(const double2 *__restrict__ src, double2 *__restrict__ dst, int64_t ns, int nr, Scales sc) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ns * nr) return;
    dst[e] = cscale(src[e], sc.s[e / ns]);
}

// x[r, q] += sum_i Z_i[r, q] y[q * J + i]
__global__ void k_gm_xupdate(const double2 *__restrict__ Z, int64_t ns, int nr, int J, const double2 *__restrict__ y,
                             double2 *__restrict__ x) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ns * nr) return;
    const int64_t q = e / ns, r = e % ns;
    double2 s = x[e];
    for (int i = 0; i < J; i++) cfma(s, Z[((int64_t)i * nr + q) * ns + r], y[q * J + i]);
    x[e] = s;
}

struct HostPinned {
    void *p = nullptr;
    ~HostPinned() {
        if (p) cudaFreeHost(p);
    }
};

struct DevBuf {
    char *p = nullptr;
    cudaStream_t st = nullptr;
    ~DevBuf() {
        if (p) cudaFreeAsync(p, st);
    }
};

}  // namespace

extern "C" gdm_status gdm_lattice_partition(const double *pos, int64_t n, double step, int block_cells,
                                            int32_t *perm, int32_t *parent, int32_t *coarse_offsets,
                                            int64_t *n_coarse) {
    if (!pos || !perm || !parent || !coarse_offsets || !n_coarse) return GDM_ERR_INVALID_ARG;
    if (n < 1 || n > (int64_t)1 << 26 || !(step > 0) || !isfinite(step) || block_cells < 1) return GDM_ERR_INVALID_ARG;
    GDM_GUARD_BEGIN
    std::vector<double> hp(pos, pos + 3 * n);
    for (double x : hp)
        if (!isfinite(x)) return GDM_ERR_INVALID_ARG;
    Partition part;
    make_partition(hp, n, step, block_cells, part);
    std::copy(part.perm.begin(), part.perm.end(), perm);
    std::copy(part.parent.begin(), part.parent.end(), parent);
    std::copy(part.coff.begin(), part.coff.end(), coarse_offsets);
    *n_coarse = (int64_t)part.coff.size() - 1;
    return GDM_OK;
    GDM_GUARD_END(nullptr)
}

static gdm_status solve_gmres(gdm_ctx *ctx, gdm_precision prec, const gdm_problem *p, const double *F0, double *F,
                              int n_rhs, const gdm_gmres_opts *opts, gdm_solve_info *info) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    if (!p || !F0 || !F) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (p->kind != 3) return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "gdm_solve_gmres: discretised structures (kind 3)");
    if (!p->pos || !p->eps) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (p->n < 1 || !(p->step > 0) || !isfinite(p->step) || !(p->wavelength > 0) || !isfinite(p->wavelength) ||
        !(p->eps_env > 0) || !isfinite(p->eps_env))
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "need n >= 1, step > 0, wavelength > 0, eps_env > 0");
    if (p->n > (int64_t)1 << 26) return gdm_fail(ctx, GDM_ERR_SHAPE, "gdm_solve_gmres: at most 2^26 cells");
    if (prec != GDM_TF32_REFINE && prec != GDM_FP32)
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "gdm_solve_gmres: the preconditioner factors in TF32 or FP32");
    if (n_rhs < 1 || n_rhs > GM_MAX_RHS)
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "gdm_solve_gmres: n_rhs must be in [1, %d]", GM_MAX_RHS);
    gdm_gmres_opts o = {0, 0, 0.0, 0, 0};
    if (opts) o = *opts;
    const int m = o.restart > 0 ? o.restart : 60;
    const int max_it = o.max_iter > 0 ? o.max_iter : 1000;
    const double tol = o.tol > 0 ? o.tol : 1e-12;
    const int bc = o.block_cells > 0 ? o.block_cells : 512;
    const bool use_blocks = !(o.flags & GDM_GMRES_NO_BLOCKS);
    bool use_coarse = !(o.flags & GDM_GMRES_NO_COARSE);
    if (m > GM_MAX_RESTART || bc > GM_MAX_BLOCK_CELLS)
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "gdm_solve_gmres: restart <= %d and block_cells <= %d",
                        GM_MAX_RESTART, GM_MAX_BLOCK_CELLS);
    if (info) memset(info, 0, sizeof(*info));
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    gdm_params_reset(ctx);
    const int64_t n = p->n, ns = 3 * n;
    const int nr = n_rhs;

    // ---- partition of the lattice (host, once)
    Partition part;
    {
        std::vector<double> hp(3 * n);
        GDM_CUDA_TRY(ctx, cudaMemcpyAsync(hp.data(), p->pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost,
                                          ctx->stream));
        GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        for (double x : hp)
            if (!isfinite(x)) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "non-finite cell position");
        make_partition(hp, n, p->step, bc, part);
    }
    const int64_t nc = (int64_t)part.coff.size() - 1, nc3 = 3 * nc;
    const int nb = (int)part.boff.size() - 1;
    // a structure inside one block: the block part is the LU of the whole system, which the additive
    // coarse term would only perturb
    if (use_blocks && nb == 1) use_coarse = false;
    const int64_t lda_c = (nc3 + 31) / 32 * 32;
    std::vector<int64_t> fac_off(nb);
    std::vector<int> fac_ld(nb);
    int64_t fac_total = 0;
    int max_m = 0;
    for (int b = 0; b < nb; b++) {
        const int mb = 3 * (part.boff[b + 1] - part.boff[b]);
        fac_ld[b] = (mb + 31) / 32 * 32;
        fac_off[b] = fac_total;
        fac_total += ((int64_t)mb * fac_ld[b] + 31) / 32 * 32;
        max_m = std::max(max_m, mb);
    }
    const int nct = (int)((ns + GM_ROWS - 1) / GM_ROWS);
    const size_t vec = (size_t)ns * nr;

    // ---- device buffers (one allocation, carved twice: sizing, then for real)
    int *d_perm, *d_parent, *d_coff, *d_boff, *d_fld, *tsync;
    int64_t *d_foff;
    int32_t *piv, *piv_c;
    double *pos_p, *pos_c, *nrm, *npart, *bnorm2;
    double2 *eps_p, *eps_c, *chi_c, *bp, *x, *zero, *w, *V, *Z, *Pbuf, *gpart, *dpart, *h1, *h2, *ybuf;
    float2 *fac, *Ac, *rc, *yc;
    void *ffws, *dinv;
    const size_t pbytes = gdm_green_partial_bytes(ctx, n, n, 3);
    auto carve = [&](char *base) {
        ScratchCarver sc(base);
        d_perm = sc.take<int>(n);
        d_parent = sc.take<int>(n);
        d_coff = sc.take<int>(nc + 1);
        d_boff = sc.take<int>(nb + 1);
        d_fld = sc.take<int>(nb);
        d_foff = sc.take<int64_t>(nb);
        piv = sc.take<int32_t>(ns);
        pos_p = sc.take<double>(3 * n);
        eps_p = sc.take<double2>(n);
        pos_c = sc.take<double>(3 * nc);
        eps_c = sc.take<double2>(nc);
        chi_c = sc.take<double2>(nc);
        fac = use_blocks ? sc.take<float2>(fac_total) : nullptr;
        Ac = use_coarse ? sc.take<float2>((size_t)nc3 * lda_c) : nullptr;
        piv_c = sc.take<int32_t>(nc3);
        tsync = sc.take<int>(gdm_trsv_sync_bytes(nc3) / sizeof(int) + 1);
        dinv = sc.take<char>(gdm_trsv_inv_bytes(nc3));
        rc = sc.take<float2>((size_t)nc3 * nr);
        yc = sc.take<float2>((size_t)nc3 * nr);
        bp = sc.take<double2>(vec);
        x = sc.take<double2>(vec);
        zero = sc.take<double2>(vec);
        w = sc.take<double2>(vec);
        V = sc.take<double2>(vec * (m + 1));
        Z = sc.take<double2>(vec * m);
        Pbuf = sc.take<double2>(vec);
        gpart = sc.take<double2>(pbytes / sizeof(double2));
        ffws = sc.take<char>(gdm_ff_scratch_bytes(n));
        dpart = sc.take<double2>((size_t)nct * (m + 1) * nr);
        h1 = sc.take<double2>((size_t)(m + 1) * nr);
        h2 = sc.take<double2>((size_t)(m + 1) * nr);
        ybuf = sc.take<double2>((size_t)(m + 1) * nr);
        npart = sc.take<double>((size_t)nct * nr);
        nrm = sc.take<double>(nr);
        bnorm2 = sc.take<double>(nr);
        return sc.off + 256;
    };
    DevBuf buf;
    buf.st = ctx->stream;
    GDM_CUDA_TRY(ctx, cudaMallocAsync((void **)&buf.p, carve(nullptr), ctx->stream));
    carve(buf.p);
    HostPinned hpin;
    const size_t hbytes = sizeof(double2) * 2 * (m + 1) * nr + sizeof(double) * 2 * nr + 256;
    GDM_CUDA_TRY(ctx, cudaMallocHost(&hpin.p, hbytes));
    double2 *hh1 = (double2 *)hpin.p, *hh2 = hh1 + (m + 1) * nr;
    double *hnrm = (double *)(hh2 + (m + 1) * nr), *hb2 = hnrm + nr;

    if (info) GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
    // ---- permuted problem, coarse model, factorisations
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(d_perm, part.perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(d_parent, part.parent.data(), sizeof(int) * n, cudaMemcpyHostToDevice,
                                      ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(d_coff, part.coff.data(), sizeof(int) * (nc + 1), cudaMemcpyHostToDevice,
                                      ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(d_boff, part.boff.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice,
                                      ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(d_fld, fac_ld.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(d_foff, fac_off.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice,
                                      ctx->stream));
    // the host vectors above must outlive the copies
    GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    k_gather_cells<<<nblk(n), GM_T, 0, ctx->stream>>>(p->pos, (const double2 *)p->eps, d_perm, n, pos_p, eps_p);
    GDM_LAUNCHED(ctx, "gather_cells");
    k_coarse_cells<<<nblk(nc), GM_T, 0, ctx->stream>>>(pos_p, eps_p, d_coff, nc, p->eps_env, pos_c, eps_c, chi_c);
    GDM_LAUNCHED(ctx, "coarse_cells");
    gdm_problem pp = *p;
    pp.pos = pos_p;
    pp.eps = (const double *)eps_p;
    double growth_max = 0.0;
    int refactored = 0;
    // The coarse model and the blocks are independent factorisations of latency-bound size: they run
    // concurrently on the context's pool of child contexts (item 0 = the coarse model when used, then the
    // blocks, largest first), each child on its own stream and scratch.
    auto assemble_on = [&](gdm_ctx *c, const gdm_problem *q, float2 *A, int64_t ld, bool coarse) -> gdm_status {
        GDM_TRY(gdm_launch_assemble(c, q, prec, A, ld));
        if (coarse) {
            k_coarse_diag<<<nblk(nc3), GM_T, 0, c->stream>>>(A, ld, chi_c, nc, 1.0 / (3.0 * p->eps_env));
            GDM_LAUNCHED(c, "gmres_coarse_diag");
        }
        return GDM_OK;
    };
    auto factor_on = [&](gdm_ctx *c, const gdm_problem *q, float2 *A, int64_t mq, int64_t ld, int32_t *ipq,
                         bool coarse, gdm_solve_info *inf) -> gdm_status {
        float growth = 1.f;
        GDM_TRY(assemble_on(c, q, A, ld, coarse));
        GDM_TRY(gdm_lu_factor(c, prec, A, mq, ld, ipq, 0, &growth));
        if (!(growth <= (float)GDM_PIVOT_GROWTH_LIMIT)) {
            GDM_TRY(assemble_on(c, q, A, ld, coarse));
            GDM_TRY(gdm_lu_factor(c, prec, A, mq, ld, ipq, 1, &growth));
            inf->refactored = 1;
        }
        inf->pivot_growth = growth;
        return gdm_ctx_check(c);
    };
    gdm_problem pc = *p;
    pc.n = nc;
    pc.pos = pos_c;
    pc.eps = (const double *)eps_c;
    pc.step = 2.0 * p->step;
    const int c0i = use_coarse ? 1 : 0;
    const int n_items = c0i + (use_blocks ? nb : 0);
    if (n_items > 0) {
        std::vector<int64_t> isize(n_items);
        if (use_coarse) isize[0] = nc3;
        for (int i = c0i; i < n_items; i++) isize[i] = 3 * (int64_t)(part.boff[i - c0i + 1] - part.boff[i - c0i]);
        std::vector<gdm_solve_info> iinfo(n_items);
        GDM_TRY(gdm_run_pool(
            ctx, n_items, isize.data(), 8, iinfo.data(),
            [&](gdm_ctx *c, int, int i, gdm_solve_info *inf) -> gdm_status {
                gdm_params_reset(c);
                if (i < c0i) return factor_on(c, &pc, Ac, nc3, lda_c, piv_c, true, inf);
                const int b = i - c0i;
                gdm_problem pb = pp;
                pb.n = part.boff[b + 1] - part.boff[b];
                pb.pos = pos_p + 3 * (int64_t)part.boff[b];
                pb.eps = (const double *)(eps_p + part.boff[b]);
                return factor_on(c, &pb, fac + fac_off[b], 3 * pb.n, fac_ld[b], piv + 3 * (int64_t)part.boff[b],
                                 false, inf);
            },
            nullptr));
        for (const gdm_solve_info &x : iinfo) {
            growth_max = std::max(growth_max, x.pivot_growth);
            refactored += x.refactored;
        }
    }
    int coarse_local = 0;
    if (use_coarse) {
        GDM_TRY(gdm_pivots_local(ctx, piv_c, nc3, 32, tsync, &coarse_local));
        if (coarse_local) GDM_TRY(gdm_trsv_prepare(ctx, prec, Ac, nc3, lda_c, piv_c, dinv, 0));
    }
    if (use_blocks) {
        const int smem = (int)(sizeof(float2) * (size_t)max_m * nr);
        GDM_TRY(launch_bj_nr(ctx, nr, nb, smem, fac, d_foff, d_fld, piv, d_boff, nullptr, ns, d_parent, rc, yc, nc3,
                             0, nullptr, true));
    }
    float setup_ms = 0.f;
    if (info) {
        GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
        GDM_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev1));
        GDM_CUDA_TRY(ctx, cudaEventElapsedTime(&setup_ms, ctx->ev0, ctx->ev1));
    }

    // phase accounting (gdm_profile_phases): preconditioner as correction solves, operator as residual
    auto precond = [&](const double2 *v, double2 *z) -> gdm_status {
        GDM_TRY(gdm_phase_begin(ctx, GDM_PH_TRSV));
        if (use_coarse) {
            k_restrict<<<nblk(nc3 * nr), GM_T, 0, ctx->stream>>>(v, ns, nr, d_coff, nc, rc, yc);
            GDM_LAUNCHED(ctx, "gmres_restrict");
            if (coarse_local)
                GDM_TRY(gdm_trsv_persistent(ctx, prec, Ac, nc3, lda_c, piv_c, yc, nc3, nr, 0, tsync, dinv));
            else
                GDM_TRY(gdm_lu_solve(ctx, prec, Ac, nc3, lda_c, piv_c, yc, nc3, nr, 0));
        }
        if (use_blocks) {
            const int smem = (int)(sizeof(float2) * (size_t)max_m * nr);
            GDM_TRY(launch_bj_nr(ctx, nr, nb, smem, fac, d_foff, d_fld, piv, d_boff, v, ns, d_parent, rc, yc, nc3,
                                 use_coarse ? 1 : 0, z, false));
        } else if (use_coarse) {
            k_coarse_only<<<nblk(vec), GM_T, 0, ctx->stream>>>(v, ns, nr, d_parent, rc, yc, nc3, z);
            GDM_LAUNCHED(ctx, "gmres_coarse_only");
        } else {
            GDM_CUDA_TRY(ctx, cudaMemcpyAsync(z, v, sizeof(double2) * vec, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        return gdm_phase_end(ctx, GDM_PH_TRSV);
    };
    // r = rhs - A X (double-float Green sums); norms2 (device, nr) optional
    bool ff_ready = false;
    auto residual = [&](const double2 *rhs, const double2 *X, double2 *r, double *norms2) -> gdm_status {
        GDM_TRY(gdm_phase_begin(ctx, GDM_PH_RESIDUAL));
        GDM_TRY(gdm_launch_residual_ws(ctx, &pp, (const double *)rhs, (const double *)X, nr, 0, (double *)r, norms2,
                                       Pbuf, gpart, ffws, ff_ready ? 0 : 1));
        ff_ready = true;
        return gdm_phase_end(ctx, GDM_PH_RESIDUAL);
    };
    // the same with the FP32 operator (positions prepared by the first double-float call)
    auto residual_fast = [&](const double2 *rhs, const double2 *X, double2 *r) -> gdm_status {
        GDM_TRY(gdm_phase_begin(ctx, GDM_PH_OPERATOR_F32));
        GDM_TRY(gdm_launch_residual_f32(ctx, &pp, (const double *)rhs, (const double *)X, nr, (double *)r, nullptr,
                                        Pbuf, gpart, gdm_ff_positions(ffws)));
        return gdm_phase_end(ctx, GDM_PH_OPERATOR_F32);
    };
    bool fast = !(o.flags & GDM_GMRES_EXACT_OPERATOR);
    double prev_rel = INFINITY;

    // ---- FGMRES(m)
    if (info) GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
    k_permute_rows<<<nblk(vec), GM_T, 0, ctx->stream>>>((const double2 *)F0, bp, d_perm, n, nr, 0);
    GDM_LAUNCHED(ctx, "gmres_permute");
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(x, 0, sizeof(double2) * vec, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(zero, 0, sizeof(double2) * vec, ctx->stream));
    typedef std::complex<double> cd;
    std::vector<cd> H((size_t)nr * (m + 1) * m), g((size_t)nr * (m + 1)), cs((size_t)nr * m), sn((size_t)nr * m);
    std::vector<double> bn(nr, 0.0);
    std::vector<int> len(nr);
    int total = 0, cycles = 0;
    double rel_true = INFINITY, rel_est = INFINITY;
    bool converged = false;
    while (true) {
        // true residual of the current iterate (the first iterate is 0: its residual is F0 itself)
        if (total == 0) {
            GDM_CUDA_TRY(ctx, cudaMemcpyAsync(w, bp, sizeof(double2) * vec, cudaMemcpyDeviceToDevice, ctx->stream));
            k_gm_orth<<<dim3((unsigned)nct, (unsigned)nr), GM_T, 0, ctx->stream>>>(V, ns, nr, 0, h1, w, npart);
            GDM_LAUNCHED(ctx, "gmres_orth");
            k_gm_norm_final<<<nr, 32, 0, ctx->stream>>>(npart, nct, bnorm2);
            GDM_LAUNCHED(ctx, "gmres_norm_final");
            if (!ff_ready) GDM_TRY(gdm_ff_prepare(ctx, &pp, ffws));
            ff_ready = true;
        } else {
            GDM_CUDA_TRY(ctx, cudaMemsetAsync(bnorm2, 0, sizeof(double) * nr, ctx->stream));
            GDM_TRY(residual(bp, x, w, bnorm2));
        }
        GDM_CUDA_TRY(ctx, cudaMemcpyAsync(hb2, bnorm2, sizeof(double) * nr, cudaMemcpyDeviceToHost, ctx->stream));
        GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        std::vector<double> beta(nr);
        rel_true = 0.0;
        bool finite = true;
        for (int q = 0; q < nr; q++) {
            beta[q] = sqrt(hb2[q]);
            if (!isfinite(beta[q])) finite = false;
            if (total == 0) bn[q] = beta[q];  // x = 0: the residual is F0
            const double rq = bn[q] > 0 ? beta[q] / bn[q] : 0.0;
            rel_true = std::max(rel_true, rq);
        }
        if (!finite) {
            if (info) info->status = GDM_ERR_NONFINITE;
            return gdm_fail(ctx, GDM_ERR_NONFINITE, "gdm_solve_gmres: non-finite residual");
        }
        if (rel_true <= tol) {
            converged = true;
            break;
        }
        if (total >= max_it) break;
        // a cycle on the FP32 operator must at least halve the true residual
        if (fast && !(rel_true <= 0.5 * prev_rel)) fast = false;
        prev_rel = rel_true;
        Scales sc;
        for (int q = 0; q < GM_MAX_RHS; q++) sc.s[q] = (q < nr && beta[q] > 0) ? 1.0 / beta[q] : 0.0;
        k_gm_scale<<<nblk(vec), GM_T, 0, ctx->stream>>>(w, V, ns, nr, sc);
        GDM_LAUNCHED(ctx, "gmres_scale");
        std::fill(H.begin(), H.end(), cd(0.0));
        std::fill(g.begin(), g.end(), cd(0.0));
        std::vector<bool> active(nr);
        std::vector<double> target(nr);
        for (int q = 0; q < nr; q++) {
            g[(size_t)q * (m + 1)] = beta[q];
            active[q] = bn[q] > 0 && beta[q] / bn[q] > tol;
            len[q] = 0;
            target[q] = fast ? std::max(tol * bn[q], GM_INNER * beta[q]) : tol * bn[q];
        }
        int j = 0;
        cycles++;
        for (; j < m && total < max_it; j++) {
            double2 *Vj = V + vec * j, *Zj = Z + vec * j;
            GDM_TRY(precond(Vj, Zj));
            if (fast) GDM_TRY(residual_fast(zero, Zj, w));  // w = -A z_j
            else GDM_TRY(residual(zero, Zj, w, nullptr));
            const int J = j + 1;
            const dim3 gr((unsigned)nct, (unsigned)nr);
            GDM_TRY(gdm_phase_begin(ctx, GDM_PH_OTHER));
            k_gm_dots<<<gr, GM_T, 0, ctx->stream>>>(V, ns, nr, J, w, dpart);
            GDM_LAUNCHED(ctx, "gmres_dots");
            k_gm_dots_final<<<dim3((unsigned)J, (unsigned)nr), 32, 0, ctx->stream>>>(dpart, nct, J, h1);
            GDM_LAUNCHED(ctx, "gmres_dots_final");
            k_gm_orth<<<gr, GM_T, 0, ctx->stream>>>(V, ns, nr, J, h1, w, nullptr);
            GDM_LAUNCHED(ctx, "gmres_orth");
            k_gm_dots<<<gr, GM_T, 0, ctx->stream>>>(V, ns, nr, J, w, dpart);
            GDM_LAUNCHED(ctx, "gmres_dots");
            k_gm_dots_final<<<dim3((unsigned)J, (unsigned)nr), 32, 0, ctx->stream>>>(dpart, nct, J, h2);
            GDM_LAUNCHED(ctx, "gmres_dots_final");
            k_gm_orth<<<gr, GM_T, 0, ctx->stream>>>(V, ns, nr, J, h2, w, npart);
            GDM_LAUNCHED(ctx, "gmres_orth");
            k_gm_norm_final<<<nr, 32, 0, ctx->stream>>>(npart, nct, nrm);
            GDM_LAUNCHED(ctx, "gmres_norm_final");
            GDM_TRY(gdm_phase_end(ctx, GDM_PH_OTHER));
            GDM_CUDA_TRY(ctx, cudaMemcpyAsync(hh1, h1, sizeof(double2) * J * nr, cudaMemcpyDeviceToHost, ctx->stream));
            GDM_CUDA_TRY(ctx, cudaMemcpyAsync(hh2, h2, sizeof(double2) * J * nr, cudaMemcpyDeviceToHost, ctx->stream));
            GDM_CUDA_TRY(ctx, cudaMemcpyAsync(hnrm, nrm, sizeof(double) * nr, cudaMemcpyDeviceToHost, ctx->stream));
            GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            total++;
            rel_est = 0.0;
            bool any = false;
            for (int q = 0; q < nr; q++) {
                const double hn = sqrt(hnrm[q]);
                // w holds -A z_j: the Arnoldi coefficients are the negated projections
                sc.s[q] = (active[q] && hn > 0) ? -1.0 / hn : 0.0;
                if (!active[q]) continue;
                cd *Hq = H.data() + (size_t)q * (m + 1) * m;
                cd *gq = g.data() + (size_t)q * (m + 1);
                cd *cq = cs.data() + (size_t)q * m, *sq = sn.data() + (size_t)q * m;
                for (int i = 0; i < J; i++) {
                    const double2 a = hh1[q * J + i], b = hh2[q * J + i];
                    Hq[(size_t)i * m + j] = -cd(a.x + b.x, a.y + b.y);
                }
                Hq[(size_t)(j + 1) * m + j] = hn;
                for (int i = 0; i < j; i++) {
                    const cd t = std::conj(cq[i]) * Hq[(size_t)i * m + j] + std::conj(sq[i]) * Hq[(size_t)(i + 1) * m + j];
                    Hq[(size_t)(i + 1) * m + j] = -sq[i] * Hq[(size_t)i * m + j] + cq[i] * Hq[(size_t)(i + 1) * m + j];
                    Hq[(size_t)i * m + j] = t;
                }
                const cd a = Hq[(size_t)j * m + j];
                const double den = sqrt(std::norm(a) + hn * hn);
                if (!(den > 0) || !isfinite(den)) {
                    active[q] = false;
                    len[q] = j;
                    continue;
                }
                cq[j] = a / den;
                sq[j] = hn / den;
                Hq[(size_t)j * m + j] = den;
                Hq[(size_t)(j + 1) * m + j] = 0.0;
                gq[j + 1] = -sq[j] * gq[j];
                gq[j] = std::conj(cq[j]) * gq[j];
                len[q] = j + 1;
                const double est = std::abs(gq[j + 1]) / bn[q];
                rel_est = std::max(rel_est, est);
                if (std::abs(gq[j + 1]) <= target[q] || !(hn > 1e-300 * den)) active[q] = false;
                else any = true;
            }
            if (!any) {
                j++;
                break;
            }
            k_gm_scale<<<nblk(vec), GM_T, 0, ctx->stream>>>(w, V + vec * (j + 1), ns, nr, sc);
            GDM_LAUNCHED(ctx, "gmres_scale");
        }
        // x += Z y, y from the triangular systems H y = g
        const int J = j;
        std::vector<double2> hy((size_t)nr * J, make_double2(0.0, 0.0));
        for (int q = 0; q < nr; q++) {
            const int L = len[q];
            const cd *Hq = H.data() + (size_t)q * (m + 1) * m;
            const cd *gq = g.data() + (size_t)q * (m + 1);
            std::vector<cd> y(L);
            for (int i = L - 1; i >= 0; i--) {
                cd s = gq[i];
                for (int k = i + 1; k < L; k++) s -= Hq[(size_t)i * m + k] * y[k];
                y[i] = s / Hq[(size_t)i * m + i];
            }
            for (int i = 0; i < L; i++) hy[(size_t)q * J + i] = make_double2(y[i].real(), y[i].imag());
        }
        if (J > 0) {
            GDM_CUDA_TRY(ctx, cudaMemcpyAsync(ybuf, hy.data(), sizeof(double2) * nr * J, cudaMemcpyHostToDevice,
                                              ctx->stream));
            k_gm_xupdate<<<nblk(vec), GM_T, 0, ctx->stream>>>(Z, ns, nr, J, ybuf, x);
            GDM_LAUNCHED(ctx, "gmres_xupdate");
            // hy must outlive the copy
            GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        }
        if (J == 0) break;
    }
    k_permute_rows<<<nblk(vec), GM_T, 0, ctx->stream>>>(x, (double2 *)F, d_perm, n, nr, 1);
    GDM_LAUNCHED(ctx, "gmres_permute");
    gdm_status dev = gdm_ctx_check(ctx);
    if (info) {
        float it_ms = 0.f;
        GDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev2, ctx->stream));
        GDM_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev2));
        GDM_CUDA_TRY(ctx, cudaEventElapsedTime(&it_ms, ctx->ev1, ctx->ev2));
        info->iterations = total;
        info->status = dev != GDM_OK ? dev : (converged ? GDM_OK : GDM_ERR_NOT_CONVERGED);
        info->rel_correction = rel_est;
        info->rel_residual = rel_true;
        info->factor_ms = setup_ms;
        info->refine_ms = it_ms;
        info->pivot_growth = growth_max;
        info->refactored = refactored;
        info->cycles = cycles;
    }
    if (dev != GDM_OK) return dev;
    if (!converged)
        return gdm_fail(ctx, GDM_ERR_NOT_CONVERGED, "gdm_solve_gmres: relative residual %.3e > tol %.3e after %d steps",
                        rel_true, tol, total);
    return GDM_OK;
}

extern "C" gdm_status gdm_solve_gmres(gdm_ctx *ctx, gdm_precision prec, const gdm_problem *p, const double *F0,
                                      double *F, int n_rhs, const gdm_gmres_opts *opts, gdm_solve_info *info) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    GDM_GUARD_BEGIN
    return solve_gmres(ctx, prec, p, F0, F, n_rhs, opts, info);
    GDM_GUARD_END(ctx)
}
