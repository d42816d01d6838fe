// Matrix-free refinement residual in double-float arithmetic (cells, kind 3; ED/MD dipoles, kind 6).
//
// The residual r = F0 - A F of the FP64 refinement needs the Green dyad G^Ep of every pair to ~1e-13
// relative. GB300 runs FP64 at ~1/64 of its FP32 rate, so this kernel regenerates G in double-float
// (FP32 pairs, ~48 significant bits: Knuth two-sum, FMA two-product) on the FP32 pipes:
//   * r_i - r_j from FP32 (hi, lo) position pairs; R, 1/R, R-hat in double-float;
//   * phase k R reduced modulo 2 pi with a three-part split of 2 pi;
//   * e^{i theta}: table of cos/sin at multiples of pi/128 (double-float entries computed on the host in
//     double precision) times cos/sin of the remainder |delta| <= pi/256 from its Taylor series
//     (cos: 1 - d^2/2 + d^4/24 - d^6/720, sin: d - d^3/6 + d^5/120; the neglected terms are < 1e-15);
//   * G s = a s + b u (u.s), accumulated in double-float, written as FP64 partial sums for the FP64 finalize;
//     for ED/MD dipoles the 6x6 dyad in its vacuum form at the host k acts on (p, n_env m):
//     (T p - C n_env m, C p + T n_env m) with T = eps_env G^Ep, C s = c (u x s), c = e^{ikR} (k^2/R + i k/R^2);
//     the residual's finalize scales the rows by (1/eps_env, 1/n_env).
#include <math.h>

#include "gdm_internal.cuh"

namespace {

struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff mk(float h, float l) { return {h, l}; }
__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ ff neg(ff x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ ff sub(ff x, ff y) { return add(x, neg(y)); }
__device__ __forceinline__ ff mul(ff x, ff y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ff mulf(ff x, float y) {
    float p = __fmul_rn(x.hi, y);
    float e = fmaf(x.hi, y, -p);
    e = fmaf(x.lo, y, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ff sqr(ff x) {
    float p = __fmul_rn(x.hi, x.hi);
    float e = fmaf(x.hi, x.hi, -p);
    e = fmaf(2.0f * x.hi, x.lo, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ffsqrt(ff x) {
    float r = sqrtf(x.hi);
    float p = __fmul_rn(r, r);
    float e = fmaf(r, r, -p);
    float res = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), e), x.lo);
    return fast_two_sum(r, __fdiv_rn(res, 2.0f * r));
}
__device__ __forceinline__ ff recip(ff x) {
    float r = __fdiv_rn(1.0f, x.hi);
    // d = 1 - x r (in double-float), y = r + r d
    float p = __fmul_rn(x.hi, r);
    float ep = fmaf(x.hi, r, -p);
    ep = fmaf(x.lo, r, ep);
    float d = __fsub_rn(__fsub_rn(1.0f, p), ep);
    return fast_two_sum(r, __fmul_rn(r, d));
}
struct cff {
    ff re, im;
};
__device__ __forceinline__ cff cmulff(cff a, cff b) {
    return {sub(mul(a.re, b.re), mul(a.im, b.im)), add(mul(a.re, b.im), mul(a.im, b.re))};
}
__device__ __forceinline__ cff caddff(cff a, cff b) { return {add(a.re, b.re), add(a.im, b.im)}; }
__device__ __forceinline__ cff cscaleff(cff a, ff s) { return {mul(a.re, s), mul(a.im, s)}; }

#define TWO_PI_C1 6.283203125f
#define TWO_PI_C2 (-1.7814338207244873e-05f)
#define TWO_PI_C3 (-3.4822063010864213e-09f)
#define INV_TWO_PI_F 0.15915494309189535f
// pi/128 = P1 + P2 + P3, P1 and P2 with 16 significant bits (i * P1, i * P2 exact for |i| <= 128)
#define PI128_P1 0.02454376220703125f
#define PI128_P2 (-6.95999915478751e-08f)
#define PI128_P3 (-8.694424303776205e-13f)
#define INV_PI128_F 40.7436637878418f

// e^{i x} for a double-float phase x >= 0; tab[i + 128] = (cos_hi, cos_lo, sin_hi, sin_lo) at i pi/128
__device__ __forceinline__ cff expi_ff(ff x, const float4 *tab) {
    float n = rintf(x.hi * INV_TWO_PI_F);
    float t1 = fmaf(-n, TWO_PI_C1, x.hi);
    ff s = two_sum(t1, -n * TWO_PI_C2);
    ff th = fast_two_sum(s.hi, fmaf(-n, TWO_PI_C3, __fadd_rn(s.lo, x.lo)));
    float fi = rintf(th.hi * INV_PI128_F);
    fi = fminf(fmaxf(fi, -128.f), 128.f);
    float u1 = fmaf(-fi, PI128_P1, th.hi);
    ff s2 = two_sum(u1, -fi * PI128_P2);
    ff d = fast_two_sum(s2.hi, fmaf(-fi, PI128_P3, __fadd_rn(s2.lo, th.lo)));
    ff d2 = sqr(d);
    float d2f = d2.hi;
    // cos d = 1 - d^2/2 + (d^4/24 - d^6/720);  sin d = d - d^3/6 + d^5/120
    ff cd = sub(mk(1.0f, 0.0f), mulf(d2, 0.5f));
    cd = add(cd, mk(d2f * d2f * (1.0f / 24.0f - d2f * (1.0f / 720.0f)), 0.0f));
    ff d3 = mul(d2, d);
    ff sd = sub(d, mul(d3, mk(0.16666667163372040f, -4.967053879312289e-09f)));  // 1/6 in double-float
    sd = add(sd, mk(d3.hi * d2f * (1.0f / 120.0f), 0.0f));
    float4 t = tab[(int)fi + 128];
    ff c0 = mk(t.x, t.y), s0 = mk(t.z, t.w);
    return {sub(mul(c0, cd), mul(s0, sd)), add(mul(s0, cd), mul(c0, sd))};
}

struct DipF {
    float xh, yh, zh, xl, yl, zl;
    float2 alpha;
    float2 diag;
    float pad[2];
};

#define RF_T 128
#define RF_S 32

// Source records, one per source, laid out so that a tile of RF_S consecutive sources is one contiguous
// block that a single bulk copy moves into shared memory: 8 floats (x, y, z hi; x, y, z lo; 2 pad), then
// the moments of the NR right-hand sides of this launch as double-float complex numbers, float4
// (re_hi, re_lo, im_hi, im_lo) per component, [KIND][NR].
template <int KIND, int NR> struct SrcRecLayout {
    static constexpr int FLOATS = 8 + 4 * KIND * NR;
    static constexpr int BYTES = 4 * FLOATS;  // a multiple of 16
};

template <int KIND, int NR>
__global__ void k_prep_src(const DipF *__restrict__ dip, int64_t n, const double2 *__restrict__ P, int rhs0,
                           int nr_here, float *__restrict__ rec, int conj = 0) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    float *o = rec + j * SrcRecLayout<KIND, NR>::FLOATS;
    const DipF d = dip[j];
    o[0] = d.xh;
    o[1] = d.yh;
    o[2] = d.zh;
    o[3] = d.xl;
    o[4] = d.yl;
    o[5] = d.zl;
    o[6] = 0.f;
    o[7] = 0.f;
    const int64_t ld = KIND * n;
    float4 *m = (float4 *)(o + 8);
#pragma unroll
    for (int a = 0; a < KIND; a++)
#pragma unroll
        for (int q = 0; q < NR; q++) {
            double2 v = make_double2(0.0, 0.0);
            if (q < nr_here) v = P[(rhs0 + q) * ld + KIND * j + a];
            if (conj) v.y = -v.y;
            const float rh = (float)v.x, ih = (float)v.y;
            m[a * NR + q] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
        }
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait (~2 s) for the phase of the given parity
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = gtimer_ns();
    for (;;) {
        if (mbar_test(bar, parity)) return true;
        if (gtimer_ns() - t0 > 2000000000ull) return false;
    }
}
// one bulk copy global -> shared completing on an mbarrier (addresses 16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// partial[c][q][t][OUT] (FP64) = sum over the sources j of chunk c (j != t when self_exclude) of the dyad of
// (r_t - r_j) times the moments of source j: OUT = 3: G^Ep s (cells' residual); OUT = 6 with KIND = 3:
// (G^Ep p, G^Hp-form cross term c (u x p)) (cells' near field); OUT = 6 with KIND = 6: the 6x6 vacuum-form
// dyad on (p, n_env m) (ED/MD residual and near field). Targets and sources are FP32 (hi, lo) position
// pairs. Source tiles (RF_S records) are double-buffered in shared memory by bulk copies issued one tile
// ahead by one thread; every wait on them is bounded (on timeout the device error record gets
// GDM_ERR_TIMEOUT and the CTA stops summing).
// (the body takes the target block bx and the chunk c explicitly, so that the grouped sums of a batch run it
// for any problem)
template <int KIND, int OUT, int NR>
__device__ __forceinline__ void green_sum_ff_body(const DipF *__restrict__ tgt, int64_t m,
                                                  const float *__restrict__ rec, int64_t n, float khi, float klo,
                                                  float k2hi, float k2lo, float ie_hi, float ie_lo,
                                                  const float4 *__restrict__ gtab, int64_t chunk, int self_exclude,
                                                  double2 *__restrict__ partial, int *flags, int64_t bx, int64_t c) {
    using L = SrcRecLayout<KIND, NR>;
    __shared__ float4 tab[257];
    __shared__ __align__(16) float sbuf[2][RF_S * L::FLOATS];
    __shared__ uint64_t bar[2];
    __shared__ int abort_cta;
    for (int e = threadIdx.x; e < 257; e += RF_T) tab[e] = gtab[e];
    const int64_t t = bx * RF_T + threadIdx.x;
    const bool valid = t < m;
    const int64_t jb = c * chunk, je = min(n, jb + chunk);
    const int ntile = je > jb ? (int)((je - jb + RF_S - 1) / RF_S) : 0;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_cta = 0;
    }
    __syncthreads();
    auto tile_src = [&](int it, uint32_t *bytes) {
        const int64_t s0 = jb + (int64_t)it * RF_S;
        *bytes = (uint32_t)(min((int64_t)RF_S, je - s0) * L::BYTES);
        return rec + s0 * L::FLOATS;
    };
    if (threadIdx.x == 0 && ntile > 0) {
        uint32_t by;
        const float *src = tile_src(0, &by);
        bulk_load(sbuf[0], src, by, &bar[0]);
    }
    const DipF ti = valid ? tgt[t] : tgt[0];
    const ff kf = mk(khi, klo), k2 = mk(k2hi, k2lo), ie = mk(ie_hi, ie_lo);
    cff acc[NR][OUT];
#pragma unroll
    for (int q = 0; q < NR; q++)
#pragma unroll
        for (int a = 0; a < OUT; a++) acc[q][a] = {mk(0, 0), mk(0, 0)};
    int it = 0;
    for (; it < ntile; it++) {
        const int b = it & 1;
        // the other buffer was read in the previous iteration, which every thread has left (barrier below)
        if (threadIdx.x == 0 && it + 1 < ntile) {
            uint32_t by;
            const float *src = tile_src(it + 1, &by);
            bulk_load(sbuf[b ^ 1], src, by, &bar[b ^ 1]);
        }
        const int64_t s0 = jb + (int64_t)it * RF_S;
        const int sn = (int)min((int64_t)RF_S, je - s0);
        const bool landed = mbar_wait_bounded(&bar[b], (uint32_t)((it >> 1) & 1));
        if (!landed) {
            abort_cta = 1;
            gdm_dev_error(flags, GDM_ERR_TIMEOUT, 3);
        }
        if (valid && landed) {
            const float *tb = sbuf[b];
            for (int jj = 0; jj < sn; jj++) {
                if (self_exclude && s0 + jj == t) continue;
                const float *sr = tb + jj * L::FLOATS;
                ff dx = add(two_sum(ti.xh, -sr[0]), mk(__fsub_rn(ti.xl, sr[3]), 0.f));
                ff dy = add(two_sum(ti.yh, -sr[1]), mk(__fsub_rn(ti.yl, sr[4]), 0.f));
                ff dz = add(two_sum(ti.zh, -sr[2]), mk(__fsub_rn(ti.zl, sr[5]), 0.f));
                ff r2 = add(add(sqr(dx), sqr(dy)), sqr(dz));
                ff r = ffsqrt(r2);
                ff r1 = recip(r);
                ff ri2 = sqr(r1);
                ff ri3 = mul(ri2, r1);
                ff u[3] = {mul(dx, r1), mul(dy, r1), mul(dz, r1)};
                cff e = expi_ff(mul(kf, r), tab);
                e = cscaleff(e, ie);
                ff k2r1 = mul(k2, r1);
                ff kri2 = mul(kf, ri2);
                // a = e (k^2/R - 1/R^3 + i k/R^2),  b = e (3/R^3 - k^2/R - 3 i k/R^2)
                cff ca = {sub(k2r1, ri3), kri2};
                cff cb = {sub(mulf(ri3, 3.0f), k2r1), neg(mulf(kri2, 3.0f))};
                cff a = cmulff(e, ca), bb = cmulff(e, cb);
                // electric-magnetic coupling: c = e (k^2/R + i k/R^2)
                cff cc = {mk(0, 0), mk(0, 0)};
                if (OUT == 6) cc = cmulff(e, cff{k2r1, kri2});
                const float4 *mom = (const float4 *)(sr + 8);
#pragma unroll
                for (int q = 0; q < NR; q++) {
#pragma unroll
                    for (int h = 0; h < KIND / 3; h++) {  // h = 0: electric moment, h = 1: magnetic moment
                        cff sv[3];
#pragma unroll
                        for (int aa = 0; aa < 3; aa++) {
                            const float4 v = mom[(3 * h + aa) * NR + q];
                            sv[aa] = {mk(v.x, v.y), mk(v.z, v.w)};
                        }
                        cff us = {add(add(mul(u[0], sv[0].re), mul(u[1], sv[1].re)), mul(u[2], sv[2].re)),
                                  add(add(mul(u[0], sv[0].im), mul(u[1], sv[1].im)), mul(u[2], sv[2].im))};
                        cff bus = cmulff(bb, us);
#pragma unroll
                        for (int aa = 0; aa < 3; aa++) {
                            cff v = caddff(cmulff(a, sv[aa]), cscaleff(bus, u[aa]));
                            acc[q][3 * h + aa] = caddff(acc[q][3 * h + aa], v);
                        }
                        if (OUT == 6) {
                            // u x s, added as +c (u x p) to the magnetic rows (h = 0) or -c (u x m) to the electric
                            // rows (h = 1)
                            cff x[3];
                            x[0] = {sub(mul(u[1], sv[2].re), mul(u[2], sv[1].re)),
                                    sub(mul(u[1], sv[2].im), mul(u[2], sv[1].im))};
                            x[1] = {sub(mul(u[2], sv[0].re), mul(u[0], sv[2].re)),
                                    sub(mul(u[2], sv[0].im), mul(u[0], sv[2].im))};
                            x[2] = {sub(mul(u[0], sv[1].re), mul(u[1], sv[0].re)),
                                    sub(mul(u[0], sv[1].im), mul(u[1], sv[0].im))};
#pragma unroll
                            for (int aa = 0; aa < 3; aa++) {
                                cff v = cmulff(cc, x[aa]);
                                if (h == 0) acc[q][3 + aa] = caddff(acc[q][3 + aa], v);
                                else acc[q][aa] = caddff(acc[q][aa], cff{neg(v.re), neg(v.im)});
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (abort_cta) break;
    }
    if (abort_cta && threadIdx.x == 0 && it + 1 < ntile) {
        // the copy issued for the next tile must land before the CTA's shared memory goes away
        mbar_wait_bounded(&bar[(it + 1) & 1], (uint32_t)(((it + 1) >> 1) & 1));
    }
    if (!valid) return;
#pragma unroll
    for (int q = 0; q < NR; q++) {
        double2 *o = partial + ((c * 2 + q) * m + t) * OUT;
#pragma unroll
        for (int a = 0; a < OUT; a++)
            o[a] = make_double2((double)acc[q][a].re.hi + (double)acc[q][a].re.lo,
                                (double)acc[q][a].im.hi + (double)acc[q][a].im.lo);
    }
}
template <int KIND, int OUT, int NR>
__global__ void __launch_bounds__(RF_T) k_green_sum_ff(const DipF *__restrict__ tgt, int64_t m,
                                                      const float *__restrict__ rec, int64_t n, float khi, float klo,
                                                      float k2hi, float k2lo, float ie_hi, float ie_lo,
                                                      const float4 *__restrict__ gtab, int64_t chunk, int self_exclude,
                                                      double2 *__restrict__ partial, int *flags) {
    green_sum_ff_body<KIND, OUT, NR>(tgt, m, rec, n, khi, klo, k2hi, k2lo, ie_hi, ie_lo, gtab, chunk, self_exclude,
                                     partial, flags, blockIdx.x, blockIdx.y);
}

// Gradient pair sums of the adjoint (cells), double-float on the FP32 pipes: partial[c][q][t][15] (FP64) =
// sum over the sources j != t of chunk c of, for s = the source's vector (one right-hand side per launch):
//   [0..2]   G s,   [3 + 3c + a]  (dG/dR_c s)_a,   [12..14]  dG/dk s,
// with G = a I + b u u^T, a = e (k^2/R - 1/R^3 + i k/R^2), b = e (3/R^3 - k^2/R - 3 i k/R^2), e = exp(ikR)/eps_env:
//   d/dR_c (G s)_a = u_c [a' s_a + b' u_a (u.s)] + (b/R) [delta_ca (u.s) + u_a s_c - 2 u_c u_a (u.s)],
//   a' = da/dR = i k a + e (-k^2/R^2 + 3/R^4 - 2 i k/R^3),  b' = i k b + e (k^2/R^2 - 9/R^4 + 6 i k/R^3),
//   d/dk (G s) = (i R a + e (2k/R + i/R^2)) s + (i R b + e (-2k/R - 3i/R^2)) u (u.s).
// The same sums as the FP64 kernel of the adjoint (to ~1e-13 relative instead of FP64's 1e-16), at about six
// times its rate on GB300, whose FP64 pipe runs at ~1/64 of FP32. Source tiles as in k_green_sum_ff.
#define DGF_OUT 15
__global__ void __launch_bounds__(RF_T) k_dgreen_sum_ff(const DipF *__restrict__ tgt, int64_t m,
                                                       const float *__restrict__ rec, int64_t n, float khi, float klo,
                                                       float k2hi, float k2lo, float ie_hi, float ie_lo,
                                                       const float4 *__restrict__ gtab, int64_t chunk,
                                                       int self_exclude, int qslot, double2 *__restrict__ partial,
                                                       int *flags) {
    using L = SrcRecLayout<3, 1>;
    __shared__ float4 tab[257];
    __shared__ __align__(16) float sbuf[2][RF_S * L::FLOATS];
    __shared__ uint64_t bar[2];
    __shared__ int abort_cta;
    for (int e = threadIdx.x; e < 257; e += RF_T) tab[e] = gtab[e];
    const int64_t t = (int64_t)blockIdx.x * RF_T + threadIdx.x;
    const bool valid = t < m;
    const int64_t c = blockIdx.y;
    const int64_t jb = c * chunk, je = min(n, jb + chunk);
    const int ntile = je > jb ? (int)((je - jb + RF_S - 1) / RF_S) : 0;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_cta = 0;
    }
    __syncthreads();
    auto tile_src = [&](int it, uint32_t *bytes) {
        const int64_t s0 = jb + (int64_t)it * RF_S;
        *bytes = (uint32_t)(min((int64_t)RF_S, je - s0) * L::BYTES);
        return rec + s0 * L::FLOATS;
    };
    if (threadIdx.x == 0 && ntile > 0) {
        uint32_t by;
        const float *src = tile_src(0, &by);
        bulk_load(sbuf[0], src, by, &bar[0]);
    }
    const DipF ti = valid ? tgt[t] : tgt[0];
    const ff kf = mk(khi, klo), k2 = mk(k2hi, k2lo), ie = mk(ie_hi, ie_lo);
    cff acc[DGF_OUT];
#pragma unroll
    for (int a = 0; a < DGF_OUT; a++) acc[a] = {mk(0, 0), mk(0, 0)};
    int it = 0;
    for (; it < ntile; it++) {
        const int b = it & 1;
        if (threadIdx.x == 0 && it + 1 < ntile) {
            uint32_t by;
            const float *src = tile_src(it + 1, &by);
            bulk_load(sbuf[b ^ 1], src, by, &bar[b ^ 1]);
        }
        const int64_t s0 = jb + (int64_t)it * RF_S;
        const int sn = (int)min((int64_t)RF_S, je - s0);
        const bool landed = mbar_wait_bounded(&bar[b], (uint32_t)((it >> 1) & 1));
        if (!landed) {
            abort_cta = 1;
            gdm_dev_error(flags, GDM_ERR_TIMEOUT, 5);
        }
        if (valid && landed) {
            const float *tb = sbuf[b];
            for (int jj = 0; jj < sn; jj++) {
                if (self_exclude && s0 + jj == t) continue;
                const float *sr = tb + jj * L::FLOATS;
                ff dx = add(two_sum(ti.xh, -sr[0]), mk(__fsub_rn(ti.xl, sr[3]), 0.f));
                ff dy = add(two_sum(ti.yh, -sr[1]), mk(__fsub_rn(ti.yl, sr[4]), 0.f));
                ff dz = add(two_sum(ti.zh, -sr[2]), mk(__fsub_rn(ti.zl, sr[5]), 0.f));
                const ff r = ffsqrt(add(add(sqr(dx), sqr(dy)), sqr(dz)));
                const ff r1 = recip(r);
                const ff ri2 = sqr(r1);
                const ff ri3 = mul(ri2, r1);
                const ff ri4 = sqr(ri2);
                const ff u[3] = {mul(dx, r1), mul(dy, r1), mul(dz, r1)};
                const cff e = cscaleff(expi_ff(mul(kf, r), tab), ie);
                const ff k2r1 = mul(k2, r1), kri2 = mul(kf, ri2), k2ri2 = mul(k2, ri2), kri3 = mul(kf, ri3);
                const ff kr1 = mul(kf, r1);
                const cff a = cmulff(e, cff{sub(k2r1, ri3), kri2});
                const cff bb = cmulff(e, cff{sub(mulf(ri3, 3.0f), k2r1), neg(mulf(kri2, 3.0f))});
                // i k x = (-k x.im, k x.re);  i R x = (-R x.im, R x.re)
                const cff da = caddff(cff{neg(mul(kf, a.im)), mul(kf, a.re)},
                                      cmulff(e, cff{add(neg(k2ri2), mulf(ri4, 3.0f)), neg(mulf(kri3, 2.0f))}));
                const cff db = caddff(cff{neg(mul(kf, bb.im)), mul(kf, bb.re)},
                                      cmulff(e, cff{sub(k2ri2, mulf(ri4, 9.0f)), mulf(kri3, 6.0f)}));
                const cff dka = caddff(cff{neg(mul(r, a.im)), mul(r, a.re)}, cmulff(e, cff{mulf(kr1, 2.0f), ri2}));
                const cff dkb = caddff(cff{neg(mul(r, bb.im)), mul(r, bb.re)},
                                       cmulff(e, cff{neg(mulf(kr1, 2.0f)), neg(mulf(ri2, 3.0f))}));
                const float4 *mom = (const float4 *)(sr + 8);
                cff sv[3];
#pragma unroll
                for (int aa = 0; aa < 3; aa++) {
                    const float4 v = mom[aa];
                    sv[aa] = {mk(v.x, v.y), mk(v.z, v.w)};
                }
                const cff us = {add(add(mul(u[0], sv[0].re), mul(u[1], sv[1].re)), mul(u[2], sv[2].re)),
                                add(add(mul(u[0], sv[0].im), mul(u[1], sv[1].im)), mul(u[2], sv[2].im))};
                const cff bus = cmulff(bb, us), dbus = cmulff(db, us), dkbus = cmulff(dkb, us);
                const cff bor = cscaleff(bb, r1);
#pragma unroll
                for (int aa = 0; aa < 3; aa++) {
                    acc[aa] = caddff(acc[aa], caddff(cmulff(a, sv[aa]), cscaleff(bus, u[aa])));
                    acc[12 + aa] = caddff(acc[12 + aa], caddff(cmulff(dka, sv[aa]), cscaleff(dkbus, u[aa])));
                }
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
#pragma unroll
                    for (int aa = 0; aa < 3; aa++) {
                        const cff t1 = caddff(cmulff(da, sv[aa]), cscaleff(dbus, u[aa]));
                        // delta_ca (u.s) + u_a s_c - 2 u_c u_a (u.s)
                        ff w = neg(mulf(mul(u[cc], u[aa]), 2.0f));
                        if (cc == aa) w = add(w, mk(1.0f, 0.0f));
                        const cff t2 = caddff(cscaleff(sv[cc], u[aa]), cscaleff(us, w));
                        acc[3 + 3 * cc + aa] = caddff(acc[3 + 3 * cc + aa], caddff(cscaleff(t1, u[cc]), cmulff(bor, t2)));
                    }
                }
            }
        }
        __syncthreads();
        if (abort_cta) break;
    }
    if (abort_cta && threadIdx.x == 0 && it + 1 < ntile) {
        mbar_wait_bounded(&bar[(it + 1) & 1], (uint32_t)(((it + 1) >> 1) & 1));
    }
    if (!valid) return;
    double2 *o = partial + ((c * 2 + qslot) * m + t) * DGF_OUT;  // chunk stride of two right-hand sides
#pragma unroll
    for (int a = 0; a < DGF_OUT; a++)
        o[a] = make_double2((double)acc[a].re.hi + (double)acc[a].re.lo, (double)acc[a].im.hi + (double)acc[a].im.lo);
}

__global__ void k_prep_dipf_pos(const double *__restrict__ pos, int64_t n, DipF *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    DipF d;
    double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    d.xh = (float)x;
    d.yh = (float)y;
    d.zh = (float)z;
    d.xl = (float)(x - (double)d.xh);
    d.yl = (float)(y - (double)d.yh);
    d.zl = (float)(z - (double)d.zh);
    d.alpha = make_float2(0.f, 0.f);
    d.diag = make_float2(0.f, 0.f);
    d.pad[0] = d.pad[1] = 0.f;
    out[i] = d;
}

void split(double v, float *h, float *l) {
    *h = (float)v;
    *l = (float)(v - (double)*h);
}

}  // namespace

// workspace: the sources' FP32-pair positions (DipF records, first, so that other kernels can use them),
// the (cos, sin) table of the phase reduction, and the source records of one launch (up to KIND 6, NR 2)
size_t gdm_ff_scratch_bytes(int64_t n) {
    return ScratchCarver::round(n * sizeof(DipF)) + ScratchCarver::round(257 * 16) +
           ScratchCarver::round((size_t)n * SrcRecLayout<6, 2>::BYTES) + 512;
}

// the hi/lo FP32 position pairs (48-byte records) that gdm_launch_green_sum_ff prepares at the start of its
// workspace; valid after a call with prepare = 1 on the same problem
const void *gdm_ff_positions(void *ffws) {
    ScratchCarver sc(ffws);
    return sc.take<DipF>(0);
}

// fill the workspace for the problem: FP32-pair positions and the (cos, sin) table of the phase reduction
gdm_status gdm_ff_prepare(gdm_ctx *ctx, const gdm_problem *p, void *ffws) {
    const int64_t n = p->n;
    ScratchCarver sc(ffws);
    DipF *dip = sc.take<DipF>(n);
    float4 *tab = sc.take<float4>(257);
    k_prep_dipf_pos<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(p->pos, n, dip);
    GDM_LAUNCHED(ctx, "prep_dipf_pos");
    float4 h[257];
    for (int i = -128; i <= 128; i++) {
        double a = i * (3.14159265358979323846 / 128.0);
        float ch, cl, sh, sl;
        split(cos(a), &ch, &cl);
        split(sin(a), &sh, &sl);
        h[i + 128] = make_float4(ch, cl, sh, sl);
    }
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(tab, h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));  // h is a stack array
    return GDM_OK;
}

namespace {
template <int KIND, int OUT, int NR>
gdm_status launch_ff(gdm_ctx *ctx, const DipF *tgt, int64_t m, const DipF *dip, int64_t n, const double2 *P, int rhs0,
                     int nr, float *rec, const float *kk, const float4 *tab, int64_t chunk, int nchunks,
                     int self_exclude, double2 *partial) {
    k_prep_src<KIND, NR><<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(dip, n, P, rhs0, nr, rec);
    GDM_LAUNCHED(ctx, "prep_src");
    dim3 grid((unsigned)((m + RF_T - 1) / RF_T), (unsigned)nchunks);
    k_green_sum_ff<KIND, OUT, NR><<<grid, RF_T, 0, ctx->stream>>>(tgt, m, rec, n, kk[0], kk[1], kk[2], kk[3], kk[4],
                                                                   kk[5], tab, chunk, self_exclude, partial,
                                                                   ctx->dflags);
    GDM_LAUNCHED(ctx, "green_sum_ff");
    return GDM_OK;
}
}  // namespace

// Double-float Green sums from the problem's dipoles (moments P: (KIND n) x n_rhs, right-hand sides
// rhs0 .. rhs0 + nr - 1, nr <= 2) to m targets. tgt = NULL: the targets are the dipoles themselves, each
// without its own term (the residual); otherwise FP32-pair target positions (gdm_ff_targets). out = KIND for
// the residual, 6 for near fields. partial[c][q][t][out] as the FP64 Green sum writes it.
gdm_status gdm_ff_green_sum(gdm_ctx *ctx, const gdm_problem *p, const void *tgt, int64_t m, int out,
                            const double2 *P, int rhs0, int nr, int64_t chunk, int nchunks, void *ffws,
                            double2 *partial, int prepare) {
    const int64_t n = p->n;
    ScratchCarver sc(ffws);
    DipF *dip = sc.take<DipF>(n);
    float4 *tab = sc.take<float4>(257);
    float *rec = (float *)sc.take<char>((size_t)n * SrcRecLayout<6, 2>::BYTES);
    if (prepare) GDM_TRY(gdm_ff_prepare(ctx, p, ffws));
    const double k = sqrt(p->eps_env) * gdm_k0(p);
    float kk[6];
    split(k, &kk[0], &kk[1]);
    split(k * k, &kk[2], &kk[3]);
    // the E kernel of cells carries 1/eps_env; ED/MD sums run the vacuum-form kernel (rows scaled afterwards)
    split(p->kind == 6 ? 1.0 : 1.0 / p->eps_env, &kk[4], &kk[5]);
    const DipF *t = tgt ? (const DipF *)tgt : dip;
    const int self = tgt ? 0 : 1;
    if (!tgt) m = n;
    if (p->kind == 6) {
        if (nr == 1) return launch_ff<6, 6, 1>(ctx, t, m, dip, n, P, rhs0, nr, rec, kk, tab, chunk, nchunks, self, partial);
        return launch_ff<6, 6, 2>(ctx, t, m, dip, n, P, rhs0, nr, rec, kk, tab, chunk, nchunks, self, partial);
    }
    if (out == 6) {
        if (nr == 1) return launch_ff<3, 6, 1>(ctx, t, m, dip, n, P, rhs0, nr, rec, kk, tab, chunk, nchunks, self, partial);
        return launch_ff<3, 6, 2>(ctx, t, m, dip, n, P, rhs0, nr, rec, kk, tab, chunk, nchunks, self, partial);
    }
    if (nr == 1) return launch_ff<3, 3, 1>(ctx, t, m, dip, n, P, rhs0, nr, rec, kk, tab, chunk, nchunks, self, partial);
    return launch_ff<3, 3, 2>(ctx, t, m, dip, n, P, rhs0, nr, rec, kk, tab, chunk, nchunks, self, partial);
}

// resident CTAs per SM of the double-float kernel for (kind, out, nr) (cached; 4 if the query fails)
namespace {
template <int KIND, int OUT, int NR> int ff_occ() {
    static int cached = 0;
    if (!cached) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_green_sum_ff<KIND, OUT, NR>, RF_T, 0) != cudaSuccess ||
            b < 1) {
            cudaGetLastError();
            b = 4;
        }
        cached = b > 8 ? 8 : b;
    }
    return cached;
}
}  // namespace

int gdm_ff_occupancy(int kind, int out, int nr) {
    if (kind == 6) return nr == 1 ? ff_occ<6, 6, 1>() : ff_occ<6, 6, 2>();
    if (out == 6) return nr == 1 ? ff_occ<3, 6, 1>() : ff_occ<3, 6, 2>();
    return nr == 1 ? ff_occ<3, 3, 1>() : ff_occ<3, 3, 2>();
}

// Same output as the FP64 Green sum used by the residual (partial sums per chunk, two RHS per launch).
gdm_status gdm_launch_green_sum_ff(gdm_ctx *ctx, const gdm_problem *p, const double2 *P, int rhs0, int nr,
                                   int64_t chunk, int nchunks, void *ffws, double2 *partial, int prepare) {
    return gdm_ff_green_sum(ctx, p, nullptr, p->n, p->kind, P, rhs0, nr, chunk, nchunks, ffws, partial, prepare);
}

// FP32-pair positions of m evaluation points (48-byte records into out, m of them)
gdm_status gdm_ff_targets(gdm_ctx *ctx, const double *r, int64_t m, void *out) {
    k_prep_dipf_pos<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(r, m, (DipF *)out);
    GDM_LAUNCHED(ctx, "prep_dipf_pos");
    return GDM_OK;
}

size_t gdm_ff_target_bytes(int64_t m) { return (size_t)m * sizeof(DipF); }

// occupancy (resident CTAs per SM) of the gradient pair kernel, cached
int gdm_ff_dgreen_occupancy() {
    static int cached = 0;
    if (!cached) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dgreen_sum_ff, RF_T, 0) != cudaSuccess || b < 1) {
            cudaGetLastError();
            b = 2;
        }
        cached = b > 8 ? 8 : b;
    }
    return cached;
}

// Gradient pair sums of the adjoint for the problem's cells, one right-hand side (column q of S, 3 n entries
// per column, conjugated when conj): sources and targets are the cells (each without its own term); output
// as the FP64 kernel's partial sums for slot qslot of a right-hand-side pair (partial[c][qslot][t][15]). The
// workspace must have been prepared (gdm_ff_prepare) for the problem.
gdm_status gdm_ff_dgreen_sum(gdm_ctx *ctx, const gdm_problem *p, const double2 *S, int q, int conj, int qslot,
                             int64_t chunk, int nchunks, void *ffws, double2 *partial) {
    const int64_t n = p->n;
    ScratchCarver sc(ffws);
    DipF *dip = sc.take<DipF>(n);
    float4 *tab = sc.take<float4>(257);
    float *rec = (float *)sc.take<char>((size_t)n * SrcRecLayout<6, 2>::BYTES);
    k_prep_src<3, 1><<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(dip, n, S, q, 1, rec, conj);
    GDM_LAUNCHED(ctx, "prep_src");
    const double k = sqrt(p->eps_env) * gdm_k0(p);
    float kk[6];
    split(k, &kk[0], &kk[1]);
    split(k * k, &kk[2], &kk[3]);
    split(1.0 / p->eps_env, &kk[4], &kk[5]);
    dim3 grid((unsigned)((n + RF_T - 1) / RF_T), (unsigned)nchunks);
    k_dgreen_sum_ff<<<grid, RF_T, 0, ctx->stream>>>(dip, n, rec, n, kk[0], kk[1], kk[2], kk[3], kk[4], kk[5], tab, chunk,
                                                    1, qslot, partial, ctx->dflags);
    GDM_LAUNCHED(ctx, "dgreen_sum_ff");
    return GDM_OK;
}

// ---------------------------------------------------------------- grouped sums of a batch's refinement
namespace {
// FP32-pair positions of every listed problem: ceil(n / 256) CTAs of 256 per problem
__global__ void __launch_bounds__(256) k_gr_prep_dip(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                     const int *__restrict__ prefix, int na) {
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const int64_t j = (int64_t)local * 256 + threadIdx.x;
    if (j >= items[i].n) return;
    const double *pos = items[i].pos;
    DipF d;
    const double x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2];
    d.xh = (float)x;
    d.yh = (float)y;
    d.zh = (float)z;
    d.xl = (float)(x - (double)d.xh);
    d.yl = (float)(y - (double)d.yh);
    d.zl = (float)(z - (double)d.zh);
    d.alpha = make_float2(0.f, 0.f);
    d.diag = make_float2(0.f, 0.f);
    d.pad[0] = d.pad[1] = 0.f;
    ((DipF *)items[i].dip)[j] = d;
}

// source records (positions and the moments P of both right-hand sides as double-float pairs):
// ceil(n / 256) CTAs of 256 per problem
__global__ void __launch_bounds__(256) k_gr_prep_src(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                     const int *__restrict__ prefix, int na) {
    using L = SrcRecLayout<3, 2>;
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const GrItem &g = items[i];
    const int64_t j = (int64_t)local * 256 + threadIdx.x;
    if (j >= g.n) return;
    float *o = g.rec + j * L::FLOATS;
    const DipF d = ((const DipF *)g.dip)[j];
    o[0] = d.xh;
    o[1] = d.yh;
    o[2] = d.zh;
    o[3] = d.xl;
    o[4] = d.yl;
    o[5] = d.zl;
    o[6] = 0.f;
    o[7] = 0.f;
    const int64_t ld = 3 * g.n;
    float4 *m = (float4 *)(o + 8);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int q = 0; q < 2; q++) {
            double2 v = make_double2(0.0, 0.0);
            if (q < g.nr) v = g.P[q * ld + 3 * j + a];
            const float rh = (float)v.x, ih = (float)v.y;
            m[a * 2 + q] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
        }
}

// the residual's double-float sums, every pair (t, j != t) of each listed problem: ceil(n / RF_T) target
// blocks x nc chunks per problem
__global__ void __launch_bounds__(RF_T) k_gr_green_ff(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                      const int *__restrict__ prefix, int na,
                                                      const float4 *__restrict__ tab, int *flags) {
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const GrItem &g = items[i];
    const int64_t tb = (g.n + RF_T - 1) / RF_T;
    green_sum_ff_body<3, 3, 2>((const DipF *)g.dip, g.n, g.rec, g.n, g.kk[0], g.kk[1], g.kk[2], g.kk[3], g.kk[4],
                               g.kk[5], tab, g.chunk, 1, g.partial, flags, local % tb, local / tb);
}
}  // namespace

gdm_status gdm_gr_prep_dip(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units) {
    if (units <= 0) return GDM_OK;
    k_gr_prep_dip<<<(unsigned)units, 256, 0, ctx->stream>>>(it, list, prefix, na);
    GDM_LAUNCHED(ctx, "gr_prep_dip");
    return GDM_OK;
}

gdm_status gdm_gr_prep_src(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units) {
    if (units <= 0) return GDM_OK;
    k_gr_prep_src<<<(unsigned)units, 256, 0, ctx->stream>>>(it, list, prefix, na);
    GDM_LAUNCHED(ctx, "gr_prep_src");
    return GDM_OK;
}

gdm_status gdm_gr_green_ff(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units,
                           const void *tab) {
    if (units <= 0) return GDM_OK;
    k_gr_green_ff<<<(unsigned)units, RF_T, 0, ctx->stream>>>(it, list, prefix, na, (const float4 *)tab, ctx->dflags);
    GDM_LAUNCHED(ctx, "gr_green_ff");
    return GDM_OK;
}

gdm_status gdm_ff_table_fill(gdm_ctx *ctx, void *dev_tab) {
    static float4 h[257];
    static bool made = false;
    if (!made) {
        for (int i = -128; i <= 128; i++) {
            const double a = i * (3.14159265358979323846 / 128.0);
            float ch, cl, sh, sl;
            split(cos(a), &ch, &cl);
            split(sin(a), &sh, &sl);
            h[i + 128] = make_float4(ch, cl, sh, sl);
        }
        made = true;
    }
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(dev_tab, h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
    return GDM_OK;
}
