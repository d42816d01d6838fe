// Green-dyad kernels of the GDM hot path:
//   * plane-wave illumination,
//   * pair-tiled assembly of A = I - G alpha (complex64 with a double-float phase, or complex128),
//   * FP64 matrix-free Green sums: refinement residual F0 - A F (and the adjoint A^H form), near field,
//   * FP64 cross-section reductions.
//
// Physics (Gaussian units, exp(-i w t)), following the paper's Eq. (superprop_G) blocks:
//   G^Ep(R) = e^{ikR}/eps_env [ (k^2/R + ik/R^2 - 1/R^3) I + (-k^2/R - 3ik/R^2 + 3/R^3) u u^T ]
//   G^Hp(R) = k0 k e^{ikR} (1/R + i/(k R^2)) [u]_x          ([u]_x v = u x v)
//   ED/MD dyad in a non-magnetic host: G^Em = -G^Hp, G^Hm = eps_env G^Ep (vacuum: G^Hm = G^Ep).
// ED/MD sums run the dyad in its vacuum form at the host wavenumber k (kernel T = eps_env G^Ep,
// cross term C = e^{ikR}(k^2/R + ik/R^2) [u]_x = n_env G^Hp) on the moments (p, n_env m) and scale the
// rows afterwards: E = (T p - C n_env m)/eps_env, H = (C p + T n_env m)/n_env.
// Cells (kind 3): alpha = (eps - eps_env) d^3/(4 pi), self-term S = -4 pi/(3 eps_env d^3) I
// (Sec. "Volume discretization polarizabilities", Eq. selfterm_SEp_cubic).
#include <math.h>

#include <mutex>

#include "gdm_internal.cuh"

#define PI_D 3.14159265358979323846

// ================================================================== double-float (FP32 pair) arithmetic
// Error-free transformations (Knuth two-sum, FMA two-product) give ~48-bit precision on the FP32
// pipes, which on GB300 run ~64x faster than FP64. Used for the phase k R of the assembled matrix.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_sqr(ff x) {
    float p = __fmul_rn(x.hi, x.hi);
    float e = fmaf(x.hi, x.hi, -p);
    e = fmaf(2.0f * x.hi, x.lo, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_sqrt(ff x) {
    float r = sqrtf(x.hi);
    float p = __fmul_rn(r, r);
    float e = fmaf(r, r, -p);
    float res = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), e), x.lo);
    return fast_two_sum(r, __fdiv_rn(res, 2.0f * r));
}
// x - y for two FP32-pair coordinates
__device__ __forceinline__ ff ff_diff(float xh, float xl, float yh, float yl) {
    ff s = two_sum(xh, -yh);
    float e = __fadd_rn(s.lo, __fsub_rn(xl, yl));
    return fast_two_sum(s.hi, e);
}

// 2 pi = C1 + C2 + C3: C1 and C2 carry 12 significant bits each (so n*C1, n*C2 are exact FP32
// products for |n| < 4096), C3 is the FP32-rounded remainder. Split of the number 2 pi computed
// with 50-digit arithmetic (Cody-Waite style argument reduction).
#define TWO_PI_C1 6.283203125f
#define TWO_PI_C2 (-1.7814338207244873e-05f)
#define TWO_PI_C3 (-3.4822063010864213e-09f)
#define INV_TWO_PI_F 0.15915494309189535f

// e^{i x} for a double-float phase x >= 0 (|x| < 2.5e4): reduce to [-pi, pi] keeping the low part,
// then FP32 sincos of the high part with a first-order correction for the low part. FAST: the hardware
// sine/cosine approximations for the reduced argument (absolute error about 4e-7 on [-pi, pi]), for the
// iterative solver's low-precision operator only.
template <bool FAST = false>
__device__ __forceinline__ float2 ff_expi(ff x) {
    float n = rintf(x.hi * INV_TWO_PI_F);
    float t1 = fmaf(-n, TWO_PI_C1, x.hi);  // exact
    ff s = two_sum(t1, -n * TWO_PI_C2);    // -n*C2 exact
    float lo = fmaf(-n, TWO_PI_C3, __fadd_rn(s.lo, x.lo));
    ff th = fast_two_sum(s.hi, lo);
    float sn, cs;
    if (FAST) __sincosf(th.hi, &sn, &cs);
    else sincosf(th.hi, &sn, &cs);
    return make_float2(fmaf(-sn, th.lo, cs), fmaf(cs, th.lo, sn));
}

// ================================================================== plane wave
__global__ void k_planewave(const double *__restrict__ r, int64_t m, double k, double n_env, const double *__restrict__ e0,
                            double kx, double ky, double kz, int n_rhs, int kind_out, double2 *__restrict__ F0) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    double ph = k * (kx * r[3 * i] + ky * r[3 * i + 1] + kz * r[3 * i + 2]);
    double s, c;
    sincos(ph, &s, &c);
    double2 e = make_double2(c, s);
    int64_t ld = (int64_t)kind_out * m;
    for (int q = 0; q < n_rhs; q++) {
        double2 E[3];
        for (int a = 0; a < 3; a++) E[a] = cmul(make_double2(e0[6 * q + 2 * a], e0[6 * q + 2 * a + 1]), e);
        double2 *out = F0 + q * ld + (int64_t)kind_out * i;
        for (int a = 0; a < 3; a++) out[a] = E[a];
        if (kind_out == 6) {
            // H0 = n_env khat x E0
            out[3] = cscale(csub(cscale(E[2], ky), cscale(E[1], kz)), n_env);
            out[4] = cscale(csub(cscale(E[0], kz), cscale(E[2], kx)), n_env);
            out[5] = cscale(csub(cscale(E[1], kx), cscale(E[0], ky)), n_env);
        }
    }
}

// Paraxial Gaussian beam at points (one thread per point and illumination): beam frame x' = (cos t, 0, -sin t),
// y' = y, z' = (sin t, 0, cos t) about the focus; z0 = k w0^2/2, g = 1 + i z'/z0,
// u = exp(i k z') exp(-(x'^2 + y'^2)/(w0^2 g)) / g; E_t = e0 u, E_z' = (i/k) (-2/(w0^2 g)) (x' e0x + y' e0y) u;
// H_t = n z' x E_t and H_z' from the same divergence condition.
__global__ void k_gaussian(const double *__restrict__ r, int64_t m, double k, double n_env, double w0, double fx,
                           double fy, double fz, double ct, double st, const double *__restrict__ e0, int n_rhs,
                           int kind_out, double2 *__restrict__ F0) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (i >= m || q >= n_rhs) return;
    const double rx = r[3 * i] - fx, ry = r[3 * i + 1] - fy, rz = r[3 * i + 2] - fz;
    const double xp = ct * rx - st * rz, yp = ry, zp = st * rx + ct * rz;
    const double z0 = 0.5 * k * w0 * w0;
    const double2 g = make_double2(1.0, zp / z0);
    const double2 ig = crecip(g);
    // exp(-(x'^2 + y'^2) ig / w0^2) exp(i k z')
    const double2 ex = cscale(ig, -(xp * xp + yp * yp) / (w0 * w0));
    double s, c;
    sincos(k * zp + ex.y, &s, &c);
    const double2 u = cmul(cscale(make_double2(c, s), exp(ex.x)), ig);
    const double2 a = make_double2(e0[6 * q], e0[6 * q + 1]), b = make_double2(e0[6 * q + 2], e0[6 * q + 3]);
    const double2 d = cscale(ig, -2.0 / (w0 * w0));                 // derivative factor
    const double2 ik = make_double2(0.0, 1.0 / k);
    const double2 Ex = cmul(a, u), Ey = cmul(b, u);
    const double2 Ez = cmul(cmul(ik, d), cmul(cadd(cscale(a, xp), cscale(b, yp)), u));
    const double2 Hx = cscale(cmul(b, u), -n_env), Hy = cscale(cmul(a, u), n_env);
    const double2 Hz = cmul(cmul(ik, d), cmul(cadd(cscale(b, -n_env * xp), cscale(a, n_env * yp)), u));
    double2 *o = F0 + (int64_t)q * kind_out * m + (int64_t)kind_out * i;
    // lab = x' ex + y' ey + z' ez with ex = (ct, 0, -st), ey = (0, 1, 0), ez = (st, 0, ct)
    o[0] = cadd(cscale(Ex, ct), cscale(Ez, st));
    o[1] = Ey;
    o[2] = cadd(cscale(Ex, -st), cscale(Ez, ct));
    if (kind_out == 6) {
        o[3] = cadd(cscale(Hx, ct), cscale(Hz, st));
        o[4] = Hy;
        o[5] = cadd(cscale(Hx, -st), cscale(Hz, ct));
    }
}

gdm_status gdm_launch_gaussian(gdm_ctx *ctx, const double *r, int64_t m, double k, double n_env, double w0,
                               const double *focus, double theta, const double *e0, int n_rhs, int kind_out,
                               double *F0) {
    double *de0;
    GDM_TRY(gdm_upload(ctx, e0, sizeof(double) * 6 * n_rhs, (void **)&de0));
    dim3 grid((unsigned)((m + 127) / 128), (unsigned)n_rhs);
    k_gaussian<<<grid, 128, 0, ctx->stream>>>(r, m, k, n_env, w0, focus[0], focus[1], focus[2], cos(theta),
                                              sin(theta), de0, n_rhs, kind_out, (double2 *)F0);
    GDM_LAUNCHED(ctx, "gaussian");
    return GDM_OK;
}

// Lorentzian ED/MD polarisabilities: one thread per dipole writes its 6x6 block (zeros off the diagonal)
__global__ void k_alpha6_lorentz(int64_t n, const double *__restrict__ w0e, const double *__restrict__ w0m, double g,
                                 double a3, double w, double rad_e, double rad_m, double2 *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 a[2];
    for (int h = 0; h < 2; h++) {
        const double w0 = h ? w0m[i] : w0e[i];
        // 1/alpha0 = (w0^2 - w^2 - i g w) / (a^3 w0^2); minus i rad; then invert
        const double s = 1.0 / (a3 * w0 * w0);
        const double re = (w0 * w0 - w * w) * s, im = -g * w * s - (h ? rad_m : rad_e);
        const double d = re * re + im * im;
        a[h] = make_double2(re / d, -im / d);
    }
    double2 *o = out + 36 * i;
    for (int e = 0; e < 36; e++) {
        const int r = e / 6, c = e % 6;
        o[e] = (r == c) ? a[r / 3] : make_double2(0.0, 0.0);
    }
}

// radiative dressing in the host: Im G^Ep(0) = (2/3) k^3/eps_env (electric), Im G^Hm(0) = (2/3) k^3 (magnetic)
gdm_status gdm_launch_alpha6_lorentz(gdm_ctx *ctx, int64_t n, const double *w0e, const double *w0m, double gamma_ev,
                                     double amp_nm, double wavelength, double eps_env, double *out) {
    const double hc_ev_nm = 1239.84198;  // h c in eV nm
    const double w = hc_ev_nm / wavelength, k = sqrt(eps_env) * 2.0 * PI_D / wavelength;
    const double rad_m = (2.0 / 3.0) * k * k * k;
    k_alpha6_lorentz<<<(unsigned)((n + 127) / 128), 128, 0, ctx->stream>>>(
        n, w0e, w0m, gamma_ev, amp_nm * amp_nm * amp_nm, w, rad_m / eps_env, rad_m, (double2 *)out);
    GDM_LAUNCHED(ctx, "alpha6_lorentz");
    return GDM_OK;
}

gdm_status gdm_launch_planewave(gdm_ctx *ctx, const double *r, int64_t m, double k, double n_env, const double *e0,
                                const double *khat, int n_rhs, int kind_out, double *F0) {
    double *de0;
    GDM_TRY(gdm_upload(ctx, e0, sizeof(double) * 6 * n_rhs, (void **)&de0));
    int bs = 256;
    k_planewave<<<(unsigned)((m + bs - 1) / bs), bs, 0, ctx->stream>>>(r, m, k, n_env, de0, khat[0], khat[1], khat[2],
                                                                       n_rhs, kind_out, (double2 *)F0);
    GDM_LAUNCHED(ctx, "planewave");
    return GDM_OK;
}


// ================================================================== per-dipole preparation
// FP32 assembly operands: positions split into (hi, lo) FP32 pairs so that r_i - r_j keeps ~48 bits,
// alpha_j rounded to complex64, and the diagonal block value 1 - S alpha_j (kind 3).
struct DipF {
    float xh, yh, zh, xl, yl, zl;
    float2 alpha;
    float2 diag;
    float pad[2];
};
static_assert(sizeof(DipF) == 48, "DipF layout");

__global__ void k_prep_dipf(const double *__restrict__ pos, const double2 *__restrict__ eps, int64_t n, double eps_env,
                            double d3_4pi, DipF *__restrict__ out) {
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
    d.diag = make_float2(1.f, 0.f);
    if (eps) {
        double2 e = eps[i];
        double ar = (e.x - eps_env) * d3_4pi, ai = e.y * d3_4pi;
        d.alpha = make_float2((float)ar, (float)ai);
        // 1 - S alpha with S = -4 pi / (3 eps_env d^3): 1 + (eps - eps_env) / (3 eps_env)
        d.diag = make_float2((float)(1.0 + (e.x - eps_env) / (3.0 * eps_env)), (float)(e.y / (3.0 * eps_env)));
    }
    d.pad[0] = d.pad[1] = 0.f;
    out[i] = d;
}

// FP64 cell polarisabilities alpha_j = (eps_j - eps_env) d^3 / (4 pi)
__global__ void k_alpha3_f64(const double2 *__restrict__ eps, int64_t n, double eps_env, double d3_4pi,
                             double2 *__restrict__ alpha) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 e = eps[i];
    alpha[i] = make_double2((e.x - eps_env) * d3_4pi, e.y * d3_4pi);
}

__global__ void k_alpha6_f32(const double2 *__restrict__ a6, int64_t count, float2 *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    out[i] = make_float2((float)a6[i].x, (float)a6[i].y);
}

// ================================================================== assembly
// Green coefficients of one ordered pair: G^Ep = a I + b u u^T, G^Hp = c [u]_x.
template <class T> struct PairG {
    typename cplx<T>::t a, b, c;
    T ux, uy, uz;
};

// FP32 with a double-float phase: the phase k R needs ~1e-9 absolute accuracy for kR up to ~1e3,
// the amplitudes 1/R^n only FP32 relative accuracy.
// FAST (the iterative solver's FP32 operator): R and 1/R from one hardware reciprocal square root refined
// by a Newton step (1/R to ~1e-7, R to double-float through the usual correction term), and the hardware
// sine/cosine in the phase; about 4e-7 on e^{ikR} instead of ~1e-7, well inside that operator's 1e-6.
template <bool FAST = false>
__device__ __forceinline__ PairG<float> pair_green_f32(const DipF &ti, const DipF &sj, ff kff, float kf, float k2,
                                                       float k0k, float inv_eps, bool need_c) {
    ff dx = ff_diff(ti.xh, ti.xl, sj.xh, sj.xl);
    ff dy = ff_diff(ti.yh, ti.yl, sj.yh, sj.yl);
    ff dz = ff_diff(ti.zh, ti.zl, sj.zh, sj.zl);
    ff r2 = ff_add(ff_add(ff_sqr(dx), ff_sqr(dy)), ff_sqr(dz));
    ff r;
    float r1;
    if (FAST) {
        float y = rsqrtf(r2.hi);
        y = y * fmaf(-0.5f * r2.hi * y, y, 1.5f);
        const float h = r2.hi * y;
        const float p = __fmul_rn(h, h);
        const float ep = fmaf(h, h, -p);
        const float res = __fadd_rn(__fsub_rn(__fsub_rn(r2.hi, p), ep), r2.lo);
        r = fast_two_sum(h, res * (0.5f * y));
        r1 = y;
    } else {
        r = ff_sqrt(r2);
        r1 = 1.0f / r.hi;
    }
    float r2i = r1 * r1, r3i = r2i * r1;
    float2 e = ff_expi<FAST>(ff_mul(kff, r));
    PairG<float> g;
    if (need_c) g.c = cmul(e, make_float2(k0k * r1, k0k * r2i / kf));
    e = cscale(e, inv_eps);
    g.a = cmul(e, make_float2(k2 * r1 - r3i, kf * r2i));
    g.b = cmul(e, make_float2(3.0f * r3i - k2 * r1, -3.0f * kf * r2i));
    g.ux = dx.hi * r1;
    g.uy = dy.hi * r1;
    g.uz = dz.hi * r1;
    return g;
}

__device__ __forceinline__ PairG<double> pair_green_f64(double dx, double dy, double dz, double k, double k2,
                                                        double k0k, double inv_eps, bool need_c) {
    double r2 = dx * dx + dy * dy + dz * dz;
    double r1 = rsqrt(r2);
    double r = r2 * r1;
    double r2i = r1 * r1, r3i = r2i * r1;
    double s, c;
    sincos(k * r, &s, &c);
    double2 e = make_double2(c, s);
    PairG<double> g;
    if (need_c) g.c = cmul(e, make_double2(k0k * r1, k0k * r2i / k));
    e = cscale(e, inv_eps);
    g.a = cmul(e, make_double2(k2 * r1 - r3i, k * r2i));
    g.b = cmul(e, make_double2(3.0 * r3i - k2 * r1, -3.0 * k * r2i));
    g.ux = dx * r1;
    g.uy = dy * r1;
    g.uz = dz * r1;
    return g;
}

// y = G^Ep x = a x + b u (u.x)
template <class C, class T>
__device__ __forceinline__ void apply_gep(const PairG<T> &g, const C *x, C *y) {
    C ud;
    ud.x = g.ux * x[0].x + g.uy * x[1].x + g.uz * x[2].x;
    ud.y = g.ux * x[0].y + g.uy * x[1].y + g.uz * x[2].y;
    C bu = cmul(g.b, ud);
    y[0] = cadd(cmul(g.a, x[0]), cscale(bu, g.ux));
    y[1] = cadd(cmul(g.a, x[1]), cscale(bu, g.uy));
    y[2] = cadd(cmul(g.a, x[2]), cscale(bu, g.uz));
}
// y = c (u x x)
template <class C, class T>
__device__ __forceinline__ void apply_ghp(const PairG<T> &g, const C *x, C *y) {
    C v0, v1, v2;
    v0.x = g.uy * x[2].x - g.uz * x[1].x;
    v0.y = g.uy * x[2].y - g.uz * x[1].y;
    v1.x = g.uz * x[0].x - g.ux * x[2].x;
    v1.y = g.uz * x[0].y - g.ux * x[2].y;
    v2.x = g.ux * x[1].x - g.uy * x[0].x;
    v2.y = g.ux * x[1].y - g.uy * x[0].y;
    y[0] = cmul(g.c, v0);
    y[1] = cmul(g.c, v1);
    y[2] = cmul(g.c, v2);
}
// 6x6 vacuum dyad on (x_e, x_m): (G x_e - C x_m, C x_e + G x_m)
template <class C, class T>
__device__ __forceinline__ void apply_g6(const PairG<T> &g, const C *x, C *y) {
    C ge[3], gm[3], ce[3], cm[3];
    apply_gep(g, x, ge);
    apply_gep(g, x + 3, gm);
    apply_ghp(g, x, ce);
    apply_ghp(g, x + 3, cm);
    for (int a = 0; a < 3; a++) {
        y[a] = csub(ge[a], cm[a]);
        y[3 + a] = cadd(ce[a], gm[a]);
    }
}

#define ASM_TI 128
#define ASM_TJ3 16
#define ASM_TJ6 4

// kind 3, complex64 output. Block (128 targets i) x (16 sources j). Column-major A, lda in complex.
__global__ void __launch_bounds__(ASM_TI) k_assemble3_f32(float2 *__restrict__ A, int64_t lda, int64_t n,
                                                         const DipF *__restrict__ dip, float khi, float klo,
                                                         float inv_eps) {
    __shared__ DipF sj[ASM_TJ3];
    int64_t j0 = (int64_t)blockIdx.y * ASM_TJ3;
    if (threadIdx.x < ASM_TJ3 && j0 + threadIdx.x < n) sj[threadIdx.x] = dip[j0 + threadIdx.x];
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * ASM_TI + threadIdx.x;
    if (i >= n) return;
    const DipF ti = dip[i];
    ff kff = {khi, klo};
    float kf = khi, k2 = khi * khi;
    int jn = (int)min((int64_t)ASM_TJ3, n - j0);
    for (int jj = 0; jj < jn; jj++) {
        int64_t j = j0 + jj;
        float2 *col = A + (3 * j) * lda + 3 * i;
        if (j == i) {
            float2 dg = sj[jj].diag;
            float2 z = make_float2(0.f, 0.f);
            col[0] = dg; col[1] = z; col[2] = z;
            col += lda;
            col[0] = z; col[1] = dg; col[2] = z;
            col += lda;
            col[0] = z; col[1] = z; col[2] = dg;
            continue;
        }
        PairG<float> g = pair_green_f32(ti, sj[jj], kff, kf, k2, 0.f, inv_eps, false);
        float2 al = sj[jj].alpha;
        float2 na = cmul(g.a, al), nb = cmul(g.b, al);
        na = make_float2(-na.x, -na.y);
        nb = make_float2(-nb.x, -nb.y);
        float u[3] = {g.ux, g.uy, g.uz};
#pragma unroll
        for (int b = 0; b < 3; b++) {
            float2 v0 = cscale(nb, u[0] * u[b]);
            float2 v1 = cscale(nb, u[1] * u[b]);
            float2 v2 = cscale(nb, u[2] * u[b]);
            if (b == 0) v0 = cadd(v0, na);
            if (b == 1) v1 = cadd(v1, na);
            if (b == 2) v2 = cadd(v2, na);
            col[0] = v0; col[1] = v1; col[2] = v2;
            col += lda;
        }
    }
}

// kind 3, complex128 output (plain FP64 path)
__global__ void __launch_bounds__(ASM_TI) k_assemble3_f64(double2 *__restrict__ A, int64_t lda, int64_t n,
                                                         const double *__restrict__ pos,
                                                         const double2 *__restrict__ alpha, double self_fac, double k,
                                                         double inv_eps) {
    __shared__ double sp[ASM_TJ3][3];
    __shared__ double2 sa[ASM_TJ3];
    int64_t j0 = (int64_t)blockIdx.y * ASM_TJ3;
    if (threadIdx.x < ASM_TJ3 && j0 + threadIdx.x < n) {
        int64_t j = j0 + threadIdx.x;
        sp[threadIdx.x][0] = pos[3 * j];
        sp[threadIdx.x][1] = pos[3 * j + 1];
        sp[threadIdx.x][2] = pos[3 * j + 2];
        sa[threadIdx.x] = alpha[j];
    }
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * ASM_TI + threadIdx.x;
    if (i >= n) return;
    double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    double k2 = k * k;
    int jn = (int)min((int64_t)ASM_TJ3, n - j0);
    for (int jj = 0; jj < jn; jj++) {
        int64_t j = j0 + jj;
        double2 *col = A + (3 * j) * lda + 3 * i;
        double2 al = sa[jj];
        if (j == i) {
            // 1 - S alpha with the cubic self-term S = -4 pi / (3 eps_env d^3) = -self_fac
            double2 dg = make_double2(1.0 + self_fac * al.x, self_fac * al.y);
            double2 z = make_double2(0.0, 0.0);
            col[0] = dg; col[1] = z; col[2] = z;
            col += lda;
            col[0] = z; col[1] = dg; col[2] = z;
            col += lda;
            col[0] = z; col[1] = z; col[2] = dg;
            continue;
        }
        PairG<double> g = pair_green_f64(xi - sp[jj][0], yi - sp[jj][1], zi - sp[jj][2], k, k2, 0.0, inv_eps, false);
        double2 na = cmul(g.a, al), nb = cmul(g.b, al);
        na = make_double2(-na.x, -na.y);
        nb = make_double2(-nb.x, -nb.y);
        double u[3] = {g.ux, g.uy, g.uz};
#pragma unroll
        for (int b = 0; b < 3; b++) {
            double2 v0 = cscale(nb, u[0] * u[b]);
            double2 v1 = cscale(nb, u[1] * u[b]);
            double2 v2 = cscale(nb, u[2] * u[b]);
            if (b == 0) v0 = cadd(v0, na);
            if (b == 1) v1 = cadd(v1, na);
            if (b == 2) v2 = cadd(v2, na);
            col[0] = v0; col[1] = v1; col[2] = v2;
            col += lda;
        }
    }
}

// kind 6 (ED/MD dipoles), generic 6x6 alpha_j. Block (128 targets) x (4 sources). Host medium: the
// dyad in its vacuum form at k acts on (x_e, n_env x_m); the rows are scaled by (1/eps_env, 1/n_env).
template <class T>
__global__ void __launch_bounds__(ASM_TI) k_assemble6(typename cplx<T>::t *__restrict__ A, int64_t lda, int64_t n,
                                                     const DipF *__restrict__ dipf, const double *__restrict__ pos,
                                                     const typename cplx<T>::t *__restrict__ alpha6, float khi,
                                                     float klo, double k, T n_env, T inv_eps, T inv_n) {
    typedef typename cplx<T>::t C;
    __shared__ C sa[ASM_TJ6][36];
    __shared__ DipF sjf[ASM_TJ6];
    __shared__ double sjp[ASM_TJ6][3];
    int64_t j0 = (int64_t)blockIdx.y * ASM_TJ6;
    int jn = (int)min((int64_t)ASM_TJ6, n - j0);
    for (int t = threadIdx.x; t < jn * 36; t += blockDim.x) sa[t / 36][t % 36] = alpha6[(j0 + t / 36) * 36 + t % 36];
    if (threadIdx.x < jn) {
        if (sizeof(T) == 4) sjf[threadIdx.x] = dipf[j0 + threadIdx.x];
        else {
            for (int c = 0; c < 3; c++) sjp[threadIdx.x][c] = pos[3 * (j0 + threadIdx.x) + c];
        }
    }
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * ASM_TI + threadIdx.x;
    if (i >= n) return;
    for (int jj = 0; jj < jn; jj++) {
        int64_t j = j0 + jj;
        C *col = A + (6 * j) * lda + 6 * i;
        if (j == i) {
            for (int q = 0; q < 6; q++) {
                for (int a = 0; a < 6; a++) {
                    C v;
                    v.x = (a == q) ? (T)1 : (T)0;
                    v.y = (T)0;
                    col[a] = v;
                }
                col += lda;
            }
            continue;
        }
        PairG<T> g;
        if constexpr (sizeof(T) == 4) {
            const DipF ti = dipf[i];
            ff kff = {khi, klo};
            g = pair_green_f32(ti, sjf[jj], kff, khi, khi * khi, khi * khi, 1.0f, true);
        } else {
            g = pair_green_f64(pos[3 * i] - sjp[jj][0], pos[3 * i + 1] - sjp[jj][1], pos[3 * i + 2] - sjp[jj][2], k,
                               k * k, k * k, 1.0, true);
        }
        for (int q = 0; q < 6; q++) {
            C x[6], y[6];
            for (int a = 0; a < 6; a++) x[a] = a < 3 ? sa[jj][a * 6 + q] : cscale(sa[jj][a * 6 + q], n_env);
            apply_g6(g, x, y);
            for (int a = 0; a < 6; a++) {
                const T sc = a < 3 ? -inv_eps : -inv_n;
                C v;
                v.x = sc * y[a].x;
                v.y = sc * y[a].y;
                col[a] = v;
            }
            col += lda;
        }
    }
}

// kind 3, complex64 output, stores through the bulk-copy engine. Block (128 targets i) x (8 sources j):
// the CTA builds its 384-row x 24-column tile of A in shared memory (each thread its 3x3 blocks, plain
// shared stores), then one cp.async.bulk per column moves the 3 KB column segment to HBM. A warp's
// direct stores of interleaved 3-row blocks would touch every 32-byte sector three times through L1.
#define ASB_TI 128
#define ASB_TJ 8
#define ASB_ROWS (3 * ASB_TI)
__device__ __forceinline__ void assemble3_f32_bulk_body(float2 *__restrict__ A, int64_t lda, int64_t n,
                                                        const DipF *__restrict__ dip, float khi, float klo,
                                                        float inv_eps, int64_t bx, int64_t by) {
    extern __shared__ __align__(128) float2 stile[];  // [3 * ASB_TJ columns][ASB_ROWS rows]
    __shared__ DipF sj[ASB_TJ];
    const int64_t i0 = bx * ASB_TI, j0 = by * ASB_TJ;
    if (threadIdx.x < ASB_TJ && j0 + threadIdx.x < n) sj[threadIdx.x] = dip[j0 + threadIdx.x];
    __syncthreads();
    const int64_t i = i0 + threadIdx.x;
    const int jn = (int)min((int64_t)ASB_TJ, n - j0);
    const int ni = (int)min((int64_t)ASB_TI, n - i0);
    if (i < n) {
        const DipF ti = dip[i];
        const ff kff = {khi, klo};
        const float kf = khi, k2 = khi * khi;
        for (int jj = 0; jj < jn; jj++) {
            float2 *col = stile + (3 * jj) * ASB_ROWS + 3 * threadIdx.x;
            if (j0 + jj == i) {
                const float2 dg = sj[jj].diag, z = make_float2(0.f, 0.f);
                col[0] = dg; col[1] = z; col[2] = z;
                col += ASB_ROWS;
                col[0] = z; col[1] = dg; col[2] = z;
                col += ASB_ROWS;
                col[0] = z; col[1] = z; col[2] = dg;
                continue;
            }
            PairG<float> g = pair_green_f32(ti, sj[jj], kff, kf, k2, 0.f, inv_eps, false);
            const float2 al = sj[jj].alpha;
            float2 na = cmul(g.a, al), nb = cmul(g.b, al);
            na = make_float2(-na.x, -na.y);
            nb = make_float2(-nb.x, -nb.y);
            const float u[3] = {g.ux, g.uy, g.uz};
#pragma unroll
            for (int b = 0; b < 3; b++) {
                float2 v0 = cscale(nb, u[0] * u[b]);
                float2 v1 = cscale(nb, u[1] * u[b]);
                float2 v2 = cscale(nb, u[2] * u[b]);
                if (b == 0) v0 = cadd(v0, na);
                if (b == 1) v1 = cadd(v1, na);
                if (b == 2) v2 = cadd(v2, na);
                col[0] = v0; col[1] = v1; col[2] = v2;
                col += ASB_ROWS;
            }
        }
    }
    // shared-memory writes of the generic proxy must be visible to the bulk-copy (async) proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const int rows = 3 * ni;
    const int rows16 = rows & ~1;  // a whole number of 16-byte units
    if ((int)threadIdx.x < 3 * jn) {
        const int c = threadIdx.x;
        float2 *dst = A + (3 * j0 + c) * lda + 3 * i0;
        const float2 *src = stile + c * ASB_ROWS;
        if (rows16 > 0) {
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                         "r"((uint32_t)__cvta_generic_to_shared(src)), "r"((uint32_t)(rows16 * sizeof(float2)))
                         : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        if (rows & 1) dst[rows - 1] = src[rows - 1];
        // the shared tile must stay until the engine has read it
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
}
__global__ void __launch_bounds__(ASB_TI) k_assemble3_f32_bulk(float2 *__restrict__ A, int64_t lda, int64_t n,
                                                              const DipF *__restrict__ dip, float khi, float klo,
                                                              float inv_eps) {
    assemble3_f32_bulk_body(A, lda, n, dip, khi, klo, inv_eps, blockIdx.x, blockIdx.y);
}

// kind 6 (ED/MD dipoles), complex64 output through the bulk-copy engine. Block (AS6_TI targets) x (4 sources),
// one thread per ordered pair: the CTA builds its (6 AS6_TI)-row x 24-column tile of A in shared memory
// (each thread its 6x6 block), then one cp.async.bulk per column moves the column segment to HBM. The direct
// stores of k_assemble6 (8 bytes per lane at a 48-byte stride) are bound by the L1 store path, not by HBM.
#define AS6_TJ 4
template <int AS6_TI>
__global__ void __launch_bounds__(AS6_TI * AS6_TJ) k_assemble6_f32_bulk(float2 *__restrict__ A, int64_t lda, int64_t n,
                                                                       const DipF *__restrict__ dipf,
                                                                       const float2 *__restrict__ alpha6, float khi,
                                                                       float klo, float n_env, float inv_eps,
                                                                       float inv_n) {
    constexpr int AS6_ROWS = 6 * AS6_TI;
    extern __shared__ __align__(128) float2 stile6[];  // [6 * AS6_TJ columns][AS6_ROWS rows]
    __shared__ float2 sa[AS6_TJ][36];
    __shared__ DipF sjf[AS6_TJ];
    const int64_t i0 = (int64_t)blockIdx.x * AS6_TI, j0 = (int64_t)blockIdx.y * AS6_TJ;
    const int jn = (int)min((int64_t)AS6_TJ, n - j0);
    const int ni = (int)min((int64_t)AS6_TI, n - i0);
    for (int t = threadIdx.x; t < jn * 36; t += blockDim.x) sa[t / 36][t % 36] = alpha6[(j0 + t / 36) * 36 + t % 36];
    if ((int)threadIdx.x < jn) sjf[threadIdx.x] = dipf[j0 + threadIdx.x];
    __syncthreads();
    const int il = threadIdx.x % AS6_TI, jj = threadIdx.x / AS6_TI;
    const int64_t i = i0 + il, j = j0 + jj;
    if (il < ni && jj < jn) {
        float2 *col = stile6 + (6 * jj) * AS6_ROWS + 6 * il;
        if (j == i) {
            for (int q = 0; q < 6; q++) {
                for (int a = 0; a < 6; a++) col[a] = make_float2(a == q ? 1.f : 0.f, 0.f);
                col += AS6_ROWS;
            }
        } else {
            const DipF ti = dipf[i];
            const ff kff = {khi, klo};
            const PairG<float> g = pair_green_f32(ti, sjf[jj], kff, khi, khi * khi, khi * khi, 1.0f, true);
            for (int q = 0; q < 6; q++) {
                float2 x[6], y[6];
#pragma unroll
                for (int a = 0; a < 6; a++) x[a] = a < 3 ? sa[jj][a * 6 + q] : cscale(sa[jj][a * 6 + q], n_env);
                apply_g6(g, x, y);
#pragma unroll
                for (int a = 0; a < 6; a++) {
                    const float sc = a < 3 ? -inv_eps : -inv_n;
                    col[a] = make_float2(sc * y[a].x, sc * y[a].y);
                }
                col += AS6_ROWS;
            }
        }
    }
    // shared-memory writes of the generic proxy must be visible to the bulk-copy (async) proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // 6 ni rows per column: always a whole number of 16-byte units; the column segment starts at row 6 i0
    // of a column of an lda-even, 16-byte aligned matrix, so it is 16-byte aligned too
    if ((int)threadIdx.x < 6 * jn) {
        const int c = threadIdx.x;
        float2 *dst = A + (6 * j0 + c) * lda + 6 * i0;
        const float2 *src = stile6 + c * AS6_ROWS;
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                     "r"((uint32_t)__cvta_generic_to_shared(src)), "r"((uint32_t)(6 * ni * sizeof(float2)))
                     : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        // the shared tile must stay until the engine has read it
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
}

template <int TI>
static gdm_status launch_assemble6_bulk(gdm_ctx *ctx, float2 *A, int64_t lda, int64_t n, const DipF *dipf,
                                        const float2 *a6, float khi, float klo, double n_env, double eps_env) {
    const int smem = 6 * AS6_TJ * 6 * TI * (int)sizeof(float2);
    static bool attr = false;
    if (!attr) {
        GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_assemble6_f32_bulk<TI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               smem));
        attr = true;
    }
    dim3 g6((unsigned)((n + TI - 1) / TI), (unsigned)((n + AS6_TJ - 1) / AS6_TJ));
    k_assemble6_f32_bulk<TI><<<g6, TI * AS6_TJ, smem, ctx->stream>>>(A, lda, n, dipf, a6, khi, klo, (float)n_env,
                                                                     (float)(1.0 / eps_env), (float)(1.0 / n_env));
    GDM_LAUNCHED(ctx, "assemble6_f32_bulk");
    return GDM_OK;
}

gdm_status gdm_launch_assemble(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, void *A, int64_t lda) {
    int64_t n = p->n;
    double k0 = gdm_k0(p);
    double k = sqrt(p->eps_env) * k0;
    double d3_4pi = p->kind == 3 ? p->step * p->step * p->step / (4.0 * PI_D) : 0.0;
    size_t need = ScratchCarver::round(n * sizeof(DipF)) + ScratchCarver::round(n * sizeof(double2)) +
                  (p->kind == 6 ? ScratchCarver::round(n * 36 * sizeof(float2)) : 0) + 1024;
    void *ws;
    GDM_TRY(gdm_scratch(ctx, need, &ws));
    ScratchCarver sc(ws);
    DipF *dipf = sc.take<DipF>(n);
    double2 *alpha = sc.take<double2>(n);
    int bs = 256;
    unsigned nb = (unsigned)((n + bs - 1) / bs);
    float khi = (float)k, klo = (float)(k - (double)khi);
    dim3 blk(ASM_TI);
    if (p->kind == 3) {
        if (prec == GDM_FP64) {
            k_alpha3_f64<<<nb, bs, 0, ctx->stream>>>((const double2 *)p->eps, n, p->eps_env, d3_4pi, alpha);
            GDM_LAUNCHED(ctx, "alpha3_f64");
            dim3 grid((unsigned)((n + ASM_TI - 1) / ASM_TI), (unsigned)((n + ASM_TJ3 - 1) / ASM_TJ3));
            double self_fac = 4.0 * PI_D / (3.0 * p->eps_env * p->step * p->step * p->step);
            k_assemble3_f64<<<grid, blk, 0, ctx->stream>>>((double2 *)A, lda, n, p->pos, alpha, self_fac, k,
                                                          1.0 / p->eps_env);
            GDM_LAUNCHED(ctx, "assemble3_f64");
        } else {
            k_prep_dipf<<<nb, bs, 0, ctx->stream>>>(p->pos, (const double2 *)p->eps, n, p->eps_env, d3_4pi, dipf);
            GDM_LAUNCHED(ctx, "prep_dipf");
            if (((uintptr_t)A & 15) == 0 && (lda & 1) == 0 && !getenv("GDM_ASSEMBLE_DIRECT")) {
                const int smem = 3 * ASB_TJ * ASB_ROWS * (int)sizeof(float2);
                static bool attr = false;
                if (!attr) {
                    GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_assemble3_f32_bulk,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                    attr = true;
                }
                dim3 grid((unsigned)((n + ASB_TI - 1) / ASB_TI), (unsigned)((n + ASB_TJ - 1) / ASB_TJ));
                k_assemble3_f32_bulk<<<grid, ASB_TI, smem, ctx->stream>>>((float2 *)A, lda, n, dipf, khi, klo,
                                                                         (float)(1.0 / p->eps_env));
                GDM_LAUNCHED(ctx, "assemble3_f32_bulk");
            } else {
                dim3 grid((unsigned)((n + ASM_TI - 1) / ASM_TI), (unsigned)((n + ASM_TJ3 - 1) / ASM_TJ3));
                k_assemble3_f32<<<grid, blk, 0, ctx->stream>>>((float2 *)A, lda, n, dipf, khi, klo,
                                                              (float)(1.0 / p->eps_env));
                GDM_LAUNCHED(ctx, "assemble3_f32");
            }
        }
    } else {
        dim3 grid((unsigned)((n + ASM_TI - 1) / ASM_TI), (unsigned)((n + ASM_TJ6 - 1) / ASM_TJ6));
        const double n_env = sqrt(p->eps_env);
        if (prec == GDM_FP64) {
            k_assemble6<double><<<grid, blk, 0, ctx->stream>>>((double2 *)A, lda, n, nullptr, p->pos,
                                                              (const double2 *)p->alpha6, khi, klo, k, n_env,
                                                              1.0 / p->eps_env, 1.0 / n_env);
            GDM_LAUNCHED(ctx, "assemble6_f64");
        } else {
            float2 *a6 = sc.take<float2>(n * 36);
            k_prep_dipf<<<nb, bs, 0, ctx->stream>>>(p->pos, nullptr, n, 1.0, 0.0, dipf);
            GDM_LAUNCHED(ctx, "prep_dipf");
            k_alpha6_f32<<<(unsigned)((n * 36 + bs - 1) / bs), bs, 0, ctx->stream>>>((const double2 *)p->alpha6,
                                                                                     n * 36, a6);
            GDM_LAUNCHED(ctx, "alpha6_f32");
            if (((uintptr_t)A & 15) == 0 && (lda & 1) == 0 && !getenv("GDM_ASSEMBLE_DIRECT")) {
                const char *e = getenv("GDM_AS6_TI");
                const int ti = e ? atoi(e) : 64;
                if (ti == 32) GDM_TRY(launch_assemble6_bulk<32>(ctx, (float2 *)A, lda, n, dipf, a6, khi, klo, n_env, p->eps_env));
                else if (ti == 48) GDM_TRY(launch_assemble6_bulk<48>(ctx, (float2 *)A, lda, n, dipf, a6, khi, klo, n_env, p->eps_env));
                else GDM_TRY(launch_assemble6_bulk<64>(ctx, (float2 *)A, lda, n, dipf, a6, khi, klo, n_env, p->eps_env));
            } else {
                k_assemble6<float><<<grid, blk, 0, ctx->stream>>>((float2 *)A, lda, n, dipf, p->pos, a6, khi, klo, k,
                                                                 (float)n_env, (float)(1.0 / p->eps_env),
                                                                 (float)(1.0 / n_env));
                GDM_LAUNCHED(ctx, "assemble6_f32");
            }
        }
    }
    return GDM_OK;
}

// ================================================================== FP64 matrix-free Green sums
// Dipole moments P = alpha X (forward) or P = conj(X) (adjoint sources, kind 3); (kind*n) x n_rhs.
// ED/MD (kind 6): the magnetic moments are stored times n_env, the form the Green sums and the far
// field take them in.
__global__ void k_moments(const double2 *__restrict__ X, int64_t n, int kind, int n_rhs, const double2 *__restrict__ eps,
                          double eps_env, double d3_4pi, const double2 *__restrict__ alpha6, int conj_only,
                          double2 *__restrict__ P) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int q = blockIdx.y;
    if (i >= n || q >= n_rhs) return;
    int64_t ld = kind * n;
    const double2 *x = X + q * ld + kind * i;
    double2 *o = P + q * ld + kind * i;
    if (conj_only) {
        for (int a = 0; a < kind; a++) o[a] = conjd(x[a]);
        return;
    }
    if (kind == 3) {
        double2 al = make_double2((eps[i].x - eps_env) * d3_4pi, eps[i].y * d3_4pi);
        for (int a = 0; a < 3; a++) o[a] = cmul(al, x[a]);
    } else {
        const double2 *al = alpha6 + 36 * i;
        const double n_env = sqrt(eps_env);
        for (int a = 0; a < 6; a++) {
            double2 s = make_double2(0.0, 0.0);
            for (int b = 0; b < 6; b++) cfma(s, al[6 * a + b], x[b]);
            o[a] = a < 3 ? s : cscale(s, n_env);
        }
    }
}

#define GS_T 128
#define GS_S 32

// partial[c][q][t][OUT] = sum over sources j of chunk c of G(r_t - r_j) P_j  (q < NR RHS of this group)
// OUT = 3 (G^Ep only), or 6 (G^Ep and G^Hp for kind 3 near fields / full 6x6 dyad for kind 6).
template <int KIND, int OUT, int NR>
__global__ void __launch_bounds__(GS_T) k_green_sum(const double *__restrict__ tpos, int64_t m,
                                                   const double *__restrict__ spos, const double2 *__restrict__ P,
                                                   int64_t n, int rhs0, int nr_here, double k, double k0,
                                                   double inv_eps, int64_t chunk, int self_exclude,
                                                   double2 *__restrict__ partial) {
    __shared__ double sp[GS_S][3];
    __shared__ double2 sm[GS_S][KIND][NR];
    const int64_t t = (int64_t)blockIdx.x * GS_T + threadIdx.x;
    const bool valid = t < m;
    const int64_t c = blockIdx.y;
    const int64_t jb = c * chunk, je = min(n, jb + chunk);
    double tx = 0, ty = 0, tz = 0;
    if (valid) {
        tx = tpos[3 * t];
        ty = tpos[3 * t + 1];
        tz = tpos[3 * t + 2];
    }
    double2 acc[NR][OUT];
#pragma unroll
    for (int q = 0; q < NR; q++)
#pragma unroll
        for (int a = 0; a < OUT; a++) acc[q][a] = make_double2(0.0, 0.0);
    const double k2 = k * k, k0k = k0 * k;
    const int64_t ldp = (int64_t)KIND * n;
    for (int64_t s0 = jb; s0 < je; s0 += GS_S) {
        int sn = (int)min((int64_t)GS_S, je - s0);
        for (int e = threadIdx.x; e < sn * 3; e += GS_T) sp[e / 3][e % 3] = spos[3 * s0 + e];
        for (int e = threadIdx.x; e < sn * KIND * NR; e += GS_T) {
            int jj = e / (KIND * NR), rem = e % (KIND * NR), a = rem / NR, q = rem % NR;
            double2 v = make_double2(0.0, 0.0);
            if (q < nr_here) v = P[(rhs0 + q) * ldp + KIND * (s0 + jj) + a];
            sm[jj][a][q] = v;
        }
        __syncthreads();
        if (valid) {
            for (int jj = 0; jj < sn; jj++) {
                if (self_exclude && s0 + jj == t) continue;
                PairG<double> g = pair_green_f64(tx - sp[jj][0], ty - sp[jj][1], tz - sp[jj][2], k, k2, k0k, inv_eps,
                                                 OUT == 6);
#pragma unroll
                for (int q = 0; q < NR; q++) {
                    double2 x[KIND], y[OUT];
#pragma unroll
                    for (int a = 0; a < KIND; a++) x[a] = sm[jj][a][q];
                    if constexpr (KIND == 6) {
                        apply_g6(g, x, y);
                    } else {
                        apply_gep(g, x, y);
                        if constexpr (OUT == 6) apply_ghp(g, x, y + 3);
                    }
#pragma unroll
                    for (int a = 0; a < OUT; a++) acc[q][a] = cadd(acc[q][a], y[a]);
                }
            }
        }
        __syncthreads();
    }
    if (!valid) return;
#pragma unroll
    for (int q = 0; q < NR; q++) {
        if (q >= nr_here) break;
        double2 *o = partial + ((c * NR + q) * m + t) * OUT;
#pragma unroll
        for (int a = 0; a < OUT; a++) o[a] = acc[q][a];
    }
}

// r = rhs - X + (G P)  [forward, P = alpha X, self-term S P_t for cells]
// r = rhs - X + conj(alpha_t) conj(G P)  [adjoint kind 3, P = conj(X): (A^H X)_t = X_t - conj(alpha_t (G conj X)_t)]
template <int KIND, int NR>
__device__ __forceinline__ void residual_finalize_body(const double2 *__restrict__ partial, int nchunks, int64_t n,
                                                       int rhs0, int nr_here, const double2 *__restrict__ rhs,
                                                       const double2 *__restrict__ X, const double2 *__restrict__ P,
                                                       double self_S, int adjoint, const double2 *__restrict__ eps,
                                                       double eps_env, double d3_4pi, double sE, double sH,
                                                       double2 *__restrict__ r, double *__restrict__ norms2,
                                                       int64_t bx) {
    int64_t t = bx * (int64_t)blockDim.x + threadIdx.x;
    double nrm[NR];
#pragma unroll
    for (int q = 0; q < NR; q++) nrm[q] = 0.0;
    if (t < n) {
        const int64_t ld = (int64_t)KIND * n;
        double2 al = make_double2(0.0, 0.0);
        if (adjoint && KIND == 3) al = make_double2((eps[t].x - eps_env) * d3_4pi, eps[t].y * d3_4pi);
#pragma unroll
        for (int q = 0; q < NR; q++) {
            if (q >= nr_here) break;
            int64_t col = (int64_t)(rhs0 + q) * ld + KIND * t;
            for (int a = 0; a < KIND; a++) {
                double2 s = make_double2(0.0, 0.0);
                for (int c = 0; c < nchunks; c++) s = cadd(s, partial[((c * NR + q) * n + t) * KIND + a]);
                if (KIND == 3) s = cadd(s, cscale(P[col + a], self_S));
                else s = cscale(s, a < 3 ? sE : sH);
                double2 v;
                if (adjoint) v = cadd(csub(rhs[col + a], X[col + a]), cmul(conjd(al), conjd(s)));
                else v = cadd(csub(rhs[col + a], X[col + a]), s);
                r[col + a] = v;
                nrm[q] += v.x * v.x + v.y * v.y;
            }
        }
    }
    // block reduction of the squared norms
    __shared__ double red[NR][32];
#pragma unroll
    for (int q = 0; q < NR; q++) {
        double v = nrm[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32 && norms2) {
        int nw = blockDim.x >> 5;
#pragma unroll
        for (int q = 0; q < NR; q++) {
            double v = threadIdx.x < nw ? red[q][threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (threadIdx.x == 0 && q < nr_here) atomicAdd(&norms2[rhs0 + q], v);
        }
    }
}
template <int KIND, int NR>
__global__ void k_residual_finalize(const double2 *__restrict__ partial, int nchunks, int64_t n, int rhs0, int nr_here,
                                    const double2 *__restrict__ rhs, const double2 *__restrict__ X,
                                    const double2 *__restrict__ P, double self_S, int adjoint,
                                    const double2 *__restrict__ eps, double eps_env, double d3_4pi, double sE,
                                    double sH, double2 *__restrict__ r, double *__restrict__ norms2) {
    residual_finalize_body<KIND, NR>(partial, nchunks, n, rhs0, nr_here, rhs, X, P, self_S, adjoint, eps, eps_env,
                                     d3_4pi, sE, sH, r, norms2, blockIdx.x);
}

// Grid of a Green-sum launch: ceil(m / GS_T) target blocks times nc source chunks of ceil(n / nc) sources.
// The kernels are ALU-bound and a CTA's time is about proportional to its chunk, so the last partial wave of
// CTAs idles the rest of the GPU; nc is the number of chunks (at most 64) that wastes the least of the
// occ x SMs resident-CTA slots over the whole launch (fewest chunks among equals); a context that shares the
// GPU with concurrent work counts only its share of the SMs.
static void green_grid(gdm_ctx *ctx, int64_t m, int64_t n, int occ, int64_t *chunk, int *nchunks) {
    const int64_t tb = (m + GS_T - 1) / GS_T;
    const int sms = ctx->share_sms > 0 && ctx->share_sms < ctx->sm_count ? ctx->share_sms : ctx->sm_count;
    const int64_t slots = (int64_t)(occ < 1 ? 1 : occ) * sms;
    int64_t maxc = (n + GS_S - 1) / GS_S;
    if (maxc > 64) maxc = 64;
    int64_t best_ch = n;
    double best = -1.0;
    for (int64_t nc = 1; nc <= maxc; nc++) {
        const int64_t ch = (n + nc - 1) / nc;  // any chunk length: the kernels stage partial tiles
        const int64_t ctas = tb * ((n + ch - 1) / ch);
        const int64_t waves = (ctas + slots - 1) / slots;
        const double eff = (double)ctas / (double)(waves * slots);
        if (eff > best + 1e-9) {
            best = eff;
            best_ch = ch;
        }
    }
    *chunk = best_ch;
    *nchunks = (int)((n + best_ch - 1) / best_ch);
}

// partial-sum bytes that any Green-sum launch over m targets and n sources may use (every occupancy the
// kernels have: 1 to 8 resident CTAs per SM)
size_t gdm_green_partial_bytes(gdm_ctx *ctx, int64_t m, int64_t n, int out) {
    int mx = 1;
    for (int occ = 1; occ <= 8; occ++) {
        int64_t chunk;
        int nc;
        green_grid(ctx, m, n, occ, &chunk, &nc);
        if (nc > mx) mx = nc;
    }
    return (size_t)mx * 2 * m * out * sizeof(double2);
}

// resident CTAs per SM of a kernel launched with GS_T threads and no dynamic shared memory (cached per kernel)
template <class K> static int occupancy_of(K kernel) {
    static int cached = 0;
    if (!cached) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, GS_T, 0) != cudaSuccess || b < 1) {
            cudaGetLastError();
            b = 4;
        }
        cached = b > 8 ? 8 : b;
    }
    return cached;
}
int gdm_ff_occupancy(int kind, int out, int nr);

template <int KIND, int OUT>
static gdm_status launch_green_sum(gdm_ctx *ctx, const double *tpos, int64_t m, const double *spos,
                                   const double2 *P, int64_t n, int rhs0, int nr_here, double k, double k0,
                                   double inv_eps, int self_exclude, double2 *partial, int *nchunks_out) {
    int64_t chunk;
    int nc;
    green_grid(ctx, m, n, occupancy_of(k_green_sum<KIND, OUT, 2>), &chunk, &nc);
    dim3 grid((unsigned)((m + GS_T - 1) / GS_T), (unsigned)nc);
    k_green_sum<KIND, OUT, 2><<<grid, GS_T, 0, ctx->stream>>>(tpos, m, spos, P, n, rhs0, nr_here, k, k0, inv_eps,
                                                              chunk, self_exclude, partial);
    GDM_LAUNCHED(ctx, "green_sum");
    *nchunks_out = nc;
    return GDM_OK;
}

gdm_status gdm_launch_green_sum_ff(gdm_ctx *ctx, const gdm_problem *p, const double2 *P, int rhs0, int nr,
                                   int64_t chunk, int nchunks, void *ffws, double2 *partial, int prepare);

// partial[c][q][t][3] = sum over sources j != t of chunk c of G^Ep(r_t - r_j) P_j for cells, in FP32 with the
// double-float position differences and phase of the FP32 assembly (about 1e-7 relative per pair, some 1e-6
// for a sum): the low-precision operator of the iterative solver, ~1/9 of the double-float kernel's work
template <int NR>
__device__ __forceinline__ void green_sum_f32_body(const DipF *__restrict__ dip, int64_t n,
                                                   const double2 *__restrict__ P, int rhs0, int nr_here, float khi,
                                                   float klo, float inv_eps, int64_t chunk,
                                                   double2 *__restrict__ partial, int64_t bx, int64_t c) {
    __shared__ DipF sj[GS_S];
    __shared__ float2 sm[GS_S][NR][3];
    const int64_t t = bx * GS_T + threadIdx.x;
    const bool valid = t < n;
    const int64_t jb = c * chunk, je = min(n, jb + chunk);
    const DipF ti = dip[valid ? t : 0];
    const ff kff = {khi, klo};
    const float k2 = khi * khi;
    float2 acc[NR][3];
#pragma unroll
    for (int q = 0; q < NR; q++)
#pragma unroll
        for (int a = 0; a < 3; a++) acc[q][a] = make_float2(0.f, 0.f);
    const int64_t ld = 3 * n;
    for (int64_t s0 = jb; s0 < je; s0 += GS_S) {
        const int sn = (int)min((int64_t)GS_S, je - s0);
        if (threadIdx.x < sn) sj[threadIdx.x] = dip[s0 + threadIdx.x];
        for (int e = threadIdx.x; e < sn * 3 * NR; e += GS_T) {
            const int jj = e / (3 * NR), rem = e % (3 * NR), q = rem / 3, a = rem % 3;
            double2 v = make_double2(0.0, 0.0);
            if (q < nr_here) v = P[(rhs0 + q) * ld + 3 * (s0 + jj) + a];
            sm[jj][q][a] = make_float2((float)v.x, (float)v.y);
        }
        __syncthreads();
        if (valid) {
            for (int jj = 0; jj < sn; jj++) {
                if (s0 + jj == t) continue;
                const PairG<float> g = pair_green_f32<true>(ti, sj[jj], kff, khi, k2, 0.f, inv_eps, false);
#pragma unroll
                for (int q = 0; q < NR; q++) {
                    float2 y[3];
                    apply_gep(g, sm[jj][q], y);
#pragma unroll
                    for (int a = 0; a < 3; a++) acc[q][a] = cadd(acc[q][a], y[a]);
                }
            }
        }
        __syncthreads();
    }
    if (!valid) return;
#pragma unroll
    for (int q = 0; q < NR; q++) {
        if (q >= nr_here) break;
        double2 *o = partial + ((c * NR + q) * n + t) * 3;
#pragma unroll
        for (int a = 0; a < 3; a++) o[a] = make_double2((double)acc[q][a].x, (double)acc[q][a].y);
    }
}
template <int NR>
__global__ void __launch_bounds__(GS_T) k_green_sum_f32(const DipF *__restrict__ dip, int64_t n,
                                                       const double2 *__restrict__ P, int rhs0, int nr_here,
                                                       float khi, float klo, float inv_eps, int64_t chunk,
                                                       double2 *__restrict__ partial) {
    green_sum_f32_body<NR>(dip, n, P, rhs0, nr_here, khi, klo, inv_eps, chunk, partial, blockIdx.x, blockIdx.y);
}

// residual of the FP64 system (matrix-free); scratch: P (kN x n_rhs) + partial buffer; ffws (nullable):
// double-float workspace (gdm_ff_scratch_bytes) selecting the double-float pair kernel for cells.
gdm_status gdm_launch_residual_ws(gdm_ctx *ctx, const gdm_problem *p, const double *rhs, const double *X, int n_rhs,
                                  int adjoint, double *r, double *norms2, double2 *Pbuf, double2 *partial, void *ffws,
                                  int ff_prepare) {
    const int64_t n = p->n;
    const int kind = p->kind;
    if (adjoint && kind != 3) return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "adjoint residual implemented for kind 3");
    double k0 = gdm_k0(p), k = sqrt(p->eps_env) * k0;
    double d3_4pi = kind == 3 ? p->step * p->step * p->step / (4.0 * PI_D) : 0.0;
    double S = kind == 3 ? -4.0 * PI_D / (3.0 * p->eps_env * p->step * p->step * p->step) : 0.0;
    dim3 g1((unsigned)((n + 127) / 128), (unsigned)n_rhs);
    k_moments<<<g1, 128, 0, ctx->stream>>>((const double2 *)X, n, kind, n_rhs, (const double2 *)p->eps, p->eps_env,
                                            d3_4pi, (const double2 *)p->alpha6, adjoint, Pbuf);
    GDM_LAUNCHED(ctx, "moments");
    if (norms2) GDM_CUDA_TRY(ctx, cudaMemsetAsync(norms2, 0, sizeof(double) * n_rhs, ctx->stream));
    for (int q0 = 0; q0 < n_rhs; q0 += 2) {
        int nr = n_rhs - q0 < 2 ? n_rhs - q0 : 2;
        int nc;
        if (ffws) {
            int64_t chunk;
            green_grid(ctx, n, n, gdm_ff_occupancy(kind, kind, nr), &chunk, &nc);
            GDM_TRY(gdm_launch_green_sum_ff(ctx, p, Pbuf, q0, nr, chunk, nc, ffws, partial, ff_prepare && q0 == 0));
        } else if (kind == 3)
            GDM_TRY(launch_green_sum<3, 3>(ctx, p->pos, n, p->pos, Pbuf, n, q0, nr, k, k0, 1.0 / p->eps_env, 1,
                                           partial, &nc));
        else
            GDM_TRY(launch_green_sum<6, 6>(ctx, p->pos, n, p->pos, Pbuf, n, q0, nr, k, k, 1.0, 1, partial, &nc));
        unsigned nb = (unsigned)((n + 255) / 256);
        if (kind == 3)
            k_residual_finalize<3, 2><<<nb, 256, 0, ctx->stream>>>(
                partial, nc, n, q0, nr, (const double2 *)rhs, (const double2 *)X, Pbuf, S, adjoint,
                (const double2 *)p->eps, p->eps_env, d3_4pi, 1.0, 1.0, (double2 *)r, norms2);
        else
            k_residual_finalize<6, 2><<<nb, 256, 0, ctx->stream>>>(
                partial, nc, n, q0, nr, (const double2 *)rhs, (const double2 *)X, Pbuf, 0.0, 0, nullptr, 1.0, 0.0,
                1.0 / p->eps_env, 1.0 / sqrt(p->eps_env), (double2 *)r, norms2);
        GDM_LAUNCHED(ctx, "residual_finalize");
    }
    return GDM_OK;
}

// r = rhs - X + G P for cells with the FP32 Green sums above (the iterative solver's low-precision operator);
// same scratch as gdm_launch_residual_ws; dipf: the FP32-pair positions of gdm_launch_green_sum_ff's
// workspace (prepared by an earlier double-float call on the same problem)
gdm_status gdm_launch_residual_f32(gdm_ctx *ctx, const gdm_problem *p, const double *rhs, const double *X, int n_rhs,
                                   double *r, double *norms2, double2 *Pbuf, double2 *partial, const void *dipf) {
    const int64_t n = p->n;
    if (p->kind != 3) return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "FP32 operator implemented for kind 3");
    const double k0 = gdm_k0(p), k = sqrt(p->eps_env) * k0;
    const double d3_4pi = p->step * p->step * p->step / (4.0 * PI_D);
    const double S = -4.0 * PI_D / (3.0 * p->eps_env * p->step * p->step * p->step);
    const float khi = (float)k, klo = (float)(k - (double)khi);
    dim3 g1((unsigned)((n + 127) / 128), (unsigned)n_rhs);
    k_moments<<<g1, 128, 0, ctx->stream>>>((const double2 *)X, n, 3, n_rhs, (const double2 *)p->eps, p->eps_env,
                                            d3_4pi, nullptr, 0, Pbuf);
    GDM_LAUNCHED(ctx, "moments");
    if (norms2) GDM_CUDA_TRY(ctx, cudaMemsetAsync(norms2, 0, sizeof(double) * n_rhs, ctx->stream));
    for (int q0 = 0; q0 < n_rhs; q0 += 2) {
        const int nr = n_rhs - q0 < 2 ? n_rhs - q0 : 2;
        int64_t chunk;
        int nc;
        green_grid(ctx, n, n, occupancy_of(k_green_sum_f32<2>), &chunk, &nc);
        dim3 grid((unsigned)((n + GS_T - 1) / GS_T), (unsigned)nc);
        k_green_sum_f32<2><<<grid, GS_T, 0, ctx->stream>>>((const DipF *)dipf, n, Pbuf, q0, nr, khi, klo,
                                                          (float)(1.0 / p->eps_env), chunk, partial);
        GDM_LAUNCHED(ctx, "green_sum_f32");
        k_residual_finalize<3, 2><<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
            partial, nc, n, q0, nr, (const double2 *)rhs, (const double2 *)X, Pbuf, S, 0, (const double2 *)p->eps,
            p->eps_env, d3_4pi, 1.0, 1.0, (double2 *)r, norms2);
        GDM_LAUNCHED(ctx, "residual_finalize");
    }
    return GDM_OK;
}

// ================================================================== near field
template <int OUT>
__global__ void k_nearfield_finalize(const double2 *__restrict__ partial, int nchunks, int64_t m, int rhs0, int nr_here,
                                     const double2 *__restrict__ F0e, int n_rhs_total, double sE, double sH,
                                     double2 *__restrict__ E, double2 *__restrict__ H) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= m) return;
    for (int q = 0; q < nr_here; q++) {
        int qq = rhs0 + q;
        for (int a = 0; a < OUT; a++) {
            double2 s = make_double2(0.0, 0.0);
            for (int c = 0; c < nchunks; c++) s = cadd(s, partial[((c * 2 + q) * m + t) * OUT + a]);
            s = cscale(s, a < 3 ? sE : sH);
            if (F0e) s = cadd(s, F0e[(int64_t)qq * 6 * m + 6 * t + a]);
            if (a < 3) E[(int64_t)qq * 3 * m + 3 * t + a] = s;
            else if (H) H[(int64_t)qq * 3 * m + 3 * t + a - 3] = s;
        }
    }
}

gdm_status gdm_ff_green_sum(gdm_ctx *ctx, const gdm_problem *p, const void *tgt, int64_t m, int out,
                            const double2 *P, int rhs0, int nr, int64_t chunk, int nchunks, void *ffws,
                            double2 *partial, int prepare);
gdm_status gdm_ff_targets(gdm_ctx *ctx, const double *r, int64_t m, void *out);
size_t gdm_ff_target_bytes(int64_t m);
size_t gdm_ff_scratch_bytes(int64_t n);

// Near fields by repropagation. The Green sums run in double-float arithmetic on the FP32 pipes (the
// refinement residual's kernel with separate evaluation points and both field blocks); GDM_NEARFIELD_FP64
// selects FP64 sums on the FP64 pipe instead.
gdm_status gdm_launch_nearfield(gdm_ctx *ctx, const gdm_problem *p, const double *F, const double *r_eval, int64_t m,
                                const double *F0_eval, int n_rhs, double *E_out, double *H_out) {
    const int64_t n = p->n;
    const int kind = p->kind;
    double k0 = gdm_k0(p), k = sqrt(p->eps_env) * k0;
    double d3_4pi = kind == 3 ? p->step * p->step * p->step / (4.0 * PI_D) : 0.0;
    const bool ff = !getenv("GDM_NEARFIELD_FP64");
    size_t need = ScratchCarver::round((size_t)kind * n * n_rhs * sizeof(double2)) +
                  ScratchCarver::round(gdm_green_partial_bytes(ctx, m, n, 6)) + 1024;
    if (ff) need += ScratchCarver::round(gdm_ff_scratch_bytes(n)) + ScratchCarver::round(gdm_ff_target_bytes(m));
    void *ws;
    GDM_TRY(gdm_scratch(ctx, need, &ws));
    ScratchCarver sc(ws);
    double2 *Pbuf = sc.take<double2>((size_t)kind * n * n_rhs);
    double2 *partial = sc.take<double2>(gdm_green_partial_bytes(ctx, m, n, 6) / sizeof(double2));
    void *ffws = ff ? sc.take<char>(gdm_ff_scratch_bytes(n)) : nullptr;
    void *tgt = ff ? sc.take<char>(gdm_ff_target_bytes(m)) : nullptr;
    dim3 g1((unsigned)((n + 127) / 128), (unsigned)n_rhs);
    k_moments<<<g1, 128, 0, ctx->stream>>>((const double2 *)F, n, kind, n_rhs, (const double2 *)p->eps, p->eps_env,
                                            d3_4pi, (const double2 *)p->alpha6, 0, Pbuf);
    GDM_LAUNCHED(ctx, "moments");
    if (ff) GDM_TRY(gdm_ff_targets(ctx, r_eval, m, tgt));
    for (int q0 = 0; q0 < n_rhs; q0 += 2) {
        int nr = n_rhs - q0 < 2 ? n_rhs - q0 : 2;
        int nc;
        if (ff) {
            int64_t chunk;
            green_grid(ctx, m, n, gdm_ff_occupancy(kind, 6, nr), &chunk, &nc);
            GDM_TRY(gdm_ff_green_sum(ctx, p, tgt, m, 6, Pbuf, q0, nr, chunk, nc, ffws, partial, q0 == 0));
        } else if (kind == 3)
            GDM_TRY(launch_green_sum<3, 6>(ctx, r_eval, m, p->pos, Pbuf, n, q0, nr, k, k0, 1.0 / p->eps_env, 0,
                                           partial, &nc));
        else
            GDM_TRY(launch_green_sum<6, 6>(ctx, r_eval, m, p->pos, Pbuf, n, q0, nr, k, k, 1.0, 0, partial, &nc));
        // rows: ED/MD sums use the vacuum-form dyad (E / eps_env, H / n_env); the cells' double-float cross
        // term carries the 1/eps_env of the E kernel, so G^Hp p = n_env times it
        double sE = 1.0, sH = 1.0;
        if (kind == 6) {
            sE = 1.0 / p->eps_env;
            sH = 1.0 / sqrt(p->eps_env);
        } else if (ff) {
            sH = sqrt(p->eps_env);
        }
        k_nearfield_finalize<6><<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(
            partial, nc, m, q0, nr, (const double2 *)F0_eval, n_rhs, sE, sH, (double2 *)E_out, (double2 *)H_out);
        GDM_LAUNCHED(ctx, "nearfield_finalize");
    }
    return GDM_OK;
}

// ================================================================== far field
// f(rhat) = k^2/eps_env sum_j exp(-i k rhat.r_j) [p_j - rhat (rhat.p_j) - rhat x (n_env m_j)] for q directions
// (the moment buffer holds n_env m_j); one
// thread per direction, sources staged through shared memory, FP64. Optional quadrature: per CTA the
// weighted sum of |f|^2 per RHS (partials for a deterministic final reduction).
#define FF_T 128
#define FF_S 64
template <int KIND, int NR>
__global__ void __launch_bounds__(FF_T) k_farfield(const double *__restrict__ dirs, int64_t q, const double *__restrict__ pos,
                                                  const double2 *__restrict__ P, int64_t n, int rhs0, int nr_here,
                                                  double k, double pref, double2 *__restrict__ f_out, int64_t n_rhs_out,
                                                  const double *__restrict__ wts, double *__restrict__ part) {
    __shared__ double sp[FF_S][3];
    __shared__ double2 sm[FF_S][KIND][NR];
    const int64_t t = blockIdx.x * (int64_t)FF_T + threadIdx.x;
    const bool valid = t < q;
    double rx = 0, ry = 0, rz = 1;
    if (valid) {
        rx = dirs[3 * t];
        ry = dirs[3 * t + 1];
        rz = dirs[3 * t + 2];
    }
    double2 acc[NR][KIND];
#pragma unroll
    for (int r = 0; r < NR; r++)
#pragma unroll
        for (int a = 0; a < KIND; a++) acc[r][a] = make_double2(0.0, 0.0);
    const int64_t ld = (int64_t)KIND * n;
    for (int64_t s0 = 0; s0 < n; s0 += FF_S) {
        const int sn = (int)min((int64_t)FF_S, n - s0);
        __syncthreads();
        for (int e = threadIdx.x; e < sn * 3; e += FF_T) sp[e / 3][e % 3] = pos[3 * s0 + e];
        for (int e = threadIdx.x; e < sn * KIND * NR; e += FF_T) {
            const int jj = e / (KIND * NR), rem = e % (KIND * NR), a = rem / NR, r = rem % NR;
            sm[jj][a][r] = (r < nr_here) ? P[(rhs0 + r) * ld + KIND * (s0 + jj) + a] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        if (valid)
            for (int jj = 0; jj < sn; jj++) {
                double sn_, cs_;
                sincos(-k * (rx * sp[jj][0] + ry * sp[jj][1] + rz * sp[jj][2]), &sn_, &cs_);
                const double2 e = make_double2(cs_, sn_);
#pragma unroll
                for (int r = 0; r < NR; r++)
#pragma unroll
                    for (int a = 0; a < KIND; a++) acc[r][a] = cadd(acc[r][a], cmul(e, sm[jj][a][r]));
            }
    }
    double w2[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) {
        w2[r] = 0.0;
        if (!valid || r >= nr_here) continue;
        const double2 *p = acc[r];
        const double2 rp = cadd(cadd(cscale(p[0], rx), cscale(p[1], ry)), cscale(p[2], rz));
        double2 f[3] = {csub(p[0], cscale(rp, rx)), csub(p[1], cscale(rp, ry)), csub(p[2], cscale(rp, rz))};
        if (KIND == 6) {  // - rhat x m
            const double2 *m = acc[r] + 3;
            f[0] = csub(f[0], csub(cscale(m[2], ry), cscale(m[1], rz)));
            f[1] = csub(f[1], csub(cscale(m[0], rz), cscale(m[2], rx)));
            f[2] = csub(f[2], csub(cscale(m[1], rx), cscale(m[0], ry)));
        }
        double s2 = 0.0;
        for (int a = 0; a < 3; a++) {
            f[a] = cscale(f[a], pref);
            s2 += f[a].x * f[a].x + f[a].y * f[a].y;
            if (f_out) f_out[(int64_t)(rhs0 + r) * 3 * q + 3 * t + a] = f[a];
        }
        if (wts) w2[r] = wts[t] * s2;
    }
    if (part) {
        __shared__ double red[NR][FF_T / 32];
#pragma unroll
        for (int r = 0; r < NR; r++) {
            double v = w2[r];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) red[r][threadIdx.x >> 5] = v;
        }
        __syncthreads();
        if (threadIdx.x < NR) {
            double v = 0.0;
            for (int w = 0; w < FF_T / 32; w++) v += red[threadIdx.x][w];
            part[(int64_t)(rhs0 + threadIdx.x) * gridDim.x + blockIdx.x] = v;
        }
    }
}

__global__ void k_farfield_sum(const double *__restrict__ part, int nb, int n_rhs, const double *__restrict__ inv_e2,
                               double *sigma) {
    const int r = blockIdx.x;
    if (r >= n_rhs) return;
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) v += part[(int64_t)r * nb + b];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) sigma[r] = v * inv_e2[r];
}

gdm_status gdm_launch_farfield(gdm_ctx *ctx, const gdm_problem *p, const double *F, int n_rhs, const double *dirs,
                               int64_t q, double *f_out, const double *wts, const double *inv_e2, double *sigma) {
    const int64_t n = p->n;
    const int kind = p->kind;
    const double k = sqrt(p->eps_env) * gdm_k0(p);
    const double d3_4pi = kind == 3 ? p->step * p->step * p->step / (4.0 * PI_D) : 0.0;
    const unsigned nb = (unsigned)((q + FF_T - 1) / FF_T);
    size_t need = ScratchCarver::round((size_t)kind * n * n_rhs * sizeof(double2)) +
                  ScratchCarver::round((size_t)nb * n_rhs * sizeof(double)) + 1024;
    void *ws;
    GDM_TRY(gdm_scratch(ctx, need, &ws));
    ScratchCarver sc(ws);
    double2 *Pbuf = sc.take<double2>((size_t)kind * n * n_rhs);
    double *part = sc.take<double>((size_t)nb * n_rhs);
    dim3 g1((unsigned)((n + 127) / 128), (unsigned)n_rhs);
    k_moments<<<g1, 128, 0, ctx->stream>>>((const double2 *)F, n, kind, n_rhs, (const double2 *)p->eps, p->eps_env,
                                            d3_4pi, (const double2 *)p->alpha6, 0, Pbuf);
    GDM_LAUNCHED(ctx, "moments");
    const double pref = k * k / p->eps_env;
    double *pt = wts ? part : nullptr;
    for (int q0 = 0; q0 < n_rhs; q0 += 2) {
        const int nr = n_rhs - q0 < 2 ? n_rhs - q0 : 2;
        if (kind == 3) {
            if (nr == 2)
                k_farfield<3, 2><<<nb, FF_T, 0, ctx->stream>>>(dirs, q, p->pos, Pbuf, n, q0, nr, k, pref,
                                                               (double2 *)f_out, n_rhs, wts, pt);
            else
                k_farfield<3, 1><<<nb, FF_T, 0, ctx->stream>>>(dirs, q, p->pos, Pbuf, n, q0, nr, k, pref,
                                                               (double2 *)f_out, n_rhs, wts, pt);
        } else {
            if (nr == 2)
                k_farfield<6, 2><<<nb, FF_T, 0, ctx->stream>>>(dirs, q, p->pos, Pbuf, n, q0, nr, k, pref,
                                                               (double2 *)f_out, n_rhs, wts, pt);
            else
                k_farfield<6, 1><<<nb, FF_T, 0, ctx->stream>>>(dirs, q, p->pos, Pbuf, n, q0, nr, k, pref,
                                                               (double2 *)f_out, n_rhs, wts, pt);
        }
        GDM_LAUNCHED(ctx, "farfield");
    }
    if (wts) {
        k_farfield_sum<<<n_rhs, 32, 0, ctx->stream>>>(part, (int)nb, n_rhs, inv_e2, sigma);
        GDM_LAUNCHED(ctx, "farfield_sum");
    }
    return GDM_OK;
}

// ================================================================== cross sections
#define XS_BS 256
__global__ void k_xsec_partial(const double2 *__restrict__ F0, const double2 *__restrict__ F, int64_t n, int kind,
                               const double2 *__restrict__ eps, double eps_env, double d3_4pi,
                               const double2 *__restrict__ alpha6, double rad_e, double rad_m,
                               double *__restrict__ part) {
    int q = blockIdx.y;
    int64_t i = blockIdx.x * (int64_t)XS_BS + threadIdx.x;
    double se = 0.0, sa = 0.0;
    if (i < n) {
        int64_t off = (int64_t)q * kind * n + kind * i;
        const double2 *f0 = F0 + off;
        const double2 *f = F + off;
        double2 pm[6];
        if (kind == 3) {
            double2 al = make_double2((eps[i].x - eps_env) * d3_4pi, eps[i].y * d3_4pi);
            for (int a = 0; a < 3; a++) pm[a] = cmul(al, f[a]);
        } else {
            const double2 *al = alpha6 + 36 * i;
            for (int a = 0; a < 6; a++) {
                double2 s = make_double2(0.0, 0.0);
                for (int b = 0; b < 6; b++) cfma(s, al[6 * a + b], f[b]);
                pm[a] = s;
            }
        }
        for (int a = 0; a < kind; a++) {
            se += cconjmul(f0[a], pm[a]).y;
            sa += cconjmul(f[a], pm[a]).y;
            if (kind == 6) sa -= (a < 3 ? rad_e : rad_m) * (pm[a].x * pm[a].x + pm[a].y * pm[a].y);
        }
    }
    __shared__ double red[2][XS_BS / 32];
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_down_sync(0xffffffffu, se, o);
        sa += __shfl_down_sync(0xffffffffu, sa, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = se;
        red[1][threadIdx.x >> 5] = sa;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0;
        for (int w = 0; w < XS_BS / 32; w++) {
            a0 += red[0][w];
            a1 += red[1][w];
        }
        part[((int64_t)q * gridDim.x + blockIdx.x) * 2] = a0;
        part[((int64_t)q * gridDim.x + blockIdx.x) * 2 + 1] = a1;
    }
}

__global__ void k_xsec_final(const double *__restrict__ part, int nblocks, int n_rhs, const double *__restrict__ pref,
                             double *ext, double *sca, double *abs_) {
    int q = blockIdx.x;
    if (q >= n_rhs) return;
    double a0 = 0.0, a1 = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 32) {
        a0 += part[((int64_t)q * nblocks + b) * 2];
        a1 += part[((int64_t)q * nblocks + b) * 2 + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_down_sync(0xffffffffu, a0, o);
        a1 += __shfl_down_sync(0xffffffffu, a1, o);
    }
    if (threadIdx.x == 0) {
        double e = pref[q] * a0, ab = pref[q] * a1;
        if (ext) ext[q] = e;
        if (abs_) abs_[q] = ab;
        if (sca) sca[q] = e - ab;
    }
}

gdm_status gdm_launch_cross_sections(gdm_ctx *ctx, const gdm_problem *p, const double *F0, const double *F, int n_rhs,
                                     const double *e0_norm2, double *ext, double *sca, double *abs) {
    const int64_t n = p->n;
    double k = sqrt(p->eps_env) * gdm_k0(p);
    double d3_4pi = p->kind == 3 ? p->step * p->step * p->step / (4.0 * PI_D) : 0.0;
    double pref[64];
    for (int q = 0; q < n_rhs; q++) pref[q] = 4.0 * PI_D * k / (p->eps_env * e0_norm2[q]);
    double *dpref;
    GDM_TRY(gdm_upload(ctx, pref, sizeof(double) * n_rhs, (void **)&dpref));
    unsigned nb = (unsigned)((n + XS_BS - 1) / XS_BS);
    void *ws;
    GDM_TRY(gdm_scratch(ctx, (size_t)nb * n_rhs * 2 * sizeof(double) + 256, &ws));
    double *part = (double *)ws;
    // radiated power of the ED/MD dipoles in the host: (2/3) k^3/eps_env |p|^2 and (2/3) k^3 |m|^2
    const double rad = (2.0 / 3.0) * k * k * k;
    k_xsec_partial<<<dim3(nb, n_rhs), XS_BS, 0, ctx->stream>>>((const double2 *)F0, (const double2 *)F, n, p->kind,
                                                               (const double2 *)p->eps, p->eps_env, d3_4pi,
                                                               (const double2 *)p->alpha6, rad / p->eps_env, rad,
                                                               part);
    GDM_LAUNCHED(ctx, "xsec_partial");
    k_xsec_final<<<n_rhs, 32, 0, ctx->stream>>>(part, (int)nb, n_rhs, dpref, ext, sca, abs);
    GDM_LAUNCHED(ctx, "xsec_final");
    return GDM_OK;
}

// ------------------------------------------------------------------ cross sections without allocation
// A variant of the launcher above for callers that must not allocate device memory: a step that runs
// while another allocator (a PyTorch caching allocator at its limit, say) holds the free memory, or a
// latency-bound loop that cannot afford cudaMalloc/cudaFree, which may synchronise the whole device.
// The partial sums go to one fixed file-scope buffer per device instead of the context's growing
// workspace, and the prefactors travel as a kernel argument instead of through the parameter buffer.
// Every slot the final kernel reads is written earlier on the same stream by k_xsec_partial, so nothing
// in the buffer needs to start at zero. The buffer is shared by all contexts and streams of a device:
// calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_xsec_static_part[2 * GDM_XSEC_NOALLOC_MAX_PARTS];

namespace {
struct XsecPref {
    double v[64];
};

__global__ void k_xsec_final_pref(const double *__restrict__ part, int nblocks, int n_rhs, XsecPref pref, double *ext,
                                  double *sca, double *abs_) {
    int q = blockIdx.x;
    if (q >= n_rhs) return;
    double a0 = 0.0, a1 = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 32) {
        a0 += part[((int64_t)q * nblocks + b) * 2];
        a1 += part[((int64_t)q * nblocks + b) * 2 + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_down_sync(0xffffffffu, a0, o);
        a1 += __shfl_down_sync(0xffffffffu, a1, o);
    }
    if (threadIdx.x == 0) {
        double e = pref.v[q] * a0, ab = pref.v[q] * a1;
        if (ext) ext[q] = e;
        if (abs_) abs_[q] = ab;
        if (sca) sca[q] = e - ab;
    }
}

// device address of g_xsec_static_part, looked up once per device (with that device current)
#define GDM_XSEC_MAX_DEVICES 64
std::mutex g_xsec_mu;
double *g_xsec_ptr[GDM_XSEC_MAX_DEVICES];
}  // namespace

gdm_status gdm_launch_cross_sections_noalloc(gdm_ctx *ctx, const gdm_problem *p, const double *F0, const double *F,
                                             int n_rhs, const double *e0_norm2, double *ext, double *sca,
                                             double *abs) {
    const int64_t n = p->n;
    const int64_t nb = (n + XS_BS - 1) / XS_BS;
    if (nb * n_rhs > GDM_XSEC_NOALLOC_MAX_PARTS)
        return gdm_fail(ctx, GDM_ERR_SHAPE,
                        "gdm_cross_sections_noalloc: ceil(n/%d) * n_rhs = %lld exceeds its fixed scratch of %d "
                        "partial sums (n = %lld, n_rhs = %d); use gdm_cross_sections",
                        XS_BS, (long long)(nb * n_rhs), GDM_XSEC_NOALLOC_MAX_PARTS, (long long)n, n_rhs);
    if (ctx->device < 0 || ctx->device >= GDM_XSEC_MAX_DEVICES)
        return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "gdm_cross_sections_noalloc: device ordinal %d >= %d", ctx->device,
                        GDM_XSEC_MAX_DEVICES);
    double *part;
    {
        std::lock_guard<std::mutex> lock(g_xsec_mu);
        if (!g_xsec_ptr[ctx->device]) {
            void *addr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&addr, g_xsec_static_part);
            if (e != cudaSuccess || !addr)
                return gdm_fail(ctx, GDM_ERR_CUDA, "gdm_cross_sections_noalloc: cudaGetSymbolAddress failed: %s",
                                cudaGetErrorString(e));
            g_xsec_ptr[ctx->device] = (double *)addr;
        }
        part = g_xsec_ptr[ctx->device];
    }
    const double k = sqrt(p->eps_env) * gdm_k0(p);
    const double d3_4pi = p->kind == 3 ? p->step * p->step * p->step / (4.0 * PI_D) : 0.0;
    XsecPref pref;
    for (int q = 0; q < n_rhs; q++) pref.v[q] = 4.0 * PI_D * k / (p->eps_env * e0_norm2[q]);
    const double rad = (2.0 / 3.0) * k * k * k;
    k_xsec_partial<<<dim3((unsigned)nb, n_rhs), XS_BS, 0, ctx->stream>>>(
        (const double2 *)F0, (const double2 *)F, n, p->kind, (const double2 *)p->eps, p->eps_env, d3_4pi,
        (const double2 *)p->alpha6, rad / p->eps_env, rad, part);
    GDM_LAUNCHED(ctx, "xsec_partial");
    k_xsec_final_pref<<<n_rhs, 32, 0, ctx->stream>>>(part, (int)nb, n_rhs, pref, ext, sca, abs);
    GDM_LAUNCHED(ctx, "xsec_final_pref");
    return GDM_OK;
}

// ================================================================== grouped refinement residual of a batch
namespace {
// P = alpha X of every listed problem (cells): ceil(3n nr / 256) CTAs of 256 per problem
__global__ void __launch_bounds__(256) k_gr_moments(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                    const int *__restrict__ prefix, int na) {
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const GrItem &g = items[i];
    const int64_t ld = 3 * g.n, e = (int64_t)local * 256 + threadIdx.x;
    if (e >= ld * g.nr) return;
    const int64_t c = e % ld, q = e / ld, cell = c / 3;
    const double2 ep = g.eps[cell];
    const double2 al = make_double2((ep.x - g.eps_env) * g.d3_4pi, ep.y * g.d3_4pi);
    g.P[q * ld + c] = cmul(al, g.X[q * ld + c]);
}

// the first refinement steps' FP32 sums: ceil(n / GS_T) target blocks x nc chunks per problem
__global__ void __launch_bounds__(GS_T) k_gr_green_f32(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                       const int *__restrict__ prefix, int na) {
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const GrItem &g = items[i];
    const int64_t tb = (g.n + GS_T - 1) / GS_T;
    green_sum_f32_body<2>((const DipF *)g.dip, g.n, g.P, 0, g.nr, g.khi, g.klo, g.inv_eps, g.chunk, g.partial,
                          local % tb, local / tb);
}

// r = rhs - X + (G P + S P) and ||r_q||^2: ceil(n / 256) CTAs of 256 per problem
__global__ void __launch_bounds__(256) k_gr_finalize(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                     const int *__restrict__ prefix, int na) {
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const GrItem &g = items[i];
    residual_finalize_body<3, 2>(g.partial, g.nc, g.n, 0, g.nr, g.rhs, g.X, g.P, g.self_S, 0, g.eps, g.eps_env,
                                 g.d3_4pi, 1.0, 1.0, g.r, g.norms + 4, local);
}
}  // namespace

gdm_status gdm_gr_moments(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units) {
    if (units <= 0) return GDM_OK;
    k_gr_moments<<<(unsigned)units, 256, 0, ctx->stream>>>(it, list, prefix, na);
    GDM_LAUNCHED(ctx, "gr_moments");
    return GDM_OK;
}

gdm_status gdm_gr_green_f32(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units) {
    if (units <= 0) return GDM_OK;
    k_gr_green_f32<<<(unsigned)units, GS_T, 0, ctx->stream>>>(it, list, prefix, na);
    GDM_LAUNCHED(ctx, "gr_green_f32");
    return GDM_OK;
}

gdm_status gdm_gr_finalize(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units) {
    if (units <= 0) return GDM_OK;
    k_gr_finalize<<<(unsigned)units, 256, 0, ctx->stream>>>(it, list, prefix, na);
    GDM_LAUNCHED(ctx, "gr_finalize");
    return GDM_OK;
}

// ================================================================== grouped inputs and cross sections of a batch
namespace {
// plane wave E0 = e0 exp(i k khat . r) at every cell of the listed problems that carry amplitudes:
// ceil(n / 256) CTAs per problem
__global__ void __launch_bounds__(256) k_gr_planewave(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                      const int *__restrict__ prefix, int na) {
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const GrItem &g = items[i];
    const int64_t c = (int64_t)local * 256 + threadIdx.x;
    if (!g.has_e0 || c >= g.n) return;
    const double ph = g.k * (g.khat[0] * g.pos[3 * c] + g.khat[1] * g.pos[3 * c + 1] + g.khat[2] * g.pos[3 * c + 2]);
    double sn, cs;
    sincos(ph, &sn, &cs);
    const double2 e = make_double2(cs, sn);
    const int64_t ld = 3 * g.n;
    double2 *F0 = (double2 *)g.rhs;  // written here, read by the refinement
    for (int q = 0; q < g.nr; q++)
        for (int a = 0; a < 3; a++)
            F0[q * ld + 3 * c + a] = cmul(make_double2(g.e0[6 * q + 2 * a], g.e0[6 * q + 2 * a + 1]), e);
}

// FP32 assembly records (positions as FP32 pairs, alpha, 1 - S alpha): ceil(n / 256) CTAs per problem
__global__ void __launch_bounds__(256) k_gr_prep_dipa(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                      const int *__restrict__ prefix, int na) {
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const GrItem &g = items[i];
    const int64_t c = (int64_t)local * 256 + threadIdx.x;
    if (c >= g.n) return;
    DipF d;
    const double x = g.pos[3 * c], y = g.pos[3 * c + 1], z = g.pos[3 * c + 2];
    d.xh = (float)x;
    d.yh = (float)y;
    d.zh = (float)z;
    d.xl = (float)(x - (double)d.xh);
    d.yl = (float)(y - (double)d.yh);
    d.zl = (float)(z - (double)d.zh);
    const double2 e = g.eps[c];
    d.alpha = make_float2((float)((e.x - g.eps_env) * g.d3_4pi), (float)(e.y * g.d3_4pi));
    d.diag = make_float2((float)(1.0 + (e.x - g.eps_env) / (3.0 * g.eps_env)), (float)(e.y / (3.0 * g.eps_env)));
    d.pad[0] = d.pad[1] = 0.f;
    ((DipF *)g.dipa)[c] = d;
}

// A = I - G alpha in complex64 through the bulk-copy tiles: ceil(n / ASB_TI) x ceil(n / ASB_TJ) CTAs per problem
__global__ void __launch_bounds__(ASB_TI) k_gr_assemble(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                        const int *__restrict__ prefix, int na) {
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const GrItem &g = items[i];
    const int64_t tb = (g.n + ASB_TI - 1) / ASB_TI;
    assemble3_f32_bulk_body((float2 *)g.A, g.lda, g.n, (const DipF *)g.dipa, g.khi, g.klo, g.inv_eps, local % tb,
                            local / tb);
}

// sum Im(E0* . p) and sum Im(E* . p) per right-hand side into xs (zeroed before): ceil(n / XS_BS) CTAs per problem
__global__ void __launch_bounds__(XS_BS) k_gr_xsec_partial(const GrItem *__restrict__ items, const int *__restrict__ list,
                                                           const int *__restrict__ prefix, int na) {
    __shared__ double red[4][XS_BS / 32];
    int local;
    const int i = gr_unit(list, prefix, na, (int)blockIdx.x, &local);
    const GrItem &g = items[i];
    const int64_t c = (int64_t)local * XS_BS + threadIdx.x;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    if (c < g.n) {
        const double2 e = g.eps[c];
        const double2 al = make_double2((e.x - g.eps_env) * g.d3_4pi, e.y * g.d3_4pi);
        for (int q = 0; q < g.nr; q++) {
            const int64_t off = q * 3 * g.n + 3 * c;
            for (int a = 0; a < 3; a++) {
                const double2 pm = cmul(al, g.X[off + a]);
                s[2 * q] += cconjmul(g.rhs[off + a], pm).y;
                s[2 * q + 1] += cconjmul(g.X[off + a], pm).y;
            }
        }
    }
    for (int v = 0; v < 4; v++) {
        double x = s[v];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[v][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double x = 0.0;
        for (int w = 0; w < XS_BS / 32; w++) x += red[threadIdx.x][w];
        if (threadIdx.x < 2 * g.nr) atomicAdd(&g.xs[threadIdx.x], x);
    }
}

// ext, sca, abs of every listed problem with cross sections: one thread per problem
__global__ void k_gr_xsec_final(const GrItem *__restrict__ items, const int *__restrict__ list, int na) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    const GrItem &g = items[list[k]];
    if (!g.has_sigma) return;
    for (int q = 0; q < g.nr; q++) {
        const double e = g.pref[q] * g.xs[2 * q], ab = g.pref[q] * g.xs[2 * q + 1];
        g.sigma[q] = e;
        g.sigma[g.nr + q] = e - ab;
        g.sigma[2 * g.nr + q] = ab;
    }
}
}  // namespace

gdm_status gdm_gr_planewave(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units) {
    if (units <= 0) return GDM_OK;
    k_gr_planewave<<<(unsigned)units, 256, 0, ctx->stream>>>(it, list, prefix, na);
    GDM_LAUNCHED(ctx, "gr_planewave");
    return GDM_OK;
}

gdm_status gdm_gr_prep_dipa(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units) {
    if (units <= 0) return GDM_OK;
    k_gr_prep_dipa<<<(unsigned)units, 256, 0, ctx->stream>>>(it, list, prefix, na);
    GDM_LAUNCHED(ctx, "gr_prep_dipa");
    return GDM_OK;
}

gdm_status gdm_gr_assemble(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na, int units) {
    if (units <= 0) return GDM_OK;
    const int smem = 3 * ASB_TJ * ASB_ROWS * (int)sizeof(float2);
    static bool attr = false;
    if (!attr) {
        GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_gr_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = true;
    }
    k_gr_assemble<<<(unsigned)units, ASB_TI, smem, ctx->stream>>>(it, list, prefix, na);
    GDM_LAUNCHED(ctx, "gr_assemble");
    return GDM_OK;
}

gdm_status gdm_gr_xsec_partial(gdm_ctx *ctx, const GrItem *it, const int *list, const int *prefix, int na,
                               int units) {
    if (units <= 0) return GDM_OK;
    k_gr_xsec_partial<<<(unsigned)units, XS_BS, 0, ctx->stream>>>(it, list, prefix, na);
    GDM_LAUNCHED(ctx, "gr_xsec_partial");
    return GDM_OK;
}

gdm_status gdm_gr_xsec_final(gdm_ctx *ctx, const GrItem *it, const int *list, int na) {
    if (na <= 0) return GDM_OK;
    k_gr_xsec_final<<<(unsigned)((na + 127) / 128), 128, 0, ctx->stream>>>(it, list, na);
    GDM_LAUNCHED(ctx, "gr_xsec_final");
    return GDM_OK;
}
