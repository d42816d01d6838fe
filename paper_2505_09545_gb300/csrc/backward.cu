// Adjoint backward of the GDM solve, cross sections and near field (cells, kind 3).
//
// For A F = F0 with real loss L and g = dL/dF^* (conjugate Wirtinger derivative):
//   A^H mu = g,   dL = 2 Re[mu^H (dF0 - dA F)] + explicit terms,
// following the LU-based solve of Sec. "Numerical solution" (whose derivative the paper obtains by
// automatic differentiation; here the adjoint is written out). With P = alpha F, mub = conj(mu),
// R_lj = r_l - r_j, the pair sums below give (c = x, y, z; symmetric G, odd dG/dR):
//   dL/dr_lc  = 2 Re[ mub_l . sum_j dG_c(R_lj) P_j + P_l . sum_j dG_c(R_lj) mub_j + mub_l . (i k khat_c E0_l) ] + sigma terms
//   dL/dalpha_l = 2 F_l . (G mub)_l (+ sigma terms)            (alpha = (eps - eps_env) d^3 / (4 pi))
//   dL/dk     = 2 Re[ mub . (i (khat.r) E0) + mub . sum_j dG_k P_j ] + sigma terms;  dk/dlambda = -k/lambda.
// Near field E_m = E0(r_m) + sum_j G(r_m - r_j) P_j with gE = dL/dE^*: pair sums over evaluation points with
// sources conj(gE_m) give dL/dF^*, dL/deps, dL/dr and dL/dk the same way.
#include <math.h>
#include <stdlib.h>

#include "gdm_internal.cuh"

#define PI_D 3.14159265358979323846

size_t gdm_green_partial_bytes(gdm_ctx *ctx, int64_t m, int64_t n, int out);
size_t gdm_ff_scratch_bytes(int64_t n);
gdm_status gdm_ff_prepare(gdm_ctx *ctx, const gdm_problem *p, void *ffws);
gdm_status gdm_ff_dgreen_sum(gdm_ctx *ctx, const gdm_problem *p, const double2 *S, int q, int conj, int qslot,
                             int64_t chunk, int nchunks, void *ffws, double2 *partial);
int gdm_ff_dgreen_occupancy();


namespace {

#define DG_T 128
#define DG_S 32
#define DG_OUT 15  // G s (3), dG_x s, dG_y s, dG_z s (3 each), dG_k s (3)

// per pair: G s, dG_c s, dG_k s for the electric dyad G^Ep (eps_env medium)
__device__ __forceinline__ void pair_dgreen(double dx, double dy, double dz, double k, double inv_eps,
                                            const double2 *s, double2 *out /*[15]*/) {
    double r2 = dx * dx + dy * dy + dz * dz;
    double r1 = rsqrt(r2);
    double r = r2 * r1;
    double ri2 = r1 * r1, ri3 = ri2 * r1, ri4 = ri2 * ri2;
    double sn, cs;
    sincos(k * r, &sn, &cs);
    double2 e = make_double2(cs * inv_eps, sn * inv_eps);
    double k2 = k * k;
    double2 a = cmul(e, make_double2(k2 * r1 - ri3, k * ri2));
    double2 b = cmul(e, make_double2(3.0 * ri3 - k2 * r1, -3.0 * k * ri2));
    double2 ik = make_double2(0.0, k);
    double2 da = cadd(cmul(ik, a), cmul(e, make_double2(-k2 * ri2 + 3.0 * ri4, -2.0 * k * ri3)));
    double2 db = cadd(cmul(ik, b), cmul(e, make_double2(k2 * ri2 - 9.0 * ri4, 6.0 * k * ri3)));
    double2 ir = make_double2(0.0, r);
    double2 dka = cadd(cmul(ir, a), cmul(e, make_double2(2.0 * k * r1, ri2)));
    double2 dkb = cadd(cmul(ir, b), cmul(e, make_double2(-2.0 * k * r1, -3.0 * ri2)));
    double u[3] = {dx * r1, dy * r1, dz * r1};
    double2 us;  // u . s
    us.x = u[0] * s[0].x + u[1] * s[1].x + u[2] * s[2].x;
    us.y = u[0] * s[0].y + u[1] * s[1].y + u[2] * s[2].y;
    double2 bus = cmul(b, us), dbus = cmul(db, us), dkbus = cmul(dkb, us);
    double2 bor = cscale(b, r1);
#pragma unroll
    for (int aa = 0; aa < 3; aa++) {
        out[aa] = cadd(out[aa], cadd(cmul(a, s[aa]), cscale(bus, u[aa])));
        out[12 + aa] = cadd(out[12 + aa], cadd(cmul(dka, s[aa]), cscale(dkbus, u[aa])));
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
#pragma unroll
        for (int aa = 0; aa < 3; aa++) {
            // u_c [da s_a + db u_a (u.s)] + (b/r) [delta_ca (u.s) + u_a s_c - 2 u_c u_a (u.s)]
            double2 t1 = cadd(cmul(da, s[aa]), cscale(dbus, u[aa]));
            double2 t2 = cadd(cscale(s[c], u[aa]), cscale(us, (c == aa ? 1.0 : 0.0) - 2.0 * u[c] * u[aa]));
            out[3 + 3 * c + aa] = cadd(out[3 + 3 * c + aa], cadd(cscale(t1, u[c]), cmul(bor, t2)));
        }
    }
}

// partial[c][q][t][15] over sources of chunk c; sources: positions spos, vectors S (3*nsrc per RHS column),
// optionally conjugated on load (conj_src).
template <int NR>
__global__ void __launch_bounds__(DG_T) k_dgreen_sum(const double *__restrict__ tpos, int64_t m,
                                                    const double *__restrict__ spos, const double2 *__restrict__ S,
                                                    int64_t nsrc, int rhs0, int nr_here, int conj_src, double k,
                                                    double inv_eps, int64_t chunk, int self_exclude,
                                                    double2 *__restrict__ partial) {
    __shared__ double sp[DG_S][3];
    __shared__ double2 sv[DG_S][3][NR];
    const int64_t t = (int64_t)blockIdx.x * DG_T + threadIdx.x;
    const bool valid = t < m;
    const int64_t c = blockIdx.y;
    const int64_t jb = c * chunk, je = min(nsrc, jb + chunk);
    double tx = 0, ty = 0, tz = 0;
    if (valid) {
        tx = tpos[3 * t];
        ty = tpos[3 * t + 1];
        tz = tpos[3 * t + 2];
    }
    double2 acc[NR][DG_OUT];
#pragma unroll
    for (int q = 0; q < NR; q++)
#pragma unroll
        for (int a = 0; a < DG_OUT; a++) acc[q][a] = make_double2(0.0, 0.0);
    const int64_t ld = 3 * nsrc;
    for (int64_t s0 = jb; s0 < je; s0 += DG_S) {
        int sn = (int)min((int64_t)DG_S, je - s0);
        for (int e = threadIdx.x; e < sn * 3; e += DG_T) sp[e / 3][e % 3] = spos[3 * s0 + e];
        for (int e = threadIdx.x; e < sn * 3 * NR; e += DG_T) {
            int jj = e / (3 * NR), rem = e % (3 * NR), a = rem / NR, q = rem % NR;
            double2 v = make_double2(0.0, 0.0);
            if (q < nr_here) v = S[(rhs0 + q) * ld + 3 * (s0 + jj) + a];
            if (conj_src) v.y = -v.y;
            sv[jj][a][q] = v;
        }
        __syncthreads();
        if (valid) {
            for (int jj = 0; jj < sn; jj++) {
                if (self_exclude && s0 + jj == t) continue;
                double dx = tx - sp[jj][0], dy = ty - sp[jj][1], dz = tz - sp[jj][2];
#pragma unroll
                for (int q = 0; q < NR; q++) {
                    double2 s[3] = {sv[jj][0][q], sv[jj][1][q], sv[jj][2][q]};
                    pair_dgreen(dx, dy, dz, k, inv_eps, s, acc[q]);
                }
            }
        }
        __syncthreads();
    }
    if (!valid) return;
#pragma unroll
    for (int q = 0; q < NR; q++) {
        if (q >= nr_here) break;
        double2 *o = partial + ((c * 2 + q) * m + t) * DG_OUT;  // chunk stride of two RHS for any NR
#pragma unroll
        for (int a = 0; a < DG_OUT; a++) o[a] = acc[q][a];
    }
}

void dg_grid(gdm_ctx *ctx, int64_t m, int64_t n, int64_t *chunk, int *nchunks) {
    int64_t tb = (m + DG_T - 1) / DG_T;
    int64_t want = (4 * (int64_t)ctx->sm_count + tb - 1) / tb;
    int64_t maxc = (n + DG_S - 1) / DG_S;
    int64_t nc = want < 1 ? 1 : (want > maxc ? maxc : want);
    if (nc > 64) nc = 64;
    int64_t ch = (n + nc - 1) / nc;
    ch = (ch + DG_S - 1) / DG_S * DG_S;
    *chunk = ch;
    *nchunks = (int)((n + ch - 1) / ch);
}

size_t dg_partial_bytes(gdm_ctx *ctx, int64_t m, int64_t n) {
    int64_t ch;
    int nc;
    dg_grid(ctx, m, n, &ch, &nc);
    return (size_t)nc * 2 * m * DG_OUT * sizeof(double2);
}

// chunking of the double-float gradient sums: at most the chunks dg_grid gives (the partial buffers are sized
// by it), chosen so that the last wave of CTAs wastes the fewest resident slots at the kernel's occupancy
void dg_grid_ff(gdm_ctx *ctx, int64_t m, int64_t n, int64_t *chunk, int *nchunks) {
    int64_t ch0;
    int nc_max;
    dg_grid(ctx, m, n, &ch0, &nc_max);
    const int64_t tb = (m + DG_T - 1) / DG_T;
    const int64_t slots = (int64_t)gdm_ff_dgreen_occupancy() * ctx->sm_count;
    double best = -1.0;
    *chunk = ch0;
    *nchunks = nc_max;
    for (int nc = 1; nc <= nc_max; nc++) {
        const int64_t ch = (n + nc - 1) / nc;  // any chunk length: the kernel stages partial tiles
        const int ncr = (int)((n + ch - 1) / ch);
        if (ncr > nc_max) continue;
        const int64_t ctas = tb * ncr, waves = (ctas + slots - 1) / slots;
        const double eff = (double)ctas / (double)(waves * slots);
        if (eff > best + 1e-9) {
            best = eff;
            *chunk = ch;
            *nchunks = ncr;
        }
    }
}

// launch for one RHS pair (q0, q0+1); returns the number of chunks
gdm_status launch_dg(gdm_ctx *ctx, const double *tpos, int64_t m, const double *spos, const double2 *S, int64_t nsrc,
                     int q0, int nr, int conj_src, double k, double inv_eps, int self_exclude, double2 *partial,
                     int *nc_out) {
    int64_t ch;
    int nc;
    dg_grid(ctx, m, nsrc, &ch, &nc);
    dim3 grid((unsigned)((m + DG_T - 1) / DG_T), (unsigned)nc);
    if (nr == 1)
        k_dgreen_sum<1><<<grid, DG_T, 0, ctx->stream>>>(tpos, m, spos, S, nsrc, q0, nr, conj_src, k, inv_eps, ch,
                                                         self_exclude, partial);
    else
        k_dgreen_sum<2><<<grid, DG_T, 0, ctx->stream>>>(tpos, m, spos, S, nsrc, q0, nr, conj_src, k, inv_eps, ch,
                                                         self_exclude, partial);
    GDM_LAUNCHED(ctx, "dgreen_sum");
    *nc_out = nc;
    return GDM_OK;
}

__device__ __forceinline__ double2 sum_partial(const double2 *partial, int nc, int nrs, int q, int64_t m, int64_t t,
                                               int a) {
    double2 s = make_double2(0.0, 0.0);
    for (int c = 0; c < nc; c++) s = cadd(s, partial[((c * nrs + q) * m + t) * DG_OUT + a]);
    return s;
}

struct PW {
    double k, khx, khy, khz;
};
__device__ __forceinline__ void planewave_at(const PW &pw, const double *e0q, double x, double y, double z,
                                             double2 *E0, double *zdot) {
    double ph = pw.k * (pw.khx * x + pw.khy * y + pw.khz * z);
    double s, c;
    sincos(ph, &s, &c);
    double2 e = make_double2(c, s);
    for (int a = 0; a < 3; a++) E0[a] = cmul(make_double2(e0q[2 * a], e0q[2 * a + 1]), e);
    *zdot = pw.khx * x + pw.khy * y + pw.khz * z;
}

__device__ __forceinline__ void block_atomic_add(double v, double *dst) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
        if (s != 0.0) atomicAdd(dst, s);
    }
}

// g = gF + sigma terms (per RHS weights w_ext, w_abs and prefactor c)
__global__ void k_adjoint_rhs(const double2 *__restrict__ F, const double2 *__restrict__ gF, int64_t n, int n_rhs,
                              const double2 *__restrict__ eps, double eps_env, double d3_4pi, const double *__restrict__ e0,
                              PW pw, const double *__restrict__ wts /*[q][3]: w_ext, w_abs, c*/, const double *pos,
                              double2 *__restrict__ g) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int q = blockIdx.y;
    if (i >= n || q >= n_rhs) return;
    double2 al = make_double2((eps[i].x - eps_env) * d3_4pi, eps[i].y * d3_4pi);
    double2 E0[3];
    double zd;
    planewave_at(pw, e0 + 6 * q, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], E0, &zd);
    double wext = wts[3 * q], wabs = wts[3 * q + 1], c = wts[3 * q + 2];
    int64_t off = (int64_t)q * 3 * n + 3 * i;
    for (int a = 0; a < 3; a++) {
        double2 v = gF ? gF[off + a] : make_double2(0.0, 0.0);
        // d sigma_ext / dF^* = (i/2) c conj(alpha) E0 ; d sigma_abs / dF^* = c Im(alpha) F
        double2 t = cmul(make_double2(0.0, 0.5 * c * wext), cmul(conjd(al), E0[a]));
        v = cadd(v, t);
        v = cadd(v, cscale(F[off + a], c * wabs * al.y));
        g[off + a] = v;
    }
}

// gradients from the solve adjoint (partials: A from sources P = alpha F, B from sources conj(mu))
__global__ void k_backward_finalize(const double2 *__restrict__ F, const double2 *__restrict__ mu, int64_t n, int n_rhs,
                                    const double2 *__restrict__ eps, double eps_env, double d3_4pi, double S,
                                    const double *__restrict__ pos, const double *__restrict__ e0, PW pw,
                                    const double *__restrict__ wts, const double2 *__restrict__ partA, int ncA,
                                    const double2 *__restrict__ partB, int ncB, int q0, int nr, double dk_dlambda,
                                    double *grad_pos, double2 *grad_eps, double *grad_lambda) {
    int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double dLdk = 0.0;
    if (l < n) {
        double2 al = make_double2((eps[l].x - eps_env) * d3_4pi, eps[l].y * d3_4pi);
        double gp[3] = {0, 0, 0};
        double2 C = make_double2(0.0, 0.0);
        double kh[3] = {pw.khx, pw.khy, pw.khz};
        for (int qq = 0; qq < nr; qq++) {
            int q = q0 + qq;
            int64_t off = (int64_t)q * 3 * n + 3 * l;
            double2 E0[3];
            double zd;
            planewave_at(pw, e0 + 6 * q, pos[3 * l], pos[3 * l + 1], pos[3 * l + 2], E0, &zd);
            double wext = wts[3 * q], wabs = wts[3 * q + 1], c = wts[3 * q + 2];
            double2 f[3], P[3], mb[3];
            for (int a = 0; a < 3; a++) {
                f[a] = F[off + a];
                P[a] = cmul(al, f[a]);
                mb[a] = conjd(mu[off + a]);
            }
            for (int cc = 0; cc < 3; cc++) {
                double2 s = make_double2(0.0, 0.0);
                for (int a = 0; a < 3; a++) {
                    double2 dgp = sum_partial(partA, ncA, 2, qq, n, l, 3 + 3 * cc + a);
                    double2 dgm = sum_partial(partB, ncB, 2, qq, n, l, 3 + 3 * cc + a);
                    s = cadd(s, cadd(cmul(mb[a], dgp), cmul(P[a], dgm)));
                    // dF0/dr_c = i k khat_c E0
                    s = cadd(s, cmul(mb[a], cmul(make_double2(0.0, pw.k * kh[cc]), E0[a])));
                }
                gp[cc] += 2.0 * s.x;
                // sigma_ext explicit: c Im( conj(dE0/dr_c) . P ), conj(i k khat_c E0) = -i k khat_c conj(E0)
                double2 t = make_double2(0.0, 0.0);
                for (int a = 0; a < 3; a++) t = cadd(t, cconjmul(E0[a], P[a]));
                t = cmul(make_double2(0.0, -pw.k * kh[cc]), t);
                gp[cc] += wext * c * t.y;
            }
            // eps: C = 2 F . (G mub + S mub) - i c w_ext E0^H F - i c w_abs |F|^2
            double2 dotE0F = make_double2(0.0, 0.0);
            double f2 = 0.0;
            double2 fg = make_double2(0.0, 0.0);
            for (int a = 0; a < 3; a++) {
                double2 gm = cadd(sum_partial(partB, ncB, 2, qq, n, l, a), cscale(mb[a], S));
                fg = cadd(fg, cmul(f[a], gm));
                dotE0F = cadd(dotE0F, cconjmul(E0[a], f[a]));
                f2 += f[a].x * f[a].x + f[a].y * f[a].y;
            }
            C = cadd(C, cscale(fg, 2.0));
            C = cadd(C, cmul(make_double2(0.0, -c * wext), dotE0F));
            C = cadd(C, make_double2(0.0, -c * wabs * f2));
            // k: 2 Re[ mub . (i z E0) + mub . dG_k P ] + w_ext c Im( conj(i z E0) . P )
            double2 s = make_double2(0.0, 0.0);
            double2 t = make_double2(0.0, 0.0);
            for (int a = 0; a < 3; a++) {
                double2 dkE0 = cmul(make_double2(0.0, zd), E0[a]);
                s = cadd(s, cmul(mb[a], cadd(dkE0, sum_partial(partA, ncA, 2, qq, n, l, 12 + a))));
                t = cadd(t, cconjmul(dkE0, P[a]));
            }
            dLdk += 2.0 * s.x + wext * c * t.y;
        }
        if (grad_pos)
            for (int cc = 0; cc < 3; cc++) grad_pos[3 * l + cc] += gp[cc];
        if (grad_eps) {
            double2 ge = conjd(cscale(C, d3_4pi));
            grad_eps[l] = cadd(grad_eps[l], ge);
        }
    }
    if (grad_lambda) block_atomic_add(dLdk * dk_dlambda, grad_lambda);
}

// P = alpha F (cells)
__global__ void k_alpha_times(const double2 *__restrict__ F, int64_t n, const double2 *__restrict__ eps, double eps_env,
                              double d3_4pi, double2 *__restrict__ P) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int q = blockIdx.y;
    if (i >= n) return;
    double2 al = make_double2((eps[i].x - eps_env) * d3_4pi, eps[i].y * d3_4pi);
    int64_t off = (int64_t)q * 3 * n + 3 * i;
    for (int a = 0; a < 3; a++) P[off + a] = cmul(al, F[off + a]);
}

// per-RHS sigma / k terms of dL/dk (c is proportional to k): w_ext ext/k + w_abs abs/k
__global__ void k_sigma_k_terms(const double *__restrict__ xs /*[3][n_rhs]: ext, sca, abs*/, int n_rhs,
                                const double *__restrict__ wts, double k, double dk_dlambda, double *grad_lambda) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || !grad_lambda) return;
    double s = 0.0;
    for (int q = 0; q < n_rhs; q++) s += (wts[3 * q] * xs[q] + wts[3 * q + 1] * xs[2 * n_rhs + q]) / k;
    *grad_lambda += s * dk_dlambda;
}

// near-field backward finalize: targets = dipoles j, sources = evaluation points with conj(gE)
__global__ void k_nf_backward_finalize(const double2 *__restrict__ F, int64_t n, const double2 *__restrict__ eps,
                                       double eps_env, double d3_4pi, const double2 *__restrict__ part, int nc, int q0,
                                       int nr, double2 *gF_accum, double *grad_pos, double2 *grad_eps,
                                       double dk_dlambda, double *grad_lambda) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double dLdk = 0.0;
    if (j < n) {
        double2 al = make_double2((eps[j].x - eps_env) * d3_4pi, eps[j].y * d3_4pi);
        double gp[3] = {0, 0, 0};
        double2 C = make_double2(0.0, 0.0);
        for (int qq = 0; qq < nr; qq++) {
            int q = q0 + qq;
            int64_t off = (int64_t)q * 3 * n + 3 * j;
            double2 f[3], P[3], w[3];
            for (int a = 0; a < 3; a++) {
                f[a] = F[off + a];
                P[a] = cmul(al, f[a]);
                w[a] = sum_partial(part, nc, 2, qq, n, j, a);
            }
            if (gF_accum)
                for (int a = 0; a < 3; a++) gF_accum[off + a] = cadd(gF_accum[off + a], cmul(conjd(al), conjd(w[a])));
            double2 fw = make_double2(0.0, 0.0);
            for (int a = 0; a < 3; a++) fw = cadd(fw, cmul(f[a], w[a]));
            C = cadd(C, cscale(fw, 2.0));
            for (int cc = 0; cc < 3; cc++) {
                double2 s = make_double2(0.0, 0.0);
                for (int a = 0; a < 3; a++) s = cadd(s, cmul(P[a], sum_partial(part, nc, 2, qq, n, j, 3 + 3 * cc + a)));
                gp[cc] += 2.0 * s.x;
            }
            double2 s = make_double2(0.0, 0.0);
            for (int a = 0; a < 3; a++) s = cadd(s, cmul(P[a], sum_partial(part, nc, 2, qq, n, j, 12 + a)));
            dLdk += 2.0 * s.x;
        }
        if (grad_pos)
            for (int cc = 0; cc < 3; cc++) grad_pos[3 * j + cc] += gp[cc];
        if (grad_eps) grad_eps[j] = cadd(grad_eps[j], conjd(cscale(C, d3_4pi)));
    }
    if (grad_lambda) block_atomic_add(dLdk * dk_dlambda, grad_lambda);
}

// incident-field part of dL/dk for the near field: sum_m 2 Re[ conj(gE_m) . (i (khat.r_m) E0_m) ]
__global__ void k_nf_incident_k(const double *__restrict__ r_eval, int64_t m, int n_rhs, const double2 *__restrict__ gE,
                                const double *__restrict__ e0, PW pw, double dk_dlambda, double *grad_lambda) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double v = 0.0;
    if (t < m) {
        for (int q = 0; q < n_rhs; q++) {
            double2 E0[3];
            double zd;
            planewave_at(pw, e0 + 6 * q, r_eval[3 * t], r_eval[3 * t + 1], r_eval[3 * t + 2], E0, &zd);
            for (int a = 0; a < 3; a++) {
                double2 d = cmul(make_double2(0.0, zd), E0[a]);
                v += 2.0 * cconjmul(gE[(int64_t)q * 3 * m + 3 * t + a], d).x;
            }
        }
    }
    if (grad_lambda) block_atomic_add(v * dk_dlambda, grad_lambda);
}

}  // namespace

gdm_status gdm_launch_backward(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, const void *A, int64_t lda,
                               const int32_t *ipiv, const double *F, int n_rhs, const double *e0, const double *khat,
                               const double *gF, const double *g_sigma, double *grad_pos, double *grad_eps,
                               double *grad_wavelength, gdm_solve_info *info) {
    gdm_params_reset(ctx);
    const int64_t n = p->n, ns = 3 * n, cnt = ns * n_rhs;
    const double k0 = gdm_k0(p), k = sqrt(p->eps_env) * k0;
    const double d3_4pi = p->step * p->step * p->step / (4.0 * PI_D);
    const double S = -4.0 * PI_D / (3.0 * p->eps_env * p->step * p->step * p->step);
    const double dk_dl = -k / p->wavelength;
    // weights per RHS: w_ext = dL/dext + dL/dsca, w_abs = dL/dabs - dL/dsca, prefactor c
    double hw[3 * 64];
    for (int q = 0; q < n_rhs; q++) {
        double ge = g_sigma ? g_sigma[3 * q] : 0.0, gs = g_sigma ? g_sigma[3 * q + 1] : 0.0,
               ga = g_sigma ? g_sigma[3 * q + 2] : 0.0;
        double e2 = 0.0;
        for (int a = 0; a < 6; a++) e2 += e0[6 * q + a] * e0[6 * q + a];
        hw[3 * q] = ge + gs;
        hw[3 * q + 1] = ga - gs;
        hw[3 * q + 2] = 4.0 * PI_D * k / (p->eps_env * e2);
    }
    double *dw, *de0;
    GDM_TRY(gdm_upload(ctx, hw, sizeof(double) * 3 * n_rhs, (void **)&dw));
    GDM_TRY(gdm_upload(ctx, e0, sizeof(double) * 6 * n_rhs, (void **)&de0));
    PW pw = {k, khat[0], khat[1], khat[2]};
    // adjoint right-hand side and the refined adjoint solve (its own scratch)
    // gradient pair sums in double-float on the FP32 pipes unless GDM_GRADIENT_FP64 is set
    const bool ffg = !getenv("GDM_GRADIENT_FP64");
    size_t own = ScratchCarver::round(cnt * sizeof(double2)) * 3 + ScratchCarver::round(3 * n_rhs * sizeof(double)) +
                 ScratchCarver::round(2 * dg_partial_bytes(ctx, n, n)) +
                 (ffg ? ScratchCarver::round(gdm_ff_scratch_bytes(n)) : 0) + 4096;
    // g and mu live in a separate allocation because the refined solve reuses the context arena
    double2 *g = nullptr, *mu = nullptr;
    GDM_CUDA_TRY(ctx, cudaMallocAsync((void **)&g, cnt * sizeof(double2) * 2, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(g, 0, cnt * sizeof(double2) * 2, ctx->stream));
    mu = g + cnt;
    unsigned nb = (unsigned)((n + 127) / 128);
    k_adjoint_rhs<<<dim3(nb, n_rhs), 128, 0, ctx->stream>>>((const double2 *)F, (const double2 *)gF, n, n_rhs,
                                                            (const double2 *)p->eps, p->eps_env, d3_4pi, de0, pw, dw,
                                                            p->pos, g);
    GDM_LAUNCHED(ctx, "adjoint_rhs");
    gdm_solve_opts o = {prec == GDM_FP64 ? 3 : 40, 0, 1e-12};
    gdm_status st = gdm_refined_solve(ctx, p, prec, A, lda, ipiv, (const double *)g, (double *)mu, n_rhs, 1, &o, info);
    if (st != GDM_OK) {
        cudaFreeAsync(g, ctx->stream);
        return st;
    }
    void *ws;
    GDM_TRY(gdm_scratch(ctx, own, &ws));
    ScratchCarver sc(ws);
    double2 *Pm = sc.take<double2>(cnt);
    double *xs = sc.take<double>(3 * n_rhs);
    double2 *partA = sc.take<double2>(dg_partial_bytes(ctx, n, n) / sizeof(double2));
    double2 *partB = sc.take<double2>(dg_partial_bytes(ctx, n, n) / sizeof(double2));
    double2 *F0 = sc.take<double2>(cnt);
    void *ffws = ffg ? sc.take<char>(gdm_ff_scratch_bytes(n)) : nullptr;
    // sigma values for the k-derivative of the prefactor (c is proportional to k)
    double e2[64];
    for (int q = 0; q < n_rhs; q++) {
        e2[q] = 0.0;
        for (int a = 0; a < 6; a++) e2[q] += e0[6 * q + a] * e0[6 * q + a];
    }
    GDM_TRY(gdm_launch_planewave(ctx, p->pos, n, k, sqrt(p->eps_env), e0, khat, n_rhs, 3, (double *)F0));
    GDM_TRY(gdm_launch_cross_sections(ctx, p, (const double *)F0, F, n_rhs, e2, xs, xs + n_rhs, xs + 2 * n_rhs));
    // moments P = alpha F
    k_alpha_times<<<dim3(nb, n_rhs), 128, 0, ctx->stream>>>((const double2 *)F, n, (const double2 *)p->eps,
                                                            p->eps_env, d3_4pi, Pm);
    GDM_LAUNCHED(ctx, "alpha_times");
    for (int q0 = 0; q0 < n_rhs; q0 += 2) {
        int nr = n_rhs - q0 < 2 ? n_rhs - q0 : 2;
        int ncA, ncB;
        GDM_TRY(gdm_phase_begin(ctx, GDM_PH_GRADIENT));
        if (ffg) {
            if (q0 == 0) GDM_TRY(gdm_ff_prepare(ctx, p, ffws));
            int64_t ch;
            int nc;
            dg_grid_ff(ctx, n, n, &ch, &nc);
            for (int q = 0; q < nr; q++) {
                GDM_TRY(gdm_ff_dgreen_sum(ctx, p, Pm, q0 + q, 0, q, ch, nc, ffws, partA));
                GDM_TRY(gdm_ff_dgreen_sum(ctx, p, mu, q0 + q, 1, q, ch, nc, ffws, partB));
            }
            ncA = ncB = nc;
        } else {
            GDM_TRY(launch_dg(ctx, p->pos, n, p->pos, Pm, n, q0, nr, 0, k, 1.0 / p->eps_env, 1, partA, &ncA));
            GDM_TRY(launch_dg(ctx, p->pos, n, p->pos, mu, n, q0, nr, 1, k, 1.0 / p->eps_env, 1, partB, &ncB));
        }
        GDM_TRY(gdm_phase_end(ctx, GDM_PH_GRADIENT));
        k_backward_finalize<<<nb, 128, 0, ctx->stream>>>((const double2 *)F, mu, n, n_rhs, (const double2 *)p->eps,
                                                         p->eps_env, d3_4pi, S, p->pos, de0, pw, dw, partA, ncA, partB,
                                                         ncB, q0, nr, dk_dl, grad_pos, (double2 *)grad_eps,
                                                         grad_wavelength);
        GDM_LAUNCHED(ctx, "backward_finalize");
    }
    k_sigma_k_terms<<<1, 32, 0, ctx->stream>>>(xs, n_rhs, dw, k, dk_dl, grad_wavelength);
    GDM_LAUNCHED(ctx, "sigma_k_terms");
    GDM_CUDA_TRY(ctx, cudaFreeAsync(g, ctx->stream));
    return GDM_OK;
}

gdm_status gdm_launch_nearfield_backward(gdm_ctx *ctx, const gdm_problem *p, const double *F, const double *r_eval,
                                         int64_t m, int n_rhs, const double *e0, const double *khat, const double *gE,
                                         double *gF_accum, double *grad_pos, double *grad_eps,
                                         double *grad_wavelength) {
    gdm_params_reset(ctx);
    const int64_t n = p->n;
    const double k0 = gdm_k0(p), k = sqrt(p->eps_env) * k0;
    const double d3_4pi = p->step * p->step * p->step / (4.0 * PI_D);
    const double dk_dl = -k / p->wavelength;
    double *de0;
    GDM_TRY(gdm_upload(ctx, e0, sizeof(double) * 6 * n_rhs, (void **)&de0));
    PW pw = {k, khat[0], khat[1], khat[2]};
    void *ws;
    GDM_TRY(gdm_scratch(ctx, dg_partial_bytes(ctx, n, m) + 1024, &ws));
    double2 *part = (double2 *)ws;
    unsigned nb = (unsigned)((n + 127) / 128);
    for (int q0 = 0; q0 < n_rhs; q0 += 2) {
        int nr = n_rhs - q0 < 2 ? n_rhs - q0 : 2;
        int nc;
        // targets: dipoles; sources: evaluation points with vectors conj(gE) (R = r_j - r_m)
        GDM_TRY(launch_dg(ctx, p->pos, n, r_eval, (const double2 *)gE, m, q0, nr, 1, k, 1.0 / p->eps_env, 0, part,
                          &nc));
        k_nf_backward_finalize<<<nb, 128, 0, ctx->stream>>>((const double2 *)F, n, (const double2 *)p->eps, p->eps_env,
                                                            d3_4pi, part, nc, q0, nr, (double2 *)gF_accum, grad_pos,
                                                            (double2 *)grad_eps, dk_dl, grad_wavelength);
        GDM_LAUNCHED(ctx, "nf_backward_finalize");
    }
    k_nf_incident_k<<<(unsigned)((m + 127) / 128), 128, 0, ctx->stream>>>(r_eval, m, n_rhs, (const double2 *)gE, de0,
                                                                          pw, dk_dl, grad_wavelength);
    GDM_LAUNCHED(ctx, "nf_incident_k");
    return GDM_OK;
}
