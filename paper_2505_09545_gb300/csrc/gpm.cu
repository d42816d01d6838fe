// Point-dipole illuminations, the local density of states (LDOS) of a structured environment, and
// effective-model (global polarizability matrix, GPM) extraction from a discretised structure
// (Sec. "Effective polarizabilities", GPM extraction), all steps on the GPU:
//   1. illumination fields: plane waves and local dipole sources, at the cells (E) and at the effective
//      sites (E, H);
//   2. full simulations: one factorisation, refined solves of all illuminations (chunks of 64 RHS);
//   3. scattered (E, H) at the probe positions by repropagation;
//   4. effective moments at the sites: least squares through the 6x6 dyads Gp (probe <- unit site dipole);
//   5. alpha_eff = P F0^+ in the least-squares sense over the illuminations.
// The least-squares steps use FP64 semi-normal equations (Gram matrix, Cholesky) with one refinement
// step on the residual, which brings the solution to the accuracy of a QR solve for these well-scaled,
// modestly conditioned problems. Homogeneous host of permittivity eps_env: plane waves, dipole sources and
// the site-to-probe dyads all propagate through the host.
#include <math.h>

#include "gdm_internal.cuh"

namespace {

#define GPM_MAX_ILL 512
#define GPM_MAX_SITES 64

__device__ __forceinline__ double2 cz2() { return make_double2(0.0, 0.0); }

// alpha6 = identity for every site (its "fields" F are then its moments)
__global__ void k_identity6(double2 *a, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 36 * n) return;
    const int r = (int)(e % 36) / 6, c = (int)(e % 6);
    a[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
}

// one-hot moment columns: column q holds mom[q] (6 complex) at dipole q, zero elsewhere; (6 n) x n
__global__ void k_onehot(const double2 *__restrict__ mom, int64_t n, double2 *out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 36 * n * n / 6) return;  // (6n) x n entries
    const int64_t q = e / (6 * n), r = e % (6 * n);
    out[e] = (r / 6 == q) ? (mom ? mom[6 * q + r % 6] : make_double2(r % 6 == 0 ? 1.0 : 0.0, 0.0)) : cz2();
}

// unit moment columns for the propagation matrix: column c (c < 6 M) is the unit vector e_c
__global__ void k_eye(int64_t n6, double2 *out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n6 * n6) return;
    out[e] = make_double2((e / n6) == (e % n6) ? 1.0 : 0.0, 0.0);
}

// out[(r) + c ld] for r < 3m from E[r + c 3m], for 3m <= r < 6m from H: stacked rows [E; H]
__global__ void k_stack(const double2 *__restrict__ E, const double2 *__restrict__ H, int64_t m, int64_t ncol,
                        double2 *out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 6 * m * ncol) return;
    const int64_t c = e / (6 * m), r = e % (6 * m);
    out[e] = r < 3 * m ? E[r + c * 3 * m] : H[r - 3 * m + c * 3 * m];
}

// per-point interleave: out[6 t + a + c ld] = a < 3 ? E[3 t + a + c 3m] : H[3 t + a - 3 + c 3m]
__global__ void k_interleave(const double2 *__restrict__ E, const double2 *__restrict__ H, int64_t m, int64_t ncol,
                             double2 *out, int64_t ld) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= 6 * m * ncol) return;
    const int64_t c = e / (6 * m), r = e % (6 * m), t = r / 6, a = r % 6;
    out[r + c * ld] = a < 3 ? E[3 * t + a + c * 3 * m] : H[3 * t + a - 3 + c * 3 * m];
}

// out[i + j ldo] = sum_k conj(A(k, i)) B(k, j), A(k, i) = A[k + i lda] (or A[i + k lda] when ta), same for B
__global__ void k_gram(const double2 *__restrict__ A, int64_t lda, int ta, const double2 *__restrict__ B, int64_t ldb,
                       int tb, int64_t m, int n, int r, double2 *out, int64_t ldo) {
    const int i = blockIdx.x, j0 = blockIdx.y * 8;
    double2 acc[8];
#pragma unroll
    for (int q = 0; q < 8; q++) acc[q] = cz2();
    for (int64_t k = threadIdx.x; k < m; k += blockDim.x) {
        const double2 a = ta ? A[i + k * lda] : A[k + (int64_t)i * lda];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            if (j0 + q < r) {
                const double2 b = tb ? B[(j0 + q) + k * ldb] : B[k + (int64_t)(j0 + q) * ldb];
                acc[q].x += a.x * b.x + a.y * b.y;
                acc[q].y += a.x * b.y - a.y * b.x;
            }
        }
    }
    __shared__ double2 red[8][32];
#pragma unroll
    for (int q = 0; q < 8; q++) {
        double x = acc[q].x, y = acc[q].y;
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
        }
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = make_double2(x, y);
    }
    __syncthreads();
    if (threadIdx.x < 8 && j0 + (int)threadIdx.x < r) {
        double2 s = cz2();
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s = cadd(s, red[threadIdx.x][w]);
        out[i + (int64_t)(j0 + threadIdx.x) * ldo] = s;
    }
}

// In-place Cholesky G = L L^H of the n x n Hermitian positive definite G (one CTA), then X := G^{-1} X for
// r columns (forward and backward substitution, one thread per column). flag[0] set when a pivot is not
// positive.
__global__ void __launch_bounds__(1024) k_chol_solve(double2 *G, int n, double2 *X, int64_t ldx, int r, int *flag) {
    for (int k = 0; k < n; k++) {
        __syncthreads();
        const double d = G[k + (int64_t)k * n].x;
        if (!(d > 0.0)) {
            if (threadIdx.x == 0) flag[0] = 1;
            return;
        }
        const double s = sqrt(d);
        __syncthreads();
        for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
            double2 v = G[i + (int64_t)k * n];
            G[i + (int64_t)k * n] = make_double2(v.x / s, v.y / s);
        }
        __syncthreads();
        // trailing update of the lower triangle: G[i, j] -= L[i, k] conj(L[j, k]), k < j <= i
        const int w = n - k - 1;
        for (int64_t e = threadIdx.x; e < (int64_t)w * w; e += blockDim.x) {
            const int i = k + 1 + (int)(e % w), j = k + 1 + (int)(e / w);
            if (j > i) continue;
            const double2 li = G[i + (int64_t)k * n], lj = G[j + (int64_t)k * n];
            double2 &g = G[i + (int64_t)j * n];
            g.x -= li.x * lj.x + li.y * lj.y;
            g.y -= li.y * lj.x - li.x * lj.y;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < r; c += blockDim.x) {
        double2 *x = X + (int64_t)c * ldx;
        for (int i = 0; i < n; i++) {  // L y = x
            double2 s = x[i];
            for (int j = 0; j < i; j++) s = csub(s, cmul(G[i + (int64_t)j * n], x[j]));
            const double li = G[i + (int64_t)i * n].x;
            x[i] = make_double2(s.x / li, s.y / li);
        }
        for (int i = n - 1; i >= 0; i--) {  // L^H x = y
            double2 s = x[i];
            for (int j = i + 1; j < n; j++) {
                const double2 l = G[j + (int64_t)i * n];
                s = csub(s, cmul(make_double2(l.x, -l.y), x[j]));
            }
            const double li = G[i + (int64_t)i * n].x;
            x[i] = make_double2(s.x / li, s.y / li);
        }
    }
}

// R = B - A X (A(k, i) as in k_gram); one thread per entry of R (m x r); norms[0..1] += ||R||^2, ||B||^2
__global__ void k_lsq_residual(const double2 *__restrict__ A, int64_t lda, int ta, const double2 *__restrict__ B,
                               int64_t ldb, int tb, const double2 *__restrict__ X, int64_t ldx, int64_t m, int n, int r,
                               double2 *R, double *norms) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double rr = 0.0, bb = 0.0;
    if (e < m * r) {
        const int64_t k = e % m;
        const int j = (int)(e / m);
        const double2 b = tb ? B[j + k * ldb] : B[k + (int64_t)j * ldb];
        double2 s = b;
        for (int i = 0; i < n; i++) {
            const double2 a = ta ? A[i + k * lda] : A[k + (int64_t)i * lda];
            s = csub(s, cmul(a, X[i + (int64_t)j * ldx]));
        }
        R[e] = s;
        rr = s.x * s.x + s.y * s.y;
        bb = b.x * b.x + b.y * b.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        bb += __shfl_down_sync(0xffffffffu, bb, o);
    }
    if ((threadIdx.x & 31) == 0 && (rr != 0.0 || bb != 0.0)) {
        atomicAdd(&norms[0], rr);
        atomicAdd(&norms[1], bb);
    }
}

__global__ void k_add(double2 *X, const double2 *D, int64_t cnt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < cnt) X[e] = cadd(X[e], D[e]);
}

// out[j + i ld] = in[i + j n] (plain transpose, n x n)
__global__ void k_transpose(const double2 *__restrict__ in, int n, double2 *out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int i = (int)(e % n), j = (int)(e / n);
    out[j + (int64_t)i * n] = in[e];
}

unsigned nblk(int64_t cnt, int bs = 256) { return (unsigned)((cnt + bs - 1) / bs); }

// X (n x r, ld n) = argmin ||A X - B||, A: m x n, B: m x r (A(k, i) / B(k, j) read transposed when ta / tb).
// Scratch: G (n x n), C (n x r), R (m x r), flag, norms (4 doubles). rel: host ||A X - B|| / ||B|| (or null).
gdm_status lstsq(gdm_ctx *ctx, const double2 *A, int64_t lda, int ta, const double2 *B, int64_t ldb, int tb, int64_t m,
                 int n, int r, double2 *X, double2 *G, double2 *C, double2 *R, int *flag, double *norms,
                 double *rel) {
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemsetAsync(norms, 0, 4 * sizeof(double), ctx->stream));
    for (int pass = 0; pass < 2; pass++) {
        // pass 0: X = (A^H A)^{-1} A^H B; pass 1: X += (A^H A)^{-1} A^H (B - A X)
        k_gram<<<dim3((unsigned)n, (unsigned)((n + 7) / 8)), 256, 0, ctx->stream>>>(A, lda, ta, A, lda, ta, m, n, n, G,
                                                                                   n);
        GDM_LAUNCHED(ctx, "gram");
        const double2 *rhs = pass == 0 ? B : R;
        const int64_t ldr = pass == 0 ? ldb : m;
        const int tr = pass == 0 ? tb : 0;
        k_gram<<<dim3((unsigned)n, (unsigned)((r + 7) / 8)), 256, 0, ctx->stream>>>(A, lda, ta, rhs, ldr, tr, m, n, r, C,
                                                                                   n);
        GDM_LAUNCHED(ctx, "gram_rhs");
        k_chol_solve<<<1, 1024, 0, ctx->stream>>>(G, n, C, n, r, flag);
        GDM_LAUNCHED(ctx, "chol_solve");
        if (pass == 0) {
            GDM_CUDA_TRY(ctx, cudaMemcpyAsync(X, C, sizeof(double2) * n * r, cudaMemcpyDeviceToDevice, ctx->stream));
        } else {
            k_add<<<nblk((int64_t)n * r), 256, 0, ctx->stream>>>(X, C, (int64_t)n * r);
            GDM_LAUNCHED(ctx, "lsq_add");
        }
        GDM_CUDA_TRY(ctx, cudaMemsetAsync(norms, 0, 2 * sizeof(double), ctx->stream));
        k_lsq_residual<<<nblk(m * r), 256, 0, ctx->stream>>>(A, lda, ta, B, ldb, tb, X, n, m, n, r, R, norms);
        GDM_LAUNCHED(ctx, "lsq_residual");
    }
    int hf = 0;
    double hn[2];
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaMemcpyAsync(hn, norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    GDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (hf)
        return gdm_fail(ctx, GDM_ERR_SINGULAR,
                        "GPM fit: the normal matrix is not positive definite (too few or ill-placed probes / "
                        "illuminations for the number of effective dipoles)");
    if (rel) *rel = hn[1] > 0 ? sqrt(hn[0] / hn[1]) : 0.0;
    return GDM_OK;
}

// moments of the LDOS emitters: source 3 e + u is a unit dipole along u (electric or magnetic) at r0[e]
__global__ void k_ldos_sources(const double *__restrict__ r0, int n_pos, int magnetic, double *pos3, double2 *mom) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 3 * n_pos) return;
    const int e = q / 3, u = q % 3;
    for (int c = 0; c < 3; c++) pos3[3 * q + c] = r0[3 * e + c];
    for (int c = 0; c < 6; c++) mom[6 * q + c] = make_double2(c == u + (magnetic ? 3 : 0) ? 1.0 : 0.0, 0.0);
}

// rho_u / rho_0 = 1 + 3/(2 k^3) Im(field_u at the emitter, from the emitter's own illumination)
__global__ void k_ldos_extract(const double2 *__restrict__ field, int n_pos, double c, double *out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 3 * n_pos) return;
    const int e = q / 3, u = q % 3;
    out[q] = 1.0 + c * field[(int64_t)q * 3 * n_pos + 3 * e + u].y;
}

// E (and H) at m points of n_src point dipoles (device positions n_src x 3, moments n_src x 6), column q
// = source q; id6 (36 n_src) and onehot (6 n_src x n_src) are scratch
gdm_status dipole_fields(gdm_ctx *ctx, double wavelength, double eps_env, const double *src_pos, const double2 *mom,
                         int n_src, const double *r_eval, int64_t m, double2 *E, double2 *H, double2 *id6,
                         double2 *onehot) {
    k_identity6<<<nblk(36 * (int64_t)n_src), 256, 0, ctx->stream>>>(id6, n_src);
    GDM_LAUNCHED(ctx, "identity6");
    k_onehot<<<nblk(6 * (int64_t)n_src * n_src), 256, 0, ctx->stream>>>(mom, n_src, onehot);
    GDM_LAUNCHED(ctx, "onehot");
    gdm_problem src = {n_src, 6, 0, src_pos, nullptr, (const double *)id6, 0.0, eps_env, wavelength};
    return gdm_launch_nearfield(ctx, &src, (const double *)onehot, r_eval, m, nullptr, n_src, (double *)E, (double *)H);
}

}  // namespace

extern "C" gdm_status gdm_incident_dipole(gdm_ctx *ctx, const double *r_eval, int64_t m, double wavelength,
                                          double eps_env, const double *src_pos, const double *src_mom, int n_src,
                                          int kind_out, double *F0) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    if (!r_eval || !src_pos || !src_mom || !F0) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (m < 1 || n_src < 1 || n_src > 1024) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "need m >= 1, 1 <= n_src <= 1024");
    if (kind_out != 3 && kind_out != 6) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "kind_out must be 3 or 6");
    if (!(wavelength > 0) || !isfinite(wavelength) || !(eps_env > 0) || !isfinite(eps_env))
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "bad wavelength or eps_env");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    gdm_params_reset(ctx);
    double2 *buf = nullptr;
    const size_t cnt = (size_t)36 * n_src + (size_t)6 * n_src * n_src + (kind_out == 6 ? (size_t)6 * m * n_src : 0);
    GDM_CUDA_TRY(ctx, cudaMallocAsync((void **)&buf, cnt * sizeof(double2), ctx->stream));
    double2 *id6 = buf, *onehot = buf + 36 * n_src, *E = onehot + (size_t)6 * n_src * n_src, *H = E + 3 * m * n_src;
    gdm_status st;
    if (kind_out == 3) {
        st = dipole_fields(ctx, wavelength, eps_env, src_pos, (const double2 *)src_mom, n_src, r_eval, m,
                           (double2 *)F0, nullptr, id6, onehot);
    } else {
        st = dipole_fields(ctx, wavelength, eps_env, src_pos, (const double2 *)src_mom, n_src, r_eval, m, E, H, id6,
                           onehot);
        if (st == GDM_OK) {
            k_interleave<<<nblk(6 * m * (int64_t)n_src), 256, 0, ctx->stream>>>(E, H, m, n_src, (double2 *)F0, 6 * m);
            st = gdm_after_launch(ctx, "interleave");
        }
    }
    cudaFreeAsync(buf, ctx->stream);
    return st;
}

extern "C" gdm_status gdm_ldos(gdm_ctx *ctx, gdm_precision prec, const gdm_problem *p, void *A, int64_t lda,
                               int32_t *ipiv, const double *r0, int n_pos, int magnetic, double *ldos) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    GDM_TRY(gdm_check_solve_args(ctx, p, prec, A, lda, ipiv, r0, r0, 1));
    if (p->kind != 3) return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "LDOS: discretised structures (kind 3)");
    if (!ldos) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (n_pos < 1 || n_pos > 340) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "n_pos must be in [1, 340]");
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    gdm_params_reset(ctx);
    const int64_t n = p->n;
    const int ns = 3 * n_pos;
    const size_t c16 = sizeof(double2);
    const size_t bytes = c16 * ((size_t)36 * ns + (size_t)6 * ns * ns + (size_t)6 * ns + (size_t)3 * n * ns * 2 +
                                (size_t)3 * n_pos * ns * 2) +
                         sizeof(double) * 3 * ns + 4096;
    char *buf = nullptr;
    GDM_CUDA_TRY(ctx, cudaMallocAsync((void **)&buf, bytes, ctx->stream));
    ScratchCarver sc(buf);
    double2 *id6 = sc.take<double2>((size_t)36 * ns), *onehot = sc.take<double2>((size_t)6 * ns * ns);
    double2 *mom = sc.take<double2>((size_t)6 * ns);
    double2 *F0 = sc.take<double2>((size_t)3 * n * ns), *F = sc.take<double2>((size_t)3 * n * ns);
    double2 *Es = sc.take<double2>((size_t)3 * n_pos * ns), *Hs = sc.take<double2>((size_t)3 * n_pos * ns);
    double *pos3 = sc.take<double>((size_t)3 * ns);
    auto run = [&]() -> gdm_status {
        k_ldos_sources<<<nblk(ns), 256, 0, ctx->stream>>>(r0, n_pos, magnetic, pos3, mom);
        GDM_LAUNCHED(ctx, "ldos_sources");
        GDM_TRY(dipole_fields(ctx, p->wavelength, p->eps_env, pos3, mom, ns, p->pos, n, F0, nullptr, id6, onehot));
        GDM_TRY(gdm_launch_assemble(ctx, p, prec, A, lda));
        for (int q0 = 0; q0 < ns; q0 += 64) {
            const int nr = ns - q0 < 64 ? ns - q0 : 64;
            gdm_solve_opts o = {0, q0 ? GDM_SOLVE_FACTORED : 0, 0.0};
            GDM_TRY(gdm_solve_core(ctx, p, prec, A, lda, ipiv, (const double *)(F0 + (int64_t)q0 * 3 * n),
                                   (double *)(F + (int64_t)q0 * 3 * n), nr, &o, nullptr));
        }
        GDM_TRY(gdm_launch_nearfield(ctx, p, (const double *)F, r0, n_pos, nullptr, ns, (double *)Es, (double *)Hs));
        // emitted power over that of the bare host: c k0 k^3/(3 eps_env) (electric), c k0 k^3/3 (magnetic)
        const double k = sqrt(p->eps_env) * 2.0 * 3.14159265358979323846 / p->wavelength;
        const double c = 1.5 * (magnetic ? 1.0 : p->eps_env) / (k * k * k);
        k_ldos_extract<<<nblk(ns), 256, 0, ctx->stream>>>(magnetic ? Hs : Es, n_pos, c, ldos);
        GDM_LAUNCHED(ctx, "ldos_extract");
        return GDM_OK;
    };
    gdm_status st = run();
    cudaFreeAsync(buf, ctx->stream);
    return st;
}

extern "C" gdm_status gdm_gpm_extract(gdm_ctx *ctx, gdm_precision prec, const gdm_problem *p, void *A, int64_t lda,
                                      int32_t *ipiv, const double *r_gpm, int n_sites, const double *r_probe,
                                      int n_probe, int n_pw, const double *pw_khat, const double *pw_e0, int n_ds,
                                      const double *ds_pos, const double *ds_mom, double *alpha_eff, double *moments,
                                      double *rel_fit) {
    if (!ctx) return GDM_ERR_INVALID_ARG;
    GDM_TRY(gdm_check_solve_args(ctx, p, prec, A, lda, ipiv, r_gpm, r_gpm, 1));
    if (p->kind != 3) return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "GPM extraction: discretised structures (kind 3)");
    const int n_ill = n_pw + n_ds;
    if (!r_gpm || !r_probe || !alpha_eff || (n_pw && (!pw_khat || !pw_e0)) || (n_ds && (!ds_pos || !ds_mom)))
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "null pointer");
    if (n_sites < 1 || n_sites > GPM_MAX_SITES || n_pw < 0 || n_ds < 0 || n_ill > GPM_MAX_ILL)
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "GPM extraction: need 1..%d sites and at most %d illuminations",
                        GPM_MAX_SITES, GPM_MAX_ILL);
    if (n_ill < 6 * n_sites || n_probe < n_sites)
        return gdm_fail(ctx, GDM_ERR_INVALID_ARG,
                        "GPM extraction: need at least 6 illuminations and one probe per effective dipole "
                        "(%d illuminations, %d probes, %d sites)",
                        n_ill, n_probe, n_sites);
    for (int q = 0; q < n_pw; q++) {
        double kn = 0;
        for (int c = 0; c < 3; c++) kn += pw_khat[3 * q + c] * pw_khat[3 * q + c];
        if (fabs(kn - 1.0) > 1e-9) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "khat %d is not a unit vector", q);
    }
    GDM_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    gdm_params_reset(ctx);
    const int64_t n = p->n, M = n_sites, P = n_probe, M6 = 6 * M;
    const double n_env = sqrt(p->eps_env), k = n_env * 2.0 * 3.14159265358979323846 / p->wavelength;
    // device buffers of the extraction (separate from the context arena, which the solves reuse); the
    // carving runs once on a null base to size the allocation
    const size_t c16 = sizeof(double2);
    const int64_t maxr = n_ill > M6 ? n_ill : M6;
    const int64_t nid = M > n_ds ? M : n_ds;
    double2 *F0c, *F, *S, *Et, *Ht, *Gp, *F0g, *X, *Es, *Hs, *id6, *unit, *onehot, *Gm, *Cm, *R, *aT, *Rt;
    int *flag;
    double *norms;
    auto carve = [&](char *base) {
        ScratchCarver sc(base);
        F0c = sc.take<double2>((size_t)3 * n * n_ill);
        F = sc.take<double2>((size_t)3 * n * n_ill);
        S = sc.take<double2>((size_t)6 * P * n_ill);
        Et = sc.take<double2>((size_t)3 * P * maxr);
        Ht = sc.take<double2>((size_t)3 * P * maxr);
        Gp = sc.take<double2>((size_t)6 * P * M6);
        F0g = sc.take<double2>((size_t)M6 * n_ill);
        X = sc.take<double2>((size_t)M6 * n_ill);
        Es = sc.take<double2>((size_t)3 * M * (n_ds > 0 ? n_ds : 1));
        Hs = sc.take<double2>((size_t)3 * M * (n_ds > 0 ? n_ds : 1));
        id6 = sc.take<double2>((size_t)36 * nid);
        unit = sc.take<double2>((size_t)M6 * M6);
        onehot = sc.take<double2>((size_t)6 * (n_ds > 0 ? n_ds : 1) * (n_ds > 0 ? n_ds : 1));
        Gm = sc.take<double2>((size_t)M6 * M6);
        Cm = sc.take<double2>((size_t)M6 * maxr);
        R = sc.take<double2>((size_t)6 * P * maxr);
        aT = sc.take<double2>((size_t)n_ill * M6);
        Rt = sc.take<double2>((size_t)n_ill * M6);
        flag = sc.take<int>(4);
        norms = sc.take<double>(4);
        return sc.off + 256;
    };
    const size_t bytes = carve(nullptr);
    char *buf = nullptr;
    GDM_CUDA_TRY(ctx, cudaMallocAsync((void **)&buf, bytes, ctx->stream));
    carve(buf);
    gdm_status st = GDM_OK;
    auto run = [&]() -> gdm_status {
        k_identity6<<<nblk(36 * nid), 256, 0, ctx->stream>>>(id6, nid);
        GDM_LAUNCHED(ctx, "identity6");
        // 1. illuminations: plane waves (E at the cells, E and H at the sites)
        for (int q = 0; q < n_pw; q++) {
            // the amplitudes go through the context's parameter buffer; its copies are ordered on the stream
            // after the launches that read the previous contents, so it can restart for every wave
            gdm_params_reset(ctx);
            GDM_TRY(gdm_launch_planewave(ctx, p->pos, n, k, n_env, pw_e0 + 6 * q, pw_khat + 3 * q, 1, 3,
                                         (double *)(F0c + (int64_t)q * 3 * n)));
            GDM_TRY(gdm_launch_planewave(ctx, r_gpm, M, k, n_env, pw_e0 + 6 * q, pw_khat + 3 * q, 1, 6,
                                         (double *)(F0g + (int64_t)q * M6)));
        }
        //    and local dipole sources (an ED/MD "structure" in the host with alpha = I and one-hot moments)
        if (n_ds > 0) {
            k_onehot<<<nblk(6 * (int64_t)n_ds * n_ds), 256, 0, ctx->stream>>>((const double2 *)ds_mom, n_ds, onehot);
            GDM_LAUNCHED(ctx, "onehot");
            gdm_problem src = {n_ds, 6, 0, ds_pos, nullptr, (const double *)id6, 0.0, p->eps_env, p->wavelength};
            GDM_TRY(gdm_launch_nearfield(ctx, &src, (const double *)onehot, p->pos, n, nullptr, n_ds,
                                         (double *)(F0c + (int64_t)n_pw * 3 * n), nullptr));
            GDM_TRY(gdm_launch_nearfield(ctx, &src, (const double *)onehot, r_gpm, M, nullptr, n_ds, (double *)Es,
                                         (double *)Hs));
            k_interleave<<<nblk(6 * M * (int64_t)n_ds), 256, 0, ctx->stream>>>(Es, Hs, M, n_ds, F0g + (int64_t)n_pw * M6,
                                                                             M6);
            GDM_LAUNCHED(ctx, "interleave");
        }
        // 2. full simulations: assemble, factor once, refined solves in chunks of 64 illuminations
        GDM_TRY(gdm_launch_assemble(ctx, p, prec, A, lda));
        for (int q0 = 0; q0 < n_ill; q0 += 64) {
            const int nr = n_ill - q0 < 64 ? n_ill - q0 : 64;
            gdm_solve_opts o = {0, q0 ? GDM_SOLVE_FACTORED : 0, 0.0};
            GDM_TRY(gdm_solve_core(ctx, p, prec, A, lda, ipiv, (const double *)(F0c + (int64_t)q0 * 3 * n),
                                   (double *)(F + (int64_t)q0 * 3 * n), nr, &o, nullptr));
        }
        // 3. scattered fields at the probes, stacked [E; H]
        GDM_TRY(gdm_launch_nearfield(ctx, p, (const double *)F, r_probe, P, nullptr, n_ill, (double *)Et,
                                     (double *)Ht));
        k_stack<<<nblk(6 * P * (int64_t)n_ill), 256, 0, ctx->stream>>>(Et, Ht, P, n_ill, S);
        GDM_LAUNCHED(ctx, "stack");
        //    propagation from unit moments at the sites to the probes, stacked the same way
        k_eye<<<nblk(M6 * M6), 256, 0, ctx->stream>>>(M6, unit);
        GDM_LAUNCHED(ctx, "eye");
        gdm_problem sites = {M, 6, 0, r_gpm, nullptr, (const double *)id6, 0.0, p->eps_env, p->wavelength};
        GDM_TRY(gdm_launch_nearfield(ctx, &sites, (const double *)unit, r_probe, P, nullptr, (int)M6, (double *)Et,
                                     (double *)Ht));
        k_stack<<<nblk(6 * P * M6), 256, 0, ctx->stream>>>(Et, Ht, P, M6, Gp);
        GDM_LAUNCHED(ctx, "stack");
        // 4. effective moments: min || Gp X - S ||
        GDM_TRY(lstsq(ctx, Gp, 6 * P, 0, S, 6 * P, 0, 6 * P, (int)M6, n_ill, X, Gm, Cm, R, flag, norms, rel_fit));
        // 5. alpha_eff F0g = X: F0g^T alpha^T = X^T over the illuminations
        GDM_TRY(lstsq(ctx, F0g, M6, 1, X, M6, 1, n_ill, (int)M6, (int)M6, aT, Gm, Cm, Rt, flag, norms, nullptr));
        k_transpose<<<nblk(M6 * M6), 256, 0, ctx->stream>>>(aT, (int)M6, (double2 *)alpha_eff);
        GDM_LAUNCHED(ctx, "transpose");
        if (moments)
            GDM_CUDA_TRY(ctx, cudaMemcpyAsync(moments, X, c16 * M6 * n_ill, cudaMemcpyDeviceToDevice, ctx->stream));
        return GDM_OK;
    };
    st = run();
    cudaFreeAsync(buf, ctx->stream);
    return st;
}
