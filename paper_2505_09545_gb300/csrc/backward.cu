// Adjoint backward of the GDM solve (filled in below).
#include "gdm_internal.cuh"

gdm_status gdm_launch_backward(gdm_ctx *ctx, const gdm_problem *p, gdm_precision prec, const void *A, int64_t lda,
                               const int32_t *ipiv, const double *F, int n_rhs, const double *e0, const double *khat,
                               const double *gF, const double *g_sigma, double *grad_pos, double *grad_eps,
                               double *grad_wavelength, gdm_solve_info *info) {
    return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "gdm_backward not built yet");
}

gdm_status gdm_launch_nearfield_backward(gdm_ctx *ctx, const gdm_problem *p, const double *F, const double *r_eval,
                                         int64_t m, int n_rhs, const double *e0, const double *khat, const double *gE,
                                         double *gF_accum, double *grad_pos, double *grad_eps,
                                         double *grad_wavelength) {
    return gdm_fail(ctx, GDM_ERR_UNSUPPORTED, "gdm_nearfield_backward not built yet");
}
