// tcgen05 tensor-core trailing update for the FP32 LU (filled in below).
#include "gdm_internal.cuh"

size_t gdm_tc_workspace_bytes(int64_t n, int64_t nb, gdm_precision prec) { return 0; }

gdm_status gdm_tc_trailing_update(gdm_ctx *ctx, gdm_precision prec, float2 *A, int64_t lda, int64_t n, int64_t b0,
                                  int64_t nb, void *ws, size_t ws_bytes) {
    return GDM_ERR_UNSUPPORTED;
}
