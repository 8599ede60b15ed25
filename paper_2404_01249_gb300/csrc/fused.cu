// Fused per-iteration kernels of fa_register (FA_MODE_FUSED).
#include "register.h"
#include "validate.h"

namespace fa {

void fused_carve(WsCarver &c, long long n, FusedBuffers *fb) {
    fb->coef = c.take<float>(3 * n);
    fb->g = c.take<float>(3 * n);
    fb->dir = c.take<float>(3 * n);
    fb->J = c.take<float>(n);
}

fa_status fused_iteration(FusedBuffers &, WsHeader *, const fa_params *, Dims, const FusedIter &,
                          const GaussTaps &, const GaussTaps &, fa_kernel_timer *, int,
                          cudaStream_t) {
    set_error("fused mode is not built yet");
    return FA_ERR_UNSUPPORTED;
}

cudaError_t fused_lncc_forward_only(const float *, const float *, Dims, int, float, WsHeader *,
                                    FusedBuffers &, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace fa
