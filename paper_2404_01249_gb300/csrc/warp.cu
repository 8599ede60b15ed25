// Trilinear warp J(x) = I_m(x + u(x)) with the interpolant's gradient
// (section "Preliminaries"; pushforward form of section "Alternative
// formulations for Eulerian differential").
#include "ops.h"
#include "validate.h"

namespace fa {

template <bool GRAD>
__global__ void __launch_bounds__(256) k_warp(const float *__restrict__ Im,
                                              const float *__restrict__ u, float *__restrict__ J,
                                              float *__restrict__ grad, int D, int H, int W) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    if (x >= W || y >= H) return;
    long long N = (long long)D * H * W;
    long long i = ((long long)z * H + y) * W + x;
    float gz, gy, gx;
    float v = tri_sample<GRAD>(Im, D, H, W, z, y, x, __ldg(u + i), __ldg(u + N + i),
                               __ldg(u + 2 * N + i), gz, gy, gx);
    J[i] = v;
    if (GRAD) {
        grad[i] = gz;
        grad[N + i] = gy;
        grad[2 * N + i] = gx;
    }
}

cudaError_t launch_warp(const float *Im, const float *u, float *J, float *grad, Dims d,
                        cudaStream_t s) {
    VoxGrid g(d.D, d.H, d.W);
    if (grad) {
        k_warp<true><<<g.grid, g.block, 0, s>>>(Im, u, J, grad, d.D, d.H, d.W); note_launch();
    }
    else {
        k_warp<false><<<g.grid, g.block, 0, s>>>(Im, u, J, nullptr, d.D, d.H, d.W); note_launch();
    }
    return cudaGetLastError();
}

}  // namespace fa

extern "C" fa_status fa_warp(const fa_vol *moving, const fa_vol *u, fa_vol *out, fa_vol *grad_opt,
                             void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_vol(moving, "moving", 1));
    FA_TRY(check_vol(u, "u", 3));
    FA_TRY(check_vol(out, "out", 1));
    FA_TRY(same_grid(moving, u, "moving", "u"));
    FA_TRY(same_grid(moving, out, "moving", "out"));
    if (grad_opt) {
        FA_TRY(check_vol(grad_opt, "grad", 3));
        FA_TRY(same_grid(moving, grad_opt, "moving", "grad"));
    }
    Dims d{moving->D, moving->H, moving->W};
    FA_CUDA_TRY(launch_warp((const float *)moving->data, (const float *)u->data,
                            (float *)out->data, grad_opt ? (float *)grad_opt->data : nullptr, d,
                            (cudaStream_t)stream));
    return FA_OK;
}
