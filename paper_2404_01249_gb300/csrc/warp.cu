// Trilinear warp J(x) = I_m(x + u(x)) with the interpolant's gradient
// (section "Preliminaries"; pushforward form of section "Alternative
// formulations for Eulerian differential").
#include "ops.h"
#include "validate.h"

namespace fa {

// Every buffer has rows of P (>= W) elements; only x < W is read or written.
// u: FP32 or FP16 values.
template <bool GRAD, class TU>
__global__ void __launch_bounds__(256) k_warp(const float *__restrict__ Im,
                                              const TU *__restrict__ u, float *__restrict__ J,
                                              float *__restrict__ grad, int D, int H, int W,
                                              int P) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    if (x >= W || y >= H) return;
    long long N = (long long)D * H * P;
    long long i = ((long long)z * H + y) * P + x;
    float gz, gy, gx;
    float v = tri_sample_p<GRAD>(Im, D, H, W, P, z, y, x, ld_field(u + i), ld_field(u + N + i),
                                 ld_field(u + 2 * N + i), gz, gy, gx);
    J[i] = v;
    if (GRAD) {
        grad[i] = gz;
        grad[N + i] = gy;
        grad[2 * N + i] = gx;
    }
}

template <class TU>
static cudaError_t launch_warp_t(const float *Im, const TU *u, float *J, float *grad, Dims d,
                                 cudaStream_t s) {
    VoxGrid g(d.D, d.H, d.W);
    if (grad)
        k_warp<true><<<g.grid, g.block, 0, s>>>(Im, u, J, grad, d.D, d.H, d.W, d.pitch());
    else
        k_warp<false><<<g.grid, g.block, 0, s>>>(Im, u, J, nullptr, d.D, d.H, d.W, d.pitch());
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_warp(const float *Im, const float *u, float *J, float *grad, Dims d,
                        cudaStream_t s) {
    return launch_warp_t(Im, u, J, grad, d, s);
}

cudaError_t launch_warp_field(const float *Im, const void *u, int field, float *J, float *grad,
                              Dims d, cudaStream_t s) {
    if (field == FA_F16) return launch_warp_t(Im, (const __half *)u, J, grad, d, s);
    return launch_warp_t(Im, (const float *)u, J, grad, d, s);
}


// Steepest Eulerian direction (section "Exploiting the group structure of
// diffeomorphisms", the use_jac option of Algorithm 1): g <- J(phi)^T g with
// J(phi) = I + grad u, grad u by central differences inside the grid and
// one-sided first differences at its ends (zero on an axis of length 1).
// In place: each output reads only its own voxel of g.
__device__ __forceinline__ float fd_axis(const float *__restrict__ f, int n, int k, long long i,
                                         long long stride) {
    if (n < 2) return 0.0f;
    if (k == 0) return __ldg(f + i + stride) - __ldg(f + i);
    if (k == n - 1) return __ldg(f + i) - __ldg(f + i - stride);
    return 0.5f * (__ldg(f + i + stride) - __ldg(f + i - stride));
}

__global__ void __launch_bounds__(256) k_jac_direction(const float *gin, const float *__restrict__ u,
                                                       float *gout, int D, int H, int W) {
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= W || y >= H) return;
    const long long N = (long long)D * H * W, HW = (long long)H * W;
    const long long i = (long long)z * HW + (long long)y * W + x;
    const float g0 = gin[i], g1 = gin[N + i], g2 = gin[2 * N + i];
    float out[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {  // component a: g_a + sum_j (d u_j / d x_a) g_j
        const int n = a == 0 ? D : (a == 1 ? H : W), k = a == 0 ? z : (a == 1 ? y : x);
        const long long st = a == 0 ? HW : (a == 1 ? (long long)W : 1ll);
        const float ga = a == 0 ? g0 : (a == 1 ? g1 : g2);
        float s = ga;
        s = fmaf(fd_axis(u, n, k, i, st), g0, s);
        s = fmaf(fd_axis(u + N, n, k, i, st), g1, s);
        s = fmaf(fd_axis(u + 2 * N, n, k, i, st), g2, s);
        out[a] = s;
    }
    gout[i] = out[0];
    gout[N + i] = out[1];
    gout[2 * N + i] = out[2];
}

cudaError_t launch_jac_direction(const float *gin, const float *u, float *gout, Dims d,
                                 cudaStream_t s) {
    VoxGrid g(d.D, d.H, d.W);
    k_jac_direction<<<g.grid, g.block, 0, s>>>(gin, u, gout, d.D, d.H, d.W);
    note_launch();
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

extern "C" fa_status fa_jac_direction(const fa_vol *g_in, const fa_vol *u, fa_vol *g_out,
                                      void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_vol(g_in, "g_in", 3));
    FA_TRY(check_vol(u, "u", 3));
    FA_TRY(check_vol(g_out, "g_out", 3));
    FA_TRY(same_grid(g_in, u, "g_in", "u"));
    FA_TRY(same_grid(g_in, g_out, "g_in", "g_out"));
    if (g_out->data != g_in->data) {
        const size_t n = 3 * (size_t)g_in->D * g_in->H * g_in->W * sizeof(float);
        const char *a = (const char *)g_in->data, *b = (const char *)g_out->data;
        if (a < b + n && b < a + n) {
            set_error("fa_jac_direction: g_out must equal g_in or not overlap it");
            return FA_ERR_INVALID;
        }
    }
    Dims d{g_in->D, g_in->H, g_in->W};
    FA_CUDA_TRY(launch_jac_direction((const float *)g_in->data, (const float *)u->data,
                                     (float *)g_out->data, d, (cudaStream_t)stream));
    return FA_OK;
}
