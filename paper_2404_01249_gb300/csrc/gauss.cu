// Separable Gaussian smoothing (sigma_grad / sigma_warp of the
// hyper-parameter study): taps exp(-k^2 / 2 sigma^2), |k| <= ceil(3 sigma),
// normalised to sum 1, zero padding; one launch per axis (plain form).
#include <math.h>
#include <string.h>

#include "ops.h"
#include "validate.h"

namespace fa {

bool make_gauss_taps(float sigma, GaussTaps *t) {
    memset(t, 0, sizeof(*t));
    if (!(sigma >= 0.0f) || sigma > kMaxSigma) return false;
    if (sigma == 0.0f) {
        t->R = 0;
        t->w[0] = 1.0f;
        return true;
    }
    double sd = (double)sigma;
    int R = (int)ceil(3.0 * sd);
    if (2 * R + 1 > 64) return false;
    double w[64], s = 0.0;
    for (int k = -R; k <= R; ++k) {
        w[k + R] = exp(-(double)k * k / (2.0 * sd * sd));
        s += w[k + R];
    }
    t->R = R;
    for (int k = 0; k <= 2 * R; ++k) t->w[k] = (float)(w[k] / s);
    return true;
}

template <int AXIS>
__global__ void __launch_bounds__(256) k_gauss_axis(const float *__restrict__ in,
                                                    float *__restrict__ out, int C, int D, int H,
                                                    int W, GaussTaps t) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    if (x >= W || y >= H) return;
    long long N = (long long)D * H * W;
    long long i = ((long long)z * H + y) * W + x;
    const int c0 = AXIS == 0 ? x : (AXIS == 1 ? y : z);
    const int n = AXIS == 0 ? W : (AXIS == 1 ? H : D);
    const long long stride = AXIS == 0 ? 1ll : (AXIS == 1 ? (long long)W : (long long)H * W);
    const int R = t.R;
    int lo = max(-R, -c0), hi = min(R, n - 1 - c0);
    for (int c = 0; c < C; ++c) {
        const float *src = in + c * N + i;
        float acc = 0.0f;
        for (int k = lo; k <= hi; ++k) acc = fmaf(t.w[k + R], __ldg(src + k * stride), acc);
        out[c * N + i] = acc;
    }
}

cudaError_t launch_gauss_axis(const float *in, float *out, int C, Dims d, const GaussTaps &t,
                              int axis, cudaStream_t s) {
    VoxGrid g(d.D, d.H, d.W);
    if (axis == 0) {
        k_gauss_axis<0><<<g.grid, g.block, 0, s>>>(in, out, C, d.D, d.H, d.W, t); note_launch();
    }
    else if (axis == 1) {
        k_gauss_axis<1><<<g.grid, g.block, 0, s>>>(in, out, C, d.D, d.H, d.W, t); note_launch();
    }
    else {
        k_gauss_axis<2><<<g.grid, g.block, 0, s>>>(in, out, C, d.D, d.H, d.W, t); note_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_gauss3(const float *in, float *out, float *t1, float *t2, int C, Dims d,
                          const GaussTaps &t, cudaStream_t s) {
    if (t.R == 0) {
        if (in == out) return cudaSuccess;
        return cudaMemcpyAsync(out, in, sizeof(float) * C * d.N(), cudaMemcpyDeviceToDevice, s);
    }
    cudaError_t e;
    if ((e = launch_gauss_axis(in, t1, C, d, t, 0, s)) != cudaSuccess) return e;
    if ((e = launch_gauss_axis(t1, t2, C, d, t, 1, s)) != cudaSuccess) return e;
    return launch_gauss_axis(t2, out, C, d, t, 2, s);
}

}  // namespace fa

extern "C" size_t fa_gauss_workspace_size(int32_t C, int32_t D, int32_t H, int32_t W) {
    if (C < 1 || D < 1 || H < 1 || W < 1) return 0;
    fa::WsCarver c(nullptr, ~size_t(0));
    c.take<float>((size_t)C * D * H * W);
    c.take<float>((size_t)C * D * H * W);
    return c.off;
}

extern "C" fa_status fa_gauss_smooth(const fa_vol *in, fa_vol *out, float sigma, void *ws,
                                     size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    if (!in) {
        set_error("in: descriptor is NULL");
        return FA_ERR_INVALID;
    }
    FA_TRY(check_vol(in, "in", in->C));
    FA_TRY(check_vol(out, "out", in->C));
    FA_TRY(same_grid(in, out, "in", "out"));
    GaussTaps t;
    if (!make_gauss_taps(sigma, &t)) {
        set_error("fa_gauss_smooth: sigma must be in [0, %g] (got %g)", (double)kMaxSigma,
                  (double)sigma);
        return FA_ERR_INVALID;
    }
    size_t need = t.R ? fa_gauss_workspace_size(in->C, in->D, in->H, in->W) : 0;
    FA_TRY(check_ws(ws, ws_bytes, need, "fa_gauss_smooth"));
    Dims d{in->D, in->H, in->W};
    float *t1 = nullptr, *t2 = nullptr;
    if (t.R) {
        WsCarver c(ws, ws_bytes);
        t1 = c.take<float>((size_t)in->C * d.N());
        t2 = c.take<float>((size_t)in->C * d.N());
    }
    FA_CUDA_TRY(launch_gauss3((const float *)in->data, (float *)out->data, t1, t2, in->C, d, t,
                              (cudaStream_t)stream));
    return FA_OK;
}
