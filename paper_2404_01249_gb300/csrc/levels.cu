// Pyramid levels (Algorithm 1 "downsample"; section "Interpolation strategies
// for multi-scale registration") and the trilinear level hand-off of u, m, nu
// (Algorithm 1 "Upsample").  Align-corners: index i of an n_dst axis samples
// source coordinate i (n_src - 1) / (n_dst - 1).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ops.h"
#include "validate.h"

namespace fa {

__device__ __forceinline__ float ac_coord(int i, int ns, int nd) {
    if (nd <= 1 || ns <= 1) return 0.0f;
    return (float)(i * (ns - 1)) / (float)(nd - 1);  // both exact; one rounding
}

struct Scale3 {
    float s[3];
};

// Rows of Ps (source) and Pd (destination) elements; only x < W is read or
// written.  TS, TD: FP32 or FP16 (a 16-bit destination is rounded to nearest).
template <class TS, class TD>
__global__ void __launch_bounds__(256) k_resample(const TS *__restrict__ src, int Ds, int Hs,
                                                  int Ws, int Ps, TD *__restrict__ dst, int Dd,
                                                  int Hd, int Wd, int Pd, int C, Scale3 sc) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    if (x >= Wd || y >= Hd) return;
    long long Ns = (long long)Ds * Hs * Ps, Nd = (long long)Dd * Hd * Pd;
    long long i = ((long long)z * Hd + y) * Pd + x;
    float cz = ac_coord(z, Ds, Dd), cy = ac_coord(y, Hs, Hd), cx = ac_coord(x, Ws, Wd);
    float gz, gy, gx;
    for (int c = 0; c < C; ++c) {
        float v = tri_sample_p<false>(src + c * Ns, Ds, Hs, Ws, Ps, 0, 0, 0, cz, cy, cx, gz, gy,
                                      gx);
        dst[c * Nd + i] = st_store<TD>(v * sc.s[c]);
    }
}

template <class TS, class TD>
static cudaError_t launch_resample_t(const TS *src, Dims ds, TD *dst, Dims dd, int C,
                                     const float *scale3, cudaStream_t s) {
    Scale3 sc;
    for (int c = 0; c < 3; ++c) sc.s[c] = scale3 ? scale3[c] : 1.0f;
    VoxGrid g(dd.D, dd.H, dd.W);
    k_resample<<<g.grid, g.block, 0, s>>>(src, ds.D, ds.H, ds.W, ds.pitch(), dst, dd.D, dd.H, dd.W,
                                          dd.pitch(), C, sc);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_resample(const float *src, Dims ds, float *dst, Dims dd, int C,
                            const float *scale3, cudaStream_t s) {
    return launch_resample_t(src, ds, dst, dd, C, scale3, s);
}

cudaError_t launch_resample_field(const void *src, int sfield, Dims ds, void *dst, int dfield,
                                  Dims dd, int C, const float *scale3, cudaStream_t s) {
    if (sfield == FA_F16 && dfield == FA_F16)
        return launch_resample_t((const __half *)src, ds, (__half *)dst, dd, C, scale3, s);
    if (sfield == FA_F16)
        return launch_resample_t((const __half *)src, ds, (float *)dst, dd, C, scale3, s);
    if (dfield == FA_F16)
        return launch_resample_t((const float *)src, ds, (__half *)dst, dd, C, scale3, s);
    return launch_resample_t((const float *)src, ds, (float *)dst, dd, C, scale3, s);
}

int level_size(int n, int s) {
    int m = s > 0 ? n / s : 0;
    return m < 1 ? 1 : m;
}

// Per-axis hand-off factor s_a^power, s_a = (nf - 1) / (nc - 1) (1 if degenerate).
void handoff_scales(Dims c, Dims f, int power, float out[3]) {
    int nc[3] = {c.D, c.H, c.W}, nf[3] = {f.D, f.H, f.W};
    for (int a = 0; a < 3; ++a) {
        double s = (nc[a] <= 1 || nf[a] <= 1) ? 1.0 : (double)(nf[a] - 1) / (double)(nc[a] - 1);
        double v = power == 1 ? s : (power == -1 ? 1.0 / s : 1.0 / (s * s));
        out[a] = (float)v;
    }
}

// Blur (sigma = s / 2) then resample; t1, t2: N floats of the input grid
// (which has no row padding); the level may have a row pitch of its own.
cudaError_t launch_pyramid_level(const float *img, Dims d, int s, float *out, Dims dl, float *t1,
                                 float *t2, cudaStream_t st) {
    if (s == 1)
        return cudaMemcpy2DAsync(out, sizeof(float) * dl.pitch(), img, sizeof(float) * d.pitch(),
                                 sizeof(float) * d.W, (size_t)d.D * d.H, cudaMemcpyDeviceToDevice,
                                 st);
    GaussTaps t;
    if (!make_gauss_taps(0.5f * (float)s, &t)) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = launch_gauss_axis(img, t1, 1, d, t, 0, st)) != cudaSuccess) return e;
    if ((e = launch_gauss_axis(t1, t2, 1, d, t, 1, st)) != cudaSuccess) return e;
    if ((e = launch_gauss_axis(t2, t1, 1, d, t, 2, st)) != cudaSuccess) return e;
    return launch_resample(t1, d, out, dl, 1, nullptr, st);
}

// 16-bit input images widened to FP32 (exact for both formats).
__global__ void __launch_bounds__(256) k_widen(const unsigned short *__restrict__ src, int dtype,
                                               float *__restrict__ dst, long long n) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned short b = src[i];
        dst[i] = dtype == FA_BF16 ? __uint_as_float((unsigned)b << 16)
                                  : __half2float(__ushort_as_half(b));
    }
}

cudaError_t launch_widen(const void *src, int dtype, float *dst, long long n, cudaStream_t s) {
    const long long blocks = (n + 255) / 256;
    k_widen<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(
        (const unsigned short *)src, dtype, dst, n);
    note_launch();
    return cudaGetLastError();
}

// FP32 values rounded to nearest into 16-bit storage (the inverse of k_widen
// up to that rounding).
__global__ void __launch_bounds__(256) k_narrow(const float *__restrict__ src, int dtype,
                                                unsigned short *__restrict__ dst, long long n) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = dtype == FA_BF16 ? __bfloat16_as_ushort(__float2bfloat16_rn(src[i]))
                                  : __half_as_ushort(__float2half_rn(src[i]));
}

cudaError_t launch_narrow(const float *src, int dtype, void *dst, long long n, cudaStream_t s) {
    const long long blocks = (n + 255) / 256;
    k_narrow<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(
        src, dtype, (unsigned short *)dst, n);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fa

extern "C" fa_status fa_pyramid_level(const fa_vol *img, int32_t s, fa_vol *out, void *ws,
                                      size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_vol(img, "img", 1));
    FA_TRY(check_vol(out, "out", 1));
    if (s < 1 || 0.5f * (float)s > kMaxSigma) {
        set_error("fa_pyramid_level: scale must be in 1..%d (got %d)", (int)(2 * kMaxSigma),
                  (int)s);
        return FA_ERR_INVALID;
    }
    Dims d{img->D, img->H, img->W};
    Dims dl{level_size(d.D, s), level_size(d.H, s), level_size(d.W, s)};
    if (out->D != dl.D || out->H != dl.H || out->W != dl.W) {
        set_error("fa_pyramid_level: out must be %dx%dx%d for scale %d", dl.D, dl.H, dl.W, (int)s);
        return FA_ERR_SHAPE;
    }
    size_t need = s == 1 ? 0 : fa_gauss_workspace_size(1, d.D, d.H, d.W);
    FA_TRY(check_ws(ws, ws_bytes, need, "fa_pyramid_level"));
    float *t1 = nullptr, *t2 = nullptr;
    if (s > 1) {
        WsCarver c(ws, ws_bytes);
        t1 = c.take<float>(d.N());
        t2 = c.take<float>(d.N());
    }
    FA_CUDA_TRY(launch_pyramid_level((const float *)img->data, d, s, (float *)out->data, dl, t1, t2,
                                     (cudaStream_t)stream));
    return FA_OK;
}

extern "C" fa_status fa_upsample_field(const fa_vol *coarse, fa_vol *fine, int32_t power,
                                       void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_vol(coarse, "coarse", 3));
    FA_TRY(check_vol(fine, "fine", 3));
    if (power != 1 && power != -1 && power != -2) {
        set_error("fa_upsample_field: power must be 1, -1 or -2");
        return FA_ERR_INVALID;
    }
    if (coarse->data == fine->data) {
        set_error("fa_upsample_field: fine must not alias coarse");
        return FA_ERR_INVALID;
    }
    Dims c{coarse->D, coarse->H, coarse->W}, f{fine->D, fine->H, fine->W};
    float sc[3];
    handoff_scales(c, f, power, sc);
    FA_CUDA_TRY(launch_resample((const float *)coarse->data, c, (float *)fine->data, f, 3, sc,
                                (cudaStream_t)stream));
    return FA_OK;
}

extern "C" size_t fa_pyramid_workspace_size(int32_t D, int32_t H, int32_t W, const fa_params *p) {
    using namespace fa;
    clear_error();
    if (D < 1 || H < 1 || W < 1 || !p || p->n_levels < 1 || p->n_levels > 8) return 0;
    bool blur = false;
    for (int l = 0; l < p->n_levels; ++l) {
        if (p->scales[l] < 1 || 0.5f * (float)p->scales[l] > kMaxSigma) return 0;
        blur = blur || p->scales[l] > 1;
    }
    // two full-grid temporaries shared by every blurred level (256 bytes
    // when no level is blurred, so that a valid request never reads as 0)
    return blur ? fa_gauss_workspace_size(1, D, H, W) : 256;
}

extern "C" fa_status fa_pyramid(const fa_vol *img, const fa_params *p, fa_vol *levels, void *ws,
                                size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_vol(img, "img", 1));
    if (!p || !levels) {
        set_error("fa_pyramid: params and levels must not be NULL");
        return FA_ERR_INVALID;
    }
    if (p->n_levels < 1 || p->n_levels > 8) {
        set_error("fa_pyramid: n_levels must be in 1..8 (got %d)", (int)p->n_levels);
        return FA_ERR_INVALID;
    }
    const Dims d{img->D, img->H, img->W};
    for (int l = 0; l < p->n_levels; ++l) {
        const int sc = p->scales[l];
        if (sc < 1 || 0.5f * (float)sc > kMaxSigma) {
            set_error("fa_pyramid: scales[%d] must be in 1..%d (got %d)", l, (int)(2 * kMaxSigma),
                      sc);
            return FA_ERR_INVALID;
        }
        FA_TRY(check_vol(&levels[l], "levels[l]", 1));
        const Dims dl{level_size(d.D, sc), level_size(d.H, sc), level_size(d.W, sc)};
        if (levels[l].D != dl.D || levels[l].H != dl.H || levels[l].W != dl.W) {
            set_error("fa_pyramid: levels[%d] must be %dx%dx%d for scale %d", l, dl.D, dl.H, dl.W,
                      sc);
            return FA_ERR_SHAPE;
        }
        if (levels[l].data == img->data) {
            set_error("fa_pyramid: levels[%d] must not alias img", l);
            return FA_ERR_INVALID;
        }
    }
    FA_TRY(check_ws(ws, ws_bytes, fa_pyramid_workspace_size(d.D, d.H, d.W, p), "fa_pyramid"));
    WsCarver c(ws, ws_bytes);
    float *t1 = c.take<float>(d.N());
    float *t2 = c.take<float>(d.N());
    for (int l = 0; l < p->n_levels; ++l) {
        const int sc = p->scales[l];
        const Dims dl{level_size(d.D, sc), level_size(d.H, sc), level_size(d.W, sc)};
        FA_CUDA_TRY(launch_pyramid_level((const float *)img->data, d, sc, (float *)levels[l].data,
                                         dl, t1, t2, (cudaStream_t)stream));
    }
    return FA_OK;
}
