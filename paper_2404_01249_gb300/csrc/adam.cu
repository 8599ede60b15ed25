// Adam on the Jacobian-free descent directions (section "Adaptive
// optimization on diffeomorphisms"), the step size eps_t = lr / (c_lp
// max|d|) of the appendix "Limitations of Stationary Velocity Fields", and
// the compositive update phi <- phi o (id + delta) (section "Minimizing the
// Eulerian differential", Algorithm 1).  Plain per-op kernels.
#include <math.h>

#include "ops.h"
#include "validate.h"

namespace fa {

template <class TS>
__device__ __forceinline__ void adam_body(const float *__restrict__ g, TS *__restrict__ m,
                                          TS *__restrict__ v, float *__restrict__ d, long long N,
                                          const AdamConsts &c, WsHeader *h, int parity) {
    __shared__ float red[32];
    float nrm2 = 0.0f;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    bool bad = false;
    if (i < N) {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            long long k = ch * N + i;
            float gv = g[k];
            float mv = fmaf(c.b1, st_load(m[k]), (1.0f - c.b1) * gv);
            float vv = fmaf(c.b2, st_load(v[k]), (1.0f - c.b2) * gv * gv);
            m[k] = st_store<TS>(mv);
            v[k] = st_store<TS>(vv);
            float dv = adam_dir(mv, vv, c.rbc1, c.rbc2, c.eps);
            d[k] = dv;
            nrm2 = fmaf(dv, dv, nrm2);
        }
        if (!(nrm2 <= 3.4e38f)) {
            bad = true;
            nrm2 = 0.0f;
        }
    }
    if (bad) status_set(&h->status, ST_NONFINITE);
    block_max_to(&h->step_max_bits[parity], sqrtf(nrm2), red);
}

template <class TS>
__global__ void __launch_bounds__(256) k_adam(const float *__restrict__ g, TS *__restrict__ m,
                                              TS *__restrict__ v, float *__restrict__ d,
                                              long long N, AdamConsts c, WsHeader *h,
                                              int parity) {
    adam_body<TS>(g, m, v, d, N, c, h, parity);
}

// 1 / (1 - b^t) in FP32: 1 - b^t = -expm1(t log1p(b - 1)), with b - 1 exact
// for b in [0.5, 1); log1p and expm1 keep their relative accuracy where b^t
// is close to 1 (large beta2, small t), which 1 - powf(b, t) would not.
__device__ __forceinline__ float bias_recip(float b, int t) {
    return -1.0f / expm1f((float)t * log1pf(b - 1.0f));
}

// The same step with the step number taken from the device counter:
// t = *t_dev + 1 (the counter itself is advanced by k_count_step after the
// compose, so that every block here reads the same value).
template <class TS>
__global__ void __launch_bounds__(256) k_adam_tdev(const float *__restrict__ g,
                                                   TS *__restrict__ m, TS *__restrict__ v,
                                                   float *__restrict__ d, long long N, float b1,
                                                   float b2, float eps,
                                                   const int *__restrict__ t_dev, WsHeader *h) {
    const int t = *t_dev + 1;
    if (t < 1) {  // a counter below zero: uniform over the block
        if (threadIdx.x == 0) status_set(&h->status, ST_NONFINITE);
        return;
    }
    AdamConsts c;
    c.b1 = b1;
    c.b2 = b2;
    c.eps = eps;
    c.rbc1 = bias_recip(b1, t);
    c.rbc2 = bias_recip(b2, t);
    adam_body<TS>(g, m, v, d, N, c, h, 0);
}

__global__ void k_count_step(int *t_dev) { *t_dev += 1; }

__global__ void __launch_bounds__(256) k_compose(const float *__restrict__ u,
                                                 const float *__restrict__ d,
                                                 float *__restrict__ uo, int D, int H, int W,
                                                 float lr, float c_lp, WsHeader *h, int parity,
                                                 float *eps_out) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    float mx = __uint_as_float(h->step_max_bits[parity]);
    float e = (mx > 0.0f) ? lr / (c_lp * mx) : 0.0f;
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
        threadIdx.y == 0) {
        h->step_max_bits[parity ^ 1] = 0u;  // slot of the next iteration
        h->eps_t = e;
        if (eps_out) *eps_out = e;
    }
    if (x >= W || y >= H) return;
    long long N = (long long)D * H * W;
    long long i = ((long long)z * H + y) * W + x;
    float dz = -e * d[i], dy = -e * d[N + i], dx = -e * d[2 * N + i];
    float gz, gy, gx;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        TriPending q;  // the compose's cell (the same as the fused schedule's)
        tri_issue_step(q, u + ch * N, D, H, W, W, z, y, x, dz, dy, dx);
        float s = tri_finish<false>(q, gz, gy, gx);
        float dc = ch == 0 ? dz : (ch == 1 ? dy : dx);
        uo[ch * N + i] = dc + s;
    }
}

// u'(x) = delta(x) + u(x + delta(x)) (the compositive update with a given
// step field; zero outside).  uo must not alias u; it may alias delta only
// if each thread's delta is read before its writes (it is).
__global__ void __launch_bounds__(256) k_compose_fields(const float *__restrict__ u,
                                                        const float *delta, float *uo, int D,
                                                        int H, int W) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    if (x >= W || y >= H) return;
    long long N = (long long)D * H * W;
    long long i = ((long long)z * H + y) * W + x;
    const float dz = delta[i], dy = delta[N + i], dx = delta[2 * N + i];
    float gz, gy, gx, r[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch)
        r[ch] = tri_sample<false>(u + ch * N, D, H, W, z, y, x, dz, dy, dx, gz, gy, gx);
    uo[i] = dz + r[0];
    uo[N + i] = dy + r[1];
    uo[2 * N + i] = dx + r[2];
}

__global__ void __launch_bounds__(256) k_scale_field(const float *__restrict__ v, float *out,
                                                     long long n, float s) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = v[i] * s;
}

cudaError_t launch_compose_fields(const float *u, const float *delta, float *uo, Dims d,
                                  cudaStream_t s) {
    VoxGrid g(d.D, d.H, d.W);
    k_compose_fields<<<g.grid, g.block, 0, s>>>(u, delta, uo, d.D, d.H, d.W);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_adam(const float *g, float *m, float *v, float *d, long long N, AdamConsts c,
                        WsHeader *h, int parity, cudaStream_t s) {
    long long blocks = (N + 255) / 256;
    k_adam<float><<<(unsigned)blocks, 256, 0, s>>>(g, m, v, d, N, c, h, parity); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_adam_state(const float *g, void *m, void *v, int state, float *d, long long N,
                              AdamConsts c, WsHeader *h, int parity, cudaStream_t s) {
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (state == FA_BF16)
        k_adam<__nv_bfloat16><<<blocks, 256, 0, s>>>(g, (__nv_bfloat16 *)m, (__nv_bfloat16 *)v, d,
                                                     N, c, h, parity);
    else if (state == FA_F16)
        k_adam<__half><<<blocks, 256, 0, s>>>(g, (__half *)m, (__half *)v, d, N, c, h, parity);
    else
        k_adam<float><<<blocks, 256, 0, s>>>(g, (float *)m, (float *)v, d, N, c, h, parity);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_adam_tdev(const float *g, void *m, void *v, int state, float *d, long long N,
                             const fa_params *p, const int *t_dev, WsHeader *h, cudaStream_t s) {
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (state == FA_BF16)
        k_adam_tdev<__nv_bfloat16><<<blocks, 256, 0, s>>>(g, (__nv_bfloat16 *)m, (__nv_bfloat16 *)v,
                                                          d, N, p->beta1, p->beta2, p->adam_eps,
                                                          t_dev, h);
    else if (state == FA_F16)
        k_adam_tdev<__half><<<blocks, 256, 0, s>>>(g, (__half *)m, (__half *)v, d, N, p->beta1,
                                                   p->beta2, p->adam_eps, t_dev, h);
    else
        k_adam_tdev<float><<<blocks, 256, 0, s>>>(g, (float *)m, (float *)v, d, N, p->beta1,
                                                  p->beta2, p->adam_eps, t_dev, h);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_compose(const float *u_in, const float *d, float *u_out, Dims dm, float lr,
                           float c_lp, WsHeader *h, int parity, float *eps_out, cudaStream_t s) {
    VoxGrid g(dm.D, dm.H, dm.W);
    k_compose<<<g.grid, g.block, 0, s>>>(u_in, d, u_out, dm.D, dm.H, dm.W, lr, c_lp, h, parity,
                                         eps_out); note_launch();
    return cudaGetLastError();
}

AdamConsts adam_consts(const fa_params *p, int t) {
    AdamConsts c;
    c.b1 = p->beta1;
    c.b2 = p->beta2;
    c.eps = p->adam_eps;
    c.rbc1 = (float)(1.0 / (1.0 - pow((double)p->beta1, (double)t)));
    c.rbc2 = (float)(1.0 / (1.0 - pow((double)p->beta2, (double)t)));
    return c;
}

fa_status check_adam_params(const fa_params *p, const char *who, bool state16_ok) {
    if (!p) {
        set_error("%s: params are NULL", who);
        return FA_ERR_INVALID;
    }
    if (!state16_ok && p->state_storage != FA_F32) {
        set_error("%s: keeps its Adam moments in FP32 (state_storage must be FA_F32)", who);
        return FA_ERR_UNSUPPORTED;
    }
    if (!state16_ok && p->field_storage != FA_F32) {
        set_error("%s: keeps its fields in FP32 (field_storage must be FA_F32)", who);
        return FA_ERR_UNSUPPORTED;
    }
    if (!(p->beta1 >= 0.0f && p->beta1 < 1.0f) || !(p->beta2 >= 0.0f && p->beta2 < 1.0f) ||
        !(p->adam_eps >= 0.0f) || !(p->lr > 0.0f && p->lr < 1e30f) ||
        !(p->c_lp > 0.0f && p->c_lp < 1e30f)) {
        set_error("%s: need 0 <= beta < 1, adam_eps >= 0, lr > 0, c_lp > 0", who);
        return FA_ERR_INVALID;
    }
    return FA_OK;
}

}  // namespace fa

extern "C" size_t fa_radam_workspace_size(int32_t D, int32_t H, int32_t W) {
    if (D < 1 || H < 1 || W < 1) return 0;
    fa::WsCarver c(nullptr, ~size_t(0));
    c.take<fa::WsHeader>(1);
    c.take<float>(3 * (size_t)D * H * W);
    return c.off;
}

extern "C" fa_status fa_radam_step(const fa_vol *u_in, fa_vol *u_out, fa_vol *m, fa_vol *v,
                                   const fa_vol *g, int32_t *t_dev, const fa_params *p,
                                   float *eps_t_dev, void *ws, size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_vol(u_in, "u_in", 3));
    FA_TRY(check_vol(u_out, "u_out", 3));
    if (m && m->dtype != FA_F32 && m->dtype != FA_BF16 && m->dtype != FA_F16) {
        set_error("fa_radam_step: m must be FA_F32, FA_BF16 or FA_F16 (got %d)", (int)m->dtype);
        return FA_ERR_DTYPE;
    }
    FA_TRY(check_vol_dtype(m, "m", 3, m ? m->dtype : FA_F32));
    FA_TRY(check_vol_dtype(v, "v", 3, m->dtype));
    FA_TRY(check_vol(g, "g", 3));
    FA_TRY(same_grid(u_in, u_out, "u_in", "u_out"));
    FA_TRY(same_grid(u_in, m, "u_in", "m"));
    FA_TRY(same_grid(u_in, v, "u_in", "v"));
    FA_TRY(same_grid(u_in, g, "u_in", "g"));
    if (u_in->data == u_out->data) {
        set_error("fa_radam_step: u_out must not alias u_in");
        return FA_ERR_INVALID;
    }
    if (!t_dev || ((uintptr_t)t_dev & 3u)) {
        set_error("fa_radam_step: t_dev must be a 4-byte aligned device int32");
        return FA_ERR_INVALID;
    }
    FA_TRY(check_adam_params(p, "fa_radam_step", true));  // m, v carry their own dtype
    FA_TRY(check_ws(ws, ws_bytes, fa_radam_workspace_size(u_in->D, u_in->H, u_in->W),
                    "fa_radam_step"));
    cudaStream_t s = (cudaStream_t)stream;
    Dims d{u_in->D, u_in->H, u_in->W};
    WsCarver c(ws, ws_bytes);
    WsHeader *h = c.take<WsHeader>(1);
    float *dir = c.take<float>(3 * d.N());
    FA_CUDA_TRY(launch_header_reset(h, s));
    FA_CUDA_TRY(launch_adam_tdev((const float *)g->data, m->data, v->data, m->dtype, dir, d.N(), p,
                                 t_dev, h, s));
    FA_CUDA_TRY(launch_compose((const float *)u_in->data, dir, (float *)u_out->data, d, p->lr,
                               p->c_lp, h, 0, eps_t_dev, s));
    k_count_step<<<1, 1, 0, s>>>(t_dev);
    note_launch();
    FA_CUDA_TRY(cudaGetLastError());
    return FA_OK;
}

extern "C" fa_status fa_compose(const fa_vol *u, const fa_vol *delta, fa_vol *out, void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_vol(u, "u", 3));
    FA_TRY(check_vol(delta, "delta", 3));
    FA_TRY(check_vol(out, "out", 3));
    FA_TRY(same_grid(u, delta, "u", "delta"));
    FA_TRY(same_grid(u, out, "u", "out"));
    if (out->data == u->data) {
        set_error("fa_compose: out must not be u");
        return FA_ERR_INVALID;
    }
    Dims d{u->D, u->H, u->W};
    FA_CUDA_TRY(launch_compose_fields((const float *)u->data, (const float *)delta->data,
                                      (float *)out->data, d, (cudaStream_t)stream));
    return FA_OK;
}

extern "C" size_t fa_svf_exp_workspace_size(int32_t D, int32_t H, int32_t W) {
    fa::clear_error();
    if (D < 1 || H < 1 || W < 1) return 0;
    return ((size_t)3 * D * H * W * sizeof(float) + 255) & ~(size_t)255;
}

extern "C" fa_status fa_svf_exp(const fa_vol *v, int32_t steps, fa_vol *out, void *ws,
                                size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_vol(v, "v", 3));
    FA_TRY(check_vol(out, "out", 3));
    FA_TRY(same_grid(v, out, "v", "out"));
    if (steps < 0 || steps > 30) {
        set_error("fa_svf_exp: steps must be in 0..30 (got %d)", (int)steps);
        return FA_ERR_INVALID;
    }
    Dims d{v->D, v->H, v->W};
    FA_TRY(check_ws(ws, ws_bytes, fa_svf_exp_workspace_size(d.D, d.H, d.W), "fa_svf_exp"));
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = 3 * d.N();
    float *a = (float *)out->data, *b = (float *)ws;
    // an odd number of squarings starts in the workspace so the last lands in out
    float *cur = (steps & 1) ? b : a, *nxt = (steps & 1) ? a : b;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_scale_field<<<(unsigned)blocks, 256, 0, s>>>((const float *)v->data, cur, n,
                                                   ldexpf(1.0f, -steps));
    note_launch();
    FA_CUDA_TRY(cudaGetLastError());
    for (int k = 0; k < steps; ++k) {  // phi <- phi o phi
        FA_CUDA_TRY(launch_compose_fields(cur, cur, nxt, d, s));
        float *t = cur;
        cur = nxt;
        nxt = t;
    }
    return FA_OK;
}
