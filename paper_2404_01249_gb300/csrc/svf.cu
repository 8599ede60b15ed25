// The Lie-algebra ("exp") registration the paper compares its method with
// (section "Euclidean gradient descent using the Lie algebra in shooting
// methods"): a stationary velocity v is optimised, phi = exp(v) by scaling
// and squaring (Eqs. ssbasecase and scalingandsquaring: u_0 = v / 2^M,
// u_{k+1} = u_k + u_k o (id + u_k)), and dL/dphi is pulled back into the
// algebra by the exact adjoint of the squarings,
//   gbar_k(x) = (I + grad u_k(x + u_k(x)))^T gbar_{k+1}(x)
//               + sum_y w_x(y + u_k(y)) gbar_{k+1}(y),
// grad_v L = gbar_0 / 2^M.  The update is Algorithm 1's with the retraction
// replaced by the algebra's addition: Gaussian(sigma_grad), Adam, step
// scaling, v <- v - eps_t d, Gaussian(sigma_warp).  Per-op kernels; the
// scatter accumulates in 64-bit fixed point (order-independent).
#include <string.h>

#include "ops.h"
#include "register.h"
#include "validate.h"

namespace fa {

namespace {

constexpr int kSlotG = 7;  // header slot of max |gbar|
constexpr int kMaxSteps = 12;

struct SvfWs {
    WsHeader *h;
    Dims lvl[8];
    float *If[8], *Im[8];
    float *If0, *Im0;
    float *v[2], *m[2], *nu[2];
    float *us;  // (M + 1) x 3n: u_0 .. u_M of the squarings
    float *J, *grad, *g, *g2, *dir, *t1, *t2, *partials;
    long long *acc;
    LnccBuffers lb;
    MiBuffers mi;
    long long n;
};

void svf_carve(WsCarver &c, Dims full, const fa_params *p, int steps, SvfWs *q) {
    memset(q, 0, sizeof(*q));
    q->h = c.take<WsHeader>(1);
    long long n = 0;
    for (int l = 0; l < p->n_levels; ++l) {
        const int s = p->scales[l];
        q->lvl[l] = Dims{level_size(full.D, s), level_size(full.H, s), level_size(full.W, s)};
        n = q->lvl[l].N() > n ? q->lvl[l].N() : n;
    }
    q->n = n;
    if (p->storage != FA_F32) {
        q->If0 = c.take<float>(full.N());
        q->Im0 = c.take<float>(full.N());
    }
    for (int l = 0; l < p->n_levels; ++l) {
        if (p->scales[l] == 1) continue;
        q->If[l] = c.take<float>(q->lvl[l].N());
        q->Im[l] = c.take<float>(q->lvl[l].N());
    }
    for (int k = 0; k < 2; ++k) {
        q->v[k] = c.take<float>(3 * n);
        q->m[k] = c.take<float>(3 * n);
        q->nu[k] = c.take<float>(3 * n);
    }
    q->us = c.take<float>((size_t)(steps + 1) * 3 * n);
    const long long tmp = 3 * n > full.N() ? 3 * n : full.N();
    q->t1 = c.take<float>(tmp);
    q->t2 = c.take<float>(tmp);
    q->J = c.take<float>(n);
    q->grad = c.take<float>(3 * n);
    q->g = c.take<float>(3 * n);
    q->g2 = c.take<float>(3 * n);
    q->dir = c.take<float>(3 * n);
    long long np = 0;
    for (int l = 0; l < p->n_levels; ++l)
        np = mse_partials_count(q->lvl[l]) > np ? mse_partials_count(q->lvl[l]) : np;
    q->partials = c.take<float>(np);
    q->acc = c.take<long long>(3 * n);
    q->lb = lncc_carve(c, n);
    if (p->loss == FA_LOSS_MI) q->mi = mi_carve(c, p->mi_bins);
}

__global__ void __launch_bounds__(256) k_scale(const float *__restrict__ a, float *b, long long n,
                                               float s) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        b[i] = a[i] * s;
}

// out = (I + grad u(x + u(x)))^T gb(x) (the direct term of a squaring's
// adjoint) and max |gb| into h->coef_max_bits[kSlotG] (the scatter's scale).
__global__ void __launch_bounds__(256) k_square_adjoint_direct(const float *__restrict__ u,
                                                               const float *__restrict__ gb,
                                                               float *__restrict__ out,
                                                               WsHeader *h, int D, int H, int W) {
    __shared__ float red[32];
    const long long N = (long long)D * H * W, HW = (long long)H * W;
    float amax = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(i / HW), r = (int)(i - (long long)z * HW), y = r / W, x = r - y * W;
        const float uz = u[i], uy = u[N + i], ux = u[2 * N + i];
        float G[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            tri_sample<true>(u + c * N, D, H, W, z, y, x, uz, uy, ux, G[c][0], G[c][1], G[c][2]);
        const float b[3] = {gb[i], gb[N + i], gb[2 * N + i]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float s = b[a];
#pragma unroll
            for (int j = 0; j < 3; ++j) s = fmaf(G[j][a], b[j], s);
            out[a * N + i] = s;
            const float ab = fabsf(b[a]);
            if (ab < 3.4e38f) amax = fmaxf(amax, ab);
        }
    }
    block_max_to(&h->coef_max_bits[kSlotG], amax, red);
}

// v_out = v - eps_t d with eps_t = lr / (c_lp max |d|) from the Adam kernel's
// maximum (the additive update in the algebra); resets the other parity slot.
__global__ void __launch_bounds__(256) k_svf_step(const float *__restrict__ v,
                                                  const float *__restrict__ d, float *v_out,
                                                  long long n3, float lr, float c_lp, WsHeader *h,
                                                  int parity) {
    const float mx = __uint_as_float(h->step_max_bits[parity]);
    const float e = (mx > 0.0f) ? lr / (c_lp * mx) : 0.0f;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        h->step_max_bits[parity ^ 1] = 0u;
        h->eps_t = e;
    }
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (long long)gridDim.x * blockDim.x)
        v_out[i] = fmaf(-e, d[i], v[i]);
}

unsigned blocks_for(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b > 152 * 8 ? 152 * 8 : (b < 1 ? 1 : b));
}

cudaError_t eval_reset(WsHeader *h, cudaStream_t s) {
    const size_t a = offsetof(WsHeader, coef_max_bits), b = offsetof(WsHeader, loss);
    return cudaMemsetAsync((char *)h + a, 0, b - a, s);
}

// u_M = exp(v) - id into q.us + M 3N; with grads, grad_v L into q.g; the loss
// into loss_dev (may be NULL).
fa_status svf_eval(SvfWs &q, const fa_params *p, int steps, Dims d, const float *If,
                   const float *Im, const float *v, bool grads, float *loss_dev, cudaStream_t s) {
    const long long N = d.N(), n3 = 3 * N;
    // the squarings' intermediates are packed at the level's size
    auto uk = [&](int k) { return q.us + (size_t)k * n3; };
    FA_CUDA_TRY(eval_reset(q.h, s));
    k_scale<<<blocks_for(n3), 256, 0, s>>>(v, uk(0), n3, ldexpf(1.0f, -steps));
    note_launch();
    FA_CUDA_TRY(cudaGetLastError());
    for (int k = 0; k < steps; ++k) FA_CUDA_TRY(launch_compose_fields(uk(k), uk(k), uk(k + 1), d, s));
    FA_CUDA_TRY(launch_warp(Im, uk(steps), q.J, grads ? q.grad : nullptr, d, s));
    if (p->loss == FA_LOSS_LNCC) {
        FA_CUDA_TRY(launch_lncc_forward(If, q.J, d, p->window, p->cc_eps, false, q.h, q.lb, s));
        FA_CUDA_TRY(launch_loss_finalize(q.h, N, -1.0f, loss_dev, s));
        if (grads)
            FA_CUDA_TRY(launch_lncc_backward(If, q.J, q.grad, d, p->window, q.h, q.lb, nullptr,
                                             nullptr, q.g, s));
    } else if (p->loss == FA_LOSS_MI) {
        FA_CUDA_TRY(launch_mi(If, q.J, grads ? q.grad : nullptr, d, p->mi_bins, q.h, q.mi,
                              loss_dev, nullptr, grads ? q.g : nullptr, s));
    } else {
        FA_CUDA_TRY(launch_mse(If, q.J, grads ? q.grad : nullptr, d, q.h, q.partials, nullptr,
                               nullptr, grads ? q.g : nullptr, s));
        if (loss_dev)
            FA_CUDA_TRY(cudaMemcpyAsync(loss_dev, &q.h->loss, sizeof(float),
                                        cudaMemcpyDeviceToDevice, s));
    }
    if (!grads) return FA_OK;
    for (int k = steps - 1; k >= 0; --k) {
        FA_CUDA_TRY(cudaMemsetAsync(&q.h->coef_max_bits[kSlotG], 0, sizeof(unsigned), s));
        k_square_adjoint_direct<<<blocks_for(N), 256, 0, s>>>(uk(k), q.g, q.g2, q.h, d.D, d.H,
                                                             d.W);
        note_launch();
        FA_CUDA_TRY(cudaGetLastError());
        FA_CUDA_TRY(cudaMemsetAsync(q.acc, 0, sizeof(long long) * n3, s));
        FA_CUDA_TRY(launch_field_scatter(uk(k), q.g, q.acc, q.h, kSlotG, d, s));
        FA_CUDA_TRY(launch_field_scatter_add(q.acc, q.h, kSlotG, 1.0f, q.g2, n3, s));
        float *t = q.g;
        q.g = q.g2;
        q.g2 = t;
    }
    k_scale<<<blocks_for(n3), 256, 0, s>>>(q.g, q.g, n3, ldexpf(1.0f, -steps));
    note_launch();
    FA_CUDA_TRY(cudaGetLastError());
    return FA_OK;
}

fa_status check_svf(const fa_vol *fixed, const fa_vol *moving, const fa_params *p, int steps,
                    const fa_vol *u_out) {
    if (steps < 0 || steps > kMaxSteps) {
        set_error("fa_register_svf: steps must be in 0..%d (got %d)", kMaxSteps, steps);
        return FA_ERR_INVALID;
    }
    if (p && p->use_jac) {
        set_error("fa_register_svf: use_jac does not apply to the velocity update");
        return FA_ERR_INVALID;
    }
    if (p) FA_TRY(check_adam_params(p, "fa_register_svf"));
    return register_check(fixed, moving, p, u_out);
}

}  // namespace

}  // namespace fa

extern "C" size_t fa_register_svf_workspace_size(int32_t D, int32_t H, int32_t W,
                                                 const fa_params *p, int32_t steps) {
    using namespace fa;
    clear_error();
    if (D < 1 || H < 1 || W < 1 || !p || p->n_levels < 1 || p->n_levels > 8) return 0;
    const int L = p->n_levels - 1;
    const int sl = p->scales[L] > 0 ? p->scales[L] : 1;
    fa_vol f{(void *)256, p->storage, 1, D, H, W};
    fa_vol u{(void *)256, FA_F32, 3, level_size(D, sl), level_size(H, sl), level_size(W, sl)};
    if (check_svf(&f, &f, p, steps, &u) != FA_OK) return 0;
    WsCarver c(nullptr, ~size_t(0));
    SvfWs q;
    svf_carve(c, Dims{D, H, W}, p, steps, &q);
    return c.off;
}

extern "C" fa_status fa_register_svf(const fa_vol *fixed, const fa_vol *moving,
                                     const fa_params *p, int32_t steps, fa_vol *u_out,
                                     fa_vol *v_out_opt, float *final_loss_dev, void *ws,
                                     size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_svf(fixed, moving, p, steps, u_out));
    if (v_out_opt) {
        FA_TRY(check_vol(v_out_opt, "v_out", 3));
        FA_TRY(same_grid(u_out, v_out_opt, "u_out", "v_out"));
    }
    const Dims full{fixed->D, fixed->H, fixed->W};
    FA_TRY(check_ws(ws, ws_bytes, fa_register_svf_workspace_size(full.D, full.H, full.W, p, steps),
                    "fa_register_svf"));
    WsCarver c(ws, ws_bytes);
    SvfWs q;
    svf_carve(c, full, p, steps, &q);
    cudaStream_t s = (cudaStream_t)stream;
    const float *If0 = (const float *)fixed->data, *Im0 = (const float *)moving->data;
    if (p->storage != FA_F32) {
        FA_CUDA_TRY(launch_widen(fixed->data, p->storage, q.If0, full.N(), s));
        FA_CUDA_TRY(launch_widen(moving->data, p->storage, q.Im0, full.N(), s));
        If0 = q.If0;
        Im0 = q.Im0;
    }
    GaussTaps tg, tw;
    make_gauss_taps(p->sigma_grad, &tg);
    make_gauss_taps(p->sigma_warp, &tw);
    FA_CUDA_TRY(launch_header_reset(q.h, s));
    for (int l = 0; l < p->n_levels; ++l) {
        if (p->scales[l] == 1) continue;
        FA_CUDA_TRY(launch_pyramid_level(If0, full, p->scales[l], q.If[l], q.lvl[l], q.t1, q.t2, s));
        FA_CUDA_TRY(launch_pyramid_level(Im0, full, p->scales[l], q.Im[l], q.lvl[l], q.t1, q.t2, s));
    }
    const int L = p->n_levels - 1;
    int cur = 0, t = 0;
    for (int l = 0; l < p->n_levels; ++l) {
        const Dims d = q.lvl[l];
        const long long n3 = 3 * d.N();
        const float *If = p->scales[l] == 1 ? If0 : q.If[l];
        const float *Im = p->scales[l] == 1 ? Im0 : q.Im[l];
        if (l == 0) {
            FA_CUDA_TRY(cudaMemsetAsync(q.v[cur], 0, sizeof(float) * n3, s));
            FA_CUDA_TRY(cudaMemsetAsync(q.m[cur], 0, sizeof(float) * n3, s));
            FA_CUDA_TRY(cudaMemsetAsync(q.nu[cur], 0, sizeof(float) * n3, s));
        } else {
            const Dims pc = q.lvl[l - 1];
            float s1[3], s2[3], s3[3];
            handoff_scales(pc, d, 1, s1);
            handoff_scales(pc, d, -1, s2);
            handoff_scales(pc, d, -2, s3);
            const int nx = cur ^ 1;
            FA_CUDA_TRY(launch_resample(q.v[cur], pc, q.v[nx], d, 3, s1, s));
            FA_CUDA_TRY(launch_resample(q.m[cur], pc, q.m[nx], d, 3, s2, s));
            FA_CUDA_TRY(launch_resample(q.nu[cur], pc, q.nu[nx], d, 3, s3, s));
            cur = nx;
        }
        FA_CUDA_TRY(cudaMemsetAsync(q.h->absmax_bits, 0, sizeof(q.h->absmax_bits), s));
        FA_CUDA_TRY(launch_absmax2(If, Im, d.N(), q.h, s));
        if (p->loss == FA_LOSS_MI) FA_CUDA_TRY(launch_mi_range(If, Im, d.N(), q.mi, s));
        for (int it = 0; it < p->iters[l]; ++it) {
            ++t;
            const int parity = t & 1;
            FA_TRY(svf_eval(q, p, steps, d, If, Im, q.v[cur], true, nullptr, s));
            FA_CUDA_TRY(launch_gauss3(q.g, q.g, q.t1, q.t2, 3, d, tg, s));
            FA_CUDA_TRY(launch_adam(q.g, q.m[cur], q.nu[cur], q.dir, d.N(), adam_consts(p, t), q.h,
                                    parity, s));
            k_svf_step<<<blocks_for(n3), 256, 0, s>>>(q.v[cur], q.dir, q.v[cur ^ 1], n3, p->lr,
                                                      p->c_lp, q.h, parity);
            note_launch();
            FA_CUDA_TRY(cudaGetLastError());
            FA_CUDA_TRY(launch_gauss3(q.v[cur ^ 1], q.v[cur], q.t1, q.t2, 3, d, tw, s));
        }
        if (l == L) {
            FA_TRY(svf_eval(q, p, steps, d, If, Im, q.v[cur], false, final_loss_dev, s));
            FA_CUDA_TRY(cudaMemcpyAsync(u_out->data, q.us + (size_t)steps * n3,
                                        sizeof(float) * n3, cudaMemcpyDeviceToDevice, s));
            if (v_out_opt)
                FA_CUDA_TRY(cudaMemcpyAsync(v_out_opt->data, q.v[cur], sizeof(float) * n3,
                                            cudaMemcpyDeviceToDevice, s));
        }
    }
    return FA_OK;
}

extern "C" fa_status fa_svf_loss_grad(const fa_vol *fixed, const fa_vol *moving, const fa_vol *v,
                                      const fa_params *p, int32_t steps, float *loss_dev,
                                      fa_vol *grad_v_out, fa_vol *u_out_opt, void *ws,
                                      size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    if (!p) {
        set_error("fa_svf_loss_grad: params are NULL");
        return FA_ERR_INVALID;
    }
    fa_params p1 = *p;
    p1.n_levels = 1;
    p1.scales[0] = 1;
    p1.iters[0] = 0;
    FA_TRY(check_svf(fixed, moving, &p1, steps, v));
    FA_TRY(check_vol(grad_v_out, "grad_v", 3));
    FA_TRY(same_grid(v, grad_v_out, "v", "grad_v"));
    if (u_out_opt) {
        FA_TRY(check_vol(u_out_opt, "u_out", 3));
        FA_TRY(same_grid(v, u_out_opt, "v", "u_out"));
    }
    const Dims d{fixed->D, fixed->H, fixed->W};
    FA_TRY(check_ws(ws, ws_bytes, fa_register_svf_workspace_size(d.D, d.H, d.W, &p1, steps),
                    "fa_svf_loss_grad"));
    WsCarver c(ws, ws_bytes);
    SvfWs q;
    svf_carve(c, d, &p1, steps, &q);
    cudaStream_t s = (cudaStream_t)stream;
    const float *If = (const float *)fixed->data, *Im = (const float *)moving->data;
    FA_CUDA_TRY(launch_header_reset(q.h, s));
    FA_CUDA_TRY(launch_absmax2(If, Im, d.N(), q.h, s));
    if (p1.loss == FA_LOSS_MI) FA_CUDA_TRY(launch_mi_range(If, Im, d.N(), q.mi, s));
    FA_TRY(svf_eval(q, &p1, steps, d, If, Im, (const float *)v->data, true, loss_dev, s));
    const size_t b = sizeof(float) * 3 * d.N();
    FA_CUDA_TRY(cudaMemcpyAsync(grad_v_out->data, q.g, b, cudaMemcpyDeviceToDevice, s));
    if (u_out_opt)
        FA_CUDA_TRY(cudaMemcpyAsync(u_out_opt->data, q.us + (size_t)steps * 3 * d.N(), b,
                                    cudaMemcpyDeviceToDevice, s));
    return FA_OK;
}
