// Symmetric registration (section "Alternative formulations for Eulerian
// differential": the symmetric objective takes its final map as
// phi = phi_M o phi_F^-1, with phi_F^-1 from the post-hoc inverse).  Two maps
// phi_F = id + u_F and phi_M = id + u_M start at the identity and minimise
// L(I_f o phi_F, I_m o phi_M) (LNCC or MSE, symmetric in its arguments).
// Each iteration takes Algorithm 1's update of each map from its own
// Gateaux derivative
//   dL/dphi_F = dL/dJ_F grad I_f(phi_F),   dL/dphi_M = dL/dJ_M grad I_m(phi_M)
// with its own Adam moments and step scale (one step counter).  On the last
// level u = w + u_M o (id + w), w the post-hoc inverse of u_F.
// Built from the per-op kernels: J_F takes the fixed-image role of the LNCC
// kernels and J_M the warped-image role, so dL/dJ_F is their fixed-image
// adjoint.
#include <stddef.h>
#include <string.h>

#include "ops.h"
#include "register.h"
#include "validate.h"

namespace fa {

namespace {

struct SymWs {
    WsHeader *h;
    Dims lvl[8];
    float *If[8], *Im[8];
    float *If0, *Im0;                 // FP32 copies of 16-bit inputs (else nullptr)
    float *u[2][2], *m[2][2], *v[2][2];  // [map F/M][buffer]
    float *JF, *JM, *gIF, *gIM, *dF, *gF, *gM, *dir, *t1, *t2, *partials, *w;
    LnccBuffers lb;
    void *inv_ws;
    size_t inv_bytes;
};

// p_inv == nullptr: one grid, loss and gradients only (no fields, no inverse).
void sym_carve(WsCarver &c, Dims full, const fa_params *p, const fa_params *p_inv, int storage,
               SymWs *q) {
    memset(q, 0, sizeof(*q));
    q->h = c.take<WsHeader>(1);
    long long n = 0;
    const int L = p_inv ? p->n_levels : 1;
    for (int l = 0; l < L; ++l) {
        const int s = p_inv ? p->scales[l] : 1;
        q->lvl[l] = Dims{level_size(full.D, s), level_size(full.H, s), level_size(full.W, s)};
        n = q->lvl[l].N() > n ? q->lvl[l].N() : n;
    }
    if (storage != FA_F32) {
        q->If0 = c.take<float>(full.N());
        q->Im0 = c.take<float>(full.N());
    }
    for (int l = 0; l < L; ++l) {
        if (!p_inv || p->scales[l] == 1) continue;
        q->If[l] = c.take<float>(q->lvl[l].N());
        q->Im[l] = c.take<float>(q->lvl[l].N());
    }
    if (p_inv)
        for (int k = 0; k < 2; ++k)
            for (int b = 0; b < 2; ++b) {
                q->u[k][b] = c.take<float>(3 * n);
                q->m[k][b] = c.take<float>(3 * n);
                q->v[k][b] = c.take<float>(3 * n);
            }
    const long long tmp = 3 * n > full.N() ? 3 * n : full.N();
    q->t1 = c.take<float>(tmp);
    q->t2 = c.take<float>(tmp);
    q->JF = c.take<float>(n);
    q->JM = c.take<float>(n);
    q->gIF = c.take<float>(3 * n);
    q->gIM = c.take<float>(3 * n);
    q->dF = c.take<float>(n);
    q->gF = c.take<float>(3 * n);
    q->gM = c.take<float>(3 * n);
    q->dir = c.take<float>(3 * n);
    long long np = 0;
    for (int l = 0; l < L; ++l) np = mse_partials_count(q->lvl[l]) > np ? mse_partials_count(q->lvl[l]) : np;
    q->partials = c.take<float>(np);
    q->lb = lncc_carve(c, n);
    if (p_inv) {
        const Dims d = q->lvl[p->n_levels - 1];
        q->w = c.take<float>(3 * d.N());
        q->inv_bytes = fa_inverse_workspace_size(d.D, d.H, d.W, p_inv);
        q->inv_ws = c.take<char>(q->inv_bytes);
    }
}

__global__ void __launch_bounds__(256) k_scale_channels(const float *__restrict__ a,
                                                        const float *__restrict__ grad,
                                                        float *__restrict__ g, long long N) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const float s = a[i];
        g[i] = s * grad[i];
        g[N + i] = s * grad[N + i];
        g[2 * N + i] = s * grad[2 * N + i];
    }
}

// Bytes [offsetof(coef_max_bits), offsetof(loss)) are per-evaluation state.
cudaError_t eval_reset(WsHeader *h, cudaStream_t s) {
    const size_t a = offsetof(WsHeader, coef_max_bits), b = offsetof(WsHeader, loss);
    return cudaMemsetAsync((char *)h + a, 0, b - a, s);
}

// L(I_f o phi_F, I_m o phi_M) into loss_dev (may be NULL); with grads,
// dL/du_F into q.gF and dL/du_M into q.gM.  Needs the images' maxima in h.
fa_status sym_loss(SymWs &q, int loss, int window, float cc_eps, Dims d, const float *If,
                   const float *Im, const float *uF, const float *uM, bool grads,
                   float *loss_dev, cudaStream_t s) {
    const long long N = d.N();
    FA_CUDA_TRY(eval_reset(q.h, s));
    FA_CUDA_TRY(launch_warp(If, uF, q.JF, grads ? q.gIF : nullptr, d, s));
    FA_CUDA_TRY(launch_warp(Im, uM, q.JM, grads ? q.gIM : nullptr, d, s));
    if (loss == FA_LOSS_LNCC) {
        FA_CUDA_TRY(launch_lncc_forward(q.JF, q.JM, d, window, cc_eps, grads, q.h, q.lb, s));
        FA_CUDA_TRY(launch_loss_finalize(q.h, N, -1.0f, loss_dev, s));
        if (grads)
            FA_CUDA_TRY(launch_lncc_backward(q.JF, q.JM, q.gIM, d, window, q.h, q.lb, nullptr,
                                             q.dF, q.gM, s));
    } else {
        FA_CUDA_TRY(launch_mse(q.JF, q.JM, grads ? q.gIM : nullptr, d, q.h, q.partials, nullptr,
                               grads ? q.dF : nullptr, grads ? q.gM : nullptr, s));
        if (loss_dev)
            FA_CUDA_TRY(cudaMemcpyAsync(loss_dev, &q.h->loss, sizeof(float),
                                        cudaMemcpyDeviceToDevice, s));
    }
    if (grads) {
        long long blocks = (N + 255) / 256;
        blocks = blocks > 152 * 8 ? 152 * 8 : blocks;
        k_scale_channels<<<(unsigned)blocks, 256, 0, s>>>(q.dF, q.gIF, q.gF, N);
        note_launch();
        FA_CUDA_TRY(cudaGetLastError());
    }
    return FA_OK;
}

// Algorithm 1's update of one map (k) from its derivative g (overwritten).
fa_status sym_update(SymWs &q, const fa_params *p, Dims d, float *g, int k, int cur, int t,
                     const GaussTaps &tg, const GaussTaps &tw, cudaStream_t s) {
    float *u = q.u[k][cur], *alt = q.u[k][cur ^ 1];
    const int parity = t & 1;
    // the two maps share the step-maximum slot of this parity
    FA_CUDA_TRY(cudaMemsetAsync(&q.h->step_max_bits[parity], 0, sizeof(unsigned), s));
    if (p->use_jac) FA_CUDA_TRY(launch_jac_direction(g, u, g, d, s));
    FA_CUDA_TRY(launch_gauss3(g, g, q.t1, q.t2, 3, d, tg, s));
    FA_CUDA_TRY(launch_adam(g, q.m[k][cur], q.v[k][cur], q.dir, d.N(), adam_consts(p, t), q.h,
                            parity, s));
    FA_CUDA_TRY(launch_compose(u, q.dir, alt, d, p->lr, p->c_lp, q.h, parity, nullptr, s));
    FA_CUDA_TRY(launch_gauss3(alt, u, q.t1, q.t2, 3, d, tw, s));
    return FA_OK;
}

fa_status check_loss_args(int loss, int window, float cc_eps, const char *who) {
    if (loss != FA_LOSS_LNCC && loss != FA_LOSS_MSE) {
        set_error("%s: loss must be FA_LOSS_LNCC or FA_LOSS_MSE", who);
        return FA_ERR_INVALID;
    }
    if (loss == FA_LOSS_LNCC && (window < 1 || window > 15 || (window % 2) == 0)) {
        set_error("%s: window must be odd and in 1..15 (got %d)", who, window);
        return FA_ERR_INVALID;
    }
    if (!(cc_eps >= 0.0f && cc_eps < 3e38f)) {
        set_error("%s: cc_eps must be finite and >= 0", who);
        return FA_ERR_INVALID;
    }
    return FA_OK;
}

fa_status check_inverse_schedule(Dims full, const fa_params *p, const fa_params *p_inv,
                                 size_t *inv_bytes) {
    if (!p_inv || p_inv->n_levels < 1 || p_inv->n_levels > 8 ||
        p_inv->scales[p_inv->n_levels - 1] != 1) {
        set_error("fa_register_symmetric: p_inv needs 1..8 levels, the last at scale 1");
        return FA_ERR_INVALID;
    }
    const int L = p->n_levels - 1;
    const Dims d{level_size(full.D, p->scales[L]), level_size(full.H, p->scales[L]),
                 level_size(full.W, p->scales[L])};
    *inv_bytes = fa_inverse_workspace_size(d.D, d.H, d.W, p_inv);
    return *inv_bytes ? FA_OK : FA_ERR_INVALID;  // the inverse set the message
}

}  // namespace

}  // namespace fa

extern "C" size_t fa_symmetric_loss_grad_workspace_size(int32_t D, int32_t H, int32_t W) {
    using namespace fa;
    clear_error();
    if (D < 1 || H < 1 || W < 1) return 0;
    fa_params p;
    fa_params_default(&p);
    WsCarver c(nullptr, ~size_t(0));
    SymWs q;
    sym_carve(c, Dims{D, H, W}, &p, nullptr, FA_F32, &q);
    return c.off;
}

extern "C" fa_status fa_symmetric_loss_grad(const fa_vol *fixed, const fa_vol *moving,
                                            const fa_vol *uF, const fa_vol *uM, int32_t loss,
                                            int32_t window, float cc_eps, float *loss_dev,
                                            fa_vol *gF_out, fa_vol *gM_out, void *ws,
                                            size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_loss_args(loss, window, cc_eps, "fa_symmetric_loss_grad"));
    FA_TRY(check_vol(fixed, "fixed", 1));
    FA_TRY(check_vol(moving, "moving", 1));
    FA_TRY(check_vol(uF, "uF", 3));
    FA_TRY(check_vol(uM, "uM", 3));
    FA_TRY(check_vol(gF_out, "gF", 3));
    FA_TRY(check_vol(gM_out, "gM", 3));
    FA_TRY(same_grid(fixed, moving, "fixed", "moving"));
    FA_TRY(same_grid(fixed, uF, "fixed", "uF"));
    FA_TRY(same_grid(fixed, uM, "fixed", "uM"));
    FA_TRY(same_grid(fixed, gF_out, "fixed", "gF"));
    FA_TRY(same_grid(fixed, gM_out, "fixed", "gM"));
    const Dims d{fixed->D, fixed->H, fixed->W};
    FA_TRY(check_ws(ws, ws_bytes, fa_symmetric_loss_grad_workspace_size(d.D, d.H, d.W),
                    "fa_symmetric_loss_grad"));
    fa_params p;
    fa_params_default(&p);
    WsCarver c(ws, ws_bytes);
    SymWs q;
    sym_carve(c, d, &p, nullptr, FA_F32, &q);
    cudaStream_t s = (cudaStream_t)stream;
    const float *If = (const float *)fixed->data, *Im = (const float *)moving->data;
    FA_CUDA_TRY(launch_header_reset(q.h, s));
    FA_CUDA_TRY(launch_absmax2(If, Im, d.N(), q.h, s));
    FA_TRY(sym_loss(q, loss, window, cc_eps, d, If, Im, (const float *)uF->data,
                    (const float *)uM->data, true, loss_dev, s));
    const size_t b = sizeof(float) * 3 * d.N();
    FA_CUDA_TRY(cudaMemcpyAsync(gF_out->data, q.gF, b, cudaMemcpyDeviceToDevice, s));
    FA_CUDA_TRY(cudaMemcpyAsync(gM_out->data, q.gM, b, cudaMemcpyDeviceToDevice, s));
    return FA_OK;
}

extern "C" size_t fa_register_symmetric_workspace_size(int32_t D, int32_t H, int32_t W,
                                                       const fa_params *p,
                                                       const fa_params *p_inv) {
    using namespace fa;
    clear_error();
    if (D < 1 || H < 1 || W < 1 || !p) return 0;
    fa_vol f{nullptr, p->storage, 1, D, H, W};
    const int L = p->n_levels >= 1 && p->n_levels <= 8 ? p->n_levels - 1 : 0;
    fa_vol u{nullptr, FA_F32, 3, level_size(D, p->scales[L] > 0 ? p->scales[L] : 1),
             level_size(H, p->scales[L] > 0 ? p->scales[L] : 1),
             level_size(W, p->scales[L] > 0 ? p->scales[L] : 1)};
    f.data = u.data = (void *)256;  // shape checks only
    if (check_adam_params(p, "fa_register_symmetric") != FA_OK ||
        register_check(&f, &f, p, &u) != FA_OK ||
        check_loss_args(p->loss, p->window, p->cc_eps, "fa_register_symmetric") != FA_OK)
        return 0;
    size_t inv = 0;
    if (check_inverse_schedule(Dims{D, H, W}, p, p_inv, &inv) != FA_OK) return 0;
    WsCarver c(nullptr, ~size_t(0));
    SymWs q;
    sym_carve(c, Dims{D, H, W}, p, p_inv, p->storage, &q);
    return c.off;
}

extern "C" fa_status fa_register_symmetric(const fa_vol *fixed, const fa_vol *moving,
                                           const fa_params *p, const fa_params *p_inv,
                                           fa_vol *u_out, fa_vol *uF_out_opt, fa_vol *uM_out_opt,
                                           float *final_loss_dev, float *mid_loss_dev, void *ws,
                                           size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_adam_params(p, "fa_register_symmetric"));
    FA_TRY(register_check(fixed, moving, p, u_out));
    FA_TRY(check_loss_args(p->loss, p->window, p->cc_eps, "fa_register_symmetric"));
    if (uF_out_opt) {
        FA_TRY(check_vol(uF_out_opt, "uF_out", 3));
        FA_TRY(same_grid(u_out, uF_out_opt, "u_out", "uF_out"));
    }
    if (uM_out_opt) {
        FA_TRY(check_vol(uM_out_opt, "uM_out", 3));
        FA_TRY(same_grid(u_out, uM_out_opt, "u_out", "uM_out"));
    }
    const Dims full{fixed->D, fixed->H, fixed->W};
    size_t inv = 0;
    FA_TRY(check_inverse_schedule(full, p, p_inv, &inv));
    {
        WsCarver c(nullptr, ~size_t(0));
        SymWs q0;
        sym_carve(c, full, p, p_inv, p->storage, &q0);
        FA_TRY(check_ws(ws, ws_bytes, c.off, "fa_register_symmetric"));
    }
    WsCarver c(ws, ws_bytes);
    SymWs q;
    sym_carve(c, full, p, p_inv, p->storage, &q);
    cudaStream_t s = (cudaStream_t)stream;
    const float *If0 = (const float *)fixed->data, *Im0 = (const float *)moving->data;
    if (p->storage != FA_F32) {  // 16-bit images: widened once, exactly
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
        const float *If = p->scales[l] == 1 ? If0 : q.If[l];
        const float *Im = p->scales[l] == 1 ? Im0 : q.Im[l];
        const size_t b = sizeof(float) * 3 * d.N();
        if (l == 0) {
            for (int k = 0; k < 2; ++k) {
                FA_CUDA_TRY(cudaMemsetAsync(q.u[k][cur], 0, b, s));
                FA_CUDA_TRY(cudaMemsetAsync(q.m[k][cur], 0, b, s));
                FA_CUDA_TRY(cudaMemsetAsync(q.v[k][cur], 0, b, s));
            }
        } else {
            const Dims pc = q.lvl[l - 1];
            float su[3], sm[3], sv[3];
            handoff_scales(pc, d, 1, su);
            handoff_scales(pc, d, -1, sm);
            handoff_scales(pc, d, -2, sv);
            const int nx = cur ^ 1;
            for (int k = 0; k < 2; ++k) {
                FA_CUDA_TRY(launch_resample(q.u[k][cur], pc, q.u[k][nx], d, 3, su, s));
                FA_CUDA_TRY(launch_resample(q.m[k][cur], pc, q.m[k][nx], d, 3, sm, s));
                FA_CUDA_TRY(launch_resample(q.v[k][cur], pc, q.v[k][nx], d, 3, sv, s));
            }
            cur = nx;
        }
        // fixed-point scale of this level's images (bounds of J_F and J_M)
        FA_CUDA_TRY(cudaMemsetAsync(q.h->absmax_bits, 0, sizeof(q.h->absmax_bits), s));
        FA_CUDA_TRY(launch_absmax2(If, Im, d.N(), q.h, s));
        for (int it = 0; it < p->iters[l]; ++it) {
            ++t;
            FA_TRY(sym_loss(q, p->loss, p->window, p->cc_eps, d, If, Im, q.u[0][cur], q.u[1][cur],
                            true, nullptr, s));
            FA_TRY(sym_update(q, p, d, q.gF, 0, cur, t, tg, tw, s));
            FA_TRY(sym_update(q, p, d, q.gM, 1, cur, t, tg, tw, s));
        }
        if (l == L) {
            if (mid_loss_dev)
                FA_TRY(sym_loss(q, p->loss, p->window, p->cc_eps, d, If, Im, q.u[0][cur],
                                q.u[1][cur], false, mid_loss_dev, s));
            fa_vol uf{q.u[0][cur], FA_F32, 3, d.D, d.H, d.W};
            fa_vol wv{q.w, FA_F32, 3, d.D, d.H, d.W};
            FA_TRY(fa_inverse(&uf, p_inv, &wv, nullptr, q.inv_ws, q.inv_bytes, stream));
            // phi_M o phi_F^-1 - id = w + u_M o (id + w)
            FA_CUDA_TRY(launch_compose_fields(q.u[1][cur], q.w, (float *)u_out->data, d, s));
            // final loss L(I_f, I_m o (id + u)) with zero-displacement F map
            FA_CUDA_TRY(cudaMemsetAsync(q.u[0][cur ^ 1], 0, b, s));
            FA_TRY(sym_loss(q, p->loss, p->window, p->cc_eps, d, If, Im, q.u[0][cur ^ 1],
                            (const float *)u_out->data, false, final_loss_dev, s));
            if (uF_out_opt)
                FA_CUDA_TRY(cudaMemcpyAsync(uF_out_opt->data, q.u[0][cur], b,
                                            cudaMemcpyDeviceToDevice, s));
            if (uM_out_opt)
                FA_CUDA_TRY(cudaMemcpyAsync(uM_out_opt->data, q.u[1][cur], b,
                                            cudaMemcpyDeviceToDevice, s));
        }
    }
    return FA_OK;
}
