// Whole registration (Algorithm 1, Jacobian-free direction): pyramid, level
// loop, iteration loop, level hand-off, final loss.  Host-side driver; every
// step runs in this library's kernels.
#include <math.h>
#include <string.h>

#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "ops.h"
#include "register.h"
#include "validate.h"

namespace fa {

// A 16-bit u is kept where the four fused kernels run every step of every
// level (their tile copies read it; the per-op kernels keep u in FP32).
static bool field16_ok(const fa_params *p) {
    if (p->mode != FA_MODE_FUSED || p->loss != FA_LOSS_LNCC || p->use_jac) return false;
    GaussTaps tg, tw;
    if (!make_gauss_taps(p->sigma_grad, &tg) || !make_gauss_taps(p->sigma_warp, &tw)) return false;
    return tg.R <= kMaxFusedRadius && tw.R <= kMaxFusedRadius;
}

static fa_status check_params(const fa_params *p) {
    if (!p) {
        set_error("params are NULL");
        return FA_ERR_INVALID;
    }
    if (p->n_levels < 1 || p->n_levels > 8) {
        set_error("n_levels must be in 1..8 (got %d)", (int)p->n_levels);
        return FA_ERR_INVALID;
    }
    for (int l = 0; l < p->n_levels; ++l) {
        if (p->scales[l] < 1 || 0.5f * (float)p->scales[l] > kMaxSigma || p->iters[l] < 0) {
            set_error("level %d: scale must be in 1..%d and iterations >= 0", l,
                      (int)(2 * kMaxSigma));
            return FA_ERR_INVALID;
        }
    }
    if (p->loss != FA_LOSS_LNCC && p->loss != FA_LOSS_MSE && p->loss != FA_LOSS_MI) {
        set_error("loss must be FA_LOSS_LNCC, FA_LOSS_MSE or FA_LOSS_MI");
        return FA_ERR_INVALID;
    }
    if (p->loss == FA_LOSS_MI && (p->mi_bins < kMiMinBins || p->mi_bins > kMiMaxBins)) {
        set_error("mi_bins must be in %d..%d (got %d)", kMiMinBins, kMiMaxBins, (int)p->mi_bins);
        return FA_ERR_INVALID;
    }
    if (p->loss == FA_LOSS_LNCC &&
        (p->window < 1 || p->window > 15 || (p->window % 2) == 0)) {
        set_error("window must be odd and in 1..15 (got %d)", (int)p->window);
        return FA_ERR_INVALID;
    }
    if (!(p->cc_eps >= 0.0f && p->cc_eps < 3e38f)) {
        set_error("cc_eps must be finite and >= 0");
        return FA_ERR_INVALID;
    }
    GaussTaps t;
    if (!make_gauss_taps(p->sigma_grad, &t) || !make_gauss_taps(p->sigma_warp, &t)) {
        set_error("sigma_grad and sigma_warp must be in [0, %g]", (double)kMaxSigma);
        return FA_ERR_INVALID;
    }
    if (p->use_jac != 0 && p->use_jac != 1) {
        set_error("use_jac must be 0 or 1");
        return FA_ERR_INVALID;
    }
    if (p->mode != FA_MODE_FUSED && p->mode != FA_MODE_PLAIN && p->mode != FA_MODE_PERSISTENT) {
        set_error("mode must be FA_MODE_FUSED, FA_MODE_PLAIN or FA_MODE_PERSISTENT");
        return FA_ERR_INVALID;
    }
    if (p->storage != FA_F32 && p->storage != FA_BF16 && p->storage != FA_F16) {
        set_error("storage must be FA_F32, FA_BF16 or FA_F16 (got %d)", (int)p->storage);
        return FA_ERR_UNSUPPORTED;
    }
    if (p->state_storage != FA_F32 && p->state_storage != FA_BF16) {
        // FP16's smallest normal value (6.1e-5) lies far above the moments of
        // a loss gradient that scales as 1/N: they would flush to zero
        set_error("state_storage must be FA_F32 or FA_BF16 (got %d)", (int)p->state_storage);
        return FA_ERR_UNSUPPORTED;
    }
    if (p->field_storage != FA_F32 && p->field_storage != FA_F16) {
        set_error("field_storage must be FA_F32 or FA_F16 (got %d)", (int)p->field_storage);
        return FA_ERR_UNSUPPORTED;
    }
    if (p->field_storage == FA_F16 && !field16_ok(p)) {
        set_error("field_storage FA_F16 needs FA_MODE_FUSED, the LNCC loss, use_jac = 0 and "
                  "Gaussian radii up to %d", kMaxFusedRadius);
        return FA_ERR_UNSUPPORTED;
    }
    return check_adam_params(p, "fa_register", true);
}

// Row pitch of a level's buffers: the width rounded up to a multiple of 4
// (8 with an FP16 u) where the four fused LNCC kernels run every step of the
// level, so that they take TMA tiles at any width; 0 (the width itself)
// elsewhere.  The padding is never read as data: TMA tiles describe the
// D x H x W grid and fill beyond it with zeros, and every other access
// checks x < W.
static int level_pitch(const fa_params *p, Dims d) {
    // FP16 u: rows of a multiple of 8 elements (16 bytes of FP16)
    if (p->field_storage == FA_F16) return d.W % 8 == 0 ? 0 : (d.W + 7) & ~7;
    if (p->loss != FA_LOSS_LNCC || p->use_jac || d.W % 4 == 0) return 0;
    if (p->mode == FA_MODE_PLAIN || (p->mode == FA_MODE_PERSISTENT && persistent_eligible(p, d)))
        return 0;
    GaussTaps tg, tw;
    make_gauss_taps(p->sigma_grad, &tg);
    make_gauss_taps(p->sigma_warp, &tw);
    if (tg.R > kMaxFusedRadius || tw.R > kMaxFusedRadius) return 0;  // separable passes, unpitched
    return (d.W + 3) & ~3;
}

// Workspace plan; with base == nullptr only sizes are computed.  Level l's
// images, u, m, nu and the fused buffers have rows of lvl[l].pitch()
// elements; the full-resolution inputs and u_out have none.
struct Plan {
    Dims full;
    Dims lvl[8];
    long long nmax;
    WsHeader *h;
    float *If[8], *Im[8];  // nullptr: the level is the unpadded input grid
    float *If0, *Im0;  // FP32 copies of 16-bit input images (else nullptr)
    float *u[2];
    void *m[2], *v[2];  // Adam moments, stored as p->state_storage
    float *J, *grad, *g, *dir, *t1, *t2;
    LnccBuffers lb;
    MiBuffers mi;
    float *partials;
    FusedBuffers fb;
    long long *pxy;  // in-plane window sums of the persistent coarse levels
    size_t bytes;
    bool ok;
};

static void make_plan(Plan &P, void *base, size_t cap, Dims full, const fa_params *p) {
    P.full = full;
    P.nmax = 0;
    for (int l = 0; l < p->n_levels; ++l) {
        int s = p->scales[l];
        Dims d{level_size(full.D, s), level_size(full.H, s), level_size(full.W, s)};
        d.P = level_pitch(p, d);
        P.lvl[l] = d;
        if (d.NP() > P.nmax) P.nmax = d.NP();
    }
    long long n = P.nmax;
    WsCarver c(base, cap);
    P.h = c.take<WsHeader>(1);
    P.If0 = P.Im0 = nullptr;
    if (p->storage != FA_F32) {
        P.If0 = c.take<float>(full.N());
        P.Im0 = c.take<float>(full.N());
    }
    for (int l = 0; l < p->n_levels; ++l) {
        if (p->scales[l] == 1 && P.lvl[l].pitch() == full.W) {
            P.If[l] = P.Im[l] = nullptr;  // the inputs themselves
        } else {
            P.If[l] = c.take<float>(P.lvl[l].NP());
            P.Im[l] = c.take<float>(P.lvl[l].NP());
        }
    }
    for (int k = 0; k < 2; ++k) {
        P.u[k] = c.take<float>(3 * n);
        if (p->state_storage == FA_F32) {
            P.m[k] = c.take<float>(3 * n);
            P.v[k] = c.take<float>(3 * n);
        } else {
            P.m[k] = c.take<unsigned short>(3 * n);
            P.v[k] = c.take<unsigned short>(3 * n);
        }
    }
    long long tmp = 3 * n > full.N() ? 3 * n : full.N();
    P.t1 = c.take<float>(tmp);
    P.t2 = c.take<float>(tmp);
    P.J = c.take<float>(n);
    P.grad = c.take<float>(3 * n);
    P.g = c.take<float>(3 * n);
    P.dir = c.take<float>(3 * n);
    Dims dmax{1, 1, (int)n};
    long long np = 0;
    for (int l = 0; l < p->n_levels; ++l) {
        long long k = mse_partials_count(P.lvl[l]);
        if (k > np) np = k;
    }
    (void)dmax;
    P.partials = c.take<float>(np);
    memset(&P.lb, 0, sizeof(P.lb));
    memset(&P.fb, 0, sizeof(P.fb));
    P.pxy = nullptr;
    if (p->mode == FA_MODE_PLAIN) {
        P.lb = lncc_carve(c, n);
    } else {
        fused_carve(c, n, &P.fb);
        long long np_ = 0;  // largest level that runs persistent
        for (int l = 0; l < p->n_levels; ++l)
            if (persistent_eligible(p, P.lvl[l]) && P.lvl[l].N() > np_) np_ = P.lvl[l].N();
        if (np_ > 0) P.pxy = c.take<long long>(3 * np_);
    }
    memset(&P.mi, 0, sizeof(P.mi));
    if (p->loss == FA_LOSS_MI) P.mi = P.fb.mi = mi_carve(c, p->mi_bins);
    P.bytes = c.off;
    P.ok = c.ok;
}

// Bytes [offsetof(coef_max_bits), offsetof(loss) ) are per-iteration state.
static cudaError_t iter_reset(WsHeader *h, cudaStream_t s) {
    size_t a = offsetof(WsHeader, coef_max_bits), b = offsetof(WsHeader, loss);
    return cudaMemsetAsync((char *)h + a, 0, b - a, s);
}

struct Timer {
    fa_kernel_timer *t;
    int level;
    bool on(int kernel_id) const {
        return t && t->kernel_id == kernel_id && (t->level < 0 || t->level == level) &&
               t->count < t->capacity;
    }
    cudaError_t start(int kernel_id, cudaStream_t s) const {
        if (!on(kernel_id)) return cudaSuccess;
        return timer_record(t->start_events[t->count], s);
    }
    cudaError_t stop(int kernel_id, cudaStream_t s) const {
        if (!on(kernel_id)) return cudaSuccess;
        cudaError_t e = timer_record(t->stop_events[t->count], s);
        t->count++;
        return e;
    }
};

// One plain-mode iteration: u <- G_warp(compose(u, step(Adam(G_grad(dL/du))))).
static fa_status plain_iteration(Plan &P, const fa_params *p, int l, const float *If,
                                 const float *Im, float *u, float *u_alt, void *m, void *v,
                                 int t, const GaussTaps &tg, const GaussTaps &tw, Timer &tm,
                                 cudaStream_t s) {
    Dims d = P.lvl[l];
    long long N = d.N();
    FA_CUDA_TRY(tm.start(FA_K_PLAIN_ANY, s));
    FA_CUDA_TRY(iter_reset(P.h, s));
    FA_CUDA_TRY(launch_warp(Im, u, P.J, P.grad, d, s));
    if (p->loss == FA_LOSS_LNCC) {
        FA_CUDA_TRY(launch_lncc_forward(If, P.J, d, p->window, p->cc_eps, false, P.h, P.lb, s));
        FA_CUDA_TRY(launch_lncc_backward(If, P.J, P.grad, d, p->window, P.h, P.lb, nullptr,
                                         nullptr, P.g, s));
    } else if (p->loss == FA_LOSS_MI) {
        FA_CUDA_TRY(launch_mi(If, P.J, P.grad, d, p->mi_bins, P.h, P.mi, nullptr, nullptr, P.g, s));
    } else {
        FA_CUDA_TRY(launch_mse(If, P.J, P.grad, d, P.h, P.partials, nullptr, nullptr, P.g, s));
    }
    if (p->use_jac) FA_CUDA_TRY(launch_jac_direction(P.g, u, P.g, d, s));
    FA_CUDA_TRY(launch_gauss3(P.g, P.g, P.t1, P.t2, 3, d, tg, s));
    int parity = t & 1;
    FA_CUDA_TRY(launch_adam_state(P.g, m, v, p->state_storage, P.dir, N, adam_consts(p, t), P.h,
                                  parity, s));
    FA_CUDA_TRY(launch_compose(u, P.dir, u_alt, d, p->lr, p->c_lp, P.h, parity, nullptr, s));
    FA_CUDA_TRY(launch_gauss3(u_alt, u, P.t1, P.t2, 3, d, tw, s));
    FA_CUDA_TRY(tm.stop(FA_K_PLAIN_ANY, s));
    return FA_OK;
}

static fa_status final_loss(Plan &P, const fa_params *p, int l, const float *If, const float *Im,
                            const float *u, float *loss_dev, cudaStream_t s) {
    Dims d = P.lvl[l];
    FA_CUDA_TRY(iter_reset(P.h, s));
    if (p->mode == FA_MODE_PLAIN || p->loss != FA_LOSS_LNCC)
        FA_CUDA_TRY(launch_warp(Im, u, P.J, nullptr, d, s));
    if (p->loss == FA_LOSS_LNCC) {
        if (p->mode == FA_MODE_PLAIN) {
            FA_CUDA_TRY(launch_lncc_forward(If, P.J, d, p->window, p->cc_eps, false, P.h, P.lb, s));
        } else {
            FA_CUDA_TRY(fused_lncc_forward_only(If, P.fb, d, p->window, p->cc_eps, P.h, s));
        }
        FA_CUDA_TRY(launch_loss_finalize(P.h, d.N(), -1.0f, loss_dev, s));
    } else if (p->loss == FA_LOSS_MI) {
        FA_CUDA_TRY(launch_mi(If, P.J, nullptr, d, p->mi_bins, P.h, P.mi, loss_dev, nullptr,
                              nullptr, s));
    } else {
        FA_CUDA_TRY(launch_mse(If, P.J, nullptr, d, P.h, P.partials, nullptr, nullptr, nullptr, s));
        if (loss_dev)
            FA_CUDA_TRY(
                cudaMemcpyAsync(loss_dev, &P.h->loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    }
    return FA_OK;
}

fa_status register_check(const fa_vol *fixed, const fa_vol *moving, const fa_params *p,
                         const fa_vol *u_out) {
    FA_TRY(check_params(p));
    FA_TRY(check_vol_dtype(fixed, "fixed", 1, p->storage));
    FA_TRY(check_vol_dtype(moving, "moving", 1, p->storage));
    FA_TRY(same_grid(fixed, moving, "fixed", "moving"));
    FA_TRY(check_vol(u_out, "u_out", 3));
    Dims full{fixed->D, fixed->H, fixed->W};
    int L = p->n_levels - 1;
    Dims last{level_size(full.D, p->scales[L]), level_size(full.H, p->scales[L]),
              level_size(full.W, p->scales[L])};
    if (u_out->D != last.D || u_out->H != last.H || u_out->W != last.W) {
        set_error("u_out must be 3 x %d x %d x %d (the last level's grid)", last.D, last.H, last.W);
        return FA_ERR_SHAPE;
    }
    return FA_OK;
}

// Start of a registration: 16-bit images widened once (exactly) and the
// pyramid (once per level); If0/Im0 receive the FP32 full-resolution images.
static fa_status registration_begin(Plan &P, const fa_vol *fixed, const fa_vol *moving,
                                    const fa_params *p, const float **If0, const float **Im0,
                                    cudaStream_t s) {
    const Dims full = P.full;
    *If0 = (const float *)fixed->data;
    *Im0 = (const float *)moving->data;
    if (p->storage != FA_F32) {
        FA_CUDA_TRY(launch_widen(fixed->data, p->storage, P.If0, full.N(), s));
        FA_CUDA_TRY(launch_widen(moving->data, p->storage, P.Im0, full.N(), s));
        *If0 = P.If0;
        *Im0 = P.Im0;
    }
    FA_CUDA_TRY(launch_header_reset(P.h, s));
    for (int l = 0; l < p->n_levels; ++l) {
        if (!P.If[l]) continue;
        const Dims d = P.lvl[l];
        if (d.pitch() != d.W) {  // zero padding: the level's max |I| reads whole rows
            FA_CUDA_TRY(cudaMemsetAsync(P.If[l], 0, sizeof(float) * d.NP(), s));
            FA_CUDA_TRY(cudaMemsetAsync(P.Im[l], 0, sizeof(float) * d.NP(), s));
        }
        FA_CUDA_TRY(launch_pyramid_level(*If0, full, p->scales[l], P.If[l], P.lvl[l], P.t1, P.t2, s));
        FA_CUDA_TRY(launch_pyramid_level(*Im0, full, p->scales[l], P.Im[l], P.lvl[l], P.t1, P.t2, s));
    }
    return FA_OK;
}

// Start of level l: the initial (or handed-off) u, m, nu in slot *cur, the
// level's image maxima, the MI range and the fused path's set-up.
static fa_status level_begin(Plan &P, const fa_params *p, int l, const float *u_init,
                             const float *If, const float *Im, int *cur, cudaStream_t s) {
    const Dims d = P.lvl[l];
    if (l == 0) {
        size_t b = sizeof(float) * 3 * d.NP();
        if (u_init) {  // start from a given displacement of the input grid
            float sc[3];
            handoff_scales(P.full, d, 1, sc);
            if (d.pitch() != d.W) FA_CUDA_TRY(cudaMemsetAsync(P.u[*cur], 0, b, s));
            FA_CUDA_TRY(launch_resample_field(u_init, FA_F32, P.full, P.u[*cur],
                                              p->field_storage, d, 3, sc, s));
        } else {
            FA_CUDA_TRY(cudaMemsetAsync(P.u[*cur], 0, b, s));
        }
        const size_t bs = state_bytes(p->state_storage) * 3 * d.NP();
        FA_CUDA_TRY(cudaMemsetAsync(P.m[*cur], 0, bs, s));
        FA_CUDA_TRY(cudaMemsetAsync(P.v[*cur], 0, bs, s));
    } else {
        Dims c = P.lvl[l - 1];
        float su[3], sm[3], sv[3];
        handoff_scales(c, d, 1, su);
        handoff_scales(c, d, -1, sm);
        handoff_scales(c, d, -2, sv);
        int nx = *cur ^ 1;
        FA_CUDA_TRY(launch_resample_field(P.u[*cur], p->field_storage, c, P.u[nx],
                                          p->field_storage, d, 3, su, s));
        if (p->state_storage == FA_F32) {
            FA_CUDA_TRY(launch_resample((const float *)P.m[*cur], c, (float *)P.m[nx], d, 3, sm, s));
            FA_CUDA_TRY(launch_resample((const float *)P.v[*cur], c, (float *)P.v[nx], d, 3, sv, s));
        } else {  // 16-bit moments: widened, resampled in FP32, rounded back
            const int st = p->state_storage;
            const long long nc = 3 * c.NP(), nf = 3 * d.NP();
            FA_CUDA_TRY(launch_widen(P.m[*cur], st, P.t1, nc, s));
            FA_CUDA_TRY(launch_resample(P.t1, c, P.t2, d, 3, sm, s));
            FA_CUDA_TRY(launch_narrow(P.t2, st, P.m[nx], nf, s));
            FA_CUDA_TRY(launch_widen(P.v[*cur], st, P.t1, nc, s));
            FA_CUDA_TRY(launch_resample(P.t1, c, P.t2, d, 3, sv, s));
            FA_CUDA_TRY(launch_narrow(P.t2, st, P.v[nx], nf, s));
        }
        *cur = nx;
    }
    // fixed-point scale of this level's images (max |I_f|, max |I_m|)
    FA_CUDA_TRY(cudaMemsetAsync(P.h->absmax_bits, 0, sizeof(P.h->absmax_bits), s));
    FA_CUDA_TRY(launch_absmax2(If, Im, d.NP(), P.h, s));  // padding (if any) holds zeros
    if (p->loss == FA_LOSS_MI) FA_CUDA_TRY(launch_mi_range(If, Im, d.N(), P.mi, s));
    if (p->mode != FA_MODE_PLAIN)
        FA_CUDA_TRY(fused_level_start(If, Im, P.u[*cur], d, p, P.h, P.fb, s));
    return FA_OK;
}

// After the last level's iterations: the final loss and u_out.
static fa_status registration_end(Plan &P, const fa_params *p, const float *If, const float *Im,
                                  const float *u, fa_vol *u_out, float *final_loss_dev,
                                  cudaStream_t s) {
    const int L = p->n_levels - 1;
    FA_TRY(final_loss(P, p, L, If, Im, u, final_loss_dev, s));
    const Dims d = P.lvl[L];
    if (p->field_storage == FA_F16) {  // widened (exactly) into the caller's dense FP32 field
        FA_CUDA_TRY(launch_resample_field(u, FA_F16, d, u_out->data, FA_F32,
                                          Dims{d.D, d.H, d.W}, 3, nullptr, s));
        return FA_OK;
    }
    FA_CUDA_TRY(cudaMemcpy2DAsync(u_out->data, sizeof(float) * d.W, u, sizeof(float) * d.pitch(),
                                  sizeof(float) * d.W, (size_t)3 * d.D * d.H,
                                  cudaMemcpyDeviceToDevice, s));
    return FA_OK;
}

// The images of level l (an unpadded scale-1 level is the full-resolution
// input itself).
static const float *level_image(const float *const *lv, int l, const float *full) {
    return lv[l] ? lv[l] : full;
}

// Everything one registration enqueues on stream s (arguments checked).
static fa_status enqueue_registration(const fa_vol *fixed, const fa_vol *moving,
                                      const fa_params *p, const float *u_init, fa_vol *u_out,
                                      float *final_loss_dev, void *ws, size_t ws_bytes,
                                      cudaStream_t s, fa_kernel_timer *timer) {
    Dims full{fixed->D, fixed->H, fixed->W};
    const int L = p->n_levels - 1;
    Plan P;
    make_plan(P, ws, ws_bytes, full, p);
    const float *If0, *Im0;
    FA_TRY(registration_begin(P, fixed, moving, p, &If0, &Im0, s));
    GaussTaps tg, tw;
    make_gauss_taps(p->sigma_grad, &tg);
    make_gauss_taps(p->sigma_warp, &tw);
    int cur = 0, t = 0;
    for (int l = 0; l < p->n_levels; ++l) {
        const float *If = level_image(P.If, l, If0);
        const float *Im = level_image(P.Im, l, Im0);
        FA_TRY(level_begin(P, p, l, l == 0 ? u_init : nullptr, If, Im, &cur, s));
        Timer tm{timer, l};
        // a level whose fused kernels are timed runs them
        const bool timed = timer && timer->kernel_id != FA_K_PLAIN_ANY &&
                           (timer->level < 0 || timer->level == l);
        if (!timed && persistent_eligible(p, P.lvl[l])) {  // the whole level in one launch
            const int T = p->iters[l];
            FA_TRY(persistent_level(P.fb, P.pxy, P.h, p, P.lvl[l], If, Im, P.u[cur], P.u[cur ^ 1],
                                    P.m[cur], P.v[cur], t, T, tg, tw, s));
            t += T;
            if (T & 1) {  // the result is in the other buffer: swap roles
                float *tmpu = P.u[cur];
                P.u[cur] = P.u[cur ^ 1];
                P.u[cur ^ 1] = tmpu;
            }
            if (l == L) FA_TRY(registration_end(P, p, If, Im, P.u[cur], u_out, final_loss_dev, s));
            continue;
        }
        for (int it = 0; it < p->iters[l]; ++it) {
            ++t;
            if (p->mode == FA_MODE_PLAIN) {
                FA_TRY(plain_iteration(P, p, l, If, Im, P.u[cur], P.u[cur ^ 1], P.m[cur], P.v[cur],
                                       t, tg, tw, tm, s));
            } else {
                FusedIter fi;
                fi.If = If;
                fi.Im = Im;
                fi.u = P.u[cur];
                fi.u_alt = P.u[cur ^ 1];
                fi.m = P.m[cur];
                fi.v = P.v[cur];
                fi.t = t;
                FA_TRY(fused_iteration(P.fb, P.h, p, P.lvl[l], fi, tg, tw, tm.t, l, s));
                // the fused compose writes u_alt: swap roles
                float *tmpu = P.u[cur];
                P.u[cur] = P.u[cur ^ 1];
                P.u[cur ^ 1] = tmpu;
            }
        }
        if (l == L) FA_TRY(registration_end(P, p, If, Im, P.u[cur], u_out, final_loss_dev, s));
    }
    return FA_OK;
}

__global__ void k_status_copy(const WsHeader *h, unsigned *out) { *out = h->status; }

// Lockstep: n registrations advance level by level and iteration by
// iteration together; job k works in the workspace slice ws + k * slot.
// Set-up, hand-off and final loss run per job; every iteration is one
// fused_iteration_lockstep over all jobs.  The jobs were checked with
// lockstep_check.
static fa_status enqueue_lockstep(int n, const LockstepArgs *a, char *ws, size_t slot,
                                  cudaStream_t s) {
    std::vector<Plan> P((size_t)n);
    std::vector<const float *> If0((size_t)n), Im0((size_t)n);
    std::vector<GaussTaps> tg((size_t)n), tw((size_t)n);
    std::vector<int> cur((size_t)n, 0);
    std::vector<LockstepJob> jobs((size_t)n);
    for (int k = 0; k < n; ++k) {
        const fa_params *p = a[k].p;
        make_plan(P[k], ws + slot * (size_t)k, slot,
                  Dims{a[k].fixed->D, a[k].fixed->H, a[k].fixed->W}, p);
        FA_TRY(registration_begin(P[k], a[k].fixed, a[k].moving, p, &If0[k], &Im0[k], s));
        make_gauss_taps(p->sigma_grad, &tg[k]);
        make_gauss_taps(p->sigma_warp, &tw[k]);
    }
    const fa_params *p0 = a[0].p;
    const int L = p0->n_levels - 1;
    int t = 0;
    for (int l = 0; l < p0->n_levels; ++l) {
        for (int k = 0; k < n; ++k) {
            const fa_params *p = a[k].p;
            LockstepJob &j = jobs[(size_t)k];
            j.d = P[k].lvl[l];
            j.If = level_image(P[k].If, l, If0[k]);
            j.Im = level_image(P[k].Im, l, Im0[k]);
            j.fb = &P[k].fb;
            j.h = P[k].h;
            j.p = p;
            j.tg = &tg[k];
            j.tw = &tw[k];
            FA_TRY(level_begin(P[k], p, l, nullptr, j.If, j.Im, &cur[k], s));
        }
        for (int it = 0; it < p0->iters[l]; ++it) {
            ++t;
            for (int k = 0; k < n; ++k) {
                LockstepJob &j = jobs[(size_t)k];
                const int c = cur[k];
                j.u = P[k].u[c];
                j.u_alt = P[k].u[c ^ 1];
                j.m = P[k].m[c];
                j.v = P[k].v[c];
            }
            FA_TRY(fused_iteration_lockstep(n, jobs.data(), t, s));
            for (int k = 0; k < n; ++k) {  // the compose wrote u_alt: swap roles
                const int c = cur[k];
                float *tmpu = P[k].u[c];
                P[k].u[c] = P[k].u[c ^ 1];
                P[k].u[c ^ 1] = tmpu;
            }
        }
        if (l == L)
            for (int k = 0; k < n; ++k) {
                const LockstepJob &j = jobs[(size_t)k];
                FA_TRY(registration_end(P[k], a[k].p, j.If, j.Im, P[k].u[cur[k]], a[k].u_out,
                                        a[k].final_loss_dev, s));
                if (a[k].status_dev) {
                    k_status_copy<<<1, 1, 0, s>>>(P[k].h, a[k].status_dev);
                    note_launch();
                    FA_CUDA_TRY(cudaGetLastError());
                }
            }
    }
    return FA_OK;
}

// ------------------------------------------------------------- graph cache
// A registration is a fixed sequence of launches for given pointers, shapes
// and parameters.  With p->graph set, the first call records that sequence
// as a CUDA graph (stream capture on a private stream of this host thread)
// and later calls with the same arguments replay it with one launch.
namespace {

constexpr size_t kMaxGraphs = 64;

// An instantiated graph, destroyed when its last holder lets go: a caller
// that found an entry keeps it alive across its cudaGraphLaunch even if
// another thread evicts the entry or clears the cache meanwhile (a graph
// destroyed while it runs on the GPU is freed when the run completes).
struct ExecHolder {
    cudaGraphExec_t exec;
    explicit ExecHolder(cudaGraphExec_t e) : exec(e) {}
    ~ExecHolder() {
        if (exec) cudaGraphExecDestroy(exec);
    }
    ExecHolder(const ExecHolder &) = delete;
    ExecHolder &operator=(const ExecHolder &) = delete;
};
using ExecRef = std::shared_ptr<ExecHolder>;

struct GraphEntry {
    std::string key;
    ExecRef exec;
    unsigned long long kernels;  // kernel launches recorded in the graph
    int timer_count;             // event pairs recorded in the graph
    unsigned long long last_use;
};

std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;
unsigned long long g_graph_clock = 0;

std::string graph_key(int dev, const fa_vol *fixed, const fa_vol *moving, const fa_params *p,
                      const float *u_init, const fa_vol *u_out, const float *final_loss_dev,
                      const void *ws, size_t ws_bytes, const fa_kernel_timer *timer) {
    // field by field: the structs may carry uninitialised padding
    std::string k;
    auto add = [&](const void *b, size_t n) { k.append((const char *)b, n); };
    auto vol = [&](const fa_vol *v) {
        add(&v->data, sizeof(v->data));
        const int32_t f[5] = {v->dtype, v->C, v->D, v->H, v->W};
        add(f, sizeof(f));
    };
    add(&dev, sizeof(dev));
    vol(fixed);
    vol(moving);
    vol(u_out);
    static_assert(sizeof(fa_params) == 34 * 4, "fa_params holds 34 four-byte fields, no padding");
    add(p, sizeof(*p));
    add(&u_init, sizeof(u_init));
    add(&final_loss_dev, sizeof(final_loss_dev));
    add(&ws, sizeof(ws));
    add(&ws_bytes, sizeof(ws_bytes));
    if (timer) {
        const int32_t f[3] = {timer->kernel_id, timer->level, timer->capacity};
        add(f, sizeof(f));
        add(&timer->start_events, sizeof(timer->start_events));
        add(&timer->stop_events, sizeof(timer->stop_events));
        if (timer->capacity > 0) {  // the event handles themselves
            add(timer->start_events, sizeof(void *) * (size_t)timer->capacity);
            add(timer->stop_events, sizeof(void *) * (size_t)timer->capacity);
        }
    }
    return k;
}

ExecRef graph_find(const std::string &key, unsigned long long *kernels, int *timer_count) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (auto &e : g_graphs)
        if (e.key == key) {
            e.last_use = ++g_graph_clock;
            *kernels = e.kernels;
            *timer_count = e.timer_count;
            return e.exec;
        }
    return nullptr;
}

void graph_store(const std::string &key, const ExecRef &exec, unsigned long long kernels,
                 int timer_count) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    if (g_graphs.size() >= kMaxGraphs) {
        size_t old = 0;
        for (size_t i = 1; i < g_graphs.size(); ++i)
            if (g_graphs[i].last_use < g_graphs[old].last_use) old = i;
        g_graphs.erase(g_graphs.begin() + (long)old);
    }
    g_graphs.push_back(GraphEntry{key, exec, kernels, timer_count, ++g_graph_clock});
}

// A private non-blocking stream of this host thread for captures (captures
// cannot run on the legacy default stream the caller may be using).
// The stream is kept per device and CUDA context: a stream of a context
// that a device reset destroyed is not reused.
cudaError_t capture_stream(cudaStream_t *out) {
    thread_local cudaStream_t cs[64] = {};
    thread_local unsigned long long cs_ctx[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    unsigned long long ctx = 0;
    if ((e = current_context_id(&ctx)) != cudaSuccess) return e;
    if (!cs[dev] || cs_ctx[dev] != ctx) {
        e = cudaStreamCreateWithFlags(&cs[dev], cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        cs_ctx[dev] = ctx;
    }
    *out = cs[dev];
    return cudaSuccess;
}

// Records what enqueue() launches on a private capture stream and
// instantiates it; the launch counter counts the recorded kernels once now.
template <class F>
fa_status graph_record(F enqueue, ExecRef *out, unsigned long long *kernels) {
    cudaStream_t cs;
    FA_CUDA_TRY(capture_stream(&cs));
    FA_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const unsigned long long k0 = launches_so_far();
    const fa_status st = enqueue(cs);
    *kernels = launches_so_far() - k0;
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (st != FA_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    FA_CUDA_TRY(ce);
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    FA_CUDA_TRY(ie);
    *out = std::make_shared<ExecHolder>(exec);
    return FA_OK;
}

}  // namespace

void graph_cache_clear() {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    g_graphs.clear();  // each graph is destroyed once no launch holds it
}

fa_status register_impl(const fa_vol *fixed, const fa_vol *moving, const fa_params *p,
                        const fa_vol *u_init, fa_vol *u_out, float *final_loss_dev,
                        float *final_loss_host, void *ws, size_t ws_bytes, cudaStream_t s,
                        fa_kernel_timer *timer) {
    FA_TRY(register_check(fixed, moving, p, u_out));
    if (u_init) {
        FA_TRY(check_vol(u_init, "u_init", 3));
        FA_TRY(same_grid(fixed, u_init, "fixed", "u_init"));
    }
    const float *ui = u_init ? (const float *)u_init->data : nullptr;
    Dims full{fixed->D, fixed->H, fixed->W};
    Plan P;
    make_plan(P, nullptr, ~size_t(0), full, p);
    FA_TRY(check_ws(ws, ws_bytes, P.bytes, "fa_register"));
    if (timer) {
        if (timer->capacity < 0 || (timer->capacity > 0 && (!timer->start_events || !timer->stop_events))) {
            set_error("fa_register_timed: bad timer");
            return FA_ERR_INVALID;
        }
        timer->count = 0;
    }
    if (p->graph) {
        int dev = 0;
        FA_CUDA_TRY(cudaGetDevice(&dev));
        const std::string key =
            graph_key(dev, fixed, moving, p, ui, u_out, final_loss_dev, ws, ws_bytes, timer);
        unsigned long long kernels = 0;
        int timer_count = 0;
        ExecRef exec = graph_find(key, &kernels, &timer_count);
        if (!exec) {
            // record (the launch counter counts the recorded kernels once now,
            // for this first run, and again at every later replay)
            FA_TRY(graph_record(
                [&](cudaStream_t cs) {
                    return enqueue_registration(fixed, moving, p, ui, u_out, final_loss_dev, ws,
                                                ws_bytes, cs, timer);
                },
                &exec, &kernels));
            graph_store(key, exec, kernels, timer ? timer->count : 0);
        } else {
            note_launches(kernels);
            if (timer) timer->count = timer_count;
        }
        FA_CUDA_TRY(cudaGraphLaunch(exec->exec, s));
    } else {
        FA_TRY(enqueue_registration(fixed, moving, p, ui, u_out, final_loss_dev, ws, ws_bytes, s,
                                    timer));
    }
    if (final_loss_host) {
        FA_CUDA_TRY(cudaStreamSynchronize(s));
        FA_CUDA_TRY(cudaMemcpy(final_loss_host, &((const WsHeader *)ws)->loss, sizeof(float),
                               cudaMemcpyDeviceToHost));
        return fa_ws_status(ws, s);
    }
    return FA_OK;
}

fa_status lockstep_check(int n, const LockstepArgs *a) {
    if (n < 1 || n > kMaxLockstepJobs) {
        set_error("lockstep: 1..%d jobs at a time (got %d)", kMaxLockstepJobs, n);
        return FA_ERR_INVALID;
    }
    const fa_params *p0 = a[0].p;
    for (int k = 0; k < n; ++k) {
        const fa_params *p = a[k].p;
        if ((p->mode != FA_MODE_FUSED && p->mode != FA_MODE_PERSISTENT) ||
            p->loss != FA_LOSS_LNCC || p->use_jac) {
            set_error("lockstep: job %d: needs the fused LNCC path without use_jac", k);
            return FA_ERR_UNSUPPORTED;
        }
        bool same = p->n_levels == p0->n_levels && p->window == p0->window &&
                    p->beta1 == p0->beta1 && p->beta2 == p0->beta2 &&
                    p->adam_eps == p0->adam_eps;
        for (int l = 0; same && l < p0->n_levels; ++l)
            same = p->scales[l] == p0->scales[l] && p->iters[l] == p0->iters[l];
        if (!same) {
            set_error("lockstep: job %d: every job needs the same levels, iterations, window "
                      "and Adam constants", k);
            return FA_ERR_UNSUPPORTED;
        }
        GaussTaps tg, tw;
        make_gauss_taps(p->sigma_grad, &tg);
        make_gauss_taps(p->sigma_warp, &tw);
        if (tg.R > kMaxFusedRadius || tw.R > kMaxFusedRadius) {
            set_error("lockstep: job %d: Gaussian radius above %d (sigma above %g)", k,
                      kMaxFusedRadius, (double)kMaxFusedRadius / 3.0);
            return FA_ERR_UNSUPPORTED;
        }
    }
    return FA_OK;
}

fa_status register_lockstep(int n, const LockstepArgs *a, void *ws, size_t slot, cudaStream_t s) {
    FA_TRY(lockstep_check(n, a));
    bool graph = true;
    for (int k = 0; k < n; ++k) graph = graph && a[k].p->graph;
    if (!graph) return enqueue_lockstep(n, a, (char *)ws, slot, s);
    int dev = 0;
    FA_CUDA_TRY(cudaGetDevice(&dev));
    std::string key("lockstep");
    for (int k = 0; k < n; ++k) {
        key += graph_key(dev, a[k].fixed, a[k].moving, a[k].p, nullptr, a[k].u_out,
                         a[k].final_loss_dev, (char *)ws + slot * (size_t)k, slot, nullptr);
        key.append((const char *)&a[k].status_dev, sizeof(a[k].status_dev));
    }
    unsigned long long kernels = 0;
    int timer_count = 0;
    ExecRef exec = graph_find(key, &kernels, &timer_count);
    if (!exec) {
        FA_TRY(graph_record([&](cudaStream_t cs) { return enqueue_lockstep(n, a, (char *)ws, slot, cs); },
                            &exec, &kernels));
        graph_store(key, exec, kernels, 0);
    } else {
        note_launches(kernels);
    }
    FA_CUDA_TRY(cudaGraphLaunch(exec->exec, s));
    return FA_OK;
}

size_t register_ws_bytes(int D, int H, int W, const fa_params *p) {
    if (D < 1 || H < 1 || W < 1 || check_params(p) != FA_OK) return 0;
    Plan P;
    make_plan(P, nullptr, ~size_t(0), Dims{D, H, W}, p);
    return P.bytes;
}

}  // namespace fa

extern "C" size_t fa_register_workspace_size(int32_t D, int32_t H, int32_t W, const fa_params *p) {
    fa::clear_error();
    return fa::register_ws_bytes(D, H, W, p);
}

extern "C" size_t fa_workspace_size(const fa_vol *fixed, const fa_params *p) {
    fa::clear_error();
    if (!fixed) return 0;
    return fa::register_ws_bytes(fixed->D, fixed->H, fixed->W, p);
}

extern "C" fa_status fa_register(const fa_vol *fixed, const fa_vol *moving, const fa_params *p,
                                 fa_vol *u_out, float *final_loss_dev, float *final_loss_host,
                                 void *ws, size_t ws_bytes, void *stream) {
    fa::clear_error();
    return fa::register_impl(fixed, moving, p, nullptr, u_out, final_loss_dev, final_loss_host, ws,
                             ws_bytes, (cudaStream_t)stream, nullptr);
}

extern "C" fa_status fa_register_from(const fa_vol *fixed, const fa_vol *moving,
                                      const fa_params *p, const fa_vol *u_init, fa_vol *u_out,
                                      float *final_loss_dev, float *final_loss_host, void *ws,
                                      size_t ws_bytes, void *stream) {
    fa::clear_error();
    return fa::register_impl(fixed, moving, p, u_init, u_out, final_loss_dev, final_loss_host, ws,
                             ws_bytes, (cudaStream_t)stream, nullptr);
}

extern "C" fa_status fa_autotune(int32_t D, int32_t H, int32_t W, const fa_params *p, void *ws,
                                 size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    if (D < 1 || H < 1 || W < 1) {
        set_error("fa_autotune: grid must be positive");
        return FA_ERR_SHAPE;
    }
    FA_TRY(check_params(p));
    if (p->mode == FA_MODE_PLAIN) return FA_OK;  // the per-op kernels have no choices
    Dims full{D, H, W};
    Plan P;
    make_plan(P, nullptr, ~size_t(0), full, p);
    FA_TRY(check_ws(ws, ws_bytes, P.bytes, "fa_autotune"));
    make_plan(P, ws, ws_bytes, full, p);
    cudaStream_t s = (cudaStream_t)stream;
    FA_CUDA_TRY(cudaMemsetAsync(ws, 0, P.bytes, s));
    GaussTaps tg, tw;
    make_gauss_taps(p->sigma_grad, &tg);
    make_gauss_taps(p->sigma_warp, &tw);
    for (int l = 0; l < p->n_levels; ++l) {
        const Dims d = P.lvl[l];
        // stand-in images (zeros): timing does not depend on the values much,
        // and every choice computes the same bits
        const float *If = P.If[l] ? P.If[l] : P.t1;
        const float *Im = P.Im[l] ? P.Im[l] : P.t2;
        FA_TRY(fused_autotune_level(P.fb, P.h, p, d, If, Im, P.u[0], P.u[1], P.m[0], P.v[0], tg,
                                    tw, s));
    }
    graph_cache_clear();  // recorded graphs hold the previous choices
    return FA_OK;
}

extern "C" fa_status fa_graph_cache_clear(void) {
    fa::clear_error();
    fa::graph_cache_clear();
    return FA_OK;
}

extern "C" fa_status fa_autotune_reset(void) {
    fa::clear_error();
    fa::fused_autotune_reset();
    fa::graph_cache_clear();
    return FA_OK;
}

extern "C" fa_status fa_autotune_set(const int32_t *row) {
    using namespace fa;
    clear_error();
    if (!row || row[0] < 0 || row[0] > 3 || row[1] < 0 || row[1] > 7 || row[2] < 0 || row[2] > 1 ||
        row[3] < 1 || row[4] < 1 || row[5] < 1 || row[6] < 0 || row[6] > 1 || row[7] < 0) {
        set_error("fa_autotune_set: row must be (kernel 0..3, radius 0..7, variant 0..1, D, H, W "
                  "> 0, wide 0..1, tz >= 0)");
        return FA_ERR_INVALID;
    }
    fused_tile_set(row);
    graph_cache_clear();
    return FA_OK;
}

extern "C" int32_t fa_autotune_choices(int32_t *rows, int32_t capacity) {
    fa::clear_error();
    return fa::fused_tile_choices(rows, capacity);
}

extern "C" fa_status fa_register_timed(const fa_vol *fixed, const fa_vol *moving,
                                       const fa_params *p, fa_vol *u_out, float *final_loss_dev,
                                       float *final_loss_host, void *ws, size_t ws_bytes,
                                       void *stream, fa_kernel_timer *timer) {
    fa::clear_error();
    return fa::register_impl(fixed, moving, p, nullptr, u_out, final_loss_dev, final_loss_host, ws,
                             ws_bytes, (cudaStream_t)stream, timer);
}
