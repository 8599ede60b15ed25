// Affine pre-registration (the paper aligns affinely before the
// diffeomorphic stage, with Adam at learning rate 3e-3 over a multi-scale
// schedule; section "Lung CT mapping challenges").
//
// The map acts on align-corners normalised coordinates p_a = 2 x_a / (n_a - 1)
// - 1 (0 on an axis of length 1): p' = A p + t, theta = (A row-major, t), so
// the parameters mean the same at every pyramid level.  Per iteration: the
// displacement of theta, the warp with its gradient, the LNCC (or MSE)
// gradient g = dL/dJ grad I_m(phi) from the per-op kernels, the 12 sums
//   dL/dA_ab = sum_x g_a h_a p_b,   dL/dt_a = sum_x g_a h_a   (h_a = (n_a - 1)/2)
// in a fixed order (block partials, then one float-float pass), and a plain
// Adam step on theta in a 12-thread kernel: no host synchronisation, so the
// whole stage records into a graph.
#include "ops.h"
#include "validate.h"

namespace fa {

namespace {

constexpr int kRedBlocks = 152 * 4;  // partial sums per iteration (fixed: deterministic order)

struct AffineWs {
    WsHeader *h;
    float *If[8], *Im[8];   // pyramid levels (nullptr for scale 1)
    Dims lvl[8];
    float *u, *J, *grad, *g, *t1, *t2, *partials;
    float *theta, *m, *v;   // 12 each
    float *rp;              // 6 rigid parameters (rigid stage only)
    LnccBuffers lb;
};

void affine_carve(WsCarver &c, Dims full, const fa_params *p, AffineWs *w) {
    long long nmax = 0;
    w->h = c.take<WsHeader>(1);
    for (int l = 0; l < p->n_levels; ++l) {
        const int s = p->scales[l];
        w->lvl[l] = Dims{level_size(full.D, s), level_size(full.H, s), level_size(full.W, s)};
        nmax = w->lvl[l].N() > nmax ? w->lvl[l].N() : nmax;
        if (s == 1) {
            w->If[l] = w->Im[l] = nullptr;
        } else {
            w->If[l] = c.take<float>(w->lvl[l].N());
            w->Im[l] = c.take<float>(w->lvl[l].N());
        }
    }
    const long long tmp = full.N() > 3 * nmax ? full.N() : 3 * nmax;
    w->t1 = c.take<float>(tmp);
    w->t2 = c.take<float>(tmp);
    w->u = c.take<float>(3 * nmax);
    w->J = c.take<float>(nmax);
    w->grad = c.take<float>(3 * nmax);
    w->g = c.take<float>(3 * nmax);
    long long np = kRedBlocks * 12;
    for (int l = 0; l < p->n_levels; ++l) {
        const long long k = mse_partials_count(w->lvl[l]);
        np = k > np ? k : np;
    }
    w->partials = c.take<float>(np);
    w->theta = c.take<float>(12);
    w->m = c.take<float>(12);
    w->v = c.take<float>(12);
    w->rp = c.take<float>(6);
    w->lb = lncc_carve(c, nmax);
}

__device__ __forceinline__ void norm_coords(int z, int y, int x, const int n[3], const float half[3],
                                            float p[3]) {
    const int xi[3] = {z, y, x};
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] = n[a] > 1 ? (float)xi[a] / half[a] - 1.0f : 0.0f;
}

__global__ void __launch_bounds__(256) k_affine_field(const float *__restrict__ theta,
                                                      float *__restrict__ u, int D, int H, int W) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y,
              z = blockIdx.z;
    if (x >= W || y >= H) return;
    const int n[3] = {D, H, W};
    float half[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) half[a] = n[a] > 1 ? 0.5f * (float)(n[a] - 1) : 0.0f;
    float pv[3];
    norm_coords(z, y, x, n, half, pv);
    const long long N = (long long)D * H * W, i = ((long long)z * H + y) * W + x;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float q = theta[9 + a];
#pragma unroll
        for (int b = 0; b < 3; ++b) q = fmaf(theta[3 * a + b], pv[b], q);
        u[a * N + i] = (q - pv[a]) * half[a];
    }
}

// Block b sums the 12 gradient terms of its voxels (grid-stride, fixed
// order) into partials[b][12].
__global__ void __launch_bounds__(256) k_affine_partials(const float *__restrict__ g, int D, int H,
                                                         int W, float *__restrict__ partials) {
    __shared__ float red[12][8];
    const int n[3] = {D, H, W};
    float half[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) half[a] = n[a] > 1 ? 0.5f * (float)(n[a] - 1) : 0.0f;
    const long long N = (long long)D * H * W, HW = (long long)H * W;
    float acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(i / HW), rem = (int)(i - (long long)z * HW), y = rem / W, x = rem - y * W;
        float pv[3];
        norm_coords(z, y, x, n, half, pv);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float ga = g[a * N + i] * half[a];
#pragma unroll
            for (int b = 0; b < 3; ++b) acc[3 * a + b] = fmaf(ga, pv[b], acc[3 * a + b]);
            acc[9 + a] += ga;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        float s = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[k][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        float s = 0.0f;
        for (int w = 0; w < 8; ++w) s += red[threadIdx.x][w];
        partials[(long long)blockIdx.x * 12 + threadIdx.x] = s;
    }
}

// 12 warps: warp k sums parameter k's partials in float-float (fixed order),
// then one Adam step theta_k -= lr m^ / (sqrt(v^) + eps).
__global__ void __launch_bounds__(384) k_affine_adam(const float *__restrict__ partials, int nblocks,
                                                     float *theta, float *m, float *v,
                                                     AdamConsts ac, float lr) {
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float hi = 0.0f, lo = 0.0f;
    for (int b = lane; b < nblocks; b += 32) ff_add(hi, lo, partials[(long long)b * 12 + k], 0.0f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
        ff_add(hi, lo, oh, ol);
    }
    if (lane == 0) {
        const float gk = hi + lo;
        const float mk = fmaf(ac.b1, m[k], (1.0f - ac.b1) * gk);
        const float vk = fmaf(ac.b2, v[k], (1.0f - ac.b2) * gk * gk);
        m[k] = mk;
        v[k] = vk;
        theta[k] -= lr * adam_dir(mk, vk, ac.rbc1, ac.rbc2, ac.eps);
    }
}

__global__ void k_affine_init(float *theta, float *m, float *v) {
    const int k = threadIdx.x;
    if (k < 12) {
        theta[k] = (k == 0 || k == 4 || k == 8) ? 1.0f : 0.0f;
        m[k] = 0.0f;
        v[k] = 0.0f;
    }
}

// ---------------------------------------------------------------- rigid
// Rigid stage: rp = (w, t), R = exp([w]x) by the Rodrigues formula, the
// affine map A = S^-1 R S, t on normalised coordinates (S = diag((n_a - 1)/2)
// of the input grid, 1 on an axis of length 1), so that the motion is rigid
// in the input grid's voxels about its centre.  The 12 affine sums are pulled
// back exactly: dL/dt = dL/dt_aff, dL/dw_k = sum_ij dL/dA_ij (s_j / s_i)
// dR_ij/dw_k, with
//   R = I + a K + b K^2,  dR/dw_k = c1 w_k K + a E_k + c2 w_k K^2 + b (E_k K + K E_k)
// (K = [w]x, E_k = [e_k]x, a = sin th / th, b = (1 - cos th) / th^2,
// c1 = a'(th) / th, c2 = b'(th) / th).  One thread evaluates this in FP32
// (six parameters): below th = 1 the four coefficients come from their
// Taylor series (terms to th^14, so the truncation lies far below FP32's
// unit roundoff there), where the closed forms for c1 and c2 would cancel;
// from th = 1 up the closed forms, with 1 - cos th taken as 2 sin^2(th / 2).
// sin and cos without FP64 (the library's sincosf brings FP64 instructions
// in through its reduction of huge arguments): the Cody-Waite reduction
// x = k pi/2 + r with pi/2 split into three floats P1 + P2 + P3 whose
// leading two have 8 and 11 significant bits, so k P1 and k P2 are exact for
// |k| < 2^12 (|x| below about 6400; beyond that the error grows with k), then
// the Taylor polynomials of sin (to r^13) and cos (to r^14) on |r| <= pi/4,
// whose truncation lies below 2^-40, and the quadrant k mod 4.
__device__ void sincos_cw(float x, float *sn, float *cs) {
    const float P1 = 1.5703125f, P2 = 0x1.fb4p-12f, P3 = 0x1.4442d2p-24f;
    const float k = rintf(x * 0.636619772f);
    float r = fmaf(-k, P1, x);
    r = fmaf(-k, P2, r);
    r = fmaf(-k, P3, r);
    const float r2 = r * r;
    float ps = 1.0f / 6227020800.0f;                 // 1/13!
    ps = fmaf(ps, -r2, 1.0f / 39916800.0f);
    ps = fmaf(ps, -r2, 1.0f / 362880.0f);
    ps = fmaf(ps, -r2, 1.0f / 5040.0f);
    ps = fmaf(ps, -r2, 1.0f / 120.0f);
    ps = fmaf(ps, -r2, 1.0f / 6.0f);
    const float sr = fmaf(r * r2, -ps, r);           // r - r^3 (1/6 - ...)
    float pc = 1.0f / 87178291200.0f;                // 1/14!
    pc = fmaf(pc, -r2, 1.0f / 479001600.0f);
    pc = fmaf(pc, -r2, 1.0f / 3628800.0f);
    pc = fmaf(pc, -r2, 1.0f / 40320.0f);
    pc = fmaf(pc, -r2, 1.0f / 720.0f);
    pc = fmaf(pc, -r2, 1.0f / 24.0f);
    pc = fmaf(pc, -r2, 0.5f);
    const float cr = fmaf(r2, -pc, 1.0f);             // 1 - r^2 (1/2 - ...)
    const int q = ((int)k) & 3;
    *sn = q == 0 ? sr : (q == 1 ? cr : (q == 2 ? -sr : -cr));
    *cs = q == 0 ? cr : (q == 1 ? -sr : (q == 2 ? -cr : sr));
}

__device__ void rodrigues_f(const float w[3], float R[9], float dR[27]) {
    const float th2 = fmaf(w[0], w[0], fmaf(w[1], w[1], w[2] * w[2])), th = sqrtf(th2);
    float a, b, c1, c2;
    if (th < 1.0f) {
        // a = sum (-1)^k th^2k / (2k+1)!,   b = sum (-1)^k th^2k / (2k+2)!,
        // c1 = sum_{k>=1} (-1)^k 2k th^(2k-2) / (2k+1)!,
        // c2 = sum_{k>=1} (-1)^k 2k th^(2k-2) / (2k+2)!   (Horner in th^2)
        a = 1.0f / 6227020800.0f;                    // 1/13!
        a = fmaf(a, -th2, 1.0f / 39916800.0f);       // 1/11!
        a = fmaf(a, -th2, 1.0f / 362880.0f);
        a = fmaf(a, -th2, 1.0f / 5040.0f);
        a = fmaf(a, -th2, 1.0f / 120.0f);
        a = fmaf(a, -th2, 1.0f / 6.0f);
        a = fmaf(a, -th2, 1.0f);
        b = 1.0f / 87178291200.0f;                   // 1/14!
        b = fmaf(b, -th2, 1.0f / 479001600.0f);      // 1/12!
        b = fmaf(b, -th2, 1.0f / 3628800.0f);
        b = fmaf(b, -th2, 1.0f / 40320.0f);
        b = fmaf(b, -th2, 1.0f / 720.0f);
        b = fmaf(b, -th2, 1.0f / 24.0f);
        b = fmaf(b, -th2, 0.5f);
        c1 = -14.0f / 1307674368000.0f;              // k = 7: -14/15!
        c1 = fmaf(c1, th2, 12.0f / 6227020800.0f);   // k = 6: 12/13!
        c1 = fmaf(c1, th2, -10.0f / 39916800.0f);
        c1 = fmaf(c1, th2, 8.0f / 362880.0f);
        c1 = fmaf(c1, th2, -6.0f / 5040.0f);
        c1 = fmaf(c1, th2, 4.0f / 120.0f);
        c1 = fmaf(c1, th2, -2.0f / 6.0f);
        c2 = -14.0f / 20922789888000.0f;             // k = 7: -14/16!
        c2 = fmaf(c2, th2, 12.0f / 87178291200.0f);  // k = 6: 12/14!
        c2 = fmaf(c2, th2, -10.0f / 479001600.0f);
        c2 = fmaf(c2, th2, 8.0f / 3628800.0f);
        c2 = fmaf(c2, th2, -6.0f / 40320.0f);
        c2 = fmaf(c2, th2, 4.0f / 720.0f);
        c2 = fmaf(c2, th2, -2.0f / 24.0f);
    } else {
        float sn, cs, sh, ch;
        sincos_cw(th, &sn, &cs);
        sincos_cw(0.5f * th, &sh, &ch);
        const float omc = 2.0f * sh * sh;  // 1 - cos th
        a = sn / th;
        b = omc / th2;
        c1 = fmaf(th, cs, -sn) / (th2 * th);
        c2 = fmaf(th, sn, -2.0f * omc) / (th2 * th2);
    }
    const float K[9] = {0.0f, -w[2], w[1], w[2], 0.0f, -w[0], -w[1], w[0], 0.0f};
    float K2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            float s = 0.0f;
            for (int q = 0; q < 3; ++q) s = fmaf(K[3 * i + q], K[3 * q + j], s);
            K2[3 * i + j] = s;
        }
    for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0 ? 1.0f : 0.0f) + fmaf(a, K[i], b * K2[i]);
    if (!dR) return;
    for (int k = 0; k < 3; ++k) {
        const float e0 = k == 0, e1 = k == 1, e2 = k == 2;
        const float E[9] = {0.0f, -e2, e1, e2, 0.0f, -e0, -e1, e0, 0.0f};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                float ek = 0.0f, ke = 0.0f;
                for (int q = 0; q < 3; ++q) {
                    ek = fmaf(E[3 * i + q], K[3 * q + j], ek);
                    ke = fmaf(K[3 * i + q], E[3 * q + j], ke);
                }
                const int ij = 3 * i + j;
                dR[9 * k + ij] =
                    fmaf(c1 * w[k], K[ij], fmaf(a, E[ij], fmaf(c2 * w[k], K2[ij], b * (ek + ke))));
            }
    }
}

struct RigidScales {
    float s[3];
};

__device__ void rigid_theta_f(const float *rp, RigidScales sc, float *theta) {
    const float w[3] = {rp[0], rp[1], rp[2]};
    float R[9];
    rodrigues_f(w, R, nullptr);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) theta[3 * i + j] = R[3 * i + j] * (sc.s[j] / sc.s[i]);
        theta[9 + i] = rp[3 + i];
    }
}

__global__ void k_rigid_theta(const float *rp, float *theta, RigidScales sc) {
    if (threadIdx.x == 0) rigid_theta_f(rp, sc, theta);
}

__global__ void k_rigid_init(float *rp, float *m, float *v, float *theta, RigidScales sc) {
    const int k = threadIdx.x;
    if (k < 6) {
        rp[k] = 0.0f;
        m[k] = 0.0f;
        v[k] = 0.0f;
    }
    __syncthreads();
    if (k == 0) rigid_theta_f(rp, sc, theta);
}

// 12 warps sum the affine partials (float-float, fixed order); thread 0 pulls
// them back to the 6 rigid parameters, takes one Adam step and rewrites theta.
__global__ void __launch_bounds__(384) k_rigid_adam(const float *__restrict__ partials,
                                                    int nblocks, float *rp, float *m, float *v,
                                                    float *theta, RigidScales sc, AdamConsts ac,
                                                    float lr) {
    __shared__ float gaff[12];
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float hi = 0.0f, lo = 0.0f;
    for (int b = lane; b < nblocks; b += 32) ff_add(hi, lo, partials[(long long)b * 12 + k], 0.0f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
        ff_add(hi, lo, oh, ol);
    }
    if (lane == 0) gaff[k] = hi + lo;
    __syncthreads();
    if (threadIdx.x != 0) return;
    const float w[3] = {rp[0], rp[1], rp[2]};
    float R[9], dR[27];
    rodrigues_f(w, R, dR);
    float g[6];
    for (int q = 0; q < 3; ++q) {
        float acc = 0.0f;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                acc = fmaf(gaff[3 * i + j] * (sc.s[j] / sc.s[i]), dR[9 * q + 3 * i + j], acc);
        g[q] = acc;
        g[3 + q] = gaff[9 + q];
    }
    for (int q = 0; q < 6; ++q) {
        const float mq = fmaf(ac.b1, m[q], (1.0f - ac.b1) * g[q]);
        const float vq = fmaf(ac.b2, v[q], (1.0f - ac.b2) * g[q] * g[q]);
        m[q] = mq;
        v[q] = vq;
        rp[q] -= lr * adam_dir(mq, vq, ac.rbc1, ac.rbc2, ac.eps);
    }
    rigid_theta_f(rp, sc, theta);
}

RigidScales rigid_scales(Dims full) {
    RigidScales sc;
    const int n[3] = {full.D, full.H, full.W};
    for (int a = 0; a < 3; ++a) sc.s[a] = n[a] > 1 ? 0.5f * (float)(n[a] - 1) : 1.0f;
    return sc;
}

fa_status check_affine_params(const fa_params *p) {
    if (!p || p->n_levels < 1 || p->n_levels > 8) {
        set_error("fa_affine_register: n_levels must be in 1..8");
        return FA_ERR_INVALID;
    }
    for (int l = 0; l < p->n_levels; ++l)
        if (p->scales[l] < 1 || 0.5f * (float)p->scales[l] > kMaxSigma || p->iters[l] < 0) {
            set_error("fa_affine_register: level %d: scale in 1..%d, iterations >= 0", l,
                      (int)(2 * kMaxSigma));
            return FA_ERR_INVALID;
        }
    if (p->loss != FA_LOSS_LNCC && p->loss != FA_LOSS_MSE) {
        set_error("fa_affine_register: loss must be FA_LOSS_LNCC or FA_LOSS_MSE");
        return FA_ERR_INVALID;
    }
    if (p->loss == FA_LOSS_LNCC && (p->window < 1 || p->window > 15 || p->window % 2 == 0)) {
        set_error("fa_affine_register: window must be odd and in 1..15");
        return FA_ERR_INVALID;
    }
    if (!(p->cc_eps >= 0.0f && p->cc_eps < 3e38f)) {
        set_error("fa_affine_register: cc_eps must be finite and >= 0");
        return FA_ERR_INVALID;
    }
    return check_adam_params(p, "fa_affine_register");
}

size_t affine_ws_bytes(Dims full, const fa_params *p) {
    WsCarver c(nullptr, ~size_t(0));
    AffineWs w;
    affine_carve(c, full, p, &w);
    return c.off;
}

// loss gradient g (3 channels) of level l at the current theta, and the loss
// accumulator in h when want_loss
cudaError_t affine_gradient(AffineWs &w, const fa_params *p, const float *If, const float *Im,
                            Dims d, bool want_grad, cudaStream_t s) {
    VoxGrid vg(d.D, d.H, d.W);
    k_affine_field<<<vg.grid, vg.block, 0, s>>>(w.theta, w.u, d.D, d.H, d.W);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_warp(Im, w.u, w.J, want_grad ? w.grad : nullptr, d, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(w.h, 0, sizeof(WsHeader), s);
    if (e != cudaSuccess) return e;
    if (p->loss == FA_LOSS_LNCC) {
        e = launch_absmax2(If, w.J, d.N(), w.h, s);
        if (e == cudaSuccess)
            e = launch_lncc_forward(If, w.J, d, p->window, p->cc_eps, false, w.h, w.lb, s);
        if (e == cudaSuccess && want_grad)
            e = launch_lncc_backward(If, w.J, w.grad, d, p->window, w.h, w.lb, nullptr, nullptr,
                                     w.g, s);
        return e;
    }
    return launch_mse(If, w.J, want_grad ? w.grad : nullptr, d, w.h, w.partials, nullptr,
                      nullptr, want_grad ? w.g : nullptr, s);
}

}  // namespace

}  // namespace fa

extern "C" size_t fa_affine_workspace_size(int32_t D, int32_t H, int32_t W, const fa_params *p) {
    using namespace fa;
    clear_error();
    if (D < 1 || H < 1 || W < 1 || check_affine_params(p) != FA_OK) return 0;
    return affine_ws_bytes(Dims{D, H, W}, p);
}

namespace fa {
namespace {

// The affine stage, or with rp_dev the rigid one (its 6 parameters are
// written to rp_dev, the equivalent affine map to theta_dev).
fa_status linear_stage(const fa_vol *fixed, const fa_vol *moving, const fa_params *p, bool rigid,
                       float *theta_dev, float *rp_dev, fa_vol *u_out_opt, float *final_loss_dev,
                       void *ws, size_t ws_bytes, void *stream) {
    FA_TRY(check_affine_params(p));
    FA_TRY(check_vol(fixed, "fixed", 1));
    FA_TRY(check_vol(moving, "moving", 1));
    FA_TRY(same_grid(fixed, moving, "fixed", "moving"));
    if (!theta_dev && !rigid) {
        set_error("fa_affine_register: theta_dev must not be NULL");
        return FA_ERR_INVALID;
    }
    const Dims full{fixed->D, fixed->H, fixed->W};
    const int L = p->n_levels - 1;
    const Dims last{level_size(full.D, p->scales[L]), level_size(full.H, p->scales[L]),
                    level_size(full.W, p->scales[L])};
    if (u_out_opt) {
        FA_TRY(check_vol(u_out_opt, "u_out", 3));
        if (u_out_opt->D != last.D || u_out_opt->H != last.H || u_out_opt->W != last.W) {
            set_error("u_out must be 3 x %d x %d x %d (the last level's grid)", last.D, last.H,
                      last.W);
            return FA_ERR_SHAPE;
        }
    }
    FA_TRY(check_ws(ws, ws_bytes, affine_ws_bytes(full, p), "fa_affine_register"));
    WsCarver c(ws, ws_bytes);
    AffineWs w;
    affine_carve(c, full, p, &w);
    cudaStream_t s = (cudaStream_t)stream;
    const float *If0 = (const float *)fixed->data, *Im0 = (const float *)moving->data;
    const RigidScales sc = rigid_scales(full);
    if (rigid)
        k_rigid_init<<<1, 32, 0, s>>>(w.rp, w.m, w.v, w.theta, sc);
    else
        k_affine_init<<<1, 32, 0, s>>>(w.theta, w.m, w.v);
    note_launch();
    FA_CUDA_TRY(cudaGetLastError());
    for (int l = 0; l < p->n_levels; ++l) {
        if (p->scales[l] == 1) continue;
        FA_CUDA_TRY(launch_pyramid_level(If0, full, p->scales[l], w.If[l], w.lvl[l], w.t1, w.t2, s));
        FA_CUDA_TRY(launch_pyramid_level(Im0, full, p->scales[l], w.Im[l], w.lvl[l], w.t1, w.t2, s));
    }
    int t = 0;
    for (int l = 0; l < p->n_levels; ++l) {
        const Dims d = w.lvl[l];
        const float *If = p->scales[l] == 1 ? If0 : w.If[l];
        const float *Im = p->scales[l] == 1 ? Im0 : w.Im[l];
        for (int it = 0; it < p->iters[l]; ++it) {
            FA_CUDA_TRY(affine_gradient(w, p, If, Im, d, true, s));
            k_affine_partials<<<kRedBlocks, 256, 0, s>>>(w.g, d.D, d.H, d.W, w.partials);
            note_launch();
            FA_CUDA_TRY(cudaGetLastError());
            ++t;
            if (rigid)
                k_rigid_adam<<<1, 384, 0, s>>>(w.partials, kRedBlocks, w.rp, w.m, w.v, w.theta, sc,
                                               adam_consts(p, t), p->lr);
            else
                k_affine_adam<<<1, 384, 0, s>>>(w.partials, kRedBlocks, w.theta, w.m, w.v,
                                                adam_consts(p, t), p->lr);
            note_launch();
            FA_CUDA_TRY(cudaGetLastError());
        }
        if (l == L) {
            FA_CUDA_TRY(affine_gradient(w, p, If, Im, d, false, s));
            if (p->loss == FA_LOSS_LNCC) {
                FA_CUDA_TRY(launch_loss_finalize(w.h, d.N(), -1.0f, final_loss_dev, s));
            } else if (final_loss_dev) {
                FA_CUDA_TRY(cudaMemcpyAsync(final_loss_dev, &w.h->loss, sizeof(float),
                                            cudaMemcpyDeviceToDevice, s));
            }
            if (u_out_opt)
                FA_CUDA_TRY(cudaMemcpyAsync(u_out_opt->data, w.u, sizeof(float) * 3 * d.N(),
                                            cudaMemcpyDeviceToDevice, s));
        }
    }
    if (theta_dev)
        FA_CUDA_TRY(
            cudaMemcpyAsync(theta_dev, w.theta, 12 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (rigid)
        FA_CUDA_TRY(cudaMemcpyAsync(rp_dev, w.rp, 6 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return FA_OK;
}

}  // namespace
}  // namespace fa

extern "C" fa_status fa_affine_register(const fa_vol *fixed, const fa_vol *moving,
                                        const fa_params *p, float *theta_dev, fa_vol *u_out_opt,
                                        float *final_loss_dev, void *ws, size_t ws_bytes,
                                        void *stream) {
    fa::clear_error();
    return fa::linear_stage(fixed, moving, p, false, theta_dev, nullptr, u_out_opt,
                            final_loss_dev, ws, ws_bytes, stream);
}

extern "C" fa_status fa_rigid_register(const fa_vol *fixed, const fa_vol *moving,
                                       const fa_params *p, float *rp_dev, float *theta_dev,
                                       fa_vol *u_out_opt, float *final_loss_dev, void *ws,
                                       size_t ws_bytes, void *stream) {
    fa::clear_error();
    if (!rp_dev) {
        fa::set_error("fa_rigid_register: rp_dev must not be NULL");
        return FA_ERR_INVALID;
    }
    return fa::linear_stage(fixed, moving, p, true, theta_dev, rp_dev, u_out_opt,
                            final_loss_dev, ws, ws_bytes, stream);
}

extern "C" fa_status fa_affine_field(const float *theta_dev, fa_vol *u_out, void *stream) {
    using namespace fa;
    clear_error();
    if (!theta_dev) {
        set_error("fa_affine_field: theta_dev must not be NULL");
        return FA_ERR_INVALID;
    }
    FA_TRY(check_vol(u_out, "u_out", 3));
    VoxGrid vg(u_out->D, u_out->H, u_out->W);
    k_affine_field<<<vg.grid, vg.block, 0, (cudaStream_t)stream>>>(
        theta_dev, (float *)u_out->data, u_out->D, u_out->H, u_out->W);
    note_launch();
    FA_CUDA_TRY(cudaGetLastError());
    return FA_OK;
}

extern "C" fa_status fa_rigid_theta(const float *rp_dev, int32_t D, int32_t H, int32_t W,
                                    float *theta_dev, void *stream) {
    using namespace fa;
    clear_error();
    if (!rp_dev || !theta_dev) {
        set_error("fa_rigid_theta: rp_dev and theta_dev must not be NULL");
        return FA_ERR_INVALID;
    }
    if (D < 1 || H < 1 || W < 1) {
        set_error("fa_rigid_theta: grid must be positive");
        return FA_ERR_SHAPE;
    }
    k_rigid_theta<<<1, 32, 0, (cudaStream_t)stream>>>(rp_dev, theta_dev,
                                                       rigid_scales(Dims{D, H, W}));
    note_launch();
    FA_CUDA_TRY(cudaGetLastError());
    return FA_OK;
}
