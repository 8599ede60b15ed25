// LNCC and MSE losses with their analytic gradients, one kernel per
// operation (the plain per-op form; fa_register's fused form lives in
// fused.cu).
//
// LNCC (the local normalised cross-correlation cost used with
// Eq. (image-reg)): box window of width w = 2R + 1 with zero padding and
// fixed divisor n = w^3;
//   cross = S_IJ - S_I S_J / n, var_I = S_II - S_I^2 / n, var_J likewise,
//   cc = cross^2 / (var_I var_J + eps),  L = -(1/N) sum_x cc(x).
// Gradient (section "Jacobian-Free Eulerian Descent" uses the Gateaux
// derivative): with A = 2 cross / den, B = -cc var_I / den,
// C = -(A S_I + 2 B S_J) / n (and B', C' mirrored for I),
//   dL/dJ(y) = -(1/N) sum_{x in win(y)} [A(x) I(y) + 2 B(x) J(y) + C(x)].
//
// Precision: images are quantised to b-bit fixed point (b from the window,
// see lncc_image_bits) and all window sums are exact int64 sums; the
// variance / covariance numerators n S_II - S_I^2 are formed exactly in
// 128-bit integers before rounding to float.  The adjoint window sums
// quantise A, B, C to 2^-(47 - ceil(log2 n)) of their maxima and are exact
// int64 sums too; the final I SA + 2 J SB + SC is combined in float-float.
#include "ops.h"
#include "validate.h"

namespace fa {

__host__ __device__ inline int log2_ceil_window(int window) {
    long long n = (long long)window * window * window;
    int lg = 0;
    while ((1ll << lg) < n) ++lg;
    return lg;
}

// ------------------------------------------------------------------ kernels

__global__ void k_absmax2(const float *__restrict__ I, const float *__restrict__ J, long long N,
                          WsHeader *h) {
    __shared__ float red[32];
    float a = 0.0f, b = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        float vi = fabsf(I[i]), vj = fabsf(J[i]);
        if (!(vi <= 3.4e38f) || !(vj <= 3.4e38f)) status_set(&h->status, ST_NONFINITE);
        a = fmaxf(a, vi);
        b = fmaxf(b, vj);
    }
    block_max_to(&h->absmax_bits[0], a, red);
    block_max_to(&h->absmax_bits[1], b, red);
}

__device__ __forceinline__ float image_scale(const WsHeader *h, int bits) {
    float amax = fmaxf(__uint_as_float(h->absmax_bits[0]), __uint_as_float(h->absmax_bits[1]));
    return pow2f(fixed_shift(amax, bits));
}

// x-window sums of q_I, q_J, q_I^2, q_J^2, q_I q_J -> p[5][N]
template <int R>
__global__ void __launch_bounds__(256) k_lncc_xpass(const float *__restrict__ I,
                                                    const float *__restrict__ J,
                                                    const WsHeader *__restrict__ h,
                                                    long long *__restrict__ p, int D, int H,
                                                    int W, int bits) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    if (x >= W || y >= H) return;
    long long N = (long long)D * H * W;
    long long row = ((long long)z * H + y) * W;
    float sc = image_scale(h, bits);
    long long sI = 0, sJ = 0, sII = 0, sJJ = 0, sIJ = 0;
#pragma unroll
    for (int k = -R; k <= R; ++k) {
        int xx = x + k;
        if (xx < 0 || xx >= W) continue;
        long long qi = quantize(__ldg(I + row + xx), sc);
        long long qj = quantize(__ldg(J + row + xx), sc);
        sI += qi;
        sJ += qj;
        sII += qi * qi;
        sJJ += qj * qj;
        sIJ += qi * qj;
    }
    long long i = row + x;
    p[i] = sI;
    p[N + i] = sJ;
    p[2 * N + i] = sII;
    p[3 * N + i] = sJJ;
    p[4 * N + i] = sIJ;
}

// window sums along y (AXIS 1) or z (AXIS 2) of C int64 channels (rows of P
// elements, P >= W)
template <int C, int AXIS>
__global__ void __launch_bounds__(256) k_box_axis(const long long *__restrict__ in,
                                                  long long *__restrict__ out, int D, int H,
                                                  int W, int P, int R) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    if (x >= W || y >= H) return;
    long long N = (long long)D * H * P;
    long long i = ((long long)z * H + y) * P + x;
    const int c0 = AXIS == 1 ? y : z;
    const int n = AXIS == 1 ? H : D;
    const long long stride = AXIS == 1 ? (long long)P : (long long)H * P;
    int lo = max(-R, -c0), hi = min(R, n - 1 - c0);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        long long s = 0;
        for (int k = lo; k <= hi; ++k) s += in[c * N + i + k * stride];
        out[c * N + i] = s;
    }
}

// cc, adjoint coefficients, loss accumulator and coefficient maxima
template <bool WANT_DI>
__global__ void __launch_bounds__(256) k_lncc_coef(const long long *__restrict__ S,
                                                   WsHeader *h, float *__restrict__ coef, int D,
                                                   int H, int W, int window, int bits,
                                                   float cc_eps) {
    __shared__ float redf[32];
    __shared__ unsigned long long redu[32];
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    bool live = x < W && y < H;
    long long N = (long long)D * H * W;
    long long i = ((long long)z * H + y) * W + x;
    const long long n = (long long)window * window * window;
    const float nf = (float)n, inv_nf = 1.0f / nf;
    float amax = fmaxf(__uint_as_float(h->absmax_bits[0]), __uint_as_float(h->absmax_bits[1]));
    int s = fixed_shift(amax, bits);
    float inv_s = pow2f(-s);
    // numerators are n^2 2^(2s) times the statistic: scale by 2^-s twice
    // (exact) and divide by n once (one rounding)
    float A = 0.f, B = 0.f, Cc = 0.f, Bp = 0.f, Cp = 0.f;
    unsigned long long qcc = 0;
    if (live) {
        long long sI = S[i], sJ = S[N + i], sII = S[2 * N + i], sJJ = S[3 * N + i],
                  sIJ = S[4 * N + i];
        float varI = diff_i128_to_float(n, sII, sI, sI) * inv_s * inv_s * inv_nf;
        float varJ = diff_i128_to_float(n, sJJ, sJ, sJ) * inv_s * inv_s * inv_nf;
        float cross = diff_i128_to_float(n, sIJ, sI, sJ) * inv_s * inv_s * inv_nf;
        float den = fmaf(varI, varJ, cc_eps);
        float rden = __frcp_rn(den);
        float cc = cross * cross * rden;
        A = 2.0f * cross * rden;
        B = -cc * varI * rden;
        float clo;
        lncc_c_ff(A, B, sI, sJ, inv_s, nf, inv_nf, Cc, clo);
        coef[i] = A;
        coef[N + i] = B;
        coef[2 * N + i] = Cc;
        coef[3 * N + i] = clo;
        if (WANT_DI) {
            Bp = -cc * varJ * rden;
            lncc_c_ff(A, Bp, sJ, sI, inv_s, nf, inv_nf, Cp, clo);
            coef[4 * N + i] = Bp;
            coef[5 * N + i] = Cp;
            coef[6 * N + i] = clo;
        }
        if (cc >= 0.0f && cc <= 2.0f) {
            qcc = (unsigned long long)quantize(cc, 4294967296.0f);  // cc in [0, 2]
        } else {
            status_set(&h->status, ST_NONFINITE);
        }
    }
    block_sum_to(&h->loss_acc, qcc, redu);
    block_max_to(&h->coef_max_bits[0], fabsf(A), redf);
    block_max_to(&h->coef_max_bits[1], fabsf(B), redf);
    block_max_to(&h->coef_max_bits[2], fabsf(Cc), redf);
    if (WANT_DI) {
        block_max_to(&h->coef_max_bits[3], fabsf(Bp), redf);
        block_max_to(&h->coef_max_bits[4], fabsf(Cp), redf);
    }
}

// x-window sums of the quantised adjoint coefficients.  Output channel c
// quantises coef[hi[c]] (+ coef[lo[c]] when lo[c] >= 0, the low half of a
// float-float coefficient) with the scale of coef_max_bits[mx[c]].
struct CoefSel {
    int hi[4], lo[4], mx[4];
};

template <int NC, int R>
__global__ void __launch_bounds__(256) k_coef_xpass(const float *__restrict__ coef,
                                                    const WsHeader *__restrict__ h,
                                                    long long *__restrict__ p, int D, int H,
                                                    int W, int cbits, CoefSel sel) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    if (x >= W || y >= H) return;
    long long N = (long long)D * H * W;
    long long row = ((long long)z * H + y) * W;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const float *src = coef + sel.hi[c] * N + row;
        const float *lo = sel.lo[c] >= 0 ? coef + sel.lo[c] * N + row : nullptr;
        float sc = pow2f(fixed_shift(__uint_as_float(h->coef_max_bits[sel.mx[c]]), cbits));
        long long acc = 0;
#pragma unroll
        for (int k = -R; k <= R; ++k) {
            int xx = x + k;
            if (xx >= 0 && xx < W) {
                acc += quantize(__ldg(src + xx), sc);
                if (lo) acc += quantize(__ldg(lo + xx), sc);
            }
        }
        p[c * N + row + x] = acc;
    }
}

// dL/dJ and/or dL/dI from the adjoint window sums; g = dL/dJ * grad.
// Channel order of S: SA, SB, SC, [SB', SC'] (the last two only if dI).
__global__ void __launch_bounds__(256) k_lncc_grad(const long long *__restrict__ S,
                                                   const float *__restrict__ I,
                                                   const float *__restrict__ J,
                                                   const float *__restrict__ grad,
                                                   const WsHeader *__restrict__ h,
                                                   float *__restrict__ dJ, float *__restrict__ dI,
                                                   float *__restrict__ g, int D, int H, int W,
                                                   int cbits, int nsum) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    if (x >= W || y >= H) return;
    long long N = (long long)D * H * W;
    long long i = ((long long)z * H + y) * W + x;
    float inv_n = 1.0f / (float)N;
    float Iv = I[i], Jv = J[i];
    // channel scales (exact powers of two)
    float uA = pow2f(-fixed_shift(__uint_as_float(h->coef_max_bits[0]), cbits));
    float ah, al;
    i64_to_ff(S[i], ah, al);
    ah *= uA;
    al *= uA;
    bool wantJ = dJ || g;
    if (wantJ) {
        float uB = pow2f(-fixed_shift(__uint_as_float(h->coef_max_bits[1]), cbits));
        float uC = pow2f(-fixed_shift(__uint_as_float(h->coef_max_bits[2]), cbits));
        float bh, bl, ch, cl, th, tl, rh, rl;
        i64_to_ff(S[N + i], bh, bl);
        i64_to_ff(S[2 * N + i], ch, cl);
        ff_mul_f(Iv, ah, al, rh, rl);                  // I SA
        ff_mul_f(2.0f * Jv, bh * uB, bl * uB, th, tl);  // 2 J SB
        ff_add(rh, rl, th, tl);
        ff_add(rh, rl, ch * uC, cl * uC);               // + SC
        float dj = -(rh + rl) * inv_n;
        if (dJ) dJ[i] = dj;
        if (g) {
            g[i] = dj * grad[i];
            g[N + i] = dj * grad[N + i];
            g[2 * N + i] = dj * grad[2 * N + i];
        }
    }
    if (dI) {
        int o = wantJ ? 3 : 1;  // SB', SC' follow SB, SC when both are present
        float uB = pow2f(-fixed_shift(__uint_as_float(h->coef_max_bits[3]), cbits));
        float uC = pow2f(-fixed_shift(__uint_as_float(h->coef_max_bits[4]), cbits));
        float bh, bl, ch, cl, th, tl, rh, rl;
        i64_to_ff(S[o * N + i], bh, bl);
        i64_to_ff(S[(o + 1) * N + i], ch, cl);
        ff_mul_f(Jv, ah, al, rh, rl);                  // J SA
        ff_mul_f(2.0f * Iv, bh * uB, bl * uB, th, tl);  // 2 I SB'
        ff_add(rh, rl, th, tl);
        ff_add(rh, rl, ch * uC, cl * uC);               // + SC'
        dI[i] = -(rh + rl) * inv_n;
    }
    (void)nsum;
}

__global__ void k_loss_finalize(WsHeader *h, long long N, float sign, float *out) {
    unsigned long long a = h->loss_acc;
    // a < 2^63: split so both halves convert exactly
    float hi = __ull2float_rn(a >> 32), lo = __ull2float_rn(a & 0xffffffffull);
    float mean = (hi + lo * 2.3283064365386963e-10f) / (float)N;
    float L = sign * mean;
    h->loss = L;
    if (out) *out = L;
}

// MSE: per-block partial sums of (J - I)^2 in block order for a fixed-order
// final sum.
__global__ void __launch_bounds__(256) k_mse(const float *__restrict__ I,
                                             const float *__restrict__ J,
                                             const float *__restrict__ grad, float *dJ, float *dI,
                                             float *g, float *partials, int D, int H, int W) {
    __shared__ float red[8];
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    long long N = (long long)D * H * W;
    float e2 = 0.0f;
    if (x < W && y < H) {
        long long i = ((long long)z * H + y) * W + x;
        float e = J[i] - I[i];
        e2 = e * e;
        float dj = 2.0f * e / (float)N;
        if (dJ) dJ[i] = dj;
        if (dI) dI[i] = -dj;
        if (g) {
            g[i] = dj * grad[i];
            g[N + i] = dj * grad[N + i];
            g[2 * N + i] = dj * grad[2 * N + i];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    int lane = threadIdx.x + 32 * threadIdx.y;
    if ((lane & 31) == 0) red[lane >> 5] = e2;
    __syncthreads();
    if (lane == 0) {
        float s = 0.0f;
        for (int k = 0; k < 8; ++k) s += red[k];
        long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[b] = s;
    }
}

__global__ void k_partials_finalize(const float *partials, long long nb, long long N, WsHeader *h,
                                    float *out) {
    __shared__ float red[256];
    float s = 0.0f;
    for (long long k = threadIdx.x; k < nb; k += blockDim.x) s += partials[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        float L = red[0] / (float)N;
        if (!(L <= 3.4e38f)) status_set(&h->status, ST_NONFINITE);
        h->loss = L;
        if (out) *out = L;
    }
}

// Window statistics of the fixed image alone (constant during a level): the
// exact sum S_I and the rounded variance var_I, both as the LNCC kernels
// compute them.  Buffers have rows of P (>= W) elements.
template <int R>
__global__ void __launch_bounds__(256) k_fixed_xpass(const float *__restrict__ I,
                                                     const WsHeader *__restrict__ h,
                                                     long long *__restrict__ p, int D, int H,
                                                     int W, int P, int bits) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    if (x >= W || y >= H) return;
    long long N = (long long)D * H * P;
    long long row = ((long long)z * H + y) * P;
    float sc = image_scale(h, bits);
    long long sI = 0, sII = 0;
#pragma unroll
    for (int k = -R; k <= R; ++k) {
        int xx = x + k;
        if (xx < 0 || xx >= W) continue;
        long long qi = quantize(__ldg(I + row + xx), sc);
        sI += qi;
        sII += qi * qi;
    }
    p[row + x] = sI;
    p[N + row + x] = sII;
}

__global__ void __launch_bounds__(256) k_fixed_finalize(const long long *__restrict__ S,
                                                        const WsHeader *__restrict__ h,
                                                        long long *__restrict__ sI_out,
                                                        float *__restrict__ varI_out, int D,
                                                        int H, int W, int P, int window,
                                                        int bits) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    if (x >= W || y >= H) return;
    long long N = (long long)D * H * P;
    long long i = ((long long)z * H + y) * P + x;
    const long long n = (long long)window * window * window;
    const float inv_nf = 1.0f / (float)n;
    float amax = fmaxf(__uint_as_float(h->absmax_bits[0]), __uint_as_float(h->absmax_bits[1]));
    float inv_s = pow2f(-fixed_shift(amax, bits));
    long long sI = S[i], sII = S[N + i];
    sI_out[i] = sI;
    varI_out[i] = diff_i128_to_float(n, sII, sI, sI) * inv_s * inv_s * inv_nf;
}

// ---------------------------------------------------------------- launchers

LnccBuffers lncc_carve(WsCarver &c, long long N) {
    LnccBuffers b;
    b.p0 = c.take<long long>(5 * N);
    b.p1 = c.take<long long>(5 * N);
    b.coef = c.take<float>(7 * N);
    return b;
}

size_t lncc_plain_bytes(long long N) {
    WsCarver c(nullptr, ~size_t(0));
    c.take<WsHeader>(1);
    lncc_carve(c, N);
    return c.off;
}

cudaError_t launch_header_reset(WsHeader *h, cudaStream_t s) {
    return cudaMemsetAsync(h, 0, sizeof(WsHeader), s);
}

cudaError_t launch_absmax2(const float *I, const float *J, long long N, WsHeader *h,
                           cudaStream_t s) {
    long long blocks = (N + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_absmax2<<<(unsigned)blocks, 256, 0, s>>>(I, J, N, h); note_launch();
    return cudaGetLastError();
}

template <int R>
static void xpass_img(const float *I, const float *J, WsHeader *h, long long *p, Dims d, int bits,
                      cudaStream_t s) {
    VoxGrid g(d.D, d.H, d.W);
    k_lncc_xpass<R><<<g.grid, g.block, 0, s>>>(I, J, h, p, d.D, d.H, d.W, bits); note_launch();
}

template <int NC, int R>
static void xpass_coef(const float *coef, const WsHeader *h, long long *p, Dims d, int cbits,
                       CoefSel sel, cudaStream_t s) {
    VoxGrid g(d.D, d.H, d.W);
    k_coef_xpass<NC, R><<<g.grid, g.block, 0, s>>>(coef, h, p, d.D, d.H, d.W, cbits, sel); note_launch();
}

template <int C>
static void box_yz(long long *a, long long *b, Dims d, int R, cudaStream_t s) {
    VoxGrid g(d.D, d.H, d.W);
    k_box_axis<C, 1><<<g.grid, g.block, 0, s>>>(a, b, d.D, d.H, d.W, d.pitch(), R); note_launch();
    k_box_axis<C, 2><<<g.grid, g.block, 0, s>>>(b, a, d.D, d.H, d.W, d.pitch(), R); note_launch();
}

#define FA_DISPATCH_R(R, ...)                          \
    switch (R) {                                       \
        case 0: { constexpr int RR = 0; __VA_ARGS__; } break; \
        case 1: { constexpr int RR = 1; __VA_ARGS__; } break; \
        case 2: { constexpr int RR = 2; __VA_ARGS__; } break; \
        case 3: { constexpr int RR = 3; __VA_ARGS__; } break; \
        case 4: { constexpr int RR = 4; __VA_ARGS__; } break; \
        case 5: { constexpr int RR = 5; __VA_ARGS__; } break; \
        case 6: { constexpr int RR = 6; __VA_ARGS__; } break; \
        case 7: { constexpr int RR = 7; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;         \
    }

cudaError_t launch_lncc_forward(const float *I, const float *J, Dims d, int window, float cc_eps,
                                bool want_dI, WsHeader *h, LnccBuffers b, cudaStream_t s) {
    int R = window / 2;
    int bits = lncc_image_bits(window);
    FA_DISPATCH_R(R, xpass_img<RR>(I, J, h, b.p0, d, bits, s));
    box_yz<5>(b.p0, b.p1, d, R, s);
    VoxGrid g(d.D, d.H, d.W);
    if (want_dI) {
        k_lncc_coef<true><<<g.grid, g.block, 0, s>>>(b.p0, h, b.coef, d.D, d.H, d.W, window, bits,
                                                     cc_eps); note_launch();
    }
    else {
        k_lncc_coef<false><<<g.grid, g.block, 0, s>>>(b.p0, h, b.coef, d.D, d.H, d.W, window,
                                                      bits, cc_eps); note_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_lncc_backward(const float *I, const float *J, const float *grad, Dims d,
                                 int window, WsHeader *h, LnccBuffers b, float *dJ, float *dI,
                                 float *g, cudaStream_t s) {
    int R = window / 2;
    int cbits = lncc_coef_bits(window);
    bool wantJ = dJ || g;
    // coefficient channels: 0 A, 1 B, 2/3 C (hi/lo), 4 B', 5/6 C' (hi/lo);
    // maxima: 0 A, 1 B, 2 C, 3 B', 4 C'
    const CoefSel cA{{0, 0, 0, 0}, {-1, -1, -1, -1}, {0, 0, 0, 0}};
    CoefSel sel = cA;
    int nc;
    if (wantJ && dI) {
        sel = CoefSel{{0, 1, 2, 4}, {-1, -1, 3, -1}, {0, 1, 2, 3}};  // SA, SB, SC, SB'
        nc = 5;
    } else if (wantJ) {
        sel = CoefSel{{0, 1, 2, 0}, {-1, -1, 3, -1}, {0, 1, 2, 0}};
        nc = 3;
    } else {
        sel = CoefSel{{0, 4, 5, 0}, {-1, -1, 6, -1}, {0, 3, 4, 0}};  // SA, SB', SC'
        nc = 3;
    }
    if (nc == 3) {
        FA_DISPATCH_R(R, (xpass_coef<3, RR>(b.coef, h, b.p0, d, cbits, sel, s)));
        box_yz<3>(b.p0, b.p1, d, R, s);
    } else {
        FA_DISPATCH_R(R, (xpass_coef<4, RR>(b.coef, h, b.p0, d, cbits, sel, s)));
        long long N = d.N();
        const CoefSel sc5{{5, 0, 0, 0}, {6, -1, -1, -1}, {4, 0, 0, 0}};  // SC'
        FA_DISPATCH_R(R, (xpass_coef<1, RR>(b.coef, h, b.p0 + 4 * N, d, cbits, sc5, s)));
        box_yz<5>(b.p0, b.p1, d, R, s);
    }
    VoxGrid gg(d.D, d.H, d.W);
    k_lncc_grad<<<gg.grid, gg.block, 0, s>>>(b.p0, I, J, grad, h, dJ, dI, g, d.D, d.H, d.W, cbits,
                                            nc); note_launch();
    return cudaGetLastError();
}

long long mse_partials_count(Dims d) {
    VoxGrid gg(d.D, d.H, d.W);
    return (long long)gg.grid.x * gg.grid.y * gg.grid.z;
}

cudaError_t launch_mse(const float *I, const float *J, const float *grad, Dims d, WsHeader *h,
                       float *partials, float *dJ, float *dI, float *g, cudaStream_t s) {
    VoxGrid gg(d.D, d.H, d.W);
    long long nb = mse_partials_count(d);
    k_mse<<<gg.grid, gg.block, 0, s>>>(I, J, grad, dJ, dI, g, partials, d.D, d.H, d.W); note_launch();
    k_partials_finalize<<<1, 256, 0, s>>>(partials, nb, d.N(), h, nullptr); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_fixed_stats(const float *I, Dims d, int window, const WsHeader *h,
                               long long *p0, long long *p1, long long *sI, float *varI,
                               cudaStream_t s) {
    int R = window / 2;
    int bits = lncc_image_bits(window);
    VoxGrid g(d.D, d.H, d.W);
    FA_DISPATCH_R(R, (k_fixed_xpass<RR><<<g.grid, g.block, 0, s>>>(I, h, p0, d.D, d.H, d.W,
                                                                   d.pitch(), bits)));
    note_launch();
    k_box_axis<2, 1><<<g.grid, g.block, 0, s>>>(p0, p1, d.D, d.H, d.W, d.pitch(), R); note_launch();
    k_box_axis<2, 2><<<g.grid, g.block, 0, s>>>(p1, p0, d.D, d.H, d.W, d.pitch(), R); note_launch();
    k_fixed_finalize<<<g.grid, g.block, 0, s>>>(p0, h, sI, varI, d.D, d.H, d.W, d.pitch(), window,
                                                bits);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_loss_finalize(WsHeader *h, long long N, float sign, float *loss_out,
                                 cudaStream_t s) {
    k_loss_finalize<<<1, 1, 0, s>>>(h, N, sign, loss_out); note_launch();
    return cudaGetLastError();
}

}  // namespace fa

// ---------------------------------------------------------------- C ABI

extern "C" size_t fa_lncc_workspace_size(int32_t D, int32_t H, int32_t W) {
    if (D < 1 || H < 1 || W < 1) return 0;
    return fa::lncc_plain_bytes((long long)D * H * W);
}

static fa_status loss_args(const fa_vol *fixed, const fa_vol *warped, fa_vol *dJ, fa_vol *dI,
                           void *ws, size_t ws_bytes, const char *who) {
    using namespace fa;
    FA_TRY(check_vol(fixed, "fixed", 1));
    FA_TRY(check_vol(warped, "warped", 1));
    FA_TRY(same_grid(fixed, warped, "fixed", "warped"));
    if (dJ) {
        FA_TRY(check_vol(dJ, "dL_dwarped", 1));
        FA_TRY(same_grid(fixed, dJ, "fixed", "dL_dwarped"));
    }
    if (dI) {
        FA_TRY(check_vol(dI, "dL_dfixed", 1));
        FA_TRY(same_grid(fixed, dI, "fixed", "dL_dfixed"));
    }
    FA_TRY(check_ws(ws, ws_bytes, fa_lncc_workspace_size(fixed->D, fixed->H, fixed->W), who));
    return FA_OK;
}

extern "C" fa_status fa_lncc_fwd_bwd(const fa_vol *fixed, const fa_vol *warped, int32_t window,
                                     float cc_eps, float *loss_dev, fa_vol *dL_dwarped_opt,
                                     fa_vol *dL_dfixed_opt, void *ws, size_t ws_bytes,
                                     void *stream) {
    using namespace fa;
    clear_error();
    if (window < 1 || window > 15 || (window % 2) == 0) {
        set_error("fa_lncc_fwd_bwd: window must be odd and in 1..15 (got %d)", (int)window);
        return FA_ERR_INVALID;
    }
    if (!(cc_eps >= 0.0f) || !(cc_eps < 3.0e38f)) {
        set_error("fa_lncc_fwd_bwd: cc_eps must be finite and >= 0");
        return FA_ERR_INVALID;
    }
    FA_TRY(loss_args(fixed, warped, dL_dwarped_opt, dL_dfixed_opt, ws, ws_bytes,
                     "fa_lncc_fwd_bwd"));
    cudaStream_t s = (cudaStream_t)stream;
    Dims d{fixed->D, fixed->H, fixed->W};
    long long N = d.N();
    WsCarver c(ws, ws_bytes);
    WsHeader *h = c.take<WsHeader>(1);
    LnccBuffers b = lncc_carve(c, N);
    const float *I = (const float *)fixed->data, *J = (const float *)warped->data;
    FA_CUDA_TRY(launch_header_reset(h, s));
    FA_CUDA_TRY(launch_absmax2(I, J, N, h, s));
    FA_CUDA_TRY(launch_lncc_forward(I, J, d, window, cc_eps, dL_dfixed_opt != nullptr, h, b, s));
    FA_CUDA_TRY(launch_loss_finalize(h, N, -1.0f, loss_dev, s));
    if (dL_dwarped_opt || dL_dfixed_opt)
        FA_CUDA_TRY(launch_lncc_backward(
            I, J, nullptr, d, window, h, b, dL_dwarped_opt ? (float *)dL_dwarped_opt->data : nullptr,
            dL_dfixed_opt ? (float *)dL_dfixed_opt->data : nullptr, nullptr, s));
    return FA_OK;
}

extern "C" fa_status fa_mse_fwd_bwd(const fa_vol *fixed, const fa_vol *warped, float *loss_dev,
                                    fa_vol *dL_dwarped_opt, fa_vol *dL_dfixed_opt, void *ws,
                                    size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(loss_args(fixed, warped, dL_dwarped_opt, dL_dfixed_opt, ws, ws_bytes,
                     "fa_mse_fwd_bwd"));
    cudaStream_t s = (cudaStream_t)stream;
    Dims d{fixed->D, fixed->H, fixed->W};
    WsCarver c(ws, ws_bytes);
    WsHeader *h = c.take<WsHeader>(1);
    float *partials = c.take<float>(mse_partials_count(d));
    FA_CUDA_TRY(launch_header_reset(h, s));
    FA_CUDA_TRY(launch_mse((const float *)fixed->data, (const float *)warped->data, nullptr, d, h,
                           partials,
                           dL_dwarped_opt ? (float *)dL_dwarped_opt->data : nullptr,
                           dL_dfixed_opt ? (float *)dL_dfixed_opt->data : nullptr, nullptr, s));
    if (loss_dev)
        FA_CUDA_TRY(cudaMemcpyAsync(loss_dev, &h->loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    return FA_OK;
}
