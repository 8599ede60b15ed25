// Mutual-information loss (named with LNCC among the costs of the problem
// statement, section "Deformable Image Registration"; its bin count is one of
// the hyper-parameters of the hyper-parameter study).  Parzen-window estimate
// with the cubic B-spline beta3 on B bins for both images: an intensity v of
// an image with range [lo, hi] sits at bin coordinate
//   xi = 1 + (v - lo) (B - 3) / (hi - lo), clamped to [1, B - 2],
// where the weights beta3(xi - k) of the bins k = 0..B-1 sum to one.
//   P(a,b) = (1/N) sum_x beta3(xi_f(x) - a) beta3(xi_m(x) - b),
//   L = -MI = -sum P log(P / (p_f p_m)),
//   dL/dJ(x) = -(1/N) (B - 3) / (hi_m - lo_m)
//              sum_{a,b} log(P / (p_f p_m)) beta3(xi_f - a) beta3'(xi_m - b).
// The joint histogram is accumulated in 2^-32 fixed point with integer
// atomics, so it does not depend on thread order.
#include "ops.h"
#include "validate.h"

namespace fa {

namespace {

constexpr int kMiBits = 32;  // fixed-point scale of the histogram terms (< 2^31 each)

__device__ __forceinline__ unsigned fkey(float f) {  // order-preserving float key
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fval(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

struct MiMap {
    float lo, s;  // xi = 1 + (v - lo) s
    int B;
    __device__ float coord(float v) const {
        const float xi = fmaf(v - lo, s, 1.0f);
        return fminf(fmaxf(xi, 1.0f), (float)(B - 2));
    }
};

__device__ __forceinline__ MiMap mi_map(const unsigned *keys, int k, int B) {
    MiMap m;
    m.lo = fval(keys[2 * k]);
    const float hi = fval(keys[2 * k + 1]);
    m.s = hi > m.lo ? (float)(B - 3) / (hi - m.lo) : 0.0f;
    m.B = B;
    return m;
}

// cubic B-spline weights of bins floor(xi) - 1 .. floor(xi) + 2, t = xi - floor(xi)
__device__ __forceinline__ void bspline_w(float t, float w[4]) {
    const float t2 = t * t, t3 = t2 * t, r = 1.0f - t;
    w[0] = r * r * r * (1.0f / 6.0f);
    w[1] = fmaf(0.5f, t3, fmaf(-1.0f, t2, 2.0f / 3.0f));
    w[2] = fmaf(-0.5f, t3, fmaf(0.5f, t2, fmaf(0.5f, t, 1.0f / 6.0f)));
    w[3] = t3 * (1.0f / 6.0f);
}
// their derivatives with respect to xi
__device__ __forceinline__ void bspline_dw(float t, float w[4]) {
    const float t2 = t * t, r = 1.0f - t;
    w[0] = -0.5f * r * r;
    w[1] = fmaf(1.5f, t2, -2.0f * t);
    w[2] = fmaf(-1.5f, t2, t + 0.5f);
    w[3] = 0.5f * t2;
}

__global__ void k_mi_range_init(unsigned *keys) {
    keys[0] = 0xffffffffu;   // lo_f: min over the fixed image
    keys[1] = 0u;            // hi_f
    keys[2] = fkey(0.0f);    // lo_m, hi_m: the moving image with 0 included
    keys[3] = fkey(0.0f);
}

__global__ void k_mi_range_set(const float *range, unsigned *keys) {
    if (threadIdx.x < 4) keys[threadIdx.x] = fkey(range[threadIdx.x]);
}

__global__ void __launch_bounds__(256) k_mi_range(const float *__restrict__ If,
                                                  const float *__restrict__ Im, long long N,
                                                  unsigned *keys) {
    unsigned k[4] = {0xffffffffu, 0u, 0xffffffffu, 0u};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const float a = If[i], b = Im[i];
        if (fabsf(a) <= 3.4e38f) {
            k[0] = min(k[0], fkey(a));
            k[1] = max(k[1], fkey(a));
        }
        if (fabsf(b) <= 3.4e38f) {
            k[2] = min(k[2], fkey(b));
            k[3] = max(k[3], fkey(b));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        k[0] = min(k[0], __shfl_xor_sync(0xffffffffu, k[0], o));
        k[1] = max(k[1], __shfl_xor_sync(0xffffffffu, k[1], o));
        k[2] = min(k[2], __shfl_xor_sync(0xffffffffu, k[2], o));
        k[3] = max(k[3], __shfl_xor_sync(0xffffffffu, k[3], o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(keys + 0, k[0]);
        atomicMax(keys + 1, k[1]);
        atomicMin(keys + 2, k[2]);
        atomicMax(keys + 3, k[3]);
    }
}

// Joint histogram.  Each weight product is quantised to 2^-32 (q < 2^31) and
// added as two halves, q mod 2^16 and q / 2^16, with 32-bit shared atomics
// into one of NH private copies (NH = 4 when they fit, so the block's warps
// never share one; 1 otherwise).  A copy takes at most 4 warps x 32 lanes x
// kHistWarpIters voxels, so each half-sum stays below 2^13 * 2^16 = 2^29;
// the block recombines the halves exactly in 64 bits and adds its non-zero
// bins to the global histogram.
constexpr int kHistThreads = 128, kHistWarpIters = 64;

__global__ void __launch_bounds__(kHistThreads) k_mi_hist(const float *__restrict__ I,
                                                          const float *__restrict__ J, long long N,
                                                          int B, int NH,
                                                          const unsigned *__restrict__ keys,
                                                          unsigned long long *ghist, WsHeader *h) {
    extern __shared__ unsigned shu[];  // [NH][2][B*B]: low and high halves
    const int nb = B * B, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < 2 * nb * NH; k += blockDim.x) shu[k] = 0u;
    __syncthreads();
    unsigned *lo_h = shu + (warp % NH) * 2 * nb, *hi_h = lo_h + nb;
    const MiMap mf = mi_map(keys, 0, B), mm = mi_map(keys, 1, B);
    const float scale = pow2f(kMiBits);
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const float a = I[i], b = J[i];
        if (!(fabsf(a) <= 3.4e38f && fabsf(b) <= 3.4e38f)) {
            bad = true;
            continue;
        }
        const float xf = mf.coord(a), xm = mm.coord(b);
        const float ff = floorf(xf), fm = floorf(xm);
        float wf[4], wm[4];
        bspline_w(xf - ff, wf);
        bspline_w(xm - fm, wm);
        const int a0 = (int)ff - 1, b0 = (int)fm - 1;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            if (a0 + p >= B) continue;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const unsigned v = (unsigned)quantize(wf[p] * wm[q], scale);
                if (v == 0u || b0 + q >= B) continue;
                const int k = (a0 + p) * B + b0 + q;
                atomicAdd(lo_h + k, v & 0xffffu);
                if (v >> 16) atomicAdd(hi_h + k, v >> 16);
            }
        }
    }
    if (bad) status_set(&h->status, ST_NONFINITE);
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        unsigned long long t = 0ull;
        for (int c = 0; c < NH; ++c)
            t += (unsigned long long)shu[c * 2 * nb + k] +
                 ((unsigned long long)shu[c * 2 * nb + nb + k] << 16);
        if (t) atomicAdd(ghist + k, t);
    }
}

// P, marginals, MI and the table log(P / (p_f p_m)), in FP32.  The
// marginals are exact integer sums of the fixed-point histogram, so every
// probability is one rounding of an exact count; the ratio adds two
// roundings and logf one more.  MI = sum P log(...) is accumulated as a
// float-float pair per thread (exact products by fmaf, two-sum additions)
// and the pairs are combined in a fixed tree order, so the loss carries
// about FP32's unit roundoff and does not depend on scheduling.
__global__ void __launch_bounds__(1024) k_mi_table(const unsigned long long *__restrict__ ghist,
                                                   int B, long long N, float *T, WsHeader *h,
                                                   float *loss_out) {
    extern __shared__ float shf[];
    float *P = shf, *pf = shf + B * B, *pm = pf + B, *rh = pm + B, *rl = rh + blockDim.x;
    const int nb = B * B, tid = threadIdx.x;
    const float Nf = (float)N, unit = pow2f(-kMiBits);
    for (int k = tid; k < nb; k += blockDim.x)
        P[k] = __fdiv_rn(u64_to_float_rn(ghist[k]) * unit, Nf);
    if (tid < B) {
        unsigned long long s = 0ull;
        for (int b = 0; b < B; ++b) s += ghist[tid * B + b];
        pf[tid] = __fdiv_rn(u64_to_float_rn(s) * unit, Nf);
    } else if (tid < 2 * B) {
        unsigned long long s = 0ull;
        for (int a = 0; a < B; ++a) s += ghist[a * B + tid - B];
        pm[tid - B] = __fdiv_rn(u64_to_float_rn(s) * unit, Nf);
    }
    __syncthreads();
    float hi = 0.0f, lo = 0.0f;
    for (int k = tid; k < nb; k += blockDim.x) {
        const float q = P[k];
        float tv = 0.0f;
        if (q > 0.0f) {
            tv = logf(__fdiv_rn(q, pf[k / B] * pm[k % B]));
            const float ph = q * tv, pl = fmaf(q, tv, -ph);
            ff_add(hi, lo, ph, pl);
        }
        T[k] = tv;
    }
    rh[tid] = hi;
    rl[tid] = lo;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) {
            float a = rh[tid], b = rl[tid];
            ff_add(a, b, rh[tid + o], rl[tid + o]);
            rh[tid] = a;
            rl[tid] = b;
        }
        __syncthreads();
    }
    if (tid == 0) {
        const float L = -(rh[0] + rl[0]);
        h->loss = L;
        if (loss_out) *loss_out = L;
    }
}

__global__ void __launch_bounds__(256) k_mi_grad(const float *__restrict__ I,
                                                 const float *__restrict__ J,
                                                 const float *__restrict__ grad, long long N,
                                                 int B, const unsigned *__restrict__ keys,
                                                 const float *__restrict__ Tg, float *dJ,
                                                 float *g) {
    extern __shared__ float T[];
    for (int k = threadIdx.x; k < B * B; k += blockDim.x) T[k] = Tg[k];
    __syncthreads();
    const MiMap mf = mi_map(keys, 0, B), mm = mi_map(keys, 1, B);
    const float c = -mm.s / (float)N;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const float xf = mf.coord(I[i]), xm = mm.coord(J[i]);
        const float ff = floorf(xf), fm = floorf(xm);
        float wf[4], dm[4];
        bspline_w(xf - ff, wf);
        bspline_dw(xm - fm, dm);
        const int a0 = (int)ff - 1, b0 = (int)fm - 1;
        float acc = 0.0f;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            if (a0 + p >= B) continue;
            float r = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (b0 + q < B) r = fmaf(T[(a0 + p) * B + b0 + q], dm[q], r);
            acc = fmaf(wf[p], r, acc);
        }
        const float dj = c * acc;
        if (dJ) dJ[i] = dj;
        if (g) {
            g[i] = dj * grad[i];
            g[N + i] = dj * grad[N + i];
            g[2 * N + i] = dj * grad[2 * N + i];
        }
    }
}

unsigned grid_blocks(long long N) {
    long long b = (N + 255) / 256;
    return (unsigned)(b > 152 * 4 ? 152 * 4 : (b < 1 ? 1 : b));
}

}  // namespace

MiBuffers mi_carve(WsCarver &c, int bins) {
    MiBuffers b;
    b.hist = c.take<unsigned long long>((size_t)bins * bins);
    b.T = c.take<float>((size_t)bins * bins);
    b.range = c.take<unsigned>(4);
    return b;
}

cudaError_t launch_mi_range(const float *If, const float *Im, long long N, MiBuffers b,
                            cudaStream_t s) {
    k_mi_range_init<<<1, 1, 0, s>>>(b.range);
    note_launch();
    k_mi_range<<<grid_blocks(N), 256, 0, s>>>(If, Im, N, b.range);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_mi_range_set(const float *range4, MiBuffers b, cudaStream_t s) {
    k_mi_range_set<<<1, 32, 0, s>>>(range4, b.range);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_mi(const float *I, const float *J, const float *grad, Dims d, int bins,
                      WsHeader *h, MiBuffers b, float *loss_out, float *dJ, float *g,
                      cudaStream_t s) {
    const long long N = d.N();
    const int nb = bins * bins;
    cudaError_t e = cudaMemsetAsync(b.hist, 0, sizeof(unsigned long long) * nb, s);
    if (e != cudaSuccess) return e;
    // four private copies when they fit in 48 KB (bins <= 38), else one
    const int nh = 2 * nb * 4 * (int)sizeof(unsigned) <= 49152 ? 4 : 1;
    const size_t hist_smem = sizeof(unsigned) * 2 * nb * nh;
    long long hb = (N + (long long)kHistThreads * kHistWarpIters - 1) /
                   ((long long)kHistThreads * kHistWarpIters);
    hb = hb < 152 * 4 ? 152 * 4 : hb;
    k_mi_hist<<<(unsigned)hb, kHistThreads, hist_smem, s>>>(I, J, N, bins, nh, b.range, b.hist,
                                                           h);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t tab_smem = sizeof(float) * (nb + 2 * bins + 2 * 1024);
    k_mi_table<<<1, 1024, tab_smem, s>>>(b.hist, bins, N, b.T, h, loss_out);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (dJ || g) {
        k_mi_grad<<<grid_blocks(N), 256, sizeof(float) * nb, s>>>(I, J, grad, N, bins, b.range,
                                                                   b.T, dJ, g);
        note_launch();
    }
    return cudaGetLastError();
}

}  // namespace fa

extern "C" size_t fa_mi_workspace_size(int32_t bins) {
    fa::clear_error();
    if (bins < fa::kMiMinBins || bins > fa::kMiMaxBins) return 0;
    fa::WsCarver c(nullptr, ~size_t(0));
    c.take<fa::WsHeader>(1);
    fa::mi_carve(c, bins);
    return c.off;
}

extern "C" fa_status fa_mi_fwd_bwd(const fa_vol *fixed, const fa_vol *warped, int32_t bins,
                                   const float *range_dev_opt, float *loss_dev,
                                   fa_vol *dL_dwarped_opt, void *ws, size_t ws_bytes,
                                   void *stream) {
    using namespace fa;
    clear_error();
    if (bins < kMiMinBins || bins > kMiMaxBins) {
        set_error("fa_mi_fwd_bwd: bins must be in %d..%d (got %d)", kMiMinBins, kMiMaxBins,
                  (int)bins);
        return FA_ERR_INVALID;
    }
    FA_TRY(check_vol(fixed, "fixed", 1));
    FA_TRY(check_vol(warped, "warped", 1));
    FA_TRY(same_grid(fixed, warped, "fixed", "warped"));
    if (dL_dwarped_opt) {
        FA_TRY(check_vol(dL_dwarped_opt, "dL_dwarped", 1));
        FA_TRY(same_grid(fixed, dL_dwarped_opt, "fixed", "dL_dwarped"));
    }
    FA_TRY(check_ws(ws, ws_bytes, fa_mi_workspace_size(bins), "fa_mi_fwd_bwd"));
    WsCarver c(ws, ws_bytes);
    WsHeader *h = c.take<WsHeader>(1);
    MiBuffers b = mi_carve(c, bins);
    cudaStream_t s = (cudaStream_t)stream;
    const Dims d{fixed->D, fixed->H, fixed->W};
    const float *I = (const float *)fixed->data, *J = (const float *)warped->data;
    FA_CUDA_TRY(launch_header_reset(h, s));
    if (range_dev_opt)
        FA_CUDA_TRY(launch_mi_range_set(range_dev_opt, b, s));
    else
        FA_CUDA_TRY(launch_mi_range(I, J, d.N(), b, s));
    FA_CUDA_TRY(launch_mi(I, J, nullptr, d, bins, h, b, loss_dev,
                          dL_dwarped_opt ? (float *)dL_dwarped_opt->data : nullptr, nullptr, s));
    return FA_OK;
}
