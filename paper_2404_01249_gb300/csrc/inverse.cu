// Post-hoc inverse of a displacement (section "Alternative formulations for
// Eulerian differential": phi^-1 is found after the registration by
// minimising |psi(phi(x)) - x|^2 + |phi(psi(x)) - x|^2 over a multi-scale
// schedule like the image matching objective).  With phi = id + u and
// psi = id + w:
//   E(w) = (1/N) sum_x |A(x)|^2 + |B(x)|^2,
//   A(x) = u(x) + w(x + u(x)),   B(x) = w(x) + u(x + w(x)).
// Its Gateaux derivative: the A term scatters 2 A(x) / N to the trilinear
// corners of x + u(x) (accumulated in 2^-40-relative fixed point with
// integer atomics: order-independent); the B term gives
// 2 (I + grad u(x + w(x)))^T B(x) / N with the interpolant's derivative.
// The descent is Algorithm 1's: Gaussian(sigma_grad), Adam, step scaling,
// compose, Gaussian(sigma_warp), with the per-op kernels.
#include "ops.h"
#include "validate.h"

namespace fa {

namespace {

constexpr int kInvBits = 40;
constexpr int kSlotA = 7;  // header slot of max |A|
constexpr int kEnergyBlocks = 152 * 4;

struct InverseWs {
    WsHeader *h;
    Dims lvl[8];
    float *ul, *w[2], *m[2], *v[2], *A, *g, *dir, *t1, *t2, *partials;
    long long *acc;
};

void inverse_carve(WsCarver &c, Dims full, const fa_params *p, InverseWs *q) {
    long long n = 0;
    q->h = c.take<WsHeader>(1);
    for (int l = 0; l < p->n_levels; ++l) {
        const int s = p->scales[l];
        q->lvl[l] = Dims{level_size(full.D, s), level_size(full.H, s), level_size(full.W, s)};
        n = q->lvl[l].N() > n ? q->lvl[l].N() : n;
    }
    q->ul = c.take<float>(3 * n);
    for (int k = 0; k < 2; ++k) {
        q->w[k] = c.take<float>(3 * n);
        q->m[k] = c.take<float>(3 * n);
        q->v[k] = c.take<float>(3 * n);
    }
    q->A = c.take<float>(3 * n);
    q->g = c.take<float>(3 * n);
    q->dir = c.take<float>(3 * n);
    q->t1 = c.take<float>(3 * n);
    q->t2 = c.take<float>(3 * n);
    q->partials = c.take<float>(kEnergyBlocks);
    q->acc = c.take<long long>(3 * n);
}

// A (stored), the B-term gradient (written to g), max |A| (header), and
// optionally the energy terms |A|^2 + |B|^2 (block partials).
__global__ void __launch_bounds__(256) k_inverse_terms(const float *__restrict__ u,
                                                       const float *__restrict__ w,
                                                       float *__restrict__ Aout,
                                                       float *__restrict__ g, WsHeader *h,
                                                       float *__restrict__ energy_partials,
                                                       int D, int H, int W) {
    __shared__ float red[32];
    const long long N = (long long)D * H * W, HW = (long long)H * W;
    const float inv_n = 1.0f / (float)N;
    float amax = 0.0f, esum = 0.0f;
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(i / HW), r = (int)(i - (long long)z * HW), y = r / W, x = r - y * W;
        const float uz = u[i], uy = u[N + i], ux = u[2 * N + i];
        const float wz = w[i], wy = w[N + i], wx = w[2 * N + i];
        float A[3], B[3], G[3][3], gz, gy, gx;
        A[0] = uz + tri_sample<false>(w, D, H, W, z, y, x, uz, uy, ux, gz, gy, gx);
        A[1] = uy + tri_sample<false>(w + N, D, H, W, z, y, x, uz, uy, ux, gz, gy, gx);
        A[2] = ux + tri_sample<false>(w + 2 * N, D, H, W, z, y, x, uz, uy, ux, gz, gy, gx);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float wc = c == 0 ? wz : (c == 1 ? wy : wx);
            B[c] = wc + tri_sample<true>(u + c * N, D, H, W, z, y, x, wz, wy, wx, G[c][0], G[c][1],
                                         G[c][2]);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float s = B[a];
#pragma unroll
            for (int j = 0; j < 3; ++j) s = fmaf(G[j][a], B[j], s);
            g[a * N + i] = 2.0f * s * inv_n;
            Aout[a * N + i] = A[a];
            const float aa = fabsf(A[a]);
            if (aa < 3.4e38f)
                amax = fmaxf(amax, aa);
            else
                bad = true;
            esum = fmaf(A[a], A[a], fmaf(B[a], B[a], esum));
        }
    }
    if (bad) status_set(&h->status, ST_NONFINITE);
    block_max_to(&h->coef_max_bits[kSlotA], amax, red);
    if (energy_partials) {
        // fixed-order block sum of the energy terms
        float s = esum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        __shared__ float es[8];
        if ((threadIdx.x & 31) == 0) es[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int k = 0; k < 8; ++k) t += es[k];
            energy_partials[blockIdx.x] = t;
        }
    }
}

// scatter of a (3 channels) to the corners of x + u(x), quantised relative
// to max |a| (float bits in h->coef_max_bits[slot])
__global__ void __launch_bounds__(256) k_field_scatter(const float *__restrict__ u,
                                                       const float *__restrict__ A,
                                                       unsigned long long *acc, const WsHeader *h,
                                                       int slot, int D, int H, int W) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
    if (x >= W || y >= H) return;
    const long long N = (long long)D * H * W, i = ((long long)z * H + y) * W + x;
    const float uz = u[i], uy = u[N + i], ux = u[2 * N + i];
    const float LIM = 1048576.0f;
    if (!(fabsf(uz) < LIM && fabsf(uy) < LIM && fabsf(ux) < LIM)) return;
    const int sh = fixed_shift(__uint_as_float(h->coef_max_bits[slot]), kInvBits);
    const float scale = pow2f(sh);
    const float a[3] = {A[i], A[N + i], A[2 * N + i]};
    if (!(fabsf(a[0]) < 3.4e38f && fabsf(a[1]) < 3.4e38f && fabsf(a[2]) < 3.4e38f)) return;
    const float fz = floorf(uz), fy = floorf(uy), fx = floorf(ux);
    const int iz = z + (int)fz, iy = y + (int)fy, ix = x + (int)fx;
    const float tz = uz - fz, ty = uy - fy, tx = ux - fx;
    const float wz[2] = {1.0f - tz, tz}, wy[2] = {1.0f - ty, ty}, wx[2] = {1.0f - tx, tx};
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int zz = iz + p;
        if (zz < 0 || zz >= D) continue;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int yy = iy + q;
            if (yy < 0 || yy >= H) continue;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int xx = ix + r;
                if (xx < 0 || xx >= W) continue;
                const float wt = wz[p] * wy[q] * wx[r];
                const long long j = ((long long)zz * H + yy) * W + xx;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const long long qv = quantize(a[c] * wt, scale);
                    if (qv != 0) atomicAdd(acc + c * N + j, (unsigned long long)qv);
                }
            }
        }
    }
}

// g += factor * (scattered a)
__global__ void __launch_bounds__(256) k_field_scatter_add(const long long *__restrict__ acc,
                                                           const WsHeader *h, int slot, float *g,
                                                           long long n3, float factor) {
    const int sh = fixed_shift(__uint_as_float(h->coef_max_bits[slot]), kInvBits);
    const float f = factor * pow2f(-sh);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (long long)gridDim.x * blockDim.x)
        g[i] = fmaf(i64_to_float_rn(acc[i]), f, g[i]);
}

__global__ void k_energy_finalize(const float *__restrict__ partials, int nb, long long N,
                                  float *out) {
    float hi = 0.0f, lo = 0.0f;
    for (int b = threadIdx.x; b < nb; b += 32) ff_add(hi, lo, partials[b], 0.0f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
        ff_add(hi, lo, oh, ol);
    }
    if (threadIdx.x == 0) *out = (hi + lo) / (float)N;
}

// energy gradient g of w at level d (and the energy into *energy when given)
cudaError_t inverse_gradient(InverseWs &q, const float *u, const float *w, Dims d, float *g,
                             float *energy, cudaStream_t s) {
    const long long N = d.N();
    cudaError_t e = cudaMemsetAsync(&q.h->coef_max_bits[kSlotA], 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k_inverse_terms<<<kEnergyBlocks, 256, 0, s>>>(u, w, q.A, g, q.h, energy ? q.partials : nullptr,
                                                  d.D, d.H, d.W);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (energy) {
        k_energy_finalize<<<1, 32, 0, s>>>(q.partials, kEnergyBlocks, N, energy);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemsetAsync(q.acc, 0, sizeof(long long) * 3 * N, s)) != cudaSuccess) return e;
    if ((e = launch_field_scatter(u, q.A, q.acc, q.h, kSlotA, d, s)) != cudaSuccess) return e;
    return launch_field_scatter_add(q.acc, q.h, kSlotA, 2.0f / (float)N, g, 3 * N, s);
}

fa_status check_inverse_params(const fa_params *p) {
    if (!p || p->n_levels < 1 || p->n_levels > 8) {
        set_error("fa_inverse: n_levels must be in 1..8");
        return FA_ERR_INVALID;
    }
    for (int l = 0; l < p->n_levels; ++l)
        if (p->scales[l] < 1 || 0.5f * (float)p->scales[l] > kMaxSigma || p->iters[l] < 0) {
            set_error("fa_inverse: level %d: scale in 1..%d, iterations >= 0", l,
                      (int)(2 * kMaxSigma));
            return FA_ERR_INVALID;
        }
    GaussTaps t;
    if (!make_gauss_taps(p->sigma_grad, &t) || !make_gauss_taps(p->sigma_warp, &t)) {
        set_error("fa_inverse: sigma_grad and sigma_warp must be in [0, %g]", (double)kMaxSigma);
        return FA_ERR_INVALID;
    }
    return check_adam_params(p, "fa_inverse");
}

size_t inverse_ws_bytes(Dims full, const fa_params *p) {
    WsCarver c(nullptr, ~size_t(0));
    InverseWs q;
    inverse_carve(c, full, p, &q);
    return c.off;
}

}  // namespace

cudaError_t launch_field_scatter(const float *u, const float *a, long long *acc,
                                 const WsHeader *h, int slot, Dims d, cudaStream_t s) {
    VoxGrid vg(d.D, d.H, d.W);
    k_field_scatter<<<vg.grid, vg.block, 0, s>>>(u, a, (unsigned long long *)acc, h, slot, d.D,
                                                 d.H, d.W);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_field_scatter_add(const long long *acc, const WsHeader *h, int slot,
                                     float factor, float *g, long long n3, cudaStream_t s) {
    k_field_scatter_add<<<kEnergyBlocks, 256, 0, s>>>(acc, h, slot, g, n3, factor);
    note_launch();
    return cudaGetLastError();
}

}  // namespace fa

extern "C" size_t fa_inverse_workspace_size(int32_t D, int32_t H, int32_t W, const fa_params *p) {
    using namespace fa;
    clear_error();
    if (D < 1 || H < 1 || W < 1 || check_inverse_params(p) != FA_OK) return 0;
    return inverse_ws_bytes(Dims{D, H, W}, p);
}

extern "C" fa_status fa_inverse_energy_grad(const fa_vol *u, const fa_vol *w, float *energy_dev,
                                            fa_vol *g_out, void *ws, size_t ws_bytes,
                                            void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_vol(u, "u", 3));
    FA_TRY(check_vol(w, "w", 3));
    FA_TRY(check_vol(g_out, "g", 3));
    FA_TRY(same_grid(u, w, "u", "w"));
    FA_TRY(same_grid(u, g_out, "u", "g"));
    fa_params p;
    fa_params_default(&p);
    p.n_levels = 1;
    p.scales[0] = 1;
    p.iters[0] = 0;
    const Dims d{u->D, u->H, u->W};
    FA_TRY(check_ws(ws, ws_bytes, inverse_ws_bytes(d, &p), "fa_inverse_energy_grad"));
    WsCarver c(ws, ws_bytes);
    InverseWs q;
    inverse_carve(c, d, &p, &q);
    cudaStream_t s = (cudaStream_t)stream;
    FA_CUDA_TRY(cudaMemsetAsync(q.h, 0, sizeof(WsHeader), s));
    FA_CUDA_TRY(inverse_gradient(q, (const float *)u->data, (const float *)w->data, d,
                                 (float *)g_out->data, energy_dev, s));
    return FA_OK;
}

extern "C" fa_status fa_inverse(const fa_vol *u, const fa_params *p, fa_vol *w_out,
                                float *final_energy_dev, void *ws, size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_inverse_params(p));
    FA_TRY(check_vol(u, "u", 3));
    FA_TRY(check_vol(w_out, "w_out", 3));
    const Dims full{u->D, u->H, u->W};
    const int L = p->n_levels - 1;
    const Dims last{level_size(full.D, p->scales[L]), level_size(full.H, p->scales[L]),
                    level_size(full.W, p->scales[L])};
    if (w_out->D != last.D || w_out->H != last.H || w_out->W != last.W) {
        set_error("w_out must be 3 x %d x %d x %d (the last level's grid)", last.D, last.H, last.W);
        return FA_ERR_SHAPE;
    }
    FA_TRY(check_ws(ws, ws_bytes, inverse_ws_bytes(full, p), "fa_inverse"));
    WsCarver c(ws, ws_bytes);
    InverseWs q;
    inverse_carve(c, full, p, &q);
    cudaStream_t s = (cudaStream_t)stream;
    GaussTaps tg, tw;
    make_gauss_taps(p->sigma_grad, &tg);
    make_gauss_taps(p->sigma_warp, &tw);
    FA_CUDA_TRY(cudaMemsetAsync(q.h, 0, sizeof(WsHeader), s));
    int cur = 0, t = 0;
    for (int l = 0; l < p->n_levels; ++l) {
        const Dims d = q.lvl[l];
        const size_t b = sizeof(float) * 3 * d.N();
        float su[3];
        handoff_scales(full, d, 1, su);  // phi at this level
        FA_CUDA_TRY(launch_resample((const float *)u->data, full, q.ul, d, 3, su, s));
        if (l == 0) {
            FA_CUDA_TRY(cudaMemsetAsync(q.w[cur], 0, b, s));
            FA_CUDA_TRY(cudaMemsetAsync(q.m[cur], 0, b, s));
            FA_CUDA_TRY(cudaMemsetAsync(q.v[cur], 0, b, s));
        } else {
            const Dims pc = q.lvl[l - 1];
            float s1[3], s2[3], s3[3];
            handoff_scales(pc, d, 1, s1);
            handoff_scales(pc, d, -1, s2);
            handoff_scales(pc, d, -2, s3);
            const int nx = cur ^ 1;
            FA_CUDA_TRY(launch_resample(q.w[cur], pc, q.w[nx], d, 3, s1, s));
            FA_CUDA_TRY(launch_resample(q.m[cur], pc, q.m[nx], d, 3, s2, s));
            FA_CUDA_TRY(launch_resample(q.v[cur], pc, q.v[nx], d, 3, s3, s));
            cur = nx;
        }
        for (int it = 0; it < p->iters[l]; ++it) {
            ++t;
            const int parity = t & 1;
            FA_CUDA_TRY(inverse_gradient(q, q.ul, q.w[cur], d, q.g, nullptr, s));
            FA_CUDA_TRY(launch_gauss3(q.g, q.g, q.t1, q.t2, 3, d, tg, s));
            FA_CUDA_TRY(launch_adam(q.g, q.m[cur], q.v[cur], q.dir, d.N(), adam_consts(p, t),
                                    q.h, parity, s));
            FA_CUDA_TRY(launch_compose(q.w[cur], q.dir, q.w[cur ^ 1], d, p->lr, p->c_lp, q.h,
                                       parity, nullptr, s));
            FA_CUDA_TRY(launch_gauss3(q.w[cur ^ 1], q.w[cur], q.t1, q.t2, 3, d, tw, s));
        }
        if (l == L) {
            FA_CUDA_TRY(inverse_gradient(q, q.ul, q.w[cur], d, q.g, final_energy_dev, s));
            FA_CUDA_TRY(cudaMemcpyAsync(w_out->data, q.w[cur], b, cudaMemcpyDeviceToDevice, s));
        }
    }
    return FA_OK;
}
