// fa_warp_lncc_adjoint: the loss L = LNCC(I_f, I_m o (id + u)) and its
// derivatives with respect to all three inputs, for callers that
// differentiate through a registration (template building, learned
// components around the registration).
//
//   dL/du      = dL/dJ grad I_m(phi)              (the Gateaux derivative of
//                section "Jacobian-free Eulerian descent")
//   dL/dI_f    = the LNCC adjoint with respect to the fixed image
//   dL/dI_m(p) = sum_x dL/dJ(x) w_p(x)            (the adjoint of the warp:
//                w_p(x) is the trilinear weight of corner p at x + u(x))
//
// Without dL/dI_f the call runs on the fused kernels of the registration
// loop: the warp (J and grad I_m at x + u), the fixed image's window
// statistics, K1 (exact window sums, cc, the adjoint coefficients, the loss)
// and K2 (the adjoint window sums, dL/du, and dL/dJ for the scatter).  With
// dL/dI_f it runs the per-op LNCC kernels, which also form the fixed image's
// coefficients.  The scatter of dL/dI_m accumulates quantised contributions
// in int64 with integer atomics, so the result does not depend on the order
// in which threads add (the same fixed-point scheme as the window sums).
#include "ops.h"
#include "register.h"
#include "validate.h"

namespace fa {

namespace {

constexpr int kScatterBits = 40;  // |term| <= 2^40: sums of 2^23 terms fit int64
constexpr int kSlotDJ = 7;        // header slot of max |dL/dJ|

struct AdjointBuffers {
    WsHeader *h;
    LnccBuffers lb;
    float *J, *grad, *dJ;
    long long *acc;
};

// The fused route (no dL/dI_f): the fused kernels' buffers, dL/dJ and the
// scatter accumulator.
struct AdjointFusedBuffers {
    WsHeader *h;
    FusedBuffers fb;
    float *dJ;
    long long *acc;
};

AdjointFusedBuffers adjoint_fused_carve(void *base, size_t cap, long long N, size_t *bytes) {
    WsCarver c(base, cap);
    AdjointFusedBuffers b;
    b.h = c.take<WsHeader>(1);
    fused_carve(c, N, &b.fb);
    b.dJ = c.take<float>(N);
    b.acc = c.take<long long>(N);
    *bytes = c.off;
    return b;
}

AdjointBuffers adjoint_carve(void *base, size_t cap, long long N, size_t *bytes) {
    WsCarver c(base, cap);
    AdjointBuffers b;
    b.h = c.take<WsHeader>(1);
    b.lb = lncc_carve(c, N);
    b.J = c.take<float>(N);
    b.grad = c.take<float>(3 * N);
    b.dJ = c.take<float>(N);
    b.acc = c.take<long long>(N);
    *bytes = c.off;
    return b;
}

__global__ void __launch_bounds__(256) k_absmax1(const float *__restrict__ x, long long n,
                                                 unsigned *slot) {
    __shared__ float red[32];
    float m = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));  // NaN is dropped by fmaxf; the loss reports it
    block_max_to(slot, m, red);
}

// Scatter of dJ through the trilinear weights of x + u(x) (zero outside).
__global__ void __launch_bounds__(256) k_warp_adjoint_scatter(const float *__restrict__ dJ,
                                                              const float *__restrict__ u,
                                                              unsigned long long *acc,
                                                              const WsHeader *h, int D, int H,
                                                              int W) {
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= W || y >= H) return;
    const long long N = (long long)D * H * W;
    const long long i = ((long long)z * H + y) * W + x;
    const float g = dJ[i];
    const float uz = u[i], uy = u[N + i], ux = u[2 * N + i];
    const float LIM = 1048576.0f;
    // zero, non-finite (reported by the loss) or far-outside samples add nothing
    if (!(fabsf(g) > 0.0f && fabsf(g) < 3.4e38f) ||
        !(fabsf(uz) < LIM && fabsf(uy) < LIM && fabsf(ux) < LIM))
        return;
    const int sh = fixed_shift(__uint_as_float(h->coef_max_bits[kSlotDJ]), kScatterBits);
    const float scale = pow2f(sh);
    const float fz = floorf(uz), fy = floorf(uy), fx = floorf(ux);
    const int iz = z + (int)fz, iy = y + (int)fy, ix = x + (int)fx;
    const float tz = uz - fz, ty = uy - fy, tx = ux - fx;
    const float wz[2] = {1.0f - tz, tz}, wy[2] = {1.0f - ty, ty}, wx[2] = {1.0f - tx, tx};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int zz = iz + a;
        if (zz < 0 || zz >= D) continue;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int yy = iy + b;
            if (yy < 0 || yy >= H) continue;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int xx = ix + c;
                if (xx < 0 || xx >= W) continue;
                const float w = wz[a] * wy[b] * wx[c];
                const long long q = quantize(g * w, scale);
                if (q != 0)
                    atomicAdd(acc + ((long long)zz * H + yy) * W + xx, (unsigned long long)q);
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_scatter_finalize(const long long *__restrict__ acc,
                                                          const WsHeader *h, float *out,
                                                          long long n) {
    const int sh = fixed_shift(__uint_as_float(h->coef_max_bits[kSlotDJ]), kScatterBits);
    const float inv = pow2f(-sh);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = i64_to_float_rn(acc[i]) * inv;
}

// dL/dI_m(p) = sum_x dL/dJ(x) w_p(x + u(x)): fixed point at 2^-40 of
// max |dL/dJ| with integer atomics (order-independent), then back to float.
fa_status scatter_to_moving(const float *dJ, const float *u, long long *acc, WsHeader *h,
                            Dims d, float *dIm, cudaStream_t s) {
    const long long N = d.N();
    long long blocks = (N + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_absmax1<<<(unsigned)blocks, 256, 0, s>>>(dJ, N, &h->coef_max_bits[kSlotDJ]);
    note_launch();
    FA_CUDA_TRY(cudaGetLastError());
    FA_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(long long) * N, s));
    VoxGrid g(d.D, d.H, d.W);
    k_warp_adjoint_scatter<<<g.grid, g.block, 0, s>>>(dJ, u, (unsigned long long *)acc, h, d.D,
                                                      d.H, d.W);
    note_launch();
    FA_CUDA_TRY(cudaGetLastError());
    k_scatter_finalize<<<(unsigned)blocks, 256, 0, s>>>(acc, h, dIm, N);
    note_launch();
    FA_CUDA_TRY(cudaGetLastError());
    return FA_OK;
}

}  // namespace

}  // namespace fa

extern "C" size_t fa_warp_lncc_adjoint_workspace_size(int32_t D, int32_t H, int32_t W) {
    fa::clear_error();
    if (D < 1 || H < 1 || W < 1) return 0;
    size_t plain = 0, fused = 0;
    fa::adjoint_carve(nullptr, ~size_t(0), (long long)D * H * W, &plain);
    fa::adjoint_fused_carve(nullptr, ~size_t(0), (long long)D * H * W, &fused);
    return plain > fused ? plain : fused;
}

extern "C" fa_status fa_warp_lncc_adjoint(const fa_vol *fixed, const fa_vol *moving,
                                          const fa_vol *u, int32_t window, float cc_eps,
                                          float *loss_dev, fa_vol *dL_du_opt,
                                          fa_vol *dL_dfixed_opt, fa_vol *dL_dmoving_opt, void *ws,
                                          size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    if (window < 1 || window > 15 || (window % 2) == 0) {
        set_error("fa_warp_lncc_adjoint: window must be odd and in 1..15 (got %d)", (int)window);
        return FA_ERR_INVALID;
    }
    if (!(cc_eps >= 0.0f) || !(cc_eps < 3.0e38f)) {
        set_error("fa_warp_lncc_adjoint: cc_eps must be finite and >= 0");
        return FA_ERR_INVALID;
    }
    FA_TRY(check_vol(fixed, "fixed", 1));
    FA_TRY(check_vol(moving, "moving", 1));
    FA_TRY(check_vol(u, "u", 3));
    FA_TRY(same_grid(fixed, moving, "fixed", "moving"));
    FA_TRY(same_grid(fixed, u, "fixed", "u"));
    if (dL_du_opt) {
        FA_TRY(check_vol(dL_du_opt, "dL_du", 3));
        FA_TRY(same_grid(fixed, dL_du_opt, "fixed", "dL_du"));
    }
    if (dL_dfixed_opt) {
        FA_TRY(check_vol(dL_dfixed_opt, "dL_dfixed", 1));
        FA_TRY(same_grid(fixed, dL_dfixed_opt, "fixed", "dL_dfixed"));
    }
    if (dL_dmoving_opt) {
        FA_TRY(check_vol(dL_dmoving_opt, "dL_dmoving", 1));
        FA_TRY(same_grid(fixed, dL_dmoving_opt, "fixed", "dL_dmoving"));
    }
    Dims d{fixed->D, fixed->H, fixed->W};
    const long long N = d.N();
    FA_TRY(check_ws(ws, ws_bytes, fa_warp_lncc_adjoint_workspace_size(d.D, d.H, d.W),
                    "fa_warp_lncc_adjoint"));
    cudaStream_t s = (cudaStream_t)stream;
    const float *I = (const float *)fixed->data, *Im = (const float *)moving->data;
    const float *uu = (const float *)u->data;
    float *du = dL_du_opt ? (float *)dL_du_opt->data : nullptr;
    float *dIf = dL_dfixed_opt ? (float *)dL_dfixed_opt->data : nullptr;
    float *dIm = dL_dmoving_opt ? (float *)dL_dmoving_opt->data : nullptr;

    if (!dIf) {  // the fused kernels: warp, K1 (forward), K2 (dL/du and dL/dJ), scatter
        size_t need = 0;
        AdjointFusedBuffers b = adjoint_fused_carve(ws, ws_bytes, N, &need);
        FA_CUDA_TRY(launch_header_reset(b.h, s));
        float *g = du ? du : (dIm ? b.fb.g : nullptr);
        FA_CUDA_TRY(fused_warp_lncc_adjoint(I, Im, uu, b.fb, d, window, cc_eps, b.h, loss_dev, g,
                                            dIm ? b.dJ : nullptr, s));
        if (dIm) FA_TRY(scatter_to_moving(b.dJ, uu, b.acc, b.h, d, dIm, s));
        return FA_OK;
    }

    size_t need = 0;
    AdjointBuffers b = adjoint_carve(ws, ws_bytes, N, &need);

    FA_CUDA_TRY(launch_header_reset(b.h, s));
    FA_CUDA_TRY(launch_warp(Im, uu, b.J, du ? b.grad : nullptr, d, s));
    FA_CUDA_TRY(launch_absmax2(I, b.J, N, b.h, s));
    FA_CUDA_TRY(launch_lncc_forward(I, b.J, d, window, cc_eps, dIf != nullptr, b.h, b.lb, s));
    FA_CUDA_TRY(launch_loss_finalize(b.h, N, -1.0f, loss_dev, s));
    if (du || dIf || dIm)
        FA_CUDA_TRY(launch_lncc_backward(I, b.J, du ? b.grad : nullptr, d, window, b.h, b.lb,
                                         dIm ? b.dJ : nullptr, dIf, du, s));
    if (dIm) FA_TRY(scatter_to_moving(b.dJ, uu, b.acc, b.h, d, dIm, s));
    return FA_OK;
}
