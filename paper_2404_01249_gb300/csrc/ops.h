// Internal launchers shared by the entry points and the registration driver.
// Every launcher enqueues on `s` and returns the launch error (if any).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace fa {

// A grid of D x H x W voxels.  P, when set, is the row pitch of the buffers
// that hold it (a multiple of 4 >= W, so that every row starts on a 16-byte
// boundary and the fused kernels can take TMA tiles); 0 means pitch W.  N()
// counts voxels; NP() the elements of one channel of a buffer (D H pitch).
struct Dims {
    int D, H, W;
    int P = 0;
    long long N() const { return (long long)D * H * W; }
    int pitch() const { return P > 0 ? P : W; }
    long long NP() const { return (long long)D * H * pitch(); }
};

// Gaussian taps of the method (exp(-k^2 / 2 sigma^2), |k| <= ceil(3 sigma),
// normalised); computed on the host in double, rounded to float.
struct GaussTaps {
    int R;          // radius; 0 = identity
    float w[64];    // w[k + R]
};
bool make_gauss_taps(float sigma, GaussTaps *t);
constexpr float kMaxSigma = 10.0f;

// ---- warp (warp.cu)
cudaError_t launch_warp(const float *Im, const float *u, float *J, float *grad, Dims d,
                        cudaStream_t s);
// The same for a displacement stored as `field` (FA_F32 or FA_F16).
cudaError_t launch_warp_field(const float *Im, const void *u, int field, float *J, float *grad,
                              Dims d, cudaStream_t s);
// uo = delta + u o (id + delta) (uo must not be u).
cudaError_t launch_compose_fields(const float *u, const float *delta, float *uo, Dims d,
                                  cudaStream_t s);
// g_out = J(phi)^T g_in with J(phi) = I + grad u (g_out may equal g_in).
cudaError_t launch_jac_direction(const float *gin, const float *u, float *gout, Dims d,
                                 cudaStream_t s);

// ---- plain LNCC / MSE (lncc.cu)
// Header fields used: absmax_bits, coef_max_bits, loss_acc, status.
struct LnccBuffers {
    long long *p0, *p1;   // [5][N] int64 each
    float *coef;          // [7][N]: A, B, C hi, C lo, B', C' hi, C' lo
};
size_t lncc_plain_bytes(long long N);
LnccBuffers lncc_carve(WsCarver &c, long long N);  // the plain-path scratch of an N-voxel grid
cudaError_t launch_absmax2(const float *I, const float *J, long long N, WsHeader *h,
                           cudaStream_t s);
// Forward: coefficients and loss accumulator.  want_dI selects B', C'.
cudaError_t launch_lncc_forward(const float *I, const float *J, Dims d, int window, float cc_eps,
                                bool want_dI, WsHeader *h, LnccBuffers b, cudaStream_t s);
// Backward: dJ = dL/dJ (may be NULL), dI = dL/dI (may be NULL),
// g = dL/dJ * grad (3 channels, may be NULL; needs grad).
cudaError_t launch_lncc_backward(const float *I, const float *J, const float *grad, Dims d,
                                 int window, WsHeader *h, LnccBuffers b, float *dJ, float *dI,
                                 float *g, cudaStream_t s);
long long mse_partials_count(Dims d);  // floats of `partials` launch_mse needs
cudaError_t launch_mse(const float *I, const float *J, const float *grad, Dims d, WsHeader *h,
                       float *partials, float *dJ, float *dI, float *g, cudaStream_t s);
// ---- field adjoints (inverse.cu)
// acc (3 channels, int64, zeroed by the caller) += a scattered through the
// trilinear weights of the corners of x + u(x) (zero outside), each term
// quantised to 2^-40 of max |a|, whose float bits the caller has put in
// h->coef_max_bits[slot]: the sums do not depend on the order of the adds.
cudaError_t launch_field_scatter(const float *u, const float *a, long long *acc,
                                 const WsHeader *h, int slot, Dims d, cudaStream_t s);
// g += factor * acc, converted back with the same scale.
cudaError_t launch_field_scatter_add(const long long *acc, const WsHeader *h, int slot,
                                     float factor, float *g, long long n3, cudaStream_t s);

// ---- mutual information (mi.cu)
struct MiBuffers {
    unsigned long long *hist;  // [B*B] joint histogram, 2^-26 fixed point
    float *T;                  // [B*B] log(P / (p_f p_m)), 0 where P = 0
    unsigned *range;           // [4] order-preserving keys of lo_f, hi_f, lo_m, hi_m
};
constexpr int kMiMinBins = 6, kMiMaxBins = 64;
MiBuffers mi_carve(WsCarver &c, int bins);
// [lo, hi] of I_f, and of I_m with 0 included (samples outside the grid are 0)
cudaError_t launch_mi_range(const float *If, const float *Im, long long N, MiBuffers b,
                            cudaStream_t s);
cudaError_t launch_mi_range_set(const float *range4, MiBuffers b, cudaStream_t s);
// L = -MI(I, J) into h->loss (and loss_out if not NULL); dJ = dL/dJ and
// g = dL/dJ * grad (3 channels) when not NULL.
cudaError_t launch_mi(const float *I, const float *J, const float *grad, Dims d, int bins,
                      WsHeader *h, MiBuffers b, float *loss_out, float *dJ, float *g,
                      cudaStream_t s);
// Exact window sum S_I and rounded variance of the fixed image (p0, p1:
// 2N int64 scratch each).
cudaError_t launch_fixed_stats(const float *I, Dims d, int window, const WsHeader *h,
                               long long *p0, long long *p1, long long *sI, float *varI,
                               cudaStream_t s);
// loss_out = sign * loss_acc * 2^-32 / N; also stored in h->loss.
cudaError_t launch_loss_finalize(WsHeader *h, long long N, float sign, float *loss_out,
                                 cudaStream_t s);
cudaError_t launch_header_reset(WsHeader *h, cudaStream_t s);

// ---- Gaussian (gauss.cu)
cudaError_t launch_gauss_axis(const float *in, float *out, int C, Dims d, const GaussTaps &t,
                              int axis, cudaStream_t s);
// Three passes in -> t1 -> t2 -> out (t1, t2: C*N floats each).  R == 0 copies.
cudaError_t launch_gauss3(const float *in, float *out, float *t1, float *t2, int C, Dims d,
                          const GaussTaps &t, cudaStream_t s);

// ---- Adam, step scale, compose (adam.cu)
// Records a kernel timer's event on s: as an external event node while s is
// being captured into a graph (so that the replay records it), else plainly.
inline cudaError_t timer_record(void *event, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cudaEventRecordWithFlags((cudaEvent_t)event, s,
                                    cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                        : cudaEventRecordDefault);
}

struct AdamConsts {
    float b1, b2, eps, rbc1, rbc2;  // rbc = 1 / (1 - beta^t)
};
AdamConsts adam_consts(const fa_params *p, int t);
// state16_ok: the caller can keep its Adam moments in 16-bit storage
// (fa_params.state_storage); otherwise only FA_F32 is accepted.
fa_status check_adam_params(const fa_params *p, const char *who, bool state16_ok = false);
// d = Adam direction over N voxels of 3 channels (planar, 3N floats each);
// block max of the voxel norm |d| into h->step_max_bits[parity].
cudaError_t launch_adam(const float *g, float *m, float *v, float *d, long long N, AdamConsts c,
                        WsHeader *h, int parity, cudaStream_t s);
// The same with m, v stored as `state` (FA_F32, FA_BF16 or FA_F16).
cudaError_t launch_adam_state(const float *g, void *m, void *v, int state, float *d, long long N,
                              AdamConsts c, WsHeader *h, int parity, cudaStream_t s);
// Bytes of one element of the Adam moments stored as `state`.
inline size_t state_bytes(int state) { return state == FA_F32 ? 4 : 2; }
// u_out = delta + u_in o (id + delta), delta = -lr / (c_lp max) d; resets the
// other parity's max slot; eps_t to h->eps_t and eps_out (if not NULL).
cudaError_t launch_compose(const float *u_in, const float *d, float *u_out, Dims dm, float lr,
                           float c_lp, WsHeader *h, int parity, float *eps_out, cudaStream_t s);

// ---- pyramid and hand-off (levels.cu)
// dst channel c = scale[c] * trilinear align-corners resample of src channel c
cudaError_t launch_resample(const float *src, Dims ds, float *dst, Dims dd, int C,
                            const float *scale3, cudaStream_t s);
// The same between fields stored as sfield and dfield (FA_F32 or FA_F16).
cudaError_t launch_resample_field(const void *src, int sfield, Dims ds, void *dst, int dfield,
                                  Dims dd, int C, const float *scale3, cudaStream_t s);

int level_size(int n, int s);
void handoff_scales(Dims c, Dims f, int power, float out[3]);
cudaError_t launch_pyramid_level(const float *img, Dims d, int s, float *out, Dims dl, float *t1,
                                 float *t2, cudaStream_t st);

// dst[i] = src[i] widened to FP32 (src FA_BF16 or FA_F16; exact).
cudaError_t launch_widen(const void *src, int dtype, float *dst, long long n, cudaStream_t s);
// dst[i] = src[i] rounded to nearest in dtype (FA_BF16 or FA_F16).
cudaError_t launch_narrow(const float *src, int dtype, void *dst, long long n, cudaStream_t s);

}  // namespace fa
