// Persistent form of the fused iteration for the coarse pyramid levels.
//
// A coarse level is small (10^5 - 10^6 voxels): the z-marching fused
// kernels then run one to a few output planes per CTA against a z-halo of
// 2R planes, and four launches per iteration leave the GPU latency-bound.
// Here one cooperative launch runs ALL iterations of a level: its CTAs stay
// resident and meet at grid barriers, and every separable stencil is split
// into an in-plane part (x and y, in shared memory, per item) and a z part
// (a gather of 2R + 1 planes per voxel), so no plane is processed twice
// except the few halo rows of an item.
//
// An item is one z-plane and a band of PBY rows (all W columns).  Per
// iteration, with a grid barrier after each line:
//   B   z-sums of the forward window sums -> cc, the adjoint coefficients
//       A, B, C (hi, lo), loss, coefficient maxima
//   C   quantised A, B, C summed along x and y (needs the global maxima)
//   DE  z-sums of those -> dL/dJ -> g = dL/dJ grad I_m(phi) on the band and
//       RG halo rows -> Gaussian(sigma_grad) along x and y
//   F   Gaussian along z -> Adam (m, nu, d) -> max |d|
//   G   compose u' = delta + u o (id + delta) on the band and RW halo rows
//       (delta = -eps_t d, eps_t from the global max) -> Gaussian(sigma_warp)
//       along x and y
//   HA  Gaussian along z -> u_new; J = I_m o (id + u_new) and grad I_m(phi)
//       on the band and R halo rows; J, J^2, I J summed along x and y for
//       the next iteration's B (the level's first sums run before the loop)
// Six barriers per iteration.
//
// Every arithmetic step is the one the fused kernels take, in the same
// order: exact int64 window sums, the same quantisation and conversions, the
// same epilogues, and the Gaussian taps accumulated with fmaf in the same
// tap order along x, then y, then z.  The persistent form therefore computes
// the bits of the four fused kernels.
//
// Measured on GB300 it is slower than those kernels (brain-shaped pair:
// 59 against 52 us per iteration at 40x48x56, 326 against 121 at
// 80x96x112): every phase gathers 2R + 1 planes per voxel from L2 where the
// z-marching kernels read each plane once, and a phase is a chain of L2
// round trips and CTA barriers.  It is therefore an opt-in schedule
// (FA_MODE_PERSISTENT).
//
// Data written inside the launch by other CTAs is read with ld.global.cg
// (L2, never a stale L1 line); the level's images and window statistics,
// which no CTA writes, are read through the read-only path.  Every grid
// barrier wait is bounded: on expiry a CTA sets ST_TIMEOUT and an abort flag,
// and every CTA leaves at its next barrier.
#include <cuda_bf16.h>

#include <string.h>

#include <mutex>

#include "register.h"
#include "validate.h"

namespace fa {

namespace {

constexpr int PT = 256;        // threads per CTA
constexpr int PBY = 8;         // rows per item
constexpr int PWMAX = 128;     // widest level row this form takes
constexpr int PRMAX = 3;       // widest LNCC box radius (window 7)
constexpr int PGMAX = 6;       // widest Gaussian radius
constexpr int PGT = 2 * PGMAX + 1;  // tap loops run to this length, predicated
constexpr int kMaxPersistIters = 512;  // iterations per launch (bias-correction table)

struct PersistArgs {
    const float *If, *Im;     // level images (constant during the launch)
    const long long *sI;      // window sum of I_f (constant)
    const float *varI;        // its window variance (constant)
    float *u[2];              // iteration i reads u[i & 1] and writes u[(i + 1) & 1]
    void *m, *v;              // Adam moments (storage TS)
    float *J, *gJ;            // warped image and grad I_m(phi)
    float *coef;              // [4][N] A, B, C hi, C lo
    float *gxy;               // [3][N] in-plane Gaussian of g
    float *uxy;               // [3][N] in-plane Gaussian of u'
    float *dir;               // [3][N] Adam direction
    long long *xy;            // [3][N] in-plane window sums
    WsHeader *h;
    int D, H, W, R, window, bits, cbits, RG, RW, T, t0;
    float cc_eps, lr, c_lp, b1, b2, eps;
    float wg[2 * PGMAX + 1], ww[2 * PGMAX + 1];
    float rbc1[kMaxPersistIters], rbc2[kMaxPersistIters];
};

// ------------------------------------------------------------ shared layout
// The phases use disjoint lifetimes of one dynamic buffer:
//   A : qI, qJ int32 [PBY + 2R][WQ]; xb int64 [3][PBY + 2R][W]
//   C : xb int64 [3][PBY + 2R][W]
//   DE, G: in-plane values float [3][PBY + 2RG][WG]; xb float [3][PBY + 2RG][W]
//   HA: J of the item's rows float [PBY + 2R][W] (kept across A)
// with WQ = round4(W) + 2R + 4 and WG = round4(W) + 2RG + 4 (the x passes
// read four outputs' taps with one row of slack).
__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

struct PLayout {
    int rowsA, WQ, rowsG, WG;
    size_t oJ, oQI, oQJ, oXB, oGS, oGX, bytes;
};

__host__ __device__ inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

__host__ __device__ inline PLayout playout(int W, int R, int RG, int RW) {
    PLayout L;
    const int RGm = RG > RW ? RG : RW;
    L.rowsA = PBY + 2 * R;
    L.WQ = round4(W) + 2 * R + 4;
    L.rowsG = PBY + 2 * RGm;
    L.WG = round4(W) + 2 * RGm + 4;
    L.oJ = 0;
    const size_t sJ = al256((size_t)L.rowsA * W * 4);
    // region after sJ: union of A's / C's int buffers and DE/G's float buffers
    L.oQI = sJ;
    L.oQJ = L.oQI + al256((size_t)L.rowsA * L.WQ * 4);
    L.oXB = L.oQJ + al256((size_t)L.rowsA * L.WQ * 4);
    const size_t endA = L.oXB + al256((size_t)3 * L.rowsA * W * 8);
    L.oGS = sJ;
    L.oGX = L.oGS + al256((size_t)3 * L.rowsG * L.WG * 4);
    const size_t endG = L.oGX + al256((size_t)3 * L.rowsG * W * 4);
    L.bytes = endA > endG ? endA : endG;
    return L;
}

// ------------------------------------------------------------ grid barrier
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Every CTA arrives once per barrier; barrier k completes when the counter
// reaches k * gridDim.x.  Returns false (uniformly over the CTA) when the
// launch is being abandoned.
__device__ __forceinline__ bool grid_barrier(WsHeader *h, unsigned &k, int *flag,
                                             long long limit = 1ll << 28) {
    __syncthreads();
    ++k;
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        red_release_add(&h->pbar_count, 1u);
        const unsigned target = k * gridDim.x;
        const long long c0 = clock64();
        while (ld_acquire_u32(&h->pbar_count) < target) {
            if (ld_acquire_u32(&h->pbar_abort) != 0u) {
                ok = 0;
                break;
            }
            if (clock64() - c0 > limit) {  // 2^28: 0.13 s at 2 GHz; a barrier takes ~1.5 us
                status_set(&h->status, ST_TIMEOUT);
                atomicExch(&h->pbar_abort, 1u);
                ok = 0;
                break;
            }
        }
        __threadfence();
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

// Trilinear sample of a field written inside this launch (L2 loads); the
// same cell, fractions and zero fill as tri_issue.
__device__ __forceinline__ void tri_issue_cg(TriPending &p, const float *v, int D, int H, int W,
                                             int z, int y, int x, float uz, float uy, float ux) {
    p.c000 = p.c001 = p.c010 = p.c011 = p.c100 = p.c101 = p.c110 = p.c111 = 0.0f;
    p.tz = p.ty = p.tx = 0.0f;
    const float LIM = 1048576.0f;
    if (!(fabsf(uz) < LIM && fabsf(uy) < LIM && fabsf(ux) < LIM)) {
        if (isnan(uz) || isnan(uy) || isnan(ux)) p.c000 = __int_as_float(0x7fc00000);
        p.tz = p.ty = p.tx = isnan(uz) || isnan(uy) || isnan(ux) ? __int_as_float(0x7fc00000) : 0.0f;
        return;
    }
    float fz = floorf(uz), fy = floorf(uy), fx = floorf(ux);
    int iz = z + (int)fz, iy = y + (int)fy, ix = x + (int)fx;
    p.tz = uz - fz;
    p.ty = uy - fy;
    p.tx = ux - fx;
    if (iz < -1 || iz >= D || iy < -1 || iy >= H || ix < -1 || ix >= W) return;
    const bool z0 = iz >= 0, z1 = iz + 1 < D;
    const bool y0 = iy >= 0, y1 = iy + 1 < H;
    const bool x0 = ix >= 0, x1 = ix + 1 < W;
    const int b = (iz * H + iy) * W + ix;
    const float *q0 = v + b, *q1 = q0 + H * W;
    if (z0 && y0 && x0) p.c000 = __ldcg(q0);
    if (z0 && y0 && x1) p.c001 = __ldcg(q0 + 1);
    if (z0 && y1 && x0) p.c010 = __ldcg(q0 + W);
    if (z0 && y1 && x1) p.c011 = __ldcg(q0 + W + 1);
    if (z1 && y0 && x0) p.c100 = __ldcg(q1);
    if (z1 && y0 && x1) p.c101 = __ldcg(q1 + 1);
    if (z1 && y1 && x0) p.c110 = __ldcg(q1 + W);
    if (z1 && y1 && x1) p.c111 = __ldcg(q1 + W + 1);
}

// The compose's sample of a field written inside this launch: the cell and
// weights of tri_issue_step (this voxel and its neighbours on the side of the
// step's sign for a step shorter than one voxel, tri_issue_cg's cell
// otherwise), L2 loads.
__device__ __forceinline__ void tri_issue_step_cg(TriPending &p, const float *v, int D, int H,
                                                  int W, int z, int y, int x, float uz, float uy,
                                                  float ux) {
    if (!(fabsf(uz) < 1.0f && fabsf(uy) < 1.0f && fabsf(ux) < 1.0f)) {
        tri_issue_cg(p, v, D, H, W, z, y, x, uz, uy, ux);
        return;
    }
    p.tz = fabsf(uz);
    p.ty = fabsf(uy);
    p.tx = fabsf(ux);
    const int sz = uz < 0.0f ? -1 : 1, sy = uy < 0.0f ? -1 : 1, sx = ux < 0.0f ? -1 : 1;
    const bool zo = z + sz >= 0 && z + sz < D, yo = y + sy >= 0 && y + sy < H,
               xo = x + sx >= 0 && x + sx < W;
    const float *q0 = v + (z * H + y) * W + x, *q1 = q0 + sz * H * W;
    const int oy = sy * W;
    p.c000 = __ldcg(q0);
    p.c001 = xo ? __ldcg(q0 + sx) : 0.0f;
    p.c010 = yo ? __ldcg(q0 + oy) : 0.0f;
    p.c011 = yo && xo ? __ldcg(q0 + oy + sx) : 0.0f;
    p.c100 = zo ? __ldcg(q1) : 0.0f;
    p.c101 = zo && xo ? __ldcg(q1 + sx) : 0.0f;
    p.c110 = zo && yo ? __ldcg(q1 + oy) : 0.0f;
    p.c111 = zo && yo && xo ? __ldcg(q1 + oy + sx) : 0.0f;
}

// Sliding window sums of 4 adjacent outputs from 4 + 2R values.
template <int R, class T>
__device__ __forceinline__ void slide4(const T *p, T s[4]) {
    T a = 0;
#pragma unroll
    for (int t = 0; t <= 2 * R; ++t) a += p[t];
    s[0] = a;
#pragma unroll
    for (int jj = 1; jj < 4; ++jj) {
        a += p[2 * R + jj] - p[jj - 1];
        s[jj] = a;
    }
}

// ---------------------------------------------------------------- phase A
// J (in sJ, rows y0 - R .. y0 + PBY + R - 1) and I_f of the item's plane:
// exact in-plane window sums of J, J^2, I J -> xy[3][z][y][x] for the band.
template <int R>
__device__ void phase_A(const PersistArgs &a, unsigned char *sm, const PLayout &L, int z, int y0,
                        int nrows, float scale) {
    const int W = a.W, H = a.H, rows = L.rowsA, WQ = L.WQ;
    const long long HW = (long long)H * W, N = HW * a.D;
    const float *sJ = (const float *)(sm + L.oJ);
    int *qI = (int *)(sm + L.oQI), *qJ = (int *)(sm + L.oQJ);
    long long *xb = (long long *)(sm + L.oXB);
    for (int k = threadIdx.x; k < rows * WQ; k += PT) {
        const int r = k / WQ, c = k - r * WQ, y = y0 - R + r, x = c - R;
        const bool ok = y >= 0 && y < H && x >= 0 && x < W;
        const float jv = ok ? sJ[r * W + x] : 0.0f;
        const float iv = ok ? __ldg(a.If + (long long)z * HW + (long long)y * W + x) : 0.0f;
        qJ[k] = __float2int_rn(jv * scale);
        qI[k] = __float2int_rn(iv * scale);
    }
    __syncthreads();
    const int NX4 = round4(W) / 4;
    for (int k = threadIdx.x; k < 3 * rows * NX4; k += PT) {
        const int c = k / (rows * NX4), rest = k - c * rows * NX4, r = rest / NX4,
                  x = 4 * (rest - r * NX4);
        const int *pj = qJ + r * WQ + x, *pi = qI + r * WQ + x;
        long long out[4];
        if (c == 0) {
            int s4[4];
            slide4<R, int>(pj, s4);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) out[jj] = s4[jj];
        } else {
            long long pr[4 + 2 * R];
#pragma unroll
            for (int t = 0; t < 4 + 2 * R; ++t)
                pr[t] = (long long)(c == 2 ? pi[t] : pj[t]) * pj[t];
            slide4<R, long long>(pr, out);
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
            if (x + jj < W) xb[(c * rows + r) * W + x + jj] = out[jj];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * nrows * W; k += PT) {
        const int c = k / (nrows * W), rest = k - c * nrows * W, yb = rest / W,
                  x = rest - yb * W;
        long long s = 0;
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) s += xb[(c * rows + yb + t) * W + x];
        __stcg(a.xy + c * N + (long long)z * HW + (long long)(y0 + yb) * W + x, s);
    }
    __syncthreads();
}

// ----------------------------------------------------------------- kernel
template <class TS, int R>
__global__ void __launch_bounds__(PT, 3) k_level_persistent(const __grid_constant__ PersistArgs a) {
    extern __shared__ __align__(256) unsigned char sm[];
    __shared__ int flag;
    __shared__ float redf[32];
    __shared__ unsigned long long redu[32];
    WsHeader *h = a.h;
    const int D = a.D, H = a.H, W = a.W, tid = threadIdx.x;
    const long long HW = (long long)H * W, N = HW * D;
    const int nb = (H + PBY - 1) / PBY, items = D * nb;
    const PLayout L = playout(W, R, a.RG, a.RW);
    if (tid == 0) flag = (int)(*(volatile const unsigned *)&h->status & ST_TIMEOUT);
    __syncthreads();
    if (flag) return;

    const float amax =
        fmaxf(__uint_as_float(h->absmax_bits[0]), __uint_as_float(h->absmax_bits[1]));
    const int sh = fixed_shift(amax, a.bits);
    const float scale = pow2f(sh), inv_s = pow2f(-sh);
    const long long n = (long long)a.window * a.window * a.window;
    const float nf = (float)n, inv_nf = 1.0f / nf, inv_n = 1.0f / (float)N;
    float *sJ = (float *)(sm + L.oJ);
    unsigned kb = 0;  // grid barriers passed
    float us[3];      // de-quantisation of the adjoint sums, set in C, used in DE

    // the level's first in-plane sums, from J as the level start left it
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int z = it / nb, y0 = (it - z * nb) * PBY, nrows = min(PBY, H - y0);
        for (int k = tid; k < L.rowsA * W; k += PT) {
            const int r = k / W, x = k - r * W, y = y0 - R + r;
            sJ[k] = (y >= 0 && y < H) ? __ldcg(a.J + (long long)z * HW + (long long)y * W + x)
                                      : 0.0f;
        }
        __syncthreads();
        phase_A<R>(a, sm, L, z, y0, nrows, scale);
    }

    for (int itn = 0; itn < a.T; ++itn) {
        const int t = a.t0 + itn + 1, parity = t & 1;
        const float *u = a.u[itn & 1];
        float *un = a.u[(itn + 1) & 1];
        const bool last = itn + 1 == a.T;

        // ---------------------------------------------------------- B
        if (!grid_barrier(h, kb, &flag)) return;
        {
            unsigned long long qcc = 0;
            float mA = 0.f, mB = 0.f, mC = 0.f;
            bool bad = false;
            for (int it = blockIdx.x; it < items; it += gridDim.x) {
                const int z = it / nb, y0 = (it - z * nb) * PBY, nrows = min(PBY, H - y0);
                for (int k = tid; k < nrows * W; k += PT) {
                    const int yb = k / W, x = k - yb * W;
                    const long long vox = (long long)z * HW + (long long)(y0 + yb) * W + x;
                    long long acc[3] = {0, 0, 0};
#pragma unroll
                    for (int dz = -R; dz <= R; ++dz) {
                        const int zz = z + dz;
                        const long long o = vox + (long long)dz * HW;
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            acc[c] += (zz >= 0 && zz < D) ? __ldcg(a.xy + c * N + o) : 0ll;
                    }
                    const long long a1 = __ldg(a.sI + vox), a2 = acc[0];
                    const float varI = __ldg(a.varI + vox);
                    const float varJ =
                        diff_i128_to_float(n, acc[1], a2, a2) * inv_s * inv_s * inv_nf;
                    const float cross =
                        diff_i128_to_float(n, acc[2], a1, a2) * inv_s * inv_s * inv_nf;
                    const float den = fmaf(varI, varJ, a.cc_eps);
                    const float rden = __frcp_rn(den);
                    const float cc = cross * cross * rden;
                    if (cc >= 0.0f && cc <= 2.0f)
                        qcc += (unsigned long long)quantize(cc, 4294967296.0f);
                    else
                        bad = true;
                    const float A = 2.0f * cross * rden;
                    const float B = -cc * varI * rden;
                    float Ch, Cl;
                    lncc_c_ff(A, B, a1, a2, inv_s, nf, inv_nf, Ch, Cl);
                    __stcg(a.coef + vox, A);
                    __stcg(a.coef + N + vox, B);
                    __stcg(a.coef + 2 * N + vox, Ch);
                    __stcg(a.coef + 3 * N + vox, Cl);
                    mA = fmaxf(mA, fabsf(A));
                    mB = fmaxf(mB, fabsf(B));
                    mC = fmaxf(mC, fabsf(Ch));
                }
            }
            if (bad) status_set(&h->status, ST_NONFINITE);
            block_sum_to(&h->loss_acc, qcc, redu);
            block_max_to(&h->coef_max_bits[0], mA, redf);
            block_max_to(&h->coef_max_bits[1], mB, redf);
            block_max_to(&h->coef_max_bits[2], mC, redf);
        }

        // ---------------------------------------------------------- C
        if (!grid_barrier(h, kb, &flag)) return;
        {
            float qs[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int e = fixed_shift(__uint_as_float(__ldcg(&h->coef_max_bits[c])), a.cbits);
                qs[c] = pow2f(e);
                us[c] = pow2f(-e);
            }
            const int rows = L.rowsA, NX4 = round4(W) / 4;
            long long *xb = (long long *)(sm + L.oXB);
            for (int it = blockIdx.x; it < items; it += gridDim.x) {
                const int z = it / nb, y0 = (it - z * nb) * PBY, nrows = min(PBY, H - y0);
                for (int k = tid; k < rows * NX4; k += PT) {
                    const int r = k / NX4, x = 4 * (k - r * NX4), y = y0 - R + r;
                    long long qa[4 + 2 * R], qb[4 + 2 * R], qc[4 + 2 * R];
#pragma unroll
                    for (int tt = 0; tt < 4 + 2 * R; ++tt) {
                        const int xx = x - R + tt;
                        float A = 0.f, B = 0.f, Ch = 0.f, Cl = 0.f;
                        if (y >= 0 && y < H && xx >= 0 && xx < W) {
                            const long long o = (long long)z * HW + (long long)y * W + xx;
                            A = __ldcg(a.coef + o);
                            B = __ldcg(a.coef + N + o);
                            Ch = __ldcg(a.coef + 2 * N + o);
                            Cl = __ldcg(a.coef + 3 * N + o);
                        }
                        qa[tt] = quantize(A, qs[0]);
                        qb[tt] = quantize(B, qs[1]);
                        qc[tt] = quantize(Ch, qs[2]) + quantize(Cl, qs[2]);
                    }
                    long long oa[4], ob[4], oc[4];
                    slide4<R, long long>(qa, oa);
                    slide4<R, long long>(qb, ob);
                    slide4<R, long long>(qc, oc);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj)
                        if (x + jj < W) {
                            xb[(0 * rows + r) * W + x + jj] = oa[jj];
                            xb[(1 * rows + r) * W + x + jj] = ob[jj];
                            xb[(2 * rows + r) * W + x + jj] = oc[jj];
                        }
                }
                __syncthreads();
                for (int k = tid; k < 3 * nrows * W; k += PT) {
                    const int c = k / (nrows * W), rest = k - c * nrows * W, yb = rest / W,
                              x = rest - yb * W;
                    long long s = 0;
#pragma unroll
                    for (int tt = 0; tt <= 2 * R; ++tt) s += xb[(c * rows + yb + tt) * W + x];
                    __stcg(a.xy + c * N + (long long)z * HW + (long long)(y0 + yb) * W + x, s);
                }
                __syncthreads();
            }
        }

        // --------------------------------------------------------- DE
        if (!grid_barrier(h, kb, &flag)) return;
        {
            const int RG = a.RG, rows = PBY + 2 * RG, WG = L.WG;
            float *gs = (float *)(sm + L.oGS), *gx = (float *)(sm + L.oGX);
            for (int it = blockIdx.x; it < items; it += gridDim.x) {
                const int z = it / nb, y0 = (it - z * nb) * PBY, nrows = min(PBY, H - y0);
                for (int k = tid; k < rows * WG; k += PT) {
                    const int r = k / WG, cc = k - r * WG, y = y0 - RG + r, x = cc - RG;
                    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
                    if (y >= 0 && y < H && x >= 0 && x < W) {
                        const long long vox = (long long)z * HW + (long long)y * W + x;
                        long long acc[3] = {0, 0, 0};
#pragma unroll
                        for (int dz = -R; dz <= R; ++dz) {
                            const int zz = z + dz;
                            const long long o = vox + (long long)dz * HW;
#pragma unroll
                            for (int c = 0; c < 3; ++c)
                                acc[c] += (zz >= 0 && zz < D) ? __ldcg(a.xy + c * N + o) : 0ll;
                        }
                        const float Iv = __ldg(a.If + vox), Jv = __ldcg(a.J + vox);
                        float ah, al, bh, bl, ch, cl, rh, rl, th, tl;
                        i64_to_ff(acc[0], ah, al);
                        i64_to_ff(acc[1], bh, bl);
                        i64_to_ff(acc[2], ch, cl);
                        ff_mul_f(Iv, ah * us[0], al * us[0], rh, rl);
                        ff_mul_f(2.0f * Jv, bh * us[1], bl * us[1], th, tl);
                        ff_add(rh, rl, th, tl);
                        ff_add(rh, rl, ch * us[2], cl * us[2]);
                        const float dj = -(rh + rl) * inv_n;
                        g0 = dj * __ldcg(a.gJ + vox);
                        g1 = dj * __ldcg(a.gJ + N + vox);
                        g2 = dj * __ldcg(a.gJ + 2 * N + vox);
                    }
                    gs[(0 * rows + r) * WG + cc] = g0;
                    gs[(1 * rows + r) * WG + cc] = g1;
                    gs[(2 * rows + r) * WG + cc] = g2;
                }
                __syncthreads();
                const int NX4 = round4(W) / 4;
                for (int k = tid; k < 3 * rows * NX4; k += PT) {
                    const int c = k / (rows * NX4), rest = k - c * rows * NX4, r = rest / NX4,
                              x = 4 * (rest - r * NX4);
                    const float *p = gs + (c * rows + r) * WG + x;
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        float s = 0.0f;
#pragma unroll
                        for (int tt = 0; tt < PGT; ++tt)
                            if (tt <= 2 * RG) s = fmaf(a.wg[tt], p[jj + tt], s);
                        if (x + jj < W) gx[(c * rows + r) * W + x + jj] = s;
                    }
                }
                __syncthreads();
                for (int k = tid; k < 3 * nrows * W; k += PT) {
                    const int c = k / (nrows * W), rest = k - c * nrows * W, yb = rest / W,
                              x = rest - yb * W;
                    float s = 0.0f;
#pragma unroll
                    for (int tt = 0; tt < PGT; ++tt)
                        if (tt <= 2 * RG) s = fmaf(a.wg[tt], gx[(c * rows + yb + tt) * W + x], s);
                    __stcg(a.gxy + c * N + (long long)z * HW + (long long)(y0 + yb) * W + x, s);
                }
                __syncthreads();
            }
        }

        // ---------------------------------------------------------- F
        if (!grid_barrier(h, kb, &flag)) return;
        if (blockIdx.x == 0 && tid == 0) {  // every CTA has used this iteration's maxima
            for (int c = 0; c < 8; ++c) h->coef_max_bits[c] = 0u;
            h->loss_acc = 0ull;
        }
        {
            const int RG = a.RG;
            const float rbc1 = a.rbc1[itn], rbc2 = a.rbc2[itn];
            TS *m = (TS *)a.m, *v = (TS *)a.v;
            float mx = 0.0f;
            bool bad = false;
            for (int it = blockIdx.x; it < items; it += gridDim.x) {
                const int z = it / nb, y0 = (it - z * nb) * PBY, nrows = min(PBY, H - y0);
                for (int k = tid; k < nrows * W; k += PT) {
                    const int yb = k / W, x = k - yb * W;
                    const long long vox = (long long)z * HW + (long long)(y0 + yb) * W + x;
                    float sz[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                    for (int tt = 0; tt < PGT; ++tt) {
                        const int zz = z - RG + tt;
                        const long long o = vox + (long long)(tt - RG) * HW;
                        if (tt <= 2 * RG && zz >= 0 && zz < D) {
#pragma unroll
                            for (int c = 0; c < 3; ++c)
                                sz[c] = fmaf(a.wg[tt], __ldcg(a.gxy + c * N + o), sz[c]);
                        }
                    }
                    float nrm2 = 0.0f;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float sg = sz[c];
                        const float mo = st_load(m[c * N + vox]), vo = st_load(v[c * N + vox]);
                        const float mvv = fmaf(a.b1, mo, (1.0f - a.b1) * sg);
                        const float vvv = fmaf(a.b2, vo, (1.0f - a.b2) * sg * sg);
                        m[c * N + vox] = st_store<TS>(mvv);
                        v[c * N + vox] = st_store<TS>(vvv);
                        const float dv = adam_dir(mvv, vvv, rbc1, rbc2, a.eps);
                        __stcg(a.dir + c * N + vox, dv);
                        nrm2 = fmaf(dv, dv, nrm2);
                    }
                    if (nrm2 <= 3.4e38f)
                        mx = fmaxf(mx, sqrtf(nrm2));
                    else
                        bad = true;
                }
            }
            if (bad) status_set(&h->status, ST_NONFINITE);
            block_max_to(&h->step_max_bits[parity], mx, redf);
        }

        // ---------------------------------------------------------- G
        if (!grid_barrier(h, kb, &flag)) return;
        {
            const float mxd = __uint_as_float(__ldcg(&h->step_max_bits[parity]));
            const float e = (mxd > 0.0f) ? a.lr / (a.c_lp * mxd) : 0.0f;
            if (blockIdx.x == 0 && tid == 0) {  // every CTA has read this iteration's max
                h->step_max_bits[parity ^ 1] = 0u;
                h->eps_t = e;
            }
            const int RW = a.RW, rows = PBY + 2 * RW, WG = L.WG;
            float *us = (float *)(sm + L.oGS), *ux = (float *)(sm + L.oGX);
            for (int it = blockIdx.x; it < items; it += gridDim.x) {
                const int z = it / nb, y0 = (it - z * nb) * PBY, nrows = min(PBY, H - y0);
                for (int k = tid; k < rows * WG; k += PT) {
                    const int r = k / WG, cc = k - r * WG, y = y0 - RW + r, x = cc - RW;
                    float p0 = 0.f, p1 = 0.f, p2 = 0.f;
                    if (y >= 0 && y < H && x >= 0 && x < W) {
                        const long long vox = (long long)z * HW + (long long)y * W + x;
                        const float dz = -e * __ldcg(a.dir + vox);
                        const float dy = -e * __ldcg(a.dir + N + vox);
                        const float dx = -e * __ldcg(a.dir + 2 * N + vox);
                        float gz, gy, gx;
                        TriPending t0, t1, t2;
                        tri_issue_step_cg(t0, u, D, H, W, z, y, x, dz, dy, dx);
                        tri_issue_step_cg(t1, u + N, D, H, W, z, y, x, dz, dy, dx);
                        tri_issue_step_cg(t2, u + 2 * N, D, H, W, z, y, x, dz, dy, dx);
                        p0 = dz + tri_finish<false>(t0, gz, gy, gx);
                        p1 = dy + tri_finish<false>(t1, gz, gy, gx);
                        p2 = dx + tri_finish<false>(t2, gz, gy, gx);
                    }
                    us[(0 * rows + r) * WG + cc] = p0;
                    us[(1 * rows + r) * WG + cc] = p1;
                    us[(2 * rows + r) * WG + cc] = p2;
                }
                __syncthreads();
                const int NX4 = round4(W) / 4;
                for (int k = tid; k < 3 * rows * NX4; k += PT) {
                    const int c = k / (rows * NX4), rest = k - c * rows * NX4, r = rest / NX4,
                              x = 4 * (rest - r * NX4);
                    const float *p = us + (c * rows + r) * WG + x;
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        float s = 0.0f;
#pragma unroll
                        for (int tt = 0; tt < PGT; ++tt)
                            if (tt <= 2 * RW) s = fmaf(a.ww[tt], p[jj + tt], s);
                        if (x + jj < W) ux[(c * rows + r) * W + x + jj] = s;
                    }
                }
                __syncthreads();
                for (int k = tid; k < 3 * nrows * W; k += PT) {
                    const int c = k / (nrows * W), rest = k - c * nrows * W, yb = rest / W,
                              x = rest - yb * W;
                    float s = 0.0f;
#pragma unroll
                    for (int tt = 0; tt < PGT; ++tt)
                        if (tt <= 2 * RW) s = fmaf(a.ww[tt], ux[(c * rows + yb + tt) * W + x], s);
                    __stcg(a.uxy + c * N + (long long)z * HW + (long long)(y0 + yb) * W + x, s);
                }
                __syncthreads();
            }
        }

        // --------------------------------------------------------- HA
        if (!grid_barrier(h, kb, &flag)) return;
        {
            const int RW = a.RW;
            for (int it = blockIdx.x; it < items; it += gridDim.x) {
                const int z = it / nb, y0 = (it - z * nb) * PBY, nrows = min(PBY, H - y0);
                // rows of this item: its band, plus R halo rows unless this is
                // the last iteration (the next sums need J there)
                const int rlo = last ? R : 0, rhi = last ? R + nrows : L.rowsA;
                for (int k = tid; k < (rhi - rlo) * W; k += PT) {
                    const int r = rlo + k / W, x = k - (k / W) * W, y = y0 - R + r;
                    float jv = 0.0f;
                    if (y >= 0 && y < H) {
                        const long long vox = (long long)z * HW + (long long)y * W + x;
                        float s3[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                        for (int tt = 0; tt < PGT; ++tt) {
                            const int zz = z - RW + tt;
                            const long long o = vox + (long long)(tt - RW) * HW;
                            if (tt <= 2 * RW && zz >= 0 && zz < D) {
#pragma unroll
                                for (int c = 0; c < 3; ++c)
                                    s3[c] = fmaf(a.ww[tt], __ldcg(a.uxy + c * N + o), s3[c]);
                            }
                        }
                        TriPending jp;
                        tri_issue(jp, a.Im, D, H, W, z, y, x, s3[0], s3[1], s3[2]);
                        float gz, gy, gx;
                        jv = tri_finish<true>(jp, gz, gy, gx);
                        if (r >= R && r < R + nrows) {  // the item's own rows
                            __stcg(un + vox, s3[0]);
                            __stcg(un + N + vox, s3[1]);
                            __stcg(un + 2 * N + vox, s3[2]);
                            __stcg(a.J + vox, jv);
                            __stcg(a.gJ + vox, gz);
                            __stcg(a.gJ + N + vox, gy);
                            __stcg(a.gJ + 2 * N + vox, gx);
                        }
                    }
                    sJ[r * W + x] = jv;
                }
                __syncthreads();
                if (!last) phase_A<R>(a, sm, L, z, y0, nrows, scale);
            }
        }
    }
}

// Failure-detection self-test of the grid barrier: CTA 0 never arrives, so
// the other CTAs' bounded waits give up after `limit` cycles and record
// ST_TIMEOUT; nothing hangs.
__global__ void k_grid_barrier_selftest(WsHeader *h, long long limit) {
    __shared__ int flag;
    if (blockIdx.x == 0) return;
    unsigned k = 0;
    grid_barrier(h, k, &flag, limit);
}

std::mutex g_pmu;

template <class TS, int R>
int persistent_occupancy(size_t smem) {
    auto kern = k_level_persistent<TS, R>;
    static const bool attr = [&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)playout(PWMAX, PRMAX, PGMAX, PGMAX).bytes);
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        return true;
    }();
    (void)attr;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, PT, smem) != cudaSuccess)
        occ = 0;
    return occ;
}

template <class TS, int R>
fa_status launch_persistent(PersistArgs &a, cudaStream_t s) {
    const PLayout L = playout(a.W, a.R, a.RG, a.RW);
    int occ;
    {
        std::lock_guard<std::mutex> lock(g_pmu);
        occ = persistent_occupancy<TS, R>(L.bytes);
    }
    if (occ < 1) {
        set_error("persistent level: the kernel does not fit an SM");
        return FA_ERR_UNSUPPORTED;
    }
    int dev = 0, sms = 0;
    FA_CUDA_TRY(cudaGetDevice(&dev));
    FA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int items = a.D * ((a.H + PBY - 1) / PBY);
    const int slots = sms * (occ < 4 ? occ : 4);
    const int G = items < slots ? items : slots;
    FA_CUDA_TRY(cudaMemsetAsync(&a.h->pbar_count, 0, 2 * sizeof(unsigned), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(PT);
    cfg.dynamicSmemBytes = L.bytes;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    FA_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_level_persistent<TS, R>, a));
    note_launch();
    return FA_OK;
}

}  // namespace

bool persistent_eligible(const fa_params *p, Dims d) {
    if (p->mode != FA_MODE_PERSISTENT || p->loss != FA_LOSS_LNCC || p->use_jac) return false;
    if (p->state_storage != FA_F32 && p->state_storage != FA_BF16) return false;
    if (p->window / 2 < 1 || p->window / 2 > PRMAX || d.W > PWMAX) return false;
    GaussTaps tg, tw;
    if (!make_gauss_taps(p->sigma_grad, &tg) || !make_gauss_taps(p->sigma_warp, &tw)) return false;
    if (tg.R > PGMAX || tw.R > PGMAX) return false;
    // coarse levels only: on larger grids the tiled kernels keep the GPU busy
    // and stream each field once per iteration
    return d.N() <= kPersistMaxVoxels;
}

size_t persistent_xy_bytes(long long n) { return (size_t)3 * (size_t)n * sizeof(long long); }

fa_status persistent_level(const FusedBuffers &fb, long long *xy, WsHeader *h, const fa_params *p,
                           Dims d, const float *If, const float *Im, float *u0, float *u1, void *m,
                           void *v, int t0, int T, const GaussTaps &tg, const GaussTaps &tw,
                           cudaStream_t s) {
    if (T <= 0) return FA_OK;
    PersistArgs a;
    memset(&a, 0, sizeof(a));
    a.If = If;
    a.Im = Im;
    a.sI = fb.sI;
    a.varI = fb.varI;
    a.m = m;
    a.v = v;
    a.J = fb.J;
    a.gJ = fb.gJ;
    a.coef = fb.coef;
    a.gxy = fb.g;
    a.uxy = fb.t1;
    a.dir = fb.dir;
    a.xy = xy;
    a.h = h;
    a.D = d.D;
    a.H = d.H;
    a.W = d.W;
    a.window = p->window;
    a.R = p->window / 2;
    a.bits = lncc_image_bits(p->window);
    a.cbits = lncc_coef_bits(p->window);
    a.RG = tg.R;
    a.RW = tw.R;
    for (int k = 0; k <= 2 * tg.R; ++k) a.wg[k] = tg.w[k];
    for (int k = 0; k <= 2 * tw.R; ++k) a.ww[k] = tw.w[k];
    a.cc_eps = p->cc_eps;
    a.lr = p->lr;
    a.c_lp = p->c_lp;
    a.b1 = p->beta1;
    a.b2 = p->beta2;
    a.eps = p->adam_eps;
    float *ub[2] = {u0, u1};
    for (int done = 0; done < T; done += kMaxPersistIters) {
        const int chunk = T - done < kMaxPersistIters ? T - done : kMaxPersistIters;
        a.u[0] = ub[done & 1];
        a.u[1] = ub[(done + 1) & 1];
        a.T = chunk;
        a.t0 = t0 + done;
        for (int k = 0; k < chunk; ++k) {
            const AdamConsts ac = adam_consts(p, t0 + done + k + 1);
            a.rbc1[k] = ac.rbc1;
            a.rbc2[k] = ac.rbc2;
        }
        const bool b16 = p->state_storage == FA_BF16;
        fa_status st;
        if (a.R == 1)
            st = b16 ? launch_persistent<__nv_bfloat16, 1>(a, s) : launch_persistent<float, 1>(a, s);
        else if (a.R == 2)
            st = b16 ? launch_persistent<__nv_bfloat16, 2>(a, s) : launch_persistent<float, 2>(a, s);
        else
            st = b16 ? launch_persistent<__nv_bfloat16, 3>(a, s) : launch_persistent<float, 3>(a, s);
        FA_TRY(st);
    }
    return FA_OK;
}

}  // namespace fa

extern "C" fa_status fa_selftest_grid_barrier(void *ws, size_t ws_bytes, int64_t limit_cycles,
                                              void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_ws(ws, ws_bytes, sizeof(WsHeader), "fa_selftest_grid_barrier"));
    if (limit_cycles < 0 || limit_cycles > (1ll << 31)) {
        set_error("fa_selftest_grid_barrier: limit_cycles must be in 0..2^31");
        return FA_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    FA_CUDA_TRY(launch_header_reset((WsHeader *)ws, s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(32);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    FA_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_grid_barrier_selftest, (WsHeader *)ws,
                                   (long long)limit_cycles));
    note_launch();
    return FA_OK;
}
