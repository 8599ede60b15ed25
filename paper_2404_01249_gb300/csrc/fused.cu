// Fused per-iteration kernels of fa_register (FA_MODE_FUSED).
//
// One iteration of Algorithm 1 (Jacobian-free direction) is four launches:
//   K1 k_lncc_fwd       LNCC forward on J = I_m o phi: exact int64 window
//                       sums, cc, the adjoint coefficients A, B, C, the loss
//                       accumulator and the coefficient maxima.
//   K2 k_lncc_grad      adjoint window sums of A, B, C; J and grad I_m o phi
//                       at the output voxel; g = dL/dJ grad.
//   K3 k_smooth_adam    Gaussian(sigma_grad) of g, Adam update of m, nu, the
//                       direction d and the grid max |d|.
//   K4 k_compose        delta = -eps_t d, u' = delta + u o (id + delta),
//                       Gaussian(sigma_warp) of u', and J = I_m o (id + u) of
//                       the new map for the next iteration's K1.
// The grid max of K3 is a global dependency, so K4 cannot join K3; the
// adjoint window sums need A, B, C around every output, so K2 cannot join K1
// without recomputing a much wider halo.
//
// Every kernel marches along z ("2.5-D" tiling): a CTA owns a 32 x TY tile of
// (x, y) columns and a slab of TZ output planes.  Plane inputs (tile plus
// halo) arrive through a three-stage cp.async pipeline two planes ahead of
// the plane being reduced; the plane is reduced along x and then y in shared
// memory, and the last 2R + 1 in-plane results per output column sit in a
// shared-memory ring from which the z-reduction reads.  No intermediate of
// the separable sums goes to HBM; halo re-reads hit L2.
//
// Thread layout: warp w of NW covers region rows w, w + NW, ...; lane l
// covers columns l and l + 32.  All trip counts are compile-time, the
// in-plane offsets of a thread's positions are computed once per CTA, and a
// thread consumes exactly the stage positions it copied itself wherever
// possible, so those reads need no barrier.
#include <math.h>

#include <mutex>

#include "register.h"
#include "validate.h"

namespace fa {

namespace {

constexpr int FX = 32;  // tile width along x (one warp)

__device__ __forceinline__ void cp4(void *dst, const float *src, bool ok) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(ok ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp8(void *dst, const void *src, bool ok) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
                 "r"(ok ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Row stride of an RX-wide shared region: a multiple of 4 elements, so that
// 16-byte vector loads of a row start aligned.
constexpr int pad4(int x) { return (x + 3) & ~3; }

// A thread's positions in an RY x RX region (RX <= 64) stored with row
// stride RXP.
template <int RY, int RX, int NW, int RXP = pad4(RX)>
struct Region {
    static constexpr int NJ = (RY + NW - 1) / NW;  // row slots
    static constexpr int NC = (RX + 31) / 32;      // column slots
    static constexpr int NP = NJ * NC;
    int off[NP];  // y W + x inside the grid, -1 outside the grid, -2 outside the region
    int sbase;    // shared index of slot (0, 0): wy RXP + tx

    __device__ __forceinline__ void init(int wy, int tx, int ybase, int xbase, int H, int W) {
        sbase = wy * RXP + tx;
#pragma unroll
        for (int j = 0; j < NJ; ++j)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int ry = wy + NW * j, rx = tx + 32 * c;
                const int y = ybase + ry, x = xbase + rx;
                int o = -2;
                if (ry < RY && rx < RX) o = (y >= 0 && y < H && x >= 0 && x < W) ? y * W + x : -1;
                off[j * NC + c] = o;
            }
    }
    static __device__ __forceinline__ int sofs(int j, int c) { return NW * j * RXP + 32 * c; }
};

// Copies C channels of plane zp onto [C][RY][RXP] shared floats (zero outside).
template <int C, int RY, int RX, int NW, int RXP>
__device__ __forceinline__ void load_plane(float *dst, const float *src, long long N,
                                           long long zoff, bool zok,
                                           const Region<RY, RX, NW, RXP> &rg) {
    using G = Region<RY, RX, NW, RXP>;
#pragma unroll
    for (int j = 0; j < G::NJ; ++j)
#pragma unroll
        for (int c = 0; c < G::NC; ++c) {
            const int o = rg.off[j * G::NC + c];
            if (o == -2) continue;
            const bool ok = zok && o >= 0;
            const float *s = src + (ok ? zoff + o : 0);
            float *d = dst + rg.sbase + G::sofs(j, c);
#pragma unroll
            for (int ch = 0; ch < C; ++ch) cp4(d + ch * RY * RXP, s + ch * N, ok);
        }
}

// A thread's OPT output voxels of the 32 x TY tile.
template <int OPT>
struct Outs {
    int off[OPT];  // y W + x, -1 outside the grid
    __device__ __forceinline__ void init(int wy, int tx, int y0, int x0, int NW, int H, int W) {
#pragma unroll
        for (int o = 0; o < OPT; ++o) {
            const int y = y0 + wy + NW * o, x = x0 + tx;
            off[o] = (y < H && x < W) ? y * W + x : -1;
        }
    }
};

template <int C, int OPT, int NOUT>
__device__ __forceinline__ void load_outs(float *dst, const float *src, long long N,
                                          long long zoff, const Outs<OPT> &ou, int tid, int NT) {
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
        const bool ok = ou.off[o] >= 0;
        const float *s = src + (ok ? zoff + ou.off[o] : 0);
#pragma unroll
        for (int ch = 0; ch < C; ++ch) cp4(dst + ch * NOUT + o * NT + tid, s + ch * N, ok);
    }
}

// ------------------------------------------------- register-blocked x passes
// A work item is (channel, row, group of 4 adjacent output columns); items
// are spread over all threads.  Rows are read with 16-byte shared loads.

// Gaussian x pass: pl [C][RY][RXP] -> xb [C][RY][FX].
template <int RG, int C, int RY, int RXP, int NT>
__device__ __forceinline__ void gauss_x4(const float *pl, float *xb, const GaussTaps &t, int tid) {
    constexpr int ITEMS = C * RY * 8, NL = (4 + 2 * RG + 3) / 4;
    static_assert(28 + 4 * NL <= RXP, "row too short for the vector loads");
#pragma unroll
    for (int j = 0; j < (ITEMS + NT - 1) / NT; ++j) {
        const int it = tid + j * NT;
        if (ITEMS % NT != 0 && it >= ITEMS) break;
        const int k = it & 7, rest = it >> 3, ry = rest % RY, c = rest / RY;
        const float4 *src = (const float4 *)(pl + (c * RY + ry) * RXP + 4 * k);
        float v[4 * NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const float4 q = src[l];
            v[4 * l] = q.x;
            v[4 * l + 1] = q.y;
            v[4 * l + 2] = q.z;
            v[4 * l + 3] = q.w;
        }
        float o[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            float a = 0.0f;
#pragma unroll
            for (int tt = 0; tt <= 2 * RG; ++tt) a = fmaf(t.w[tt], v[jj + tt], a);
            o[jj] = a;
        }
        *(float4 *)(xb + (c * RY + ry) * FX + 4 * k) = make_float4(o[0], o[1], o[2], o[3]);
    }
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

__device__ __forceinline__ void store_ll4(long long *d, const long long s[4]) {
    ((longlong2 *)d)[0] = make_longlong2(s[0], s[1]);
    ((longlong2 *)d)[1] = make_longlong2(s[2], s[3]);
}

// LNCC forward x pass on quantised planes qI, qJ [RY][RXP] (int32) ->
// xL [3][RY][FX] int64: channel 0 sum J, 1 sum J^2, 2 sum I J.
template <int R, int RY, int RXP, int NT>
__device__ __forceinline__ void box_x4_fwd(const int *qI, const int *qJ, long long *xL, int tid) {
    constexpr int ITEMS = 3 * RY * 8, NL = (4 + 2 * R + 3) / 4, NV = 4 + 2 * R;
    static_assert(28 + 4 * NL <= RXP, "row too short for the vector loads");
#pragma unroll
    for (int j = 0; j < (ITEMS + NT - 1) / NT; ++j) {
        const int it = tid + j * NT;
        if (ITEMS % NT != 0 && it >= ITEMS) break;
        const int k = it & 7, rest = it >> 3, ry = rest % RY, c = rest / RY;
        int vj[4 * NL], vi[4 * NL];
        const int4 *sj = (const int4 *)(qJ + ry * RXP + 4 * k);
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const int4 q = sj[l];
            vj[4 * l] = q.x;
            vj[4 * l + 1] = q.y;
            vj[4 * l + 2] = q.z;
            vj[4 * l + 3] = q.w;
        }
        long long out[4];
        if (c == 0) {
            int s4[4];
            slide4<R, int>(vj, s4);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) out[jj] = s4[jj];
        } else {
            if (c == 2) {
                const int4 *si = (const int4 *)(qI + ry * RXP + 4 * k);
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    const int4 q = si[l];
                    vi[4 * l] = q.x;
                    vi[4 * l + 1] = q.y;
                    vi[4 * l + 2] = q.z;
                    vi[4 * l + 3] = q.w;
                }
            } else {
#pragma unroll
                for (int l = 0; l < 4 * NL; ++l) vi[l] = vj[l];
            }
            long long pr[NV];
#pragma unroll
            for (int t = 0; t < NV; ++t) pr[t] = (long long)vi[t] * vj[t];
            slide4<R, long long>(pr, out);
        }
        store_ll4(xL + (c * RY + ry) * FX + 4 * k, out);
    }
}

// LNCC adjoint x pass on quantised coefficients q [3][RY][RXP] (int64) ->
// xL [3][RY][FX].
template <int R, int RY, int RXP, int NT>
__device__ __forceinline__ void box_x4_adj(const long long *q, long long *xL, int tid) {
    constexpr int ITEMS = 3 * RY * 8, NL = (4 + 2 * R + 1) / 2, NV = 4 + 2 * R;
    static_assert(28 + 2 * NL <= RXP, "row too short for the vector loads");
#pragma unroll
    for (int j = 0; j < (ITEMS + NT - 1) / NT; ++j) {
        const int it = tid + j * NT;
        if (ITEMS % NT != 0 && it >= ITEMS) break;
        const int k = it & 7, rest = it >> 3, ry = rest % RY, c = rest / RY;
        const longlong2 *src = (const longlong2 *)(q + (c * RY + ry) * RXP + 4 * k);
        long long v[2 * NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const longlong2 a = src[l];
            v[2 * l] = a.x;
            v[2 * l + 1] = a.y;
        }
        long long out[4];
        slide4<R, long long>(v, out);
        (void)NV;
        store_ll4(xL + (c * RY + ry) * FX + 4 * k, out);
    }
}

// ====================================================================== K1
// Box channels: J, J^2, I J (the fixed image's S_I and var_I come
// precomputed per level).
template <int R, int NW, int OPT, int NSTG>
struct K1S {
    static constexpr int NT = FX * NW, TY = NW * OPT, RX = FX + 2 * R, RY = TY + 2 * R;
    static constexpr int RXP = pad4(RX), NR = RXP * RY, NS = 2 * R + 1, NOUT = NT * OPT;
    static constexpr size_t o_ring = 0;                                   // [NS][3][NOUT] int64
    static constexpr size_t o_xL = o_ring + (size_t)NS * 3 * NOUT * 8;    // [3][RY][FX] int64
    static constexpr size_t o_os = o_xL + (size_t)3 * RY * FX * 8;        // [NSTG][NOUT] int64 S_I
    static constexpr size_t o_q = o_os + (size_t)NSTG * NOUT * 8;         // [2][RY][RXP] int32
    static constexpr size_t o_st = o_q + (size_t)2 * NR * 4;              // [NSTG][2][RY][RXP] f32
    static constexpr size_t o_ov = o_st + (size_t)NSTG * 2 * NR * 4;      // [NSTG][NOUT] f32 var_I
    static constexpr size_t bytes = o_ov + (size_t)NSTG * NOUT * 4;
};

template <int R, int NW, int OPT, int NSTG>
__global__ void __launch_bounds__(FX *NW) k_lncc_fwd(const float *__restrict__ If,
                                                     const float *__restrict__ J,
                                                     const long long *__restrict__ SIg,
                                                     const float *__restrict__ varIg,
                                                     float *__restrict__ coef,
                                                     WsHeader *__restrict__ h, int D, int H, int W,
                                                     int TZ, int bits, float cc_eps, int window,
                                                     int write_coef) {
    using S = K1S<R, NW, OPT, NSTG>;
    using G = Region<S::RY, S::RX, NW, S::RXP>;
    constexpr int NT = S::NT, TY = S::TY, RX = S::RX, RY = S::RY, RXP = S::RXP, NR = S::NR,
                  NS = S::NS, NOUT = S::NOUT;
    extern __shared__ __align__(16) unsigned char smem[];
    long long *ring = (long long *)(smem + S::o_ring);
    long long *xL = (long long *)(smem + S::o_xL);
    long long *os = (long long *)(smem + S::o_os);
    int *qI = (int *)(smem + S::o_q), *qJ = qI + NR;
    float *st = (float *)(smem + S::o_st);
    float *ov = (float *)(smem + S::o_ov);
    __shared__ float redf[32];
    __shared__ unsigned long long redu[32];

    const int tx = threadIdx.x, wy = threadIdx.y, tid = wy * FX + tx;
    const int x0 = blockIdx.x * FX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int zend = min(z0 + TZ, D);
    const long long N = (long long)D * H * W, HW = (long long)H * W;
    const float amax =
        fmaxf(__uint_as_float(h->absmax_bits[0]), __uint_as_float(h->absmax_bits[1]));
    const int sh = fixed_shift(amax, bits);
    const float scale = pow2f(sh), inv_s = pow2f(-sh);
    const long long n = (long long)window * window * window;
    const float nf = (float)n, inv_nf = 1.0f / nf;
    G rg;
    rg.init(wy, tx, y0 - R, x0 - R, H, W);
    Outs<OPT> ou;
    ou.init(wy, tx, y0, x0, NW, H, W);

    for (int k = tid; k < NS * 3 * NOUT; k += NT) ring[k] = 0;
    long long acc[OPT][3];
#pragma unroll
    for (int o = 0; o < OPT; ++o)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[o][c] = 0;

    const int zs = z0 - R, np = zend - z0 + 2 * R;
    auto issue = [&](int i) {
        if (i < np) {
            const int zp = zs + i, zo = zp - R;
            const bool zok = zp >= 0 && zp < D;
            float *dst = st + (i % NSTG) * 2 * NR;
            load_plane<1, RY, RX, NW, RXP>(dst, If, N, (long long)zp * HW, zok, rg);
            load_plane<1, RY, RX, NW, RXP>(dst + NR, J, N, (long long)zp * HW, zok, rg);
            if (zo >= z0 && zo < zend) {
                const long long zoff = (long long)zo * HW;
#pragma unroll
                for (int o = 0; o < OPT; ++o) {
                    const bool ok = ou.off[o] >= 0;
                    const long long gi = ok ? zoff + ou.off[o] : 0;
                    cp8(os + (i % NSTG) * NOUT + o * NT + tid, SIg + gi, ok);
                    cp4(ov + (i % NSTG) * NOUT + o * NT + tid, varIg + gi, ok);
                }
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int k = 0; k < NSTG - 1; ++k) issue(k);

    unsigned long long qcc = 0;
    float mA = 0.f, mB = 0.f, mC = 0.f;
    bool bad = false;
    int slot = 0;
    for (int i = 0; i < np; ++i) {
        const int zp = zs + i;
        issue(i + NSTG - 1);
        cp_wait<NSTG - 1>();
        long long P[OPT][3];
        if (zp >= 0 && zp < D) {
            const float *sI = st + (i % NSTG) * 2 * NR, *sJ = sI + NR;
#pragma unroll
            for (int j = 0; j < G::NJ; ++j)
#pragma unroll
                for (int c = 0; c < G::NC; ++c) {  // own copies: no barrier needed
                    if (rg.off[j * G::NC + c] == -2) continue;
                    const int k = rg.sbase + G::sofs(j, c);
                    qI[k] = __float2int_rn(sI[k] * scale);
                    qJ[k] = __float2int_rn(sJ[k] * scale);
                }
            __syncthreads();
            box_x4_fwd<R, RY, RXP, NT>(qI, qJ, xL, tid);
            __syncthreads();
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                const long long *xi = xL + (wy + NW * o) * FX + tx;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    long long sum = 0;
#pragma unroll
                    for (int t = 0; t <= 2 * R; ++t) sum += xi[c * RY * FX + t * FX];
                    P[o][c] = sum;
                }
            }
        } else {
#pragma unroll
            for (int o = 0; o < OPT; ++o)
#pragma unroll
                for (int c = 0; c < 3; ++c) P[o][c] = 0;
        }
        long long *rb = ring + slot * 3 * NOUT + tid;
#pragma unroll
        for (int o = 0; o < OPT; ++o)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                long long *r = rb + c * NOUT + o * NT;
                acc[o][c] += P[o][c] - *r;
                *r = P[o][c];
            }
        slot = (slot + 1 == NS) ? 0 : slot + 1;
        const int z = zp - R;
        if (z >= z0 && z < zend) {
            const long long zoff = (long long)z * HW;
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                if (ou.off[o] < 0) continue;
                const long long a1 = os[(i % NSTG) * NOUT + o * NT + tid];  // own copy
                const float varI = ov[(i % NSTG) * NOUT + o * NT + tid];
                const long long a2 = acc[o][0];
                const float varJ = diff_i128_to_float(n, acc[o][1], a2, a2) * inv_s * inv_s * inv_nf;
                const float cross = diff_i128_to_float(n, acc[o][2], a1, a2) * inv_s * inv_s * inv_nf;
                const float den = fmaf(varI, varJ, cc_eps);
                const float rden = __frcp_rn(den);
                const float cc = cross * cross * rden;
                if (cc >= 0.0f && cc <= 2.0f)
                    qcc += (unsigned long long)__float2ull_rn(cc * 4294967296.0f);
                else
                    bad = true;
                if (write_coef) {
                    const float A = 2.0f * cross * rden;
                    const float B = -cc * varI * rden;
                    float Ch, Cl;
                    lncc_c_ff(A, B, a1, a2, inv_s, nf, inv_nf, Ch, Cl);
                    float *cp = coef + zoff + ou.off[o];
                    cp[0] = A;
                    cp[N] = B;
                    cp[2 * N] = Ch;
                    cp[3 * N] = Cl;
                    mA = fmaxf(mA, fabsf(A));
                    mB = fmaxf(mB, fabsf(B));
                    mC = fmaxf(mC, fabsf(Ch));
                }
            }
        }
    }
    cp_wait<0>();
    if (bad) status_set(&h->status, ST_NONFINITE);
    block_sum_to(&h->loss_acc, qcc, redu);
    if (write_coef) {
        block_max_to(&h->coef_max_bits[0], mA, redf);
        block_max_to(&h->coef_max_bits[1], mB, redf);
        block_max_to(&h->coef_max_bits[2], mC, redf);
    }
}

// ====================================================================== K2
template <int R, int NW, int OPT, int NSTG>
struct K2S {
    static constexpr int NT = FX * NW, TY = NW * OPT, RX = FX + 2 * R, RY = TY + 2 * R;
    static constexpr int RXP = pad4(RX), NR = RXP * RY, NS = 2 * R + 1, NOUT = NT * OPT;
    static constexpr size_t o_ring = 0;
    static constexpr size_t o_xL = o_ring + (size_t)NS * 3 * NOUT * 8;
    static constexpr size_t o_q = o_xL + (size_t)3 * RY * FX * 8;
    static constexpr size_t o_st = o_q + (size_t)3 * NR * 8;
    static constexpr size_t o_ost = o_st + (size_t)NSTG * 4 * NR * 4;
    static constexpr size_t bytes = o_ost + (size_t)NSTG * 4 * NOUT * 4;
};

// coef holds A, B and C as a float-float pair (C hi, C lo).
template <int R, int NW, int OPT, int NSTG>
__global__ void __launch_bounds__(FX *NW) k_lncc_grad(const float *__restrict__ If,
                                                      const float *__restrict__ Im,
                                                      const float *__restrict__ u,
                                                      const float *__restrict__ coef,
                                                      const WsHeader *__restrict__ h,
                                                      float *__restrict__ g, int D, int H, int W,
                                                      int TZ, int cbits) {
    using S = K2S<R, NW, OPT, NSTG>;
    using G = Region<S::RY, S::RX, NW, S::RXP>;
    constexpr int NT = S::NT, TY = S::TY, RX = S::RX, RY = S::RY, RXP = S::RXP, NR = S::NR,
                  NS = S::NS, NOUT = S::NOUT;
    extern __shared__ __align__(16) unsigned char smem[];
    long long *ring = (long long *)(smem + S::o_ring);
    long long *xL = (long long *)(smem + S::o_xL);
    long long *q = (long long *)(smem + S::o_q);
    float *st = (float *)(smem + S::o_st);
    float *ost = (float *)(smem + S::o_ost);

    const int tx = threadIdx.x, wy = threadIdx.y, tid = wy * FX + tx;
    const int x0 = blockIdx.x * FX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int zend = min(z0 + TZ, D);
    const long long N = (long long)D * H * W, HW = (long long)H * W;
    float qs[3], us[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int e = fixed_shift(__uint_as_float(h->coef_max_bits[c]), cbits);
        qs[c] = pow2f(e);
        us[c] = pow2f(-e);
    }
    const float inv_n = 1.0f / (float)N;
    G rg;
    rg.init(wy, tx, y0 - R, x0 - R, H, W);
    Outs<OPT> ou;
    ou.init(wy, tx, y0, x0, NW, H, W);

    for (int k = tid; k < NS * 3 * NOUT; k += NT) ring[k] = 0;
    long long acc[OPT][3];
#pragma unroll
    for (int o = 0; o < OPT; ++o)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[o][c] = 0;

    const int zs = z0 - R, np = zend - z0 + 2 * R;
    auto issue = [&](int i) {
        if (i < np) {
            const int zp = zs + i, zo = zp - R;
            load_plane<4, RY, RX, NW, RXP>(st + (i % NSTG) * 4 * NR, coef, N, (long long)zp * HW,
                                           zp >= 0 && zp < D, rg);
            if (zo >= z0 && zo < zend) {
                float *o = ost + (i % NSTG) * 4 * NOUT;
                load_outs<3, OPT, NOUT>(o, u, N, (long long)zo * HW, ou, tid, NT);
                load_outs<1, OPT, NOUT>(o + 3 * NOUT, If, N, (long long)zo * HW, ou, tid, NT);
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int k = 0; k < NSTG - 1; ++k) issue(k);

    int slot = 0;
    for (int i = 0; i < np; ++i) {
        const int zp = zs + i, zo = zp - R;
        issue(i + NSTG - 1);
        cp_wait<NSTG - 1>();
        const bool out = zo >= z0 && zo < zend;
        // gathers for this plane's outputs, consumed after the reductions
        TriPending tp[OPT];
        float Iv[OPT];
        if (out) {
            const float *o = ost + (i % NSTG) * 4 * NOUT + tid;
#pragma unroll
            for (int k = 0; k < OPT; ++k) {
                tri_issue(tp[k], Im, D, H, W, zo, y0 + wy + NW * k, x0 + tx, o[k * NT],
                          o[NOUT + k * NT], o[2 * NOUT + k * NT]);
                Iv[k] = o[3 * NOUT + k * NT];
            }
        }
        long long P[OPT][3];
        if (zp >= 0 && zp < D) {
            const float *s = st + (i % NSTG) * 4 * NR;
#pragma unroll
            for (int j = 0; j < G::NJ; ++j)
#pragma unroll
                for (int c = 0; c < G::NC; ++c) {  // own copies
                    if (rg.off[j * G::NC + c] == -2) continue;
                    const int k = rg.sbase + G::sofs(j, c);
                    q[k] = quantize(s[k], qs[0]);
                    q[NR + k] = quantize(s[NR + k], qs[1]);
                    q[2 * NR + k] = quantize(s[2 * NR + k], qs[2]) + quantize(s[3 * NR + k], qs[2]);
                }
            __syncthreads();
            box_x4_adj<R, RY, RXP, NT>(q, xL, tid);
            __syncthreads();
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                const long long *xi = xL + (wy + NW * o) * FX + tx;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    long long sum = 0;
#pragma unroll
                    for (int t = 0; t <= 2 * R; ++t) sum += xi[c * RY * FX + t * FX];
                    P[o][c] = sum;
                }
            }
        } else {
#pragma unroll
            for (int o = 0; o < OPT; ++o)
#pragma unroll
                for (int c = 0; c < 3; ++c) P[o][c] = 0;
        }
        long long *rb = ring + slot * 3 * NOUT + tid;
#pragma unroll
        for (int o = 0; o < OPT; ++o)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                long long *r = rb + c * NOUT + o * NT;
                acc[o][c] += P[o][c] - *r;
                *r = P[o][c];
            }
        slot = (slot + 1 == NS) ? 0 : slot + 1;
        if (out) {
            const long long zoff = (long long)zo * HW;
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                if (ou.off[o] < 0) continue;
                float gz, gy, gx;
                const float Jv = tri_finish<true>(tp[o], gz, gy, gx);
                float ah, al, bh, bl, ch, cl, rh, rl, th, tl;
                i64_to_ff(acc[o][0], ah, al);
                i64_to_ff(acc[o][1], bh, bl);
                i64_to_ff(acc[o][2], ch, cl);
                ff_mul_f(Iv[o], ah * us[0], al * us[0], rh, rl);       // I SA
                ff_mul_f(2.0f * Jv, bh * us[1], bl * us[1], th, tl);   // 2 J SB
                ff_add(rh, rl, th, tl);
                ff_add(rh, rl, ch * us[2], cl * us[2]);                // + SC
                const float dj = -(rh + rl) * inv_n;
                float *gp = g + zoff + ou.off[o];
                gp[0] = dj * gz;
                gp[N] = dj * gy;
                gp[2 * N] = dj * gx;
            }
        }
    }
    cp_wait<0>();
}

// MSE: g = 2 (J - I) / N * grad I_m o phi (pointwise).
__global__ void __launch_bounds__(256) k_fused_mse_grad(const float *__restrict__ If,
                                                        const float *__restrict__ Im,
                                                        const float *__restrict__ u,
                                                        float *__restrict__ g, int D, int H,
                                                        int W) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    if (x >= W || y >= H) return;
    long long N = (long long)D * H * W;
    long long i = ((long long)z * H + y) * W + x;
    float gz, gy, gx;
    float Jv = tri_sample<true>(Im, D, H, W, z, y, x, __ldg(u + i), __ldg(u + N + i),
                                __ldg(u + 2 * N + i), gz, gy, gx);
    float dj = 2.0f * (Jv - __ldg(If + i)) / (float)N;
    g[i] = dj * gz;
    g[N + i] = dj * gy;
    g[2 * N + i] = dj * gx;
}

// ====================================================== separable Gaussian
// x pass of a [3][RY][RXP] plane onto [3][RY][FX] and this thread's y pass.
template <int RG, int RY, int RXP, int NW, int OPT>
__device__ __forceinline__ void gauss_xy(const float *pl, float *xb, const GaussTaps &t, int wy,
                                         int tx, float Q[OPT][3]) {
    gauss_x4<RG, 3, RY, RXP, FX * NW>(pl, xb, t, wy * FX + tx);
    __syncthreads();
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
        const float *xi = xb + (wy + NW * o) * FX + tx;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k <= 2 * RG; ++k) s = fmaf(t.w[k], xi[c * RY * FX + k * FX], s);
            Q[o][c] = s;
        }
    }
}

// Ring of the last NS in-plane results, every slot stored twice (k, k + NS)
// so that the z window is contiguous.  Writes plane results at `slot` and
// returns the first slot of the window (oldest plane first).
template <int NS, int OPT, int NOUT, int NT>
__device__ __forceinline__ int ring_push(float *ring, int slot, int tid, const float Q[OPT][3]) {
#pragma unroll
    for (int o = 0; o < OPT; ++o)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = Q[o][c];
            ring[(slot * 3 + c) * NOUT + o * NT + tid] = v;
            ring[((slot + NS) * 3 + c) * NOUT + o * NT + tid] = v;
        }
    return slot + 1;  // window slots slot+1 .. slot+NS
}

template <int RG, int NOUT>
__device__ __forceinline__ float gauss_z(const float *win, const GaussTaps &t, int c) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k <= 2 * RG; ++k) s = fmaf(t.w[k], win[(k * 3 + c) * NOUT], s);
    return s;
}

// ====================================================================== K3
template <int RG, int NW, int OPT, int NSTG>
struct K3S {
    static constexpr int NT = FX * NW, TY = NW * OPT, RX = FX + 2 * RG, RY = TY + 2 * RG;
    static constexpr int RXP = pad4(RX), NR = RXP * RY, NS = 2 * RG + 1, NOUT = NT * OPT;
    static constexpr size_t o_ring = 0;
    static constexpr size_t o_xb = o_ring + (size_t)2 * NS * 3 * NOUT * 4;
    static constexpr size_t o_st = o_xb + (size_t)3 * RY * FX * 4;
    static constexpr size_t o_mv = o_st + (size_t)NSTG * 3 * NR * 4;
    static constexpr size_t bytes = o_mv + (size_t)NSTG * 6 * NOUT * 4;
};

template <int RG, int NW, int OPT, int NSTG>
__global__ void __launch_bounds__(FX *NW) k_smooth_adam(const float *__restrict__ g,
                                                        float *__restrict__ m,
                                                        float *__restrict__ v,
                                                        float *__restrict__ dir,
                                                        WsHeader *__restrict__ h, int D, int H,
                                                        int W, int TZ, GaussTaps t, AdamConsts ac,
                                                        int parity) {
    using S = K3S<RG, NW, OPT, NSTG>;
    using G = Region<S::RY, S::RX, NW, S::RXP>;
    constexpr int NT = S::NT, TY = S::TY, RX = S::RX, RY = S::RY, RXP = S::RXP, NR = S::NR,
                  NS = S::NS, NOUT = S::NOUT;
    extern __shared__ __align__(16) unsigned char smem[];
    float *ring = (float *)(smem + S::o_ring);
    float *xb = (float *)(smem + S::o_xb);
    float *st = (float *)(smem + S::o_st);
    float *mvs = (float *)(smem + S::o_mv);
    __shared__ float redf[32];

    const int tx = threadIdx.x, wy = threadIdx.y, tid = wy * FX + tx;
    const int x0 = blockIdx.x * FX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int zend = min(z0 + TZ, D);
    const long long N = (long long)D * H * W, HW = (long long)H * W;
    G rg;
    rg.init(wy, tx, y0 - RG, x0 - RG, H, W);
    Outs<OPT> ou;
    ou.init(wy, tx, y0, x0, NW, H, W);
    for (int k = tid; k < 2 * NS * 3 * NOUT; k += NT) ring[k] = 0.0f;

    const int zs = z0 - RG, np = zend - z0 + 2 * RG;
    auto issue = [&](int i) {
        if (i < np) {
            const int zp = zs + i, zo = zp - RG;
            load_plane<3, RY, RX, NW, RXP>(st + (i % NSTG) * 3 * NR, g, N, (long long)zp * HW,
                                           zp >= 0 && zp < D, rg);
            if (zo >= z0 && zo < zend) {
                float *o = mvs + (i % NSTG) * 6 * NOUT;
                load_outs<3, OPT, NOUT>(o, m, N, (long long)zo * HW, ou, tid, NT);
                load_outs<3, OPT, NOUT>(o + 3 * NOUT, v, N, (long long)zo * HW, ou, tid, NT);
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int k = 0; k < NSTG - 1; ++k) issue(k);

    float mx = 0.0f;
    bool bad = false;
    int slot = 0;
    for (int i = 0; i < np; ++i) {
        const int zp = zs + i, zo = zp - RG;
        issue(i + NSTG - 1);
        cp_wait<NSTG - 1>();
        float Q[OPT][3];
        if (zp >= 0 && zp < D) {
            __syncthreads();  // the x pass reads neighbours' copies
            gauss_xy<RG, RY, RXP, NW, OPT>(st + (i % NSTG) * 3 * NR, xb, t, wy, tx, Q);
        } else {
#pragma unroll
            for (int o = 0; o < OPT; ++o) Q[o][0] = Q[o][1] = Q[o][2] = 0.0f;
        }
        const int wbase = ring_push<NS, OPT, NOUT, NT>(ring, slot, tid, Q);
        slot = (slot + 1 == NS) ? 0 : slot + 1;
        if (zo >= z0 && zo < zend) {
            const float *mv = mvs + (i % NSTG) * 6 * NOUT + tid;
            const long long zoff = (long long)zo * HW;
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                if (ou.off[o] < 0) continue;
                const float *win = ring + wbase * 3 * NOUT + o * NT + tid;
                const long long gi = zoff + ou.off[o];
                float nrm2 = 0.0f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float s = gauss_z<RG, NOUT>(win, t, c);
                    const float mvv = fmaf(ac.b1, mv[c * NOUT + o * NT], (1.0f - ac.b1) * s);
                    const float vvv =
                        fmaf(ac.b2, mv[(3 + c) * NOUT + o * NT], (1.0f - ac.b2) * s * s);
                    m[c * N + gi] = mvv;
                    v[c * N + gi] = vvv;
                    const float dv = adam_dir(mvv, vvv, ac.rbc1, ac.rbc2, ac.eps);
                    dir[c * N + gi] = dv;
                    nrm2 = fmaf(dv, dv, nrm2);
                }
                if (nrm2 <= 3.4e38f)
                    mx = fmaxf(mx, sqrtf(nrm2));
                else
                    bad = true;
            }
        }
    }
    cp_wait<0>();
    if (bad) status_set(&h->status, ST_NONFINITE);
    block_max_to(&h->step_max_bits[parity], mx, redf);
}

// ====================================================================== K4
// SU: u is staged in shared memory (planes z-1..z+1, halo RG + 1); valid when
// the step is shorter than one voxel (lr / c_lp < 1).
template <int RG, int NW, int OPT, bool SU, int NSTG>
struct K4S {
    static constexpr int NT = FX * NW, TY = NW * OPT, RX = FX + 2 * RG, RY = TY + 2 * RG;
    static constexpr int RXP = pad4(RX), NR = RXP * RY, NS = 2 * RG + 1, NOUT = NT * OPT;
    // u planes z-1, z, z+1 in use plus NSTG - 1 in flight
    static constexpr int URX = RX + 2, URY = RY + 2, URXP = pad4(URX), NRU = URXP * URY,
                         NSU = NSTG + 2;
    static constexpr size_t o_ring = 0;
    static constexpr size_t o_xb = o_ring + (size_t)2 * NS * 3 * NOUT * 4;
    static constexpr size_t o_up = o_xb + (size_t)3 * RY * FX * 4;
    static constexpr size_t o_dst = o_up + (size_t)3 * NR * 4;
    static constexpr size_t o_ust = o_dst + (size_t)NSTG * 3 * NR * 4;
    static constexpr size_t bytes = o_ust + (SU ? (size_t)NSU * 3 * NRU * 4 : 0);
};

template <int RG, int NW, int OPT, bool SU, int NSTG>
__global__ void __launch_bounds__(FX *NW) k_compose(const float *__restrict__ u,
                                                    const float *__restrict__ dir,
                                                    float *__restrict__ uo,
                                                    const float *__restrict__ Im,
                                                    float *__restrict__ Jout,
                                                    WsHeader *__restrict__ h, int D, int H, int W,
                                                    int TZ, GaussTaps t, float lr, float c_lp,
                                                    int parity) {
    using S = K4S<RG, NW, OPT, SU, NSTG>;
    using G = Region<S::RY, S::RX, NW, S::RXP>;
    using GU = Region<S::URY, S::URX, NW, S::URXP>;
    constexpr int NT = S::NT, TY = S::TY, RX = S::RX, RY = S::RY, RXP = S::RXP, NR = S::NR,
                  NS = S::NS, NOUT = S::NOUT, URX = S::URX, URY = S::URY, URXP = S::URXP,
                  NRU = S::NRU, NSU = S::NSU;
    extern __shared__ __align__(16) unsigned char smem[];
    float *ring = (float *)(smem + S::o_ring);
    float *xb = (float *)(smem + S::o_xb);
    float *up = (float *)(smem + S::o_up);
    float *dst = (float *)(smem + S::o_dst);
    float *ust = (float *)(smem + S::o_ust);

    const int tx = threadIdx.x, wy = threadIdx.y, tid = wy * FX + tx;
    const int x0 = blockIdx.x * FX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int zend = min(z0 + TZ, D);
    const long long N = (long long)D * H * W, HW = (long long)H * W;
    const float mxd = __uint_as_float(h->step_max_bits[parity]);
    const float e = (mxd > 0.0f) ? lr / (c_lp * mxd) : 0.0f;
    G rg;
    rg.init(wy, tx, y0 - RG, x0 - RG, H, W);
    GU rgu;
    if (SU) rgu.init(wy, tx, y0 - RG - 1, x0 - RG - 1, H, W);
    Outs<OPT> ou;
    ou.init(wy, tx, y0, x0, NW, H, W);
    for (int k = tid; k < 2 * NS * 3 * NOUT; k += NT) ring[k] = 0.0f;

    const int zs = z0 - RG, np = zend - z0 + 2 * RG;
    // u plane q lives in stage (q - (zs - 1)) % NSU
    auto issue_u = [&](int q) {
        load_plane<3, URY, URX, NW, URXP>(ust + ((q - (zs - 1)) % NSU) * 3 * NRU, u, N,
                                          (long long)q * HW, q >= 0 && q < D, rgu);
    };
    auto issue = [&](int i) {
        if (i < np) {
            const int zp = zs + i;
            load_plane<3, RY, RX, NW, RXP>(dst + (i % NSTG) * 3 * NR, dir, N,
                                           (long long)zp * HW, zp >= 0 && zp < D, rg);
            if (SU) issue_u(zp + 1);
        }
        cp_commit();
    };
    if (SU) {
        issue_u(zs - 1);
        issue_u(zs);
    }
#pragma unroll
    for (int k = 0; k < NSTG - 1; ++k) issue(k);  // the u planes above join group 0

    TriPending jp[OPT];
    long long jidx[OPT];
    bool jlive[OPT];
#pragma unroll
    for (int o = 0; o < OPT; ++o) jlive[o] = false;

    int slot = 0;
    for (int i = 0; i < np; ++i) {
        const int zp = zs + i, zo = zp - RG;
        issue(i + NSTG - 1);
        cp_wait<NSTG - 1>();
        float Q[OPT][3];
        if (zp >= 0 && zp < D) {
            if (SU) __syncthreads();  // u stages hold neighbours' copies
            const float *ds = dst + (i % NSTG) * 3 * NR;
            const float *um = ust + ((zp - 1 - (zs - 1)) % NSU) * 3 * NRU;
            const float *u0 = ust + ((zp - (zs - 1)) % NSU) * 3 * NRU;
            const float *u1 = ust + ((zp + 1 - (zs - 1)) % NSU) * 3 * NRU;
#pragma unroll
            for (int j = 0; j < G::NJ; ++j)
#pragma unroll
                for (int cc = 0; cc < G::NC; ++cc) {  // own copies of d
                    const int o = rg.off[j * G::NC + cc];
                    if (o == -2) continue;
                    const int k = rg.sbase + G::sofs(j, cc);
                    float a = 0.f, b = 0.f, c = 0.f;
                    if (o >= 0) {
                        const float dz = -e * ds[k], dy = -e * ds[NR + k], dx = -e * ds[2 * NR + k];
                        if (SU) {
                            // cell corners lie within one voxel: planes zp-1..zp+1
                            if (dz > -1.0f && dz < 1.0f && dy > -1.0f && dy < 1.0f &&
                                dx > -1.0f && dx < 1.0f) {
                                const float fz = floorf(dz), fy = floorf(dy), fx = floorf(dx);
                                const float tz = dz - fz, ty = dy - fy, tx2 = dx - fx;
                                const float *pa = fz < 0.0f ? um : u0;
                                const float *pb = fz < 0.0f ? u0 : u1;
                                const int ry = wy + NW * j, rx = tx + 32 * cc;
                                const int b0 = (ry + 1 + (int)fy) * URXP + (rx + 1 + (int)fx);
                                float r[3];
#pragma unroll
                                for (int ch = 0; ch < 3; ++ch) {
                                    const float *A = pa + ch * NRU + b0, *B = pb + ch * NRU + b0;
                                    const float c00 = fmaf(tx2, A[1] - A[0], A[0]);
                                    const float c01 = fmaf(tx2, A[URXP + 1] - A[URXP], A[URXP]);
                                    const float c10 = fmaf(tx2, B[1] - B[0], B[0]);
                                    const float c11 = fmaf(tx2, B[URXP + 1] - B[URXP], B[URXP]);
                                    const float c0 = fmaf(ty, c01 - c00, c00);
                                    const float c1 = fmaf(ty, c11 - c10, c10);
                                    r[ch] = fmaf(tz, c1 - c0, c0);
                                }
                                a = dz + r[0];
                                b = dy + r[1];
                                c = dx + r[2];
                            } else {
                                a = b = c = __int_as_float(0x7fc00000);  // impossible step: flag it
                            }
                        } else {
                            const int y = y0 - RG + wy + NW * j, x = x0 - RG + tx + 32 * cc;
                            float gz, gy, gx;
                            a = dz + tri_sample<false>(u, D, H, W, zp, y, x, dz, dy, dx, gz, gy, gx);
                            b = dy + tri_sample<false>(u + N, D, H, W, zp, y, x, dz, dy, dx, gz, gy,
                                                       gx);
                            c = dx + tri_sample<false>(u + 2 * N, D, H, W, zp, y, x, dz, dy, dx, gz,
                                                       gy, gx);
                        }
                    }
                    up[k] = a;
                    up[NR + k] = b;
                    up[2 * NR + k] = c;
                }
            __syncthreads();
            gauss_xy<RG, RY, RXP, NW, OPT>(up, xb, t, wy, tx, Q);
        } else {
#pragma unroll
            for (int o = 0; o < OPT; ++o) Q[o][0] = Q[o][1] = Q[o][2] = 0.0f;
        }
        const int wbase = ring_push<NS, OPT, NOUT, NT>(ring, slot, tid, Q);
        slot = (slot + 1 == NS) ? 0 : slot + 1;
        if (zo >= z0 && zo < zend) {
            const long long zoff = (long long)zo * HW;
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                // finish the previous plane's warped value first (its loads have landed)
                if (jlive[o]) {
                    float gz, gy, gx;
                    Jout[jidx[o]] = tri_finish<false>(jp[o], gz, gy, gx);
                    jlive[o] = false;
                }
                if (ou.off[o] < 0) continue;
                const float *win = ring + wbase * 3 * NOUT + o * NT + tid;
                const long long gi = zoff + ou.off[o];
                const float a = gauss_z<RG, NOUT>(win, t, 0);
                const float b = gauss_z<RG, NOUT>(win, t, 1);
                const float c = gauss_z<RG, NOUT>(win, t, 2);
                uo[gi] = a;
                uo[N + gi] = b;
                uo[2 * N + gi] = c;
                tri_issue(jp[o], Im, D, H, W, zo, y0 + wy + NW * o, x0 + tx, a, b, c);
                jidx[o] = gi;
                jlive[o] = true;
            }
        }
    }
#pragma unroll
    for (int o = 0; o < OPT; ++o)
        if (jlive[o]) {
            float gz, gy, gx;
            Jout[jidx[o]] = tri_finish<false>(jp[o], gz, gy, gx);
        }
    cp_wait<0>();
    // per-iteration header fields for the next iteration (nobody else reads them now)
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tid == 0) {
        for (int c = 0; c < 8; ++c) h->coef_max_bits[c] = 0u;
        h->step_max_bits[parity ^ 1] = 0u;
        h->loss_acc = 0ull;
        h->eps_t = e;
    }
}

// ================================================================ launching

std::mutex g_mu;
int g_num_sms = 0;

int num_sms() {
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_num_sms == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            g_num_sms = n;
        else
            g_num_sms = 152;
    }
    return g_num_sms;
}

// Slab depth TZ minimising (waves x planes per CTA) for a z-marching kernel.
int choose_tz(int D, int tiles_xy, int halo, int ctas_per_sm) {
    const long long slots = (long long)num_sms() * (ctas_per_sm > 0 ? ctas_per_sm : 1);
    int best = D;
    long long bestcost = -1;
    for (int tz = 1; tz <= D && tz <= 64; ++tz) {
        const long long ctas = (long long)tiles_xy * ((D + tz - 1) / tz);
        const long long waves = (ctas + slots - 1) / slots;
        const long long cost = waves * (tz + 2 * halo);
        if (bestcost < 0 || cost < bestcost) {
            bestcost = cost;
            best = tz;
        }
    }
    return best;
}

// Opts the kernel into its dynamic shared memory and returns its resident
// CTAs per SM (called once per kernel instantiation).
template <class K>
int prepare(K kernel, size_t smem, int threads) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess ||
        n < 1)
        n = 1;
    return n;
}

struct LaunchGeom {
    dim3 grid, block;
    int tz;
};

inline LaunchGeom geometry(int occ, int nw, int ty, int halo, Dims d) {
    LaunchGeom g;
    const int gx = (d.W + FX - 1) / FX, gy = (d.H + ty - 1) / ty;
    g.tz = choose_tz(d.D, gx * gy, halo, occ);
    g.grid = dim3(gx, gy, (d.D + g.tz - 1) / g.tz);
    g.block = dim3(FX, nw);
    return g;
}

// tile shapes (warps per CTA, outputs per thread along y) and pipeline depth
constexpr int K1_NW = 8, K1_OPT = 1, K1_ST = 3;
constexpr int K2_NW = 8, K2_OPT = 1, K2_ST = 2;
constexpr int K3_NW = 8, K3_OPT = 1, K3_ST = 2;
constexpr int K4_NW = 8, K4_OPT = 1, K4_ST = 2;

template <int R>
cudaError_t launch_k1(const float *If, const float *J, const long long *sI, const float *varI,
                      float *coef, WsHeader *h, Dims d, int window, float cc_eps, bool wc,
                      cudaStream_t s) {
    using S = K1S<R, K1_NW, K1_OPT, K1_ST>;
    auto kern = k_lncc_fwd<R, K1_NW, K1_OPT, K1_ST>;
    static const int occ = prepare(kern, S::bytes, S::NT);
    LaunchGeom g = geometry(occ, K1_NW, S::TY, R, d);
    kern<<<g.grid, g.block, S::bytes, s>>>(If, J, sI, varI, coef, h, d.D, d.H, d.W, g.tz,
                                           lncc_image_bits(window), cc_eps, window, wc ? 1 : 0);
    note_launch();
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_k2(const float *If, const float *Im, const float *u, const float *coef,
                      const WsHeader *h, float *g, Dims d, int window, cudaStream_t s) {
    using S = K2S<R, K2_NW, K2_OPT, K2_ST>;
    auto kern = k_lncc_grad<R, K2_NW, K2_OPT, K2_ST>;
    static const int occ = prepare(kern, S::bytes, S::NT);
    LaunchGeom gg = geometry(occ, K2_NW, S::TY, R, d);
    kern<<<gg.grid, gg.block, S::bytes, s>>>(If, Im, u, coef, h, g, d.D, d.H, d.W, gg.tz,
                                             lncc_coef_bits(window));
    note_launch();
    return cudaGetLastError();
}

template <int RG>
cudaError_t launch_k3(const float *g, float *m, float *v, float *dir, WsHeader *h, Dims d,
                      const GaussTaps &t, AdamConsts ac, int parity, cudaStream_t s) {
    using S = K3S<RG, K3_NW, K3_OPT, K3_ST>;
    auto kern = k_smooth_adam<RG, K3_NW, K3_OPT, K3_ST>;
    static const int occ = prepare(kern, S::bytes, S::NT);
    LaunchGeom gg = geometry(occ, K3_NW, S::TY, RG, d);
    kern<<<gg.grid, gg.block, S::bytes, s>>>(g, m, v, dir, h, d.D, d.H, d.W, gg.tz, t, ac, parity);
    note_launch();
    return cudaGetLastError();
}

template <int RG, bool SU>
cudaError_t launch_k4(const float *u, const float *dir, float *uo, const float *Im, float *J,
                      WsHeader *h, Dims d, const GaussTaps &t, float lr, float c_lp, int parity,
                      cudaStream_t s) {
    using S = K4S<RG, K4_NW, K4_OPT, SU, K4_ST>;
    auto kern = k_compose<RG, K4_NW, K4_OPT, SU, K4_ST>;
    static const int occ = prepare(kern, S::bytes, S::NT);
    LaunchGeom gg = geometry(occ, K4_NW, S::TY, RG, d);
    kern<<<gg.grid, gg.block, S::bytes, s>>>(u, dir, uo, Im, J, h, d.D, d.H, d.W, gg.tz, t, lr,
                                             c_lp, parity);
    note_launch();
    return cudaGetLastError();
}

#define FA_CASE(n, call)      \
    case n: {                 \
        constexpr int RR = n; \
        return call;          \
    }

cudaError_t dispatch_k1(const float *If, const float *J, const long long *sI, const float *varI,
                        float *coef, WsHeader *h, Dims d, int window, float cc_eps, bool wc,
                        cudaStream_t s) {
    switch (window / 2) {
        FA_CASE(0, (launch_k1<RR>(If, J, sI, varI, coef, h, d, window, cc_eps, wc, s)))
        FA_CASE(1, (launch_k1<RR>(If, J, sI, varI, coef, h, d, window, cc_eps, wc, s)))
        FA_CASE(2, (launch_k1<RR>(If, J, sI, varI, coef, h, d, window, cc_eps, wc, s)))
        FA_CASE(3, (launch_k1<RR>(If, J, sI, varI, coef, h, d, window, cc_eps, wc, s)))
        FA_CASE(4, (launch_k1<RR>(If, J, sI, varI, coef, h, d, window, cc_eps, wc, s)))
        FA_CASE(5, (launch_k1<RR>(If, J, sI, varI, coef, h, d, window, cc_eps, wc, s)))
        FA_CASE(6, (launch_k1<RR>(If, J, sI, varI, coef, h, d, window, cc_eps, wc, s)))
        FA_CASE(7, (launch_k1<RR>(If, J, sI, varI, coef, h, d, window, cc_eps, wc, s)))
    }
    return cudaErrorInvalidValue;
}

cudaError_t dispatch_k2(const float *If, const float *Im, const float *u, const float *coef,
                        const WsHeader *h, float *g, Dims d, int window, cudaStream_t s) {
    switch (window / 2) {
        FA_CASE(0, (launch_k2<RR>(If, Im, u, coef, h, g, d, window, s)))
        FA_CASE(1, (launch_k2<RR>(If, Im, u, coef, h, g, d, window, s)))
        FA_CASE(2, (launch_k2<RR>(If, Im, u, coef, h, g, d, window, s)))
        FA_CASE(3, (launch_k2<RR>(If, Im, u, coef, h, g, d, window, s)))
        FA_CASE(4, (launch_k2<RR>(If, Im, u, coef, h, g, d, window, s)))
        FA_CASE(5, (launch_k2<RR>(If, Im, u, coef, h, g, d, window, s)))
        FA_CASE(6, (launch_k2<RR>(If, Im, u, coef, h, g, d, window, s)))
        FA_CASE(7, (launch_k2<RR>(If, Im, u, coef, h, g, d, window, s)))
    }
    return cudaErrorInvalidValue;
}

constexpr int kMaxFusedRG = 6;

cudaError_t dispatch_k3(const float *g, float *m, float *v, float *dir, WsHeader *h, Dims d,
                        const GaussTaps &t, AdamConsts ac, int parity, cudaStream_t s) {
    switch (t.R) {
        FA_CASE(0, (launch_k3<RR>(g, m, v, dir, h, d, t, ac, parity, s)))
        FA_CASE(1, (launch_k3<RR>(g, m, v, dir, h, d, t, ac, parity, s)))
        FA_CASE(2, (launch_k3<RR>(g, m, v, dir, h, d, t, ac, parity, s)))
        FA_CASE(3, (launch_k3<RR>(g, m, v, dir, h, d, t, ac, parity, s)))
        FA_CASE(4, (launch_k3<RR>(g, m, v, dir, h, d, t, ac, parity, s)))
        FA_CASE(5, (launch_k3<RR>(g, m, v, dir, h, d, t, ac, parity, s)))
        FA_CASE(6, (launch_k3<RR>(g, m, v, dir, h, d, t, ac, parity, s)))
    }
    return cudaErrorInvalidValue;
}

cudaError_t dispatch_k4(const float *u, const float *dir, float *uo, const float *Im, float *J,
                        WsHeader *h, Dims d, const GaussTaps &t, float lr, float c_lp, int parity,
                        bool su, cudaStream_t s) {
    if (su) {
        switch (t.R) {
            FA_CASE(0, (launch_k4<RR, true>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(1, (launch_k4<RR, true>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(2, (launch_k4<RR, true>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(3, (launch_k4<RR, true>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(4, (launch_k4<RR, true>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(5, (launch_k4<RR, true>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(6, (launch_k4<RR, true>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
        }
    } else {
        switch (t.R) {
            FA_CASE(0, (launch_k4<RR, false>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(1, (launch_k4<RR, false>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(2, (launch_k4<RR, false>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(3, (launch_k4<RR, false>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(4, (launch_k4<RR, false>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(5, (launch_k4<RR, false>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(6, (launch_k4<RR, false>(u, dir, uo, Im, J, h, d, t, lr, c_lp, parity, s)))
        }
    }
    return cudaErrorInvalidValue;
}
#undef FA_CASE

struct KTimer {
    fa_kernel_timer *t;
    int level;
    bool on(int id) const {
        return t && t->kernel_id == id && (t->level < 0 || t->level == level) &&
               t->count < t->capacity;
    }
};

}  // namespace

void fused_carve(WsCarver &c, long long n, FusedBuffers *fb) {
    fb->coef = c.take<float>(4 * n);  // also the first int64 scratch of the fixed statistics
    fb->g = c.take<float>(4 * n);     // also the second one
    fb->dir = c.take<float>(3 * n);
    fb->J = c.take<float>(n);
    fb->t1 = c.take<float>(3 * n);
    fb->t2 = c.take<float>(3 * n);
    fb->sI = c.take<long long>(n);
    fb->varI = c.take<float>(n);
}

cudaError_t fused_level_start(const float *If, const float *Im, const float *u, Dims d,
                              const fa_params *p, const WsHeader *h, FusedBuffers &fb,
                              cudaStream_t s) {
    if (p->loss == FA_LOSS_LNCC) {
        cudaError_t e = launch_fixed_stats(If, d, p->window, h, (long long *)fb.coef,
                                           (long long *)fb.g, fb.sI, fb.varI, s);
        if (e != cudaSuccess) return e;
    }
    return launch_warp(Im, u, fb.J, nullptr, d, s);
}

fa_status fused_iteration(FusedBuffers &fb, WsHeader *h, const fa_params *p, Dims d,
                          const FusedIter &it, const GaussTaps &tg, const GaussTaps &tw,
                          fa_kernel_timer *timer, int level, cudaStream_t s) {
    KTimer kt{timer, level};
    auto start = [&](int id) -> cudaError_t {
        return kt.on(id) ? cudaEventRecord((cudaEvent_t)timer->start_events[timer->count], s)
                         : cudaSuccess;
    };
    auto stop = [&](int id) -> cudaError_t {
        if (!kt.on(id)) return cudaSuccess;
        cudaError_t e = cudaEventRecord((cudaEvent_t)timer->stop_events[timer->count], s);
        timer->count++;
        return e;
    };
    const int parity = it.t & 1;
    if (p->loss == FA_LOSS_LNCC) {
        FA_CUDA_TRY(start(FA_K_FUSED_WARP_LNCC));
        FA_CUDA_TRY(dispatch_k1(it.If, fb.J, fb.sI, fb.varI, fb.coef, h, d, p->window, p->cc_eps,
                                true, s));
        FA_CUDA_TRY(stop(FA_K_FUSED_WARP_LNCC));
        FA_CUDA_TRY(start(FA_K_FUSED_LNCC_GRAD));
        FA_CUDA_TRY(dispatch_k2(it.If, it.Im, it.u, fb.coef, h, fb.g, d, p->window, s));
        FA_CUDA_TRY(stop(FA_K_FUSED_LNCC_GRAD));
    } else {
        VoxGrid gg(d.D, d.H, d.W);
        FA_CUDA_TRY(start(FA_K_FUSED_LNCC_GRAD));
        k_fused_mse_grad<<<gg.grid, gg.block, 0, s>>>(it.If, it.Im, it.u, fb.g, d.D, d.H, d.W);
        note_launch();
        FA_CUDA_TRY(cudaGetLastError());
        FA_CUDA_TRY(stop(FA_K_FUSED_LNCC_GRAD));
    }
    // Gaussians wider than the fused kernels' rings run as separable passes
    // around the identity-width fused kernel.
    static const GaussTaps ident = [] {
        GaussTaps t;
        make_gauss_taps(0.0f, &t);
        return t;
    }();
    const bool wide_g = tg.R > kMaxFusedRG, wide_w = tw.R > kMaxFusedRG;
    // the compose reads u from shared memory when every step is under a voxel
    const bool su = (double)p->lr / (double)p->c_lp < 0.999;
    if (wide_g) FA_CUDA_TRY(launch_gauss3(fb.g, fb.g, fb.t1, fb.t2, 3, d, tg, s));
    FA_CUDA_TRY(start(FA_K_FUSED_SMOOTH_ADAM));
    FA_CUDA_TRY(dispatch_k3(fb.g, it.m, it.v, fb.dir, h, d, wide_g ? ident : tg,
                            adam_consts(p, it.t), parity, s));
    FA_CUDA_TRY(stop(FA_K_FUSED_SMOOTH_ADAM));
    FA_CUDA_TRY(start(FA_K_FUSED_COMPOSE));
    FA_CUDA_TRY(dispatch_k4(it.u, fb.dir, it.u_alt, it.Im, fb.J, h, d, wide_w ? ident : tw, p->lr,
                            p->c_lp, parity, su, s));
    FA_CUDA_TRY(stop(FA_K_FUSED_COMPOSE));
    if (wide_w) {
        FA_CUDA_TRY(launch_gauss3(it.u_alt, it.u_alt, fb.t1, fb.t2, 3, d, tw, s));
        FA_CUDA_TRY(launch_warp(it.Im, it.u_alt, fb.J, nullptr, d, s));  // J of the smoothed map
    }
    return FA_OK;
}

cudaError_t fused_lncc_forward_only(const float *If, const FusedBuffers &fb, Dims d, int window,
                                    float cc_eps, WsHeader *h, cudaStream_t s) {
    return dispatch_k1(If, fb.J, fb.sI, fb.varI, nullptr, h, d, window, cc_eps, false, s);
}

}  // namespace fa
