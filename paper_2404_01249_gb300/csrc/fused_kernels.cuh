// Fused per-iteration kernels of fa_register (FA_MODE_FUSED).
//
// One iteration of Algorithm 1 (Jacobian-free direction) is four launches:
//   K1 k_lncc_fwd       LNCC forward on J = I_m o phi: exact int64 window
//                       sums of J, J^2 and I J (the fixed image's window sum
//                       and variance come precomputed per level), cc, the
//                       adjoint coefficients A, B, C, the loss accumulator and
//                       the coefficient maxima.
//   K2 k_lncc_grad      adjoint window sums of A, B, C; g = dL/dJ grad I_m(phi)
//                       with J and grad I_m(phi) as the compose kernel stored
//                       them.
//   K3 k_smooth_adam    Gaussian(sigma_grad) of g, Adam update of m, nu, the
//                       direction d and the grid max |d|.
//   K4 k_compose        delta = -eps_t d, u' = delta + u o (id + delta),
//                       Gaussian(sigma_warp) of u', and J = I_m o (id + u')
//                       with its gradient grad I_m(phi') for the next
//                       iteration's K1 and K2 (one gather per iteration).
// The grid max of K3 is a global dependency, so K4 cannot join K3; the
// adjoint window sums need A, B, C around every output, so K2 cannot join K1
// without recomputing a much wider halo.
//
// Every kernel marches along z ("2.5-D" tiling): a CTA owns a 32 x TY tile of
// (x, y) columns and a slab of TZ output planes.  A plane's inputs (the tile
// plus its halo, and the operands of the plane's outputs) arrive NSTG - 1
// planes ahead of use.  When the buffers' rows start on 16-byte boundaries
// (a registration pads its levels' rows to a multiple of 4 floats) they come
// as TMA tile copies issued by one thread and completed on an mbarrier (zero
// fill outside the grid); otherwise each thread copies its own positions with
// cp.async.  A plane is reduced along x (register-blocked, 16-byte shared
// loads) and then y in shared memory; the last 2R + 1 in-plane results per
// output column sit in a shared-memory ring from which the z reduction reads.
// No intermediate of the separable sums goes to HBM; halo re-reads hit L2.
//
// Shared plane layout: [C][RY][BXW] with BXW = 32 + 2 XB and XB = R rounded
// up to a multiple of 4.  Column c holds x = x0 - XB + c and row r holds
// y = y0 - R + r, so that a TMA box starts on a 16-byte boundary.
//
// Every wait on a TMA barrier is bounded; a wait that gives up sets
// ST_TIMEOUT in the status word, waits (bounded again) for the CTA's copies
// in flight and ends the CTA, and later CTAs that see the bit drain their
// first copies and return.
#pragma once

#include <cuda.h>
#include <type_traits>
#include <math.h>

#include <map>
#include <mutex>

#include "register.h"
#include "validate.h"

namespace fa {

namespace {


constexpr int FX = 32;  // tile width along x (one warp)

__host__ __device__ constexpr int halo4(int r) { return (r + 3) / 4 * 4; }
__host__ __device__ constexpr size_t al128(size_t b) { return (b + 127) & ~size_t(127); }

__device__ __forceinline__ unsigned su32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// ----------------------------------------------------------- cp.async path
__device__ __forceinline__ void cp4(void *dst, const void *src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(su32(dst)), "l"(src),
                 "r"(ok ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp8(void *dst, const void *src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(su32(dst)), "l"(src),
                 "r"(ok ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------- TMA path
__device__ __forceinline__ void mbar_init(unsigned long long *b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(b)) : "memory");
}
// Makes initialised barriers visible to the TMA unit.
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Orders this thread's shared-memory stores before later tile copies into the
// same bytes (a buffer refilled by TMA after the threads wrote to it).
__device__ __forceinline__ void proxy_fence_async() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// The arrival of the one expected thread, announcing `bytes` of copies.
__device__ __forceinline__ void mbar_expect(unsigned long long *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase of parity `parity` to complete; gives up after about
// `limit` SM cycles (default 2^28: 0.13 s at 2 GHz; a tile copy takes
// microseconds).
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity,
                                          long long limit = 1ll << 28) {
    if (mbar_try(b, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(b, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
// One tile copy of a rank-4 map ([C][D][H][W]) into shared memory.
__device__ __forceinline__ void tma4(void *dst, const CUtensorMap *m, int x, int y, int z, int c,
                                     unsigned long long *b) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(su32(dst)),
        "l"(reinterpret_cast<unsigned long long>(m)), "r"(x), "r"(y), "r"(z), "r"(c),
        "r"(su32(b))
        : "memory");
}

// Tensor maps of one launch (the ones a kernel does not use stay zero).
struct Maps {
    CUtensorMap a, b, c, d;
};

// The tensor maps a CTA's body loads through: generic addresses of maps in
// the kernel's parameter space (a launch's Maps, or one job's entries of a
// lockstep table); null where the body takes no TMA tiles.
struct MapRef {
    const CUtensorMap *a, *b, *c;
};
__device__ __forceinline__ MapRef map_ref(const Maps &m) { return MapRef{&m.a, &m.b, &m.c}; }

}  // namespace
// Map of a [C][D][H][W] field of 4- or 8-byte elements with rows of
// d.pitch() elements, a {bx, by, 1, bc} box and zero fill outside the grid;
// false when the field does not meet TMA's alignment rules.
bool tmap(CUtensorMap *m, const void *base, int esize, Dims d, int C, int bx, int by, int bc);
namespace {

// Programmatic dependent launch: the fused kernels are launched so that a
// kernel's CTAs may start while the previous kernel in the stream finishes.
// Everything before pdl_wait() touches no data the previous kernel writes;
// pdl_wait() returns once that kernel has completed and its writes are
// visible.  pdl_trigger() lets the next kernel begin launching once every
// CTA of this one has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// For a CTA that has waited for the previous kernel (pdl_wait) and issued its
// first copies and header loads (so that they are in flight while the status
// word is read): true, uniformly over the CTA, when an earlier CTA reported a
// timeout; the caller then drains its copies (drain_first) and returns.
__device__ __forceinline__ bool status_timed_out(const WsHeader *h, int tid, int *flag) {
    if (tid == 0) *flag = (int)(*(volatile const unsigned *)&h->status & ST_TIMEOUT);
    __syncthreads();
    pdl_trigger();
    return *flag != 0;
}

// Bounded wait for the first min(n, NSTG - 1) stage copies a CTA issued
// before it returns early (TMA), or for its copy groups (cp.async).
template <bool TMA, int NSTG>
__device__ __forceinline__ void drain_first(unsigned long long *bar, int n, int tid) {
    if (TMA) {
        if (tid == 0)
            for (int j = 0; j < n && j < NSTG - 1; ++j) mbar_wait(bar + j, 0u);
    } else {
        cp_wait<0>();
    }
}

// --------------------------------------------- cp.async position mapping
// A thread's positions in the RY x RX logical region of a plane (RX <= 64):
// warp w covers rows w, w + NW, ...; lane l covers columns l and l + 32.
// Logical column rx is stored at column rx + COFF of a BXW-wide row.
template <int RY, int RX, int NW, int BXW, int COFF>
struct Region {
    static constexpr int NJ = (RY + NW - 1) / NW;
    static constexpr int NC = (RX + 31) / 32;
    int off[NJ * NC];  // y P + x inside the grid, -1 outside the grid, -2 outside the region
    int sbase;
    __device__ __forceinline__ void init(int wy, int tx, int ybase, int xbase, int H, int W,
                                         int P) {
        sbase = wy * BXW + tx + COFF;
#pragma unroll
        for (int j = 0; j < NJ; ++j)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int ry = wy + NW * j, rx = tx + 32 * c;
                const int y = ybase + ry, x = xbase + rx;
                int o = -2;
                if (ry < RY && rx < RX) o = (y >= 0 && y < H && x >= 0 && x < W) ? y * P + x : -1;
                off[j * NC + c] = o;
            }
    }
    static __device__ __forceinline__ int sofs(int j, int c) { return NW * j * BXW + 32 * c; }
    // C channels of plane zoff / W H (zero outside the grid) -> [C][RY][BXW]
    template <int C>
    __device__ __forceinline__ void load(float *dst, const float *src, long long N, long long zoff,
                                         bool zok) const {
#pragma unroll
        for (int j = 0; j < NJ; ++j)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int o = off[j * NC + c];
                if (o == -2) continue;
                const bool ok = zok && o >= 0;
                const float *s = src + (ok ? zoff + o : 0);
                float *d = dst + sbase + sofs(j, c);
#pragma unroll
                for (int ch = 0; ch < C; ++ch) cp4(d + ch * RY * BXW, s + ch * N, ok);
            }
    }
};

// This thread's OPT output voxels; its slot o of a [C][TY][32] output tile is
// o NT + tid (the layout a {32, TY, 1, C} TMA box lands in).
template <int OPT, int NW>
struct Outs {
    static constexpr int NT = 32 * NW, NOUT = OPT * NT;
    int off[OPT];  // y P + x (P: the row pitch), -1 outside the grid
    __device__ __forceinline__ void init(int wy, int tx, int y0, int x0, int H, int W, int P) {
#pragma unroll
        for (int o = 0; o < OPT; ++o) {
            const int y = y0 + wy + NW * o, x = x0 + tx;
            off[o] = (y < H && x < W) ? y * P + x : -1;
        }
    }
    // C channels of this thread's outputs on plane zoff / (H W), to registers
    // (zero outside the grid)
    template <int C, class T>
    __device__ __forceinline__ void fetch(T (&r)[OPT][C], const T *src, long long N,
                                          long long zoff) const {
#pragma unroll
        for (int o = 0; o < OPT; ++o)
#pragma unroll
            for (int c = 0; c < C; ++c) r[o][c] = off[o] >= 0 ? src[c * N + zoff + off[o]] : T(0);
    }
    template <int C, class T>
    __device__ __forceinline__ void load(T *dst, const T *src, long long N, long long zoff,
                                         int tid) const {
#pragma unroll
        for (int o = 0; o < OPT; ++o) {
            const bool ok = off[o] >= 0;
            const T *s = src + (ok ? zoff + off[o] : 0);
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                if (sizeof(T) == 8)
                    cp8(dst + ch * NOUT + o * NT + tid, s + ch * N, ok);
                else
                    cp4(dst + ch * NOUT + o * NT + tid, s + ch * N, ok);
            }
        }
    }
};

// ------------------------------------------------- register-blocked x passes
// A work item is (channel, row, group of 4 adjacent output columns); items
// are spread over all threads.  The taps of output column ox start at plane
// column ox + COFF; rows are read with 16-byte shared loads from column 4k.

// Gaussian x pass: pl [C][RY][BXW] -> xb [C][RY][FX].
template <int RG, int C, int RY, int BXW, int COFF, int NT, class TT>
__device__ __forceinline__ void gauss_x4(const float *pl, float *xb, const TT &t, int tid) {
    constexpr int ITEMS = C * RY * 8, NL = (4 + COFF + 2 * RG + 3) / 4;
    static_assert(28 + 4 * NL <= BXW, "row too short for the vector loads");
#pragma unroll
    for (int j = 0; j < (ITEMS + NT - 1) / NT; ++j) {
        const int it = tid + j * NT;
        if (ITEMS % NT != 0 && it >= ITEMS) break;
        const int k = it & 7, rest = it >> 3, ry = rest % RY, c = rest / RY;
        const float4 *src = (const float4 *)(pl + (c * RY + ry) * BXW + 4 * k);
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
            for (int tt = 0; tt <= 2 * RG; ++tt) a = fmaf(t.w[tt], v[jj + COFF + tt], a);
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

// LNCC forward x pass on quantised planes qI, qJ [RY][BXW] (int32) ->
// xL [3][RY][FX] int64: channel 0 sum J, 1 sum J^2, 2 sum I J.
template <int R, int RY, int BXW, int COFF, int NT>
__device__ __forceinline__ void box_x4_fwd(const int *qI, const int *qJ, long long *xL, int tid) {
    constexpr int ITEMS = 3 * RY * 8, NL = (4 + COFF + 2 * R + 3) / 4, NV = 4 + 2 * R;
    static_assert(28 + 4 * NL <= BXW, "row too short for the vector loads");
#pragma unroll
    for (int j = 0; j < (ITEMS + NT - 1) / NT; ++j) {
        const int it = tid + j * NT;
        if (ITEMS % NT != 0 && it >= ITEMS) break;
        const int k = it & 7, rest = it >> 3, ry = rest % RY, c = rest / RY;
        int vj[4 * NL], vi[4 * NL];
        const int4 *sj = (const int4 *)(qJ + ry * BXW + 4 * k);
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
            slide4<R, int>(vj + COFF, s4);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) out[jj] = s4[jj];
        } else {
            if (c == 2) {
                const int4 *si = (const int4 *)(qI + ry * BXW + 4 * k);
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
            for (int tt = 0; tt < NV; ++tt) pr[tt] = (long long)vi[tt + COFF] * vj[tt + COFF];
            slide4<R, long long>(pr, out);
        }
        store_ll4(xL + (c * RY + ry) * FX + 4 * k, out);
    }
}

// LNCC adjoint x pass on quantised coefficients q [3][RY][BXW] (int64) ->
// xL [3][RY][FX].
template <int R, int RY, int BXW, int COFF, int NT>
__device__ __forceinline__ void box_x4_adj(const long long *q, long long *xL, int tid) {
    constexpr int ITEMS = 3 * RY * 8, NL = (4 + COFF + 2 * R + 1) / 2;
    static_assert(28 + 2 * NL <= BXW, "row too short for the vector loads");
#pragma unroll
    for (int j = 0; j < (ITEMS + NT - 1) / NT; ++j) {
        const int it = tid + j * NT;
        if (ITEMS % NT != 0 && it >= ITEMS) break;
        const int k = it & 7, rest = it >> 3, ry = rest % RY, c = rest / RY;
        const longlong2 *src = (const longlong2 *)(q + (c * RY + ry) * BXW + 4 * k);
        long long v[2 * NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const longlong2 a = src[l];
            v[2 * l] = a.x;
            v[2 * l + 1] = a.y;
        }
        long long out[4];
        slide4<R, long long>(v + COFF, out);
        store_ll4(xL + (c * RY + ry) * FX + 4 * k, out);
    }
}

// y pass of this thread's outputs from xL [C][RY][FX].
template <int R, int RY, int NW, int OPT>
__device__ __forceinline__ void box_y3(const long long *xL, int wy, int tx, long long P[OPT][3]) {
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
}

// Channels 0 and 1 of the y and z passes run as one packed FP32 pair
// (__ffma2_rn: each component is exactly fmaf), channel 2 alone; every
// channel's taps accumulate in the same order as a scalar loop would.
template <int RG, int RY, int NW, int OPT, class TT>
__device__ __forceinline__ void gauss_y3(const float *xb, const TT &t, int wy, int tx,
                                         float Q[OPT][3]) {
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
        const float *xi = xb + (wy + NW * o) * FX + tx;
        float2 s01 = make_float2(0.0f, 0.0f);
        float s2 = 0.0f;
#pragma unroll
        for (int k = 0; k <= 2 * RG; ++k) {
            const float w = t.w[k];
            s01 = __ffma2_rn(make_float2(w, w),
                             make_float2(xi[k * FX], xi[RY * FX + k * FX]), s01);
            s2 = fmaf(w, xi[2 * RY * FX + k * FX], s2);
        }
        Q[o][0] = s01.x;
        Q[o][1] = s01.y;
        Q[o][2] = s2;
    }
}

// Running z window sums: ring of the last NS plane results per output.
template <int NS, int OPT, int NOUT, int NT>
__device__ __forceinline__ void zslide(long long *ring, int slot, int tid,
                                       const long long P[OPT][3], long long acc[OPT][3]) {
    long long *rb = ring + slot * 3 * NOUT + tid;
#pragma unroll
    for (int o = 0; o < OPT; ++o)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            long long *r = rb + c * NOUT + o * NT;
            acc[o][c] += P[o][c] - *r;
            *r = P[o][c];
        }
}

// Ring of the last NS in-plane results of this thread's outputs, [NS][3][NOUT]
// floats; slot `newest` holds the current plane.
template <int NS, int OPT, int NOUT, int NT>
__device__ __forceinline__ void ring_put(float *ring, int newest, int tid, const float Q[OPT][3]) {
#pragma unroll
    for (int o = 0; o < OPT; ++o)
#pragma unroll
        for (int c = 0; c < 3; ++c) ring[(newest * 3 + c) * NOUT + o * NT + tid] = Q[o][c];
}

// Weighted z window of all three channels of one output: tap k takes the
// plane k - R of the window, i.e. ring slot (newest + 1 + k) mod NS.
template <int RG, int NOUT, class TT>
__device__ __forceinline__ void gauss_z3(const float *ring_o, int newest, const TT &t,
                                         float out[3]) {
    constexpr int NS = 2 * RG + 1;
    float2 s01 = make_float2(0.0f, 0.0f);
    float s2 = 0.0f;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        int j = newest + 1 + k;
        j = j >= NS ? j - NS : j;
        const float *r = ring_o + j * 3 * NOUT;
        const float w = t.w[k];
        s01 = __ffma2_rn(make_float2(w, w), make_float2(r[0], r[NOUT]), s01);
        s2 = fmaf(w, r[2 * NOUT], s2);
    }
    out[0] = s01.x;
    out[1] = s01.y;
    out[2] = s2;
}

// Bounded wait, by thread 0, for the copies of planes i .. i + NSTG - 1 that
// may still be in flight when a CTA stops early.
template <int NSTG>
__device__ __forceinline__ void drain(unsigned long long *bar, int i, int np) {
    for (int j = i; j < i + NSTG && j < np; ++j) mbar_wait(bar + j % NSTG, (unsigned)(j / NSTG) & 1u);
}

// ====================================================================== K1
template <int R, int NW, int OPT, int NSTG>
struct K1S {
    static constexpr int NT = FX * NW, TY = NW * OPT, RX = FX + 2 * R, RY = TY + 2 * R;
    static constexpr int XB = halo4(R), BXW = FX + 2 * XB, COFF = XB - R;
    static constexpr int NR = BXW * RY, NS = 2 * R + 1, NOUT = NT * OPT;
    static constexpr size_t plane = al128((size_t)NR * 4);  // I_f plane, then J plane
    static constexpr size_t st_bytes = 2 * plane;
    static constexpr unsigned tx_plane = 2u * NR * 4;
    static constexpr size_t o_st = 0;
    static constexpr size_t o_ring = o_st + st_bytes * NSTG;             // [NS][3][NOUT] int64
    static constexpr size_t o_xL = o_ring + (size_t)NS * 3 * NOUT * 8;   // [3][RY][FX] int64
    static constexpr size_t o_q = o_xL + (size_t)3 * RY * FX * 8;        // [2][RY][BXW] int32
    static constexpr size_t o_bar = al128(o_q + (size_t)2 * NR * 4);
    static constexpr size_t bytes = o_bar + 8 * NSTG;
};

// K1's output voxel from its window sums acc = (S_J, S_JJ, S_IJ) and the
// fixed image's S_I (a1) and variance: cc into the loss sum qcc (bad when cc
// leaves [0, 2]), and with write_coef the adjoint coefficients A, B and C
// (float-float) at cp[0], cp[N], cp[2N], cp[3N] with their running maxima.
__device__ __forceinline__ void lncc_fwd_output(const long long acc[3], long long a1, float varI,
                                                long long n, float nf, float inv_nf, float inv_s,
                                                float cc_eps, int write_coef, float *cp,
                                                long long N, unsigned long long &qcc, bool &bad,
                                                float &mA, float &mB, float &mC) {
    const long long a2 = acc[0];
    const float varJ = diff_i128_to_float(n, acc[1], a2, a2) * inv_s * inv_s * inv_nf;
    const float cross = diff_i128_to_float(n, acc[2], a1, a2) * inv_s * inv_s * inv_nf;
    const float den = fmaf(varI, varJ, cc_eps);
    const float rden = __frcp_rn(den);
    const float cc = cross * cross * rden;
    if (cc >= 0.0f && cc <= 2.0f)
        qcc += (unsigned long long)quantize(cc, 4294967296.0f);  // cc in [0, 2]
    else
        bad = true;
    if (write_coef) {
        const float A = 2.0f * cross * rden;
        const float B = -cc * varI * rden;
        float Ch, Cl;
        lncc_c_ff(A, B, a1, a2, inv_s, nf, inv_nf, Ch, Cl);
        cp[0] = A;
        cp[N] = B;
        cp[2 * N] = Ch;
        cp[3 * N] = Cl;
        mA = fmaxf(mA, fabsf(A));
        mB = fmaxf(mB, fabsf(B));
        mC = fmaxf(mC, fabsf(Ch));
    }
}

// The body of K1 for the CTA with tile coordinates (bx, by, bz).
template <int R, int NW, int OPT, int NSTG, bool TMA>
__device__ __forceinline__ void lncc_fwd_body(MapRef maps, const float *__restrict__ If,
                                              const float *__restrict__ J,
                                              const long long *__restrict__ SIg,
                                              const float *__restrict__ varIg,
                                              float *__restrict__ coef, WsHeader *__restrict__ h,
                                              int D, int H, int W, int P, int TZ, int bits,
                                              float cc_eps,
                                              int window, int write_coef, int bx, int by, int bz) {
    using S = K1S<R, NW, OPT, NSTG>;
    constexpr int NT = S::NT, TY = S::TY, RX = S::RX, RY = S::RY, BXW = S::BXW, COFF = S::COFF,
                  XB = S::XB, NR = S::NR, NS = S::NS, NOUT = S::NOUT;
    constexpr int CS = (int)(S::plane / 4);
    using G = Region<RY, RX, NW, BXW, COFF>;
    extern __shared__ __align__(128) unsigned char smem[];
    long long *ring = (long long *)(smem + S::o_ring);
    long long *xL = (long long *)(smem + S::o_xL);
    int *qI = (int *)(smem + S::o_q), *qJ = qI + NR;
    unsigned long long *bar = (unsigned long long *)(smem + S::o_bar);
    __shared__ float redf[32];
    __shared__ unsigned long long redu[32];
    __shared__ int flag;
    auto stage = [&](int s) { return (float *)(smem + S::o_st + S::st_bytes * s); };

    const int tx = threadIdx.x, wy = threadIdx.y, tid = wy * FX + tx;
    const int x0 = bx * FX, y0 = by * TY, z0 = bz * TZ;
    const int zend = min(z0 + TZ, D);
    const long long N = (long long)D * H * P, HW = (long long)H * P;  // channel, plane strides
    const long long n = (long long)window * window * window;
    const float nf = (float)n, inv_nf = 1.0f / nf;
    G rg;
    if (!TMA) rg.init(wy, tx, y0 - R, x0 - R, H, W, P);
    Outs<OPT, NW> ou;
    ou.init(wy, tx, y0, x0, H, W, P);
    if (TMA && tid == 0) {
        for (int k = 0; k < NSTG; ++k) mbar_init(bar + k);
        mbar_init_fence();
    }
    for (int k = tid; k < NS * 3 * NOUT; k += NT) ring[k] = 0;

    long long acc[OPT][3];
#pragma unroll
    for (int o = 0; o < OPT; ++o)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[o][c] = 0;

    const int zs = z0 - R, np = zend - z0 + 2 * R;
    auto issue = [&](int i) {
        const int zp = zs + i, s = i % NSTG;
        if (TMA) {
            if (tid == 0 && i < np) {
                mbar_expect(bar + s, S::tx_plane);
                tma4(stage(s), maps.a, x0 - XB, y0 - R, zp, 0, bar + s);
                tma4(stage(s) + CS, maps.b, x0 - XB, y0 - R, zp, 0, bar + s);
            }
        } else {
            if (i < np) {
                const bool zok = zp >= 0 && zp < D;
                rg.template load<1>(stage(s), If, N, (long long)zp * HW, zok);
                rg.template load<1>(stage(s) + CS, J, N, (long long)zp * HW, zok);
            }
            cp_commit();
        }
    };
    // the outputs' operands S_I, var_I, loaded one plane ahead into registers
    long long a1n[OPT][1];
    float vIn[OPT][1];
    auto fetch_ops = [&](int i) {
        const int zo = zs + i - R;
        if (i < np && zo >= z0 && zo < zend) {
            ou.fetch(a1n, SIg, N, (long long)zo * HW);
            ou.fetch(vIn, varIg, N, (long long)zo * HW);
        }
    };
    // after the previous kernel: first copies, operands and header loads in
    // flight together, then the status check
    pdl_wait();
    fetch_ops(0);
#pragma unroll
    for (int k = 0; k < NSTG - 1; ++k) issue(k);
    const float amax =
        fmaxf(__uint_as_float(h->absmax_bits[0]), __uint_as_float(h->absmax_bits[1]));
    if (status_timed_out(h, tid, &flag)) {
        drain_first<TMA, NSTG>(bar, np, tid);
        return;
    }
    const int sh = fixed_shift(amax, bits);
    const float scale = pow2f(sh), inv_s = pow2f(-sh);

    unsigned long long qcc = 0;
    float mA = 0.f, mB = 0.f, mC = 0.f;
    bool bad = false;
    int fail = -1, slot = 0;
    for (int i = 0; i < np; ++i) {
        const int zp = zs + i, z = zp - R, s = i % NSTG;
        issue(i + NSTG - 1);
        const bool out = z >= z0 && z < zend;
        long long a1[OPT];
        float vI[OPT];
#pragma unroll
        for (int o = 0; o < OPT; ++o) {
            a1[o] = a1n[o][0];
            vI[o] = vIn[o][0];
        }
        fetch_ops(i + 1);
        bool ok = true;
        if (TMA)
            ok = mbar_wait(bar + s, (unsigned)(i / NSTG) & 1u);
        else
            cp_wait<NSTG - 1>();
        const bool zin = zp >= 0 && zp < D;
        if (zin) {
            const float *sI = stage(s), *sJ = sI + CS;
            if (TMA) {
                for (int k = tid; k < NR; k += NT) {
                    qI[k] = __float2int_rn(sI[k] * scale);
                    qJ[k] = __float2int_rn(sJ[k] * scale);
                }
            } else {
#pragma unroll
                for (int j = 0; j < G::NJ; ++j)
#pragma unroll
                    for (int c = 0; c < G::NC; ++c) {  // own copies
                        if (rg.off[j * G::NC + c] == -2) continue;
                        const int k = rg.sbase + G::sofs(j, c);
                        qI[k] = __float2int_rn(sI[k] * scale);
                        qJ[k] = __float2int_rn(sJ[k] * scale);
                    }
            }
        }
        if (__syncthreads_or(!ok)) {
            fail = i;
            break;
        }
        long long P[OPT][3];
        if (zin) {
            box_x4_fwd<R, RY, BXW, COFF, NT>(qI, qJ, xL, tid);
            __syncthreads();
            box_y3<R, RY, NW, OPT>(xL, wy, tx, P);
        } else {
#pragma unroll
            for (int o = 0; o < OPT; ++o)
#pragma unroll
                for (int c = 0; c < 3; ++c) P[o][c] = 0;
        }
        zslide<NS, OPT, NOUT, NT>(ring, slot, tid, P, acc);
        slot = (slot + 1 == NS) ? 0 : slot + 1;
        if (out) {
            const long long zoff = (long long)z * HW;
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                if (ou.off[o] < 0) continue;
                lncc_fwd_output(acc[o], a1[o], vI[o], n, nf, inv_nf, inv_s, cc_eps, write_coef,
                                coef + zoff + ou.off[o], N, qcc, bad, mA, mB, mC);
            }
        }
    }
    if (fail >= 0) {  // a tile copy never landed
        if (tid == 0) {
            status_set(&h->status, ST_TIMEOUT);
            drain<NSTG>(bar, fail, np);
        }
        return;
    }
    if (!TMA) cp_wait<0>();
    if (bad) status_set(&h->status, ST_NONFINITE);
    block_sum_to(&h->loss_acc, qcc, redu);
    if (write_coef) {
        block_max_to(&h->coef_max_bits[0], mA, redf);
        block_max_to(&h->coef_max_bits[1], mB, redf);
        block_max_to(&h->coef_max_bits[2], mC, redf);
    }
}

template <int R, int NW, int OPT, int NSTG, bool TMA>
__global__ void __launch_bounds__(FX *NW) k_lncc_fwd(const __grid_constant__ Maps maps,
                                                     const float *__restrict__ If,
                                                     const float *__restrict__ J,
                                                     const long long *__restrict__ SIg,
                                                     const float *__restrict__ varIg,
                                                     float *__restrict__ coef,
                                                     WsHeader *__restrict__ h, int D, int H, int W,
                                                     int P, int TZ, int bits, float cc_eps,
                                                     int window, int write_coef) {
    lncc_fwd_body<R, NW, OPT, NSTG, TMA>(map_ref(maps), If, J, SIg, varIg, coef, h, D, H, W, P, TZ, bits,
                                         cc_eps, window, write_coef, blockIdx.x, blockIdx.y,
                                         blockIdx.z);
}

// ====================================================================== K2
// coef holds A, B and C as a float-float pair (C hi, C lo): [4][N].
template <int R, int NW, int OPT, int NSTG>
struct K2S {
    static constexpr int NT = FX * NW, TY = NW * OPT, RX = FX + 2 * R, RY = TY + 2 * R;
    static constexpr int XB = halo4(R), BXW = FX + 2 * XB, COFF = XB - R;
    static constexpr int NR = BXW * RY, NS = 2 * R + 1, NOUT = NT * OPT;
    static constexpr size_t st_bytes = al128((size_t)4 * NR * 4);    // A, B, C hi, C lo
    static constexpr unsigned tx_plane = 4u * NR * 4;
    static constexpr size_t o_st = 0;
    static constexpr size_t o_ring = o_st + st_bytes * NSTG;
    static constexpr size_t o_xL = o_ring + (size_t)NS * 3 * NOUT * 8;
    static constexpr size_t o_q = o_xL + (size_t)3 * RY * FX * 8;
    static constexpr size_t o_bar = al128(o_q + (size_t)3 * NR * 8);
    static constexpr size_t bytes = o_bar + 8 * NSTG;
};

// The body of K2 for the CTA with tile coordinates (bx, by, bz).  WDJ: also
// write dL/dJ itself to dJout (the adjoint's scatter into dL/dI_m needs it).
template <int R, int NW, int OPT, int NSTG, bool TMA, bool WDJ = false>
__device__ __forceinline__ void lncc_grad_body(MapRef maps, const float *__restrict__ If,
                                               const float *__restrict__ gJ,
                                               const float *__restrict__ J,
                                               const float *__restrict__ coef,
                                               WsHeader *__restrict__ h, float *__restrict__ g,
                                               int D, int H, int W, int P, int TZ, int cbits,
                                               int bx,
                                               int by, int bz, float *__restrict__ dJout = nullptr) {
    using S = K2S<R, NW, OPT, NSTG>;
    constexpr int NT = S::NT, TY = S::TY, RX = S::RX, RY = S::RY, BXW = S::BXW, COFF = S::COFF,
                  XB = S::XB, NR = S::NR, NS = S::NS, NOUT = S::NOUT;
    using G = Region<RY, RX, NW, BXW, COFF>;
    extern __shared__ __align__(128) unsigned char smem[];
    long long *ring = (long long *)(smem + S::o_ring);
    long long *xL = (long long *)(smem + S::o_xL);
    long long *q = (long long *)(smem + S::o_q);
    unsigned long long *bar = (unsigned long long *)(smem + S::o_bar);
    __shared__ int flag;
    auto stage = [&](int s) { return (float *)(smem + S::o_st + S::st_bytes * s); };

    const int tx = threadIdx.x, wy = threadIdx.y, tid = wy * FX + tx;
    const int x0 = bx * FX, y0 = by * TY, z0 = bz * TZ;
    const int zend = min(z0 + TZ, D);
    const long long N = (long long)D * H * P, HW = (long long)H * P;  // channel, plane strides
    const float inv_n = 1.0f / (float)((long long)D * H * W);  // 1 / voxel count
    G rg;
    if (!TMA) rg.init(wy, tx, y0 - R, x0 - R, H, W, P);
    Outs<OPT, NW> ou;
    ou.init(wy, tx, y0, x0, H, W, P);
    if (TMA && tid == 0) {
        for (int k = 0; k < NSTG; ++k) mbar_init(bar + k);
        mbar_init_fence();
    }
    for (int k = tid; k < NS * 3 * NOUT; k += NT) ring[k] = 0;
    long long acc[OPT][3];
#pragma unroll
    for (int o = 0; o < OPT; ++o)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[o][c] = 0;

    const int zs = z0 - R, np = zend - z0 + 2 * R;
    auto issue = [&](int i) {
        const int zp = zs + i, s = i % NSTG;
        if (TMA) {
            if (tid == 0 && i < np) {
                mbar_expect(bar + s, S::tx_plane);
                tma4(stage(s), maps.a, x0 - XB, y0 - R, zp, 0, bar + s);
            }
        } else {
            if (i < np)
                rg.template load<4>(stage(s), coef, N, (long long)zp * HW, zp >= 0 && zp < D);
            cp_commit();
        }
    };
    // the outputs' operands grad I_m(phi), I_f, J, loaded one plane ahead
    float gn[OPT][3], In[OPT][1], Jn[OPT][1];
    auto fetch_ops = [&](int i) {
        const int zo = zs + i - R;
        if (i < np && zo >= z0 && zo < zend) {
            ou.fetch(gn, gJ, N, (long long)zo * HW);
            ou.fetch(In, If, N, (long long)zo * HW);
            ou.fetch(Jn, J, N, (long long)zo * HW);
        }
    };
    // after the previous kernel: first copies, operands and header loads in
    // flight together, then the status check
    pdl_wait();
    fetch_ops(0);
#pragma unroll
    for (int k = 0; k < NSTG - 1; ++k) issue(k);
    float cmax[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) cmax[c] = __uint_as_float(h->coef_max_bits[c]);
    if (status_timed_out(h, tid, &flag)) {
        drain_first<TMA, NSTG>(bar, np, tid);
        return;
    }
    float qs[3], us[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int e = fixed_shift(cmax[c], cbits);
        qs[c] = pow2f(e);
        us[c] = pow2f(-e);
    }

    int fail = -1, slot = 0;
    for (int i = 0; i < np; ++i) {
        const int zp = zs + i, zo = zp - R, s = i % NSTG;
        issue(i + NSTG - 1);
        const bool out = zo >= z0 && zo < zend;
        float Gz[OPT], Gy[OPT], Gx[OPT], Iv[OPT], Jv[OPT];
#pragma unroll
        for (int k = 0; k < OPT; ++k) {
            Gz[k] = gn[k][0];
            Gy[k] = gn[k][1];
            Gx[k] = gn[k][2];
            Iv[k] = In[k][0];
            Jv[k] = Jn[k][0];
        }
        fetch_ops(i + 1);
        bool ok = true;
        if (TMA)
            ok = mbar_wait(bar + s, (unsigned)(i / NSTG) & 1u);
        else
            cp_wait<NSTG - 1>();
        const bool zin = zp >= 0 && zp < D;
        if (zin) {
            const float *sp = stage(s);
            auto quant = [&](int k) {
                q[k] = quantize(sp[k], qs[0]);
                q[NR + k] = quantize(sp[NR + k], qs[1]);
                q[2 * NR + k] = quantize(sp[2 * NR + k], qs[2]) + quantize(sp[3 * NR + k], qs[2]);
            };
            if (TMA) {
                for (int k = tid; k < NR; k += NT) quant(k);
            } else {
#pragma unroll
                for (int j = 0; j < G::NJ; ++j)
#pragma unroll
                    for (int c = 0; c < G::NC; ++c) {  // own copies
                        if (rg.off[j * G::NC + c] == -2) continue;
                        quant(rg.sbase + G::sofs(j, c));
                    }
            }
        }
        if (__syncthreads_or(!ok)) {
            fail = i;
            break;
        }
        long long P[OPT][3];
        if (zin) {
            box_x4_adj<R, RY, BXW, COFF, NT>(q, xL, tid);
            __syncthreads();
            box_y3<R, RY, NW, OPT>(xL, wy, tx, P);
        } else {
#pragma unroll
            for (int o = 0; o < OPT; ++o)
#pragma unroll
                for (int c = 0; c < 3; ++c) P[o][c] = 0;
        }
        zslide<NS, OPT, NOUT, NT>(ring, slot, tid, P, acc);
        slot = (slot + 1 == NS) ? 0 : slot + 1;
        if (out) {
            const long long zoff = (long long)zo * HW;
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                if (ou.off[o] < 0) continue;
                float ah, al, bh, bl, ch, cl, rh, rl, th, tl;
                i64_to_ff(acc[o][0], ah, al);
                i64_to_ff(acc[o][1], bh, bl);
                i64_to_ff(acc[o][2], ch, cl);
                ff_mul_f(Iv[o], ah * us[0], al * us[0], rh, rl);      // I SA
                ff_mul_f(2.0f * Jv[o], bh * us[1], bl * us[1], th, tl);  // 2 J SB
                ff_add(rh, rl, th, tl);
                ff_add(rh, rl, ch * us[2], cl * us[2]);               // + SC
                const float dj = -(rh + rl) * inv_n;
                float *gp = g + zoff + ou.off[o];
                gp[0] = dj * Gz[o];
                gp[N] = dj * Gy[o];
                gp[2 * N] = dj * Gx[o];
                if (WDJ) dJout[zoff + ou.off[o]] = dj;
            }
        }
    }
    if (fail >= 0) {
        if (tid == 0) {
            status_set(&h->status, ST_TIMEOUT);
            drain<NSTG>(bar, fail, np);
        }
        return;
    }
    if (!TMA) cp_wait<0>();
}

template <int R, int NW, int OPT, int NSTG, bool TMA, bool WDJ = false>
__global__ void __launch_bounds__(FX *NW) k_lncc_grad(const __grid_constant__ Maps maps,
                                                      const float *__restrict__ If,
                                                      const float *__restrict__ gJ,
                                                      const float *__restrict__ J,
                                                      const float *__restrict__ coef,
                                                      WsHeader *__restrict__ h,
                                                      float *__restrict__ g, int D, int H, int W,
                                                      int P, int TZ, int cbits,
                                                      float *__restrict__ dJout) {
    lncc_grad_body<R, NW, OPT, NSTG, TMA, WDJ>(map_ref(maps), If, gJ, J, coef, h, g, D, H, W, P, TZ, cbits,
                                               blockIdx.x, blockIdx.y, blockIdx.z, dJout);
}

// MSE: g = 2 (J - I) / N * grad I_m(phi) (pointwise, J and the gradient as
// the compose kernel stored them).
__global__ void __launch_bounds__(256) k_fused_mse_grad(const float *__restrict__ If,
                                                        const float *__restrict__ J,
                                                        const float *__restrict__ gJ,
                                                        float *__restrict__ g, int D, int H,
                                                        int W) {
    int x = blockIdx.x * 32 + threadIdx.x;
    int y = blockIdx.y * 8 + threadIdx.y;
    int z = blockIdx.z;
    if (x >= W || y >= H) return;
    long long N = (long long)D * H * W;
    long long i = ((long long)z * H + y) * W + x;
    float dj = 2.0f * (__ldg(J + i) - __ldg(If + i)) / (float)N;
    g[i] = dj * __ldg(gJ + i);
    g[N + i] = dj * __ldg(gJ + N + i);
    g[2 * N + i] = dj * __ldg(gJ + 2 * N + i);
}

// ====================================================================== K3
// STAGED: the moments m, nu (FP32) arrive with the plane's TMA copies;
// otherwise (16-bit moments, or the per-thread copy variant) each thread loads
// its outputs' moments straight into registers one plane ahead.
template <int RG, int NW, int OPT, int NSTG, bool STAGED = true>
struct K3S {
    static constexpr int NT = FX * NW, TY = NW * OPT, RX = FX + 2 * RG, RY = TY + 2 * RG;
    static constexpr int XB = halo4(RG), BXW = FX + 2 * XB, COFF = XB - RG;
    static constexpr int NR = BXW * RY, NS = 2 * RG + 1, NOUT = NT * OPT;
    static constexpr size_t st_bytes = al128((size_t)3 * NR * 4);    // g
    static constexpr size_t ost_bytes = STAGED ? al128((size_t)6 * NOUT * 4) : 0;  // m, v
    static constexpr unsigned tx_plane = 3u * NR * 4, tx_out = 6u * NOUT * 4;
    static constexpr size_t o_st = 0;
    static constexpr size_t o_ost = o_st + st_bytes * NSTG;
    static constexpr size_t o_ring = o_ost + ost_bytes * NSTG;
    static constexpr size_t o_xb = o_ring + (size_t)NS * 3 * NOUT * 4;
    static constexpr size_t o_bar = al128(o_xb + (size_t)3 * RY * FX * 4);
    static constexpr size_t bytes = o_bar + 8 * NSTG;
};

// The body of K3 for the CTA with tile coordinates (bx, by, bz).
template <int RG, int NW, int OPT, int NSTG, bool TMA, class TT, class TS>
__device__ __forceinline__ void smooth_adam_body(MapRef maps, const float *__restrict__ g,
                                                 TS *__restrict__ m, TS *__restrict__ v,
                                                 float *__restrict__ dir, WsHeader *__restrict__ h,
                                                 int D, int H, int W, int P, int TZ, const TT t,
                                                 const AdamConsts ac, int parity, int bx, int by,
                                                 int bz) {
    constexpr bool S32 = sizeof(TS) == 4, STAGED = S32 && TMA;
    using S = K3S<RG, NW, OPT, NSTG, STAGED>;
    // moments as loaded into registers: FP32 values or 16-bit patterns
    using FT = typename std::conditional<S32, float, unsigned short>::type;
    constexpr int NT = S::NT, TY = S::TY, RX = S::RX, RY = S::RY, BXW = S::BXW, COFF = S::COFF,
                  XB = S::XB, NS = S::NS, NOUT = S::NOUT;
    using G = Region<RY, RX, NW, BXW, COFF>;
    extern __shared__ __align__(128) unsigned char smem[];
    float *ring = (float *)(smem + S::o_ring);
    float *xb = (float *)(smem + S::o_xb);
    unsigned long long *bar = (unsigned long long *)(smem + S::o_bar);
    __shared__ float redf[32];
    __shared__ int flag;
    auto stage = [&](int s) { return (float *)(smem + S::o_st + S::st_bytes * s); };
    auto ostage = [&](int s) { return (float *)(smem + S::o_ost + S::ost_bytes * s); };

    const int tx = threadIdx.x, wy = threadIdx.y, tid = wy * FX + tx;
    const int x0 = bx * FX, y0 = by * TY, z0 = bz * TZ;
    const int zend = min(z0 + TZ, D);
    const long long N = (long long)D * H * P, HW = (long long)H * P;  // channel, plane strides
    G rg;
    if (!TMA) rg.init(wy, tx, y0 - RG, x0 - RG, H, W, P);
    Outs<OPT, NW> ou;
    ou.init(wy, tx, y0, x0, H, W, P);
    if (TMA && tid == 0) {
        for (int k = 0; k < NSTG; ++k) mbar_init(bar + k);
        mbar_init_fence();
    }
    for (int k = tid; k < NS * 3 * NOUT; k += NT) ring[k] = 0.0f;

    const int zs = z0 - RG, np = zend - z0 + 2 * RG;
    auto issue = [&](int i) {
        const int zp = zs + i, zo = zp - RG, s = i % NSTG;
        const bool out = STAGED && zo >= z0 && zo < zend;
        if (TMA) {
            if (tid == 0 && i < np) {
                mbar_expect(bar + s, S::tx_plane + (out ? S::tx_out : 0u));
                tma4(stage(s), maps.a, x0 - XB, y0 - RG, zp, 0, bar + s);
                if (out) {
                    tma4(ostage(s), maps.b, x0, y0, zo, 0, bar + s);
                    tma4(ostage(s) + 3 * NOUT, maps.c, x0, y0, zo, 0, bar + s);
                }
            }
        } else {
            if (i < np) {
                rg.template load<3>(stage(s), g, N, (long long)zp * HW, zp >= 0 && zp < D);
            }
            cp_commit();
        }
    };
    // unstaged moments of the next output plane, loaded one plane ahead
    FT mn[OPT][3], vn[OPT][3];
    auto fetch_mv = [&](int i) {
        if constexpr (!STAGED) {
            const int zo = zs + i - RG;
            if (i < np && zo >= z0 && zo < zend) {
                ou.fetch(mn, (const FT *)m, N, (long long)zo * HW);
                ou.fetch(vn, (const FT *)v, N, (long long)zo * HW);
            }
        }
    };
    // after the previous kernel: first copies and loads in flight, then the
    // status check
    pdl_wait();
    fetch_mv(0);
#pragma unroll
    for (int k = 0; k < NSTG - 1; ++k) issue(k);
    if (status_timed_out(h, tid, &flag)) {
        drain_first<TMA, NSTG>(bar, np, tid);
        return;
    }

    float mx = 0.0f;
    bool bad = false;
    int fail = -1, slot = 0;
    for (int i = 0; i < np; ++i) {
        const int zp = zs + i, zo = zp - RG, s = i % NSTG;
        issue(i + NSTG - 1);
        bool ok = true;
        if (TMA)
            ok = mbar_wait(bar + s, (unsigned)(i / NSTG) & 1u);
        else
            cp_wait<NSTG - 1>();
        const bool out = zo >= z0 && zo < zend;
        float mo[OPT][3], vo[OPT][3];
        if (out) {
            if constexpr (STAGED) {
                const float *od = ostage(s) + tid;
#pragma unroll
                for (int o = 0; o < OPT; ++o)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        mo[o][c] = od[c * NOUT + o * NT];
                        vo[o][c] = od[(3 + c) * NOUT + o * NT];
                    }
            } else {
#pragma unroll
                for (int o = 0; o < OPT; ++o)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        mo[o][c] = st_value<TS>(mn[o][c]);
                        vo[o][c] = st_value<TS>(vn[o][c]);
                    }
            }
        }
        fetch_mv(i + 1);
        if (__syncthreads_or(!ok)) {  // also: the x pass reads neighbours' copies
            fail = i;
            break;
        }
        float Q[OPT][3];
        if (zp >= 0 && zp < D) {
            gauss_x4<RG, 3, RY, BXW, COFF, NT>(stage(s), xb, t, tid);
            __syncthreads();
            gauss_y3<RG, RY, NW, OPT>(xb, t, wy, tx, Q);
        } else {
#pragma unroll
            for (int o = 0; o < OPT; ++o) Q[o][0] = Q[o][1] = Q[o][2] = 0.0f;
        }
        ring_put<NS, OPT, NOUT, NT>(ring, slot, tid, Q);
        const int newest = slot;
        slot = (slot + 1 == NS) ? 0 : slot + 1;
        if (out) {
            const long long zoff = (long long)zo * HW;
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                if (ou.off[o] < 0) continue;
                float sz[3];
                gauss_z3<RG, NOUT>(ring + o * NT + tid, newest, t, sz);
                const long long gi = zoff + ou.off[o];
                float nrm2 = 0.0f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float sg = sz[c];
                    const float mvv = fmaf(ac.b1, mo[o][c], (1.0f - ac.b1) * sg);
                    const float vvv = fmaf(ac.b2, vo[o][c], (1.0f - ac.b2) * sg * sg);
                    m[c * N + gi] = st_store<TS>(mvv);
                    v[c * N + gi] = st_store<TS>(vvv);
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
    if (fail >= 0) {
        if (tid == 0) {
            status_set(&h->status, ST_TIMEOUT);
            drain<NSTG>(bar, fail, np);
        }
        return;
    }
    if (!TMA) cp_wait<0>();
    if (bad) status_set(&h->status, ST_NONFINITE);
    block_max_to(&h->step_max_bits[parity], mx, redf);
}

template <int RG, int NW, int OPT, int NSTG, bool TMA, class TS = float>
__global__ void __launch_bounds__(FX *NW, NW >= 16 ? 2 : 1) k_smooth_adam(const __grid_constant__ Maps maps,
                                                        const float *__restrict__ g,
                                                        TS *__restrict__ m,
                                                        TS *__restrict__ v,
                                                        float *__restrict__ dir,
                                                        WsHeader *__restrict__ h, int D, int H,
                                                        int W, int P, int TZ, GaussTaps t,
                                                        AdamConsts ac, int parity) {
    smooth_adam_body<RG, NW, OPT, NSTG, TMA>(map_ref(maps), g, m, v, dir, h, D, H, W, P, TZ, t, ac, parity,
                                             blockIdx.x, blockIdx.y, blockIdx.z);
}

// ====================================================================== K4
// SU: u is staged in shared memory (planes z-1..z+1, halo RG + 1); valid when
// the step is shorter than one voxel (lr / c_lp < 1).
// TU: storage of u (float, or __half for an FP16 u).
// The u tile's rows are 48 (or 64) elements long: an FP32 row is 16 banks
// (mod 32) long, so that the compose's reads of a neighbour row on either side
// of a lane's own voxel fall in the same bank, and an FP16 tile row starts on
// 16 bytes.  Its planes are whole multiples of 32 banks apart.
template <int RG, int NW, int OPT, bool SU, int NSTG, class TU = float>
struct K4S {
    static constexpr int NT = FX * NW, TY = NW * OPT, RX = FX + 2 * RG, RY = TY + 2 * RG;
    static constexpr int XB = halo4(RG), BXW = FX + 2 * XB, COFF = XB - RG;
    static constexpr int NR = BXW * RY, NS = 2 * RG + 1, NOUT = NT * OPT;
    // u planes z-1, z, z+1 in use plus NSTG - 1 in flight, halo RG + 1
    static constexpr int EU = (int)sizeof(TU);
    static constexpr int URX = RX + 2, URY = RY + 2, UXB = (RG + 1 + 7) / 8 * 8,
                         UBXW = FX + 2 * UXB;
    static constexpr int UCOFF = UXB - RG - 1, NRU = UBXW * URY, NSU = NSTG + 2;
    static constexpr int NP = RY * RX, NJP = (NP + NT - 1) / NT;  // compose positions
    static constexpr size_t st_bytes = al128((size_t)3 * NR * 4);     // d, then u' in place
    static constexpr size_t ust_bytes = al128((size_t)3 * NRU * EU);  // u
    static constexpr unsigned tx_plane = 3u * NR * 4, tx_u = 3u * NRU * EU;
    static constexpr size_t o_st = 0;
    static constexpr size_t o_ust = o_st + st_bytes * NSTG;
    static constexpr size_t o_ring = o_ust + (SU ? ust_bytes * NSU : 0);
    static constexpr size_t o_xb = o_ring + (size_t)NS * 3 * NOUT * 4;
    static constexpr size_t o_bar = al128(o_xb + (size_t)3 * RY * FX * 4);
    static constexpr size_t bytes = o_bar + 8 * (NSTG + 1);
    static_assert(EU == 2 || UBXW % 32 == 16 || UBXW % 32 == 0, "u rows of 16 or 32 banks");
};

// Compose position of slot pidx in the RY x RX region (RX = 32 + 2 RG): the
// first 32 RY slots are the region's first 32 columns row by row, so that a
// warp's positions lie in one row and its shared-memory reads and writes of
// them (d, the u cell corners, u') hit 32 consecutive words; the last 2 RG
// columns follow.
template <int RY, int RX>
__device__ __forceinline__ void compose_position(int pidx, int &ry, int &rx) {
    if (RX == 32 || pidx < 32 * RY) {
        ry = pidx >> 5;
        rx = pidx & 31;
    } else {
        const int e = pidx - 32 * RY;
        ry = e / (RX - 32);
        rx = 32 + e % (RX - 32);
    }
}

// The body of K4 for the CTA with tile coordinates (bx, by, bz).
template <int RG, int NW, int OPT, bool SU, int NSTG, bool TMA, class TT, class TU>
__device__ __forceinline__ void compose_body(MapRef maps, const TU *__restrict__ u,
                                             const float *__restrict__ dir,
                                             TU *__restrict__ uo,
                                             const float *__restrict__ Im,
                                             float *__restrict__ Jout, float *__restrict__ gJout,
                                             WsHeader *__restrict__ h, int D, int H, int W, int P,
                                             int TZ,
                                             const TT t, float lr, float c_lp, int parity, int bx,
                                             int by, int bz) {
    static_assert(TMA || sizeof(TU) == 4, "an FP16 u is staged by tile copies only");
    using S = K4S<RG, NW, OPT, SU, NSTG, TU>;
    constexpr int NT = S::NT, TY = S::TY, RX = S::RX, RY = S::RY, BXW = S::BXW, COFF = S::COFF,
                  XB = S::XB, NR = S::NR, NS = S::NS, NOUT = S::NOUT, URX = S::URX,
                  URY = S::URY, UXB = S::UXB, UBXW = S::UBXW, UCOFF = S::UCOFF, NRU = S::NRU,
                  NSU = S::NSU, NP = S::NP, NJP = S::NJP;
    using G = Region<RY, RX, NW, BXW, COFF>;
    using GU = Region<URY, URX, NW, UBXW, UCOFF>;
    extern __shared__ __align__(128) unsigned char smem[];
    float *ring = (float *)(smem + S::o_ring);
    float *xb = (float *)(smem + S::o_xb);
    unsigned long long *bar = (unsigned long long *)(smem + S::o_bar);
    __shared__ int flag;
    auto stage = [&](int s) { return (float *)(smem + S::o_st + S::st_bytes * s); };

    const int tx = threadIdx.x, wy = threadIdx.y, tid = wy * FX + tx;
    const int x0 = bx * FX, y0 = by * TY, z0 = bz * TZ;
    const int zend = min(z0 + TZ, D);
    const long long N = (long long)D * H * P, HW = (long long)H * P;  // channel, plane strides
    G rg;
    GU rgu;
    if (!TMA) {
        rg.init(wy, tx, y0 - RG, x0 - RG, H, W, P);
        if (SU) rgu.init(wy, tx, y0 - RG - 1, x0 - RG - 1, H, W, P);
    }
    Outs<OPT, NW> ou;
    ou.init(wy, tx, y0, x0, H, W, P);
    if (TMA && tid == 0) {
        for (int k = 0; k <= NSTG; ++k) mbar_init(bar + k);
        mbar_init_fence();
    }
    for (int k = tid; k < NS * 3 * NOUT; k += NT) ring[k] = 0.0f;

    const int zs = z0 - RG, np = zend - z0 + 2 * RG;
    // u plane q lives in u stage (q - (zs - 1)) % NSU
    auto uslot = [&](int q) {
        return (TU *)(smem + S::o_ust + S::ust_bytes * ((q - (zs - 1)) % NSU));
    };
    // group i: d plane zs + i and u plane zs + i + 1
    auto issue = [&](int i) {
        const int zp = zs + i, s = i % NSTG;
        if (TMA) {
            if (tid == 0 && i < np) {
                mbar_expect(bar + s, S::tx_plane + (SU ? S::tx_u : 0u));
                tma4(stage(s), maps.a, x0 - XB, y0 - RG, zp, 0, bar + s);
                if (SU) tma4(uslot(zp + 1), maps.b, x0 - UXB, y0 - RG - 1, zp + 1, 0, bar + s);
            }
        } else {
            if (i < np) {
                rg.template load<3>(stage(s), dir, N, (long long)zp * HW, zp >= 0 && zp < D);
                if constexpr (SU && sizeof(TU) == 4)
                    rgu.template load<3>(uslot(zp + 1), u, N, (long long)(zp + 1) * HW,
                                         zp + 1 >= 0 && zp + 1 < D);
            }
            cp_commit();
        }
    };
    // after the previous kernel: first copies and the step maximum in flight
    // together, then the status check
    pdl_wait();
    // u planes zs - 1 and zs: barrier NSTG (TMA), or cp.async group 0
    if (SU) {
        if (TMA) {
            if (tid == 0) {
                mbar_expect(bar + NSTG, 2u * S::tx_u);
                tma4(uslot(zs - 1), maps.b, x0 - UXB, y0 - RG - 1, zs - 1, 0, bar + NSTG);
                tma4(uslot(zs), maps.b, x0 - UXB, y0 - RG - 1, zs, 0, bar + NSTG);
            }
        } else if constexpr (sizeof(TU) == 4) {
            rgu.template load<3>(uslot(zs - 1), u, N, (long long)(zs - 1) * HW,
                                 zs - 1 >= 0 && zs - 1 < D);
            rgu.template load<3>(uslot(zs), u, N, (long long)zs * HW, zs >= 0 && zs < D);
        }
    }
#pragma unroll
    for (int k = 0; k < NSTG - 1; ++k) issue(k);
    const float mxd = __uint_as_float(h->step_max_bits[parity]);
    if (status_timed_out(h, tid, &flag)) {
        if (SU && TMA && tid == 0) mbar_wait(bar + NSTG, 0u);
        drain_first<TMA, NSTG>(bar, np, tid);
        return;
    }
    const float e = (mxd > 0.0f) ? lr / (c_lp * mxd) : 0.0f;
    bool ok0 = true;
    if (SU && TMA) ok0 = mbar_wait(bar + NSTG, 0u);

    TriPending jp[OPT];
    long long jidx[OPT];
    bool jlive[OPT];
#pragma unroll
    for (int o = 0; o < OPT; ++o) jlive[o] = false;

    // this thread's compose positions (fixed for every plane): plane-layout
    // index (-1: none), inside the grid, and the u stage index of the position
    int pk[NJP], pub[NJP];
    bool pin[NJP];
#pragma unroll
    for (int j = 0; j < NJP; ++j) {
        const int pidx = tid + j * NT;
        int ry, rx;
        compose_position<RY, RX>(pidx, ry, rx);
        const int y = y0 - RG + ry, x = x0 - RG + rx;
        pk[j] = pidx < NP ? ry * BXW + rx + COFF : -1;
        pin[j] = pidx < NP && y >= 0 && y < H && x >= 0 && x < W;
        pub[j] = (ry + 1) * UBXW + (rx + 1) + UCOFF;
    }

    int fail = -1, slot = 0;
    for (int i = 0; i < np; ++i) {
        const int zp = zs + i, zo = zp - RG, s = i % NSTG;
        issue(i + NSTG - 1);
        bool ok = ok0;
        if (TMA)
            ok = mbar_wait(bar + s, (unsigned)(i / NSTG) & 1u) && ok;
        else
            cp_wait<NSTG - 1>();
        if (__syncthreads_or(!ok)) {  // the stages hold neighbours' copies
            fail = i;
            break;
        }
        float Q[OPT][3];
        if (zp >= 0 && zp < D) {
            // u' replaces d in the stage, position by position (each thread
            // reads its positions' d before it writes them)
            float *ds = stage(s);
            const TU *um = uslot(zp - 1), *u0 = uslot(zp), *u1 = uslot(zp + 1);
            // u' on the RY x RX region (positions spread over all threads),
            // at the plane layout's columns
#pragma unroll
            for (int j = 0; j < NJP; ++j) {
                const int k = pk[j];
                if (NP % NT != 0 && k < 0) break;
                float a = 0.f, b = 0.f, c = 0.f;
                if (pin[j]) {
                    const float dz = -e * ds[k], dy = -e * ds[NR + k], dx = -e * ds[2 * NR + k];
                    if (SU) {
                        // cell corners lie within one voxel: planes zp-1..zp+1
                        if (dz > -1.0f && dz < 1.0f && dy > -1.0f && dy < 1.0f &&
                            dx > -1.0f && dx < 1.0f) {
                            // the corners are this voxel and its neighbours on
                            // the side of the step's sign, weighted by |delta|
                            // (the cell and weights of tri_issue_step)
                            const float tz = fabsf(dz), ty = fabsf(dy), tx2 = fabsf(dx);
                            const TU *pa = u0, *pb = dz < 0.0f ? um : u1;
                            const int b0 = pub[j], oy = dy < 0.0f ? -UBXW : UBXW,
                                      ox = dx < 0.0f ? -1 : 1;
                            // channels 0 and 1 as a packed pair (each component
                            // exactly the scalar fadd / fmaf), channel 2 alone
                            auto pair = [&](const TU *P, int o) {
                                return make_float2(st_load(P[b0 + o]), st_load(P[NRU + b0 + o]));
                            };
                            auto lerp2 = [](float t, float2 lo, float2 hi) {
                                return __ffma2_rn(make_float2(t, t),
                                                  __fadd2_rn(hi, make_float2(-lo.x, -lo.y)), lo);
                            };
                            const float2 c00 = lerp2(tx2, pair(pa, 0), pair(pa, ox));
                            const float2 c01 = lerp2(tx2, pair(pa, oy), pair(pa, oy + ox));
                            const float2 c10 = lerp2(tx2, pair(pb, 0), pair(pb, ox));
                            const float2 c11 = lerp2(tx2, pair(pb, oy), pair(pb, oy + ox));
                            const float2 r01 = lerp2(tz, lerp2(ty, c00, c01), lerp2(ty, c10, c11));
                            const TU *Ap = pa + 2 * NRU + b0, *Bp = pb + 2 * NRU + b0;
                            const float A[2] = {st_load(Ap[0]), st_load(Ap[ox])},
                                        A2[2] = {st_load(Ap[oy]), st_load(Ap[oy + ox])},
                                        B[2] = {st_load(Bp[0]), st_load(Bp[ox])},
                                        B2[2] = {st_load(Bp[oy]), st_load(Bp[oy + ox])};
                            const float e00 = fmaf(tx2, A[1] - A[0], A[0]);
                            const float e01 = fmaf(tx2, A2[1] - A2[0], A2[0]);
                            const float e10 = fmaf(tx2, B[1] - B[0], B[0]);
                            const float e11 = fmaf(tx2, B2[1] - B2[0], B2[0]);
                            const float e0 = fmaf(ty, e01 - e00, e00);
                            const float e1 = fmaf(ty, e11 - e10, e10);
                            const float2 ab = __fadd2_rn(make_float2(dz, dy), r01);
                            a = ab.x;
                            b = ab.y;
                            c = dx + fmaf(tz, e1 - e0, e0);
                        } else {
                            a = b = c = __int_as_float(0x7fc00000);  // impossible step: flag it
                        }
                    } else {
                        int ry, rx;
                        compose_position<RY, RX>(tid + j * NT, ry, rx);
                        const int y = y0 - RG + ry, x = x0 - RG + rx;
                        float gz, gy, gx;
                        TriPending q;
                        tri_issue_step(q, u, D, H, W, P, zp, y, x, dz, dy, dx);
                        a = dz + tri_finish<false>(q, gz, gy, gx);
                        tri_issue_step(q, u + N, D, H, W, P, zp, y, x, dz, dy, dx);
                        b = dy + tri_finish<false>(q, gz, gy, gx);
                        tri_issue_step(q, u + 2 * N, D, H, W, P, zp, y, x, dz, dy, dx);
                        c = dx + tri_finish<false>(q, gz, gy, gx);
                    }
                }
                ds[k] = a;
                ds[NR + k] = b;
                ds[2 * NR + k] = c;
            }
            if (TMA) proxy_fence_async();  // the stage is refilled by a tile copy later
            __syncthreads();
            gauss_x4<RG, 3, RY, BXW, COFF, NT>(ds, xb, t, tid);
            __syncthreads();
            gauss_y3<RG, RY, NW, OPT>(xb, t, wy, tx, Q);
        } else {
#pragma unroll
            for (int o = 0; o < OPT; ++o) Q[o][0] = Q[o][1] = Q[o][2] = 0.0f;
        }
        ring_put<NS, OPT, NOUT, NT>(ring, slot, tid, Q);
        const int newest = slot;
        slot = (slot + 1 == NS) ? 0 : slot + 1;
        if (zo >= z0 && zo < zend) {
            const long long zoff = (long long)zo * HW;
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                // finish the previous plane's warped value first (its loads have landed)
                if (jlive[o]) {
                    float gz, gy, gx;
                    Jout[jidx[o]] = tri_finish<true>(jp[o], gz, gy, gx);
                    gJout[jidx[o]] = gz;
                    gJout[N + jidx[o]] = gy;
                    gJout[2 * N + jidx[o]] = gx;
                    jlive[o] = false;
                }
                if (ou.off[o] < 0) continue;
                float sz[3];
                gauss_z3<RG, NOUT>(ring + o * NT + tid, newest, t, sz);
                const long long gi = zoff + ou.off[o];
                const float a = sz[0], b = sz[1], c = sz[2];
                // the stored (for FP16, rounded) u is the one the next steps read
                const TU sa = st_store<TU>(a), sb = st_store<TU>(b), sc = st_store<TU>(c);
                uo[gi] = sa;
                uo[N + gi] = sb;
                uo[2 * N + gi] = sc;
                tri_issue_p(jp[o], Im, D, H, W, P, zo, y0 + wy + NW * o, x0 + tx, st_load(sa),
                            st_load(sb), st_load(sc));
                jidx[o] = gi;
                jlive[o] = true;
            }
        }
    }
    if (fail >= 0) {
        if (tid == 0) {
            status_set(&h->status, ST_TIMEOUT);
            if (SU && !ok0) mbar_wait(bar + NSTG, 0u);
            drain<NSTG>(bar, fail, np);
        }
        return;
    }
#pragma unroll
    for (int o = 0; o < OPT; ++o)
        if (jlive[o]) {
            float gz, gy, gx;
            Jout[jidx[o]] = tri_finish<true>(jp[o], gz, gy, gx);
            gJout[jidx[o]] = gz;
            gJout[N + jidx[o]] = gy;
            gJout[2 * N + jidx[o]] = gx;
        }
    if (!TMA) cp_wait<0>();
    // per-iteration header fields for the next iteration (nobody else reads them now)
    if (bx == 0 && by == 0 && bz == 0 && tid == 0) {
        for (int c = 0; c < 8; ++c) h->coef_max_bits[c] = 0u;
        h->step_max_bits[parity ^ 1] = 0u;
        h->loss_acc = 0ull;
        h->eps_t = e;
    }
}

template <int RG, int NW, int OPT, bool SU, int NSTG, bool TMA, class TU = float>
__global__ void __launch_bounds__(FX *NW, NW >= 16 ? 2 : 1) k_compose(const __grid_constant__ Maps maps,
                                                    const TU *__restrict__ u,
                                                    const float *__restrict__ dir,
                                                    TU *__restrict__ uo,
                                                    const float *__restrict__ Im,
                                                    float *__restrict__ Jout,
                                                    float *__restrict__ gJout,
                                                    WsHeader *__restrict__ h, int D, int H, int W,
                                                    int P, int TZ, GaussTaps t, float lr,
                                                    float c_lp, int parity) {
    compose_body<RG, NW, OPT, SU, NSTG, TMA>(map_ref(maps), u, dir, uo, Im, Jout, gJout, h, D, H, W, P, TZ,
                                             t, lr, c_lp, parity, blockIdx.x, blockIdx.y,
                                             blockIdx.z);
}

// ================================================================ launch helpers

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

// Opts the kernel into its dynamic shared memory and returns its resident
// CTAs per SM (called once per kernel instantiation).
template <class K>
int prepare(K kernel, size_t smem, int threads) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
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

// Launch with programmatic stream serialization (see pdl_wait).
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), const LaunchGeom &g, size_t smem, cudaStream_t s,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g.grid;
    cfg.blockDim = g.block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// tile shapes (warps per CTA, outputs per thread along y) and pipeline depths
// of the TMA and of the cp.async variant
constexpr int K1_NW = 8, K1_OPT = 1, K1_ST_TMA = 3, K1_ST_CP = 3;
constexpr int K2_NW = 8, K2_OPT = 1, K2_ST_TMA = 2, K2_ST_CP = 2;
constexpr int K3_NW = 8, K3_OPT = 1, K3_ST_TMA = 2, K3_ST_CP = 2;
constexpr int K4_NW = 8, K4_OPT = 1, K4_ST_TMA = 2, K4_ST_CP = 2;

// Gaussians up to this radius run inside the fused kernels
constexpr int kMaxFusedRG = kMaxFusedRadius;

}  // namespace

}  // namespace fa
