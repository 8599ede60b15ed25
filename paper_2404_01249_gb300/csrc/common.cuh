// Shared device helpers of libfa (sm_103a).  Nothing here is numerical
// policy beyond what fa.h states: trilinear sampling with zero outside the
// grid, fixed-point scaling for exact window sums, status-word bits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fa.h"

namespace fa {

// ---------------------------------------------------------------- host side
void set_error(const char *fmt, ...);
void clear_error();
fa_status cuda_fail(cudaError_t e, const char *where);
// Counts kernel launches made by this library (read with fa_launch_count);
// a replayed graph adds the kernels it holds.
void note_launch();
void note_launches(unsigned long long n);
unsigned long long launches_so_far();
// Identity of the CUDA context current on the calling thread (the
// runtime's primary context of the current device, made current first):
// the driver's unique context id, which a new context after a device reset
// never repeats.  0 when the driver does not provide it.  Host caches of
// device addresses or streams key on it.
cudaError_t current_context_id(unsigned long long *id);

#define FA_CUDA_TRY(expr)                                           \
    do {                                                            \
        cudaError_t _e = (expr);                                    \
        if (_e != cudaSuccess) return ::fa::cuda_fail(_e, #expr);   \
    } while (0)

#define FA_TRY(expr)                        \
    do {                                    \
        fa_status _s = (expr);              \
        if (_s != FA_OK) return _s;         \
    } while (0)

// Device status word bits (FA_ERR_NONFINITE / FA_ERR_TIMEOUT on the host).
enum : unsigned { ST_NONFINITE = 1u, ST_TIMEOUT = 2u };

// Workspace header, at offset 0 of every workspace libfa uses.  256 bytes.
struct WsHeader {
    unsigned status;           // sticky status bits of this call
    unsigned absmax_bits[2];   // max |I|, max |J| (float bits, non-negative)
    unsigned coef_max_bits[8]; // max |coefficient| per LNCC adjoint channel
    unsigned step_max_bits[2]; // max_x |d(x)| per iteration parity (float bits)
    unsigned pad0;
    unsigned long long loss_acc; // sum of cc (or squared error) in 2^-32 fixed point
    float loss;                // final loss of the last reduction
    float eps_t;               // last step size
    unsigned pbar_count;       // grid barriers of a persistent launch: arrivals
    unsigned pbar_abort;       // set when a persistent launch is abandoned
    unsigned char pad[256 - 4 - 8 - 32 - 8 - 4 - 8 - 8 - 8];
};
static_assert(sizeof(WsHeader) == 256, "header must be 256 bytes");

// Carves 256-byte aligned regions from a caller workspace.
struct WsCarver {
    char *base;
    size_t cap, off;
    bool ok;
    WsCarver(void *b, size_t c) : base((char *)b), cap(c), off(0), ok(true) {}
    template <class T>
    T *take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (off + bytes > cap) {
            ok = false;
            return nullptr;
        }
        T *p = base ? (T *)(base + off) : nullptr;
        off += bytes;
        return p;
    }
};

// -------------------------------------------------------------- device side
__device__ __forceinline__ void status_set(unsigned *st, unsigned bits) { atomicOr(st, bits); }

// Non-negative floats order like their bit patterns.
__device__ __forceinline__ void atomic_max_nonneg(unsigned *slot, float v) {
    atomicMax(slot, __float_as_uint(v));
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide max of non-negative values, then one atomic per block.
// Every thread of the block must call it.
__device__ __forceinline__ void block_max_to(unsigned *slot, float v, float *red /*>=32*/) {
    int lane = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    int nthr = blockDim.x * blockDim.y * blockDim.z;
    v = warp_max(v);
    if ((lane & 31) == 0) red[lane >> 5] = v;
    __syncthreads();
    if (lane < 32) {
        float w = (lane < (nthr + 31) / 32) ? red[lane] : 0.0f;
        w = warp_max(w);
        if (lane == 0 && w > 0.0f) atomic_max_nonneg(slot, w);
    }
    __syncthreads();
}

__device__ __forceinline__ void block_sum_to(unsigned long long *slot, unsigned long long v,
                                             unsigned long long *red /*>=32*/) {
    int lane = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    int nthr = blockDim.x * blockDim.y * blockDim.z;
    v = warp_sum_u64(v);
    if ((lane & 31) == 0) red[lane >> 5] = v;
    __syncthreads();
    if (lane < 32) {
        unsigned long long w = (lane < (nthr + 31) / 32) ? red[lane] : 0ull;
        w = warp_sum_u64(w);
        if (lane == 0 && w) atomicAdd(slot, w);
    }
    __syncthreads();
}

// Trilinear sample of v at (z + uz, y + uy, x + ux) with zero outside the
// grid, split in two halves so that the eight corner loads can be issued
// early and consumed later.  The cell is floor of the position (integer
// part taken from u so the fraction keeps full precision); gradients are the
// interpolant's partial derivatives inside that cell.  NaN displacement
// gives NaN; a displacement of magnitude >= 2^20 voxels samples outside.
struct TriPending {
    float c000, c001, c010, c011, c100, c101, c110, c111;
    float tz, ty, tx;
};

// A stored field value as FP32 (FP32, or FP16 read exactly).
__device__ __forceinline__ float ld_field(const float *q) { return __ldg(q); }
__device__ __forceinline__ float ld_field(const __half *q) { return __half2float(__ldg(q)); }

// tri_issue_p: the same for a buffer of row pitch P (>= W; zero outside the
// logical D x H x W grid whatever the padding holds), of FP32 or FP16 values.
template <class T>
__device__ __forceinline__ void tri_issue_p(TriPending &p, const T *__restrict__ v, int D,
                                            int H, int W, int P, int z, int y, int x, float uz,
                                            float uy, float ux) {
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
    // 32-bit offsets: buffers hold fewer than 2^31 elements and iz >= -1
    if (iz >= 0 && iz + 1 < D && iy >= 0 && iy + 1 < H && ix >= 0 && ix + 1 < W) {
        const T *q0 = v + (iz * H + iy) * P + ix, *q1 = q0 + H * P;  // the whole cell inside
        p.c000 = ld_field(q0);
        p.c001 = ld_field(q0 + 1);
        p.c010 = ld_field(q0 + P);
        p.c011 = ld_field(q0 + P + 1);
        p.c100 = ld_field(q1);
        p.c101 = ld_field(q1 + 1);
        p.c110 = ld_field(q1 + P);
        p.c111 = ld_field(q1 + P + 1);
        return;
    }
    if (iz < -1 || iz >= D || iy < -1 || iy >= H || ix < -1 || ix >= W) return;
    const bool z0 = iz >= 0, z1 = iz + 1 < D;
    const bool y0 = iy >= 0, y1 = iy + 1 < H;
    const bool x0 = ix >= 0, x1 = ix + 1 < W;
    const int b = (iz * H + iy) * P + ix;
    const T *q0 = v + b, *q1 = q0 + H * P;
    if (z0 && y0 && x0) p.c000 = ld_field(q0);
    if (z0 && y0 && x1) p.c001 = ld_field(q0 + 1);
    if (z0 && y1 && x0) p.c010 = ld_field(q0 + P);
    if (z0 && y1 && x1) p.c011 = ld_field(q0 + P + 1);
    if (z1 && y0 && x0) p.c100 = ld_field(q1);
    if (z1 && y0 && x1) p.c101 = ld_field(q1 + 1);
    if (z1 && y1 && x0) p.c110 = ld_field(q1 + P);
    if (z1 && y1 && x1) p.c111 = ld_field(q1 + P + 1);
}

// The compose's sample u(x + delta) at a grid voxel (z, y, x): for a step
// shorter than one voxel on every axis the cell's corners are the voxel itself
// and its neighbours on the side of each component's sign, with the exact
// weights |delta| (so u is sampled exactly when delta is 0 on an axis); longer
// steps take tri_issue_p's cell.  tri_finish completes either.
template <class T>
__device__ __forceinline__ void tri_issue_step(TriPending &p, const T *__restrict__ v, int D,
                                               int H, int W, int P, int z, int y, int x,
                                               float uz, float uy, float ux) {
    if (!(fabsf(uz) < 1.0f && fabsf(uy) < 1.0f && fabsf(ux) < 1.0f)) {
        tri_issue_p(p, v, D, H, W, P, z, y, x, uz, uy, ux);
        return;
    }
    p.tz = fabsf(uz);
    p.ty = fabsf(uy);
    p.tx = fabsf(ux);
    const int sz = uz < 0.0f ? -1 : 1, sy = uy < 0.0f ? -1 : 1, sx = ux < 0.0f ? -1 : 1;
    const bool zo = z + sz >= 0 && z + sz < D, yo = y + sy >= 0 && y + sy < H,
               xo = x + sx >= 0 && x + sx < W;
    // 32-bit offsets: buffers hold fewer than 2^31 elements
    const T *q0 = v + (z * H + y) * P + x, *q1 = q0 + sz * H * P;
    const int oy = sy * P;
    p.c000 = ld_field(q0);
    p.c001 = xo ? ld_field(q0 + sx) : 0.0f;
    p.c010 = yo ? ld_field(q0 + oy) : 0.0f;
    p.c011 = yo && xo ? ld_field(q0 + oy + sx) : 0.0f;
    p.c100 = zo ? ld_field(q1) : 0.0f;
    p.c101 = zo && xo ? ld_field(q1 + sx) : 0.0f;
    p.c110 = zo && yo ? ld_field(q1 + oy) : 0.0f;
    p.c111 = zo && yo && xo ? ld_field(q1 + oy + sx) : 0.0f;
}

__device__ __forceinline__ void tri_issue(TriPending &p, const float *__restrict__ v, int D,
                                          int H, int W, int z, int y, int x, float uz, float uy,
                                          float ux) {
    tri_issue_p(p, v, D, H, W, W, z, y, x, uz, uy, ux);
}

template <bool GRAD>
__device__ __forceinline__ float tri_finish(const TriPending &p, float &gz, float &gy, float &gx) {
    const float tz = p.tz, ty = p.ty, tx = p.tx;
    float c00 = fmaf(tx, p.c001 - p.c000, p.c000);
    float c01 = fmaf(tx, p.c011 - p.c010, p.c010);
    float c10 = fmaf(tx, p.c101 - p.c100, p.c100);
    float c11 = fmaf(tx, p.c111 - p.c110, p.c110);
    float c0 = fmaf(ty, c01 - c00, c00);
    float c1 = fmaf(ty, c11 - c10, c10);
    if (GRAD) {
        gz = c1 - c0;
        gy = fmaf(tz, (c11 - c10) - (c01 - c00), c01 - c00);
        float d00 = p.c001 - p.c000, d01 = p.c011 - p.c010, d10 = p.c101 - p.c100,
              d11 = p.c111 - p.c110;
        float d0 = fmaf(ty, d01 - d00, d00), d1 = fmaf(ty, d11 - d10, d10);
        gx = fmaf(tz, d1 - d0, d0);
    } else {
        gz = gy = gx = 0.0f;
    }
    return fmaf(tz, c1 - c0, c0);
}

template <bool GRAD>
__device__ __forceinline__ float tri_sample(const float *__restrict__ v, int D, int H, int W,
                                            int z, int y, int x, float uz, float uy, float ux,
                                            float &gz, float &gy, float &gx) {
    TriPending p;
    tri_issue(p, v, D, H, W, z, y, x, uz, uy, ux);
    return tri_finish<GRAD>(p, gz, gy, gx);
}

template <bool GRAD, class T>
__device__ __forceinline__ float tri_sample_p(const T *__restrict__ v, int D, int H, int W,
                                              int P, int z, int y, int x, float uz, float uy,
                                              float ux, float &gz, float &gy, float &gx) {
    TriPending p;
    tri_issue_p(p, v, D, H, W, P, z, y, x, uz, uy, ux);
    return tri_finish<GRAD>(p, gz, gy, gx);
}

// ---------------------------------------------------------- fixed point
// Window sums of images run in 64-bit integers: values are quantised as
// q = rint(v * 2^s) with |q| <= 2^b (b from lncc_image_bits), so every sum
// is exact (associative, order-independent).

// Image bits used by every LNCC path: with |q| <= 2^b every 3-D window sum
// of n products stays below 2^62 (b = floor((62 - ceil(log2 n)) / 2)); the
// numerators n S_II - S_I^2 are then formed exactly in 128-bit integers.
__host__ __device__ inline int lncc_image_bits(int window) {
    long long n = (long long)window * window * window;
    int lg = 0;
    while ((1ll << lg) < n) ++lg;
    return (62 - lg) / 2;
}

// Bits of the quantised LNCC adjoint coefficients: 3-D sums stay below 2^47
// so that they convert to float-float exactly, and every quantised value
// stays below 2^41 (the range of quantize below).
__host__ __device__ inline int lncc_coef_bits(int window) {
    long long n = (long long)window * window * window;
    int lg = 0;
    while ((1ll << lg) < n) ++lg;
    return 47 - lg < 41 ? 47 - lg : 41;
}

// Exponent s with max|v| * 2^s <= 2^bits (0 if amax is 0 or not finite).
__device__ __forceinline__ int fixed_shift(float amax, int bits) {
    if (!(amax > 0.0f) || !(amax <= 3.4e38f)) return 0;
    int e;
    frexpf(amax, &e);  // amax = m 2^e, m in [0.5, 1)  =>  amax < 2^e
    int s = bits - e;
    return s < -126 ? -126 : (s > 127 ? 127 : s);
}

// q = rint(v * scale) (round half to even) for |v * scale| < 2^42, scale a
// power of two.  Built from FP32 adds instead of the 64-bit float-to-integer
// conversion, which issues at a small fraction of the ALU rate on sm_103:
// adding and subtracting 1.5 * 2^43 rounds x to a multiple of 2^20, the
// remainder (exact, |r| <= 2^19) is rounded by adding 1.5 * 2^23, and both
// integers are read from the bits of floats in the binade [2^23, 2^24).
__device__ __forceinline__ long long quantize(float v, float scale) {
    const float x = v * scale;
    const float M43 = 13194139533312.0f, M23 = 12582912.0f;
    const float h = __fsub_rn(__fadd_rn(x, M43), M43);
    const float r = __fsub_rn(x, h);
    const int k = __float_as_int(__fmaf_rn(h, 9.5367431640625e-07f, M23)) - 0x4B400000;
    const int l = __float_as_int(__fadd_rn(r, M23)) - 0x4B400000;
    return ((long long)k << 20) + l;
}

// The conversions below avoid the 64-bit integer-to-float instruction, which
// on sm_103 runs on the narrow FP64 pipe (about 2 per clock per SM) and
// limited the exact-sum kernels; they use 32-bit conversions, integer
// operations and FP32 adds, and give the same bits as that instruction.

// uint64 -> float, rounded to nearest even: the leading 24 bits, rounded by
// the 40 bits below them (a carry out of the mantissa raises the exponent).
__device__ __forceinline__ float u64_to_float_rn(unsigned long long u) {
    if (u == 0ull) return 0.0f;
    const int lz = __clzll((long long)u);
    const unsigned long long m = u << lz;  // bit 63 set
    unsigned mant = (unsigned)(m >> 40);   // 24 bits, the leading one included
    const unsigned long long rest = m & 0xFFFFFFFFFFull, half = 1ull << 39;
    mant += (rest > half || (rest == half && (mant & 1u))) ? 1u : 0u;
    return __uint_as_float(((unsigned)(190 - lz) << 23) + (mant - 0x800000u));
}

__device__ __forceinline__ float i64_to_float_rn(long long x) {
    const float f = u64_to_float_rn(x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x);
    return x < 0 ? -f : f;
}

// int64 -> (hi, lo) floats with hi + lo == x exactly for |x| < 2^48: hi is x
// rounded to nearest, lo = x - hi.  x = a 2^24 + b with |a| < 2^24 and
// 0 <= b < 2^24, both exact in FP32; hi = a 2^24 + b rounded, and lo is the
// exact error of that sum (|a 2^24| >= b unless a = 0).
__device__ __forceinline__ void i64_to_ff(long long x, float &hi, float &lo) {
    const float fh = __int2float_rn((int)(x >> 24)) * 16777216.0f;
    const float fl = __uint2float_rn((unsigned)x & 0xFFFFFFu);
    hi = __fadd_rn(fh, fl);
    lo = __fsub_rn(fl, __fsub_rn(hi, fh));
}

// n a - b c for int64 operands, formed exactly in 128 bits and rounded to
// float (one rounding when the result fits 64 bits; otherwise the two halves
// are scaled and added, within one float ulp).
__device__ __forceinline__ float diff_i128_to_float(long long n, long long a, long long b,
                                                    long long c) {
    const __int128 r = (__int128)n * a - (__int128)b * c;
    const long long hi = (long long)(r >> 64);
    const unsigned long long lo = (unsigned long long)r;
    if (hi == 0) return u64_to_float_rn(lo);
    if (hi == -1 && (long long)lo < 0) return i64_to_float_rn((long long)lo);
    // |hi| < 2^24 here (|r| < 2^88), so its 32-bit conversion is exact
    return fmaf(__int2float_rn((int)hi), 18446744073709551616.0f, u64_to_float_rn(lo));
}

// ---------------------------------------------------------- float-float
__device__ __forceinline__ void ff_two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void ff_add(float &h, float &l, float bh, float bl) {
    float s, e;
    ff_two_sum(h, bh, s, e);
    e += l + bl;
    h = s + e;
    l = e - (h - s);
}

// (hi, lo) of a * (xh + xl) for a float a and a float-float x.
__device__ __forceinline__ void ff_mul_f(float a, float xh, float xl, float &h, float &l) {
    h = a * xh;
    l = fmaf(a, xh, -h);
    l = fmaf(a, xl, l);
}

// Adjoint coefficient C = -(A S_I + 2 B S_J) / n of the LNCC gradient as a
// float-float pair, from the exact window sums (scaled by 2^s, inv_s = 2^-s)
// and the rounded float A, B.  Forming C from the same rounded A, B that are
// summed keeps I(y) sum A + sum C free of their rounding; the pair keeps the
// ~2^-44 relative accuracy the cancellation between those two sums needs.
__device__ __forceinline__ void lncc_c_ff(float A, float B, long long sI, long long sJ,
                                          float inv_s, float nf, float inv_nf, float &ch,
                                          float &cl) {
    float ih, il, jh, jl;
    i64_to_ff(sI, ih, il);
    i64_to_ff(sJ, jh, jl);
    ih *= inv_s;
    il *= inv_s;
    jh *= inv_s;
    jl *= inv_s;
    const float i1 = ih * inv_nf, i2 = (fmaf(-i1, nf, ih) + il) * inv_nf;  // mean of I
    const float j1 = jh * inv_nf, j2 = (fmaf(-j1, nf, jh) + jl) * inv_nf;  // mean of J
    float ph, pl, th, tl;
    ff_mul_f(A, i1, i2, ph, pl);
    ff_mul_f(2.0f * B, j1, j2, th, tl);
    ff_add(ph, pl, th, tl);
    ch = -ph;
    cl = -pl;
}

// Storage of the Adam moments: FP32, or 16-bit values read as FP32 and
// written rounded to nearest (all arithmetic is FP32).
__device__ __forceinline__ float st_load(float x) { return x; }
__device__ __forceinline__ float st_load(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float st_load(__half x) { return __half2float(x); }
template <class T>
__device__ __forceinline__ T st_store(float x);
template <>
__device__ __forceinline__ float st_store<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 st_store<__nv_bfloat16>(float x) {
    return __float2bfloat16_rn(x);
}
template <>
__device__ __forceinline__ __half st_store<__half>(float x) { return __float2half_rn(x); }
// A 16-bit stored value given by its bits, as FP32 (exact).
template <class T>
__device__ __forceinline__ float st_bits(unsigned short b);
template <>
__device__ __forceinline__ float st_bits<__nv_bfloat16>(unsigned short b) {
    return __uint_as_float((unsigned)b << 16);
}
template <>
__device__ __forceinline__ float st_bits<__half>(unsigned short b) {
    return __half2float(__ushort_as_half(b));
}
// A stored moment as loaded (an FP32 value, or the bits of a 16-bit one), as FP32.
template <class T>
__device__ __forceinline__ float st_value(float x) { return x; }
template <class T>
__device__ __forceinline__ float st_value(unsigned short b) { return st_bits<T>(b); }

// Adam direction d = (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps) with the
// bias corrections passed as reciprocals; square root and quotient use the
// hardware approximations (a few ulp).
__device__ __forceinline__ float adam_dir(float m, float v, float rbc1, float rbc2, float eps) {
    const float vh = v * rbc2;
    const float sq = vh > 0.0f ? vh * rsqrtf(vh) : 0.0f;
    return __fdividef(m * rbc1, sq + eps);
}

// 2^s as a float for s in [-126, 127] (clamped).
__device__ __forceinline__ float pow2f(int s) {
    s = s < -126 ? -126 : (s > 127 ? 127 : s);
    return __int_as_float((127 + s) << 23);
}

// Launch geometry for voxel-parallel kernels: 32 x 8 threads per (x, y)
// tile, one grid layer per z-slice.
struct VoxGrid {
    dim3 block, grid;
    VoxGrid(int D, int H, int W) : block(32, 8, 1), grid((W + 31) / 32, (H + 7) / 8, D) {}
};

}  // namespace fa
