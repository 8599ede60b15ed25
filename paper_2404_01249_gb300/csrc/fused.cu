// Fused per-iteration kernels of fa_register (FA_MODE_FUSED): launching,
// tile choices, tensor maps and the per-iteration driver.  The kernels
// themselves are in fused_kernels.cuh.
#include "fused_kernels.cuh"

#include <map>
#include <mutex>
#include <unordered_map>

namespace fa {

namespace {

// ================================================================ launching

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

// ------------------------------------------------------------- tile choices
// Per (kernel, radius, compose variant, level grid): the slab depth TZ
// (0: the cost model above) and, for K3/K4 on the TMA path, 32 x 16 tiles
// of 16 warps instead of 32 x 8.  fa_autotune measures candidates and fills
// the table; every choice computes the same bits.
struct TileChoice {
    int wide, tz;
};
struct TuneKey {
    int kernel, radius, su, D, H, W;
    bool operator<(const TuneKey &o) const {
        const int a[6] = {kernel, radius, su, D, H, W}, b[6] = {o.kernel, o.radius, o.su, o.D, o.H, o.W};
        for (int i = 0; i < 6; ++i)
            if (a[i] != b[i]) return a[i] < b[i];
        return false;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, TileChoice> g_tune;
thread_local const TileChoice *g_force = nullptr;  // a candidate under measurement

constexpr int kDefaultWide[4] = {0, 0, 0, 1};

TileChoice tile_choice(int kernel, int radius, int su, Dims d) {
    if (g_force) return *g_force;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(TuneKey{kernel, radius, su, d.D, d.H, d.W});
    if (it != g_tune.end()) return it->second;
    return TileChoice{kDefaultWide[kernel], 0};
}

inline LaunchGeom geometry(int occ, int nw, int ty, int halo, Dims d, int tz = 0) {
    LaunchGeom g;
    const int gx = (d.W + FX - 1) / FX, gy = (d.H + ty - 1) / ty;
    g.tz = tz > 0 ? (tz < d.D ? tz : d.D) : choose_tz(d.D, gx * gy, halo, occ);
    g.grid = dim3(gx, gy, (d.D + g.tz - 1) / g.tz);
    g.block = dim3(FX, nw);
    return g;
}

// ------------------------------------------------------------- tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (EncodeTiledFn)p;
    }();
    return fn;
}

struct MapKey {
    const void *base;
    int esize, D, H, W, P, C, bx, by, bc;
    bool operator==(const MapKey &o) const {
        return base == o.base && esize == o.esize && D == o.D && H == o.H && W == o.W &&
               P == o.P && C == o.C && bx == o.bx && by == o.by && bc == o.bc;
    }
};
struct MapKeyHash {
    size_t operator()(const MapKey &k) const {
        unsigned long long h = (unsigned long long)(uintptr_t)k.base;
        const int f[9] = {k.esize, k.D, k.H, k.W, k.P, k.C, k.bx, k.by, k.bc};
        for (int v : f) h = (h ^ (unsigned)v) * 0x100000001b3ull;
        return (size_t)h;
    }
};

}  // namespace

// Map of a [C][D][H][W] field of 2- (FP16), 4- or 8-byte elements (rows of d.pitch()
// elements) with a {bx, by, 1, bc} box, zero fill outside the D x H x W grid
// (so a padded row's tail is never read).  Encoded maps are kept per host
// thread (a map is a function of its key alone; a lockstep batch reuses a
// few hundred).  False when the field does not meet TMA's alignment rules
// (base and row pitch multiples of 16 bytes).
bool tmap(CUtensorMap *m, const void *base, int esize, Dims d, int C, int bx, int by, int bc) {
    thread_local std::unordered_map<MapKey, CUtensorMap, MapKeyHash> cache;
    const MapKey key{base, esize, d.D, d.H, d.W, d.pitch(), C, bx, by, bc};
    auto it = cache.find(key);
    if (it != cache.end()) {
        *m = it->second;
        return true;
    }
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const long long P = d.pitch();
    if (((uintptr_t)base & 15u) != 0 || (P * esize) % 16 != 0 || (d.NP() * esize) % 16 != 0)
        return false;
    cuuint64_t dims[4] = {(cuuint64_t)d.W, (cuuint64_t)d.H, (cuuint64_t)d.D, (cuuint64_t)C};
    cuuint64_t strides[3] = {(cuuint64_t)P * esize, (cuuint64_t)P * d.H * esize,
                             (cuuint64_t)d.NP() * esize};
    cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1u, (cuuint32_t)bc};
    cuuint32_t es[4] = {1u, 1u, 1u, 1u};
    CUtensorMap tm;
    const CUtensorMapDataType dt = esize == 8   ? CU_TENSOR_MAP_DATA_TYPE_INT64
                                   : esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = fn(&tm, dt,
                    4, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    if (cache.size() >= 4096) cache.clear();
    cache.emplace(key, tm);
    *m = tm;
    return true;
}

namespace {


template <int R>
cudaError_t launch_k1(const float *If, const float *J, const long long *sI, const float *varI,
                      float *coef, WsHeader *h, Dims d, int window, float cc_eps, bool wc,
                      cudaStream_t s) {
    const int bits = lncc_image_bits(window);
    Maps mp{};
    cudaError_t le;
    using ST = K1S<R, K1_NW, K1_OPT, K1_ST_TMA>;
    const bool tma = tmap(&mp.a, If, 4, d, 1, ST::BXW, ST::RY, 1) &&
                     tmap(&mp.b, J, 4, d, 1, ST::BXW, ST::RY, 1);
    const TileChoice tc = tile_choice(0, R, 0, d);
    if (tma) {
        auto kern = k_lncc_fwd<R, K1_NW, K1_OPT, K1_ST_TMA, true>;
        static const int occ = prepare(kern, ST::bytes, ST::NT);
        LaunchGeom g = geometry(occ, K1_NW, ST::TY, R, d, tc.tz);
        le = launch_pdl(kern, g, ST::bytes, s, mp, If, J, sI, varI, coef, h, d.D, d.H, d.W, d.pitch(), g.tz,
                                                bits, cc_eps, window, wc ? 1 : 0);
    } else {
        using SC = K1S<R, K1_NW, K1_OPT, K1_ST_CP>;
        auto kern = k_lncc_fwd<R, K1_NW, K1_OPT, K1_ST_CP, false>;
        static const int occ = prepare(kern, SC::bytes, SC::NT);
        LaunchGeom g = geometry(occ, K1_NW, SC::TY, R, d, tc.tz);
        le = launch_pdl(kern, g, SC::bytes, s, mp, If, J, sI, varI, coef, h, d.D, d.H, d.W, d.pitch(), g.tz,
                                                bits, cc_eps, window, wc ? 1 : 0);
    }
    note_launch();
    return le;
}

// WDJ: the adjoint's variant, which also writes dL/dJ to dJout.
template <int R, bool WDJ = false>
cudaError_t launch_k2(const float *If, const float *gJ, const float *J, const float *coef,
                      WsHeader *h, float *g, Dims d, int window, cudaStream_t s,
                      float *dJout = nullptr) {
    const int cb = lncc_coef_bits(window);
    Maps mp{};
    cudaError_t le;
    using ST = K2S<R, K2_NW, K2_OPT, K2_ST_TMA>;
    const bool tma = tmap(&mp.a, coef, 4, d, 4, ST::BXW, ST::RY, 4);
    const TileChoice tc = tile_choice(1, R, 0, d);
    if (tma) {
        auto kern = k_lncc_grad<R, K2_NW, K2_OPT, K2_ST_TMA, true, WDJ>;
        static const int occ = prepare(kern, ST::bytes, ST::NT);
        LaunchGeom gg = geometry(occ, K2_NW, ST::TY, R, d, tc.tz);
        le = launch_pdl(kern, gg, ST::bytes, s, mp, If, gJ, J, coef, h, g, d.D, d.H, d.W, d.pitch(), gg.tz,
                        cb, dJout);
    } else {
        using SC = K2S<R, K2_NW, K2_OPT, K2_ST_CP>;
        auto kern = k_lncc_grad<R, K2_NW, K2_OPT, K2_ST_CP, false, WDJ>;
        static const int occ = prepare(kern, SC::bytes, SC::NT);
        LaunchGeom gg = geometry(occ, K2_NW, SC::TY, R, d, tc.tz);
        le = launch_pdl(kern, gg, SC::bytes, s, mp, If, gJ, J, coef, h, g, d.D, d.H, d.W, d.pitch(), gg.tz,
                        cb, dJout);
    }
    note_launch();
    return le;
}

template <int RG, int NW, class TS>
cudaError_t launch_k3_tma(const Maps &mp, const float *g, TS *m, TS *v, float *dir, WsHeader *h,
                          Dims d, const GaussTaps &t, AdamConsts ac, int parity, int tz,
                          cudaStream_t s) {
    using ST = K3S<RG, NW, K3_OPT, K3_ST_TMA, sizeof(TS) == 4>;
    auto kern = k_smooth_adam<RG, NW, K3_OPT, K3_ST_TMA, true, TS>;
    static const int occ = prepare(kern, ST::bytes, ST::NT);
    LaunchGeom gg = geometry(occ, NW, ST::TY, RG, d, tz);
    return launch_pdl(kern, gg, ST::bytes, s, mp, g, m, v, dir, h, d.D, d.H, d.W, d.pitch(), gg.tz, t, ac,
                      parity);
}

// TS: storage of the moments (float, __nv_bfloat16 or __half); 16-bit moments
// take the 32 x 8 tiles only.
template <int RG, class TS>
cudaError_t launch_k3(const float *g, TS *m, TS *v, float *dir, WsHeader *h, Dims d,
                      const GaussTaps &t, AdamConsts ac, int parity, cudaStream_t s) {
    constexpr bool S32 = sizeof(TS) == 4;
    Maps mp{};
    cudaError_t le;
    const TileChoice tc = tile_choice(2, RG, 0, d);
    const bool wide = S32 && tc.wide;
    const int nw = wide ? 16 : 8;
    const bool tma = tmap(&mp.a, g, 4, d, 3, FX + 2 * halo4(RG), nw + 2 * RG, 3) &&
                     (!S32 || (tmap(&mp.b, m, 4, d, 3, FX, nw, 3) &&
                               tmap(&mp.c, v, 4, d, 3, FX, nw, 3)));
    if (tma) {
        if constexpr (S32)
            le = wide ? launch_k3_tma<RG, 16, TS>(mp, g, m, v, dir, h, d, t, ac, parity, tc.tz, s)
                      : launch_k3_tma<RG, 8, TS>(mp, g, m, v, dir, h, d, t, ac, parity, tc.tz, s);
        else
            le = launch_k3_tma<RG, 8, TS>(mp, g, m, v, dir, h, d, t, ac, parity, tc.tz, s);
    } else {
        using SC = K3S<RG, K3_NW, K3_OPT, K3_ST_CP, false>;  // moments unstaged
        auto kern = k_smooth_adam<RG, K3_NW, K3_OPT, K3_ST_CP, false, TS>;
        static const int occ = prepare(kern, SC::bytes, SC::NT);
        LaunchGeom gg = geometry(occ, K3_NW, SC::TY, RG, d, tc.tz);
        le = launch_pdl(kern, gg, SC::bytes, s, mp, g, m, v, dir, h, d.D, d.H, d.W, d.pitch(), gg.tz, t, ac,
                        parity);
    }
    note_launch();
    return le;
}

template <int RG, bool SU, int NW, class TU>
cudaError_t launch_k4_tma(const Maps &mp, const TU *u, const float *dir, TU *uo,
                          const float *Im, float *J, float *gJ, WsHeader *h, Dims d, const GaussTaps &t,
                          float lr, float c_lp, int parity, int tz, cudaStream_t s) {
    using ST = K4S<RG, NW, K4_OPT, SU, K4_ST_TMA, TU>;
    auto kern = k_compose<RG, NW, K4_OPT, SU, K4_ST_TMA, true, TU>;
    static const int occ = prepare(kern, ST::bytes, ST::NT);
    LaunchGeom gg = geometry(occ, NW, ST::TY, RG, d, tz);
    return launch_pdl(kern, gg, ST::bytes, s, mp, u, dir, uo, Im, J, gJ, h, d.D, d.H, d.W, d.pitch(), gg.tz, t,
                      lr, c_lp, parity);
}

// TU: storage of u (float, or __half: tile copies only; cudaErrorNotSupported
// when a field does not take them).
template <int RG, bool SU, class TU>
cudaError_t launch_k4(const TU *u, const float *dir, TU *uo, const float *Im, float *J,
                      float *gJ, WsHeader *h, Dims d, const GaussTaps &t, float lr, float c_lp, int parity,
                      cudaStream_t s) {
    constexpr int EU = (int)sizeof(TU);
    using S16 = K4S<RG, 16, K4_OPT, SU, K4_ST_TMA, TU>;
    using S8 = K4S<RG, 8, K4_OPT, SU, K4_ST_TMA, TU>;
    Maps mp{};
    cudaError_t le;
    const TileChoice tc = tile_choice(3, RG, SU ? 1 : 0, d);
    const int nw = tc.wide ? 16 : 8;
    const int ubx = tc.wide ? S16::UBXW : S8::UBXW;
    const bool tma = tmap(&mp.a, dir, 4, d, 3, FX + 2 * halo4(RG), nw + 2 * RG, 3) &&
                     (!SU || tmap(&mp.b, u, EU, d, 3, ubx, nw + 2 * RG + 2, 3));
    if (tma) {
        le = tc.wide ? launch_k4_tma<RG, SU, 16>(mp, u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity,
                                                 tc.tz, s)
                     : launch_k4_tma<RG, SU, 8>(mp, u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity,
                                                tc.tz, s);
    } else if constexpr (EU == 4) {
        using SC = K4S<RG, K4_NW, K4_OPT, SU, K4_ST_CP>;
        auto kern = k_compose<RG, K4_NW, K4_OPT, SU, K4_ST_CP, false>;
        static const int occ = prepare(kern, SC::bytes, SC::NT);
        LaunchGeom gg = geometry(occ, K4_NW, SC::TY, RG, d, tc.tz);
        le = launch_pdl(kern, gg, SC::bytes, s, mp, u, dir, uo, Im, J, gJ, h, d.D, d.H, d.W, d.pitch(), gg.tz, t,
                        lr, c_lp, parity);
    } else {
        return cudaErrorNotSupported;
    }
    note_launch();
    return le;
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

cudaError_t dispatch_k2(const float *If, const float *gJ, const float *J, const float *coef,
                        WsHeader *h, float *g, Dims d, int window, cudaStream_t s) {
    switch (window / 2) {
        FA_CASE(0, (launch_k2<RR>(If, gJ, J, coef, h, g, d, window, s)))
        FA_CASE(1, (launch_k2<RR>(If, gJ, J, coef, h, g, d, window, s)))
        FA_CASE(2, (launch_k2<RR>(If, gJ, J, coef, h, g, d, window, s)))
        FA_CASE(3, (launch_k2<RR>(If, gJ, J, coef, h, g, d, window, s)))
        FA_CASE(4, (launch_k2<RR>(If, gJ, J, coef, h, g, d, window, s)))
        FA_CASE(5, (launch_k2<RR>(If, gJ, J, coef, h, g, d, window, s)))
        FA_CASE(6, (launch_k2<RR>(If, gJ, J, coef, h, g, d, window, s)))
        FA_CASE(7, (launch_k2<RR>(If, gJ, J, coef, h, g, d, window, s)))
    }
    return cudaErrorInvalidValue;
}

// The adjoint's K2 (windows 1..15): g and dL/dJ.
cudaError_t dispatch_k2_dj(const float *If, const float *gJ, const float *J, const float *coef,
                           WsHeader *h, float *g, float *dJ, Dims d, int window, cudaStream_t s) {
    switch (window / 2) {
        FA_CASE(0, (launch_k2<RR, true>(If, gJ, J, coef, h, g, d, window, s, dJ)))
        FA_CASE(1, (launch_k2<RR, true>(If, gJ, J, coef, h, g, d, window, s, dJ)))
        FA_CASE(2, (launch_k2<RR, true>(If, gJ, J, coef, h, g, d, window, s, dJ)))
        FA_CASE(3, (launch_k2<RR, true>(If, gJ, J, coef, h, g, d, window, s, dJ)))
        FA_CASE(4, (launch_k2<RR, true>(If, gJ, J, coef, h, g, d, window, s, dJ)))
        FA_CASE(5, (launch_k2<RR, true>(If, gJ, J, coef, h, g, d, window, s, dJ)))
        FA_CASE(6, (launch_k2<RR, true>(If, gJ, J, coef, h, g, d, window, s, dJ)))
        FA_CASE(7, (launch_k2<RR, true>(If, gJ, J, coef, h, g, d, window, s, dJ)))
    }
    return cudaErrorInvalidValue;
}


template <class TS>
cudaError_t dispatch_k3_ts(const float *g, TS *m, TS *v, float *dir, WsHeader *h, Dims d,
                           const GaussTaps &t, AdamConsts ac, int parity, cudaStream_t s) {
    switch (t.R) {
        FA_CASE(0, (launch_k3<RR, TS>(g, m, v, dir, h, d, t, ac, parity, s)))
        FA_CASE(1, (launch_k3<RR, TS>(g, m, v, dir, h, d, t, ac, parity, s)))
        FA_CASE(2, (launch_k3<RR, TS>(g, m, v, dir, h, d, t, ac, parity, s)))
        FA_CASE(3, (launch_k3<RR, TS>(g, m, v, dir, h, d, t, ac, parity, s)))
        FA_CASE(4, (launch_k3<RR, TS>(g, m, v, dir, h, d, t, ac, parity, s)))
        FA_CASE(5, (launch_k3<RR, TS>(g, m, v, dir, h, d, t, ac, parity, s)))
        FA_CASE(6, (launch_k3<RR, TS>(g, m, v, dir, h, d, t, ac, parity, s)))
    }
    return cudaErrorInvalidValue;
}

// m, v stored as `state` (FA_F32 or FA_BF16)
cudaError_t dispatch_k3(const float *g, void *m, void *v, int state, float *dir, WsHeader *h,
                        Dims d, const GaussTaps &t, AdamConsts ac, int parity, cudaStream_t s) {
    if (state == FA_BF16)
        return dispatch_k3_ts(g, (__nv_bfloat16 *)m, (__nv_bfloat16 *)v, dir, h, d, t, ac, parity,
                              s);
    if (state != FA_F32) return cudaErrorInvalidValue;
    return dispatch_k3_ts(g, (float *)m, (float *)v, dir, h, d, t, ac, parity, s);
}

template <class TU>
cudaError_t dispatch_k4_t(const TU *u, const float *dir, TU *uo, const float *Im, float *J,
                          float *gJ, WsHeader *h, Dims d, const GaussTaps &t, float lr,
                          float c_lp, int parity, bool su, cudaStream_t s) {
    if (su) {
        switch (t.R) {
            FA_CASE(0, (launch_k4<RR, true, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(1, (launch_k4<RR, true, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(2, (launch_k4<RR, true, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(3, (launch_k4<RR, true, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(4, (launch_k4<RR, true, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(5, (launch_k4<RR, true, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(6, (launch_k4<RR, true, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
        }
    } else {
        switch (t.R) {
            FA_CASE(0, (launch_k4<RR, false, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(1, (launch_k4<RR, false, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(2, (launch_k4<RR, false, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(3, (launch_k4<RR, false, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(4, (launch_k4<RR, false, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(5, (launch_k4<RR, false, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
            FA_CASE(6, (launch_k4<RR, false, TU>(u, dir, uo, Im, J, gJ, h, d, t, lr, c_lp, parity, s)))
        }
    }
    return cudaErrorInvalidValue;
}
// u, uo: displacements stored as `field` (FA_F32 or FA_F16)
cudaError_t dispatch_k4(const void *u, const float *dir, void *uo, int field, const float *Im,
                        float *J, float *gJ, WsHeader *h, Dims d, const GaussTaps &t, float lr,
                        float c_lp, int parity, bool su, cudaStream_t s) {
    if (field == FA_F16)
        return dispatch_k4_t((const __half *)u, dir, (__half *)uo, Im, J, gJ, h, d, t, lr, c_lp,
                             parity, su, s);
    return dispatch_k4_t((const float *)u, dir, (float *)uo, Im, J, gJ, h, d, t, lr, c_lp, parity,
                         su, s);
}
#undef FA_CASE

struct KTimer {
    fa_kernel_timer *t;
    int level;
    bool on(int id) const {
        return t && (t->kernel_id == id || (t->kernel_id == FA_K_FUSED_ALL && id <= 3)) &&
               (t->level < 0 || t->level == level) && t->count < t->capacity;
    }
};

}  // namespace

void fused_carve(WsCarver &c, long long n, FusedBuffers *fb) {
    fb->coef = c.take<float>(4 * n);  // also the first int64 scratch of the fixed statistics
    fb->g = c.take<float>(4 * n);     // also the second one
    fb->dir = c.take<float>(3 * n);
    fb->J = c.take<float>(n);
    fb->gJ = c.take<float>(3 * n);
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
    return launch_warp_field(Im, u, p->field_storage, fb.J, fb.gJ, d, s);
}

fa_status fused_iteration(FusedBuffers &fb, WsHeader *h, const fa_params *p, Dims d,
                          const FusedIter &it, const GaussTaps &tg, const GaussTaps &tw,
                          fa_kernel_timer *timer, int level, cudaStream_t s) {
    KTimer kt{timer, level};
    auto start = [&](int id) -> cudaError_t {
        return kt.on(id) ? timer_record(timer->start_events[timer->count], s) : cudaSuccess;
    };
    auto stop = [&](int id) -> cudaError_t {
        if (!kt.on(id)) return cudaSuccess;
        cudaError_t e = timer_record(timer->stop_events[timer->count], s);
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
        FA_CUDA_TRY(dispatch_k2(it.If, fb.gJ, fb.J, fb.coef, h, fb.g, d, p->window, s));
        FA_CUDA_TRY(stop(FA_K_FUSED_LNCC_GRAD));
    } else if (p->loss == FA_LOSS_MI) {
        FA_CUDA_TRY(start(FA_K_FUSED_LNCC_GRAD));
        FA_CUDA_TRY(launch_mi(it.If, fb.J, fb.gJ, d, p->mi_bins, h, fb.mi, nullptr, nullptr, fb.g,
                              s));
        FA_CUDA_TRY(stop(FA_K_FUSED_LNCC_GRAD));
    } else {
        VoxGrid gg(d.D, d.H, d.W);
        FA_CUDA_TRY(start(FA_K_FUSED_LNCC_GRAD));
        k_fused_mse_grad<<<gg.grid, gg.block, 0, s>>>(it.If, fb.J, fb.gJ, fb.g, d.D, d.H, d.W);
        note_launch();
        FA_CUDA_TRY(cudaGetLastError());
        FA_CUDA_TRY(stop(FA_K_FUSED_LNCC_GRAD));
    }
    if (p->use_jac) FA_CUDA_TRY(launch_jac_direction(fb.g, it.u, fb.g, d, s));
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
    FA_CUDA_TRY(dispatch_k3(fb.g, it.m, it.v, p->state_storage, fb.dir, h, d, wide_g ? ident : tg,
                            adam_consts(p, it.t), parity, s));
    FA_CUDA_TRY(stop(FA_K_FUSED_SMOOTH_ADAM));
    FA_CUDA_TRY(start(FA_K_FUSED_COMPOSE));
    FA_CUDA_TRY(dispatch_k4(it.u, fb.dir, it.u_alt, p->field_storage, it.Im, fb.J, fb.gJ, h, d,
                            wide_w ? ident : tw, p->lr,
                            p->c_lp, parity, su, s));
    FA_CUDA_TRY(stop(FA_K_FUSED_COMPOSE));
    if (wide_w) {
        FA_CUDA_TRY(launch_gauss3(it.u_alt, it.u_alt, fb.t1, fb.t2, 3, d, tw, s));
        FA_CUDA_TRY(launch_warp(it.Im, it.u_alt, fb.J, fb.gJ, d, s));  // J, grad of the smoothed map
    }
    return FA_OK;
}

fa_status fused_autotune_level(FusedBuffers &fb, WsHeader *h, const fa_params *p, Dims d,
                               const float *If, const float *Im, float *u, float *u_alt, void *m,
                               void *v, const GaussTaps &tg, const GaussTaps &tw,
                               cudaStream_t s) {
    static const GaussTaps ident = [] {
        GaussTaps t;
        make_gauss_taps(0.0f, &t);
        return t;
    }();
    const GaussTaps &g3 = tg.R > kMaxFusedRG ? ident : tg;
    const GaussTaps &g4 = tw.R > kMaxFusedRG ? ident : tw;
    const bool su = (double)p->lr / (double)p->c_lp < 0.999;
    const AdamConsts ac = adam_consts(p, 1);
    auto launch = [&](int kernel) -> cudaError_t {
        switch (kernel) {
            case 0:
                return dispatch_k1(If, fb.J, fb.sI, fb.varI, fb.coef, h, d, p->window, p->cc_eps,
                                   true, s);
            case 1: return dispatch_k2(If, fb.gJ, fb.J, fb.coef, h, fb.g, d, p->window, s);
            case 2: return dispatch_k3(fb.g, m, v, p->state_storage, fb.dir, h, d, g3, ac, 0, s);
            default:
                return dispatch_k4(u, fb.dir, u_alt, p->field_storage, Im, fb.J, fb.gJ, h, d, g4,
                                   p->lr, p->c_lp, 0,
                                   su, s);
        }
    };
    cudaEvent_t e0, e1;
    FA_CUDA_TRY(cudaEventCreate(&e0));
    FA_CUDA_TRY(cudaEventCreate(&e1));
    const int tzs[] = {0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64};
    fa_status result = FA_OK;
    for (int kernel = (p->loss == FA_LOSS_LNCC ? 0 : 2); kernel < 4 && result == FA_OK; ++kernel) {
        const int radius = kernel < 2 ? p->window / 2 : (kernel == 2 ? g3.R : g4.R);
        const int sukey = kernel == 3 && su ? 1 : 0;
        TileChoice best{kDefaultWide[kernel], 0};
        float best_ms = -1.0f;
        for (int wide = 0; wide < (kernel >= 2 ? 2 : 1) && result == FA_OK; ++wide)
            for (int tz : tzs) {
                if (tz > d.D) continue;
                const TileChoice c{wide, tz};
                g_force = &c;
                cudaError_t e = launch(kernel);  // warm
                if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                // 12 launches: the coarse levels' launches take 10-20 us, so
                // fewer would leave the choice to timer noise
                for (int r = 0; r < 12 && e == cudaSuccess; ++r) e = launch(kernel);
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                g_force = nullptr;
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    result = cuda_fail(e, "fa_autotune");
                    break;
                }
                if (best_ms < 0.0f || ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
        if (result == FA_OK) {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tune[TuneKey{kernel, radius, sukey, d.D, d.H, d.W}] = best;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return result;
}

void fused_tile_set(const int32_t *r) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[TuneKey{r[0], r[1], r[2], r[3], r[4], r[5]}] = TileChoice{r[6] ? 1 : 0, r[7]};
}

void fused_autotune_reset() {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
}

int fused_tile_choices(int32_t *out, int capacity) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    int n = 0;
    for (const auto &kv : g_tune) {
        if (n < capacity && out) {
            int32_t *r = out + 8 * n;
            r[0] = kv.first.kernel;
            r[1] = kv.first.radius;
            r[2] = kv.first.su;
            r[3] = kv.first.D;
            r[4] = kv.first.H;
            r[5] = kv.first.W;
            r[6] = kv.second.wide;
            r[7] = kv.second.tz;
        }
        ++n;
    }
    return n;
}

cudaError_t fused_lncc_forward_only(const float *If, const FusedBuffers &fb, Dims d, int window,
                                    float cc_eps, WsHeader *h, cudaStream_t s) {
    return dispatch_k1(If, fb.J, fb.sI, fb.varI, nullptr, h, d, window, cc_eps, false, s);
}

cudaError_t fused_warp_lncc_adjoint(const float *If, const float *Im, const float *u,
                                    const FusedBuffers &fb, Dims d, int window, float cc_eps,
                                    WsHeader *h, float *loss_dev, float *g, float *dJ,
                                    cudaStream_t s) {
    cudaError_t e;
    if ((e = launch_warp(Im, u, fb.J, g ? fb.gJ : nullptr, d, s)) != cudaSuccess) return e;
    if ((e = launch_absmax2(If, fb.J, d.N(), h, s)) != cudaSuccess) return e;
    if ((e = launch_fixed_stats(If, d, window, h, (long long *)fb.coef, (long long *)fb.g, fb.sI,
                                fb.varI, s)) != cudaSuccess)
        return e;
    if ((e = dispatch_k1(If, fb.J, fb.sI, fb.varI, fb.coef, h, d, window, cc_eps, g != nullptr,
                         s)) != cudaSuccess)
        return e;
    if ((e = launch_loss_finalize(h, d.N(), -1.0f, loss_dev, s)) != cudaSuccess) return e;
    if (!g) return cudaSuccess;
    return dJ ? dispatch_k2_dj(If, fb.gJ, fb.J, fb.coef, h, g, dJ, d, window, s)
              : dispatch_k2(If, fb.gJ, fb.J, fb.coef, h, g, d, window, s);
}

// Self-test of the bounded wait: one thread waits on an mbarrier that no
// thread arrives at, gives up after `limit` cycles and records ST_TIMEOUT,
// exactly as a fused kernel does when a tile copy never lands.
__global__ void k_wait_selftest(WsHeader *h, long long limit) {
    __shared__ unsigned long long bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar);
    mbar_init_fence();
    if (!mbar_wait(&bar, 0u, limit)) status_set(&h->status, ST_TIMEOUT);
}

}  // namespace fa

extern "C" fa_status fa_selftest_wait_timeout(void *ws, size_t ws_bytes, int64_t limit_cycles,
                                              void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_ws(ws, ws_bytes, sizeof(WsHeader), "fa_selftest_wait_timeout"));
    if (limit_cycles < 0 || limit_cycles > (1ll << 31)) {
        set_error("fa_selftest_wait_timeout: limit_cycles must be in 0..2^31");
        return FA_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    FA_CUDA_TRY(launch_header_reset((WsHeader *)ws, s));
    k_wait_selftest<<<1, 32, 0, s>>>((WsHeader *)ws, (long long)limit_cycles);
    note_launch();
    FA_CUDA_TRY(cudaGetLastError());
    return FA_OK;
}
