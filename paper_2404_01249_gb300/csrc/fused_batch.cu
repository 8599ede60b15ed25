// Lockstep batches of the fused kernels: many registrations advance together,
// one launch of each fused kernel per iteration over the tiles of every job.
#include "fused_kernels.cuh"

namespace fa {

namespace {

// ------------------------------------------------------------ lockstep batches
// Many registrations advance together: one launch of a fused kernel covers the
// tiles of every job in the launch's table.  CTA b belongs to the job k with
// first[k] <= b < first[k + 1]; its tile inside that job's grid is
// b - first[k] in x-fastest order.  The table travels in the kernel's
// parameter space (read through the constant cache; every thread of a CTA
// reads the same entry), and so do the jobs' tensor maps: a CTA hands the
// TMA unit the address of its job's maps in that space.  A launch takes TMA
// tiles when every job's buffers meet TMA's alignment rules (the row pitch
// of a level's buffers is a multiple of 4 floats whenever the fused kernels
// run it), else the per-thread copy variant (cp.async) for all its jobs.
// The compose kernel of a batch takes 32 x 16 tiles of 16 warps: its u' region
// (the tile plus the sigma_warp halo) is then 1.25 instead of 1.5 times the
// tile, the choice the single-job launches make by default.
constexpr int K4B_NW = 16;

struct BGeom {
    int D, H, W, P, TZ, gx, gy;  // P: row pitch of the job's buffers
};
struct BTaps {
    float w[2 * kMaxFusedRG + 1];
};
struct K1Job {
    const float *If, *J;
    const long long *SI;
    const float *varI;
    float *coef;
    WsHeader *h;
    BGeom g;
    float cc_eps;
};
struct K1Batch {
    CUtensorMap tm[2 * kMaxLockstepJobs];  // job k: I_f at 2k, J at 2k + 1
    int n, bits, window, write_coef;
    int first[kMaxLockstepJobs + 1];
    K1Job j[kMaxLockstepJobs];
};
struct K2Job {
    const float *If, *gJ, *J, *coef;
    float *g;
    WsHeader *h;
    BGeom geo;
};
struct K2Batch {
    CUtensorMap tm[kMaxLockstepJobs];  // job k: the A, B, C coefficients
    int n, cbits;
    int first[kMaxLockstepJobs + 1];
    K2Job j[kMaxLockstepJobs];
};
struct K3Job {
    const float *g;
    void *m, *v;  // stored as the launch's moment type
    float *dir;
    WsHeader *h;
    BGeom geo;
    BTaps t;
};
// NM maps per job: the gradient, then (FP32 moments) m and nu.
template <int NM>
struct K3Batch {
    CUtensorMap tm[NM * kMaxLockstepJobs];
    int n, parity;
    AdamConsts ac;
    int first[kMaxLockstepJobs + 1];
    K3Job j[kMaxLockstepJobs];
};
struct K4Job {
    const void *u;  // stored as the launch's u type
    const float *dir;
    void *uo;
    const float *Im;
    float *J, *gJ;
    WsHeader *h;
    BGeom geo;
    BTaps t;
    float lr, c_lp;
};
// NM maps per job: the direction, then (u read from shared memory) u.
template <int NM>
struct K4Batch {
    CUtensorMap tm[NM * kMaxLockstepJobs];
    int n, parity;
    int first[kMaxLockstepJobs + 1];
    K4Job j[kMaxLockstepJobs];
};
// CUDA's limit on a launch's parameters
constexpr size_t kMaxParamBytes = 32764;
static_assert(sizeof(K1Batch) <= kMaxParamBytes && sizeof(K2Batch) <= kMaxParamBytes &&
                  sizeof(K3Batch<3>) <= kMaxParamBytes && sizeof(K4Batch<2>) <= kMaxParamBytes,
              "a lockstep table must fit the kernel parameter space");

// The job of CTA b: the largest k with first[k] <= b (first[0] = 0).
__device__ __forceinline__ int batch_job(const int *first, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void batch_tile(const BGeom &g, int t, int &bx, int &by, int &bz) {
    bx = t % g.gx;
    const int r = t / g.gx;
    by = r % g.gy;
    bz = r / g.gy;
}

// Job k's maps tm[NM k ...] of a table (TMA launches), else none.
template <int NM, bool TMA>
__device__ __forceinline__ MapRef job_maps(const CUtensorMap *tm, int k) {
    MapRef r{nullptr, nullptr, nullptr};
    if (TMA) {
        r.a = tm + NM * k;
        if (NM > 1) r.b = tm + NM * k + 1;
        if (NM > 2) r.c = tm + NM * k + 2;
    }
    return r;
}

template <int R, bool TMA>
__global__ void __launch_bounds__(FX *K1_NW) k_lncc_fwd_batch(const __grid_constant__ K1Batch b) {
    const int k = batch_job(b.first, b.n, (int)blockIdx.x);
    const K1Job &j = b.j[k];
    int bx, by, bz;
    batch_tile(j.g, (int)blockIdx.x - b.first[k], bx, by, bz);
    lncc_fwd_body<R, K1_NW, K1_OPT, TMA ? K1_ST_TMA : K1_ST_CP, TMA>(
        job_maps<2, TMA>(b.tm, k), j.If, j.J, j.SI, j.varI, j.coef, j.h, j.g.D, j.g.H, j.g.W,
        j.g.P, j.g.TZ, b.bits, j.cc_eps, b.window, b.write_coef, bx, by, bz);
}

template <int R, bool TMA>
__global__ void __launch_bounds__(FX *K2_NW) k_lncc_grad_batch(const __grid_constant__ K2Batch b) {
    const int k = batch_job(b.first, b.n, (int)blockIdx.x);
    const K2Job &j = b.j[k];
    int bx, by, bz;
    batch_tile(j.geo, (int)blockIdx.x - b.first[k], bx, by, bz);
    lncc_grad_body<R, K2_NW, K2_OPT, TMA ? K2_ST_TMA : K2_ST_CP, TMA>(
        job_maps<1, TMA>(b.tm, k), j.If, j.gJ, j.J, j.coef, j.h, j.g, j.geo.D, j.geo.H, j.geo.W,
        j.geo.P, j.geo.TZ, b.cbits, bx, by, bz);
}

template <class TS>
constexpr int k3_maps() {
    return sizeof(TS) == 4 ? 3 : 1;
}

template <int RG, class TS, bool TMA>
__global__ void __launch_bounds__(FX *K3_NW) k_smooth_adam_batch(
    const __grid_constant__ K3Batch<k3_maps<TS>()> b) {
    const int k = batch_job(b.first, b.n, (int)blockIdx.x);
    const K3Job &j = b.j[k];
    int bx, by, bz;
    batch_tile(j.geo, (int)blockIdx.x - b.first[k], bx, by, bz);
    smooth_adam_body<RG, K3_NW, K3_OPT, TMA ? K3_ST_TMA : K3_ST_CP, TMA>(
        job_maps<k3_maps<TS>(), TMA>(b.tm, k), j.g, (TS *)j.m, (TS *)j.v, j.dir, j.h, j.geo.D,
        j.geo.H, j.geo.W, j.geo.P, j.geo.TZ, j.t, b.ac, b.parity, bx, by, bz);
}

// TU: storage of u (float, or __half: tile copies only).
template <int RG, bool SU, bool TMA, class TU>
__global__ void __launch_bounds__(FX *K4B_NW, 2) k_compose_batch(
    const __grid_constant__ K4Batch<SU ? 2 : 1> b) {
    const int k = batch_job(b.first, b.n, (int)blockIdx.x);
    const K4Job &j = b.j[k];
    int bx, by, bz;
    batch_tile(j.geo, (int)blockIdx.x - b.first[k], bx, by, bz);
    compose_body<RG, K4B_NW, K4_OPT, SU, TMA ? K4_ST_TMA : K4_ST_CP, TMA>(
        job_maps<SU ? 2 : 1, TMA>(b.tm, k), (const TU *)j.u, j.dir, (TU *)j.uo, j.Im, j.J, j.gJ,
        j.h, j.geo.D, j.geo.H, j.geo.W, j.geo.P, j.geo.TZ, j.t, j.lr, j.c_lp, b.parity, bx, by,
        bz);
}

// Slab depth of a lockstep launch: one TZ for all its jobs (each capped at its
// own depth), minimising (waves x planes per CTA) over the whole launch, whose
// CTAs fill the GPU's resident slots together.  A coarse level of many jobs
// then takes short slabs (more CTAs), a fine level long ones (less halo).
int launch_tz(const Dims *d, int n, int ty, int halo, int occ) {
    const long long slots = (long long)num_sms() * (occ > 0 ? occ : 1);
    int best = 64;
    long long bestcost = -1;
    for (int tz = 1; tz <= 64; ++tz) {
        long long ctas = 0;
        for (int k = 0; k < n; ++k) {
            const long long txy = (long long)((d[k].W + FX - 1) / FX) * ((d[k].H + ty - 1) / ty);
            const int t = tz < d[k].D ? tz : d[k].D;
            ctas += txy * ((d[k].D + t - 1) / t);
        }
        const long long cost = (ctas + slots - 1) / slots * (tz + 2 * halo);
        if (bestcost < 0 || cost < bestcost) {
            bestcost = cost;
            best = tz;
        }
    }
    return best;
}

// Fills a job's tile geometry for a kernel with `ty` rows per CTA and slab
// depth tz (capped at the job's depth) and returns its CTA count.
int batch_geom(BGeom &g, Dims d, int ty, int tz) {
    g.D = d.D;
    g.H = d.H;
    g.W = d.W;
    g.P = d.pitch();
    g.gx = (d.W + FX - 1) / FX;
    g.gy = (d.H + ty - 1) / ty;
    g.TZ = tz < d.D ? tz : d.D;
    return g.gx * g.gy * ((d.D + g.TZ - 1) / g.TZ);
}

BGeom *geom_of(K1Job &j) { return &j.g; }
BGeom *geom_of(K2Job &j) { return &j.geo; }
BGeom *geom_of(K3Job &j) { return &j.geo; }
BGeom *geom_of(K4Job &j) { return &j.geo; }

void batch_taps(BTaps &b, const GaussTaps &t) {
    for (int k = 0; k < 2 * kMaxFusedRG + 1; ++k) b.w[k] = k <= 2 * t.R ? t.w[k] : 0.0f;
}

template <class K, class B>
cudaError_t launch_batch(K kern, const B &b, int nw, size_t smem, cudaStream_t s) {
    LaunchGeom g;
    g.grid = dim3((unsigned)b.first[b.n]);
    g.block = dim3(FX, nw);
    g.tz = 0;
    return launch_pdl(kern, g, smem, s, b);
}

// Tile geometry of every job of a launch (jobs[idx[k]], k < b.n) for a kernel
// of `ty` rows per CTA, halo `halo` and `occ` resident CTAs per SM.
template <class B>
void batch_layout(B &b, const LockstepJob *jobs, const int *idx, int ty, int halo, int occ) {
    Dims dd[kMaxLockstepJobs];
    for (int k = 0; k < b.n; ++k) dd[k] = jobs[idx[k]].d;
    const int tz = launch_tz(dd, b.n, ty, halo, occ);
    b.first[0] = 0;
    for (int k = 0; k < b.n; ++k) {
        BGeom &g = *geom_of(b.j[k]);
        b.first[k + 1] = b.first[k] + batch_geom(g, dd[k], ty, tz);
    }
}

template <int R>
cudaError_t launch_k1_batch(K1Batch &b, const LockstepJob *jobs, const int *idx, cudaStream_t s) {
    using ST = K1S<R, K1_NW, K1_OPT, K1_ST_TMA>;
    bool tma = true;
    for (int k = 0; k < b.n && tma; ++k) {
        const LockstepJob &q = jobs[idx[k]];
        tma = tmap(&b.tm[2 * k], q.If, 4, q.d, 1, ST::BXW, ST::RY, 1) &&
              tmap(&b.tm[2 * k + 1], q.fb->J, 4, q.d, 1, ST::BXW, ST::RY, 1);
    }
    if (tma) {
        auto kern = k_lncc_fwd_batch<R, true>;
        static const int occ = prepare(kern, ST::bytes, ST::NT);
        batch_layout(b, jobs, idx, ST::TY, R, occ);
        return launch_batch(kern, b, ST::NT / FX, ST::bytes, s);
    }
    using SC = K1S<R, K1_NW, K1_OPT, K1_ST_CP>;
    auto kern = k_lncc_fwd_batch<R, false>;
    static const int occ = prepare(kern, SC::bytes, SC::NT);
    batch_layout(b, jobs, idx, SC::TY, R, occ);
    return launch_batch(kern, b, SC::NT / FX, SC::bytes, s);
}

template <int R>
cudaError_t launch_k2_batch(K2Batch &b, const LockstepJob *jobs, const int *idx, cudaStream_t s) {
    using ST = K2S<R, K2_NW, K2_OPT, K2_ST_TMA>;
    bool tma = true;
    for (int k = 0; k < b.n && tma; ++k) {
        const LockstepJob &q = jobs[idx[k]];
        tma = tmap(&b.tm[k], q.fb->coef, 4, q.d, 4, ST::BXW, ST::RY, 4);
    }
    if (tma) {
        auto kern = k_lncc_grad_batch<R, true>;
        static const int occ = prepare(kern, ST::bytes, ST::NT);
        batch_layout(b, jobs, idx, ST::TY, R, occ);
        return launch_batch(kern, b, ST::NT / FX, ST::bytes, s);
    }
    using SC = K2S<R, K2_NW, K2_OPT, K2_ST_CP>;
    auto kern = k_lncc_grad_batch<R, false>;
    static const int occ = prepare(kern, SC::bytes, SC::NT);
    batch_layout(b, jobs, idx, SC::TY, R, occ);
    return launch_batch(kern, b, SC::NT / FX, SC::bytes, s);
}

template <int RG, class TS>
cudaError_t launch_k3_batch(K3Batch<k3_maps<TS>()> &b, const LockstepJob *jobs, const int *idx,
                            cudaStream_t s) {
    constexpr bool S32 = sizeof(TS) == 4;
    constexpr int NM = k3_maps<TS>();
    using ST = K3S<RG, K3_NW, K3_OPT, K3_ST_TMA, S32>;  // FP32 moments staged
    bool tma = true;
    for (int k = 0; k < b.n && tma; ++k) {
        const LockstepJob &q = jobs[idx[k]];
        tma = tmap(&b.tm[NM * k], q.fb->g, 4, q.d, 3, ST::BXW, ST::RY, 3);
        if constexpr (S32)
            tma = tma && tmap(&b.tm[NM * k + 1], q.m, 4, q.d, 3, FX, ST::TY, 3) &&
                  tmap(&b.tm[NM * k + 2], q.v, 4, q.d, 3, FX, ST::TY, 3);
    }
    if (tma) {
        auto kern = k_smooth_adam_batch<RG, TS, true>;
        static const int occ = prepare(kern, ST::bytes, ST::NT);
        batch_layout(b, jobs, idx, ST::TY, RG, occ);
        return launch_batch(kern, b, ST::NT / FX, ST::bytes, s);
    }
    using SC = K3S<RG, K3_NW, K3_OPT, K3_ST_CP, false>;  // moments unstaged
    auto kern = k_smooth_adam_batch<RG, TS, false>;
    static const int occ = prepare(kern, SC::bytes, SC::NT);
    batch_layout(b, jobs, idx, SC::TY, RG, occ);
    return launch_batch(kern, b, SC::NT / FX, SC::bytes, s);
}

// TU: storage of u of every job of the launch (an FP16 u takes tile copies
// only: cudaErrorNotSupported when a job's buffers do not meet their rules).
template <int RG, bool SU, class TU>
cudaError_t launch_k4_batch(K4Batch<SU ? 2 : 1> &b, const LockstepJob *jobs, const int *idx,
                            cudaStream_t s) {
    constexpr int NM = SU ? 2 : 1, EU = (int)sizeof(TU);
    using ST = K4S<RG, K4B_NW, K4_OPT, SU, K4_ST_TMA, TU>;
    bool tma = true;
    for (int k = 0; k < b.n && tma; ++k) {
        const LockstepJob &q = jobs[idx[k]];
        tma = tmap(&b.tm[NM * k], q.fb->dir, 4, q.d, 3, ST::BXW, ST::RY, 3);
        if constexpr (SU)
            tma = tma && tmap(&b.tm[NM * k + 1], q.u, EU, q.d, 3, ST::UBXW, ST::URY, 3);
    }
    if (tma) {
        auto kern = k_compose_batch<RG, SU, true, TU>;
        static const int occ = prepare(kern, ST::bytes, ST::NT);
        batch_layout(b, jobs, idx, ST::TY, RG, occ);
        return launch_batch(kern, b, ST::NT / FX, ST::bytes, s);
    }
    if constexpr (EU == 4) {
        using SC = K4S<RG, K4B_NW, K4_OPT, SU, K4_ST_CP>;
        auto kern = k_compose_batch<RG, SU, false, float>;
        static const int occ = prepare(kern, SC::bytes, SC::NT);
        batch_layout(b, jobs, idx, SC::TY, RG, occ);
        return launch_batch(kern, b, SC::NT / FX, SC::bytes, s);
    } else {
        return cudaErrorNotSupported;
    }
}

#define FA_CASE(n, call)      \
    case n: {                 \
        constexpr int RR = n; \
        return call;          \
    }

cudaError_t dispatch_k1_batch(int R, K1Batch &b, const LockstepJob *jobs, const int *idx,
                              cudaStream_t s) {
    switch (R) {
        FA_CASE(0, launch_k1_batch<RR>(b, jobs, idx, s))
        FA_CASE(1, launch_k1_batch<RR>(b, jobs, idx, s))
        FA_CASE(2, launch_k1_batch<RR>(b, jobs, idx, s))
        FA_CASE(3, launch_k1_batch<RR>(b, jobs, idx, s))
        FA_CASE(4, launch_k1_batch<RR>(b, jobs, idx, s))
        FA_CASE(5, launch_k1_batch<RR>(b, jobs, idx, s))
        FA_CASE(6, launch_k1_batch<RR>(b, jobs, idx, s))
        FA_CASE(7, launch_k1_batch<RR>(b, jobs, idx, s))
    }
    return cudaErrorInvalidValue;
}

cudaError_t dispatch_k2_batch(int R, K2Batch &b, const LockstepJob *jobs, const int *idx,
                              cudaStream_t s) {
    switch (R) {
        FA_CASE(0, launch_k2_batch<RR>(b, jobs, idx, s))
        FA_CASE(1, launch_k2_batch<RR>(b, jobs, idx, s))
        FA_CASE(2, launch_k2_batch<RR>(b, jobs, idx, s))
        FA_CASE(3, launch_k2_batch<RR>(b, jobs, idx, s))
        FA_CASE(4, launch_k2_batch<RR>(b, jobs, idx, s))
        FA_CASE(5, launch_k2_batch<RR>(b, jobs, idx, s))
        FA_CASE(6, launch_k2_batch<RR>(b, jobs, idx, s))
        FA_CASE(7, launch_k2_batch<RR>(b, jobs, idx, s))
    }
    return cudaErrorInvalidValue;
}

template <class TS>
cudaError_t dispatch_k3_batch_ts(int RG, K3Batch<k3_maps<TS>()> &b, const LockstepJob *jobs,
                                 const int *idx, cudaStream_t s) {
    switch (RG) {
        FA_CASE(0, (launch_k3_batch<RR, TS>(b, jobs, idx, s)))
        FA_CASE(1, (launch_k3_batch<RR, TS>(b, jobs, idx, s)))
        FA_CASE(2, (launch_k3_batch<RR, TS>(b, jobs, idx, s)))
        FA_CASE(3, (launch_k3_batch<RR, TS>(b, jobs, idx, s)))
        FA_CASE(4, (launch_k3_batch<RR, TS>(b, jobs, idx, s)))
        FA_CASE(5, (launch_k3_batch<RR, TS>(b, jobs, idx, s)))
        FA_CASE(6, (launch_k3_batch<RR, TS>(b, jobs, idx, s)))
    }
    return cudaErrorInvalidValue;
}

// One K3 launch over jobs[idx[0..m)], whose moments are stored as TS.
template <class TS>
cudaError_t k3_batch(int RG, int m, const LockstepJob *jobs, const int *idx, AdamConsts ac,
                     int parity, cudaStream_t s) {
    K3Batch<k3_maps<TS>()> b;
    b.n = m;
    b.parity = parity;
    b.ac = ac;
    for (int i = 0; i < m; ++i) {
        const LockstepJob &q = jobs[idx[i]];
        K3Job &j = b.j[i];
        j.g = q.fb->g;
        j.m = q.m;
        j.v = q.v;
        j.dir = q.fb->dir;
        j.h = q.h;
        batch_taps(j.t, *q.tg);
    }
    return dispatch_k3_batch_ts<TS>(RG, b, jobs, idx, s);
}

template <bool SU, class TU>
cudaError_t dispatch_k4_batch(int RG, K4Batch<SU ? 2 : 1> &b, const LockstepJob *jobs,
                              const int *idx, cudaStream_t s) {
    switch (RG) {
        FA_CASE(0, (launch_k4_batch<RR, SU, TU>(b, jobs, idx, s)))
        FA_CASE(1, (launch_k4_batch<RR, SU, TU>(b, jobs, idx, s)))
        FA_CASE(2, (launch_k4_batch<RR, SU, TU>(b, jobs, idx, s)))
        FA_CASE(3, (launch_k4_batch<RR, SU, TU>(b, jobs, idx, s)))
        FA_CASE(4, (launch_k4_batch<RR, SU, TU>(b, jobs, idx, s)))
        FA_CASE(5, (launch_k4_batch<RR, SU, TU>(b, jobs, idx, s)))
        FA_CASE(6, (launch_k4_batch<RR, SU, TU>(b, jobs, idx, s)))
    }
    return cudaErrorInvalidValue;
}

// One K4 launch over jobs[idx[0..m)], whose u is stored as TU.
template <bool SU, class TU>
cudaError_t k4_batch(int RG, int m, const LockstepJob *jobs, const int *idx, int parity,
                     cudaStream_t s) {
    K4Batch<SU ? 2 : 1> b;
    b.n = m;
    b.parity = parity;
    for (int i = 0; i < m; ++i) {
        const LockstepJob &q = jobs[idx[i]];
        K4Job &j = b.j[i];
        j.u = q.u;
        j.dir = q.fb->dir;
        j.uo = q.u_alt;
        j.Im = q.Im;
        j.J = q.fb->J;
        j.gJ = q.fb->gJ;
        j.h = q.h;
        batch_taps(j.t, *q.tw);
        j.lr = q.p->lr;
        j.c_lp = q.p->c_lp;
    }
    return dispatch_k4_batch<SU, TU>(RG, b, jobs, idx, s);
}
#undef FA_CASE

}  // namespace

fa_status fused_iteration_lockstep(int n, const LockstepJob *jobs, int t, cudaStream_t s) {
    if (n < 1 || n > kMaxLockstepJobs) {
        set_error("lockstep iteration: 1..%d jobs per launch (got %d)", kMaxLockstepJobs, n);
        return FA_ERR_INVALID;
    }
    const fa_params *p0 = jobs[0].p;
    const int parity = t & 1, R = p0->window / 2;
    int idx[kMaxLockstepJobs];
    for (int k = 0; k < n; ++k) idx[k] = k;
    {
        K1Batch b;
        b.n = n;
        b.bits = lncc_image_bits(p0->window);
        b.window = p0->window;
        b.write_coef = 1;
        for (int k = 0; k < n; ++k) {
            const LockstepJob &q = jobs[k];
            K1Job &j = b.j[k];
            j.If = q.If;
            j.J = q.fb->J;
            j.SI = q.fb->sI;
            j.varI = q.fb->varI;
            j.coef = q.fb->coef;
            j.h = q.h;
            j.cc_eps = q.p->cc_eps;
        }
        FA_CUDA_TRY(dispatch_k1_batch(R, b, jobs, idx, s));
        note_launch();
    }
    {
        K2Batch b;
        b.n = n;
        b.cbits = lncc_coef_bits(p0->window);
        for (int k = 0; k < n; ++k) {
            const LockstepJob &q = jobs[k];
            K2Job &j = b.j[k];
            j.If = q.If;
            j.gJ = q.fb->gJ;
            j.J = q.fb->J;
            j.coef = q.fb->coef;
            j.g = q.fb->g;
            j.h = q.h;
        }
        FA_CUDA_TRY(dispatch_k2_batch(R, b, jobs, idx, s));
        note_launch();
    }
    const AdamConsts ac = adam_consts(p0, t);
    const int states[2] = {FA_F32, FA_BF16};
    for (int st : states) {
        for (int rg = 0; rg <= kMaxFusedRG; ++rg) {
            int m = 0;
            for (int k = 0; k < n; ++k)
                if (jobs[k].tg->R == rg && jobs[k].p->state_storage == st) idx[m++] = k;
            if (m == 0) continue;
            FA_CUDA_TRY(st == FA_F32 ? k3_batch<float>(rg, m, jobs, idx, ac, parity, s)
                                     : k3_batch<__nv_bfloat16>(rg, m, jobs, idx, ac, parity, s));
            note_launch();
        }
    }
    const int fields[2] = {FA_F32, FA_F16};
    for (int fs : fields)
        for (int su = 0; su < 2; ++su)
            for (int rg = 0; rg <= kMaxFusedRG; ++rg) {
                int m = 0;
                for (int k = 0; k < n; ++k) {
                    const fa_params *p = jobs[k].p;
                    const int ksu = (double)p->lr / (double)p->c_lp < 0.999 ? 1 : 0;
                    if (jobs[k].tw->R == rg && ksu == su && p->field_storage == fs) idx[m++] = k;
                }
                if (m == 0) continue;
                cudaError_t e;
                if (fs == FA_F16)
                    e = su ? k4_batch<true, __half>(rg, m, jobs, idx, parity, s)
                           : k4_batch<false, __half>(rg, m, jobs, idx, parity, s);
                else
                    e = su ? k4_batch<true, float>(rg, m, jobs, idx, parity, s)
                           : k4_batch<false, float>(rg, m, jobs, idx, parity, s);
                if (e == cudaErrorNotSupported) {
                    set_error("lockstep: an FP16 u needs tile copies (rows of 8 elements)");
                    return FA_ERR_UNSUPPORTED;
                }
                FA_CUDA_TRY(e);
                note_launch();
            }
    return FA_OK;
}

}  // namespace fa
