// Fused-path interface used by the registration driver (register.cu).
#pragma once
#include "ops.h"

namespace fa {

// Scratch of the fused iteration (carved from the registration workspace).
struct FusedBuffers {
    float *coef;   // [4][N]: A, B, C hi, C lo of the LNCC adjoint
    float *g;      // [3][N]: dL/dphi before smoothing
    float *dir;    // [3][N]: Adam direction d
    float *J;      // [N]    : warped image I_m o phi of the current map
    float *gJ;     // [3][N]: grad I_m at phi (the interpolant's derivative)
    float *t1, *t2;  // [3][N]: separable passes when a Gaussian is wider than the fused kernels take
    long long *sI; // [N]    : exact window sum of the level's fixed image
    float *varI;   // [N]    : its window variance
    MiBuffers mi;  // histogram scratch of the MI loss (set by the driver)
};
void fused_carve(WsCarver &c, long long n, FusedBuffers *fb);

struct FusedIter {
    const float *If, *Im;
    float *u, *u_alt;  // u_alt receives the updated displacement
    void *m, *v;       // Adam moments, stored as fa_params.state_storage
    int t;
};

fa_status fused_iteration(FusedBuffers &fb, WsHeader *h, const fa_params *p, Dims d,
                          const FusedIter &it, const GaussTaps &tg, const GaussTaps &tw,
                          fa_kernel_timer *timer, int level, cudaStream_t s);
// Per-level set-up of the fused path: the fixed image's window statistics
// (LNCC) and J = I_m o (id + u) with its gradient for the first iteration
// (later iterations get both from the compose kernel).  Needs the level's image maxima in h.
cudaError_t fused_level_start(const float *If, const float *Im, const float *u, Dims d,
                              const fa_params *p, const WsHeader *h, FusedBuffers &fb,
                              cudaStream_t s);
// Measures candidate tile choices of the fused kernels on grid d (any
// buffer contents) and records the fastest for later launches.
fa_status fused_autotune_level(FusedBuffers &fb, WsHeader *h, const fa_params *p, Dims d,
                               const float *If, const float *Im, float *u, float *u_alt, void *m,
                               void *v, const GaussTaps &tg, const GaussTaps &tw, cudaStream_t s);
void fused_autotune_reset();
void fused_tile_set(const int32_t *row);  // one row as fused_tile_choices writes it
// Recorded choices as rows of 8 int32 (kernel, radius, compose variant, D, H,
// W, 16-warp tiles, TZ); returns the number of rows.
int fused_tile_choices(int32_t *out, int capacity);
// The warp + LNCC adjoint on the fused kernels: J and grad I_m at x + u
// (fb.J, fb.gJ), the fixed image's window statistics, K1 (coefficients and
// loss, finalised into loss_dev and h->loss), and when g is not NULL K2: g =
// dL/du and, when dJ is not NULL, dL/dJ.  h must be reset by the caller.
cudaError_t fused_warp_lncc_adjoint(const float *If, const float *Im, const float *u,
                                    const FusedBuffers &fb, Dims d, int window, float cc_eps,
                                    WsHeader *h, float *loss_dev, float *g, float *dJ,
                                    cudaStream_t s);
// LNCC loss accumulator only (no coefficients) for the warped image fb.J.
cudaError_t fused_lncc_forward_only(const float *If, const FusedBuffers &fb, Dims d, int window,
                                    float cc_eps, WsHeader *h, cudaStream_t s);

// One iteration of many registrations that advance together (lockstep): each
// fused kernel runs as one launch over the tiles of every job (K3 and K4 one
// launch per Gaussian radius and compose variant).  The jobs share the loss
// (LNCC), the window, the Adam constants and the step counter t; each Gaussian
// is at most kMaxFusedRadius wide.  K3 runs one launch per Gaussian radius and
// moment storage type.
constexpr int kMaxLockstepJobs = 64;
constexpr int kMaxFusedRadius = 6;
struct LockstepJob {
    Dims d;
    const float *If, *Im;
    float *u, *u_alt;  // u_alt receives the updated displacement
    void *m, *v;       // Adam moments, stored as p->state_storage
    FusedBuffers *fb;
    WsHeader *h;
    const fa_params *p;
    const GaussTaps *tg, *tw;
};
fa_status fused_iteration_lockstep(int n, const LockstepJob *jobs, int t, cudaStream_t s);

// One job of a lockstep call (arguments of fa_register plus a status word).
struct LockstepArgs {
    const fa_vol *fixed, *moving;
    const fa_params *p;
    fa_vol *u_out;
    float *final_loss_dev;  // may be NULL
    uint32_t *status_dev;   // may be NULL
};
// FA_OK when the jobs (each already checked with register_check) can advance
// together, else FA_ERR_UNSUPPORTED with the reason in fa_last_error.
fa_status lockstep_check(int n, const LockstepArgs *a);
// Enqueues n <= kMaxLockstepJobs checked jobs; job k works in ws + k * slot.
// Records the call as a CUDA graph and replays it when every job asks for it.
fa_status register_lockstep(int n, const LockstepArgs *a, void *ws, size_t slot, cudaStream_t s);

// Persistent form of a coarse level (persistent.cu): one cooperative launch
// runs every iteration of the level with grid barriers between its phases,
// computing the bits of fused_iteration.  Eligible: FA_MODE_PERSISTENT, LNCC
// with window 3..7, no use_jac, Gaussian radii <= 6, width <= 128 and at
// most kPersistMaxVoxels voxels.  xy: persistent_xy_bytes(N) of scratch.  The
// displacement after T iterations is in u0 if T is even, else in u1.
constexpr long long kPersistMaxVoxels = 2ll << 20;
bool persistent_eligible(const fa_params *p, Dims d);
size_t persistent_xy_bytes(long long n);
fa_status persistent_level(const FusedBuffers &fb, long long *xy, WsHeader *h, const fa_params *p,
                           Dims d, const float *If, const float *Im, float *u0, float *u1, void *m,
                           void *v, int t0, int T, const GaussTaps &tg, const GaussTaps &tw,
                           cudaStream_t s);

// Argument checks of fa_register (no launch).
fa_status register_check(const fa_vol *fixed, const fa_vol *moving, const fa_params *p,
                         const fa_vol *u_out);
size_t register_ws_bytes(int D, int H, int W, const fa_params *p);

fa_status register_impl(const fa_vol *fixed, const fa_vol *moving, const fa_params *p,
                        const fa_vol *u_init, fa_vol *u_out, float *final_loss_dev, float *final_loss_host, void *ws,
                        size_t ws_bytes, cudaStream_t s, fa_kernel_timer *timer);

}  // namespace fa
