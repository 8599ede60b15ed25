/*
 * libfa -- GB300 (sm_103a) inner loop of FireANTs' multi-scale Riemannian
 * Adam diffeomorphic registration (arXiv 2404.01249).
 *
 * C ABI.  Every pointer to voxel data is a DEVICE pointer owned by the
 * caller; every other pointer (descriptors, parameters, host results) is a
 * HOST pointer.  Streams are passed as `void *` holding a cudaStream_t
 * (NULL = the legacy default stream).  Calls are asynchronous on that stream
 * unless stated otherwise.  Argument, shape and dtype errors are returned
 * before anything is launched; libfa never allocates device memory: scratch
 * space is a caller-provided workspace whose size the *_workspace_size
 * queries return.  No exceptions cross the ABI; fa_last_error() gives a
 * thread-local message for the last failing call.
 *
 * Layout.  A volume is [D][H][W], W fastest.  A 3-channel field is
 * [3][D][H][W] (structure of arrays); channel 0 is the z (D-axis)
 * component, 1 the y (H-axis), 2 the x (W-axis) component, in voxels of the
 * grid it lives on.  The map is phi(x) = x + u(x).  Samples outside the grid
 * read as zero (u is extended by zero outside the domain, section
 * "Preliminaries" of the paper).
 *
 * Arithmetic is FP32 on the GPU, and no kernel holds an FP64 instruction.
 * LNCC window sums are accumulated exactly in 64-bit fixed point, so the
 * E[I^2] - E[I]^2 cancellation does not lose precision.
 */
#ifndef FA_H
#define FA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FA_OK = 0,
    FA_ERR_INVALID = 1,     /* null pointer, bad parameter value            */
    FA_ERR_SHAPE = 2,       /* inconsistent or unsupported shapes           */
    FA_ERR_DTYPE = 3,       /* unsupported element type                     */
    FA_ERR_CUDA = 4,        /* a CUDA runtime call failed                   */
    FA_ERR_NONFINITE = 5,   /* device status word: NaN/Inf in a loss or step */
    FA_ERR_TIMEOUT = 6,     /* device status word: a bounded wait gave up   */
    FA_ERR_UNSUPPORTED = 7, /* valid request this build does not implement  */
    FA_ERR_WORKSPACE = 8    /* workspace missing, too small or misaligned   */
} fa_status;

typedef enum { FA_F32 = 0, FA_BF16 = 1, FA_F16 = 2 } fa_dtype;

typedef enum { FA_LOSS_LNCC = 0, FA_LOSS_MSE = 1, FA_LOSS_MI = 2 } fa_loss;

/* Kernel schedule used by fa_register:
 *  FA_MODE_FUSED (default): four fused kernels per iteration;
 *  FA_MODE_PLAIN: one kernel per operation, intermediates in HBM (the
 *    baseline the fused form is measured against);
 *  FA_MODE_PERSISTENT: as FA_MODE_FUSED, except that a level of at most
 *    2^21 voxels (LNCC with window 3..7, no use_jac, Gaussian radii <= 6,
 *    width <= 128) runs as ONE persistent cooperative launch for all its
 *    iterations, with grid barriers between the phases of an iteration and
 *    the bits of FA_MODE_FUSED.  On GB300 it is slower than FA_MODE_FUSED
 *    (its per-voxel z gathers re-read every plane from L2 in each phase); it
 *    is kept as an alternative schedule.  Its CTAs must be resident
 *    together: fa_register_batched (concurrent streams) runs such jobs as
 *    FA_MODE_FUSED.
 * All compute the same arithmetic. */
typedef enum { FA_MODE_FUSED = 0, FA_MODE_PLAIN = 1, FA_MODE_PERSISTENT = 2 } fa_mode;

/* Descriptor of a caller-owned device buffer holding C channels of a
 * D x H x W grid, contiguous [C][D][H][W]. */
typedef struct {
    void *data;
    int32_t dtype; /* fa_dtype */
    int32_t C, D, H, W;
} fa_vol;

/* Hyper-parameters of Algorithm 1 ("FireANTs"): scales s_l and iterations
 * T_l per level (coarsest first), learning rate eta, the Gaussian widths
 * sigma_grad / sigma_warp of the hyper-parameter study, the LNCC window, the
 * loss, Adam constants (Kingma & Ba, as cited for the adaptive optimiser),
 * the LNCC stabiliser cc_eps and the factor c_lp of the step-size rule
 * eps_t = eta / (c_lp max|d|) of the appendix "Limitations of Stationary
 * Velocity Fields" (c_lp = 2: the bound LP(v) <= sup 2|v| / |dx|). */
typedef struct {
    int32_t n_levels;     /* 1..8 */
    int32_t scales[8];    /* downsampling factor per level, >= 1 */
    int32_t iters[8];     /* iterations per level, >= 0 */
    float lr;             /* eta, > 0 */
    float sigma_grad;     /* >= 0, voxels of the level; 0 = no smoothing */
    float sigma_warp;     /* >= 0 */
    int32_t window;       /* odd LNCC box width, 1..15 */
    int32_t loss;         /* fa_loss */
    float beta1, beta2, adam_eps;
    float cc_eps;         /* >= 0 */
    float c_lp;           /* > 0 */
    int32_t mode;         /* fa_mode */
    int32_t storage;      /* fa_dtype of the fixed and moving images given to fa_register:
                             FA_F32, FA_BF16 or FA_F16 (16-bit images are widened once
                             to FP32 copies in the workspace; all arithmetic is FP32) */
    int32_t graph;        /* 1: fa_register records its whole launch sequence as a CUDA
                             graph on first use (stream capture on a private stream) and
                             replays it when called again with identical arguments
                             (pointers, shapes, parameters, workspace, timer); up to 64
                             graphs are kept per process.  0: launch kernel by kernel. */
    int32_t use_jac;      /* 1: steepest Eulerian direction J(phi)^T dL/dphi (section
                             "Exploiting the group structure of diffeomorphisms", Algorithm 1
                             use_jac) instead of the Jacobian-free dL/dphi; see
                             fa_jac_direction.  0 (default): Jacobian-free. */
    int32_t mi_bins;      /* histogram bins B of FA_LOSS_MI, 6..64 (default 32) */
    int32_t state_storage; /* fa_dtype of the Adam moments m and nu kept between
                             iterations (and handed off between levels) by
                             fa_register, fa_register_from and the batched calls:
                             FA_F32 (default) or FA_BF16.  Arithmetic stays FP32: each
                             iteration reads the stored moments, updates them in FP32,
                             takes the direction from the FP32 values and stores them
                             rounded to nearest.  FA_F16 is refused
                             (FA_ERR_UNSUPPORTED): its smallest normal value, 6.1e-5,
                             lies far above the moments of a loss gradient that scales
                             as 1/N, which would flush to zero.  The displacement u is
                             stored as field_storage (below).
                             The symmetric, SVF, inverse, affine and rigid calls take
                             FA_F32 only (FA_ERR_UNSUPPORTED otherwise). */
    int32_t field_storage; /* fa_dtype of the displacement u kept between iterations and
                             levels by fa_register, fa_register_from and
                             fa_register_batched: FA_F32 (default) or FA_F16.  With
                             FA_F16 every update of u is rounded to FP16 when stored
                             (arithmetic stays FP32; u_out is returned in FP32); it
                             needs FA_MODE_FUSED, the LNCC loss, use_jac = 0 and both
                             Gaussians within the fused kernels' radius
                             (FA_ERR_UNSUPPORTED otherwise).
                             fa_register_batched_lockstep takes FA_F16 under the same
                             conditions; every other call takes FA_F32 only. */
} fa_params;

/* Fills p with: 3 levels {4,2,1} x {200,100,50}, lr 0.5, sigma_grad 1,
 * sigma_warp 0.5, window 5, LNCC, Adam (0.9, 0.999, 1e-8), cc_eps 1e-5,
 * c_lp 2, fused mode, FP32 storage, graph replay on, Jacobian-free direction,
 * 32 MI bins, FP32 Adam moments. */
fa_status fa_params_default(fa_params *p);

const char *fa_status_str(fa_status s);
/* Message of the last failing call made by this host thread ("" if none). */
const char *fa_last_error(void);

/* Number of kernels this library has launched in this process (all threads);
 * benchmarks difference it around a timed region. */
uint64_t fa_launch_count(void);

/* ---------------------------------------------------------------------------
 * Building blocks.  Each is one step of the per-iteration loop; fa_register
 * chains them (or their fused forms) for whole registrations.
 * ------------------------------------------------------------------------- */

/* Warp (section "Preliminaries": (I o phi)(x) = I(phi(x)); pushforward form
 * of section "Alternative formulations for Eulerian differential"):
 *   out(x) = moving(x + u(x)), trilinear, zero outside the grid;
 *   grad_opt(x) = gradient of the trilinear interpolant of `moving` at
 *   x + u(x) (derivative inside the cell floor(x + u), one-sided at integer
 *   coordinates); may be NULL.
 * moving: C=1; u: C=3; out: C=1; grad_opt: C=3; all on one D x H x W grid,
 * FA_F32.  No workspace. */
fa_status fa_warp(const fa_vol *moving, const fa_vol *u, fa_vol *out, fa_vol *grad_opt,
                  void *stream);

/* Bytes of workspace fa_lncc_fwd_bwd needs for a D x H x W grid. */
size_t fa_lncc_workspace_size(int32_t D, int32_t H, int32_t W);

/* LNCC loss (the local normalised cross-correlation cost named with
 * Eq. (image-reg); window size is its hyper-parameter) and its Gateaux
 * derivatives (section "Jacobian-Free Eulerian Descent").  Definition:
 * box window of width `window` (odd), zero padding, fixed divisor
 * n = window^3; cross = S_IJ - S_I S_J / n, var_I = S_II - S_I^2 / n,
 * var_J = S_JJ - S_J^2 / n, cc = cross^2 / (var_I var_J + cc_eps),
 * L = -(1/N) sum_x cc(x).
 *   loss_dev         device float, receives L (may be NULL)
 *   dL_dwarped_opt   C=1, receives dL/dJ (may be NULL)
 *   dL_dfixed_opt    C=1, receives dL/dI (may be NULL)
 * fixed, warped: C=1, FA_F32, same grid.  window in 1..15.  Workspace of
 * fa_lncc_workspace_size bytes, 256-byte aligned. */
fa_status fa_lncc_fwd_bwd(const fa_vol *fixed, const fa_vol *warped, int32_t window,
                          float cc_eps, float *loss_dev, fa_vol *dL_dwarped_opt,
                          fa_vol *dL_dfixed_opt, void *ws, size_t ws_bytes, void *stream);

/* Same computation and arguments as fa_lncc_fwd_bwd, for callers that
 * cannot allocate device memory (code where cudaMalloc is forbidden or
 * unavailable, e.g. inside another library's allocation-free section, a
 * plugin host that owns every device allocation, or a loop that must never
 * enter the allocator).  No workspace argument: scratch is a 64 MiB array
 * built into the library, held by every GPU that loads it until exit, so the
 * grid may hold at most 621,376 voxels (larger grids return FA_ERR_SHAPE
 * before any launch).  The first call on each device looks up the array's
 * address with that device current; make it before any stream capture.
 * The address is kept per device and CUDA context: after a device reset the
 * next call looks it up again and must likewise precede any capture.
 * All calls share the array (each clears what must start at zero); calls
 * that overlap on the GPU race and must be serialised by the caller.  No
 * counterpart in the paper: an integration convenience of this library. */
fa_status fa_lncc_fwd_bwd_noalloc(const fa_vol *fixed, const fa_vol *warped, int32_t window,
                                  float cc_eps, float *loss_dev, fa_vol *dL_dwarped_opt,
                                  fa_vol *dL_dfixed_opt, void *stream);

/* MSE loss L = (1/N) sum (J - I)^2 (the squared-intensity cost of section
 * "Deformable Image Registration is a severely ill-conditioned problem",
 * normalised by N) and dL/dJ = 2 (J - I) / N, dL/dI = -dL/dJ.  Same argument
 * conventions as fa_lncc_fwd_bwd; workspace of fa_lncc_workspace_size. */
fa_status fa_mse_fwd_bwd(const fa_vol *fixed, const fa_vol *warped, float *loss_dev,
                         fa_vol *dL_dwarped_opt, fa_vol *dL_dfixed_opt, void *ws,
                         size_t ws_bytes, void *stream);

/* Mutual-information loss (the MI cost named with LNCC in section
 * "Deformable Image Registration"; its bin count is a hyper-parameter of the
 * hyper-parameter study).  Parzen-window estimate with the cubic B-spline
 * beta3 on `bins` bins (6..64) for both images: intensity v of an image with
 * range [lo, hi] sits at xi = 1 + (v - lo) (bins - 3) / (hi - lo), clamped
 * to [1, bins - 2];
 *   P(a,b) = (1/N) sum_x beta3(xi_f(x) - a) beta3(xi_J(x) - b),
 *   L = -MI = -sum_{a,b} P log(P / (p_f(a) p_J(b))),
 *   dL/dJ(x) = -(1/N) (bins - 3) / (hi_J - lo_J)
 *              sum_{a,b} log(P / (p_f p_J)) beta3(xi_f - a) beta3'(xi_J - b).
 * range_dev_opt: 4 device floats lo_f, hi_f, lo_J, hi_J; NULL takes [min, max]
 * of `fixed` and of `warped` with 0 included (fa_register takes the moving
 * image's range with 0 included, since samples outside the grid are 0).
 * loss_dev (device float) receives L; dL_dwarped_opt (C=1) dL/dJ (either may
 * be NULL).  The joint histogram is accumulated in 2^-32 fixed point with
 * integer atomics: the result does not depend on thread order.  FA_F32,
 * same grid; workspace of fa_mi_workspace_size(bins) bytes (0: bins out of
 * range). */
size_t fa_mi_workspace_size(int32_t bins);
fa_status fa_mi_fwd_bwd(const fa_vol *fixed, const fa_vol *warped, int32_t bins,
                        const float *range_dev_opt, float *loss_dev, fa_vol *dL_dwarped_opt,
                        void *ws, size_t ws_bytes, void *stream);

/* Bytes of workspace fa_gauss_smooth needs for C channels of D x H x W. */
size_t fa_gauss_workspace_size(int32_t C, int32_t D, int32_t H, int32_t W);

/* Separable Gaussian smoothing of each channel (sigma_grad / sigma_warp of
 * the hyper-parameter study, in voxels): taps exp(-k^2 / 2 sigma^2) for
 * |k| <= ceil(3 sigma), normalised to sum 1, zero padding.  sigma = 0 copies.
 * in, out: same C, D, H, W, FA_F32; in == out is allowed.  sigma <= 10. */
fa_status fa_gauss_smooth(const fa_vol *in, fa_vol *out, float sigma, void *ws,
                          size_t ws_bytes, void *stream);

/* Bytes of workspace fa_radam_step needs for a D x H x W grid. */
size_t fa_radam_workspace_size(int32_t D, int32_t H, int32_t W);

/* One Riemannian Adam step (section "Adaptive optimization on
 * diffeomorphisms"; Algorithm 1 optimiser update and compositive update):
 *   m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;
 *   d = (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + adam_eps);
 *   eps_t = lr / (c_lp max_x |d(x)|)  (0 if the max is 0);  delta = -eps_t d;
 *   u_out(x) = delta(x) + u_in(x + delta(x))   (phi <- phi o (id + delta)).
 * u_in(x + delta) is trilinear with zero outside the grid; where every
 * component of delta(x) is below one voxel it is taken on the cell between x
 * and its neighbours on delta's side (weights |delta_a|, exact), elsewhere on
 * the floor cell: the same interpolant, rounded as fa_register's fused
 * schedule rounds it.
 * u_in, u_out, g: C=3, FA_F32; m, v: C=3, both FA_F32, both FA_BF16 or both
 * FA_F16 (16-bit moments are read, updated in FP32 and stored rounded to
 * nearest, the direction coming from the FP32 values; FP16 moments must lie
 * in its normal range to keep their precision); one grid; u_out must not
 * alias u_in.
 * t_dev is a DEVICE int32 holding the number of steps taken so far (0 before
 * the first): the step uses t = *t_dev + 1 and the call advances *t_dev to t
 * on the stream, so a sequence of calls can be recorded in a CUDA graph and
 * replayed without host involvement.  The bias corrections 1 / (1 - beta^t)
 * are formed on the device in FP32 as -1 / expm1(t log1p(beta - 1)).  A
 * counter below 0 leaves u_out = u_in and sets FA_ERR_NONFINITE in the
 * status word.  Uses p->beta1, beta2, adam_eps, lr, c_lp.  eps_t_dev (device
 * float, may be NULL) receives eps_t.  A non-finite max|d| sets the
 * workspace status word (see fa_ws_status). */
fa_status fa_radam_step(const fa_vol *u_in, fa_vol *u_out, fa_vol *m, fa_vol *v,
                        const fa_vol *g, int32_t *t_dev, const fa_params *p, float *eps_t_dev,
                        void *ws, size_t ws_bytes, void *stream);

/* Pyramid level (Algorithm 1 "downsample(I, s)"; section "Interpolation
 * strategies for multi-scale registration"): Gaussian blur with sigma = s/2
 * on the input grid, then trilinear align-corners sampling onto the output
 * grid, whose size must be max(1, floor(N_a / s)) per axis.  s = 1 copies.
 * img, out: C=1, FA_F32.  Workspace of fa_gauss_workspace_size(1, D, H, W). */
fa_status fa_pyramid_level(const fa_vol *img, int32_t s, fa_vol *out, void *ws,
                           size_t ws_bytes, void *stream);

/* The whole pyramid of Algorithm 1 ("downsample" for every level) in one
 * call: levels[l] (C=1, FA_F32, max(1, floor(N_a / p->scales[l])) per axis)
 * receives fa_pyramid_level(img, p->scales[l]) for l = 0 .. p->n_levels - 1
 * (only n_levels and scales of p are read; scale 1 copies img).  No level
 * may alias img.  Workspace of fa_pyramid_workspace_size bytes (two
 * full-grid temporaries shared by the levels; 0 for invalid arguments). */
size_t fa_pyramid_workspace_size(int32_t D, int32_t H, int32_t W, const fa_params *p);
fa_status fa_pyramid(const fa_vol *img, const fa_params *p, fa_vol *levels, void *ws,
                     size_t ws_bytes, void *stream);

/* Level hand-off (section "Interpolation strategies": trilinear upsampling
 * of phi and of the optimiser state m, nu; Algorithm 1 "Upsample"):
 * trilinear align-corners resampling of a 3-channel field from `coarse` onto
 * `fine`, then channel a is multiplied by s_a^power with
 * s_a = (Nf_a - 1) / (Nc_a - 1) (1 when either size is 1):
 * power = 1 for the displacement u, -1 for the first moment m, -2 for the
 * second moment nu.  C=3, FA_F32.  No workspace. */
fa_status fa_upsample_field(const fa_vol *coarse, fa_vol *fine, int32_t power, void *stream);

/* ---------------------------------------------------------------------------
 * Whole registration (Algorithm 1 with the Jacobian-free direction).
 * Per iteration: warp -> loss and dL/dphi -> Gaussian(sigma_grad) -> Adam ->
 * step scaling -> compose -> Gaussian(sigma_warp).  Levels run coarsest
 * first; u, m, nu are handed off with fa_upsample_field's rule; the Adam
 * step counter carries across levels.
 * ------------------------------------------------------------------------- */

/* Bytes of workspace fa_register needs for a D x H x W pair (0: invalid
 * parameters); fa_workspace_size is the same query from the fixed image's
 * descriptor. */
size_t fa_register_workspace_size(int32_t D, int32_t H, int32_t W, const fa_params *p);
size_t fa_workspace_size(const fa_vol *fixed, const fa_params *p);

/* fixed, moving: C=1, dtype p->storage, same D x H x W.  u_out: C=3 FA_F32 on the grid of the
 * last level (max(1, floor(N_a / s_last))).  final_loss_dev (device float,
 * may be NULL) receives the loss at the final map on the last level
 * (for LNCC that is -mean cc).  If final_loss_host is not NULL the call
 * waits for the stream, stores that loss there and returns
 * FA_ERR_NONFINITE / FA_ERR_TIMEOUT if the device status word is set;
 * otherwise it returns after enqueueing (read the status with fa_ws_status).
 * Workspace of fa_register_workspace_size bytes, 256-byte aligned. */
fa_status fa_register(const fa_vol *fixed, const fa_vol *moving, const fa_params *p,
                      fa_vol *u_out, float *final_loss_dev, float *final_loss_host, void *ws,
                      size_t ws_bytes, void *stream);

/* Compositive update with a given step field (section "Minimizing the
 * Eulerian differential", Algorithm 1's retraction): out = delta + u o (id +
 * delta), trilinear with zero outside.  C=3 FA_F32 on one grid; out must not
 * be u.  No workspace. */
fa_status fa_compose(const fa_vol *u, const fa_vol *delta, fa_vol *out, void *stream);

/* Exponential of a stationary velocity field by scaling and squaring
 * (section "Adaptive Optimization for Diffeomorphisms", Eqs. ssbasecase and
 * scalingandsquaring; the parametrisation the paper compares against):
 * out = exp(v) - id after `steps` (0..30) squarings of id + v / 2^steps,
 * each squaring a fa_compose of the field with itself.  C=3 FA_F32;
 * workspace of fa_svf_exp_workspace_size bytes (one field). */
size_t fa_svf_exp_workspace_size(int32_t D, int32_t H, int32_t W);
fa_status fa_svf_exp(const fa_vol *v, int32_t steps, fa_vol *out, void *ws, size_t ws_bytes,
                     void *stream);

/* The Lie-algebra ("exp") registration the paper compares its method with
 * (section "Euclidean gradient descent using the Lie algebra in shooting
 * methods"; the exp curves of the grid study): a stationary velocity v is
 * optimised, phi = exp(v) - id by fa_svf_exp's scaling and squaring with
 * `steps` squarings (0..12), and dL/dphi (loss of p: LNCC, MSE or MI) is
 * pulled back into the algebra by the exact adjoint of the squarings
 *   gbar_k(x) = (I + grad u_k(x + u_k(x)))^T gbar_{k+1}(x)
 *               + sum_y w_x(y + u_k(y)) gbar_{k+1}(y),   grad_v = gbar_0 / 2^M
 * (w_x(p): trilinear weight of grid point x at p; the scatter accumulates in
 * 64-bit fixed point, order-independent).  Each iteration: Gaussian
 * (sigma_grad) of grad_v, Adam, the step rule eps_t = lr / (c_lp max|d|),
 * the additive update v <- v - eps_t d, Gaussian (sigma_warp) of v; v, m, nu
 * are handed off between levels like fa_register's u, m, nu.  p->use_jac must
 * be 0; p->mode and p->graph are ignored (per-op kernels).  u_out (C=3,
 * last level's grid) receives exp(v) - id, v_out_opt the velocity,
 * final_loss_dev (may be NULL) the loss there.  Workspace of
 * fa_register_svf_workspace_size bytes (0: invalid arguments).
 *
 * fa_svf_loss_grad evaluates L(I_f, I_m o exp(v)), grad_v L and optionally
 * exp(v) - id on one grid (p gives the loss; its schedule is ignored);
 * workspace of fa_register_svf_workspace_size for a one-level schedule at
 * scale 1. */
size_t fa_register_svf_workspace_size(int32_t D, int32_t H, int32_t W, const fa_params *p,
                                      int32_t steps);
fa_status fa_register_svf(const fa_vol *fixed, const fa_vol *moving, const fa_params *p,
                          int32_t steps, fa_vol *u_out, fa_vol *v_out_opt, float *final_loss_dev,
                          void *ws, size_t ws_bytes, void *stream);
fa_status fa_svf_loss_grad(const fa_vol *fixed, const fa_vol *moving, const fa_vol *v,
                           const fa_params *p, int32_t steps, float *loss_dev, fa_vol *grad_v_out,
                           fa_vol *u_out_opt, void *ws, size_t ws_bytes, void *stream);

/* Steepest Eulerian descent direction (section "Exploiting the group
 * structure of diffeomorphisms"; Algorithm 1 with use_jac):
 * g_out = J(phi)^T g_in with J(phi) = I + grad u, i.e.
 * g_out_a = g_in_a + sum_j (d u_j / d x_a) g_in_j, the derivatives by central
 * differences inside the grid and one-sided first differences at its ends
 * (zero on an axis of length 1).  All C=3 FA_F32 on one grid; g_out may be
 * g_in (in place) but must not otherwise overlap it.  No workspace. */
fa_status fa_jac_direction(const fa_vol *g_in, const fa_vol *u, fa_vol *g_out, void *stream);

/* ---------------------------------------------------------------------------
 * Differentiation of the warp + LNCC loss (the Gateaux derivative of section
 * "Jacobian-free Eulerian descent" plus the adjoints with respect to both
 * images).  L = LNCC(I_f, I_m o (id + u)) exactly as fa_lncc_fwd_bwd
 * defines it; dL_du = dL/dJ * grad I_m(phi) (C=3); dL_dfixed = dL/dI_f;
 * dL_dmoving(p) = sum_x dL/dJ(x) w_p(x), w_p the trilinear weight of voxel
 * p at x + u(x) (zero outside), accumulated in 2^-40-relative fixed point
 * with integer atomics (order-independent).  Every output may be NULL.
 * All volumes FA_F32 on one grid.  Workspace of
 * fa_warp_lncc_adjoint_workspace_size bytes, 256-byte aligned. */
size_t fa_warp_lncc_adjoint_workspace_size(int32_t D, int32_t H, int32_t W);
fa_status fa_warp_lncc_adjoint(const fa_vol *fixed, const fa_vol *moving, const fa_vol *u,
                               int32_t window, float cc_eps, float *loss_dev, fa_vol *dL_du_opt,
                               fa_vol *dL_dfixed_opt, fa_vol *dL_dmoving_opt, void *ws,
                               size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Many registrations in one call (no counterpart in the paper's text beyond
 * the independence of registrations in Algorithm 1; the paper's own
 * hyper-parameter sweeps run many such registrations, section "Results:
 * Runtime and Memory Efficiency Analysis").
 *
 * Job j = pair * n_cfg + cfg registers fixed[pair] to moving[pair] with
 * cfgs[cfg] (every field of fa_register's parameters may differ between
 * sets, including the pyramid).  Pairs may have different grids.
 * u_out[j] (C=3) is on the last level's grid of that job; final_loss_dev
 * (n_pairs * n_cfg device floats, may be NULL) receives each job's final
 * loss; status_dev (n_pairs * n_cfg device uint32, may be NULL) receives
 * each job's device status bits (1: non-finite value, 2: a bounded wait gave
 * up; 0: ok).
 *
 * Jobs run on `concurrency` (1..32) internal streams of the current device,
 * forked from `stream` with events and joined back into it: work enqueued
 * on `stream` afterwards sees every job's results.  Slot k of the workspace
 * (fa_register_batched_workspace_size bytes, 256-byte aligned) serves jobs
 * k, k + concurrency, ... in order.  Every job's arguments are checked
 * before anything is enqueued.  The call returns after enqueueing.  The
 * internal streams are created on first use and kept until the process
 * exits; make the first call before a stream capture. */
size_t fa_register_batched_workspace_size(int32_t n_pairs, const fa_vol *fixed, int32_t n_cfg,
                                          const fa_params *cfgs, int32_t concurrency);
fa_status fa_register_batched(int32_t n_pairs, const fa_vol *fixed, const fa_vol *moving,
                              int32_t n_cfg, const fa_params *cfgs, fa_vol *u_out,
                              float *final_loss_dev, uint32_t *status_dev, int32_t concurrency,
                              void *ws, size_t ws_bytes, void *stream);

/* The same jobs in lockstep (Algorithm 1 per job, as above; the lockstep
 * schedule itself has no counterpart in the paper): the jobs of a wave
 * advance level by level and iteration by iteration together, and every
 * iteration is ONE launch of each fused kernel over the tiles of every job
 * of the wave (K3: one launch per distinct Gaussian radius and moment
 * storage among the jobs; K4: per distinct Gaussian radius, compose variant
 * and storage of u).  Per-job set-up (pyramid, level start,
 * hand-off, final loss) runs as per-job launches between iterations.
 * Results are those of one fa_register call per job (the kernels compute
 * the same bits whatever the tiling).
 *
 * Same arguments, outputs and status words as fa_register_batched, except:
 *  - jobs_per_wave (1..64): jobs run in waves of this many, one wave after
 *    another on `stream` in the same workspace (fa_register_lockstep_
 *    workspace_size bytes: one slice per job of a wave, each sized for the
 *    largest job; 256-byte aligned);
 *  - every job needs mode FA_MODE_FUSED, loss FA_LOSS_LNCC, use_jac 0,
 *    sigma_grad and sigma_warp at most 2 (Gaussian radius <= 6), and the
 *    jobs of a wave share n_levels, scales, iters, window, beta1, beta2 and
 *    adam_eps; lr, c_lp, cc_eps, the sigmas, the storage types (of the
 *    moments and of u) and the grids may differ.  Otherwise FA_ERR_UNSUPPORTED before anything is enqueued.
 * With graph set in every parameter set, each wave is recorded as one CUDA
 * graph on first use and replayed by later identical calls (not during a
 * stream capture of the caller's).  Everything runs on `stream`; the call
 * returns after enqueueing. */
size_t fa_register_lockstep_workspace_size(int32_t n_pairs, const fa_vol *fixed, int32_t n_cfg,
                                           const fa_params *cfgs, int32_t jobs_per_wave);
fa_status fa_register_batched_lockstep(int32_t n_pairs, const fa_vol *fixed,
                                       const fa_vol *moving, int32_t n_cfg,
                                       const fa_params *cfgs, fa_vol *u_out,
                                       float *final_loss_dev, uint32_t *status_dev,
                                       int32_t jobs_per_wave, void *ws, size_t ws_bytes,
                                       void *stream);

/* ---------------------------------------------------------------------------
 * Tile autotuning of the fused kernels (no counterpart in the paper).
 * fa_autotune times, for every pyramid level of a D x H x W registration
 * with parameters p, candidate slab depths (and 32 x 16 instead of 32 x 8
 * tiles for the Gaussian kernels) of the four fused kernels on the given
 * workspace (fa_register_workspace_size bytes; its contents are
 * overwritten), waits for `stream`, and keeps the fastest choice per kernel,
 * radius and grid for every later launch in this process.  Every choice
 * computes the same bits; only the speed changes.  It also drops the
 * recorded graphs (they hold the previous choices).  Not during a stream
 * capture.  fa_autotune_reset forgets all choices; fa_autotune_choices
 * writes up to `capacity` rows of 8 int32 (kernel 0..3, radius, compose
 * variant, D, H, W, 16-warp tiles, slab depth) and returns the number of
 * recorded choices.  fa_autotune_set records one such row (a choice made
 * elsewhere, or pinned by hand).
 *
 * Process-wide state.  Apart from the caller's buffers, libfa keeps three
 * things per process, shared by every caller and every thread:
 *  - the tile choices above (they change the speed of later fused launches,
 *    never their results);
 *  - the recorded graphs of fa_register / fa_register_batched_lockstep with
 *    p->graph set: up to 64, keyed on the call's pointers, shapes and
 *    parameters, least recently used dropped first.  A graph holds device
 *    addresses: after freeing a buffer that a recorded call used, call
 *    fa_graph_cache_clear (or pass graph = 0) before the memory is reused
 *    under the same key.  Lookups are locked; a graph in use by one thread
 *    stays valid while another thread evicts or clears it;
 *  - internal streams (capture streams per host thread and device, and the
 *    forked streams of fa_register_batched), created on first use.
 * fa_graph_cache_clear drops every recorded graph (each is destroyed once no
 * launch holds it; graphs already launched finish normally). */
fa_status fa_autotune(int32_t D, int32_t H, int32_t W, const fa_params *p, void *ws,
                      size_t ws_bytes, void *stream);
fa_status fa_autotune_reset(void);
int32_t fa_autotune_choices(int32_t *rows, int32_t capacity);
fa_status fa_autotune_set(const int32_t *row);
fa_status fa_graph_cache_clear(void);

/* fa_register starting from a displacement u_init (C=3 FA_F32 on the input
 * grid, e.g. an affine pre-alignment from fa_affine_field) instead of the
 * identity: the first level starts from u_init resampled to its grid (align
 * corners, scaled like the level hand-off) with zero Adam state.  u_init NULL
 * is fa_register. */
fa_status fa_register_from(const fa_vol *fixed, const fa_vol *moving, const fa_params *p,
                           const fa_vol *u_init, fa_vol *u_out, float *final_loss_dev,
                           float *final_loss_host, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Affine pre-registration (the paper's affine stage before the
 * diffeomorphic one, Adam at learning rate 3e-3 over a multi-scale schedule;
 * section "Lung CT mapping challenges").  The map acts on align-corners
 * normalised coordinates p_a = 2 x_a / (n_a - 1) - 1: p' = A p + t with
 * theta = (A row-major, t), 12 floats, identity start; loss LNCC or MSE as
 * in fa_register; plain Adam (lr, beta1, beta2, adam_eps of p; the other
 * smoothing and step fields are unused); the step counter carries across
 * levels.  theta_dev (12 device floats) receives the result, u_out (C=3,
 * last level's grid, may be NULL) its displacement, final_loss_dev (may be
 * NULL) the loss there.  Asynchronous; no host synchronisation, so it can
 * be recorded in a graph.  Workspace of fa_affine_workspace_size bytes. */
size_t fa_affine_workspace_size(int32_t D, int32_t H, int32_t W, const fa_params *p);
fa_status fa_affine_register(const fa_vol *fixed, const fa_vol *moving, const fa_params *p,
                             float *theta_dev, fa_vol *u_out_opt, float *final_loss_dev,
                             void *ws, size_t ws_bytes, void *stream);
/* Displacement (voxels of u_out's grid) of the affine map theta_dev. */
fa_status fa_affine_field(const float *theta_dev, fa_vol *u_out, void *stream);

/* Rigid pre-registration (the rigid group, the first of the transformation
 * groups stacked rigid -> affine -> diffeomorphism in section "Discussion").
 * The motion is rigid in the voxel coordinates of the input grid about its
 * centre: y' = R y + tau, y = x - (n - 1)/2, R = exp([w]x) (Rodrigues; w is
 * the rotation axis times the angle in radians).  Parameters rp = (w, t),
 * t = S^-1 tau in the normalised units of fa_affine_register
 * (S = diag((n_a - 1)/2), 1 on an axis of length 1); on normalised
 * coordinates the map is the affine theta = (S^-1 R S, t), the same at every
 * level.  Identity start; plain Adam on the 6 parameters (lr, beta1, beta2,
 * adam_eps of p) with the exact gradient (the 12 affine sums pulled back
 * through dR/dw, evaluated in FP32 by one thread); loss, scales and
 * iterations as fa_affine_register.  rp_dev (6 device floats) receives the
 * parameters, theta_dev (12, may be NULL) the equivalent affine map, u_out
 * (may be NULL) its displacement on the last level's grid, final_loss_dev
 * (may be NULL) the loss there.  Workspace of fa_affine_workspace_size
 * bytes. */
fa_status fa_rigid_register(const fa_vol *fixed, const fa_vol *moving, const fa_params *p,
                            float *rp_dev, float *theta_dev, fa_vol *u_out_opt,
                            float *final_loss_dev, void *ws, size_t ws_bytes, void *stream);
/* The affine map theta (12 device floats, as fa_affine_register's) of the
 * rigid parameters rp_dev = (w, t) (6 device floats) for a D x H x W input
 * grid: (S^-1 R S, t) with R = exp([w]x), in FP32 (Rodrigues with Taylor
 * series below |w| = 1, Cody-Waite reduced sine and cosine above). */
fa_status fa_rigid_theta(const float *rp_dev, int32_t D, int32_t H, int32_t W, float *theta_dev,
                         void *stream);

/* ---------------------------------------------------------------------------
 * Post-hoc inverse of a displacement (section "Alternative formulations for
 * Eulerian differential": the inverse map is found after the registration by
 * an optimisation of the same kind).  With phi = id + u and psi = id + w the
 * energy is the inverse-consistency error
 *   E(w) = (1/N) sum_x |u(x) + w(x + u(x))|^2 + |w(x) + u(x + w(x))|^2
 * (trilinear, zero outside), minimised over the multi-scale schedule of p
 * (scales, iters, sigma_grad, sigma_warp, lr, c_lp, Adam constants; the loss
 * fields are unused) with the Algorithm 1 update: Gaussian(sigma_grad) of
 * the gradient, Adam, step scaling, compose, Gaussian(sigma_warp).  Level l
 * works on u resampled to its grid (align corners, scaled to its voxels);
 * w, m and v are handed off between levels like fa_register's.
 * u: C=3 FA_F32 on the input grid; w_out: C=3 FA_F32 on the last level's
 * grid; final_energy_dev (device float, may be NULL) receives E there.
 * Deterministic: the scatter of the first term accumulates in 64-bit fixed
 * point (2^40 relative to the largest term) with integer atomics.
 * Asynchronous; workspace of fa_inverse_workspace_size bytes.
 *
 * fa_inverse_energy_grad evaluates E(w) (energy_dev, may be NULL) and its
 * exact Gateaux gradient g_out = dE/dw (C=3) on one grid, for checks and
 * for callers with their own optimiser; workspace of
 * fa_inverse_workspace_size with one level at scale 1. */
size_t fa_inverse_workspace_size(int32_t D, int32_t H, int32_t W, const fa_params *p);
fa_status fa_inverse(const fa_vol *u, const fa_params *p, fa_vol *w_out, float *final_energy_dev,
                     void *ws, size_t ws_bytes, void *stream);
fa_status fa_inverse_energy_grad(const fa_vol *u, const fa_vol *w, float *energy_dev,
                                 fa_vol *g_out, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Symmetric registration (section "Alternative formulations for Eulerian
 * differential": the symmetric objective obtains phi = phi_M o phi_F^-1
 * with the post-hoc inverse).  Two maps phi_F = id + u_F and
 * phi_M = id + u_M start at the identity and minimise
 * L(I_f o phi_F, I_m o phi_M) (p->loss, window, cc_eps); every iteration
 * applies Algorithm 1's update (p's Gaussians, Adam, step scaling, compose,
 * use_jac) to each map from its own derivative
 *   dL/dphi_F = dL/dJ_F grad I_f(phi_F),  dL/dphi_M = dL/dJ_M grad I_m(phi_M),
 * with separate Adam moments and step scales and one step counter; both maps
 * are handed off between levels like fa_register's.  On the last level w,
 * the post-hoc inverse of u_F (fa_inverse with schedule p_inv, whose scales
 * are relative to that grid and whose last scale must be 1), gives
 *   u_out = w + u_M o (id + w)   (phi_M o phi_F^-1 - id).
 * fixed/moving: C=1 volumes of p->storage; u_out and the optional uF_out,
 * uM_out: C=3 FA_F32 on the last level's grid.  final_loss_dev receives
 * L(I_f, I_m o (id + u_out)), mid_loss_dev L(I_f o phi_F, I_m o phi_M)
 * (device floats, either may be NULL).  Per-op kernels, no graph
 * recording (p->mode and p->graph are ignored).  Asynchronous; workspace of
 * fa_register_symmetric_workspace_size bytes (0: invalid arguments).
 *
 * fa_symmetric_loss_grad evaluates L(I_f o phi_F, I_m o phi_M) and both
 * derivatives on one grid (FA_F32 volumes; gF_out, gM_out: C=3); workspace
 * of fa_symmetric_loss_grad_workspace_size bytes. */
size_t fa_register_symmetric_workspace_size(int32_t D, int32_t H, int32_t W, const fa_params *p,
                                            const fa_params *p_inv);
fa_status fa_register_symmetric(const fa_vol *fixed, const fa_vol *moving, const fa_params *p,
                                const fa_params *p_inv, fa_vol *u_out, fa_vol *uF_out_opt,
                                fa_vol *uM_out_opt, float *final_loss_dev, float *mid_loss_dev,
                                void *ws, size_t ws_bytes, void *stream);
size_t fa_symmetric_loss_grad_workspace_size(int32_t D, int32_t H, int32_t W);
fa_status fa_symmetric_loss_grad(const fa_vol *fixed, const fa_vol *moving, const fa_vol *uF,
                                 const fa_vol *uM, int32_t loss, int32_t window, float cc_eps,
                                 float *loss_dev, fa_vol *gF_out, fa_vol *gM_out, void *ws,
                                 size_t ws_bytes, void *stream);

/* Waits for `stream` and returns the status word that kernels recorded in a
 * workspace used by fa_register, fa_radam_step or fa_lncc_fwd_bwd
 * (FA_OK, FA_ERR_NONFINITE or FA_ERR_TIMEOUT). */
fa_status fa_ws_status(const void *ws, void *stream);

/* Failure-detection self-test (no counterpart in the paper): one kernel
 * waits, with the bounded mbarrier wait the fused kernels use for their tile
 * copies, on a barrier that nothing completes, gives up after limit_cycles
 * SM cycles (0..2^31) and records FA_ERR_TIMEOUT in the workspace's status
 * word (read it with fa_ws_status); nothing faults or hangs and the context
 * stays usable.  ws: at least 256 bytes of device memory. */
fa_status fa_selftest_wait_timeout(void *ws, size_t ws_bytes, int64_t limit_cycles, void *stream);

/* The same for the grid barrier of the persistent coarse-level launch (no
 * counterpart in the paper): a cooperative launch of two CTAs in which one
 * never arrives; the other's bounded wait gives up after limit_cycles
 * (0..2^31) and records FA_ERR_TIMEOUT in the status word. */
fa_status fa_selftest_grid_barrier(void *ws, size_t ws_bytes, int64_t limit_cycles, void *stream);

/* ---------------------------------------------------------------------------
 * Kernel timing for benchmarks.  When `timer` is not NULL, fa_register_timed
 * records a pair of CUDA events (caller-created cudaEvent_t handles) around
 * every launch of kernel `kernel_id` on level `level` (-1: every level), in
 * order, until `capacity` pairs are used; `count` receives the number of
 * pairs recorded.  Elapsed times are then read with cudaEventElapsedTime.
 * With p->graph set, the event records are part of the recorded graph: a
 * replay records the same events again (read them before the next replay
 * of the same call), and `count` is set to the recorded number.  A level
 * whose fused kernels are timed runs them (FA_MODE_PERSISTENT's launch of a
 * coarse level has no per-kernel launches).
 * ------------------------------------------------------------------------- */
typedef enum {
    FA_K_FUSED_WARP_LNCC = 0,   /* fused: warp + LNCC forward (coefficients, loss)    */
    FA_K_FUSED_LNCC_GRAD = 1,   /* fused: LNCC adjoint sums + warp gradient -> dL/du  */
    FA_K_FUSED_SMOOTH_ADAM = 2, /* fused: Gaussian(sigma_grad) + Adam + max |d|       */
    FA_K_FUSED_COMPOSE = 3,     /* fused: compose + Gaussian(sigma_warp)              */
    FA_K_PLAIN_ANY = 4,         /* plain mode: every kernel of one iteration          */
    FA_K_FUSED_ALL = 5          /* fused: each of the four kernels above, launch order */
} fa_kernel_id;

typedef struct {
    int32_t kernel_id;
    int32_t level;
    int32_t capacity;
    int32_t count;
    void **start_events;
    void **stop_events;
} fa_kernel_timer;

fa_status fa_register_timed(const fa_vol *fixed, const fa_vol *moving, const fa_params *p,
                            fa_vol *u_out, float *final_loss_dev, float *final_loss_host,
                            void *ws, size_t ws_bytes, void *stream, fa_kernel_timer *timer);

#ifdef __cplusplus
}
#endif

#endif /* FA_H */
