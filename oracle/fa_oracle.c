/*
 * FP64 reference ("oracle") for the FireANTs registration inner loop.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA library; it is written from the paper
 * (arXiv 2404.01249, "FireANTs: Adaptive Riemannian Optimization for
 * Multi-Scale Diffeomorphic Matching") and from the readings listed below.
 *
 * Everything is plain double precision.  Loops follow the definitions: no
 * separable box sums, no sliding windows, no fusion.  The only structure
 * beyond the definitions is the separable Gaussian (the method itself smooths
 * with a separable Gaussian) and OpenMP over z-slices, which changes no
 * arithmetic (per-slice partial sums are added in slice order).
 *
 * Conventions
 *   volume  : [D][H][W] doubles, W fastest, index (z*H + y)*W + x.
 *   field   : [3][D][H][W]; channel 0 is the z (D-axis) component,
 *             channel 1 the y (H-axis), channel 2 the x (W-axis) component.
 *   coordinates are voxel units of the current level; phi(x) = x + u(x).
 *
 * Readings of points the paper leaves open (each marked "reading" below):
 *   R-sym     symmetric objective: L(I_f o phi_F, I_m o phi_M), Algorithm 1's
 *             update of each map, phi = phi_M o phi_F^-1 with the post-hoc
 *             inverse (or_register_symmetric).
 *   R-inv     post-hoc inverse: Algorithm 1's update on the
 *             inverse-consistency energy, exact Gateaux gradient (or_inverse).
 *   R-svfreg  Lie-algebra variant: v optimised, phi = exp(v) by scaling and
 *             squaring, exact adjoint of the squarings, additive update
 *             (or_register_svf).
 *   R-rigid   rigid stage: rotation exp([w]x) (Rodrigues) and translation in
 *             the input grid's voxel coordinates about its centre, as the
 *             affine map S^-1 R S, t of reading R-aff (or_rigid_register).
 *   R-aff     affine stage: p' = A p + t on align-corners normalised
 *             coordinates, identity start, plain Adam (or_affine_register).
 *   R-jac     with use_jac, grad u by central differences inside the grid and
 *             one-sided first differences at its ends (zero on an axis of 1).
 *   R-interp  trilinear interpolation, samples outside the grid are zero
 *             (u is extended by zero outside Omega, section Preliminaries).
 *   R-kink    at integer coordinates the interpolant's derivative is taken in
 *             the cell floor(p) (one-sided).
 *   R-lncc    LNCC = squared local correlation over a w^3 box with zero
 *             padding and fixed divisor n = w^3:
 *               cross = S_IJ - S_I S_J / n, varI = S_II - S_I^2 / n,
 *               varJ = S_JJ - S_J^2 / n, cc = cross^2 / (varI varJ + eps),
 *               L = -(1/N) sum_x cc(x).
 *   R-mse     L = (1/N) sum (J - I_f)^2 (the printed sum, normalised).
 *   R-mi      mutual information with cubic B-spline Parzen windows on B
 *             bins, intensities mapped to [1, B - 2] (or_mi), L = -MI.
 *   R-gauss   taps exp(-k^2 / 2 sigma^2), k in [-ceil(3 sigma), ceil(3 sigma)],
 *             normalised to sum 1, zero padding; sigma == 0 is the identity.
 *   R-adam    Kingma-Ba Adam with bias correction; t carries across levels.
 *   R-step    eps_t = eta / (c_LP * max_x |d(x)|), c_LP = 2 (the Lipschitz
 *             bound of the appendix "Limitations of Stationary Velocity
 *             Fields" with voxel spacing 1); delta = -eps_t d; eps_t = 0 when
 *             max |d| == 0.
 *   R-pyr     level size max(1, floor(N_a / s)); Gaussian blur sigma = s/2 on
 *             the fine grid, then trilinear align-corners sampling; s == 1 is
 *             the identity.
 *   R-up      level hand-off: trilinear align-corners; u scaled by
 *             s_a = (Nf_a - 1)/(Nc_a - 1) per axis, m by 1/s_a and v by
 *             1/s_a^2 (state kept fixed in normalised coordinates);
 *             s_a = 1 when Nc_a == 1 or Nf_a == 1.  m and v are statistics
 *             of dL/du, which the chain rule makes a covector (dL/du_fine =
 *             dL/du_coarse / s_a), so these factors are the ones for which
 *             the handed-off state equals the state of a fine-level Adam fed
 *             the same gradient history.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL 1

#define IDX(z, y, x) (((size_t)(z) * (size_t)H + (size_t)(y)) * (size_t)W + (size_t)(x))

static int in_grid(int z, int y, int x, int D, int H, int W) {
    return z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W;
}

/* Trilinear interpolant of vol at (pz, py, px) with zero outside the grid
 * (reading R-interp) and its gradient with respect to the sample position
 * (reading R-kink).  grad may be NULL. */
static double trilinear(const double *vol, int D, int H, int W,
                        double pz, double py, double px, double *grad) {
    if (grad) grad[0] = grad[1] = grad[2] = 0.0;
    if (isnan(pz) || isnan(py) || isnan(px)) {
        if (grad) grad[0] = grad[1] = grad[2] = NAN;
        return NAN;
    }
    /* every corner is outside: value and gradient are exactly zero */
    if (pz < -1.0 || py < -1.0 || px < -1.0 ||
        pz >= (double)D || py >= (double)H || px >= (double)W)
        return 0.0;
    double fz = floor(pz), fy = floor(py), fx = floor(px);
    int z0 = (int)fz, y0 = (int)fy, x0 = (int)fx;
    double tz = pz - fz, ty = py - fy, tx = px - fx;
    double c[2][2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e) {
                int z = z0 + a, y = y0 + b, x = x0 + e;
                c[a][b][e] = in_grid(z, y, x, D, H, W) ? vol[IDX(z, y, x)] : 0.0;
            }
    double wz[2] = {1.0 - tz, tz}, wy[2] = {1.0 - ty, ty}, wx[2] = {1.0 - tx, tx};
    double val = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e)
                val += wz[a] * wy[b] * wx[e] * c[a][b][e];
    if (grad) {
        double gz = 0.0, gy = 0.0, gx = 0.0;
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e)
                gz += (c[1][b][e] - c[0][b][e]) * wy[b] * wx[e];
        for (int a = 0; a < 2; ++a)
            for (int e = 0; e < 2; ++e)
                gy += (c[a][1][e] - c[a][0][e]) * wz[a] * wx[e];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                gx += (c[a][b][1] - c[a][b][0]) * wz[a] * wy[b];
        grad[0] = gz; grad[1] = gy; grad[2] = gx;
    }
    return val;
}

/* Pointwise sample of a volume; exported so tests can probe the interpolant. */
double or_sample(const double *vol, int D, int H, int W,
                 double pz, double py, double px, double *grad3) {
    return trilinear(vol, D, H, W, pz, py, px, grad3);
}

/* Warp (section Preliminaries: (I o phi)(x) = I(phi(x)), pushforward form of
 * section "Alternative formulations"): J(x) = I_m(x + u(x)) and, if requested,
 * gradJ(x) = (grad I_m)(x + u(x)), the interpolant's gradient at the sampled
 * point (needed by the MSE gradient of section "Deformable Image Registration
 * is a severely ill-conditioned problem" and by the LNCC chain rule). */
int or_warp(const double *Im, int D, int H, int W, const double *u,
            double *J, double *gradJ) {
    if (D <= 0 || H <= 0 || W <= 0) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                size_t i = IDX(z, y, x);
                double g[3];
                double v = trilinear(Im, D, H, W, z + u[i], y + u[N + i], x + u[2 * N + i], g);
                J[i] = v;
                if (gradJ) {
                    gradJ[i] = g[0];
                    gradJ[N + i] = g[1];
                    gradJ[2 * N + i] = g[2];
                }
            }
    return OR_OK;
}

/* Adjoint of the warp with respect to the moving intensities: for a cotangent
 * dJ on the fixed grid, dIm[k] = sum_x dJ(x) * w_k(x + u(x)) where w_k is the
 * trilinear weight of voxel k.  This is the derivative a template update needs
 * (the template is the moving image).  Serial scatter: exact order. */
int or_warp_adjoint(const double *dJ, const double *u, int D, int H, int W,
                    int Dm, int Hm, int Wm, double *dIm) {
    if (D <= 0 || H <= 0 || W <= 0 || Dm <= 0 || Hm <= 0 || Wm <= 0) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
    size_t Nm = (size_t)Dm * Hm * Wm;
    memset(dIm, 0, Nm * sizeof(double));
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                size_t i = IDX(z, y, x);
                double pz = z + u[i], py = y + u[N + i], px = x + u[2 * N + i];
                if (isnan(pz) || isnan(py) || isnan(px)) continue;
                if (pz < -1.0 || py < -1.0 || px < -1.0 ||
                    pz >= (double)Dm || py >= (double)Hm || px >= (double)Wm)
                    continue;
                double fz = floor(pz), fy = floor(py), fx = floor(px);
                int z0 = (int)fz, y0 = (int)fy, x0 = (int)fx;
                double tz = pz - fz, ty = py - fy, tx = px - fx;
                double wz[2] = {1.0 - tz, tz}, wy[2] = {1.0 - ty, ty}, wx[2] = {1.0 - tx, tx};
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        for (int e = 0; e < 2; ++e) {
                            int zz = z0 + a, yy = y0 + b, xx = x0 + e;
                            if (zz < 0 || zz >= Dm || yy < 0 || yy >= Hm || xx < 0 || xx >= Wm) continue;
                            dIm[((size_t)zz * Hm + yy) * Wm + xx] += dJ[i] * wz[a] * wy[b] * wx[e];
                        }
            }
    return OR_OK;
}

/* Window sum of v over the w^3 box centred at (z, y, x), zero padding. */
static double box_at(const double *v, int D, int H, int W, int r, int z, int y, int x) {
    double s = 0.0;
    for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx) {
                int zz = z + dz, yy = y + dy, xx = x + dx;
                if (in_grid(zz, yy, xx, D, H, W)) s += v[IDX(zz, yy, xx)];
            }
    return s;
}

/* Box sum of a whole volume, straight from the definition (exported so that
 * tests can check window extent against brute force). */
int or_box_sum(const double *in, int D, int H, int W, int win, double *out) {
    if (D <= 0 || H <= 0 || W <= 0 || win < 1 || (win % 2) == 0) return OR_EINVAL;
    int r = win / 2;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) out[IDX(z, y, x)] = box_at(in, D, H, W, r, z, y, x);
    return OR_OK;
}

/* LNCC loss (reading R-lncc; the cost named in Eq. (image-reg) and tuned by
 * its window in section "FireANTs enables rapid prototyping") and its
 * analytic Gateaux derivative with respect to the warped image J and the
 * fixed image I.
 *
 * With A = d cc / d S_IJ = 2 cross / Dn, B = d cc / d S_JJ = -cross^2 varI / Dn^2,
 * C = d cc / d S_J = -A S_I / n - 2 B S_J / n (Dn = varI varJ + eps) and the
 * mirrored B', C' for I, the chain rule through the window sums gives
 *   dL/dJ(y) = -(1/N) sum_{x : y in win(x)} [A(x) I(y) + 2 B(x) J(y) + C(x)]
 *   dL/dI(y) = -(1/N) sum_{x : y in win(x)} [A(x) J(y) + 2 B'(x) I(y) + C'(x)]
 * and {x in grid : y in win(x)} = win(y) ∩ grid for the symmetric box.
 *
 * loss   : L (scalar).  cc (nullable): per-voxel cc.  dJ, dI (nullable). */
int or_lncc(const double *I, const double *J, int D, int H, int W, int win, double cc_eps,
            double *loss, double *cc, double *dJ, double *dI) {
    if (D <= 0 || H <= 0 || W <= 0 || win < 1 || (win % 2) == 0 || cc_eps < 0.0) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
    int r = win / 2;
    double n = (double)win * win * win;
    double *II = malloc(N * sizeof(double)), *JJ = malloc(N * sizeof(double)),
           *IJ = malloc(N * sizeof(double));
    double *A = malloc(N * sizeof(double)), *B = malloc(N * sizeof(double)),
           *C = malloc(N * sizeof(double)), *Bp = malloc(N * sizeof(double)),
           *Cp = malloc(N * sizeof(double));
    double *slice = calloc((size_t)D, sizeof(double));
    if (!II || !JJ || !IJ || !A || !B || !C || !Bp || !Cp || !slice) {
        free(II); free(JJ); free(IJ); free(A); free(B); free(C); free(Bp); free(Cp); free(slice);
        return OR_EINVAL;
    }
    for (size_t i = 0; i < N; ++i) {
        II[i] = I[i] * I[i];
        JJ[i] = J[i] * J[i];
        IJ[i] = I[i] * J[i];
    }
#pragma omp parallel for schedule(static)
    for (int z = 0; z < D; ++z) {
        double acc = 0.0;
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                double sI = box_at(I, D, H, W, r, z, y, x);
                double sJ = box_at(J, D, H, W, r, z, y, x);
                double sII = box_at(II, D, H, W, r, z, y, x);
                double sJJ = box_at(JJ, D, H, W, r, z, y, x);
                double sIJ = box_at(IJ, D, H, W, r, z, y, x);
                double cross = sIJ - sI * sJ / n;
                double varI = sII - sI * sI / n;
                double varJ = sJJ - sJ * sJ / n;
                double den = varI * varJ + cc_eps;
                double c = cross * cross / den;
                size_t i = IDX(z, y, x);
                if (cc) cc[i] = c;
                acc += c;
                A[i] = 2.0 * cross / den;
                B[i] = -cross * cross * varI / (den * den);
                Bp[i] = -cross * cross * varJ / (den * den);
                C[i] = -A[i] * sI / n - 2.0 * B[i] * sJ / n;
                Cp[i] = -A[i] * sJ / n - 2.0 * Bp[i] * sI / n;
            }
        slice[z] = acc;
    }
    double total = 0.0;
    for (int z = 0; z < D; ++z) total += slice[z];
    *loss = -total / (double)N;
    if (dJ || dI) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < D; ++z)
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    size_t i = IDX(z, y, x);
                    double sA = box_at(A, D, H, W, r, z, y, x);
                    if (dJ) {
                        double sB = box_at(B, D, H, W, r, z, y, x);
                        double sC = box_at(C, D, H, W, r, z, y, x);
                        dJ[i] = -(sA * I[i] + 2.0 * sB * J[i] + sC) / (double)N;
                    }
                    if (dI) {
                        double sBp = box_at(Bp, D, H, W, r, z, y, x);
                        double sCp = box_at(Cp, D, H, W, r, z, y, x);
                        dI[i] = -(sA * J[i] + 2.0 * sBp * I[i] + sCp) / (double)N;
                    }
                }
    }
    free(II); free(JJ); free(IJ); free(A); free(B); free(C); free(Bp); free(Cp); free(slice);
    return OR_OK;
}

/* MSE loss (reading R-mse of the cost in section "Deformable Image
 * Registration is a severely ill-conditioned problem") and its derivative
 * dL/dJ = 2 (J - I) / N, dL/dI = -dL/dJ. */
int or_mse(const double *I, const double *J, int D, int H, int W,
           double *loss, double *dJ, double *dI) {
    if (D <= 0 || H <= 0 || W <= 0) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
    double total = 0.0;
    for (size_t i = 0; i < N; ++i) {
        double e = J[i] - I[i];
        total += e * e;
        if (dJ) dJ[i] = 2.0 * e / (double)N;
        if (dI) dI[i] = -2.0 * e / (double)N;
    }
    *loss = total / (double)N;
    return OR_OK;
}

/* Mutual information (the cost named with LNCC in the problem statement of
 * section "Deformable Image Registration", with a bin-count hyper-parameter
 * in the hyper-parameter study).  Reading R-mi: Parzen-window estimate with
 * the cubic B-spline beta3 on B bins (B >= 6) for both images; intensity v of
 * an image with range [lo, hi] sits at bin coordinate
 *   xi = 1 + (v - lo) (B - 3) / (hi - lo)   (xi = 1 when hi == lo),
 * clamped to [1, B - 2], so that the weights beta3(xi - k), k = 0..B-1, sum
 * to one;  P(a,b) = (1/N) sum_x beta3(xi_f(x) - a) beta3(xi_m(x) - b),
 * p_f, p_m its marginals, MI = sum P log(P / (p_f p_m)) (0 log 0 = 0),
 * L = -MI.  The exact derivative (the marginals depend on J through P; the
 * constant part of dMI/dP cancels because the weights sum to one):
 *   dL/dJ(x) = -(1/N) (B - 3) / (hi_m - lo_m)
 *              sum_{a,b} log(P / (p_f p_m)) beta3(xi_f - a) beta3'(xi_m - b).
 * The registration takes [lo, hi] of I_f from the fixed image and of J from
 * the moving image with 0 included (samples outside the grid are 0). */
static double bspline3(double t) {
    double a = fabs(t);
    if (a < 1.0) return (4.0 - 6.0 * a * a + 3.0 * a * a * a) / 6.0;
    if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
    return 0.0;
}

static double bspline3_d(double t) {
    double a = fabs(t);
    if (a < 1.0) return -2.0 * t + 1.5 * t * a;
    if (a < 2.0) return (t > 0.0 ? -1.0 : 1.0) * 0.5 * (2.0 - a) * (2.0 - a);
    return 0.0;
}

static double mi_coord(double v, double lo, double hi, int B) {
    if (!(hi > lo)) return 1.0;
    double xi = 1.0 + (v - lo) * (double)(B - 3) / (hi - lo);
    return xi < 1.0 ? 1.0 : (xi > (double)(B - 2) ? (double)(B - 2) : xi);
}

int or_mi(const double *I, const double *J, int D, int H, int W, int B, const double *range,
          double *loss, double *dJ) {
    if (D <= 0 || H <= 0 || W <= 0 || B < 6 || B > 256) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
    double *P = calloc((size_t)B * B, sizeof(double)), *pf = calloc((size_t)B, sizeof(double)),
           *pm = calloc((size_t)B, sizeof(double)), *T = calloc((size_t)B * B, sizeof(double));
    if (!P || !pf || !pm || !T) { free(P); free(pf); free(pm); free(T); return OR_EINVAL; }
    for (size_t i = 0; i < N; ++i) {
        double xf = mi_coord(I[i], range[0], range[1], B), xm = mi_coord(J[i], range[2], range[3], B);
        for (int a = 0; a < B; ++a) {
            double wa = bspline3(xf - a);
            if (wa == 0.0) continue;
            for (int b = 0; b < B; ++b) P[(size_t)a * B + b] += wa * bspline3(xm - b);
        }
    }
    for (int a = 0; a < B; ++a)
        for (int b = 0; b < B; ++b) {
            P[(size_t)a * B + b] /= (double)N;
            pf[a] += P[(size_t)a * B + b];
            pm[b] += P[(size_t)a * B + b];
        }
    double mi = 0.0;
    for (int a = 0; a < B; ++a)
        for (int b = 0; b < B; ++b) {
            double q = P[(size_t)a * B + b];
            if (q > 0.0) {
                T[(size_t)a * B + b] = log(q / (pf[a] * pm[b]));
                mi += q * T[(size_t)a * B + b];
            }
        }
    *loss = -mi;
    if (dJ) {
        double sm = range[3] > range[2] ? (double)(B - 3) / (range[3] - range[2]) : 0.0;
        for (size_t i = 0; i < N; ++i) {
            double xf = mi_coord(I[i], range[0], range[1], B), xm = mi_coord(J[i], range[2], range[3], B);
            double acc = 0.0;
            for (int a = 0; a < B; ++a) {
                double wa = bspline3(xf - a);
                if (wa == 0.0) continue;
                for (int b = 0; b < B; ++b) acc += T[(size_t)a * B + b] * wa * bspline3_d(xm - b);
            }
            dJ[i] = -acc * sm / (double)N;
        }
    }
    free(P); free(pf); free(pm); free(T);
    return OR_OK;
}

/* [lo, hi] of the fixed image and of the moving image with 0 included
 * (reading R-mi). */
int or_mi_range(const double *If, const double *Im, size_t N, double *range) {
    if (N == 0) return OR_EINVAL;
    range[0] = range[1] = If[0];
    range[2] = range[3] = 0.0;
    for (size_t i = 0; i < N; ++i) {
        range[0] = If[i] < range[0] ? If[i] : range[0];
        range[1] = If[i] > range[1] ? If[i] : range[1];
        range[2] = Im[i] < range[2] ? Im[i] : range[2];
        range[3] = Im[i] > range[3] ? Im[i] : range[3];
    }
    return OR_OK;
}

/* Gaussian taps (reading R-gauss).  Returns the radius R, fills taps[0..2R]
 * (taps[k + R] is the weight of offset k); -1 if cap is too small. */
int or_gauss_taps(double sigma, double *taps, int cap) {
    if (!(sigma >= 0.0)) return -1;
    if (sigma == 0.0) {
        if (cap < 1) return -1;
        taps[0] = 1.0;
        return 0;
    }
    int R = (int)ceil(3.0 * sigma);
    if (2 * R + 1 > cap) return -1;
    double s = 0.0;
    for (int k = -R; k <= R; ++k) {
        taps[k + R] = exp(-(double)k * k / (2.0 * sigma * sigma));
        s += taps[k + R];
    }
    for (int k = 0; k <= 2 * R; ++k) taps[k] /= s;
    return R;
}

/* One axial pass of a 1-D correlation with zero padding. axis 0 = z, 1 = y, 2 = x. */
static void axial_pass(const double *in, double *out, int D, int H, int W,
                       const double *taps, int R, int axis) {
#pragma omp parallel for schedule(static)
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                double s = 0.0;
                for (int k = -R; k <= R; ++k) {
                    int zz = z + (axis == 0 ? k : 0);
                    int yy = y + (axis == 1 ? k : 0);
                    int xx = x + (axis == 2 ? k : 0);
                    if (in_grid(zz, yy, xx, D, H, W)) s += taps[k + R] * in[IDX(zz, yy, xx)];
                }
                out[IDX(z, y, x)] = s;
            }
}

/* Separable Gaussian smoothing of C channels ([C][D][H][W]) with sigma in
 * voxels (sigma_grad / sigma_warp of the hyper-parameter study, reading
 * R-gauss).  in and out may alias. */
int or_gauss_smooth(const double *in, double *out, int C, int D, int H, int W, double sigma) {
    if (C <= 0 || D <= 0 || H <= 0 || W <= 0) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
    double taps[4096];
    int R = or_gauss_taps(sigma, taps, 4096);
    if (R < 0) return OR_EINVAL;
    if (R == 0) {
        if (out != in) memmove(out, in, (size_t)C * N * sizeof(double));
        return OR_OK;
    }
    double *a = malloc(N * sizeof(double)), *b = malloc(N * sizeof(double));
    if (!a || !b) { free(a); free(b); return OR_EINVAL; }
    for (int c = 0; c < C; ++c) {
        axial_pass(in + (size_t)c * N, a, D, H, W, taps, R, 2);
        axial_pass(a, b, D, H, W, taps, R, 1);
        axial_pass(b, out + (size_t)c * N, D, H, W, taps, R, 0);
    }
    free(a); free(b);
    return OR_OK;
}

/* Adam (section "Adaptive optimization on diffeomorphisms", Algorithm 1 step
 * "Update (v_d', optstate)"; constants of reading R-adam) applied to the
 * descent directions, which all live in the tangent space at identity:
 *   m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2) g^2,
 *   d = (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
 * t is the step number after increment (t >= 1). */
int or_adam(const double *g, double *m, double *v, double *d, size_t n, int t,
            double b1, double b2, double eps) {
    if (t < 1) return OR_EINVAL;
    double bc1 = 1.0 - pow(b1, t), bc2 = 1.0 - pow(b2, t);
    for (size_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        d[i] = (m[i] / bc1) / (sqrt(v[i] / bc2) + eps);
    }
    return OR_OK;
}

/* max_x |d(x)|_2 over a 3-channel field: the quantity that bounds the
 * Lipschitz constant in the appendix "Limitations of Stationary Velocity
 * Fields".  Returns NaN if any component is NaN. */
double or_max_norm(const double *d, int D, int H, int W) {
    size_t N = (size_t)D * H * W;
    double mx = 0.0;
    for (size_t i = 0; i < N; ++i) {
        double s = d[i] * d[i] + d[N + i] * d[N + i] + d[2 * N + i] * d[2 * N + i];
        double nrm = sqrt(s);
        if (isnan(nrm)) return NAN;
        if (nrm > mx) mx = nrm;
    }
    return mx;
}

/* Step scaling (appendix "Limitations of Stationary Velocity Fields", reading
 * R-step): delta = -eta / (c_LP max|d|) * d.  Returns the step size eps_t. */
double or_step_scale(const double *d, double *delta, int D, int H, int W, double eta, double c_lp) {
    size_t N = (size_t)D * H * W;
    double mx = or_max_norm(d, D, H, W);
    double e = (mx > 0.0) ? eta / (c_lp * mx) : 0.0;
    if (isnan(mx)) e = NAN;
    for (size_t i = 0; i < 3 * N; ++i) delta[i] = -e * d[i];
    return e;
}

/* Compositive retraction update (section "Minimizing the Eulerian
 * differential": phi_{t+1} = phi_t o (id + eta_t v_d); Algorithm 1):
 *   phi'(x) = phi(x + delta(x))  =>  u'(x) = delta(x) + u(x + delta(x)),
 * u interpolated trilinearly with zero outside (reading R-interp).
 * out must not alias u. */
int or_compose(const double *u, const double *delta, double *out, int D, int H, int W) {
    if (D <= 0 || H <= 0 || W <= 0 || out == u) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                size_t i = IDX(z, y, x);
                double pz = z + delta[i], py = y + delta[N + i], px = x + delta[2 * N + i];
                for (int c = 0; c < 3; ++c)
                    out[(size_t)c * N + i] =
                        delta[(size_t)c * N + i] + trilinear(u + (size_t)c * N, D, H, W, pz, py, px, NULL);
            }
    return OR_OK;
}

/* Exponential of a stationary velocity field by scaling and squaring
 * (section "Adaptive Optimization for Diffeomorphisms", Eqs. ssbasecase and
 * scalingandsquaring): phi^(1/2^M) = id + v / 2^M, then M squarings
 * phi <- phi o phi, i.e. u <- u + u(x + u(x)) with the zero-outside
 * trilinear interpolation of or_compose.  out receives exp(v) - id. */
int or_svf_exp(const double *v, int D, int H, int W, int steps, double *out) {
    if (D <= 0 || H <= 0 || W <= 0 || steps < 0 || out == v) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
    double *tmp = malloc(3 * N * sizeof(double));
    if (!tmp) return OR_EINVAL;
    double scale = ldexp(1.0, -steps);
    for (size_t i = 0; i < 3 * N; ++i) out[i] = v[i] * scale;
    for (int k = 0; k < steps; ++k) {
        or_compose(out, out, tmp, D, H, W);
        memcpy(out, tmp, 3 * N * sizeof(double));
    }
    free(tmp);
    return OR_OK;
}

/* Size of a pyramid level (reading R-pyr). */
int or_level_size(int n, int s) {
    int m = (s > 0) ? n / s : 0;
    return m < 1 ? 1 : m;
}

/* Align-corners source coordinate of destination index i when resampling
 * an axis of length n_src onto one of length n_dst. */
static double ac_coord(int i, int n_src, int n_dst) {
    if (n_dst <= 1 || n_src <= 1) return 0.0;
    return (double)i * (double)(n_src - 1) / (double)(n_dst - 1);
}

/* Trilinear align-corners resampling of C channels from (Ds,Hs,Ws) onto
 * (Dd,Hd,Wd); all sample points lie inside the source grid. */
static void resample_ac(const double *src, int C, int Ds, int Hs, int Ws,
                        double *dst, int Dd, int Hd, int Wd) {
    size_t Ns = (size_t)Ds * Hs * Ws, Nd = (size_t)Dd * Hd * Wd;
    for (int c = 0; c < C; ++c) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < Dd; ++z)
            for (int y = 0; y < Hd; ++y)
                for (int x = 0; x < Wd; ++x)
                    dst[(size_t)c * Nd + ((size_t)z * Hd + y) * Wd + x] =
                        trilinear(src + (size_t)c * Ns, Ds, Hs, Ws, ac_coord(z, Ds, Dd),
                                  ac_coord(y, Hs, Hd), ac_coord(x, Ws, Wd), NULL);
    }
}

/* Pyramid level (section "Interpolation strategies for multi-scale
 * registration"; Algorithm 1 "downsample(I, s_l)"; reading R-pyr): Gaussian
 * blur sigma = s/2 then trilinear align-corners sampling to
 * (max(1, D/s), max(1, H/s), max(1, W/s)). */
int or_downsample(const double *I, int D, int H, int W, int s, double *out) {
    if (D <= 0 || H <= 0 || W <= 0 || s < 1) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
    if (s == 1) {
        memmove(out, I, N * sizeof(double));
        return OR_OK;
    }
    double *blur = malloc(N * sizeof(double));
    if (!blur) return OR_EINVAL;
    int rc = or_gauss_smooth(I, blur, 1, D, H, W, 0.5 * (double)s);
    if (rc != OR_OK) { free(blur); return rc; }
    resample_ac(blur, 1, D, H, W, out, or_level_size(D, s), or_level_size(H, s), or_level_size(W, s));
    free(blur);
    return OR_OK;
}

/* Per-axis voxel-unit scale factor of the level hand-off (reading R-up). */
static double up_scale(int nc, int nf) {
    if (nc <= 1 || nf <= 1) return 1.0;
    return (double)(nf - 1) / (double)(nc - 1);
}

/* Level hand-off of a 3-channel field (section "Interpolation strategies":
 * trilinear upsampling of phi and of the optimiser state m, nu; Algorithm 1
 * "Upsample(phi, s_{l+1})").  power = 1 multiplies channel a by s_a (the
 * displacement u), power = -1 divides by s_a (the first moment m), power = -2
 * divides by s_a^2 (the second moment nu); reading R-up. */
int or_upsample_field(const double *src, int Dc, int Hc, int Wc,
                      double *dst, int Df, int Hf, int Wf, int power) {
    if (Dc <= 0 || Hc <= 0 || Wc <= 0 || Df <= 0 || Hf <= 0 || Wf <= 0) return OR_EINVAL;
    if (power != 1 && power != -1 && power != -2) return OR_EINVAL;
    size_t Nf = (size_t)Df * Hf * Wf;
    resample_ac(src, 3, Dc, Hc, Wc, dst, Df, Hf, Wf);
    double s[3] = {up_scale(Dc, Df), up_scale(Hc, Hf), up_scale(Wc, Wf)};
    for (int c = 0; c < 3; ++c) {
        double f = power == 1 ? s[c] : (power == -1 ? 1.0 / s[c] : 1.0 / (s[c] * s[c]));
        for (size_t i = 0; i < Nf; ++i) dst[(size_t)c * Nf + i] *= f;
    }
    return OR_OK;
}

/* Steepest Eulerian descent direction of section "Exploiting the group
 * structure of diffeomorphisms" (the use_jac option of Algorithm 1):
 * out = J(phi)^T g with J(phi) = I + grad u, i.e.
 *   out_i(x) = g_i(x) + sum_j (d u_j / d x_i)(x) g_j(x),
 * reading R-jac: the derivatives are central differences (u[k+1] - u[k-1]) / 2
 * inside the grid and one-sided first differences at its first and last
 * index (zero on an axis of length 1).  out must not alias g. */
static double dfd(const double *f, int D, int H, int W, int axis, int z, int y, int x) {
    int n = axis == 0 ? D : (axis == 1 ? H : W);
    int k = axis == 0 ? z : (axis == 1 ? y : x);
    if (n < 2) return 0.0;
    int dz = axis == 0, dy = axis == 1, dx = axis == 2;
    if (k == 0) return f[IDX(z + dz, y + dy, x + dx)] - f[IDX(z, y, x)];
    if (k == n - 1) return f[IDX(z, y, x)] - f[IDX(z - dz, y - dy, x - dx)];
    return 0.5 * (f[IDX(z + dz, y + dy, x + dx)] - f[IDX(z - dz, y - dy, x - dx)]);
}

int or_jac_direction(const double *g, const double *u, int D, int H, int W, double *out) {
    if (D <= 0 || H <= 0 || W <= 0 || out == g) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                size_t i = IDX(z, y, x);
                for (int a = 0; a < 3; ++a) {          /* component of the output */
                    double s = g[(size_t)a * N + i];
                    for (int j = 0; j < 3; ++j)        /* J_ja = delta_ja + d u_j / d x_a */
                        s += dfd(u + (size_t)j * N, D, H, W, a, z, y, x) * g[(size_t)j * N + i];
                    out[(size_t)a * N + i] = s;
                }
            }
    return OR_OK;
}

/* Hyper-parameters of Algorithm 1 plus the smoothing widths of the grid
 * study and the Adam constants.  Plain struct, mirrored in oracle/__init__.py. */
typedef struct {
    int n_levels;
    int scales[8];
    int iters[8];
    double lr;          /* eta */
    double sigma_grad;
    double sigma_warp;
    int window;         /* LNCC box width w (odd) */
    int loss;           /* 0 = LNCC, 1 = MSE, 2 = MI (reading R-mi) */
    double beta1, beta2, adam_eps;
    double cc_eps;
    double c_lp;        /* Lipschitz-bound factor of reading R-step (2) */
    int use_jac;        /* 1: steepest Eulerian direction J(phi)^T dL/dphi (or_jac_direction) */
    int mi_bins;        /* MI histogram bins B (loss 2) */
} or_params;

/* range: the level's MI intensity ranges (or_mi_range), used by loss 2 only */
static int loss_and_grad(const or_params *p, const double *If, const double *J,
                         int D, int H, int W, const double *range, double *L, double *dJ) {
    if (p->loss == 0) return or_lncc(If, J, D, H, W, p->window, p->cc_eps, L, NULL, dJ, NULL);
    if (p->loss == 2) return or_mi(If, J, D, H, W, p->mi_bins, range, L, dJ);
    return or_mse(If, J, D, H, W, L, dJ, NULL);
}

/* Algorithm 1 (FireANTs), Jacobian-free descent direction (section
 * "Jacobian-Free Eulerian Descent"; with use_jac the steepest direction
 * J(phi)^T dL/dphi instead), with the per-iteration order
 *   warp -> loss and dL/dphi -> Gaussian(sigma_grad) -> Adam -> step scale
 *   -> compose -> Gaussian(sigma_warp).
 * u_out receives the finest-level displacement (level size of the last
 * scale); final_loss receives L(phi_final) on the last level;
 * loss_trace (nullable, sum(iters) entries) receives the loss of every
 * iteration before its update. */
int or_register_from(const double *If, const double *Im, int D, int H, int W, const or_params *p,
                     const double *u_init, double *u_out, double *final_loss, double *loss_trace);

int or_register(const double *If, const double *Im, int D, int H, int W, const or_params *p,
                double *u_out, double *final_loss, double *loss_trace) {
    return or_register_from(If, Im, D, H, W, p, NULL, u_out, final_loss, loss_trace);
}

/* or_register starting from a displacement u_init given on the input grid
 * (NULL: the identity), e.g. an affine pre-alignment: the first level starts
 * from u_init resampled to its grid (align corners, scaled like the level
 * hand-off), with zero Adam state. */
int or_register_from(const double *If, const double *Im, int D, int H, int W, const or_params *p,
                     const double *u_init, double *u_out, double *final_loss, double *loss_trace) {
    if (D <= 0 || H <= 0 || W <= 0 || !p || p->n_levels < 1 || p->n_levels > 8) return OR_EINVAL;
    for (int l = 0; l < p->n_levels; ++l)
        if (p->scales[l] < 1 || p->iters[l] < 0) return OR_EINVAL;
    int t = 0, pd = 0, ph = 0, pw = 0, trace_i = 0;
    double *u = NULL, *m = NULL, *v = NULL;
    for (int l = 0; l < p->n_levels; ++l) {
        int s = p->scales[l];
        int d = or_level_size(D, s), h = or_level_size(H, s), w = or_level_size(W, s);
        size_t N = (size_t)d * h * w;
        double *fl = malloc(N * sizeof(double)), *ml = malloc(N * sizeof(double));
        double *nu = calloc(3 * N, sizeof(double)), *nm = calloc(3 * N, sizeof(double)),
               *nv = calloc(3 * N, sizeof(double));
        double *J = malloc(N * sizeof(double)), *gJ = malloc(3 * N * sizeof(double)),
               *dJ = malloc(N * sizeof(double)), *g = malloc(3 * N * sizeof(double)),
               *dir = malloc(3 * N * sizeof(double)), *tmp = malloc(3 * N * sizeof(double));
        if (!fl || !ml || !nu || !nm || !nv || !J || !gJ || !dJ || !g || !dir || !tmp) return OR_EINVAL;
        or_downsample(If, D, H, W, s, fl);
        or_downsample(Im, D, H, W, s, ml);
        double range[4];
        or_mi_range(fl, ml, N, range);
        if (l == 0 && u_init)
            or_upsample_field(u_init, D, H, W, nu, d, h, w, 1);
        if (l > 0) {   /* Algorithm 1: phi <- Upsample(phi), state likewise */
            or_upsample_field(u, pd, ph, pw, nu, d, h, w, 1);
            or_upsample_field(m, pd, ph, pw, nm, d, h, w, -1);
            or_upsample_field(v, pd, ph, pw, nv, d, h, w, -2);
        }
        free(u); free(m); free(v);
        u = nu; m = nm; v = nv;
        pd = d; ph = h; pw = w;
        for (int it = 0; it < p->iters[l]; ++it) {
            double L;
            or_warp(ml, d, h, w, u, J, gJ);
            loss_and_grad(p, fl, J, d, h, w, range, &L, dJ);
            if (loss_trace) loss_trace[trace_i++] = L;
            for (int c = 0; c < 3; ++c)          /* dL/dphi(x) = dL/dJ(x) grad I_m(phi(x)) */
                for (size_t i = 0; i < N; ++i) g[(size_t)c * N + i] = dJ[i] * gJ[(size_t)c * N + i];
            if (p->use_jac) {                      /* J(phi)^T dL/dphi instead */
                or_jac_direction(g, u, d, h, w, tmp);
                memcpy(g, tmp, 3 * N * sizeof(double));
            }
            or_gauss_smooth(g, g, 3, d, h, w, p->sigma_grad);
            ++t;
            or_adam(g, m, v, dir, 3 * N, t, p->beta1, p->beta2, p->adam_eps);
            or_step_scale(dir, dir, d, h, w, p->lr, p->c_lp);
            or_compose(u, dir, tmp, d, h, w);
            or_gauss_smooth(tmp, u, 3, d, h, w, p->sigma_warp);
        }
        if (l == p->n_levels - 1) {
            double L;
            or_warp(ml, d, h, w, u, J, NULL);
            loss_and_grad(p, fl, J, d, h, w, range, &L, NULL);
            *final_loss = L;
            memcpy(u_out, u, 3 * N * sizeof(double));
        }
        free(fl); free(ml); free(J); free(gJ); free(dJ); free(g); free(dir); free(tmp);
    }
    free(u); free(m); free(v);
    return OR_OK;
}

/* ------------------------------------------------------------ affine stage
 * Affine pre-registration (the paper aligns affinely before the
 * diffeomorphic stage, with Adam at learning rate 3e-3 over a multi-scale
 * schedule; section "Lung CT mapping challenges").  Reading R-aff: the map
 * acts on align-corners normalised coordinates, p_a = 2 x_a / (n_a - 1) - 1
 * (0 on an axis of length 1), p' = A p + t, so that theta = (A row-major, t)
 * means the same at every pyramid level; identity start; the loss is LNCC or
 * MSE of I_f and I_m o phi; plain Adam on the 12 parameters (no step
 * scaling); the Adam step counter carries across levels. */

/* Displacement (level voxels) of theta on a D x H x W grid:
 * u_a(x) = (p'_a - p_a) (n_a - 1) / 2. */
int or_affine_field(const double *theta, int D, int H, int W, double *u) {
    if (D <= 0 || H <= 0 || W <= 0) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
    const int n[3] = {D, H, W};
    double half[3];
    for (int a = 0; a < 3; ++a) half[a] = n[a] > 1 ? 0.5 * (n[a] - 1) : 0.0;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const int xi[3] = {z, y, x};
                double pv[3];
                for (int a = 0; a < 3; ++a) pv[a] = n[a] > 1 ? xi[a] / half[a] - 1.0 : 0.0;
                for (int a = 0; a < 3; ++a) {
                    double q = theta[9 + a];
                    for (int b = 0; b < 3; ++b) q += theta[3 * a + b] * pv[b];
                    u[(size_t)a * N + IDX(z, y, x)] = (q - pv[a]) * half[a];
                }
            }
    return OR_OK;
}

/* Loss of theta and its gradient: with g = dL/dJ grad I_m(phi) (dL/du),
 * dL/dA_ab = sum_x g_a h_a p_b and dL/dt_a = sum_x g_a h_a, h_a = (n_a - 1)/2. */
int or_affine_loss_grad(const double *If, const double *Im, int D, int H, int W,
                        const double *theta, int loss, int window, double cc_eps, double *L,
                        double *grad) {
    if (loss != 0 && loss != 1) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
    double *u = malloc(3 * N * sizeof(double)), *J = malloc(N * sizeof(double)),
           *gJ = malloc(3 * N * sizeof(double)), *dJ = malloc(N * sizeof(double));
    if (!u || !J || !gJ || !dJ) return OR_EINVAL;
    or_affine_field(theta, D, H, W, u);
    or_warp(Im, D, H, W, u, J, gJ);
    int rc = loss == 0 ? or_lncc(If, J, D, H, W, window, cc_eps, L, NULL, grad ? dJ : NULL, NULL)
                       : or_mse(If, J, D, H, W, L, grad ? dJ : NULL, NULL);
    if (rc == OR_OK && grad) {
        const int n[3] = {D, H, W};
        double half[3];
        for (int a = 0; a < 3; ++a) half[a] = n[a] > 1 ? 0.5 * (n[a] - 1) : 0.0;
        for (int k = 0; k < 12; ++k) grad[k] = 0.0;
        /* z-slices summed in order: partial sums per slice, then slice order */
        double *part = calloc((size_t)D * 12, sizeof(double));
        if (!part) return OR_EINVAL;
#pragma omp parallel for schedule(static)
        for (int z = 0; z < D; ++z) {
            double *ps = part + (size_t)z * 12;
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    size_t i = IDX(z, y, x);
                    const int xi[3] = {z, y, x};
                    double pv[3];
                    for (int a = 0; a < 3; ++a) pv[a] = n[a] > 1 ? xi[a] / half[a] - 1.0 : 0.0;
                    for (int a = 0; a < 3; ++a) {
                        double ga = dJ[i] * gJ[(size_t)a * N + i] * half[a];
                        for (int b = 0; b < 3; ++b) ps[3 * a + b] += ga * pv[b];
                        ps[9 + a] += ga;
                    }
                }
        }
        for (int z = 0; z < D; ++z)
            for (int k = 0; k < 12; ++k) grad[k] += part[(size_t)z * 12 + k];
        free(part);
    }
    free(u); free(J); free(gJ); free(dJ);
    return rc;
}

int or_affine_register(const double *If, const double *Im, int D, int H, int W,
                       const or_params *p, double *theta, double *final_loss) {
    if (D <= 0 || H <= 0 || W <= 0 || !p || p->n_levels < 1 || p->n_levels > 8) return OR_EINVAL;
    double m[12] = {0}, v[12] = {0}, g[12], dir[12];
    for (int k = 0; k < 12; ++k) theta[k] = (k == 0 || k == 4 || k == 8) ? 1.0 : 0.0;
    int t = 0;
    for (int l = 0; l < p->n_levels; ++l) {
        int s = p->scales[l];
        int d = or_level_size(D, s), h = or_level_size(H, s), w = or_level_size(W, s);
        size_t N = (size_t)d * h * w;
        double *fl = malloc(N * sizeof(double)), *ml = malloc(N * sizeof(double));
        if (!fl || !ml) return OR_EINVAL;
        or_downsample(If, D, H, W, s, fl);
        or_downsample(Im, D, H, W, s, ml);
        for (int it = 0; it < p->iters[l]; ++it) {
            double L;
            int rc = or_affine_loss_grad(fl, ml, d, h, w, theta, p->loss, p->window, p->cc_eps, &L, g);
            if (rc != OR_OK) return rc;
            ++t;
            or_adam(g, m, v, dir, 12, t, p->beta1, p->beta2, p->adam_eps);
            for (int k = 0; k < 12; ++k) theta[k] -= p->lr * dir[k];
        }
        if (l == p->n_levels - 1)
            or_affine_loss_grad(fl, ml, d, h, w, theta, p->loss, p->window, p->cc_eps, final_loss, NULL);
        free(fl); free(ml);
    }
    return OR_OK;
}

/* ------------------------------------------------ stationary velocity field
 * The Lie-algebra ("exp") variant the paper compares against (section
 * "Euclidean gradient descent using the Lie algebra in shooting methods"): a
 * velocity v is optimised, phi = exp(v) by scaling and squaring
 * (or_svf_exp), and dL/dphi is pulled back into the algebra,
 * grad_v L = (dphi/dv)^T grad_phi L.  Reading R-svfreg: the pull-back is the
 * exact adjoint of the squarings; one squaring u' = u + u o (id + u) has the
 * adjoint
 *   gbar(x) = (I + grad u(x + u(x)))^T gbar'(x) + sum_y w_x(y + u(y)) gbar'(y)
 * (w_x(p): trilinear weight of grid point x at p, zero outside), and
 * u_0 = v / 2^M gives grad_v L = gbar_0 / 2^M.  The update is Algorithm 1's
 * with the retraction replaced by the algebra's addition: Gaussian(sigma_grad)
 * of grad_v L, Adam, step scaling, v <- v - eps_t d, Gaussian(sigma_warp) of
 * v; v, m and nu are handed off between levels as u is. */

/* gbar of one squaring of u from gbar' (gp); out must not alias gp. */
static void svf_square_adjoint(const double *u, const double *gp, int D, int H, int W,
                               double *out) {
    size_t N = (size_t)D * H * W;
    memset(out, 0, 3 * N * sizeof(double));
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                size_t i = IDX(z, y, x);
                double pz = z + u[i], py = y + u[N + i], px = x + u[2 * N + i];
                double G[3][3];
                for (int c = 0; c < 3; ++c) trilinear(u + (size_t)c * N, D, H, W, pz, py, px, G[c]);
                for (int a = 0; a < 3; ++a) {
                    double acc = gp[(size_t)a * N + i];
                    for (int j = 0; j < 3; ++j) acc += G[j][a] * gp[(size_t)j * N + i];
                    out[(size_t)a * N + i] += acc;
                }
                if (isnan(pz) || isnan(py) || isnan(px) || pz < -1.0 || py < -1.0 || px < -1.0 ||
                    pz >= (double)D || py >= (double)H || px >= (double)W)
                    continue;
                double fz = floor(pz), fy = floor(py), fx = floor(px);
                int z0 = (int)fz, y0 = (int)fy, x0 = (int)fx;
                double tz = pz - fz, ty = py - fy, tx = px - fx;
                double wz[2] = {1.0 - tz, tz}, wy[2] = {1.0 - ty, ty}, wx[2] = {1.0 - tx, tx};
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        for (int e = 0; e < 2; ++e) {
                            int zz = z0 + a, yy = y0 + b, xx = x0 + e;
                            if (!in_grid(zz, yy, xx, D, H, W)) continue;
                            double wt = wz[a] * wy[b] * wx[e];
                            for (int c = 0; c < 3; ++c)
                                out[(size_t)c * N + IDX(zz, yy, xx)] += wt * gp[(size_t)c * N + i];
                        }
            }
}

/* L(I_f, I_m o exp(v)) with loss p->loss (range: the MI ranges of the level),
 * grad_v L (gv, nullable) and exp(v) - id (u_out, nullable). */
int or_svf_loss_grad(const double *If, const double *Im, int D, int H, int W, const or_params *p,
                     int steps, const double *range, const double *v, double *L, double *gv,
                     double *u_out) {
    if (D <= 0 || H <= 0 || W <= 0 || steps < 0 || steps > 16) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
    double *us = malloc((size_t)(steps + 1) * 3 * N * sizeof(double));
    double *J = malloc(N * sizeof(double)), *gJ = malloc(3 * N * sizeof(double)),
           *dJ = malloc(N * sizeof(double)), *g = malloc(3 * N * sizeof(double)),
           *g2 = malloc(3 * N * sizeof(double));
    if (!us || !J || !gJ || !dJ || !g || !g2) return OR_EINVAL;
    double sc = ldexp(1.0, -steps);
    for (size_t i = 0; i < 3 * N; ++i) us[i] = v[i] * sc;
    for (int k = 0; k < steps; ++k)
        or_compose(us + (size_t)k * 3 * N, us + (size_t)k * 3 * N, us + (size_t)(k + 1) * 3 * N,
                   D, H, W);
    const double *uM = us + (size_t)steps * 3 * N;
    or_warp(Im, D, H, W, uM, J, gJ);
    int rc = loss_and_grad(p, If, J, D, H, W, range, L, gv ? dJ : NULL);
    if (rc == OR_OK && gv) {
        for (int c = 0; c < 3; ++c)
            for (size_t i = 0; i < N; ++i) g[(size_t)c * N + i] = dJ[i] * gJ[(size_t)c * N + i];
        for (int k = steps - 1; k >= 0; --k) {
            svf_square_adjoint(us + (size_t)k * 3 * N, g, D, H, W, g2);
            memcpy(g, g2, 3 * N * sizeof(double));
        }
        for (size_t i = 0; i < 3 * N; ++i) gv[i] = g[i] * sc;
    }
    if (u_out) memcpy(u_out, uM, 3 * N * sizeof(double));
    free(us); free(J); free(gJ); free(dJ); free(g); free(g2);
    return rc;
}

int or_register_svf(const double *If, const double *Im, int D, int H, int W, const or_params *p,
                    int steps, double *v_out, double *u_out, double *final_loss) {
    if (D <= 0 || H <= 0 || W <= 0 || !p || p->n_levels < 1 || p->n_levels > 8 || steps < 0 ||
        steps > 16 || p->use_jac)
        return OR_EINVAL;
    int t = 0, pd = 0, ph = 0, pw = 0;
    double *v = NULL, *m = NULL, *nu = NULL;
    for (int l = 0; l < p->n_levels; ++l) {
        int s = p->scales[l];
        int d = or_level_size(D, s), h = or_level_size(H, s), w = or_level_size(W, s);
        size_t N = (size_t)d * h * w;
        double *fl = malloc(N * sizeof(double)), *ml = malloc(N * sizeof(double));
        double *nv = calloc(3 * N, sizeof(double)), *nm = calloc(3 * N, sizeof(double)),
               *nn = calloc(3 * N, sizeof(double));
        double *g = malloc(3 * N * sizeof(double)), *dir = malloc(3 * N * sizeof(double));
        if (!fl || !ml || !nv || !nm || !nn || !g || !dir) return OR_EINVAL;
        or_downsample(If, D, H, W, s, fl);
        or_downsample(Im, D, H, W, s, ml);
        double range[4];
        or_mi_range(fl, ml, N, range);
        if (l > 0) {
            or_upsample_field(v, pd, ph, pw, nv, d, h, w, 1);
            or_upsample_field(m, pd, ph, pw, nm, d, h, w, -1);
            or_upsample_field(nu, pd, ph, pw, nn, d, h, w, -2);
        }
        free(v); free(m); free(nu);
        v = nv; m = nm; nu = nn;
        pd = d; ph = h; pw = w;
        for (int it = 0; it < p->iters[l]; ++it) {
            double L;
            int rc = or_svf_loss_grad(fl, ml, d, h, w, p, steps, range, v, &L, g, NULL);
            if (rc != OR_OK) return rc;
            or_gauss_smooth(g, g, 3, d, h, w, p->sigma_grad);
            ++t;
            or_adam(g, m, nu, dir, 3 * N, t, p->beta1, p->beta2, p->adam_eps);
            or_step_scale(dir, dir, d, h, w, p->lr, p->c_lp);   /* dir <- -eps_t d */
            for (size_t i = 0; i < 3 * N; ++i) g[i] = v[i] + dir[i];
            or_gauss_smooth(g, v, 3, d, h, w, p->sigma_warp);
        }
        if (l == p->n_levels - 1) {
            or_svf_loss_grad(fl, ml, d, h, w, p, steps, range, v, final_loss, NULL, u_out);
            if (v_out) memcpy(v_out, v, 3 * N * sizeof(double));
        }
        free(fl); free(ml); free(g); free(dir);
    }
    free(v); free(m); free(nu);
    return OR_OK;
}

/* ------------------------------------------------------------- rigid stage
 * Rigid pre-registration (the rigid group among the transformation groups
 * the paper's framework offers before the affine and deformable stages,
 * section "Discussion": rigid -> affine -> diffeomorphism).  Reading R-rigid:
 * the motion is rigid in the voxel coordinates of the input grid about its
 * centre, y' = R y + tau with y = x - (n - 1) / 2; R = exp([w]x) by the
 * Rodrigues formula (w: axis times angle, radians); the translation is kept in
 * the normalised units of reading R-aff, t = S^-1 tau, S = diag((n_a - 1)/2)
 * of the input grid (1 on an axis of length 1).  On normalised coordinates
 * this is the affine map A = S^-1 R S, t, the same at every pyramid level.
 * rp = (w, t); identity start; plain Adam on the 6 parameters; the gradient
 * is the affine one pulled back exactly: dL/dt = dL/dt_aff and
 * dL/dw_k = sum_ij dL/dA_ij (s_j / s_i) dR_ij/dw_k. */

/* R = I + a K + b K^2 and dR/dw_k = c1 w_k K + a E_k + c2 w_k K^2 + b (E_k K + K E_k)
 * (K = [w]x, E_k = [e_k]x, a = sin th / th, b = (1 - cos th) / th^2,
 * c1 = a'(th) / th, c2 = b'(th) / th; power series below th = 1e-2). */
void or_rodrigues(const double *w, double *R, double *dR /* 3 x 9, nullable */) {
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2], th = sqrt(th2);
    double a, b, c1, c2;
    if (th < 1e-2) {
        a = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        b = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        c1 = -1.0 / 3.0 + th2 / 30.0 - th2 * th2 / 840.0;
        c2 = -1.0 / 12.0 + th2 / 180.0 - th2 * th2 / 6720.0;
    } else {
        double sn = sin(th), cs = cos(th);
        a = sn / th;
        b = (1.0 - cs) / th2;
        c1 = (th * cs - sn) / (th2 * th);
        c2 = (th * sn - 2.0 * (1.0 - cs)) / (th2 * th2);
    }
    double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0}, K2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += K[3 * i + k] * K[3 * k + j];
            K2[3 * i + j] = acc;
        }
    for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + a * K[i] + b * K2[i];
    if (!dR) return;
    for (int k = 0; k < 3; ++k) {
        double e[3] = {0.0, 0.0, 0.0}, E[9], EK[9], KE[9];
        e[k] = 1.0;
        double Et[9] = {0.0, -e[2], e[1], e[2], 0.0, -e[0], -e[1], e[0], 0.0};
        memcpy(E, Et, sizeof(E));
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s1 = 0.0, s2 = 0.0;
                for (int q = 0; q < 3; ++q) {
                    s1 += E[3 * i + q] * K[3 * q + j];
                    s2 += K[3 * i + q] * E[3 * q + j];
                }
                EK[3 * i + j] = s1;
                KE[3 * i + j] = s2;
            }
        for (int i = 0; i < 9; ++i)
            dR[9 * k + i] = c1 * w[k] * K[i] + a * E[i] + c2 * w[k] * K2[i] + b * (EK[i] + KE[i]);
    }
}

static void rigid_scales(int D, int H, int W, double s[3]) {
    const int n[3] = {D, H, W};
    for (int a = 0; a < 3; ++a) s[a] = n[a] > 1 ? 0.5 * (n[a] - 1) : 1.0;
}

/* theta (reading R-aff) of the rigid parameters rp on a D x H x W input grid */
int or_rigid_theta(const double *rp, int D, int H, int W, double *theta) {
    if (D <= 0 || H <= 0 || W <= 0) return OR_EINVAL;
    double R[9], s[3];
    or_rodrigues(rp, R, NULL);
    rigid_scales(D, H, W, s);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) theta[3 * i + j] = R[3 * i + j] * s[j] / s[i];
        theta[9 + i] = rp[3 + i];
    }
    return OR_OK;
}

/* the 6-parameter gradient from the affine one (gaff: 12) */
static void rigid_pullback(const double *rp, const double s[3], const double *gaff, double *g) {
    double R[9], dR[27];
    or_rodrigues(rp, R, dR);
    for (int k = 0; k < 3; ++k) {
        double acc = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) acc += gaff[3 * i + j] * s[j] / s[i] * dR[9 * k + 3 * i + j];
        g[k] = acc;
        g[3 + k] = gaff[9 + k];
    }
}

/* loss of level images (fl, ml) at rp (input grid D0 x H0 x W0) and its
 * 6-parameter gradient (nullable) */
int or_rigid_loss_grad(const double *If, const double *Im, int D, int H, int W, int D0, int H0,
                       int W0, const double *rp, int loss, int window, double cc_eps, double *L,
                       double *grad) {
    double theta[12], gaff[12], s[3];
    int rc = or_rigid_theta(rp, D0, H0, W0, theta);
    if (rc != OR_OK) return rc;
    rc = or_affine_loss_grad(If, Im, D, H, W, theta, loss, window, cc_eps, L, grad ? gaff : NULL);
    if (rc != OR_OK || !grad) return rc;
    rigid_scales(D0, H0, W0, s);
    rigid_pullback(rp, s, gaff, grad);
    return OR_OK;
}

int or_rigid_register(const double *If, const double *Im, int D, int H, int W,
                      const or_params *p, double *rp, double *final_loss) {
    if (D <= 0 || H <= 0 || W <= 0 || !p || p->n_levels < 1 || p->n_levels > 8) return OR_EINVAL;
    double m[6] = {0}, v[6] = {0}, g[6], dir[6];
    for (int k = 0; k < 6; ++k) rp[k] = 0.0;
    int t = 0;
    for (int l = 0; l < p->n_levels; ++l) {
        int s = p->scales[l];
        int d = or_level_size(D, s), h = or_level_size(H, s), w = or_level_size(W, s);
        size_t N = (size_t)d * h * w;
        double *fl = malloc(N * sizeof(double)), *ml = malloc(N * sizeof(double));
        if (!fl || !ml) return OR_EINVAL;
        or_downsample(If, D, H, W, s, fl);
        or_downsample(Im, D, H, W, s, ml);
        for (int it = 0; it < p->iters[l]; ++it) {
            double L;
            int rc = or_rigid_loss_grad(fl, ml, d, h, w, D, H, W, rp, p->loss, p->window,
                                        p->cc_eps, &L, g);
            if (rc != OR_OK) return rc;
            ++t;
            or_adam(g, m, v, dir, 6, t, p->beta1, p->beta2, p->adam_eps);
            for (int k = 0; k < 6; ++k) rp[k] -= p->lr * dir[k];
        }
        if (l == p->n_levels - 1)
            or_rigid_loss_grad(fl, ml, d, h, w, D, H, W, rp, p->loss, p->window, p->cc_eps,
                               final_loss, NULL);
        free(fl); free(ml);
    }
    return OR_OK;
}

/* ------------------------------------------------------------ inverse map
 * Post-hoc inverse of phi = id + u (section "Alternative formulations for
 * Eulerian differential"): psi = id + w minimises
 *   E(w) = (1/N) sum_x |psi(phi(x)) - x|^2 + |phi(psi(x)) - x|^2
 *        = (1/N) sum_x |u(x) + w(x + u(x))|^2 + |w(x) + u(x + w(x))|^2
 * over a multi-scale schedule with Algorithm 1's update (reading R-inv).
 * The gradient is the exact Gateaux derivative: the first term scatters
 * 2 A(x) / N through the trilinear weights of w at x + u(x); the second gives
 * 2 (I + grad u(x + w(x)))^T B(x) / N with the interpolant's derivative. */
int or_inverse_energy_grad(const double *u, const double *w, int D, int H, int W, double *E,
                           double *g) {
    if (D <= 0 || H <= 0 || W <= 0) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
    if (g) memset(g, 0, 3 * N * sizeof(double));
    double e = 0.0;
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                size_t i = IDX(z, y, x);
                double pa[3] = {z + u[i], y + u[N + i], x + u[2 * N + i]};
                double pb[3] = {z + w[i], y + w[N + i], x + w[2 * N + i]};
                double A[3], B[3], G[3][3];
                for (int c = 0; c < 3; ++c) {
                    A[c] = u[(size_t)c * N + i] +
                           trilinear(w + (size_t)c * N, D, H, W, pa[0], pa[1], pa[2], NULL);
                    B[c] = w[(size_t)c * N + i] +
                           trilinear(u + (size_t)c * N, D, H, W, pb[0], pb[1], pb[2], G[c]);
                    e += A[c] * A[c] + B[c] * B[c];
                }
                if (!g) continue;
                for (int a = 0; a < 3; ++a) {       /* (I + grad u)^T B */
                    double s = B[a];
                    for (int j = 0; j < 3; ++j) s += G[j][a] * B[j];
                    g[(size_t)a * N + i] += 2.0 * s / (double)N;
                }
                /* scatter of 2 A / N to the corners of x + u(x) */
                if (isnan(pa[0]) || isnan(pa[1]) || isnan(pa[2])) continue;
                if (pa[0] < -1.0 || pa[1] < -1.0 || pa[2] < -1.0 || pa[0] >= (double)D ||
                    pa[1] >= (double)H || pa[2] >= (double)W)
                    continue;
                double fz = floor(pa[0]), fy = floor(pa[1]), fx = floor(pa[2]);
                int z0 = (int)fz, y0 = (int)fy, x0 = (int)fx;
                double tz = pa[0] - fz, ty = pa[1] - fy, tx = pa[2] - fx;
                double wz[2] = {1.0 - tz, tz}, wy[2] = {1.0 - ty, ty}, wx[2] = {1.0 - tx, tx};
                for (int a2 = 0; a2 < 2; ++a2)
                    for (int b2 = 0; b2 < 2; ++b2)
                        for (int e2 = 0; e2 < 2; ++e2) {
                            int zz = z0 + a2, yy = y0 + b2, xx = x0 + e2;
                            if (!in_grid(zz, yy, xx, D, H, W)) continue;
                            double wt = wz[a2] * wy[b2] * wx[e2];
                            for (int c = 0; c < 3; ++c)
                                g[(size_t)c * N + IDX(zz, yy, xx)] += 2.0 * A[c] * wt / (double)N;
                        }
            }
    if (E) *E = e / (double)N;
    return OR_OK;
}

int or_inverse(const double *u, int D, int H, int W, const or_params *p, double *w_out,
               double *final_energy) {
    if (D <= 0 || H <= 0 || W <= 0 || !p || p->n_levels < 1 || p->n_levels > 8) return OR_EINVAL;
    int t = 0, pd = 0, ph = 0, pw = 0;
    double *w = NULL, *m = NULL, *v = NULL;
    for (int l = 0; l < p->n_levels; ++l) {
        int s = p->scales[l];
        int d = or_level_size(D, s), h = or_level_size(H, s), wd = or_level_size(W, s);
        size_t N = (size_t)d * h * wd;
        double *ul = malloc(3 * N * sizeof(double));
        double *nw = calloc(3 * N, sizeof(double)), *nm = calloc(3 * N, sizeof(double)),
               *nv = calloc(3 * N, sizeof(double));
        double *g = malloc(3 * N * sizeof(double)), *dir = malloc(3 * N * sizeof(double)),
               *tmp = malloc(3 * N * sizeof(double));
        if (!ul || !nw || !nm || !nv || !g || !dir || !tmp) return OR_EINVAL;
        or_upsample_field(u, D, H, W, ul, d, h, wd, 1);   /* phi at this level */
        if (l > 0) {
            or_upsample_field(w, pd, ph, pw, nw, d, h, wd, 1);
            or_upsample_field(m, pd, ph, pw, nm, d, h, wd, -1);
            or_upsample_field(v, pd, ph, pw, nv, d, h, wd, -2);
        }
        free(w); free(m); free(v);
        w = nw; m = nm; v = nv;
        pd = d; ph = h; pw = wd;
        for (int it = 0; it < p->iters[l]; ++it) {
            or_inverse_energy_grad(ul, w, d, h, wd, NULL, g);
            or_gauss_smooth(g, g, 3, d, h, wd, p->sigma_grad);
            ++t;
            or_adam(g, m, v, dir, 3 * N, t, p->beta1, p->beta2, p->adam_eps);
            or_step_scale(dir, dir, d, h, wd, p->lr, p->c_lp);
            or_compose(w, dir, tmp, d, h, wd);
            or_gauss_smooth(tmp, w, 3, d, h, wd, p->sigma_warp);
        }
        if (l == p->n_levels - 1) {
            or_inverse_energy_grad(ul, w, d, h, wd, final_energy, NULL);
            memcpy(w_out, w, 3 * N * sizeof(double));
        }
        free(ul); free(g); free(dir); free(tmp);
    }
    free(w); free(m); free(v);
    return OR_OK;
}


/* ------------------------------------------------------- symmetric objective
 * Symmetric registration (section "Alternative formulations for Eulerian
 * differential": the symmetric objective gets its final map as
 * phi = phi_M o phi_F^-1, with phi_F^-1 from the post-hoc inverse).
 * Reading R-sym: two maps phi_F = id + u_F and phi_M = id + u_M, both from
 * the identity, minimise L(I_f o phi_F, I_m o phi_M), the loss of the two
 * warped images (LNCC or MSE, symmetric in its arguments).  Each iteration
 * takes Algorithm 1's update of each map from its own Gateaux derivative,
 *   dL/dphi_F = dL/dJ_F grad I_f(phi_F),  dL/dphi_M = dL/dJ_M grad I_m(phi_M),
 * with its own Adam moments and step scale (one step counter); the level
 * hand-off treats both as or_register treats u.  On the last level w, the
 * inverse of u_F, comes from or_inverse (schedule p_inv, scales relative to
 * that grid, last scale 1), and u = w + u_M o (id + w) = phi_M o phi_F^-1 - id. */

/* L(I_f o phi_F, I_m o phi_M) and both derivatives (gF, gM nullable). */
int or_symmetric_loss_grad(const double *If, const double *Im, int D, int H, int W,
                           const or_params *p, const double *uF, const double *uM, double *L,
                           double *gF, double *gM) {
    if (D <= 0 || H <= 0 || W <= 0 || !p || (p->loss != 0 && p->loss != 1)) return OR_EINVAL;
    size_t N = (size_t)D * H * W;
    double *JF = malloc(N * sizeof(double)), *JM = malloc(N * sizeof(double));
    double *gIF = malloc(3 * N * sizeof(double)), *gIM = malloc(3 * N * sizeof(double));
    double *dF = malloc(N * sizeof(double)), *dM = malloc(N * sizeof(double));
    int rc = OR_EINVAL;
    if (!JF || !JM || !gIF || !gIM || !dF || !dM) goto done;
    or_warp(If, D, H, W, uF, JF, gIF);
    or_warp(Im, D, H, W, uM, JM, gIM);
    /* J_F takes the fixed role of the loss, J_M the warped one */
    if (p->loss == 0)
        rc = or_lncc(JF, JM, D, H, W, p->window, p->cc_eps, L, NULL, dM, dF);
    else
        rc = or_mse(JF, JM, D, H, W, L, dM, dF);
    if (rc != OR_OK) goto done;
    for (int c = 0; c < 3; ++c)
        for (size_t i = 0; i < N; ++i) {
            if (gF) gF[(size_t)c * N + i] = dF[i] * gIF[(size_t)c * N + i];
            if (gM) gM[(size_t)c * N + i] = dM[i] * gIM[(size_t)c * N + i];
        }
done:
    free(JF); free(JM); free(gIF); free(gIM); free(dF); free(dM);
    return rc;
}

/* Algorithm 1's update of one map from its derivative g (g is overwritten). */
static void sym_update(const or_params *p, double *g, double *u, double *m, double *v, int t,
                       int d, int h, int w, double *dir, double *tmp) {
    size_t N = (size_t)d * h * w;
    if (p->use_jac) {
        or_jac_direction(g, u, d, h, w, tmp);
        memcpy(g, tmp, 3 * N * sizeof(double));
    }
    or_gauss_smooth(g, g, 3, d, h, w, p->sigma_grad);
    or_adam(g, m, v, dir, 3 * N, t, p->beta1, p->beta2, p->adam_eps);
    or_step_scale(dir, dir, d, h, w, p->lr, p->c_lp);
    or_compose(u, dir, tmp, d, h, w);
    or_gauss_smooth(tmp, u, 3, d, h, w, p->sigma_warp);
}

int or_register_symmetric(const double *If, const double *Im, int D, int H, int W,
                          const or_params *p, const or_params *p_inv, double *u_out,
                          double *uF_out, double *uM_out, double *final_loss, double *mid_loss) {
    if (D <= 0 || H <= 0 || W <= 0 || !p || !p_inv || p->n_levels < 1 || p->n_levels > 8 ||
        (p->loss != 0 && p->loss != 1) ||
        p_inv->n_levels < 1 || p_inv->n_levels > 8 || p_inv->scales[p_inv->n_levels - 1] != 1)
        return OR_EINVAL;
    for (int l = 0; l < p->n_levels; ++l)
        if (p->scales[l] < 1 || p->iters[l] < 0) return OR_EINVAL;
    int t = 0, pd = 0, ph = 0, pw = 0;
    double *u[2] = {NULL, NULL}, *m[2] = {NULL, NULL}, *v[2] = {NULL, NULL};
    for (int l = 0; l < p->n_levels; ++l) {
        int s = p->scales[l];
        int d = or_level_size(D, s), h = or_level_size(H, s), w = or_level_size(W, s);
        size_t N = (size_t)d * h * w;
        double *fl = malloc(N * sizeof(double)), *ml = malloc(N * sizeof(double));
        double *gF = malloc(3 * N * sizeof(double)), *gM = malloc(3 * N * sizeof(double));
        double *dir = malloc(3 * N * sizeof(double)), *tmp = malloc(3 * N * sizeof(double));
        if (!fl || !ml || !gF || !gM || !dir || !tmp) return OR_EINVAL;
        or_downsample(If, D, H, W, s, fl);
        or_downsample(Im, D, H, W, s, ml);
        for (int k = 0; k < 2; ++k) {   /* k = 0: phi_F, k = 1: phi_M */
            double *nu = calloc(3 * N, sizeof(double)), *nm = calloc(3 * N, sizeof(double)),
                   *nv = calloc(3 * N, sizeof(double));
            if (!nu || !nm || !nv) return OR_EINVAL;
            if (l > 0) {
                or_upsample_field(u[k], pd, ph, pw, nu, d, h, w, 1);
                or_upsample_field(m[k], pd, ph, pw, nm, d, h, w, -1);
                or_upsample_field(v[k], pd, ph, pw, nv, d, h, w, -2);
            }
            free(u[k]); free(m[k]); free(v[k]);
            u[k] = nu; m[k] = nm; v[k] = nv;
        }
        pd = d; ph = h; pw = w;
        for (int it = 0; it < p->iters[l]; ++it) {
            double L;
            or_symmetric_loss_grad(fl, ml, d, h, w, p, u[0], u[1], &L, gF, gM);
            ++t;
            sym_update(p, gF, u[0], m[0], v[0], t, d, h, w, dir, tmp);
            sym_update(p, gM, u[1], m[1], v[1], t, d, h, w, dir, tmp);
        }
        if (l == p->n_levels - 1) {
            double L, *winv = malloc(3 * N * sizeof(double)), *J = malloc(N * sizeof(double));
            if (!winv || !J) return OR_EINVAL;
            if (mid_loss) {
                or_symmetric_loss_grad(fl, ml, d, h, w, p, u[0], u[1], &L, NULL, NULL);
                *mid_loss = L;
            }
            or_inverse(u[0], d, h, w, p_inv, winv, NULL);
            or_compose(u[1], winv, u_out, d, h, w);      /* phi_M o phi_F^-1 */
            or_warp(ml, d, h, w, u_out, J, NULL);
            if (p->loss == 0)
                or_lncc(fl, J, d, h, w, p->window, p->cc_eps, &L, NULL, NULL, NULL);
            else
                or_mse(fl, J, d, h, w, &L, NULL, NULL);
            *final_loss = L;
            if (uF_out) memcpy(uF_out, u[0], 3 * N * sizeof(double));
            if (uM_out) memcpy(uM_out, u[1], 3 * N * sizeof(double));
            free(winv); free(J);
        }
        free(fl); free(ml); free(gF); free(gM); free(dir); free(tmp);
    }
    for (int k = 0; k < 2; ++k) { free(u[k]); free(m[k]); free(v[k]); }
    return OR_OK;
}
