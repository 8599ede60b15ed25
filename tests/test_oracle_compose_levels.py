"""Pins for the oracle's compositive update (phi <- phi o (id + delta)), the
pyramid (Algorithm 1 "downsample") and the level hand-off (trilinear
upsampling of phi, m and nu, section "Interpolation strategies")."""
import math

import numpy as np
import pytest
from scipy.ndimage import gaussian_filter, map_coordinates

from conftest import rng


def grid(shape):
    return np.stack(np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij"))


def jac_det(u):
    """det(I + grad u) by central differences (np.gradient), voxel units."""
    G = np.empty((3, 3) + u.shape[1:])
    for a in range(3):
        gr = np.gradient(u[a])
        for b in range(3):
            G[a, b] = gr[b] + (1.0 if a == b else 0.0)
    return np.linalg.det(np.moveaxis(G, (0, 1), (-2, -1)))


def test_compose_identities(orc):
    shape = (5, 6, 7)
    u = rng(40).standard_normal((3,) + shape)
    assert np.array_equal(orc.compose(u, np.zeros_like(u)), u)
    d = 0.7 * rng(41).standard_normal((3,) + shape)
    assert np.array_equal(orc.compose(np.zeros_like(u), d), d)


def test_compose_affine_fields_exact_in_interior(orc):
    shape = (9, 10, 11)
    x = grid(shape)
    A = 0.05 * rng(42).standard_normal((3, 3))
    b = np.array([0.3, -0.2, 0.1])
    C = 0.03 * rng(43).standard_normal((3, 3))
    e = np.array([-0.1, 0.25, 0.05])
    u = np.einsum("ab,b...->a...", A, x) + b[:, None, None, None]
    d = np.einsum("ab,b...->a...", C, x) + e[:, None, None, None]
    out = orc.compose(u, d)
    p = x + d
    exact = d + np.einsum("ab,b...->a...", A, p) + b[:, None, None, None]
    ok = np.all((p >= 0) & (np.floor(p) + 1 <= np.array(shape)[:, None, None, None] - 1), axis=0)
    assert ok.sum() > 100
    assert np.allclose(out[:, ok], exact[:, ok], atol=1e-12)


def test_compose_matches_scipy(orc):
    shape = (6, 7, 8)
    u = rng(44).standard_normal((3,) + shape)
    d = 1.5 * rng(45).standard_normal((3,) + shape)
    out = orc.compose(u, d)
    p = grid(shape) + d
    for c in range(3):
        ref = d[c] + map_coordinates(u[c], list(p), order=1, mode="grid-constant", cval=0.0)
        assert np.allclose(out[c], ref, atol=1e-12)


def test_compose_sign_side_cell_gives_the_oracle_value(orc):
    """For a step below one voxel on every axis, the trilinear sample may be
    taken on the cell between x and its neighbours on each component's sign
    side, with weights |delta_a| (the CUDA path's compose cell): the
    interpolant is continuous across cell faces, so this equals the oracle's
    floor-cell compose, including at the grid's faces (zero outside) and for
    components that are exactly zero."""
    shape = (6, 7, 9)
    u = rng(46).standard_normal((3,) + shape)
    d = rng(47).uniform(-0.999, 0.999, (3,) + shape)
    d[0, 2] = 0.0  # a plane of zero z components
    d[2, :, :, 4] = -0.0
    D, H, W = shape

    def at(c, z, y, x):
        return u[c, z, y, x] if (0 <= z < D and 0 <= y < H and 0 <= x < W) else 0.0

    out = np.empty_like(u)
    for z in range(D):
        for y in range(H):
            for x in range(W):
                dz, dy, dx = d[:, z, y, x]
                sz, sy, sx = (-1 if v < 0 else 1 for v in (dz, dy, dx))
                tz, ty, tx = abs(dz), abs(dy), abs(dx)
                for c in range(3):
                    v = 0.0
                    for a, wa in ((0, 1 - tz), (sz, tz)):
                        for b, wb in ((0, 1 - ty), (sy, ty)):
                            for e, we in ((0, 1 - tx), (sx, tx)):
                                v += wa * wb * we * at(c, z + a, y + b, x + e)
                    out[c, z, y, x] = d[c, z, y, x] + v
    assert np.allclose(out, orc.compose(u, d), rtol=0, atol=1e-13)


def test_small_step_keeps_jacobian_positive(orc):
    """Theorem (appendix): id + eps v is a diffeomorphism for eps < 1/LP(v);
    the step scaling keeps the update inside that bound, so composing a
    diffeomorphic u with the scaled step keeps det J > 0."""
    shape = (16, 16, 16)
    from paper_2404_01249_gb300 import synth
    u = synth.random_field(shape, 3.0, 1.5, 46).astype(np.float64)
    assert jac_det(u)[1:-1, 1:-1, 1:-1].min() > 0
    d = rng(47).standard_normal((3,) + shape)
    d = gaussian_filter(d, (0, 1, 1, 1))
    delta, _ = orc.step_scale(d, 0.5)
    out = orc.compose(u, delta)
    assert jac_det(out)[1:-1, 1:-1, 1:-1].min() > 0


def test_level_sizes(orc):
    assert orc.level_shape((160, 192, 224), 4) == (40, 48, 56)
    assert orc.level_shape((33, 7, 3), 4) == (8, 1, 1)
    assert orc.level_shape((5, 5, 5), 1) == (5, 5, 5)


def test_downsample_identity_at_scale_one(orc):
    I = rng(48).standard_normal((5, 6, 7))
    assert np.array_equal(orc.downsample(I, 1), I)


@pytest.mark.parametrize("s", [2, 4])
def test_downsample_matches_scipy(orc, s):
    shape = (17, 20, 23)
    I = rng(49).standard_normal(shape)
    out = orc.downsample(I, s)
    sig = 0.5 * s
    R = math.ceil(3 * sig)
    blur = gaussian_filter(I, sig, mode="constant", cval=0.0, truncate=R / sig)
    cs = [np.arange(m) * (n - 1) / (m - 1) for n, m in zip(shape, out.shape)]
    pts = np.meshgrid(*cs, indexing="ij")
    ref = map_coordinates(blur, pts, order=1, mode="grid-constant")
    assert out.shape == tuple(n // s for n in shape)
    assert np.allclose(out, ref, atol=1e-12)


def test_downsample_affine_image_in_interior(orc):
    shape = (33, 29, 41)
    x = grid(shape)
    a = np.array([0.5, -0.25, 1.5])
    I = np.einsum("a,a...->...", a, x) + 2.0
    s = 2
    out = orc.downsample(I, s)
    M = out.shape
    fine = [np.arange(m) * (n - 1) / (m - 1) for n, m in zip(shape, M)]
    pz, py, px = np.meshgrid(*fine, indexing="ij")
    exact = a[0] * pz + a[1] * py + a[2] * px + 2.0
    R = 3  # blur radius for sigma = 1: interior points see no padding
    ok = (pz >= R) & (pz <= shape[0] - 1 - R - 1) & (py >= R) & (py <= shape[1] - 1 - R - 1) & \
         (px >= R) & (px <= shape[2] - 1 - R - 1)
    assert ok.sum() > 100
    assert np.allclose(out[ok], exact[ok], atol=1e-11)


def test_upsample_affine_field_exact(orc):
    cshape, fshape = (5, 6, 7), (10, 12, 14)
    xc = grid(cshape)
    A = 0.1 * rng(50).standard_normal((3, 3))
    b = np.array([0.4, -0.3, 0.2])
    u = np.einsum("ab,b...->a...", A, xc) + b[:, None, None, None]
    s = np.array([(f - 1) / (c - 1) for c, f in zip(cshape, fshape)])
    out = orc.upsample_field(u, fshape, 1)
    xf = grid(fshape)
    xcf = xf / s[:, None, None, None]           # fine voxel -> coarse coordinate
    exact = (np.einsum("ab,b...->a...", A, xcf) + b[:, None, None, None]) * s[:, None, None, None]
    assert np.allclose(out, exact, atol=1e-12)


def _level_fields(shape, funcs, power):
    """Covector fields of one level from smooth functions F_a(p) of the
    normalised coordinate p in [-1, 1]^3 (align-corners): by the chain rule
    for u_norm,a = u_vox,a * 2 / (n_a - 1), a derivative with respect to the
    voxel displacement is F_a(p) * (2 / (n_a - 1)), a squared one
    F_a(p) * (2 / (n_a - 1))^2 (power 1 or 2)."""
    p = np.stack(np.meshgrid(*[np.linspace(-1.0, 1.0, n) for n in shape], indexing="ij"))
    return np.stack([funcs[a](p) * (2.0 / (shape[a] - 1)) ** power for a in range(3)])


def test_moment_handoff_commutes_with_adam(orc):
    """Reading R-up (section "Interpolation strategies", Algorithm 1's
    upsampling of phi and the optimiser state): m and nu are running
    statistics of dL/du, and the chain rule makes that derivative a covector
    (the fine-level gradient at a point shared by both grids is the coarse one
    divided by s_a, since u_fine = s_a u_coarse).  Handing off the moments is
    therefore right exactly when the handed-off state equals the state a
    fine-level Adam would hold after the same gradient history expressed at
    the fine level.  Run Adam T steps on both levels from zero with the two
    levels' chain-rule gradients of one smooth sequence, hand the coarse state
    off with or_upsample_field(-1) and (-2), and compare on the coincident
    grid points (where trilinear interpolation is exact); then one more step
    on both sides gives the same direction d.  The other readings (m * s_a,
    nu * s_a^2) and no scaling both fail the same check."""
    cshape, fshape = (5, 7, 9), (9, 13, 25)          # s_a = 2, 2, 3
    s = np.array([(f - 1) / (c - 1) for c, f in zip(cshape, fshape)])
    T = 6
    r = rng(61)

    def grad_funcs(k):
        a = r.standard_normal((3, 4))
        return [lambda p, q=a[c]: q[0] + q[1] * np.sin(1.3 * p[0] + q[2]) * np.cos(0.7 * p[1])
                + q[3] * p[2] * p[1] for c in range(3)]

    hist = [grad_funcs(k) for k in range(T + 1)]
    # eps = 0: with eps > 0 Adam is not scale-invariant, so the check would
    # test eps instead of the hand-off
    zc, zf = np.zeros((3,) + cshape), np.zeros((3,) + fshape)
    mc, vc, mf, vf = zc, zc, zf, zf
    for k in range(T):
        _, mc, vc = orc.adam(_level_fields(cshape, hist[k], 1), mc, vc, k + 1, eps=0.0)
        _, mf, vf = orc.adam(_level_fields(fshape, hist[k], 1), mf, vf, k + 1, eps=0.0)
    co = tuple(slice(0, None, int(sa)) for sa in s)   # fine points on the coarse grid
    assert all(len(range(n)[sl]) == c for n, sl, c in zip(fshape, co, cshape))
    m_up = orc.upsample_field(mc, fshape, -1)
    v_up = orc.upsample_field(vc, fshape, -2)
    for a in range(3):
        np.testing.assert_allclose(m_up[a][co], mf[a][co], rtol=1e-12,
                                   atol=1e-12 * np.abs(mf[a]).max())
        np.testing.assert_allclose(v_up[a][co], vf[a][co], rtol=1e-12)
    # the next step's direction is the same on both sides
    gf = _level_fields(fshape, hist[T], 1)
    d_up, _, _ = orc.adam(gf, m_up, v_up, T + 1, eps=0.0)
    d_ref, _, _ = orc.adam(gf, mf, vf, T + 1, eps=0.0)
    for a in range(3):
        np.testing.assert_allclose(d_up[a][co], d_ref[a][co], rtol=1e-10, atol=1e-12)
    # the alternatives: m * s_a, nu * s_a^2 (power +1 on both, then once more
    # s_a on nu), and no scaling (power +1 divided back out of the values)
    m_alt = orc.upsample_field(mc, fshape, 1)
    v_alt = orc.upsample_field(vc, fshape, 1) * s[:, None, None, None]
    m_raw = m_alt / s[:, None, None, None]
    v_raw = v_alt / s[:, None, None, None] ** 2
    for mm, vv in ((m_alt, v_alt), (m_raw, v_raw)):
        d_alt, _, _ = orc.adam(gf, mm, vv, T + 1, eps=0.0)
        err = max(np.abs(d_alt[a][co] - d_ref[a][co]).max() for a in range(3))
        assert err > 1e-2


def test_upsample_preserves_positive_jacobian(orc):
    """Section "Interpolation strategies": trilinear upsampling of a
    diffeomorphic warp does not introduce folds."""
    from paper_2404_01249_gb300 import synth
    cshape = (12, 12, 12)
    u = synth.random_field(cshape, 2.0, 1.2, 51).astype(np.float64)
    assert jac_det(u)[1:-1, 1:-1, 1:-1].min() > 0
    up = orc.upsample_field(u, (24, 24, 24), 1)
    assert jac_det(up)[1:-1, 1:-1, 1:-1].min() > 0


def test_svf_exp_zero_and_affine_power(orc):
    """Scaling and squaring: exp(0) = id; for an affine velocity A x the M
    squarings give (I + A / 2^M)^(2^M) exactly wherever every intermediate
    point stays inside the grid (trilinear is exact on affine fields)."""
    shape = (16, 17, 18)
    assert np.array_equal(orc.svf_exp(np.zeros((3,) + shape), 5), np.zeros((3,) + shape))
    X = grid(shape)
    c = np.array([(n - 1) / 2 for n in shape])[:, None, None, None]
    A = 0.02 * rng(60).standard_normal((3, 3))
    v = np.einsum("ab,b...->a...", A, X - c)               # zero at the centre
    M = 4
    out = orc.svf_exp(v, M)
    P = np.linalg.matrix_power(np.eye(3) + A / 2 ** M, 2 ** M)
    exact = np.einsum("ab,b...->a...", P - np.eye(3), X - c)
    inner = (slice(4, -4),) * 3
    assert np.allclose(out[(slice(None),) + inner], exact[(slice(None),) + inner], atol=1e-12)


def test_svf_exp_constant_velocity_is_a_translation(orc):
    shape = (12, 12, 12)
    v = np.zeros((3,) + shape)
    v[0], v[1], v[2] = 0.4, -0.3, 0.25
    out = orc.svf_exp(v, 3)
    # the zero outside the grid reaches one voxel further in at every
    # squaring (each interpolation mixes in a neighbour)
    inner = (slice(4, -4),) * 3
    for a, val in enumerate((0.4, -0.3, 0.25)):
        assert np.allclose(out[a][inner], val, atol=1e-14)
