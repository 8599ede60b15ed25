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


def test_upsample_affine_field_exact_and_moment_scaling(orc):
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
    const = np.ones((3,) + cshape)
    m = orc.upsample_field(const, fshape, -1)
    v = orc.upsample_field(const, fshape, -2)
    for a in range(3):
        assert np.allclose(m[a], 1.0 / s[a], rtol=1e-15)
        assert np.allclose(v[a], 1.0 / s[a] ** 2, rtol=1e-15)


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
