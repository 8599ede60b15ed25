"""Pins for the oracle's trilinear warp (section Preliminaries, pushforward
I(phi(x)); zero outside the grid) and its adjoint."""
import numpy as np
import pytest
from scipy.ndimage import map_coordinates

from conftest import rng


def _grid(shape):
    return np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")


def test_identity_is_exact(orc):
    I = rng(1).standard_normal((5, 6, 7))
    J, g = orc.warp(I, np.zeros((3, 5, 6, 7)))
    assert np.array_equal(J, I)


def test_integer_translation_is_exact_shift_with_zero_fill(orc):
    I = rng(2).standard_normal((6, 5, 7))
    u = np.zeros((3, 6, 5, 7))
    u[0], u[1], u[2] = 1.0, -2.0, 3.0
    J = orc.warp(I, u, want_grad=False)
    ref = np.zeros_like(I)
    # J(z, y, x) = I(z + 1, y - 2, x + 3), zero where that leaves the grid
    ref[:5, 2:, :4] = I[1:, :3, 3:]
    assert np.array_equal(J, ref)


def test_matches_scipy_grid_constant(orc):
    shape = (7, 8, 9)
    I = rng(3).standard_normal(shape)
    u = 1.7 * rng(4).standard_normal((3,) + shape)
    J = orc.warp(I, u, want_grad=False)
    z, y, x = _grid(shape)
    ref = map_coordinates(I, [z + u[0], y + u[1], x + u[2]], order=1, mode="grid-constant", cval=0.0)
    assert np.allclose(J, ref, rtol=0, atol=1e-12)


def test_affine_image_reproduced_with_exact_gradient(orc):
    shape = (6, 7, 8)
    z, y, x = _grid(shape)
    a = np.array([0.3, -1.25, 2.0])
    I = a[0] * z + a[1] * y + a[2] * x + 0.7
    u = 0.45 * rng(5).uniform(-1, 1, size=(3,) + shape)
    J, g = orc.warp(I, u)
    pz, py, px = z + u[0], y + u[1], x + u[2]
    inside = (pz >= 0) & (pz <= shape[0] - 1) & (py >= 0) & (py <= shape[1] - 1) & \
             (px >= 0) & (px <= shape[2] - 1)
    # the sample's whole cell must be in the grid for the interpolant to be affine
    inside &= (np.floor(pz) + 1 <= shape[0] - 1) & (np.floor(py) + 1 <= shape[1] - 1) & \
              (np.floor(px) + 1 <= shape[2] - 1)
    assert inside.sum() > 50
    exact = a[0] * pz + a[1] * py + a[2] * px + 0.7
    assert np.allclose(J[inside], exact[inside], atol=1e-12)
    for c in range(3):
        assert np.allclose(g[c][inside], a[c], atol=1e-12)


def test_gradient_matches_central_differences(orc):
    I = rng(6).standard_normal((5, 6, 7))
    r = rng(7)
    h = 1e-6
    for _ in range(40):
        p = r.uniform(-0.9, [4.9, 5.9, 6.9])
        # keep 10 h away from integers (the interpolant has kinks there)
        p = np.where(np.abs(p - np.round(p)) < 1e-3, p + 0.01, p)
        _, g = orc.sample(I, p)
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            fd = (orc.sample(I, p + e)[0] - orc.sample(I, p - e)[0]) / (2 * h)
            assert abs(fd - g[c]) <= 1e-8 * max(1.0, abs(g[c]))


def test_one_sided_derivative_at_integer(orc):
    I = np.zeros((3, 3, 3))
    I[1, 1, 1] = 1.0
    # at z = 1 exactly the cell is [1, 2): derivative is I[2] - I[1] = -1
    _, g = orc.sample(I, (1.0, 1.0, 1.0))
    assert g[0] == -1.0
    # at z = -1 exactly the cell is [-1, 0): derivative = I(0,...) - 0
    J = np.ones((2, 2, 2))
    _, g = orc.sample(J, (-1.0, 0.0, 0.0))
    assert g[0] == 1.0


def test_adjoint_dot_product(orc):
    shape = (6, 5, 7)
    r = rng(8)
    I = r.standard_normal(shape)
    y = r.standard_normal(shape)
    u = 1.3 * r.standard_normal((3,) + shape)
    J = orc.warp(I, u, want_grad=False)
    At = orc.warp_adjoint(y, u, shape)
    assert abs(np.vdot(J, y) - np.vdot(I, At)) <= 1e-11 * np.abs(J * y).sum()


def test_adjoint_is_derivative_of_linear_functional(orc):
    shape = (4, 5, 4)
    r = rng(9)
    I = r.standard_normal(shape)
    y = r.standard_normal(shape)
    u = 0.8 * r.standard_normal((3,) + shape)
    At = orc.warp_adjoint(y, u, shape)
    h = 1e-4
    for k in [(0, 0, 0), (2, 3, 1), (3, 4, 3), (1, 2, 2)]:
        e = np.zeros(shape)
        e[k] = h
        fd = (np.vdot(orc.warp(I + e, u, False), y) - np.vdot(orc.warp(I - e, u, False), y)) / (2 * h)
        assert abs(fd - At[k]) <= 1e-9
