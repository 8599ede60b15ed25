"""Pins for the oracle's LNCC (squared local correlation over a w^3 box, zero
padding, fixed divisor w^3, L = -mean cc) and MSE, and their analytic
gradients (the Gateaux derivatives the Jacobian-free descent direction uses,
section "Jacobian-Free Eulerian Descent")."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from conftest import rng


def smooth_volume(shape, seed):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(rng(seed).standard_normal(shape), 1.0) + 0.5


def test_hand_worked_1x1x3_window3(orc):
    # D = H = 1, W = 3, w = 3 (n = 27).  Windows clipped by the grid keep the
    # divisor 27.  x = 0 sees voxels {0, 1}: S_I = 3, S_J = 3, S_II = 5,
    # S_JJ = 5, S_IJ = 4 -> cross = 11/3, varI = varJ = 14/3, cc = 121/196.
    # x = 1 sees all: S_I = 7, S_J = 6, S_II = 21, S_JJ = 14, S_IJ = 16 ->
    # cross = 130/9, varI = 518/27, varJ = 38/3, cc = 4225/4921.
    # x = 2 sees {1, 2}: S_I = 6, S_J = 4, S_II = 20, S_JJ = 10, S_IJ = 14 ->
    # cross = 118/9, varI = 56/3, varJ = 254/27, cc = 3481/3556.
    I = np.array([1.0, 2.0, 4.0]).reshape(1, 1, 3)
    J = np.array([2.0, 1.0, 3.0]).reshape(1, 1, 3)
    out = orc.lncc(I, J, 3, 0.0, want_cc=True)
    expect = [Fr(121, 196), Fr(4225, 4921), Fr(3481, 3556)]
    assert np.allclose(out["cc"].ravel(), [float(e) for e in expect], rtol=1e-14, atol=0)
    assert abs(out["loss"] + float(sum(expect) / 3)) < 1e-14


def test_box_sum_is_window_sum(orc):
    x = rng(11).standard_normal((5, 6, 7))
    for w in (1, 3, 5, 7):
        r = w // 2
        pad = np.pad(x, r)
        ref = np.zeros_like(x)
        for dz in range(w):
            for dy in range(w):
                for dx in range(w):
                    ref += pad[dz:dz + 5, dy:dy + 6, dx:dx + 7]
        assert np.allclose(orc.box_sum(x, w), ref, atol=1e-12)


def test_self_correlation_is_one_with_zero_gradient(orc):
    I = smooth_volume((8, 9, 10), 12)
    out = orc.lncc(I, I, 5, 0.0, want_cc=True, want_dI=True)
    assert np.allclose(out["cc"], 1.0, atol=1e-10)
    assert abs(out["loss"] + 1.0) < 1e-10
    N = I.size
    assert np.abs(out["dJ"]).max() * N < 1e-8
    assert np.abs(out["dI"]).max() * N < 1e-8


def test_range_and_affine_invariance(orc):
    shape = (9, 8, 10)
    I = smooth_volume(shape, 13)
    J = smooth_volume(shape, 14)
    cc = orc.lncc(I, J, 5, 0.0, want_cc=True)["cc"]
    assert cc.min() >= 0.0 and cc.max() <= 1.0 + 1e-12
    cc2 = orc.lncc(I, -2.5 * J + 4.0, 5, 0.0, want_cc=True)["cc"]
    full = (slice(2, -2),) * 3   # windows entirely inside the grid
    assert np.allclose(cc[full], cc2[full], rtol=1e-9, atol=1e-12)
    # swapping the images leaves cc unchanged (symmetry of the definition)
    cc3 = orc.lncc(J, I, 5, 0.0, want_cc=True)["cc"]
    assert np.allclose(cc, cc3, rtol=1e-12, atol=1e-14)


def test_locality_of_window(orc):
    shape = (9, 9, 9)
    I = smooth_volume(shape, 15)
    J = smooth_volume(shape, 16)
    base = orc.lncc(I, J, 5, 1e-5, want_cc=True)["cc"]
    J2 = J.copy()
    J2[4, 4, 7] += 1.0
    cc = orc.lncc(I, J2, 5, 1e-5, want_cc=True)["cc"]
    changed = np.argwhere(np.abs(cc - base) > 0)
    dist = np.abs(changed - np.array([4, 4, 7])).max(axis=1)
    assert dist.max() == 2          # exactly the voxels whose window holds it
    assert len(changed) == 5 * 5 * 4  # x clipped at W = 9


@pytest.mark.parametrize("cc_eps", [0.0, 1e-5, 1e-2])
def test_gradients_match_central_differences(orc, cc_eps):
    shape = (6, 7, 8)
    I = smooth_volume(shape, 17)
    J = smooth_volume(shape, 18)
    out = orc.lncc(I, J, 3, cc_eps, want_dI=True)
    h = 1e-4
    r = rng(19)
    for _ in range(12):
        k = tuple(int(r.integers(0, n)) for n in shape)
        for key, arr in (("dJ", J), ("dI", I)):
            e = np.zeros(shape)
            e[k] = h
            if key == "dJ":
                lp = orc.lncc(I, J + e, 3, cc_eps, want_dJ=False)["loss"]
                lm = orc.lncc(I, J - e, 3, cc_eps, want_dJ=False)["loss"]
            else:
                lp = orc.lncc(I + e, J, 3, cc_eps, want_dJ=False)["loss"]
                lm = orc.lncc(I - e, J, 3, cc_eps, want_dJ=False)["loss"]
            fd = (lp - lm) / (2 * h)
            an = out[key][k]
            # relative to the gradient's max norm: a voxel whose gradient
            # nearly cancels still carries the O(h^2) truncation of its
            # neighbours' curvature
            assert abs(fd - an) <= 1e-6 * np.abs(out[key]).max(), (key, k, fd, an)


def test_loss_gradient_wrt_displacement_matches_fd(orc):
    """dL/du(x) = dL/dJ(x) * grad I_m(x + u(x)), checked by central
    differences (h = 1e-4) at sample points away from cell faces."""
    shape = (6, 7, 8)
    If = smooth_volume(shape, 20)
    Im = smooth_volume(shape, 21)
    u = 0.6 * rng(22).uniform(-1, 1, (3,) + shape)
    # keep every sample point >= 0.02 from integer coordinates
    grid = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"))
    frac = (grid + u) - np.floor(grid + u)
    u = np.where(frac < 0.02, u + 0.03, u)
    u = np.where(frac > 0.98, u - 0.03, u)
    J, gJ = orc.warp(Im, u)
    out = orc.lncc(If, J, 5, 1e-5)
    g = out["dJ"][None] * gJ
    h = 1e-4
    r = rng(23)
    for _ in range(15):
        k = tuple(int(r.integers(0, n)) for n in shape)
        c = int(r.integers(0, 3))
        e = np.zeros_like(u)
        e[(c,) + k] = h
        lp = orc.lncc(If, orc.warp(Im, u + e, False), 5, 1e-5, want_dJ=False)["loss"]
        lm = orc.lncc(If, orc.warp(Im, u - e, False), 5, 1e-5, want_dJ=False)["loss"]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[(c,) + k]) <= 1e-6 * np.abs(g).max()


def test_mse_closed_form_and_gradient(orc):
    shape = (4, 5, 6)
    I = rng(24).standard_normal(shape)
    J = rng(25).standard_normal(shape)
    out = orc.mse(I, J)
    assert abs(out["loss"] - np.mean((J - I) ** 2)) < 1e-14
    h = 1e-5
    for k in [(0, 0, 0), (3, 4, 5), (2, 1, 3)]:
        e = np.zeros(shape)
        e[k] = h
        fd = (orc.mse(I, J + e)["loss"] - orc.mse(I, J - e)["loss"]) / (2 * h)
        assert abs(fd - out["dJ"][k]) <= 1e-8 * abs(out["dJ"][k]) + 1e-13
        fd = (orc.mse(I + e, J)["loss"] - orc.mse(I - e, J)["loss"]) / (2 * h)
        assert abs(fd - out["dI"][k]) <= 1e-8 * abs(out["dI"][k]) + 1e-13
