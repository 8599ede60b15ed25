"""Symmetric registration in the oracle (reading R-sym: the loss of
I_f o phi_F and I_m o phi_M, Algorithm 1's update of each map, and the
final map phi_M o phi_F^-1 through the post-hoc inverse).  Pinned to FP64
central differences of the loss, the exact exchange symmetry of the
objective, the zero-gradient case, and the composition with a zero inverse."""
import numpy as np
import pytest

from paper_2404_01249_gb300 import synth


@pytest.mark.parametrize("loss", ["lncc", "mse"])
def test_gradients_match_central_differences(orc, loss):
    shape = (10, 11, 12)
    f, m, _ = synth.blobs_pair(shape=shape, sigma=2.0, seed=1003)
    uF = synth.random_field(shape, 2.0, 1.3, seed=7).astype(np.float64)
    uM = synth.random_field(shape, 2.0, 1.1, seed=8).astype(np.float64)
    _, gF, gM = orc.symmetric_loss_grad(f, m, uF, uM, window=3, loss=loss)
    h = 1e-6
    rng = np.random.default_rng(3)
    for which, u, g in (("F", uF, gF), ("M", uM, gM)):
        for _ in range(8):
            c, a, b, d = (int(rng.integers(0, n)) for n in (3,) + shape)
            up, um = u.copy(), u.copy()
            up[c, a, b, d] += h
            um[c, a, b, d] -= h
            if which == "F":
                Lp = orc.symmetric_loss_grad(f, m, up, uM, 3, loss, want_grad=False)[0]
                Lm = orc.symmetric_loss_grad(f, m, um, uM, 3, loss, want_grad=False)[0]
            else:
                Lp = orc.symmetric_loss_grad(f, m, uF, up, 3, loss, want_grad=False)[0]
                Lm = orc.symmetric_loss_grad(f, m, uF, um, 3, loss, want_grad=False)[0]
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[c, a, b, d]) <= 1e-6 * np.abs(g).max() + 1e-12, (which, loss)


@pytest.mark.parametrize("loss", ["lncc", "mse"])
def test_exchanging_the_images_exchanges_the_maps(orc, loss):
    f, m, _ = synth.blobs_pair(shape=(14, 15, 16), sigma=2.5, seed=1001)
    kw = dict(scales=[2, 1], iters=[6, 4], inv_scales=(1,), inv_iters=(5,), loss=loss)
    a = orc.register_symmetric(f, m, **kw)
    b = orc.register_symmetric(m, f, **kw)
    assert np.array_equal(a["uF"], b["uM"]) and np.array_equal(a["uM"], b["uF"])
    assert a["mid_loss"] == b["mid_loss"]


def test_identical_images_mse_stay_at_identity(orc):
    f, _, _ = synth.blobs_pair(shape=(12, 13, 14), sigma=2.5)
    r = orc.register_symmetric(f, f, [2, 1], [5, 5], loss="mse")
    assert not r["u"].any() and not r["uF"].any() and not r["uM"].any()
    assert r["final_loss"] == 0.0 and r["mid_loss"] == 0.0


def test_identical_images_lncc_move_both_maps_alike(orc):
    f, _, _ = synth.blobs_pair(shape=(12, 13, 14), sigma=2.5)
    r = orc.register_symmetric(f, f, [2, 1], [5, 5])
    assert np.array_equal(r["uF"], r["uM"])


def test_zero_inverse_composes_to_the_moving_map(orc):
    f, m, _ = synth.blobs_pair(shape=(14, 15, 16), sigma=2.5, seed=1002)
    r = orc.register_symmetric(f, m, [2, 1], [8, 4], inv_scales=(1,), inv_iters=(0,))
    assert np.array_equal(r["u"], r["uM"])
    J = orc.warp(m, r["uM"], want_grad=False)
    assert r["final_loss"] == orc.lncc(f, J, 5, 1e-5)["loss"]


def test_symmetric_registration_improves_the_loss(orc):
    f, m, _ = synth.blobs_pair(shape=(24, 26, 28), sigma=3.0)
    L0 = orc.lncc(f, m, 5, 1e-5)["loss"]
    r = orc.register_symmetric(f, m, [2, 1], [40, 20], inv_scales=(2, 1), inv_iters=(30, 20))
    assert r["mid_loss"] < L0 - 0.1 and r["final_loss"] < L0
