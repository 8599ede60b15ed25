"""The Lie-algebra ("exp") variant in the oracle (reading R-svfreg: phi =
exp(v) by scaling and squaring, grad_v L by the exact adjoint of the
squarings, additive update of v).  Pinned to FP64 central differences of the
loss in v, the no-squaring case (exp(v) = id + v: the gradient is the warp's
chain rule), zero iterations, and recovery of a known translation."""
import numpy as np
import pytest

from paper_2404_01249_gb300 import synth


@pytest.mark.parametrize("loss,steps", [("lncc", 3), ("mse", 4), ("lncc", 0), ("mi", 2)])
def test_gradient_matches_central_differences(orc, loss, steps):
    shape = (10, 11, 12)
    f, m, _ = synth.blobs_pair(shape=shape, sigma=2.0, seed=1010)
    v = synth.random_field(shape, 2.0, 1.2, seed=12).astype(np.float64)
    _, g, _ = orc.svf_loss_grad(f, m, v, steps, window=3, loss=loss, mi_bins=16)
    h = 1e-6
    rng = np.random.default_rng(2)
    for _ in range(10):
        c, a, b, d = (int(rng.integers(0, n)) for n in (3,) + shape)
        vp, vq = v.copy(), v.copy()
        vp[c, a, b, d] += h
        vq[c, a, b, d] -= h
        fd = (orc.svf_loss_grad(f, m, vp, steps, 3, loss, mi_bins=16, want_grad=False)[0] -
              orc.svf_loss_grad(f, m, vq, steps, 3, loss, mi_bins=16, want_grad=False)[0]) / (2 * h)
        assert abs(fd - g[c, a, b, d]) <= 1e-6 * np.abs(g).max() + 1e-14, (loss, steps)


def test_without_squarings_the_gradient_is_the_warp_chain_rule(orc):
    shape = (9, 10, 11)
    f, m, _ = synth.blobs_pair(shape=shape, sigma=2.0, seed=1011)
    v = synth.random_field(shape, 2.0, 1.0, seed=13).astype(np.float64)
    L, g, u = orc.svf_loss_grad(f, m, v, 0)
    J, gJ = orc.warp(m, v)
    r = orc.lncc(f, J, 5, 1e-5)
    assert np.array_equal(u, v) and L == r["loss"]
    assert np.abs(g - r["dJ"][None] * gJ).max() <= 1e-15 * max(1.0, np.abs(g).max())


def test_zero_iterations_is_the_identity(orc):
    f, m, _ = synth.blobs_pair(shape=(10, 11, 12), sigma=2.0)
    r = orc.register_svf(f, m, [2, 1], [0, 0], steps=5)
    assert not r["u"].any() and not r["v"].any()


def test_recovers_a_subvoxel_translation(orc):
    shape = (20, 22, 24)
    f, _, _ = synth.blobs_pair(shape=shape, sigma=3.0)
    t = np.array([0.4, -0.3, 0.5])
    m = orc.warp(f, np.broadcast_to(t[:, None, None, None], (3,) + shape).copy(), want_grad=False)
    r = orc.register_svf(f, m, [2, 1], [60, 40], steps=5, loss="mse")
    inner = (slice(None),) + (slice(5, -5),) * 3
    est = r["u"][inner].reshape(3, -1).mean(1)
    assert np.abs(est + t).max() < 0.1   # the map that undoes the shift
