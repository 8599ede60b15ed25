"""Mutual-information loss in the oracle (reading R-mi: cubic B-spline Parzen
windows on B bins, intensities mapped to [1, B - 2], L = -MI).  Pinned to a
closed form (a two-valued image against itself has MI equal to the binary
entropy of its mixing fraction), the zero-information case, invariance to
monotone affine intensity maps (both orientations), symmetry in the two
images, and FP64 central differences of the loss."""
import numpy as np
import pytest

from paper_2404_01249_gb300 import synth


def test_two_valued_image_against_itself_is_the_binary_entropy(orc):
    rng = np.random.default_rng(0)
    for q, B in ((0.3, 16), (0.5, 8), (0.1, 32)):
        I = np.where(rng.random((9, 10, 11)) < q, 1.7, 0.2)
        qq = float((I == 1.7).mean())
        L = orc.mi(I, I, B, rng=[0.2, 1.7, 0.2, 1.7])["loss"]
        H = -qq * np.log(qq) - (1 - qq) * np.log(1 - qq)
        assert abs(-L - H) < 1e-13


def test_constant_image_carries_no_information(orc):
    I = synth.blobs_pair(shape=(10, 11, 12), sigma=2.0)[0].astype(np.float64)
    J = np.full_like(I, 0.4)
    r = orc.mi(I, J, 32, rng=[I.min(), I.max(), 0.0, 1.0])
    assert abs(r["loss"]) < 1e-14 and np.abs(r["dJ"]).max() < 1e-14


@pytest.mark.parametrize("alpha,beta", [(2.5, -0.3), (-0.7, 1.1)])
def test_invariant_to_affine_intensity_maps(orc, alpha, beta):
    f, m, _ = synth.blobs_pair(shape=(12, 13, 14), sigma=2.0)
    f, m = f.astype(np.float64), m.astype(np.float64)
    r = orc.mi_range(f, m)
    lo, hi = alpha * r[2] + beta, alpha * r[3] + beta
    r2 = [r[0], r[1], min(lo, hi), max(lo, hi)]
    a = orc.mi(f, m, 24, rng=r)["loss"]
    b = orc.mi(f, alpha * m + beta, 24, rng=r2)["loss"]
    assert abs(a - b) < 1e-12


def test_symmetric_in_the_two_images(orc):
    f, m, _ = synth.blobs_pair(shape=(12, 13, 14), sigma=2.0)
    r = orc.mi_range(f, m)
    a = orc.mi(f, m, 32, rng=r)["loss"]
    b = orc.mi(m, f, 32, rng=[r[2], r[3], r[0], r[1]])["loss"]
    assert abs(a - b) < 1e-13


def test_gradient_matches_central_differences(orc):
    shape = (10, 11, 12)
    f, m, _ = synth.blobs_pair(shape=shape, sigma=2.0, seed=1005)
    f, m = f.astype(np.float64), m.astype(np.float64)
    r = orc.mi_range(f, m)
    dJ = orc.mi(f, m, 16, rng=r)["dJ"]
    h = 1e-6
    rng = np.random.default_rng(4)
    inside = np.argwhere((m > r[2] + 1e-3) & (m < r[3] - 1e-3))
    for k in rng.choice(len(inside), 12, replace=False):
        a, b, c = inside[k]
        mp, mq = m.copy(), m.copy()
        mp[a, b, c] += h
        mq[a, b, c] -= h
        fd = (orc.mi(f, mp, 16, rng=r, want_dJ=False)["loss"] -
              orc.mi(f, mq, 16, rng=r, want_dJ=False)["loss"]) / (2 * h)
        assert abs(fd - dJ[a, b, c]) <= 1e-6 * np.abs(dJ).max()


def test_mi_registration_raises_mutual_information(orc):
    f, m, _ = synth.blobs_pair(shape=(20, 22, 24), sigma=3.0)
    L0 = orc.mi(f, m, 32)["loss"]
    r = orc.register(f, m, [2, 1], [30, 20], loss="mi", mi_bins=32)
    assert r["final_loss"] < L0 - 0.05
