"""Invariant pins for the oracle's whole registration (Algorithm 1).  The paper
prints no worked example of a registration, so these check properties the
method guarantees: the similarity improves, the map stays diffeomorphic
(theorem of the appendix "Limitations of Stationary Velocity Fields" plus
trilinear hand-off), and a known translation is recovered with the right sign
and size (phi = id - s undoes moving(x) = fixed(x + s))."""
import numpy as np
import pytest

from paper_2404_01249_gb300 import synth
from test_oracle_compose_levels import jac_det


def test_blobs_32_improves_and_stays_diffeomorphic(orc):
    f, m, _ = synth.blobs_pair()
    init = orc.lncc(f, m, 5, 1e-5, want_dJ=False)["loss"]
    r = orc.register(f, m, [2, 1], [50, 25], want_trace=True)
    assert r["u"].shape == (3, 32, 32, 32)
    assert r["final_loss"] < init - 0.05          # LNCC (= -loss) rises
    assert jac_det(r["u"]).min() > 0.0
    # trace holds one loss per iteration; the last coarse-level iterates
    # improve on the first
    tr = r["trace"]
    assert len(tr) == 75 and tr[49] < tr[0] and tr[-1] < tr[50]


def test_translation_recovered(orc):
    shift = np.array([0.6, -0.4, 0.8])
    f, m = synth.translated_blob_pair(shift=tuple(shift))
    r = orc.register(f, m, [2, 1], [80, 80])
    g = np.stack(np.gradient(f.astype(np.float64)))
    mag = np.sqrt((g ** 2).sum(0))
    sel = mag > 0.5 * mag.max()
    est = np.array([-r["u"][c][sel].mean() for c in range(3)])
    assert np.all(np.sign(est) == np.sign(shift))
    assert np.abs(est - shift).max() < 0.2, est


def test_mse_variant_runs_and_improves(orc):
    f, m, _ = synth.blobs_pair(shape=(16, 16, 16), sigma=2.0, max_disp=1.0)
    init = orc.mse(f, m)["loss"]
    r = orc.register(f, m, [1], [30], loss="mse")
    assert r["final_loss"] < 0.5 * init
    assert jac_det(r["u"]).min() > 0.0
