"""Post-hoc inverse of a displacement in the oracle (reading R-inv: Algorithm
1's update on E(w) = mean |u + w o (id + u)|^2 + |w + u o (id + w)|^2, the
objective the paper states for phi^-1).  Pinned to the identity, FP64
central differences of E, the exact inverse of a translation, and the
energy decrease on a smooth random field."""
import numpy as np

from paper_2404_01249_gb300 import synth


def test_identity_inverts_to_identity(orc):
    u = np.zeros((3, 8, 9, 10))
    r = orc.inverse(u, [2, 1], [5, 5])
    assert np.array_equal(r["w"], u) and r["final_energy"] == 0.0


def test_energy_gradient_matches_central_differences(orc):
    shape = (12, 13, 14)
    u = synth.random_field(shape, 3.0, 1.5, seed=5).astype(np.float64)
    w = synth.random_field(shape, 3.0, 1.0, seed=6).astype(np.float64)
    _, g = orc.inverse_energy_grad(u, w)
    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(10):
        c, a, b, d = (int(rng.integers(0, n)) for n in (3,) + shape)
        wp, wm = w.copy(), w.copy()
        wp[c, a, b, d] += h
        wm[c, a, b, d] -= h
        fd = (orc.inverse_energy_grad(u, wp, False)[0] - orc.inverse_energy_grad(u, wm, False)[0]) / (2 * h)
        assert abs(fd - g[c, a, b, d]) <= 1e-5 * np.abs(g).max()


def test_translation_inverse(orc):
    shape = (16, 17, 18)
    v = np.zeros((3,) + shape)
    v[0], v[1], v[2] = 0.7, -0.4, 0.5
    r = orc.inverse(v, [2, 1], [80, 60])
    inner = (slice(None),) + (slice(4, -4),) * 3
    assert np.abs(r["w"][inner] + v[inner]).max() < 0.02


def test_energy_decreases_on_a_smooth_field(orc):
    shape = (16, 17, 18)
    u = synth.random_field(shape, 3.0, 1.5, seed=5).astype(np.float64)
    E0, _ = orc.inverse_energy_grad(u, np.zeros_like(u), False)
    r = orc.inverse(u, [2, 1], [60, 40])
    assert r["final_energy"] < 0.1 * E0
