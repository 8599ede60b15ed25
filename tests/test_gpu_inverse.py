"""Post-hoc inverse of a displacement against the oracle (reading R-inv:
E(w) = mean |u + w o (id + u)|^2 + |w + u o (id + w)|^2, its exact Gateaux
gradient, and Algorithm 1's update over a multi-scale schedule)."""
import numpy as np
import pytest
import torch

from paper_2404_01249_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def fa():
    from paper_2404_01249_gb300 import build, fa
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fa.load()
    return fa


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("shape,amp", [((19, 23, 37), 1.5), ((9, 40, 33), 4.0), ((1, 7, 12), 0.8)])
def test_energy_gradient(fa, orc, shape, amp):
    u = synth.random_field(shape, 3.0, amp, seed=11).astype(np.float32)
    w = synth.random_field(shape, 3.0, 0.7 * amp, seed=12).astype(np.float32)
    E, g = fa.fa_inverse_energy_grad(cuda(u), cuda(w))
    Er, gr = orc.inverse_energy_grad(u, w)
    assert abs(float(E) - Er) <= TOL * max(Er, 1e-30)
    err = float(np.abs(g.cpu().double().numpy() - gr).max())
    assert err <= TOL * np.abs(gr).max(), err


def test_energy_gradient_at_zero(fa, orc):
    # w = 0: every B sample sits on the grid (the kink convention of the warp)
    shape = (12, 14, 17)
    u = synth.random_field(shape, 3.0, 2.0, seed=3).astype(np.float32)
    w = np.zeros_like(u)
    E, g = fa.fa_inverse_energy_grad(cuda(u), cuda(w))
    Er, gr = orc.inverse_energy_grad(u, w)
    assert abs(float(E) - Er) <= TOL * Er
    assert float(np.abs(g.cpu().double().numpy() - gr).max()) <= TOL * np.abs(gr).max()


def test_inverse_matches_oracle(fa, orc):
    shape = (20, 22, 26)
    u = synth.random_field(shape, 3.0, 1.5, seed=5).astype(np.float32)
    P = fa.RegParams(scales=(2, 1), iters=(30, 20))
    r = fa.fa_inverse(cuda(u), P)
    ref = orc.inverse(u, [2, 1], [30, 20])
    d = np.sqrt(((r["w"].cpu().double().numpy() - ref["w"]) ** 2).sum(0))
    assert d.mean() <= 0.01 and d.max() <= 0.05, (d.mean(), d.max())
    assert abs(r["final_energy"] - ref["final_energy"]) <= 1e-3 * max(ref["final_energy"], 1e-6)
    E0, _ = orc.inverse_energy_grad(u, np.zeros_like(u), False)
    assert r["final_energy"] < 0.1 * E0


def test_translation_inverse(fa):
    shape = (16, 17, 18)
    v = np.zeros((3,) + shape, np.float32)
    v[0], v[1], v[2] = 0.7, -0.4, 0.5
    r = fa.fa_inverse(cuda(v), fa.RegParams(scales=(2, 1), iters=(80, 60)))
    inner = (slice(None),) + (slice(4, -4),) * 3
    assert float((r["w"].cpu()[inner] + torch.from_numpy(v)[inner]).abs().max()) < 0.02


def test_deterministic_and_coarse_output(fa):
    shape = (18, 20, 21)
    u = cuda(synth.random_field(shape, 3.0, 1.5, seed=8))
    P = fa.RegParams(scales=(4, 2), iters=(10, 10))
    a = fa.fa_inverse(u, P)
    b = fa.fa_inverse(u, P)
    assert a["w"].shape == (3, 9, 10, 10)
    assert torch.equal(a["w"], b["w"]) and a["final_energy"] == b["final_energy"]


def test_invalid(fa):
    u = cuda(np.zeros((3, 8, 8, 8)))
    with pytest.raises(ValueError):
        fa.fa_inverse(u, fa.RegParams(scales=(), iters=()))
    with pytest.raises(fa.FAError):
        fa.fa_inverse(u, fa.RegParams(scales=(1,), iters=(1,), sigma_grad=50.0))
