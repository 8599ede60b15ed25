"""The Lie-algebra (exp) registration variant against the oracle (reading
R-svfreg: exp(v) by scaling and squaring, the exact adjoint of the squarings,
additive update of v)."""
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


def rel(a, b):
    a = a.detach().cpu().double().numpy()
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


@pytest.mark.parametrize("shape,loss,steps", [((20, 24, 28), "lncc", 5), ((17, 31, 22), "mse", 3),
                                              ((13, 19, 37), "mi", 4), ((16, 18, 20), "lncc", 0)])
def test_loss_grad_matches_oracle(fa, orc, shape, loss, steps):
    f, m, _ = synth.blobs_pair(shape=shape, sigma=2.5, seed=1012)
    v = synth.random_field(shape, 3.0, 1.5, seed=41)
    P = fa.RegParams(scales=(1,), iters=(0,), loss=loss, mi_bins=16)
    L, g, u = fa.fa_svf_loss_grad(cuda(f), cuda(m), cuda(v), steps, P)
    Lr, gr, ur = orc.svf_loss_grad(f, m, v, steps, loss=loss, mi_bins=16)
    assert abs(float(L) - Lr) <= TOL * max(1.0, abs(Lr))
    assert rel(u, ur) < TOL
    assert rel(g, gr) < TOL


def test_registration_matches_oracle(fa, orc):
    f, m, _ = synth.blobs_pair(shape=(24, 26, 28), sigma=3.0)
    r = fa.fa_register_svf(cuda(f), cuda(m), fa.RegParams(scales=(2, 1), iters=(40, 20)), steps=5)
    ref = orc.register_svf(f, m, [2, 1], [40, 20], steps=5)
    assert abs(r["final_loss"] - ref["final_loss"]) < 1e-3
    for k in ("u", "v"):
        d = r[k].cpu().double().numpy() - ref[k]
        assert float(np.sqrt((d ** 2).sum(0)).mean()) < 0.05, k


def test_deterministic(fa):
    f, m, _ = synth.blobs_pair(shape=(16, 18, 20), sigma=2.5)
    P = fa.RegParams(scales=(2, 1), iters=(6, 4))
    a = fa.fa_register_svf(cuda(f), cuda(m), P, steps=4)
    b = fa.fa_register_svf(cuda(f), cuda(m), P, steps=4)
    assert torch.equal(a["u"], b["u"]) and a["final_loss"] == b["final_loss"]


def test_invalid(fa):
    f = cuda(np.zeros((8, 8, 8)))
    with pytest.raises(fa.FAError):
        fa.fa_register_svf(f, f, fa.RegParams(scales=(1,), iters=(1,)), steps=13)
    with pytest.raises(fa.FAError):
        fa.fa_register_svf(f, f, fa.RegParams(scales=(1,), iters=(1,), use_jac=True), steps=2)
