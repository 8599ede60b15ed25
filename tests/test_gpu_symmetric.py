"""Symmetric registration against the oracle (reading R-sym: the loss of
I_f o phi_F and I_m o phi_M, Algorithm 1's update of each map, and the final
map phi_M o phi_F^-1 through the post-hoc inverse)."""
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


def mean_disp(a, b):
    d = a.cpu().double().numpy() - b
    return float(np.sqrt((d ** 2).sum(0)).mean())


@pytest.mark.parametrize("shape,loss,window", [((20, 24, 28), "lncc", 5),
                                               ((17, 31, 22), "lncc", 3),
                                               ((13, 19, 37), "mse", 5)])
def test_loss_grad_matches_oracle(fa, orc, shape, loss, window):
    f, m, _ = synth.blobs_pair(shape=shape, sigma=3.0, seed=1004)
    uF = synth.random_field(shape, 3.0, 1.5, seed=21)
    uM = synth.random_field(shape, 3.0, 1.2, seed=22)
    L, gF, gM = fa.fa_symmetric_loss_grad(cuda(f), cuda(m), cuda(uF), cuda(uM), window, loss)
    Lr, gFr, gMr = orc.symmetric_loss_grad(f, m, uF, uM, window, loss)
    assert abs(float(L) - Lr) <= TOL * abs(Lr)
    assert rel(gF, gFr) < TOL and rel(gM, gMr) < TOL


def test_registration_matches_oracle(fa, orc):
    f, m, _ = synth.blobs_pair(shape=(24, 26, 28), sigma=3.0)
    P = fa.RegParams(scales=(2, 1), iters=(40, 20))
    Pi = fa.RegParams(scales=(2, 1), iters=(30, 20))
    r = fa.fa_register_symmetric(cuda(f), cuda(m), P, Pi)
    ref = orc.register_symmetric(f, m, [2, 1], [40, 20], inv_scales=(2, 1), inv_iters=(30, 20))
    assert abs(r["final_loss"] - ref["final_loss"]) < 1e-3
    assert abs(r["final_mid_loss"] - ref["mid_loss"]) < 1e-3
    for k in ("uF", "uM", "u"):
        assert mean_disp(r[k], ref[k]) < 0.05, k


def test_mse_identical_images_stay_at_identity(fa):
    f, _, _ = synth.blobs_pair(shape=(12, 13, 14), sigma=2.5)
    P = fa.RegParams(scales=(2, 1), iters=(5, 5), loss="mse")
    r = fa.fa_register_symmetric(cuda(f), cuda(f), P, fa.RegParams(scales=(1,), iters=(5,)))
    assert not r["u"].any() and not r["uF"].any() and not r["uM"].any()
    assert r["final_loss"] == 0.0


def test_bf16_storage_equals_f32_on_rounded_images(fa):
    f, m, _ = synth.blobs_pair(shape=(16, 18, 20), sigma=2.5)
    fb, mb = cuda(f).bfloat16(), cuda(m).bfloat16()
    P16 = fa.RegParams(scales=(2, 1), iters=(6, 4))
    Pi = fa.RegParams(scales=(1,), iters=(10,))
    a = fa.fa_register_symmetric(fb, mb, P16, Pi)
    b = fa.fa_register_symmetric(fb.float(), mb.float(), fa.RegParams(scales=(2, 1), iters=(6, 4)), Pi)
    assert torch.equal(a["u"], b["u"]) and a["final_loss"] == b["final_loss"]


def test_deterministic(fa):
    f, m, _ = synth.blobs_pair(shape=(16, 18, 20), sigma=2.5)
    P = fa.RegParams(scales=(2, 1), iters=(6, 4))
    Pi = fa.RegParams(scales=(1,), iters=(10,))
    a = fa.fa_register_symmetric(cuda(f), cuda(m), P, Pi)
    b = fa.fa_register_symmetric(cuda(f), cuda(m), P, Pi)
    assert torch.equal(a["u"], b["u"]) and a["final_loss"] == b["final_loss"]


def test_invalid_inverse_schedule(fa):
    f = cuda(np.zeros((8, 8, 8)))
    with pytest.raises(fa.FAError):
        fa.fa_register_symmetric(f, f, fa.RegParams(scales=(1,), iters=(1,)),
                                 fa.RegParams(scales=(2,), iters=(1,)))
