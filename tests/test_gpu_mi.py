"""Mutual-information loss against the oracle (reading R-mi: cubic B-spline
Parzen windows on B bins, L = -MI, exact derivative), standalone and inside
whole registrations (both schedules)."""
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


@pytest.mark.parametrize("shape,bins", [((20, 24, 28), 32), ((17, 31, 22), 8),
                                        ((13, 19, 37), 64), ((1, 9, 40), 16)])
def test_mi_matches_oracle(fa, orc, shape, bins):
    f, m, _ = synth.blobs_pair(shape=shape, sigma=2.5, seed=1006)
    u = synth.random_field(shape, 3.0, 1.5, seed=31)
    J = orc.warp(m, u, want_grad=False).astype(np.float32)
    r = fa.fa_mi_fwd_bwd(cuda(f), cuda(J), bins)
    ref = orc.mi(f, J, bins)
    assert abs(float(r["loss"]) - ref["loss"]) <= TOL * max(1.0, abs(ref["loss"]))
    assert rel(r["dJ"], ref["dJ"]) < TOL


def test_mi_explicit_range_and_closed_form(fa):
    rng = np.random.default_rng(0)
    I = np.where(rng.random((9, 10, 11)) < 0.3, 1.7, 0.2).astype(np.float32)
    q = float((I == np.float32(1.7)).mean())
    r = fa.fa_mi_fwd_bwd(cuda(I), cuda(I), 16, rng=cuda([0.2, 1.7, 0.2, 1.7]))
    H = -q * np.log(q) - (1 - q) * np.log(1 - q)
    assert abs(-float(r["loss"]) - H) < 1e-6


def test_mi_is_deterministic(fa):
    f, m, _ = synth.voronoi_pair(shape=(40, 48, 56), seed=9)
    a = fa.fa_mi_fwd_bwd(cuda(f), cuda(m), 32)
    b = fa.fa_mi_fwd_bwd(cuda(f), cuda(m), 32)
    assert float(a["loss"]) == float(b["loss"]) and torch.equal(a["dJ"], b["dJ"])


@pytest.mark.parametrize("mode", ["fused", "plain"])
def test_mi_registration_matches_oracle(fa, orc, mode):
    f, m, _ = synth.blobs_pair(shape=(24, 26, 28), sigma=3.0)
    P = fa.RegParams(scales=(2, 1), iters=(30, 20), loss="mi", mi_bins=32, mode=mode)
    out = fa.fa_register(cuda(f), cuda(m), P)
    ref = orc.register(f, m, [2, 1], [30, 20], loss="mi", mi_bins=32)
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    d = out["u"].cpu().double().numpy() - ref["u"]
    assert float(np.sqrt((d ** 2).sum(0)).mean()) < 0.05


def test_mi_invalid_bins(fa):
    f = cuda(np.zeros((4, 4, 4)))
    with pytest.raises(fa.FAError):
        fa.fa_mi_fwd_bwd(f, f, 5)
    with pytest.raises(fa.FAError):
        fa.fa_register(f, f, fa.RegParams(scales=(1,), iters=(1,), loss="mi", mi_bins=65))
