"""End-to-end parity of fa_register with the oracle's Algorithm 1 on the
32^3 blobs workload (final LNCC within 1e-3, mean displacement difference
below 0.05 voxel), plus edge cases and device status reporting."""
import numpy as np
import pytest
import torch

from paper_2404_01249_gb300 import synth

pytestmark = pytest.mark.gpu

C1 = dict(scales=(2, 1), iters=(50, 25), lr=0.5, sigma_grad=1.0, sigma_warp=0.5, window=5)


@pytest.fixture(scope="module")
def fa():
    from paper_2404_01249_gb300 import build, fa
    build.build()
    assert torch.cuda.is_available()
    fa.load()
    return fa


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def mean_disp_diff(u, ur):
    d = u.detach().cpu().double().numpy() - ur
    return float(np.sqrt((d ** 2).sum(0)).mean())


@pytest.fixture(scope="module")
def c1_oracle(orc):
    f, m, _ = synth.blobs_pair()
    r = orc.register(f, m, list(C1["scales"]), list(C1["iters"]), lr=0.5, sigma_grad=1.0,
                     sigma_warp=0.5, window=5, cc_eps=float(np.float32(1e-5)),
                     beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)),
                     adam_eps=float(np.float32(1e-8)))
    return f, m, r


@pytest.mark.parametrize("mode", ["plain"])
def test_c1_matches_oracle(fa, c1_oracle, mode):
    f, m, ref = c1_oracle
    out = fa.fa_register(cuda(f), cuda(m), fa.RegParams(mode=mode, **C1))
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    assert mean_disp_diff(out["u"], ref["u"]) < 0.05


def test_zero_iterations_is_identity(fa, orc):
    f, m, _ = synth.blobs_pair(shape=(12, 14, 16), sigma=2.0)
    out = fa.fa_register(cuda(f), cuda(m), fa.RegParams(scales=(2, 1), iters=(0, 0), mode="plain"))
    assert float(out["u"].abs().max()) == 0.0
    ref = orc.lncc(f, m, 5, np.float32(1e-5), want_dJ=False)["loss"]
    assert abs(out["final_loss"] - ref) < 1e-5


def test_mse_single_level(fa, orc):
    f, m, _ = synth.blobs_pair(shape=(16, 16, 16), sigma=2.0, max_disp=1.0)
    out = fa.fa_register(cuda(f), cuda(m), fa.RegParams(scales=(1,), iters=(30,), loss="mse",
                                                         mode="plain"))
    ref = orc.register(f, m, [1], [30], loss="mse", cc_eps=0.0, beta1=float(np.float32(0.9)),
                       beta2=float(np.float32(0.999)), adam_eps=float(np.float32(1e-8)))
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3 * max(1.0, abs(ref["final_loss"]))
    assert mean_disp_diff(out["u"], ref["u"]) < 0.05


def test_nonfinite_input_is_reported(fa):
    f, m, _ = synth.blobs_pair(shape=(8, 8, 8), sigma=2.0)
    m[3, 3, 3] = np.nan
    with pytest.raises(fa.FAError) as e:
        fa.fa_register(cuda(f), cuda(m), fa.RegParams(scales=(1,), iters=(3,), mode="plain"))
    assert e.value.status == 5


def test_tiny_and_degenerate_grids(fa, orc):
    for shape in [(1, 1, 1), (1, 4, 9), (3, 2, 5)]:
        r = np.random.default_rng(9)
        f = r.random(shape).astype(np.float32)
        m = r.random(shape).astype(np.float32)
        p = fa.RegParams(scales=(2, 1), iters=(3, 2), mode="plain")
        out = fa.fa_register(cuda(f), cuda(m), p)
        ref = orc.register(f, m, [2, 1], [3, 2], cc_eps=float(np.float32(1e-5)),
                           beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)),
                           adam_eps=float(np.float32(1e-8)))
        assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
        assert mean_disp_diff(out["u"], ref["u"]) < 0.05
