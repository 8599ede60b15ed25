"""fa_register_batched: jobs (pairs of different grids x parameter sets) run
concurrently on forked streams and give exactly the results of one
fa_register call per job (the kernels are deterministic: window sums are
exact integers and reductions are order-independent)."""
import numpy as np
import pytest
import torch

from paper_2404_01249_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fa():
    from paper_2404_01249_gb300 import build, fa
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fa.load()
    return fa


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_batched_equals_one_call_per_job(fa):
    shapes = [(20, 24, 28), (17, 22, 26), (24, 20, 16)]
    pairs = [synth.voronoi_pair(shape=s, seed=500 + i) for i, s in enumerate(shapes)]
    fixed = [cuda(p[0]) for p in pairs]
    moving = [cuda(p[1]) for p in pairs]
    cfgs = [fa.RegParams(scales=(2, 1), iters=(12, 6)),
            fa.RegParams(scales=(2, 1), iters=(8, 8), lr=0.25, sigma_grad=2.0, window=3),
            fa.RegParams(scales=(1,), iters=(5,), loss="mse", sigma_warp=0.0)]
    out = fa.fa_register_batched(fixed, moving, cfgs, concurrency=4)
    assert len(out) == len(shapes) * len(cfgs)
    for i in range(len(shapes)):
        for c, p in enumerate(cfgs):
            r = out[i * len(cfgs) + c]
            ref = fa.fa_register(fixed[i], moving[i], p)
            assert r["status"] == 0
            assert torch.equal(r["u"], ref["u"]), (i, c)
            assert r["final_loss"] == ref["final_loss"], (i, c)


@pytest.mark.parametrize("concurrency", [1, 3, 32])
def test_batched_concurrency_does_not_change_results(fa, concurrency):
    f, m, _ = synth.blobs_pair(shape=(16, 18, 20), sigma=2.5)
    fixed, moving = [cuda(f), cuda(m)], [cuda(m), cuda(f)]
    cfgs = [fa.RegParams(scales=(2, 1), iters=(6, 4), lr=lr) for lr in (0.25, 0.5)]
    base = fa.fa_register_batched(fixed, moving, cfgs, concurrency=1)
    out = fa.fa_register_batched(fixed, moving, cfgs, concurrency=concurrency)
    for a, b in zip(base, out):
        assert torch.equal(a["u"], b["u"]) and a["final_loss"] == b["final_loss"]


def test_batched_reports_nonfinite_job(fa):
    f, m, _ = synth.blobs_pair(shape=(8, 8, 8), sigma=2.0)
    bad = m.copy()
    bad[3, 3, 3] = np.nan
    out = fa.fa_register_batched([cuda(f), cuda(f)], [cuda(m), cuda(bad)],
                                 [fa.RegParams(scales=(1,), iters=(3,))], concurrency=2)
    assert out[0]["status"] == 0
    assert out[1]["status"] & 1
