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


# ------------------------------------------------------------------ lockstep
# One launch per fused kernel per iteration covers every job of a wave; the
# per-job results must be those of one fa_register call per job, bit for bit
# (window sums are exact integers, every output's filters run in the same
# order whatever the tiling, and reductions are order-independent).

def _lockstep_jobs(fa, dtype=torch.float32):
    # widths: multiples of 4 and uneven ones (whose level rows the fused
    # schedule pads to a multiple of 4 floats)
    shapes = [(20, 24, 28), (17, 22, 26), (24, 20, 16), (9, 13, 35)]
    pairs = [synth.voronoi_pair(shape=s, seed=700 + i) for i, s in enumerate(shapes)]
    fixed = [cuda(p[0]).to(dtype) for p in pairs]
    moving = [cuda(p[1]).to(dtype) for p in pairs]
    cfgs = [fa.RegParams(scales=(2, 1), iters=(10, 6)),
            fa.RegParams(scales=(2, 1), iters=(10, 6), lr=0.25, sigma_grad=2.0, cc_eps=1e-4),
            fa.RegParams(scales=(2, 1), iters=(10, 6), lr=1.0, sigma_grad=0.5, sigma_warp=1.0),
            fa.RegParams(scales=(2, 1), iters=(10, 6), lr=2.5, sigma_warp=0.0)]
    return fixed, moving, cfgs


@pytest.mark.parametrize("graph", [True, False])
def test_lockstep_equals_one_call_per_job(fa, graph):
    fixed, moving, cfgs = _lockstep_jobs(fa)
    for c in cfgs:
        c.graph = graph
    out = fa.fa_register_batched_lockstep(fixed, moving, cfgs, jobs_per_wave=64)
    assert len(out) == len(fixed) * len(cfgs)
    for i in range(len(fixed)):
        for c, p in enumerate(cfgs):
            r = out[i * len(cfgs) + c]
            ref = fa.fa_register(fixed[i], moving[i], p)
            assert r["status"] == 0, (i, c)
            d = (r["u"] - ref["u"]).abs().max().item()
            assert torch.equal(r["u"], ref["u"]), (i, c, d)
            assert r["final_loss"] == ref["final_loss"], (i, c)


def test_lockstep_copy_variant_equals_tma_variant(fa):
    """The fused schedule gives a level of uneven width rows padded to a
    multiple of 4 floats, so its kernels take TMA tiles; a job of the
    persistent schedule keeps its small levels unpadded, and in a lockstep
    wave those run the per-thread copy (cp.async) variant of the batch
    kernels.  Both give the bits of one padded fa_register call per job."""
    import dataclasses
    fixed, moving, cfgs = _lockstep_jobs(fa)
    for mode in ("fused", "persistent"):
        mc = [dataclasses.replace(c, mode=mode) for c in cfgs]
        out = fa.fa_register_batched_lockstep(fixed, moving, mc, jobs_per_wave=64)
        for i in range(len(fixed)):
            for c, p in enumerate(cfgs):
                r = out[i * len(cfgs) + c]
                ref = fa.fa_register(fixed[i], moving[i], p)
                assert r["status"] == 0, (mode, i, c)
                assert torch.equal(r["u"], ref["u"]), (mode, i, c)
                assert r["final_loss"] == ref["final_loss"], (mode, i, c)


def test_lockstep_full_wave_of_64_jobs(fa):
    """64 jobs in one wave (the largest launch table, FP32 moments: three
    tensor maps per job in K3's parameters) over uneven grids; sampled jobs
    against one call each."""
    r = np.random.default_rng(77)
    shapes = [tuple(int(v) for v in r.integers(9, 23, size=3)) for _ in range(16)]
    pairs = [synth.voronoi_pair(shape=s, seed=900 + i) for i, s in enumerate(shapes)]
    fixed = [cuda(p[0]) for p in pairs]
    moving = [cuda(p[1]) for p in pairs]
    cfgs = [fa.RegParams(scales=(2, 1), iters=(4, 3), lr=lr, sigma_grad=sg)
            for lr in (0.25, 1.0) for sg in (0.5, 2.0)]
    out = fa.fa_register_batched_lockstep(fixed, moving, cfgs, jobs_per_wave=64)
    assert len(out) == 64
    for k in (0, 5, 22, 37, 50, 63):
        i, c = divmod(k, len(cfgs))
        ref = fa.fa_register(fixed[i], moving[i], cfgs[c])
        assert out[k]["status"] == 0, k
        assert torch.equal(out[k]["u"], ref["u"]), (k, shapes[i])
        assert out[k]["final_loss"] == ref["final_loss"], k


def test_lockstep_waves_and_replay_do_not_change_results(fa):
    fixed, moving, cfgs = _lockstep_jobs(fa)
    base = fa.fa_register_batched_lockstep(fixed, moving, cfgs, jobs_per_wave=64)
    for wave in (1, 3, 7):
        out = fa.fa_register_batched_lockstep(fixed, moving, cfgs, jobs_per_wave=wave)
        for a, b in zip(base, out):
            assert torch.equal(a["u"], b["u"]) and a["final_loss"] == b["final_loss"], wave
    again = fa.fa_register_batched_lockstep(fixed, moving, cfgs, jobs_per_wave=64)  # replay
    for a, b in zip(base, again):
        assert torch.equal(a["u"], b["u"]) and a["final_loss"] == b["final_loss"]


def test_lockstep_bf16_images_equal_one_call_per_job(fa):
    fixed, moving, cfgs = _lockstep_jobs(fa, torch.bfloat16)
    out = fa.fa_register_batched_lockstep(fixed[:2], moving[:2], cfgs[:2])
    for i in range(2):
        for c in range(2):
            ref = fa.fa_register(fixed[i], moving[i], cfgs[c])
            assert torch.equal(out[i * 2 + c]["u"], ref["u"]), (i, c)


def test_lockstep_reports_nonfinite_job(fa):
    f, m, _ = synth.blobs_pair(shape=(8, 8, 12), sigma=2.0)
    bad = m.copy()
    bad[3, 3, 3] = np.nan
    out = fa.fa_register_batched_lockstep([cuda(f), cuda(f)], [cuda(m), cuda(bad)],
                                          [fa.RegParams(scales=(1,), iters=(3,))])
    assert out[0]["status"] == 0
    assert out[1]["status"] & 1


def test_lockstep_brain_shaped_level_vs_oracle(fa, orc):
    """Two jobs of the uneven brain-like generator, each at scale 4 of its
    grid (200 iterations, two learning rates), in one lockstep call against
    the FP64 oracle: final LNCC within 1e-3 and mean displacement difference
    below 0.05 voxel."""
    f32 = lambda x: float(np.float32(x))
    fixed, moving, host = [], [], []
    for i, s in enumerate(synth.uneven_shapes(n=2, seed=3000)):
        f, m, _ = synth.voronoi_pair(shape=tuple(s), seed=3100 + i)
        fl = orc.downsample(f, 4).astype(np.float32)
        ml = orc.downsample(m, 4).astype(np.float32)
        host.append((fl, ml))
        fixed.append(cuda(fl))
        moving.append(cuda(ml))
    cfgs = [fa.RegParams(scales=(1,), iters=(200,), lr=lr) for lr in (0.5, 0.25)]
    out = fa.fa_register_batched_lockstep(fixed, moving, cfgs)
    for i, (fl, ml) in enumerate(host):
        for c, p in enumerate(cfgs):
            ref = orc.register(fl, ml, [1], [200], lr=f32(p.lr), cc_eps=f32(1e-5),
                               beta1=f32(0.9), beta2=f32(0.999), adam_eps=f32(1e-8))
            r = out[i * len(cfgs) + c]
            du = r["u"].cpu().double().numpy() - ref["u"]
            assert np.sqrt((du ** 2).sum(0)).mean() < 0.05, (i, c)
            assert abs(r["final_loss"] - ref["final_loss"]) < 1e-3, (i, c)
