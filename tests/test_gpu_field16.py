"""FP16 storage of the displacement u (fa_params.field_storage = FA_F16): every
stored update of u is rounded to FP16 (arithmetic stays FP32), u_out comes back
in FP32 holding those FP16 values, and the registration stays within the
end-to-end bar of the FP64 oracle (final LNCC within 1e-3, mean displacement
difference below 0.05 voxel) on the C1 pair, a brain-shaped coarse level and
grids of uneven width; lockstep waves may mix FP16 and FP32 u.  Calls outside
the fused LNCC path refuse FA_F16."""
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
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def mean_disp_diff(u, ur):
    d = u.detach().cpu().double().numpy() - ur
    return float(np.sqrt((d ** 2).sum(0)).mean())


def f32(x):
    return float(np.float32(x))


def oracle_run(orc, f, m, scales, iters):
    return orc.register(f, m, list(scales), list(iters), cc_eps=f32(1e-5), beta1=f32(0.9),
                        beta2=f32(0.999), adam_eps=f32(1e-8))


@pytest.mark.parametrize("case", ["c1", "uneven", "brain_level"])
def test_fp16_field_against_oracle(fa, orc, case):
    if case == "c1":
        f, m, _ = synth.blobs_pair()
        scales, iters = (2, 1), (50, 25)
    elif case == "uneven":
        f, m, _ = synth.voronoi_pair(shape=(17, 30, 41), seed=81)
        scales, iters = (2, 1), (20, 10)
    else:
        fb, mb, _ = synth.voronoi_pair(shape=(160, 192, 224), seed=1000)
        f = orc.downsample(fb, 4).astype(np.float32)
        m = orc.downsample(mb, 4).astype(np.float32)
        scales, iters = (1,), (200,)
    out = fa.fa_register(cuda(f), cuda(m), fa.RegParams(scales=scales, iters=iters, field="f16"))
    ref = oracle_run(orc, f, m, scales, iters)
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    assert mean_disp_diff(out["u"], ref["u"]) < 0.05
    u = out["u"]
    assert u.dtype == torch.float32
    assert torch.equal(u, u.half().float())  # the stored FP16 values, widened exactly


def test_fp16_field_close_to_fp32_and_deterministic(fa):
    f, m, _ = synth.voronoi_pair(shape=(40, 48, 56), seed=91)
    fx, mv = cuda(f), cuda(m)
    p16 = fa.RegParams(scales=(2, 1), iters=(40, 20), field="f16")
    a = fa.fa_register(fx, mv, fa.RegParams(scales=(2, 1), iters=(40, 20)))
    b = fa.fa_register(fx, mv, p16)
    assert abs(a["final_loss"] - b["final_loss"]) < 1e-3
    assert float((a["u"] - b["u"]).norm(dim=0).mean()) < 0.05
    ws = fa.workspace(fa.fa_register_workspace_size(f.shape, p16), "cuda")
    outs = [fa.fa_register(fx, mv, p16, ws=ws) for _ in range(3)]  # record, replay, replay
    for o in outs:
        assert torch.equal(o["u"], b["u"]) and o["final_loss"] == b["final_loss"]


@pytest.mark.parametrize("field", ["f32", "f16"])
def test_steps_above_a_voxel_against_oracle(fa, orc, field):
    """lr 2.5 allows steps of 1.25 voxels, so the fused compose samples u
    (FP32 or FP16) from global memory (sign-side cells below a voxel, floor
    cells above) instead of from its staged tile; against the oracle with the
    same bar."""
    f, m, _ = synth.voronoi_pair(shape=(24, 28, 36), seed=87)
    scales, iters = (2, 1), (20, 10)
    out = fa.fa_register(cuda(f), cuda(m),
                         fa.RegParams(scales=scales, iters=iters, lr=2.5, field=field))
    ref = orc.register(f, m, list(scales), list(iters), lr=2.5, cc_eps=f32(1e-5),
                       beta1=f32(0.9), beta2=f32(0.999), adam_eps=f32(1e-8))
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    assert mean_disp_diff(out["u"], ref["u"]) < 0.05
    if field == "f16":
        assert torch.equal(out["u"], out["u"].half().float())


@pytest.mark.parametrize("kw", [dict(mode="plain"), dict(mode="persistent"), dict(use_jac=True),
                                dict(loss="mse"), dict(sigma_warp=3.0)])
def test_fp16_field_refused_outside_the_fused_lncc_path(fa, kw):
    f, m, _ = synth.blobs_pair(shape=(12, 14, 16), sigma=2.0)
    with pytest.raises(fa.FAError) as e:  # refused by the workspace query or the call
        fa.fa_register(cuda(f), cuda(m), fa.RegParams(scales=(1,), iters=(2,), field="f16", **kw))
    assert e.value.status in (fa.FA_ERR_INVALID, fa.FA_ERR_UNSUPPORTED)
    assert "field_storage" in str(e.value)


def test_fp16_field_in_lockstep_equals_one_call_per_job(fa):
    """Jobs with FP16 and FP32 u (and BF16 moments, steps below and above a
    voxel) in one lockstep wave: each job's u and final loss are those of its
    own fa_register call, bit for bit (K4 runs once per u storage)."""
    shapes = [(20, 23, 29), (17, 30, 41)]
    pairs = [synth.voronoi_pair(shape=sh, seed=300 + i) for i, sh in enumerate(shapes)]
    fixed = [cuda(p[0]) for p in pairs]
    moving = [cuda(p[1]) for p in pairs]
    cfgs = [fa.RegParams(scales=(2, 1), iters=(8, 6), field="f16"),
            fa.RegParams(scales=(2, 1), iters=(8, 6)),
            fa.RegParams(scales=(2, 1), iters=(8, 6), field="f16", state="bf16", lr=2.5)]
    out = fa.fa_register_batched_lockstep(fixed, moving, cfgs)
    for i in range(len(shapes)):
        for c, p in enumerate(cfgs):
            r = out[i * len(cfgs) + c]
            ref = fa.fa_register(fixed[i], moving[i], p)
            assert r["status"] == 0
            assert torch.equal(r["u"], ref["u"]), (i, c)
            assert r["final_loss"] == ref["final_loss"], (i, c)
