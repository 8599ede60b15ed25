"""Adam moments stored in BF16 (fa_params.state_storage; FP16 too for the
per-op fa_radam_step), arithmetic in FP32.  Per kernel the bar is 2e-3 in the
normwise relative error against the FP64 oracle fed the same stored inputs,
and elementwise the format's unit roundoff; end to end it is the FP32 path's
bar: final LNCC within 1e-3 and mean displacement difference below 0.05
voxel.  Lockstep batches with BF16 moments equal one fa_register call per
job."""
import numpy as np
import pytest
import torch

from paper_2404_01249_gb300 import synth

pytestmark = pytest.mark.gpu

TOL16 = 2e-3
DT = {"bf16": torch.bfloat16, "f16": torch.float16}


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
    a = a.detach().cpu().double().numpy() if torch.is_tensor(a) else np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def f32(x):
    return float(np.float32(x))


def mean_disp_diff(u, ur):
    d = u.detach().cpu().double().numpy() - ur
    return float(np.sqrt((d ** 2).sum(0)).mean())


# unit roundoff of the 16-bit formats (8 and 11 significant bits)
U16 = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}


@pytest.mark.parametrize("state", ["bf16", "f16"])
def test_radam_step_with_16bit_moments(fa, orc, state):
    """a5-a7 with 16-bit m, nu.  The stored moments after the step are the
    oracle's FP64 update (from the same stored inputs) up to the format's
    rounding: elementwise within its unit roundoff (plus the FP32 bar), and
    within 2e-3 in the normwise relative error.  The direction, the step
    size and the composed field come from the FP32 values before rounding,
    so they meet the FP32 bar of 1e-5.  The FP16 moments are drawn inside
    FP16's normal range."""
    shape = (19, 37, 45)
    r = np.random.default_rng(15)
    u = synth.random_field(shape, 3.0, 6.0, 16)
    scale = 1e-3 if state == "bf16" else 1.0
    g = (r.standard_normal((3,) + shape) * scale).astype(np.float32)
    m0 = torch.from_numpy((r.standard_normal((3,) + shape) * scale).astype(np.float32))
    v0 = torch.from_numpy((0.5 + r.random((3,) + shape)) * scale ** 2).float()
    params = fa.RegParams(lr=0.5)
    for t in (1, 9):
        mt = m0.to(DT[state]).cuda()
        vt = v0.to(DT[state]).cuda()
        m_in = mt.float().cpu().double().numpy()  # the stored inputs, exactly
        v_in = vt.float().cpu().double().numpy()
        u_out, eps = fa.fa_radam_step(cuda(u), mt, vt, cuda(g), t, params)
        d, mr, vr = orc.adam(g, m_in, v_in, t, f32(0.9), f32(0.999), f32(1e-8))
        delta, er = orc.step_scale(d, 0.5, 2.0)
        ur = orc.compose(u, delta)
        assert mt.dtype == DT[state]
        for got, want in ((mt, mr), (vt, vr)):
            a = got.float().cpu().double().numpy()
            assert np.all(np.abs(a - want) <= U16[state] * np.abs(want) +
                          1e-5 * np.abs(want).max())
            assert np.linalg.norm(a - want) / np.linalg.norm(want) < TOL16
        assert abs(float(eps) - er) <= 1e-5 * er
        assert rel(u_out, ur) < 1e-5


@pytest.mark.parametrize("mode", ["fused", "plain"])
@pytest.mark.parametrize("state", ["bf16"])
def test_c1_with_16bit_moments_matches_oracle(fa, orc, mode, state):
    """The 32^3 blobs workload (two levels, so the 16-bit hand-off is
    exercised) against the oracle's FP64 Algorithm 1."""
    f, m, _ = synth.blobs_pair()
    p = fa.RegParams(scales=(2, 1), iters=(50, 25), mode=mode, state=state)
    out = fa.fa_register(cuda(f), cuda(m), p)
    ref = orc.register(f, m, [2, 1], [50, 25], cc_eps=f32(1e-5), beta1=f32(0.9),
                       beta2=f32(0.999), adam_eps=f32(1e-8))
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    assert mean_disp_diff(out["u"], ref["u"]) < 0.05


def test_brain_level_with_bf16_moments_matches_oracle(fa, orc):
    """The brain workload's coarse level (40x48x56, 200 iterations): the
    longest run of rounded moments in the tests."""
    f, m, _ = synth.voronoi_pair(shape=(160, 192, 224), seed=1000)
    fl = orc.downsample(f, 4).astype(np.float32)
    ml = orc.downsample(m, 4).astype(np.float32)
    out = fa.fa_register(cuda(fl), cuda(ml), fa.RegParams(scales=(1,), iters=(200,),
                                                          state="bf16"))
    ref = orc.register(fl, ml, [1], [200], cc_eps=f32(1e-5), beta1=f32(0.9), beta2=f32(0.999),
                       adam_eps=f32(1e-8))
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    assert mean_disp_diff(out["u"], ref["u"]) < 0.05


def test_lockstep_mixed_moment_storage_equals_one_call_per_job(fa):
    shapes = [(20, 24, 28), (17, 22, 26)]
    pairs = [synth.voronoi_pair(shape=s, seed=900 + i) for i, s in enumerate(shapes)]
    fixed = [cuda(p[0]).to(torch.bfloat16) for p in pairs]
    moving = [cuda(p[1]).to(torch.bfloat16) for p in pairs]
    cfgs = [fa.RegParams(scales=(2, 1), iters=(8, 5), state=st, sigma_grad=sg)
            for st in ("f32", "bf16") for sg in (1.0, 2.0)]
    out = fa.fa_register_batched_lockstep(fixed, moving, cfgs)
    for i in range(len(shapes)):
        for c, p in enumerate(cfgs):
            ref = fa.fa_register(fixed[i], moving[i], p)
            r = out[i * len(cfgs) + c]
            assert r["status"] == 0
            assert torch.equal(r["u"], ref["u"]), (i, c)
            assert r["final_loss"] == ref["final_loss"], (i, c)


def test_16bit_moments_halve_their_workspace(fa):
    lib = fa.load()
    import ctypes
    a = fa.RegParams().to_c()
    b = fa.RegParams(state="bf16").to_c()
    full = lib.fa_register_workspace_size(160, 192, 224, ctypes.byref(a))
    half = lib.fa_register_workspace_size(160, 192, 224, ctypes.byref(b))
    n = 160 * 192 * 224
    # u, m, nu twice (ping-pong): m and nu lose 2 bytes per channel each
    assert full - half >= 2 * 2 * 3 * 2 * n - 4096
