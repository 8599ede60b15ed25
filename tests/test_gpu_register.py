"""End-to-end parity of fa_register with the oracle's Algorithm 1 on the
32^3 blobs workload (final LNCC within 1e-3, mean displacement difference
below 0.05 voxel), plus edge cases and device status reporting."""
import ctypes
import dataclasses

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


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_c1_matches_oracle(fa, c1_oracle, mode):
    f, m, ref = c1_oracle
    out = fa.fa_register(cuda(f), cuda(m), fa.RegParams(mode=mode, **C1))
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    assert mean_disp_diff(out["u"], ref["u"]) < 0.05


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_zero_iterations_is_identity(fa, orc, mode):
    f, m, _ = synth.blobs_pair(shape=(12, 14, 16), sigma=2.0)
    out = fa.fa_register(cuda(f), cuda(m), fa.RegParams(scales=(2, 1), iters=(0, 0), mode=mode))
    assert float(out["u"].abs().max()) == 0.0
    ref = orc.lncc(f, m, 5, np.float32(1e-5), want_dJ=False)["loss"]
    assert abs(out["final_loss"] - ref) < 1e-5


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_mse_single_level(fa, orc, mode):
    f, m, _ = synth.blobs_pair(shape=(16, 16, 16), sigma=2.0, max_disp=1.0)
    out = fa.fa_register(cuda(f), cuda(m), fa.RegParams(scales=(1,), iters=(30,), loss="mse",
                                                         mode=mode))
    ref = orc.register(f, m, [1], [30], loss="mse", cc_eps=0.0, beta1=float(np.float32(0.9)),
                       beta2=float(np.float32(0.999)), adam_eps=float(np.float32(1e-8)))
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3 * max(1.0, abs(ref["final_loss"]))
    assert mean_disp_diff(out["u"], ref["u"]) < 0.05


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_nonfinite_input_is_reported(fa, mode):
    f, m, _ = synth.blobs_pair(shape=(8, 8, 8), sigma=2.0)
    m[3, 3, 3] = np.nan
    with pytest.raises(fa.FAError) as e:
        fa.fa_register(cuda(f), cuda(m), fa.RegParams(scales=(1,), iters=(3,), mode=mode))
    assert e.value.status == 5


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_tiny_and_degenerate_grids(fa, orc, mode):
    # the fused schedule stores every level with rows padded to a multiple of
    # 4 floats and takes tile copies (TMA) with boxes larger than the grid
    for shape in [(1, 1, 1), (1, 4, 9), (3, 2, 5), (2, 3, 4), (5, 6, 8)]:
        r = np.random.default_rng(9)
        f = r.random(shape).astype(np.float32)
        m = r.random(shape).astype(np.float32)
        p = fa.RegParams(scales=(2, 1), iters=(3, 2), mode=mode)
        out = fa.fa_register(cuda(f), cuda(m), p)
        ref = orc.register(f, m, [2, 1], [3, 2], cc_eps=float(np.float32(1e-5)),
                           beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)),
                           adam_eps=float(np.float32(1e-8)))
        assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
        assert mean_disp_diff(out["u"], ref["u"]) < 0.05


@pytest.mark.parametrize("shape", [(37, 45, 53), (40, 48, 56)])
@pytest.mark.parametrize("kw", [
    dict(),                                         # the brain workload's hyper-parameters
    dict(window=7, sigma_grad=2.0, sigma_warp=0.0),  # wider window, no warp smoothing
    dict(window=3, sigma_grad=3.0, sigma_warp=2.5),  # Gaussians wider than the fused rings
    dict(loss="mse", sigma_grad=0.5),
    dict(lr=2.5),  # steps up to 1.25 voxel: K4 samples u from global memory
])
def test_fused_equals_plain(fa, kw, shape):
    """Both schedules compute the same arithmetic in the same order, so their
    results agree to float32 rounding over a whole multi-level run on a
    brain-shaped grid, of uneven width (the fused levels' rows padded) and
    with widths that are multiples of 4."""
    f, m, _ = synth.voronoi_pair(shape=shape, seed=31)
    base = dict(scales=(2, 1), iters=(15, 8))
    base.update(kw)
    a = fa.fa_register(cuda(f), cuda(m), fa.RegParams(mode="plain", **base))
    b = fa.fa_register(cuda(f), cuda(m), fa.RegParams(mode="fused", **base))
    assert abs(a["final_loss"] - b["final_loss"]) < 1e-5
    assert float((a["u"] - b["u"]).abs().max()) < 1e-4


@pytest.mark.parametrize("shape", [(20, 23, 29), (17, 30, 41)])
def test_padded_rows_against_oracle(fa, orc, shape):
    """Uneven widths at every level (29 -> 15, 41 -> 21): the fused
    schedule's padded level buffers (resampling, hand-off, u_out copy) give
    the oracle's registration."""
    f, m, _ = synth.voronoi_pair(shape=shape, seed=81)
    out = fa.fa_register(cuda(f), cuda(m), fa.RegParams(scales=(2, 1), iters=(20, 10)))
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    ref = orc.register(f, m, [2, 1], [20, 10], cc_eps=f32(1e-5), beta1=f32(0.9),
                       beta2=f32(0.999), adam_eps=f32(1e-8))
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    assert mean_disp_diff(out["u"], ref["u"]) < 0.05


def test_fused_brain_level_against_oracle(fa, orc):
    """One level of the brain workload at scale 4 (40x48x56, 200 iterations)
    against the oracle: final LNCC within 1e-3 and mean displacement
    difference below 0.05 voxel."""
    f, m, _ = synth.voronoi_pair(shape=(160, 192, 224), seed=1000)
    fl = orc.downsample(f, 4).astype(np.float32)
    ml = orc.downsample(m, 4).astype(np.float32)
    out = fa.fa_register(cuda(fl), cuda(ml), fa.RegParams(scales=(1,), iters=(200,), mode="fused"))
    f32 = lambda x: float(np.float32(x))
    ref = orc.register(fl, ml, [1], [200], cc_eps=f32(1e-5), beta1=f32(0.9), beta2=f32(0.999),
                       adam_eps=f32(1e-8))
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    assert mean_disp_diff(out["u"], ref["u"]) < 0.05


def test_brain_workload_full_size_against_oracle(fa, orc):
    """The benchmarked workload itself, end to end at full size: the
    160x192x224 brain-shaped pair with scales {4,2,1} x iterations
    {200,100,50} in the fused schedule against the oracle's FP64 Algorithm 1
    on the same pair: final LNCC within 1e-3 and mean displacement difference
    below 0.05 voxel (the oracle takes about a minute on 16 cores)."""
    f, m, _ = synth.voronoi_pair(shape=(160, 192, 224), seed=1000)
    out = fa.fa_register(cuda(f), cuda(m), fa.RegParams())
    f32 = lambda x: float(np.float32(x))
    ref = orc.register(f, m, [4, 2, 1], [200, 100, 50], cc_eps=f32(1e-5), beta1=f32(0.9),
                       beta2=f32(0.999), adam_eps=f32(1e-8))
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    assert mean_disp_diff(out["u"], ref["u"]) < 0.05


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_16bit_images_equal_fp32_of_the_rounded_images(fa, dtype):
    """16-bit images are widened exactly, so registering them equals
    registering their FP32 values bit for bit (and inherits the FP32 path's
    parity with the oracle)."""
    f, m, _ = synth.voronoi_pair(shape=(24, 28, 32), seed=77)
    fh, mh = cuda(f).to(dtype), cuda(m).to(dtype)
    p = fa.RegParams(scales=(2, 1), iters=(10, 5))
    a = fa.fa_register(fh, mh, p)
    b = fa.fa_register(fh.float().contiguous(), mh.float().contiguous(), p)
    assert torch.equal(a["u"], b["u"]) and a["final_loss"] == b["final_loss"]


def test_graph_replay_equals_launch_by_launch(fa):
    """The recorded-graph path replays exactly the launches of the direct
    path: same bits, same launch count, and the in-graph kernel timer
    reports its events on every replay."""
    f, m, _ = synth.voronoi_pair(shape=(24, 28, 32), seed=13)
    fx, mv = cuda(f), cuda(m)
    direct = fa.fa_register(fx, mv, fa.RegParams(scales=(2, 1), iters=(8, 6), graph=False))
    pg = fa.RegParams(scales=(2, 1), iters=(8, 6), graph=True)
    ws = fa.workspace(fa.load().fa_register_workspace_size(24, 28, 32, ctypes.byref(pg.to_c())),
                      fx.device)
    u = torch.empty_like(direct["u"])
    loss = torch.empty((), device=fx.device)
    n0 = fa.fa_launch_count()
    fa.fa_register(fx, mv, pg, ws=ws, u_out=u, loss_out=loss)          # records the graph
    n1 = fa.fa_launch_count()
    u.zero_()
    r = fa.fa_register(fx, mv, pg, ws=ws, u_out=u, loss_out=loss)      # replays it
    n2 = fa.fa_launch_count()
    assert torch.equal(u, direct["u"]) and r["final_loss"] == direct["final_loss"]
    assert n2 - n1 == n1 - n0 > 0
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(4 * 6)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(4 * 6)]
    tm = fa.make_timer(fa.FA_K_FUSED_ALL, 1, ev0, ev1)
    for _ in range(2):
        fa.fa_register(fx, mv, pg, ws=ws, u_out=u, loss_out=loss, timer=tm)
        torch.cuda.synchronize()
        assert tm.count == 24
        assert all(a.elapsed_time(b) > 0 for a, b in zip(ev0, ev1))
    assert torch.equal(u, direct["u"])
    # without graph recording the events are recorded on the stream directly
    tm = fa.make_timer(fa.FA_K_FUSED_ALL, 1, ev0, ev1)
    fa.fa_register(fx, mv, dataclasses.replace(pg, graph=False), ws=ws, u_out=u, loss_out=loss,
                   timer=tm)
    torch.cuda.synchronize()
    assert tm.count == 24
    assert all(a.elapsed_time(b) > 0 for a, b in zip(ev0, ev1))
    assert torch.equal(u, direct["u"])


def test_tile_choices_change_speed_not_bits(fa):
    """Every tile choice (slab depth, 32x8 or 32x16 tiles) of the fused
    kernels computes the same bits: the window sums are exact integers and
    each output's filters run in the same order; the autotuner only picks
    the fastest."""
    shape = (40, 48, 56)
    f, m, _ = synth.voronoi_pair(shape=shape, seed=17)
    fx, mv = cuda(f), cuda(m)
    p = fa.RegParams(scales=(2, 1), iters=(6, 4), graph=False)
    fa.fa_autotune_reset()
    base = fa.fa_register(fx, mv, p)
    lv = [(20, 24, 28), shape]
    try:
        for wide, tz in [(0, 1), (1, 3), (0, 7), (1, 64)]:
            for (D, H, W) in lv:
                for k, rad in [(0, 2), (1, 2), (2, 3), (3, 2)]:
                    fa.fa_autotune_set(k, rad, 1 if k == 3 else 0, D, H, W, wide, tz)
            r = fa.fa_register(fx, mv, p)
            assert torch.equal(r["u"], base["u"]) and r["final_loss"] == base["final_loss"]
        fa.fa_autotune_reset()
        choices = fa.fa_autotune(shape, p)
        assert len(choices) == 8 and all(c["tz"] >= 0 for c in choices)
        r = fa.fa_register(fx, mv, p)
        assert torch.equal(r["u"], base["u"]) and r["final_loss"] == base["final_loss"]
    finally:
        fa.fa_autotune_reset()


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_jacobian_direction_against_oracle(fa, orc, mode):
    """use_jac (steepest Eulerian direction) end to end against the oracle."""
    f, m, _ = synth.blobs_pair()
    p = fa.RegParams(scales=(2, 1), iters=(20, 10), mode=mode, use_jac=True)
    out = fa.fa_register(cuda(f), cuda(m), p)
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    ref = orc.register(f, m, [2, 1], [20, 10], cc_eps=f32(1e-5), beta1=f32(0.9),
                       beta2=f32(0.999), adam_eps=f32(1e-8), use_jac=True)
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    assert mean_disp_diff(out["u"], ref["u"]) < 0.05


def test_jacobian_direction_fused_equals_plain(fa):
    f, m, _ = synth.voronoi_pair(shape=(40, 48, 56), seed=33)
    base = dict(scales=(2, 1), iters=(10, 6), use_jac=True)
    a = fa.fa_register(cuda(f), cuda(m), fa.RegParams(mode="plain", **base))
    b = fa.fa_register(cuda(f), cuda(m), fa.RegParams(mode="fused", **base))
    assert abs(a["final_loss"] - b["final_loss"]) < 1e-5
    assert float((a["u"] - b["u"]).abs().max()) < 1e-4
