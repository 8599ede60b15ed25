"""The persistent schedule (FA_MODE_PERSISTENT: one cooperative launch for
all of a coarse level's iterations, grid barriers between the phases)
computes the bits of the four fused kernels (FA_MODE_FUSED): same
displacement and final loss, bit for bit, over window sizes, Gaussian radii,
both compose variants, BF16 moments, ragged grids, iteration counts that
take several launches, and the brain-shaped pair's coarse levels at full
length.  The bounded grid-barrier wait gives up on a CTA that never arrives
and reports a timeout."""
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


def run(fa, f, m, mode, **kw):
    out = fa.fa_register(f, m, fa.RegParams(mode=mode, **kw))
    return out["u"].clone(), out["final_loss"]


CASES = [
    # (shape, parameters)
    ((32, 32, 32), dict(scales=(2, 1), iters=(50, 25))),
    ((37, 45, 53), dict(scales=(2, 1), iters=(7, 5), window=3, sigma_grad=2.0, sigma_warp=0.0)),
    ((29, 31, 27), dict(scales=(1,), iters=(9,), window=7, sigma_grad=0.5, sigma_warp=1.0,
                        lr=1.0, state="bf16")),
    ((24, 17, 61), dict(scales=(1,), iters=(6,), lr=2.5, sigma_warp=0.4)),  # steps above a voxel
    ((5, 3, 2), dict(scales=(1,), iters=(4,))),
    ((1, 9, 70), dict(scales=(1,), iters=(4,), window=3)),
    ((12, 14, 16), dict(scales=(2, 1), iters=(0, 3))),
]


@pytest.mark.parametrize("shape,kw", CASES)
def test_persistent_equals_fused(fa, shape, kw):
    if min(shape) >= 8:
        f, m, _ = synth.voronoi_pair(shape=shape, seed=71)
    else:
        r = np.random.default_rng(72)
        f = r.random(shape).astype(np.float32)
        m = np.roll(f, 1, axis=-1).copy()
    ft, mt = torch.from_numpy(f).cuda(), torch.from_numpy(m).cuda()
    u_p, l_p = run(fa, ft, mt, "persistent", **kw)
    u_t, l_t = run(fa, ft, mt, "fused", **kw)
    assert np.isfinite(l_p)
    assert l_p == l_t
    assert torch.equal(u_p, u_t)


def test_persistent_several_launches(fa):
    """600 iterations take two launches (512 per launch): the displacement
    buffer parity and the step counter carry across them."""
    shape = (20, 22, 24)
    f, m, _ = synth.voronoi_pair(shape=shape, seed=73)
    ft, mt = torch.from_numpy(f).cuda(), torch.from_numpy(m).cuda()
    kw = dict(scales=(1,), iters=(600,), lr=0.25)
    u_p, l_p = run(fa, ft, mt, "persistent", **kw)
    u_t, l_t = run(fa, ft, mt, "fused", **kw)
    assert l_p == l_t and torch.equal(u_p, u_t)


def test_brain_coarse_levels_full_length(fa):
    """The benchmarked pair's two coarse levels (40x48x56 and 80x96x112, 200
    and 100 iterations) in both schedules, and the full three-level
    registration, whose finest level runs the four fused kernels in both."""
    f, m, _ = synth.voronoi_pair(shape=(160, 192, 224), seed=1000)
    ft, mt = torch.from_numpy(f).cuda(), torch.from_numpy(m).cuda()
    for kw in (dict(scales=(4, 2), iters=(200, 100)),
               dict(scales=(4, 2, 1), iters=(200, 100, 5))):
        u_p, l_p = run(fa, ft, mt, "persistent", **kw)
        u_t, l_t = run(fa, ft, mt, "fused", **kw)
        assert l_p == l_t and torch.equal(u_p, u_t)


def test_persistent_graph_replay_and_status(fa):
    """A recorded registration replays the persistent launches with the same
    bits, and the status word stays clean."""
    shape = (32, 36, 40)
    f, m, _ = synth.voronoi_pair(shape=shape, seed=74)
    ft, mt = torch.from_numpy(f).cuda(), torch.from_numpy(m).cuda()
    P = fa.RegParams(scales=(2, 1), iters=(30, 10), mode="persistent")
    ws = fa.workspace(fa.fa_register_workspace_size(shape, P), "cuda")
    outs = [fa.fa_register(ft, mt, P, ws=ws) for _ in range(3)]  # record, replay, replay
    for o in outs[1:]:
        assert o["final_loss"] == outs[0]["final_loss"]
        assert torch.equal(o["u"], outs[0]["u"])
    fa.fa_ws_status(ws)


@pytest.mark.parametrize("limit", [0, 1 << 20])
def test_grid_barrier_reports_timeout(fa, limit):
    lib = fa.load()
    ws = fa.workspace(256, "cuda")
    fa._check(lib.fa_selftest_grid_barrier(fa._ptr(ws), ws.numel(), int(limit), fa._stream()))
    assert int(lib.fa_ws_status(fa._ptr(ws), fa._stream())) == fa.FA_ERR_TIMEOUT
    # the context still runs a registration with persistent levels
    f, m, _ = synth.blobs_pair(shape=(16, 18, 20), sigma=2.5)
    out = fa.fa_register(torch.from_numpy(f).cuda(), torch.from_numpy(m).cuda(),
                         fa.RegParams(scales=(2, 1), iters=(5, 5), mode="persistent"))
    assert np.isfinite(out["final_loss"])
