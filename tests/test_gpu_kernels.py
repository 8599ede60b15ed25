"""Parity of every libfa kernel entry point with the FP64 oracle (same seeded
inputs; the oracle reads the float32 inputs as doubles).  Bar: max-abs error
over max-abs reference <= 1e-5 for FP32 arithmetic."""
import numpy as np
import pytest
import torch

from paper_2404_01249_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel(a, b):
    a = a.detach().cpu().double().numpy() if torch.is_tensor(a) else np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


@pytest.fixture(scope="module")
def fa():
    from paper_2404_01249_gb300 import build, fa
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fa.load()
    return fa


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def voronoi(shape, seed=1000):
    f, m, _ = synth.voronoi_pair(shape=shape, seed=seed)
    return f, m


def smooth_field(shape, max_disp, seed):
    return synth.random_field(shape, 3.0, max_disp, seed)


SHAPES = [(19, 37, 45), (40, 48, 56), (1, 9, 70), (5, 3, 2)]


@pytest.mark.parametrize("shape", SHAPES)
def test_warp(fa, orc, shape):
    f, m = voronoi(shape) if min(shape) > 3 else (None, np.random.default_rng(1).random(shape))
    img = m.astype(np.float32)
    u = smooth_field(shape, 4.0, 5)
    J, g = fa.fa_warp(cuda(img), cuda(u))
    Jr, gr = orc.warp(img, u)
    assert rel(J, Jr) < TOL
    assert rel(g, gr) < TOL


def test_warp_outside_and_identity(fa, orc):
    shape = (6, 7, 8)
    img = np.random.default_rng(2).random(shape).astype(np.float32)
    u = np.zeros((3,) + shape, np.float32)
    J = fa.fa_warp(cuda(img), cuda(u), want_grad=False)
    assert torch.equal(J.cpu(), torch.from_numpy(img))
    u[:] = 50.0  # everything outside
    J, g = fa.fa_warp(cuda(img), cuda(u))
    assert float(J.abs().max()) == 0.0 and float(g.abs().max()) == 0.0
    u[0] = 1.0
    u[1] = -2.0
    u[2] = 3.0
    J = fa.fa_warp(cuda(img), cuda(u), want_grad=False)
    assert np.array_equal(J.cpu().numpy(), orc.warp(img, u, want_grad=False).astype(np.float32))


@pytest.mark.parametrize("window", [3, 5, 7])
@pytest.mark.parametrize("shape", [(19, 37, 45), (40, 48, 56)])
def test_lncc_fwd_bwd(fa, orc, shape, window):
    f, m = voronoi(shape, seed=11)
    out = fa.fa_lncc_fwd_bwd(cuda(f), cuda(m), window, 1e-5, want_dJ=True, want_dI=True)
    ref = orc.lncc(f, m, window, np.float32(1e-5), want_dI=True)
    assert abs(float(out["loss"]) - ref["loss"]) <= TOL * abs(ref["loss"])
    assert rel(out["dJ"], ref["dJ"]) < TOL
    assert rel(out["dI"], ref["dI"]) < TOL


def test_lncc_eps_zero_and_single_outputs(fa, orc):
    shape = (12, 17, 33)
    r = np.random.default_rng(3)
    f = r.random(shape).astype(np.float32)
    m = r.random(shape).astype(np.float32)
    for want_dJ, want_dI in [(True, False), (False, True)]:
        out = fa.fa_lncc_fwd_bwd(cuda(f), cuda(m), 5, 0.0, want_dJ=want_dJ, want_dI=want_dI)
        ref = orc.lncc(f, m, 5, 0.0, want_dI=True)
        assert abs(float(out["loss"]) - ref["loss"]) <= TOL * abs(ref["loss"])
        if want_dJ:
            assert rel(out["dJ"], ref["dJ"]) < TOL
        if want_dI:
            assert rel(out["dI"], ref["dI"]) < TOL


def test_lncc_self_is_one(fa):
    f, _ = voronoi((20, 24, 28), seed=12)
    out = fa.fa_lncc_fwd_bwd(cuda(f), cuda(f), 5, 0.0, want_dJ=True)
    assert abs(float(out["loss"]) + 1.0) < 1e-6
    assert float(out["dJ"].abs().max()) * f.size < 1e-3


def test_mse(fa, orc):
    shape = (19, 37, 45)
    f, m = voronoi(shape, seed=13)
    out = fa.fa_mse_fwd_bwd(cuda(f), cuda(m), want_dI=True)
    ref = orc.mse(f, m)
    assert abs(float(out["loss"]) - ref["loss"]) <= TOL * ref["loss"]
    assert rel(out["dJ"], ref["dJ"]) < TOL
    assert rel(out["dI"], ref["dI"]) < TOL


@pytest.mark.parametrize("sigma", [0.0, 0.5, 1.0, 2.0, 6.0])
def test_gauss(fa, orc, sigma):
    shape = (19, 37, 45)
    x = np.random.default_rng(4).standard_normal((3,) + shape).astype(np.float32)
    y = fa.fa_gauss_smooth(cuda(x), sigma)
    assert rel(y, orc.gauss_smooth(x, sigma)) < TOL
    xin = cuda(x)
    fa.fa_gauss_smooth(xin, sigma, out=xin)  # in place
    assert rel(xin, orc.gauss_smooth(x, sigma)) < TOL


@pytest.mark.parametrize("lr", [0.5, 20.0])
def test_radam_step(fa, orc, lr):
    """Adam, step scale and compose against the oracle.  lr 0.5 keeps every
    step below half a voxel (the compose's sign-side cells); lr 20 allows 10
    voxels, so one call mixes those cells with floor cells (about 1% of the
    voxels step a voxel or more on some axis), and steps at the grid's faces
    sample the zero outside."""
    shape = (19, 37, 45)
    r = np.random.default_rng(5)
    u = smooth_field(shape, 2.0, 6)
    m = (r.standard_normal((3,) + shape) * 1e-6).astype(np.float32)
    v = (r.random((3,) + shape) * 1e-12).astype(np.float32)
    g = (r.standard_normal((3,) + shape) * 1e-6).astype(np.float32)
    params = fa.RegParams(lr=lr)
    mt, vt = cuda(m), cuda(v)
    for t in (1, 7):
        mt, vt = cuda(m), cuda(v)
        u_out, eps = fa.fa_radam_step(cuda(u), mt, vt, cuda(g), t, params)
        f32 = lambda x: float(np.float32(x))
        d, mr, vr = orc.adam(g, m, v, t, f32(0.9), f32(0.999), f32(1e-8))
        delta, er = orc.step_scale(d, lr, 2.0)
        if lr > 2.0:  # both cell rules occur
            big = (np.abs(delta) >= 1.0).any(0)
            assert 0 < big.sum() < big.size
        ur = orc.compose(u, delta)
        assert rel(mt, mr) < TOL and rel(vt, vr) < TOL
        assert abs(float(eps) - er) <= TOL * er
        assert rel(u_out, ur) < TOL


def test_radam_step_device_counter_in_a_graph(fa, orc):
    """fa_radam_step with its device step counter, recorded in a CUDA graph:
    two steps per replay (ping-pong of u), two replays, so t runs 1..4 on the
    device with no host involvement; u, m, v and the counter against the
    oracle's four Adam steps (Algorithm 1 optimiser update and retraction)."""
    import ctypes
    shape = (19, 37, 45)
    r = np.random.default_rng(8)
    u0 = smooth_field(shape, 2.0, 9)
    gs = [(r.standard_normal((3,) + shape) * 1e-6).astype(np.float32) for _ in range(2)]
    params = fa.RegParams(lr=0.5)
    lib = fa.load()
    D, H, W = shape
    ua, ub = cuda(u0), torch.empty((3,) + shape, device="cuda")
    m = torch.zeros((3,) + shape, device="cuda")
    v = torch.zeros((3,) + shape, device="cuda")
    g = [cuda(x) for x in gs]
    t_dev = torch.zeros(1, dtype=torch.int32, device="cuda")
    eps = torch.empty((), device="cuda")
    ws = fa.workspace(lib.fa_radam_workspace_size(D, H, W), "cuda")
    pc = params.to_c()

    def step(src, dst, gk):
        assert lib.fa_radam_step(fa._vol(src, 3), fa._vol(dst, 3), fa._vol(m, 3), fa._vol(v, 3),
                                 fa._vol(gk, 3), fa._ptr(t_dev), ctypes.byref(pc), fa._ptr(eps),
                                 fa._ptr(ws), ws.numel(), fa._stream()) == 0

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            step(ua, ub, g[0])
            step(ub, ua, g[1])
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    assert int(t_dev.item()) == 0  # capture does not run anything
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    assert int(t_dev.item()) == 4
    f32 = lambda x: float(np.float32(x))
    ur, mr, vr = u0.astype(np.float64), np.zeros((3,) + shape), np.zeros((3,) + shape)
    for t in range(1, 5):
        d, mr, vr = orc.adam(gs[(t - 1) % 2], mr, vr, t, f32(0.9), f32(0.999), f32(1e-8))
        delta, er = orc.step_scale(d, 0.5, 2.0)
        ur = orc.compose(ur, delta)
    assert rel(m, mr) < TOL and rel(v, vr) < TOL
    assert rel(ua, ur) < TOL
    assert abs(float(eps) - er) <= TOL * er


def test_pyramid_all_levels(fa, orc):
    """fa_pyramid builds every level of Algorithm 1's downsample in one call;
    each level against the oracle's downsample (a ragged grid, four levels
    including an odd scale and the copy at scale 1)."""
    shape = (37, 45, 53)
    f, _ = voronoi(shape, seed=15)
    scales = (8, 3, 2, 1)
    levels = fa.fa_pyramid(cuda(f), fa.RegParams(scales=scales, iters=(1, 1, 1, 1)))
    assert len(levels) == len(scales)
    for lv, s in zip(levels, scales):
        ref = orc.downsample(f, s)
        assert tuple(lv.shape) == ref.shape
        assert rel(lv, ref) < TOL
    assert torch.equal(levels[-1], cuda(f))


@pytest.mark.parametrize("s", [1, 2, 3, 4])
def test_pyramid_level(fa, orc, s):
    shape = (19, 37, 45)
    f, _ = voronoi(shape, seed=14)
    y = fa.fa_pyramid_level(cuda(f), s)
    assert rel(y, orc.downsample(f, s)) < TOL


@pytest.mark.parametrize("power", [1, -1, -2])
def test_upsample_field(fa, orc, power):
    c = smooth_field((10, 12, 14), 1.5, 7)
    fine = (19, 24, 28)
    y = fa.fa_upsample_field(cuda(c), fine, power)
    assert rel(y, orc.upsample_field(c, fine, power)) < TOL


def test_full_size_warp_and_lncc(fa, orc):
    """160x192x224 (brain-MRI shape): warp and LNCC forward/backward in the
    launch configuration fa_register uses, against the oracle on the whole
    volume."""
    shape = (160, 192, 224)
    f, m, psi = synth.voronoi_pair(shape=shape, seed=1000)
    u = (-0.5 * psi).astype(np.float32)
    J, g = fa.fa_warp(cuda(m), cuda(u))
    Jr, gr = orc.warp(m, u)
    assert rel(J, Jr) < TOL and rel(g, gr) < TOL
    # the LNCC kernels take the oracle's own warped image (rounded to FP32),
    # so no CUDA output feeds the oracle
    Jn = Jr.astype(np.float32)
    out = fa.fa_lncc_fwd_bwd(cuda(f), cuda(Jn), 5, 1e-5)
    ref = orc.lncc(f, Jn, 5, np.float32(1e-5))
    assert abs(float(out["loss"]) - ref["loss"]) <= TOL * abs(ref["loss"])
    assert rel(out["dJ"], ref["dJ"]) < TOL


@pytest.mark.parametrize("shape", [(19, 37, 45), (1, 9, 70), (5, 3, 2)])
def test_jac_direction(fa, orc, shape):
    g = np.random.default_rng(31).standard_normal((3,) + shape).astype(np.float32)
    u = smooth_field(shape, 2.0, 32).astype(np.float32)
    out = fa.fa_jac_direction(cuda(g), cuda(u))
    assert rel(out, orc.jac_direction(g, u)) < TOL
    gi = cuda(g)
    fa.fa_jac_direction(gi, cuda(u), out=gi)          # in place
    assert torch.equal(gi, out)


@pytest.mark.parametrize("shape", [(19, 37, 45), (5, 3, 2)])
def test_compose_fields(fa, orc, shape):
    u = smooth_field(shape, 2.5, 41).astype(np.float32)
    delta = smooth_field(shape, 1.2, 42).astype(np.float32)
    assert rel(fa.fa_compose(cuda(u), cuda(delta)), orc.compose(u, delta)) < TOL


@pytest.mark.parametrize("steps", [0, 1, 6])
def test_svf_exp(fa, orc, steps):
    shape = (24, 28, 20)
    v = smooth_field(shape, 6.0, 43).astype(np.float32)
    assert rel(fa.fa_svf_exp(cuda(v), steps), orc.svf_exp(v, steps)) < TOL
