"""fa_warp_lncc_adjoint and the autograd wrapper against the oracle: the loss,
dL/du = dL/dJ grad I_m(phi), dL/dI_f and the warp adjoint dL/dI_m (oracle:
lncc + warp + warp_adjoint in FP64).  Bar: max-abs error over max-abs
reference <= 1e-5."""
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
    b = np.asarray(b, np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


@pytest.mark.parametrize("shape,window", [((20, 24, 28), 5), ((17, 31, 22), 3),
                                          ((12, 16, 40), 7)])
def test_adjoint_matches_oracle(fa, orc, shape, window):
    f, m, _ = synth.voronoi_pair(shape=shape, seed=321)
    u = synth.random_field(shape, 3.0, 2.5, seed=9).astype(np.float32)
    r = fa.fa_warp_lncc_adjoint(cuda(f), cuda(m), cuda(u), window, 1e-5)
    # the oracle's own warped image, LNCC, gradient and warp adjoint in FP64
    J, _ = fa.fa_warp(cuda(m), cuda(u))
    Jr, gr = orc.warp(m, u)
    assert rel(J, Jr) < TOL
    ref = orc.lncc(f, Jr, window, np.float32(1e-5), want_dJ=True, want_dI=True)
    assert abs(float(r["loss"]) - ref["loss"]) <= TOL * abs(ref["loss"])
    assert rel(r["dL_dfixed"], ref["dI"]) < TOL
    assert rel(r["dL_du"], ref["dJ"][None] * gr) < TOL
    assert rel(r["dL_dmoving"], orc.warp_adjoint(ref["dJ"], u, shape)) < TOL


def test_adjoint_full_brain_size_matches_oracle(fa, orc):
    """The warp+LNCC adjoint at the brain workload's size (160x192x224, the
    differentiation config's large case) against the oracle on every voxel:
    loss and the three gradients within 1e-5 (max-norm relative)."""
    shape = (160, 192, 224)
    f, m, _ = synth.voronoi_pair(shape=shape, seed=1000)
    u = synth.random_field(shape, 8.0, 4.0, seed=1001).astype(np.float32)
    r = fa.fa_warp_lncc_adjoint(cuda(f), cuda(m), cuda(u), 5, 1e-5)
    Jr, gr = orc.warp(m, u)
    ref = orc.lncc(f, Jr, 5, np.float32(1e-5), want_dJ=True, want_dI=True)
    assert abs(float(r["loss"]) - ref["loss"]) <= TOL * abs(ref["loss"])
    assert rel(r["dL_dfixed"], ref["dI"]) < TOL
    assert rel(r["dL_du"], ref["dJ"][None] * gr) < TOL
    assert rel(r["dL_dmoving"], orc.warp_adjoint(ref["dJ"], u, shape)) < TOL


def test_adjoint_outputs_are_optional_and_deterministic(fa):
    shape = (16, 20, 24)
    f, m, _ = synth.voronoi_pair(shape=shape, seed=5)
    u = cuda(synth.random_field(shape, 3.0, 2.0, seed=4))
    a = fa.fa_warp_lncc_adjoint(cuda(f), cuda(m), u, 5, 1e-5)
    b = fa.fa_warp_lncc_adjoint(cuda(f), cuda(m), u, 5, 1e-5, want_u=False, want_fixed=False)
    c = fa.fa_warp_lncc_adjoint(cuda(f), cuda(m), u, 5, 1e-5)
    assert b["dL_du"] is None and b["dL_dfixed"] is None
    assert torch.equal(a["dL_dmoving"], c["dL_dmoving"])   # order-independent scatter
    # without dL/dI_f the call takes the fused kernels: same values within the bar
    assert rel(b["dL_dmoving"], a["dL_dmoving"].cpu().double().numpy()) < TOL
    assert abs(float(a["loss"]) - float(b["loss"])) <= TOL * abs(float(a["loss"]))
    d = fa.fa_warp_lncc_adjoint(cuda(f), cuda(m), u, 5, 1e-5, want_u=False, want_fixed=False)
    assert torch.equal(b["dL_dmoving"], d["dL_dmoving"])


@pytest.mark.parametrize("shape,window", [((20, 24, 28), 5), ((17, 31, 22), 3),
                                          ((12, 16, 40), 7), ((160, 192, 224), 5)])
def test_fused_adjoint_matches_oracle(fa, orc, shape, window):
    """Without dL/dI_f the adjoint runs the registration loop's fused kernels
    (warp, K1, K2 with dL/dJ, scatter): loss, dL/du and dL/dI_m against the
    oracle, on TMA-width and ragged grids and at the brain size."""
    f, m, _ = synth.voronoi_pair(shape=shape, seed=322)
    u = synth.random_field(shape, 3.0, 2.5, seed=10).astype(np.float32)
    r = fa.fa_warp_lncc_adjoint(cuda(f), cuda(m), cuda(u), window, 1e-5, want_fixed=False)
    assert r["dL_dfixed"] is None
    Jr, gr = orc.warp(m, u)
    ref = orc.lncc(f, Jr, window, np.float32(1e-5), want_dJ=True)
    assert abs(float(r["loss"]) - ref["loss"]) <= TOL * abs(ref["loss"])
    assert rel(r["dL_du"], ref["dJ"][None] * gr) < TOL
    assert rel(r["dL_dmoving"], orc.warp_adjoint(ref["dJ"], u, shape)) < TOL
    only_loss = fa.fa_warp_lncc_adjoint(cuda(f), cuda(m), cuda(u), window, 1e-5, want_u=False,
                                        want_fixed=False, want_moving=False)
    assert float(only_loss["loss"]) == float(r["loss"])


def test_autograd_forward_keeps_no_gradient_volume(fa):
    """The autograd forward evaluates the loss alone and keeps only its
    inputs; backward recomputes and forms the gradients it is asked for."""
    from paper_2404_01249_gb300.autograd import warp_lncc
    shape = (32, 36, 40)
    n = 32 * 36 * 40
    f, m, _ = synth.voronoi_pair(shape=shape, seed=11)
    u0 = synth.random_field(shape, 3.0, 1.5, seed=12)
    mv = cuda(m).requires_grad_(True)
    u = cuda(u0).requires_grad_(True)
    fx = cuda(f)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    loss = warp_lncc(fx, mv, u, 5, 1e-5)
    torch.cuda.synchronize()
    kept = torch.cuda.memory_allocated() - before
    assert kept < 4 * n          # the loss scalar, not a volume
    loss.backward()
    r = fa.fa_warp_lncc_adjoint(fx, cuda(m), cuda(u0), 5, 1e-5, want_fixed=False)
    assert torch.equal(mv.grad, r["dL_dmoving"]) and torch.equal(u.grad, r["dL_du"])


def test_autograd_function(fa):
    from paper_2404_01249_gb300.autograd import warp_lncc
    shape = (14, 18, 22)
    f, m, _ = synth.voronoi_pair(shape=shape, seed=8)
    u0 = synth.random_field(shape, 3.0, 1.5, seed=3)
    fx = cuda(f).requires_grad_(True)
    mv = cuda(m).requires_grad_(True)
    u = cuda(u0).requires_grad_(True)
    loss = 3.0 * warp_lncc(fx, mv, u, 5, 1e-5)
    loss.backward()
    r = fa.fa_warp_lncc_adjoint(cuda(f), cuda(m), cuda(u0), 5, 1e-5)
    assert torch.allclose(fx.grad, 3.0 * r["dL_dfixed"], rtol=0, atol=0)
    assert torch.allclose(mv.grad, 3.0 * r["dL_dmoving"], rtol=0, atol=0)
    assert torch.allclose(u.grad, 3.0 * r["dL_du"], rtol=0, atol=0)
    # only what is asked for is computed
    u2 = cuda(u0).requires_grad_(True)
    warp_lncc(cuda(f), cuda(m), u2).backward()
    assert u2.grad is not None


def test_template_gradient_on_gpu_matches_oracle(fa, orc):
    from paper_2404_01249_gb300.template import template_gradient
    shape = (12, 14, 16)
    T, _, _ = synth.voronoi_pair(shape=shape, seed=60)
    subs = [synth.voronoi_pair(shape=shape, seed=61 + i)[1] for i in range(3)]
    us = [synth.random_field(shape, 3.0, 1.0, seed=70 + i).astype(np.float32) for i in range(3)]
    loss, g = template_gradient(cuda(T), [cuda(s) for s in subs], [cuda(u) for u in us])
    ref_g = np.zeros(shape)
    ref_l = 0.0
    for s, u in zip(subs, us):
        r = orc.lncc(s, orc.warp(T, u, want_grad=False), 5, np.float32(1e-5), want_dJ=True)
        ref_g += orc.warp_adjoint(r["dJ"], u, shape)
        ref_l += r["loss"]
    assert rel(g, ref_g / 3) < TOL
    assert abs(float(loss) - ref_l / 3) < 1e-5


def test_adjoint_against_fp64_central_differences(fa, orc):
    """dL/du, dL/dI_m and dL/dI_f from the GPU against FP64 central finite
    differences (h = 1e-4) of the oracle's loss at 48^3, on voxels whose
    warped position stays at least 10 h away from the trilinear kinks."""
    shape = (48, 48, 48)
    f, m, _ = synth.voronoi_pair(shape=shape, seed=48)
    u = synth.random_field(shape, 3.0, 2.0, seed=49).astype(np.float32)
    r = fa.fa_warp_lncc_adjoint(cuda(f), cuda(m), cuda(u), 5, 1e-5)
    du, dm, dfx = (r[k].cpu().double().numpy() for k in ("dL_du", "dL_dmoving", "dL_dfixed"))
    f64, m64, u64 = f.astype(np.float64), m.astype(np.float64), u.astype(np.float64)

    def loss(ff, mm, uu):
        return orc.lncc(ff, orc.warp(mm, uu, want_grad=False), 5, float(np.float32(1e-5)),
                        want_dJ=False)["loss"]

    h = 1e-4
    rng = np.random.default_rng(7)
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    pos = np.stack([z, y, x]) + u64
    frac = np.abs(pos - np.round(pos)).min(axis=0)
    inner = (frac > 10 * h)
    inner[:4], inner[-4:], inner[:, :4], inner[:, -4:], inner[:, :, :4], inner[:, :, -4:] = (False,) * 6
    cand = np.argwhere(inner & (np.abs(m64) > 0))
    picks = cand[rng.choice(len(cand), 6, replace=False)]
    for (a, b, c) in picks:
        for ch in range(3):
            up, um = u64.copy(), u64.copy()
            up[ch, a, b, c] += h
            um[ch, a, b, c] -= h
            fd = (loss(f64, m64, up) - loss(f64, m64, um)) / (2 * h)
            assert abs(du[ch, a, b, c] - fd) <= 1e-4 * np.abs(du).max(), (a, b, c, ch)
        mp, mq = m64.copy(), m64.copy()
        mp[a, b, c] += h
        mq[a, b, c] -= h
        fd = (loss(f64, mp, u64) - loss(f64, mq, u64)) / (2 * h)
        assert abs(dm[a, b, c] - fd) <= 1e-4 * np.abs(dm).max(), (a, b, c)
        fp, fq = f64.copy(), f64.copy()
        fp[a, b, c] += h
        fq[a, b, c] -= h
        fd = (loss(fp, m64, u64) - loss(fq, m64, u64)) / (2 * h)
        assert abs(dfx[a, b, c] - fd) <= 1e-4 * np.abs(dfx).max(), (a, b, c)


def test_template_gradient_eight_subjects_48(fa, orc):
    """The template step of the atlas workload: 8 subjects at 48^3, the mean
    template gradient on the GPU against the oracle's."""
    from paper_2404_01249_gb300.template import template_gradient
    shape = (48, 48, 48)
    T = synth.voronoi_pair(shape=shape, seed=400)[0]
    subs = [synth.voronoi_pair(shape=shape, seed=401 + i)[1] for i in range(8)]
    us = [synth.random_field(shape, 3.0, 1.5, seed=420 + i).astype(np.float32) for i in range(8)]
    loss, g = template_gradient(cuda(T), [cuda(s) for s in subs], [cuda(u) for u in us])
    ref_g, ref_l = np.zeros(shape), 0.0
    for s, u in zip(subs, us):
        r = orc.lncc(s, orc.warp(T, u, want_grad=False), 5, np.float32(1e-5), want_dJ=True)
        ref_g += orc.warp_adjoint(r["dJ"], u, shape)
        ref_l += r["loss"]
    assert rel(g, ref_g / 8) < TOL
    assert abs(float(loss) - ref_l / 8) < 1e-5
