"""Affine pre-stage and registration from an initial displacement against
the oracle (reading R-aff: p' = A p + t on align-corners normalised
coordinates, plain Adam at the paper's learning rate 3e-3)."""
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


def theta_of(A, t):
    return np.concatenate([np.asarray(A, float).ravel(), np.asarray(t, float)])


def mean_disp(a, b):
    d = a.cpu().double().numpy() - b
    return float(np.sqrt((d ** 2).sum(0)).mean())


def affine_pair(orc, shape=(28, 30, 32)):
    f, _, _ = synth.blobs_pair(shape=shape, sigma=3.0)
    A = np.eye(3) + np.array([[0.04, 0.02, 0.0], [-0.01, 0.03, 0.02], [0.0, 0.01, -0.03]])
    m = orc.warp(f, orc.affine_field(theta_of(A, [0.03, -0.04, 0.02]), shape), want_grad=False)
    return f, m.astype(np.float32)


@pytest.mark.parametrize("shape", [(17, 23, 31), (1, 9, 12)])
def test_affine_field(fa, orc, shape):
    th = theta_of(np.eye(3) + 0.05 * np.random.default_rng(1).standard_normal((3, 3)),
                  [0.02, -0.03, 0.01])
    u = fa.fa_affine_field(cuda(th), shape)
    ref = orc.affine_field(th.astype(np.float32), shape)
    assert float(np.abs(u.cpu().double().numpy() - ref).max()) <= TOL * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("loss", ["mse", "lncc"])
def test_affine_register_against_oracle(fa, orc, loss):
    f, m = affine_pair(orc)
    p = fa.RegParams(scales=(2, 1), iters=(60, 30), lr=3e-3, loss=loss)
    out = fa.fa_affine_register(cuda(f), cuda(m), p)
    ref = orc.affine_register(f, m, [2, 1], [60, 30], lr=3e-3, loss=loss,
                              cc_eps=float(np.float32(1e-5)), beta1=float(np.float32(0.9)),
                              beta2=float(np.float32(0.999)), adam_eps=float(np.float32(1e-8)))
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    uref = orc.affine_field(ref["theta"], f.shape)
    assert mean_disp(out["u"], uref) < 0.05
    assert float((out["theta"].cpu().double() - torch.from_numpy(ref["theta"])).abs().max()) < 1e-3


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_deformable_from_affine_start(fa, orc, mode):
    """The paper's pipeline: affine stage, then the diffeomorphic stage from
    its displacement (fa_register_from), against the oracle."""
    f, m = affine_pair(orc, shape=(24, 26, 28))
    th = theta_of(np.eye(3) + 0.02 * np.random.default_rng(5).standard_normal((3, 3)),
                  [0.01, -0.02, 0.01])
    u0 = orc.affine_field(th, f.shape).astype(np.float32)
    p = fa.RegParams(scales=(2, 1), iters=(15, 8), mode=mode)
    out = fa.fa_register(cuda(f), cuda(m), p, u_init=cuda(u0))
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    ref = orc.register(f, m, [2, 1], [15, 8], u_init=u0, cc_eps=f32(1e-5), beta1=f32(0.9),
                       beta2=f32(0.999), adam_eps=f32(1e-8))
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    assert mean_disp(out["u"], ref["u"]) < 0.05
    zero = fa.fa_register(cuda(f), cuda(m), fa.RegParams(scales=(2, 1), iters=(0, 0), mode=mode),
                          u_init=cuda(u0))
    assert float((zero["u"].cpu() - torch.from_numpy(u0)).abs().max()) < 1e-5


def rigid_pair(orc, shape=(26, 28, 30)):
    f, _, _ = synth.blobs_pair(shape=shape, sigma=3.0, n_blobs=12, seed=1009)
    th = orc.rigid_theta(np.array([0.04, -0.05, 0.03, 0.03, -0.04, 0.035]), shape)
    m = orc.warp(f, orc.affine_field(th, shape), want_grad=False)
    return f, m.astype(np.float32)


@pytest.mark.parametrize("loss", ["mse", "lncc"])
def test_rigid_register_against_oracle(fa, orc, loss):
    f, m = rigid_pair(orc)
    p = fa.RegParams(scales=(2, 1), iters=(60, 30), lr=3e-3, loss=loss)
    out = fa.fa_rigid_register(cuda(f), cuda(m), p)
    ref = orc.rigid_register(f, m, [2, 1], [60, 30], lr=3e-3, loss=loss,
                             cc_eps=float(np.float32(1e-5)), beta1=float(np.float32(0.9)),
                             beta2=float(np.float32(0.999)), adam_eps=float(np.float32(1e-8)))
    assert abs(out["final_loss"] - ref["final_loss"]) < 1e-3
    assert float((out["rp"].cpu().double() - torch.from_numpy(ref["rp"])).abs().max()) < 2e-3
    assert float((out["theta"].cpu().double() - torch.from_numpy(ref["theta"])).abs().max()) < 2e-3
    uref = orc.affine_field(ref["theta"], f.shape)
    assert mean_disp(out["u"], uref) < 0.05


def test_rigid_zero_iterations_is_identity(fa):
    f = cuda(np.random.default_rng(0).random((9, 10, 11)))
    out = fa.fa_rigid_register(f, f, fa.RegParams(scales=(1,), iters=(0,), lr=3e-3))
    assert not out["rp"].any() and not out["u"].any()
    assert torch.equal(out["theta"].cpu(), torch.tensor([1.0, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0]))



@pytest.mark.parametrize("angle", [0.0, 1e-3, 0.3, 0.999, 1.0, 1.7, 3.1, 5.0, 40.0])
def test_rigid_theta_fp32_against_oracle(fa, orc, angle):
    """The rigid parameters' affine map in FP32 (no FP64 on the GPU): both
    branches of the Rodrigues coefficients (Taylor series below |w| = 1,
    closed forms with the Cody-Waite reduced sine and cosine above) against
    the oracle's double-precision map, on an anisotropic grid."""
    shape = (26, 41, 33)
    axis = np.array([0.3, -0.8, 0.52])
    rp = np.concatenate([angle * axis / np.linalg.norm(axis), [0.05, -0.02, 0.1]])
    rp32 = rp.astype(np.float32)
    lib = fa.load()
    rp_dev = cuda(rp32)
    th = torch.empty(12, device="cuda")
    fa._check(lib.fa_rigid_theta(fa._ptr(rp_dev), *shape, fa._ptr(th), fa._stream()))
    ref = orc.rigid_theta(rp32.astype(np.float64), shape)
    got = th.cpu().double().numpy()
    # FP32 rounding of O(10) operations on entries of size up to s_max/s_min
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()
