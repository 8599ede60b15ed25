"""The rigid stage in the oracle (reading R-rigid: rotation exp([w]x) by the
Rodrigues formula and translation, rigid in the input grid's voxel
coordinates about its centre, expressed as the affine map of reading R-aff).
Pinned to scipy's rotation-vector routine, the properties of rotations, FP64
central differences of R and of the loss, distance preservation on an
anisotropic grid, and recovery of a known rigid motion."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2404_01249_gb300 import synth

WS = [np.array([0.0, 0.0, 0.0]), np.array([1e-5, -2e-5, 3e-6]), np.array([4e-3, -6e-3, 5e-3]),
      np.array([0.3, -0.2, 0.5]), np.array([-1.9, 0.7, 1.2])]


@pytest.mark.parametrize("w", WS)
def test_rodrigues_is_the_rotation_of_the_vector(orc, w):
    R, _ = orc.rodrigues(w, want_grad=False)
    assert np.abs(R - Rotation.from_rotvec(w).as_matrix()).max() < 1e-14
    assert np.abs(R @ R.T - np.eye(3)).max() < 1e-14 and abs(np.linalg.det(R) - 1) < 1e-14
    assert np.abs(R @ w - w).max() < 1e-14
    assert abs(np.trace(R) - 1 - 2 * np.cos(np.linalg.norm(w))) < 1e-14


@pytest.mark.parametrize("w", WS + [np.array([0.0, 0.0, 0.0099]), np.array([0.0, 0.0, 0.0101])])
def test_rotation_derivative_matches_central_differences(orc, w):
    _, dR = orc.rodrigues(w)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (orc.rodrigues(w + e, False)[0] - orc.rodrigues(w - e, False)[0]) / (2 * h)
        assert np.abs(fd - dR[k]).max() < 1e-8


def test_rigid_map_preserves_voxel_distances(orc):
    shape = (9, 14, 23)
    rp = np.array([0.2, -0.35, 0.15, 0.05, -0.1, 0.08])
    u = orc.affine_field(orc.rigid_theta(rp, shape), shape)
    grid = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")).astype(float)
    phi = (grid + u).reshape(3, -1)
    x = grid.reshape(3, -1)
    rng = np.random.default_rng(1)
    i, j = rng.integers(0, x.shape[1], (2, 200))
    d0 = np.linalg.norm(x[:, i] - x[:, j], axis=0)
    d1 = np.linalg.norm(phi[:, i] - phi[:, j], axis=0)
    assert np.abs(d1 - d0).max() < 1e-12
    assert not orc.affine_field(orc.rigid_theta(np.zeros(6), shape), shape).any()


@pytest.mark.parametrize("loss", ["lncc", "mse"])
def test_loss_gradient_matches_central_differences(orc, loss):
    f, m, _ = synth.blobs_pair(shape=(14, 16, 18), sigma=2.5, seed=1007)
    rp = np.array([0.03, -0.02, 0.04, 0.01, -0.02, 0.015])
    _, g = orc.rigid_loss_grad(f, m, rp, window=5, loss=loss)
    h = 1e-6
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        fd = (orc.rigid_loss_grad(f, m, rp + e, loss=loss)[0] -
              orc.rigid_loss_grad(f, m, rp - e, loss=loss)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * np.abs(g).max(), k


def _blobs(shape, P, seed=5, n=20, sigma=2.5):
    """Gaussian blobs evaluated analytically at the positions P [3, ...]."""
    rng = np.random.default_rng(seed)
    C = rng.uniform([4, 4, 4], np.array(shape) - 4, (n, 3))
    amp = rng.uniform(0.5, 1.0, n)
    out = np.zeros(P.shape[1:])
    for c, a in zip(C, amp):
        out += a * np.exp(-sum((P[i] - c[i]) ** 2 for i in range(3)) / (2 * sigma ** 2))
    return out


@pytest.mark.parametrize("loss,tol_max,tol_mean", [("mse", 0.06, 0.04), ("lncc", 0.15, 0.12)])
def test_recovers_a_known_rigid_motion(orc, loss, tol_max, tol_mean):
    """moving = fixed o psi for a rigid psi of about 4 degrees and 0.5-0.7
    voxel, both images evaluated analytically (no interpolation in the
    data): the registration finds psi^-1 (theta o psi = id) to a small
    fraction of a voxel, starting 1.1 voxel away on average."""
    shape = (28, 32, 36)
    true = np.array([0.04, -0.05, 0.03, 0.03, -0.04, 0.035])
    th = orc.rigid_theta(true, shape)
    grid = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")).astype(float)
    u = orc.affine_field(th, shape)
    f, m = _blobs(shape, grid), _blobs(shape, grid + u)
    r = orc.rigid_register(f, m, [2, 1], [150, 60], lr=3e-3, loss=loss)
    A, t = r["theta"][:9].reshape(3, 3), r["theta"][9:]
    A0, t0 = th[:9].reshape(3, 3), th[9:]
    comp = orc.affine_field(np.concatenate([(A0 @ A).ravel(), A0 @ t + t0]), shape)
    inner = (slice(None),) + (slice(6, -6),) * 3
    e = np.sqrt((comp[inner] ** 2).sum(0))
    assert np.sqrt((u[inner] ** 2).sum(0)).mean() > 1.0
    assert e.max() < tol_max and e.mean() < tol_mean
