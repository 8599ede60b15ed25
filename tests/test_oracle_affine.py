"""The affine pre-stage in the oracle (reading R-aff: p' = A p + t on
align-corners normalised coordinates, plain Adam).  Pinned to the identity,
to level invariance of the normalised parametrisation, to the group law
(an affine map composed with its inverse is the identity), to FP64 central
differences of the loss, and to recovery of a known affine map."""
import numpy as np

from paper_2404_01249_gb300 import synth

ID = np.array([1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0, 0, 0, 0])


def theta_of(A, t):
    return np.concatenate([np.asarray(A, float).ravel(), np.asarray(t, float)])


def test_identity_is_zero(orc):
    assert np.array_equal(orc.affine_field(ID, (5, 6, 7)), np.zeros((3, 5, 6, 7)))


def test_level_invariance(orc):
    """Where a coarse grid point coincides with a fine one (align corners),
    the fine displacement is the coarse one times the grid ratio."""
    A = np.eye(3) + 0.05 * np.random.default_rng(1).standard_normal((3, 3))
    th = theta_of(A, [0.03, -0.02, 0.05])
    coarse, fine = (5, 7, 9), (9, 13, 17)          # (n_f - 1) = 2 (n_c - 1)
    uc = orc.affine_field(th, coarse)
    uf = orc.affine_field(th, fine)
    assert np.allclose(uf[:, ::2, ::2, ::2], 2.0 * uc, rtol=0, atol=1e-12)


def test_group_law_with_the_inverse(orc):
    A = np.eye(3) + 0.04 * np.random.default_rng(2).standard_normal((3, 3))
    t = np.array([0.02, 0.01, -0.03])
    Ai = np.linalg.inv(A)
    th, thi = theta_of(A, t), theta_of(Ai, -Ai @ t)
    shape = (20, 21, 22)
    comp = orc.compose(orc.affine_field(th, shape), orc.affine_field(thi, shape))
    inner = (slice(None),) + (slice(3, -3),) * 3
    assert np.abs(comp[inner]).max() < 1e-9


def test_gradient_matches_central_differences(orc):
    f, m, _ = synth.blobs_pair(shape=(14, 15, 16), sigma=2.5)
    th = theta_of(np.eye(3) + 0.02 * np.random.default_rng(3).standard_normal((3, 3)),
                  [0.01, -0.02, 0.015])
    for loss in ("lncc", "mse"):
        _, g = orc.affine_loss_grad(f, m, th, window=5, loss=loss)
        h = 1e-6
        fd = np.empty(12)
        for k in range(12):
            a, b = th.copy(), th.copy()
            a[k] += h
            b[k] -= h
            fd[k] = (orc.affine_loss_grad(f, m, a, loss=loss)[0] -
                     orc.affine_loss_grad(f, m, b, loss=loss)[0]) / (2 * h)
        assert np.abs(g - fd).max() <= 1e-5 * np.abs(fd).max(), (loss, g, fd)


def test_recovers_a_known_affine_map(orc):
    """moving = fixed o phi for a known small affine phi: the registration
    (which aligns moving o psi with fixed) finds psi = phi^-1 to a fraction of
    a voxel, starting 0.68 voxel away."""
    shape = (24, 24, 24)
    f, _, _ = synth.blobs_pair(shape=shape, sigma=3.0)
    A = np.eye(3) + np.array([[0.04, 0.02, 0.0], [-0.01, 0.03, 0.02], [0.0, 0.01, -0.03]])
    t = np.array([0.03, -0.04, 0.02])
    m = orc.warp(f, orc.affine_field(theta_of(A, t), shape), want_grad=False)
    Ai = np.linalg.inv(A)
    expect = orc.affine_field(theta_of(Ai, -Ai @ t), shape)
    r = orc.affine_register(f, m, [2, 1], [150, 80], lr=3e-3, loss="mse")
    err = orc.affine_field(r["theta"], shape) - expect
    inner = (slice(None),) + (slice(3, -3),) * 3
    assert np.sqrt((expect[inner] ** 2).sum(0)).mean() > 0.5
    assert np.sqrt((err[inner] ** 2).sum(0)).mean() < 0.15


def test_register_from_an_affine_start_with_zero_iterations(orc):
    """Starting the deformable stage from an affine displacement: with no
    iterations the result is that displacement, carried through the pyramid
    exactly (align-corners resampling is exact on affine fields)."""
    shape = (13, 15, 17)
    f, m, _ = synth.blobs_pair(shape=shape, sigma=2.5)
    A = np.eye(3) + 0.03 * np.random.default_rng(7).standard_normal((3, 3))
    u0 = orc.affine_field(theta_of(A, [0.02, -0.01, 0.03]), shape)
    r = orc.register(f, m, [2, 1], [0, 0], u_init=u0)
    assert np.allclose(r["u"], u0, rtol=0, atol=1e-12)
    r1 = orc.register(f, m, [1], [0], u_init=u0)
    assert np.array_equal(r1["u"], u0)
