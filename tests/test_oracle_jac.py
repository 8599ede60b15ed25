"""The steepest Eulerian descent direction J(phi)^T dL/dphi (use_jac,
section "Exploiting the group structure of diffeomorphisms") in the oracle:
pinned to the identity, to NumPy's finite-difference gradient (a library
routine the oracle does not use) and to the closed form for affine maps."""
import numpy as np

from conftest import rng
from paper_2404_01249_gb300 import synth


def test_zero_displacement_leaves_the_gradient(orc):
    g = rng(1).standard_normal((3, 5, 6, 7))
    assert np.array_equal(orc.jac_direction(g, np.zeros_like(g)), g)


def test_matches_numpy_gradient(orc):
    shape = (6, 7, 9)
    g = rng(2).standard_normal((3,) + shape)
    u = synth.random_field(shape, 1.5, 2.0, seed=3).astype(np.float64)
    grads = [np.gradient(u[j], axis=a) for j in range(3) for a in range(3)]  # d u_j / d x_a
    du = np.array(grads).reshape(3, 3, *shape)                               # [j][a]
    ref = g + np.einsum("ja...,j...->a...", du, g)
    assert np.allclose(orc.jac_direction(g, u), ref, rtol=0, atol=1e-13)


def test_affine_map_closed_form(orc):
    shape = (5, 6, 7)
    z, y, x = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    X = np.stack([z, y, x])
    A = 0.1 * rng(4).standard_normal((3, 3))
    u = np.einsum("jb,b...->j...", A, X) + np.array([0.3, -0.2, 0.1])[:, None, None, None]
    g = rng(5).standard_normal((3,) + shape)
    # J = I + A everywhere (differences are exact on linear functions): out = (I + A)^T g
    ref = np.einsum("ja,j...->a...", np.eye(3) + A, g)
    assert np.allclose(orc.jac_direction(g, u), ref, rtol=0, atol=1e-12)


def test_register_with_jacobian_direction_improves(orc):
    f, m, _ = synth.blobs_pair(shape=(16, 16, 16), sigma=2.5)
    init = orc.lncc(f, m, 5, 1e-5, want_dJ=False)["loss"]
    r = orc.register(f, m, [2, 1], [20, 10], use_jac=True)
    assert r["final_loss"] < init - 0.02
    plain = orc.register(f, m, [2, 1], [20, 10])
    assert not np.array_equal(r["u"], plain["u"])
