"""Pins for the oracle's Gaussian smoothing (sigma_grad / sigma_warp of the
hyper-parameter study), Adam (Kingma & Ba, used on the tangent-space
directions of section "Adaptive optimization on diffeomorphisms") and the
step scaling of the appendix "Limitations of Stationary Velocity Fields"."""
import json
import math
import os

import numpy as np
import pytest
from scipy.ndimage import gaussian_filter

from conftest import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("sigma", [0.4, 0.5, 1.0, 2.0, 6.0])
def test_taps(orc, sigma):
    t = orc.gauss_taps(sigma)
    R = math.ceil(3 * sigma)
    assert len(t) == 2 * R + 1
    assert abs(t.sum() - 1.0) < 1e-15
    assert np.allclose(t, t[::-1], rtol=0, atol=0)
    k = np.arange(-R, R + 1)
    assert np.allclose(t / t[R], np.exp(-k ** 2 / (2 * sigma ** 2)), rtol=1e-14)


def test_zero_sigma_is_identity(orc):
    x = rng(30).standard_normal((3, 4, 5, 6))
    assert np.array_equal(orc.gauss_smooth(x, 0.0), x)


@pytest.mark.parametrize("sigma", [0.5, 1.0, 2.0])
def test_matches_scipy_zero_padded(orc, sigma):
    x = rng(31).standard_normal((2, 9, 11, 13))
    R = math.ceil(3 * sigma)
    out = orc.gauss_smooth(x, sigma)
    for c in range(2):
        ref = gaussian_filter(x[c], sigma, mode="constant", cval=0.0, truncate=R / sigma)
        assert np.allclose(out[c], ref, atol=1e-13)


def test_separable_equals_direct_3d_and_impulse(orc):
    sigma = 1.0
    t = orc.gauss_taps(sigma)
    R = len(t) // 2
    shape = (7, 8, 9)
    x = rng(32).standard_normal(shape)
    kern = t[:, None, None] * t[None, :, None] * t[None, None, :]
    pad = np.pad(x, R)
    ref = np.zeros(shape)
    for a in range(2 * R + 1):
        for b in range(2 * R + 1):
            for c in range(2 * R + 1):
                ref += kern[a, b, c] * pad[a:a + shape[0], b:b + shape[1], c:c + shape[2]]
    assert np.allclose(orc.gauss_smooth(x, sigma), ref, atol=1e-13)
    imp = np.zeros((9, 9, 9))
    imp[4, 4, 4] = 1.0
    resp = orc.gauss_smooth(imp, sigma)
    assert np.allclose(resp[4 - R:5 + R, 4 - R:5 + R, 4 - R:5 + R], kern, atol=1e-16)
    assert abs(resp.sum() - 1.0) < 1e-14


def test_constant_preserved_away_from_border(orc):
    x = np.full((12, 12, 12), 3.25)
    out = orc.gauss_smooth(x, 1.0)
    assert np.allclose(out[3:-3, 3:-3, 3:-3], 3.25, rtol=1e-15)
    assert out[0, 0, 0] < 3.25   # zero padding at the border


def test_adam_matches_torch(orc):
    torch = pytest.importorskip("torch")
    shape = (3, 4, 5, 6)
    r = rng(33)
    p = torch.zeros(shape, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=1.0, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(shape)
    v = np.zeros(shape)
    for t in range(1, 8):
        g = r.standard_normal(shape) * 10.0 ** r.uniform(-8, 1)
        before = p.detach().clone()
        p.grad = torch.from_numpy(g.copy())
        opt.step()
        d_torch = (before - p.detach()).numpy()
        d, m, v = orc.adam(g, m, v, t)
        assert np.allclose(d, d_torch, rtol=1e-12, atol=1e-14)


def test_adam_condition_number_invariance():
    """Appendix "On the Ill-conditioning of Image Registration": on
    f(x, y) = x_t^2 + kappa y_t^2 rotated by theta = pi/3, Adam from (5, 5)
    ends within 1e-3 of the minimum after 1000 steps for kappa = 1000.  The
    learning rate is not printed; the fixture fixes one."""
    import oracle
    with open(os.path.join(GOLDEN, "adam_toy.json")) as f:
        gold = json.load(f)
    th = gold["theta"]
    Rm = np.array([[math.cos(th), math.sin(th)], [-math.sin(th), math.cos(th)]])
    for kappa in gold["kappas"]:
        Hm = Rm.T @ np.diag([2.0, 2.0 * kappa]) @ Rm
        x = np.array(gold["start"], dtype=np.float64)
        m = np.zeros(2)
        v = np.zeros(2)
        for t in range(1, gold["iterations"] + 1):
            g = Hm @ x
            d, m, v = oracle.adam(g, m, v, t)
            x = x - gold["lr"] * d
        assert np.linalg.norm(x) < gold["max_final_distance"], (kappa, np.linalg.norm(x))


def test_step_scale_bounds_max_step(orc):
    d = rng(34).standard_normal((3, 5, 6, 7))
    for eta in (0.25, 0.5, 1.0):
        delta, e = orc.step_scale(d, eta, 2.0)
        n = np.sqrt((delta ** 2).sum(axis=0))
        assert abs(n.max() - eta / 2.0) < 1e-15
        assert np.allclose(delta, -e * d, rtol=0, atol=0)
        assert e > 0
    delta, e = orc.step_scale(np.zeros((3, 2, 2, 2)), 0.5, 2.0)
    assert e == 0.0 and not delta.any()


def test_max_norm(orc):
    d = np.zeros((3, 2, 3, 4))
    d[:, 1, 2, 3] = [3.0, 4.0, 12.0]
    d[:, 0, 0, 0] = [-5.0, 0.0, 0.0]
    assert orc.max_norm(d) == 13.0
