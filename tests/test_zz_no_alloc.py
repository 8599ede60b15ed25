"""fa_lncc_fwd_bwd_noalloc (no workspace argument, built-in device scratch)
gives the same loss and gradients as fa_lncc_fwd_bwd, on two calls in a row
with different inputs, called through the C ABI.  This file sorts last so a
run that stops at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2404_01249_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel(a, b):
    a = a.detach().cpu().double().numpy()
    b = b.detach().cpu().double().numpy()
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


@pytest.fixture(scope="module")
def fa():
    from paper_2404_01249_gb300 import build, fa
    build.build()
    assert torch.cuda.is_available()
    fa.load()
    return fa


def call_noalloc(fa, fixed, warped, window, cc_eps):
    D, H, W = fixed.shape
    loss = torch.empty((), device="cuda")
    dJ = torch.empty_like(fixed)
    dI = torch.empty_like(fixed)
    st = fa.load().fa_lncc_fwd_bwd_noalloc(fa._vol(fixed, 1), fa._vol(warped, 1), window, cc_eps,
                                          fa._ptr(loss), fa._vol(dJ, 1), fa._vol(dI, 1),
                                          fa._stream())
    fa._check(st)
    return loss, dJ, dI


def test_noalloc_matches_workspace_entry_point_twice(fa):
    for k, (shape, window) in enumerate([((40, 48, 56), 5), ((31, 17, 45), 7)]):
        f, m, _ = synth.voronoi_pair(shape=shape, seed=21 + k)
        ft = torch.from_numpy(f).cuda()
        mt = torch.from_numpy(m).cuda()
        loss, dJ, dI = call_noalloc(fa, ft, mt, window, 1e-5)
        ref = fa.fa_lncc_fwd_bwd(ft, mt, window, 1e-5, want_dJ=True, want_dI=True)
        torch.cuda.synchronize()
        assert abs(float(loss) - float(ref["loss"])) <= TOL * abs(float(ref["loss"]))
        assert rel(dJ, ref["dJ"]) <= TOL
        assert rel(dI, ref["dI"]) <= TOL


def test_noalloc_at_its_exact_limit(fa):
    """64 x 133 x 73 = 621,376 voxels fill the 64 MiB scratch with no slack;
    the result still equals the workspace entry point's."""
    shape = (64, 133, 73)
    assert fa.load().fa_lncc_workspace_size(*shape) == 64 << 20
    f, m, _ = synth.voronoi_pair(shape=shape, seed=23)
    ft, mt = torch.from_numpy(f).cuda(), torch.from_numpy(m).cuda()
    loss, dJ, dI = call_noalloc(fa, ft, mt, 5, 1e-5)
    ref = fa.fa_lncc_fwd_bwd(ft, mt, 5, 1e-5, want_dJ=True, want_dI=True)
    torch.cuda.synchronize()
    assert abs(float(loss) - float(ref["loss"])) <= TOL * abs(float(ref["loss"]))
    assert rel(dJ, ref["dJ"]) <= TOL
    assert rel(dI, ref["dI"]) <= TOL


@pytest.mark.parametrize("shape", [(64, 133, 74), (100, 100, 100)])
def test_noalloc_rejects_grids_beyond_its_scratch(fa, shape):
    big = torch.empty(shape, device="cuda")
    with pytest.raises(fa.FAError) as e:
        call_noalloc(fa, big, big, 5, 1e-5)
    assert e.value.status == 2
    assert "621376" in str(e.value)
