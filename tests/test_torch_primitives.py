"""The PyTorch-primitives form of the iteration (`bench.py --mode torch`, a
comparison point for the benchmark) follows the oracle's registration: one
level and two levels on a small Voronoi pair, on the CPU.  The bounds are
looser than the library's (final LNCC 1e-2, mean displacement 0.15 voxel):
its pyramid blur and resampling are PyTorch's conv3d and interpolate, and
its float32 rounding differs from the exact window sums."""
import numpy as np
import pytest
import torch

import bench
from paper_2404_01249_gb300 import synth


@pytest.mark.parametrize("scales,iters", [((1,), (12,)), ((2, 1), (10, 6))])
def test_torch_primitives_form_matches_oracle(orc, scales, iters):
    f, m, _ = synth.voronoi_pair(shape=(14, 16, 18), seed=5)
    u, cc = bench._torch_register(torch.from_numpy(f), torch.from_numpy(m), scales, iters,
                                  0.5, 1.0, 0.5, 5, 1e-5)
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    ref = orc.register(f, m, list(scales), list(iters), cc_eps=f32(1e-5), beta1=f32(0.9),
                       beta2=f32(0.999), adam_eps=f32(1e-8))
    assert abs(cc + ref["final_loss"]) < 1e-2
    d = u.double().numpy() - ref["u"]
    assert float(np.sqrt((d ** 2).sum(0)).mean()) < 0.15
