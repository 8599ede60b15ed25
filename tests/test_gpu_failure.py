"""Failure detection on the GPU without a fault: the bounded wait the fused
kernels use for their tile copies gives up on a barrier that nothing
completes, records a timeout in the workspace status word, and the context
stays usable for the next registration."""
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


@pytest.mark.parametrize("limit", [0, 1 << 20])
def test_bounded_wait_reports_timeout(fa, limit):
    assert fa.fa_selftest_wait_timeout(limit) == fa.FA_ERR_TIMEOUT


def test_context_usable_after_timeout(fa):
    assert fa.fa_selftest_wait_timeout(1 << 16) == fa.FA_ERR_TIMEOUT
    f, m, _ = synth.blobs_pair(shape=(16, 18, 20), sigma=2.5)
    out = fa.fa_register(torch.from_numpy(f).cuda(), torch.from_numpy(m).cuda(),
                         fa.RegParams(scales=(2, 1), iters=(5, 5)))
    assert np.isfinite(out["final_loss"]) and torch.isfinite(out["u"]).all()


def test_invalid_limit(fa):
    with pytest.raises(fa.FAError):
        fa.fa_selftest_wait_timeout(-1)
