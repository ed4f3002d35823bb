"""The FP32 -> FP64 conversion the FP64 kernels use on complex64 data is written with integer
instructions from the IEEE-754 layouts (a converting instruction issues on this GPU's FP64
pipe).  It must give the hardware conversion's bits for every input: random bit patterns over
the whole range (zeros, subnormals, infinities and NaNs included), both zeros and the extremes
of the normal range."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2308_06085_gb300 import helm as h

    torch.cuda.set_device(0)
    return h


def test_conversion_matches_the_hardware_bit_for_bit(helm):
    rng = np.random.default_rng(2308)
    bits = rng.integers(0, 2 ** 32, size=1 << 23, dtype=np.uint64).astype(np.uint32)
    fi = np.finfo(np.float32)
    edges = np.array([0.0, -0.0, 1.0, -1.0, fi.max, -fi.max, fi.tiny, -fi.tiny, fi.tiny / 2, fi.smallest_subnormal,
                      np.inf, -np.inf, np.nan, 0.1, 3.0e-39], dtype=np.float32)
    x = torch.from_numpy(np.concatenate([bits.view(np.float32), edges])).cuda()
    got = helm.convert_check(x)
    ref = x.to(torch.float64)  # the hardware conversion
    same = (got.view(torch.int64) == ref.view(torch.int64)) | (torch.isnan(got) & torch.isnan(ref))
    assert int((~same).sum()) == 0, x[~same][:8]
    assert int(torch.isnan(x).sum()) > 0 and int((x.abs() < fi.tiny).sum()) > 2  # the slow path ran too
