"""The allocation-free entry point helm_vcycle_down_noalloc.

It serves callers that may not allocate device memory themselves (their framework's pool
owns every allocation).  It must give the same coarse right-hand side as the context-based
stage helm_vcycle_stage(level 0, stage 0), within the FP64 tolerance used for every stage
(1e-12 relative), on two calls in a row: the static scratch array is shared by all calls,
so the second call must not see anything left by the first.  This file is collected last
so that a run stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2308_06085_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2308_06085_gb300 import helm as h

    torch.cuda.set_device(0)
    return h


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,bc", [((32, 24, 40), 1), ((16, 16, 16), 0)])
def test_noalloc_matches_stage_twice(helm, n, bc):
    h = 1.0 / max(n)
    shape = I.unknown_shape(n, bc)
    k2 = I.random_k2(shape, seed=17, kmin=2.0, kmax=0.6 / h)
    s = helm.Solver(n, h, k2, bc, coarsest_n=2)
    k2d = torch.from_numpy(k2).cuda()
    for call, seed in enumerate((101, 202)):
        b = torch.from_numpy(I.random_vector(shape, seed)).cuda()
        want = s.vcycle_stage(0, 0, b).cpu().numpy()
        # through the C ABI directly
        cshape = want.shape
        out = torch.full(cshape, float("nan"), dtype=torch.complex128, device="cuda")
        st = helm.lib().helm_vcycle_down_noalloc(n[0], n[1], n[2], h, C.c_void_p(k2d.data_ptr()), bc, 1.0, -0.5, 0.8,
                                                 C.c_void_p(b.data_ptr()), C.c_void_p(out.data_ptr()),
                                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == helm.OK, helm.lib().helm_last_error(None)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel(got, want) <= 1e-12, (call, rel(got, want))
        # and through the binding
        got2 = helm.vcycle_down_noalloc(n, h, k2d, b, bc=bc).cpu().numpy()
        assert rel(got2, want) <= 1e-12


def test_noalloc_rejects_oversize_and_odd_grids(helm):
    k2 = torch.ones(1, dtype=torch.float64, device="cuda")
    b = torch.zeros(1, dtype=torch.complex128, device="cuda")
    o = torch.zeros(1, dtype=torch.complex128, device="cuda")
    args = (0.01, C.c_void_p(k2.data_ptr()), 1, 1.0, -0.5, 0.8, C.c_void_p(b.data_ptr()), C.c_void_p(o.data_ptr()),
            None)
    st = helm.lib().helm_vcycle_down_noalloc(64, 64, 64, *args)  # 65^3 > 262144 unknowns
    assert st == helm.EINVAL and b"static scratch limit" in helm.lib().helm_last_error(None)
    st = helm.lib().helm_vcycle_down_noalloc(15, 16, 16, *args)
    assert st == helm.EINVAL
