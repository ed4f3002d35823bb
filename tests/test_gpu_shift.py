"""GPU parity of the CSLP shift sweep (Sec. 5.1.4: beta2 from -0.5 to -1, V- and F-cycle):
at beta2 = -0.75 and -1 the preconditioner M = -Lap - (beta1 - beta2 i) k^2 on every level,
one V-cycle and one F-cycle, and GMRES solves preconditioned by either, against the FP64 CPU
oracle with the same shift.

Tolerances as for the paper's own shift (beta2 = -0.5) in test_gpu_parity.py: FP64 cycles
1e-12 relative, complex64 cycles 2e-5 (V) and 4e-5 (F), solves #Matvec within +-1 of the
oracle and solutions within 1e-5, with the true residual checked by the oracle's operator."""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_06085_gb300 import inputs as I

pytestmark = pytest.mark.gpu

D, S = 0, 1
CASES = [
    ("dir_ragged", (40, 20, 12), D, 2),
    ("som_ragged", (40, 20, 12), S, 2),
    ("som_noncubic", (24, 8, 16), S, 2),
]
SHIFTS = [-0.75, -1.0]


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2308_06085_gb300 import helm as h

    torch.cuda.set_device(0)
    return h


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def make(helm, name, n, bc, coarsest, beta2, **kw):
    h = 1.0 / max(n)
    shape = I.unknown_shape(n, bc)
    k2 = I.random_k2(shape, seed=sum(map(ord, name)), kmin=2.0, kmax=0.6 / h)
    s = helm.Solver(n, h, k2, bc, coarsest_n=coarsest, beta2=beta2, **kw)
    o = oracle.Solver(n, h, bc, k2, coarsest_n=coarsest, beta2=beta2)
    return s, o, shape, k2, h


@pytest.mark.parametrize("beta2", SHIFTS)
@pytest.mark.parametrize("name,n,bc,coarsest", CASES)
def test_shifted_cycles(helm, name, n, bc, coarsest, beta2):
    s, o, shape, k2, h = make(helm, name, n, bc, coarsest, beta2)
    r = I.random_vector(shape, 31)
    # the shifted operator M = -Lap - (1 - beta2 i) k^2 itself
    v = s.apply(dev(r), "M").cpu().numpy()
    assert rel(v, oracle.apply(r, k2, h, bc, (1.0, -beta2))) <= 1e-12
    assert rel(s.vcycle(dev(r)).cpu().numpy(), o.vcycle(r)) <= 1e-12
    assert rel(s.fcycle(dev(r)).cpu().numpy(), o.fcycle(r)) <= 1e-12
    r32 = r.astype(np.complex64)
    r64 = r32.astype(np.complex128)
    assert rel(s.vcycle(dev(r32)).cpu().numpy(), o.vcycle(r64)) <= 2e-5
    assert rel(s.fcycle(dev(r32)).cpu().numpy(), o.fcycle(r64)) <= 4e-5


@pytest.mark.parametrize("beta2", SHIFTS)
@pytest.mark.parametrize("cycle", ["v", "f"])
def test_shifted_gmres_vs_oracle(helm, beta2, cycle):
    """GMRES(30) on the n = 32 wedge with the shifted CSLP, V- or F-cycle."""
    w = I.workload("wedge", 32)
    s = helm.Solver(w["n"], w["h"], w["k2"], S, beta2=beta2, cycle=cycle)
    o = oracle.Solver(w["n"], w["h"], S, w["k2"], beta2=beta2, cycle=cycle)
    b = s.rhs_point(w["sources"])
    x, info = s.solve(b)
    bn = b.cpu().numpy()
    ro = o.gmres(bn, restart=30, tol=1e-6)
    assert info["status"] == 0 and ro["status"] == 0
    assert abs(info["iterations"] - ro["iters"]) <= 1, (info, ro["iters"])
    assert rel(x.cpu().numpy(), ro["x"]) <= 1e-5
    ax = oracle.apply(x.cpu().numpy(), w["k2"], w["h"], S)
    assert np.linalg.norm(bn - ax) / np.linalg.norm(bn) <= 1.01e-6
