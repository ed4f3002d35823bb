"""The paper's own coarsest-grid solve on the GPU (helm_params.coarse_tol > 0): full GMRES on
M_c e = b from a zero guess to a relative residual of coarse_tol (1e-11 in the paper, Sec. 5),
run by one thread-block cluster, in place of the library's default dense inverse.

- On a hierarchy of one level the V-cycle is the coarse solve alone: its residual is checked
  with the oracle's operator, and it must equal the dense inverse's answer to the tolerance.
- On several hierarchies the whole V- and F-cycle must equal the oracle's cycles with the
  oracle's own coarse GMRES at the same tolerance (both FP64; the two GMRES runs differ in
  rounding and Gram-Schmidt form, so by up to the tolerance times the coarse operator's
  condition number: 1e-7 relative is asked).
- Table 1 (65^3 closed-off, 17-node coarsest grid) with the paper's coarse solver: left GMRES
  and Bi-CGSTAB counts against the oracle run the same way and against the paper's spread.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_06085_gb300 import inputs as I

pytestmark = pytest.mark.gpu

D, S = 0, 1
TOL = 1e-11


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


@pytest.mark.parametrize("n,bc", [((12, 10, 8), S), ((15, 16, 14), D), ((14, 14, 14), S)])
def test_single_level_is_the_coarse_solve(helm, n, bc):
    h = 1.0 / max(n)
    shape = I.unknown_shape(n, bc)
    k2 = I.random_k2(shape, seed=41, kmin=2.0, kmax=0.6 / h)
    r = I.random_vector(shape, 43)
    big = 64  # no level can be halved: the hierarchy is the coarsest grid alone
    s = helm.Solver(n, h, k2, bc, coarsest_n=big, coarse_tol=TOL)
    assert s.nlevels == 1
    e = s.vcycle(dev(r)).cpu().numpy()
    steps, converged = s.coarse_info()
    assert converged and 0 < steps <= min(256, int(np.prod(shape))), (steps, converged)
    again = s.vcycle(dev(r)).cpu().numpy()
    s.close()
    assert np.array_equal(e, again)  # deterministic: every CTA sums the partials in rank order
    me = oracle.apply(e, k2, h, bc, (1.0, 0.5))  # M = -Lap - (1 + 0.5 i) k^2 (beta2 = -0.5)
    assert np.linalg.norm(r - me) <= 2 * TOL * np.linalg.norm(r)
    t = helm.Solver(n, h, k2, bc, coarsest_n=big)
    with pytest.raises(helm.HelmError):
        t.coarse_info()  # the dense inverse keeps no GMRES report
    exact = t.vcycle(dev(r)).cpu().numpy()
    t.close()
    assert rel(e, exact) <= 1e-7  # tol times the coarse operator's condition number, with room


@pytest.mark.parametrize("n,bc,coarsest", [((32, 32, 32), D, 8), ((32, 32, 32), S, 8), ((40, 20, 12), S, 3)])
def test_cycles_match_the_oracle_with_its_coarse_gmres(helm, n, bc, coarsest):
    h = 1.0 / max(n)
    shape = I.unknown_shape(n, bc)
    k2 = I.random_k2(shape, seed=47, kmin=2.0, kmax=0.6 / h)
    r = I.random_vector(shape, 53)
    s = helm.Solver(n, h, k2, bc, coarsest_n=coarsest, coarse_tol=TOL)
    o = oracle.Solver(n, h, bc, k2, coarsest_n=coarsest, coarse_tol=TOL)
    assert s.nlevels > 1
    assert rel(s.vcycle(dev(r)).cpu().numpy(), o.vcycle(r)) <= 1e-7
    assert rel(s.fcycle(dev(r)).cpu().numpy(), o.fcycle(r)) <= 1e-7
    r32 = r.astype(np.complex64)
    assert rel(s.vcycle(dev(r32)).cpu().numpy(), o.vcycle(r32.astype(np.complex128))) <= 2e-5
    s.close()


def test_table1_with_the_papers_coarse_solver(helm):
    """65^3 closed-off problem at k = 40 as the paper runs it: 17-node coarsest grid solved by
    GMRES to 1e-11.  Left GMRES within one of the oracle run the same way and within two of the
    printed 145; Bi-CGSTAB within 10% of the oracle's count (short recurrences move with rounding
    order) and inside the paper's spread over layouts (359-407, Table 1) widened to 0.85x-1.1x."""
    w = I.workload("closed_off", 64)
    assert w["coarsest_n"] == 16
    o = oracle.Solver(64, w["h"], oracle.DIRICHLET, w["k2"], coarsest_n=16, coarse_tol=TOL)
    counts = {}
    for krylov, side in (("gmres", "left"), ("bicgstab", "right")):
        s = helm.Solver(w["n"], w["h"], w["k2"], helm.DIRICHLET, coarsest_n=16, krylov=krylov, restart=200,
                        max_iter=3000, side=side, coarse_tol=TOL)
        _, info = s.solve(dev(w["rhs"]))
        s.close()
        assert info["status"] == 0, info
        counts[krylov] = info["iterations"]
    ro = o.gmres(w["rhs"], restart=400, tol=1e-6, max_iter=400, left=True)
    assert abs(counts["gmres"] - ro["iters"]) <= 1, (counts, ro["iters"])
    assert abs(counts["gmres"] - 145) <= 2, counts
    rb = o.bicgstab(w["rhs"], tol=1e-6, max_iter=2000)
    assert abs(counts["bicgstab"] - rb["iters"]) <= 0.1 * rb["iters"], (counts, rb["iters"])
    assert 0.85 * 359 <= counts["bicgstab"] <= 1.1 * 407, counts


@pytest.mark.parametrize("precision,krylov,cycle", [("mixed", "fgmres", "v"), ("fp64", "gmres", "f"),
                                                    ("fp64", "idrs", "v")])
def test_solves_with_the_coarse_gmres(helm, precision, krylov, cycle):
    """Whole solves (captured in CUDA graphs, the complex64 cycle included) with the coarse GMRES:
    they reach the true relative residual 1e-6 with the oracle's operator, in the iteration count
    of the same solve with the dense coarsest inverse (within one for GMRES, 10% for IDR(s))."""
    w = I.workload("wedge", 32)
    counts = []
    for tol in (TOL, 0.0):
        s = helm.Solver(w["n"], w["h"], w["k2"], S, coarsest_n=8, krylov=krylov, precision=precision, cycle=cycle,
                        coarse_tol=tol, max_iter=3000)
        b = s.rhs_point(w["sources"])
        x, info = s.solve(b)
        s.close()
        assert info["status"] == 0, info
        bn = b.cpu().numpy()
        ax = oracle.apply(x.cpu().numpy(), w["k2"], w["h"], S)
        assert np.linalg.norm(bn - ax) <= 1.01e-6 * np.linalg.norm(bn)
        counts.append(info["iterations"])
    slack = 1 if krylov != "idrs" else max(2, 0.1 * counts[1])
    assert abs(counts[0] - counts[1]) <= slack, counts
