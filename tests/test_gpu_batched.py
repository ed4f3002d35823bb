"""Batched right-hand sides (helm_solve_batched): every right-hand side of a lockstep
batched FGMRES(30) against the same right-hand side solved alone, and against the FP64
oracle.  Widths that need padding (3 -> 4), a full 32-wide chunk and two chunks (33) are
covered, in FP64 and in mixed precision.

Tolerances: true relative residual <= 1e-6 for every right-hand side; iteration counts within
+-1 of the single solve (the batched second Gram-Schmidt pass is taken when any right-hand side
needs it, which changes rounding only); solutions within 1e-5 of the single solve and, in
FP64, of the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_06085_gb300 import inputs as I

pytestmark = pytest.mark.gpu
S = 1


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2308_06085_gb300 import helm as h

    torch.cuda.set_device(0)
    return h


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def sources(n, count):
    grid = I.source_grid(n, 4, 8, 0.1)
    return [grid[i % len(grid)] if i < len(grid) else (n // 2, n // 2, (i * 3) % (n + 1)) for i in range(count)]


@pytest.mark.parametrize("orth", ["fp64", "df"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("count", [3, 8])
def test_batched_matches_single(helm, precision, count, orth):
    w = I.workload("batched", 32)
    s = helm.Solver(w["n"], w["h"], w["k2"], S, krylov="fgmres", precision=precision, orth=orth)
    src = sources(32, count)
    B = torch.stack([s.rhs_point([p]) for p in src])
    X, infos = s.solve_batched(B)
    for r in range(count):
        x1, i1 = s.solve(B[r])
        assert infos[r]["status"] == 0 and infos[r]["rel_residual"] <= 1e-6, infos[r]
        assert abs(infos[r]["iterations"] - i1["iterations"]) <= 1, (r, infos[r], i1)
        assert rel(X[r].cpu().numpy(), x1.cpu().numpy()) <= 1e-5
        # the residual, with the oracle's operator
        ax = oracle.apply(X[r].cpu().numpy(), w["k2"], w["h"], S)
        b = B[r].cpu().numpy()
        assert np.linalg.norm(b - ax) / np.linalg.norm(b) <= 1.01e-6


def test_batched_fp64_matches_oracle(helm):
    w = I.workload("batched", 16)
    s = helm.Solver(w["n"], w["h"], w["k2"], S, krylov="fgmres")
    o = oracle.Solver(w["n"], w["h"], S, w["k2"])
    src = sources(16, 4)
    B = torch.stack([s.rhs_point([p]) for p in src])
    X, infos = s.solve_batched(B)
    for r in range(4):
        ro = o.gmres(B[r].cpu().numpy(), restart=30, tol=1e-6, flexible=True)
        assert abs(infos[r]["iterations"] - ro["iters"]) <= 1
        assert rel(X[r].cpu().numpy(), ro["x"]) <= 1e-5


def test_batched_two_chunks_and_warm_start(helm):
    w = I.workload("batched", 16)
    s = helm.Solver(w["n"], w["h"], w["k2"], S, krylov="fgmres", precision="mixed")
    src = sources(16, 33)
    B = torch.stack([s.rhs_point([p]) for p in src])
    X, infos = s.solve_batched(B)
    assert all(i["status"] == 0 and i["rel_residual"] <= 1e-6 for i in infos)
    x1, _ = s.solve(B[32])
    assert rel(X[32].cpu().numpy(), x1.cpu().numpy()) <= 1e-5
    # warm start from the solutions: nothing left to do
    X2, infos2 = s.solve_batched(B, X.clone())
    assert all(i["iterations"] == 0 for i in infos2)
    # a zero right-hand side inside a batch
    B[1].zero_()
    X3, infos3 = s.solve_batched(B[:4])
    assert infos3[1]["iterations"] == 0 and torch.count_nonzero(X3[1]) == 0
    assert infos3[0]["rel_residual"] <= 1e-6


def test_batched_fcycle_matches_single(helm):
    """The batched solver with F-cycle preconditioning against the same right-hand sides solved
    one at a time with the F-cycle (mixed precision, double-float Gram-Schmidt)."""
    w = I.workload("batched", 32)
    s = helm.Solver(w["n"], w["h"], w["k2"], S, krylov="fgmres", precision="mixed", orth="df", cycle="f")
    src = sources(32, 5)
    B = torch.stack([s.rhs_point([p]) for p in src])
    X, infos = s.solve_batched(B)
    for r in range(5):
        x1, i1 = s.solve(B[r])
        assert infos[r]["status"] == 0 and infos[r]["rel_residual"] <= 1e-6, infos[r]
        assert abs(infos[r]["iterations"] - i1["iterations"]) <= 1, (r, infos[r], i1)
        assert rel(X[r].cpu().numpy(), x1.cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_summed_basis_matches_textbook(helm, precision):
    """Batched FP64 Gram-Schmidt against the summed basis (three FMAs per complex multiply-add,
    the default) and in the textbook four-FMA form: the same solves to 1e-10, so #Matvec within
    +-1 and solutions within 1e-8 for every right-hand side; the default also against the oracle."""
    w = I.workload("batched", 16)
    src = sources(16, 6)
    out = []
    for sums in (True, False):
        s = helm.Solver(w["n"], w["h"], w["k2"], S, krylov="fgmres", precision=precision, gs_sums=sums, tol=1e-10,
                        max_iter=4000)
        B = torch.stack([s.rhs_point([p]) for p in src])
        X, infos = s.solve_batched(B)
        assert all(i["status"] == 0 and i["rel_residual"] <= 1e-10 for i in infos)
        out.append((X.cpu().numpy(), [i["iterations"] for i in infos], B.cpu().numpy()))
        s.close()
    (xa, ia, B), (xb, ib, _) = out
    for r in range(len(src)):
        assert abs(ia[r] - ib[r]) <= 1, (r, ia, ib)
        assert rel(xa[r], xb[r]) <= 1e-8
    if precision == "fp64":
        o = oracle.Solver(w["n"], w["h"], S, w["k2"])
        for r in range(2):
            ro = o.gmres(B[r], restart=30, tol=1e-10, max_iter=4000, flexible=True)
            assert abs(ia[r] - ro["iters"]) <= 1 and rel(xa[r], ro["x"]) <= 1e-8
