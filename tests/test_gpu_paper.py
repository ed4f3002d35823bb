"""The paper's own numbers for the 3D closed-off problem (Sec. 2.1, k = 40) reproduced by the
GPU path through the C ABI, in the paper's configuration: coarsest grid by the 17-node rule
(Sec. 4.2), full GMRES preconditioned from the left with the preconditioned stopping rule, and
Bi-CGSTAB / IDR(4) on the true residual (Sec. 5), all in FP64.

- Table 1 (65^3 nodes): the GPU's #Matvec against the oracle's on the same inputs (GMRES within
  +-1, the short-recurrence methods within 10%, since their counts move with rounding order) and
  against the paper's spread over processor layouts, widened by 10% (IDR(4)) and 20% / 10%
  (Bi-CGSTAB, whose count the paper shows moving by 13% with the layout alone).
- Table 2 (129^3, 193^3 and 257^3 nodes): against the oracle's counts on the same inputs, stored
  by tests/golden/make_closed_off_counts.py because the oracle takes up to half an hour there
  (GMRES within +-1, IDR(4) within 10%), and against the paper's (GMRES within 5%, IDR(4) within
  10%).  The oracle reproduces the paper's 146 at 129^3 and 143 at 257^3 exactly but takes 140
  where the paper prints 137 at 193^3, which the 5% admits.
- Sec. 5.1.1: the solution equals the closed-form discrete solution and converges to the
  analytic one at second order in h.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2308_06085_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def table1():
    return {r[0]: [int(v) for v in r[1:]] for r in golden_rows("table1_matvec.txt")}


def table2():
    return {int(r[0]) - 1: dict(gmres=int(r[2]), idr4=int(r[4]))
            for r in golden_rows("weak_scaling_matvec.txt") if r[0] != "per_iter"}


def oracle_counts():
    """The oracle's counts at the Table 2 sizes, written by make_closed_off_counts.py."""
    return {int(r[0]) - 1: dict(gmres=int(r[1]), idr4=int(r[2])) for r in golden_rows("closed_off_oracle_counts.txt")}


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2308_06085_gb300 import helm as h

    torch.cuda.set_device(0)
    return h


def gpu_solver(helm, w, krylov, side="right", restart=200, **kw):
    return helm.Solver(w["n"], w["h"], w["k2"], helm.DIRICHLET, coarsest_n=w["coarsest_n"], krylov=krylov,
                       restart=restart, max_iter=3000, side=side, **kw)


def gpu_count(helm, w, krylov, side="right"):
    s = gpu_solver(helm, w, krylov, side)
    try:
        _, info = s.solve(torch.from_numpy(w["rhs"]).cuda())
    finally:
        s.close()
    assert info["status"] == 0, info
    return info["iterations"]


def test_table1_counts(helm):
    w = I.workload("closed_off", 64)
    assert w["coarsest_n"] == 16
    o = oracle.Solver(64, w["h"], oracle.DIRICHLET, w["k2"], coarsest_n=16)
    t = table1()
    shape = w["k2"].shape

    g = gpu_count(helm, w, "gmres", "left")
    ro = o.gmres(w["rhs"], restart=400, tol=1e-6, max_iter=400, left=True)
    assert abs(g - ro["iters"]) <= 1, (g, ro["iters"])
    assert abs(g - t["GMRES"][0]) <= 2, g

    g = gpu_count(helm, w, "idrs")
    ro = o.idrs(w["rhs"], I.shadow_space(shape, 4), tol=1e-6, max_iter=2000)
    assert abs(g - ro["iters"]) <= 0.1 * ro["iters"], (g, ro["iters"])
    assert 0.9 * min(t["IDR(4)"]) <= g <= 1.1 * max(t["IDR(4)"]), g

    # Bi-CGSTAB's count moves most with rounding order (Sec. 5.1.3: 359-407 over layouts) and with
    # the coarsest-grid solve: the library solves it exactly, where the paper runs GMRES to 1e-11,
    # and the oracle measures 321 products exactly against 347 with the paper's coarse solver
    # (test_oracle_paper); the coarsest inverse alone, eliminated in another order, moves the
    # GPU's count by 5%.  Hence the lower bound of 0.8 of the paper's smallest count.
    g = gpu_count(helm, w, "bicgstab")
    ro = o.bicgstab(w["rhs"], tol=1e-6, max_iter=2000)
    assert abs(g - ro["iters"]) <= 0.1 * ro["iters"], (g, ro["iters"])
    assert 0.8 * min(t["Bi-CGSTAB"]) <= g <= 1.1 * max(t["Bi-CGSTAB"]), g


@pytest.mark.parametrize("n", [128, 192, 256])
def test_table2_counts(helm, n):
    w = I.workload("closed_off", n)
    assert w["coarsest_n"] == {128: 16, 192: 12, 256: 16}[n]
    t, o = table2()[n], oracle_counts()[n]
    g = gpu_count(helm, w, "gmres", "left")
    i = gpu_count(helm, w, "idrs")
    assert abs(g - o["gmres"]) <= 1, (g, o)
    assert abs(i - o["idr4"]) <= 0.1 * o["idr4"], (i, o)
    assert abs(g - t["gmres"]) <= 0.05 * t["gmres"], (g, t)
    assert abs(i - t["idr4"]) <= 0.1 * t["idr4"], (i, t)


def test_closed_off_solution_against_closed_forms(helm):
    """Sec. 5.1.1 validates the solver on the closed-off problem, whose analytic solution is
    u = S + 1 with S = sin(pi x1) sin(2 pi x2) sin(4 pi x3).  S is an eigenvector of the 7-point
    Laplacian with Dirichlet data (eigenvalue lam_h = sum over m in (1, 2, 4) of
    (4 / h^2) sin^2(m pi h / 2)) and the constant 1 is annihilated by it, so the discrete
    solution is u_h = 1 + a S with a = (21 pi^2 - k^2) / (lam_h - k^2).  Solved to 1e-10, the GPU
    solution must match u_h to 1e-6 and its error against u must fall by four when h halves."""
    k = 40.0
    errs = []
    for n in (64, 128, 256):
        w = I.workload("closed_off", n)
        s = gpu_solver(helm, w, "gmres", restart=200, tol=1e-10)
        try:
            x, info = s.solve(torch.from_numpy(w["rhs"]).cuda())
        finally:
            s.close()
        assert info["status"] == 0 and info["rel_residual"] <= 1e-10, info
        h = 1.0 / n
        c = np.arange(1, n) * h
        S = np.sin(4 * np.pi * c)[:, None, None] * np.sin(2 * np.pi * c)[None, :, None] * np.sin(np.pi * c)[None, None, :]
        lam = sum(4.0 / h ** 2 * np.sin(m * np.pi * h / 2) ** 2 for m in (1, 2, 4))
        u_h = 1.0 + (21 * np.pi ** 2 - k * k) / (lam - k * k) * S
        xh = x.cpu().numpy()
        assert np.abs(xh - u_h).max() <= 1e-6, (n, np.abs(xh - u_h).max())
        errs.append(float(np.abs(xh - (S + 1.0)).max()))
        del x
        torch.cuda.empty_cache()
    for coarse, fine in zip(errs, errs[1:]):
        assert 3.8 <= coarse / fine <= 4.2, errs
