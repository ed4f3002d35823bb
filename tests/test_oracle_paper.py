"""The paper's own iteration counts as a soft pin of the whole method (operator, CSLP shift,
V-cycle, transfers, Krylov methods and their stopping rules): Table 1 of Sec. 5.1.3, the 3D
closed-off problem at 65^3 nodes and k = 40.

The oracle runs the paper's configuration: coarsest grid 17^3 nodes (coarsest_n = 16
intervals, which is the paper's 17-node rule on this grid), left-preconditioned full GMRES with
the preconditioned stopping rule, and Bi-CGSTAB / IDR(4) on the true residual.  GMRES is
insensitive to rounding order (the paper prints 145 for every layout) and must land within
+-2 of it.  Bi-CGSTAB and IDR(4) move with rounding order and, for IDR, the random shadow
space (the paper's counts spread 359-407 and 192-211 across layouts); they must fall inside
that spread widened by 15% / 10%.  The coarsest solve is exact here where the paper runs GMRES
to 1e-11 on it, a difference far below the outer tolerance.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2308_06085_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_matvec.txt")


def table1():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, *vals = line.split()
            out[name] = [int(v) for v in vals]
    return out


@pytest.fixture(scope="module")
def closed_off():
    n, k = 64, 40.0
    shape = I.unknown_shape(n, oracle.DIRICHLET)
    o = oracle.Solver(n, 1.0 / n, oracle.DIRICHLET, np.full(shape, k * k), coarsest_n=16)
    assert o.nlevels == 3 and o.level(2)["n"] == (16, 16, 16)
    return o, oracle.rhs_closed_off(n, k), shape


@pytest.mark.slow
def test_table1_gmres(closed_off):
    o, b, _ = closed_off
    r = o.gmres(b, restart=400, tol=1e-6, max_iter=400, left=True)
    assert r["status"] == 0
    assert abs(r["iters"] - table1()["GMRES"][0]) <= 2, r["iters"]


@pytest.mark.slow
def test_table1_idr4(closed_off):
    o, b, shape = closed_off
    r = o.idrs(b, I.shadow_space(shape, 4), tol=1e-6, max_iter=2000)
    t = table1()["IDR(4)"]
    assert r["status"] == 0
    assert 0.9 * min(t) <= r["iters"] <= 1.1 * max(t), r["iters"]


@pytest.mark.slow
def test_table1_bicgstab(closed_off):
    o, b, _ = closed_off
    r = o.bicgstab(b, tol=1e-6, max_iter=2000)
    t = table1()["Bi-CGSTAB"]
    assert r["status"] == 0
    assert 0.85 * min(t) <= r["iters"] <= 1.1 * max(t), r["iters"]


@pytest.mark.slow
def test_table1_gmres_with_the_papers_coarse_solver():
    """The paper solves the 17^3 coarsest grid by full GMRES to 1e-11 (Sec. 5) where the
    default oracle and the library solve it exactly; with the paper's coarse solver the count stays at Table 1's."""
    n, k = 64, 40.0
    shape = I.unknown_shape(n, oracle.DIRICHLET)
    o = oracle.Solver(n, 1.0 / n, oracle.DIRICHLET, np.full(shape, k * k), coarsest_n=16, coarse_tol=1e-11)
    r = o.gmres(oracle.rhs_closed_off(n, k), restart=400, tol=1e-6, max_iter=400, left=True)
    assert r["status"] == 0
    assert abs(r["iters"] - table1()["GMRES"][0]) <= 2, r["iters"]


@pytest.mark.slow
def test_table1_bicgstab_with_the_papers_coarse_solver():
    """Bi-CGSTAB's count depends on the coarsest-grid solve: with the exact solve the oracle
    takes 321 products with A, 11% under the paper's 359 on one process (Table 1), while with
    the paper's own coarse solver, full GMRES to 1e-11 (Sec. 5), it takes 347, inside the spread
    the paper prints over its processor layouts (359-407) widened by 5%.  GMRES, whose count is
    insensitive to this (previous test), and IDR(4) agree either way."""
    n, k = 64, 40.0
    shape = I.unknown_shape(n, oracle.DIRICHLET)
    o = oracle.Solver(n, 1.0 / n, oracle.DIRICHLET, np.full(shape, k * k), coarsest_n=16, coarse_tol=1e-11)
    r = o.bicgstab(oracle.rhs_closed_off(n, k), tol=1e-6, max_iter=2000)
    t = table1()["Bi-CGSTAB"]
    assert r["status"] == 0
    assert 0.95 * min(t) <= r["iters"] <= 1.05 * max(t), r["iters"]


def test_seventeen_node_rule():
    """Sec. 4.2's coarsening stop, on the grids the paper names: the closed-off cubes of
    Tables 1-2 and the salt grid, whose coarsest grid the paper gives as 41 x 41 x 13 nodes
    (Sec. 5.1.2).  With coarsest_n = m, a direction of n intervals halves while the shortest
    one stays >= m, so the salt grid's 640-interval sides end at 640 / (192 / m) intervals."""
    assert [I.coarsest_by_node_rule(n) for n in (64, 128, 192, 256)] == [16, 16, 12, 16]
    m = I.coarsest_by_node_rule((640, 640, 192))
    halvings = int(np.log2(192 // m))
    assert (640 >> halvings) + 1 == 41 and (192 >> halvings) + 1 == 13


def test_stored_table2_counts_against_paper():
    """The oracle's counts at Table 2's 129^3, 193^3 and 257^3 nodes (stored by
    golden/make_closed_off_counts.py, which calls only the oracle, because the solves take tens
    of minutes) against the paper's (Sec. 5.2, Table 2): left-preconditioned GMRES within 3%
    (146 against 146, 140 against 137, 143 against 143), IDR(4) within 10% (its count moves
    with the shadow space and rounding order, Sec. 5.1.3)."""
    def rows(name):
        with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
            return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]

    paper = {int(r[0]): (int(r[2]), int(r[4])) for r in rows("weak_scaling_matvec.txt") if r[0] != "per_iter"}
    stored = {int(r[0]): (int(r[1]), int(r[2])) for r in rows("closed_off_oracle_counts.txt")}
    assert set(stored) == set(paper) == {129, 193, 257}
    for nodes, (g, i) in stored.items():
        pg, pi = paper[nodes]
        assert abs(g - pg) <= 0.03 * pg, (nodes, g, pg)
        assert abs(i - pi) <= 0.1 * pi, (nodes, i, pi)
