"""Pins for the oracle's preconditioned GMRES (Sec. 3.1-3.3, Sec. 5 stopping rule).

  * tiny problems against a dense direct solve of the Kronecker-built A,
  * the closed-off problem of Sec. 2.1 (analytic solution): second-order error decay,
  * Green's-function reciprocity for interior source/receiver pairs,
  * GMRES invariants: monotone residual estimates, the estimate equal to the explicit
    residual at the end, flexible and plain right preconditioning agreeing, and the
    complex-conjugate symmetry between the two signs of the CSLP shift on a real problem.
"""
import numpy as np
import pytest

import oracle
from dense_ref import helmholtz_3d
from paper_2308_06085_gb300 import inputs as I

D, S = oracle.DIRICHLET, oracle.SOMMERFELD


@pytest.mark.parametrize("bc,n", [(D, 8), (S, 6), (S, (6, 4, 8))])
def test_tiny_solve_matches_dense(bc, n):
    nn = (n, n, n) if np.isscalar(n) else n
    h = 1.0 / max(nn)
    shape = I.unknown_shape(nn, bc)
    k2 = I.random_k2(shape, seed=41, kmin=1.0, kmax=0.6 / h)
    b = I.random_vector(shape, 42)
    o = oracle.Solver(nn, h, bc, k2, coarsest_n=2)
    res = o.gmres(b, restart=400, tol=1e-12, max_iter=400)
    assert res["status"] == 0
    x = np.linalg.solve(helmholtz_3d(nn, h, bc, k2), b.ravel())
    assert np.linalg.norm(res["x"].ravel() - x) <= 1e-10 * np.linalg.norm(x)


def test_closed_off_second_order():
    """Sec. 2.1: u = sin(pi x) sin(2 pi y) sin(4 pi z) + 1 with Dirichlet u = 1.  The
    max error of the discrete solution falls by ~4 per halving of h."""
    k = 5.0
    errs = []
    for n in (16, 32, 64):
        shape = I.unknown_shape(n, D)
        b = oracle.rhs_closed_off(n, k)
        o = oracle.Solver(n, 1.0 / n, D, np.full(shape, k * k), coarsest_n=4)
        res = o.gmres(b, restart=60, tol=1e-11, max_iter=300)
        assert res["status"] == 0
        x = (np.arange(1, n) / n)
        exact = (np.sin(np.pi * x)[None, None, :] * np.sin(2 * np.pi * x)[None, :, None]
                 * np.sin(4 * np.pi * x)[:, None, None] + 1.0)
        errs.append(np.abs(res["x"] - exact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2, errs


def test_reciprocity():
    """A = D^-1 S with S symmetric and D = 1 at interior nodes, so the discrete Green's
    function is reciprocal between interior nodes: G(s -> r) = G(r -> s)."""
    n = 12
    h = 1.0 / n
    shape = I.unknown_shape(n, S)
    c = I.wedge_velocity(n)
    k2 = I.k2_from_velocity(c, I.wedge_omega(n))
    o = oracle.Solver(n, h, S, k2, coarsest_n=3)
    s, r = (3, 5, 2), (8, 4, 9)  # node coordinates (i1, i2, i3)
    us = o.gmres(oracle.rhs_point(shape, S, h, [s]), tol=1e-11, max_iter=500)
    ur = o.gmres(oracle.rhs_point(shape, S, h, [r]), tol=1e-11, max_iter=500)
    a = us["x"][r[2], r[1], r[0]]
    bb = ur["x"][s[2], s[1], s[0]]
    assert abs(a - bb) <= 1e-8 * abs(a)


def test_gmres_invariants():
    n = 16
    h = 1.0 / n
    shape = I.unknown_shape(n, S)
    w = I.workload("wedge", n)
    b = oracle.rhs_point(shape, S, h, w["sources"])
    o = oracle.Solver(n, h, S, w["k2"], coarsest_n=4)
    full = o.gmres(b, restart=200, tol=1e-8, max_iter=200, history=True)
    hist = full["history"]
    assert full["status"] == 0 and np.all(np.diff(hist) <= 1e-12)
    assert abs(hist[-1] - full["relres"]) <= 1e-4 * full["relres"]
    fl = o.gmres(b, restart=200, tol=1e-8, max_iter=200, flexible=True)
    assert abs(fl["iters"] - full["iters"]) <= 1
    assert np.linalg.norm(fl["x"] - full["x"]) <= 1e-6 * np.linalg.norm(full["x"])
    r30 = o.gmres(b, restart=5, tol=1e-8, max_iter=400)
    assert r30["status"] == 0 and r30["iters"] >= full["iters"]
    Ax = oracle.apply(r30["x"], w["k2"], h, S)
    assert np.linalg.norm(b - Ax) / np.linalg.norm(b) <= 1e-8


def test_cslp_sign_conjugate_symmetry():
    """Real Dirichlet problem: beta2 = -0.5 and +0.5 give complex-conjugate iterates, so
    the same iteration counts (the two readings of the CSLP sign agree here)."""
    n = 16
    shape = I.unknown_shape(n, D)
    k2 = np.full(shape, 10.0**2)
    b = oracle.rhs_point(shape, D, 1.0 / n, [(8, 8, 8)])
    a = oracle.Solver(n, 1 / n, D, k2, beta2=-0.5).gmres(b, tol=1e-8)
    c = oracle.Solver(n, 1 / n, D, k2, beta2=+0.5).gmres(b, tol=1e-8)
    assert a["iters"] == c["iters"]
    assert np.linalg.norm(a["x"] - np.conj(c["x"])) <= 1e-12 * np.linalg.norm(a["x"])


def test_zero_rhs_and_max_iter():
    n = 8
    shape = I.unknown_shape(n, S)
    o = oracle.Solver(n, 1 / n, S, np.full(shape, 25.0))
    z = o.gmres(np.zeros(shape))
    assert z["status"] == 0 and z["iters"] == 0 and np.all(z["x"] == 0)
    b = I.random_vector(shape, 1)
    one = o.gmres(b, max_iter=1, tol=1e-14)
    assert one["status"] == 1 and one["iters"] == 1
