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


def test_closed_off_discrete_closed_form():
    """S = sin(pi x1) sin(2 pi x2) sin(4 pi x3) is an eigenvector of the 7-point Dirichlet
    Laplacian (eigenvalue lam_h = sum over m in (1, 2, 4) of (4 / h^2) sin^2(m pi h / 2)) and
    the boundary value 1 is annihilated by it, so the closed-off problem's discrete solution is
    u_h = 1 + a S, a = (21 pi^2 - k^2) / (lam_h - k^2), here indefinite (k^2 = 400 lies above
    the smallest eigenvalue, about 3 pi^2, and above lam_h, so a < 0).  The preconditioned solve must reach it; a wrong sign or scale of the boundary
    data, of k^2 or of the right-hand side moves the solution off u_h."""
    n, k = 32, 20.0
    h = 1.0 / n
    b = oracle.rhs_closed_off(n, k)
    o = oracle.Solver(n, h, D, np.full(I.unknown_shape(n, D), k * k), coarsest_n=4)
    res = o.gmres(b, restart=100, tol=1e-12, max_iter=1000)
    assert res["status"] == 0
    c = np.arange(1, n) * h
    S = np.sin(4 * np.pi * c)[:, None, None] * np.sin(2 * np.pi * c)[None, :, None] * np.sin(np.pi * c)[None, None, :]
    lam = sum(4.0 / h ** 2 * np.sin(m * np.pi * h / 2) ** 2 for m in (1, 2, 4))
    assert k * k > lam > 3 * np.pi ** 2
    u_h = 1.0 + (21 * np.pi ** 2 - k * k) / (lam - k * k) * S
    assert np.abs(res["x"] - u_h).max() <= 1e-9


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


@pytest.mark.parametrize("bc,n", [(D, 8), (S, (6, 4, 8))])
def test_bicgstab_tiny_matches_dense(bc, n):
    nn = (n, n, n) if np.isscalar(n) else n
    h = 1.0 / max(nn)
    shape = I.unknown_shape(nn, bc)
    k2 = I.random_k2(shape, seed=43, kmin=1.0, kmax=0.6 / h)
    b = I.random_vector(shape, 44)
    o = oracle.Solver(nn, h, bc, k2, coarsest_n=2)
    res = o.bicgstab(b, tol=1e-12, max_iter=2000)
    assert res["status"] == 0 and res["relres"] <= 1e-12
    x = np.linalg.solve(helmholtz_3d(nn, h, bc, k2), b.ravel())
    assert np.linalg.norm(res["x"].ravel() - x) <= 1e-9 * np.linalg.norm(x)


def test_bicgstab_agrees_with_gmres_and_counts_matvecs():
    """Both Krylov methods reach the same solution; Bi-CGSTAB spends two A-products per
    step (Sec. 5 counts #Matvec as products with A)."""
    n = 16
    h = 1.0 / n
    shape = I.unknown_shape(n, S)
    w = I.workload("wedge", n)
    b = oracle.rhs_point(shape, S, h, w["sources"])
    o = oracle.Solver(n, h, S, w["k2"])
    g = o.gmres(b, restart=200, tol=1e-10, max_iter=400)
    bi = o.bicgstab(b, tol=1e-10, max_iter=2000, history=True)
    assert bi["status"] == 0 and bi["relres"] <= 1e-10
    assert np.linalg.norm(bi["x"] - g["x"]) <= 1e-8 * np.linalg.norm(g["x"])
    # the recursive residual history ends below tol and the iteration count is the number of
    # history entries (one per A-product)
    assert len(bi["history"]) == bi["iters"] and bi["history"][-1] <= 1e-10


def test_fcycle_preconditioned_krylov():
    """Sec. 3.4.5: the F-cycle does more coarse work per application than the V-cycle, so as
    a preconditioner it needs no more outer iterations; both solves reach the dense solution."""
    n = (8, 8, 8)
    h = 1.0 / 8
    shape = I.unknown_shape(n, S)
    k2 = I.random_k2(shape, seed=45, kmin=1.0, kmax=0.6 / h)
    b = I.random_vector(shape, 46)
    x = np.linalg.solve(helmholtz_3d(n, h, S, k2), b.ravel())
    ov = oracle.Solver(n, h, S, k2, coarsest_n=2)
    of = oracle.Solver(n, h, S, k2, coarsest_n=2, cycle="f")
    for o in (ov, of):
        r = o.gmres(b, restart=200, tol=1e-12, max_iter=200)
        assert r["status"] == 0
        assert np.linalg.norm(r["x"].ravel() - x) <= 1e-10 * np.linalg.norm(x)
        bi = o.bicgstab(b, tol=1e-12, max_iter=2000)
        assert bi["status"] == 0
        assert np.linalg.norm(bi["x"].ravel() - x) <= 1e-9 * np.linalg.norm(x)
    w = I.workload("wedge", 16)
    b = oracle.rhs_point(w["k2"].shape, S, w["h"], w["sources"])
    itv = oracle.Solver(16, w["h"], S, w["k2"]).gmres(b, tol=1e-8)["iters"]
    itf = oracle.Solver(16, w["h"], S, w["k2"], cycle="f").gmres(b, tol=1e-8)["iters"]
    assert itf <= itv, (itf, itv)


@pytest.mark.parametrize("bc,n,s", [(D, 8, 4), (S, (6, 4, 8), 4), (S, 6, 2)])
def test_idrs_tiny_matches_dense(bc, n, s):
    nn = (n, n, n) if np.isscalar(n) else n
    h = 1.0 / max(nn)
    shape = I.unknown_shape(nn, bc)
    k2 = I.random_k2(shape, seed=47, kmin=1.0, kmax=0.6 / h)
    b = I.random_vector(shape, 48)
    o = oracle.Solver(nn, h, bc, k2, coarsest_n=2)
    res = o.idrs(b, I.shadow_space(shape, s), tol=1e-12, max_iter=2000)
    assert res["status"] == 0 and res["relres"] <= 1e-12
    x = np.linalg.solve(helmholtz_3d(nn, h, bc, k2), b.ravel())
    assert np.linalg.norm(res["x"].ravel() - x) <= 1e-9 * np.linalg.norm(x)


def test_idr1_is_bicgstab():
    """IDR(1) with the initial residual as its shadow vector and the minimal-residual omega
    (kappa = 0) is mathematically Bi-CGSTAB: both build their residuals from the same Krylov
    polynomials, so the residual norm after every A-product agrees until rounding takes over."""
    n = 16
    h = 1.0 / n
    shape = I.unknown_shape(n, S)
    w = I.workload("wedge", n)
    b = oracle.rhs_point(shape, S, h, w["sources"])
    o = oracle.Solver(n, h, S, w["k2"])
    bi = o.bicgstab(b, tol=1e-8, max_iter=400, history=True)
    idr = o.idrs(b, b[None], kappa=0.0, tol=1e-8, max_iter=400, history=True)
    assert idr["iters"] == bi["iters"] > 20
    np.testing.assert_allclose(idr["history"], bi["history"], rtol=1e-8)


@pytest.mark.parametrize("s", [1, 4, 8])
def test_idrs_agrees_with_gmres(s):
    """Every s reaches the GMRES solution; larger s needs fewer A-products (Sec. 3.1: IDR(s)
    moves from Bi-CGSTAB towards GMRES as s grows), and no method beats GMRES's optimal count."""
    n = 16
    h = 1.0 / n
    shape = I.unknown_shape(n, S)
    w = I.workload("wedge", n)
    b = oracle.rhs_point(shape, S, h, w["sources"])
    o = oracle.Solver(n, h, S, w["k2"])
    g = o.gmres(b, restart=400, tol=1e-10, max_iter=400)
    r = o.idrs(b, I.shadow_space(shape, s), tol=1e-10, max_iter=2000, history=True)
    assert r["status"] == 0 and r["relres"] <= 1e-10
    assert np.linalg.norm(r["x"] - g["x"]) <= 1e-8 * np.linalg.norm(g["x"])
    assert r["iters"] >= g["iters"]
    assert len(r["history"]) == r["iters"]


@pytest.mark.parametrize("nn,s,bound", [((3, 3, 3), 8, 8), ((5, 3, 3), 16, 16), ((5, 3, 3), 2, 24),
                                         ((5, 3, 3), 4, 20), ((5, 5, 3), 2, 48), ((5, 5, 5), 4, 80)])
def test_idrs_finite_termination(nn, s, bound):
    """The dimension-reduction theorem: in exact arithmetic IDR(s) reaches r = 0 within
    N + N / s products with A on N unknowns.  With s = N the first s steps make r orthogonal
    to a basis of the whole space, so r = 0 after exactly N products."""
    h = 1.0 / 5
    shape = I.unknown_shape(nn, D)
    N = int(np.prod(shape))
    k2 = I.random_k2(shape, seed=49, kmin=1.0, kmax=3.0 / h)
    b = I.random_vector(shape, 50)
    o = oracle.Solver(nn, h, D, k2, coarsest_n=2)
    r = o.idrs(b, I.shadow_space(shape, s), tol=1e-11, max_iter=500, history=True)
    assert r["status"] == 0 and r["relres"] <= 1e-11
    assert r["iters"] <= bound
    if s == N:
        assert r["iters"] == N and r["history"][-2] > 1e-6


def test_closed_off_rhs_generators_agree():
    """The synthetic-input module's closed-off right-hand side (used by the benchmark) and the
    oracle's own (used by the pins) are written independently; they must agree."""
    for n, k in ((8, 5.0), (64, 40.0)):
        a = I.closed_off_rhs(n, k)
        b = oracle.rhs_closed_off(n, k)
        assert a.shape == b.shape
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
