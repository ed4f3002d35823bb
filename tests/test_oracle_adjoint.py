"""Pins for the oracle's adjoint state and gradient with respect to k^2.

  * lambda from the D-scaled forward solve equals a dense solve with A^H (Kronecker-built A),
  * the adjoint-state gradient equals central finite differences of the loss, node by node,
    at interior, face, edge and corner nodes.
"""
import numpy as np
import pytest

import oracle
from dense_ref import helmholtz_3d
from paper_2308_06085_gb300 import inputs as I

D, S = oracle.DIRICHLET, oracle.SOMMERFELD


@pytest.mark.parametrize("bc,n", [(S, (6, 4, 8)), (D, (8, 8, 8)), (S, (6, 6, 6))])
def test_adjoint_matches_dense_hermitian_solve(bc, n):
    h = 1.0 / max(n)
    shape = I.unknown_shape(n, bc)
    k2 = I.random_k2(shape, seed=51, kmin=1.0, kmax=0.6 / h)
    g = I.random_vector(shape, 52)
    o = oracle.Solver(n, h, bc, k2, coarsest_n=2)
    lam = o.solve_adjoint(g, restart=400, tol=1e-13, max_iter=400)["x"]
    A = helmholtz_3d(n, h, bc, k2)
    want = np.linalg.solve(A.conj().T, g.ravel())
    assert np.linalg.norm(lam.ravel() - want) <= 1e-10 * np.linalg.norm(want)


def _loss(n, h, bc, k2, sources, rec, d):
    o = oracle.Solver(n, h, bc, k2, coarsest_n=2)
    loss = 0.0
    for s, src in enumerate(sources):
        b = oracle.rhs_point(o.shape, bc, h, [src])
        u = o.gmres(b, restart=200, tol=1e-13, max_iter=400)["x"]
        loss += 0.5 * float(np.sum(np.abs(u.ravel()[rec] - d[s]) ** 2))
    return loss


def test_adjoint_gradient_matches_central_differences():
    n, bc = (8, 8, 8), S
    h = 1.0 / 8
    shape = I.unknown_shape(n, bc)
    c = I.smooth_random_velocity(n, sigma=1.5)
    k2 = I.k2_from_velocity(c, I.wedge_omega(n, cmin=float(c.min())))
    sources = [(2, 3, 0), (6, 5, 0)]
    plane = 7
    N3, N2, N1 = shape
    rec = np.array([plane * N2 * N1 + j * N1 + i for j in range(N2) for i in range(N1)])
    # observed data from a perturbed model
    k2_true = k2 * I.gaussian_bump(n, amp=-0.08, width=0.2) ** -2
    ot = oracle.Solver(n, h, bc, k2_true, coarsest_n=2)
    d = [ot.gmres(oracle.rhs_point(shape, bc, h, [s]), restart=200, tol=1e-13, max_iter=400)["x"].ravel()[rec]
         for s in sources]
    o = oracle.Solver(n, h, bc, k2, coarsest_n=2)
    loss, grad = o.adjoint_grad(sources, rec, d, restart=200, tol=1e-13, max_iter=400)
    assert abs(loss - _loss(n, h, bc, k2, sources, rec, d)) <= 1e-10 * loss
    # corner, edges, faces, interior and receiver-plane nodes
    nodes = [(0, 0, 0), (8, 0, 0), (0, 8, 8), (4, 0, 0), (0, 4, 8), (4, 4, 0), (8, 4, 4), (4, 4, 4), (3, 5, 2),
             (2, 6, 7), (5, 5, 6), (7, 1, 3)]
    for (i, j, k) in nodes:
        p = (k, j, i)
        eps = 1e-4 * k2[p]
        kp, km = k2.copy(), k2.copy()
        kp[p] += eps
        km[p] -= eps
        fd = (_loss(n, h, bc, kp, sources, rec, d) - _loss(n, h, bc, km, sources, rec, d)) / (2 * eps)
        assert abs(grad[p] - fd) <= 1e-4 * abs(fd) + 1e-9 * np.abs(grad).max(), (i, j, k, grad[p], fd)
