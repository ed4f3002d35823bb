"""Pins for the oracle's operators A_h and M_h (Sec. 2.4, Sec. 3.3, Algorithm 2).

Each check ties the oracle to the paper or to mathematics, not to itself:
  * the printed stencil (golden fixture),
  * closed-form eigenpairs of sine modes (Dirichlet),
  * the Kronecker-sum structure of the ghost-eliminated Sommerfeld operator,
  * consistency of the ghost elimination with the continuous radiation condition,
  * symmetry of A (Dirichlet) and of D A (Sommerfeld).
"""
import numpy as np
import pytest

import oracle
from conftest import load_stencil
from dense_ref import helmholtz_3d, second_diff_1d
from paper_2308_06085_gb300 import inputs as I

D, S = oracle.DIRICHLET, oracle.SOMMERFELD
CSLP = (1.0, 0.5)  # beta1 - beta2 i with beta2 = -0.5 (Sec. 3.3)


def test_printed_helmholtz_stencil():
    """A delta at an interior node returns the Sec. 2.4 stencil: (6 - k^2 h^2)/h^2 at the
    centre, -1/h^2 at the six neighbours, 0 elsewhere."""
    n, h, k = 8, 1.0 / 8, 3.0
    shape = I.unknown_shape(n, D)
    u = np.zeros(shape, complex)
    c = (3, 3, 3)
    u[c] = 1.0
    v = oracle.apply(u, np.full(shape, k * k), h, D)
    lap = load_stencil("laplace_stencil.txt")
    got = v[2:5, 2:5, 2:5] * h * h
    want = lap.astype(complex)
    want[1, 1, 1] -= k * k * h * h
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    v[2:5, 2:5, 2:5] = 0
    assert np.abs(v).max() == 0


@pytest.mark.parametrize("n", [(8, 8, 8), (6, 10, 12)])
@pytest.mark.parametrize("shift", [(1.0, 0.0), CSLP, (0.7, -1.3)])
def test_dirichlet_sine_modes(n, shift):
    """v = prod_d sin(p_d pi i_d / n_d) gives (A v)_p = (lambda - s k_p^2) v_p with
    lambda = (4/h^2) sum_d sin^2(p_d pi / (2 n_d)), pointwise even for variable k."""
    h = 0.1
    n1, n2, n3 = n
    shape = I.unknown_shape(n, D)
    k2 = I.random_k2(shape, seed=7, kmin=1.0, kmax=6.0)
    s = shift[0] + 1j * shift[1]
    for p in [(1, 1, 1), (2, 3, 1), (n1 - 1, 1, n3 - 2), (3, n2 - 1, 2)]:
        i1 = np.arange(1, n1)[None, None, :]
        i2 = np.arange(1, n2)[None, :, None]
        i3 = np.arange(1, n3)[:, None, None]
        v = np.sin(p[0] * np.pi * i1 / n1) * np.sin(p[1] * np.pi * i2 / n2) * np.sin(p[2] * np.pi * i3 / n3)
        lam = 4.0 / h**2 * sum(np.sin(pd * np.pi / (2 * nd)) ** 2 for pd, nd in zip(p, n))
        got = oracle.apply(v.astype(complex), k2, h, D, shift)
        want = (lam - s * k2) * v
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("n", [(6, 6, 6), (4, 7, 5)])
def test_sommerfeld_kronecker_sum(n):
    """With constant k, A = A1(x) + A1(y) + A1(z) - k^2 I, where A1 is the 1D operator with
    the ghost point eliminated at both ends (its -2ik/h end terms split per direction).
    Tensor products of A1 eigenvectors must be eigenvectors of the oracle's 3D operator,
    which pins edge and corner handling and the axis ordering."""
    h, k = 0.07, 9.0
    shape = I.unknown_shape(n, S)
    A1 = []
    for m in n:
        T = second_diff_1d(m, h, S).astype(complex)
        T[0, 0] -= 2j * k / h
        T[-1, -1] -= 2j * k / h
        A1.append(T)
    ev = [np.linalg.eig(T) for T in A1]
    rng = np.random.default_rng(3)
    for _ in range(4):
        a, b, c = (rng.integers(0, len(e[0])) for e in ev)
        v = np.einsum("k,j,i->kji", ev[2][1][:, c], ev[1][1][:, b], ev[0][1][:, a])
        mu = ev[0][0][a] + ev[1][0][b] + ev[2][0][c] - k * k
        got = oracle.apply(v, np.full(shape, k * k), h, S)
        assert np.abs(got - mu * v).max() <= 1e-10 * np.abs(mu * v).max()


@pytest.mark.parametrize("axis,side", [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1)])
def test_sommerfeld_outgoing_wave_consistency(axis, side):
    """A plane wave leaving through a face satisfies du/dn - i k u = 0 there, so the
    discrete residual (A u)_p at that face's nodes is the truncation error,
    -i k^3 h / 3 + O(h^2) (Taylor expansion of the eliminated stencil).  A wrong sign
    or factor in the ghost formula would leave an O(k/h) residual instead."""
    k = 6.0
    errs = []
    for n in (16, 32, 64):
        h = 1.0 / n
        shape = I.unknown_shape(n, S)
        x = np.arange(n + 1) * h
        sgn = 1.0 if side == 1 else -1.0
        w = np.exp(1j * sgn * k * x)
        u = [np.ones(n + 1)] * 3
        u = list(u)
        u[axis] = w
        U = np.einsum("k,j,i->kji", u[2], u[1], u[0])
        v = oracle.apply(U, np.full(shape, k * k), h, S)
        idx = [slice(1, n), slice(1, n), slice(1, n)]  # (i1, i2, i3) interior
        idx[axis] = n if side == 1 else 0
        face = v[idx[2], idx[1], idx[0]] / U[idx[2], idx[1], idx[0]]
        np.testing.assert_allclose(face, face.ravel()[0], rtol=1e-9, atol=1e-9)
        val = face.ravel()[0]
        assert abs(val - (-1j * k**3 * h / 3.0)) <= 0.2 * k**3 * h / 3.0
        errs.append(abs(val))
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


@pytest.mark.parametrize("bc", [D, S])
@pytest.mark.parametrize("shift", [(1.0, 0.0), CSLP])
def test_symmetry(bc, shift):
    """Dirichlet: A is complex symmetric, u^T A v = v^T A u.  Sommerfeld: the eliminated
    rows are scaled by 2 per face, so D A is symmetric with D = diag(2^-faces)."""
    n = (6, 5, 7)
    h = 0.11
    shape = I.unknown_shape(n, bc)
    k2 = I.random_k2(shape, seed=11, kmin=2.0, kmax=9.0)
    u = I.random_vector(shape, 1)
    v = I.random_vector(shape, 2)
    Au = oracle.apply(u, k2, h, bc, shift)
    Av = oracle.apply(v, k2, h, bc, shift)
    if bc == S:
        fc = np.zeros(shape)
        for ax, N in zip((2, 1, 0), shape[::-1]):
            sl = [slice(None)] * 3
            for e in (0, -1):
                sl[ax] = e
                fc[tuple(sl)] += 1
        Dg = 2.0 ** (-fc)
    else:
        Dg = np.ones(shape)
    lhs = np.sum(u * Dg * Av)
    rhs = np.sum(v * Dg * Au)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("bc", [D, S])
def test_apply_matches_kronecker_assembly(bc):
    """Heterogeneous k: the oracle's matrix-free product equals the dense Kronecker-sum
    assembly (1D second differences + diagonal -s k^2 - 2 i k_p nf_p / h)."""
    n = (5, 6, 4)
    h = 0.13
    shape = I.unknown_shape(n, bc)
    k2 = I.random_k2(shape, seed=5, kmin=1.0, kmax=7.0)
    u = I.random_vector(shape, 9)
    s = 1.0 + 0.5j
    M = helmholtz_3d(n, h, bc, k2, shift=s)
    want = (M @ u.ravel()).reshape(shape)
    got = oracle.apply(u, k2, h, bc, (s.real, s.imag))
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    d = oracle.diag(k2, h, bc, (s.real, s.imag))
    np.testing.assert_allclose(d.ravel(), np.diag(M), rtol=1e-14)


def test_rhs_point_is_discrete_dirac():
    """Sec. 2.4 discrete Dirac: 1/h^3 at the source node, zero elsewhere."""
    n = 8
    h = 1.0 / n
    b = oracle.rhs_point(I.unknown_shape(n, S), S, h, [(4, 4, 0)])
    assert b[0, 4, 4] == 1.0 / h**3 and np.count_nonzero(b) == 1
    bd = oracle.rhs_point(I.unknown_shape(n, D), D, h, [(4, 2, 3), (0, 3, 3)])  # 2nd on boundary
    assert bd[2, 1, 3] == 1.0 / h**3 and np.count_nonzero(bd) == 1
