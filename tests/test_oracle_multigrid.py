"""Pins for the oracle's transfers, smoother and V-cycle (Sec. 3.4, Algorithm 1).

  * printed restriction / prolongation stencils (golden fixtures, Sec. 3.4.2-3.4.3),
  * the exact adjoint relation 8 <R r, e> = <r, P e> and exactness on linear functions,
  * the V-cycle against an independent dense composition from Kronecker-built matrices,
  * textbook multigrid behaviour on the k = 0 Poisson problem: an h-independent V(1,1)
    contraction factor below the damped-Jacobi smoothing bound.
"""
import numpy as np
import pytest

import oracle
from conftest import load_stencil
from dense_ref import dense_fcycle, dense_vcycle, helmholtz_3d, inject_k2, levels
from paper_2308_06085_gb300 import inputs as I

D, S = oracle.DIRICHLET, oracle.SOMMERFELD


def test_printed_restriction_stencil():
    """Row of I_h^H at an interior coarse node = the printed (1/64) 3x3x3 stencil."""
    nf = 8
    fs, cs = I.unknown_shape(nf, S), I.unknown_shape(nf // 2, S)
    C = (2, 2, 2)  # coarse node (i3, i2, i1) -> fine node 2C
    table = np.zeros((3, 3, 3))
    for dk in range(3):
        for dj in range(3):
            for di in range(3):
                r = np.zeros(fs, complex)
                r[2 * C[0] + dk - 1, 2 * C[1] + dj - 1, 2 * C[2] + di - 1] = 1.0
                table[dk, dj, di] = oracle.restrict(r, cs, S)[C].real
    np.testing.assert_allclose(table * 64, load_stencil("restriction_stencil.txt"), rtol=0, atol=1e-13)


@pytest.mark.parametrize("bc", [D, S])
def test_printed_prolongation_stencil(bc):
    """Column of I_H^h at an interior coarse node = the printed (1/8) 3x3x3 stencil."""
    nf = 8
    fs, cs = I.unknown_shape(nf, bc), I.unknown_shape(nf // 2, bc)
    e = np.zeros(cs, complex)
    Cn = (2, 2, 2)  # coarse node coordinates
    off = 1 if bc == D else 0
    e[tuple(c - off for c in Cn)] = 1.0
    out = oracle.prolong(e, fs, bc)
    f = [2 * c - off for c in Cn]
    blk = out[f[0] - 1:f[0] + 2, f[1] - 1:f[1] + 2, f[2] - 1:f[2] + 2].real
    np.testing.assert_allclose(blk * 8, load_stencil("prolongation_stencil.txt"), rtol=0, atol=1e-13)
    out[f[0] - 1:f[0] + 2, f[1] - 1:f[1] + 2, f[2] - 1:f[2] + 2] = 0
    assert np.abs(out).max() == 0


@pytest.mark.parametrize("bc", [D, S])
@pytest.mark.parametrize("nf", [(8, 8, 8), (4, 8, 6)])
def test_transfer_adjoint(bc, nf):
    """8 <R r, e>_H = <r, P e>_h (bilinear), i.e. full weighting is P^T / 8."""
    fs, cs = I.unknown_shape(nf, bc), I.unknown_shape(tuple(m // 2 for m in nf), bc)
    r = I.random_vector(fs, 21)
    e = I.random_vector(cs, 22)
    lhs = 8 * np.sum(oracle.restrict(r, cs, bc) * e)
    rhs = np.sum(r * oracle.prolong(e, fs, bc))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_transfers_exact_on_linear_functions():
    """Trilinear interpolation reproduces a linear function at every fine node, and full
    weighting reproduces it at every coarse node whose 27-point patch is in the domain."""
    nf = (8, 12, 10)
    fs, cs = I.unknown_shape(nf, S), I.unknown_shape(tuple(m // 2 for m in nf), S)
    lin = lambda i1, i2, i3: 0.3 + 1.7 * i1 - 0.4 * i2 + 2.5 * i3 + 1j * (0.1 * i1 + i3)
    k3, k2_, k1 = np.meshgrid(*[np.arange(m) for m in cs], indexing="ij")
    e = lin(2.0 * k1, 2.0 * k2_, 2.0 * k3)  # coarse node c sits at fine coordinate 2c
    f3, f2, f1 = np.meshgrid(*[np.arange(m) for m in fs], indexing="ij")
    np.testing.assert_allclose(oracle.prolong(e, fs, S), lin(1.0 * f1, 1.0 * f2, 1.0 * f3), rtol=1e-14, atol=1e-12)
    R = oracle.restrict(lin(1.0 * f1, 1.0 * f2, 1.0 * f3), cs, S)
    np.testing.assert_allclose(R[1:-1, 1:-1, 1:-1], e[1:-1, 1:-1, 1:-1], rtol=1e-14, atol=1e-12)


def test_coarse_k2_is_injection():
    n = (8, 16, 8)
    shape = I.unknown_shape(n, S)
    k2 = I.random_k2(shape, 4)
    o = oracle.Solver(n, 1.0 / 16, S, k2, coarsest_n=2)
    assert o.nlevels == 3
    np.testing.assert_array_equal(o.level(1)["k2"], k2[::2, ::2, ::2])
    np.testing.assert_array_equal(o.level(2)["k2"], k2[::4, ::4, ::4])
    od = oracle.Solver(n, 1.0 / 16, D, I.random_k2(I.unknown_shape(n, D), 4), coarsest_n=2)
    assert od.level(2)["shape"] == (1, 3, 1)


def test_hierarchy_depths():
    """Coarsening rule: halve while every n_d is even and n_d / 2 >= coarsest_n (4)."""
    for n, nl in [(32, 4), (128, 6), (192, 6), (256, 7), (12, 2), (10, 2), (6, 1)]:
        assert len(levels((n, n, n), 4)) == nl
    for n, nl in [(32, 4), (12, 2), (10, 2), (6, 1), ((16, 8, 24), 2)]:
        nn = (n, n, n) if np.isscalar(n) else n
        shape = I.unknown_shape(nn, S)
        assert oracle.Solver(nn, 0.1, S, np.ones(shape), coarsest_n=4).nlevels == nl


@pytest.mark.parametrize("bc,n,coarsest", [(D, (8, 8, 8), 2), (S, (8, 8, 8), 2), (S, (8, 12, 4), 2), (D, (16, 8, 8), 2)])
def test_vcycle_matches_dense_composition(bc, n, coarsest):
    """The matrix-free V-cycle equals z = S(x1 + P M_H^{-1} R (b - M x1)), x1 = w D^-1 b,
    applied recursively with dense Kronecker-built matrices."""
    h = 1.0 / max(n)
    shape = I.unknown_shape(n, bc)
    k2 = I.random_k2(shape, seed=31, kmin=2.0, kmax=0.6 / h)
    b = I.random_vector(shape, 32)
    o = oracle.Solver(n, h, bc, k2, beta1=1.0, beta2=-0.5, omega=0.8, coarsest_n=coarsest)
    got = o.vcycle(b).ravel()
    want = dense_vcycle(n, h, bc, k2, b, 1.0 + 0.5j, 0.8, coarsest)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_vcycle_stages_compose():
    """Down stage, coarse solve and up stage chained level by level give the V-cycle."""
    n = (16, 16, 16)
    shape = I.unknown_shape(n, S)
    k2 = I.random_k2(shape, seed=3, kmin=2.0, kmax=8.0)
    b = I.random_vector(shape, 4)
    o = oracle.Solver(n, 1 / 16, S, k2, coarsest_n=4)
    L = o.nlevels
    bs = [b]
    for l in range(L - 1):
        bs.append(o.vcycle_down(l, bs[-1]))
    e = o.coarse_solve(bs[-1])
    for l in range(L - 2, -1, -1):
        e = o.vcycle_up(l, bs[l], e)
    np.testing.assert_allclose(e, o.vcycle(b), rtol=0, atol=1e-13 * np.abs(e).max())


def test_poisson_vcycle_contraction():
    """k = 0 Poisson, Dirichlet: V(1,1) with w = 0.8 damped Jacobi as a stationary
    iteration.  Its error contraction is h-independent and below the smoothing bound
    mu^2, mu = max(|1 - w/3|, |1 - 2w|) = 0.733 (3D Jacobi smoothing factor)."""
    rhos = []
    for n in (16, 32, 64):
        shape = I.unknown_shape(n, D)
        k2 = np.zeros(shape)
        o = oracle.Solver(n, 1.0 / n, D, k2, coarsest_n=4)
        x = I.random_vector(shape, 77).real.astype(complex)
        ratios = []
        for _ in range(12):
            r = -oracle.apply(x, k2, 1.0 / n, D)
            xn = x + o.vcycle(r)
            ratios.append(np.linalg.norm(xn) / np.linalg.norm(x))
            x = xn / np.linalg.norm(xn)
        rhos.append(np.mean(ratios[-4:]))
    mu = max(abs(1 - 0.8 / 3), abs(1 - 1.6))
    assert all(r < mu**2 for r in rhos), rhos
    assert abs(rhos[1] - rhos[2]) < 0.05 and abs(rhos[0] - rhos[1]) < 0.05, rhos


@pytest.mark.parametrize("bc,n,coarsest", [(D, (16, 8, 8), 2), (S, (8, 12, 8), 2), (S, (16, 16, 16), 2)])
def test_fcycle_matches_dense_composition(bc, n, coarsest):
    """The F-cycle (Sec. 3.4.5) equals its dense recursive composition."""
    h = 1.0 / max(n)
    shape = I.unknown_shape(n, bc)
    k2 = I.random_k2(shape, seed=33, kmin=2.0, kmax=0.6 / h)
    b = I.random_vector(shape, 34)
    o = oracle.Solver(n, h, bc, k2, coarsest_n=coarsest)
    assert o.nlevels >= 3
    got = o.fcycle(b).ravel()
    want = dense_fcycle(n, h, bc, k2, b, 1.0 + 0.5j, 0.8, coarsest)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_poisson_fcycle_contracts_at_least_as_well_as_vcycle():
    n = 32
    shape = I.unknown_shape(n, D)
    k2 = np.zeros(shape)
    o = oracle.Solver(n, 1.0 / n, D, k2, coarsest_n=4)
    out = {}
    for name, cyc in (("v", o.vcycle), ("f", o.fcycle)):
        x = I.random_vector(shape, 78).real.astype(complex)
        ratios = []
        for _ in range(10):
            xn = x + cyc(-oracle.apply(x, k2, 1.0 / n, D))
            ratios.append(np.linalg.norm(xn) / np.linalg.norm(x))
            x = xn / np.linalg.norm(xn)
        out[name] = np.mean(ratios[-4:])
    assert out["f"] <= out["v"] + 1e-3, out


def test_coarse_gmres_matches_exact_coarse_solve():
    """The paper's coarsest solver (full GMRES to 1e-11, Sec. 5) against the exact LU solve:
    the coarse error of GMRES is at the 1e-11 level, so one V-cycle agrees to ~1e-9."""
    import oracle
    from paper_2308_06085_gb300 import inputs as I

    for bc, n in ((oracle.SOMMERFELD, 16), (oracle.DIRICHLET, 16)):
        shape = I.unknown_shape(n, bc)
        k2 = I.random_k2(shape, seed=61, kmin=1.0, kmax=0.6 * n)
        r = I.random_vector(shape, 62)
        exact = oracle.Solver(n, 1.0 / n, bc, k2, coarsest_n=4).vcycle(r)
        for tol, bound in ((1e-11, 1e-8), (1e-14, 1e-11)):
            z = oracle.Solver(n, 1.0 / n, bc, k2, coarsest_n=4, coarse_tol=tol).vcycle(r)
            assert np.linalg.norm(z - exact) <= bound * np.linalg.norm(exact), (bc, tol)
        # GMRES with a loose tolerance leaves a visible coarse error: the option is really used
        z = oracle.Solver(n, 1.0 / n, bc, k2, coarsest_n=4, coarse_tol=1e-2).vcycle(r)
        assert np.linalg.norm(z - exact) > 1e-6 * np.linalg.norm(exact)
