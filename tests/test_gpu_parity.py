"""GPU parity: every step of the hot path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.

Tolerances (relative, in the 2-norm over the whole grid unless stated):
  FP64 operator, V-cycle stages, full V-cycle : 1e-12   (both sides FP64; only rounding order
                                                          and FMA contraction differ)
  FP32 operator / V-cycle (complex64)          : 1e-5 / 2e-5 (unit roundoff 6e-8 times the
                                                          stencil's cancellation, see design notes)
  solves (FP64)  : true relative residual <= tol, iterations within +-1 of the oracle,
                   solution difference <= 1e-5
Grids are chosen to span several 32 x 8 thread tiles with ragged tails in x and y, odd
unknown counts, non-cubic boxes and the degenerate one-level hierarchy.
"""
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
    ("som_wedge32", (32, 32, 32), S, 4),
    ("som_noncubic", (24, 8, 16), S, 2),
]


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2308_06085_gb300 import helm as h

    torch.cuda.set_device(0)
    return h


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def orth_kw(orth):
    """Gram-Schmidt arithmetic under test: FP64 against the summed basis (three FMAs per complex
    multiply-add, the default), FP64 in the textbook four-FMA form, or double-float."""
    return {"fp64": dict(orth="fp64"), "fp64-4fma": dict(orth="fp64", gs_sums=False), "df": dict(orth="df")}[orth]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def check_mixed_accuracy(o, bn, x, ro):
    """Mixed precision has no FP64 twin to follow step by step (parity unpinned by the paper,
    which is all FP64).  Its true residual is checked by the caller; here its error against the
    oracle's solve to 1e-11 is bounded by 1e-4.  Solves that stop at 1e-6 sit ~1e-5 from the
    exact discrete solution on these grids whatever their arithmetic (the oracle's own 1e-6
    solves measure 3e-6 .. 2e-5), so two of them can differ by a few 1e-5."""
    tight = o.gmres(bn, restart=200, tol=1e-11, max_iter=2000)["x"]
    e_gpu = rel(x, tight)
    assert e_gpu <= 1e-4, (e_gpu, rel(ro["x"], tight))


def make(helm, name, n, bc, coarsest, **kw):
    h = 1.0 / max(n)
    shape = I.unknown_shape(n, bc)
    if name.endswith("wedge32"):
        k2 = I.workload("wedge", 32)["k2"]
    else:
        k2 = I.random_k2(shape, seed=sum(map(ord, name)), kmin=2.0, kmax=0.6 / h)
    s = helm.Solver(n, h, k2, bc, coarsest_n=coarsest, **kw)
    o = oracle.Solver(n, h, bc, k2, coarsest_n=coarsest)
    return s, o, k2, h, shape


@pytest.mark.parametrize("name,n,bc,coarsest", CASES)
@pytest.mark.parametrize("op", ["A", "M"])
def test_apply_c128(helm, name, n, bc, coarsest, op):
    s, o, k2, h, shape = make(helm, name, n, bc, coarsest)
    u = I.random_vector(shape, 3)
    v = s.apply(dev(u), op).cpu().numpy()
    shift = (1.0, 0.0) if op == "A" else (1.0, 0.5)
    vo = oracle.apply(u, k2, h, bc, shift)
    assert np.abs(v - vo).max() <= 1e-12 * np.abs(vo).max()
    assert rel(v, vo) <= 1e-12


@pytest.mark.parametrize("name,n,bc,coarsest", CASES)
def test_apply_c64(helm, name, n, bc, coarsest):
    s, o, k2, h, shape = make(helm, name, n, bc, coarsest)
    u = I.random_vector(shape, 4)
    v = s.apply(dev(u.astype(np.complex64)), "M").cpu().numpy()
    vo = oracle.apply(u.astype(np.complex64).astype(np.complex128), k2, h, bc, (1.0, 0.5))
    assert rel(v, vo) <= 1e-5


@pytest.mark.parametrize("name,n,bc,coarsest", CASES)
def test_vcycle_stages_c128(helm, name, n, bc, coarsest):
    s, o, k2, h, shape = make(helm, name, n, bc, coarsest)
    L = s.nlevels
    assert L == o.nlevels
    for l in range(L - 1):
        fs = s.level_dims(l)["shape"]
        cs = s.level_dims(l + 1)["shape"]
        b = I.random_vector(fs, 10 + l)
        e = I.random_vector(cs, 20 + l)
        down = s.vcycle_stage(l, 0, dev(b)).cpu().numpy()
        assert rel(down, o.vcycle_down(l, b)) <= 1e-12, l
        up = s.vcycle_stage(l, 1, dev(b), dev(e)).cpu().numpy()
        assert rel(up, o.vcycle_up(l, b, e)) <= 1e-12, l
    bl = I.random_vector(s.level_dims(L - 1)["shape"], 5)
    ec = s.vcycle_stage(L - 1, 2, dev(bl)).cpu().numpy()
    assert rel(ec, o.coarse_solve(bl)) <= 1e-12


@pytest.mark.parametrize("name,n,bc,coarsest", CASES)
def test_vcycle_c128(helm, name, n, bc, coarsest):
    s, o, k2, h, shape = make(helm, name, n, bc, coarsest)
    r = I.random_vector(shape, 6)
    z = s.vcycle(dev(r)).cpu().numpy()
    assert rel(z, o.vcycle(r)) <= 1e-12


@pytest.mark.parametrize("name,n,bc,coarsest", CASES)
def test_vcycle_c64(helm, name, n, bc, coarsest):
    s, o, k2, h, shape = make(helm, name, n, bc, coarsest)
    r = I.random_vector(shape, 7).astype(np.complex64)
    z = s.vcycle(dev(r)).cpu().numpy()
    err = rel(z, o.vcycle(r.astype(np.complex128)))
    assert err <= 2e-5, err


def test_rhs_point_bit_exact(helm):
    for n, bc, src in [((16, 16, 16), S, [(8, 8, 0), (0, 0, 0), (16, 3, 16), (8, 8, 0)]),
                       ((16, 12, 8), D, [(8, 6, 4), (0, 6, 4), (15, 11, 7)])]:
        shape = I.unknown_shape(n, bc)
        s = helm.Solver(n, 1 / 16, np.ones(shape), bc)
        b = s.rhs_point(src).cpu().numpy()
        np.testing.assert_array_equal(b, oracle.rhs_point(shape, bc, 1 / 16, src))


@pytest.mark.parametrize("orth", ["fp64", "fp64-4fma", "df"])
@pytest.mark.parametrize("krylov,restart", [("gmres", 30), ("fgmres", 30), ("gmres", 200)])
def test_solve_small_dirichlet(helm, krylov, restart, orth):
    """The small workload itself: n = 32, constant k = 20 (kh = 0.625), Dirichlet, centre source."""
    w = I.workload("small")
    s = helm.Solver(w["n"], w["h"], w["k2"], D, krylov=krylov, restart=restart, max_iter=600, **orth_kw(orth))
    o = oracle.Solver(w["n"], w["h"], D, w["k2"])
    b = s.rhs_point(w["sources"])
    x, info = s.solve(b)
    ro = o.gmres(b.cpu().numpy(), restart=restart, tol=1e-6, max_iter=600, flexible=krylov == "fgmres")
    assert info["status"] == 0 and ro["status"] == 0
    assert info["rel_residual"] <= 1e-6
    assert abs(info["iterations"] - ro["iters"]) <= 1, (info, ro["iters"])
    assert rel(x.cpu().numpy(), ro["x"]) <= 1e-5
    # independent check of the residual with the oracle's operator
    ax = oracle.apply(x.cpu().numpy(), w["k2"], w["h"], D)
    assert np.linalg.norm(b.cpu().numpy() - ax) / np.linalg.norm(b.cpu().numpy()) <= 1.01e-6


@pytest.mark.parametrize("orth", ["fp64", "fp64-4fma", "df"])
@pytest.mark.parametrize("krylov", ["gmres", "fgmres"])
def test_solve_wedge_scaled(helm, krylov, orth):
    w = I.workload("wedge", 32)
    s = helm.Solver(w["n"], w["h"], w["k2"], S, krylov=krylov, **orth_kw(orth))
    o = oracle.Solver(w["n"], w["h"], S, w["k2"])
    b = s.rhs_point(w["sources"])
    x, info = s.solve(b)
    ro = o.gmres(b.cpu().numpy(), restart=30, tol=1e-6, flexible=krylov == "fgmres")
    assert info["status"] == 0 and info["rel_residual"] <= 1e-6
    assert abs(info["iterations"] - ro["iters"]) <= 1, (info, ro["iters"])
    assert rel(x.cpu().numpy(), ro["x"]) <= 1e-5


@pytest.mark.parametrize("orth", ["fp64", "df"])
def test_solve_mixed_precision(helm, orth):
    """complex64 V-cycle under FP64 FGMRES(30): the true residual still reaches 1e-6; the
    error against a tight FP64 oracle solution is reported (the paper fixes no bound)."""
    w = I.workload("mixed", 32)
    s = helm.Solver(w["n"], w["h"], w["k2"], S, precision="mixed", orth=orth)
    o = oracle.Solver(w["n"], w["h"], S, w["k2"])
    b = s.rhs_point(w["sources"])
    x, info = s.solve(b)
    ro = o.gmres(b.cpu().numpy(), restart=30, tol=1e-10, max_iter=2000)
    ro6 = o.gmres(b.cpu().numpy(), restart=30, tol=1e-6)
    err = rel(x.cpu().numpy(), ro["x"])
    print(f"mixed: iters {info['iterations']} (fp64 oracle {ro6['iters']}), relres {info['rel_residual']:.2e}, "
          f"error vs tight oracle {err:.2e}")
    assert info["status"] == 0 and info["rel_residual"] <= 1e-6
    assert abs(info["iterations"] - ro6["iters"]) <= 3
    assert err <= 1e-4


def test_solve_host_buffers_and_warm_start(helm):
    w = I.workload("wedge", 16)
    s = helm.Solver(w["n"], w["h"], w["k2"], S)
    b = s.rhs_point(w["sources"])
    xd, infod = s.solve(b)
    bh = b.cpu().pin_memory()
    xh, infoh = s.solve(bh, torch.zeros_like(bh).pin_memory())
    assert infoh["iterations"] == infod["iterations"]
    np.testing.assert_array_equal(xh.numpy(), xd.cpu().numpy())
    # pageable host memory works too
    xp, infop = s.solve(b.cpu().clone(), torch.zeros(s.shape, dtype=torch.complex128))
    np.testing.assert_array_equal(xp.numpy(), xd.cpu().numpy())
    # warm start from the solution: converged at entry, no Arnoldi step
    x2, info2 = s.solve(b, xd.clone())
    assert info2["iterations"] == 0 and info2["rel_residual"] <= 1e-6
    # helm_solve_zero ignores what x holds on entry (device and pinned host buffers): the same
    # solve as from a zero guess, bit for bit
    junk = torch.full(s.shape, 7.0 + 3.0j, dtype=torch.complex128)
    xz, infoz = s.solve(b, junk.clone().cuda(), zero_guess=True)
    assert infoz["iterations"] == infod["iterations"] and torch.equal(xz, xd)
    xzh, infozh = s.solve(bh, junk.clone().pin_memory(), zero_guess=True)
    np.testing.assert_array_equal(xzh.numpy(), xd.cpu().numpy())


def test_solve_edge_cases(helm):
    # zero right-hand side
    w = I.workload("wedge", 16)
    s = helm.Solver(w["n"], w["h"], w["k2"], S, max_iter=1)
    x, info = s.solve(torch.zeros(s.shape, dtype=torch.complex128, device="cuda"))
    assert info["iterations"] == 0 and torch.count_nonzero(x) == 0
    # iteration cap
    b = s.rhs_point(w["sources"])
    x, info = s.solve(b)
    assert info["status"] == 4 and info["iterations"] == 1
    # one-level hierarchies (coarsest solve only) and the smallest grids
    for n, bc in [((2, 2, 2), D), ((2, 2, 2), S), ((6, 10, 8), S), ((3, 5, 7), D)]:
        shape = I.unknown_shape(n, bc)
        k2 = I.random_k2(shape, 3, 1.0, 3.0)
        s = helm.Solver(n, 0.2, k2, bc)
        o = oracle.Solver(n, 0.2, bc, k2)
        assert s.nlevels == o.nlevels == 1
        r = I.random_vector(shape, 8)
        assert rel(s.vcycle(dev(r)).cpu().numpy(), o.vcycle(r)) <= 1e-12
        x, info = s.solve(dev(r))
        assert info["status"] == 0 and info["iterations"] <= 30


def test_full_size_wedge_apply_and_vcycle(helm):
    """The n = 128 wedge (129^3 unknowns) in the configuration the benchmark times: the
    operator and one V-cycle against the oracle on the whole grid."""
    w = I.workload("wedge")
    s = helm.Solver(w["n"], w["h"], w["k2"], S)
    o = oracle.Solver(w["n"], w["h"], S, w["k2"])
    u = I.random_vector(s.shape, 12)
    v = s.apply(dev(u)).cpu().numpy()
    assert rel(v, oracle.apply(u, w["k2"], w["h"], S)) <= 1e-12
    z = s.vcycle(dev(u)).cpu().numpy()
    assert rel(z, o.vcycle(u)) <= 1e-12


@pytest.mark.parametrize("orth", ["fp64", "df"])
def test_full_size_wedge_solve_residual(helm, orth):
    """Full-size FP64 solve: the oracle's own operator confirms ||b - A x|| / ||b|| <= 1e-6."""
    w = I.workload("wedge")
    s = helm.Solver(w["n"], w["h"], w["k2"], S, orth=orth)
    b = s.rhs_point(w["sources"])
    x, info = s.solve(b)
    assert info["status"] == 0
    bn = b.cpu().numpy()
    ax = oracle.apply(x.cpu().numpy(), w["k2"], w["h"], S)
    rr = np.linalg.norm(bn - ax) / np.linalg.norm(bn)
    assert rr <= 1.01e-6 and abs(rr - info["rel_residual"]) <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("bc,n", [(D, (32, 32, 32)), (S, (32, 32, 32))])
def test_bicgstab_vs_oracle(helm, precision, bc, n):
    """Right-preconditioned Bi-CGSTAB (the paper's short-recurrence solver): the true
    residual reaches tol; #Matvec within 10% of the oracle's (the recurrence is sensitive to
    rounding, Sec. 5.1.3); solutions agree with the oracle's to the solve accuracy.

    FP64 runs to 1e-9 with #Matvec within 10% of the oracle's.  Mixed precision runs to the
    paper's 1e-6: Bi-CGSTAB assumes a fixed preconditioner, and the complex64 V-cycle is one
    only up to its FP32 rounding (V-cycle parity 2e-5), which short recurrences amplify (the
    paper sees 12% spread from reordering alone); its count is bounded by 1.5x the FP64
    oracle's and its accuracy must match the FP64 oracle's solve to the same tolerance."""
    tol = 1e-9 if precision == "fp64" else 1e-6
    w = I.workload("small") if bc == D else I.workload("wedge", 32)
    s = helm.Solver(w["n"], w["h"], w["k2"], bc, krylov="bicgstab", precision=precision, tol=tol, max_iter=4000)
    o = oracle.Solver(w["n"], w["h"], bc, w["k2"])
    b = s.rhs_point(w["sources"])
    x, info = s.solve(b)
    ro = o.bicgstab(b.cpu().numpy(), tol=tol, max_iter=4000)
    assert info["status"] == 0 and info["rel_residual"] <= tol and ro["status"] == 0
    bn = b.cpu().numpy()
    if precision == "fp64":
        assert abs(info["iterations"] - ro["iters"]) <= max(2, 0.1 * ro["iters"]), (info, ro["iters"])
        assert rel(x.cpu().numpy(), ro["x"]) <= 1e-5
    else:
        assert info["iterations"] <= 1.5 * ro["iters"] + 2, (info, ro["iters"])
        check_mixed_accuracy(o, bn, x.cpu().numpy(), ro)
    ax = oracle.apply(x.cpu().numpy(), w["k2"], w["h"], bc)
    assert np.linalg.norm(bn - ax) / np.linalg.norm(bn) <= 1.01 * tol


@pytest.mark.parametrize("name,n,bc,coarsest", CASES)
def test_fcycle_c128(helm, name, n, bc, coarsest):
    """One F-cycle (Sec. 3.4.5) in FP64 against the oracle's, same bound as the V-cycle."""
    s, o, k2, h, shape = make(helm, name, n, bc, coarsest)
    r = I.random_vector(shape, 8)
    z = s.fcycle(dev(r)).cpu().numpy()
    assert rel(z, o.fcycle(r)) <= 1e-12


@pytest.mark.parametrize("name,n,bc,coarsest", CASES)
def test_fcycle_c64(helm, name, n, bc, coarsest):
    s, o, k2, h, shape = make(helm, name, n, bc, coarsest)
    r = I.random_vector(shape, 9).astype(np.complex64)
    z = s.fcycle(dev(r)).cpu().numpy()
    err = rel(z, o.fcycle(r.astype(np.complex128)))
    assert err <= 4e-5, err


@pytest.mark.parametrize("krylov,precision", [("gmres", "fp64"), ("fgmres", "mixed"), ("bicgstab", "fp64")])
def test_solve_fcycle_vs_oracle(helm, krylov, precision):
    """F-cycle preconditioned solves on the wedge at n=32 against the oracle with the same
    preconditioner: residual, iteration counts and solutions at the solve bounds."""
    w = I.workload("wedge", 32)
    s = helm.Solver(w["n"], w["h"], w["k2"], S, krylov=krylov, precision=precision, cycle="f", max_iter=4000)
    o = oracle.Solver(w["n"], w["h"], S, w["k2"], cycle="f")
    b = s.rhs_point(w["sources"])
    x, info = s.solve(b)
    bn = b.cpu().numpy()
    if krylov == "bicgstab":
        ro = o.bicgstab(bn, tol=1e-6, max_iter=4000)
        slack = max(2, 0.1 * ro["iters"])
    else:
        ro = o.gmres(bn, restart=30, tol=1e-6, flexible=krylov == "fgmres")
        slack = 1
    assert info["status"] == 0 and ro["status"] == 0
    assert abs(info["iterations"] - ro["iters"]) <= slack, (info, ro["iters"])
    assert rel(x.cpu().numpy(), ro["x"]) <= 1e-5
    ax = oracle.apply(x.cpu().numpy(), w["k2"], w["h"], S)
    assert np.linalg.norm(bn - ax) / np.linalg.norm(bn) <= 1.01e-6


@pytest.mark.parametrize("s", [1, 4, 8])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("bc", [D, S])
def test_idrs_vs_oracle(helm, bc, precision, s):
    """Right-preconditioned IDR(s), biorthogonal form (the paper's outer solver, as IDR(4)),
    with the same seeded shadow space on both sides.  FP64: true residual to 1e-9, #Matvec
    within 10% of the oracle's (short recurrences amplify rounding-order differences, Sec.
    5.1.3).  Mixed precision: to the paper's 1e-6, #Matvec within 1.5x the FP64 oracle's
    (the complex64 V-cycle is a fixed preconditioner only up to its FP32 rounding)."""
    tol = 1e-9 if precision == "fp64" else 1e-6
    w = I.workload("small") if bc == D else I.workload("wedge", 32)
    s_ = helm.Solver(w["n"], w["h"], w["k2"], bc, krylov="idrs", idr_s=s, precision=precision, tol=tol,
                     max_iter=4000)
    shape = w["k2"].shape
    o = oracle.Solver(w["n"], w["h"], bc, w["k2"])
    b = s_.rhs_point(w["sources"])
    x, info = s_.solve(b)
    bn = b.cpu().numpy()
    ro = o.idrs(bn, I.shadow_space(shape, s), tol=tol, max_iter=4000)
    assert info["status"] == 0 and info["rel_residual"] <= tol and ro["status"] == 0, (info, ro["status"])
    if precision == "fp64":
        assert abs(info["iterations"] - ro["iters"]) <= max(2, 0.1 * ro["iters"]), (info, ro["iters"])
        assert rel(x.cpu().numpy(), ro["x"]) <= 1e-5
    else:
        assert info["iterations"] <= 1.5 * ro["iters"] + 2, (info, ro["iters"])
        check_mixed_accuracy(o, bn, x.cpu().numpy(), ro)
    ax = oracle.apply(x.cpu().numpy(), w["k2"], w["h"], bc)
    assert np.linalg.norm(bn - ax) / np.linalg.norm(bn) <= 1.01 * tol


def test_idrs_edge_cases(helm):
    """Zero right-hand side, warm start from the solution, the #Matvec cap, a replaced shadow
    space, and a shadow space beyond the largest s."""
    w = I.workload("wedge", 16)
    s = helm.Solver(w["n"], w["h"], w["k2"], S, krylov="idrs", idr_s=4, max_iter=400, tol=1e-9)
    b = s.rhs_point(w["sources"])
    z, iz = s.solve(torch.zeros_like(b))
    assert iz["iterations"] == 0 and torch.count_nonzero(z) == 0
    x, info = s.solve(b)
    assert info["status"] == 0
    x2, info2 = s.solve(b, x.clone())
    assert info2["iterations"] == 0
    s.set_shadow_space(I.shadow_space(w["k2"].shape, 2, seed=7))
    x3, info3 = s.solve(b)
    assert info3["status"] == 0 and rel(x3.cpu().numpy(), x.cpu().numpy()) <= 1e-5
    capped = helm.Solver(w["n"], w["h"], w["k2"], S, krylov="idrs", idr_s=4, max_iter=7, tol=1e-12)
    _, ic = capped.solve(b)
    assert ic["status"] == helm.ENOCONV and ic["iterations"] == 7
    with pytest.raises(helm.HelmError):
        s.set_shadow_space(I.shadow_space(w["k2"].shape, 9))


@pytest.mark.parametrize("krylov,precision", [("gmres", "fp64"), ("fgmres", "fp64"), ("fgmres", "mixed")])
def test_summed_basis_matches_textbook_gram_schmidt(helm, krylov, precision):
    """The three-FMA inner products and updates against the summed basis (gs_sums) compute the
    same Gram-Schmidt as the four-FMA textbook form up to rounding: on a ragged Sommerfeld wedge
    solved to 1e-10 the iteration counts agree within one and the solutions to 1e-8."""
    n = (40, 20, 12)
    h = 1.0 / 40
    k2 = I.k2_from_velocity(I.wedge_velocity(n), I.wedge_omega(40))
    out = []
    for sums in (True, False):
        s = helm.Solver(n, h, k2, S, krylov=krylov, precision=precision, tol=1e-10, max_iter=2000, gs_sums=sums)
        b = s.rhs_point([(20, 10, 0)])
        x, info = s.solve(b)
        assert info["status"] == 0 and info["rel_residual"] <= 1e-10, info
        out.append((x.cpu().numpy(), info["iterations"]))
        s.close()
    assert abs(out[0][1] - out[1][1]) <= 1, (out[0][1], out[1][1])
    assert rel(out[0][0], out[1][0]) <= 1e-8


@pytest.mark.parametrize("krylov,precision", [("gmres", "fp64"), ("fgmres", "mixed")])
def test_reorthogonalisation_threshold(helm, krylov, precision):
    """The selective second Gram-Schmidt pass at keep = 0.1 (default), 0.5 (the conservative
    eta = 1/sqrt(2)) and 0 (never, short of total cancellation), and always: on a ragged
    Sommerfeld wedge solved to 1e-10 the iteration counts agree within one and the solutions to
    1e-8, and the FP64 default solve matches the oracle's modified Gram-Schmidt GMRES."""
    n = (40, 20, 12)
    h = 1.0 / 40
    k2 = I.k2_from_velocity(I.wedge_velocity(n), I.wedge_omega(40))
    out = []
    for keep, reorth in ((0.1, None), (0.5, None), (0.0, None), (0.1, "always")):
        s = helm.Solver(n, h, k2, S, krylov=krylov, precision=precision, tol=1e-10, max_iter=2000, reorth_keep=keep,
                        reorth=reorth)
        b = s.rhs_point([(20, 10, 0)])
        x, info = s.solve(b)
        assert info["status"] == 0 and info["rel_residual"] <= 1e-10, (keep, reorth, info)
        out.append((x.cpu().numpy(), info["iterations"], b.cpu().numpy()))
        s.close()
    for x, it, _ in out[1:]:
        assert abs(it - out[0][1]) <= 1, (it, out[0][1])
        assert rel(x, out[0][0]) <= 1e-8
    if precision == "fp64":
        o = oracle.Solver(n, h, S, k2)
        ro = o.gmres(out[0][2], restart=30, tol=1e-10, max_iter=2000)
        assert ro["status"] == 0 and abs(ro["iters"] - out[0][1]) <= 1, (ro["iters"], out[0][1])
        assert rel(out[0][0], ro["x"]) <= 1e-8


@pytest.mark.parametrize("bc", [D, S])
def test_left_preconditioned_gmres_vs_oracle(helm, bc):
    """The paper's own GMRES (Sec. 3.2): left preconditioning with the preconditioned stopping
    rule (Sec. 5).  Same iterates as the oracle's left mode: iterations within +-1, solution
    within 1e-5, and the reported preconditioned relative residual below tol on both sides."""
    w = I.workload("small") if bc == D else I.workload("wedge", 32)
    s = helm.Solver(w["n"], w["h"], w["k2"], bc, krylov="gmres", side="left", restart=30)
    o = oracle.Solver(w["n"], w["h"], bc, w["k2"])
    b = s.rhs_point(w["sources"])
    x, info = s.solve(b)
    ro = o.gmres(b.cpu().numpy(), restart=30, tol=1e-6, left=True)
    assert info["status"] == 0 and ro["status"] == 0
    assert info["rel_residual"] <= 1e-6 and ro["relres"] <= 1e-6
    assert abs(info["iterations"] - ro["iters"]) <= 1, (info, ro["iters"])
    # with equal counts both sides stop on the same iterate up to rounding; when the last
    # estimate sits at the tolerance one side may take one more step (the +-1 above)
    if info["iterations"] == ro["iters"]:
        assert abs(info["rel_residual"] - ro["relres"]) <= 0.02 * ro["relres"]
    assert rel(x.cpu().numpy(), ro["x"]) <= 1e-5
    with pytest.raises(helm.HelmError):
        helm.Solver(w["n"], w["h"], w["k2"], bc, krylov="fgmres", side="left")


@pytest.mark.parametrize("name,n,bc,coarsest", CASES)
def test_apply_c64_double_float(helm, name, n, bc, coarsest):
    """A u for a complex64 u in double-float arithmetic (the A-product of the mixed-precision
    solver with double-float Gram-Schmidt) against the FP64 oracle on the same (exactly
    representable) input: about 48 significant bits, 2^-46 of the largest term, so 1e-12
    relative allows a cancellation factor of ~100 (kh <= 0.6)."""
    s, o, k2, h, shape = make(helm, name, n, bc, coarsest, precision="mixed", orth="df")
    u = I.random_vector(shape, 11).astype(np.complex64)
    v = s.apply_c64_df(dev(u)).cpu().numpy()
    vo = oracle.apply(u.astype(np.complex128), k2, h, bc)
    err = rel(v, vo)
    assert err <= 1e-12, err


def test_full_size_mixed_n256(helm):
    """The n = 256 mixed-precision workload (257^3 unknowns) at full size: the complex64
    V-cycle against the FP64 oracle's on the whole grid, and the mixed-precision double-float
    solve's true residual from the oracle's own operator."""
    w = I.workload("mixed", 256)
    s = helm.Solver(w["n"], w["h"], w["k2"], S, krylov="fgmres", precision="mixed", orth="df")
    o = oracle.Solver(w["n"], w["h"], S, w["k2"])
    r = I.random_vector(s.shape, 14).astype(np.complex64)
    z = s.vcycle(dev(r)).cpu().numpy()
    err = rel(z, o.vcycle(r.astype(np.complex128)))
    assert err <= 2e-5, err
    del o
    b = s.rhs_point(w["sources"])
    x, info = s.solve(b)
    assert info["status"] == 0
    bn = b.cpu().numpy()
    ax = oracle.apply(x.cpu().numpy(), w["k2"], w["h"], S)
    rr = np.linalg.norm(bn - ax) / np.linalg.norm(bn)
    assert rr <= 1.01e-6 and abs(rr - info["rel_residual"]) <= 1e-3 * rr


def test_full_size_batched_sources(helm):
    """Batched sources on the n = 128 wedge in the benchmark's batched configuration (complex64
    cycle, double-float Gram-Schmidt, F-cycle): every source's true residual from the oracle's
    operator."""
    w = I.workload("batched", 128)
    s = helm.Solver(w["n"], w["h"], w["k2"], S, krylov="fgmres", precision="mixed", orth="df", cycle="f")
    B = torch.stack([s.rhs_point([p]) for p in w["sources"][:4]])
    X, infos = s.solve_batched(B)
    for r in range(4):
        assert infos[r]["status"] == 0
        bn = B[r].cpu().numpy()
        ax = oracle.apply(X[r].cpu().numpy(), w["k2"], w["h"], S)
        rr = np.linalg.norm(bn - ax) / np.linalg.norm(bn)
        assert rr <= 1.01e-6, (r, rr)


def test_bicgstab_stall_window(helm):
    """Bi-CGSTAB's stagnation guard.  A window of 2 products asks the residual to halve on every
    step (two products).  In the oracle's Bi-CGSTAB on the n = 32 wedge the second step takes
    the true residual only from 3.4e-2 to 2.0e-2 (56 products in all to 1e-6), so the guarded
    solve stops after a few products with HELM_ENOCONV and says why.  With the guard off it converges, and the default window leaves the FP64 solve
    unchanged, bit for bit."""
    w = I.workload("wedge", 32)
    runs = {}
    for win in (2, 0, 1000):
        s = helm.Solver(w["n"], w["h"], w["k2"], S, krylov="bicgstab", stall_window=win, max_iter=4000)
        x, info = s.solve(s.rhs_point(w["sources"]))
        runs[win] = (x.cpu().numpy(), info)
        s.close()
    x0, i0 = runs[0]
    x1, i1 = runs[1000]
    assert i0["status"] == 0 and i1["status"] == 0 and i0["iterations"] == i1["iterations"]
    assert np.array_equal(x0, x1)
    x2, i2 = runs[2]
    assert i2["status"] == 4 and i2["iterations"] < i0["iterations"] and "stagnated" in i2["message"], i2
    assert np.all(np.isfinite(x2))
