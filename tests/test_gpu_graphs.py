"""CUDA-graph replay of solver steps (helm_params.graphs): a step captured once and replayed
runs the same kernels with the same launch shapes and the same deterministic reductions, so a
solve with graphs must equal the plain-launch solve bit for bit, on first use (capture) and on
replay, for every Krylov method and precision mode, and into a second solution buffer (steps
that write x are captured per buffer)."""
import numpy as np
import pytest
import torch

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


@pytest.mark.parametrize("krylov,precision,orth,cycle", [
    ("gmres", "fp64", "fp64", "v"), ("fgmres", "mixed", "df", "v"), ("gmres", "fp64", "df", "f"),
    ("bicgstab", "fp64", None, "v"), ("idrs", "fp64", None, "v"), ("idrs", "mixed", None, "f")])
def test_graph_replay_is_bit_exact(helm, krylov, precision, orth, cycle):
    w = I.workload("wedge", 32)
    kw = dict(krylov=krylov, precision=precision, orth=orth, cycle=cycle, restart=12, max_iter=4000)
    plain = helm.Solver(w["n"], w["h"], w["k2"], S, graphs=False, **kw)
    graph = helm.Solver(w["n"], w["h"], w["k2"], S, graphs=True, **kw)
    b = plain.rhs_point(w["sources"])
    x0, i0 = plain.solve(b)
    x1, i1 = graph.solve(b)                # first use: captures
    x2, i2 = graph.solve(b)                # replay; steps that write x captured for the new buffer
    x2b, i3 = graph.solve(b, torch.zeros_like(x2).copy_(x2).zero_())  # replay into another buffer
    x4, i4 = graph.solve(b, x2.zero_())    # replay into the second solve's buffer
    for xi, ii in ((x1, i1), (x2b, i3), (x4, i4)):
        assert ii["status"] == 0 and ii["iterations"] == i0["iterations"], (ii, i0)
        assert torch.equal(xi, x0)
    assert i2["iterations"] == i0["iterations"]


def test_graph_cycle_shorter_than_restart(helm):
    """A cycle cut short by max_iter (jmax < m) runs its columns as plain launches."""
    w = I.workload("wedge", 16)
    kw = dict(krylov="gmres", restart=30, tol=1e-14, max_iter=35)
    a = helm.Solver(w["n"], w["h"], w["k2"], S, graphs=False, **kw)
    g = helm.Solver(w["n"], w["h"], w["k2"], S, graphs=True, **kw)
    b = a.rhs_point(w["sources"])
    xa, ia = a.solve(b)
    xg, ig = g.solve(b)
    assert ia["iterations"] == ig["iterations"] == 35
    assert torch.equal(xa, xg)


@pytest.mark.parametrize("n,bc,coarsest", [((32, 32, 32), 1, 4), ((40, 20, 12), 0, 2), ((24, 8, 16), 1, 2)])
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_fused_coarse_cycle_is_bit_exact(helm, n, bc, coarsest, dtype):
    """The coarse levels run as one single-CTA kernel (helm_params.fuse_coarse) with the same
    arithmetic per point as the level-by-level kernels: V-cycles, F-cycles and whole solves
    must agree bit for bit with fusion off."""
    h = 1.0 / max(n)
    shape = I.unknown_shape(n, bc)
    k2 = I.random_k2(shape, seed=5, kmin=2.0, kmax=0.6 / h)
    a = helm.Solver(n, h, k2, bc, coarsest_n=coarsest, fuse_coarse=False)
    f = helm.Solver(n, h, k2, bc, coarsest_n=coarsest, fuse_coarse=True)
    r = torch.from_numpy(I.random_vector(shape, 12)).cuda().to(dtype)
    assert torch.equal(a.vcycle(r), f.vcycle(r))
    assert torch.equal(a.fcycle(r), f.fcycle(r))
    if dtype == torch.complex128:
        b = a.rhs_point([(n[0] // 2, n[1] // 2, n[2] // 2)])
        xa, ia = a.solve(b)
        xf, i_f = f.solve(b)
        assert ia["iterations"] == i_f["iterations"] and torch.equal(xa, xf)


@pytest.mark.parametrize("orth,cycle", [("fp64", "v"), ("df", "f")])
def test_batched_graph_replay_is_bit_exact(helm, orth, cycle):
    """The batched solver's Arnoldi columns replayed from graphs (per batch width) against plain
    launches, for two widths in a row (the wider one reallocates the workspace)."""
    w = I.workload("batched", 16)
    kw = dict(krylov="fgmres", precision="mixed", orth=orth, cycle=cycle)
    plain = helm.Solver(w["n"], w["h"], w["k2"], S, graphs=False, **kw)
    graph = helm.Solver(w["n"], w["h"], w["k2"], S, graphs=True, **kw)
    src = [(4 + 2 * (i % 4), 4 + 3 * (i // 4), 2) for i in range(8)]
    B = torch.stack([plain.rhs_point([p]) for p in src])
    for width in (3, 8, 8):
        X0, i0 = plain.solve_batched(B[:width])
        X1, i1 = graph.solve_batched(B[:width])
        assert [a["iterations"] for a in i0] == [a["iterations"] for a in i1]
        assert torch.equal(X0, X1)


@pytest.mark.parametrize("n", [32, 64])
def test_autotuned_shapes_are_bit_exact(helm, n):
    """Launch shapes (and the shared-memory tiled FP32 stencils the autotuner may pick) change
    the schedule, not the arithmetic of a point: complex64 V-cycles and mixed-precision solves
    with the autotuner equal those with the fixed default shape bit for bit."""
    w = I.workload("wedge", n)
    a = helm.Solver(w["n"], w["h"], w["k2"], S, krylov="fgmres", precision="mixed", autotune=False)
    t = helm.Solver(w["n"], w["h"], w["k2"], S, krylov="fgmres", precision="mixed", autotune=True)
    tiled = any(rec[1] == 12 for rec in t.tune_log())
    assert tiled, "the tiled FP32 stencil was never timed"
    r = torch.from_numpy(I.random_vector(t.shape, 13).astype(np.complex64)).cuda()
    assert torch.equal(a.vcycle(r), t.vcycle(r))
    b = a.rhs_point(w["sources"])
    xa, ia = a.solve(b)
    xt, it = t.solve(b)
    assert ia["iterations"] == it["iterations"] and torch.equal(xa, xt)


@pytest.mark.parametrize("name,n,bc", [("wedge32", 32, S), ("som_ragged", (40, 20, 12), S), ("dir_ragged", (40, 20, 12), 0),
                                       ("wedge64", 64, S)])
def test_sweep_forms_are_bit_exact(helm, name, n, bc):
    """The complex64 down-sweep as three kernels, as pre-smoothing + residual then restriction,
    as one kernel that keeps the residual in shared memory, or as pre-smoothing then residual +
    restriction in one kernel (fuse_down 0 / 1 / 2 / 3), and the up-sweep as two kernels or one
    (fuse_up 0 / 1), also with the autotuner's planes per CTA, compute every point with the same
    arithmetic: V-cycles, F-cycles and mixed-precision solves agree bit for bit."""
    h = 1.0 / (n if np.isscalar(n) else max(n))
    if name.startswith("wedge"):
        k2 = I.workload("wedge", n)["k2"]
    else:
        k2 = I.random_k2(I.unknown_shape(n, bc), seed=sum(map(ord, name)), kmin=2.0, kmax=0.6 / h)
    outs = []
    for fuse, up, tune in ((0, 0, False), (1, 0, False), (2, 1, False), (3, 1, False), (3, 0, False), (2, 1, True),
                           (0, 1, True)):
        s = helm.Solver(n, h, k2, bc, krylov="fgmres", precision="mixed", coarsest_n=2, fuse_down=fuse, fuse_up=up,
                        autotune=tune)
        for lev in range(s.nlevels - 1):
            v = s.kernel_variants(lev)
            assert v["down_full"] == (fuse == 2) and v["fused_down"] == (fuse == 1), (lev, v)
            assert v["rr"] == (fuse == 3) and v["up_full"] == (up == 1), (lev, v)
        r = torch.from_numpy(I.random_vector(s.shape, 21).astype(np.complex64)).cuda()
        src = [tuple(m // 2 for m in ((n, n, n) if np.isscalar(n) else n))]
        b = s.rhs_point(src)
        x, info = s.solve(b)
        outs.append((s.vcycle(r), s.fcycle(r), x, info["iterations"]))
        s.close()
    for o in outs[1:]:
        assert torch.equal(o[0], outs[0][0]) and torch.equal(o[1], outs[0][1])
        assert o[3] == outs[0][3] and torch.equal(o[2], outs[0][2])


@pytest.mark.parametrize("name,n,bc", [("wedge32", 32, S), ("som_ragged", (40, 20, 12), S), ("dir_ragged", (40, 20, 12), 0),
                                       ("som_noncubic", (24, 8, 16), S)])
def test_fp64_sweep_forms_are_bit_exact(helm, name, n, bc):
    """The FP64 cycle's down-sweep as three kernels or as pre-smoothing then residual +
    restriction in one kernel (fuse_down 0 / 3), its up-sweep as two kernels or one (fuse_up
    0 / 1), and the autotuner's choice among them: V-cycles, F-cycles and FP64 solves agree bit
    for bit (the fused kernels read the same coefficient table and sum in the same order)."""
    h = 1.0 / (n if np.isscalar(n) else max(n))
    if name.startswith("wedge"):
        k2 = I.workload("wedge", n)["k2"]
    else:
        k2 = I.random_k2(I.unknown_shape(n, bc), seed=sum(map(ord, name)), kmin=2.0, kmax=0.6 / h)
    outs = []
    for fuse, up, tune in ((0, 0, False), (3, 1, False), (3, 0, False), (0, 1, False), (-1, -1, True)):
        s = helm.Solver(n, h, k2, bc, krylov="gmres", coarsest_n=2, fuse_down=fuse, fuse_up=up, autotune=tune)
        if not tune:
            for lev in range(s.nlevels - 1):
                v = s.kernel_variants(lev)
                assert v["rr"] == (fuse == 3) and v["up_full"] == (up == 1), (lev, v)
        r = torch.from_numpy(I.random_vector(s.shape, 22)).cuda()
        src = [tuple(m // 2 for m in ((n, n, n) if np.isscalar(n) else n))]
        b = s.rhs_point(src)
        x, info = s.solve(b)
        outs.append((s.vcycle(r), s.fcycle(r), x, info["iterations"]))
        s.close()
    for o in outs[1:]:
        assert torch.equal(o[0], outs[0][0]) and torch.equal(o[1], outs[0][1])
        assert o[3] == outs[0][3] and torch.equal(o[2], outs[0][2])


@pytest.mark.parametrize("orth,sums", [("fp64", True), ("fp64", False), ("df", True)])
def test_dot_variants_are_bit_exact(helm, orth, sums):
    """Every Gram-Schmidt inner-product kernel variant the autotuner chooses from (w staged or
    not, 2, 4 or 8 basis vectors per warp pass) sums each inner product over the same points in
    the same order: solves agree bit for bit whichever variant runs."""
    w = I.workload("wedge", 32)
    s = helm.Solver(w["n"], w["h"], w["k2"], S, krylov="gmres", orth=orth, gs_sums=sums, restart=20)
    b = s.rhs_point(w["sources"])
    out = []
    nvar = 3 if orth == "df" else 2
    for v in range(nvar):
        assert s.dot_variant(v) == v
        x, info = s.solve(b)
        out.append((x.clone(), info["iterations"]))
    for x, it in out[1:]:
        assert it == out[0][1] and torch.equal(x, out[0][0])
    with pytest.raises(helm.HelmError):
        s.dot_variant(nvar)


def test_autotuned_batched_double_float_is_bit_exact(helm):
    """The batched double-float inner products: whichever slots-per-pass variant and launch
    shapes the autotuner picks for a width, the batched solve equals the untuned one bit for bit."""
    w = I.workload("wedge", 32)
    kw = dict(krylov="fgmres", precision="mixed", orth="df", restart=12)
    a = helm.Solver(w["n"], w["h"], w["k2"], S, autotune=False, **kw)
    t = helm.Solver(w["n"], w["h"], w["k2"], S, autotune=True, **kw)
    src = [(8 + 4 * i, 8 + 4 * j, 1) for i in range(3) for j in range(3)]
    B = torch.stack([a.rhs_point([p]) for p in src])
    Xa, ia = a.solve_batched(B)
    Xt, it = t.solve_batched(B)
    assert [q["iterations"] for q in ia] == [q["iterations"] for q in it]
    assert torch.equal(Xa, Xt)
