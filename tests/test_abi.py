"""The C ABI library builds, loads without a GPU, and exports every entry point that
include/helm.h declares; argument validation that happens before any device work is
checked here too (host logic only, no kernels run)."""
import ctypes as C
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "helm.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^HELM_API\s+[\w\s\*]+?\b(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libhelm():
    from paper_2308_06085_gb300 import build_ext

    path = build_ext.build()
    return C.CDLL(path)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for want in ("helm_create", "helm_destroy", "helm_apply", "cslp_vcycle", "helm_solve", "helm_last_error",
                 "helm_rhs_point", "helm_vcycle_stage", "helm_default_params"):
        assert want in names


def test_every_declared_symbol_is_exported(libhelm):
    for name in declared_functions():
        assert hasattr(libhelm, name), name


def test_default_params_are_the_papers(libhelm):
    from paper_2308_06085_gb300 import helm

    p = helm.Params()
    libhelm.helm_default_params(C.byref(p))
    assert (p.beta1, p.beta2, p.omega, p.nu1, p.nu2) == (1.0, -0.5, 0.8, 1, 1)
    assert (p.restart, p.tol, p.krylov, p.precision) == (30, 1e-6, 0, 0)
    assert (p.graphs, p.autotune, p.side, p.fuse_coarse, p.gs_sums, p.fuse_down, p.fuse_up) == (1, 1, 0, 0, 1, -1, -1)
    assert p.stall_window == 1000 and p.reorth_keep == 0.1 and p.coarse_tol == 0.0


@pytest.mark.parametrize("args,msg", [
    ((1, 8, 8, 0.1, 1, 0), "interval counts"),
    ((8, 8, 8, 0.0, 1, 0), "h must be"),
    ((8, 8, 8, 0.1, 0, 0), "k2 is NULL"),
    ((8, 8, 8, 0.1, 1, 5), "boundary"),
])
def test_create_rejects_bad_arguments_before_device_work(libhelm, args, msg):
    libhelm.helm_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_int, C.c_void_p,
                                    C.c_void_p, C.POINTER(C.c_void_p)]
    libhelm.helm_last_error.argtypes = [C.c_void_p]
    libhelm.helm_last_error.restype = C.c_char_p
    n1, n2, n3, h, k2_nonnull, bc = args
    dummy = (C.c_double * 4)()
    out = C.c_void_p(123)
    st = libhelm.helm_create(n1, n2, n3, h, C.cast(dummy, C.c_void_p) if k2_nonnull else None, bc, None, None,
                             C.byref(out))
    assert st == 1 and not out.value
    assert msg in libhelm.helm_last_error(None).decode()


def test_bad_parameters_rejected(libhelm):
    from paper_2308_06085_gb300 import helm

    dummy = (C.c_double * 4)()
    for field, val, msg in [("nu1", 2, "nu1"), ("restart", 0, "restart"), ("coarsest_n", 1, "coarsest_n"),
                            ("omega", 0.0, "omega"), ("tol", 0.0, "tol"), ("precision", 7, "precision"),
                            ("gs_sums", 2, "gs_sums"), ("side", 3, "side"), ("cycle", 2, "cycle"),
                            ("fuse_down", 4, "fuse_down"), ("fuse_up", 2, "fuse_up"),
                            ("stall_window", -1, "stall_window"), ("reorth_keep", 1.0, "reorth_keep"),
                            ("coarse_tol", -1.0, "coarse_tol")]:
        p = helm.Params()
        libhelm.helm_default_params(C.byref(p))
        setattr(p, field, val)
        out = C.c_void_p()
        st = libhelm.helm_create(8, 8, 8, 0.1, C.cast(dummy, C.c_void_p), 1, C.cast(C.pointer(p), C.c_void_p), None,
                                 C.byref(out))
        assert st == 1, field
        assert msg in libhelm.helm_last_error(None).decode()


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2308_06085_gb300 import helm

    monkeypatch.setattr(helm, "_lib", None)
    monkeypatch.setattr(helm, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        helm.lib()


def test_noalloc_binding_rejects_bad_tensors_before_any_launch():
    """The binding of the allocation-free entry point checks dtype, size and device of k^2 and
    b on the host, so a wrong tensor never reaches the kernels as a raw pointer."""
    import torch

    from paper_2308_06085_gb300 import helm

    n, bc = (8, 8, 8), helm.SOMMERFELD
    fine = 9 ** 3
    k2 = torch.ones(fine, dtype=torch.float64)
    b = torch.zeros(fine, dtype=torch.complex128)
    with pytest.raises(TypeError):  # complex64 b would be read as complex128: twice its bytes
        helm.vcycle_down_noalloc(n, 0.125, k2, b.to(torch.complex64), bc=bc)
    with pytest.raises(TypeError):
        helm.vcycle_down_noalloc(n, 0.125, k2.float(), b, bc=bc)
    with pytest.raises(ValueError):  # one unknown short
        helm.vcycle_down_noalloc(n, 0.125, k2[:-1], b, bc=bc)
    with pytest.raises(ValueError):  # the Dirichlet grid of the same n has 7^3 unknowns
        helm.vcycle_down_noalloc(n, 0.125, k2, b, bc=helm.DIRICHLET)
    with pytest.raises(ValueError):  # host tensors are not device pointers
        helm.vcycle_down_noalloc(n, 0.125, k2, b, bc=bc)
    with pytest.raises(ValueError):
        helm.vcycle_down_noalloc(n, 0.125, k2, b, bc=7)
