"""FP64 CPU oracle for the CSLP-preconditioned matrix-free Helmholtz solver (arXiv 2308.06085).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  The CUDA library never loads it, and it shares
no code with the library: the arithmetic lives in ``oracle.c`` (plain loops written from the
paper) and this module only marshals numpy arrays to it.

Parity pins that tie this oracle to the paper and to mathematics, not to itself, live in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build_oracle import build as _build

DIRICHLET = 0
SOMMERFELD = 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = C.CDLL(path)
        dp, ip, vp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p
        i, d = C.c_int, C.c_double
        L.oracle_apply.argtypes = [i, i, i, d, i, dp, d, d, dp, dp]
        L.oracle_diag.argtypes = [i, i, i, d, i, dp, d, d, dp]
        L.oracle_jacobi.argtypes = [i, i, i, d, i, dp, d, d, d, dp, dp]
        L.oracle_restrict.argtypes = [i, i, i, i, dp, i, i, i, dp]
        L.oracle_prolong.argtypes = [i, i, i, i, dp, i, i, i, dp]
        L.oracle_create.argtypes = [i, i, i, d, i, dp, d, d, d, i, i, i]
        L.oracle_create.restype = vp
        L.oracle_destroy.argtypes = [vp]
        L.oracle_nlevels.argtypes = [vp]
        L.oracle_nlevels.restype = i
        L.oracle_level_info.argtypes = [vp, i, ip, dp]
        L.oracle_level_k2.argtypes = [vp, i, dp]
        L.oracle_vcycle.argtypes = [vp, dp, dp]
        L.oracle_fcycle.argtypes = [vp, dp, dp]
        L.oracle_set_cycle.argtypes = [vp, C.c_int]
        L.oracle_set_coarse_tol.argtypes = [vp, C.c_double]
        L.oracle_vcycle_down.argtypes = [vp, i, dp, dp]
        L.oracle_vcycle_up.argtypes = [vp, i, dp, dp, dp]
        L.oracle_coarse_solve.argtypes = [vp, dp, dp]
        L.oracle_gmres.argtypes = [vp, dp, dp, i, d, i, i, ip, dp, dp, i]
        L.oracle_gmres.restype = i
        L.oracle_rhs_point.argtypes = [i, i, i, i, d, i, ip, dp]
        L.oracle_rhs_closed_off.argtypes = [i, d, dp]
        L.oracle_adjoint_rhs.argtypes = [i, i, i, i, dp, dp]
        L.oracle_adjoint_finish.argtypes = [i, i, i, i, dp, dp]
        L.oracle_grad_k2.argtypes = [i, i, i, d, i, dp, dp, dp, dp]
        L.oracle_bicgstab.argtypes = [vp, dp, dp, d, i, ip, dp, dp, i]
        L.oracle_bicgstab.restype = i
        L.oracle_idrs.argtypes = [vp, i, dp, d, dp, dp, d, i, ip, dp, dp, i]
        L.oracle_idrs.restype = i
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def unknown_dims(n, bc):
    """Unknown count per direction for n intervals: n-1 (Dirichlet) or n+1 (Sommerfeld)."""
    return tuple(int(x) - 1 if bc == DIRICHLET else int(x) + 1 for x in n)


def apply(u, k2, h, bc, shift=(1.0, 0.0)):
    """v = (-Lap_h - s k^2) u on a 3D array shaped (N3, N2, N1) (x fastest)."""
    u = _c128(u)
    k2 = _f64(k2)
    N3, N2, N1 = u.shape
    v = np.empty_like(u)
    lib().oracle_apply(N1, N2, N3, h, bc, _dp(k2), shift[0], shift[1], _dp(u), _dp(v))
    return v


def diag(k2, h, bc, shift=(1.0, 0.0)):
    k2 = _f64(k2)
    N3, N2, N1 = k2.shape
    d = np.empty(k2.shape, dtype=np.complex128)
    lib().oracle_diag(N1, N2, N3, h, bc, _dp(k2), shift[0], shift[1], _dp(d))
    return d


def jacobi(u, b, k2, h, bc, shift, omega):
    u = _c128(u).copy()
    b = _c128(b)
    k2 = _f64(k2)
    N3, N2, N1 = u.shape
    lib().oracle_jacobi(N1, N2, N3, h, bc, _dp(k2), shift[0], shift[1], omega, _dp(b), _dp(u))
    return u


def restrict(r, coarse_shape, bc):
    r = _c128(r)
    Nf3, Nf2, Nf1 = r.shape
    Nc3, Nc2, Nc1 = coarse_shape
    out = np.empty(coarse_shape, dtype=np.complex128)
    lib().oracle_restrict(Nf1, Nf2, Nf3, bc, _dp(r), Nc1, Nc2, Nc3, _dp(out))
    return out


def prolong(e, fine_shape, bc):
    e = _c128(e)
    Nc3, Nc2, Nc1 = e.shape
    Nf3, Nf2, Nf1 = fine_shape
    out = np.empty(fine_shape, dtype=np.complex128)
    lib().oracle_prolong(Nc1, Nc2, Nc3, bc, _dp(e), Nf1, Nf2, Nf3, _dp(out))
    return out


def rhs_point(shape, bc, h, nodes):
    """Discrete Dirac RHS: 1/h^3 at each source node (node coordinates, 0..n)."""
    N3, N2, N1 = shape
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.int32).reshape(-1, 3))
    b = np.empty(shape, dtype=np.complex128)
    lib().oracle_rhs_point(N1, N2, N3, bc, h, len(nodes), nodes.ctypes.data_as(C.POINTER(C.c_int)), _dp(b))
    return b


def rhs_closed_off(n, k):
    N = n - 1
    b = np.empty((N, N, N), dtype=np.complex128)
    lib().oracle_rhs_closed_off(n, k, _dp(b))
    return b


def grad_k2(u, lam, k2, h, bc, grad=None):
    """grad += -Re(conj(lambda) dA/dk2 u) at every node (adjoint-state gradient)."""
    u, lam, k2 = _c128(u), _c128(lam), _f64(k2)
    N3, N2, N1 = u.shape
    g = np.zeros(u.shape) if grad is None else np.ascontiguousarray(grad, dtype=np.float64)
    lib().oracle_grad_k2(N1, N2, N3, h, bc, _dp(k2), _dp(u), _dp(lam), _dp(g))
    return g


class Solver:
    """Oracle multigrid hierarchy + V-cycle + right-preconditioned GMRES(m)."""

    def __init__(self, n, h, bc, k2, beta1=1.0, beta2=-0.5, omega=0.8, nu1=1, nu2=1, coarsest_n=4, cycle="v",
                 coarse_tol=0.0):
        n1, n2, n3 = (n, n, n) if np.isscalar(n) else tuple(n)
        self.bc = bc
        self.h = h
        self.shape = unknown_dims((n3, n2, n1), bc)
        self._k2 = _f64(k2).reshape(self.shape)
        self._ctx = lib().oracle_create(n1, n2, n3, h, bc, _dp(self._k2), beta1, beta2, omega, nu1, nu2, coarsest_n)
        if not self._ctx:
            raise ValueError("oracle_create rejected the arguments")
        self.beta1, self.beta2, self.omega = beta1, beta2, omega
        lib().oracle_set_cycle(self._ctx, {"v": 0, "f": 1}[cycle])
        # 0: exact coarsest solve; > 0: the paper's full GMRES to that relative residual
        lib().oracle_set_coarse_tol(self._ctx, coarse_tol)

    def __del__(self):
        ctx = getattr(self, "_ctx", None)
        if ctx and _lib is not None:
            _lib.oracle_destroy(ctx)
            self._ctx = None

    @property
    def nlevels(self):
        return lib().oracle_nlevels(self._ctx)

    def level(self, l):
        dims = (C.c_int * 6)()
        h = C.c_double()
        lib().oracle_level_info(self._ctx, l, dims, C.byref(h))
        N = (dims[5], dims[4], dims[3])
        k2 = np.empty(N, dtype=np.float64)
        lib().oracle_level_k2(self._ctx, l, _dp(k2))
        return {"n": (dims[0], dims[1], dims[2]), "shape": N, "h": h.value, "k2": k2}

    def vcycle(self, b):
        b = _c128(b).reshape(self.shape)
        z = np.empty_like(b)
        lib().oracle_vcycle(self._ctx, _dp(b), _dp(z))
        return z

    def fcycle(self, b):
        b = _c128(b).reshape(self.shape)
        z = np.empty_like(b)
        lib().oracle_fcycle(self._ctx, _dp(b), _dp(z))
        return z

    def vcycle_down(self, l, b):
        shape_c = self.level(l + 1)["shape"]
        b = _c128(b).reshape(self.level(l)["shape"])
        out = np.empty(shape_c, dtype=np.complex128)
        lib().oracle_vcycle_down(self._ctx, l, _dp(b), _dp(out))
        return out

    def vcycle_up(self, l, b, e):
        shape = self.level(l)["shape"]
        b = _c128(b).reshape(shape)
        e = _c128(e).reshape(self.level(l + 1)["shape"])
        out = np.empty(shape, dtype=np.complex128)
        lib().oracle_vcycle_up(self._ctx, l, _dp(b), _dp(e), _dp(out))
        return out

    def coarse_solve(self, b):
        L = self.level(self.nlevels - 1)
        b = _c128(b).reshape(L["shape"])
        e = np.empty_like(b)
        lib().oracle_coarse_solve(self._ctx, _dp(b), _dp(e))
        return e

    def solve_adjoint(self, g, restart=30, tol=1e-6, max_iter=1000):
        """lambda with A^H lambda = g: solve A nu = D^-1 conj(g) by the same GMRES, then
        lambda = conj(D nu), D = diag(2^-faces)."""
        g = _c128(g).reshape(self.shape)
        N3, N2, N1 = self.shape
        q = np.empty_like(g)
        lib().oracle_adjoint_rhs(N1, N2, N3, self.bc, _dp(g), _dp(q))
        r = self.gmres(q, restart=restart, tol=tol, max_iter=max_iter)
        lam = np.empty_like(g)
        lib().oracle_adjoint_finish(N1, N2, N3, self.bc, _dp(r["x"]), _dp(lam))
        r["x"] = lam
        return r

    def adjoint_grad(self, sources, rec_idx, d_obs, restart=30, tol=1e-6, max_iter=1000):
        """Loss 1/2 sum_s |u_s(R) - d_s|^2 over point sources and its gradient w.r.t. k^2.
        rec_idx: flat unknown indices of the receivers; d_obs: (nsrc, nrec) complex."""
        rec_idx = np.asarray(rec_idx, dtype=np.int64)
        grad = np.zeros(self.shape)
        loss = 0.0
        for s, src in enumerate(sources):
            b = rhs_point(self.shape, self.bc, self.h, [src])
            u = self.gmres(b, restart=restart, tol=tol, max_iter=max_iter)["x"]
            res = u.ravel()[rec_idx] - np.asarray(d_obs)[s]
            loss += 0.5 * float(np.sum(np.abs(res) ** 2))
            g = np.zeros(u.size, dtype=np.complex128)
            g[rec_idx] = res
            lam = self.solve_adjoint(g.reshape(self.shape), restart=restart, tol=tol, max_iter=max_iter)["x"]
            grad = grad_k2(u, lam, self._k2, self.h, self.bc, grad)
        return loss, grad

    def bicgstab(self, b, x0=None, tol=1e-6, max_iter=2000, history=False):
        """Right-preconditioned Bi-CGSTAB with one V-cycle as M^{-1}; iters counts A-products."""
        b = _c128(b).reshape(self.shape)
        x = np.zeros_like(b) if x0 is None else _c128(x0).reshape(self.shape).copy()
        it, rr = C.c_int(), C.c_double()
        hist = np.zeros(max(max_iter, 1))
        st = lib().oracle_bicgstab(self._ctx, _dp(b), _dp(x), tol, max_iter, C.byref(it), C.byref(rr), _dp(hist),
                                   len(hist))
        out = {"x": x, "iters": it.value, "relres": rr.value, "status": st}
        if history:
            out["history"] = hist[: it.value].copy()
        return out

    def idrs(self, b, P, x0=None, kappa=0.7, tol=1e-6, max_iter=2000, history=False):
        """Right-preconditioned biorthogonal IDR(s), s = number of shadow vectors in P (shaped
        (s,) + unknown shape, complex); iters counts A-products."""
        b = _c128(b).reshape(self.shape)
        P = _c128(P).reshape((-1,) + self.shape)
        x = np.zeros_like(b) if x0 is None else _c128(x0).reshape(self.shape).copy()
        it, rr = C.c_int(), C.c_double()
        hist = np.zeros(max(max_iter, 1))
        st = lib().oracle_idrs(self._ctx, P.shape[0], _dp(P), kappa, _dp(b), _dp(x), tol, max_iter, C.byref(it),
                               C.byref(rr), _dp(hist), len(hist))
        if st == -2:
            raise ValueError("s out of range")
        out = {"x": x, "iters": it.value, "relres": rr.value, "status": st}
        if history:
            out["history"] = hist[: it.value].copy()
        return out

    def gmres(self, b, x0=None, restart=30, tol=1e-6, max_iter=1000, flexible=False, history=False, left=False):
        """Right-preconditioned GMRES(m) (FGMRES with flexible=True); left=True runs the paper's
        left-preconditioned form, whose relres is the preconditioned residual."""
        b = _c128(b).reshape(self.shape)
        x = np.zeros_like(b) if x0 is None else _c128(x0).reshape(self.shape).copy()
        it = C.c_int()
        rr = C.c_double()
        hist = np.zeros(max(max_iter, 1), dtype=np.float64)
        st = lib().oracle_gmres(self._ctx, _dp(b), _dp(x), restart, tol, max_iter, 2 if left else int(flexible),
                                C.byref(it), C.byref(rr), _dp(hist), len(hist))
        out = {"x": x, "iters": it.value, "relres": rr.value, "status": st}
        if history:
            out["history"] = hist[: it.value].copy()
        return out
