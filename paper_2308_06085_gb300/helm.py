"""Python binding of libhelm (include/helm.h): argument marshalling only.

Every step of the solve runs in the CUDA kernels of ``libhelm.so``; this module converts
torch tensors to pointers, passes torch's current CUDA stream, and raises on error codes.
There is no CPU fallback: without the built library every call raises.

Tensor layout: a grid vector is a contiguous tensor shaped (N3, N2, N1) (x fastest) of
dtype complex128 (FP64 path) or complex64 (FP32 path) on a CUDA device.  k^2 is float64.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhelm.so")

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ETIMEOUT, ENUMERIC = range(7)
STATUS = {0: "HELM_OK", 1: "HELM_EINVAL", 2: "HELM_ENOMEM", 3: "HELM_ECUDA", 4: "HELM_ENOCONV",
          5: "HELM_ETIMEOUT", 6: "HELM_ENUMERIC"}
DIRICHLET, SOMMERFELD = 0, 1
C128, C64 = 0, 1
OP_A, OP_M = 0, 1
GMRES, FGMRES, BICGSTAB, IDRS = 0, 1, 2, 3
PREC_FP64, PREC_MIXED = 0, 1
ORTH_FP64, ORTH_DF = 0, 1
REORTH_ALWAYS, REORTH_SELECTIVE = 0, 1


class HelmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("beta1", C.c_double), ("beta2", C.c_double), ("omega", C.c_double), ("nu1", C.c_int),
                ("nu2", C.c_int), ("coarsest_n", C.c_int), ("krylov", C.c_int), ("restart", C.c_int),
                ("tol", C.c_double), ("max_iter", C.c_int), ("precision", C.c_int), ("orth", C.c_int),
                ("reorth", C.c_int), ("cycle", C.c_int), ("idr_kappa", C.c_double),
                ("graphs", C.c_int), ("autotune", C.c_int), ("side", C.c_int),
                ("fuse_coarse", C.c_int), ("gs_sums", C.c_int), ("fuse_down", C.c_int), ("fuse_up", C.c_int),
                ("stall_window", C.c_int), ("reorth_keep", C.c_double), ("coarse_tol", C.c_double)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_longlong), ("ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("status", C.c_int),
                ("rel_residual", C.c_double), ("ms_total", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libhelm.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libhelm.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    L.helm_default_params.argtypes = [C.POINTER(Params)]
    L.helm_default_params.restype = None
    L.helm_create.argtypes = [i, i, i, d, vp, i, C.POINTER(Params), vp, C.POINTER(vp)]
    L.helm_destroy.argtypes = [vp]
    L.helm_levels.argtypes = [vp, C.POINTER(i)]
    L.helm_level_dims.argtypes = [vp, i, C.POINTER(i), C.POINTER(d)]
    L.helm_apply.argtypes = [vp, i, i, vp, vp, vp]
    L.cslp_vcycle.argtypes = [vp, i, vp, vp, vp]
    L.cslp_fcycle.argtypes = [vp, i, vp, vp, vp]
    L.helm_set_shadow_space.argtypes = [vp, i, vp, vp]
    L.helm_apply_c64_df.argtypes = [vp, vp, vp, vp]
    L.helm_launch_shapes.argtypes = [vp, i, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.helm_launch_shapes.restype = i
    L.helm_tune_log.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_float), i, C.POINTER(C.c_int)]
    L.helm_tune_log.restype = i
    L.helm_dot_variant.argtypes = [vp, i, C.POINTER(C.c_int)]
    L.helm_dot_variant.restype = i
    L.helm_kernel_variants.argtypes = [vp, i, C.POINTER(C.c_int)]
    L.helm_kernel_variants.restype = i
    L.helm_apply_c64_df.restype = i
    L.helm_set_shadow_space.restype = i
    L.cslp_fcycle.restype = i
    L.helm_vcycle_stage.argtypes = [vp, i, i, i, vp, vp, vp, vp]
    L.helm_rhs_point.argtypes = [vp, i, C.POINTER(i), vp, vp]
    L.helm_solve.argtypes = [vp, vp, vp, C.POINTER(SolveInfo), vp]
    L.helm_solve_zero.argtypes = [vp, vp, vp, C.POINTER(SolveInfo), vp]
    L.helm_coarse_info.argtypes = [vp, C.POINTER(i), C.POINTER(i)]
    L.helm_coarse_info.restype = i
    L.helm_profile.argtypes = [vp, i]
    L.helm_profile_read.argtypes = [vp, C.POINTER(KernelStat), i, C.POINTER(i), C.POINTER(C.c_longlong)]
    L.helm_solve_batched.argtypes = [vp, i, vp, vp, C.POINTER(SolveInfo), vp]
    L.helm_solve_batched.restype = i
    L.helm_solve_adjoint.argtypes = [vp, vp, vp, C.POINTER(SolveInfo), vp]
    L.helm_solve_adjoint_batched.argtypes = [vp, i, vp, vp, C.POINTER(SolveInfo), vp]
    L.helm_solve_adjoint_batched.restype = i
    L.helm_grad_k2.argtypes = [vp, vp, vp, vp, vp]
    L.helm_adjoint_grad.argtypes = [vp, i, C.POINTER(i), i, C.POINTER(i), vp, vp, C.POINTER(d), C.POINTER(SolveInfo),
                                    vp]
    for f in ("helm_solve_adjoint", "helm_grad_k2", "helm_adjoint_grad"):
        getattr(L, f).restype = i
    L.helm_vcycle_down_noalloc.argtypes = [i, i, i, d, vp, i, d, d, d, vp, vp, vp]
    L.helm_vcycle_down_noalloc.restype = i
    L.helm_convert_check.argtypes = [vp, vp, C.c_size_t, vp]
    L.helm_convert_check.restype = i
    L.helm_last_error.argtypes = [vp]
    L.helm_last_error.restype = C.c_char_p
    for f in ("helm_create", "helm_destroy", "helm_levels", "helm_level_dims", "helm_apply", "cslp_vcycle",
              "helm_vcycle_stage", "helm_rhs_point", "helm_solve", "helm_solve_zero", "helm_profile", "helm_profile_read"):
        getattr(L, f).restype = i
    _lib = L
    return L


def default_params():
    p = Params()
    lib().helm_default_params(C.byref(p))
    return p


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


_DT = {torch.complex128: C128, torch.complex64: C64}


def convert_check(x32):
    """The kernels' own FP32 -> FP64 conversion (integer instructions) applied to a float32 CUDA
    tensor; returns float64."""
    x32 = x32.reshape(-1).contiguous()
    if x32.dtype != torch.float32:
        raise TypeError("convert_check takes a float32 tensor")
    o64 = torch.empty(x32.shape, dtype=torch.float64, device=x32.device)
    st = lib().helm_convert_check(_ptr(x32), _ptr(o64), x32.numel(), _stream())
    if st != OK:
        raise HelmError(st, lib().helm_last_error(None).decode())
    return o64


NOALLOC_MAX_POINTS = 262144


def vcycle_down_noalloc(n, h, k2, b, bc=SOMMERFELD, beta1=1.0, beta2=-0.5, omega=0.8):
    """Finest-level down stage R(b - M omega D^-1 b) with no context and no device allocation
    inside the library (for callers that may not allocate).  k2: float64 CUDA tensor at the
    fine unknowns; b: complex128 CUDA tensor; returns the coarse right-hand side (the output
    tensor is the caller's allocation)."""
    n1, n2, n3 = (n, n, n) if np.isscalar(n) else tuple(int(x) for x in n)
    if bc not in (DIRICHLET, SOMMERFELD):
        raise ValueError(f"unknown boundary condition {bc}")
    d = -1 if bc == DIRICHLET else 1
    fine = (n3 + d) * (n2 + d) * (n1 + d)
    # the library reads fine-grid vectors through raw pointers: check type, device, layout and
    # size here, before anything is launched
    args = (("k2", k2, torch.float64), ("b", b, torch.complex128))
    for name, t, dt in args:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if t.dtype != dt:
            raise TypeError(f"{name} must be {dt}, got {t.dtype}")
    for name, t, _ in args:
        if t.numel() != fine:
            raise ValueError(f"{name} has {t.numel()} elements; the fine grid has {fine} unknowns")
    for name, t, _ in args:
        if t.device.type != "cuda" or t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must be on the current CUDA device, got {t.device}")
    k2 = k2.reshape(-1).contiguous()
    b = b.reshape(-1).contiguous()
    cshape = (n3 // 2 + d, n2 // 2 + d, n1 // 2 + d)
    out = torch.empty(cshape, dtype=torch.complex128, device=b.device)
    st = lib().helm_vcycle_down_noalloc(n1, n2, n3, float(h), _ptr(k2), bc, beta1, beta2, omega, _ptr(b), _ptr(out),
                                        _stream())
    if st != OK:
        raise HelmError(st, lib().helm_last_error(None).decode())
    return out


class Solver:
    """A libhelm context: hierarchy, coarsest inverse and Krylov workspace on one GPU."""

    def __init__(self, n, h, k2, bc=SOMMERFELD, *, beta1=1.0, beta2=-0.5, omega=0.8, coarsest_n=4,
                 krylov="gmres", restart=30, tol=1e-6, max_iter=2000, precision="fp64", orth=None,
                 reorth=None, cycle="v", idr_s=4, idr_kappa=0.7, shadow=None, graphs=True, autotune=True, side="right", fuse_coarse=False, gs_sums=True, fuse_down=-1, fuse_up=-1, stall_window=1000,
                 reorth_keep=0.1, coarse_tol=0.0, device=None):
        n1, n2, n3 = (n, n, n) if np.isscalar(n) else tuple(int(x) for x in n)
        self.n = (n1, n2, n3)
        self.h = float(h)
        self.bc = bc
        d = -1 if bc == DIRICHLET else 1
        self.shape = (n3 + d, n2 + d, n1 + d)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        k2t = torch.as_tensor(k2, dtype=torch.float64)
        if tuple(k2t.shape) != self.shape:
            k2t = k2t.reshape(self.shape)
        k2t = k2t.to(self.device).contiguous()
        p = default_params()
        p.beta1, p.beta2, p.omega, p.coarsest_n = beta1, beta2, omega, coarsest_n
        p.krylov = {"gmres": GMRES, "fgmres": FGMRES, "bicgstab": BICGSTAB, "idrs": IDRS}[krylov]
        p.idr_kappa = idr_kappa
        p.graphs = int(bool(graphs))
        p.autotune = int(bool(autotune))
        p.side = {"right": 0, "left": 1}[side]
        p.fuse_coarse = int(bool(fuse_coarse))
        p.gs_sums = int(bool(gs_sums))
        p.fuse_down = int(fuse_down)
        p.fuse_up = int(fuse_up)
        p.stall_window = int(stall_window)
        p.reorth_keep = float(reorth_keep)
        p.coarse_tol = float(coarse_tol)
        p.restart, p.tol, p.max_iter = restart, tol, max_iter
        p.precision = {"fp64": PREC_FP64, "mixed": PREC_MIXED}[precision]
        if orth is not None:
            p.orth = {"fp64": ORTH_FP64, "df": ORTH_DF}[orth]
        p.cycle = {"v": 0, "f": 1}[cycle]
        if reorth is not None:
            p.reorth = {"always": REORTH_ALWAYS, "selective": REORTH_SELECTIVE}[reorth]
        self.params = p
        ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            st = lib().helm_create(n1, n2, n3, self.h, _ptr(k2t), bc, C.byref(p), _stream(), C.byref(ctx))
        if st != OK:
            raise HelmError(st, lib().helm_last_error(None).decode())
        self._ctx = ctx
        if krylov == "idrs":
            # IDR(s) draws its shadow space at random (Sec. 3.1); by default the seeded draw of
            # the synthetic-input module, so runs are repeatable
            if shadow is None:
                from . import inputs

                shadow = inputs.shadow_space(self.shape, idr_s)
            self.set_shadow_space(shadow)

    # -- housekeeping -----------------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None):
            lib().helm_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise HelmError(st, lib().helm_last_error(self._ctx).decode())

    @property
    def nlevels(self):
        n = C.c_int()
        self._check(lib().helm_levels(self._ctx, C.byref(n)))
        return n.value

    def level_dims(self, level):
        dims = (C.c_int * 6)()
        h = C.c_double()
        self._check(lib().helm_level_dims(self._ctx, level, dims, C.byref(h)))
        return {"n": (dims[0], dims[1], dims[2]), "shape": (dims[5], dims[4], dims[3]), "h": h.value}

    def _vec(self, t, shape=None, dtype=None):
        shape = self.shape if shape is None else shape
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise TypeError("expected a CUDA tensor")
        if dtype is not None and t.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {t.dtype}")
        if t.dtype not in _DT:
            raise TypeError("grid vectors are complex128 or complex64")
        if tuple(t.shape) != tuple(shape):
            t = t.reshape(shape)
        return t.contiguous()

    # -- operators ----------------------------------------------------------------------
    def apply(self, u, op="A", out=None):
        u = self._vec(u)
        v = torch.empty_like(u) if out is None else out
        self._check(lib().helm_apply(self._ctx, {"A": OP_A, "M": OP_M}[op], _DT[u.dtype], _ptr(u), _ptr(v), _stream()))
        return v

    def vcycle(self, r, out=None):
        r = self._vec(r)
        z = torch.empty_like(r) if out is None else out
        self._check(lib().cslp_vcycle(self._ctx, _DT[r.dtype], _ptr(r), _ptr(z), _stream()))
        return z

    def launch_shapes(self, level):
        """(rows per CTA, CTA target) per slot on `level`: slots 0-3 FP64 stencil / pre-smoothing /
        restriction / prolongation, 4-7 the same in FP32; (0, 0) = default."""
        ty, ct = (C.c_int * 8)(), (C.c_int * 8)()
        self._check(lib().helm_launch_shapes(self._ctx, level, ty, ct))
        return [(ty[q], ct[q]) for q in range(8)]

    def dot_variant(self, variant=None):
        """The Gram-Schmidt inner-product kernel variant in use; with `variant`, replace it."""
        v = C.c_int(-1 if variant is None else int(variant))
        self._check(lib().helm_dot_variant(self._ctx, 0 if variant is None else 1, C.byref(v)))
        return v.value

    def coarse_info(self):
        """(steps, converged) of the last coarsest-grid GMRES (contexts with coarse_tol > 0)."""
        steps, conv = C.c_int(), C.c_int()
        self._check(lib().helm_coarse_info(self._ctx, C.byref(steps), C.byref(conv)))
        return steps.value, bool(conv.value)

    def kernel_variants(self, level):
        """{'tiled', 'fused_down', 'down_full', 'up_full', 'rr'} in use on `level`: the
        shared-memory tiled FP32 stencils, pre-smoothing + residual as one kernel, the whole
        down-sweep as one, the whole up-sweep as one, residual + restriction as one."""
        f = C.c_int()
        self._check(lib().helm_kernel_variants(self._ctx, level, C.byref(f)))
        return {"tiled": bool(f.value & 1), "fused_down": bool(f.value & 2), "down_full": bool(f.value & 4),
                "up_full": bool(f.value & 8), "rr": bool(f.value & 16)}

    def tune_log(self):
        """Every launch shape the autotuner timed: (level, slot, ty, ctas, ms per launch)."""
        cnt = C.c_int()
        self._check(lib().helm_tune_log(self._ctx, None, None, 0, C.byref(cnt)))
        n = cnt.value
        rec, ms = (C.c_int * (4 * max(n, 1)))(), (C.c_float * max(n, 1))()
        self._check(lib().helm_tune_log(self._ctx, rec, ms, n, C.byref(cnt)))
        return [(rec[4 * i], rec[4 * i + 1], rec[4 * i + 2], rec[4 * i + 3], ms[i]) for i in range(n)]

    def apply_c64_df(self, u):
        """A u for a complex64 u in double-float arithmetic (mixed precision + double-float
        orth contexts), returned as complex128."""
        u = self._vec(u)
        if u.dtype != torch.complex64:
            raise TypeError("apply_c64_df takes a complex64 vector")
        v = torch.empty(u.shape, dtype=torch.complex128, device=u.device)
        self._check(lib().helm_apply_c64_df(self._ctx, _ptr(u), _ptr(v), _stream()))
        return v

    def set_shadow_space(self, P):
        """The s shadow vectors of IDR(s), shaped (s,) + grid shape, complex."""
        P = torch.as_tensor(P, dtype=torch.complex128).to(self.device).contiguous()
        if P.dim() != 4 or tuple(P.shape[1:]) != self.shape:
            raise ValueError(f"shadow space must be shaped (s,) + {self.shape}")
        self._check(lib().helm_set_shadow_space(self._ctx, P.shape[0], _ptr(P), _stream()))

    def fcycle(self, r, out=None):
        r = self._vec(r)
        z = torch.empty_like(r) if out is None else out
        self._check(lib().cslp_fcycle(self._ctx, _DT[r.dtype], _ptr(r), _ptr(z), _stream()))
        return z

    def vcycle_stage(self, level, stage, b, e=None):
        L = self.nlevels
        dt = b.dtype
        if stage == 0:
            out = torch.empty(self.level_dims(level + 1)["shape"], dtype=dt, device=b.device)
        else:
            out = torch.empty(self.level_dims(level)["shape"], dtype=dt, device=b.device)
        b = self._vec(b, self.level_dims(level)["shape"])
        ep = None
        if stage == 1:
            e = self._vec(e, self.level_dims(level + 1)["shape"], dt)
            ep = _ptr(e)
        assert 0 <= level < L
        self._check(lib().helm_vcycle_stage(self._ctx, level, stage, _DT[dt], _ptr(b), ep, _ptr(out), _stream()))
        return out

    def rhs_point(self, nodes):
        nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.int32).reshape(-1, 3))
        b = torch.empty(self.shape, dtype=torch.complex128, device=self.device)
        self._check(lib().helm_rhs_point(self._ctx, len(nodes), nodes.ctypes.data_as(C.POINTER(C.c_int)), _ptr(b),
                                         _stream()))
        return b

    # -- instrumentation ----------------------------------------------------------------
    def profile(self, enable=True):
        """Turn per-kernel CUDA-event timing on/off (resets the totals and launch count)."""
        self._check(lib().helm_profile(self._ctx, int(enable)))

    def profile_read(self):
        stats = (KernelStat * 32)()
        cnt = C.c_int()
        launches = C.c_longlong()
        self._check(lib().helm_profile_read(self._ctx, stats, 32, C.byref(cnt), C.byref(launches)))
        fams = [{"name": s.name.decode(), "launches": s.launches, "ms": s.ms, "bytes": s.bytes, "flops": s.flops}
                for s in stats[: cnt.value]]
        return fams, launches.value

    def solve_batched(self, B, X=None):
        """Solve for nrhs right-hand sides together: B is complex128 CUDA, shaped
        (nrhs, N3, N2, N1); X the initial guesses (zeros if None).  Returns (X, infos)."""
        B = B.reshape((-1,) + self.shape).contiguous()
        if B.dtype != torch.complex128 or B.device.type != "cuda":
            raise TypeError("B must be a complex128 CUDA tensor")
        nrhs = B.shape[0]
        X = torch.zeros_like(B) if X is None else X.reshape(B.shape).contiguous()
        infos = (SolveInfo * nrhs)()
        st = lib().helm_solve_batched(self._ctx, nrhs, _ptr(B), _ptr(X), infos, _stream())
        if st not in (OK, ENOCONV):
            self._check(st)
        return X, [infos[r].as_dict() for r in range(nrhs)]

    def solve_adjoint(self, g):
        """lambda with A^H lambda = g (device complex128 tensors); returns (lambda, info)."""
        g = self._vec(g, dtype=torch.complex128)
        lam = torch.empty_like(g)
        info = SolveInfo()
        st = lib().helm_solve_adjoint(self._ctx, _ptr(g), _ptr(lam), C.byref(info), _stream())
        if st not in (OK, ENOCONV):
            self._check(st)
        return lam, info.as_dict()

    def solve_adjoint_batched(self, G):
        """Lambda with A^H Lambda_r = G_r for every r at once (complex128 CUDA, shaped
        (nrhs, N3, N2, N1)); returns (Lambda, infos)."""
        G = G.reshape((-1,) + self.shape).contiguous()
        if G.dtype != torch.complex128 or G.device.type != "cuda":
            raise TypeError("G must be a complex128 CUDA tensor")
        nrhs = G.shape[0]
        L = torch.empty_like(G)
        infos = (SolveInfo * nrhs)()
        st = lib().helm_solve_adjoint_batched(self._ctx, nrhs, _ptr(G), _ptr(L), infos, _stream())
        if st not in (OK, ENOCONV):
            self._check(st)
        return L, [infos[r].as_dict() for r in range(nrhs)]

    def grad_k2(self, u, lam, grad=None):
        """grad += -Re(conj(lambda) dA/dk^2 u) at every node (float64 tensor shaped like u)."""
        u = self._vec(u, dtype=torch.complex128)
        lam = self._vec(lam, dtype=torch.complex128)
        if grad is None:
            grad = torch.zeros(self.shape, dtype=torch.float64, device=u.device)
        self._check(lib().helm_grad_k2(self._ctx, _ptr(u), _ptr(lam), _ptr(grad), _stream()))
        return grad

    def adjoint_grad(self, sources, rec_idx, d_obs):
        """Loss 1/2 sum_s |u_s(rec) - d_obs[s]|^2 for point sources and its gradient w.r.t. k^2.
        rec_idx: distinct flat unknown indices; d_obs: complex128 CUDA tensor (nsrc, nrec)."""
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32).reshape(-1, 3))
        rec = np.ascontiguousarray(np.asarray(rec_idx, dtype=np.int32).ravel())
        d_obs = d_obs.contiguous()
        if d_obs.dtype != torch.complex128 or d_obs.numel() != len(src) * len(rec):
            raise TypeError("d_obs must be complex128 with nsrc * nrec values")
        grad = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        loss = C.c_double()
        info = SolveInfo()
        st = lib().helm_adjoint_grad(self._ctx, len(src), src.ctypes.data_as(C.POINTER(C.c_int)), len(rec),
                                     rec.ctypes.data_as(C.POINTER(C.c_int)), _ptr(d_obs), _ptr(grad), C.byref(loss),
                                     C.byref(info), _stream())
        if st not in (OK, ENOCONV):
            self._check(st)
        return loss.value, grad, info.as_dict()

    def solve(self, b, x=None, zero_guess=False):
        """Solve A x = b.  b (and x, the initial guess) are complex128 tensors on the GPU, or
        both on the host (pinned or pageable), in which case the library stages the copies.
        zero_guess: start from x = 0 (helm_solve_zero); x, when given, only receives the
        solution."""
        host = b.device.type == "cpu"
        b = b.reshape(self.shape).contiguous()
        if b.dtype != torch.complex128:
            raise TypeError("helm_solve takes complex128 vectors")
        if x is None:
            x = torch.empty_like(b) if zero_guess else torch.zeros_like(b)
        x = x.reshape(self.shape)
        if (x.device.type == "cpu") != host or not x.is_contiguous() or x.dtype != torch.complex128:
            raise TypeError("x must be a contiguous complex128 tensor on the same kind of device as b")
        info = SolveInfo()
        entry = lib().helm_solve_zero if zero_guess else lib().helm_solve
        st = entry(self._ctx, _ptr(b), _ptr(x), C.byref(info), _stream())
        if st not in (OK, ENOCONV):
            self._check(st)
        out = info.as_dict()
        if st == ENOCONV:
            out["message"] = lib().helm_last_error(self._ctx).decode()
        return x, out


class HelmholtzSolve(torch.autograd.Function):
    """x = A(k^2)^{-1} b as a differentiable torch op.

    b is one right-hand side shaped like the grid, or several sources shaped (nsrc,) + grid
    (solved together by helm_solve_batched).  forward builds a context for k^2 and solves;
    backward solves the adjoint systems A^H lambda = dL/d conj(x) with the same preconditioned
    solver (helm_solve_adjoint_batched for several sources) and returns
    dL/dk^2 = -sum_s Re(conj(lambda_s) dA/dk^2 x_s) and dL/d conj(b) = lambda.

    recompute: True drops the forward wavefields and solves for them again in backward
    (checkpointing); False keeps them; None (default) keeps them when they take at most a
    quarter of the device memory that is free after the forward solve (cudaMemGetInfo), so
    that the adjoint solves still have room, and recomputes otherwise."""

    @staticmethod
    def forward(ctx, k2, b, n, h, bc, opts=None, recompute=None):
        opts = dict(opts or {})
        s = Solver(n, h, k2.detach(), bc, **opts)
        batched = b.dim() == 4
        bb = b.detach().reshape(((-1,) if batched else ()) + s.shape).contiguous()
        if batched:
            x, infos = s.solve_batched(bb)
        else:
            x, info = s.solve(bb)
            infos = [info]
        if any(i["status"] != OK for i in infos):
            raise HelmError(max(i["status"] for i in infos), "forward solve did not converge")
        if recompute is None:
            free, _ = torch.cuda.mem_get_info(x.device)
            recompute = x.numel() * x.element_size() > free // 4
        ctx.solver = s
        ctx.batched = batched
        ctx.recompute = bool(recompute)
        ctx.save_for_backward(bb if ctx.recompute else x)
        return x

    @staticmethod
    def backward(ctx, gx):
        s = ctx.solver
        (saved,) = ctx.saved_tensors
        if ctx.recompute:
            x = s.solve_batched(saved)[0] if ctx.batched else s.solve(saved)[0]
        else:
            x = saved
        g = gx.reshape(x.shape).contiguous()
        if ctx.batched:
            lam, _ = s.solve_adjoint_batched(g)
            gk2 = torch.zeros(s.shape, dtype=torch.float64, device=x.device)
            for r in range(x.shape[0]):
                s.grad_k2(x[r], lam[r], gk2)
        else:
            lam, _ = s.solve_adjoint(g)
            gk2 = s.grad_k2(x, lam)
        return gk2, lam, None, None, None, None, None


def helmholtz_solve(k2, b, n, h, bc=SOMMERFELD, opts=None, recompute=None):
    """Differentiable x = A(k^2)^{-1} b (see HelmholtzSolve)."""
    return HelmholtzSolve.apply(k2, b, n, h, bc, opts, recompute)
