"""Dense numpy constructions used to pin the oracle (tests only).

Every matrix here is built from one-dimensional pieces by Kronecker products, a route
independent of the oracle's node-by-node loops:
  * the 1D second-difference matrix on the unknown set, with either the Dirichlet row
    truncation or the Sommerfeld ghost elimination u_ghost = u_opposite + 2 h i k u_p
    (Sec. 2.4, Eq. elimination) which doubles the off-diagonal of the first/last row;
  * the 1D full-weighting row (1, 2, 1)/4 and linear interpolation column (1, 2, 1)/2,
    whose tensor products are the paper's 27-point stencils (Sec. 3.4.2-3.4.3).
The x index runs fastest, so a 3D operator is kron(T3, I, I) + kron(I, T2, I) + kron(I, I, T1).
"""
import numpy as np

DIRICHLET = 0
SOMMERFELD = 1


def n_unknowns(n, bc):
    return n - 1 if bc == DIRICHLET else n + 1


def second_diff_1d(n, h, bc):
    N = n_unknowns(n, bc)
    T = np.zeros((N, N))
    for i in range(N):
        T[i, i] = 2.0
        if i > 0:
            T[i, i - 1] = -1.0
        if i < N - 1:
            T[i, i + 1] = -1.0
    if bc == SOMMERFELD:
        T[0, 1] = -2.0
        T[N - 1, N - 2] = -2.0
    return T / (h * h)


def face_count(n3, bc):
    """Number of Sommerfeld faces each unknown node lies on, shaped (N3, N2, N1)."""
    n1, n2, n3_ = n3
    if bc != SOMMERFELD:
        return np.zeros((n3_ - 1, n2 - 1, n1 - 1))
    f = []
    for n in (n1, n2, n3_):
        v = np.zeros(n + 1)
        v[0] = 1
        v[-1] = 1
        f.append(v)
    return f[2][:, None, None] + f[1][None, :, None] + f[0][None, None, :]


def laplacian_3d(n, h, bc):
    n1, n2, n3 = n
    T1, T2, T3 = (second_diff_1d(m, h, bc) for m in (n1, n2, n3))
    I1, I2, I3 = (np.eye(T.shape[0]) for T in (T1, T2, T3))
    return np.kron(np.kron(I3, I2), T1) + np.kron(np.kron(I3, T2), I1) + np.kron(np.kron(T3, I2), I1)


def helmholtz_3d(n, h, bc, k2, shift=1.0):
    """Dense (-Lap_h - shift k^2) with Sommerfeld face terms -2 i k_p / h per face."""
    L = laplacian_3d(n, h, bc).astype(np.complex128)
    k2f = np.asarray(k2, dtype=np.float64).ravel()
    d = -shift * k2f
    if bc == SOMMERFELD:
        d = d - 2j * np.sqrt(k2f) / h * face_count(n, bc).ravel()
    return L + np.diag(d)


def restriction_1d(nf, bc):
    Nf = n_unknowns(nf, bc)
    Nc = n_unknowns(nf // 2, bc)
    R = np.zeros((Nc, Nf))
    off = 1 if bc == DIRICHLET else 0
    for I in range(Nc):
        f = 2 * (I + off) - off
        R[I, f] = 0.5
        if f - 1 >= 0:
            R[I, f - 1] = 0.25
        if f + 1 < Nf:
            R[I, f + 1] = 0.25
    return R


def prolongation_1d(nf, bc):
    Nf = n_unknowns(nf, bc)
    Nc = n_unknowns(nf // 2, bc)
    P = np.zeros((Nf, Nc))
    off = 1 if bc == DIRICHLET else 0
    for I in range(Nc):
        f = 2 * (I + off) - off
        P[f, I] = 1.0
        if f - 1 >= 0:
            P[f - 1, I] = 0.5
        if f + 1 < Nf:
            P[f + 1, I] = 0.5
    return P


def restriction_3d(nf, bc):
    R1, R2, R3 = (restriction_1d(m, bc) for m in nf)
    return np.kron(np.kron(R3, R2), R1)


def prolongation_3d(nf, bc):
    P1, P2, P3 = (prolongation_1d(m, bc) for m in nf)
    return np.kron(np.kron(P3, P2), P1)


def inject_k2(k2, bc):
    k2 = np.asarray(k2)
    return k2[::2, ::2, ::2].copy() if bc == SOMMERFELD else k2[1::2, 1::2, 1::2].copy()


def levels(n, coarsest_n):
    out = [tuple(n)]
    while all(m % 2 == 0 for m in out[-1]) and all(m // 2 >= coarsest_n for m in out[-1]):
        out.append(tuple(m // 2 for m in out[-1]))
    return out


def dense_vcycle(n, h, bc, k2, b, shift, omega, coarsest_n):
    """One V-cycle z ~= M^{-1} b by dense algebra, zero initial guess, one damped-Jacobi
    sweep before and after each coarse correction, exact solve on the last level."""
    levs = levels(n, coarsest_n)
    k2s = [np.asarray(k2, dtype=np.float64)]
    for _ in levs[1:]:
        k2s.append(inject_k2(k2s[-1], bc))
    hs = [h * 2 ** l for l in range(len(levs))]
    Ms = [helmholtz_3d(levs[l], hs[l], bc, k2s[l], shift) for l in range(len(levs))]

    def cycle(l, bl):
        M = Ms[l]
        if l == len(levs) - 1:
            return np.linalg.solve(M, bl)
        D = np.diag(M)
        x1 = omega * bl / D
        r = bl - M @ x1
        bc_ = restriction_3d(levs[l], bc) @ r
        e = cycle(l + 1, bc_)
        x2 = x1 + prolongation_3d(levs[l], bc) @ e
        return x2 + omega * (bl - M @ x2) / D

    return cycle(0, np.asarray(b, dtype=np.complex128).ravel())


def dense_fcycle(n, h, bc, k2, b, shift, omega, coarsest_n):
    """One F-cycle by dense algebra: the coarse-grid error of each level is an F-cycle on the
    next level followed by one V-cycle there started from it (zero start on the way down)."""
    levs = levels(n, coarsest_n)
    k2s = [np.asarray(k2, dtype=np.float64)]
    for _ in levs[1:]:
        k2s.append(inject_k2(k2s[-1], bc))
    hs = [h * 2 ** l for l in range(len(levs))]
    Ms = [helmholtz_3d(levs[l], hs[l], bc, k2s[l], shift) for l in range(len(levs))]
    Rs = [restriction_3d(levs[l], bc) for l in range(len(levs) - 1)]
    Ps = [prolongation_3d(levs[l], bc) for l in range(len(levs) - 1)]
    last = len(levs) - 1

    def smooth(l, x, bl):
        return x + omega * (bl - Ms[l] @ x) / np.diag(Ms[l])

    def vcyc(l, x, bl):
        if l == last:
            return np.linalg.solve(Ms[l], bl)
        x = smooth(l, x, bl)
        e = vcyc(l + 1, np.zeros(Ms[l + 1].shape[0], complex), Rs[l] @ (bl - Ms[l] @ x))
        return smooth(l, x + Ps[l] @ e, bl)

    def fcyc(l, bl):
        if l == last:
            return np.linalg.solve(Ms[l], bl)
        x = smooth(l, np.zeros(Ms[l].shape[0], complex), bl)
        bc_ = Rs[l] @ (bl - Ms[l] @ x)
        e = fcyc(l + 1, bc_)
        e = vcyc(l + 1, e, bc_)
        return smooth(l, x + Ps[l] @ e, bl)

    return fcyc(0, np.asarray(b, dtype=np.complex128).ravel())
