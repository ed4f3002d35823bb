"""Seeded synthetic inputs: grids, velocity / wavenumber fields, source and receiver nodes.

This module generates inputs only.  It holds none of the solver's arithmetic (no operator,
smoother, transfer or Krylov step), so both the CUDA library and the CPU oracle can be fed
from it.  The paper's own benchmark data (the SEG/EAGE salt model) is not available, so
these seeded models stand in for its shapes and value ranges: velocities 1500-4482 m/s and
the three-layer wedge structure of Sec. 2.2.

Array convention: 3D arrays are shaped (N3, N2, N1), x fastest.  Node coordinates are
(i1, i2, i3) with 0 <= i_d <= n_d on a grid of n_d intervals.  The unit cube is used for
every model, with x3 increasing with depth (the top plane is x3 = 0).
"""
from __future__ import annotations

import math

import numpy as np

DIRICHLET = 0
SOMMERFELD = 1

# Seed fixed for the smooth random velocity model (arXiv id digits).
SMOOTH_MODEL_SEED = 2308060085


def unknown_shape(n, bc):
    """Shape (N3, N2, N1) of the unknown set for (n1, n2, n3) intervals."""
    n1, n2, n3 = (n, n, n) if np.isscalar(n) else tuple(n)
    d = -1 if bc == DIRICHLET else 1
    return (n3 + d, n2 + d, n1 + d)




def _grid(n, bc):
    n1, n2, n3 = (n, n, n) if np.isscalar(n) else tuple(n)
    off = 1 if bc == DIRICHLET else 0
    N3, N2, N1 = unknown_shape((n1, n2, n3), bc)
    x1 = ((np.arange(N1) + off) / n1)[None, None, :]
    x2 = ((np.arange(N2) + off) / n2)[None, :, None]
    x3 = ((np.arange(N3) + off) / n3)[:, None, None]
    return x1, x2, x3


def wedge_velocity(n, bc=SOMMERFELD):
    """Three-layer wedge (Sec. 2.2) on the unit cube: 2000 m/s above x3 = 0.4 + 0.2 x1,
    1500 m/s down to x3 = 0.8 - 0.2 x2, 3000 m/s below."""
    x1, x2, x3 = _grid(n, bc)
    shape = unknown_shape(n, bc)
    c = np.full(shape, 3000.0)
    mid = x3 < (0.8 - 0.2 * x2)
    top = x3 < (0.4 + 0.2 * x1)
    c = np.where(mid, 1500.0, c)
    c = np.where(top, 2000.0, c)
    return c


def wedge_omega(n, kh=0.625, cmin=1500.0):
    """Angular frequency that puts max k*h at `kh` on the finest grid (k = omega / c)."""
    n1 = n if np.isscalar(n) else max(n)
    return kh * cmin * n1


def k2_from_velocity(c, omega):
    """Wavenumber field k^2 = (omega / c)^2 at every node (Sec. 2: k = 2 pi f / c)."""
    return (omega / np.asarray(c, dtype=np.float64)) ** 2


def smooth_random_velocity(n, bc=SOMMERFELD, seed=SMOOTH_MODEL_SEED, sigma=8.0, amp=0.2, c0=2000.0):
    """c = c0 (1 + amp * m), m = uniform(-1, 1) noise, Gaussian-filtered (sigma in nodes,
    reflect boundary, truncated at 4 sigma), rescaled to max |m| = 1."""
    from scipy.ndimage import gaussian_filter

    shape = unknown_shape(n, bc)
    rng = np.random.default_rng(seed)
    m = rng.uniform(-1.0, 1.0, size=shape)
    m = gaussian_filter(m, sigma=sigma, mode="reflect", truncate=4.0)
    m /= np.abs(m).max()
    return c0 * (1.0 + amp * m)


def gaussian_bump(n, bc=SOMMERFELD, centre=(0.5, 0.5, 0.5), width=0.1, amp=0.05):
    """Multiplicative perturbation 1 + amp * exp(-|x - centre|^2 / (2 width^2))."""
    x1, x2, x3 = _grid(n, bc)
    r2 = (x1 - centre[0]) ** 2 + (x2 - centre[1]) ** 2 + (x3 - centre[2]) ** 2
    return 1.0 + amp * np.exp(-r2 / (2.0 * width * width))


def round_half_up(x):
    return int(math.floor(x + 0.5))


def top_centre_source(n):
    n1, n2, n3 = (n, n, n) if np.isscalar(n) else tuple(n)
    return [(n1 // 2, n2 // 2, 0)]


def source_grid(n, nx, ny, depth):
    """nx * ny sources at x1 = (i + 1/2)/nx, x2 = (j + 1/2)/ny, x3 = depth, rounded half-up
    to the nearest node; ordered x1 fastest."""
    n1, n2, n3 = (n, n, n) if np.isscalar(n) else tuple(n)
    out = []
    for j in range(ny):
        for i in range(nx):
            out.append((round_half_up((i + 0.5) / nx * n1), round_half_up((j + 0.5) / ny * n2),
                        round_half_up(depth * n3)))
    return out


def receiver_plane(n, depth):
    """Node index of the receiver plane x3 = depth."""
    n3 = n if np.isscalar(n) else n[2]
    return round_half_up(depth * n3)


def random_vector(shape, seed, dtype=np.complex128):
    """Seeded complex vector with independent U(-1, 1) real and imaginary parts."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(-1.0, 1.0, size=shape)
    im = rng.uniform(-1.0, 1.0, size=shape)
    return (re + 1j * im).astype(dtype)


def closed_off_rhs(n, k):
    """Right-hand side of the closed-off problem (Sec. 2.1) on the (n-1)^3 interior unknowns,
    x1 fastest: the source f = (21 pi^2 - k^2) sin(pi x1) sin(2 pi x2) sin(4 pi x3) - k^2 of the
    exact solution u = sin(pi x1) sin(2 pi x2) sin(4 pi x3) + 1, plus the Dirichlet data u = 1
    moved to the right (1 / h^2 for every neighbour on the boundary)."""
    h = 1.0 / n
    x = np.arange(1, n) * h
    f = ((21.0 * np.pi ** 2 - k * k) * np.sin(4 * np.pi * x)[:, None, None] * np.sin(2 * np.pi * x)[None, :, None]
         * np.sin(np.pi * x)[None, None, :] - k * k)
    edge = np.zeros(n - 1)
    edge[0] += 1
    edge[-1] += 1
    nb = edge[:, None, None] + edge[None, :, None] + edge[None, None, :]
    return (f + nb / (h * h)).astype(np.complex128)


IDR_SEED = 2308060085 + 4


def shadow_space(shape, s, seed=IDR_SEED):
    """The s random shadow vectors of IDR(s), shaped (s,) + shape: independent complex
    Gaussians of variance 1 / (2 N) per part, so each column has an expected norm of 1 and,
    at the sizes solved here, nearly orthogonal columns (IDR depends only on their span)."""
    rng = np.random.default_rng(seed)
    N = int(np.prod(shape))
    sd = 1.0 / np.sqrt(2.0 * N)
    re = rng.normal(0.0, sd, size=(s,) + tuple(shape))
    im = rng.normal(0.0, sd, size=(s,) + tuple(shape))
    return re + 1j * im


def random_k2(shape, seed, kmin=5.0, kmax=40.0):
    """Seeded positive k^2 field with k uniform in [kmin, kmax] (a rough heterogeneous model)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(kmin, kmax, size=shape) ** 2


# ---------------------------------------------------------------------------------------
# The workloads.  `n` may be overridden to scale a workload down for parity tests
# while keeping its structure (model, boundary, source placement, max k*h).
# ---------------------------------------------------------------------------------------
def workload(name, n=None):
    if name == "small":  # constant k = 20 at n = 32 (kh = 0.625), Dirichlet, centre source
        n = 32 if n is None else n
        k = 20.0 * n / 32.0
        shape = unknown_shape(n, DIRICHLET)
        return dict(name=name, n=(n, n, n), h=1.0 / n, bc=DIRICHLET, k2=np.full(shape, k * k),
                    sources=[(n // 2, n // 2, n // 2)], precision="fp64", restart=30)
    if name in ("wedge", "mixed", "batched"):
        n = {"wedge": 128, "mixed": 256, "batched": 128}[name] if n is None else n
        # one frequency for the wedge family: max k h = 0.625 at n = 128 (kh 0.3125 at n = 256)
        omega = wedge_omega(128) * (n / 128.0) if name != "mixed" else wedge_omega(128) * (n / 256.0)
        c = wedge_velocity(n)
        src = top_centre_source(n) if name != "batched" else source_grid(n, 4, 8, 0.1)
        return dict(name=name, n=(n, n, n), h=1.0 / n, bc=SOMMERFELD, k2=k2_from_velocity(c, omega),
                    omega=omega, sources=src, precision="fp64" if name == "wedge" else "mixed",
                    restart=30)
    if name == "adjoint":
        n = 192 if n is None else n
        c = smooth_random_velocity(n, sigma=8.0 * n / 192.0)
        omega = wedge_omega(n, kh=0.625, cmin=float(c.min()))
        return dict(name=name, n=(n, n, n), h=1.0 / n, bc=SOMMERFELD, k2=k2_from_velocity(c, omega),
                    omega=omega, velocity=c, sources=source_grid(n, 2, 4, 0.1),
                    receiver_plane=receiver_plane(n, 0.9), precision="mixed", restart=30)
    if name == "closed_off":  # Sec. 2.1 at k = 40 (Tables 1-3), Dirichlet u = 1, no point source
        n = 64 if n is None else n
        k = 40.0
        return dict(name=name, n=(n, n, n), h=1.0 / n, bc=DIRICHLET, k2=np.full(unknown_shape(n, DIRICHLET), k * k),
                    rhs=closed_off_rhs(n, k), coarsest_n=coarsest_by_node_rule(n), precision="fp64")
    raise ValueError(name)


def coarsest_by_node_rule(n, nodes=17):
    """Coarsest-grid interval count (the solver's `coarsest_n`) under the stopping rule of
    Sec. 4.2: coarsen by two until some direction has at most `nodes` grid points.  n is the
    interval count, or a tuple of them for a box, where the shortest direction decides:
    65 -> 17, 129 -> 17, 193 -> 13, 257 -> 17 nodes, and 641 x 641 x 193 -> 41 x 41 x 13 as the
    paper states for the salt grid (Sec. 5.1.2)."""
    m = min(n) if isinstance(n, (tuple, list)) else n
    while m + 1 > nodes and m % 2 == 0:
        m //= 2
    return m
