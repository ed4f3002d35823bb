// stencil.cu -- matrix-free grid kernels of libhelm: the 7-point Helmholtz / CSLP operator
// (Sec. 2.4, Sec. 3.5 Algorithm 2), damped Jacobi (Sec. 3.4.1), full-weighting restriction
// (Sec. 3.4.2), trilinear interpolation (Sec. 3.4.3), k^2 injection for the DCG coarse
// operators (Sec. 3.4.4) and the exact coarsest-grid solve.
//
// Every grid kernel maps a 32 x 8 tile of (x, y) columns to a 256-thread block and streams
// along z: the z-1 / z / z+1 values of a thread's own column stay in registers (2.5D
// streaming), the in-plane neighbours come through the read-only L1 path.
#include "internal.cuh"

#include <type_traits>

namespace helm {

namespace {

constexpr int TX = 32, TY = 8;

template <typename T>
__device__ __forceinline__ cx<T> zero_c() {
  return mkc<T>((T)0, (T)0);
}

// One stencil kernel for three uses (MODE):
//   APPLY  : out = Op u
//   RESID  : out = b - Op u
//   JACOBI : out = u + (omega / d) (b - Op u)
// with Op = -Lap_h - s k^2 (s in OpCoef).  DINV: read omega/d from a precomputed array
// (FP64 path, where a complex division costs more than the 16-byte read) instead of
// computing it.  With g.nb right-hand sides per node, a thread owns one (node column, rhs)
// pair; for nb = 32 a warp covers the 32 right-hand sides of one node with one 256-byte
// (complex64) row and reads k^2 once.
template <typename R, int MODE, bool DINV, typename TU, typename TB, typename TO, bool SPLIT = false>
__global__ void __launch_bounds__(TX* TY)
    k_stencil(Grid g, OpCoef<R> c, const R* __restrict__ k2, const cx<R>* __restrict__ dinv,
              const cx<TU>* __restrict__ u, const cx<TB>* __restrict__ b, cx<TO>* __restrict__ out,
              int zchunk, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int nb = g.nb;
  const int f = blockIdx.x * TX + threadIdx.x;
  const int i = f / nb, r = f - (f / nb) * nb;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.N1 || j >= g.N2) return;
  const int k0 = blockIdx.z * zchunk;
  if (k0 >= g.N3) return;
  const int k1 = min(k0 + zchunk, g.N3);
  const bool som = g.bc == 1;
  const size_t S = (size_t)g.N1 * g.N2;  // nodes per plane
  const size_t Se = S * nb;              // elements per plane
  const long Xe = nb, Ye = (long)g.N1 * nb;
  const bool hxm = i > 0, hxp = i < g.N1 - 1, hym = j > 0, hyp = j < g.N2 - 1;
  const int nfxy = som ? (!hxm) + (!hxp) + (!hym) + (!hyp) : 0;
  auto ld = [&](size_t q) { return cvt<R>(ldg(u + q)); };
  size_t p = gidx(i, j, k0, g.N1, g.N2);  // node index
  size_t e = p * nb + r;                  // element index
  cx<R> uc = ld(e);
  cx<R> um = (k0 > 0) ? ld(e - Se) : zero_c<R>();
  for (int k = k0; k < k1; ++k, p += S, e += Se) {
    const bool hzp = k + 1 < g.N3;
    cx<R> up = hzp ? ld(e + Se) : zero_c<R>();
    int nf = nfxy;
    cx<R> zm, zp;
    if (k > 0) zm = um;
    else if (som) { zm = up; ++nf; }
    else zm = zero_c<R>();
    if (hzp) zp = up;
    else if (som) { zp = um; ++nf; }
    else zp = zero_c<R>();
    cx<R> xm = hxm ? ld(e - Xe) : (som ? ld(e + Xe) : zero_c<R>());
    cx<R> xp = hxp ? ld(e + Xe) : (som ? ld(e - Xe) : zero_c<R>());
    cx<R> ym = hym ? ld(e - Ye) : (som ? ld(e + Ye) : zero_c<R>());
    cx<R> yp = hyp ? ld(e + Ye) : (som ? ld(e - Ye) : zero_c<R>());
    const R kk = __ldg(k2 + p);
    const cx<R> d = op_diag(c, kk, nf, nf ? face_k<R>(g, p, kk) : (R)0);
    const bool real_d = c.real_shift && nf == 0;
    if (MODE == 0) {
      const cx<R> v = op_apply(d, real_d, uc, c.ih2, xm, xp, ym, yp, zm, zp);
      if (SPLIT)  // the output buffer holds double-float values (16 bytes, like complex128)
        reinterpret_cast<zdf*>(out)[e] = df_from(cvt<double>(v));
      else
        out[e] = cvt<TO>(v);
    } else {
      const cx<R> res = op_resid(cvt<R>(ldg(b + e)), d, real_d, uc, c.ih2, xm, xp, ym, yp, zm, zp);
      if (MODE == 1) {
        out[e] = cvt<TO>(res);
      } else {
        const cx<R> w = DINV ? ldg(dinv + p) : omega_over(d, c.omega);
        out[e] = cvt<TO>(cfma(w, res, uc));
      }
    }
    um = uc;
    uc = up;
  }
}

// The FP32 7-point kernels (one right-hand side) with the x-y neighbours staged in shared
// memory: a CTA of 32 x TYT threads covers a 32 x TYT tile of each plane and streams its z-chunk;
// each plane's values go to a (TYT + 2) x 34 tile (halo loaded by the edge threads), so a point
// costs one coalesced load of u plus the halo share instead of five L1 requests.  The z
// neighbours stay in registers.  Same arithmetic per point as k_stencil (op_apply / op_resid /
// omega_over, same neighbour substitution at Sommerfeld faces), so the results are identical.
constexpr int TYT = 8;
template <int MODE, typename TU, typename TB, typename TO>
__global__ void __launch_bounds__(TX* TYT)
    k_stencil32_tiled(Grid g, OpCoef<float> c, const float* __restrict__ k2, const cx<TU>* __restrict__ u,
                      const cx<TB>* __restrict__ b, cx<TO>* __restrict__ out, int zchunk,
                      const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ z64 tile[TYT + 2][TX + 2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * TX + tx, j = blockIdx.y * TYT + ty;
  const int k0 = blockIdx.z * zchunk;
  if (k0 >= g.N3) return;  // the whole CTA
  const int k1 = min(k0 + zchunk, g.N3);
  const bool inside = i < g.N1 && j < g.N2;
  const bool som = g.bc == 1;
  const size_t S = (size_t)g.N1 * g.N2;
  const bool hxm = i > 0, hxp = i < g.N1 - 1, hym = j > 0, hyp = j < g.N2 - 1;
  const int nfxy = som ? (!hxm) + (!hxp) + (!hym) + (!hyp) : 0;
  const z64 z0 = mkc<float>(0.f, 0.f);
  auto ld = [&](size_t q) { return cvt<float>(ldg(u + q)); };
  // halo duties of this thread (loads that stay inside the grid)
  const bool ld_xm = inside && tx == 0 && i > 0;
  const bool ld_xp = inside && tx == TX - 1 && i + 1 < g.N1;
  const bool ld_ym = inside && ty == 0 && j > 0;
  const bool ld_yp = inside && ty == TYT - 1 && j + 1 < g.N2;
  size_t p = inside ? gidx(i, j, k0, g.N1, g.N2) : 0;
  z64 uc = inside ? ld(p) : z0;
  z64 um = (inside && k0 > 0) ? ld(p - S) : z0;
  z64 up = (inside && k0 + 1 < g.N3) ? ld(p + S) : z0;
  for (int k = k0; k < k1; ++k, p += S) {
    // stage plane k; load what this plane's update needs besides the neighbours
    z64 hx0 = z0, hx1 = z0, hy0 = z0, hy1 = z0;
    if (ld_xm) hx0 = ld(p - 1);
    if (ld_xp) hx1 = ld(p + 1);
    if (ld_ym) hy0 = ld(p - g.N1);
    if (ld_yp) hy1 = ld(p + g.N1);
    const float kk = inside ? __ldg(k2 + p) : 0.f;
    const z64 bv = (MODE != 0 && inside) ? cvt<float>(ldg(b + p)) : z0;
    const bool hzp = k + 1 < g.N3;
    const z64 un = (inside && k + 2 < g.N3 && k + 1 < k1) ? ld(p + 2 * S) : z0;  // next plane's up
    __syncthreads();  // the previous plane's readers are done with the tile
    tile[ty + 1][tx + 1] = uc;
    if (ld_xm) tile[ty + 1][0] = hx0;
    if (ld_xp) tile[ty + 1][TX + 1] = hx1;
    if (ld_ym) tile[0][tx + 1] = hy0;
    if (ld_yp) tile[TYT + 1][tx + 1] = hy1;
    __syncthreads();
    if (inside) {
      int nf = nfxy;
      z64 zm, zp;
      if (k > 0) zm = um;
      else if (som) { zm = up; ++nf; }
      else zm = z0;
      if (hzp) zp = up;
      else if (som) { zp = um; ++nf; }
      else zp = z0;
      const z64 xm = hxm ? tile[ty + 1][tx] : (som ? tile[ty + 1][tx + 2] : z0);
      const z64 xp = hxp ? tile[ty + 1][tx + 2] : (som ? tile[ty + 1][tx] : z0);
      const z64 ym = hym ? tile[ty][tx + 1] : (som ? tile[ty + 2][tx + 1] : z0);
      const z64 yp = hyp ? tile[ty + 2][tx + 1] : (som ? tile[ty][tx + 1] : z0);
      const z64 d = op_diag(c, kk, nf, nf ? face_k<float>(g, p, kk) : 0.f);
      const bool real_d = c.real_shift && nf == 0;
      if (MODE == 0) {
        out[p] = cvt<TO>(op_apply(d, real_d, uc, c.ih2, xm, xp, ym, yp, zm, zp));
      } else {
        const z64 res = op_resid(bv, d, real_d, uc, c.ih2, xm, xp, ym, yp, zm, zp);
        if (MODE == 1) out[p] = cvt<TO>(res);
        else out[p] = cvt<TO>(cfma(omega_over(d, c.omega), res, uc));
      }
    }
    um = uc;
    uc = up;
    up = un;
  }
}

// FP32 pre-smoothing from zero fused with the residual (one right-hand side): u1 = (omega/d) b
// is written for the interpolation step, and r = b - M u1 is formed from u1 values recomputed at
// the six neighbours (b and k^2 there), so neither u1 nor b is read back from memory.  Each u1
// value is the same product as in k_smooth0, so the results equal those of the two separate
// kernels.
template <typename TB>
__global__ void __launch_bounds__(TX* TY)
    k_smooth0_resid32(Grid g, OpCoef<float> c, const float* __restrict__ k2, const cx<TB>* __restrict__ b,
                      z64* __restrict__ u1, z64* __restrict__ r, int zchunk, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int i = blockIdx.x * TX + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.N1 || j >= g.N2) return;
  const int k0 = blockIdx.z * zchunk;
  if (k0 >= g.N3) return;
  const int k1 = min(k0 + zchunk, g.N3);
  const bool som = g.bc == 1;
  const size_t S = (size_t)g.N1 * g.N2;
  const z64 z0 = mkc<float>(0.f, 0.f);
  // u1 at node (ii, jj, kk) of the grid (the caller keeps it inside)
  auto u1_at = [&](int ii, int jj, int kk, size_t q) {
    const int nf = som ? (ii == 0) + (ii == g.N1 - 1) + (jj == 0) + (jj == g.N2 - 1) + (kk == 0) + (kk == g.N3 - 1) : 0;
    const float kq = __ldg(k2 + q);
    const z64 w = omega_over(op_diag(c, kq, nf, nf ? face_k<float>(g, q, kq) : 0.f), c.omega);
    return cmul(w, cvt<float>(ldg(b + q)));
  };
  const bool hxm = i > 0, hxp = i < g.N1 - 1, hym = j > 0, hyp = j < g.N2 - 1;
  const int nfxy = som ? (!hxm) + (!hxp) + (!hym) + (!hyp) : 0;
  size_t p = gidx(i, j, k0, g.N1, g.N2);
  z64 uc = u1_at(i, j, k0, p);
  z64 um = k0 > 0 ? u1_at(i, j, k0 - 1, p - S) : z0;
  for (int k = k0; k < k1; ++k, p += S) {
    const bool hzp = k + 1 < g.N3;
    const z64 up = hzp ? u1_at(i, j, k + 1, p + S) : z0;
    int nf = nfxy;
    z64 zm, zp;
    if (k > 0) zm = um;
    else if (som) { zm = up; ++nf; }
    else zm = z0;
    if (hzp) zp = up;
    else if (som) { zp = um; ++nf; }
    else zp = z0;
    const z64 xm = hxm ? u1_at(i - 1, j, k, p - 1) : (som ? u1_at(i + 1, j, k, p + 1) : z0);
    const z64 xp = hxp ? u1_at(i + 1, j, k, p + 1) : (som ? u1_at(i - 1, j, k, p - 1) : z0);
    const z64 ym = hym ? u1_at(i, j - 1, k, p - g.N1) : (som ? u1_at(i, j + 1, k, p + g.N1) : z0);
    const z64 yp = hyp ? u1_at(i, j + 1, k, p + g.N1) : (som ? u1_at(i, j - 1, k, p - g.N1) : z0);
    const float kk = __ldg(k2 + p);
    const z64 d = op_diag(c, kk, nf, nf ? face_k<float>(g, p, kk) : 0.f);
    const bool real_d = c.real_shift && nf == 0;
    u1[p] = uc;
    r[p] = op_resid(cvt<float>(ldg(b + p)), d, real_d, uc, c.ih2, xm, xp, ym, yp, zm, zp);
    um = uc;
    uc = up;
  }
}

// Pre-smoothing from a zero initial guess: one damped-Jacobi sweep gives u1 = (omega/d) b.
template <typename R, bool DINV, typename TB>
__global__ void __launch_bounds__(TX* TY)
    k_smooth0(Grid g, OpCoef<R> c, const R* __restrict__ k2, const cx<R>* __restrict__ dinv,
              const cx<TB>* __restrict__ b, cx<R>* __restrict__ out, int zchunk,
              const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int nb = g.nb;
  const int f = blockIdx.x * TX + threadIdx.x;
  const int i = f / nb, r = f - (f / nb) * nb;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.N1 || j >= g.N2) return;
  const int k0 = blockIdx.z * zchunk;
  const int k1 = min(k0 + zchunk, g.N3);
  const bool som = g.bc == 1;
  const int nfxy = som ? (i == 0) + (i == g.N1 - 1) + (j == 0) + (j == g.N2 - 1) : 0;
  const size_t S = (size_t)g.N1 * g.N2;
  size_t p = gidx(i, j, k0, g.N1, g.N2);
  size_t e = p * nb + r;
  for (int k = k0; k < k1; ++k, p += S, e += S * nb) {
    cx<R> w;
    if (DINV) {
      w = ldg(dinv + p);
    } else {
      const int nf = nfxy + (som ? (k == 0) + (k == g.N3 - 1) : 0);
      const R kk = __ldg(k2 + p);
      w = omega_over(op_diag(c, kk, nf, nf ? face_k<R>(g, p, kk) : (R)0), c.omega);
    }
    out[e] = cmul(w, cvt<R>(ldg(b + e)));
  }
}

// omega / diag(M) at every node (FP64 path; computed once per level at set-up).
__global__ void k_dinv(Grid g, OpCoef<double> c, const double* __restrict__ k2, z128* __restrict__ out) {
  const size_t n = g.npts();
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % g.N1);
    const int j = (int)((p / g.N1) % g.N2);
    const int k = (int)(p / ((size_t)g.N1 * g.N2));
    const int nf = g.bc == 1 ? (i == 0) + (i == g.N1 - 1) + (j == 0) + (j == g.N2 - 1) + (k == 0) + (k == g.N3 - 1) : 0;
    const z128 d = op_diag(c, k2[p], nf, sqrt(k2[p]));
    // omega / d as omega conj(d) / |d|^2 in FP64 (set-up only)
    const double m2 = d.re * d.re + d.im * d.im;
    out[p] = mkc<double>(c.omega * d.re / m2, -c.omega * d.im / m2);
  }
}

// Full weighting (Sec. 3.4.2): b_H(I) = (1/64) sum over the 27 fine neighbours of the fine
// node 2I of weight 8 / 4 / 2 / 1 (centre / face / edge / corner) times r_h; fine values
// outside the unknown set count as 0.
template <typename R>
__global__ void __launch_bounds__(TX* TY)
    k_restrict(Grid gf, Grid gc, const cx<R>* __restrict__ r, cx<R>* __restrict__ out, int zchunk,
               const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int nb = gc.nb;
  const int f = blockIdx.x * TX + threadIdx.x;
  const int I = f / nb, q = f - (f / nb) * nb;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= gc.N1 || J >= gc.N2) return;
  const int K0 = blockIdx.z * zchunk;
  const int K1 = min(K0 + zchunk, gc.N3);
  const int off = gf.bc == 0 ? 1 : 0;
  const int fi = 2 * (I + off) - off, fj = 2 * (J + off) - off;
  for (int K = K0; K < K1; ++K) {
    const int fk = 2 * (K + off) - off;
    R are = 0, aim = 0;
    for (int dz = -1; dz <= 1; ++dz) {
      const int z = fk + dz;
      if (z < 0 || z >= gf.N3) continue;
      const R wz = dz ? (R)1 : (R)2;
      for (int dy = -1; dy <= 1; ++dy) {
        const int y = fj + dy;
        if (y < 0 || y >= gf.N2) continue;
        const R wyz = wz * (dy ? (R)1 : (R)2);
        for (int dx = -1; dx <= 1; ++dx) {
          const int x = fi + dx;
          if (x < 0 || x >= gf.N1) continue;
          const R w = wyz * (dx ? (R)1 : (R)2);
          const cx<R> v = ldg(r + gidx(x, y, z, gf.N1, gf.N2) * nb + q);
          are = fma(w, v.re, are);
          aim = fma(w, v.im, aim);
        }
      }
    }
    out[gidx(I, J, K, gc.N1, gc.N2) * nb + q] = mkc<R>(are * (R)(1.0 / 64.0), aim * (R)(1.0 / 64.0));
  }
}

// Trilinear interpolation (Sec. 3.4.3) added to u1: out = u1 + I_H^h e.  A fine node at
// an odd node index along an axis averages the two coarse nodes either side; coarse
// values outside the unknown set (Dirichlet boundary) are 0.
template <typename R>
__global__ void __launch_bounds__(TX* TY)
    k_prolong_add(Grid gf, Grid gc, const cx<R>* __restrict__ u1, const cx<R>* __restrict__ e,
                  cx<R>* __restrict__ out, int zchunk, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int nb = gf.nb;
  const int f = blockIdx.x * TX + threadIdx.x;
  const int i = f / nb, q = f - (f / nb) * nb;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= gf.N1 || j >= gf.N2) return;
  const int k0 = blockIdx.z * zchunk;
  const int k1 = min(k0 + zchunk, gf.N3);
  const int off = gf.bc == 0 ? 1 : 0;
  int cx_[2], cy_[2];
  const int fi = i + off, fj = j + off;
  cx_[0] = (fi >> 1) - off; cx_[1] = ((fi + 1) >> 1) - off;
  cy_[0] = (fj >> 1) - off; cy_[1] = ((fj + 1) >> 1) - off;
  const int nx = (cx_[0] == cx_[1]) ? 1 : 2, ny = (cy_[0] == cy_[1]) ? 1 : 2;
  for (int k = k0; k < k1; ++k) {
    const int fk = k + off;
    int cz_[2] = {(fk >> 1) - off, ((fk + 1) >> 1) - off};
    const int nz = (cz_[0] == cz_[1]) ? 1 : 2;
    R are = 0, aim = 0;
    for (int c = 0; c < nz; ++c) {
      if (cz_[c] < 0 || cz_[c] >= gc.N3) continue;
      for (int bq = 0; bq < ny; ++bq) {
        if (cy_[bq] < 0 || cy_[bq] >= gc.N2) continue;
        for (int a = 0; a < nx; ++a) {
          if (cx_[a] < 0 || cx_[a] >= gc.N1) continue;
          const cx<R> v = ldg(e + gidx(cx_[a], cy_[bq], cz_[c], gc.N1, gc.N2) * nb + q);
          are += v.re;
          aim += v.im;
        }
      }
    }
    const R s = (R)1 / (R)(nx * ny * nz);
    const size_t p = gidx(i, j, k, gf.N1, gf.N2) * nb + q;
    const cx<R> base = ldg(u1 + p);
    out[p] = mkc<R>(fma(are, s, base.re), fma(aim, s, base.im));
  }
}

// k^2 on a coarse grid by injection (coarse node c = fine node 2c, Sec. 3.4.4 DCG).
__global__ void k_inject(Grid gf, Grid gc, const double* __restrict__ kf, double* __restrict__ kc) {
  const size_t n = gc.npts();
  const int off = gf.bc == 0 ? 1 : 0;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const int I = (int)(p % gc.N1);
    const int J = (int)((p / gc.N1) % gc.N2);
    const int K = (int)(p / ((size_t)gc.N1 * gc.N2));
    kc[p] = kf[gidx(2 * (I + off) - off, 2 * (J + off) - off, 2 * (K + off) - off, gf.N1, gf.N2)];
  }
}

__global__ void k_sqrt_table(const double* __restrict__ k2, double* __restrict__ sk, float* __restrict__ skf, size_t n) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const double v = sqrt(k2[p]);
    sk[p] = v;
    skf[p] = sqrtf((float)k2[p]);
  }
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    b[p] = (float)a[p];
}

// k^2 sanity check at set-up: counts non-finite or non-positive entries.
__global__ void k_check_k2(const double* __restrict__ a, size_t n, int* __restrict__ bad) {
  int local = 0;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    local += !(isfinite(a[p]) && a[p] > 0.0);
  if (local) atomicAdd(bad, local);
}

// Exact coarsest-grid solve as a dense FP64 product with the precomputed inverse:
// one warp per row, lanes over columns in a fixed order.
template <typename TI, typename TO>
__global__ void k_coarse(int nc, const z128* __restrict__ Minv, const cx<TI>* __restrict__ b,
                         cx<TO>* __restrict__ e, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= nc) return;
  double re = 0, im = 0;
  const z128* a = Minv + (size_t)row * nc;
  for (int c = lane; c < nc; c += 32) {
    const z128 m = a[c];
    const z128 v = cvt<double>(ldg(b + c));
    re = fma(m.re, v.re, re);
    re = fma(-m.im, v.im, re);
    im = fma(m.re, v.im, im);
    im = fma(m.im, v.re, im);
  }
  for (int o = 16; o; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) e[row] = mkc<TO>((TO)re, (TO)im);
}

// The same product for nb right-hand sides (row-major Minv, vectors node-major with the
// right-hand side innermost): one thread per (row, rhs), columns in a fixed order.
template <typename TI, typename TO>
__global__ void k_coarse_b(int nc, int nb, const z128* __restrict__ Minv, const cx<TI>* __restrict__ b,
                           cx<TO>* __restrict__ e, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * nb) return;
  const int row = t / nb, q = t - (t / nb) * nb;
  const z128* a = Minv + (size_t)row * nc;
  double re = 0, im = 0;
  for (int c = 0; c < nc; ++c) {
    const z128 m = a[c];
    const z128 v = cvt<double>(ldg(b + (size_t)c * nb + q));
    re = fma(m.re, v.re, re);
    re = fma(-m.im, v.im, re);
    im = fma(m.re, v.im, im);
    im = fma(m.im, v.re, im);
  }
  e[t] = mkc<TO>((TO)re, (TO)im);
}

// v = A u for a complex64 u in double-float arithmetic (FP32 instructions only, about 48
// significant bits, 2^-46 relative to the largest term): the exact double-float sum of the six
// neighbours (TwoSum), times 1/h^2, subtracted from the diagonal term d u_c with
// d = 6/h^2 - k^2 - i (2 k / h) nf (the operator A, Sec. 2.4).  k^2 and k come from
// double-float tables (hi, lo per node).  The float inputs are exact, so this is A applied to
// the complex64 vector to FP64-class accuracy without FP64 instructions, whose issue rate on
// this GPU is 1/64 of FP32's.  OUT: zdf (double-float, 16 B) or z128.
template <typename OUT>
__global__ void __launch_bounds__(TX* TY)
    k_apply_c64_df(Grid g, float2 ih2, float2 six_ih2, float2 two_over_h, const float2* __restrict__ k2df,
                   const float2* __restrict__ skdf, const z64* __restrict__ u, OUT* __restrict__ out, int zchunk,
                   const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int nb = g.nb;
  const int f = blockIdx.x * TX + threadIdx.x;
  const int i = f / nb, r = f - (f / nb) * nb;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.N1 || j >= g.N2) return;
  const int k0 = blockIdx.z * zchunk;
  if (k0 >= g.N3) return;
  const int k1 = min(k0 + zchunk, g.N3);
  const bool som = g.bc == 1;
  const size_t S = (size_t)g.N1 * g.N2;
  const size_t Se = S * nb;
  const long Xe = nb, Ye = (long)g.N1 * nb;
  const bool hxm = i > 0, hxp = i < g.N1 - 1, hym = j > 0, hyp = j < g.N2 - 1;
  const int nfxy = som ? (!hxm) + (!hxp) + (!hym) + (!hyp) : 0;
  auto ld = [&](size_t q) { return ldg(u + q); };
  const z64 z0 = mkc<float>(0.f, 0.f);
  size_t p = gidx(i, j, k0, g.N1, g.N2);
  size_t e = p * nb + r;
  z64 uc = ld(e);
  z64 um = (k0 > 0) ? ld(e - Se) : z0;
  for (int k = k0; k < k1; ++k, p += S, e += Se) {
    const bool hzp = k + 1 < g.N3;
    const z64 up = hzp ? ld(e + Se) : z0;
    int nf = nfxy;
    z64 zm, zp;
    if (k > 0) zm = um;
    else if (som) { zm = up; ++nf; }
    else zm = z0;
    if (hzp) zp = up;
    else if (som) { zp = um; ++nf; }
    else zp = z0;
    const z64 xm = hxm ? ld(e - Xe) : (som ? ld(e + Xe) : z0);
    const z64 xp = hxp ? ld(e + Xe) : (som ? ld(e - Xe) : z0);
    const z64 ym = hym ? ld(e - Ye) : (som ? ld(e + Ye) : z0);
    const z64 yp = hyp ? ld(e + Ye) : (som ? ld(e - Ye) : z0);
    // exact neighbour sums as (hi, lo)
    float sr, cr, si, ci, t;
    two_sum(xm.re, xp.re, sr, cr);
    two_sum(xm.im, xp.im, si, ci);
    const float nre[4] = {ym.re, yp.re, zm.re, zp.re}, nim[4] = {ym.im, yp.im, zm.im, zp.im};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      two_sum(sr, nre[q], sr, t);
      cr = __fadd_rn(cr, t);
      two_sum(si, nim[q], si, t);
      ci = __fadd_rn(ci, t);
    }
    df_renorm(sr, cr, sr, cr);
    df_renorm(si, ci, si, ci);
    // N = (1/h^2) * sum
    float nrh, nrl, nih, nil;
    df_mul(ih2.x, ih2.y, sr, cr, nrh, nrl);
    df_mul(ih2.x, ih2.y, si, ci, nih, nil);
    // d_re = 6/h^2 - k^2
    const float2 kk = __ldg(k2df + p);
    float drh, drl;
    df_add(six_ih2.x, six_ih2.y, -kk.x, -kk.y, drh, drl);
    // v = d_re u_c - N (+ i d_im u_c at faces)
    float ah, al, bh, bl, vrh, vrl, vih, vil;
    df_mul_f(drh, drl, uc.re, ah, al);
    df_add(ah, al, -nrh, -nrl, vrh, vrl);
    df_mul_f(drh, drl, uc.im, bh, bl);
    df_add(bh, bl, -nih, -nil, vih, vil);
    if (nf) {
      // d_im = -(2/h) k nf
      const float2 kf = __ldg(skdf + p);
      float dih, dil;
      df_mul(two_over_h.x, two_over_h.y, kf.x, kf.y, dih, dil);
      df_mul_f(dih, dil, -(float)nf, dih, dil);
      // re -= d_im u_c.im ; im += d_im u_c.re
      df_mul_f(dih, dil, uc.im, ah, al);
      df_add(vrh, vrl, -ah, -al, vrh, vrl);
      df_mul_f(dih, dil, uc.re, bh, bl);
      df_add(vih, vil, bh, bl, vih, vil);
    }
    if constexpr (std::is_same<OUT, zdf>::value) {
      zdf o;
      o.rh = vrh; o.rl = vrl; o.ih = vih; o.il = vil;
      out[e] = o;
    } else {
      out[e] = mkc<double>((double)vrh + (double)vrl, (double)vih + (double)vil);
    }
    um = uc;
    uc = up;
  }
}

// (hi, lo) tables of k^2 and k = sqrt(k^2) from the FP64 k^2 (face terms use k).
__global__ void k_k2_df(const double* __restrict__ k2, size_t n, float2* __restrict__ k2df,
                        float2* __restrict__ skdf) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const double a = k2[q], b = sqrt(a);
    const float ah = (float)a, bh = (float)b;
    k2df[q] = make_float2(ah, (float)(a - (double)ah));
    skdf[q] = make_float2(bh, (float)(b - (double)bh));
  }
}

// ---- coarse sub-cycle in one CTA -------------------------------------------------------
// The V-cycle on the levels of cc (Sec. 3.4.5: zero start, one damped-Jacobi sweep before and
// after each coarse correction, the coarsest level solved exactly), run by one CTA with every
// vector in shared memory.  On grids of a few thousand unknowns each kernel of the level-by-level
// cycle is dominated by its launch and ramp; here the whole sub-cycle is one launch.  Every point
// takes the same arithmetic, in the same order, as the grid kernels (op_diag / op_resid /
// omega_over, the restriction's 27 weights, the interpolation average, the coarse product's
// lane-strided sum), so the results are those of the level-by-level cycle.
// q / d for 0 <= q < 2^22 and d >= 1 by a float reciprocal and one correction each way
// (an integer division takes tens of issue slots; the float estimate is within one of q / d).
__device__ __forceinline__ int cc_div(int q, int d, float rd) {
  int t = __float2int_rz((float)q * rd);
  if (t * d > q) --t;
  if ((t + 1) * d <= q) ++t;
  return t;
}
template <typename R>
__device__ __forceinline__ void cc_ijk(const Grid& g, int q, int& i, int& j, int& k) {
  const int t = cc_div(q, g.N1, 1.0f / (float)g.N1);
  i = q - t * g.N1;
  k = cc_div(t, g.N2, 1.0f / (float)g.N2);
  j = t - k * g.N2;
}

template <typename R>
__device__ __forceinline__ OpCoef<R> cc_coef(const CCycle<R>& cc, double h) {
  OpCoef<R> c;
  c.ih2 = (R)(1.0 / (h * h));
  c.six_ih2 = (R)(6.0 / (h * h));
  c.s_re = (R)cc.s_re;
  c.s_im = (R)cc.s_im;
  c.two_over_h = (R)(2.0 / h);
  c.omega = (R)cc.omega;
  c.real_shift = cc.s_im == 0.0;
  return c;
}

// out = b - M u (MODE 1) or u + (omega/d)(b - M u) (MODE 2) on one level, all in shared memory
// (k^2, sqrt(k^2) and omega/diag(M) read from their shared copies).
template <typename R, int MODE>
__device__ void cc_stencil(const CLevel<R>& F, const OpCoef<R>& c, const cx<R>* sm, const R* smr, int off_in,
                           cx<R>* out) {
  const Grid& g = F.g;
  const int n = (int)g.npts();
  const bool som = g.bc == 1;
  const cx<R> z0 = zero_c<R>();
  const cx<R>* u = sm + off_in;
  const cx<R>* b = sm + F.off_b;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    int i, j, k;
    cc_ijk<R>(g, q, i, j, k);
    const bool hxm = i > 0, hxp = i < g.N1 - 1, hym = j > 0, hyp = j < g.N2 - 1, hzp = k + 1 < g.N3;
    const int S = g.N1 * g.N2;
    int nf = som ? (!hxm) + (!hxp) + (!hym) + (!hyp) : 0;
    const cx<R> um = k > 0 ? u[q - S] : z0;
    const cx<R> up = hzp ? u[q + S] : z0;
    cx<R> zm, zp;
    if (k > 0) zm = um;
    else if (som) { zm = up; ++nf; }
    else zm = z0;
    if (hzp) zp = up;
    else if (som) { zp = um; ++nf; }
    else zp = z0;
    const cx<R> xm = hxm ? u[q - 1] : (som ? u[q + 1] : z0);
    const cx<R> xp = hxp ? u[q + 1] : (som ? u[q - 1] : z0);
    const cx<R> ym = hym ? u[q - g.N1] : (som ? u[q + g.N1] : z0);
    const cx<R> yp = hyp ? u[q + g.N1] : (som ? u[q - g.N1] : z0);
    const R kk = smr[F.off_k + q];
    const cx<R> d = op_diag(c, kk, nf, nf ? smr[F.off_s + q] : (R)0);
    const bool real_d = c.real_shift && nf == 0;
    const cx<R> uc = u[q];
    const cx<R> res = op_resid(b[q], d, real_d, uc, c.ih2, xm, xp, ym, yp, zm, zp);
    if (MODE == 1) {
      out[q] = res;
    } else {
      const cx<R> w = F.off_d >= 0 ? sm[F.off_d + q] : omega_over(d, c.omega);
      out[q] = cfma(w, res, uc);
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(CC_THREADS)
    k_coarse_cycle(CCycle<R> cc, const cx<R>* __restrict__ bin, cx<R>* __restrict__ eout,
                   const int* __restrict__ active) {
  if (active && *active == 0) return;
  extern __shared__ __align__(16) unsigned char cc_smem[];
  cx<R>* sm = reinterpret_cast<cx<R>*>(cc_smem);
  const R* smr = reinterpret_cast<const R*>(cc_smem);
  const int L = cc.L;
  // shared copies of the per-node coefficients, and the right-hand side
  for (int l = 0; l < L; ++l) {
    const CLevel<R>& F = cc.lev[l];
    const int n = (int)F.g.npts();
    R* sk = reinterpret_cast<R*>(cc_smem);
    const R* tab = grid_sqk<R>(F.g);
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const R kk = F.k2[q];
      sk[F.off_k + q] = kk;
      sk[F.off_s + q] = tab ? tab[q] : sqrt(kk);
      if (F.off_d >= 0) sm[F.off_d + q] = F.dinv[q];
    }
  }
  {
    const CLevel<R>& F = cc.lev[0];
    const int n = (int)F.g.npts();
    for (int q = threadIdx.x; q < n; q += blockDim.x) sm[F.off_b + q] = bin[q];
  }
  __syncthreads();
  // down: pre-smoothing from zero, residual, full weighting
  for (int l = 0; l < L - 1; ++l) {
    const CLevel<R>& F = cc.lev[l];
    const CLevel<R>& C = cc.lev[l + 1];
    const OpCoef<R> c = cc_coef(cc, F.g.h);
    const Grid& g = F.g;
    const int n = (int)g.npts();
    const bool som = g.bc == 1;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      cx<R> w;
      if (F.off_d >= 0) {
        w = sm[F.off_d + q];
      } else {
        int i, j, k;
        cc_ijk<R>(g, q, i, j, k);
        const int nf = som ? (i == 0) + (i == g.N1 - 1) + (j == 0) + (j == g.N2 - 1) + (k == 0) + (k == g.N3 - 1) : 0;
        const R kk = smr[F.off_k + q];
        w = omega_over(op_diag(c, kk, nf, nf ? smr[F.off_s + q] : (R)0), c.omega);
      }
      sm[F.off_u + q] = cmul(w, sm[F.off_b + q]);
    }
    __syncthreads();
    cc_stencil<R, 1>(F, c, sm, smr, F.off_u, sm + F.off_t);
    __syncthreads();
    const Grid& gc = C.g;
    const int nC = (int)gc.npts();
    const int off = g.bc == 0 ? 1 : 0;
    const cx<R>* r = sm + F.off_t;
    for (int Q = threadIdx.x; Q < nC; Q += blockDim.x) {
      int I, J, K;
      cc_ijk<R>(gc, Q, I, J, K);
      const int fi = 2 * (I + off) - off, fj = 2 * (J + off) - off, fk = 2 * (K + off) - off;
      R are = 0, aim = 0;
      for (int dz = -1; dz <= 1; ++dz) {
        const int z = fk + dz;
        if (z < 0 || z >= g.N3) continue;
        const R wz = dz ? (R)1 : (R)2;
        for (int dy = -1; dy <= 1; ++dy) {
          const int y = fj + dy;
          if (y < 0 || y >= g.N2) continue;
          const R wyz = wz * (dy ? (R)1 : (R)2);
          for (int dx = -1; dx <= 1; ++dx) {
            const int x = fi + dx;
            if (x < 0 || x >= g.N1) continue;
            const R wgt = wyz * (dx ? (R)1 : (R)2);
            const cx<R> v = r[(z * g.N2 + y) * g.N1 + x];
            are = fma(wgt, v.re, are);
            aim = fma(wgt, v.im, aim);
          }
        }
      }
      sm[C.off_b + Q] = mkc<R>(are * (R)(1.0 / 64.0), aim * (R)(1.0 / 64.0));
    }
    __syncthreads();
  }
  // coarsest: E = Minv B, one warp per row, lane-strided columns, fixed shuffle tree
  {
    const CLevel<R>& Cl = cc.lev[L - 1];
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int row = threadIdx.x >> 5; row < cc.nc; row += nw) {
      double re = 0, im = 0;
      const z128* a = cc.Minv + (size_t)row * cc.nc;
      for (int col = lane; col < cc.nc; col += 32) {
        const z128 m = a[col];
        const z128 v = cvt<double>(sm[Cl.off_b + col]);
        re = fma(m.re, v.re, re);
        re = fma(-m.im, v.im, re);
        im = fma(m.re, v.im, im);
        im = fma(m.im, v.re, im);
      }
      for (int o = 16; o; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane == 0) sm[Cl.off_u + row] = mkc<R>((R)re, (R)im);
    }
  }
  __syncthreads();
  // up: interpolation + correction, post-smoothing
  for (int l = L - 2; l >= 0; --l) {
    const CLevel<R>& F = cc.lev[l];
    const CLevel<R>& C = cc.lev[l + 1];
    const Grid& gf = F.g;
    const Grid& gc = C.g;
    const int n = (int)gf.npts();
    const int off = gf.bc == 0 ? 1 : 0;
    const cx<R>* e = sm + C.off_u;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      int i, j, k;
      cc_ijk<R>(gf, q, i, j, k);
      const int fi = i + off, fj = j + off, fk = k + off;
      const int cx_[2] = {(fi >> 1) - off, ((fi + 1) >> 1) - off};
      const int cy_[2] = {(fj >> 1) - off, ((fj + 1) >> 1) - off};
      const int cz_[2] = {(fk >> 1) - off, ((fk + 1) >> 1) - off};
      const int nx = (cx_[0] == cx_[1]) ? 1 : 2, ny = (cy_[0] == cy_[1]) ? 1 : 2, nz = (cz_[0] == cz_[1]) ? 1 : 2;
      R are = 0, aim = 0;
      for (int c = 0; c < nz; ++c) {
        if (cz_[c] < 0 || cz_[c] >= gc.N3) continue;
        for (int bq = 0; bq < ny; ++bq) {
          if (cy_[bq] < 0 || cy_[bq] >= gc.N2) continue;
          for (int a = 0; a < nx; ++a) {
            if (cx_[a] < 0 || cx_[a] >= gc.N1) continue;
            const cx<R> v = e[(cz_[c] * gc.N2 + cy_[bq]) * gc.N1 + cx_[a]];
            are += v.re;
            aim += v.im;
          }
        }
      }
      const R s = (R)1 / (R)(nx * ny * nz);
      const cx<R> base = sm[F.off_u + q];
      sm[F.off_t + q] = mkc<R>(fma(are, s, base.re), fma(aim, s, base.im));
    }
    __syncthreads();
    cc_stencil<R, 2>(F, cc_coef(cc, gf.h), sm, smr, F.off_t, sm + F.off_u);
    __syncthreads();
  }
  {
    const CLevel<R>& F = cc.lev[0];
    const int n = (int)F.g.npts();
    for (int q = threadIdx.x; q < n; q += blockDim.x) eout[q] = sm[F.off_u + q];
  }
}

// Discrete Dirac sources (Sec. 2.4): b(node) += 1/h^3, sources applied in order.
__global__ void k_rhs_point(Grid g, int nsrc, const int* __restrict__ idx, double amp, z128* __restrict__ b) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int s = 0; s < nsrc; ++s) {
    const int q = idx[s];
    if (q >= 0) b[q].re += amp;
  }
}

// Launch shape of kernel family `fam` in arithmetic R on grid g: TX x ty threads per CTA
// covering TX elements of an x-line by ty lines; CTAs along z split the N3 planes into
// chunks so that about g's CTA target runs (8 per SM unless tuned).
template <typename R>
dim3 grid_for(const Grid& g, int fam, int& zchunk, dim3& blk) {
  const int slot = tile_slot<R>(fam);
  const int ty = g.tile_ty[slot] > 0 ? g.tile_ty[slot] : TY;
  const int target = g.tile_ctas[slot] > 0 ? g.tile_ctas[slot] : 152 * 8;
  const int bx = (g.N1 * g.nb + TX - 1) / TX, by = (g.N2 + ty - 1) / ty;
  int zsplit = target / (bx * by);
  if (zsplit < 1) zsplit = 1;
  if (zsplit > g.N3) zsplit = g.N3;
  zchunk = (g.N3 + zsplit - 1) / zsplit;
  const int bz = (g.N3 + zchunk - 1) / zchunk;
  blk = dim3(TX, ty);
  return dim3(bx, by, bz);
}

template <typename R>
OpCoef<R> coef_for(double h, double s_re, double s_im, double omega) {
  OpCoef<R> c;
  c.ih2 = (R)(1.0 / (h * h));
  c.six_ih2 = (R)(6.0 / (h * h));
  c.s_re = (R)s_re;
  c.s_im = (R)s_im;
  c.two_over_h = (R)(2.0 / h);
  c.omega = (R)omega;
  c.real_shift = s_im == 0.0;
  return c;
}

}  // namespace

// ------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------
// Launch shape of the tiled FP32 kernels: 32 x TYT threads, the tuned CTA count for z.
static dim3 grid_tiled(const Grid& g, int& zchunk) {
  const int slot = tile_slot<float>(TILE_STENCIL);
  const int target = g.tile_ctas[slot] > 0 ? g.tile_ctas[slot] : 152 * 8;
  const int bx = (g.N1 + TX - 1) / TX, by = (g.N2 + TYT - 1) / TYT;
  int zsplit = target / (bx * by);
  if (zsplit < 1) zsplit = 1;
  if (zsplit > g.N3) zsplit = g.N3;
  zchunk = (g.N3 + zsplit - 1) / zsplit;
  return dim3(bx, by, (g.N3 + zchunk - 1) / zchunk);
}

template <typename R, typename TU, typename TO>
void launch_apply(const Grid& g, double s_re, double s_im, const R* k2, const cx<TU>* u, cx<TO>* v,
                  cudaStream_t st, const int* active) {
  int zc;
  if constexpr (std::is_same<R, float>::value) {
    if (g.nb == 1 && g.tiled) {
      const dim3 gr = grid_tiled(g, zc);
      k_stencil32_tiled<0, TU, TU, TO><<<gr, dim3(TX, TYT), 0, st>>>(g, coef_for<R>(g.h, s_re, s_im, 0.0), k2, u,
                                                                    nullptr, v, zc, active);
      return;
    }
  }
  dim3 blk, gr = grid_for<R>(g, TILE_STENCIL, zc, blk);
  k_stencil<R, 0, false, TU, TU, TO><<<gr, blk, 0, st>>>(g, coef_for<R>(g.h, s_re, s_im, 0.0), k2, nullptr, u,
                                                                   nullptr, v, zc, active);
}

static float2 df_const(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

template <typename OUT>
void launch_apply_c64_df(const Grid& g, const float2* k2df, const float2* skdf, const z64* u, OUT* v, cudaStream_t st,
                         const int* active) {
  int zc;
  dim3 blk, gr = grid_for<float>(g, TILE_STENCIL, zc, blk);
  k_apply_c64_df<OUT><<<gr, blk, 0, st>>>(g, df_const(1.0 / (g.h * g.h)), df_const(6.0 / (g.h * g.h)),
                                          df_const(2.0 / g.h), k2df, skdf, u, v, zc, active);
}
template void launch_apply_c64_df<zdf>(const Grid&, const float2*, const float2*, const z64*, zdf*, cudaStream_t,
                                       const int*);
template void launch_apply_c64_df<z128>(const Grid&, const float2*, const float2*, const z64*, z128*, cudaStream_t,
                                        const int*);

void launch_k2_df(const double* k2, size_t n, float2* k2df, float2* skdf, cudaStream_t st) {
  size_t b = (n + 255) / 256;
  k_k2_df<<<(int)(b < 4096 ? (b ? b : 1) : 4096), 256, 0, st>>>(k2, n, k2df, skdf);
}

template <typename TU>
void launch_apply_split(const Grid& g, double s_re, double s_im, const double* k2, const cx<TU>* u, zdf* v,
                        cudaStream_t st, const int* active) {
  int zc;
  dim3 blk, gr = grid_for<double>(g, TILE_STENCIL, zc, blk);
  k_stencil<double, 0, false, TU, TU, double, true><<<gr, blk, 0, st>>>(
      g, coef_for<double>(g.h, s_re, s_im, 0.0), k2, nullptr, u, nullptr, reinterpret_cast<z128*>(v), zc, active);
}
template void launch_apply_split<double>(const Grid&, double, double, const double*, const z128*, zdf*, cudaStream_t,
                                         const int*);
template void launch_apply_split<float>(const Grid&, double, double, const double*, const z64*, zdf*, cudaStream_t,
                                        const int*);

template <typename R, typename TU, typename TB, typename TO>
void launch_resid(const Grid& g, double s_re, double s_im, const R* k2, const cx<TU>* u, const cx<TB>* b,
                  cx<TO>* out, cudaStream_t st, const int* active) {
  int zc;
  if constexpr (std::is_same<R, float>::value) {
    if (g.nb == 1 && g.tiled) {
      const dim3 gr = grid_tiled(g, zc);
      k_stencil32_tiled<1, TU, TB, TO><<<gr, dim3(TX, TYT), 0, st>>>(g, coef_for<R>(g.h, s_re, s_im, 0.0), k2, u, b,
                                                                    out, zc, active);
      return;
    }
  }
  dim3 blk, gr = grid_for<R>(g, TILE_STENCIL, zc, blk);
  k_stencil<R, 1, false, TU, TB, TO><<<gr, blk, 0, st>>>(g, coef_for<R>(g.h, s_re, s_im, 0.0), k2, nullptr,
                                                                   u, b, out, zc, active);
}

template <typename R, typename TB, typename TO>
void launch_jacobi(const Grid& g, double s_re, double s_im, double omega, const R* k2, const cx<R>* dinv,
                   const cx<R>* u, const cx<TB>* b, cx<TO>* out, cudaStream_t st, const int* active) {
  int zc;
  OpCoef<R> c = coef_for<R>(g.h, s_re, s_im, omega);
  if constexpr (std::is_same<R, float>::value) {
    if (g.nb == 1 && g.tiled && !dinv) {
      const dim3 gr = grid_tiled(g, zc);
      k_stencil32_tiled<2, R, TB, TO><<<gr, dim3(TX, TYT), 0, st>>>(g, c, k2, u, b, out, zc, active);
      return;
    }
  }
  dim3 blk, gr = grid_for<R>(g, TILE_STENCIL, zc, blk);
  if (dinv)
    k_stencil<R, 2, true, R, TB, TO><<<gr, blk, 0, st>>>(g, c, k2, dinv, u, b, out, zc, active);
  else
    k_stencil<R, 2, false, R, TB, TO><<<gr, blk, 0, st>>>(g, c, k2, dinv, u, b, out, zc, active);
}

template <typename R, typename TB>
void launch_smooth0(const Grid& g, double s_re, double s_im, double omega, const R* k2, const cx<R>* dinv,
                    const cx<TB>* b, cx<R>* out, cudaStream_t st, const int* active) {
  int zc;
  dim3 blk, gr = grid_for<R>(g, TILE_SMOOTH0, zc, blk);
  OpCoef<R> c = coef_for<R>(g.h, s_re, s_im, omega);
  if (dinv)
    k_smooth0<R, true, TB><<<gr, blk, 0, st>>>(g, c, k2, dinv, b, out, zc, active);
  else
    k_smooth0<R, false, TB><<<gr, blk, 0, st>>>(g, c, k2, dinv, b, out, zc, active);
}

template <typename TB>
void launch_smooth0_resid32(const Grid& g, double s_re, double s_im, double omega, const float* k2, const cx<TB>* b,
                            z64* u1, z64* r, cudaStream_t st, const int* active) {
  int zc;
  dim3 blk, gr = grid_for<float>(g, TILE_SMOOTH0, zc, blk);
  k_smooth0_resid32<TB><<<gr, blk, 0, st>>>(g, coef_for<float>(g.h, s_re, s_im, omega), k2, b, u1, r, zc, active);
}
template void launch_smooth0_resid32<float>(const Grid&, double, double, double, const float*, const z64*, z64*, z64*,
                                            cudaStream_t, const int*);
template void launch_smooth0_resid32<double>(const Grid&, double, double, double, const float*, const z128*, z64*,
                                             z64*, cudaStream_t, const int*);

template <typename R>
void launch_restrict(const Grid& gf, const Grid& gc, const cx<R>* r, cx<R>* out, cudaStream_t st, const int* active) {
  int zc;
  dim3 blk, gr = grid_for<R>(gc, TILE_RESTRICT, zc, blk);
  k_restrict<R><<<gr, blk, 0, st>>>(gf, gc, r, out, zc, active);
}

template <typename R>
void launch_prolong_add(const Grid& gf, const Grid& gc, const cx<R>* u1, const cx<R>* e, cx<R>* out, cudaStream_t st,
                        const int* active) {
  int zc;
  dim3 blk, gr = grid_for<R>(gf, TILE_PROLONG, zc, blk);
  k_prolong_add<R><<<gr, blk, 0, st>>>(gf, gc, u1, e, out, zc, active);
}

template <typename TI, typename TO>
void launch_coarse(int nc, const z128* Minv, const cx<TI>* b, cx<TO>* e, cudaStream_t st, const int* active, int nb) {
  if (nb == 1) {
    const int wpb = 8;
    k_coarse<TI, TO><<<(nc + wpb - 1) / wpb, wpb * 32, 0, st>>>(nc, Minv, b, e, active);
  } else {
    k_coarse_b<TI, TO><<<(nc * nb + 255) / 256, 256, 0, st>>>(nc, nb, Minv, b, e, active);
  }
}

void launch_dinv(const Grid& g, double s_re, double s_im, double omega, const double* k2, z128* out, cudaStream_t st) {
  k_dinv<<<1216, 256, 0, st>>>(g, coef_for<double>(g.h, s_re, s_im, omega), k2, out);
}

void launch_inject(const Grid& gf, const Grid& gc, const double* kf, double* kc, cudaStream_t st) {
  k_inject<<<1216, 256, 0, st>>>(gf, gc, kf, kc);
}

void launch_sqrt_table(const double* k2, double* sk, float* skf, size_t n, cudaStream_t st) {
  k_sqrt_table<<<1216, 256, 0, st>>>(k2, sk, skf, n);
}

void launch_to_float(const double* a, float* b, size_t n, cudaStream_t st) {
  k_to_float<<<1216, 256, 0, st>>>(a, b, n);
}

void launch_check_k2(const double* a, size_t n, int* bad, cudaStream_t st) {
  k_check_k2<<<1216, 256, 0, st>>>(a, n, bad);
}

void launch_rhs_point(const Grid& g, int nsrc, const int* idx, double amp, z128* b, cudaStream_t st) {
  k_rhs_point<<<1, 32, 0, st>>>(g, nsrc, idx, amp, b);
}

template <typename R>
bool coarse_cycle_ready() {
  static const bool ok = [] {
    const bool r = cudaFuncSetAttribute(k_coarse_cycle<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)CC_SMEM_MAX) == cudaSuccess;
    cudaGetLastError();
    return r;
  }();
  return ok;
}
template <typename R>
void launch_coarse_cycle(const CCycle<R>& cc, size_t smem_bytes, const cx<R>* b, cx<R>* e, cudaStream_t st,
                         const int* active) {
  k_coarse_cycle<R><<<1, CC_THREADS, smem_bytes, st>>>(cc, b, e, active);
}
template bool coarse_cycle_ready<double>();
template bool coarse_cycle_ready<float>();
template void launch_coarse_cycle<double>(const CCycle<double>&, size_t, const z128*, z128*, cudaStream_t, const int*);
template void launch_coarse_cycle<float>(const CCycle<float>&, size_t, const z64*, z64*, cudaStream_t, const int*);

// explicit instantiations used by the library
#define HELM_INST_R(R)                                                                                   \
  template void launch_restrict<R>(const Grid&, const Grid&, const cx<R>*, cx<R>*, cudaStream_t, const int*); \
  template void launch_prolong_add<R>(const Grid&, const Grid&, const cx<R>*, const cx<R>*, cx<R>*, cudaStream_t, const int*);
HELM_INST_R(double)
HELM_INST_R(float)

template void launch_apply<double, double, double>(const Grid&, double, double, const double*, const z128*, z128*, cudaStream_t, const int*);
template void launch_apply<double, float, double>(const Grid&, double, double, const double*, const z64*, z128*, cudaStream_t, const int*);
template void launch_apply<float, float, float>(const Grid&, double, double, const float*, const z64*, z64*, cudaStream_t, const int*);
template void launch_resid<double, double, double, double>(const Grid&, double, double, const double*, const z128*, const z128*, z128*, cudaStream_t, const int*);
template void launch_resid<double, double, double, float>(const Grid&, double, double, const double*, const z128*, const z128*, z64*, cudaStream_t, const int*);
template void launch_resid<float, float, float, float>(const Grid&, double, double, const float*, const z64*, const z64*, z64*, cudaStream_t, const int*);
template void launch_resid<float, float, double, float>(const Grid&, double, double, const float*, const z64*, const z128*, z64*, cudaStream_t, const int*);
template void launch_jacobi<double, double, double>(const Grid&, double, double, double, const double*, const z128*, const z128*, const z128*, z128*, cudaStream_t, const int*);
template void launch_jacobi<float, float, float>(const Grid&, double, double, double, const float*, const z64*, const z64*, const z64*, z64*, cudaStream_t, const int*);
template void launch_jacobi<float, double, float>(const Grid&, double, double, double, const float*, const z64*, const z64*, const z128*, z64*, cudaStream_t, const int*);
template void launch_jacobi<float, double, double>(const Grid&, double, double, double, const float*, const z64*, const z64*, const z128*, z128*, cudaStream_t, const int*);
template void launch_jacobi<float, float, double>(const Grid&, double, double, double, const float*, const z64*, const z64*, const z64*, z128*, cudaStream_t, const int*);
template void launch_jacobi<double, double, float>(const Grid&, double, double, double, const double*, const z128*, const z128*, const z128*, z64*, cudaStream_t, const int*);
template void launch_smooth0<double, double>(const Grid&, double, double, double, const double*, const z128*, const z128*, z128*, cudaStream_t, const int*);
template void launch_smooth0<float, float>(const Grid&, double, double, double, const float*, const z64*, const z64*, z64*, cudaStream_t, const int*);
template void launch_smooth0<float, double>(const Grid&, double, double, double, const float*, const z64*, const z128*, z64*, cudaStream_t, const int*);
template void launch_coarse<double, double>(int, const z128*, const z128*, z128*, cudaStream_t, const int*, int);
template void launch_coarse<float, float>(int, const z128*, const z64*, z64*, cudaStream_t, const int*, int);
template void launch_coarse<double, float>(int, const z128*, const z128*, z64*, cudaStream_t, const int*, int);
template void launch_coarse<float, double>(int, const z128*, const z64*, z128*, cudaStream_t, const int*, int);

}  // namespace helm
