// stencil.cu -- matrix-free grid kernels of libhelm: the 7-point Helmholtz / CSLP operator
// (Sec. 2.4, Sec. 3.5 Algorithm 2), damped Jacobi (Sec. 3.4.1), full-weighting restriction
// (Sec. 3.4.2), trilinear interpolation (Sec. 3.4.3), k^2 injection for the DCG coarse
// operators (Sec. 3.4.4), the exact coarsest-grid solve and the set-up inverse behind it.
//
// The streaming grid kernels map a 32 x rows tile of (x, y) columns to a block and stream along
// z: the z-1 / z / z+1 values of a thread's own column stay in registers (2.5D streaming), the
// in-plane neighbours come through the read-only L1 path; in FP32 the next plane's loads are
// issued one trip ahead.  The fused sweep kernels (k_down32, k_up, k_rr) instead keep
// three-plane rings of their tile and halo in shared memory.
#include "internal.cuh"

#include <type_traits>

namespace helm {

namespace {

constexpr int TX = 32, TY = 8;

template <typename T>
__device__ __forceinline__ cx<T> zero_c() {
  return mkc<T>((T)0, (T)0);
}

// Full weighting (Sec. 3.4.2) in one fixed order that every restriction kernel shares, so that
// the separate and the fused forms give identical results.  The weights (8, 4, 2, 1) / 64 are
// the product of (1, 2, 1) / 4 along each axis, applied x first: per fine line
// fx = 2 r_0 + (r_-1 + r_+1), per fine plane p = 2 fx_0 + (fx_-1 + fx_+1), and
// b_H = (2 p_0 + (p_-1 + p_+1)) / 64, each as one FMA after one addition; fine values outside
// the grid count as 0.
template <typename R>
__device__ __forceinline__ cx<R> fw3(cx<R> m, cx<R> c, cx<R> p) {
  return mkc<R>(fma((R)2, c.re, m.re + p.re), fma((R)2, c.im, m.im + p.im));
}
template <typename R, typename Get>
__device__ __forceinline__ cx<R> fw_plane(int fi, int fj, int N1, int N2, Get&& get) {
  cx<R> fx[3];
  for (int dy = -1; dy <= 1; ++dy) {
    const int y = fj + dy;
    cx<R> v[3];
    for (int dx = -1; dx <= 1; ++dx) {
      const int x = fi + dx;
      v[dx + 1] = (y >= 0 && y < N2 && x >= 0 && x < N1) ? get(x, y) : mkc<R>((R)0, (R)0);
    }
    fx[dy + 1] = fw3(v[0], v[1], v[2]);
  }
  return fw3(fx[0], fx[1], fx[2]);
}
template <typename R>
__device__ __forceinline__ cx<R> fw_combine(cx<R> pm, cx<R> p0, cx<R> pp) {
  const cx<R> t = fw3(pm, p0, pp);
  return mkc<R>(t.re * (R)(1.0 / 64.0), t.im * (R)(1.0 / 64.0));
}

// Trilinear interpolation (Sec. 3.4.3) in one fixed order shared by every prolongation kernel.
// A fine node at an odd node index along an axis lies between the coarse nodes either side, at
// an even index on one; coarse parents outside the unknown set (Dirichlet boundary) count as 0,
// and the divisor counts every parent.  The parents are summed y first, then z, then x:
// ty(X, Z) = e(X, y0, Z) [+ e(X, y1, Z)], tz(X) = ty(X, z0) [+ ty(X, z1)],
// t = tz(x0) [+ tz(x1)], and u2 = u1 + t / (nx ny nz) as one FMA per component.
template <typename R>
__device__ __forceinline__ R tl_scale(int cnt) {  // 1 / cnt for cnt in {1, 2, 4, 8}, without a division
  return cnt == 1 ? (R)1 : cnt == 2 ? (R)0.5 : cnt == 4 ? (R)0.25 : (R)0.125;
}
template <typename R, typename Get>
__device__ __forceinline__ cx<R> tl_value(int fi, int fj, int fk, int off, const Grid& gc, cx<R> base, Get&& get) {
  const int xs[2] = {(fi >> 1) - off, ((fi + 1) >> 1) - off};
  const int ys[2] = {(fj >> 1) - off, ((fj + 1) >> 1) - off};
  const int zs[2] = {(fk >> 1) - off, ((fk + 1) >> 1) - off};
  const int nx = xs[0] == xs[1] ? 1 : 2, ny = ys[0] == ys[1] ? 1 : 2, nz = zs[0] == zs[1] ? 1 : 2;
  auto val = [&](int X, int Y, int Z) {
    return (X >= 0 && X < gc.N1 && Y >= 0 && Y < gc.N2 && Z >= 0 && Z < gc.N3) ? get(X, Y, Z) : mkc<R>((R)0, (R)0);
  };
  auto ty = [&](int X, int Z) {
    cx<R> v = val(X, ys[0], Z);
    if (ny == 2) v = cadd(v, val(X, ys[1], Z));
    return v;
  };
  auto tz = [&](int X) {
    cx<R> v = ty(X, zs[0]);
    if (nz == 2) v = cadd(v, ty(X, zs[1]));
    return v;
  };
  cx<R> t = tz(xs[0]);
  if (nx == 2) t = cadd(t, tz(xs[1]));
  const R sc = tl_scale<R>(nx * ny * nz);
  return mkc<R>(fma(t.re, sc, base.re), fma(t.im, sc, base.im));
}

// One stencil kernel for three uses (MODE):
//   APPLY  : out = Op u
//   RESID  : out = b - Op u
//   JACOBI : out = u + (omega / d) (b - Op u)
// with Op = -Lap_h - s k^2 (s in OpCoef).  DINV (FP64 multigrid levels): read the diagonal d
// of M and omega/d from the level's coefficient table (omega/d at [0, npts), d at [npts,
// 2 npts)) instead of computing them from k^2: on this GPU FP64 instructions, not bytes, bound
// these kernels, and the table holds the very values op_diag and the division would give.
// REALA (the operator A, real shift s = 1, APPLY or RESID): the diagonal is real away from the
// Sommerfeld faces, so the two products with its imaginary part are issued only at face nodes
// (same operations in the same order as the general path, so the same results).  With g.nb
// right-hand sides per node, a thread owns one (node column, rhs) pair; for nb = 32 a warp
// covers the 32 right-hand sides of one node with one 256-byte (complex64) row and reads k^2
// once.
template <typename R, int MODE, bool DINV, typename TU, typename TB, typename TO, bool SPLIT = false,
          bool REALA = false>
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
  // FP32 (memory-bound): the next trip's z neighbour, k^2 and b are loaded one trip ahead, so
  // each thread keeps two planes' loads in flight
  constexpr bool PF = std::is_same<R, float>::value;
  // the prefetched b stays in its stored precision until it is used: a conversion right after
  // the load would wait for the load and undo the prefetch
  cx<R> upf = (PF && k0 + 1 < g.N3) ? ld(e + Se) : zero_c<R>();
  R kpf = PF ? __ldg(k2 + p) : (R)0;
  cx<TB> bpf = (PF && MODE != 0) ? ldg(b + e) : zero_c<TB>();
  for (int k = k0; k < k1; ++k, p += S, e += Se) {
    const bool hzp = k + 1 < g.N3;
    cx<R> up, bv = zero_c<R>();
    R kk;
    if constexpr (PF) {
      up = upf;
      kk = kpf;
      bv = cvt<R>(bpf);
      if (k + 1 < k1) {
        upf = k + 2 < g.N3 ? ld(e + 2 * Se) : zero_c<R>();
        kpf = __ldg(k2 + p + S);
        if (MODE != 0) bpf = ldg(b + e + Se);
      }
    } else {
      up = hzp ? ld(e + Se) : zero_c<R>();
    }
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
    if constexpr (!PF) {
      if (!DINV) kk = __ldg(k2 + p);
      if (MODE != 0) bv = cvt<R>(ldg(b + e));
    }
    if constexpr (REALA && MODE != 2) {
      // real diagonal 6/h^2 - k^2; a face node adds -i (2k/h) nf (op_diag's face term)
      const cx<R> dr = mkc<R>(fma(-c.s_re, kk, c.six_ih2), (R)0);
      cx<R> v = MODE == 0 ? op_apply(dr, true, uc, c.ih2, xm, xp, ym, yp, zm, zp)
                          : op_resid(bv, dr, true, uc, c.ih2, xm, xp, ym, yp, zm, zp);
      if (nf) {
        const R dim = fma(-(R)nf * c.two_over_h, face_k<R>(g, p, kk), (R)0);
        if (MODE == 0) {
          v.re = fma(-dim, uc.im, v.re);
          v.im = fma(dim, uc.re, v.im);
        } else {
          v.re = fma(dim, uc.im, v.re);
          v.im = fma(-dim, uc.re, v.im);
        }
      }
      if (MODE == 0 && SPLIT)
        reinterpret_cast<zdf*>(out)[e] = df_from(cvt<double>(v));
      else
        out[e] = cvt<TO>(v);
      um = uc;
      uc = up;
      continue;
    }
    const cx<R> d = DINV ? ldg(dinv + g.npts() + p) : op_diag(c, kk, nf, nf ? face_k<R>(g, p, kk) : (R)0);
    const bool real_d = c.real_shift && nf == 0;
    if (MODE == 0) {
      const cx<R> v = op_apply(d, real_d, uc, c.ih2, xm, xp, ym, yp, zm, zp);
      if (SPLIT)  // the output buffer holds double-float values (16 bytes, like complex128)
        reinterpret_cast<zdf*>(out)[e] = df_from(cvt<double>(v));
      else
        out[e] = cvt<TO>(v);
    } else {
      const cx<R> res = op_resid(bv, d, real_d, uc, c.ih2, xm, xp, ym, yp, zm, zp);
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

// The whole down-sweep of one FP32 level (one right-hand side) in one kernel: pre-smoothing from
// zero (u1 = (omega/d) b, Sec. 3.4.1), the residual r = b - M u1 and its full-weighting
// restriction (Sec. 3.4.2) to the next level's right-hand side.  r never goes to memory.
// A CTA owns DCX x DCY coarse columns and a chunk of coarse planes.  It streams the fine planes
// in z: u1 over the fine window with a halo of two, r over the window with a halo of one, each
// in a three-plane ring in shared memory, and after fine plane 2K + off + 1 the coarse plane K.
// u1 is also written to memory for the fine points this CTA owns (the windows of neighbouring
// CTAs overlap; ownership tiles the grid).  Every value goes through the same arithmetic in
// the same order as k_smooth0 / k_stencil(resid) / k_restrict, so the results are identical.
constexpr int DCX = 16, DCY = 8, DNT = 256;
constexpr int DUX = 2 * DCX + 3, DUY = 2 * DCY + 3, DRX = 2 * DCX + 1, DRY = 2 * DCY + 1;
template <typename TB>
__global__ void __launch_bounds__(DNT)
    k_down32(Grid gf, Grid gc, OpCoef<float> c, const float* __restrict__ k2, const cx<TB>* __restrict__ b,
             z64* __restrict__ u1, z64* __restrict__ bco, int kchunk, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ z64 su[3][DUY][DUX];
  __shared__ z64 sr[3][DRY][DRX];
  const int off = gf.bc == 0 ? 1 : 0;  // the fine centre of coarse node I is 2 I + off
  const bool som = gf.bc == 1;
  const int N1 = gf.N1, N2 = gf.N2, N3 = gf.N3;
  const int I0 = blockIdx.x * DCX, J0 = blockIdx.y * DCY, K0 = blockIdx.z * kchunk;
  if (K0 >= gc.N3) return;
  const int K1 = min(K0 + kchunk, gc.N3);
  const int rx0 = 2 * I0 + off - 1, ry0 = 2 * J0 + off - 1, rz0 = 2 * K0 + off - 1;
  const int ux0 = rx0 - 1, uy0 = ry0 - 1;
  const int ox0 = I0 == 0 ? 0 : rx0, ox1 = I0 + DCX >= gc.N1 ? N1 : rx0 + 2 * DCX;
  const int oy0 = J0 == 0 ? 0 : ry0, oy1 = J0 + DCY >= gc.N2 ? N2 : ry0 + 2 * DCY;
  const int oz0 = K0 == 0 ? 0 : rz0, oz1 = K1 >= gc.N3 ? N3 : 2 * K1 + off - 1;
  const int zlo = max(rz0, 0), zhi = min(2 * (K1 - 1) + off + 1, N3 - 1);
  const z64 z0 = mkc<float>(0.f, 0.f);
  auto fill_u = [&](int z) {
    z64(*U)[DUX] = su[z % 3];
    for (int t = threadIdx.x; t < DUX * DUY; t += DNT) {
      const int ly = t / DUX, lx = t - ly * DUX;
      const int x = ux0 + lx, y = uy0 + ly;
      z64 v = z0;
      if (x >= 0 && x < N1 && y >= 0 && y < N2) {
        const size_t q = gidx(x, y, z, N1, N2);
        const int nf = som ? (x == 0) + (x == N1 - 1) + (y == 0) + (y == N2 - 1) + (z == 0) + (z == N3 - 1) : 0;
        const float kq = __ldg(k2 + q);
        const z64 w = omega_over(op_diag(c, kq, nf, nf ? face_k<float>(gf, q, kq) : 0.f), c.omega);
        v = cmul(w, cvt<float>(ldg(b + q)));
        if (x >= ox0 && x < ox1 && y >= oy0 && y < oy1 && z >= oz0 && z < oz1) u1[q] = v;
      }
      U[ly][lx] = v;
    }
  };
  auto fill_r = [&](int z) {
    const z64(*Um)[DUX] = su[(z + 2) % 3];
    const z64(*Uc)[DUX] = su[z % 3];
    const z64(*Up)[DUX] = su[(z + 1) % 3];
    z64(*Rz)[DRX] = sr[z % 3];
    const bool hzm = z > 0, hzp = z + 1 < N3;
    for (int t = threadIdx.x; t < DRX * DRY; t += DNT) {
      const int ly = t / DRX, lx = t - ly * DRX;
      const int x = rx0 + lx, y = ry0 + ly;
      z64 v = z0;
      if (x >= 0 && x < N1 && y >= 0 && y < N2) {
        const int li = lx + 1, lj = ly + 1;
        const bool hxm = x > 0, hxp = x < N1 - 1, hym = y > 0, hyp = y < N2 - 1;
        int nf = som ? (!hxm) + (!hxp) + (!hym) + (!hyp) : 0;
        const z64 uc = Uc[lj][li];
        z64 zm, zp;
        if (hzm) zm = Um[lj][li];
        else if (som) { zm = Up[lj][li]; ++nf; }
        else zm = z0;
        if (hzp) zp = Up[lj][li];
        else if (som) { zp = Um[lj][li]; ++nf; }
        else zp = z0;
        const z64 xm = hxm ? Uc[lj][li - 1] : (som ? Uc[lj][li + 1] : z0);
        const z64 xp = hxp ? Uc[lj][li + 1] : (som ? Uc[lj][li - 1] : z0);
        const z64 ym = hym ? Uc[lj - 1][li] : (som ? Uc[lj + 1][li] : z0);
        const z64 yp = hyp ? Uc[lj + 1][li] : (som ? Uc[lj - 1][li] : z0);
        const size_t q = gidx(x, y, z, N1, N2);
        const float kk = __ldg(k2 + q);
        const z64 d = op_diag(c, kk, nf, nf ? face_k<float>(gf, q, kk) : 0.f);
        const bool real_d = c.real_shift && nf == 0;
        v = op_resid(cvt<float>(ldg(b + q)), d, real_d, uc, c.ih2, xm, xp, ym, yp, zm, zp);
      }
      Rz[ly][lx] = v;
    }
  };
  auto restrict_plane = [&](int K) {
    const int fk = 2 * K + off;
    for (int t = threadIdx.x; t < DCX * DCY; t += DNT) {
      const int ly = t / DCX, lx = t - ly * DCX;
      const int I = I0 + lx, J = J0 + ly;
      if (I >= gc.N1 || J >= gc.N2) continue;
      const int fi = 2 * I + off, fj = 2 * J + off;
      z64 p[3];
      for (int dz = -1; dz <= 1; ++dz) {
        const int z = fk + dz;
        p[dz + 1] = z0;
        if (z < 0 || z >= N3) continue;
        const z64(*Rz)[DRX] = sr[z % 3];
        p[dz + 1] = fw_plane<float>(fi, fj, N1, N2, [&](int x, int y) { return Rz[y - ry0][x - rx0]; });
      }
      bco[gidx(I, J, K, gc.N1, gc.N2)] = fw_combine(p[0], p[1], p[2]);
    }
  };
  if (zlo > 0) fill_u(zlo - 1);
  fill_u(zlo);
  int K = K0;
  for (int z = zlo; z <= zhi; ++z) {
    if (z + 1 < N3) fill_u(z + 1);
    __syncthreads();
    fill_r(z);
    __syncthreads();
    // coarse plane K needs fine r planes 2K + off - 1 .. 2K + off + 1 (those inside the grid)
    while (K < K1 && min(2 * K + off + 1, N3 - 1) == z) restrict_plane(K++);
  }
}

// The whole up-sweep of one level (one right-hand side) in one kernel: u2 = u1 + P e
// (trilinear interpolation, Sec. 3.4.3) and the post-smoothing u3 = u2 + (omega/d)(b - M u2)
// (Sec. 3.4.1).  u2 never goes to memory: a CTA of 32 x UTY fine columns computes it over its
// window with a halo of one into a three-plane ring in shared memory while it streams its
// z-chunk.  Same arithmetic per point, in the same order, as k_prolong_add and
// k_stencil(jacobi) (DINV: the FP64 level's table of omega/d and d), so the results are
// identical.
constexpr int UTY = 8, UWX = TX + 2, UWY = UTY + 2;
template <typename R, bool DINV, typename TB, typename TO>
__global__ void __launch_bounds__(TX* UTY)
    k_up(Grid gf, Grid gc, OpCoef<R> c, const R* __restrict__ k2, const cx<R>* __restrict__ dinv,
         const cx<R>* __restrict__ u1, const cx<R>* __restrict__ e, const cx<TB>* __restrict__ b,
         cx<TO>* __restrict__ out, int zchunk, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ cx<R> su[3][UWY][UWX];
  const int N1 = gf.N1, N2 = gf.N2, N3 = gf.N3;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * UTY;
  const int k0 = blockIdx.z * zchunk;
  if (k0 >= N3) return;
  const int k1 = min(k0 + zchunk, N3);
  const int off = gf.bc == 0 ? 1 : 0;
  const bool som = gf.bc == 1;
  const size_t NP = gf.npts();
  const cx<R> z0 = zero_c<R>();
  const int tid = threadIdx.y * TX + threadIdx.x;
  auto fill = [&](int z) {
    cx<R>(*U)[UWX] = su[z % 3];
    for (int t = tid; t < UWX * UWY; t += TX * UTY) {
      const int ly = t / UWX, lx = t - ly * UWX;
      const int x = x0 - 1 + lx, y = y0 - 1 + ly;
      cx<R> v = z0;
      if (x >= 0 && x < N1 && y >= 0 && y < N2)
        v = tl_value<R>(x + off, y + off, z + off, off, gc, ldg(u1 + gidx(x, y, z, N1, N2)),
                        [&](int X, int Y, int Z) { return ldg(e + gidx(X, Y, Z, gc.N1, gc.N2)); });
      U[ly][lx] = v;
    }
  };
  const int i = x0 + threadIdx.x, j = y0 + threadIdx.y;
  const int li = threadIdx.x + 1, lj = threadIdx.y + 1;
  const bool inside = i < N1 && j < N2;
  const bool hxm = i > 0, hxp = i < N1 - 1, hym = j > 0, hyp = j < N2 - 1;
  const int nfxy = som ? (!hxm) + (!hxp) + (!hym) + (!hyp) : 0;
  if (k0 > 0) fill(k0 - 1);
  fill(k0);
  for (int k = k0; k < k1; ++k) {
    const bool hzp = k + 1 < N3;
    if (hzp) fill(k + 1);
    __syncthreads();
    if (inside) {
      const cx<R>(*Um)[UWX] = su[(k + 2) % 3];
      const cx<R>(*Uc)[UWX] = su[k % 3];
      const cx<R>(*Up)[UWX] = su[(k + 1) % 3];
      int nf = nfxy;
      const cx<R> uc = Uc[lj][li];
      cx<R> zm, zp;
      if (k > 0) zm = Um[lj][li];
      else if (som) { zm = Up[lj][li]; ++nf; }
      else zm = z0;
      if (hzp) zp = Up[lj][li];
      else if (som) { zp = Um[lj][li]; ++nf; }
      else zp = z0;
      const cx<R> xm = hxm ? Uc[lj][li - 1] : (som ? Uc[lj][li + 1] : z0);
      const cx<R> xp = hxp ? Uc[lj][li + 1] : (som ? Uc[lj][li - 1] : z0);
      const cx<R> ym = hym ? Uc[lj - 1][li] : (som ? Uc[lj + 1][li] : z0);
      const cx<R> yp = hyp ? Uc[lj + 1][li] : (som ? Uc[lj - 1][li] : z0);
      const size_t p = gidx(i, j, k, N1, N2);
      cx<R> d, w;
      if constexpr (DINV) {
        d = ldg(dinv + NP + p);
        w = ldg(dinv + p);
      } else {
        const R kk = __ldg(k2 + p);
        d = op_diag(c, kk, nf, nf ? face_k<R>(gf, p, kk) : (R)0);
        w = omega_over(d, c.omega);
      }
      const bool real_d = c.real_shift && nf == 0;
      const cx<R> res = op_resid(cvt<R>(ldg(b + p)), d, real_d, uc, c.ih2, xm, xp, ym, yp, zm, zp);
      out[p] = cvt<TO>(cfma(w, res, uc));
    }
    __syncthreads();
  }
}

// Residual and restriction of one level in one kernel (one right-hand side): r = b - M u1 on
// the fine grid and its full-weighting restriction (Sec. 3.4.2) to the next level's right-hand
// side.  r stays in a three-plane ring in shared memory and never goes to memory.  A CTA of
// RWX x RWY threads owns RCX x RCY coarse columns and a chunk of coarse planes; each thread
// computes r on one fine column of the CTA's window (the fine points of those coarse columns
// with a halo of one) while it streams the fine planes in z, u1 of its own column in registers
// and the in-plane neighbours through the read-only path, exactly as k_stencil(resid).  After
// fine plane 2K + off + 1, coarse plane K is restricted by three threads per coarse point, one
// fine plane each (fw_plane), combined by a shuffle (fw_combine) as k_restrict does, so the
// results equal those of the two separate kernels.  DINV: the FP64 level's table of d.
constexpr int RCX = 16, RCY = 8, RWX = 2 * RCX + 1, RWY = 2 * RCY + 1, RNT = RWX * RWY;
template <typename R, bool DINV, typename TB>
__global__ void __launch_bounds__(RNT, 2)
    k_rr(Grid gf, Grid gc, OpCoef<R> c, const R* __restrict__ k2, const cx<R>* __restrict__ dtab,
         const cx<R>* __restrict__ u1, const cx<TB>* __restrict__ b, cx<R>* __restrict__ bco, int kchunk,
         const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ cx<R> sr[3][RWY][RWX];
  const int off = gf.bc == 0 ? 1 : 0;
  const bool som = gf.bc == 1;
  const int N1 = gf.N1, N2 = gf.N2, N3 = gf.N3;
  const int I0 = blockIdx.x * RCX, J0 = blockIdx.y * RCY, K0 = blockIdx.z * kchunk;
  if (K0 >= gc.N3) return;  // the whole CTA
  const int K1 = min(K0 + kchunk, gc.N3);
  const int t = threadIdx.x;
  const int ly = t / RWX, lx = t - ly * RWX;
  const int rx0 = 2 * I0 + off - 1, ry0 = 2 * J0 + off - 1;
  const int x = rx0 + lx, y = ry0 + ly;
  const bool inside = x >= 0 && x < N1 && y >= 0 && y < N2;
  const int zlo = max(2 * K0 + off - 1, 0), zhi = min(2 * (K1 - 1) + off + 1, N3 - 1);
  const size_t S = (size_t)N1 * N2;
  const size_t NP = gf.npts();
  const bool hxm = x > 0, hxp = x < N1 - 1, hym = y > 0, hyp = y < N2 - 1;
  const int nfxy = som ? (!hxm) + (!hxp) + (!hym) + (!hyp) : 0;
  const cx<R> z0 = zero_c<R>();
  size_t p = inside ? gidx(x, y, zlo, N1, N2) : 0;
  cx<R> uc = inside ? ldg(u1 + p) : z0;
  cx<R> um = (inside && zlo > 0) ? ldg(u1 + p - S) : z0;
  // restriction duty: coarse point q = t / 4 of the tile, fine plane part - 1 around its centre
  // (lanes 4q .. 4q + 3 share a warp; the fourth lane only waits)
  constexpr int RQ = 4 * RCX * RCY;
  const int q = t >> 2, part = t & 3;
  const int qI = I0 + (q % RCX), qJ = J0 + (q / RCX);
  const bool rduty = t < RQ && qI < gc.N1 && qJ < gc.N2;
  int K = K0;
  for (int z = zlo; z <= zhi; ++z) {
    cx<R> v = z0;
    if (inside) {
      const bool hzp = z + 1 < N3;
      const cx<R> up = hzp ? ldg(u1 + p + S) : z0;
      int nf = nfxy;
      cx<R> zm, zp;
      if (z > 0) zm = um;
      else if (som) { zm = up; ++nf; }
      else zm = z0;
      if (hzp) zp = up;
      else if (som) { zp = um; ++nf; }
      else zp = z0;
      const cx<R> xm = hxm ? ldg(u1 + p - 1) : (som ? ldg(u1 + p + 1) : z0);
      const cx<R> xp = hxp ? ldg(u1 + p + 1) : (som ? ldg(u1 + p - 1) : z0);
      const cx<R> ym = hym ? ldg(u1 + p - N1) : (som ? ldg(u1 + p + N1) : z0);
      const cx<R> yp = hyp ? ldg(u1 + p + N1) : (som ? ldg(u1 + p - N1) : z0);
      cx<R> d;
      if constexpr (DINV) {
        d = ldg(dtab + NP + p);
      } else {
        const R kk = __ldg(k2 + p);
        d = op_diag(c, kk, nf, nf ? face_k<R>(gf, p, kk) : (R)0);
      }
      const bool real_d = c.real_shift && nf == 0;
      v = op_resid(cvt<R>(ldg(b + p)), d, real_d, uc, c.ih2, xm, xp, ym, yp, zm, zp);
      um = uc;
      uc = up;
      p += S;
    }
    sr[z % 3][ly][lx] = v;
    __syncthreads();
    // coarse plane K needs fine planes 2K + off - 1 .. 2K + off + 1 (those inside the grid)
    bool did = false;
    while (K < K1 && min(2 * K + off + 1, N3 - 1) == z) {
      if (t < RQ) {
        const int zz = 2 * K + off + part - 1;
        cx<R> pv = z0;
        if (rduty && part < 3 && zz >= 0 && zz < N3) {
          const cx<R>(*Rz)[RWX] = sr[zz % 3];
          pv = fw_plane<R>(2 * qI + off, 2 * qJ + off, N1, N2,
                           [&](int xx, int yy) { return Rz[yy - ry0][xx - rx0]; });
        }
        const int lane0 = (threadIdx.x & 31) & ~3;
        const cx<R> pm = mkc<R>(__shfl_sync(0xffffffffu, pv.re, lane0), __shfl_sync(0xffffffffu, pv.im, lane0));
        const cx<R> p0 =
            mkc<R>(__shfl_sync(0xffffffffu, pv.re, lane0 + 1), __shfl_sync(0xffffffffu, pv.im, lane0 + 1));
        const cx<R> pp =
            mkc<R>(__shfl_sync(0xffffffffu, pv.re, lane0 + 2), __shfl_sync(0xffffffffu, pv.im, lane0 + 2));
        if (rduty && part == 0) bco[gidx(qI, qJ, K, gc.N1, gc.N2)] = fw_combine(pm, p0, pp);
      }
      ++K;
      did = true;
    }
    if (did) __syncthreads();  // the next plane overwrites the oldest ring slot
  }
}

// Pre-smoothing from a zero initial guess: one damped-Jacobi sweep gives u1 = (omega/d) b.
// bout (optional): b in working precision R, written beside u1, so that the level's later
// kernels read it without converting b again.
template <typename R, bool DINV, typename TB>
__global__ void __launch_bounds__(TX* TY)
    k_smooth0(Grid g, OpCoef<R> c, const R* __restrict__ k2, const cx<R>* __restrict__ dinv,
              const cx<TB>* __restrict__ b, cx<R>* __restrict__ out, cx<R>* __restrict__ bout, int zchunk,
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
  // FP32: b and k^2 of the next trip are loaded one trip ahead (two planes of loads in flight)
  constexpr bool PF = !DINV && std::is_same<R, float>::value;
  R kpf = PF && k0 < k1 ? __ldg(k2 + p) : (R)0;
  cx<TB> bpf = PF && k0 < k1 ? ldg(b + e) : zero_c<TB>();  // converted when used (see k_stencil)
  for (int k = k0; k < k1; ++k, p += S, e += S * nb) {
    cx<R> w, bv;
    if (DINV) {
      w = ldg(dinv + p);
      bv = cvt<R>(ldg(b + e));
    } else {
      const int nf = nfxy + (som ? (k == 0) + (k == g.N3 - 1) : 0);
      R kk;
      if constexpr (PF) {
        kk = kpf;
        bv = cvt<R>(bpf);
        if (k + 1 < k1) {
          kpf = __ldg(k2 + p + S);
          bpf = ldg(b + e + S * nb);
        }
      } else {
        kk = __ldg(k2 + p);
        bv = cvt<R>(ldg(b + e));
      }
      w = omega_over(op_diag(c, kk, nf, nf ? face_k<R>(g, p, kk) : (R)0), c.omega);
    }
    out[e] = cmul(w, bv);
    if (bout) bout[e] = bv;
  }
}

// The coefficient table of an FP64 level (computed once at set-up): omega / diag(M) at every
// node in out[0, npts), diag(M) itself in out[npts, 2 npts).
__global__ void k_dinv(Grid g, OpCoef<double> c, const double* __restrict__ k2, z128* __restrict__ out) {
  const size_t n = g.npts();
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % g.N1);
    const int j = (int)((p / g.N1) % g.N2);
    const int k = (int)(p / ((size_t)g.N1 * g.N2));
    const int nf = g.bc == 1 ? (i == 0) + (i == g.N1 - 1) + (j == 0) + (j == g.N2 - 1) + (k == 0) + (k == g.N3 - 1) : 0;
    const z128 d = op_diag(c, k2[p], nf, sqrt(k2[p]));
    // omega / d as omega conj(d) / |d|^2 in FP64 (set-up only), then d itself
    const double m2 = d.re * d.re + d.im * d.im;
    out[p] = mkc<double>(c.omega * d.re / m2, -c.omega * d.im / m2);
    out[n + p] = d;
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
    cx<R> p[3];
    for (int dz = -1; dz <= 1; ++dz) {
      const int z = fk + dz;
      p[dz + 1] = zero_c<R>();
      if (z < 0 || z >= gf.N3) continue;
      p[dz + 1] = fw_plane<R>(fi, fj, gf.N1, gf.N2,
                              [&](int x, int y) { return ldg(r + gidx(x, y, z, gf.N1, gf.N2) * nb + q); });
    }
    out[gidx(I, J, K, gc.N1, gc.N2) * nb + q] = fw_combine(p[0], p[1], p[2]);
  }
}

// Full weighting for one right-hand side with the x-neighbourhood shared along a warp: lane l
// owns coarse x index X = X0 + l, loads the fine values at 2X + off and 2X + off + 1 of each fine
// line it needs and takes the one at 2X + off - 1 from the lane before (lane 0 loads it).  A
// thread streams the coarse planes of its chunk and carries the in-plane sum of the shared fine
// plane 2Z + off + 1 into the next coarse plane, so each fine plane is filtered once per coarse
// column.  Same sums in the same order as fw_plane / fw_combine, so the results equal
// k_restrict's.
constexpr int RTY = 8;
template <typename R>
__global__ void __launch_bounds__(TX* RTY)
    k_restrict2(Grid gf, Grid gc, const cx<R>* __restrict__ r, cx<R>* __restrict__ out, int zchunk,
                const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int off = gf.bc == 0 ? 1 : 0;
  const int lane = threadIdx.x;
  const int X = blockIdx.x * TX + lane, Y = blockIdx.y * blockDim.y + threadIdx.y;
  const bool own = X < gc.N1 && Y < gc.N2;
  const int fi = 2 * X + off, fj = 2 * Y + off;
  const int N1 = gf.N1, N2 = gf.N2, N3 = gf.N3;
  const size_t S = (size_t)N1 * N2;
  const cx<R> z0 = zero_c<R>();
  // the lane's three fine rows fj - 1 .. fj + 1 at x = fi: in-plane offsets and which of the
  // loads (x = fi, fi + 1, and fi - 1 for lane 0) fall inside the grid, fixed for the whole
  // z-stream; lanes without a coarse point load nothing (their values are only ever passed to
  // lanes that have none either)
  const bool cok = own && fi < N1, pok = own && fi + 1 < N1, mok = own && fi >= 1;
  bool rok[3];
  size_t rb[3];
  for (int d = 0; d < 3; ++d) {
    const int y = fj + d - 1;
    rok[d] = y >= 0 && y < N2;
    rb[d] = rok[d] ? (size_t)y * N1 + fi : 0;
  }
  // the in-plane sum p of fine plane z for this lane's coarse column (0 outside the grid)
  auto plane = [&](int z) {
    const bool zok = z >= 0 && z < N3;
    const cx<R>* P = r + (zok ? (size_t)z * S : 0);
    cx<R> fx[3];
    for (int d = 0; d < 3; ++d) {
      const bool ok = zok && rok[d];
      const cx<R> c = ok && cok ? ldg(P + rb[d]) : z0;
      const cx<R> pnext = ok && pok ? ldg(P + rb[d] + 1) : z0;
      cx<R> m = mkc<R>(__shfl_up_sync(0xffffffffu, pnext.re, 1), __shfl_up_sync(0xffffffffu, pnext.im, 1));
      if (lane == 0) m = ok && mok ? ldg(P + rb[d] - 1) : z0;
      fx[d] = fw3(m, c, pnext);
    }
    return fw3(fx[0], fx[1], fx[2]);
  };
  const int K0 = blockIdx.z * zchunk, K1 = min(K0 + zchunk, gc.N3);
  if (K0 >= K1) return;  // the whole CTA
  cx<R> pm = plane(2 * K0 + off - 1);
  for (int K = K0; K < K1; ++K) {
    const int fk = 2 * K + off;
    const cx<R> p0 = plane(fk), pp = plane(fk + 1);
    if (own) out[gidx(X, Y, K, gc.N1, gc.N2)] = fw_combine(pm, p0, pp);
    pm = pp;
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
  for (int k = k0; k < k1; ++k) {
    const size_t p = gidx(i, j, k, gf.N1, gf.N2) * nb + q;
    out[p] = tl_value<R>(i + off, j + off, k + off, off, gc, ldg(u1 + p),
                         [&](int X, int Y, int Z) { return ldg(e + gidx(X, Y, Z, gc.N1, gc.N2) * nb + q); });
  }
}

// Trilinear interpolation added to u1 for one right-hand side with two fine points per lane
// along x: lane l owns coarse x node c = c0 + l and the fine nodes 2c and 2c + 1; the odd one
// needs tz of node c + 1, taken from the next lane by a shuffle (the last lane of a warp only
// supplies it, so warps step 31 coarse nodes).  A thread streams the coarse z nodes of its
// chunk: each coarse plane's y-sum ty is formed once and serves the fine planes 2Z - 1 (with the
// previous plane's) and 2Z.  Coarse loads are coalesced and no lane branches on parity.  Same
// sums in the same order as tl_value, so the results equal k_prolong_add's.
constexpr int PTY = 8;
template <typename R>
__global__ void __launch_bounds__(TX* PTY)
    k_prolong2(Grid gf, Grid gc, const cx<R>* __restrict__ u1, const cx<R>* __restrict__ e,
               cx<R>* __restrict__ out, int zchunk, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int off = gf.bc == 0 ? 1 : 0;
  const int lane = threadIdx.x;
  const int cn = blockIdx.x * (TX - 1) + lane;         // coarse x node
  const int j = blockIdx.y * blockDim.y + threadIdx.y;  // fine y index
  const bool rowok = j < gf.N2;
  const int X = cn - off;
  const bool xok = X >= 0 && X < gc.N1;
  const int fj = j + off, y0 = (fj >> 1) - off, y1 = ((fj + 1) >> 1) - off;
  const int ny = y0 == y1 ? 1 : 2;
  const bool y0ok = rowok && xok && y0 >= 0 && y0 < gc.N2, y1ok = rowok && xok && y1 >= 0 && y1 < gc.N2;
  const int ie = 2 * cn - off, io = ie + 1;  // fine x indices of nodes 2c, 2c + 1
  const bool eok = rowok && ie >= 0 && ie < gf.N1;
  const bool ook = rowok && lane < TX - 1 && io >= 0 && io < gf.N1;
  const cx<R> z0 = zero_c<R>();
  auto ty = [&](int Zn) {  // y-sum at coarse z node Zn (0 outside the grid)
    const int Z = Zn - off;
    const bool zok = Z >= 0 && Z < gc.N3;
    cx<R> v = (y0ok && zok) ? ldg(e + gidx(X, y0, Z, gc.N1, gc.N2)) : z0;
    if (ny == 2) v = cadd(v, (y1ok && zok) ? ldg(e + gidx(X, y1, Z, gc.N1, gc.N2)) : z0);
    return v;
  };
  // one fine plane (node fz, fine index k = fz - off) from this lane's tz
  auto emit = [&](int fz, cx<R> tz, int nz) {
    const cx<R> tr = mkc<R>(__shfl_down_sync(0xffffffffu, tz.re, 1), __shfl_down_sync(0xffffffffu, tz.im, 1));
    const int k = fz - off;
    if (k < 0 || k >= gf.N3) return;
    if (eok) {
      const size_t p = gidx(ie, j, k, gf.N1, gf.N2);
      const cx<R> b = ldg(u1 + p);
      const R sc = tl_scale<R>(ny * nz);
      out[p] = mkc<R>(fma(tz.re, sc, b.re), fma(tz.im, sc, b.im));
    }
    if (ook) {
      const size_t p = gidx(io, j, k, gf.N1, gf.N2);
      const cx<R> b = ldg(u1 + p);
      const cx<R> t = cadd(tz, tr);
      const R sc = tl_scale<R>(2 * ny * nz);
      out[p] = mkc<R>(fma(t.re, sc, b.re), fma(t.im, sc, b.im));
    }
  };
  const int nzn = gc.N3 + 2 * off;  // coarse z nodes, the Dirichlet boundary nodes included
  const int zn0 = blockIdx.z * zchunk, zn1 = min(zn0 + zchunk, nzn);
  cx<R> prev = zn0 > 0 ? ty(zn0 - 1) : z0;
  for (int Zn = zn0; Zn < zn1; ++Zn) {
    const cx<R> cur = ty(Zn);
    if (Zn > 0) emit(2 * Zn - 1, cadd(prev, cur), 2);
    emit(2 * Zn, cur, 1);
    prev = cur;
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

// The kernels' FP32 -> FP64 conversion (f32_to_f64) applied elementwise, for checks against
// the hardware conversion.
__global__ void k_convert_check(const float* __restrict__ in32, double* __restrict__ out64, size_t n) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    out64[p] = f32_to_f64(in32[p]);
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

// ---- coarsest-grid inverse (set-up only): Gauss-Jordan elimination with partial pivoting ----
// A (n x n, row-major) is reduced to the identity while X, started as the identity, becomes
// A^{-1}.  Column col takes three launches: the pivot search (the largest |A[r][col]|, r >= col,
// the smallest r on ties) which also saves the column's multipliers as they stand after the row
// swap; the swap and scaling of the pivot row; the elimination of every other row with a
// nonzero multiplier.
__global__ void k_gj_identity(z128* __restrict__ X, int n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)n * n; t += (size_t)gridDim.x * blockDim.x)
    X[t] = mkc<double>((t / n) == (t % n) ? 1.0 : 0.0, 0.0);
}

constexpr int GJ_THREADS = 1024;
__global__ void __launch_bounds__(GJ_THREADS)
    k_gj_pivot(const z128* __restrict__ A, int n, int col, z128* __restrict__ fcol, int* __restrict__ piv,
               z128* __restrict__ pinv, int* __restrict__ singular) {
  __shared__ double sbest[GJ_THREADS / 32];
  __shared__ int sidx[GJ_THREADS / 32];
  __shared__ int spiv;
  double best = -1.0;
  int idx = n;
  for (int r = col + threadIdx.x; r < n; r += GJ_THREADS) {
    const z128 a = A[(size_t)r * n + col];
    const double m = a.re * a.re + a.im * a.im;
    if (m > best) { best = m; idx = r; }  // rows visited in increasing order: ties keep the first
  }
  for (int o = 16; o; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ob > best || (ob == best && oi < idx)) { best = ob; idx = oi; }
  }
  if ((threadIdx.x & 31) == 0) {
    sbest[threadIdx.x >> 5] = best;
    sidx[threadIdx.x >> 5] = idx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    best = sbest[0];
    idx = sidx[0];
    for (int w = 1; w < GJ_THREADS / 32; ++w)
      if (sbest[w] > best || (sbest[w] == best && sidx[w] < idx)) { best = sbest[w]; idx = sidx[w]; }
    if (!(best > 0.0)) {  // singular (or NaN): finish harmlessly, the host reports it
      *singular = 1;
      idx = col;
      *pinv = mkc<double>(0.0, 0.0);
    } else {
      const z128 p = A[(size_t)idx * n + col];
      const double inv = 1.0 / (p.re * p.re + p.im * p.im);
      *pinv = mkc<double>(p.re * inv, -p.im * inv);
    }
    *piv = idx;
    spiv = idx;
  }
  __syncthreads();
  const int pv = spiv;
  for (int r = threadIdx.x; r < n; r += GJ_THREADS) {
    const int src = r == col ? pv : (r == pv ? col : r);
    fcol[r] = r == col ? mkc<double>(0.0, 0.0) : A[(size_t)src * n + col];
  }
}

__global__ void k_gj_swap_scale(z128* __restrict__ A, z128* __restrict__ X, int n, int col, const int* __restrict__ piv,
                                const z128* __restrict__ pinv) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 2 * n || q < col) return;  // columns of A left of col are finished
  z128* M = q < n ? A : X;
  const int c = q < n ? q : q - n;
  const int pv = *piv;
  const z128 pi = *pinv;
  const z128 a = M[(size_t)col * n + c], b = M[(size_t)pv * n + c];
  M[(size_t)pv * n + c] = a;
  M[(size_t)col * n + c] = mkc<double>(b.re * pi.re - b.im * pi.im, b.re * pi.im + b.im * pi.re);
}

__global__ void k_gj_eliminate(z128* __restrict__ A, z128* __restrict__ X, int n, int col,
                               const z128* __restrict__ fcol) {
  const int r = blockIdx.y;
  const z128 f = fcol[r];
  if (f.re == 0.0 && f.im == 0.0) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 2 * n || q < col) return;  // columns of A left of col are finished
  z128* M = q < n ? A : X;
  const int c = q < n ? q : q - n;
  const z128 p = M[(size_t)col * n + c];
  if (p.re == 0.0 && p.im == 0.0) return;
  z128 v = M[(size_t)r * n + c];
  v.re = fma(-f.re, p.re, v.re);
  v.re = fma(f.im, p.im, v.re);
  v.im = fma(-f.re, p.im, v.im);
  v.im = fma(-f.im, p.re, v.im);
  M[(size_t)r * n + c] = v;
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
      cx<R> pz[3];
      for (int dz = -1; dz <= 1; ++dz) {
        const int z = fk + dz;
        pz[dz + 1] = mkc<R>((R)0, (R)0);
        if (z < 0 || z >= g.N3) continue;
        pz[dz + 1] = fw_plane<R>(fi, fj, g.N1, g.N2, [&](int x, int y) { return r[(z * g.N2 + y) * g.N1 + x]; });
      }
      sm[C.off_b + Q] = fw_combine(pz[0], pz[1], pz[2]);
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
      sm[F.off_t + q] = tl_value<R>(i + off, j + off, k + off, off, gc, sm[F.off_u + q],
                                    [&](int X, int Y, int Z) { return e[(Z * gc.N2 + Y) * gc.N1 + X]; });
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
  if (s_im == 0.0 && std::is_same<R, double>::value)  // the operator A: real diagonal off the faces
    k_stencil<R, 0, false, TU, TU, TO, false, true><<<gr, blk, 0, st>>>(g, coef_for<R>(g.h, s_re, s_im, 0.0), k2,
                                                                        nullptr, u, nullptr, v, zc, active);
  else
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
  if (s_im == 0.0)
    k_stencil<double, 0, false, TU, TU, double, true, true><<<gr, blk, 0, st>>>(
        g, coef_for<double>(g.h, s_re, s_im, 0.0), k2, nullptr, u, nullptr, reinterpret_cast<z128*>(v), zc, active);
  else
    k_stencil<double, 0, false, TU, TU, double, true><<<gr, blk, 0, st>>>(
        g, coef_for<double>(g.h, s_re, s_im, 0.0), k2, nullptr, u, nullptr, reinterpret_cast<z128*>(v), zc, active);
}
template void launch_apply_split<double>(const Grid&, double, double, const double*, const z128*, zdf*, cudaStream_t,
                                         const int*);
template void launch_apply_split<float>(const Grid&, double, double, const double*, const z64*, zdf*, cudaStream_t,
                                        const int*);

template <typename R, typename TU, typename TB, typename TO>
void launch_resid(const Grid& g, double s_re, double s_im, const R* k2, const cx<TU>* u, const cx<TB>* b,
                  cx<TO>* out, cudaStream_t st, const int* active, const cx<R>* dtab) {
  int zc;
  if (dtab) {
    dim3 blk, gr = grid_for<R>(g, TILE_STENCIL, zc, blk);
    k_stencil<R, 1, true, TU, TB, TO><<<gr, blk, 0, st>>>(g, coef_for<R>(g.h, s_re, s_im, 0.0), k2, dtab, u, b, out,
                                                           zc, active);
    return;
  }
  if constexpr (std::is_same<R, float>::value) {
    if (g.nb == 1 && g.tiled) {
      const dim3 gr = grid_tiled(g, zc);
      k_stencil32_tiled<1, TU, TB, TO><<<gr, dim3(TX, TYT), 0, st>>>(g, coef_for<R>(g.h, s_re, s_im, 0.0), k2, u, b,
                                                                    out, zc, active);
      return;
    }
  }
  dim3 blk, gr = grid_for<R>(g, TILE_STENCIL, zc, blk);
  if (s_im == 0.0 && std::is_same<R, double>::value)  // the operator A: real diagonal off the faces
    k_stencil<R, 1, false, TU, TB, TO, false, true><<<gr, blk, 0, st>>>(g, coef_for<R>(g.h, s_re, s_im, 0.0), k2,
                                                                        nullptr, u, b, out, zc, active);
  else
    k_stencil<R, 1, false, TU, TB, TO><<<gr, blk, 0, st>>>(g, coef_for<R>(g.h, s_re, s_im, 0.0), k2, nullptr, u, b,
                                                           out, zc, active);
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
                    const cx<TB>* b, cx<R>* out, cudaStream_t st, const int* active, cx<R>* bout) {
  int zc;
  dim3 blk, gr = grid_for<R>(g, TILE_SMOOTH0, zc, blk);
  OpCoef<R> c = coef_for<R>(g.h, s_re, s_im, omega);
  if (dinv)
    k_smooth0<R, true, TB><<<gr, blk, 0, st>>>(g, c, k2, dinv, b, out, bout, zc, active);
  else
    k_smooth0<R, false, TB><<<gr, blk, 0, st>>>(g, c, k2, dinv, b, out, bout, zc, active);
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

template <typename TB>
void launch_down32(const Grid& gf, const Grid& gc, double s_re, double s_im, double omega, const float* k2,
                   const cx<TB>* b, z64* u1, z64* bc, int kchunk, cudaStream_t st, const int* active) {
  const int kc = kchunk > 0 ? kchunk : 4;
  const dim3 gr((gc.N1 + DCX - 1) / DCX, (gc.N2 + DCY - 1) / DCY, (gc.N3 + kc - 1) / kc);
  k_down32<TB><<<gr, DNT, 0, st>>>(gf, gc, coef_for<float>(gf.h, s_re, s_im, omega), k2, b, u1, bc, kc, active);
}
template void launch_down32<float>(const Grid&, const Grid&, double, double, double, const float*, const z64*, z64*,
                                   z64*, int, cudaStream_t, const int*);
template void launch_down32<double>(const Grid&, const Grid&, double, double, double, const float*, const z128*,
                                    z64*, z64*, int, cudaStream_t, const int*);

template <typename R, typename TB, typename TO>
void launch_up(const Grid& gf, const Grid& gc, double s_re, double s_im, double omega, const R* k2, const cx<R>* dinv,
               const cx<R>* u1, const cx<R>* e, const cx<TB>* b, cx<TO>* out, int zchunk, cudaStream_t st,
               const int* active) {
  const int kz = zchunk > 0 ? zchunk : 16;
  const dim3 gr((gf.N1 + TX - 1) / TX, (gf.N2 + UTY - 1) / UTY, (gf.N3 + kz - 1) / kz);
  const OpCoef<R> c = coef_for<R>(gf.h, s_re, s_im, omega);
  if constexpr (std::is_same<R, double>::value) {
    if (dinv) {  // FP64 levels carry the coefficient table
      k_up<R, true, TB, TO><<<gr, dim3(TX, UTY), 0, st>>>(gf, gc, c, k2, dinv, u1, e, b, out, kz, active);
      return;
    }
  }
  k_up<R, false, TB, TO><<<gr, dim3(TX, UTY), 0, st>>>(gf, gc, c, k2, dinv, u1, e, b, out, kz, active);
}
#define UP_INST(R, TB, TO)                                                                                        \
  template void launch_up<R, TB, TO>(const Grid&, const Grid&, double, double, double, const R*, const cx<R>*,   \
                                     const cx<R>*, const cx<R>*, const cx<TB>*, cx<TO>*, int, cudaStream_t,      \
                                     const int*);
UP_INST(float, float, float)
UP_INST(float, double, float)
UP_INST(float, float, double)
UP_INST(float, double, double)
UP_INST(double, double, double)
#undef UP_INST

template <typename R, typename TB>
void launch_rr(const Grid& gf, const Grid& gc, double s_re, double s_im, const R* k2, const cx<R>* dtab,
               const cx<R>* u1, const cx<TB>* b, cx<R>* bc, int kchunk, cudaStream_t st, const int* active) {
  const int kc = kchunk > 0 ? kchunk : 4;
  const dim3 gr((gc.N1 + RCX - 1) / RCX, (gc.N2 + RCY - 1) / RCY, (gc.N3 + kc - 1) / kc);
  const OpCoef<R> c = coef_for<R>(gf.h, s_re, s_im, 0.0);
  if constexpr (std::is_same<R, double>::value) {
    if (dtab) {  // FP64 levels carry the coefficient table
      k_rr<R, true, TB><<<gr, RNT, 0, st>>>(gf, gc, c, k2, dtab, u1, b, bc, kc, active);
      return;
    }
  }
  k_rr<R, false, TB><<<gr, RNT, 0, st>>>(gf, gc, c, k2, dtab, u1, b, bc, kc, active);
}
template void launch_rr<float, float>(const Grid&, const Grid&, double, double, const float*, const z64*, const z64*,
                                      const z64*, z64*, int, cudaStream_t, const int*);
template void launch_rr<float, double>(const Grid&, const Grid&, double, double, const float*, const z64*,
                                       const z64*, const z128*, z64*, int, cudaStream_t, const int*);
template void launch_rr<double, double>(const Grid&, const Grid&, double, double, const double*, const z128*,
                                        const z128*, const z128*, z128*, int, cudaStream_t, const int*);

template <typename R>
void launch_restrict(const Grid& gf, const Grid& gc, const cx<R>* r, cx<R>* out, cudaStream_t st, const int* active) {
  int zc;
  dim3 blk, gr = grid_for<R>(gc, TILE_RESTRICT, zc, blk);
  if (gc.nb == 1)  // lanes along x share the fine neighbourhood; same shape rules as k_restrict
    k_restrict2<R><<<gr, blk, 0, st>>>(gf, gc, r, out, zc, active);
  else
    k_restrict<R><<<gr, blk, 0, st>>>(gf, gc, r, out, zc, active);
}

template <typename R>
void launch_prolong_add(const Grid& gf, const Grid& gc, const cx<R>* u1, const cx<R>* e, cx<R>* out, cudaStream_t st,
                        const int* active) {
  int zc;
  if (gf.nb == 1) {  // two fine points per lane; the tuned shape sets rows per CTA and the z-chunk
    const int slot = tile_slot<R>(TILE_PROLONG);
    const int ty = gf.tile_ty[slot] > 0 ? gf.tile_ty[slot] : PTY;
    const int target = gf.tile_ctas[slot] > 0 ? gf.tile_ctas[slot] : 152 * 8;
    const int off = gf.bc == 0 ? 1 : 0;
    const int bx = (gc.N1 + 2 * off + TX - 2) / (TX - 1), by = (gf.N2 + ty - 1) / ty, nzn = gc.N3 + 2 * off;
    int zsplit = target / (bx * by);
    if (zsplit < 1) zsplit = 1;
    if (zsplit > nzn) zsplit = nzn;
    zc = (nzn + zsplit - 1) / zsplit;
    k_prolong2<R><<<dim3(bx, by, (nzn + zc - 1) / zc), dim3(TX, ty), 0, st>>>(gf, gc, u1, e, out, zc, active);
    return;
  }
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

void launch_gj_invert(z128* A, z128* X, int n, z128* fcol, int* piv, z128* pinv, int* singular, cudaStream_t st) {
  k_gj_identity<<<1216, 256, 0, st>>>(X, n);
  const int bx = (2 * n + 255) / 256;
  for (int col = 0; col < n; ++col) {
    k_gj_pivot<<<1, GJ_THREADS, 0, st>>>(A, n, col, fcol, piv, pinv, singular);
    k_gj_swap_scale<<<bx, 256, 0, st>>>(A, X, n, col, piv, pinv);
    k_gj_eliminate<<<dim3(bx, n), 256, 0, st>>>(A, X, n, col, fcol);
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

void launch_convert_check(const float* in32, double* out64, size_t n, cudaStream_t st) {
  k_convert_check<<<1216, 256, 0, st>>>(in32, out64, n);
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
template void launch_resid<double, double, double, double>(const Grid&, double, double, const double*, const z128*, const z128*, z128*, cudaStream_t, const int*, const z128*);
template void launch_resid<double, double, double, float>(const Grid&, double, double, const double*, const z128*, const z128*, z64*, cudaStream_t, const int*, const z128*);
template void launch_resid<float, float, float, float>(const Grid&, double, double, const float*, const z64*, const z64*, z64*, cudaStream_t, const int*, const z64*);
template void launch_resid<float, float, double, float>(const Grid&, double, double, const float*, const z64*, const z128*, z64*, cudaStream_t, const int*, const z64*);
template void launch_jacobi<double, double, double>(const Grid&, double, double, double, const double*, const z128*, const z128*, const z128*, z128*, cudaStream_t, const int*);
template void launch_jacobi<float, float, float>(const Grid&, double, double, double, const float*, const z64*, const z64*, const z64*, z64*, cudaStream_t, const int*);
template void launch_jacobi<float, double, float>(const Grid&, double, double, double, const float*, const z64*, const z64*, const z128*, z64*, cudaStream_t, const int*);
template void launch_jacobi<float, double, double>(const Grid&, double, double, double, const float*, const z64*, const z64*, const z128*, z128*, cudaStream_t, const int*);
template void launch_jacobi<float, float, double>(const Grid&, double, double, double, const float*, const z64*, const z64*, const z64*, z128*, cudaStream_t, const int*);
template void launch_jacobi<double, double, float>(const Grid&, double, double, double, const double*, const z128*, const z128*, const z128*, z64*, cudaStream_t, const int*);
template void launch_smooth0<double, double>(const Grid&, double, double, double, const double*, const z128*, const z128*, z128*, cudaStream_t, const int*, z128*);
template void launch_smooth0<float, float>(const Grid&, double, double, double, const float*, const z64*, const z64*, z64*, cudaStream_t, const int*, z64*);
template void launch_smooth0<float, double>(const Grid&, double, double, double, const float*, const z64*, const z128*, z64*, cudaStream_t, const int*, z64*);
template void launch_coarse<double, double>(int, const z128*, const z128*, z128*, cudaStream_t, const int*, int);
template void launch_coarse<float, float>(int, const z128*, const z64*, z64*, cudaStream_t, const int*, int);
template void launch_coarse<double, float>(int, const z128*, const z128*, z64*, cudaStream_t, const int*, int);
template void launch_coarse<float, double>(int, const z128*, const z64*, z128*, cudaStream_t, const int*, int);

}  // namespace helm
