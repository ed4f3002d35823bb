// coarse_gmres.cu -- the paper's own coarsest-grid solve (Sec. 5): the error equation
// M_c e = b on the coarsest grid is solved by full (unrestarted) GMRES from e = 0 until the
// relative residual reaches a tolerance (1e-11 in the paper), instead of by the precomputed
// dense inverse the library uses by default.
//
// The coarsest grid holds at most a few thousand unknowns, too few to fill the GPU and too many
// for one SM to orthogonalise quickly, so one thread-block cluster (16 CTAs where the GPU can
// place a cluster that large, else the portable 8; distributed shared memory, hardware cluster
// barriers) runs the whole iteration in one launch: each CTA owns a contiguous slice of the
// grid (one node per thread), applies M on it, and contributes partial inner products that
// every CTA then sums from the others' shared memory in rank order, so all CTAs hold the same
// Hessenberg column, Givens rotations and stopping decision and take every barrier together.
// Classical Gram-Schmidt with the library's selective second pass (the reorth_keep test).  The
// basis lives in global memory (L2-resident); values written during the launch by other CTAs
// are read through L2 only.
#include "internal.cuh"

#include <cooperative_groups.h>

namespace helm {

namespace {

namespace cgr = cooperative_groups;

constexpr int CG_NT = 512;
constexpr int CG_NW = CG_NT / 32;
constexpr int CG_MAXB = CG_MAX + 1;

__device__ __forceinline__ z128 ld_l2(const z128* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return mkc<double>(v.x, v.y);
}
__device__ __forceinline__ void st_l2(z128* p, z128 v) {
  __stcg(reinterpret_cast<double2*>(p), make_double2(v.re, v.im));
}
__device__ __forceinline__ z128 zdiv(z128 a, z128 b) {
  const double d = b.re * b.re + b.im * b.im;
  return mkc<double>((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}

// (M v)_p on the coarsest grid: the 7-point operator with the level's k^2, Sommerfeld faces
// taking the opposite neighbour and adding the face term to the diagonal, Dirichlet faces a
// zero (the substitution of k_stencil).
__device__ z128 coarse_apply(const Grid& g, const OpCoef<double>& c, const double* __restrict__ k2,
                             const z128* v, int p) {
  const int N1 = g.N1, N2 = g.N2, N3 = g.N3, S = N1 * N2;
  const int i = p % N1, j = (p / N1) % N2, k = p / S;
  const bool som = g.bc == 1;
  const bool hxm = i > 0, hxp = i < N1 - 1, hym = j > 0, hyp = j < N2 - 1, hzm = k > 0, hzp = k < N3 - 1;
  const int nf = som ? (!hxm) + (!hxp) + (!hym) + (!hyp) + (!hzm) + (!hzp) : 0;
  const z128 z0 = mkc<double>(0.0, 0.0);
  const z128 xm = hxm ? ld_l2(v + p - 1) : (som ? ld_l2(v + p + 1) : z0);
  const z128 xp = hxp ? ld_l2(v + p + 1) : (som ? ld_l2(v + p - 1) : z0);
  const z128 ym = hym ? ld_l2(v + p - N1) : (som ? ld_l2(v + p + N1) : z0);
  const z128 yp = hyp ? ld_l2(v + p + N1) : (som ? ld_l2(v + p - N1) : z0);
  const z128 zm = hzm ? ld_l2(v + p - S) : (som ? ld_l2(v + p + S) : z0);
  const z128 zp = hzp ? ld_l2(v + p + S) : (som ? ld_l2(v + p - S) : z0);
  const double kk = k2[p];
  const z128 d = op_diag(c, kk, nf, nf ? face_k<double>(g, (size_t)p, kk) : 0.0);
  return op_apply(d, c.real_shift && nf == 0, ld_l2(v + p), c.ih2, xm, xp, ym, yp, zm, zp);
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(CG_NT)
    k_coarse_gmres(Grid g, OpCoef<double> c, const double* __restrict__ k2, const cx<TI>* __restrict__ b,
                   cx<TO>* __restrict__ e, z128* __restrict__ V, z128* __restrict__ H, int maxit, double tol,
                   double keep, int* __restrict__ info, const int* __restrict__ active) {
  if (active && *active == 0) return;  // read by every thread of every CTA: all return together
  cgr::cluster_group cl = cgr::this_cluster();
  const int rank = (int)cl.block_rank();
  const int cs = (int)cl.num_blocks();  // the grid is one cluster
  const int n = (int)g.npts();
  const int chunk = (n + cs - 1) / cs;  // <= CG_NT (n <= CG_CS * CG_NT)
  const int p0 = min(rank * chunk, n), p1 = min(p0 + chunk, n), len = p1 - p0;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int p = p0 + t;
  const bool own = t < len;
  __shared__ z128 part[2][CG_MAXB];  // this CTA's partial sums, read by every CTA of the cluster
  __shared__ z128 sw[CG_NT];         // w on this CTA's nodes
  __shared__ z128 hcol[CG_MAXB];     // the Hessenberg column being built (both passes)
  __shared__ z128 hp[CG_MAXB];       // this pass's coefficients
  __shared__ double scs[CG_MAX];
  __shared__ z128 ssn[CG_MAX];
  __shared__ z128 sg[CG_MAXB];
  __shared__ z128 sy[CG_MAX];
  __shared__ double sred[CG_NW];
  __shared__ double sval;
  __shared__ int sstop, spass2;

  // sum over the cluster of one real value per thread: block sum into part[buf][0], barrier,
  // then the CTAs' sums added in rank order (the same result in every CTA)
  auto cluster_sum = [&](double x, int buf) -> double {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sred[warp] = x;
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
      for (int w = 0; w < CG_NW; ++w) s += sred[w];
      part[buf][0] = mkc<double>(s, 0.0);
    }
    cl.sync();
    if (t == 0) {
      double s = 0.0;
      for (int r = 0; r < cs; ++r) s += cl.map_shared_rank(&part[buf][0], r)->re;
      sval = s;
    }
    __syncthreads();
    return sval;
  };
  // hp[i] = sum over the grid of conj(V_i) w, i <= j, and with `wn` hp[j + 1] = |w|^2: warp w
  // takes i = w, w + CG_NW, ...
  auto dots = [&](int j, int buf, int wn) {
    for (int i = warp; i <= j + wn; i += CG_NW) {
      double re = 0.0, im = 0.0;
      const z128* Vi = V + (size_t)i * n + p0;
      if (i > j) {
        for (int q = lane; q < len; q += 32) re = fma(sw[q].re, sw[q].re, fma(sw[q].im, sw[q].im, re));
      } else {
#pragma unroll 4
        for (int q = lane; q < len; q += 32) cdot_acc(ld_l2(Vi + q), sw[q], re, im);
      }
      for (int o = 16; o; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane == 0) part[buf][i] = mkc<double>(re, im);
    }
    cl.sync();
    for (int i = t; i <= j + wn; i += CG_NT) {
      double re = 0.0, im = 0.0;
      for (int r = 0; r < cs; ++r) {
        const z128 v = cl.map_shared_rank(&part[buf][0], r)[i];
        re += v.re;
        im += v.im;
      }
      hp[i] = mkc<double>(re, im);
    }
    __syncthreads();
  };

  // beta = |b|, v_0 = b / beta
  z128 bv = mkc<double>(0.0, 0.0);
  if (own) bv = cvt<double>(b[p]);
  const double beta = sqrt(cluster_sum(own ? bv.re * bv.re + bv.im * bv.im : 0.0, 0));
  if (beta == 0.0 || !isfinite(beta)) {
    if (own) e[p] = cvt<TO>(mkc<double>(0.0, 0.0));
    if (rank == 0 && t == 0 && info) {
      info[0] = 0;
      info[1] = beta == 0.0;
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
    return;
  }
  if (own) st_l2(V + p, mkc<double>(bv.re / beta, bv.im / beta));
  if (t == 0) sg[0] = mkc<double>(beta, 0.0);
  int k = 0, conv = 0;
  for (int j = 0; j < maxit; ++j) {
    cl.sync();  // v_j complete in every CTA's slice; the reads of part[0] are done
    if (own) sw[t] = coarse_apply(g, c, k2, V + (size_t)j * n, p);
    __syncthreads();
    // classical Gram-Schmidt; the second pass only when the first kept less than `keep` of
    // |w|^2 (the Daniel-Gragg-Kaufman-Stewart test, decided alike in every CTA)
    for (int pass = 0; pass < 2; ++pass) {
      dots(j, pass, pass == 0);
      if (pass == 0 && t == 0) {
        double h2 = 0.0;
        for (int i = 0; i <= j; ++i) h2 += hp[i].re * hp[i].re + hp[i].im * hp[i].im;
        const double w2 = hp[j + 1].re;
        spass2 = !(w2 - h2 >= keep * w2);
      }
      for (int i = t; i <= j; i += CG_NT) hcol[i] = pass == 0 ? hp[i] : cadd(hcol[i], hp[i]);
      if (own) {
        z128 w = sw[t];
#pragma unroll 8
        for (int i = 0; i <= j; ++i) w = csub(w, cmul(hp[i], ld_l2(V + (size_t)i * n + p)));
        sw[t] = w;
      }
      __syncthreads();
      if (!spass2) break;
    }
    const z128 wv = own ? sw[t] : mkc<double>(0.0, 0.0);
    const double hn = sqrt(cluster_sum(wv.re * wv.re + wv.im * wv.im, 0));
    if (own && hn > 0.0) st_l2(V + (size_t)(j + 1) * n + p, mkc<double>(wv.re / hn, wv.im / hn));
    if (t == 0) {
      // previous rotations on the new column, then the rotation that zeroes h_{j+1,j}
      hcol[j + 1] = mkc<double>(hn, 0.0);
      for (int i = 0; i < j; ++i) {
        const z128 a = hcol[i], bb = hcol[i + 1];
        const double cs = scs[i];
        const z128 sn = ssn[i];
        const z128 sb = cmul(sn, bb);
        const z128 ta = cmul(mkc<double>(-sn.re, sn.im), a);  // -conj(sn) a
        hcol[i] = mkc<double>(cs * a.re + sb.re, cs * a.im + sb.im);
        hcol[i + 1] = mkc<double>(ta.re + cs * bb.re, ta.im + cs * bb.im);
      }
      const z128 a = hcol[j], bb = hcol[j + 1];
      const double na = hypot(a.re, a.im), nbb = hypot(bb.re, bb.im), tt = hypot(na, nbb);
      double cs;
      z128 sn;
      if (na == 0.0) {
        cs = 0.0;
        sn = mkc<double>(1.0, 0.0);
        hcol[j] = bb;
      } else {
        const z128 ph = mkc<double>(a.re / na, a.im / na);
        cs = na / tt;
        sn = cmul(ph, mkc<double>(bb.re / tt, -bb.im / tt));
        hcol[j] = mkc<double>(ph.re * tt, ph.im * tt);
      }
      scs[j] = cs;
      ssn[j] = sn;
      const z128 gj = sg[j];
      sg[j + 1] = cmul(mkc<double>(-sn.re, sn.im), gj);
      sg[j] = mkc<double>(cs * gj.re, cs * gj.im);
      if (rank == 0)
        for (int i = 0; i <= j; ++i) st_l2(H + (size_t)j * CG_MAXB + i, hcol[i]);
      const double est = hypot(sg[j + 1].re, sg[j + 1].im) / beta;
      sstop = (est <= tol) ? 1 : (!(hn > 0.0) || !isfinite(est)) ? 2 : 0;
    }
    __syncthreads();
    k = j + 1;
    if (sstop) {
      conv = sstop == 1;
      break;
    }
  }
  cl.sync();  // the columns written by rank 0 are visible; no shared memory is read after this
  if (t == 0) {
    for (int i = k - 1; i >= 0; --i) {
      z128 acc = sg[i];
      for (int q = i + 1; q < k; ++q) acc = csub(acc, cmul(ld_l2(H + (size_t)q * CG_MAXB + i), sy[q]));
      sy[i] = zdiv(acc, ld_l2(H + (size_t)i * CG_MAXB + i));
    }
  }
  __syncthreads();
  if (own) {
    z128 x = mkc<double>(0.0, 0.0);
#pragma unroll 8
    for (int i = 0; i < k; ++i) x = cfma(sy[i], ld_l2(V + (size_t)i * n + p), x);
    e[p] = cvt<TO>(x);
  }
  if (rank == 0 && t == 0 && info) {
    info[0] = k;
    info[1] = conv;
  }
}

}  // namespace

template <typename TI, typename TO>
void launch_coarse_gmres(const Grid& g, double s_re, double s_im, const double* k2, const cx<TI>* b, cx<TO>* e,
                         z128* V, z128* H, double tol, double keep, int* info, cudaStream_t st, const int* active) {
  const int n = (int)g.npts();
  const int maxit = n < CG_MAX ? n : CG_MAX;
  auto kern = k_coarse_gmres<TI, TO>;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(CG_NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // the cluster size, chosen once: 16 CTAs (a non-portable size) when the GPU can place such a
  // cluster, else the portable 8 (the first call comes from helm_create's set-up or a first
  // cycle, before any graph capture)
  static const int cs = [&] {
    const bool clean = cudaPeekAtLastError() == cudaSuccess;
    int ok = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
      cudaLaunchConfig_t q = cfg;
      cudaLaunchAttribute qa = at[0];
      qa.val.clusterDim.x = 16;
      q.gridDim = dim3(16);
      q.attrs = &qa;
      if (cudaOccupancyMaxActiveClusters(&ok, kern, &q) != cudaSuccess) ok = 0;
    }
    if (clean) cudaGetLastError();  // a refused query leaves no error behind (an earlier one stays)
    return ok >= 1 ? 16 : CG_CS;
  }();
  at[0].val.clusterDim.x = cs;
  cfg.gridDim = dim3(cs);
  cudaLaunchKernelEx(&cfg, kern, g, coef_for<double>(g.h, s_re, s_im, 0.0), k2, b, e, V, H, maxit, tol, keep, info,
                     active);
}
template void launch_coarse_gmres<double, double>(const Grid&, double, double, const double*, const z128*, z128*,
                                                  z128*, z128*, double, double, int*, cudaStream_t, const int*);
template void launch_coarse_gmres<float, float>(const Grid&, double, double, const double*, const z64*, z64*, z128*,
                                                z128*, double, double, int*, cudaStream_t, const int*);
template void launch_coarse_gmres<double, float>(const Grid&, double, double, const double*, const z128*, z64*,
                                                 z128*, z128*, double, double, int*, cudaStream_t, const int*);
template void launch_coarse_gmres<float, double>(const Grid&, double, double, const double*, const z64*, z128*,
                                                 z128*, z128*, double, double, int*, cudaStream_t, const int*);

}  // namespace helm
