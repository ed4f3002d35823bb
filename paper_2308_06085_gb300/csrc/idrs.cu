// idrs.cu -- FP64 vector and scalar kernels of right-preconditioned IDR(s) (Sec. 3.1: the
// induced-dimension-reduction method the paper runs as IDR(4), stopping on ||b - A x|| / ||b||,
// Sec. 5), in its biorthogonal form.
//
// One cycle is s steps k = 0..s-1 and one dimension-reduction step.  Step k:
//   c    = Ms[k.., k..]^{-1} f[k..]                      (scalar kernel, lower triangular)
//   v    = r - G[k..] c                                  (k_idr_v)
//   U_k  = omega M^{-1} v + U[k..] c                     (V-cycle, then k_idr_u)
//   G_k  = A U_k                                         (stencil)
//   d    = P^H G_k                                       (k_idr_pdots)
//   alpha, the new column Ms[k.., k], beta = f_k / Ms[k][k], f update (scalar kernel)
//   G_k -= G[<k] alpha; U_k -= U[<k] alpha; r -= beta G_k; x += beta U_k; |r|^2  (k_idr_update)
// The biorthogonalisation coefficients come from the single product d = P^H G_k by forward
// substitution with the known lower triangle of Ms (P_i^H G_j = Ms[i][j] for j <= i), the same
// values that subtracting G_0 .. G_{k-1} one at a time gives.  Dimension reduction:
//   t = A M^{-1} r, omega from (t^H r, |t|^2, |r|) with the angle safeguard kappa,
//   r -= omega t, x += omega M^{-1} r, and f = P^H r and |r|^2 of the new r in the same pass.
// All scalars stay on the device; every reduction has a fixed grid and order.
#include "internal.cuh"
#include "vecred.cuh"

namespace helm {

namespace {

using namespace vecred;

// v = r - sum_{i=k}^{s-1} c_i G_i
__global__ void __launch_bounds__(NT)
    k_idr_v(const IdrCtl* __restrict__ ic, int k, const z128* __restrict__ r, const z128* __restrict__ G, size_t n,
            z128* __restrict__ v) {
  if (ic->active == 0) return;
  const int s = ic->s;
  z128 c[IDR_SMAX];
#pragma unroll
  for (int i = 0; i < IDR_SMAX; ++i) c[i] = i >= k && i < s ? mkc<double>(-ic->c[i].re, -ic->c[i].im) : mkc<double>(0.0, 0.0);
  for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
    z128 a = ldg(r + q);
#pragma unroll
    for (int i = 0; i < IDR_SMAX; ++i)
      if (i >= k && i < s) a = cfma(c[i], ldg(G + (size_t)i * n + q), a);
    v[q] = a;
  }
}

// U_k = omega vh + sum_{i=k}^{s-1} c_i U_i  (U_k itself is one of the terms)
__global__ void __launch_bounds__(NT)
    k_idr_u(const IdrCtl* __restrict__ ic, int k, const z128* __restrict__ vh, z128* __restrict__ U, size_t n) {
  if (ic->active == 0) return;
  const int s = ic->s;
  const z128 om = ic->om;
  z128 c[IDR_SMAX];
#pragma unroll
  for (int i = 0; i < IDR_SMAX; ++i) c[i] = i >= k && i < s ? ic->c[i] : mkc<double>(0.0, 0.0);
  z128* Uk = U + (size_t)k * n;
  for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
    z128 a = cmul(om, ldg(vh + q));
#pragma unroll
    for (int i = 0; i < IDR_SMAX; ++i)
      if (i >= k && i < s) a = cfma(c[i], U[(size_t)i * n + q], a);
    Uk[q] = a;
  }
}

// Partial sums of conj(P_i) . y for i < S (slots 0..S-1) and, with NORM, |y|^2 (slot S).
template <int S, bool NORM>
__global__ void __launch_bounds__(NT)
    k_idr_pdots(const z128* __restrict__ P, const z128* __restrict__ y, size_t n, z128* __restrict__ part,
                const int* __restrict__ active) {
  if (active && *active == 0) return;
  size_t p0, p1;
  brange(n, p0, p1);
  constexpr int NS = S + (NORM ? 1 : 0);
  double re[NS], im[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) re[i] = im[i] = 0.0;
  for (size_t q = p0 + threadIdx.x; q < p1; q += NT) {
    const z128 yv = ldg(y + q);
#pragma unroll
    for (int i = 0; i < S; ++i) cdot_acc(ldg(P + (size_t)i * n + q), yv, re[i], im[i]);
    if (NORM) {
      re[NS - 1] = fma(yv.re, yv.re, re[NS - 1]);
      re[NS - 1] = fma(yv.im, yv.im, re[NS - 1]);
    }
  }
  block_partials<NS>(re, im, part);
}

// G_k -= sum_{j<k} alpha_j G_j ; U_k -= sum_{j<k} alpha_j U_j ; r -= beta G_k ; x += beta U_k ;
// partial |r|^2 in slot 0.
__global__ void __launch_bounds__(NT)
    k_idr_update(const IdrCtl* __restrict__ ic, int k, z128* __restrict__ G, z128* __restrict__ U, z128* __restrict__ r,
                 z128* __restrict__ x, size_t n, z128* __restrict__ part) {
  if (ic->active == 0) return;
  size_t p0, p1;
  brange(n, p0, p1);
  z128 ma[IDR_SMAX];
#pragma unroll
  for (int j = 0; j < IDR_SMAX; ++j) ma[j] = j < k ? mkc<double>(-ic->alpha[j].re, -ic->alpha[j].im) : mkc<double>(0.0, 0.0);
  const z128 beta = ic->beta, mbeta = mkc<double>(-ic->beta.re, -ic->beta.im);
  z128* Gk = G + (size_t)k * n;
  z128* Uk = U + (size_t)k * n;
  double re[1] = {0.0}, im[1] = {0.0};
  for (size_t q = p0 + threadIdx.x; q < p1; q += NT) {
    z128 g = Gk[q], u = Uk[q];
#pragma unroll
    for (int j = 0; j < IDR_SMAX; ++j)
      if (j < k) {
        g = cfma(ma[j], ldg(G + (size_t)j * n + q), g);
        u = cfma(ma[j], ldg(U + (size_t)j * n + q), u);
      }
    Gk[q] = g;
    Uk[q] = u;
    const z128 rv = cfma(mbeta, g, r[q]);
    r[q] = rv;
    x[q] = cfma(beta, u, x[q]);
    re[0] = fma(rv.re, rv.re, re[0]);
    re[0] = fma(rv.im, rv.im, re[0]);
  }
  block_partials<1>(re, im, part);
}

// r -= omega t ; x += omega vh ; partials conj(P_i) . r (slots 0..S-1) and |r|^2 (slot S).
template <int S>
__global__ void __launch_bounds__(NT)
    k_idr_xr(const IdrCtl* __restrict__ ic, const z128* __restrict__ P, z128* __restrict__ r, const z128* __restrict__ t,
             z128* __restrict__ x, const z128* __restrict__ vh, size_t n, z128* __restrict__ part) {
  if (ic->active == 0) return;
  size_t p0, p1;
  brange(n, p0, p1);
  const z128 om = ic->om, mom = mkc<double>(-ic->om.re, -ic->om.im);
  double re[S + 1], im[S + 1];
#pragma unroll
  for (int i = 0; i <= S; ++i) re[i] = im[i] = 0.0;
  for (size_t q = p0 + threadIdx.x; q < p1; q += NT) {
    const z128 rv = cfma(mom, ldg(t + q), r[q]);
    r[q] = rv;
    x[q] = cfma(om, ldg(vh + q), x[q]);
#pragma unroll
    for (int i = 0; i < S; ++i) cdot_acc(ldg(P + (size_t)i * n + q), rv, re[i], im[i]);
    re[S] = fma(rv.re, rv.re, re[S]);
    re[S] = fma(rv.im, rv.im, re[S]);
  }
  block_partials<S + 1>(re, im, part);
}

__device__ __forceinline__ bool czero(z128 a) { return a.re == 0.0 && a.im == 0.0; }

__device__ __forceinline__ void idr_stop(IdrCtl* ic, int flag) {
  ic->flag = flag;
  ic->active = 0;
}

// Scalar steps, one warp (the warp sums the block partials; lane 0 updates the scalars).
//   0 (step k): c = Ms[k.., k..]^{-1} f[k..]
//   1 (step k, after d = P^H G_k): alpha, Ms[k.., k], beta, f; #Matvec += 1
//   2 (step k, after the update): |r| -> convergence / cap
//   3 (dimension reduction, after t^H r and |t|^2): omega with the angle safeguard; #Matvec += 1
//   4 (after r -= omega t): f = P^H r, |r| -> convergence / cap
//   5 (start): f = P^H r, |r|; Ms = I, omega = 1
__global__ void k_idr_scalar(IdrCtl* ic, const z128* __restrict__ part, int nb, int stage, int k, double tol,
                             int max_iter, double* hist, int hist_len) {
  if (stage != 5 && ic->active == 0) return;
  const bool lead = threadIdx.x == 0;
  const int s = ic->s;
  if (stage == 0) {
    if (!lead) return;
    for (int i = k; i < s; ++i) {
      z128 acc = ic->f[i];
      for (int j = k; j < i; ++j) acc = csub(acc, cmul(ic->Ms[i * IDR_SMAX + j], ic->c[j]));
      ic->c[i] = cdiv(acc, ic->Ms[i * IDR_SMAX + i]);
    }
  } else if (stage == 1) {
    z128 d[IDR_SMAX];
    for (int i = 0; i < s; ++i) d[i] = sum_slot(part, i, nb);
    if (!lead) return;
    ic->iters += 1;
    z128 al[IDR_SMAX];
    for (int i = 0; i < k; ++i) {
      z128 acc = d[i];
      for (int j = 0; j < i; ++j) acc = csub(acc, cmul(al[j], ic->Ms[i * IDR_SMAX + j]));
      al[i] = cdiv(acc, ic->Ms[i * IDR_SMAX + i]);
      ic->alpha[i] = al[i];
    }
    for (int i = k; i < s; ++i) {
      z128 acc = d[i];
      for (int j = 0; j < k; ++j) acc = csub(acc, cmul(al[j], ic->Ms[i * IDR_SMAX + j]));
      ic->Ms[i * IDR_SMAX + k] = acc;
    }
    const z128 mkk = ic->Ms[k * IDR_SMAX + k];
    if (czero(mkk)) {
      idr_stop(ic, 2);
      return;
    }
    const z128 beta = cdiv(ic->f[k], mkk);
    ic->beta = beta;
    for (int i = k + 1; i < s; ++i) ic->f[i] = csub(ic->f[i], cmul(beta, ic->Ms[i * IDR_SMAX + k]));
  } else if (stage == 2) {
    const double rn = sqrt(sum_slot(part, 0, nb).re) / ic->bnorm;
    if (!lead) return;
    ic->relres = rn;
    const int it = ic->iters - 1;
    if (hist && it < hist_len) hist[it] = rn;
    if (!isfinite(rn)) idr_stop(ic, 2);
    else if (rn <= tol) idr_stop(ic, 1);
    else if (ic->iters >= max_iter) idr_stop(ic, 0);
  } else if (stage == 3) {
    const z128 tr = sum_slot(part, 0, nb);
    const double tt = sum_slot(part, 1, nb).re;
    if (!lead) return;
    ic->iters += 1;
    const double tn = sqrt(tt), rn = ic->relres * ic->bnorm;
    if (!(tt > 0.0)) {
      idr_stop(ic, 2);
      return;
    }
    z128 om = mkc<double>(tr.re / tt, tr.im / tt);
    const double rho = sqrt(tr.re * tr.re + tr.im * tr.im) / (tn * rn);
    if (rho < ic->kappa) {
      const double sc = ic->kappa / rho;
      om = mkc<double>(om.re * sc, om.im * sc);
    }
    if (czero(om)) {
      idr_stop(ic, 2);
      return;
    }
    ic->om = om;
  } else {
    z128 f[IDR_SMAX];
    for (int i = 0; i < s; ++i) f[i] = sum_slot(part, i, nb);
    const double rn = sqrt(sum_slot(part, s, nb).re) / ic->bnorm;
    if (!lead) return;
    for (int i = 0; i < s; ++i) ic->f[i] = f[i];
    ic->relres = rn;
    if (stage == 5) {
      for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) ic->Ms[i * IDR_SMAX + j] = mkc<double>(i == j ? 1.0 : 0.0, 0.0);
      ic->om = mkc<double>(1.0, 0.0);
      ic->flag = 0;
      ic->active = 1;
      if (!isfinite(rn)) idr_stop(ic, 2);
      else if (rn <= tol) idr_stop(ic, 1);
      return;
    }
    const int it = ic->iters - 1;
    if (hist && it < hist_len) hist[it] = rn;
    if (!isfinite(rn)) idr_stop(ic, 2);
    else if (rn <= tol) idr_stop(ic, 1);
    else if (ic->iters >= max_iter) idr_stop(ic, 0);
  }
}

template <int S, bool NORM>
int pdots_s(const z128* P, const z128* y, size_t n, z128* part, cudaStream_t st, const int* active) {
  static const int nb = wave(k_idr_pdots<S, NORM>);
  k_idr_pdots<S, NORM><<<nb, NT, 0, st>>>(P, y, n, part, active);
  return nb;
}

template <int S>
int xr_s(const IdrCtl* ic, const z128* P, z128* r, const z128* t, z128* x, const z128* vh, size_t n, z128* part,
         cudaStream_t st) {
  static const int nb = wave(k_idr_xr<S>);
  k_idr_xr<S><<<nb, NT, 0, st>>>(ic, P, r, t, x, vh, n, part);
  return nb;
}

}  // namespace

void launch_idr_v(const IdrCtl* ic, int k, const z128* r, const z128* G, size_t n, z128* v, cudaStream_t st) {
  k_idr_v<<<sblocks(n), NT, 0, st>>>(ic, k, r, G, n, v);
}
void launch_idr_u(const IdrCtl* ic, int k, const z128* vh, z128* U, size_t n, cudaStream_t st) {
  k_idr_u<<<sblocks(n), NT, 0, st>>>(ic, k, vh, U, n);
}
int launch_idr_pdots(int s, bool with_norm, const z128* P, const z128* y, size_t n, z128* part, cudaStream_t st,
                     const int* active) {
#define IDR_PD(S) \
  case S: return with_norm ? pdots_s<S, true>(P, y, n, part, st, active) : pdots_s<S, false>(P, y, n, part, st, active);
  switch (s) {
    IDR_PD(1) IDR_PD(2) IDR_PD(3) IDR_PD(4) IDR_PD(5) IDR_PD(6) IDR_PD(7) IDR_PD(8)
    default: return 0;
  }
#undef IDR_PD
}
int launch_idr_update(const IdrCtl* ic, int k, z128* G, z128* U, z128* r, z128* x, size_t n, z128* part,
                      cudaStream_t st) {
  static const int nb = wave(k_idr_update);
  k_idr_update<<<nb, NT, 0, st>>>(ic, k, G, U, r, x, n, part);
  return nb;
}
int launch_idr_xr(int s, const IdrCtl* ic, const z128* P, z128* r, const z128* t, z128* x, const z128* vh, size_t n,
                  z128* part, cudaStream_t st) {
  switch (s) {
    case 1: return xr_s<1>(ic, P, r, t, x, vh, n, part, st);
    case 2: return xr_s<2>(ic, P, r, t, x, vh, n, part, st);
    case 3: return xr_s<3>(ic, P, r, t, x, vh, n, part, st);
    case 4: return xr_s<4>(ic, P, r, t, x, vh, n, part, st);
    case 5: return xr_s<5>(ic, P, r, t, x, vh, n, part, st);
    case 6: return xr_s<6>(ic, P, r, t, x, vh, n, part, st);
    case 7: return xr_s<7>(ic, P, r, t, x, vh, n, part, st);
    case 8: return xr_s<8>(ic, P, r, t, x, vh, n, part, st);
    default: return 0;
  }
}
void launch_idr_scalar(IdrCtl* ic, const z128* part, int nb, int stage, int k, double tol, int max_iter, double* hist,
                       int hist_len, cudaStream_t st) {
  k_idr_scalar<<<1, 32, 0, st>>>(ic, part, nb, stage, k, tol, max_iter, hist, hist_len);
}

}  // namespace helm
