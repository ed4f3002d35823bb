// bicgstab.cu -- FP64 vector and scalar kernels of right-preconditioned Bi-CGSTAB (Sec. 3.1;
// the paper runs it with the same CSLP V-cycle and stops on ||b - A x|| / ||b||, Sec. 5).
// All scalars (rho, alpha, omega, beta) stay on the device; vector updates are fused with the
// partial sums they feed, and every reduction is deterministic (fixed grid, fixed order).
#include "internal.cuh"
#include "vecred.cuh"

namespace helm {

namespace {

using namespace vecred;

// part slot 0: conj(a) . b ; slot 1: conj(c) . d (when c != NULL)
__global__ void __launch_bounds__(NT)
    k_dots2(const z128* __restrict__ a, const z128* __restrict__ b, const z128* __restrict__ c,
            const z128* __restrict__ d, size_t n, z128* __restrict__ part, const int* __restrict__ active) {
  if (active && *active == 0) return;
  size_t p0, p1;
  brange(n, p0, p1);
  double re[2] = {0.0, 0.0}, im[2] = {0.0, 0.0};
  for (size_t p = p0 + threadIdx.x; p < p1; p += NT) {
    cdot_acc(ldg(a + p), ldg(b + p), re[0], im[0]);
    if (c) cdot_acc(ldg(c + p), ldg(d + p), re[1], im[1]);
  }
  block_partials<2>(re, im, part);
}

// p = r + beta (p - omega v)
__global__ void __launch_bounds__(NT)
    k_bicg_p(const z128* __restrict__ r, z128* __restrict__ p, const z128* __restrict__ v, const BicgCtl* __restrict__ bc,
             size_t n) {
  if (bc->active == 0) return;
  const z128 beta = bc->beta, omega = bc->omega;
  for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
    const z128 t = csub(p[q], cmul(omega, v[q]));
    p[q] = cfma(beta, t, r[q]);
  }
}

// s = r - alpha v, partial |s|^2
__global__ void __launch_bounds__(NT)
    k_bicg_s(const z128* __restrict__ r, const z128* __restrict__ v, z128* __restrict__ s, const BicgCtl* __restrict__ bc,
             size_t n, z128* __restrict__ part) {
  if (bc->active == 0) return;
  size_t p0, p1;
  brange(n, p0, p1);
  const z128 ma = mkc<double>(-bc->alpha.re, -bc->alpha.im);
  double re[1] = {0.0}, im[1] = {0.0};
  for (size_t q = p0 + threadIdx.x; q < p1; q += NT) {
    const z128 x = cfma(ma, v[q], r[q]);
    s[q] = x;
    re[0] = fma(x.re, x.re, re[0]);
    re[0] = fma(x.im, x.im, re[0]);
  }
  block_partials<1>(re, im, part);
}

// x += alpha p^ + omega s^ ; r = s - omega t ; partials |r|^2 (slot 0) and conj(rh) . r (slot 1).
// When the step ended at its half step (bc->half), only x += alpha p^ and r = s.
__global__ void __launch_bounds__(NT)
    k_bicg_xr(z128* __restrict__ x, z128* __restrict__ r, const z128* __restrict__ ph, const z128* __restrict__ sh,
              const z128* __restrict__ s, const z128* __restrict__ t, const z128* __restrict__ rh,
              const BicgCtl* __restrict__ bc, size_t n, z128* __restrict__ part) {
  if (bc->active == 0) return;
  size_t p0, p1;
  brange(n, p0, p1);
  const z128 alpha = bc->alpha, omega = bc->omega;
  const bool half = bc->half != 0;
  double re[2] = {0.0, 0.0}, im[2] = {0.0, 0.0};
  for (size_t q = p0 + threadIdx.x; q < p1; q += NT) {
    z128 xv = cfma(alpha, ph[q], x[q]);
    z128 rv = s[q];
    if (!half) {
      xv = cfma(omega, sh[q], xv);
      rv = cfma(mkc<double>(-omega.re, -omega.im), t[q], rv);
    }
    x[q] = xv;
    r[q] = rv;
    re[0] = fma(rv.re, rv.re, re[0]);
    re[0] = fma(rv.im, rv.im, re[0]);
    cdot_acc(ldg(rh + q), rv, re[1], im[1]);
  }
  block_partials<2>(re, im, part);
}

// Scalar steps, one warp (the warp sums the block partials; lane 0 updates the scalars):
// stage 0: start of a step: beta = (rho / rho_prev)(alpha / omega); breakdown if rho = 0
// stage 1: alpha = rho / (rh . v)
// stage 2: |s| -> half-step test
// stage 3: omega = (t . s) / (t . t)
// stage 4: |r|, rho_next -> convergence test; stagnation when the residual has not halved within
//          `stall` products with A (stall > 0)
__global__ void k_bicg_scalar(BicgCtl* bc, const z128* __restrict__ part, int nb, int stage, double tol, int max_iter,
                              int stall, double* hist, int hist_len) {
  if (blockIdx.x != 0) return;
  if (bc->active == 0) return;
  const bool lead = threadIdx.x == 0;
  if (stage == 0) {
    if (!lead) return;
    const z128 rho = bc->rho;
    bc->cont = 1;
    bc->half = 0;
    if ((rho.re == 0.0 && rho.im == 0.0) || (bc->omega.re == 0.0 && bc->omega.im == 0.0)) {
      bc->flag = 2;
      bc->active = 0;
      bc->cont = 0;
      return;
    }
    bc->beta = cmul(cdiv(rho, bc->rho_prev), cdiv(bc->alpha, bc->omega));
  } else if (stage == 1) {
    const z128 rv = sum_slot(part, 0, nb);
    if (!lead) return;
    bc->iters += 1;
    if (rv.re == 0.0 && rv.im == 0.0) {
      bc->flag = 2;
      bc->active = 0;
      bc->cont = 0;
      return;
    }
    bc->alpha = cdiv(bc->rho, rv);
  } else if (stage == 2) {
    const double sn = sqrt(sum_slot(part, 0, nb).re) / bc->bnorm;
    if (!lead) return;
    const int it = bc->iters - 1;
    if (hist && it < hist_len) hist[it] = sn;
    if (sn <= tol || bc->iters >= max_iter) {
      bc->half = 1;
      bc->cont = 0;
    }
  } else if (stage == 3) {
    if (bc->cont == 0) return;
    const z128 ts = sum_slot(part, 0, nb);
    const double tt = sum_slot(part, 1, nb).re;
    if (!lead) return;
    bc->iters += 1;
    if (!(tt > 0.0)) {
      bc->flag = 2;
      bc->active = 0;
      bc->cont = 0;
      return;
    }
    bc->omega = mkc<double>(ts.re / tt, ts.im / tt);
  } else {
    const double rn = sqrt(sum_slot(part, 0, nb).re) / bc->bnorm;
    const z128 rho = sum_slot(part, 1, nb);
    if (!lead) return;
    if (!bc->half) {
      const int it = bc->iters - 1;
      if (hist && it < hist_len) hist[it] = rn;
    }
    bc->relres = rn;
    bc->rho_prev = bc->rho;
    bc->rho = rho;
    if (!isfinite(rn)) {
      bc->flag = 2;
      bc->active = 0;
    } else if (rn <= tol) {
      bc->flag = 1;
      bc->active = 0;
    } else if (bc->half || bc->iters >= max_iter) {
      bc->active = 0;
    } else if (rn < 0.5 * bc->mark) {
      bc->mark = rn;
      bc->mark_it = bc->iters;
    } else if (stall > 0 && bc->iters - bc->mark_it >= stall) {
      bc->flag = 3;
      bc->active = 0;
    }
    if (bc->active == 0) bc->cont = 0;
  }
}

// Start (or restart) from r = b - A x: rh = r, p = v = 0, rho = |r|^2, alpha = omega = rho_prev = 1.
__global__ void k_bicg_init(BicgCtl* bc, const z128* __restrict__ part, int nb, const z128* __restrict__ r,
                            z128* __restrict__ rh, z128* __restrict__ p, z128* __restrict__ v, size_t n) {
  for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
    rh[q] = r[q];
    p[q] = mkc<double>(0.0, 0.0);
    v[q] = mkc<double>(0.0, 0.0);
  }
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    const double rr = sum_slot(part, 0, nb).re;
    if (threadIdx.x != 0) return;
    bc->rho = mkc<double>(rr, 0.0);
    bc->rho_prev = bc->alpha = bc->omega = mkc<double>(1.0, 0.0);
    bc->relres = sqrt(rr) / bc->bnorm;
    bc->mark = bc->relres;
    bc->mark_it = bc->iters;
    bc->half = 0;
    bc->flag = 0;
    bc->active = 1;
    bc->cont = 1;
  }
}

}  // namespace

int launch_dots2(const z128* a, const z128* b, const z128* c, const z128* d, size_t n, z128* part, cudaStream_t st,
                 const int* active) {
  static const int nb = wave(k_dots2);
  k_dots2<<<nb, NT, 0, st>>>(a, b, c, d, n, part, active);
  return nb;
}
void launch_bicg_p(const z128* r, z128* p, const z128* v, const BicgCtl* bc, size_t n, cudaStream_t st) {
  k_bicg_p<<<sblocks(n), NT, 0, st>>>(r, p, v, bc, n);
}
int launch_bicg_s(const z128* r, const z128* v, z128* s, const BicgCtl* bc, size_t n, z128* part, cudaStream_t st) {
  static const int nb = wave(k_bicg_s);
  k_bicg_s<<<nb, NT, 0, st>>>(r, v, s, bc, n, part);
  return nb;
}
int launch_bicg_xr(z128* x, z128* r, const z128* ph, const z128* sh, const z128* s, const z128* t, const z128* rh,
                   const BicgCtl* bc, size_t n, z128* part, cudaStream_t st) {
  static const int nb = wave(k_bicg_xr);
  k_bicg_xr<<<nb, NT, 0, st>>>(x, r, ph, sh, s, t, rh, bc, n, part);
  return nb;
}
void launch_bicg_scalar(BicgCtl* bc, const z128* part, int nb, int stage, double tol, int max_iter, int stall,
                        double* hist, int hist_len, cudaStream_t st) {
  k_bicg_scalar<<<1, 32, 0, st>>>(bc, part, nb, stage, tol, max_iter, stall, hist, hist_len);
}
void launch_bicg_init(BicgCtl* bc, const z128* part, int nb, const z128* r, z128* rh, z128* p, z128* v, size_t n,
                      cudaStream_t st) {
  k_bicg_init<<<sblocks(n), NT, 0, st>>>(bc, part, nb, r, rh, p, v, n);
}

}  // namespace helm
