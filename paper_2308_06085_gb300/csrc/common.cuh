// common.cuh -- shared device types for libhelm: complex values, grid descriptors and the
// pointwise pieces of the 7-point Helmholtz / CSLP operator (Sec. 2.4, Sec. 3.5).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

// Interleaved complex value; alignment makes a load one 16-byte (double) or 8-byte
// (float) vector access.
template <typename R>
struct alignas(2 * sizeof(R)) cx {
  R re, im;
};
using z128 = cx<double>;
using z64 = cx<float>;

template <typename R>
__host__ __device__ __forceinline__ cx<R> mkc(R a, R b) {
  cx<R> z;
  z.re = a;
  z.im = b;
  return z;
}
// FP32 -> FP64 conversion by the IEEE-754 bit layouts, in integer instructions.  On this GPU a
// converting instruction issues on the FP64 pipe, the one that bounds every FP64 kernel; the
// FP64 A-product on complex64 data (the mixed-precision Krylov method) spent a third of its time
// converting.  For zeros and normal numbers this gives the hardware conversion's bits: the
// exponent is rebiased by 1023 - 127 = 896 and the mantissa moved up 29 bits.  The rare other
// inputs (subnormals, infinities, NaNs) take the converting instruction in a separate call.
// (The opposite direction stays on the converting instruction: the FP32 kernels that read
// complex128 data are memory-bound, and an integer rounding measured slower there.)
static __device__ __noinline__ double f32_to_f64_hw(float f) { return (double)f; }
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned mag = u & 0x7fffffffu;
  if (mag != 0u && mag - 0x00800000u >= 0x7f000000u) return f32_to_f64_hw(f);
  const unsigned hi = (u & 0x80000000u) | (mag ? (mag >> 3) + 0x38000000u : 0u);
  return __hiloint2double((int)hi, (int)(u << 29));
}

template <typename To, typename From>
__device__ __forceinline__ cx<To> cvt(cx<From> a) {
  return mkc<To>((To)a.re, (To)a.im);
}
template <>
__device__ __forceinline__ cx<double> cvt<double, float>(cx<float> a) {
  return mkc<double>(f32_to_f64(a.re), f32_to_f64(a.im));
}

template <typename R>
__device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return mkc<R>(a.re + b.re, a.im + b.im); }
template <typename R>
__device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return mkc<R>(a.re - b.re, a.im - b.im); }
template <typename R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return mkc<R>(fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re));
}
// a + b*c
template <typename R>
__device__ __forceinline__ cx<R> cfma(cx<R> b, cx<R> c, cx<R> a) {
  R re = fma(b.re, c.re, a.re);
  re = fma(-b.im, c.im, re);
  R im = fma(b.re, c.im, a.im);
  im = fma(b.im, c.re, im);
  return mkc<R>(re, im);
}
// conj(a) * b accumulated into acc
template <typename R>
__device__ __forceinline__ void cdot_acc(cx<R> a, cx<R> b, R& re, R& im) {
  re = fma(a.re, b.re, re);
  re = fma(a.im, b.im, re);
  im = fma(a.re, b.im, im);
  im = fma(-a.im, b.re, im);
}

// Read-only (non-coherent L1) vector load of one complex value.
__device__ __forceinline__ cx<double> ldg(const cx<double>* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return mkc<double>(v.x, v.y);
}
__device__ __forceinline__ cx<float> ldg(const cx<float>* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return mkc<float>(v.x, v.y);
}

// Double-float complex: each FP64 component held as an unevaluated sum hi + lo of two FP32
// values (about 48 significant bits).  Layout (re_hi, im_hi, re_lo, im_lo), 16 bytes, so
// the first 8 bytes are the value rounded to complex64.
struct alignas(16) zdf {
  float rh, ih, rl, il;
};

__device__ __forceinline__ double ldg(const double* p) { return __ldg(p); }
__device__ __forceinline__ zdf ldg(const zdf* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  zdf z;
  z.rh = v.x; z.ih = v.y; z.rl = v.z; z.il = v.w;
  return z;
}

// x = hi + lo with hi = fl32(x), lo = fl32(x - hi).
__device__ __forceinline__ void df_split(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}
__device__ __forceinline__ zdf df_from(cx<double> z) {
  zdf r;
  df_split(z.re, r.rh, r.rl);
  df_split(z.im, r.ih, r.il);
  return r;
}
__device__ __forceinline__ cx<double> df_to_c128(const zdf& z) {
  return mkc<double>((double)z.rh + (double)z.rl, (double)z.ih + (double)z.il);
}

// (s, c) += (ah + al) (bh + bl), dropping al*bl (about 2^-48 relative).  The product's
// rounding error comes from an FMA (TwoProduct), the sum's from Knuth's TwoSum; both are
// exact in round-to-nearest FP32.  The _rn intrinsics are never contracted into FMAs, which
// keeps the error-free transformations intact.  (s, c) stays unnormalised: |c| << |s|.
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float& s, float& c) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// Double-float arithmetic on (hi, lo) pairs; results renormalised so |lo| <= ulp(hi)/2.
__device__ __forceinline__ void df_renorm(float s, float e, float& hi, float& lo) {
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}
// (ah + al) + (bh + bl): TwoSum of the leading parts, trailing parts added to the error.
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& hi, float& lo) {
  const float s = __fadd_rn(ah, bh);
  const float bp = __fsub_rn(s, ah);
  float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bp)), __fsub_rn(bh, bp));
  e = __fadd_rn(e, __fadd_rn(al, bl));
  df_renorm(s, e, hi, lo);
}
// (ah + al) (bh + bl) with the product error from an FMA; al*bl is dropped.
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& hi, float& lo) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  df_renorm(p, e, hi, lo);
}

// Error-free sum of two floats (Knuth's TwoSum): s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}
// (hi, lo) = (ah + al) * b for a float b: exact leading product by FMA, al*b added to the tail.
__device__ __forceinline__ void df_mul_f(float ah, float al, float b, float& hi, float& lo) {
  const float p = __fmul_rn(ah, b);
  float e = fmaf(ah, b, -p);
  e = fmaf(al, b, e);
  df_renorm(p, e, hi, lo);
}

// Grid of unknowns: N_d per direction, x fastest; bc 0 = Dirichlet, 1 = Sommerfeld.
struct Grid {
  int N1, N2, N3;
  int bc;
  double h;
  // sqrt(k^2) per node (FP64 and FP32 copies), read only at Sommerfeld face nodes; NULL when
  // the caller has none (the kernels then take the square root themselves)
  const double* sqk = nullptr;
  const float* sqkf = nullptr;
  // right-hand sides per node: grid vectors hold nb values per node, right-hand side
  // innermost (element index = node index * nb + rhs); per-node arrays (k^2, tables) stay
  // one value per node
  int nb = 1;
  // launch shape per kernel family (TILE_*) and arithmetic (slot = family + 4 for FP32): rows
  // of x-lines per CTA and the CTA count that sets the z-chunk each CTA streams through.  0
  // selects the default (8 rows, 8 CTAs per SM); helm_create's autotuner fills them.
  int tile_ty[8] = {};
  int tile_ctas[8] = {};
  // FP32 7-point kernels (one right-hand side): stage each plane's x-y neighbours in shared
  // memory (set per level by the autotuner when it measures faster)
  int tiled = 0;
  // FP32, one right-hand side: pre-smoothing from zero and the residual as one kernel (the
  // pre-smoothing slot then holds that kernel's shape); set by the autotuner when faster
  int fused_down = 0;
  // FP32, one right-hand side: the whole down-sweep (pre-smoothing, residual, restriction) as
  // one kernel (k_down32) with down_kc coarse planes per CTA; set by the autotuner when faster
  int down_full = 0, down_kc = 0;
  // one right-hand side (FP32 or FP64): prolongation, correction and post-smoothing as one
  // kernel (k_up) with up_kz fine planes per CTA; set by the autotuner when faster
  int up_full = 0, up_kz = 0;
  // one right-hand side (FP32 or FP64): the residual and its restriction as one kernel (k_rr)
  // with rr_kc coarse planes per CTA, after the pre-smoothing kernel; set by the autotuner when
  // faster
  int rr_full = 0, rr_kc = 0;
  __host__ __device__ size_t npts() const { return (size_t)N1 * N2 * N3; }
};

// One level of a coarse sub-cycle run by a single CTA in shared memory (k_coarse_cycle):
// the level's grid (one right-hand side), k^2, the FP64 omega/diag(M) table (NULL in FP32) and
// the offsets of its vectors in the CTA's shared buffer: B (right-hand side), U (pre-smoothed
// iterate, then the level's result E) and T (residual / corrected iterate; unused on the
// coarsest level).
constexpr int CC_MAX_LEVELS = 6;
template <typename R>
struct CLevel {
  Grid g;
  const R* k2;
  const cx<R>* dinv;
  int off_b, off_u, off_t;  // complex vectors (units of cx<R>)
  int off_k, off_s;         // k^2 and sqrt(k^2) copies (units of R)
  int off_d;                // omega/diag(M) copy (units of cx<R>; FP64 path), -1 without
};
template <typename R>
struct CCycle {
  int L;           // levels in the sub-cycle, the last one solved exactly
  int nc;          // unknowns of the coarsest level
  const cx<double>* Minv;
  double s_re, s_im, omega;
  CLevel<R> lev[CC_MAX_LEVELS];
};

// Kernel families with their own launch shape (Grid::tile_*).
enum { TILE_STENCIL = 0, TILE_SMOOTH0 = 1, TILE_RESTRICT = 2, TILE_PROLONG = 3 };
template <typename R>
constexpr int tile_slot(int fam) { return fam + (sizeof(R) == 4 ? 4 : 0); }

template <typename R>
__device__ __forceinline__ const R* grid_sqk(const Grid& g);
template <>
__device__ __forceinline__ const double* grid_sqk<double>(const Grid& g) { return g.sqk; }
template <>
__device__ __forceinline__ const float* grid_sqk<float>(const Grid& g) { return g.sqkf; }

// k at node p for the face term: from the per-node table when present.
template <typename R>
__device__ __forceinline__ R face_k(const Grid& g, size_t p, R k2p) {
  const R* t = grid_sqk<R>(g);
  return t ? __ldg(t + p) : sqrt(k2p);
}

__host__ __device__ __forceinline__ size_t gidx(int i, int j, int k, int N1, int N2) {
  return ((size_t)k * N2 + j) * N1 + i;
}

// Coefficients of (-Lap_h - s k^2) in working precision R.  s = s_re + i s_im:
// s = 1 for A_h, s = beta1 - beta2 i for M_h (Sec. 3.5).
template <typename R>
struct OpCoef {
  R ih2;      // 1 / h^2
  R six_ih2;  // 6 / h^2
  R s_re, s_im;
  R two_over_h;  // 2 / h : a Sommerfeld face adds -i (2/h) k to the diagonal
  R omega;       // damped-Jacobi relaxation (used by smoothing kernels)
  int real_shift;  // s_im == 0 (the operator A): the diagonal is real away from the faces
};

// Coefficients of a level's operator in working precision R (host side), shift s = s_re + i s_im.
template <typename R>
inline OpCoef<R> coef_for(double h, double s_re, double s_im, double omega) {
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

// Diagonal of the operator at a node lying on `nf` Sommerfeld faces (kp = sqrt(k^2), used only
// when nf > 0):
// 6/h^2 - s k^2 - i (2 k / h) nf.  The face term comes from eliminating the ghost value
// u_ghost = u_opposite + 2 h i k u_p (Sec. 2.4 Eq. elimination): its -1/h^2 coefficient
// moves 2 h i k u_p onto the diagonal.
template <typename R>
__device__ __forceinline__ cx<R> op_diag(const OpCoef<R>& c, R k2p, int nf, R kp) {
  R dre = fma(-c.s_re, k2p, c.six_ih2);
  R dim = c.real_shift ? (R)0 : -c.s_im * k2p;
  if (nf) dim = fma(-(R)nf * c.two_over_h, kp, dim);
  return mkc<R>(dre, dim);
}

// v = d u_c - (1/h^2) (sum of the six neighbour values) as an FMA chain, neighbours already
// replaced by the opposite value (Sommerfeld) or 0 (Dirichlet) where they fall outside the
// grid; real_d skips the d.im terms (d.im = 0).
template <typename R>
__device__ __forceinline__ cx<R> op_apply(cx<R> d, bool real_d, cx<R> uc, R ih2, cx<R> a, cx<R> b, cx<R> c,
                                          cx<R> e, cx<R> f, cx<R> g) {
  R re = -ih2 * a.re, im = -ih2 * a.im;
  re = fma(-ih2, b.re, re); im = fma(-ih2, b.im, im);
  re = fma(-ih2, c.re, re); im = fma(-ih2, c.im, im);
  re = fma(-ih2, e.re, re); im = fma(-ih2, e.im, im);
  re = fma(-ih2, f.re, re); im = fma(-ih2, f.im, im);
  re = fma(-ih2, g.re, re); im = fma(-ih2, g.im, im);
  re = fma(d.re, uc.re, re); im = fma(d.re, uc.im, im);
  if (!real_d) {
    re = fma(-d.im, uc.im, re);
    im = fma(d.im, uc.re, im);
  }
  return mkc<R>(re, im);
}

// Residual y - (d u_c - (1/h^2) sum) as one FMA chain starting from y.
template <typename R>
__device__ __forceinline__ cx<R> op_resid(cx<R> y, cx<R> d, bool real_d, cx<R> uc, R ih2, cx<R> a, cx<R> b,
                                          cx<R> c, cx<R> e, cx<R> f, cx<R> g) {
  R re = y.re, im = y.im;
  re = fma(ih2, a.re, re); im = fma(ih2, a.im, im);
  re = fma(ih2, b.re, re); im = fma(ih2, b.im, im);
  re = fma(ih2, c.re, re); im = fma(ih2, c.im, im);
  re = fma(ih2, e.re, re); im = fma(ih2, e.im, im);
  re = fma(ih2, f.re, re); im = fma(ih2, f.im, im);
  re = fma(ih2, g.re, re); im = fma(ih2, g.im, im);
  re = fma(-d.re, uc.re, re); im = fma(-d.re, uc.im, im);
  if (!real_d) {
    re = fma(d.im, uc.im, re);
    im = fma(-d.im, uc.re, im);
  }
  return mkc<R>(re, im);
}

// omega / d, computed as omega conj(d) / |d|^2.  The FP32 path (the complex64 V-cycle)
// takes the correctly rounded reciprocal of |d|^2 and one product instead of an IEEE division,
// which costs many more issue slots per point.
template <typename R>
__device__ __forceinline__ cx<R> omega_over(cx<R> d, R omega) {
  R inv = omega / fma(d.re, d.re, d.im * d.im);
  return mkc<R>(d.re * inv, -d.im * inv);
}
template <>
__device__ __forceinline__ cx<float> omega_over<float>(cx<float> d, float omega) {
  const float inv = omega * __frcp_rn(fmaf(d.re, d.re, d.im * d.im));
  return mkc<float>(d.re * inv, -d.im * inv);
}

// Device control block of Bi-CGSTAB: all scalars of the recurrence stay on the device.
struct BicgCtl {
  int active;  // 1 while the iteration continues
  int cont;    // 1 while the current step goes on past its half step
  int flag;    // 1 converged, 2 breakdown, 3 stagnation
  int half;    // the half step met tol (or the #Matvec cap)
  int iters;   // #Matvec
  int mark_it; // #Matvec when the residual last fell below half of mark
  double bnorm, relres;
  double mark; // residual at mark_it
  cx<double> rho, rho_prev, alpha, omega, beta;
};

// Device control block of IDR(s): the scalars of the recurrence and the small s x s system.
constexpr int IDR_SMAX = 8;
struct IdrCtl {
  int active;  // 1 while the iteration continues
  int flag;    // 1 converged, 2 breakdown
  int iters;   // #Matvec
  int s;       // shadow-space dimension
  double bnorm, relres, kappa, pad;
  cx<double> om;                          // omega of the last dimension-reduction step
  cx<double> beta;                        // step size of the current step
  cx<double> f[IDR_SMAX];                 // P^H r
  cx<double> c[IDR_SMAX];                 // coefficients of the current step
  cx<double> alpha[IDR_SMAX];             // biorthogonalisation coefficients of the current step
  cx<double> Ms[IDR_SMAX * IDR_SMAX];     // P^H G (row i, column k at i * IDR_SMAX + k), lower triangular
};

// Device control block of the batched Krylov loop (all pointers are device arrays; per
// right-hand side r unless stated).
struct BatchCtl {
  int any;       // 1 while any right-hand side is active in the current cycle
  int pass2;     // second Gram-Schmidt pass for the current step
  int max_iter;  // #Matvec cap per right-hand side
  int pad;
  int *act, *jend, *flag, *jmax, *iters;
  double *bnorm, *beta, *est;
  cx<double>* H;   // nb x (m+1) x m
  double* cs;      // nb x m
  cx<double>* sn;  // nb x m
  cx<double>* g;   // nb x (m+1)
  cx<double>* y;   // m x nb
};

// Device control block for the Krylov loop: kernels of an Arnoldi step return at once
// when `active` is 0, so the host can enqueue ahead without waiting.
struct KrylovCtl {
  int active;  // 1 while the current restart cycle continues
  int jend;    // last Arnoldi column completed in this cycle
  int flag;    // 1 = estimate reached tol, 2 = breakdown (zero or non-finite norm)
  int iter0;   // #Matvec before this cycle
  int pass2;   // 1 when the current Arnoldi step takes the second Gram-Schmidt pass
  double bnorm;
  double beta;
  double est;
};
