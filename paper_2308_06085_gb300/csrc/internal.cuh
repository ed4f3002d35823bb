// internal.cuh -- launchers shared between the translation units of libhelm.
#pragma once

#include "common.cuh"

namespace helm {

// ---- grid kernels (stencil.cu) ----
template <typename R, typename TU, typename TO>
void launch_apply(const Grid& g, double s_re, double s_im, const R* k2, const cx<TU>* u, cx<TO>* v, cudaStream_t st,
                  const int* active);
// FP64 operator product written as double-float (the Arnoldi vector of the double-float
// Gram-Schmidt)
template <typename TU>
void launch_apply_split(const Grid& g, double s_re, double s_im, const double* k2, const cx<TU>* u, zdf* v,
                        cudaStream_t st, const int* active);
// out = b - M u; with dtab (an FP64 level's coefficient table: omega/d, then d) the diagonal of
// M is read from the table instead of computed from k^2 (same values)
template <typename R, typename TU, typename TB, typename TO>
void launch_resid(const Grid& g, double s_re, double s_im, const R* k2, const cx<TU>* u, const cx<TB>* b, cx<TO>* out,
                  cudaStream_t st, const int* active, const cx<R>* dtab = nullptr);
template <typename R, typename TB, typename TO>
void launch_jacobi(const Grid& g, double s_re, double s_im, double omega, const R* k2, const cx<R>* dinv,
                   const cx<R>* u, const cx<TB>* b, cx<TO>* out, cudaStream_t st, const int* active);
// u1 = (omega/d) b; with bout, b in working precision R is written there too
template <typename R, typename TB>
void launch_smooth0(const Grid& g, double s_re, double s_im, double omega, const R* k2, const cx<R>* dinv,
                    const cx<TB>* b, cx<R>* out, cudaStream_t st, const int* active, cx<R>* bout = nullptr);
template <typename R>
void launch_restrict(const Grid& gf, const Grid& gc, const cx<R>* r, cx<R>* out, cudaStream_t st, const int* active);
template <typename R>
void launch_prolong_add(const Grid& gf, const Grid& gc, const cx<R>* u1, const cx<R>* e, cx<R>* out, cudaStream_t st,
                        const int* active);
// The paper's coarsest-grid solve: full GMRES on M_c e = b from e = 0 to the relative
// residual tol (at most CG_MAX steps; second Gram-Schmidt pass when the first kept less than
// `keep` of |w|^2), by one cluster of 16 CTAs (CG_CS = 8 where the GPU cannot place 16); V
// holds (CG_MAX + 1) grid vectors and H CG_MAX columns of CG_MAX + 1, both device scratch of
// the context; info[0] = steps taken, info[1] = 1 when tol was met.  The grid may hold at most
// CG_CS * 512 unknowns.
constexpr int CG_CS = 8;
constexpr int CG_MAX = 256;
template <typename TI, typename TO>
void launch_coarse_gmres(const Grid& g, double s_re, double s_im, const double* k2, const cx<TI>* b, cx<TO>* e,
                         z128* V, z128* H, double tol, double keep, int* info, cudaStream_t st, const int* active);
// e = Minv b for nb right-hand sides (node-major, right-hand side innermost)
template <typename TI, typename TO>
void launch_coarse(int nc, const z128* Minv, const cx<TI>* b, cx<TO>* e, cudaStream_t st, const int* active,
                   int nb = 1);
// X = A^{-1} by Gauss-Jordan elimination with partial pivoting (A, n x n row-major, is
// overwritten); scratch fcol (n), piv, pinv; *singular is set when a pivot column is zero.
void launch_gj_invert(z128* A, z128* X, int n, z128* fcol, int* piv, z128* pinv, int* singular, cudaStream_t st);
// FP64 level coefficient table: out[p] = omega / diag(M)_p, out[npts + p] = diag(M)_p
void launch_dinv(const Grid& g, double s_re, double s_im, double omega, const double* k2, z128* out, cudaStream_t st);
void launch_inject(const Grid& gf, const Grid& gc, const double* kf, double* kc, cudaStream_t st);
void launch_to_float(const double* a, float* b, size_t n, cudaStream_t st);
// out64 = the kernels' FP32 -> FP64 conversion of in32
void launch_convert_check(const float* in32, double* out64, size_t n, cudaStream_t st);
// sk = sqrt(k2) in FP64, skf = sqrtf(float(k2)) in FP32 (the face terms' k)
void launch_sqrt_table(const double* k2, double* sk, float* skf, size_t n, cudaStream_t st);
void launch_check_k2(const double* a, size_t n, int* bad, cudaStream_t st);
void launch_rhs_point(const Grid& g, int nsrc, const int* idx, double amp, z128* b, cudaStream_t st);

// ---- Krylov kernels (krylov.cu) ----
constexpr int RED_STRIDE = 2048;  // row stride of partial-sum buffers: max blocks of a reduction grid
constexpr int MAX_BASIS = 257;   // restart <= 256

// part[i * RED_STRIDE + blk] = sum over blk's points of conj(V_i) w, i < nv; with_norm also
// writes the partial |w|^2 to slot nv.  Returns the number of blocks (partials per row).
int launch_mdot(const z128* V, size_t ld, int nv, const z128* w, size_t n, z128* part, int with_norm,
                cudaStream_t st, const int* active, int variant = 0);
// The same against a basis stored with its element sums Vs[i * ld + p] = Re V + Im V (three
// FP64 FMAs per complex multiply-add instead of four).
int launch_mdot_sums(const z128* V, const double* Vs, size_t ld, int nv, const z128* w, size_t n, z128* part,
                     int with_norm, cudaStream_t st, const int* active, int variant);
// hpass[i] = sum_{blk < nb} part[i * RED_STRIDE + blk]; hacc[i] = hpass[i] (accumulate 0) or
// += (1).  decide_j >= 0: also read |w|^2 from slot nv and set *pass2 = log[decide_j] =
// (second Gram-Schmidt pass needed: the first kept less than `keep` of |w|^2)
void launch_reduce_dots(const z128* part, int nv, int nb, z128* hpass, z128* hacc, int accumulate, int decide_j,
                        int* pass2, int* log, cudaStream_t st, const int* active, double keep);
// w -= sum_i h[i] V_i
void launch_gs_update(const z128* V, size_t ld, int nv, const z128* h, z128* w, size_t n, cudaStream_t st,
                      const int* active);
void launch_gs_update_sums(const z128* V, const double* Vs, size_t ld, int nv, const z128* h, z128* w, size_t n,
                           cudaStream_t st, const int* active);
// partial sums of |x|^2 into partr[0..nb); returns nb
int launch_norm2_part(const z128* x, size_t n, double* partr, cudaStream_t st, const int* active);
// *out = sqrt(sum_{b < nb} partr[b])
void launch_reduce_norm(const double* partr, int nb, double* out, cudaStream_t st, const int* active);
// out = in * (1 / *s)   (when *s != 0)
void launch_scale_inv(const z128* in, const double* s, z128* out, size_t n, cudaStream_t st, const int* active);
// out = in / *s and outs = Re out + Im out
void launch_scale_inv_sums(const z128* in, const double* s, z128* out, double* outs, size_t n, cudaStream_t st,
                           const int* active);
// start a restart cycle: active = 1, g = (beta, 0, ...), iter0 recorded
void launch_cycle_init(KrylovCtl* ctl, z128* gvec, int m, int iter0, cudaStream_t st);
// Arnoldi step j: rotations on H(:, j) (column stored at Hcol), new rotation, g update,
// estimate, stopping flags; writes hist[iter0 + j]
void launch_givens(KrylovCtl* ctl, z128* H, int m, int j, int jmax, const z128* hcol, const double* hnorm,
                   double* cs, z128* sn, z128* gvec, double tol, double* hist, int hist_len, cudaStream_t st);
// y = H(0:k, 0:k)^{-1} g with k = jend + 1
void launch_trisolve(const KrylovCtl* ctl, const z128* H, int m, const z128* gvec, z128* y, cudaStream_t st);
// x += Z y in double-float arithmetic for complex64 Z (x FP64)
void launch_xupdate_df(const KrylovCtl* ctl, const z64* Z, size_t ld, const z128* y, z128* x, size_t n,
                       cudaStream_t st);
void launch_bxupdate_df(const BatchCtl* bc, int nb, int m, const z64* Z, size_t ld, z128* x, size_t ne,
                        cudaStream_t st);
// x += sum_{i<=jend} y_i Z_i   (Z c128 or c64)
template <typename TZ>
void launch_xupdate(const KrylovCtl* ctl, const cx<TZ>* Z, size_t ld, const z128* y, z128* x, size_t n,
                    cudaStream_t st);
// w = sum_{i<=jend} y_i V_i
void launch_combine(const KrylovCtl* ctl, const z128* V, size_t ld, const z128* y, z128* w, size_t n,
                    cudaStream_t st);
// double-float Gram-Schmidt (basis stored as zdf)
// variant: slots per warp per pass, 0: 4, 1: 2, 2: 8 (chosen by the autotuner)
int launch_mdot_df(const zdf* V, size_t ld, int nv, const zdf* w, size_t n, z128* part, int with_norm,
                   cudaStream_t st, const int* active, int variant = 0);
void launch_gs_update_df(const zdf* V, size_t ld, int nv, const z128* h, zdf* w, size_t n, cudaStream_t st,
                         const int* active);
// partial sums of |x|^2 (double-float x) into partr; returns nb
int launch_norm2_part_df(const zdf* x, size_t n, double* partr, cudaStream_t st, const int* active);
// out = in / *s as double-float, and a copy as c128 (exact) or c64 (leading part); in is
// c128 (TI = z128) or double-float (TI = zdf)
template <typename TI, typename TC>
void launch_scale_df(const TI* in, const double* s, zdf* out, cx<TC>* copy, size_t n, cudaStream_t st,
                     const int* active);
void launch_combine_df(const KrylovCtl* ctl, const zdf* V, size_t ld, const z128* y, z128* w, size_t n,
                       cudaStream_t st);
void launch_c128_to_c64(const z128* a, z64* b, size_t n, cudaStream_t st);
void launch_c64_to_c128(const z64* a, z128* b, size_t n, cudaStream_t st);
void launch_set_active(KrylovCtl* ctl, int v, cudaStream_t st);
// x += z
void launch_axpy1(const z128* z, z128* x, size_t n, cudaStream_t st);

// A u for a complex64 u in double-float arithmetic (stencil.cu); k2df / skdf are (hi, lo)
// tables of k^2 and sqrt(k^2) filled by launch_k2_df.  OUT: zdf or z128.
template <typename OUT>
void launch_apply_c64_df(const Grid& g, const float2* k2df, const float2* skdf, const z64* u, OUT* v, cudaStream_t st,
                         const int* active);
void launch_k2_df(const double* k2, size_t n, float2* k2df, float2* skdf, cudaStream_t st);

// The V-cycle on the coarse levels of cc in one CTA with every vector in shared memory
// (stencil.cu): b = the first level's right-hand side, e = its result; smem_bytes <=
// CC_SMEM_MAX.  coarse_cycle_ready() configures the kernel's shared-memory limit once and says
// whether it can run.
constexpr size_t CC_SMEM_MAX = 200 * 1024;
constexpr int CC_THREADS = 1024;
template <typename R>
bool coarse_cycle_ready();
template <typename R>
void launch_coarse_cycle(const CCycle<R>& cc, size_t smem_bytes, const cx<R>* b, cx<R>* e, cudaStream_t st,
                         const int* active);

// FP32 pre-smoothing from zero fused with the residual, one right-hand side (stencil.cu):
// u1 = (omega/d) b and r = b - M u1, u1 recomputed at the neighbours; same values as
// launch_smooth0 followed by launch_resid.
// The up-sweep of one level in one kernel (one right-hand side): out = u2 + (omega/d)(b - M u2)
// with u2 = u1 + P e (zchunk fine planes per CTA); dinv: an FP64 level's coefficient table
template <typename R, typename TB, typename TO>
void launch_up(const Grid& gf, const Grid& gc, double s_re, double s_im, double omega, const R* k2, const cx<R>* dinv,
               const cx<R>* u1, const cx<R>* e, const cx<TB>* b, cx<TO>* out, int zchunk, cudaStream_t st,
               const int* active);
// The residual b - M u1 of one level and its full-weighting restriction into bc in one kernel
// (one right-hand side, kchunk coarse planes per CTA); same values as launch_resid followed by
// launch_restrict.  dtab: an FP64 level's coefficient table.
template <typename R, typename TB>
void launch_rr(const Grid& gf, const Grid& gc, double s_re, double s_im, const R* k2, const cx<R>* dtab,
               const cx<R>* u1, const cx<TB>* b, cx<R>* bc, int kchunk, cudaStream_t st, const int* active);
// The FP32 down-sweep of one level in one kernel: u1 = (omega/d) b on the fine grid and the
// full-weighting restriction of b - M u1 into bc on the coarse grid (kchunk coarse planes per CTA)
template <typename TB>
void launch_down32(const Grid& gf, const Grid& gc, double s_re, double s_im, double omega, const float* k2,
                   const cx<TB>* b, z64* u1, z64* bc, int kchunk, cudaStream_t st, const int* active);
template <typename TB>
void launch_smooth0_resid32(const Grid& g, double s_re, double s_im, double omega, const float* k2, const cx<TB>* b,
                            z64* u1, z64* r, cudaStream_t st, const int* active);

// ---- IDR(s) (idrs.cu); part holds RED_STRIDE-strided slots of complex partial sums ----
void launch_idr_v(const IdrCtl* ic, int k, const z128* r, const z128* G, size_t n, z128* v, cudaStream_t st);
void launch_idr_u(const IdrCtl* ic, int k, const z128* vh, z128* U, size_t n, cudaStream_t st);
int launch_idr_pdots(int s, bool with_norm, const z128* P, const z128* y, size_t n, z128* part, cudaStream_t st,
                     const int* active);
int launch_idr_update(const IdrCtl* ic, int k, z128* G, z128* U, z128* r, z128* x, size_t n, z128* part,
                      cudaStream_t st);
int launch_idr_xr(int s, const IdrCtl* ic, const z128* P, z128* r, const z128* t, z128* x, const z128* vh, size_t n,
                  z128* part, cudaStream_t st);
void launch_idr_scalar(IdrCtl* ic, const z128* part, int nb, int stage, int k, double tol, int max_iter, double* hist,
                       int hist_len, cudaStream_t st);

// ---- Bi-CGSTAB (bicgstab.cu) ----
// part slot 0 = conj(a).b, slot 1 = conj(c).d (c may be NULL); returns the number of partials
int launch_dots2(const z128* a, const z128* b, const z128* c, const z128* d, size_t n, z128* part, cudaStream_t st,
                 const int* active);
void launch_bicg_p(const z128* r, z128* p, const z128* v, const BicgCtl* bc, size_t n, cudaStream_t st);
int launch_bicg_s(const z128* r, const z128* v, z128* s, const BicgCtl* bc, size_t n, z128* part, cudaStream_t st);
int launch_bicg_xr(z128* x, z128* r, const z128* ph, const z128* sh, const z128* s, const z128* t, const z128* rh,
                   const BicgCtl* bc, size_t n, z128* part, cudaStream_t st);
void launch_bicg_scalar(BicgCtl* bc, const z128* part, int nb, int stage, double tol, int max_iter, int stall,
                        double* hist, int hist_len, cudaStream_t st);
void launch_bicg_init(BicgCtl* bc, const z128* part, int nb, const z128* r, z128* rh, z128* p, z128* v, size_t n,
                      cudaStream_t st);

// ---- batched FGMRES kernels (krylov_batched.cu); vectors node-major, rhs innermost ----
int launch_bnorm2_part(const z128* x, size_t ne, int nb, double* part, cudaStream_t st, const int* active);
void launch_breduce_norm(const double* part, int nb, int nblk, double* out, cudaStream_t st, const int* active);
// Vs: the element sums Re V + Im V of a summed basis (three FP64 FMAs per complex
// multiply-add), or NULL for the textbook four-FMA form
int launch_bmdot(const z128* V, const double* Vs, size_t ld, int nv, const z128* w, size_t ne, int nb, z128* part,
                 int with_norm, cudaStream_t st, const int* active);
// decide_j >= 0: the second-pass test per right-hand side (need[r]); *pass2 = any, log[decide_j] =
// how many
void launch_breduce_dots(const z128* part, int nv, int nb, int nblk, z128* hpass, z128* hacc, int accumulate,
                         int decide_j, const int* act, int* pass2, int* log, double* sw2, int* need, cudaStream_t st,
                         const int* active, double keep);
// the second Gram-Schmidt pass for the right-hand sides with need[r] only (FP64; Vs: summed
// basis or NULL): inner products into part (k_bmdot's layout and grid; zeros for the others),
// and the update
int launch_bmdot_sel(const z128* V, const double* Vs, size_t ld, int nv, const z128* w, size_t ne, int nb,
                     const int* need, z128* part, cudaStream_t st, const int* active);
void launch_bgs_update_sel(const z128* V, const double* Vs, size_t ld, int nv, int nb, const z128* h, z128* w,
                           size_t ne, const int* need, cudaStream_t st, const int* active);
void launch_bgs_update(const z128* V, const double* Vs, size_t ld, int nv, int nb, const z128* h, z128* w, size_t ne,
                       cudaStream_t st, const int* active);
// out = in / s[r]; with outs, also the element sums Re out + Im out
void launch_bscale_inv(const z128* in, const double* s, z128* out, double* outs, size_t ne, int nb, cudaStream_t st,
                       const int* active);
// double-float Gram-Schmidt variants (basis and Arnoldi vector as zdf)
int launch_bnorm2_part_df(const zdf* x, size_t ne, int nb, double* part, cudaStream_t st, const int* active);
int launch_bmdot_df(const zdf* V, size_t ld, int nv, const zdf* w, size_t ne, int nb, z128* part, int with_norm,
                    cudaStream_t st, const int* active, int variant = 0);
void launch_bgs_update_df(const zdf* V, size_t ld, int nv, int nb, const z128* h, zdf* w, size_t ne, cudaStream_t st,
                          const int* active);
template <typename TI, typename TC>
void launch_bscale_df(const TI* in, const double* s, zdf* out, cx<TC>* copy, size_t ne, int nb, cudaStream_t st,
                      const int* active);
void launch_bcycle_init(BatchCtl* bc, int nb, int m, double tol, cudaStream_t st);
void launch_bgivens(BatchCtl* bc, int nb, int m, int j, const z128* hcol, const double* hnorm, double tol,
                    cudaStream_t st);
void launch_btrisolve(BatchCtl* bc, int nb, int m, cudaStream_t st);
template <typename TZ>
void launch_bxupdate(const BatchCtl* bc, int nb, int m, const cx<TZ>* Z, size_t ld, z128* x, size_t ne,
                     cudaStream_t st);
void launch_to_batch(const z128* src, z128* dst, size_t n, int nb, int nrhs, cudaStream_t st);
void launch_from_batch(const z128* src, z128* dst, size_t n, int nb, int nrhs, cudaStream_t st);

// ---- adjoint-state gradient (adjoint.cu) ----
// q = D^-1 conj(in), D = diag(2^-faces) (Sommerfeld) or I (Dirichlet); g.nb values per node
// (the batched layout); in == q allowed
void launch_adjoint_rhs(const Grid& g, const z128* in, z128* q, cudaStream_t st);
// x = conj(D x), g.nb values per node
void launch_adjoint_finish(const Grid& g, z128* x, cudaStream_t st);
// grad += -Re(conj(lam) (-1 - i nf / (h k)) u)
void launch_grad_k2(const Grid& g, const double* k2, const z128* u, const z128* lam, double* grad, cudaStream_t st);
// g(rec[r]) = u(rec[r]) - d[r]; partial sums of |u - d|^2 into part; returns the number of partials
int launch_receiver_residual(int nrec, const int* rec, const z128* u, const z128* d, z128* g, double* part,
                             cudaStream_t st);

}  // namespace helm
