// internal.cuh -- launchers shared between the translation units of libhelm.
#pragma once

#include "common.cuh"

namespace helm {

// ---- grid kernels (stencil.cu) ----
template <typename R, typename TU, typename TO>
void launch_apply(const Grid& g, double s_re, double s_im, const R* k2, const cx<TU>* u, cx<TO>* v, cudaStream_t st,
                  const int* active);
template <typename R, typename TU, typename TB, typename TO>
void launch_resid(const Grid& g, double s_re, double s_im, const R* k2, const cx<TU>* u, const cx<TB>* b, cx<TO>* out,
                  cudaStream_t st, const int* active);
template <typename R, typename TB, typename TO>
void launch_jacobi(const Grid& g, double s_re, double s_im, double omega, const R* k2, const cx<R>* dinv,
                   const cx<R>* u, const cx<TB>* b, cx<TO>* out, cudaStream_t st, const int* active);
template <typename R, typename TB>
void launch_smooth0(const Grid& g, double s_re, double s_im, double omega, const R* k2, const cx<R>* dinv,
                    const cx<TB>* b, cx<R>* out, cudaStream_t st, const int* active);
template <typename R>
void launch_restrict(const Grid& gf, const Grid& gc, const cx<R>* r, cx<R>* out, cudaStream_t st, const int* active);
template <typename R>
void launch_prolong_add(const Grid& gf, const Grid& gc, const cx<R>* u1, const cx<R>* e, cx<R>* out, cudaStream_t st,
                        const int* active);
template <typename TI, typename TO>
void launch_coarse(int nc, const z128* Minv, const cx<TI>* b, cx<TO>* e, cudaStream_t st, const int* active);
void launch_dinv(const Grid& g, double s_re, double s_im, double omega, const double* k2, z128* out, cudaStream_t st);
void launch_inject(const Grid& gf, const Grid& gc, const double* kf, double* kc, cudaStream_t st);
void launch_to_float(const double* a, float* b, size_t n, cudaStream_t st);
void launch_check_k2(const double* a, size_t n, int* bad, cudaStream_t st);
void launch_rhs_point(const Grid& g, int nsrc, const int* idx, double amp, z128* b, cudaStream_t st);

// ---- Krylov kernels (krylov.cu) ----
constexpr int RED_BLOCKS = 608;  // fixed grid for reductions: partial sums combine in a fixed order
constexpr int MAX_BASIS = 257;   // restart <= 256

// part[i * RED_BLOCKS + blk] = sum over blk's points of conj(V_i) w, i < nv
void launch_mdot(const z128* V, size_t ld, int nv, const z128* w, size_t n, z128* part, cudaStream_t st,
                 const int* active);
// hpass[i] = sum_blk part[i * RED_BLOCKS + blk]; hacc[i] = hpass[i] (accumulate 0) or += (1)
void launch_reduce_dots(const z128* part, int nv, z128* hpass, z128* hacc, int accumulate, cudaStream_t st,
                        const int* active);
// w -= sum_i h[i] V_i
void launch_gs_update(const z128* V, size_t ld, int nv, const z128* h, z128* w, size_t n, cudaStream_t st,
                      const int* active);
// partial sums of |x|^2 into partr[RED_BLOCKS]
void launch_norm2_part(const z128* x, size_t n, double* partr, cudaStream_t st, const int* active);
// *out = sqrt(sum partr)
void launch_reduce_norm(const double* partr, double* out, cudaStream_t st, const int* active);
// out = in * (1 / *s)   (when *s != 0)
void launch_scale_inv(const z128* in, const double* s, z128* out, size_t n, cudaStream_t st, const int* active);
// start a restart cycle: active = 1, g = (beta, 0, ...), iter0 recorded
void launch_cycle_init(KrylovCtl* ctl, z128* gvec, int m, int iter0, cudaStream_t st);
// Arnoldi step j: rotations on H(:, j) (column stored at Hcol), new rotation, g update,
// estimate, stopping flags; writes hist[iter0 + j]
void launch_givens(KrylovCtl* ctl, z128* H, int m, int j, int jmax, const z128* hcol, const double* hnorm,
                   double* cs, z128* sn, z128* gvec, double tol, double* hist, int hist_len, cudaStream_t st);
// y = H(0:k, 0:k)^{-1} g with k = jend + 1
void launch_trisolve(const KrylovCtl* ctl, const z128* H, int m, const z128* gvec, z128* y, cudaStream_t st);
// x += sum_{i<=jend} y_i Z_i   (Z c128 or c64)
template <typename TZ>
void launch_xupdate(const KrylovCtl* ctl, const cx<TZ>* Z, size_t ld, const z128* y, z128* x, size_t n,
                    cudaStream_t st);
// w = sum_{i<=jend} y_i V_i
void launch_combine(const KrylovCtl* ctl, const z128* V, size_t ld, const z128* y, z128* w, size_t n,
                    cudaStream_t st);
void launch_c128_to_c64(const z128* a, z64* b, size_t n, cudaStream_t st);
void launch_c64_to_c128(const z64* a, z128* b, size_t n, cudaStream_t st);
void launch_set_active(KrylovCtl* ctl, int v, cudaStream_t st);
// x += z
void launch_axpy1(const z128* z, z128* x, size_t n, cudaStream_t st);

}  // namespace helm
