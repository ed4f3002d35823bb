// adjoint.cu -- pointwise kernels of the adjoint-state gradient with respect to k^2.
//
// The operator of Sec. 2.4 with Sommerfeld ghost elimination is not symmetric, but D A is,
// with D = diag(2^-faces) (each eliminated face doubles one off-diagonal of the node's row).
// Hence A^T = D A D^-1 and A^H lambda = g is solved with the forward operator and the same
// preconditioned Krylov solver: A nu = D^-1 conj(g), lambda = conj(D nu).  For Dirichlet D = I.
//
// A depends on k^2_p only through its diagonal entry -k^2_p - i (2 k_p / h) nf_p, so for a real
// loss L with dL/d conj(u) = g:  dL/dk^2_p = -Re(conj(lambda_p) (-1 - i nf_p / (h k_p)) u_p).
#include "internal.cuh"

namespace helm {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ int faces_at(const Grid& g, size_t p) {
  if (g.bc != 1) return 0;
  const int i = (int)(p % g.N1);
  const int j = (int)((p / g.N1) % g.N2);
  const int k = (int)(p / ((size_t)g.N1 * g.N2));
  return (i == 0) + (i == g.N1 - 1) + (j == 0) + (j == g.N2 - 1) + (k == 0) + (k == g.N3 - 1);
}

// q = D^-1 conj(in) elementwise; g.nb values per node (node-major, right-hand side innermost).
// in and q may be the same buffer (each element is read, then written, by one thread).
__global__ void __launch_bounds__(NT) k_adjoint_rhs(Grid g, const z128* in, z128* q) {
  const size_t n = g.npts() * g.nb;
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < n; e += (size_t)gridDim.x * NT) {
    const double s = (double)(1 << faces_at(g, e / g.nb));  // D^-1, an exact power of two
    const z128 v = in[e];
    q[e] = mkc<double>(s * v.re, -s * v.im);
  }
}

// x = conj(D x) elementwise, g.nb values per node
__global__ void __launch_bounds__(NT) k_adjoint_finish(Grid g, z128* __restrict__ x) {
  const size_t n = g.npts() * g.nb;
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < n; e += (size_t)gridDim.x * NT) {
    const double s = 1.0 / (double)(1 << faces_at(g, e / g.nb));  // D, exact
    const z128 v = x[e];
    x[e] = mkc<double>(s * v.re, -s * v.im);
  }
}

__global__ void __launch_bounds__(NT)
    k_grad_k2(Grid g, const double* __restrict__ k2, const z128* __restrict__ u, const z128* __restrict__ lam,
              double* __restrict__ grad) {
  const size_t n = g.npts();
  const double ih = 1.0 / g.h;
  for (size_t p = blockIdx.x * (size_t)NT + threadIdx.x; p < n; p += (size_t)gridDim.x * NT) {
    const int nf = faces_at(g, p);
    const double beta = nf ? (double)nf * ih / sqrt(k2[p]) : 0.0;
    const z128 x = u[p], l = lam[p];
    // t = (-1 - i beta) x ; grad += -Re(conj(l) t)
    const double tre = -x.re + beta * x.im, tim = -x.im - beta * x.re;
    grad[p] -= l.re * tre + l.im * tim;
  }
}

// Residual at the receivers: g(rec[r]) = u(rec[r]) - d[r] (g zeroed beforehand; receiver
// indices distinct), and per-block partial sums of |u - d|^2.
__global__ void __launch_bounds__(NT)
    k_receiver_residual(int nrec, const int* __restrict__ rec, const z128* __restrict__ u, const z128* __restrict__ d,
                        z128* __restrict__ g, double* __restrict__ part) {
  __shared__ double sred[NT / 32];
  double s = 0.0;
  for (int r = blockIdx.x * NT + threadIdx.x; r < nrec; r += gridDim.x * NT) {
    const int q = rec[r];
    const z128 a = u[q], b = d[r];
    const z128 e = mkc<double>(a.re - b.re, a.im - b.im);
    g[q] = e;
    s = fma(e.re, e.re, s);
    s = fma(e.im, e.im, s);
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += sred[w];
    part[blockIdx.x] = t;
  }
}

int blocks_for(size_t n) {
  size_t b = (n + NT - 1) / NT;
  return (int)(b < 1216 ? (b > 0 ? b : 1) : 1216);
}

}  // namespace

void launch_adjoint_rhs(const Grid& g, const z128* in, z128* q, cudaStream_t st) {
  k_adjoint_rhs<<<blocks_for(g.npts() * g.nb), NT, 0, st>>>(g, in, q);
}
void launch_adjoint_finish(const Grid& g, z128* x, cudaStream_t st) {
  k_adjoint_finish<<<blocks_for(g.npts() * g.nb), NT, 0, st>>>(g, x);
}
void launch_grad_k2(const Grid& g, const double* k2, const z128* u, const z128* lam, double* grad, cudaStream_t st) {
  k_grad_k2<<<blocks_for(g.npts()), NT, 0, st>>>(g, k2, u, lam, grad);
}
int launch_receiver_residual(int nrec, const int* rec, const z128* u, const z128* d, z128* g, double* part,
                             cudaStream_t st) {
  const int nb = (nrec + NT - 1) / NT < 256 ? ((nrec + NT - 1) / NT > 0 ? (nrec + NT - 1) / NT : 1) : 256;
  k_receiver_residual<<<nb, NT, 0, st>>>(nrec, rec, u, d, g, part);
  return nb;
}

}  // namespace helm
