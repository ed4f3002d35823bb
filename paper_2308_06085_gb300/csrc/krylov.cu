// krylov.cu -- FP64 kernels of the right-preconditioned (flexible) GMRES(m) outer solver
// (Sec. 3.1-3.2): multi-vector inner products and updates for classical Gram-Schmidt with
// one reorthogonalisation pass, norms, and the Hessenberg least-squares problem solved by
// complex Givens rotations on the device, so the host never waits inside an Arnoldi step.
//
// Reductions are deterministic: a fixed grid of RED_BLOCKS blocks writes partial sums,
// combined by a second kernel in a fixed order.
#include "internal.cuh"

namespace helm {

namespace {

constexpr int NT = 256;
constexpr int NW = NT / 32;
constexpr int G = 8;  // basis vectors per pass of the inner-product kernel

__device__ __forceinline__ void block_range(size_t n, size_t& p0, size_t& p1) {
  const size_t chunk = (n + RED_BLOCKS - 1) / RED_BLOCKS;
  p0 = blockIdx.x * chunk;
  p1 = p0 + chunk < n ? p0 + chunk : n;
}

__global__ void __launch_bounds__(NT)
    k_mdot(const z128* __restrict__ V, size_t ld, int nv, const z128* __restrict__ w, size_t n,
           z128* __restrict__ part, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ double sred[NW][2 * G];
  size_t p0, p1;
  block_range(n, p0, p1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* partd = reinterpret_cast<double*>(part);
  for (int g0 = 0; g0 < nv; g0 += G) {
    double re[G], im[G];
#pragma unroll
    for (int q = 0; q < G; ++q) re[q] = im[q] = 0.0;
    for (size_t p = p0 + threadIdx.x; p < p1; p += NT) {
      const z128 wv = ldg(w + p);
#pragma unroll
      for (int q = 0; q < G; ++q)
        if (g0 + q < nv) cdot_acc(ldg(V + (size_t)(g0 + q) * ld + p), wv, re[q], im[q]);
    }
#pragma unroll
    for (int q = 0; q < G; ++q)
      for (int o = 16; o; o >>= 1) {
        re[q] += __shfl_xor_sync(0xffffffffu, re[q], o);
        im[q] += __shfl_xor_sync(0xffffffffu, im[q], o);
      }
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < G; ++q) {
        sred[warp][2 * q] = re[q];
        sred[warp][2 * q + 1] = im[q];
      }
    __syncthreads();
    if (threadIdx.x < 2 * G) {
      const int q = threadIdx.x >> 1, comp = threadIdx.x & 1;
      double s = 0.0;
      for (int wi = 0; wi < NW; ++wi) s += sred[wi][threadIdx.x];
      if (g0 + q < nv) partd[2 * ((size_t)(g0 + q) * RED_BLOCKS + blockIdx.x) + comp] = s;
    }
    __syncthreads();
  }
}

// One warp per basis vector: lanes sum the RED_BLOCKS partials in a fixed order.
__global__ void __launch_bounds__(NT)
    k_reduce_dots(const z128* __restrict__ part, int nv, z128* __restrict__ hpass, z128* __restrict__ hacc,
                  int accumulate, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < nv; i += NW) {
    double re = 0.0, im = 0.0;
    for (int b = lane; b < RED_BLOCKS; b += 32) {
      const z128 v = part[(size_t)i * RED_BLOCKS + b];
      re += v.re;
      im += v.im;
    }
    for (int o = 16; o; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
      hpass[i] = mkc<double>(re, im);
      if (accumulate) {
        hacc[i].re += re;
        hacc[i].im += im;
      } else {
        hacc[i] = mkc<double>(re, im);
      }
    }
  }
}

__global__ void __launch_bounds__(NT)
    k_gs_update(const z128* __restrict__ V, size_t ld, int nv, const z128* __restrict__ h, z128* __restrict__ w,
                size_t n, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ z128 sh[MAX_BASIS];
  for (int i = threadIdx.x; i < nv; i += NT) sh[i] = h[i];
  __syncthreads();
  for (size_t p = blockIdx.x * (size_t)NT + threadIdx.x; p < n; p += (size_t)gridDim.x * NT) {
    z128 acc = w[p];
    for (int i = 0; i < nv; ++i) {
      const z128 v = ldg(V + (size_t)i * ld + p);
      const z128 c = sh[i];
      acc.re = fma(-c.re, v.re, acc.re);
      acc.re = fma(c.im, v.im, acc.re);
      acc.im = fma(-c.re, v.im, acc.im);
      acc.im = fma(-c.im, v.re, acc.im);
    }
    w[p] = acc;
  }
}

__global__ void __launch_bounds__(NT)
    k_norm2_part(const z128* __restrict__ x, size_t n, double* __restrict__ part, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ double sred[NW];
  size_t p0, p1;
  block_range(n, p0, p1);
  double s = 0.0;
  for (size_t p = p0 + threadIdx.x; p < p1; p += NT) {
    const z128 v = ldg(x + p);
    s = fma(v.re, v.re, s);
    s = fma(v.im, v.im, s);
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int wi = 0; wi < NW; ++wi) t += sred[wi];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(NT)
    k_reduce_norm(const double* __restrict__ part, double* __restrict__ out, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ double sred[NW];
  double s = 0.0;
  for (int b = threadIdx.x; b < RED_BLOCKS; b += NT) s += part[b];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int wi = 0; wi < NW; ++wi) t += sred[wi];
    *out = sqrt(t);
  }
}

__global__ void __launch_bounds__(NT)
    k_scale_inv(const z128* __restrict__ in, const double* __restrict__ s, z128* __restrict__ out, size_t n,
                const int* __restrict__ active) {
  if (active && *active == 0) return;
  const double d = *s;
  if (!(d != 0.0)) return;
  const double inv = 1.0 / d;
  for (size_t p = blockIdx.x * (size_t)NT + threadIdx.x; p < n; p += (size_t)gridDim.x * NT) {
    const z128 v = in[p];
    out[p] = mkc<double>(v.re * inv, v.im * inv);
  }
}

__global__ void k_cycle_init(KrylovCtl* ctl, z128* g, int m, int iter0) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->active = 1;
    ctl->jend = -1;
    ctl->flag = 0;
    ctl->iter0 = iter0;
    ctl->est = ctl->beta / ctl->bnorm;
  }
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = mkc<double>(i == 0 ? ctl->beta : 0.0, 0.0);
}

// Arnoldi step j of the least-squares update: column j of H gets the previous rotations,
// then a new rotation (c real, s complex) that zeroes H(j+1, j):
//   c = |a| / t, s = (a / |a|) conj(b) / t, H(j, j) = (a / |a|) t, t = sqrt(|a|^2 + |b|^2),
// and the right-hand side g picks up g(j+1) = -conj(s) g(j), g(j) = c g(j).  |g(j+1)| is
// the residual norm of the current GMRES iterate (right preconditioning: the true residual).
__global__ void k_givens(KrylovCtl* ctl, z128* H, int m, int j, int jmax, const z128* __restrict__ hcol,
                         const double* __restrict__ hnorm, double* cs, z128* sn, z128* g, double tol, double* hist,
                         int hist_len) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (ctl->active == 0) return;
  for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
  const double hn = *hnorm;
  H[(size_t)(j + 1) * m + j] = mkc<double>(hn, 0.0);
  for (int i = 0; i < j; ++i) {
    const z128 a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
    const double c = cs[i];
    const z128 s = sn[i];
    // H(i) = c a + s b ; H(i+1) = -conj(s) a + c b
    const z128 sb = cmul(s, b);
    const z128 cs_a = mkc<double>(-s.re, s.im);  // -conj(s)
    const z128 t = cmul(cs_a, a);
    H[(size_t)i * m + j] = mkc<double>(c * a.re + sb.re, c * a.im + sb.im);
    H[(size_t)(i + 1) * m + j] = mkc<double>(t.re + c * b.re, t.im + c * b.im);
  }
  const z128 a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
  const double na = hypot(a.re, a.im), nb = hypot(b.re, b.im);
  const double t = hypot(na, nb);
  double c;
  z128 s;
  if (na == 0.0) {
    c = 0.0;
    s = mkc<double>(1.0, 0.0);
    H[(size_t)j * m + j] = b;
  } else {
    const z128 ph = mkc<double>(a.re / na, a.im / na);
    c = na / t;
    s = cmul(ph, mkc<double>(b.re / t, -b.im / t));
    H[(size_t)j * m + j] = mkc<double>(ph.re * t, ph.im * t);
  }
  H[(size_t)(j + 1) * m + j] = mkc<double>(0.0, 0.0);
  cs[j] = c;
  sn[j] = s;
  const z128 gj = g[j];
  const z128 ms = mkc<double>(-s.re, s.im);  // -conj(s)
  g[j + 1] = cmul(ms, gj);
  g[j] = mkc<double>(c * gj.re, c * gj.im);
  const double est = hypot(g[j + 1].re, g[j + 1].im) / ctl->bnorm;
  ctl->est = est;
  ctl->jend = j;
  const int it = ctl->iter0 + j;
  if (hist && it < hist_len) hist[it] = est;
  if (!isfinite(est) || !isfinite(hn)) {
    ctl->flag = 2;
    ctl->active = 0;
  } else if (est <= tol) {
    ctl->flag = 1;
    ctl->active = 0;
  } else if (j + 1 >= jmax) {
    ctl->active = 0;
  }
}

__global__ void k_trisolve(const KrylovCtl* ctl, const z128* H, int m, const z128* g, z128* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = ctl->jend + 1;
  for (int i = k - 1; i >= 0; --i) {
    z128 s = g[i];
    for (int q = i + 1; q < k; ++q) {
      const z128 hy = cmul(H[(size_t)i * m + q], y[q]);
      s.re -= hy.re;
      s.im -= hy.im;
    }
    const z128 d = H[(size_t)i * m + i];
    const double dd = d.re * d.re + d.im * d.im;
    y[i] = mkc<double>((s.re * d.re + s.im * d.im) / dd, (s.im * d.re - s.re * d.im) / dd);
  }
}

template <typename TZ>
__global__ void __launch_bounds__(NT)
    k_xupdate(const KrylovCtl* __restrict__ ctl, const cx<TZ>* __restrict__ Z, size_t ld, const z128* __restrict__ y,
              z128* __restrict__ x, size_t n) {
  __shared__ z128 sy[MAX_BASIS];
  const int k = ctl->jend + 1;
  for (int i = threadIdx.x; i < k; i += NT) sy[i] = y[i];
  __syncthreads();
  for (size_t p = blockIdx.x * (size_t)NT + threadIdx.x; p < n; p += (size_t)gridDim.x * NT) {
    z128 acc = x[p];
    for (int i = 0; i < k; ++i) acc = cfma(sy[i], cvt<double>(ldg(Z + (size_t)i * ld + p)), acc);
    x[p] = acc;
  }
}

__global__ void __launch_bounds__(NT)
    k_combine(const KrylovCtl* __restrict__ ctl, const z128* __restrict__ V, size_t ld, const z128* __restrict__ y,
              z128* __restrict__ w, size_t n) {
  __shared__ z128 sy[MAX_BASIS];
  const int k = ctl->jend + 1;
  for (int i = threadIdx.x; i < k; i += NT) sy[i] = y[i];
  __syncthreads();
  for (size_t p = blockIdx.x * (size_t)NT + threadIdx.x; p < n; p += (size_t)gridDim.x * NT) {
    z128 acc = mkc<double>(0.0, 0.0);
    for (int i = 0; i < k; ++i) acc = cfma(sy[i], ldg(V + (size_t)i * ld + p), acc);
    w[p] = acc;
  }
}

__global__ void k_c128_to_c64(const z128* __restrict__ a, z64* __restrict__ b, size_t n) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    b[p] = cvt<float>(a[p]);
}
__global__ void k_c64_to_c128(const z64* __restrict__ a, z128* __restrict__ b, size_t n) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    b[p] = cvt<double>(a[p]);
}
__global__ void k_set_active(KrylovCtl* ctl, int v) { ctl->active = v; }
__global__ void k_axpy1(const z128* __restrict__ z, z128* __restrict__ x, size_t n) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const z128 a = z[p], b = x[p];
    x[p] = mkc<double>(a.re + b.re, a.im + b.im);
  }
}

int stream_blocks(size_t n) {
  size_t b = (n + NT - 1) / NT;
  const size_t cap = 152 * 8;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

void launch_mdot(const z128* V, size_t ld, int nv, const z128* w, size_t n, z128* part, cudaStream_t st,
                 const int* active) {
  k_mdot<<<RED_BLOCKS, NT, 0, st>>>(V, ld, nv, w, n, part, active);
}
void launch_reduce_dots(const z128* part, int nv, z128* hpass, z128* hacc, int accumulate, cudaStream_t st,
                        const int* active) {
  k_reduce_dots<<<1, NT, 0, st>>>(part, nv, hpass, hacc, accumulate, active);
}
void launch_gs_update(const z128* V, size_t ld, int nv, const z128* h, z128* w, size_t n, cudaStream_t st,
                      const int* active) {
  k_gs_update<<<stream_blocks(n), NT, 0, st>>>(V, ld, nv, h, w, n, active);
}
void launch_norm2_part(const z128* x, size_t n, double* partr, cudaStream_t st, const int* active) {
  k_norm2_part<<<RED_BLOCKS, NT, 0, st>>>(x, n, partr, active);
}
void launch_reduce_norm(const double* partr, double* out, cudaStream_t st, const int* active) {
  k_reduce_norm<<<1, NT, 0, st>>>(partr, out, active);
}
void launch_scale_inv(const z128* in, const double* s, z128* out, size_t n, cudaStream_t st, const int* active) {
  k_scale_inv<<<stream_blocks(n), NT, 0, st>>>(in, s, out, n, active);
}
void launch_cycle_init(KrylovCtl* ctl, z128* gvec, int m, int iter0, cudaStream_t st) {
  k_cycle_init<<<1, 256, 0, st>>>(ctl, gvec, m, iter0);
}
void launch_givens(KrylovCtl* ctl, z128* H, int m, int j, int jmax, const z128* hcol, const double* hnorm, double* cs,
                   z128* sn, z128* gvec, double tol, double* hist, int hist_len, cudaStream_t st) {
  k_givens<<<1, 32, 0, st>>>(ctl, H, m, j, jmax, hcol, hnorm, cs, sn, gvec, tol, hist, hist_len);
}
void launch_trisolve(const KrylovCtl* ctl, const z128* H, int m, const z128* gvec, z128* y, cudaStream_t st) {
  k_trisolve<<<1, 32, 0, st>>>(ctl, H, m, gvec, y);
}
template <typename TZ>
void launch_xupdate(const KrylovCtl* ctl, const cx<TZ>* Z, size_t ld, const z128* y, z128* x, size_t n,
                    cudaStream_t st) {
  k_xupdate<TZ><<<stream_blocks(n), NT, 0, st>>>(ctl, Z, ld, y, x, n);
}
template void launch_xupdate<double>(const KrylovCtl*, const z128*, size_t, const z128*, z128*, size_t, cudaStream_t);
template void launch_xupdate<float>(const KrylovCtl*, const z64*, size_t, const z128*, z128*, size_t, cudaStream_t);
void launch_combine(const KrylovCtl* ctl, const z128* V, size_t ld, const z128* y, z128* w, size_t n,
                    cudaStream_t st) {
  k_combine<<<stream_blocks(n), NT, 0, st>>>(ctl, V, ld, y, w, n);
}
void launch_c128_to_c64(const z128* a, z64* b, size_t n, cudaStream_t st) {
  k_c128_to_c64<<<stream_blocks(n), NT, 0, st>>>(a, b, n);
}
void launch_c64_to_c128(const z64* a, z128* b, size_t n, cudaStream_t st) {
  k_c64_to_c128<<<stream_blocks(n), NT, 0, st>>>(a, b, n);
}
void launch_set_active(KrylovCtl* ctl, int v, cudaStream_t st) { k_set_active<<<1, 1, 0, st>>>(ctl, v); }
void launch_axpy1(const z128* z, z128* x, size_t n, cudaStream_t st) {
  k_axpy1<<<stream_blocks(n), NT, 0, st>>>(z, x, n);
}

}  // namespace helm
