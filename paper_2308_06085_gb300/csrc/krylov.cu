// krylov.cu -- FP64 kernels of the right-preconditioned (flexible) GMRES(m) outer solver
// (Sec. 3.1-3.2): multi-vector inner products and updates for classical Gram-Schmidt with
// one reorthogonalisation pass, norms, and the Hessenberg least-squares problem solved by
// complex Givens rotations on the device, so the host never waits inside an Arnoldi step.
//
// Reductions are deterministic: a grid of exactly one wave (SMs x resident blocks, fixed for
// a device) writes partial sums, combined by a second kernel in a fixed order.
#include "internal.cuh"

namespace helm {

namespace {

constexpr int NT = 256;
constexpr int NW = NT / 32;

__device__ __forceinline__ void block_range(size_t n, size_t& p0, size_t& p1) {
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  p0 = blockIdx.x * chunk;
  p1 = p0 + chunk < n ? p0 + chunk : n;
}

// ---- inner products conj(V_i) . w of nv basis vectors against one vector --------------------
// A block stages tiles of w in shared memory; each warp owns "slots" (a basis vector, or the
// extra slot nv for |w|^2 when with_norm is set).  With fewer slots than warps, several
// consecutive warps share a slot and split the tile's points.  A lane accumulates its slots
// over all the block's points, so the per-slot epilogue (warp reduction) is amortised over
// ~50-100 points per lane.  Partials per block go to part[slot * RED_STRIDE + block].
constexpr int KS = 4;  // slots per warp per pass over the block's points

struct AccD {  // FP64 accumulator, four FMAs per complex multiply-add
  static constexpr bool kBalanced = false;
  static constexpr bool kSums = false;
  double re, im;
  __device__ void zero() { re = im = 0.0; }
  __device__ void mac(const z128& v, const z128& w) { cdot_acc(v, w, re, im); }
  __device__ void norm(const z128& w) {
    re = fma(w.re, w.re, re);
    re = fma(w.im, w.im, re);
  }
  __device__ void reduce_warp(double& r, double& i) {
    r = re;
    i = im;
    for (int o = 16; o; o >>= 1) {
      r += __shfl_xor_sync(0xffffffffu, r, o);
      i += __shfl_xor_sync(0xffffffffu, i, o);
    }
  }
};

__device__ __forceinline__ void df_shfl_reduce(float& s, float& c) {
  for (int o = 16; o; o >>= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, s, o), oc = __shfl_xor_sync(0xffffffffu, c, o);
    float hi, lo;
    df_add(s, c, os, oc, hi, lo);
    s = hi;
    c = lo;
  }
}

struct AccF {  // double-float accumulator, FP32 arithmetic only
  static constexpr bool kBalanced = true;
  static constexpr bool kSums = false;
  float rs, rc, is, ic;
  __device__ void zero() { rs = rc = is = ic = 0.f; }
  __device__ void mac(const zdf& v, const zdf& w) {
    // re += vr wr + vi wi ; im += vr wi - vi wr
    df_mac(v.rh, v.rl, w.rh, w.rl, rs, rc);
    df_mac(v.ih, v.il, w.ih, w.il, rs, rc);
    df_mac(v.rh, v.rl, w.ih, w.il, is, ic);
    df_mac(-v.ih, -v.il, w.rh, w.rl, is, ic);
  }
  __device__ void norm(const zdf& w) {
    df_mac(w.rh, w.rl, w.rh, w.rl, rs, rc);
    df_mac(w.ih, w.il, w.ih, w.il, rs, rc);
  }
  __device__ void reduce_warp(double& r, double& i) {
    float a = rs, b = rc, x = is, y = ic;
    df_renorm(a, b, a, b);
    df_renorm(x, y, x, y);
    df_shfl_reduce(a, b);
    df_shfl_reduce(x, y);
    r = (double)a + (double)b;
    i = (double)x + (double)y;
  }
};

// FP64 accumulator against a basis stored with its element sums s = Re v + Im v: with
// A = sum vr wr, B = sum vi wi and C = sum s (wi - wr),
//   conj(v) . w = (A + B) + i (C + A - B),
// since s (wi - wr) = vr wi - vi wr - (vr wr - vi wi).  Three FMAs per element and slot; the
// difference wi - wr is formed once per element of w and shared by all slots.
struct AccD3 {
  static constexpr bool kBalanced = false;
  static constexpr bool kSums = true;
  double a, b, c;
  __device__ void zero() { a = b = c = 0.0; }
  __device__ void mac3(const z128& v, double sv, const z128& w, double wd) {
    a = fma(v.re, w.re, a);
    b = fma(v.im, w.im, b);
    c = fma(sv, wd, c);
  }
  __device__ void norm(const z128& w) {
    a = fma(w.re, w.re, a);
    b = fma(w.im, w.im, b);
  }
  __device__ void reduce_warp(double& r, double& i) {
    r = a + b;
    i = c + (a - b);
    for (int o = 16; o; o >>= 1) {
      r += __shfl_xor_sync(0xffffffffu, r, o);
      i += __shfl_xor_sync(0xffffffffu, i, o);
    }
  }
};

// One slot's multiply-add: the plain accumulators read V alone, AccD3 also the sums Vs.
template <typename ACC, typename E>
__device__ __forceinline__ void slot_mac(ACC& acc, const E* __restrict__ V, const double* __restrict__ Vs, size_t off,
                                         const E& w, double wd) {
  if constexpr (ACC::kSums) acc.mac3(ldg(V + off), ldg(Vs + off), w, wd);
  else acc.mac(ldg(V + off), w);
}
__device__ __forceinline__ double w_diff(const z128& w) { return w.im - w.re; }
__device__ __forceinline__ double w_diff(const zdf&) { return 0.0; }

// Warps sharing one slot: the groups of NW / wps warps take the slots round-robin, so the
// busiest group holds ceil(nslot / groups) of them.  Take the least sharing that leaves at most
// 1/8 of the warp-slots idle: less sharing means more points per lane between warp reductions,
// and fewer idle warps means more loads in flight.
__device__ __forceinline__ int share_width(int nslot) {
  for (int wps = 1; wps < NW; wps <<= 1) {
    const int groups = NW / wps;
    const int cap = (nslot + groups - 1) / groups * groups;
    if (8 * (cap - nslot) <= cap) return wps;
  }
  return NW;
}

// TILE points of w per shared-memory tile (16 KB, and 8 KB more for wi - wr with the summed
// basis): few barriers per point keep loads in flight.
// STAGE: w passes through shared memory tile by tile (two barriers per tile); without it each
// warp reads w itself (the block's warps share it through L1) and runs barrier-free.
template <typename E, typename ACC, int TILE, int KSV = KS, bool STAGE = true>
__global__ void __launch_bounds__(NT)
    k_mdot(const E* __restrict__ V, const double* __restrict__ Vs, size_t ld, int nv, const E* __restrict__ w, size_t n,
           z128* __restrict__ part, int with_norm, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ E sw[TILE];
  __shared__ double swd[ACC::kSums ? TILE : 1];  // wi - wr of the staged points (summed basis)
  __shared__ double sred[NW][2];
  size_t p0, p1;
  block_range(n, p0, p1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nslot = nv + (with_norm ? 1 : 0);
  // warps sharing one slot: FP64 accumulation is bound by FP64 issue, where the least sharing
  // (longest runs between reductions) is fastest; double-float accumulation is bound by
  // latency, where evenly loaded warps keep more loads in flight
  const int wps = ACC::kBalanced ? share_width(nslot) : (nslot >= NW ? 1 : NW / nslot);
  const int sub = warp % wps, sfirst = warp / wps, sstep = NW / wps;
  double* partd = reinterpret_cast<double*>(part);
  for (int sbase = 0; sbase * sstep < nslot; sbase += KSV) {
    ACC acc[KSV];
#pragma unroll
    for (int k = 0; k < KSV; ++k) acc[k].zero();
    if (STAGE) {
      for (size_t t0 = p0; t0 < p1; t0 += TILE) {
        const int tn = (int)min((size_t)TILE, p1 - t0);
        __syncthreads();
        for (int q = threadIdx.x; q < tn; q += NT) {
          const E wv = ldg(w + t0 + q);
          sw[q] = wv;
          if (ACC::kSums) swd[q] = w_diff(wv);  // once per point, not once per warp
        }
        __syncthreads();
#pragma unroll 2
        for (int q = sub * 32 + lane; q < tn; q += 32 * wps) {
          const E wv = sw[q];
          const double wd = ACC::kSums ? swd[q] : 0.0;
#pragma unroll
          for (int k = 0; k < KSV; ++k) {
            const int sl = sfirst + (sbase + k) * sstep;
            if (sl < nv) slot_mac(acc[k], V, Vs, (size_t)sl * ld + t0 + q, wv, wd);
            else if (sl == nv && with_norm) acc[k].norm(wv);
          }
        }
      }
    } else {
#pragma unroll 2
      for (size_t q = p0 + sub * 32 + lane; q < p1; q += 32 * wps) {
        const E wv = ldg(w + q);
        const double wd = ACC::kSums ? w_diff(wv) : 0.0;
#pragma unroll
        for (int k = 0; k < KSV; ++k) {
          const int sl = sfirst + (sbase + k) * sstep;
          if (sl < nv) slot_mac(acc[k], V, Vs, (size_t)sl * ld + q, wv, wd);
          else if (sl == nv && with_norm) acc[k].norm(wv);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KSV; ++k) {
      const int sl = sfirst + (sbase + k) * sstep;
      double r, i;
      acc[k].reduce_warp(r, i);
      __syncthreads();
      if (lane == 0) {
        sred[warp][0] = r;
        sred[warp][1] = i;
      }
      __syncthreads();
      if (sub == 0 && lane == 0 && sl < nslot) {
        double tr = 0.0, ti = 0.0;
        for (int u = 0; u < wps; ++u) {
          tr += sred[warp + u][0];
          ti += sred[warp + u][1];
        }
        partd[2 * ((size_t)sl * RED_STRIDE + blockIdx.x)] = tr;
        partd[2 * ((size_t)sl * RED_STRIDE + blockIdx.x) + 1] = sl == nv ? 0.0 : ti;
      }
    }
  }
}

// One warp per basis vector: lanes sum the nb partials in a fixed order.
// decide_j >= 0 (first pass): slot nv holds partial |w|^2; the block then applies the
// Daniel-Gragg-Kaufman-Stewart test -- a second pass is needed when the projection kept less
// than `keep` of |w|^2 (|w - V h|^2 = |w|^2 - |h|^2 < keep |w|^2) -- and records the
// decision in *pass2 and log[decide_j].
__global__ void __launch_bounds__(NT)
    k_reduce_dots(const z128* __restrict__ part, int nv, int nb, z128* __restrict__ hpass, z128* __restrict__ hacc,
                  int accumulate, int decide_j, int* __restrict__ pass2, int* __restrict__ log,
                  const int* __restrict__ active, double keep) {
  if (active && *active == 0) return;
  __shared__ double sw2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nsum = decide_j >= 0 ? nv + 1 : nv;
  for (int i = warp; i < nsum; i += NW) {
    double re = 0.0, im = 0.0;
    for (int b = lane; b < nb; b += 32) {
      const z128 v = part[(size_t)i * RED_STRIDE + b];
      re += v.re;
      im += v.im;
    }
    for (int o = 16; o; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
      if (i == nv) {
        sw2 = re;
      } else {
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
  if (decide_j < 0) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    double h2 = 0.0;
    for (int i = 0; i < nv; ++i) h2 += hpass[i].re * hpass[i].re + hpass[i].im * hpass[i].im;
    const int again = !(sw2 - h2 >= keep * sw2);  // NaN also takes the second pass
    *pass2 = again;
    log[decide_j] = again;
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

// w -= sum_i h_i v_i against the summed basis: with P = sum hr vr, Q = sum hi vi and
// R = sum (hr + hi) s,  h v = (P - Q) + i (R - P - Q) summed over i, three FMAs per element
// and basis vector (hr + hi is formed once per vector).
__global__ void __launch_bounds__(NT)
    k_gs_update_sums(const z128* __restrict__ V, const double* __restrict__ Vs, size_t ld, int nv,
                     const z128* __restrict__ h, z128* __restrict__ w, size_t n, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ double3 sh[MAX_BASIS];
  for (int i = threadIdx.x; i < nv; i += NT) {
    const z128 c = h[i];
    sh[i] = make_double3(c.re, c.im, c.re + c.im);
  }
  __syncthreads();
  for (size_t p = blockIdx.x * (size_t)NT + threadIdx.x; p < n; p += (size_t)gridDim.x * NT) {
    double P = 0.0, Q = 0.0, R = 0.0;
    for (int i = 0; i < nv; ++i) {
      const size_t off = (size_t)i * ld + p;
      const z128 v = ldg(V + off);
      const double sv = ldg(Vs + off);
      const double3 c = sh[i];
      P = fma(c.x, v.re, P);
      Q = fma(c.y, v.im, Q);
      R = fma(c.z, sv, R);
    }
    const z128 a = w[p];
    w[p] = mkc<double>(a.re - (P - Q), a.im - (R - (P + Q)));
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
    k_reduce_norm(const double* __restrict__ part, int nb, double* __restrict__ out, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ double sred[NW];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += NT) s += part[b];
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

// out = in / *s, and outs = Re out + Im out (the element sums of a summed basis vector).
__global__ void __launch_bounds__(NT)
    k_scale_inv_sums(const z128* __restrict__ in, const double* __restrict__ s, z128* __restrict__ out,
                     double* __restrict__ outs, size_t n, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const double d = *s;
  if (!(d != 0.0)) return;
  const double inv = 1.0 / d;
  for (size_t p = blockIdx.x * (size_t)NT + threadIdx.x; p < n; p += (size_t)gridDim.x * NT) {
    const z128 v = in[p];
    const z128 o = mkc<double>(v.re * inv, v.im * inv);
    out[p] = o;
    outs[p] = o.re + o.im;
  }
}

__global__ void k_cycle_init(KrylovCtl* ctl, z128* g, int m, int iter0) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->active = 1;
    ctl->pass2 = 0;
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
  // one warp: the column and the previous rotations are staged in shared memory so the
  // sequential part runs on on-chip data only
  __shared__ z128 col[MAX_BASIS + 1];
  __shared__ z128 ssn[MAX_BASIS];
  __shared__ double scs[MAX_BASIS];
  if (blockIdx.x != 0) return;
  if (ctl->active == 0) return;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = hcol[i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    scs[i] = cs[i];
    ssn[i] = sn[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double hn = *hnorm;
    col[j + 1] = mkc<double>(hn, 0.0);
    for (int i = 0; i < j; ++i) {
      const z128 a = col[i], b = col[i + 1];
      const double c = scs[i];
      const z128 s = ssn[i];
      // H(i) = c a + s b ; H(i+1) = -conj(s) a + c b
      const z128 sb = cmul(s, b);
      const z128 t = cmul(mkc<double>(-s.re, s.im), a);
      col[i] = mkc<double>(c * a.re + sb.re, c * a.im + sb.im);
      col[i + 1] = mkc<double>(t.re + c * b.re, t.im + c * b.im);
    }
    const z128 a = col[j], b = col[j + 1];
    const double na = hypot(a.re, a.im), nb = hypot(b.re, b.im);
    const double t = hypot(na, nb);
    double c;
    z128 s;
    if (na == 0.0) {
      c = 0.0;
      s = mkc<double>(1.0, 0.0);
      col[j] = b;
    } else {
      const z128 ph = mkc<double>(a.re / na, a.im / na);
      c = na / t;
      s = cmul(ph, mkc<double>(b.re / t, -b.im / t));
      col[j] = mkc<double>(ph.re * t, ph.im * t);
    }
    col[j + 1] = mkc<double>(0.0, 0.0);
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
    if (ctl->active == 0) ctl->pass2 = 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) H[(size_t)i * m + j] = col[i];
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

// x += sum_i y_i z_i for complex64 z_i in double-float arithmetic (FP32 instructions only; the
// z_i are exact, the y_i carried as (hi, lo)): the solution update of the mixed-precision solver
// with double-float Gram-Schmidt.  x itself stays FP64: the double-float sum is added once.
__global__ void __launch_bounds__(NT)
    k_xupdate_df(const KrylovCtl* __restrict__ ctl, const z64* __restrict__ Z, size_t ld, const z128* __restrict__ y,
                 z128* __restrict__ x, size_t n) {
  __shared__ zdf sy[MAX_BASIS];
  const int k = ctl->jend + 1;
  for (int i = threadIdx.x; i < k; i += NT) sy[i] = df_from(y[i]);
  __syncthreads();
  for (size_t p = blockIdx.x * (size_t)NT + threadIdx.x; p < n; p += (size_t)gridDim.x * NT) {
    float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
    for (int i = 0; i < k; ++i) {
      const z64 zv = ldg(Z + (size_t)i * ld + p);
      const zdf c = sy[i];
      // re += y.re z.re - y.im z.im ; im += y.re z.im + y.im z.re
      df_mac(c.rh, c.rl, zv.re, 0.f, rs, rc);
      df_mac(-c.ih, -c.il, zv.im, 0.f, rs, rc);
      df_mac(c.rh, c.rl, zv.im, 0.f, is, ic);
      df_mac(c.ih, c.il, zv.re, 0.f, is, ic);
    }
    const z128 xv = x[p];
    x[p] = mkc<double>(xv.re + ((double)rs + (double)rc), xv.im + ((double)is + (double)ic));
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

// ---- double-float Gram-Schmidt: basis in zdf, arithmetic on the FP32 pipes ----------------
// w -= sum_i h_i v_i, all in double-float.
__global__ void __launch_bounds__(NT)
    k_gs_update_df(const zdf* __restrict__ V, size_t ld, int nv, const z128* __restrict__ h, zdf* __restrict__ w,
                   size_t n, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ zdf sh[MAX_BASIS];
  for (int i = threadIdx.x; i < nv; i += NT) sh[i] = df_from(h[i]);
  __syncthreads();
  for (size_t p = blockIdx.x * (size_t)NT + threadIdx.x; p < n; p += (size_t)gridDim.x * NT) {
    float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
    for (int i = 0; i < nv; ++i) {
      const zdf v = ldg(V + (size_t)i * ld + p);
      const zdf c = sh[i];
      // re += cr vr - ci vi ; im += cr vi + ci vr
      df_mac(c.rh, c.rl, v.rh, v.rl, rs, rc);
      df_mac(-c.ih, -c.il, v.ih, v.il, rs, rc);
      df_mac(c.rh, c.rl, v.ih, v.il, is, ic);
      df_mac(c.ih, c.il, v.rh, v.rl, is, ic);
    }
    const zdf a = w[p];
    zdf o;
    df_add(a.rh, a.rl, -rs, -rc, o.rh, o.rl);
    df_add(a.ih, a.il, -is, -ic, o.ih, o.il);
    w[p] = o;
  }
}

__global__ void __launch_bounds__(NT)
    k_norm2_part_df(const zdf* __restrict__ x, size_t n, double* __restrict__ part, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ double sred[NW];
  size_t p0, p1;
  block_range(n, p0, p1);
  float ss = 0.f, sc = 0.f;
  for (size_t p = p0 + threadIdx.x; p < p1; p += NT) {
    const zdf v = ldg(x + p);
    df_mac(v.rh, v.rl, v.rh, v.rl, ss, sc);
    df_mac(v.ih, v.il, v.ih, v.il, ss, sc);
  }
  df_renorm(ss, sc, ss, sc);
  df_shfl_reduce(ss, sc);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = (double)ss + (double)sc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int wi = 0; wi < NW; ++wi) t += sred[wi];
    part[blockIdx.x] = t;
  }
}

// out = in / *s stored as double-float; `copy` receives the same vector as c128 (TC =
// double, exactly the double-float value) or complex64 (TC = float, its leading part).
__device__ __forceinline__ zdf scale_to_df(const z128& v, double inv, float, float) {
  return df_from(mkc<double>(v.re * inv, v.im * inv));
}
__device__ __forceinline__ zdf scale_to_df(const zdf& v, double, float ih, float il) {
  zdf z;
  df_mul(v.rh, v.rl, ih, il, z.rh, z.rl);
  df_mul(v.ih, v.il, ih, il, z.ih, z.il);
  return z;
}

template <typename TI, typename TC>
__global__ void __launch_bounds__(NT)
    k_scale_df(const TI* __restrict__ in, const double* __restrict__ s, zdf* __restrict__ out,
               cx<TC>* __restrict__ copy, size_t n, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const double d = *s;
  if (!(d != 0.0)) return;
  const double inv = 1.0 / d;
  float ih, il;
  df_split(inv, ih, il);
  for (size_t p = blockIdx.x * (size_t)NT + threadIdx.x; p < n; p += (size_t)gridDim.x * NT) {
    const zdf z = scale_to_df(in[p], inv, ih, il);
    out[p] = z;
    if (sizeof(TC) == 8) {
      const z128 c = df_to_c128(z);
      copy[p] = mkc<TC>((TC)c.re, (TC)c.im);
    } else {
      copy[p] = mkc<TC>((TC)z.rh, (TC)z.ih);
    }
  }
}

// w = sum_{i<=jend} y_i V_i, double-float accumulation.
__global__ void __launch_bounds__(NT)
    k_combine_df(const KrylovCtl* __restrict__ ctl, const zdf* __restrict__ V, size_t ld, const z128* __restrict__ y,
                 z128* __restrict__ w, size_t n) {
  __shared__ zdf sy[MAX_BASIS];
  const int k = ctl->jend + 1;
  for (int i = threadIdx.x; i < k; i += NT) sy[i] = df_from(y[i]);
  __syncthreads();
  for (size_t p = blockIdx.x * (size_t)NT + threadIdx.x; p < n; p += (size_t)gridDim.x * NT) {
    float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
    for (int i = 0; i < k; ++i) {
      const zdf v = ldg(V + (size_t)i * ld + p);
      const zdf c = sy[i];
      df_mac(c.rh, c.rl, v.rh, v.rl, rs, rc);
      df_mac(-c.ih, -c.il, v.ih, v.il, rs, rc);
      df_mac(c.rh, c.rl, v.ih, v.il, is, ic);
      df_mac(c.ih, c.il, v.rh, v.rl, is, ic);
    }
    w[p] = mkc<double>((double)rs + (double)rc, (double)is + (double)ic);
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

// One full wave of `kern` at NT threads: SMs x resident blocks (capped at RED_STRIDE).
template <typename K>
int wave_blocks(K kern) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NT, 0);
  const int nb = sms * (per > 0 ? per : 1);
  return nb < RED_STRIDE ? nb : RED_STRIDE;
}

// A wave of the least resident of two kernels at NT threads (capped at RED_STRIDE).
template <typename K1, typename K2>
int common_wave(K1 a, K2 b) {
  int dev = 0, sms = 0, pa = 0, pb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pa, a, NT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pb, b, NT, 0);
  const int per = std::max(1, std::min(pa, pb));
  return std::min(sms * per, RED_STRIDE);
}

int stream_blocks(size_t n) {
  size_t b = (n + NT - 1) / NT;
  const size_t cap = 152 * 8;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

// The variants of one inner-product family share one grid, so the points fall into the same
// block ranges whichever variant runs and the partial sums (hence the results) are identical: a
// wave of the family's least-resident variant.
template <typename ACC>
int mdot_fp64_grid() {
  static const int nb = common_wave(k_mdot<z128, ACC, 4 * NT, KS, true>, k_mdot<z128, ACC, 4 * NT, KS, false>);
  return nb;
}
template <typename ACC, bool STAGE>
int mdot_fp64(const z128* V, const double* Vs, size_t ld, int nv, const z128* w, size_t n, z128* part, int with_norm,
              cudaStream_t st, const int* active) {
  const int nb = mdot_fp64_grid<ACC>();
  k_mdot<z128, ACC, 4 * NT, KS, STAGE><<<nb, NT, 0, st>>>(V, Vs, ld, nv, w, n, part, with_norm, active);
  return nb;
}
// variant 0: w staged in shared memory; 1: each warp reads w itself.  Same sums (same grid, same
// points per lane in the same order).
template <typename ACC>
int mdot_variant(const z128* V, const double* Vs, size_t ld, int nv, const z128* w, size_t n, z128* part,
                 int with_norm, cudaStream_t st, const int* active, int variant) {
  return variant == 1 ? mdot_fp64<ACC, false>(V, Vs, ld, nv, w, n, part, with_norm, st, active)
                      : mdot_fp64<ACC, true>(V, Vs, ld, nv, w, n, part, with_norm, st, active);
}
int launch_mdot(const z128* V, size_t ld, int nv, const z128* w, size_t n, z128* part, int with_norm,
                cudaStream_t st, const int* active, int variant) {
  return mdot_variant<AccD>(V, nullptr, ld, nv, w, n, part, with_norm, st, active, variant);
}
int launch_mdot_sums(const z128* V, const double* Vs, size_t ld, int nv, const z128* w, size_t n, z128* part,
                     int with_norm, cudaStream_t st, const int* active, int variant) {
  return mdot_variant<AccD3>(V, Vs, ld, nv, w, n, part, with_norm, st, active, variant);
}
void launch_reduce_dots(const z128* part, int nv, int nb, z128* hpass, z128* hacc, int accumulate, int decide_j,
                        int* pass2, int* log, cudaStream_t st, const int* active, double keep) {
  k_reduce_dots<<<1, NT, 0, st>>>(part, nv, nb, hpass, hacc, accumulate, decide_j, pass2, log, active, keep);
}
void launch_gs_update(const z128* V, size_t ld, int nv, const z128* h, z128* w, size_t n, cudaStream_t st,
                      const int* active) {
  k_gs_update<<<stream_blocks(n), NT, 0, st>>>(V, ld, nv, h, w, n, active);
}
void launch_gs_update_sums(const z128* V, const double* Vs, size_t ld, int nv, const z128* h, z128* w, size_t n,
                           cudaStream_t st, const int* active) {
  k_gs_update_sums<<<stream_blocks(n), NT, 0, st>>>(V, Vs, ld, nv, h, w, n, active);
}
int launch_norm2_part(const z128* x, size_t n, double* partr, cudaStream_t st, const int* active) {
  static const int nb = wave_blocks(k_norm2_part);
  k_norm2_part<<<nb, NT, 0, st>>>(x, n, partr, active);
  return nb;
}
void launch_reduce_norm(const double* partr, int nb, double* out, cudaStream_t st, const int* active) {
  k_reduce_norm<<<1, NT, 0, st>>>(partr, nb, out, active);
}
void launch_scale_inv(const z128* in, const double* s, z128* out, size_t n, cudaStream_t st, const int* active) {
  k_scale_inv<<<stream_blocks(n), NT, 0, st>>>(in, s, out, n, active);
}
void launch_scale_inv_sums(const z128* in, const double* s, z128* out, double* outs, size_t n, cudaStream_t st,
                           const int* active) {
  k_scale_inv_sums<<<stream_blocks(n), NT, 0, st>>>(in, s, out, outs, n, active);
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
void launch_xupdate_df(const KrylovCtl* ctl, const z64* Z, size_t ld, const z128* y, z128* x, size_t n,
                       cudaStream_t st) {
  k_xupdate_df<<<stream_blocks(n), NT, 0, st>>>(ctl, Z, ld, y, x, n);
}
void launch_combine(const KrylovCtl* ctl, const z128* V, size_t ld, const z128* y, z128* w, size_t n,
                    cudaStream_t st) {
  k_combine<<<stream_blocks(n), NT, 0, st>>>(ctl, V, ld, y, w, n);
}
// One grid for the double-float variants: a wave of the most resident (2-slot) kernel, the one
// the autotuner measures fastest; the 4- and 8-slot kernels, with more registers, run it in more
// than one wave.
int mdot_df_grid() {
  static const int nb = wave_blocks(k_mdot<zdf, AccF, 4 * NT, 2>);
  return nb;
}
template <int KSV>
int mdot_df_ks(const zdf* V, size_t ld, int nv, const zdf* w, size_t n, z128* part, int with_norm, cudaStream_t st,
               const int* active) {
  const int nb = mdot_df_grid();
  k_mdot<zdf, AccF, 4 * NT, KSV><<<nb, NT, 0, st>>>(V, nullptr, ld, nv, w, n, part, with_norm, active);
  return nb;
}
int launch_mdot_df(const zdf* V, size_t ld, int nv, const zdf* w, size_t n, z128* part, int with_norm,
                   cudaStream_t st, const int* active, int variant) {
  switch (variant) {
    case 1: return mdot_df_ks<2>(V, ld, nv, w, n, part, with_norm, st, active);
    case 2: return mdot_df_ks<8>(V, ld, nv, w, n, part, with_norm, st, active);
    default: return mdot_df_ks<4>(V, ld, nv, w, n, part, with_norm, st, active);
  }
}
void launch_gs_update_df(const zdf* V, size_t ld, int nv, const z128* h, zdf* w, size_t n, cudaStream_t st,
                         const int* active) {
  k_gs_update_df<<<stream_blocks(n), NT, 0, st>>>(V, ld, nv, h, w, n, active);
}
int launch_norm2_part_df(const zdf* x, size_t n, double* partr, cudaStream_t st, const int* active) {
  static const int nb = wave_blocks(k_norm2_part_df);
  k_norm2_part_df<<<nb, NT, 0, st>>>(x, n, partr, active);
  return nb;
}
template <typename TI, typename TC>
void launch_scale_df(const TI* in, const double* s, zdf* out, cx<TC>* copy, size_t n, cudaStream_t st,
                     const int* active) {
  k_scale_df<TI, TC><<<stream_blocks(n), NT, 0, st>>>(in, s, out, copy, n, active);
}
template void launch_scale_df<z128, double>(const z128*, const double*, zdf*, z128*, size_t, cudaStream_t, const int*);
template void launch_scale_df<z128, float>(const z128*, const double*, zdf*, z64*, size_t, cudaStream_t, const int*);
template void launch_scale_df<zdf, double>(const zdf*, const double*, zdf*, z128*, size_t, cudaStream_t, const int*);
template void launch_scale_df<zdf, float>(const zdf*, const double*, zdf*, z64*, size_t, cudaStream_t, const int*);
void launch_combine_df(const KrylovCtl* ctl, const zdf* V, size_t ld, const z128* y, z128* w, size_t n,
                       cudaStream_t st) {
  k_combine_df<<<stream_blocks(n), NT, 0, st>>>(ctl, V, ld, y, w, n);
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
