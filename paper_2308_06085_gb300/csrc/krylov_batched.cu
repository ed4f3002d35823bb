// krylov_batched.cu -- FP64 kernels of right-preconditioned FGMRES(m) for nb right-hand sides
// solved together (nb a power of two <= 32).  Grid vectors are node-major with the right-hand
// side innermost (element e = node * nb + rhs), so a warp reads nb right-hand sides of 32/nb
// nodes in one coalesced row.  Every right-hand side keeps its own Hessenberg matrix, Givens
// rotations, residual estimate and stopping flag; the Arnoldi steps run in lockstep and a
// right-hand side that has stopped is carried along but no longer updated.
//
// A lane always works on the same right-hand side (thread strides are multiples of nb), so
// per-right-hand-side sums reduce across lanes of equal (lane mod nb) with shuffles at offsets
// >= nb, then across warps and blocks in a fixed order (deterministic).
#include "internal.cuh"

#include <type_traits>

namespace helm {

namespace {

constexpr int NT = 256;
constexpr int NW = NT / 32;
constexpr int KS = 4;        // basis vectors per warp per pass
constexpr int TILE = 1024;   // elements of w staged per shared-memory tile

__device__ __forceinline__ void block_range_e(size_t ne, int nb, size_t& e0, size_t& e1) {
  // chunk per block, a multiple of the tile and of nb
  size_t chunk = (ne + gridDim.x - 1) / gridDim.x;
  chunk = (chunk + TILE - 1) / TILE * TILE;
  e0 = blockIdx.x * chunk;
  e1 = e0 + chunk < ne ? e0 + chunk : ne;
  if (e0 > ne) e0 = ne;
  (void)nb;
}

// reduce across lanes with equal lane mod nb
__device__ __forceinline__ double lane_group_sum(double v, int nb) {
  for (int o = 16; o >= nb; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void df_group_sum(float& s, float& c, int nb) {
  for (int o = 16; o >= nb; o >>= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, s, o), oc = __shfl_xor_sync(0xffffffffu, c, o);
    float hi, lo;
    df_add(s, c, os, oc, hi, lo);
    s = hi;
    c = lo;
  }
}

// Accumulators of one lane: FP64 (z128 vectors) or double-float (zdf vectors, FP32 pipes).
struct BAccD {
  static constexpr bool kBalanced = false;
  static constexpr bool kSums = false;
  double re, im;
  __device__ void zero() { re = im = 0.0; }
  __device__ void mac(const z128& v, const z128& w) { cdot_acc(v, w, re, im); }
  __device__ void norm(const z128& w) {
    re = fma(w.re, w.re, re);
    re = fma(w.im, w.im, re);
  }
  __device__ void group(int nb, double& r, double& i) {
    r = lane_group_sum(re, nb);
    i = lane_group_sum(im, nb);
  }
  __device__ void value(double& r, double& i) const {
    r = re;
    i = im;
  }
};
// FP64 accumulator against a basis stored with its element sums s = Re v + Im v (three FMAs
// per complex multiply-add): A = sum vr wr, B = sum vi wi, C = sum s (wi - wr) give
// conj(v) . w = (A + B) + i (C + A - B).
struct BAccD3 {
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
  __device__ void group(int nb, double& r, double& i) {
    r = lane_group_sum(a + b, nb);
    i = lane_group_sum(c + (a - b), nb);
  }
  __device__ void value(double& r, double& i) const {
    r = a + b;
    i = c + (a - b);
  }
};
struct BAccF {
  static constexpr bool kBalanced = true;
  static constexpr bool kSums = false;
  float rs, rc, is, ic;
  __device__ void zero() { rs = rc = is = ic = 0.f; }
  __device__ void mac(const zdf& v, const zdf& w) {
    df_mac(v.rh, v.rl, w.rh, w.rl, rs, rc);
    df_mac(v.ih, v.il, w.ih, w.il, rs, rc);
    df_mac(v.rh, v.rl, w.ih, w.il, is, ic);
    df_mac(-v.ih, -v.il, w.rh, w.rl, is, ic);
  }
  __device__ void norm(const zdf& w) {
    df_mac(w.rh, w.rl, w.rh, w.rl, rs, rc);
    df_mac(w.ih, w.il, w.ih, w.il, rs, rc);
  }
  __device__ void group(int nb, double& r, double& i) {
    float a = rs, b = rc, x = is, y = ic;
    df_renorm(a, b, a, b);
    df_renorm(x, y, x, y);
    df_group_sum(a, b, nb);
    df_group_sum(x, y, nb);
    r = (double)a + (double)b;
    i = (double)x + (double)y;
  }
};

// |x_r|^2 partials: part[r * RED_STRIDE + blk]
template <typename E, typename ACC>
__global__ void __launch_bounds__(NT)
    k_bnorm2_part(const E* __restrict__ x, size_t ne, int nb, double* __restrict__ part, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ double sred[NW][32];
  size_t e0, e1;
  block_range_e(ne, nb, e0, e1);
  ACC acc;
  acc.zero();
  for (size_t e = e0 + threadIdx.x; e < e1; e += NT) acc.norm(ldg(x + e));
  double s, unused;
  acc.group(nb, s, unused);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < nb) sred[warp][lane] = s;
  __syncthreads();
  if ((int)threadIdx.x < nb) {
    double t = 0.0;
    for (int w = 0; w < NW; ++w) t += sred[w][threadIdx.x];
    part[(size_t)threadIdx.x * RED_STRIDE + blockIdx.x] = t;
  }
}

// out[r] = sqrt(sum_b part[r][b]), one warp per right-hand side
__global__ void __launch_bounds__(NT)
    k_breduce_norm(const double* __restrict__ part, int nb, int nblk, double* __restrict__ out, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < nb; r += NW) {
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += part[(size_t)r * RED_STRIDE + b];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[r] = sqrt(s);
  }
}

// Inner products conj(V_i) . w per right-hand side; slot nv holds |w_r|^2 when with_norm.
// Warps sharing one slot for double-float accumulation: the least sharing that leaves at most
// 1/8 of the warp-slots idle (latency-bound, so evenly loaded warps keep more loads in flight).
__device__ __forceinline__ int bshare_width(int nslot) {
  for (int wps = 1; wps < NW; wps <<= 1) {
    const int groups = NW / wps;
    const int cap = (nslot + groups - 1) / groups * groups;
    if (8 * (cap - nslot) <= cap) return wps;
  }
  return NW;
}

template <typename ACC, typename E>
__device__ __forceinline__ void bslot_mac(ACC& acc, const E* __restrict__ V, const double* __restrict__ Vs, size_t off,
                                          const E& w, double wd) {
  if constexpr (ACC::kSums) acc.mac3(ldg(V + off), ldg(Vs + off), w, wd);
  else acc.mac(ldg(V + off), w);
}
__device__ __forceinline__ double bw_diff(const z128& w) { return w.im - w.re; }
__device__ __forceinline__ double bw_diff(const zdf&) { return 0.0; }

template <typename E, typename ACC, int KSV = KS>
__global__ void __launch_bounds__(NT, 4)
    k_bmdot(const E* __restrict__ V, const double* __restrict__ Vs, size_t ld, int nv, const E* __restrict__ w,
            size_t ne, int nb, z128* __restrict__ part, int with_norm, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ E sw[TILE];
  __shared__ double swd[ACC::kSums ? TILE : 1];  // wi - wr of the staged points (summed basis)
  __shared__ double sred[NW][32][2];
  size_t e0, e1;
  block_range_e(ne, nb, e0, e1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nslot = nv + (with_norm ? 1 : 0);
  const int wps = ACC::kBalanced ? bshare_width(nslot) : (nslot >= NW ? 1 : NW / nslot);
  const int sub = warp % wps, sfirst = warp / wps, sstep = NW / wps;
  double* partd = reinterpret_cast<double*>(part);
  for (int sbase = 0; sbase * sstep < nslot; sbase += KSV) {
    ACC acc[KSV];
#pragma unroll
    for (int k = 0; k < KSV; ++k) acc[k].zero();
    for (size_t t0 = e0; t0 < e1; t0 += TILE) {
      const int tn = (int)min((size_t)TILE, e1 - t0);
      __syncthreads();
      for (int q = threadIdx.x; q < tn; q += NT) {
        const E wv = ldg(w + t0 + q);
        sw[q] = wv;
        if (ACC::kSums) swd[q] = bw_diff(wv);  // once per point, not once per warp
      }
      __syncthreads();
#pragma unroll 2
      for (int q = sub * 32 + lane; q < tn; q += 32 * wps) {
        const E wv = sw[q];
        const double wd = ACC::kSums ? swd[q] : 0.0;
#pragma unroll
        for (int k = 0; k < KSV; ++k) {
          const int sl = sfirst + (sbase + k) * sstep;
          if (sl < nv) bslot_mac(acc[k], V, Vs, (size_t)sl * ld + t0 + q, wv, wd);
          else if (sl == nv && with_norm) acc[k].norm(wv);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KSV; ++k) {
      const int sl = sfirst + (sbase + k) * sstep;
      double r, i;
      acc[k].group(nb, r, i);
      __syncthreads();
      if (lane < nb) {
        sred[warp][lane][0] = r;
        sred[warp][lane][1] = i;
      }
      __syncthreads();
      if (sub == 0 && lane < nb && sl < nslot) {
        double tr = 0.0, ti = 0.0;
        for (int u = 0; u < wps; ++u) {
          tr += sred[warp + u][lane][0];
          ti += sred[warp + u][lane][1];
        }
        const size_t row = (size_t)sl * nb + lane;
        partd[2 * (row * RED_STRIDE + blockIdx.x)] = tr;
        partd[2 * (row * RED_STRIDE + blockIdx.x) + 1] = sl == nv ? 0.0 : ti;
      }
    }
  }
}

// hpass[i * nb + r] = sum of the partials of (slot i, rhs r); hacc stores or accumulates.
// decide_j >= 0: a second Gram-Schmidt pass is taken when, for any active right-hand side,
// the projection kept less than `keep` of |w_r|^2 (k_bdecide).
__global__ void __launch_bounds__(NT)
    k_breduce_dots(const z128* __restrict__ part, int nv, int nb, int nblk, z128* __restrict__ hpass,
                   z128* __restrict__ hacc, int accumulate, int decide_j, double* __restrict__ sw2,
                   const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int lane = threadIdx.x & 31;
  const int rows = (decide_j >= 0 ? nv + 1 : nv) * nb;
  // one warp per (basis vector, right-hand side) row, over every block of the grid
  const int row = blockIdx.x * NW + (threadIdx.x >> 5);
  if (row >= rows) return;
  double re = 0.0, im = 0.0;
  for (int b = lane; b < nblk; b += 32) {
    const z128 v = part[(size_t)row * RED_STRIDE + b];
    re += v.re;
    im += v.im;
  }
  for (int o = 16; o; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    if (row >= nv * nb) {
      sw2[row - nv * nb] = re;
    } else {
      hpass[row] = mkc<double>(re, im);
      if (accumulate) {
        hacc[row].re += re;
        hacc[row].im += im;
      } else {
        hacc[row] = mkc<double>(re, im);
      }
    }
  }
}

// The Daniel-Gragg-Kaufman-Stewart test per active right-hand side: r takes a second pass when
// its first one kept less than `keep` of |w_r|^2 (need[r]); the pass runs when any r needs it,
// and log[decide_j] holds how many do.
__global__ void k_bdecide(const z128* __restrict__ hpass, const double* __restrict__ sw2, int nv, int nb,
                          int decide_j, const int* __restrict__ act, int* __restrict__ pass2, int* __restrict__ log,
                          int* __restrict__ need, const int* __restrict__ active, double keep) {
  if (active && *active == 0) return;
  if (threadIdx.x != 0) return;
  int count = 0;
  for (int r = 0; r < nb; ++r) {
    int nr = 0;
    if (act[r]) {
      double h2 = 0.0;
      for (int i = 0; i < nv; ++i) h2 += hpass[i * nb + r].re * hpass[i * nb + r].re + hpass[i * nb + r].im * hpass[i * nb + r].im;
      nr = !(sw2[r] - h2 >= keep * sw2[r]);
    }
    need[r] = nr;
    count += nr;
  }
  *pass2 = count > 0;
  log[decide_j] = count;
}

// The list of right-hand sides that need the second pass, in increasing order, in shared memory.
__device__ __forceinline__ int need_list(const int* __restrict__ need, int nb, int* list) {
  __shared__ int cnt;
  if (threadIdx.x < 32) {
    const int f = (int)threadIdx.x < nb ? need[threadIdx.x] != 0 : 0;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (f) list[__popc(m & ((1u << threadIdx.x) - 1u))] = threadIdx.x;
    if (threadIdx.x == 0) cnt = __popc(m);
  }
  __syncthreads();
  return cnt;
}

// Second Gram-Schmidt pass for the right-hand sides in need[] only (FP64, summed basis or
// textbook accumulator).  The partials keep k_bmdot's layout and block ranges, so
// k_breduce_dots sums them unchanged; the rows of the other right-hand sides get zeros.  The
// work is packed: with K selected right-hand sides, thread t of the block takes the pairs
// (node, selected right-hand side t % K) for t < (NT / K) K, so every active lane works on a
// selected right-hand side, and a warp reads a few contiguous rows of nb values; the per-thread
// sums are then added over the threads of each right-hand side in a fixed order.
template <typename ACC>
__global__ void __launch_bounds__(NT)
    k_bmdot_sel(const z128* __restrict__ V, const double* __restrict__ Vs, size_t ld, int nv,
                const z128* __restrict__ w, size_t ne, int nb, const int* __restrict__ need, z128* __restrict__ part,
                const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ int list[32];
  __shared__ double sred[KS][NT][2];
  const int cnt = need_list(need, nb, list);
  size_t e0, e1;
  block_range_e(ne, nb, e0, e1);
  const size_t q0 = e0 / nb, q1 = e1 / nb;  // node range of this block (chunks are multiples of nb)
  double* partd = reinterpret_cast<double*>(part);
  // zeros for the rows of the right-hand sides without a second pass
  for (int t = threadIdx.x; t < nv * nb; t += NT) {
    const int r = t % nb;
    bool sel = false;
    for (int k = 0; k < cnt; ++k) sel |= list[k] == r;
    if (!sel) {
      partd[2 * ((size_t)t * RED_STRIDE + blockIdx.x)] = 0.0;
      partd[2 * ((size_t)t * RED_STRIDE + blockIdx.x) + 1] = 0.0;
    }
  }
  if (cnt == 0) return;
  const int per = NT / cnt;            // nodes per block sweep
  const int tk = threadIdx.x % cnt;    // this thread's selected right-hand side
  const int tq = threadIdx.x / cnt;    // this thread's node offset in a sweep
  const bool on = tq < per;
  const int r = list[tk];
  for (int sbase = 0; sbase < nv; sbase += KS) {
    ACC acc[KS];
#pragma unroll
    for (int s = 0; s < KS; ++s) acc[s].zero();
    if (on)
      for (size_t q = q0 + tq; q < q1; q += per) {
        const size_t e = q * nb + r;
        const z128 wv = ldg(w + e);
        const double wd = bw_diff(wv);
#pragma unroll
        for (int s = 0; s < KS; ++s)
          if (sbase + s < nv) bslot_mac(acc[s], V, Vs, (size_t)(sbase + s) * ld + e, wv, wd);
      }
#pragma unroll
    for (int s = 0; s < KS; ++s) {
      double re, im;
      acc[s].value(re, im);  // this thread's own sum (no lane exchange)
      sred[s][threadIdx.x][0] = on ? re : 0.0;
      sred[s][threadIdx.x][1] = on ? im : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < KS * cnt; t += NT) {
      const int s = t / cnt, k = t % cnt;
      if (sbase + s < nv) {
        double tr = 0.0, ti = 0.0;
        for (int u = k; u < per * cnt; u += cnt) {
          tr += sred[s][u][0];
          ti += sred[s][u][1];
        }
        const size_t row = (size_t)(sbase + s) * nb + list[k];
        partd[2 * (row * RED_STRIDE + blockIdx.x)] = tr;
        partd[2 * (row * RED_STRIDE + blockIdx.x) + 1] = ti;
      }
    }
    __syncthreads();
  }
}

// w[e] -= sum_i h[i][r] V_i[e] for the right-hand sides in need[] only (the others' h is zero),
// packed as in k_bmdot_sel: thread t of the grid takes (node, selected right-hand side t % K)
template <bool SUMS>
__global__ void __launch_bounds__(NT)
    k_bgs_update_sel(const z128* __restrict__ V, const double* __restrict__ Vs, size_t ld, int nv, int nb,
                     const z128* __restrict__ h, z128* __restrict__ w, size_t ne, const int* __restrict__ need,
                     const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ int list[32];
  extern __shared__ double3 shq[];
  const int cnt = need_list(need, nb, list);
  if (cnt == 0) return;
  for (int t = threadIdx.x; t < nv * cnt; t += NT) {
    const z128 c = h[(t / cnt) * nb + list[t % cnt]];
    shq[t] = make_double3(c.re, c.im, c.re + c.im);
  }
  __syncthreads();
  const int per = NT / cnt;
  const int tk = threadIdx.x % cnt, tq = threadIdx.x / cnt;
  if (tq >= per) return;
  const int r = list[tk];
  const size_t nq = ne / nb;
  for (size_t q = blockIdx.x * (size_t)per + tq; q < nq; q += (size_t)gridDim.x * per) {
    const size_t e = q * nb + r;
    const z128 a = w[e];
    if (SUMS) {
      double P = 0.0, Q = 0.0, R = 0.0;
      for (int i = 0; i < nv; ++i) {
        const size_t off = (size_t)i * ld + e;
        const z128 v = ldg(V + off);
        const double sv = ldg(Vs + off);
        const double3 c = shq[i * cnt + tk];
        P = fma(c.x, v.re, P);
        Q = fma(c.y, v.im, Q);
        R = fma(c.z, sv, R);
      }
      w[e] = mkc<double>(a.re - (P - Q), a.im - (R - (P + Q)));
    } else {
      z128 acc = a;
      for (int i = 0; i < nv; ++i) {
        const z128 v = ldg(V + (size_t)i * ld + e);
        const double3 c = shq[i * cnt + tk];
        acc.re = fma(-c.x, v.re, acc.re);
        acc.re = fma(c.y, v.im, acc.re);
        acc.im = fma(-c.x, v.im, acc.im);
        acc.im = fma(-c.y, v.re, acc.im);
      }
      w[e] = acc;
    }
  }
}

// w[e] -= sum_i h[i][r] V_i[e]
__global__ void __launch_bounds__(NT)
    k_bgs_update(const z128* __restrict__ V, size_t ld, int nv, int nb, const z128* __restrict__ h, z128* __restrict__ w,
                 size_t ne, const int* __restrict__ active) {
  if (active && *active == 0) return;
  extern __shared__ z128 shb[];
  for (int i = threadIdx.x; i < nv * nb; i += NT) shb[i] = h[i];
  __syncthreads();
  const size_t stride = (size_t)gridDim.x * NT;
  // nb is a power of two <= 32 and divides the stride, so a thread keeps one right-hand side
  const int r = (int)((blockIdx.x * (size_t)NT + threadIdx.x) & (size_t)(nb - 1));
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < ne; e += stride) {
    z128 acc = w[e];
    for (int i = 0; i < nv; ++i) {
      const z128 v = ldg(V + (size_t)i * ld + e);
      const z128 c = shb[i * nb + r];
      acc.re = fma(-c.re, v.re, acc.re);
      acc.re = fma(c.im, v.im, acc.re);
      acc.im = fma(-c.re, v.im, acc.im);
      acc.im = fma(-c.im, v.re, acc.im);
    }
    w[e] = acc;
  }
}

// w[e] -= sum_i h[i][r] V_i[e] against the summed basis: with P = sum hr vr, Q = sum hi vi and
// R = sum (hr + hi) s, h v = (P - Q) + i (R - P - Q), three FMAs per element and vector
__global__ void __launch_bounds__(NT)
    k_bgs_update_sums(const z128* __restrict__ V, const double* __restrict__ Vs, size_t ld, int nv, int nb,
                      const z128* __restrict__ h, z128* __restrict__ w, size_t ne, const int* __restrict__ active) {
  if (active && *active == 0) return;
  extern __shared__ double3 shs[];
  for (int i = threadIdx.x; i < nv * nb; i += NT) {
    const z128 c = h[i];
    shs[i] = make_double3(c.re, c.im, c.re + c.im);
  }
  __syncthreads();
  const size_t stride = (size_t)gridDim.x * NT;
  const int r = (int)((blockIdx.x * (size_t)NT + threadIdx.x) & (size_t)(nb - 1));  // fixed per thread
  // two elements per trip, e and e + stride (the same right-hand side, as stride is a multiple
  // of nb): twice the independent loads and FMA chains, one coefficient load for both; each
  // element's sums run in the same order as with one element per trip
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < ne; e += 2 * stride) {
    const size_t e2 = e + stride;
    const bool two = e2 < ne;
    double P = 0.0, Q = 0.0, R = 0.0, P2 = 0.0, Q2 = 0.0, R2 = 0.0;
    for (int i = 0; i < nv; ++i) {
      const size_t off = (size_t)i * ld + e;
      const z128 v = ldg(V + off);
      const double sv = ldg(Vs + off);
      const double3 c = shs[i * nb + r];
      P = fma(c.x, v.re, P);
      Q = fma(c.y, v.im, Q);
      R = fma(c.z, sv, R);
      if (two) {
        const z128 v2 = ldg(V + off + stride);
        const double sv2 = ldg(Vs + off + stride);
        P2 = fma(c.x, v2.re, P2);
        Q2 = fma(c.y, v2.im, Q2);
        R2 = fma(c.z, sv2, R2);
      }
    }
    const z128 a = w[e];
    w[e] = mkc<double>(a.re - (P - Q), a.im - (R - (P + Q)));
    if (two) {
      const z128 a2 = w[e2];
      w[e2] = mkc<double>(a2.re - (P2 - Q2), a2.im - (R2 - (P2 + Q2)));
    }
  }
}

// out[e] = in[e] * (1 / s[r]) where s[r] > 0, else 0, and outs[e] = Re out + Im out (the element
// sums of a summed basis vector)
__global__ void __launch_bounds__(NT)
    k_bscale_inv_sums(const z128* __restrict__ in, const double* __restrict__ s, z128* __restrict__ out,
                      double* __restrict__ outs, size_t ne, int nb, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const size_t stride = (size_t)gridDim.x * NT;
  const double d = s[(blockIdx.x * (size_t)NT + threadIdx.x) & (size_t)(nb - 1)];  // fixed per thread
  // one division per thread (an FP64 division costs many FP64 issue slots), as k_scale_inv does
  const double inv = d > 0.0 ? 1.0 / d : 0.0;
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < ne; e += stride) {
    const z128 v = in[e];
    const z128 o = mkc<double>(v.re * inv, v.im * inv);
    out[e] = o;
    outs[e] = o.re + o.im;
  }
}

// double-float: w[e] -= sum_i h[i][r] V_i[e], all on the FP32 pipes
__global__ void __launch_bounds__(NT)
    k_bgs_update_df(const zdf* __restrict__ V, size_t ld, int nv, int nb, const z128* __restrict__ h,
                    zdf* __restrict__ w, size_t ne, const int* __restrict__ active) {
  if (active && *active == 0) return;
  extern __shared__ zdf shf[];
  for (int i = threadIdx.x; i < nv * nb; i += NT) shf[i] = df_from(h[i]);
  __syncthreads();
  const size_t stride = (size_t)gridDim.x * NT;
  const int r = (int)((blockIdx.x * (size_t)NT + threadIdx.x) & (size_t)(nb - 1));  // fixed per thread
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < ne; e += stride) {
    float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
    for (int i = 0; i < nv; ++i) {
      const zdf v = ldg(V + (size_t)i * ld + e);
      const zdf c = shf[i * nb + r];
      df_mac(c.rh, c.rl, v.rh, v.rl, rs, rc);
      df_mac(-c.ih, -c.il, v.ih, v.il, rs, rc);
      df_mac(c.rh, c.rl, v.ih, v.il, is, ic);
      df_mac(c.ih, c.il, v.rh, v.rl, is, ic);
    }
    const zdf a = w[e];
    zdf o;
    df_add(a.rh, a.rl, -rs, -rc, o.rh, o.rl);
    df_add(a.ih, a.il, -is, -ic, o.ih, o.il);
    w[e] = o;
  }
}

// double-float scaling: out[e] = in[e] / s[r] (0 when s[r] is not positive), and the copy the
// next V-cycle reads (complex128, exact value; or complex64, the leading parts)
__device__ __forceinline__ zdf bscale_one(const z128& v, double d) {
  return d > 0.0 ? df_from(mkc<double>(v.re / d, v.im / d)) : zdf{0.f, 0.f, 0.f, 0.f};
}
// the double-float reciprocal of d (0 when d is not positive), computed once per thread
struct DfRecip {
  float hi, lo;
  bool pos;
  __device__ explicit DfRecip(double d) : hi(0.f), lo(0.f), pos(d > 0.0) {
    if (pos) df_split(1.0 / d, hi, lo);
  }
};
__device__ __forceinline__ zdf bscale_one(const zdf& v, const DfRecip& q) {
  if (!q.pos) return zdf{0.f, 0.f, 0.f, 0.f};
  zdf z;
  df_mul(v.rh, v.rl, q.hi, q.lo, z.rh, z.rl);
  df_mul(v.ih, v.il, q.hi, q.lo, z.ih, z.il);
  return z;
}
template <typename TI>
__device__ __forceinline__ typename std::conditional<std::is_same<TI, zdf>::value, DfRecip, double>::type
scale_arg(double d) {
  return typename std::conditional<std::is_same<TI, zdf>::value, DfRecip, double>::type(d);
}

template <typename TI, typename TC>
__global__ void __launch_bounds__(NT)
    k_bscale_df(const TI* __restrict__ in, const double* __restrict__ s, zdf* __restrict__ out,
                cx<TC>* __restrict__ copy, size_t ne, int nb, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const size_t stride = (size_t)gridDim.x * NT;
  const double sr = s[(blockIdx.x * (size_t)NT + threadIdx.x) & (size_t)(nb - 1)];  // fixed per thread
  // the scale as the input type wants it: FP64 for complex128 input, a double-float
  // reciprocal for double-float input (one FP64 division per thread, not per element)
  const auto sc = scale_arg<TI>(sr);
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < ne; e += stride) {
    const zdf z = bscale_one(in[e], sc);
    out[e] = z;
    if (sizeof(TC) == 8) {
      const z128 c = df_to_c128(z);
      copy[e] = mkc<TC>((TC)c.re, (TC)c.im);
    } else {
      copy[e] = mkc<TC>((TC)z.rh, (TC)z.ih);
    }
  }
}

// out[e] = in[e] * (1 / s[r]) where s[r] > 0, else 0
__global__ void __launch_bounds__(NT)
    k_bscale_inv(const z128* __restrict__ in, const double* __restrict__ s, z128* __restrict__ out, size_t ne, int nb,
                 const int* __restrict__ active) {
  if (active && *active == 0) return;
  const size_t stride = (size_t)gridDim.x * NT;
  const double d = s[(blockIdx.x * (size_t)NT + threadIdx.x) & (size_t)(nb - 1)];  // fixed per thread
  // one division per thread (an FP64 division costs many FP64 issue slots), as k_scale_inv does
  const double inv = d > 0.0 ? 1.0 / d : 0.0;
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < ne; e += stride) {
    const z128 v = in[e];
    out[e] = mkc<double>(v.re * inv, v.im * inv);
  }
}

// Start a restart cycle: right-hand side r is active when its residual is above tol and it
// has Arnoldi steps left; g_r = (beta_r, 0, ...).
__global__ void k_bcycle_init(BatchCtl* bc, int nb, int m, double tol) {
  const int r = threadIdx.x;
  __shared__ int any;
  if (r == 0) any = 0;
  __syncthreads();
  if (r < nb) {
    const int a = bc->bnorm[r] > 0.0 && bc->beta[r] > tol * bc->bnorm[r] && bc->iters[r] < bc->max_iter &&
                  isfinite(bc->beta[r]);
    bc->act[r] = a;
    bc->jend[r] = -1;
    bc->flag[r] = 0;
    bc->jmax[r] = min(m, bc->max_iter - bc->iters[r]);
    for (int i = 0; i <= m; ++i) bc->g[(size_t)r * (m + 1) + i] = mkc<double>(i == 0 ? bc->beta[r] : 0.0, 0.0);
    if (a) atomicOr(&any, 1);
  }
  __syncthreads();
  if (r == 0) {
    bc->any = any;
    bc->pass2 = 0;
  }
}

// Arnoldi step j, Givens rotations per right-hand side (one thread each), as in the
// single-right-hand-side kernel.
__global__ void k_bgivens(BatchCtl* bc, int nb, int m, int j, const z128* __restrict__ hcol, const double* __restrict__ hnorm,
                          double tol) {
  const int r = threadIdx.x;
  __shared__ int any;
  if (r == 0) any = 0;
  __syncthreads();
  if (r < nb && bc->act[r]) {
    z128* H = bc->H + (size_t)r * (m + 1) * m;
    double* cs = bc->cs + (size_t)r * m;
    z128* sn = bc->sn + (size_t)r * m;
    z128* g = bc->g + (size_t)r * (m + 1);
    for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i * nb + r];
    const double hn = hnorm[r];
    H[(size_t)(j + 1) * m + j] = mkc<double>(hn, 0.0);
    for (int i = 0; i < j; ++i) {
      const z128 a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
      const double c = cs[i];
      const z128 s = sn[i];
      const z128 sb = cmul(s, b);
      const z128 t = cmul(mkc<double>(-s.re, s.im), a);
      H[(size_t)i * m + j] = mkc<double>(c * a.re + sb.re, c * a.im + sb.im);
      H[(size_t)(i + 1) * m + j] = mkc<double>(t.re + c * b.re, t.im + c * b.im);
    }
    const z128 a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
    const double na = hypot(a.re, a.im), nbv = hypot(b.re, b.im);
    const double t = hypot(na, nbv);
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
    g[j + 1] = cmul(mkc<double>(-s.re, s.im), gj);
    g[j] = mkc<double>(c * gj.re, c * gj.im);
    const double est = hypot(g[j + 1].re, g[j + 1].im) / bc->bnorm[r];
    bc->est[r] = est;
    bc->jend[r] = j;
    if (!isfinite(est) || !isfinite(hn)) {
      bc->flag[r] = 2;
      bc->act[r] = 0;
    } else if (est <= tol) {
      bc->flag[r] = 1;
      bc->act[r] = 0;
    } else if (j + 1 >= bc->jmax[r]) {
      bc->act[r] = 0;
    }
    if (bc->act[r]) atomicOr(&any, 1);
  }
  __syncthreads();
  if (r == 0) {
    bc->any = any;
    if (!any) bc->pass2 = 0;
  }
}

// y_r = H_r(0:k, 0:k)^{-1} g_r with k = jend_r + 1 (one thread per right-hand side)
__global__ void k_btrisolve(BatchCtl* bc, int nb, int m) {
  const int r = threadIdx.x;
  if (r >= nb) return;
  const int k = bc->jend[r] + 1;
  bc->iters[r] += k;
  const z128* H = bc->H + (size_t)r * (m + 1) * m;
  const z128* g = bc->g + (size_t)r * (m + 1);
  z128* y = bc->y;  // y[i * nb + r]
  for (int i = k - 1; i >= 0; --i) {
    z128 s = g[i];
    for (int q = i + 1; q < k; ++q) {
      const z128 hy = cmul(H[(size_t)i * m + q], y[q * nb + r]);
      s.re -= hy.re;
      s.im -= hy.im;
    }
    const z128 d = H[(size_t)i * m + i];
    const double dd = d.re * d.re + d.im * d.im;
    y[i * nb + r] = mkc<double>((s.re * d.re + s.im * d.im) / dd, (s.im * d.re - s.re * d.im) / dd);
  }
}

// x[e] += sum_{i <= jend_r} y[i][r] Z_i[e]
template <typename TZ>
__global__ void __launch_bounds__(NT)
    k_bxupdate(const BatchCtl* __restrict__ bc, int nb, int m, const cx<TZ>* __restrict__ Z, size_t ld, z128* __restrict__ x,
               size_t ne) {
  extern __shared__ z128 sy[];
  __shared__ int kr[32];
  __shared__ int kmax;
  if (threadIdx.x < (unsigned)nb) kr[threadIdx.x] = bc->jend[threadIdx.x] + 1;
  for (int i = threadIdx.x; i < m * nb; i += NT) sy[i] = bc->y[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    int mx = 0;
    for (int r = 0; r < nb; ++r) mx = max(mx, kr[r]);
    kmax = mx;
  }
  __syncthreads();
  const size_t stride = (size_t)gridDim.x * NT;
  const int r = (int)((blockIdx.x * (size_t)NT + threadIdx.x) & (size_t)(nb - 1));  // fixed per thread
  const int k = kr[r];
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < ne; e += stride) {
    z128 acc = x[e];
    for (int i = 0; i < kmax; ++i)
      if (i < k) acc = cfma(sy[i * nb + r], cvt<double>(ldg(Z + (size_t)i * ld + e)), acc);
    x[e] = acc;
  }
}

// The same update in double-float arithmetic for complex64 Z (mixed precision with
// double-float Gram-Schmidt): FP32 instructions only, x stays FP64.
__global__ void __launch_bounds__(NT)
    k_bxupdate_df(const BatchCtl* __restrict__ bc, int nb, int m, const z64* __restrict__ Z, size_t ld,
                  z128* __restrict__ x, size_t ne) {
  extern __shared__ zdf syd[];
  __shared__ int kr[32];
  __shared__ int kmax;
  if (threadIdx.x < (unsigned)nb) kr[threadIdx.x] = bc->jend[threadIdx.x] + 1;
  for (int i = threadIdx.x; i < m * nb; i += NT) syd[i] = df_from(bc->y[i]);
  __syncthreads();
  if (threadIdx.x == 0) {
    int mx = 0;
    for (int r = 0; r < nb; ++r) mx = max(mx, kr[r]);
    kmax = mx;
  }
  __syncthreads();
  const size_t stride = (size_t)gridDim.x * NT;
  const int r = (int)((blockIdx.x * (size_t)NT + threadIdx.x) & (size_t)(nb - 1));  // fixed per thread
  const int k = kr[r];
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < ne; e += stride) {
    float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
    for (int i = 0; i < kmax; ++i)
      if (i < k) {
        const z64 zv = ldg(Z + (size_t)i * ld + e);
        const zdf c = syd[i * nb + r];
        df_mac(c.rh, c.rl, zv.re, 0.f, rs, rc);
        df_mac(-c.ih, -c.il, zv.im, 0.f, rs, rc);
        df_mac(c.rh, c.rl, zv.im, 0.f, is, ic);
        df_mac(c.ih, c.il, zv.re, 0.f, is, ic);
      }
    const z128 xv = x[e];
    x[e] = mkc<double>(xv.re + ((double)rs + (double)rc), xv.im + ((double)is + (double)ic));
  }
}

// [rhs][node] <-> [node][rhs] (nb slots; right-hand sides r >= nrhs are zero on the way in)
__global__ void k_to_batch(const z128* __restrict__ src, z128* __restrict__ dst, size_t n, int nb, int nrhs) {
  const size_t ne = n * nb;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ne; e += (size_t)gridDim.x * blockDim.x) {
    const size_t p = e / nb;
    const int r = (int)(e - p * nb);
    dst[e] = r < nrhs ? src[(size_t)r * n + p] : mkc<double>(0.0, 0.0);
  }
}
__global__ void k_from_batch(const z128* __restrict__ src, z128* __restrict__ dst, size_t n, int nb, int nrhs) {
  const size_t ne = n * nrhs;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < ne; t += (size_t)gridDim.x * blockDim.x) {
    const size_t r = t / n, p = t - r * n;
    dst[t] = src[p * nb + r];
  }
}

template <typename K>
int wave_blocks(K kern, int smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NT, smem);
  const int nb = sms * (per > 0 ? per : 1);
  return nb < RED_STRIDE ? nb : RED_STRIDE;
}

int stream_blocks(size_t n) {
  size_t b = (n + NT - 1) / NT;
  const size_t cap = 152 * 8;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

int launch_bnorm2_part(const z128* x, size_t ne, int nb, double* part, cudaStream_t st, const int* active) {
  static const int nblk = wave_blocks(k_bnorm2_part<z128, BAccD>, 0);
  k_bnorm2_part<z128, BAccD><<<nblk, NT, 0, st>>>(x, ne, nb, part, active);
  return nblk;
}
int launch_bnorm2_part_df(const zdf* x, size_t ne, int nb, double* part, cudaStream_t st, const int* active) {
  static const int nblk = wave_blocks(k_bnorm2_part<zdf, BAccF>, 0);
  k_bnorm2_part<zdf, BAccF><<<nblk, NT, 0, st>>>(x, ne, nb, part, active);
  return nblk;
}
void launch_breduce_norm(const double* part, int nb, int nblk, double* out, cudaStream_t st, const int* active) {
  k_breduce_norm<<<1, NT, 0, st>>>(part, nb, nblk, out, active);
}
int launch_bmdot(const z128* V, const double* Vs, size_t ld, int nv, const z128* w, size_t ne, int nb, z128* part,
                 int with_norm, cudaStream_t st, const int* active) {
  if (Vs) {  // the summed basis
    static const int nblk3 = wave_blocks(k_bmdot<z128, BAccD3>, 0);
    k_bmdot<z128, BAccD3><<<nblk3, NT, 0, st>>>(V, Vs, ld, nv, w, ne, nb, part, with_norm, active);
    return nblk3;
  }
  static const int nblk = wave_blocks(k_bmdot<z128, BAccD>, 0);
  k_bmdot<z128, BAccD><<<nblk, NT, 0, st>>>(V, nullptr, ld, nv, w, ne, nb, part, with_norm, active);
  return nblk;
}
// The double-float variants share one grid, a wave of the most resident (2-slot) kernel (the 4-
// and 8-slot ones run it in more than one wave), so the points fall into the same block ranges
// whichever variant the autotuner picks and the results are identical.
int bmdot_df_grid() {
  static const int nblk = wave_blocks(k_bmdot<zdf, BAccF, 2>, 0);
  return nblk;
}
template <int KSV>
int bmdot_df_ks(const zdf* V, size_t ld, int nv, const zdf* w, size_t ne, int nb, z128* part, int with_norm,
                cudaStream_t st, const int* active) {
  const int nblk = bmdot_df_grid();
  k_bmdot<zdf, BAccF, KSV><<<nblk, NT, 0, st>>>(V, nullptr, ld, nv, w, ne, nb, part, with_norm, active);
  return nblk;
}
int launch_bmdot_df(const zdf* V, size_t ld, int nv, const zdf* w, size_t ne, int nb, z128* part, int with_norm,
                    cudaStream_t st, const int* active, int variant) {
  switch (variant) {
    case 1: return bmdot_df_ks<2>(V, ld, nv, w, ne, nb, part, with_norm, st, active);
    case 2: return bmdot_df_ks<8>(V, ld, nv, w, ne, nb, part, with_norm, st, active);
    default: return bmdot_df_ks<4>(V, ld, nv, w, ne, nb, part, with_norm, st, active);
  }
}
void launch_bgs_update_df(const zdf* V, size_t ld, int nv, int nb, const z128* h, zdf* w, size_t ne, cudaStream_t st,
                          const int* active) {
  k_bgs_update_df<<<stream_blocks(ne), NT, sizeof(zdf) * nv * nb, st>>>(V, ld, nv, nb, h, w, ne, active);
}
template <typename TI, typename TC>
void launch_bscale_df(const TI* in, const double* s, zdf* out, cx<TC>* copy, size_t ne, int nb, cudaStream_t st,
                      const int* active) {
  k_bscale_df<TI, TC><<<stream_blocks(ne), NT, 0, st>>>(in, s, out, copy, ne, nb, active);
}
template void launch_bscale_df<z128, double>(const z128*, const double*, zdf*, z128*, size_t, int, cudaStream_t, const int*);
template void launch_bscale_df<z128, float>(const z128*, const double*, zdf*, z64*, size_t, int, cudaStream_t, const int*);
template void launch_bscale_df<zdf, double>(const zdf*, const double*, zdf*, z128*, size_t, int, cudaStream_t, const int*);
template void launch_bscale_df<zdf, float>(const zdf*, const double*, zdf*, z64*, size_t, int, cudaStream_t, const int*);
void launch_breduce_dots(const z128* part, int nv, int nb, int nblk, z128* hpass, z128* hacc, int accumulate,
                         int decide_j, const int* act, int* pass2, int* log, double* sw2, int* need, cudaStream_t st,
                         const int* active, double keep) {
  const int rows = (decide_j >= 0 ? nv + 1 : nv) * nb;
  k_breduce_dots<<<(rows + NW - 1) / NW, NT, 0, st>>>(part, nv, nb, nblk, hpass, hacc, accumulate, decide_j, sw2,
                                                      active);
  if (decide_j >= 0) k_bdecide<<<1, 32, 0, st>>>(hpass, sw2, nv, nb, decide_j, act, pass2, log, need, active, keep);
}
int launch_bmdot_sel(const z128* V, const double* Vs, size_t ld, int nv, const z128* w, size_t ne, int nb,
                     const int* need, z128* part, cudaStream_t st, const int* active) {
  // the grid of the first pass's kernel, so that the block ranges and partial slots match
  if (Vs) {
    static const int nblk3 = wave_blocks(k_bmdot<z128, BAccD3>, 0);
    k_bmdot_sel<BAccD3><<<nblk3, NT, 0, st>>>(V, Vs, ld, nv, w, ne, nb, need, part, active);
    return nblk3;
  }
  static const int nblk = wave_blocks(k_bmdot<z128, BAccD>, 0);
  k_bmdot_sel<BAccD><<<nblk, NT, 0, st>>>(V, nullptr, ld, nv, w, ne, nb, need, part, active);
  return nblk;
}
void launch_bgs_update_sel(const z128* V, const double* Vs, size_t ld, int nv, int nb, const z128* h, z128* w,
                           size_t ne, const int* need, cudaStream_t st, const int* active) {
  const size_t smem = sizeof(double3) * nv * nb;
  if (Vs)
    k_bgs_update_sel<true><<<stream_blocks(ne / nb), NT, smem, st>>>(V, Vs, ld, nv, nb, h, w, ne, need, active);
  else
    k_bgs_update_sel<false><<<stream_blocks(ne / nb), NT, smem, st>>>(V, nullptr, ld, nv, nb, h, w, ne, need, active);
}
void launch_bgs_update(const z128* V, const double* Vs, size_t ld, int nv, int nb, const z128* h, z128* w, size_t ne,
                       cudaStream_t st, const int* active) {
  if (Vs)
    k_bgs_update_sums<<<stream_blocks(ne), NT, sizeof(double3) * nv * nb, st>>>(V, Vs, ld, nv, nb, h, w, ne, active);
  else
    k_bgs_update<<<stream_blocks(ne), NT, sizeof(z128) * nv * nb, st>>>(V, ld, nv, nb, h, w, ne, active);
}
void launch_bscale_inv(const z128* in, const double* s, z128* out, double* outs, size_t ne, int nb, cudaStream_t st,
                       const int* active) {
  if (outs)
    k_bscale_inv_sums<<<stream_blocks(ne), NT, 0, st>>>(in, s, out, outs, ne, nb, active);
  else
    k_bscale_inv<<<stream_blocks(ne), NT, 0, st>>>(in, s, out, ne, nb, active);
}
void launch_bcycle_init(BatchCtl* bc, int nb, int m, double tol, cudaStream_t st) {
  k_bcycle_init<<<1, 32, 0, st>>>(bc, nb, m, tol);
}
void launch_bgivens(BatchCtl* bc, int nb, int m, int j, const z128* hcol, const double* hnorm, double tol,
                    cudaStream_t st) {
  k_bgivens<<<1, 32, 0, st>>>(bc, nb, m, j, hcol, hnorm, tol);
}
void launch_btrisolve(BatchCtl* bc, int nb, int m, cudaStream_t st) { k_btrisolve<<<1, 32, 0, st>>>(bc, nb, m); }
template <typename TZ>
void launch_bxupdate(const BatchCtl* bc, int nb, int m, const cx<TZ>* Z, size_t ld, z128* x, size_t ne,
                     cudaStream_t st) {
  k_bxupdate<TZ><<<stream_blocks(ne), NT, sizeof(z128) * m * nb, st>>>(bc, nb, m, Z, ld, x, ne);
}
template void launch_bxupdate<double>(const BatchCtl*, int, int, const z128*, size_t, z128*, size_t, cudaStream_t);
template void launch_bxupdate<float>(const BatchCtl*, int, int, const z64*, size_t, z128*, size_t, cudaStream_t);
void launch_bxupdate_df(const BatchCtl* bc, int nb, int m, const z64* Z, size_t ld, z128* x, size_t ne,
                        cudaStream_t st) {
  k_bxupdate_df<<<stream_blocks(ne), NT, sizeof(zdf) * m * nb, st>>>(bc, nb, m, Z, ld, x, ne);
}
void launch_to_batch(const z128* src, z128* dst, size_t n, int nb, int nrhs, cudaStream_t st) {
  k_to_batch<<<stream_blocks(n * nb), NT, 0, st>>>(src, dst, n, nb, nrhs);
}
void launch_from_batch(const z128* src, z128* dst, size_t n, int nb, int nrhs, cudaStream_t st) {
  k_from_batch<<<stream_blocks(n * nrhs), NT, 0, st>>>(src, dst, n, nb, nrhs);
}

}  // namespace helm
