// vecred.cuh -- block-level helpers shared by the short-recurrence Krylov kernels
// (Bi-CGSTAB, IDR(s)): contiguous block ranges, deterministic per-block partial sums of
// complex values, and their warp-level final sum.
#pragma once

#include "internal.cuh"

namespace helm {
namespace vecred {

constexpr int NT = 256;
constexpr int NW = NT / 32;

__device__ __forceinline__ void brange(size_t n, size_t& p0, size_t& p1) {
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  p0 = blockIdx.x * chunk;
  p1 = p0 + chunk < n ? p0 + chunk : n;
  if (p0 > n) p0 = n;
}

// Write NS per-block partial sums (each a complex value) from per-thread values.
template <int NS>
__device__ __forceinline__ void block_partials(double (&re)[NS], double (&im)[NS], z128* part) {
  __shared__ double sred[NW][2 * NS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NS; ++k)
    for (int o = 16; o; o >>= 1) {
      re[k] += __shfl_xor_sync(0xffffffffu, re[k], o);
      im[k] += __shfl_xor_sync(0xffffffffu, im[k], o);
    }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      sred[warp][2 * k] = re[k];
      sred[warp][2 * k + 1] = im[k];
    }
  __syncthreads();
  if ((int)threadIdx.x < 2 * NS) {
    double t = 0.0;
    for (int w = 0; w < NW; ++w) t += sred[w][threadIdx.x];
    reinterpret_cast<double*>(part)[2 * ((size_t)(threadIdx.x >> 1) * RED_STRIDE + blockIdx.x) + (threadIdx.x & 1)] = t;
  }
}

// Sum of one slot's partials by a full warp (lanes stride the blocks, then a fixed tree).
__device__ __forceinline__ z128 sum_slot(const z128* part, int slot, int nb) {
  const int lane = threadIdx.x & 31;
  double re = 0.0, im = 0.0;
  for (int b = lane; b < nb; b += 32) {
    re += part[(size_t)slot * RED_STRIDE + b].re;
    im += part[(size_t)slot * RED_STRIDE + b].im;
  }
  for (int o = 16; o; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  return mkc<double>(re, im);
}

__device__ __forceinline__ z128 cdiv(z128 a, z128 b) {
  const double d = b.re * b.re + b.im * b.im;
  return mkc<double>((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}

// Blocks for a one-wave grid of kernel `kern` at NT threads, capped at RED_STRIDE.
template <typename K>
inline int wave(K kern) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NT, 0);
  const int nb = sms * (per > 0 ? per : 1);
  return nb < RED_STRIDE ? nb : RED_STRIDE;
}

inline int sblocks(size_t n) {
  size_t b = (n + NT - 1) / NT;
  return (int)(b < 1216 ? (b > 0 ? b : 1) : 1216);
}

}  // namespace vecred
}  // namespace helm
