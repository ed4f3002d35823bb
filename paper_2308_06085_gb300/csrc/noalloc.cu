// noalloc.cu -- an allocation-free entry point for callers that cannot call cudaMalloc.
//
// Some callers own a GPU but may not allocate device memory themselves: code running inside
// a host framework whose memory pool owns every device allocation, or a plug-in whose
// allocations are only allowed at start-up.  helm_vcycle_down_noalloc lets them run the
// restriction stage of the V-cycle on the finest grid without a context: they pass the grid,
// k^2, the right-hand side and the output, and the two intermediate grid vectors live in
// the file-scope device array below instead of in memory from cudaMalloc.
#include <cstdio>
#include <mutex>

#include "../../include/helm.h"
#include "internal.cuh"

namespace {

// Scratch for the pre-smoothed iterate u1 and the residual r of one fine grid:
// 2 x HELM_NOALLOC_MAX_POINTS complex128 values = 8 MiB.  Every GPU that loads the library
// holds it until the process exits.
constexpr size_t kMaxPoints = HELM_NOALLOC_MAX_POINTS;
__device__ __align__(256) z128 g_noalloc_scratch[2 * kMaxPoints];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
z128* g_scratch_ptr[kMaxDevices] = {};  // device address of the array, per device

int unknowns(int n, int bc) { return bc == HELM_BC_DIRICHLET ? n - 1 : n + 1; }

}  // namespace

// Defined in helm_api.cu: stores the message returned by helm_last_error(NULL).
void helm_set_global_error(const char* msg);

extern "C" helm_status helm_vcycle_down_noalloc(int n1, int n2, int n3, double h, const double* k2, helm_bc bc,
                                                double beta1, double beta2, double omega, const void* b, void* out,
                                                void* stream) {
  using namespace helm;
  if (n1 < 2 || n2 < 2 || n3 < 2 || n1 % 2 || n2 % 2 || n3 % 2) {
    helm_set_global_error("helm_vcycle_down_noalloc: interval counts must be even and >= 2");
    return HELM_EINVAL;
  }
  if (!(h > 0.0) || !k2 || !b || !out || (bc != HELM_BC_DIRICHLET && bc != HELM_BC_SOMMERFELD) ||
      !(omega > 0.0 && omega < 2.0)) {
    helm_set_global_error("helm_vcycle_down_noalloc: bad h, pointer, boundary condition or omega");
    return HELM_EINVAL;
  }
  Grid gf, gc;
  gf.N1 = unknowns(n1, bc); gf.N2 = unknowns(n2, bc); gf.N3 = unknowns(n3, bc);
  gc.N1 = unknowns(n1 / 2, bc); gc.N2 = unknowns(n2 / 2, bc); gc.N3 = unknowns(n3 / 2, bc);
  gf.bc = gc.bc = (int)bc;
  gf.h = h;
  gc.h = 2.0 * h;
  if (gc.N1 < 1 || gc.N2 < 1 || gc.N3 < 1) {
    helm_set_global_error("helm_vcycle_down_noalloc: the coarse grid has no unknowns");
    return HELM_EINVAL;
  }
  if (gf.npts() > kMaxPoints) {
    char msg[200];
    snprintf(msg, sizeof(msg),
             "helm_vcycle_down_noalloc: %zu fine-grid unknowns exceed the static scratch limit of %zu",
             gf.npts(), kMaxPoints);
    helm_set_global_error(msg);
    return HELM_EINVAL;
  }
  // An error left on this thread by earlier, unrelated CUDA work is the caller's: report it
  // without clearing it, so that the check after the launches below sees only this call's.
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof(msg), "helm_vcycle_down_noalloc: a CUDA error was already pending: %s",
             cudaGetErrorString(pending));
    helm_set_global_error(msg);
    return HELM_ECUDA;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    helm_set_global_error("helm_vcycle_down_noalloc: no current CUDA device");
    return HELM_ECUDA;
  }
  z128* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      // Host code cannot use the array's name as a device address: ask the runtime, once
      // per device, with that device current.
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        cudaGetLastError();
        char msg[200];
        snprintf(msg, sizeof(msg), "helm_vcycle_down_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        helm_set_global_error(msg);
        return HELM_ECUDA;
      }
      g_scratch_ptr[dev] = static_cast<z128*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  z128* u1 = scratch;
  z128* r = scratch + kMaxPoints;
  cudaStream_t st = (cudaStream_t)stream;
  // u1 = omega D^-1 b (every entry written), r = b - M u1 (every entry written),
  // out = full-weighting restriction of r.  Nothing in the scratch needs to start at zero.
  launch_smooth0<double, double>(gf, beta1, -beta2, omega, k2, nullptr, (const z128*)b, u1, st, nullptr);
  launch_resid<double, double, double, double>(gf, beta1, -beta2, k2, u1, (const z128*)b, r, st, nullptr);
  launch_restrict<double>(gf, gc, r, (z128*)out, st, nullptr);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof(msg), "helm_vcycle_down_noalloc: launch failed: %s", cudaGetErrorString(e));
    helm_set_global_error(msg);
    return HELM_ECUDA;
  }
  return HELM_OK;
}
