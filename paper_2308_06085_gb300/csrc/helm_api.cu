// helm_api.cu -- the C ABI of libhelm (include/helm.h): context and multigrid hierarchy
// set-up, the V-cycle driver, and the host side of right-preconditioned GMRES(m) /
// FGMRES(m).  All grid arithmetic runs in the kernels of stencil.cu and krylov.cu; the host
// only orders launches, except at set-up, where it inverts the small coarsest-grid matrix.
#include <algorithm>
#include <chrono>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/helm.h"
#include "internal.cuh"

using namespace helm;

namespace {

constexpr int MAX_LEVELS = 32;
constexpr int MAX_COARSE = 4096;  // unknowns of the dense coarsest solve
constexpr int TYT_TILED = 8;      // rows of the tiled FP32 stencil CTAs (stencil.cu)
constexpr int FLAG_LAG = 2;       // Arnoldi steps enqueued ahead of the host's flag check

// Message of the last failing context-free call (helm_create, helm_vcycle_down_noalloc) on
// this host thread, read by helm_last_error(NULL).  One slot per thread: concurrent failing
// calls on different threads never share the string.
thread_local std::string g_create_error;

struct Level {
  int n1, n2, n3;
  Grid g;
  double* k2 = nullptr;    // FP64 k^2
  float* k2f = nullptr;    // FP32 copy
  double* sk = nullptr;    // sqrt(k^2), FP64 (face terms)
  float* skf = nullptr;    // sqrt(k^2), FP32
  z128* dinv = nullptr;    // FP64 path: omega / diag(M) at [0, npts), diag(M) at [npts, 2 npts)
  // V-cycle work vectors: B = right-hand side (levels >= 1), U1 = pre-smoothed iterate,
  // T = residual / corrected iterate, E = result (levels >= 1)
  z128 *B64 = nullptr, *U164 = nullptr, *T64 = nullptr, *E64 = nullptr;
  z64 *B32 = nullptr, *U132 = nullptr, *T32 = nullptr, *E32 = nullptr;
};

template <typename R> struct LevelBufs;
template <> struct LevelBufs<double> {
  static z128* B(Level& L) { return L.B64; }
  static z128* U1(Level& L) { return L.U164; }
  static z128* T(Level& L) { return L.T64; }
  static z128* E(Level& L) { return L.E64; }
  static const double* k2(Level& L) { return L.k2; }
  static const z128* dinv(Level& L) { return L.dinv; }
};
template <> struct LevelBufs<float> {
  static z64* B(Level& L) { return L.B32; }
  static z64* U1(Level& L) { return L.U132; }
  static z64* T(Level& L) { return L.T32; }
  static z64* E(Level& L) { return L.E32; }
  static const float* k2(Level& L) { return L.k2f; }
  static const z64* dinv(Level&) { return nullptr; }
};

// Kernel families for the opt-in profiler (names match the kernel functions).
enum Fam {
  F_APPLY, F_RESID, F_JACOBI, F_SMOOTH0, F_RESTRICT, F_PROLONG, F_COARSE, F_MDOT, F_REDUCE_DOTS, F_GS_UPDATE,
  F_NORM, F_REDUCE_NORM, F_SCALE, F_GIVENS, F_SOLUPDATE, F_MISC, F_CCYCLE, F_DOWN, F_UP, F_RR,
  // the same multigrid kernels on the finest level, where the bytes are (kept apart so that
  // their roofline can be read off directly)
  F_SMOOTH0_F, F_RESID_F, F_RESTRICT_F, F_PROLONG_F, F_JACOBI_F, F_DOWN_F, F_UP_F, F_RR_F, F_COUNT
};
const char* const FAM_NAMES[F_COUNT] = {
    "k_stencil(apply)", "k_stencil(resid)", "k_stencil(jacobi)", "k_smooth0", "k_restrict", "k_prolong_add",
    "k_coarse", "k_mdot", "k_reduce_dots", "k_gs_update", "k_norm2_part", "k_reduce_norm", "k_scale_inv",
    "k_givens", "k_xupdate/k_combine/k_axpy1/k_trisolve", "other", "k_coarse_cycle", "k_down32", "k_up", "k_rr",
    "k_smooth0 (finest)", "k_stencil(resid) (finest)", "k_restrict (finest)", "k_prolong_add (finest)",
    "k_stencil(jacobi) (finest)", "k_down32 (finest)", "k_up (finest)", "k_rr (finest)"};

struct TuneRec {
  int level, slot, ty, ctas;
  float ms;
};

struct ProfRec {
  int fam, j, e0, e1;
  int cond;  // 1: second Gram-Schmidt pass, which ran only if the step's log entry is set; 2: the
             // same, with bytes and flops per right-hand side times the logged count
  double bytes, flops;
};

struct Prof {
  bool on = false;
  long long launches = 0;  // every kernel launch of this context, always counted
  double ms[F_COUNT] = {}, bytes[F_COUNT] = {}, flops[F_COUNT] = {};
  long long cnt[F_COUNT] = {};
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  int used = 0;
};

// Workspace of the batched solver for nb right-hand sides (allocated on first use, grown when a
// wider batch is asked for).
struct BatchWS {
  int nb = 0;
  // tuned launch shapes per batch width 2^t: the V-cycle grids of every level and the FP64
  // finest-level operator
  bool tuned[6] = {};
  int bmdot_variant[6] = {};  // slots per warp pass of the double-float dots, per width
  int tty[6][MAX_LEVELS][8] = {}, tct[6][MAX_LEVELS][8] = {};
  int g0ty[6][8] = {}, g0ct[6][8] = {};
  z128 *V = nullptr, *Z64 = nullptr, *w = nullptr, *r = nullptr, *Bt = nullptr, *Xt = nullptr;
  double* Vs = nullptr;     // (m+1) x ne element sums Re V + Im V (FP64 Gram-Schmidt, gs_sums)
  int* need = nullptr;      // per right-hand side: the current step takes the second Gram-Schmidt pass
  z64* Z32 = nullptr;
  zdf* wdf = nullptr;       // Arnoldi vector, double-float Gram-Schmidt
  z128* vcur64 = nullptr;   // V-cycle input copy of v_j (double-float basis, FP64 V-cycle)
  z64* vcur32 = nullptr;    // V-cycle input copy of v_j (double-float basis, mixed precision)
  z128 *part = nullptr, *hpass = nullptr, *hacc = nullptr;
  double *partr = nullptr, *hnorm = nullptr;
  double* sw2 = nullptr;    // |w|^2 per right-hand side for the reorthogonalisation test
  BatchCtl h;               // host copy of the device pointers
  BatchCtl* ctl = nullptr;  // device
  int* log = nullptr;
  z128 *B64[MAX_LEVELS] = {}, *U164[MAX_LEVELS] = {}, *T64[MAX_LEVELS] = {}, *E64[MAX_LEVELS] = {};
  z64 *B32[MAX_LEVELS] = {}, *U132[MAX_LEVELS] = {}, *T32[MAX_LEVELS] = {}, *E32[MAX_LEVELS] = {};
  int* hany = nullptr;  // pinned, one slot per Arnoldi step
};

}  // namespace

struct helm_ctx {
  helm_params p;
  int bc = 0;
  int nlev = 0;
  Level L[MAX_LEVELS];
  int nc = 0;
  z128* Minv = nullptr;
  // the paper's coarsest-grid GMRES (coarse_tol > 0): basis, Hessenberg columns, last report
  z128 *cgV = nullptr, *cgH = nullptr;
  int* cginfo = nullptr;
  // Krylov workspace
  int m = 0;
  size_t n0 = 0;
  z128* V = nullptr;      // (m+1) x n0
  double* Vs = nullptr;   // (m+1) x n0 element sums Re V + Im V of the FP64 basis (gs_sums)
  z128* Z64 = nullptr;    // m x n0, FGMRES in FP64
  z64* Z32 = nullptr;     // m x n0, mixed precision
  z128* zs = nullptr;     // n0 scratch (V-cycle output, GMRES)
  zdf* wdf = nullptr;     // n0 new Arnoldi vector, double-float (double-float basis)
  z128* vcur64 = nullptr; // V-cycle input v_j as c128 (double-float basis, FP64 V-cycle)
  z64* vcur32 = nullptr;  // V-cycle input v_j as c64 (double-float basis, mixed precision)
  z128* r = nullptr;      // n0 residual
  z128* xs = nullptr;     // staging for host x
  z128* bs = nullptr;     // staging for host b
  z128* part = nullptr;   // (m+2) x RED_STRIDE partial dots
  double* partr = nullptr;
  z128 *hpass = nullptr, *hacc = nullptr;
  z128* H = nullptr;
  double* cs = nullptr;
  z128* sn = nullptr;
  z128* gv = nullptr;
  z128* y = nullptr;
  double* hnorm = nullptr;
  double* hist = nullptr;
  int hist_len = 0;
  KrylovCtl* ctl = nullptr;
  int* one = nullptr;
  int* rhs_idx = nullptr;
  int rhs_cap = 0;
  int* hflags = nullptr;  // pinned
  KrylovCtl* hctl = nullptr;  // pinned
  cudaEvent_t ev[FLAG_LAG + 2];
  int nev = 0;
  std::vector<void*> allocs;
  std::string err;
  double s_re = 1.0, s_im = 0.0;  // CSLP shift beta1 - beta2 i
  Prof prof;
  int cur_j = -1;  // Arnoldi column being enqueued (-1 outside the Arnoldi loop)
  int cur_cond = 0;
  int* reorth_log = nullptr;   // device, per Arnoldi step: second pass taken
  int* hreorth_log = nullptr;  // pinned host copy
  long long reorth_steps = 0, arnoldi_steps = 0;
  // adjoint-state gradient buffers (allocated on first use)
  z128 *adj_u = nullptr, *adj_g = nullptr, *adj_l = nullptr;
  // batched adjoint gradient: wavefields, receiver residuals and adjoint states of every source
  z128 *adj_U = nullptr, *adj_G = nullptr, *adj_L = nullptr;
  int adj_cap = 0;
  double* adj_part = nullptr;
  double* adj_norm = nullptr;
  int* adj_rec = nullptr;
  int adj_rec_cap = 0;
  BatchWS bw;
  BicgCtl* bicg = nullptr;  // device
  BicgCtl* hbicg = nullptr; // pinned
  // (hi, lo) tables of k^2 and k on the finest level for the double-float A-product of the
  // mixed-precision solver (allocated for mixed precision with double-float Gram-Schmidt)
  float2* k2df = nullptr;
  float2* skdf = nullptr;
  // CUDA graphs of whole solver steps, captured on gstream on first use and replayed on the
  // caller's stream (keyed by step kind, step index and a caller pointer the step writes)
  struct GraphEnt {
    int tag, j;
    const void* p;
    cudaGraphExec_t exec;
    long long launches;
  };
  std::vector<GraphEnt> graphs;
  std::vector<TuneRec> tune_log;  // every launch shape the autotuner timed
  int mdot_df_variant = 0;        // slots per warp pass of the double-float inner products
  int mdot_variant = 0;           // FP64 inner products: 0 w staged in shared memory, 1 not
  cudaStream_t gstream = nullptr;
  // IDR(s): shadow space P (s vectors), work G, U (s each), r, v, vh, t; control block
  int idr_s = 0;
  z128* idrP = nullptr;
  z128* idrW = nullptr;
  z128* idr_part = nullptr;  // (IDR_SMAX + 1) x RED_STRIDE
  IdrCtl* idr = nullptr;     // device
  IdrCtl* hidr = nullptr;    // pinned
};

namespace {

helm_status fail(helm_ctx* c, helm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_create_error = buf;
  return st;
}

#define CU(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(c, HELM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
helm_status dalloc(helm_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return HELM_OK;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, HELM_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", count * sizeof(T), cudaGetErrorString(e));
  }
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return HELM_OK;
}

// Free one allocation made by dalloc (and forget it).
void dfree(helm_ctx* c, void* p) {
  if (!p) return;
  for (size_t i = 0; i < c->allocs.size(); ++i)
    if (c->allocs[i] == p) {
      cudaFree(p);
      c->allocs.erase(c->allocs.begin() + (long)i);
      return;
    }
}

#define TRY(x)                          \
  do {                                  \
    helm_status s_ = (x);               \
    if (s_ != HELM_OK) return s_;       \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int unknowns(int n, int bc) { return bc == HELM_BC_DIRICHLET ? n - 1 : n + 1; }

helm_status check_launch(helm_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, HELM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return HELM_OK;
}

int prof_event(helm_ctx* c) {
  Prof& P = c->prof;
  if (P.used == (int)P.pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    P.pool.push_back(e);
  }
  return P.used++;
}

void prof_pre(helm_ctx* c, cudaStream_t st, int& e0) {
  ++c->prof.launches;
  e0 = -1;
  if (!c->prof.on) return;
  e0 = prof_event(c);
  if (e0 >= 0) cudaEventRecord(c->prof.pool[e0], st);
}

void prof_post(helm_ctx* c, cudaStream_t st, int e0, int fam, double bytes, double flops) {
  if (!c->prof.on || e0 < 0) return;
  const int e1 = prof_event(c);
  if (e1 < 0) return;
  cudaEventRecord(c->prof.pool[e1], st);
  c->prof.recs.push_back(ProfRec{fam, c->cur_j, e0, e1, c->cur_cond, bytes, flops});
}

// Fold timed launches into the totals once their events completed.  Launches of Arnoldi
// columns beyond `jend` returned at once (the cycle had stopped) and are dropped.
void prof_flush(helm_ctx* c, int jend) {
  Prof& P = c->prof;
  if (!P.on || P.recs.empty()) { P.used = 0; P.recs.clear(); return; }
  cudaEventSynchronize(P.pool[P.recs.back().e1]);
  for (const ProfRec& r : P.recs) {
    if (r.j >= 0 && r.j > jend) continue;
    if (r.cond && r.j >= 0 && !c->hreorth_log[r.j]) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, P.pool[r.e0], P.pool[r.e1]) != cudaSuccess) { cudaGetLastError(); continue; }
    // cond 2: bytes and flops were given per right-hand side; the log holds how many took part
    const double f = r.cond == 2 && r.j >= 0 ? (double)c->hreorth_log[r.j] : 1.0;
    P.ms[r.fam] += ms;
    P.bytes[r.fam] += r.bytes * f;
    P.flops[r.fam] += r.flops * f;
    P.cnt[r.fam] += 1;
  }
  P.recs.clear();
  P.used = 0;
}

// Launch wrapper: counts the launch and, when profiling, brackets it with events.
#define KL(fam, bytes, flops, stmt)                      \
  do {                                                   \
    int e0_;                                             \
    prof_pre(c, st, e0_);                                \
    stmt;                                                \
    prof_post(c, st, e0_, fam, (double)(bytes), (double)(flops)); \
  } while (0)

// Profiler family of a multigrid kernel on grid g: its finest-level family when g is the
// finest grid (any batch width).
int vfam(const helm_ctx* c, const Grid& g, int fam) {
  const Grid& g0 = c->L[0].g;
  if (g.N1 != g0.N1 || g.N2 != g0.N2 || g.N3 != g0.N3) return fam;
  switch (fam) {
    case F_SMOOTH0: return F_SMOOTH0_F;
    case F_RESID: return F_RESID_F;
    case F_RESTRICT: return F_RESTRICT_F;
    case F_PROLONG: return F_PROLONG_F;
    case F_JACOBI: return F_JACOBI_F;
    case F_DOWN: return F_DOWN_F;
    case F_UP: return F_UP_F;
    case F_RR: return F_RR_F;
    default: return fam;
  }
}

// Dense coarsest operator M_L (row-major), entries as in the grid kernels: diagonal
// 6/h^2 - s k^2 - i (2 k / h) per Sommerfeld face, -1/h^2 per in-grid neighbour, and a
// neighbour beyond a Sommerfeld face folded onto the opposite node (ghost elimination).
void assemble_coarse(const Level& L, int bc, std::complex<double> s, const std::vector<double>& k2,
                     std::vector<std::complex<double>>& A) {
  const int N1 = L.g.N1, N2 = L.g.N2, N3 = L.g.N3;
  const int n = N1 * N2 * N3;
  const double h = L.g.h, ih2 = 1.0 / (h * h);
  A.assign((size_t)n * n, 0.0);
  for (int k = 0; k < N3; ++k)
    for (int j = 0; j < N2; ++j)
      for (int i = 0; i < N1; ++i) {
        const int p = (k * N2 + j) * N1 + i;
        int nf = 0;
        auto add = [&](int ii, int jj, int kk, int oi, int oj, int ok) {
          if (ii >= 0 && ii < N1 && jj >= 0 && jj < N2 && kk >= 0 && kk < N3) {
            A[(size_t)p * n + (kk * N2 + jj) * N1 + ii] += -ih2;
          } else if (bc == HELM_BC_SOMMERFELD) {
            ++nf;
            A[(size_t)p * n + (ok * N2 + oj) * N1 + oi] += -ih2;
          }
        };
        add(i - 1, j, k, i + 1, j, k);
        add(i + 1, j, k, i - 1, j, k);
        add(i, j - 1, k, i, j + 1, k);
        add(i, j + 1, k, i, j - 1, k);
        add(i, j, k - 1, i, j, k + 1);
        add(i, j, k + 1, i, j, k - 1);
        std::complex<double> d = 6.0 * ih2 - s * k2[p];
        if (nf) d += std::complex<double>(0.0, -2.0 * std::sqrt(k2[p]) / h * nf);
        A[(size_t)p * n + p] += d;
      }
}


// One V-cycle z ~= M^{-1} r in working precision R (input type TI, output type TO).
// Buffers and grid of one V-cycle level (single or batched right-hand sides).
template <typename R>
struct VLevel {
  Grid g;
  const R* k2;
  const cx<R>* dinv;
  cx<R> *B, *U1, *T, *E;
};

// Whether level F runs its pre-smoothing and residual as one kernel, and that launch (u1 into
// F.U1, the residual into F.T).
template <typename R>
bool down_fused(const VLevel<R>& F) {
  return std::is_same<R, float>::value && F.g.nb == 1 && F.g.fused_down;
}
template <typename R, typename TB>
void down_fused_launch(const VLevel<R>& F, double sr, double si, double om, const cx<TB>* b, cudaStream_t st,
                       const int* active) {
  if constexpr (std::is_same<R, float>::value)
    launch_smooth0_resid32<TB>(F.g, sr, si, om, F.k2, b, F.U1, F.T, st, active);
}
// Whether level F runs its whole down-sweep (pre-smoothing, residual, restriction into C.B) as
// one kernel, and that launch.
template <typename R>
bool down_full(const VLevel<R>& F) {
  return std::is_same<R, float>::value && F.g.nb == 1 && F.g.down_full;
}
// Whether level F runs its whole up-sweep (prolongation, correction, post-smoothing) as one
// kernel, and that launch (FP32, or FP64 with complex128 input and output).
template <typename R>
bool up_full(const VLevel<R>& F) {
  return F.g.nb == 1 && F.g.up_full;
}
template <typename R, typename TB, typename TO>
void up_full_launch(const VLevel<R>& F, const VLevel<R>& C, double sr, double si, double om, const cx<TB>* b,
                    cx<TO>* out, cudaStream_t st, const int* active) {
  if constexpr (std::is_same<R, float>::value || (std::is_same<TB, double>::value && std::is_same<TO, double>::value))
    launch_up<R, TB, TO>(F.g, C.g, sr, si, om, F.k2, F.dinv, F.U1, C.E, b, out, F.g.up_kz, st, active);
}
// Whether level F runs its residual and restriction (into C.B) as one kernel after the
// pre-smoothing, and that launch.
template <typename R>
bool rr_full(const VLevel<R>& F) {
  return F.g.nb == 1 && F.g.rr_full;
}
template <typename R, typename TB>
void rr_launch(const VLevel<R>& F, const VLevel<R>& C, double sr, double si, const cx<TB>* b, cudaStream_t st,
               const int* active) {
  if constexpr (std::is_same<R, float>::value || std::is_same<TB, double>::value)
    launch_rr<R, TB>(F.g, C.g, sr, si, F.k2, F.dinv, F.U1, b, C.B, F.g.rr_kc, st, active);
}
template <typename R, typename TB>
void down_full_launch(const VLevel<R>& F, const VLevel<R>& C, double sr, double si, double om, const cx<TB>* b,
                      cudaStream_t st, const int* active) {
  if constexpr (std::is_same<R, float>::value)
    launch_down32<TB>(F.g, C.g, sr, si, om, F.k2, b, F.U1, C.B, F.g.down_kc, st, active);
}

// Levels from which the rest of a V-cycle over lv[0..L) runs in one CTA (k_coarse_cycle):
// the first relative level lf >= 1 whose sub-cycle (at least two levels, one right-hand side)
// fits the shared-memory budget, with its vectors laid out in *cc and the byte count in
// *bytes; L when none fits or the context runs without it.
// The coarsest-grid solve e = M_c^{-1} b: the precomputed dense inverse, or with coarse_tol > 0
// (one right-hand side) the paper's GMRES to that relative residual.
template <typename TI, typename TO>
void coarse_solve(helm_ctx* c, const cx<TI>* b, cx<TO>* e, cudaStream_t st, const int* active, int nb) {
  if (c->p.coarse_tol > 0.0 && nb == 1) {
    const Level& Lc = c->L[c->nlev - 1];
    launch_coarse_gmres<TI, TO>(Lc.g, c->s_re, c->s_im, Lc.k2, b, e, c->cgV, c->cgH, c->p.coarse_tol,
                                c->p.reorth_keep, c->cginfo, st, active);
  } else {
    launch_coarse<TI, TO>(c->nc, c->Minv, b, e, st, active, nb);
  }
}

template <typename R>
int plan_coarse_cycle(helm_ctx* c, const VLevel<R>* lv, int L, CCycle<R>* cc, size_t* bytes) {
  if (!c->p.fuse_coarse || lv[0].g.nb != 1 || !coarse_cycle_ready<R>() || c->p.coarse_tol > 0.0) return L;
  for (int lf = 1; lf <= L - 2; ++lf) {
    if (L - lf > CC_MAX_LEVELS) continue;
    // layout in units of cx<R>: per level B, U (and T), then the FP64 omega/d copy, then the
    // k^2 and sqrt(k^2) copies (two R per cx<R> slot)
    size_t off = 0;
    for (int l = lf; l < L; ++l) {
      const size_t n = lv[l].g.npts();
      const size_t nv = (l == L - 1) ? 2 : 3;
      CLevel<R>& C = cc->lev[l - lf];
      C.g = lv[l].g;
      C.k2 = lv[l].k2;
      C.dinv = lv[l].dinv;
      C.off_b = (int)off;
      C.off_u = (int)(off + n);
      C.off_t = l == L - 1 ? -1 : (int)(off + 2 * n);
      off += nv * n;
      C.off_d = -1;
      if (lv[l].dinv) {
        C.off_d = (int)off;
        off += n;
      }
      C.off_k = (int)(2 * off);      // in units of R
      C.off_s = (int)(2 * off + n);
      off += n;                      // 2 n values of R
    }
    const size_t b = off * sizeof(cx<R>);
    if (b <= CC_SMEM_MAX) {
      cc->L = L - lf;
      cc->nc = c->nc;
      cc->Minv = c->Minv;
      cc->s_re = c->s_re;
      cc->s_im = c->s_im;
      cc->omega = c->p.omega;
      *bytes = b;
      return lf;
    }
  }
  return L;
}

// One V-cycle z ~= M^{-1} r in working precision R (input type TI, output type TO) over the
// levels lv[0..L); g.nb right-hand sides per node.
template <typename R, typename TI, typename TO>
void run_vcycle_levels(helm_ctx* c, const VLevel<R>* lv, int L, const cx<TI>* rin, cx<TO>* zout, cudaStream_t st,
                       const int* active) {
  const double sr = c->s_re, si = c->s_im, om = c->p.omega;
  const int nbv = lv[0].g.nb;
  const double cb = 2.0 * sizeof(R) * nbv;  // bytes of one node's complex values
  const double kb = sizeof(R), ib = 2.0 * sizeof(TI) * nbv, ob = 2.0 * sizeof(TO) * nbv;
  const double db = lv[0].dinv ? 16.0 : 0.0;  // omega/d array (FP64 path)
  const double kd = db ? 16.0 : kb;            // the diagonal: FP64 table of d, or k^2
  const double nc = c->nc;
  if (L == 1) {
    KL(F_COARSE, nc * nc * 16 + nc * (ib + ob), 8 * nc * nc * nbv,
       (coarse_solve<TI, TO>(c, rin, zout, st, active, nbv)));
    return;
  }
  // levels lf.. run as one single-CTA sub-cycle when they fit in shared memory
  CCycle<R> cc;
  size_t cc_bytes = 0;
  const int lf = plan_coarse_cycle<R>(c, lv, L, &cc, &cc_bytes);
  const int Ld = lf < L ? lf + 1 : L;  // levels run kernel by kernel, the sub-cycle's first included
  // A complex128 input to a complex64 cycle (one right-hand side, separate kernels on the
  // finest level) is converted once: the pre-smoothing writes b in complex64 to the level's B
  // buffer, which the residual and the post-smoothing then read (same values, half the bytes,
  // no FP64 -> FP32 conversion in either).
  const bool b32 = std::is_same<R, float>::value && !std::is_same<TI, float>::value && nbv == 1 && Ld > 1 &&
                   lv[0].B != nullptr && !down_full(lv[0]) && !down_fused(lv[0]) && !rr_full(lv[0]);
  // down: pre-smooth from zero, residual, restriction
  for (int l = 0; l < Ld - 1; ++l) {
    const VLevel<R>& F = lv[l];
    const VLevel<R>& C = lv[l + 1];
    const double n = (double)F.g.npts(), ncn = (double)C.g.npts();
    const double bi = l == 0 ? ib : cb;
    if (down_full(F)) {
      // pre-smoothing, residual and restriction in one kernel (FP32, one right-hand side)
      if (l == 0) KL(vfam(c, F.g, F_DOWN), n * (bi + kb + cb) + ncn * cb, 60 * n, down_full_launch(F, C, sr, si, om, rin, st, active));
      else KL(vfam(c, F.g, F_DOWN), n * (bi + kb + cb) + ncn * cb, 60 * n, down_full_launch(F, C, sr, si, om, F.B, st, active));
      continue;
    }
    // the residual and its restriction as one kernel after the pre-smoothing (one right-hand side)
    const bool rr = rr_full(F);
    if (down_fused(F) && !rr) {
      // u1 and the residual in one kernel (FP32, one right-hand side)
      if (l == 0) KL(vfam(c, F.g, F_SMOOTH0), n * (bi + kb + 2 * cb), 30 * n, down_fused_launch(F, sr, si, om, rin, st, active));
      else KL(vfam(c, F.g, F_SMOOTH0), n * (bi + kb + 2 * cb), 30 * n, down_fused_launch(F, sr, si, om, F.B, st, active));
    } else if (l == 0 && b32) {
      KL(vfam(c, F.g, F_SMOOTH0), n * (bi + kb + 2 * cb), 6 * n, (launch_smooth0<R, TI>(F.g, sr, si, om, F.k2, F.dinv, rin, F.U1, st, active, F.B)));
      KL(vfam(c, F.g, F_RESID), n * (3 * cb + kd), 24 * n, (launch_resid<R, R, R, R>(F.g, sr, si, F.k2, F.U1, F.B, F.T, st, active, F.dinv)));
    } else if (l == 0) {
      KL(vfam(c, F.g, F_SMOOTH0), n * (bi + (db ? db : kb) + cb), 6 * n * nbv, (launch_smooth0<R, TI>(F.g, sr, si, om, F.k2, F.dinv, rin, F.U1, st, active)));
      if (rr) KL(vfam(c, F.g, F_RR), n * (cb + bi + kd) + ncn * cb, 24 * n + 54 * ncn, rr_launch(F, C, sr, si, rin, st, active));
      else KL(vfam(c, F.g, F_RESID), n * (cb + bi + kd + cb), 24 * n * nbv, (launch_resid<R, R, TI, R>(F.g, sr, si, F.k2, F.U1, rin, F.T, st, active, F.dinv)));
    } else {
      KL(vfam(c, F.g, F_SMOOTH0), n * (bi + (db ? db : kb) + cb), 6 * n * nbv, (launch_smooth0<R, R>(F.g, sr, si, om, F.k2, F.dinv, F.B, F.U1, st, active)));
      if (rr) KL(vfam(c, F.g, F_RR), n * (cb + bi + kd) + ncn * cb, 24 * n + 54 * ncn, rr_launch(F, C, sr, si, F.B, st, active));
      else KL(vfam(c, F.g, F_RESID), n * (cb + bi + kd + cb), 24 * n * nbv, (launch_resid<R, R, R, R>(F.g, sr, si, F.k2, F.U1, F.B, F.T, st, active, F.dinv)));
    }
    if (!rr) KL(vfam(c, F.g, F_RESTRICT), n * cb + ncn * cb, 54 * ncn * nbv, (launch_restrict<R>(F.g, C.g, F.T, C.B, st, active)));
  }
  if (lf < L) {
    // the sub-cycle lv[lf].B -> lv[lf].E in one CTA
    KL(F_CCYCLE, 2.0 * cb * lv[lf].g.npts() + nc * nc * 16, 8 * nc * nc,
       launch_coarse_cycle<R>(cc, cc_bytes, lv[lf].B, lv[lf].E, st, active));
  } else {
    // coarsest: exact FP64 solve
    KL(F_COARSE, nc * nc * 16 + nc * 2 * cb, 8 * nc * nc * nbv,
       (coarse_solve<R, R>(c, lv[L - 1].B, lv[L - 1].E, st, active, nbv)));
  }
  // up: prolongation + correction, post-smoothing
  for (int l = Ld - 2; l >= 0; --l) {
    const VLevel<R>& F = lv[l];
    const VLevel<R>& C = lv[l + 1];
    const double n = (double)F.g.npts(), ncn = (double)C.g.npts();
    if (up_full(F)) {
      // prolongation, correction and post-smoothing in one kernel (one right-hand side)
      if (l == 0 && b32)
        KL(vfam(c, F.g, F_UP), n * (2 * cb + kb + ob) + ncn * cb, 40 * n, up_full_launch(F, C, sr, si, om, F.B, zout, st, active));
      else if (l == 0)
        KL(vfam(c, F.g, F_UP), n * (cb + ib + (db ? kd + db : kb) + ob) + ncn * cb, 40 * n, up_full_launch(F, C, sr, si, om, rin, zout, st, active));
      else
        KL(vfam(c, F.g, F_UP), n * (3 * cb + (db ? kd + db : kb)) + ncn * cb, 40 * n, up_full_launch(F, C, sr, si, om, F.B, F.E, st, active));
      continue;
    }
    KL(vfam(c, F.g, F_PROLONG), n * 2 * cb + ncn * cb, 6 * n * nbv, (launch_prolong_add<R>(F.g, C.g, F.U1, C.E, F.T, st, active)));
    if (l == 0 && b32)
      KL(vfam(c, F.g, F_JACOBI), n * (2 * cb + kd + ob), 32 * n, (launch_jacobi<R, R, TO>(F.g, sr, si, om, F.k2, F.dinv, F.T, F.B, zout, st, active)));
    else if (l == 0)
      KL(vfam(c, F.g, F_JACOBI), n * (cb + ib + kd + db + ob), 32 * n * nbv, (launch_jacobi<R, TI, TO>(F.g, sr, si, om, F.k2, F.dinv, F.T, rin, zout, st, active)));
    else
      KL(vfam(c, F.g, F_JACOBI), n * (3 * cb + kd + db), 32 * n * nbv, (launch_jacobi<R, R, R>(F.g, sr, si, om, F.k2, F.dinv, F.T, F.B, F.E, st, active)));
  }
}

template <typename R, typename TI, typename TO>
void run_vcycle(helm_ctx* c, const cx<TI>* rin, cx<TO>* zout, cudaStream_t st, const int* active) {
  using B = LevelBufs<R>;
  VLevel<R> lv[MAX_LEVELS];
  for (int l = 0; l < c->nlev; ++l) {
    Level& L = c->L[l];
    lv[l] = VLevel<R>{L.g, B::k2(L), B::dinv(L), B::B(L), B::U1(L), B::T(L), B::E(L)};
  }
  run_vcycle_levels<R, TI, TO>(c, lv, c->nlev, rin, zout, st, active);
}

// V-cycle on level l > 0 started from u (in place): Jacobi from u, residual, restriction, a
// zero-start V-cycle below, correction, Jacobi.  The level's U1 holds the smoothed iterate: it
// is free here because the F-cycle on this level has already returned.
template <typename R>
void vcycle_from(helm_ctx* c, const VLevel<R>* lv, int L, int l, cudaStream_t st, const int* active) {
  const double sr = c->s_re, si = c->s_im, om = c->p.omega;
  const VLevel<R>& F = lv[l];
  const double nc = c->nc, cb = 2.0 * sizeof(R), kb = sizeof(R), db = F.dinv ? 16.0 : 0.0, kd = db ? 16.0 : kb;
  if (l == L - 1) {
    KL(F_COARSE, nc * nc * 16 + nc * 2 * cb, 8 * nc * nc, (coarse_solve<R, R>(c, F.B, F.E, st, active, F.g.nb)));
    return;
  }
  const VLevel<R>& C = lv[l + 1];
  const double n = (double)F.g.npts() * F.g.nb, ncn = (double)C.g.npts() * C.g.nb;
  KL(vfam(c, F.g, F_JACOBI), n * (3 * cb + kd + db), 32 * n, (launch_jacobi<R, R, R>(F.g, sr, si, om, F.k2, F.dinv, F.E, F.B, F.U1, st, active)));
  if (rr_full(F)) {
    KL(vfam(c, F.g, F_RR), n * (2 * cb + kd) + ncn * cb, 24 * n + 54 * ncn, rr_launch(F, C, sr, si, F.B, st, active));
  } else {
    KL(vfam(c, F.g, F_RESID), n * (3 * cb + kd), 24 * n, (launch_resid<R, R, R, R>(F.g, sr, si, F.k2, F.U1, F.B, F.T, st, active, F.dinv)));
    KL(vfam(c, F.g, F_RESTRICT), n * cb + ncn * cb, 54 * ncn, (launch_restrict<R>(F.g, C.g, F.T, C.B, st, active)));
  }
  run_vcycle_levels<R, R, R>(c, lv + l + 1, L - l - 1, C.B, C.E, st, active);
  if (up_full(F)) {
    KL(vfam(c, F.g, F_UP), n * (3 * cb + (db ? kd + db : kb)) + ncn * cb, 40 * n, up_full_launch(F, C, sr, si, om, F.B, F.E, st, active));
    return;
  }
  KL(vfam(c, F.g, F_PROLONG), n * 2 * cb + ncn * cb, 6 * n, (launch_prolong_add<R>(F.g, C.g, F.U1, C.E, F.T, st, active)));
  KL(vfam(c, F.g, F_JACOBI), n * (3 * cb + kd + db), 32 * n, (launch_jacobi<R, R, R>(F.g, sr, si, om, F.k2, F.dinv, F.T, F.B, F.E, st, active)));
}

// F-cycle (Sec. 3.4.5) from level l down: pre-smoothing from zero, residual, restriction; the
// coarse-grid error is an F-cycle on the next level followed by one V-cycle there, started from
// it; correction and post-smoothing.  Level l + 1 keeps its right-hand side in B and its error
// in E throughout.
template <typename R, typename TI, typename TO>
void fcycle_levels(helm_ctx* c, const VLevel<R>* lv, int L, int l, const cx<TI>* rin, cx<TO>* zout,
                   cudaStream_t st, const int* active) {
  const double sr = c->s_re, si = c->s_im, om = c->p.omega;
  const double nc = c->nc, cb = 2.0 * sizeof(R), kb = sizeof(R), ib = 2.0 * sizeof(TI), ob = 2.0 * sizeof(TO);
  if (l == L - 1) {
    KL(F_COARSE, nc * nc * 16 + nc * (ib + ob), 8 * nc * nc,
       (coarse_solve<TI, TO>(c, rin, zout, st, active, lv[l].g.nb)));
    return;
  }
  const VLevel<R>& F = lv[l];
  const VLevel<R>& C = lv[l + 1];
  const double n = (double)F.g.npts() * F.g.nb, ncn = (double)C.g.npts() * C.g.nb, db = F.dinv ? 16.0 : 0.0;
  const double kd = db ? 16.0 : kb;
  if (down_full(F)) {
    KL(vfam(c, F.g, F_DOWN), n * (ib + kb + cb) + ncn * cb, 60 * n, down_full_launch(F, C, sr, si, om, rin, st, active));
  } else if (rr_full(F)) {
    KL(vfam(c, F.g, F_SMOOTH0), n * (ib + (db ? db : kb) + cb), 6 * n, (launch_smooth0<R, TI>(F.g, sr, si, om, F.k2, F.dinv, rin, F.U1, st, active)));
    KL(vfam(c, F.g, F_RR), n * (cb + ib + kd) + ncn * cb, 24 * n + 54 * ncn, rr_launch(F, C, sr, si, rin, st, active));
  } else {
    if (down_fused(F)) {
      KL(vfam(c, F.g, F_SMOOTH0), n * (ib + kb + 2 * cb), 30 * n, down_fused_launch(F, sr, si, om, rin, st, active));
    } else {
      KL(vfam(c, F.g, F_SMOOTH0), n * (ib + (db ? db : kb) + cb), 6 * n, (launch_smooth0<R, TI>(F.g, sr, si, om, F.k2, F.dinv, rin, F.U1, st, active)));
      KL(vfam(c, F.g, F_RESID), n * (cb + ib + kd + cb), 24 * n, (launch_resid<R, R, TI, R>(F.g, sr, si, F.k2, F.U1, rin, F.T, st, active, F.dinv)));
    }
    KL(vfam(c, F.g, F_RESTRICT), n * cb + ncn * cb, 54 * ncn, (launch_restrict<R>(F.g, C.g, F.T, C.B, st, active)));
  }
  fcycle_levels<R, R, R>(c, lv, L, l + 1, C.B, C.E, st, active);
  vcycle_from<R>(c, lv, L, l + 1, st, active);
  if (up_full(F)) {
    KL(vfam(c, F.g, F_UP), n * (cb + ib + (db ? kd + db : kb) + ob) + ncn * cb, 40 * n, up_full_launch(F, C, sr, si, om, rin, zout, st, active));
    return;
  }
  KL(vfam(c, F.g, F_PROLONG), n * 2 * cb + ncn * cb, 6 * n, (launch_prolong_add<R>(F.g, C.g, F.U1, C.E, F.T, st, active)));
  KL(vfam(c, F.g, F_JACOBI), n * (cb + ib + kd + db + ob), 32 * n, (launch_jacobi<R, TI, TO>(F.g, sr, si, om, F.k2, F.dinv, F.T, rin, zout, st, active)));
}

template <typename R, typename TI, typename TO>
void run_fcycle(helm_ctx* c, const cx<TI>* rin, cx<TO>* zout, cudaStream_t st, const int* active) {
  using B = LevelBufs<R>;
  VLevel<R> lv[MAX_LEVELS];
  for (int l = 0; l < c->nlev; ++l) {
    Level& L = c->L[l];
    lv[l] = VLevel<R>{L.g, B::k2(L), B::dinv(L), B::B(L), B::U1(L), B::T(L), B::E(L)};
  }
  fcycle_levels<R, TI, TO>(c, lv, c->nlev, 0, rin, zout, st, active);
}

// The configured cycle over given level arrays (the batched solver's nb-wide grids).
template <typename R, typename TI, typename TO>
void run_cycle_levels(helm_ctx* c, const VLevel<R>* lv, const cx<TI>* rin, cx<TO>* zout, cudaStream_t st,
                      const int* active) {
  if (c->p.cycle == HELM_CYCLE_F) fcycle_levels<R, TI, TO>(c, lv, c->nlev, 0, rin, zout, st, active);
  else run_vcycle_levels<R, TI, TO>(c, lv, c->nlev, rin, zout, st, active);
}

// The configured multigrid cycle (V or F) as the preconditioner.
template <typename R, typename TI, typename TO>
void run_cycle(helm_ctx* c, const cx<TI>* rin, cx<TO>* zout, cudaStream_t st, const int* active) {
  if (c->p.cycle == HELM_CYCLE_F) run_fcycle<R, TI, TO>(c, rin, zout, st, active);
  else run_vcycle<R, TI, TO>(c, rin, zout, st, active);
}

void norm_into(helm_ctx* c, const z128* x, double* out, cudaStream_t st, const int* active) {
  const double n = (double)c->n0;
  int nb = 0;
  KL(F_NORM, 16 * n, 4 * n, nb = launch_norm2_part(x, c->n0, c->partr, st, active));
  KL(F_REDUCE_NORM, 8.0 * nb, nb, launch_reduce_norm(c->partr, nb, out, st, active));
}

void clear_graphs(helm_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

// Enqueue one solver step on `st`: replayed from a CUDA graph captured on first use when the
// context runs with graphs and without per-kernel profiling, else launched kernel by kernel.
// `enqueue(stream)` must only launch work on `stream` (no host waits, no allocation), and
// everything it launches must depend only on (tag, j, p) and on the context's own buffers.
template <typename Fn>
helm_status graph_step(helm_ctx* c, int tag, int j, const void* p, cudaStream_t st, Fn&& enqueue) {
  if (!c->p.graphs || c->prof.on) {
    enqueue(st);
    return HELM_OK;
  }
  for (auto& g : c->graphs)
    if (g.tag == tag && g.j == j && g.p == p) {
      CU(cudaGraphLaunch(g.exec, st));
      c->prof.launches += g.launches;
      return HELM_OK;
    }
  if (c->graphs.size() >= 512) clear_graphs(c);
  if (!c->gstream) CU(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
  const long long l0 = c->prof.launches;
  CU(cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeRelaxed));
  enqueue(c->gstream);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->gstream, &g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, HELM_ECUDA, "stream capture of a solver step: %s", cudaGetErrorString(e));
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return fail(c, HELM_ECUDA, "graph instantiation: %s", cudaGetErrorString(ei));
  const long long nl = c->prof.launches - l0;
  c->graphs.push_back({tag, j, p, ex, nl});
  CU(cudaGraphLaunch(ex, st));
  return HELM_OK;
}

// ---- launch-shape autotuner -------------------------------------------------------------
// For every level and kernel family, time each (rows per CTA, CTA count) candidate on the
// level's own work vectors and keep the fastest.  Stencil, transfer and smoothing results do
// not depend on the launch shape (no reductions), so tuning changes speed only.
template <typename Fn>
helm_status tune_slot(helm_ctx* c, Grid& g, int slot, int level, cudaStream_t st, Fn&& run) {
  static const int tys[] = {1, 2, 4, 8};
  static const int per_sm[] = {4, 8, 16, 32};
  constexpr int kBurst = 3;  // back-to-back launches per timing, as in a solve
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  float best = 1e30f;
  int bty = 0, bct = 0;
  for (int ty : tys)
    for (int m : per_sm) {
      g.tile_ty[slot] = ty;
      g.tile_ctas[slot] = 152 * m;
      run(g);  // warm-up
      float ms = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        CU(cudaEventRecord(e0, st));
        for (int b = 0; b < kBurst; ++b) run(g);
        CU(cudaEventRecord(e1, st));
        CU(cudaEventSynchronize(e1));
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, e0, e1));
        ms = std::min(ms, t / kBurst);
      }
      c->tune_log.push_back(TuneRec{level, slot, ty, 152 * m, ms});
      if (ms < best) { best = ms; bty = ty; bct = 152 * m; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g.tile_ty[slot] = bty;
  g.tile_ctas[slot] = bct;
  return check_launch(c, "autotune");
}

// Best of three timings of three back-to-back launches of run(), per launch, in ms.
template <typename Fn>
float time_burst(helm_ctx* c, cudaStream_t st, Fn&& run) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return 1e30f;
  run();
  float ms = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    for (int b = 0; b < 3; ++b) run();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms = std::min(ms, t / 3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  (void)c;
  return ms;
}

// Tune the V-cycle kernels of arithmetic R on the levels lv[0..L) (grids are updated in place).
template <typename R>
helm_status tune_vlevels(helm_ctx* c, VLevel<R>* lv, int L, cudaStream_t st) {
  const double sr = c->s_re, si = c->s_im, om = c->p.omega;
  for (int l = 0; l < L; ++l) {
    VLevel<R>& F = lv[l];
    const size_t ne = F.g.npts() * F.g.nb;
    // finite nonzero bytes (0x3f.. is about 0.75 in FP32 and 4.8e-4 in FP64)
    CU(cudaMemsetAsync(F.U1, 0x3f, ne * sizeof(cx<R>), st));
    CU(cudaMemsetAsync(F.T, 0x3f, ne * sizeof(cx<R>), st));
    if (l == L - 1) break;  // the coarsest level runs the dense solve only
    TRY(tune_slot(c, F.g, tile_slot<R>(TILE_STENCIL), l, st, [&](const Grid& g) {
      launch_jacobi<R, R, R>(g, sr, si, om, F.k2, F.dinv, F.U1, F.U1, F.T, st, nullptr);
    }));
    if (std::is_same<R, float>::value && F.g.nb == 1) {
      // the shared-memory tiled FP32 kernels against the best plain shape (logged as slot 12)
      const int slot = tile_slot<R>(TILE_STENCIL);
      auto run = [&] { launch_jacobi<R, R, R>(F.g, sr, si, om, F.k2, F.dinv, F.U1, F.U1, F.T, st, nullptr); };
      const int ct0 = F.g.tile_ctas[slot];
      float best = time_burst(c, st, run);
      int best_ct = -1;
      F.g.tiled = 1;
      for (int m : {4, 8, 16, 32}) {
        F.g.tile_ctas[slot] = 152 * m;
        const float t = time_burst(c, st, run);
        c->tune_log.push_back(TuneRec{l, 12, TYT_TILED, 152 * m, t});
        if (t < best) { best = t; best_ct = 152 * m; }
      }
      F.g.tiled = best_ct > 0 ? 1 : 0;
      F.g.tile_ctas[slot] = best_ct > 0 ? best_ct : ct0;
      TRY(check_launch(c, "autotune (tiled stencil)"));
    }
    TRY(tune_slot(c, F.g, tile_slot<R>(TILE_SMOOTH0), l, st, [&](const Grid& g) {
      launch_smooth0<R, R>(g, sr, si, om, F.k2, F.dinv, F.U1, F.T, st, nullptr);
    }));
    if constexpr (std::is_same<R, float>::value) {
      if (F.g.nb == 1) {
        // pre-smoothing + residual in one kernel against the two tuned kernels (logged as slot 13
        // for the fused shapes); the pre-smoothing slot keeps whichever shape is used
        const int slot = tile_slot<R>(TILE_SMOOTH0);
        // scratch for the fused kernel's u1 output: the context's complex128 work vector holds
        // at least one complex64 grid vector of any level
        z64* scratch = reinterpret_cast<z64*>(c->zs);
        const float t_plain =
            time_burst(c, st, [&] { launch_smooth0<R, R>(F.g, sr, si, om, F.k2, F.dinv, F.U1, F.T, st, nullptr); }) +
            time_burst(c, st, [&] { launch_resid<R, R, R, R>(F.g, sr, si, F.k2, F.U1, F.U1, F.T, st, nullptr, F.dinv); });
        const int ty0 = F.g.tile_ty[slot], ct0 = F.g.tile_ctas[slot];
        float best = 1e30f;
        int bty = 0, bct = 0;
        for (int ty : {1, 2, 4, 8})
          for (int m : {4, 8, 16, 32}) {
            F.g.tile_ty[slot] = ty;
            F.g.tile_ctas[slot] = 152 * m;
            const float t = time_burst(c, st, [&] {
              launch_smooth0_resid32<float>(F.g, sr, si, om, F.k2, F.U1, scratch, F.T, st, nullptr);
            });
            c->tune_log.push_back(TuneRec{l, 13, ty, 152 * m, t});
            if (t < best) { best = t; bty = ty; bct = 152 * m; }
          }
        const bool use = best < t_plain;
        F.g.fused_down = use ? 1 : 0;
        F.g.tile_ty[slot] = use ? bty : ty0;
        F.g.tile_ctas[slot] = use ? bct : ct0;
        TRY(check_launch(c, "autotune (fused pre-smoothing and residual)"));
      }
    }
    VLevel<R>& C = lv[l + 1];
    CU(cudaMemsetAsync(C.E, 0x3f, C.g.npts() * C.g.nb * sizeof(cx<R>), st));
    TRY(tune_slot(c, F.g, tile_slot<R>(TILE_PROLONG), l, st, [&](const Grid& g) {
      launch_prolong_add<R>(g, C.g, F.U1, C.E, F.T, st, nullptr);
    }));
    TRY(tune_slot(c, C.g, tile_slot<R>(TILE_RESTRICT), l + 1, st, [&](const Grid& g) {
      launch_restrict<R>(F.g, g, F.T, C.B, st, nullptr);
    }));
    if (F.g.nb != 1) continue;
    // scratch for the forms' outputs: the context's complex128 work vector holds a grid vector
    // of any level in either precision
    cx<R>* scratch = reinterpret_cast<cx<R>*>(c->zs);
    // the residual and its restriction as one kernel against the chosen pair (logged as slot 16,
    // coarse planes per CTA in the shape column); with it the pre-smoothing runs on its own
    {
      const float t_pair =
          (F.g.fused_down
               ? time_burst(c, st, [&] {
                   if constexpr (std::is_same<R, float>::value)
                     launch_smooth0_resid32<float>(F.g, sr, si, om, F.k2, F.U1, reinterpret_cast<z64*>(c->zs), F.T, st,
                                                   nullptr);
                 })
               : time_burst(c, st, [&] { launch_smooth0<R, R>(F.g, sr, si, om, F.k2, F.dinv, F.U1, F.T, st, nullptr); }) +
                     time_burst(c, st, [&] { launch_resid<R, R, R, R>(F.g, sr, si, F.k2, F.U1, F.U1, F.T, st, nullptr, F.dinv); })) +
          time_burst(c, st, [&] { launch_restrict<R>(F.g, C.g, F.T, C.B, st, nullptr); });
      const float t_s0 =
          time_burst(c, st, [&] { launch_smooth0<R, R>(F.g, sr, si, om, F.k2, F.dinv, F.U1, F.T, st, nullptr); });
      float best = 1e30f;
      int bkc = 0;
      for (int kc : {1, 2, 4, 8, 16}) {
        if (kc > 1 && (kc / 2) >= C.g.N3) break;
        const float t = time_burst(c, st, [&] {
          launch_rr<R, R>(F.g, C.g, sr, si, F.k2, F.dinv, F.U1, F.U1, C.B, kc, st, nullptr);
        });
        c->tune_log.push_back(TuneRec{l, 16, kc, 0, t});
        if (t < best) { best = t; bkc = kc; }
      }
      F.g.rr_full = t_s0 + best < t_pair ? 1 : 0;
      F.g.rr_kc = bkc;
      if (F.g.rr_full) F.g.fused_down = 0;
      TRY(check_launch(c, "autotune (residual with restriction)"));
    }
    if constexpr (std::is_same<R, float>::value) {
      // the whole down-sweep in one kernel against the chosen kernels (logged as slot 14,
      // coarse planes per CTA in the shape column)
      const float t_cur =
          (F.g.fused_down
               ? time_burst(c, st, [&] {
                   launch_smooth0_resid32<float>(F.g, sr, si, om, F.k2, F.U1, reinterpret_cast<z64*>(c->zs), F.T, st,
                                                 nullptr);
                 })
               : time_burst(c, st, [&] { launch_smooth0<R, R>(F.g, sr, si, om, F.k2, F.dinv, F.U1, F.T, st, nullptr); })) +
          (F.g.rr_full
               ? time_burst(c, st, [&] {
                   launch_rr<R, R>(F.g, C.g, sr, si, F.k2, F.dinv, F.U1, F.U1, C.B, F.g.rr_kc, st, nullptr);
                 })
               : (F.g.fused_down ? 0.f
                                 : time_burst(c, st, [&] {
                                     launch_resid<R, R, R, R>(F.g, sr, si, F.k2, F.U1, F.U1, F.T, st, nullptr);
                                   })) +
                     time_burst(c, st, [&] { launch_restrict<R>(F.g, C.g, F.T, C.B, st, nullptr); }));
      float best = 1e30f;
      int bkc = 0;
      for (int kc : {1, 2, 4, 8, 16}) {
        if (kc > 1 && (kc / 2) >= C.g.N3) break;
        const float t = time_burst(c, st, [&] {
          launch_down32<float>(F.g, C.g, sr, si, om, F.k2, F.T, reinterpret_cast<z64*>(c->zs), C.B, kc, st, nullptr);
        });
        c->tune_log.push_back(TuneRec{l, 14, kc, 0, t});
        if (t < best) { best = t; bkc = kc; }
      }
      F.g.down_full = best < t_cur ? 1 : 0;
      F.g.down_kc = bkc;
      TRY(check_launch(c, "autotune (fused down-sweep)"));
    }
    // the whole up-sweep in one kernel against prolongation + post-smoothing (logged as slot 15,
    // fine planes per CTA in the shape column)
    const float t_up =
        time_burst(c, st, [&] { launch_prolong_add<R>(F.g, C.g, F.U1, C.E, F.T, st, nullptr); }) +
        time_burst(c, st, [&] { launch_jacobi<R, R, R>(F.g, sr, si, om, F.k2, F.dinv, F.T, F.U1, scratch, st, nullptr); });
    float bu = 1e30f;
    int bkz = 0;
    for (int kz : {4, 8, 16, 32, 64}) {
      if (kz > 4 && kz / 2 >= F.g.N3) break;
      const float t = time_burst(c, st, [&] {
        launch_up<R, R, R>(F.g, C.g, sr, si, om, F.k2, F.dinv, F.U1, C.E, F.U1, scratch, kz, st, nullptr);
      });
      c->tune_log.push_back(TuneRec{l, 15, kz, 0, t});
      if (t < bu) { bu = t; bkz = kz; }
    }
    F.g.up_full = bu < t_up ? 1 : 0;
    F.g.up_kz = bkz;
    TRY(check_launch(c, "autotune (fused up-sweep)"));
  }
  return HELM_OK;
}

// Tune the single-right-hand-side kernels: the V-cycle in the context's arithmetic on every
// level, and the FP64 operator of the outer Krylov method on the finest level.
helm_status autotune(helm_ctx* c, cudaStream_t st) {
  const bool mixed = c->p.precision == HELM_PREC_MIXED;
  const int L = c->nlev;
  if (mixed) {
    VLevel<float> lv[MAX_LEVELS];
    for (int l = 0; l < L; ++l) {
      Level& Lv = c->L[l];
      lv[l] = VLevel<float>{Lv.g, Lv.k2f, nullptr, Lv.B32, Lv.U132, Lv.T32, Lv.E32};
    }
    TRY(tune_vlevels<float>(c, lv, L, st));
    for (int l = 0; l < L; ++l) c->L[l].g = lv[l].g;
  }
  VLevel<double> lv[MAX_LEVELS];
  for (int l = 0; l < L; ++l) {
    Level& Lv = c->L[l];
    lv[l] = VLevel<double>{Lv.g, Lv.k2, Lv.dinv, Lv.B64, Lv.U164, Lv.T64, Lv.E64};
  }
  if (!mixed) {
    TRY(tune_vlevels<double>(c, lv, L, st));
  } else {
    // the finest FP64 operator only (A-products and residuals of the outer method)
    Level& F = c->L[0];
    const size_t n = F.g.npts();
    CU(cudaMemsetAsync(F.U164, 0x3f, n * sizeof(z128), st));
    TRY(tune_slot(c, lv[0].g, tile_slot<double>(TILE_STENCIL), 0, st, [&](const Grid& g) {
      launch_resid<double, double, double, double>(g, 1.0, 0.0, F.k2, F.U164, F.U164, F.T64, st, nullptr);
    }));
  }
  for (int l = 0; l < L; ++l)
    for (int q = 0; q < 4; ++q) {
      c->L[l].g.tile_ty[q] = lv[l].g.tile_ty[q];
      c->L[l].g.tile_ctas[q] = lv[l].g.tile_ctas[q];
    }
  // FP64 inner products: w staged in shared memory or read by each warp (logged as level -1,
  // slot 16 + variant)
  if (c->p.orth == HELM_ORTH_FP64 && c->m >= 2) {
    const size_t n = c->n0;
    const int nv = std::min(16, c->m);
    CU(cudaMemsetAsync(c->V, 0x3f, (size_t)(nv + 1) * n * sizeof(z128), st));
    if (c->Vs) CU(cudaMemsetAsync(c->Vs, 0x3f, (size_t)nv * n * sizeof(double), st));
    float best = 1e30f;
    for (int v = 0; v < 2; ++v) {
      const float t = time_burst(c, st, [&] {
        if (c->Vs) launch_mdot_sums(c->V, c->Vs, n, nv, c->V + (size_t)nv * n, n, c->part, 1, st, nullptr, v);
        else launch_mdot(c->V, n, nv, c->V + (size_t)nv * n, n, c->part, 1, st, nullptr, v);
      });
      c->tune_log.push_back(TuneRec{-1, 16 + v, nv, 0, t});
      if (t < best) { best = t; c->mdot_variant = v; }
    }
    TRY(check_launch(c, "autotune (FP64 inner products)"));
  }
  // double-float inner products: slots per warp pass (logged as level -1, slot 8 + variant)
  if (c->p.orth == HELM_ORTH_DF && c->m >= 2) {
    const size_t n = c->n0;
    const int nv = std::min(16, c->m);
    zdf* Vdf = reinterpret_cast<zdf*>(c->V);
    CU(cudaMemsetAsync(c->V, 0x3f, (size_t)(nv + 1) * n * sizeof(z128), st));
    CU(cudaMemsetAsync(c->wdf, 0x3f, n * sizeof(zdf), st));
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int v = 0; v < 3; ++v) {
      launch_mdot_df(Vdf, n, nv, c->wdf, n, c->part, 1, st, nullptr, v);
      float ms = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        CU(cudaEventRecord(e0, st));
        launch_mdot_df(Vdf, n, nv, c->wdf, n, c->part, 1, st, nullptr, v);
        CU(cudaEventRecord(e1, st));
        CU(cudaEventSynchronize(e1));
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, e0, e1));
        ms = std::min(ms, t);
      }
      c->tune_log.push_back(TuneRec{-1, 8 + v, nv, 0, ms});
      if (ms < best) { best = ms; c->mdot_df_variant = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TRY(check_launch(c, "autotune (inner products)"));
  }
  CU(cudaStreamSynchronize(st));
  return HELM_OK;
}

enum { G_ARNOLDI = 1, G_BICG = 2, G_IDR = 3, G_IDR_DR = 4, G_BATCH = 100 };

// GMRES(m) / FGMRES(m) on device-resident b and x.
helm_status gmres_device(helm_ctx* c, const z128* b, z128* x, helm_solve_info* info, cudaStream_t st) {
  const Level& F = c->L[0];
  const size_t n = c->n0;
  const int m = c->m;
  const bool mixed = c->p.precision == HELM_PREC_MIXED;
  const bool flexible = mixed || c->p.krylov == HELM_FGMRES;
  const double tol = c->p.tol;
  KrylovCtl* ctl = c->ctl;
  const int* act = &ctl->active;
  const bool df = c->p.orth == HELM_ORTH_DF;
  const bool sums = !df && c->Vs;  // FP64 Gram-Schmidt against the summed basis
  zdf* Vdf = reinterpret_cast<zdf*>(c->V);
  // the paper's left preconditioning (Sec. 3.2): GMRES on M^{-1} A x = M^{-1} b, stopping on
  // ||M^{-1}(b - A x)|| / ||M^{-1} b|| (Sec. 5); FP64 GMRES only (checked at creation)
  const bool left = c->p.side == HELM_SIDE_LEFT;
  auto residual = [&](void) {  // c->r = b - A x, or M^{-1}(b - A x) from the left
    z128* dst = left ? c->zs : c->r;
    KL(F_RESID, 56.0 * n, 24.0 * n, (launch_resid<double, double, double, double>(F.g, 1.0, 0.0, F.k2, x, b, dst, st, c->one)));
    if (left) run_cycle<double, double, double>(c, c->zs, c->r, st, c->one);
  };

  if (left) {
    run_cycle<double, double, double>(c, b, c->zs, st, c->one);
    norm_into(c, c->zs, &ctl->bnorm, st, c->one);
  } else {
    norm_into(c, b, &ctl->bnorm, st, c->one);
  }
  residual();
  norm_into(c, c->r, &ctl->beta, st, c->one);
  CU(cudaMemcpyAsync(c->hctl, ctl, sizeof(KrylovCtl), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  prof_flush(c, -1);
  double bnorm = c->hctl->bnorm;
  int iters = 0, restarts = 0;
  helm_status status = HELM_OK;
  if (bnorm == 0.0) {
    // b = 0: the solution is x = 0
    CU(cudaMemsetAsync(x, 0, n * sizeof(z128), st));
    CU(cudaStreamSynchronize(st));
    if (info) { info->iterations = 0; info->restarts = 0; info->rel_residual = 0.0; }
    return HELM_OK;
  }
  double relres = c->hctl->beta / bnorm;
  for (;;) {
    if (!(relres == relres) || relres == HUGE_VAL) { status = HELM_ENUMERIC; break; }
    if (relres <= tol) { status = HELM_OK; break; }
    if (iters >= c->p.max_iter) { status = HELM_ENOCONV; break; }
    const int jmax = std::min(m, c->p.max_iter - iters);
    KL(F_MISC, 0, 0, launch_cycle_init(ctl, c->gv, m, iters, st));
    if (df) {
      if (mixed) KL(F_SCALE, 40.0 * n, 2.0 * n, (launch_scale_df<z128, float>(c->r, &ctl->beta, Vdf, c->vcur32, n, st, act)));
      else KL(F_SCALE, 48.0 * n, 2.0 * n, (launch_scale_df<z128, double>(c->r, &ctl->beta, Vdf, c->vcur64, n, st, act)));
    } else if (sums) {
      KL(F_SCALE, 40.0 * n, 3.0 * n, launch_scale_inv_sums(c->r, &ctl->beta, c->V, c->Vs, n, st, act));
    } else {
      KL(F_SCALE, 32.0 * n, 2.0 * n, launch_scale_inv(c->r, &ctl->beta, c->V, n, st, act));
    }
    for (int j = 0; j < jmax; ++j) {
      c->cur_j = j;
      auto step = [&](cudaStream_t st) {
        z128* vj = c->V + (size_t)j * n;
        z128* w = c->V + (size_t)(j + 1) * n;  // FP64 Gram-Schmidt works in place in V
        zdf* wd = c->wdf;                      // double-float Gram-Schmidt works in wdf
        const double nd = (double)n, nv = j + 1;
        if (mixed) {
          z64* zj = c->Z32 + (size_t)j * n;
          if (df) {
            run_cycle<float, float, float>(c, c->vcur32, zj, st, act);
            KL(F_APPLY, 32.0 * nd, 22.0 * nd, (launch_apply_c64_df<zdf>(F.g, c->k2df, c->skdf, zj, wd, st, act)));
          } else {
            run_cycle<float, double, float>(c, vj, zj, st, act);
            KL(F_APPLY, 32.0 * nd, 22.0 * nd, (launch_apply<double, float, double>(F.g, 1.0, 0.0, F.k2, zj, w, st, act)));
          }
        } else if (left) {
          KL(F_APPLY, 40.0 * nd, 22.0 * nd, (launch_apply<double, double, double>(F.g, 1.0, 0.0, F.k2, vj, c->zs, st, act)));
          run_cycle<double, double, double>(c, c->zs, w, st, act);
        } else {
          z128* zj = flexible ? c->Z64 + (size_t)j * n : c->zs;
          run_cycle<double, double, double>(c, df ? c->vcur64 : vj, zj, st, act);
          if (df)
            KL(F_APPLY, 40.0 * nd, 22.0 * nd, (launch_apply_split<double>(F.g, 1.0, 0.0, F.k2, zj, wd, st, act)));
          else
            KL(F_APPLY, 40.0 * nd, 22.0 * nd, (launch_apply<double, double, double>(F.g, 1.0, 0.0, F.k2, zj, w, st, act)));
        }
        // classical Gram-Schmidt: first pass always; the second on every step (ALWAYS) or when
        // the first pass's projection kept less than reorth_keep of |w|^2 (SELECTIVE)
        const bool sel = c->p.reorth == HELM_REORTH_SELECTIVE;
        for (int pass = 0; pass < 2; ++pass) {
          const int* a2 = (pass == 1 && sel) ? &ctl->pass2 : act;
          c->cur_cond = (pass == 1 && sel) ? 1 : 0;
          const int wn = (pass == 0 && sel) ? 1 : 0;
          int nb = 0;
          if (df)
            KL(F_MDOT, 16.0 * (nv + 1) * nd, 8.0 * nv * nd,
               nb = launch_mdot_df(Vdf, n, j + 1, wd, n, c->part, wn, st, a2, c->mdot_df_variant));
          else if (sums)
            // algorithmic flops: 8 per basis vector and unknown (a complex multiply-add), of
            // which the summed form executes 6; bytes: what its layout must move
            KL(F_MDOT, (24.0 * nv + 16.0) * nd, 8.0 * nv * nd,
               nb = launch_mdot_sums(c->V, c->Vs, n, j + 1, w, n, c->part, wn, st, a2, c->mdot_variant));
          else
            KL(F_MDOT, 16.0 * (nv + 1) * nd, 8.0 * nv * nd,
               nb = launch_mdot(c->V, n, j + 1, w, n, c->part, wn, st, a2, c->mdot_variant));
          KL(F_REDUCE_DOTS, 16.0 * nv * nb, 2.0 * nv * nb,
             launch_reduce_dots(c->part, j + 1, nb, c->hpass, c->hacc, pass, wn ? j : -1, &ctl->pass2, c->reorth_log,
                                st, a2, c->p.reorth_keep));
          if (df)
            KL(F_GS_UPDATE, 16.0 * (nv + 2) * nd, 8.0 * nv * nd, launch_gs_update_df(Vdf, n, j + 1, c->hpass, wd, n, st, a2));
          else if (sums)
            KL(F_GS_UPDATE, (24.0 * nv + 32.0) * nd, 8.0 * nv * nd,
               launch_gs_update_sums(c->V, c->Vs, n, j + 1, c->hpass, w, n, st, a2));
          else
            KL(F_GS_UPDATE, 16.0 * (nv + 2) * nd, 8.0 * nv * nd, launch_gs_update(c->V, n, j + 1, c->hpass, w, n, st, a2));
        }
        c->cur_cond = 0;
        if (df) {
          int nb = 0;
          KL(F_NORM, 16.0 * nd, 4.0 * nd, nb = launch_norm2_part_df(wd, n, c->partr, st, act));
          KL(F_REDUCE_NORM, 8.0 * nb, nb, launch_reduce_norm(c->partr, nb, c->hnorm, st, act));
        } else {
          norm_into(c, w, c->hnorm, st, act);
        }
        KL(F_GIVENS, 0, 0, launch_givens(ctl, c->H, m, j, jmax, c->hacc, c->hnorm, c->cs, c->sn, c->gv, tol, c->hist, c->hist_len, st));
        if (df) {
          zdf* vn = Vdf + (size_t)(j + 1) * n;
          if (mixed) KL(F_SCALE, 40.0 * nd, 2.0 * nd, (launch_scale_df<zdf, float>(wd, c->hnorm, vn, c->vcur32, n, st, act)));
          else KL(F_SCALE, 48.0 * nd, 2.0 * nd, (launch_scale_df<zdf, double>(wd, c->hnorm, vn, c->vcur64, n, st, act)));
        } else if (sums) {
          KL(F_SCALE, 40.0 * nd, 3.0 * nd, launch_scale_inv_sums(w, c->hnorm, w, c->Vs + (size_t)(j + 1) * n, n, st, act));
        } else {
          KL(F_SCALE, 32.0 * nd, 2.0 * nd, launch_scale_inv(w, c->hnorm, w, n, st, act));
        }
};
      // a graph per Arnoldi column, for full-length cycles (the Givens step knows jmax)
      if (jmax == m) TRY(graph_step(c, G_ARNOLDI, j, nullptr, st, step));
      else step(st);
      TRY(check_launch(c, "Arnoldi step"));
      CU(cudaMemcpyAsync(c->hflags + j, act, sizeof(int), cudaMemcpyDeviceToHost, st));
      CU(cudaEventRecord(c->ev[j % c->nev], st));
      if (j >= FLAG_LAG) {
        CU(cudaEventSynchronize(c->ev[(j - FLAG_LAG) % c->nev]));
        if (c->hflags[j - FLAG_LAG] == 0) break;
      }
    }
    c->cur_j = -1;
    CU(cudaMemcpyAsync(c->hctl, ctl, sizeof(KrylovCtl), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(c->hreorth_log, c->reorth_log, sizeof(int) * m, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    const int jend = c->hctl->jend;
    if (c->p.reorth == HELM_REORTH_SELECTIVE)
      for (int q = 0; q <= jend; ++q) c->reorth_steps += c->hreorth_log[q];
    else
      c->reorth_steps += jend + 1;
    c->arnoldi_steps += jend + 1;
    prof_flush(c, jend);
    iters += jend + 1;
    ++restarts;
    if (jend >= 0) {
      const double nd = (double)n, k = jend + 1;
      KL(F_SOLUPDATE, 0, 0, launch_trisolve(ctl, c->H, m, c->gv, c->y, st));
      if (mixed) {
        if (df)
          KL(F_SOLUPDATE, (8.0 * k + 32.0) * nd, 8.0 * k * nd, launch_xupdate_df(ctl, c->Z32, n, c->y, x, n, st));
        else
          KL(F_SOLUPDATE, (8.0 * k + 32.0) * nd, 8.0 * k * nd, launch_xupdate<float>(ctl, c->Z32, n, c->y, x, n, st));
      } else if (flexible) {
        KL(F_SOLUPDATE, (16.0 * k + 32.0) * nd, 8.0 * k * nd, launch_xupdate<double>(ctl, c->Z64, n, c->y, x, n, st));
      } else {
        if (df)
          KL(F_SOLUPDATE, (16.0 * k + 16.0) * nd, 8.0 * k * nd, launch_combine_df(ctl, Vdf, n, c->y, c->r, n, st));
        else
          KL(F_SOLUPDATE, (16.0 * k + 16.0) * nd, 8.0 * k * nd, launch_combine(ctl, c->V, n, c->y, c->r, n, st));
        if (left) {
          KL(F_SOLUPDATE, 48.0 * nd, 2.0 * nd, launch_axpy1(c->r, x, n, st));  // x += V y
        } else {
          run_cycle<double, double, double>(c, c->r, c->zs, st, c->one);
          KL(F_SOLUPDATE, 48.0 * nd, 2.0 * nd, launch_axpy1(c->zs, x, n, st));
        }
      }
    }
    residual();
    norm_into(c, c->r, &ctl->beta, st, c->one);
    TRY(check_launch(c, "solution update"));
    CU(cudaMemcpyAsync(c->hctl, ctl, sizeof(KrylovCtl), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    prof_flush(c, -1);
    relres = c->hctl->beta / bnorm;
    if (c->hctl->flag == 2 && !(relres <= tol)) { status = HELM_ENUMERIC; break; }
    if (jend < 0) { status = HELM_ENUMERIC; break; }
  }
  if (info) {
    info->iterations = iters;
    info->restarts = restarts;
    info->rel_residual = relres;
  }
  return status;
}

helm_status fcycle_entry(helm_ctx* c, helm_dtype dt, const void* r, void* z, cudaStream_t st) {
  if (dt == HELM_C128) run_fcycle<double, double, double>(c, (const z128*)r, (z128*)z, st, nullptr);
  else if (dt == HELM_C64) run_fcycle<float, float, float>(c, (const z64*)r, (z64*)z, st, nullptr);
  else return fail(c, HELM_EINVAL, "unknown dtype %d", (int)dt);
  return check_launch(c, "cslp_fcycle");
}

template <typename R>
void stage_impl(helm_ctx* c, int l, int stage, const cx<R>* b, const cx<R>* e, cx<R>* out, cudaStream_t st) {
  using B = LevelBufs<R>;
  const double sr = c->s_re, si = c->s_im, om = c->p.omega;
  Level& F = c->L[l];
  if (stage == 2) {
    coarse_solve<R, R>(c, b, out, st, nullptr, 1);
    return;
  }
  Level& C = c->L[l + 1];
  // the kernel forms the context's V-cycle uses on this level (their results are identical)
  launch_smooth0<R, R>(F.g, sr, si, om, B::k2(F), B::dinv(F), b, B::U1(F), st, nullptr);
  if (stage == 0) {
    if (F.g.rr_full) {
      launch_rr<R, R>(F.g, C.g, sr, si, B::k2(F), B::dinv(F), B::U1(F), b, out, F.g.rr_kc, st, nullptr);
    } else {
      launch_resid<R, R, R, R>(F.g, sr, si, B::k2(F), B::U1(F), b, B::T(F), st, nullptr, B::dinv(F));
      launch_restrict<R>(F.g, C.g, B::T(F), out, st, nullptr);
    }
  } else if (F.g.up_full) {
    launch_up<R, R, R>(F.g, C.g, sr, si, om, B::k2(F), B::dinv(F), B::U1(F), e, b, out, F.g.up_kz, st, nullptr);
  } else {
    launch_prolong_add<R>(F.g, C.g, B::U1(F), e, B::T(F), st, nullptr);
    launch_jacobi<R, R, R>(F.g, sr, si, om, B::k2(F), B::dinv(F), B::T(F), b, out, st, nullptr);
  }
}

}  // namespace

namespace {

helm_status batch_alloc(helm_ctx* c, int nb) {
  BatchWS& W = c->bw;
  if (W.nb >= nb) return HELM_OK;
  clear_graphs(c);  // captured batched steps hold the old workspace addresses
  const size_t n = c->n0, ne = n * nb;
  const int m = c->m;
  const bool mixed = c->p.precision == HELM_PREC_MIXED;
  TRY(dalloc(c, &W.V, (size_t)(m + 1) * ne));
  if (c->p.orth == HELM_ORTH_FP64 && c->p.gs_sums) TRY(dalloc(c, &W.Vs, (size_t)(m + 1) * ne));
  if (mixed) TRY(dalloc(c, &W.Z32, (size_t)m * ne));
  else TRY(dalloc(c, &W.Z64, (size_t)m * ne));
  TRY(dalloc(c, &W.r, ne));
  if (c->p.orth == HELM_ORTH_DF) {
    TRY(dalloc(c, &W.wdf, ne));
    if (mixed) TRY(dalloc(c, &W.vcur32, ne));
    else TRY(dalloc(c, &W.vcur64, ne));
  }
  TRY(dalloc(c, &W.Bt, ne));
  TRY(dalloc(c, &W.Xt, ne));
  TRY(dalloc(c, &W.part, (size_t)(m + 2) * nb * RED_STRIDE));
  TRY(dalloc(c, &W.partr, (size_t)nb * RED_STRIDE));
  TRY(dalloc(c, &W.hpass, (size_t)(m + 1) * nb));
  TRY(dalloc(c, &W.hacc, (size_t)(m + 1) * nb));
  TRY(dalloc(c, &W.hnorm, nb));
  TRY(dalloc(c, &W.sw2, nb));
  TRY(dalloc(c, &W.log, m));
  TRY(dalloc(c, &W.need, nb));
  CU(cudaMemset(W.need, 0, sizeof(int) * nb));
  BatchCtl& h = W.h;
  h.any = 0; h.pass2 = 0; h.max_iter = c->p.max_iter; h.pad = 0;
  TRY(dalloc(c, &h.act, nb)); TRY(dalloc(c, &h.jend, nb)); TRY(dalloc(c, &h.flag, nb));
  TRY(dalloc(c, &h.jmax, nb)); TRY(dalloc(c, &h.iters, nb));
  TRY(dalloc(c, &h.bnorm, nb)); TRY(dalloc(c, &h.beta, nb)); TRY(dalloc(c, &h.est, nb));
  TRY(dalloc(c, &h.H, (size_t)nb * (m + 1) * m));
  TRY(dalloc(c, &h.cs, (size_t)nb * m));
  TRY(dalloc(c, &h.sn, (size_t)nb * m));
  TRY(dalloc(c, &h.g, (size_t)nb * (m + 1)));
  TRY(dalloc(c, &h.y, (size_t)m * nb));
  TRY(dalloc(c, &W.ctl, 1));
  CU(cudaMemcpy(W.ctl, &h, sizeof(BatchCtl), cudaMemcpyHostToDevice));
  for (int l = 0; l < c->nlev; ++l) {
    const size_t np = c->L[l].g.npts() * nb;
    if (mixed) {
      TRY(dalloc(c, &W.U132[l], np)); TRY(dalloc(c, &W.T32[l], np));
      if (l > 0) { TRY(dalloc(c, &W.B32[l], np)); TRY(dalloc(c, &W.E32[l], np)); }
    } else {
      TRY(dalloc(c, &W.U164[l], np)); TRY(dalloc(c, &W.T64[l], np));
      if (l > 0) { TRY(dalloc(c, &W.B64[l], np)); TRY(dalloc(c, &W.E64[l], np)); }
    }
  }
  if (!W.hany) CU(cudaHostAlloc((void**)&W.hany, sizeof(int) * (m + FLAG_LAG + 1), cudaHostAllocDefault));
  W.nb = nb;
  return HELM_OK;
}

template <typename R> VLevel<R> batch_level(helm_ctx* c, int l, int nb);
template <>
VLevel<float> batch_level<float>(helm_ctx* c, int l, int nb) {
  Level& L = c->L[l];
  VLevel<float> v{L.g, L.k2f, nullptr, c->bw.B32[l], c->bw.U132[l], c->bw.T32[l], c->bw.E32[l]};
  v.g.nb = nb;
  return v;
}
template <>
VLevel<double> batch_level<double>(helm_ctx* c, int l, int nb) {
  Level& L = c->L[l];
  VLevel<double> v{L.g, L.k2, L.dinv, c->bw.B64[l], c->bw.U164[l], c->bw.T64[l], c->bw.E64[l]};
  v.g.nb = nb;
  return v;
}

// Lockstep FGMRES(m) for the nb right-hand sides held in bw.Bt / bw.Xt.
helm_status gmres_batched(helm_ctx* c, int nb, cudaStream_t st) {
  BatchWS& W = c->bw;
  const size_t n = c->n0, ne = n * nb;
  const int m = c->m;
  const bool mixed = c->p.precision == HELM_PREC_MIXED;
  const double tol = c->p.tol;
  Grid g0 = c->L[0].g;
  g0.nb = nb;
  const double* k2 = c->L[0].k2;
  BatchCtl* ctl = W.ctl;
  const int* any = &ctl->any;
  VLevel<float> lv32[MAX_LEVELS];
  VLevel<double> lv64[MAX_LEVELS];
  for (int l = 0; l < c->nlev; ++l) {
    if (mixed) lv32[l] = batch_level<float>(c, l, nb);
    else lv64[l] = batch_level<double>(c, l, nb);
  }
  if (c->p.autotune) {
    int t = 0;
    while ((1 << t) < nb) ++t;
    if (!W.tuned[t]) {
      if (mixed) {
        TRY(tune_vlevels<float>(c, lv32, c->nlev, st));
        CU(cudaMemsetAsync(W.r, 0x3f, ne * sizeof(z128), st));
        TRY(tune_slot(c, g0, tile_slot<double>(TILE_STENCIL), 0, st, [&](const Grid& g) {
          launch_resid<double, double, double, double>(g, 1.0, 0.0, k2, W.r, W.r, W.V, st, nullptr);
        }));
      } else {
        TRY(tune_vlevels<double>(c, lv64, c->nlev, st));
        for (int q = 0; q < 8; ++q) {
          g0.tile_ty[q] = lv64[0].g.tile_ty[q];
          g0.tile_ctas[q] = lv64[0].g.tile_ctas[q];
        }
      }
      for (int l = 0; l < c->nlev; ++l) {
        const Grid& g = mixed ? lv32[l].g : lv64[l].g;
        for (int q = 0; q < 8; ++q) { W.tty[t][l][q] = g.tile_ty[q]; W.tct[t][l][q] = g.tile_ctas[q]; }
      }
      for (int q = 0; q < 8; ++q) { W.g0ty[t][q] = g0.tile_ty[q]; W.g0ct[t][q] = g0.tile_ctas[q]; }
      if (c->p.orth == HELM_ORTH_DF && m >= 2) {
        // double-float dots: slots per warp pass (logged as level -2, slot 8 + variant)
        const int nvt = std::min(16, m);
        zdf* Vd = reinterpret_cast<zdf*>(W.V);
        CU(cudaMemsetAsync(W.V, 0x3f, (size_t)(nvt + 1) * ne * sizeof(z128), st));
        CU(cudaMemsetAsync(W.wdf, 0x3f, ne * sizeof(zdf), st));
        cudaEvent_t e0, e1;
        CU(cudaEventCreate(&e0));
        CU(cudaEventCreate(&e1));
        float best = 1e30f;
        for (int v = 0; v < 3; ++v) {
          launch_bmdot_df(Vd, ne, nvt, W.wdf, ne, nb, W.part, 1, st, nullptr, v);
          CU(cudaEventRecord(e0, st));
          launch_bmdot_df(Vd, ne, nvt, W.wdf, ne, nb, W.part, 1, st, nullptr, v);
          CU(cudaEventRecord(e1, st));
          CU(cudaEventSynchronize(e1));
          float ms = 0.f;
          CU(cudaEventElapsedTime(&ms, e0, e1));
          c->tune_log.push_back(TuneRec{-2, 8 + v, nvt, nb, ms});
          if (ms < best) { best = ms; W.bmdot_variant[t] = v; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        TRY(check_launch(c, "autotune (batched inner products)"));
      }
      W.tuned[t] = true;
    } else {
      for (int l = 0; l < c->nlev; ++l) {
        Grid& g = mixed ? lv32[l].g : lv64[l].g;
        for (int q = 0; q < 8; ++q) { g.tile_ty[q] = W.tty[t][l][q]; g.tile_ctas[q] = W.tct[t][l][q]; }
      }
      for (int q = 0; q < 8; ++q) { g0.tile_ty[q] = W.g0ty[t][q]; g0.tile_ctas[q] = W.g0ct[t][q]; }
    }
  }
  int bvar = 0;
  {
    int t = 0;
    while ((1 << t) < nb) ++t;
    bvar = W.bmdot_variant[t];
  }
  const double nd = (double)ne;
  int nblk = launch_bnorm2_part(W.Bt, ne, nb, W.partr, st, c->one);
  launch_breduce_norm(W.partr, nb, nblk, W.h.bnorm, st, c->one);
  KL(F_RESID, 56.0 * nd, 24.0 * nd, (launch_resid<double, double, double, double>(g0, 1.0, 0.0, k2, W.Xt, W.Bt, W.r, st, c->one)));
  nblk = launch_bnorm2_part(W.r, ne, nb, W.partr, st, c->one);
  launch_breduce_norm(W.partr, nb, nblk, W.h.beta, st, c->one);
  CU(cudaMemsetAsync(W.h.iters, 0, sizeof(int) * nb, st));
  for (int cycle = 0;; ++cycle) {
    launch_bcycle_init(ctl, nb, m, tol, st);
    CU(cudaMemcpyAsync(W.hany, any, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (W.hany[0] == 0) break;
    const bool df = c->p.orth == HELM_ORTH_DF;
    zdf* Vdf = reinterpret_cast<zdf*>(W.V);
    if (df) {
      if (mixed) KL(F_SCALE, 40.0 * nd, 2.0 * nd, (launch_bscale_df<z128, float>(W.r, W.h.beta, Vdf, W.vcur32, ne, nb, st, any)));
      else KL(F_SCALE, 48.0 * nd, 2.0 * nd, (launch_bscale_df<z128, double>(W.r, W.h.beta, Vdf, W.vcur64, ne, nb, st, any)));
    } else {
      KL(F_SCALE, (W.Vs ? 40.0 : 32.0) * nd, (W.Vs ? 3.0 : 2.0) * nd,
         launch_bscale_inv(W.r, W.h.beta, W.V, W.Vs, ne, nb, st, any));
    }
    for (int j = 0; j < m; ++j) {
      c->cur_j = j;
      auto step = [&](cudaStream_t st) {
        z128* vj = W.V + (size_t)j * ne;
        z128* w = W.V + (size_t)(j + 1) * ne;
        const double nv = j + 1;
        if (mixed) {
          z64* zj = W.Z32 + (size_t)j * ne;
          if (df) {
            run_cycle_levels<float, float, float>(c, lv32, W.vcur32, zj, st, any);
            KL(F_APPLY, 32.0 * nd, 22.0 * nd, (launch_apply_c64_df<zdf>(g0, c->k2df, c->skdf, zj, W.wdf, st, any)));
          } else {
            run_cycle_levels<float, double, float>(c, lv32, vj, zj, st, any);
            KL(F_APPLY, 32.0 * nd, 22.0 * nd, (launch_apply<double, float, double>(g0, 1.0, 0.0, k2, zj, w, st, any)));
          }
        } else {
          z128* zj = W.Z64 + (size_t)j * ne;
          run_cycle_levels<double, double, double>(c, lv64, df ? W.vcur64 : vj, zj, st, any);
          if (df)
            KL(F_APPLY, 40.0 * nd, 22.0 * nd, (launch_apply_split<double>(g0, 1.0, 0.0, k2, zj, W.wdf, st, any)));
          else
            KL(F_APPLY, 40.0 * nd, 22.0 * nd, (launch_apply<double, double, double>(g0, 1.0, 0.0, k2, zj, w, st, any)));
        }
        const bool sel = c->p.reorth == HELM_REORTH_SELECTIVE;
        for (int pass = 0; pass < 2; ++pass) {
          const int* a2 = (pass == 1 && sel) ? &ctl->pass2 : any;
          c->cur_cond = (pass == 1 && sel) ? 1 : 0;
          const int wn = (pass == 0 && sel) ? 1 : 0;
          int nbk = 0;
          // FP64 second pass with the selective test: only the right-hand sides that need it
          // (profiled per right-hand side and scaled by the logged count)
          const bool per_rhs = pass == 1 && sel && !df;
          if (per_rhs) c->cur_cond = 2;
          if (per_rhs)
            KL(F_MDOT, ((W.Vs ? 24.0 * nv + 16.0 : 16.0 * (nv + 1)) * nd) / nb, 8.0 * nv * nd / nb,
               nbk = launch_bmdot_sel(W.V, W.Vs, ne, j + 1, w, ne, nb, W.need, W.part, st, a2));
          else if (df)
            KL(F_MDOT, 16.0 * (nv + 1) * nd, 8.0 * nv * nd,
               nbk = launch_bmdot_df(Vdf, ne, j + 1, W.wdf, ne, nb, W.part, wn, st, a2, bvar));
          else if (W.Vs)
            // algorithmic flops: 8 per basis vector and element (a complex multiply-add), of which
            // the summed form executes 6; bytes: what its layout must move
            KL(F_MDOT, (24.0 * nv + 16.0) * nd, 8.0 * nv * nd,
               nbk = launch_bmdot(W.V, W.Vs, ne, j + 1, w, ne, nb, W.part, wn, st, a2));
          else
            KL(F_MDOT, 16.0 * (nv + 1) * nd, 8.0 * nv * nd,
               nbk = launch_bmdot(W.V, nullptr, ne, j + 1, w, ne, nb, W.part, wn, st, a2));
          if (per_rhs) c->cur_cond = 1;
          KL(F_REDUCE_DOTS, 16.0 * nv * nb * nbk, 2.0 * nv * nb * nbk,
             launch_breduce_dots(W.part, j + 1, nb, nbk, W.hpass, W.hacc, pass, wn ? j : -1, W.h.act, &ctl->pass2,
                                 c->reorth_log, W.sw2, W.need, st, a2, c->p.reorth_keep));
          if (per_rhs) c->cur_cond = 2;
          if (per_rhs)
            KL(F_GS_UPDATE, ((W.Vs ? 24.0 * nv + 32.0 : 16.0 * (nv + 2)) * nd) / nb, 8.0 * nv * nd / nb,
               launch_bgs_update_sel(W.V, W.Vs, ne, j + 1, nb, W.hpass, w, ne, W.need, st, a2));
          else if (df)
            KL(F_GS_UPDATE, 16.0 * (nv + 2) * nd, 8.0 * nv * nd, launch_bgs_update_df(Vdf, ne, j + 1, nb, W.hpass, W.wdf, ne, st, a2));
          else
            KL(F_GS_UPDATE, (W.Vs ? 24.0 * nv + 32.0 : 16.0 * (nv + 2)) * nd, 8.0 * nv * nd,
               launch_bgs_update(W.V, W.Vs, ne, j + 1, nb, W.hpass, w, ne, st, a2));
        }
        c->cur_cond = 0;
        int nbn = 0;
        if (df)
          KL(F_NORM, 16.0 * nd, 4.0 * nd, nbn = launch_bnorm2_part_df(W.wdf, ne, nb, W.partr, st, any));
        else
          KL(F_NORM, 16.0 * nd, 4.0 * nd, nbn = launch_bnorm2_part(w, ne, nb, W.partr, st, any));
        KL(F_REDUCE_NORM, 8.0 * nb * nbn, nb * nbn, launch_breduce_norm(W.partr, nb, nbn, W.hnorm, st, any));
        KL(F_GIVENS, 0, 0, launch_bgivens(ctl, nb, m, j, W.hacc, W.hnorm, tol, st));
        if (df) {
          zdf* vn = Vdf + (size_t)(j + 1) * ne;
          if (mixed) KL(F_SCALE, 40.0 * nd, 2.0 * nd, (launch_bscale_df<zdf, float>(W.wdf, W.hnorm, vn, W.vcur32, ne, nb, st, any)));
          else KL(F_SCALE, 48.0 * nd, 2.0 * nd, (launch_bscale_df<zdf, double>(W.wdf, W.hnorm, vn, W.vcur64, ne, nb, st, any)));
        } else {
          KL(F_SCALE, (W.Vs ? 40.0 : 32.0) * nd, (W.Vs ? 3.0 : 2.0) * nd,
             launch_bscale_inv(w, W.hnorm, w, W.Vs ? W.Vs + (size_t)(j + 1) * ne : nullptr, ne, nb, st, any));
        }
      };
      // one graph per Arnoldi column and batch width (the workspace and the tuned shapes of
      // that width are fixed)
      TRY(graph_step(c, G_BATCH + nb, j, W.V, st, step));
      TRY(check_launch(c, "batched Arnoldi step"));
      CU(cudaMemcpyAsync(W.hany + j, any, sizeof(int), cudaMemcpyDeviceToHost, st));
      CU(cudaEventRecord(c->ev[j % c->nev], st));
      if (j >= FLAG_LAG) {
        CU(cudaEventSynchronize(c->ev[(j - FLAG_LAG) % c->nev]));
        if (W.hany[j - FLAG_LAG] == 0) break;
      }
    }
    c->cur_j = -1;
    CU(cudaMemcpyAsync(c->hreorth_log, c->reorth_log, sizeof(int) * m, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    prof_flush(c, m);
    KL(F_SOLUPDATE, 0, 0, launch_btrisolve(ctl, nb, m, st));
    if (mixed)
      if (c->p.orth == HELM_ORTH_DF)
        KL(F_SOLUPDATE, 8.0 * m * nd, 8.0 * m * nd, launch_bxupdate_df(ctl, nb, m, W.Z32, ne, W.Xt, ne, st));
      else
        KL(F_SOLUPDATE, 8.0 * m * nd, 8.0 * m * nd, launch_bxupdate<float>(ctl, nb, m, W.Z32, ne, W.Xt, ne, st));
    else
      KL(F_SOLUPDATE, 16.0 * m * nd, 8.0 * m * nd, launch_bxupdate<double>(ctl, nb, m, W.Z64, ne, W.Xt, ne, st));
    KL(F_RESID, 56.0 * nd, 24.0 * nd, (launch_resid<double, double, double, double>(g0, 1.0, 0.0, k2, W.Xt, W.Bt, W.r, st, c->one)));
    nblk = launch_bnorm2_part(W.r, ne, nb, W.partr, st, c->one);
    launch_breduce_norm(W.partr, nb, nblk, W.h.beta, st, c->one);
    TRY(check_launch(c, "batched solution update"));
    prof_flush(c, -1);
  }
  return HELM_OK;
}

// Right-preconditioned Bi-CGSTAB on device-resident b and x: two V-cycles and two products
// with A per step, scalars on the device, the host checking the stop flag two steps behind.
// A converged recursion is confirmed with the explicit residual; if that is still above
// tol, the method restarts from it.
helm_status bicgstab_device(helm_ctx* c, const z128* b, z128* x, helm_solve_info* info, cudaStream_t st) {
  const Level& F = c->L[0];
  const size_t n = c->n0;
  const bool mixed = c->p.precision == HELM_PREC_MIXED;
  const double tol = c->p.tol;
  const int maxit = c->p.max_iter;
  const int stall = c->p.stall_window;
  BicgCtl* bc = c->bicg;
  z128 *r = c->V, *rh = c->V + n, *p = c->V + 2 * n, *v = c->V + 3 * n, *ph = c->V + 4 * n, *s = c->V + 5 * n,
       *sh = c->V + 6 * n, *t = c->V + 7 * n;
  const int* act = &bc->active;
  const int* cont = &bc->cont;
  const double nd = (double)n;
  CU(cudaMemsetAsync(bc, 0, sizeof(BicgCtl), st));
  norm_into(c, b, &bc->bnorm, st, c->one);
  CU(cudaMemcpyAsync(c->hbicg, bc, sizeof(BicgCtl), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (c->hbicg->bnorm == 0.0) {
    CU(cudaMemsetAsync(x, 0, n * sizeof(z128), st));
    CU(cudaStreamSynchronize(st));
    if (info) { info->iterations = 0; info->restarts = 0; info->rel_residual = 0.0; }
    return HELM_OK;
  }
  int restarts = 0, flat = 0;
  helm_status status = HELM_OK;
  double relres = 0.0, best = 0.0;
  for (;;) {
    KL(F_RESID, 56.0 * nd, 24.0 * nd, (launch_resid<double, double, double, double>(F.g, 1.0, 0.0, F.k2, x, b, r, st, c->one)));
    int nb = 0;
    KL(F_MDOT, 32.0 * nd, 4.0 * nd, nb = launch_dots2(r, r, nullptr, nullptr, n, c->part, st, c->one));
    KL(F_MISC, 0, 0, launch_bicg_init(bc, c->part, nb, r, rh, p, v, n, st));
    CU(cudaMemcpyAsync(c->hbicg, bc, sizeof(BicgCtl), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    relres = c->hbicg->relres;
    if (relres <= tol) { status = HELM_OK; break; }
    if (!(relres == relres)) { status = HELM_ENUMERIC; break; }
    if (c->hbicg->iters >= maxit) { status = HELM_ENOCONV; break; }
    for (int step = 0;; ++step) {
      c->cur_j = -1;
      auto enq = [&](cudaStream_t st) {
        KL(F_GIVENS, 0, 0, launch_bicg_scalar(bc, c->part, nb, 0, tol, maxit, stall, c->hist, c->hist_len, st));
        KL(F_GS_UPDATE, 48.0 * nd, 8.0 * nd, launch_bicg_p(r, p, v, bc, n, st));
        if (mixed) run_cycle<float, double, double>(c, p, ph, st, act);
        else run_cycle<double, double, double>(c, p, ph, st, act);
        KL(F_APPLY, 40.0 * nd, 22.0 * nd, (launch_apply<double, double, double>(F.g, 1.0, 0.0, F.k2, ph, v, st, act)));
        KL(F_MDOT, 32.0 * nd, 8.0 * nd, nb = launch_dots2(rh, v, nullptr, nullptr, n, c->part, st, act));
        KL(F_GIVENS, 0, 0, launch_bicg_scalar(bc, c->part, nb, 1, tol, maxit, stall, c->hist, c->hist_len, st));
        KL(F_GS_UPDATE, 48.0 * nd, 8.0 * nd, nb = launch_bicg_s(r, v, s, bc, n, c->part, st));
        KL(F_GIVENS, 0, 0, launch_bicg_scalar(bc, c->part, nb, 2, tol, maxit, stall, c->hist, c->hist_len, st));
        if (mixed) run_cycle<float, double, double>(c, s, sh, st, cont);
        else run_cycle<double, double, double>(c, s, sh, st, cont);
        KL(F_APPLY, 40.0 * nd, 22.0 * nd, (launch_apply<double, double, double>(F.g, 1.0, 0.0, F.k2, sh, t, st, cont)));
        KL(F_MDOT, 48.0 * nd, 12.0 * nd, nb = launch_dots2(t, s, t, t, n, c->part, st, cont));
        KL(F_GIVENS, 0, 0, launch_bicg_scalar(bc, c->part, nb, 3, tol, maxit, stall, c->hist, c->hist_len, st));
        KL(F_GS_UPDATE, 112.0 * nd, 20.0 * nd, nb = launch_bicg_xr(x, r, ph, sh, s, t, rh, bc, n, c->part, st));
        KL(F_GIVENS, 0, 0, launch_bicg_scalar(bc, c->part, nb, 4, tol, maxit, stall, c->hist, c->hist_len, st));
      };
      TRY(graph_step(c, G_BICG, 0, x, st, enq));
      TRY(check_launch(c, "Bi-CGSTAB step"));
      const int slot = step % (c->m + FLAG_LAG + 1);
      CU(cudaMemcpyAsync(c->hflags + slot, act, sizeof(int), cudaMemcpyDeviceToHost, st));
      CU(cudaEventRecord(c->ev[step % c->nev], st));
      if (step >= FLAG_LAG) {
        CU(cudaEventSynchronize(c->ev[(step - FLAG_LAG) % c->nev]));
        if (c->hflags[(step - FLAG_LAG) % (c->m + FLAG_LAG + 1)] == 0) break;
      }
    }
    CU(cudaMemcpyAsync(c->hbicg, bc, sizeof(BicgCtl), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    prof_flush(c, -1);
    const BicgCtl h = *c->hbicg;
    // explicit residual
    KL(F_RESID, 56.0 * nd, 24.0 * nd, (launch_resid<double, double, double, double>(F.g, 1.0, 0.0, F.k2, x, b, r, st, c->one)));
    norm_into(c, r, &bc->relres, st, c->one);
    double rn = 0.0;
    CU(cudaMemcpyAsync(&rn, &bc->relres, sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    relres = rn / h.bnorm;
    if (relres <= tol) { status = HELM_OK; break; }
    if (h.flag == 2 || !(relres == relres)) { status = HELM_ENUMERIC; break; }
    if (h.flag == 3) {
      status = fail(c, HELM_ENOCONV, "Bi-CGSTAB stagnated: the residual did not halve within stall_window "
                                          "products with A (with precision = mixed the complex64 cycle is not a "
                                          "fixed preconditioner; FGMRES or IDR(s) converge there)");
      break;
    }
    if (h.iters >= maxit) { status = HELM_ENOCONV; break; }
    // the recursion met tol but the explicit residual did not: restart from it, unless three
    // restarts in a row have not halved the best explicit residual
    flat = (restarts > 0 && relres > 0.5 * best) ? flat + 1 : 0;
    best = restarts > 0 ? fmin(best, relres) : relres;
    if (stall > 0 && flat >= 3) {
      status = fail(c, HELM_ENOCONV, "Bi-CGSTAB stagnated: three restarts from the explicit residual did not "
                                          "halve it (the recursive residual drifts from the true one)");
      break;
    }
    ++restarts;
  }
  CU(cudaMemcpyAsync(c->hbicg, bc, sizeof(BicgCtl), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (info) {
    info->iterations = c->hbicg->iters;
    info->restarts = restarts;
    info->rel_residual = relres;
  }
  return status;
}

// Right-preconditioned IDR(s), biorthogonal form (Sec. 3.1), on device-resident vectors.
// The host enqueues whole steps and stops on a lagged copy of the device's active flag.
helm_status idrs_device(helm_ctx* c, const z128* b, z128* x, helm_solve_info* info, cudaStream_t st) {
  if (c->idr_s < 1) return fail(c, HELM_EINVAL, "IDR(s) needs a shadow space (helm_set_shadow_space)");
  const Level& F = c->L[0];
  const size_t n = c->n0;
  const int s = c->idr_s;
  const bool mixed = c->p.precision == HELM_PREC_MIXED;
  const double tol = c->p.tol;
  const int maxit = c->p.max_iter;
  IdrCtl* ic = c->idr;
  z128 *G = c->idrW, *U = G + (size_t)s * n, *r = U + (size_t)s * n, *v = r + n, *vh = v + n, *t = vh + n;
  const z128* P = c->idrP;
  z128* part = c->idr_part;
  const int* act = &ic->active;
  const double nd = (double)n, sd = (double)s;
  IdrCtl h0;
  memset(&h0, 0, sizeof(h0));
  h0.s = s;
  h0.kappa = c->p.idr_kappa;
  CU(cudaMemcpyAsync(ic, &h0, sizeof(IdrCtl), cudaMemcpyHostToDevice, st));
  norm_into(c, b, &ic->bnorm, st, c->one);
  CU(cudaMemcpyAsync(c->hidr, ic, sizeof(IdrCtl), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (c->hidr->bnorm == 0.0) {
    CU(cudaMemsetAsync(x, 0, n * sizeof(z128), st));
    CU(cudaStreamSynchronize(st));
    if (info) { info->iterations = 0; info->restarts = 0; info->rel_residual = 0.0; }
    return HELM_OK;
  }
  const int ring = c->m + FLAG_LAG + 1;
  int restarts = 0;
  helm_status status = HELM_OK;
  double relres = 0.0;
  for (;;) {
    KL(F_RESID, 56.0 * nd, 24.0 * nd, (launch_resid<double, double, double, double>(F.g, 1.0, 0.0, F.k2, x, b, r, st, c->one)));
    CU(cudaMemsetAsync(G, 0, 2 * (size_t)s * n * sizeof(z128), st));
    int nb = 0;
    KL(F_MDOT, 16.0 * (sd + 1) * nd, 4.0 * (sd + 1) * nd, nb = launch_idr_pdots(s, true, P, r, n, part, st, c->one));
    KL(F_MISC, 0, 0, launch_idr_scalar(ic, part, nb, 5, 0, tol, maxit, c->hist, c->hist_len, st));
    CU(cudaMemcpyAsync(c->hidr, ic, sizeof(IdrCtl), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    relres = c->hidr->relres;
    if (c->hidr->active == 0) {
      status = c->hidr->flag == 1 ? HELM_OK : HELM_ENUMERIC;
      break;
    }
    if (c->hidr->iters >= maxit) { status = HELM_ENOCONV; break; }
    int step = 0;
    bool stop = false;
    auto lagged = [&](void) -> helm_status {
      const int slot = step % ring;
      CU(cudaMemcpyAsync(c->hflags + slot, act, sizeof(int), cudaMemcpyDeviceToHost, st));
      CU(cudaEventRecord(c->ev[step % c->nev], st));
      if (step >= FLAG_LAG) {
        CU(cudaEventSynchronize(c->ev[(step - FLAG_LAG) % c->nev]));
        if (c->hflags[(step - FLAG_LAG) % ring] == 0) stop = true;
      }
      ++step;
      return HELM_OK;
    };
    while (!stop) {
      for (int k = 0; k < s && !stop; ++k) {
        c->cur_j = -1;
        const double wk = (double)(s - k);
        auto enq = [&](cudaStream_t st) {
          KL(F_GIVENS, 0, 0, launch_idr_scalar(ic, part, 0, 0, k, tol, maxit, c->hist, c->hist_len, st));
          KL(F_GS_UPDATE, 16.0 * (wk + 2) * nd, 8.0 * wk * nd, launch_idr_v(ic, k, r, G, n, v, st));
          if (mixed) run_cycle<float, double, double>(c, v, vh, st, act);
          else run_cycle<double, double, double>(c, v, vh, st, act);
          KL(F_GS_UPDATE, 16.0 * (wk + 2) * nd, 8.0 * (wk + 1) * nd, launch_idr_u(ic, k, vh, U, n, st));
          KL(F_APPLY, 40.0 * nd, 22.0 * nd,
             (launch_apply<double, double, double>(F.g, 1.0, 0.0, F.k2, U + (size_t)k * n, G + (size_t)k * n, st, act)));
          KL(F_MDOT, 16.0 * (sd + 1) * nd, 8.0 * sd * nd,
             nb = launch_idr_pdots(s, false, P, G + (size_t)k * n, n, part, st, act));
          KL(F_GIVENS, 0, 0, launch_idr_scalar(ic, part, nb, 1, k, tol, maxit, c->hist, c->hist_len, st));
          KL(F_GS_UPDATE, 16.0 * (2.0 * k + 8) * nd, (16.0 * k + 20) * nd,
             nb = launch_idr_update(ic, k, G, U, r, x, n, part, st));
          KL(F_GIVENS, 0, 0, launch_idr_scalar(ic, part, nb, 2, k, tol, maxit, c->hist, c->hist_len, st));
        };
        TRY(graph_step(c, G_IDR, k, x, st, enq));
        TRY(check_launch(c, "IDR(s) step"));
        TRY(lagged());
      }
      if (stop) break;
      // dimension reduction
      auto enq_dr = [&](cudaStream_t st) {
        if (mixed) run_cycle<float, double, double>(c, r, vh, st, act);
        else run_cycle<double, double, double>(c, r, vh, st, act);
        KL(F_APPLY, 40.0 * nd, 22.0 * nd, (launch_apply<double, double, double>(F.g, 1.0, 0.0, F.k2, vh, t, st, act)));
        KL(F_MDOT, 32.0 * nd, 12.0 * nd, nb = launch_dots2(t, r, t, t, n, part, st, act));
        KL(F_GIVENS, 0, 0, launch_idr_scalar(ic, part, nb, 3, 0, tol, maxit, c->hist, c->hist_len, st));
        KL(F_GS_UPDATE, 16.0 * (sd + 6) * nd, (8.0 * sd + 20) * nd,
           nb = launch_idr_xr(s, ic, P, r, t, x, vh, n, part, st));
        KL(F_GIVENS, 0, 0, launch_idr_scalar(ic, part, nb, 4, 0, tol, maxit, c->hist, c->hist_len, st));
      };
      TRY(graph_step(c, G_IDR_DR, 0, x, st, enq_dr));
      TRY(check_launch(c, "IDR(s) dimension reduction"));
      TRY(lagged());
    }
    CU(cudaMemcpyAsync(c->hidr, ic, sizeof(IdrCtl), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    prof_flush(c, -1);
    const IdrCtl h = *c->hidr;
    // explicit residual
    KL(F_RESID, 56.0 * nd, 24.0 * nd, (launch_resid<double, double, double, double>(F.g, 1.0, 0.0, F.k2, x, b, r, st, c->one)));
    norm_into(c, r, &ic->relres, st, c->one);
    double rn = 0.0;
    CU(cudaMemcpyAsync(&rn, &ic->relres, sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    relres = rn / h.bnorm;
    if (relres <= tol) { status = HELM_OK; break; }
    if (h.flag == 2 || !(relres == relres)) { status = HELM_ENUMERIC; break; }
    if (h.iters >= maxit) { status = HELM_ENOCONV; break; }
    ++restarts;  // the recursion met tol but the explicit residual did not: restart from it
    h0.iters = h.iters;
    h0.bnorm = h.bnorm;
    CU(cudaMemcpyAsync(ic, &h0, sizeof(IdrCtl), cudaMemcpyHostToDevice, st));
  }
  CU(cudaMemcpyAsync(c->hidr, ic, sizeof(IdrCtl), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (info) {
    info->iterations = c->hidr->iters;
    info->restarts = restarts;
    info->rel_residual = relres;
  }
  return status;
}

// The configured outer Krylov method on device-resident vectors.
helm_status krylov_device(helm_ctx* c, const z128* b, z128* x, helm_solve_info* info, cudaStream_t st) {
  if (c->p.krylov == HELM_IDRS) return idrs_device(c, b, x, info, st);
  return c->p.krylov == HELM_BICGSTAB ? bicgstab_device(c, b, x, info, st) : gmres_device(c, b, x, info, st);
}

}  // namespace

// Message slot of helm_last_error(NULL), shared with the context-free entry point.
void helm_set_global_error(const char* msg) { g_create_error = msg; }

namespace {

// nrhs solves with A (or, adjoint, with A^H from a zero start) in chunks of <= 32 lockstep
// right-hand sides; B, X device, nrhs vectors each.  The adjoint goes through the forward solver:
// A nu = D^-1 conj(g), lambda = conj(D nu), applied in the batched layout.
helm_status solve_batched_core(helm_ctx* c, int nrhs, const z128* B, z128* X, helm_solve_info* infos, cudaStream_t st,
                               bool adjoint) {
  const auto t0 = std::chrono::steady_clock::now();
  const size_t n = c->n0;
  helm_status worst = HELM_OK;
  for (int start = 0; start < nrhs; start += 32) {
    const int cnt = std::min(32, nrhs - start);
    int nb = 1;
    while (nb < cnt) nb <<= 1;
    TRY(batch_alloc(c, nb));
    BatchWS& W = c->bw;
    Grid gb = c->L[0].g;
    gb.nb = nb;
    launch_to_batch(B + (size_t)start * n, W.Bt, n, nb, cnt, st);
    if (adjoint) {
      launch_adjoint_rhs(gb, W.Bt, W.Bt, st);
      CU(cudaMemsetAsync(W.Xt, 0, n * nb * sizeof(z128), st));
    } else {
      launch_to_batch(X + (size_t)start * n, W.Xt, n, nb, cnt, st);
    }
    TRY(check_launch(c, "batch transpose"));
    TRY(gmres_batched(c, nb, st));
    if (adjoint) launch_adjoint_finish(gb, W.Xt, st);
    launch_from_batch(W.Xt, X + (size_t)start * n, n, nb, cnt, st);
    std::vector<int> it(nb);
    std::vector<double> bn(nb), be(nb);
    CU(cudaMemcpyAsync(it.data(), W.h.iters, sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(bn.data(), W.h.bnorm, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(be.data(), W.h.beta, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int r = 0; r < cnt; ++r) {
      const double rr = bn[r] > 0.0 ? be[r] / bn[r] : 0.0;
      helm_status sr = HELM_OK;
      if (!(rr == rr) || rr == HUGE_VAL) sr = HELM_ENUMERIC;
      else if (rr > c->p.tol) sr = HELM_ENOCONV;
      if (sr != HELM_OK && worst != HELM_ENUMERIC) worst = sr;
      if (infos) {
        helm_solve_info& I = infos[start + r];
        I.iterations = it[r];
        I.restarts = 0;
        I.rel_residual = rr;
        I.status = (int)sr;
        I.ms_total = ms;
      }
    }
  }
  if (worst == HELM_ENOCONV) fail(c, worst, "some right-hand sides reached max_iter (%d)", c->p.max_iter);
  if (worst == HELM_ENUMERIC) fail(c, worst, "non-finite residual in a batched solve");
  return worst;
}

}  // namespace

namespace {

// helm_solve / helm_solve_zero: the solve through device or host buffers; with `zero` the
// initial guess is 0 and x is output only (not read, so not copied to the device).
helm_status solve_entry(helm_ctx* c, const void* b, void* x, helm_solve_info* info, void* stream, bool zero) {
  if (!c) return HELM_EINVAL;
  if (!b || !x || b == x) return fail(c, HELM_EINVAL, "b and x must be distinct non-NULL pointers");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)stream;
  const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
  if (bdev != xdev) return fail(c, HELM_EINVAL, "b and x must both be device or both be host pointers");
  const size_t bytes = c->n0 * sizeof(z128);
  const z128* bd = (const z128*)b;
  z128* xd = (z128*)x;
  if (!bdev) {
    CU(cudaMemcpyAsync(c->bs, b, bytes, cudaMemcpyHostToDevice, st));
    if (!zero) CU(cudaMemcpyAsync(c->xs, x, bytes, cudaMemcpyHostToDevice, st));
    bd = c->bs;
    xd = c->xs;
  }
  if (zero) CU(cudaMemsetAsync(xd, 0, bytes, st));
  helm_solve_info tmp;
  helm_solve_info* inf = info ? info : &tmp;
  c->err.clear();
  helm_status s = krylov_device(c, bd, xd, inf, st);
  if (!bdev && (s == HELM_OK || s == HELM_ENOCONV || s == HELM_ENUMERIC)) {
    CU(cudaMemcpyAsync(x, c->xs, bytes, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
  }
  inf->status = (int)s;
  inf->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (s == HELM_ENOCONV && c->err.empty())
    fail(c, s, "max_iter (%d) reached at relative residual %.3e", c->p.max_iter, inf->rel_residual);
  if (s == HELM_ENUMERIC) fail(c, s, "non-finite residual or Krylov breakdown");
  return s;
}

}  // namespace

extern "C" {

void helm_default_params(helm_params* p) {
  if (!p) return;
  p->beta1 = 1.0;
  p->beta2 = -0.5;
  p->omega = 0.8;
  p->nu1 = 1;
  p->nu2 = 1;
  p->coarsest_n = 4;
  p->krylov = HELM_GMRES;
  p->restart = 30;
  p->tol = 1e-6;
  p->max_iter = 2000;
  p->precision = HELM_PREC_FP64;
  p->orth = HELM_ORTH_FP64;
  p->reorth = HELM_REORTH_SELECTIVE;
  p->cycle = HELM_CYCLE_V;
  p->idr_kappa = 0.7;
  p->graphs = 1;
  p->autotune = 1;
  p->side = HELM_SIDE_RIGHT;
  p->fuse_coarse = 0;
  p->gs_sums = 1;
  p->fuse_down = -1;
  p->fuse_up = -1;
  p->stall_window = 1000;
  p->reorth_keep = 0.1;
  p->coarse_tol = 0.0;
}

const char* helm_last_error(const helm_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

helm_status helm_convert_check(const float* in32, double* out64, size_t n, void* stream) {
  if (n == 0) return HELM_OK;
  if (!in32 || !out64) {
    helm_set_global_error("helm_convert_check: NULL pointer");
    return HELM_EINVAL;
  }
  launch_convert_check(in32, out64, n, (cudaStream_t)stream);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    helm_set_global_error(cudaGetErrorString(e));
    return HELM_ECUDA;
  }
  return HELM_OK;
}

helm_status helm_profile(helm_ctx* c, int enable) {
  if (!c) return HELM_EINVAL;
  prof_flush(c, 1 << 30);
  Prof& P = c->prof;
  for (int f = 0; f < F_COUNT; ++f) { P.ms[f] = P.bytes[f] = P.flops[f] = 0.0; P.cnt[f] = 0; }
  P.launches = 0;
  P.on = enable != 0;
  return HELM_OK;
}

helm_status helm_profile_read(helm_ctx* c, helm_kernel_stat* stats, int cap, int* count, long long* launches) {
  if (!c) return HELM_EINVAL;
  prof_flush(c, 1 << 30);
  const Prof& P = c->prof;
  int k = 0;
  for (int f = 0; f < F_COUNT && stats && k < cap; ++f, ++k) {
    stats[k].name = FAM_NAMES[f];
    stats[k].launches = P.cnt[f];
    stats[k].ms = P.ms[f];
    stats[k].bytes = P.bytes[f];
    stats[k].flops = P.flops[f];
  }
  if (count) *count = stats ? k : F_COUNT;
  if (launches) *launches = P.launches;
  return HELM_OK;
}

helm_status helm_destroy(helm_ctx* ctx) {
  if (!ctx) return HELM_OK;
  for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
  clear_graphs(ctx);
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  for (void* q : ctx->allocs) cudaFree(q);
  if (ctx->hflags) cudaFreeHost(ctx->hflags);
  if (ctx->hidr) cudaFreeHost(ctx->hidr);
  if (ctx->hctl) cudaFreeHost(ctx->hctl);
  if (ctx->hreorth_log) cudaFreeHost(ctx->hreorth_log);
  if (ctx->bw.hany) cudaFreeHost(ctx->bw.hany);
  if (ctx->hbicg) cudaFreeHost(ctx->hbicg);
  for (int i = 0; i < ctx->nev; ++i) cudaEventDestroy(ctx->ev[i]);
  delete ctx;
  return HELM_OK;
}

static helm_status create_impl(helm_ctx* c, int n1, int n2, int n3, double h, const double* k2, int bc,
                               cudaStream_t st) {
  const helm_params& P = c->p;
  c->bc = bc;
  c->s_re = P.beta1;
  c->s_im = -P.beta2;
  // hierarchy (Sec. 4.2): halve while every n_d is even and n_d / 2 >= coarsest_n
  int a = n1, b = n2, d = n3;
  double hl = h;
  int nl = 0;
  for (;;) {
    Level& L = c->L[nl];
    L.n1 = a; L.n2 = b; L.n3 = d;
    L.g.N1 = unknowns(a, bc); L.g.N2 = unknowns(b, bc); L.g.N3 = unknowns(d, bc);
    L.g.bc = bc;
    L.g.h = hl;
    ++nl;
    const bool can = a % 2 == 0 && b % 2 == 0 && d % 2 == 0 && a / 2 >= P.coarsest_n && b / 2 >= P.coarsest_n &&
                     d / 2 >= P.coarsest_n && nl < MAX_LEVELS;
    if (!can) break;
    a /= 2; b /= 2; d /= 2;
    hl *= 2;
  }
  c->nlev = nl;
  const Level& Lc = c->L[nl - 1];
  c->nc = Lc.g.N1 * Lc.g.N2 * Lc.g.N3;
  if ((size_t)Lc.g.N1 * Lc.g.N2 * Lc.g.N3 > (size_t)MAX_COARSE)
    return fail(c, HELM_EINVAL, "coarsest grid has %zu unknowns (limit %d): use interval counts divisible by a "
                "larger power of two or a smaller coarsest_n", (size_t)Lc.g.N1 * Lc.g.N2 * Lc.g.N3, MAX_COARSE);
  for (int l = 0; l < nl; ++l) {
    Level& L = c->L[l];
    const size_t np = L.g.npts();
    TRY(dalloc(c, &L.k2, np));
    TRY(dalloc(c, &L.k2f, np));
    TRY(dalloc(c, &L.sk, np));
    TRY(dalloc(c, &L.skf, np));
    L.g.sqk = L.sk;
    L.g.sqkf = L.skf;
    TRY(dalloc(c, &L.dinv, 2 * np));
    TRY(dalloc(c, &L.U164, np));
    TRY(dalloc(c, &L.T64, np));
    TRY(dalloc(c, &L.U132, np));
    TRY(dalloc(c, &L.T32, np));
    if (l > 0) {
      TRY(dalloc(c, &L.B64, np));
      TRY(dalloc(c, &L.E64, np));
      TRY(dalloc(c, &L.B32, np));
      TRY(dalloc(c, &L.E32, np));
    } else if (P.precision == HELM_PREC_MIXED) {
      TRY(dalloc(c, &L.B32, np));  // the complex64 copy of a complex128 cycle input
    }
  }
  Level& L0 = c->L[0];
  const size_t n0 = L0.g.npts();
  c->n0 = n0;
  CU(cudaMemcpyAsync(L0.k2, k2, n0 * sizeof(double), cudaMemcpyDefault, st));
  int* bad = nullptr;
  TRY(dalloc(c, &bad, 1));
  CU(cudaMemsetAsync(bad, 0, sizeof(int), st));
  launch_check_k2(L0.k2, n0, bad, st);
  int hbad = 0;
  CU(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (hbad) return fail(c, HELM_EINVAL, "k2 has %d non-finite or non-positive entries", hbad);
  for (int l = 1; l < nl; ++l) launch_inject(c->L[l - 1].g, c->L[l].g, c->L[l - 1].k2, c->L[l].k2, st);
  for (int l = 0; l < nl; ++l) {
    Level& L = c->L[l];
    launch_to_float(L.k2, L.k2f, L.g.npts(), st);
    launch_sqrt_table(L.k2, L.sk, L.skf, L.g.npts(), st);
    launch_dinv(L.g, c->s_re, c->s_im, P.omega, L.k2, L.dinv, st);
  }
  TRY(check_launch(c, "set-up kernels"));
  // coarsest: assemble M_L on the host and invert it once
  std::vector<double> k2c(c->nc);
  CU(cudaMemcpyAsync(k2c.data(), c->L[nl - 1].k2, c->nc * sizeof(double), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  std::vector<std::complex<double>> A;
  assemble_coarse(c->L[nl - 1], bc, std::complex<double>(c->s_re, c->s_im), k2c, A);
  {
    // inverted on the device by Gauss-Jordan elimination with partial pivoting
    z128 *Aw = nullptr, *fcol = nullptr, *pinv = nullptr;
    int *piv = nullptr, *sing = nullptr;
    TRY(dalloc(c, &c->Minv, (size_t)c->nc * c->nc));
    TRY(dalloc(c, &Aw, (size_t)c->nc * c->nc));
    TRY(dalloc(c, &fcol, c->nc));
    TRY(dalloc(c, &pinv, 1));
    TRY(dalloc(c, &piv, 1));
    TRY(dalloc(c, &sing, 1));
    CU(cudaMemcpyAsync(Aw, A.data(), A.size() * sizeof(z128), cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(sing, 0, sizeof(int), st));
    launch_gj_invert(Aw, c->Minv, c->nc, fcol, piv, pinv, sing, st);
    int hsing = 0;
    CU(cudaMemcpyAsync(&hsing, sing, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    TRY(check_launch(c, "coarsest-grid inverse"));
    dfree(c, Aw);
    dfree(c, fcol);
    dfree(c, pinv);
    dfree(c, piv);
    dfree(c, sing);
    if (hsing) return fail(c, HELM_ENUMERIC, "coarsest-grid operator is singular");
  }
  if (P.coarse_tol > 0.0) {
    if (c->nc > CG_CS * 512) return fail(c, HELM_EINVAL, "coarse_tol > 0 needs a coarsest grid of at most %d unknowns", CG_CS * 512);
    TRY(dalloc(c, &c->cgV, (size_t)(CG_MAX + 1) * c->nc));
    TRY(dalloc(c, &c->cgH, (size_t)CG_MAX * (CG_MAX + 1)));
    TRY(dalloc(c, &c->cginfo, 2));
    CU(cudaMemsetAsync(c->cginfo, 0, 2 * sizeof(int), st));
  }
  // Krylov workspace
  const int m = P.restart;
  c->m = m;
  // Bi-CGSTAB keeps its eight vectors in the basis storage
  TRY(dalloc(c, &c->V, (size_t)std::max(m + 1, 8) * n0));
  if (P.gs_sums && P.orth == HELM_ORTH_FP64 && (P.krylov == HELM_GMRES || P.krylov == HELM_FGMRES))
    TRY(dalloc(c, &c->Vs, (size_t)(m + 1) * n0));
  if (P.precision == HELM_PREC_MIXED) TRY(dalloc(c, &c->Z32, (size_t)m * n0));
  else if (P.krylov == HELM_FGMRES) TRY(dalloc(c, &c->Z64, (size_t)m * n0));
  TRY(dalloc(c, &c->zs, n0));
  if (P.orth == HELM_ORTH_DF) {
    TRY(dalloc(c, &c->wdf, n0));
    if (P.precision == HELM_PREC_MIXED) TRY(dalloc(c, &c->vcur32, n0));
    else TRY(dalloc(c, &c->vcur64, n0));
  }
  if (P.orth == HELM_ORTH_DF && P.precision == HELM_PREC_MIXED) {
    TRY(dalloc(c, &c->k2df, n0));
    TRY(dalloc(c, &c->skdf, n0));
    launch_k2_df(c->L[0].k2, n0, c->k2df, c->skdf, st);
  }
  TRY(dalloc(c, &c->r, n0));
  TRY(dalloc(c, &c->xs, n0));
  TRY(dalloc(c, &c->bs, n0));
  TRY(dalloc(c, &c->part, (size_t)(m + 2) * RED_STRIDE));
  TRY(dalloc(c, &c->partr, RED_STRIDE));
  TRY(dalloc(c, &c->hpass, MAX_BASIS));
  TRY(dalloc(c, &c->hacc, MAX_BASIS));
  TRY(dalloc(c, &c->H, (size_t)(m + 1) * m));
  TRY(dalloc(c, &c->cs, m));
  TRY(dalloc(c, &c->sn, m));
  TRY(dalloc(c, &c->gv, m + 1));
  TRY(dalloc(c, &c->y, m));
  TRY(dalloc(c, &c->hnorm, 1));
  c->hist_len = P.max_iter;
  TRY(dalloc(c, &c->hist, c->hist_len));
  TRY(dalloc(c, &c->ctl, 1));
  TRY(dalloc(c, &c->bicg, 1));
  CU(cudaMemset(c->bicg, 0, sizeof(BicgCtl)));
  CU(cudaHostAlloc((void**)&c->hbicg, sizeof(BicgCtl), cudaHostAllocDefault));
  TRY(dalloc(c, &c->one, 1));
  const int one = 1;
  CU(cudaMemcpy(c->one, &one, sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemset(c->ctl, 0, sizeof(KrylovCtl)));
  CU(cudaHostAlloc((void**)&c->hflags, sizeof(int) * (m + FLAG_LAG + 1), cudaHostAllocDefault));
  CU(cudaHostAlloc((void**)&c->hctl, sizeof(KrylovCtl), cudaHostAllocDefault));
  CU(cudaHostAlloc((void**)&c->hreorth_log, sizeof(int) * m, cudaHostAllocDefault));
  TRY(dalloc(c, &c->reorth_log, m));
  CU(cudaMemset(c->reorth_log, 0, sizeof(int) * m));
  c->nev = FLAG_LAG + 2;
  for (int i = 0; i < c->nev; ++i) CU(cudaEventCreateWithFlags(&c->ev[i], cudaEventDisableTiming));
  CU(cudaStreamSynchronize(st));
  if (P.autotune) TRY(autotune(c, st));
  if (P.fuse_down >= 0)
    for (int l = 0; l + 1 < nl; ++l) {
      c->L[l].g.fused_down = P.fuse_down == 1 ? 1 : 0;
      c->L[l].g.down_full = P.fuse_down == 2 ? 1 : 0;
      c->L[l].g.rr_full = P.fuse_down == 3 ? 1 : 0;
    }
  if (P.fuse_up >= 0)
    for (int l = 0; l + 1 < nl; ++l) c->L[l].g.up_full = P.fuse_up;
  return HELM_OK;
}

helm_status helm_create(int n1, int n2, int n3, double h, const double* k2, helm_bc bc, const helm_params* p,
                        void* stream, helm_ctx** out) {
  if (!out) return fail(nullptr, HELM_EINVAL, "out is NULL");
  *out = nullptr;
  if (n1 < 2 || n2 < 2 || n3 < 2) return fail(nullptr, HELM_EINVAL, "interval counts must be >= 2 (got %d %d %d)", n1, n2, n3);
  if (!(h > 0.0) || !std::isfinite(h)) return fail(nullptr, HELM_EINVAL, "h must be positive and finite");
  if (bc != HELM_BC_DIRICHLET && bc != HELM_BC_SOMMERFELD) return fail(nullptr, HELM_EINVAL, "unknown boundary condition %d", (int)bc);
  if (!k2) return fail(nullptr, HELM_EINVAL, "k2 is NULL");
  helm_params P;
  if (p) P = *p;
  else helm_default_params(&P);
  if (!(P.omega > 0.0 && P.omega < 2.0)) return fail(nullptr, HELM_EINVAL, "omega must lie in (0, 2)");
  if (P.nu1 != 1 || P.nu2 != 1) return fail(nullptr, HELM_EINVAL, "only nu1 = nu2 = 1 is supported");
  if (P.coarsest_n < 2) return fail(nullptr, HELM_EINVAL, "coarsest_n must be >= 2");
  if (P.restart < 1 || P.restart > MAX_BASIS - 1) return fail(nullptr, HELM_EINVAL, "restart must lie in 1..%d", MAX_BASIS - 1);
  if (!(P.tol > 0.0)) return fail(nullptr, HELM_EINVAL, "tol must be positive");
  if (P.max_iter < 1) return fail(nullptr, HELM_EINVAL, "max_iter must be >= 1");
  if (!(P.idr_kappa >= 0.0 && P.idr_kappa < 1.0)) return fail(nullptr, HELM_EINVAL, "idr_kappa must lie in [0, 1)");
  if (P.side != HELM_SIDE_RIGHT && P.side != HELM_SIDE_LEFT) return fail(nullptr, HELM_EINVAL, "unknown side %d", P.side);
  if (P.side == HELM_SIDE_LEFT &&
      (P.krylov != HELM_GMRES || P.precision != HELM_PREC_FP64 || P.orth != HELM_ORTH_FP64))
    return fail(nullptr, HELM_EINVAL, "left preconditioning needs krylov = HELM_GMRES, FP64 precision and FP64 orth");
  if (P.krylov != HELM_GMRES && P.krylov != HELM_FGMRES && P.krylov != HELM_BICGSTAB && P.krylov != HELM_IDRS)
    return fail(nullptr, HELM_EINVAL, "unknown krylov %d", P.krylov);
  if (P.precision != HELM_PREC_FP64 && P.precision != HELM_PREC_MIXED) return fail(nullptr, HELM_EINVAL, "unknown precision %d", P.precision);
  if (!std::isfinite(P.beta1) || !std::isfinite(P.beta2)) return fail(nullptr, HELM_EINVAL, "beta1, beta2 must be finite");
  if (P.orth != HELM_ORTH_FP64 && P.orth != HELM_ORTH_DF) return fail(nullptr, HELM_EINVAL, "unknown orth %d", P.orth);
  if (P.cycle != HELM_CYCLE_V && P.cycle != HELM_CYCLE_F) return fail(nullptr, HELM_EINVAL, "unknown cycle %d", P.cycle);
  if (P.reorth != HELM_REORTH_ALWAYS && P.reorth != HELM_REORTH_SELECTIVE)
    return fail(nullptr, HELM_EINVAL, "unknown reorth %d", P.reorth);
  if (P.gs_sums != 0 && P.gs_sums != 1) return fail(nullptr, HELM_EINVAL, "gs_sums must be 0 or 1");
  if (P.fuse_down < -1 || P.fuse_down > 3) return fail(nullptr, HELM_EINVAL, "fuse_down must lie in -1..3");
  if (P.fuse_up < -1 || P.fuse_up > 1) return fail(nullptr, HELM_EINVAL, "fuse_up must lie in -1..1");
  if (P.stall_window < 0) return fail(nullptr, HELM_EINVAL, "stall_window must be >= 0");
  if (!(P.reorth_keep >= 0.0 && P.reorth_keep < 1.0)) return fail(nullptr, HELM_EINVAL, "reorth_keep must lie in [0, 1)");
  if (!(P.coarse_tol >= 0.0 && P.coarse_tol < 1.0)) return fail(nullptr, HELM_EINVAL, "coarse_tol must lie in [0, 1)");
  if (P.precision == HELM_PREC_MIXED && P.krylov == HELM_GMRES) P.krylov = HELM_FGMRES;
  helm_ctx* c = new (std::nothrow) helm_ctx();
  if (!c) return fail(nullptr, HELM_ENOMEM, "host allocation failed");
  c->p = P;
  helm_status s = create_impl(c, n1, n2, n3, h, k2, (int)bc, (cudaStream_t)stream);
  if (s != HELM_OK) {
    g_create_error = c->err;
    helm_destroy(c);
    return s;
  }
  *out = c;
  return HELM_OK;
}

helm_status helm_levels(const helm_ctx* ctx, int* nlevels) {
  if (!ctx || !nlevels) return HELM_EINVAL;
  *nlevels = ctx->nlev;
  return HELM_OK;
}

helm_status helm_level_dims(const helm_ctx* ctx, int level, int* dims6, double* h_out) {
  if (!ctx || !dims6 || level < 0 || level >= ctx->nlev) return HELM_EINVAL;
  const Level& L = ctx->L[level];
  dims6[0] = L.n1; dims6[1] = L.n2; dims6[2] = L.n3;
  dims6[3] = L.g.N1; dims6[4] = L.g.N2; dims6[5] = L.g.N3;
  if (h_out) *h_out = L.g.h;
  return HELM_OK;
}

helm_status helm_apply(helm_ctx* c, helm_op op, helm_dtype dt, const void* u, void* v, void* stream) {
  if (!c) return HELM_EINVAL;
  if (!u || !v || u == v) return fail(c, HELM_EINVAL, "u and v must be distinct non-NULL device pointers");
  if (op != HELM_OP_A && op != HELM_OP_M) return fail(c, HELM_EINVAL, "unknown operator %d", (int)op);
  const double sr = op == HELM_OP_A ? 1.0 : c->s_re, si = op == HELM_OP_A ? 0.0 : c->s_im;
  cudaStream_t st = (cudaStream_t)stream;
  Level& L = c->L[0];
  const double n = (double)L.g.npts();
  if (dt == HELM_C128)
    KL(F_APPLY, 40.0 * n, 22.0 * n, (launch_apply<double, double, double>(L.g, sr, si, L.k2, (const z128*)u, (z128*)v, st, nullptr)));
  else if (dt == HELM_C64)
    KL(F_APPLY, 20.0 * n, 22.0 * n, (launch_apply<float, float, float>(L.g, sr, si, L.k2f, (const z64*)u, (z64*)v, st, nullptr)));
  else
    return fail(c, HELM_EINVAL, "unknown dtype %d", (int)dt);
  return check_launch(c, "helm_apply");
}

helm_status cslp_vcycle(helm_ctx* c, helm_dtype dt, const void* r, void* z, void* stream) {
  if (!c) return HELM_EINVAL;
  if (!r || !z || r == z) return fail(c, HELM_EINVAL, "r and z must be distinct non-NULL device pointers");
  cudaStream_t st = (cudaStream_t)stream;
  if (dt == HELM_C128)
    run_vcycle<double, double, double>(c, (const z128*)r, (z128*)z, st, nullptr);
  else if (dt == HELM_C64)
    run_vcycle<float, float, float>(c, (const z64*)r, (z64*)z, st, nullptr);
  else
    return fail(c, HELM_EINVAL, "unknown dtype %d", (int)dt);
  return check_launch(c, "cslp_vcycle");
}

helm_status helm_launch_shapes(const helm_ctx* c, int level, int* ty, int* ctas) {
  if (!c || !ty || !ctas || level < 0 || level >= c->nlev) return HELM_EINVAL;
  for (int q = 0; q < 8; ++q) {
    ty[q] = c->L[level].g.tile_ty[q];
    ctas[q] = c->L[level].g.tile_ctas[q];
  }
  return HELM_OK;
}

helm_status helm_kernel_variants(const helm_ctx* c, int level, int* flags) {
  if (!c || !flags || level < 0 || level >= c->nlev) return HELM_EINVAL;
  const Grid& g = c->L[level].g;
  *flags = (g.tiled ? 1 : 0) | (g.fused_down ? 2 : 0) | (g.down_full ? 4 : 0) | (g.up_full ? 8 : 0) |
           (g.rr_full ? 16 : 0);
  return HELM_OK;
}

helm_status helm_dot_variant(helm_ctx* c, int set, int* variant) {
  if (!c || !variant) return HELM_EINVAL;
  const bool df = c->p.orth == HELM_ORTH_DF;
  int& v = df ? c->mdot_df_variant : c->mdot_variant;
  if (!set) {
    *variant = v;
    return HELM_OK;
  }
  if (*variant < 0 || *variant > (df ? 2 : 1)) return fail(c, HELM_EINVAL, "inner-product variant out of range");
  v = *variant;
  clear_graphs(c);  // captured steps hold the old kernels
  return HELM_OK;
}

helm_status helm_tune_log(const helm_ctx* c, int* rec, float* ms, int cap, int* count) {
  if (!c || !count) return HELM_EINVAL;
  *count = (int)c->tune_log.size();
  for (int i = 0; i < cap && i < *count; ++i) {
    const TuneRec& t = c->tune_log[i];
    if (rec) { rec[4 * i] = t.level; rec[4 * i + 1] = t.slot; rec[4 * i + 2] = t.ty; rec[4 * i + 3] = t.ctas; }
    if (ms) ms[i] = t.ms;
  }
  return HELM_OK;
}

helm_status helm_apply_c64_df(helm_ctx* c, const void* u, void* v, void* stream) {
  if (!c) return HELM_EINVAL;
  if (!u || !v || u == v) return fail(c, HELM_EINVAL, "u and v must be distinct non-NULL device pointers");
  if (!c->k2df) return fail(c, HELM_EINVAL, "the context was created without mixed precision and double-float orth");
  launch_apply_c64_df<z128>(c->L[0].g, c->k2df, c->skdf, (const z64*)u, (z128*)v, (cudaStream_t)stream, nullptr);
  return check_launch(c, "helm_apply_c64_df");
}

helm_status cslp_fcycle(helm_ctx* c, helm_dtype dt, const void* r, void* z, void* stream) {
  if (!c) return HELM_EINVAL;
  if (!r || !z || r == z) return fail(c, HELM_EINVAL, "r and z must be distinct non-NULL device pointers");
  return fcycle_entry(c, dt, r, z, (cudaStream_t)stream);
}

helm_status helm_vcycle_stage(helm_ctx* c, int level, int stage, helm_dtype dt, const void* b, const void* e,
                              void* out, void* stream) {
  if (!c) return HELM_EINVAL;
  if (stage < 0 || stage > 2) return fail(c, HELM_EINVAL, "stage must be 0, 1 or 2");
  if (stage == 2 && level != c->nlev - 1) return fail(c, HELM_EINVAL, "stage 2 runs on the last level only");
  if (stage < 2 && (level < 0 || level >= c->nlev - 1)) return fail(c, HELM_EINVAL, "level out of range");
  if (!b || !out || (stage == 1 && !e)) return fail(c, HELM_EINVAL, "NULL vector");
  cudaStream_t st = (cudaStream_t)stream;
  if (dt == HELM_C128)
    stage_impl<double>(c, level, stage, (const z128*)b, (const z128*)e, (z128*)out, st);
  else if (dt == HELM_C64)
    stage_impl<float>(c, level, stage, (const z64*)b, (const z64*)e, (z64*)out, st);
  else
    return fail(c, HELM_EINVAL, "unknown dtype %d", (int)dt);
  return check_launch(c, "helm_vcycle_stage");
}

helm_status helm_rhs_point(helm_ctx* c, int nsrc, const int* nodes, void* b, void* stream) {
  if (!c) return HELM_EINVAL;
  if (nsrc < 0 || (nsrc > 0 && !nodes) || !b) return fail(c, HELM_EINVAL, "bad source list or b");
  cudaStream_t st = (cudaStream_t)stream;
  const Level& L = c->L[0];
  const int off = c->bc == HELM_BC_DIRICHLET ? 1 : 0;
  std::vector<int> idx(nsrc > 0 ? nsrc : 1, -1);
  for (int s = 0; s < nsrc; ++s) {
    const int i = nodes[3 * s] - off, j = nodes[3 * s + 1] - off, k = nodes[3 * s + 2] - off;
    if (nodes[3 * s] < 0 || nodes[3 * s] > L.n1 || nodes[3 * s + 1] < 0 || nodes[3 * s + 1] > L.n2 ||
        nodes[3 * s + 2] < 0 || nodes[3 * s + 2] > L.n3)
      return fail(c, HELM_EINVAL, "source %d outside the grid", s);
    if (i < 0 || i >= L.g.N1 || j < 0 || j >= L.g.N2 || k < 0 || k >= L.g.N3) continue;
    idx[s] = (int)gidx(i, j, k, L.g.N1, L.g.N2);
  }
  CU(cudaStreamSynchronize(st));
  if (nsrc > c->rhs_cap) {
    TRY(dalloc(c, &c->rhs_idx, nsrc));
    c->rhs_cap = nsrc;
  }
  if (nsrc > 0) CU(cudaMemcpy(c->rhs_idx, idx.data(), nsrc * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemsetAsync(b, 0, c->n0 * sizeof(z128), st));
  if (nsrc > 0) launch_rhs_point(L.g, nsrc, c->rhs_idx, 1.0 / (L.g.h * L.g.h * L.g.h), (z128*)b, st);
  return check_launch(c, "helm_rhs_point");
}

helm_status helm_solve_adjoint(helm_ctx* c, const void* g, void* lambda, helm_solve_info* info, void* stream) {
  if (!c) return HELM_EINVAL;
  if (!g || !lambda || g == lambda) return fail(c, HELM_EINVAL, "g and lambda must be distinct non-NULL device pointers");
  if (!is_device_ptr(g) || !is_device_ptr(lambda)) return fail(c, HELM_EINVAL, "g and lambda must be device pointers");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)stream;
  const Level& F = c->L[0];
  launch_adjoint_rhs(F.g, (const z128*)g, c->bs, st);
  CU(cudaMemsetAsync(lambda, 0, c->n0 * sizeof(z128), st));
  helm_solve_info tmp;
  helm_solve_info* inf = info ? info : &tmp;
  helm_status s = krylov_device(c, c->bs, (z128*)lambda, inf, st);
  launch_adjoint_finish(F.g, (z128*)lambda, st);
  TRY(check_launch(c, "helm_solve_adjoint"));
  CU(cudaStreamSynchronize(st));
  inf->status = (int)s;
  inf->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (s == HELM_ENOCONV) fail(c, s, "adjoint solve: max_iter (%d) reached", c->p.max_iter);
  if (s == HELM_ENUMERIC) fail(c, s, "adjoint solve: non-finite residual or Krylov breakdown");
  return s;
}

helm_status helm_grad_k2(helm_ctx* c, const void* u, const void* lambda, double* grad_k2, void* stream) {
  if (!c) return HELM_EINVAL;
  if (!u || !lambda || !grad_k2) return fail(c, HELM_EINVAL, "NULL pointer");
  const Level& F = c->L[0];
  launch_grad_k2(F.g, F.k2, (const z128*)u, (const z128*)lambda, grad_k2, (cudaStream_t)stream);
  return check_launch(c, "helm_grad_k2");
}

helm_status helm_adjoint_grad(helm_ctx* c, int nsrc, const int* src_nodes, int nrec, const int* rec_idx,
                              const void* d_obs, double* grad_k2, double* loss, helm_solve_info* info, void* stream) {
  if (!c) return HELM_EINVAL;
  if (nsrc < 1 || !src_nodes || nrec < 1 || !rec_idx || !d_obs || !grad_k2 || !loss)
    return fail(c, HELM_EINVAL, "bad source, receiver, data or output arguments");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = c->n0;
  std::vector<int> rec(rec_idx, rec_idx + nrec);
  {
    std::vector<int> sorted(rec);
    std::sort(sorted.begin(), sorted.end());
    if (sorted.front() < 0 || (size_t)sorted.back() >= n)
      return fail(c, HELM_EINVAL, "receiver index outside 0..%zu", n - 1);
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return fail(c, HELM_EINVAL, "receiver indices must be distinct");
  }
  if (!c->adj_u) {
    TRY(dalloc(c, &c->adj_u, n));
    TRY(dalloc(c, &c->adj_g, n));
    TRY(dalloc(c, &c->adj_l, n));
    TRY(dalloc(c, &c->adj_part, 256));
    TRY(dalloc(c, &c->adj_norm, 1));
  }
  if (nrec > c->adj_rec_cap) {
    TRY(dalloc(c, &c->adj_rec, nrec));
    c->adj_rec_cap = nrec;
  }
  CU(cudaStreamSynchronize(st));
  CU(cudaMemcpy(c->adj_rec, rec.data(), sizeof(int) * nrec, cudaMemcpyHostToDevice));
  CU(cudaMemsetAsync(grad_k2, 0, n * sizeof(double), st));
  const Level& F = c->L[0];
  double total = 0.0;
  int iters = 0, restarts = 0;
  helm_status worst = HELM_OK;
  double worst_rr = 0.0;
  const bool batched =
      nsrc > 1 && (c->p.krylov == HELM_GMRES || c->p.krylov == HELM_FGMRES) && c->p.side == HELM_SIDE_RIGHT;
  if (batched) {
    // every source's forward solve in lockstep batches (helm_solve_batched), then every
    // adjoint solve the same way: nsrc wavefields, right-hand sides and adjoint states
    if (nsrc > c->adj_cap) {
      TRY(dalloc(c, &c->adj_U, (size_t)nsrc * n));
      TRY(dalloc(c, &c->adj_G, (size_t)nsrc * n));
      TRY(dalloc(c, &c->adj_L, (size_t)nsrc * n));
      c->adj_cap = nsrc;
    }
    for (int s = 0; s < nsrc; ++s) TRY(helm_rhs_point(c, 1, src_nodes + 3 * s, c->adj_G + (size_t)s * n, st));
    CU(cudaMemsetAsync(c->adj_U, 0, (size_t)nsrc * n * sizeof(z128), st));
    std::vector<helm_solve_info> fi(nsrc), ai(nsrc);
    helm_status fs = solve_batched_core(c, nsrc, c->adj_G, c->adj_U, fi.data(), st, false);
    if (fs == HELM_ENUMERIC || fs == HELM_ECUDA || fs == HELM_ENOMEM) return fs;
    CU(cudaMemsetAsync(c->adj_G, 0, (size_t)nsrc * n * sizeof(z128), st));
    for (int s = 0; s < nsrc; ++s) {
      const int nb = launch_receiver_residual(nrec, c->adj_rec, c->adj_U + (size_t)s * n,
                                              (const z128*)d_obs + (size_t)s * nrec, c->adj_G + (size_t)s * n,
                                              c->adj_part, st);
      launch_reduce_norm(c->adj_part, nb, c->adj_norm, st, nullptr);
      double rn = 0.0;
      CU(cudaMemcpyAsync(&rn, c->adj_norm, sizeof(double), cudaMemcpyDeviceToHost, st));
      CU(cudaStreamSynchronize(st));
      total += 0.5 * rn * rn;
    }
    helm_status as = solve_batched_core(c, nsrc, c->adj_G, c->adj_L, ai.data(), st, true);
    if (as == HELM_ENUMERIC || as == HELM_ECUDA || as == HELM_ENOMEM) return as;
    for (int s = 0; s < nsrc; ++s) {
      launch_grad_k2(F.g, F.k2, c->adj_U + (size_t)s * n, c->adj_L + (size_t)s * n, grad_k2, st);
      iters += fi[s].iterations + ai[s].iterations;
      worst_rr = std::max(worst_rr, std::max(fi[s].rel_residual, ai[s].rel_residual));
    }
    TRY(check_launch(c, "helm_adjoint_grad"));
    if (fs != HELM_OK) worst = fs;
    if (as != HELM_OK) worst = as;
  }
  for (int s = 0; s < nsrc && !batched; ++s) {
    TRY(helm_rhs_point(c, 1, src_nodes + 3 * s, c->bs, st));
    CU(cudaMemsetAsync(c->adj_u, 0, n * sizeof(z128), st));
    helm_solve_info fi;
    helm_status fs = krylov_device(c, c->bs, c->adj_u, &fi, st);
    if (fs == HELM_ENUMERIC || fs == HELM_ECUDA || fs == HELM_ENOMEM) return fs;
    CU(cudaMemsetAsync(c->adj_g, 0, n * sizeof(z128), st));
    const int nb = launch_receiver_residual(nrec, c->adj_rec, c->adj_u, (const z128*)d_obs + (size_t)s * nrec, c->adj_g,
                                            c->adj_part, st);
    launch_reduce_norm(c->adj_part, nb, c->adj_norm, st, nullptr);
    double rn = 0.0;
    CU(cudaMemcpyAsync(&rn, c->adj_norm, sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    total += 0.5 * rn * rn;
    launch_adjoint_rhs(F.g, c->adj_g, c->bs, st);
    CU(cudaMemsetAsync(c->adj_l, 0, n * sizeof(z128), st));
    helm_solve_info ai;
    helm_status as = krylov_device(c, c->bs, c->adj_l, &ai, st);
    if (as == HELM_ENUMERIC || as == HELM_ECUDA || as == HELM_ENOMEM) return as;
    launch_adjoint_finish(F.g, c->adj_l, st);
    launch_grad_k2(F.g, F.k2, c->adj_u, c->adj_l, grad_k2, st);
    TRY(check_launch(c, "helm_adjoint_grad"));
    iters += fi.iterations + ai.iterations;
    restarts += fi.restarts + ai.restarts;
    if (fs != HELM_OK) worst = fs;
    if (as != HELM_OK) worst = as;
    worst_rr = std::max(worst_rr, std::max(fi.rel_residual, ai.rel_residual));
  }
  CU(cudaStreamSynchronize(st));
  *loss = total;
  if (info) {
    info->iterations = iters;
    info->restarts = restarts;
    info->rel_residual = worst_rr;
    info->status = (int)worst;
    info->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  if (worst == HELM_ENOCONV) fail(c, worst, "a forward or adjoint solve reached max_iter");
  return worst;
}


helm_status helm_solve_batched(helm_ctx* c, int nrhs, const void* B, void* X, helm_solve_info* infos, void* stream) {
  if (!c) return HELM_EINVAL;
  if (nrhs < 1 || !B || !X || B == X) return fail(c, HELM_EINVAL, "bad nrhs or NULL / aliased B, X");
  if (!is_device_ptr(B) || !is_device_ptr(X)) return fail(c, HELM_EINVAL, "B and X must be device pointers");
  return solve_batched_core(c, nrhs, (const z128*)B, (z128*)X, infos, (cudaStream_t)stream, false);
}

helm_status helm_solve_adjoint_batched(helm_ctx* c, int nrhs, const void* G, void* Lambda, helm_solve_info* infos,
                                       void* stream) {
  if (!c) return HELM_EINVAL;
  if (nrhs < 1 || !G || !Lambda || G == Lambda) return fail(c, HELM_EINVAL, "bad nrhs or NULL / aliased G, Lambda");
  if (!is_device_ptr(G) || !is_device_ptr(Lambda)) return fail(c, HELM_EINVAL, "G and Lambda must be device pointers");
  return solve_batched_core(c, nrhs, (const z128*)G, (z128*)Lambda, infos, (cudaStream_t)stream, true);
}

helm_status helm_set_shadow_space(helm_ctx* c, int s, const void* P, void* stream) {
  if (!c) return HELM_EINVAL;
  if (s < 1 || s > IDR_SMAX) return fail(c, HELM_EINVAL, "IDR(s): s = %d outside 1..%d", s, IDR_SMAX);
  if (!P) return fail(c, HELM_EINVAL, "P is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = c->n0;
  CU(cudaStreamSynchronize(st));
  clear_graphs(c);  // captured IDR steps depend on s and on the workspace addresses
  if (s > c->idr_s) {
    CU(cudaStreamSynchronize(st));
    dfree(c, c->idrP);
    dfree(c, c->idrW);
    c->idrP = c->idrW = nullptr;
    c->idr_s = 0;
    TRY(dalloc(c, &c->idrP, (size_t)s * n));
    TRY(dalloc(c, &c->idrW, (2 * (size_t)s + 4) * n));
  }
  if (!c->idr) {
    TRY(dalloc(c, &c->idr_part, (size_t)(IDR_SMAX + 1) * RED_STRIDE));
    TRY(dalloc(c, &c->idr, 1));
    CU(cudaHostAlloc((void**)&c->hidr, sizeof(IdrCtl), cudaHostAllocDefault));
  }
  CU(cudaMemcpyAsync(c->idrP, P, (size_t)s * n * sizeof(z128), cudaMemcpyDefault, st));
  CU(cudaStreamSynchronize(st));
  c->idr_s = s;
  return HELM_OK;
}

helm_status helm_solve(helm_ctx* c, const void* b, void* x, helm_solve_info* info, void* stream) {
  return solve_entry(c, b, x, info, stream, false);
}

helm_status helm_solve_zero(helm_ctx* c, const void* b, void* x, helm_solve_info* info, void* stream) {
  return solve_entry(c, b, x, info, stream, true);
}

helm_status helm_coarse_info(helm_ctx* c, int* steps, int* converged) {
  if (!c || !steps || !converged) return HELM_EINVAL;
  if (!c->cginfo) return fail(c, HELM_EINVAL, "the context solves the coarsest grid exactly (coarse_tol = 0)");
  int h[2] = {0, 0};
  // the last solve may have run on any stream: wait for the device, then read
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(h, c->cginfo, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(c, HELM_ECUDA, "helm_coarse_info: %s", cudaGetErrorString(cudaGetLastError()));
  *steps = h[0];
  *converged = h[1];
  return HELM_OK;
}

}  // extern "C"
