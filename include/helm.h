/*
 * helm.h -- C ABI of libhelm, a single-GPU (sm_103a) matrix-free solver for the 3D
 * heterogeneous Helmholtz equation, preconditioned by the Complex Shifted Laplace
 * Preconditioner (CSLP) and one geometric-multigrid V-cycle.
 *
 * Method: Chen, Dwarka & Vuik, "A matrix-free parallel solution method for the
 * three-dimensional heterogeneous Helmholtz equation" (arXiv 2308.06085).
 *
 * Problem (Sec. 2): -Lap u - k(x)^2 u = b on a box of n1 x n2 x n3 intervals of equal
 * spacing h, with either homogeneous Dirichlet values or the first-order Sommerfeld
 * condition du/dn - i k u = 0 on every face.
 *
 * Grid and vector layout (shared by every entry point):
 *   - Unknowns per direction: N_d = n_d - 1 (Dirichlet, interior nodes 1..n_d-1) or
 *     N_d = n_d + 1 (Sommerfeld, all nodes 0..n_d; the boundary nodes are unknowns
 *     after ghost-point elimination, Sec. 2.4 Eq. elimination).
 *   - A grid vector holds N1*N2*N3 values, x fastest: index (i3*N2 + i2)*N1 + i1.
 *   - Complex values are interleaved (re, im): HELM_C128 = 2 doubles (16 bytes),
 *     HELM_C64 = 2 floats (8 bytes).
 *   - Vector pointers are DEVICE pointers owned by the caller unless an entry point says
 *     otherwise.  They must be 16-byte (c128) / 8-byte (c64) aligned and may not alias
 *     each other unless stated.
 *
 * Streams: every call is ordered on the CUDA stream passed as `stream` (a cudaStream_t;
 * NULL = the legacy default stream).  Calls return once the work is enqueued, except where
 * stated (helm_solve and helm_solve_batched wait for the solve to finish).
 *
 * Errors: every entry point returns a helm_status; no C++ exception crosses the ABI.
 * helm_last_error() gives a message for the last failing call on a context.  A context is
 * not thread-safe: use one context per host thread.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>

#if defined(__GNUC__)
#define HELM_API __attribute__((visibility("default")))
#else
#define HELM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct helm_ctx helm_ctx;

typedef enum {
  HELM_OK = 0,
  HELM_EINVAL = 1,   /* bad argument: sizes, pointers, enum values, unsupported option */
  HELM_ENOMEM = 2,   /* device or host allocation failed */
  HELM_ECUDA = 3,    /* a CUDA runtime call failed (message in helm_last_error) */
  HELM_ENOCONV = 4,  /* max_iter reached, or Bi-CGSTAB stagnated (stall_window), before tol; x holds
                        the last iterate */
  HELM_ETIMEOUT = 5, /* reserved: a bounded device wait gave up */
  HELM_ENUMERIC = 6  /* NaN/Inf residual or Krylov breakdown; x holds the last finite iterate */
} helm_status;

typedef enum { HELM_BC_DIRICHLET = 0, HELM_BC_SOMMERFELD = 1 } helm_bc;
typedef enum { HELM_C128 = 0, HELM_C64 = 1 } helm_dtype;
typedef enum { HELM_OP_A = 0, HELM_OP_M = 1 } helm_op;
typedef enum { HELM_GMRES = 0, HELM_FGMRES = 1, HELM_BICGSTAB = 2, HELM_IDRS = 3 } helm_krylov;
typedef enum { HELM_PREC_FP64 = 0, HELM_PREC_MIXED = 1 } helm_precision;
typedef enum { HELM_ORTH_FP64 = 0, HELM_ORTH_DF = 1 } helm_orth;
typedef enum { HELM_REORTH_ALWAYS = 0, HELM_REORTH_SELECTIVE = 1 } helm_reorth;
typedef enum { HELM_CYCLE_V = 0, HELM_CYCLE_F = 1 } helm_cycle;
typedef enum { HELM_SIDE_RIGHT = 0, HELM_SIDE_LEFT = 1 } helm_side;

/* Solver parameters (Sec. 3.3-3.4 and Sec. 5).  helm_default_params fills the paper's
 * values: beta1 = 1, beta2 = -0.5 (M = -Lap - (beta1 - beta2 i) k^2, Sec. 3.3 Eq.
 * preconditioner), omega = 0.8 (Sec. 3.4.1), one pre- and one post-smoothing sweep
 * (Sec. 3.4.5), coarsest_n = 4, GMRES(30), tol = 1e-6 on the true relative residual,
 * max_iter = 2000, FP64 precision. */
typedef struct {
  double beta1;     /* real part of the CSLP shift multiplier */
  double beta2;     /* CSLP complex shift; the shift is (beta1 - beta2 i) */
  double omega;     /* damped-Jacobi relaxation, 0 < omega < 2 */
  int nu1, nu2;     /* pre/post smoothing sweeps; the library supports nu1 = nu2 = 1 */
  int coarsest_n;   /* >= 2; coarsen while every n_d is even and n_d/2 >= coarsest_n;
                       the coarsest grid may hold at most 4096 unknowns */
  int krylov;       /* helm_krylov: right-preconditioned GMRES(m), flexible GMRES(m),
                       right-preconditioned Bi-CGSTAB, or right-preconditioned IDR(s) in its
                       biorthogonal form (Sec. 3.1; the paper's solver for its wedge and salt
                       runs, as IDR(4)).  Bi-CGSTAB and IDR(s) ignore restart; IDR(s) needs a
                       shadow space from helm_set_shadow_space before helm_solve. */
  int restart;      /* m, Krylov vectors per restart cycle, 1..256 */
  double tol;       /* stop when ||b - A x|| / ||b|| <= tol */
  int max_iter;     /* cap on products with A in the Arnoldi process (#Matvec) */
  int precision;    /* helm_precision: HELM_PREC_MIXED runs the V-cycle in complex64
                       under an FP64 outer Krylov (turns HELM_GMRES into HELM_FGMRES; Bi-CGSTAB
                       and IDR(s) keep M^{-1} p as a vector of their own, so they run as they
                       are) */
  int orth;         /* helm_orth: arithmetic of the Gram-Schmidt inner products and updates.
                       HELM_ORTH_FP64: native FP64.  HELM_ORTH_DF: the Krylov basis is held
                       as pairs of FP32 values (hi + lo, about 48 significant bits) and the
                       products and sums use error-free FP32 transformations; vectors
                       outside the basis, norms and the Hessenberg problem stay FP64. */
  int reorth;       /* helm_reorth: classical Gram-Schmidt with a second pass on every Arnoldi
                       step (ALWAYS), or only when the first pass removed more than
                       1 - reorth_keep of |w|^2 (SELECTIVE, the Daniel-Gragg-Kaufman-Stewart
                       test) */
  int cycle;        /* helm_cycle: the preconditioner is one V-cycle (default) or one F-cycle
                       (Sec. 3.4.5: each coarse-grid error is an F-cycle on the next level followed
                       by one V-cycle there); the batched solver follows it too */
  double idr_kappa; /* IDR(s) dimension-reduction step: omega minimises |r - omega A M^{-1} r|
                       and is enlarged so that the cosine of the angle between r and
                       A M^{-1} r is at least idr_kappa when it is smaller; 0 keeps the
                       minimal-residual omega.  Default 0.7, in [0, 1). */
  int graphs;       /* 1 (default): each solver step (an Arnoldi column of a full-length GMRES
                       cycle, single or batched, a Bi-CGSTAB step, an IDR(s) step) is captured
                       once into a CUDA graph and replayed, one launch instead of 30-70;
                       0: plain launches.  Graphs are bypassed while helm_profile is on.  Steps
                       that write x are keyed by the x pointer, so a solve into a new buffer
                       captures its steps again. */
  int autotune;     /* 1 (default): helm_create times every stencil, smoothing and transfer
                       kernel of every level over launch shapes (rows of x-lines per CTA x CTA
                       count) and keeps the fastest, and helm_solve_batched does the same for
                       its width on first use, and picks the Gram-Schmidt inner-product
                       kernel variant and the FP32 kernel forms (see fuse_down, fuse_up); 0:
                       the fixed default shape and forms.  Results do not depend on any of these
                       choices (the grid kernels have no reductions; the inner-product variants
                       share one grid). */
  int side;         /* helm_side: right preconditioning (default; every solver), or the paper's
                       left-preconditioned GMRES (Sec. 3.2) with its stopping rule
                       ||M^{-1}(b - A x)|| / ||M^{-1} b|| <= tol (Sec. 5), for which
                       helm_solve_info.rel_residual reports that preconditioned quantity.  Left
                       needs krylov = HELM_GMRES with FP64 precision and FP64 orth. */
  int fuse_coarse;  /* 1: the coarse levels of every V-cycle whose vectors fit in one CTA's
                       shared memory (about 200 KB; from 17^3 nodes down in complex64, 9^3 in
                       complex128) run as one single-CTA kernel instead of five kernels per
                       level, with the same arithmetic per point (bit-identical results).
                       0 (default): level by level, which measures faster on GB300 (one SM
                       cannot hide the latency of the coarse-grid product and coefficient
                       loads that many small grids spread over all SMs). */
  int gs_sums;      /* FP64 Gram-Schmidt of GMRES / FGMRES (orth = HELM_ORTH_FP64).  1 (default):
                       every basis vector is stored together with its element sums
                       Re v + Im v (8 more bytes per unknown and vector), so that the inner
                       products conj(v) w and the updates w -= h v take three FP64 FMAs per
                       complex multiply-add instead of four (the three-multiplication form of
                       a complex product); 0: the textbook four-FMA form.  The results differ
                       only by rounding. */
  int fuse_down;    /* down-sweep of the multigrid cycle (one right-hand side), per level:
                       -1 (default): the autotuner's choice (separate kernels when autotune is
                       0); 0: pre-smoothing, residual and restriction as three kernels; 1
                       (complex64 only): pre-smoothing and residual as one kernel, then the
                       restriction; 2 (complex64 only): all three as one kernel; 3
                       (complex64 and complex128): the pre-smoothing, then the residual and its
                       restriction as one kernel (the residual stays in shared memory).  The
                       arithmetic per point is the same in every form (bit-identical results). */
  int fuse_up;      /* up-sweep of the multigrid cycle (one right-hand side; complex64 and
                       complex128), per level: -1 (default): the autotuner's choice (separate
                       kernels when autotune is 0); 0: prolongation + correction, then
                       post-smoothing, as two kernels; 1: one kernel (the corrected iterate
                       stays in shared memory).  Bit-identical results either way. */
  int stall_window; /* Bi-CGSTAB only, >= 0: stop with HELM_ENOCONV (message in helm_last_error)
                       when the recursive residual has not fallen below half of its last mark
                       within this many products with A, or when three restarts from the
                       explicit residual in a row do not halve it.  0: never (run to max_iter).
                       Default 1000.  With precision = HELM_PREC_MIXED the complex64 cycle is a
                       preconditioner that changes with its input's rounding, which Bi-CGSTAB's
                       recurrences do not allow for; it can stagnate there (FGMRES and IDR(s)
                       converge). */
  double reorth_keep; /* GMRES / FGMRES with reorth = HELM_REORTH_SELECTIVE, 0 <= keep < 1: the
                       second classical Gram-Schmidt pass of an Arnoldi step is skipped when the
                       first pass kept at least this fraction of |w|^2 (|w - V h|^2 estimated
                       as |w|^2 - |h|^2): the Daniel-Gragg-Kaufman-Stewart test with
                       eta = sqrt(keep).  One pass leaves the new basis vector orthogonal to the
                       others to about eps / eta, so the second pass matters only under heavy
                       cancellation.  Default 0.1 (eta = 0.32: orthogonality to about 3 eps);
                       0.5 is the conservative eta = 1/sqrt(2). */
  double coarse_tol; /* coarsest-grid solve of every cycle.  0 (default): the dense inverse of
                       M on the coarsest grid, computed once at helm_create (exact to
                       rounding).  0 < tol < 1: the paper's own choice (Sec. 5), full GMRES on
                       the coarsest grid from a zero guess until its relative residual is
                       <= tol (the paper uses 1e-11), at most 256 steps, run by one
                       thread-block cluster of 16 CTAs (8 where the GPU cannot place 16); one
                       right-hand side at a time (the batched solver
                       keeps the dense inverse).  Needs a coarsest grid of at most 4096 unknowns
                       and (257 x that count + 65792) x 16 bytes of device memory. */
} helm_params;

/* Per-solve report (host struct). */
typedef struct {
  int iterations;      /* products with A in the Arnoldi process (#Matvec, Sec. 5) */
  int restarts;        /* restart cycles run */
  int status;          /* helm_status of the solve */
  double rel_residual; /* explicit ||b - A x|| / ||b|| at return */
  double ms_total;     /* wall time of the call, host clock */
} helm_solve_info;

/* Fill *p with the defaults listed above. */
HELM_API void helm_default_params(helm_params* p);

/* Create a context: the multigrid hierarchy (Sec. 4.2; coarse grids re-discretise M with
 * H = 2h, k^2 by injection, Sec. 3.4.4), the exact FP64 inverse of the coarsest M (the
 * paper solves it by GMRES to 1e-11, Sec. 5), and Krylov workspaces.
 *   n1, n2, n3 : intervals per direction, each >= 2
 *   h          : grid spacing, > 0
 *   k2         : k(x)^2 at the N1*N2*N3 unknown nodes (layout above), FP64, > 0 and
 *                finite; a device or host pointer, copied (the caller keeps ownership)
 *   bc         : boundary condition on all faces
 *   p          : parameters, NULL for defaults; copied
 *   stream     : stream for the set-up work; the call waits for it to finish
 *   out        : receives the context; *out is NULL on failure
 * Errors: HELM_EINVAL (sizes, h, k2 values, parameters), HELM_ENOMEM, HELM_ECUDA. */
HELM_API helm_status helm_create(int n1, int n2, int n3, double h, const double* k2, helm_bc bc,
                        const helm_params* p, void* stream, helm_ctx** out);

/* Release every device and host resource of the context (NULL is accepted). */
HELM_API helm_status helm_destroy(helm_ctx* ctx);

/* Number of multigrid levels, and the interval counts and unknown counts of one level
 * (level 0 = finest).  dims6 receives n1, n2, n3, N1, N2, N3; h_out the level's spacing. */
HELM_API helm_status helm_levels(const helm_ctx* ctx, int* nlevels);
HELM_API helm_status helm_level_dims(const helm_ctx* ctx, int level, int* dims6, double* h_out);

/* Matrix-free operator product on the finest grid (Sec. 3.5, Algorithm 2):
 *   HELM_OP_A : v = A_h u = (-Lap_h - k^2) u
 *   HELM_OP_M : v = M_h u = (-Lap_h - (beta1 - beta2 i) k^2) u
 * with the Sommerfeld ghost value u_ghost = u_opposite + 2 h i k u_p substituted on every
 * boundary face a node lies on.  u and v are device vectors of type dt; u != v. */
HELM_API helm_status helm_apply(helm_ctx* ctx, helm_op op, helm_dtype dt, const void* u, void* v,
                       void* stream);

/* One multigrid V-cycle z ~= M_h^{-1} r (Algorithm 1 applied recursively, Sec. 3.4.5):
 * zero initial guess on each level, one damped-Jacobi sweep before and after each coarse
 * correction, full-weighting restriction (Sec. 3.4.2), trilinear interpolation
 * (Sec. 3.4.3), exact FP64 solve on the coarsest level.  dt = HELM_C128 runs every level
 * in FP64; HELM_C64 runs them in FP32 (the coarsest solve stays FP64).  r, z: device. */
HELM_API helm_status cslp_vcycle(helm_ctx* ctx, helm_dtype dt, const void* r, void* z, void* stream);

/* Launch shapes in use on `level` (library instrumentation, no paper counterpart): for each of
 * the 8 slots (kernel family stencil / pre-smoothing / restriction / prolongation, FP64 then
 * FP32) the rows of x-lines per CTA (ty) and the CTA count the z-chunking aims at (ctas); 0 means
 * the default shape (8 rows, 8 CTAs per SM).  ty and ctas: host arrays of 8. */
HELM_API helm_status helm_launch_shapes(const helm_ctx* ctx, int level, int* ty, int* ctas);

/* Kernel variants in use on `level` (library instrumentation; the autotuner's picks, or
 * helm_params.fuse_down): *flags bit 0 = FP32 7-point kernels with shared-memory tiles, bit 1 =
 * FP32 pre-smoothing and residual fused into one kernel, bit 2 = the whole FP32 down-sweep
 * (pre-smoothing, residual, restriction) as one kernel, bit 3 = the whole up-sweep
 * (prolongation, correction, post-smoothing) as one kernel, bit 4 = the residual and its
 * restriction as one kernel.  All change the schedule only, not the arithmetic of a point. */
HELM_API helm_status helm_kernel_variants(const helm_ctx* ctx, int level, int* flags);

/* The variant of helm_solve's Gram-Schmidt inner-product kernel (one right-hand side; library
 * instrumentation): with set = 0,
 * *variant receives the one in use; with set = 1 it replaces it (the autotuner's choice) for the
 * context's arithmetic (helm_params.orth).  FP64: 0 = w staged in shared memory, 1 = each warp
 * reads w itself.  Double-float: 0, 1, 2 = 4, 2, 8 basis vectors per warp pass.  The variants of
 * one arithmetic share one grid and sum each inner product over the same points in the same
 * order, so the results are identical; only the speed differs.  HELM_EINVAL outside 0..1 (FP64)
 * or 0..2 (double-float). */
HELM_API helm_status helm_dot_variant(helm_ctx* ctx, int set, int* variant);

/* The autotuner's measurements (library instrumentation): *count = number of timed shapes; the
 * first min(cap, count) are written as rec[4 i .. 4 i + 3] = (level, slot, ty, ctas) and ms[i] =
 * the best of three timings of three back-to-back launches, per launch.  rec / ms may be NULL. */
HELM_API helm_status helm_tune_log(const helm_ctx* ctx, int* rec, float* ms, int cap, int* count);

/* v = A_h u (Sec. 2.4, Algorithm 2) for a complex64 u, computed in double-float arithmetic
 * (pairs of FP32 values, about 48 significant bits; FP32 instructions only): the A-product of the
 * mixed-precision solver with double-float Gram-Schmidt, exposed for parity checks.  The float
 * inputs are exact, so v is A u to FP64-class accuracy (2^-46 relative to the largest term).
 *   u : device c64 grid vector;  v : device c128 grid vector (output)
 * The context must have precision = HELM_PREC_MIXED and orth = HELM_ORTH_DF (it holds the
 * double-float k^2 table); HELM_EINVAL otherwise.  Stream-ordered. */
HELM_API helm_status helm_apply_c64_df(helm_ctx* ctx, const void* u, void* v, void* stream);

/* One multigrid F-cycle z ~= M_h^{-1} r (Sec. 3.4.5): like the V-cycle, but the coarse-grid
 * error of every level comes from an F-cycle on the next level followed by one V-cycle there,
 * started from that result.  Works on any context, whatever its `cycle` field (which only
 * chooses the preconditioner of helm_solve); uses the same work vectors as the V-cycle, so
 * the same stream rules apply.  dt, r, z as cslp_vcycle. */
HELM_API helm_status cslp_fcycle(helm_ctx* ctx, helm_dtype dt, const void* r, void* z, void* stream);

/* One stage of the V-cycle on level `level`, for stage-by-stage checks:
 *   stage 0 (down): out = R_l (b - M_l u1), u1 = omega D_l^{-1} b; out is on level l+1
 *   stage 1 (up)  : out = S_l(u1 + P_l e), u1 as above, e on level l+1, out on level l
 *   stage 2 (coarsest): out = M_L^{-1} b on the last level (level must be nlevels-1)
 * b, e, out: device vectors of type dt on the levels stated. */
HELM_API helm_status helm_vcycle_stage(helm_ctx* ctx, int level, int stage, helm_dtype dt,
                              const void* b, const void* e, void* out, void* stream);

/* Right-hand side of point sources (Sec. 2.4, discrete Dirac): b = 0, then 1/h^3 added at
 * each source node.  nodes: HOST array of 3*nsrc ints, node coordinates (i1, i2, i3) with
 * 0 <= i_d <= n_d; a node that is not an unknown (Dirichlet boundary) is skipped.
 * b: device c128 vector. */
HELM_API helm_status helm_rhs_point(helm_ctx* ctx, int nsrc, const int* nodes, void* b, void* stream);

/* Solve A_h x = b to ||b - A x|| / ||b|| <= tol by right-preconditioned GMRES(m)
 * (or FGMRES(m)) with one CSLP V-cycle as the preconditioner (Sec. 3.1-3.3).
 *   b    : c128 right-hand side
 *   x    : c128; on entry the initial guess, on exit the solution (a warm start resumes
 *          an earlier solve)
 *   b and x may both be device pointers, or both host pointers (pageable or pinned); host
 *   buffers are copied through the context's device buffers on `stream`.
 *   info : optional host struct, filled on return
 * Waits for the solve.  Returns HELM_OK, HELM_ENOCONV (max_iter hit, or Bi-CGSTAB stagnated;
 * x is the last iterate; helm_last_error(ctx) says which) or HELM_ENUMERIC (breakdown to
 * NaN/Inf). */
HELM_API helm_status helm_solve(helm_ctx* ctx, const void* b, void* x, helm_solve_info* info,
                       void* stream);

/* helm_solve from the initial guess x = 0 (Sec. 3.2 starts GMRES from a given x_0; the
 * paper's experiments start from zero).  x is output only: it is not read, and with host
 * buffers only b is copied to the device before the solve.  Same arguments, waiting and
 * return values as helm_solve. */
HELM_API helm_status helm_solve_zero(helm_ctx* ctx, const void* b, void* x, helm_solve_info* info,
                                     void* stream);

/* Report of the last coarsest-grid GMRES of a context created with coarse_tol > 0 (Sec. 5):
 * *steps = GMRES steps it took, *converged = 1 when it met coarse_tol (0 when it stopped at
 * 256 steps or on a breakdown).  Waits for the device.  HELM_EINVAL for a context that solves
 * the coarsest grid with the dense inverse. */
HELM_API helm_status helm_coarse_info(helm_ctx* ctx, int* steps, int* converged);

/* Shadow space of IDR(s): s (1..8) device c128 grid vectors P_0 .. P_{s-1}, consecutive, one
 * grid vector each (the layout of helm_solve's b).  IDR(s) builds its residuals orthogonal to
 * span(P) step by step (Sec. 3.1); the paper draws P at random, and the caller passes those
 * random vectors in.  Copied into the context (device-to-device on `stream`; the call waits),
 * so P may be freed afterwards; allocates 3 s + 4 grid vectors of context memory.  Calling
 * it again replaces the space.  HELM_EINVAL for s out of range or a NULL P. */
HELM_API helm_status helm_set_shadow_space(helm_ctx* ctx, int s, const void* P, void* stream);

/* Solve A_h X_r = B_r for nrhs right-hand sides together (the batched form of the solve; the
 * paper solves one source at a time).  The right-hand sides run through the same
 * preconditioned flexible GMRES(m) in lockstep, in chunks of up to 32: grid vectors are
 * stored node-major with the right-hand side innermost, so every stencil, transfer and
 * V-cycle kernel reads k^2 once per node for the whole chunk and each warp loads one
 * contiguous row of right-hand sides.  Each right-hand side keeps its own Hessenberg matrix,
 * rotations and stopping test; a converged one is carried along unchanged.  The V-cycle
 * runs in the context's precision (complex64 for HELM_PREC_MIXED, FP64 otherwise); the outer
 * Krylov and residuals are FP64 and the Gram-Schmidt arithmetic follows the context's orth.
 *   B, X : device c128, nrhs consecutive grid vectors (X: initial guesses in, solutions out)
 *   infos: optional host array of nrhs reports
 * Waits for completion.  HELM_ENOCONV if any right-hand side missed tol within max_iter. */
HELM_API helm_status helm_solve_batched(helm_ctx* ctx, int nrhs, const void* B, void* X, helm_solve_info* infos,
                                        void* stream);

/* Adjoint solve for frequency-domain gradients (the paper solves forward problems only;
 * the operator and boundary scheme are its Sec. 2.4).  Solves A^H lambda = g, where A^H is the
 * conjugate transpose of A_h, with the same preconditioned Krylov method as helm_solve: the
 * rows eliminated at Sommerfeld faces make D A symmetric for D = diag(2^-faces) (D = I for
 * Dirichlet), so A^T = D A D^-1 and the library solves A nu = D^-1 conj(g), lambda = conj(D nu).
 *   g, lambda : device c128 vectors (lambda is overwritten; the solve starts from zero)
 *   info      : optional host report of the inner forward-type solve
 * Waits for the solve.  Errors as helm_solve. */
HELM_API helm_status helm_solve_adjoint(helm_ctx* ctx, const void* g, void* lambda, helm_solve_info* info,
                                        void* stream);

/* The adjoint solve of helm_solve_adjoint for nrhs right-hand sides at once, through the
 * lockstep batched solver of helm_solve_batched (the D-scaling and conjugation are applied in
 * its node-major batched layout).
 *   G, Lambda : device c128, nrhs consecutive grid vectors (Lambda overwritten; zero start)
 *   infos     : optional host array of nrhs reports
 * Waits for completion.  Errors as helm_solve_batched. */
HELM_API helm_status helm_solve_adjoint_batched(helm_ctx* ctx, int nrhs, const void* G, void* Lambda,
                                                helm_solve_info* infos, void* stream);

/* Accumulate the adjoint-state gradient with respect to k^2 at every node:
 *   grad_k2[p] += -Re( conj(lambda_p) * dA_pp/dk^2_p * u_p ),  dA_pp/dk^2_p = -1 - i nf_p / (h k_p)
 * (nf_p = Sommerfeld faces at p).  u: the forward solution, lambda: the adjoint solution for
 * g = dL/d conj(u) of a real loss L; the sum over sources is the gradient of L.
 * u, lambda: device c128; grad_k2: device FP64, N1*N2*N3 values, accumulated into. */
HELM_API helm_status helm_grad_k2(helm_ctx* ctx, const void* u, const void* lambda, double* grad_k2, void* stream);

/* Full-waveform-style gradient for point sources and a receiver set:
 *   L = 1/2 sum_s sum_{r in R} |u_s(r) - d_obs[s][r]|^2,  A u_s = b_s (discrete Dirac, Sec. 2.4),
 *   grad_k2 = dL/dk^2 (one forward and one adjoint solve per source, helm_grad_k2 summed).
 *   src_nodes : HOST, 3*nsrc node coordinates (as helm_rhs_point)
 *   rec_idx   : HOST, nrec distinct unknown indices (layout index (i3*N2 + i2)*N1 + i1)
 *   d_obs     : device c128, nsrc x nrec (row per source)
 *   grad_k2   : device FP64, N1*N2*N3, overwritten;  loss : host double
 *   info      : optional host report (iterations summed over all solves, worst residual)
 * With GMRES / FGMRES (right preconditioning) and nsrc > 1 every forward solve runs in
 * helm_solve_batched's lockstep batches, then every adjoint solve the same way, so the
 * context holds nsrc forward wavefields, receiver residuals and adjoint states (3 nsrc grid
 * vectors, allocated on first use); otherwise one source at a time, holding one wavefield.
 * Waits for completion.  HELM_ENOCONV if any solve hit max_iter. */
HELM_API helm_status helm_adjoint_grad(helm_ctx* ctx, int nsrc, const int* src_nodes, int nrec, const int* rec_idx,
                                       const void* d_obs, double* grad_k2, double* loss, helm_solve_info* info,
                                       void* stream);

/* Per-kernel-family statistics of the opt-in profiler. */
typedef struct {
  const char* name;   /* kernel function(s) of the family; static string */
  long long launches; /* timed launches */
  double ms;          /* sum of CUDA-event durations of those launches */
  double bytes;       /* algorithmic bytes moved by those launches (minimum reads + writes) */
  double flops;       /* algorithmic floating-point operations (an FMA counts 2) */
} helm_kernel_stat;

/* Library instrumentation (not part of the paper's method).  enable = 1 brackets every
 * kernel launch of this context with CUDA events on the launching stream and accumulates
 * per-family durations; enable = 0 stops timing.  Either call resets the totals.  Launch
 * counting is always on. */
HELM_API helm_status helm_profile(helm_ctx* ctx, int enable);

/* Read the profiler: up to `cap` families into `stats` (count receives the number of
 * families), and the number of kernel launches this context made since the last reset
 * into *launches (either pointer may be NULL).  Waits for pending timed launches. */
HELM_API helm_status helm_profile_read(helm_ctx* ctx, helm_kernel_stat* stats, int cap, int* count,
                                       long long* launches);

/* Allocation-free variant of the finest-level down stage (helm_vcycle_stage with level 0,
 * stage 0), with no context.  The paper has no counterpart; it exists for callers that may
 * not call cudaMalloc themselves -- code inside a host framework whose memory pool owns
 * every device allocation, or a plug-in allowed to allocate only at start-up -- but still
 * want one multigrid restriction step on their own buffers.
 *
 * Computes out = R (b - M u1), u1 = omega D^{-1} b, on the grid of n1 x n2 x n3 intervals
 * (each even, >= 2) with spacing h, boundary bc and the CSLP shift (beta1 - beta2 i):
 *   k2  : device, FP64, k^2 at the fine unknowns
 *   b   : device, c128, fine unknowns;  out : device, c128, unknowns of the n/2 grid
 * The intermediate u1 and residual live in a static device array of
 * 2 x HELM_NOALLOC_MAX_POINTS complex128 values (8 MiB) that every GPU loading the library
 * holds until exit; grids with more fine unknowns than HELM_NOALLOC_MAX_POINTS are rejected
 * with HELM_EINVAL (message in helm_last_error(NULL)).  Nothing is allocated: no cudaMalloc,
 * no cudaFree, no allocating library call.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before capturing a stream into a graph.
 * Every call on a device shares the one array and overwrites all of its live part, so
 * nothing in it needs to start at zero, but calls that overlap on the GPU (other streams,
 * other threads) race on it: order them.
 * A CUDA error already pending on the calling thread when the call starts is left in place
 * (not cleared) and the call returns HELM_ECUDA without launching anything. */
#define HELM_NOALLOC_MAX_POINTS 262144
HELM_API helm_status helm_vcycle_down_noalloc(int n1, int n2, int n3, double h, const double* k2, helm_bc bc,
                                              double beta1, double beta2, double omega, const void* b, void* out,
                                              void* stream);

/* The FP32 -> FP64 conversion the FP64 kernels use on complex64 data (library instrumentation;
 * the paper has no counterpart).  It is written with integer instructions from the IEEE-754
 * layouts, since a converting instruction issues on this GPU's FP64 pipe, and must give the
 * hardware conversion's bits: out64[i] = (double)in32[i].  Both arrays are device buffers of n
 * elements owned by the caller; stream-ordered.  HELM_EINVAL for a NULL pointer (message in
 * helm_last_error(NULL)). */
HELM_API helm_status helm_convert_check(const float* in32, double* out64, size_t n, void* stream);

/* Message for the last failing call on ctx, or, when ctx is NULL, for the last failing
 * context-free call (helm_create, helm_vcycle_down_noalloc, helm_convert_check) made on the
 * calling host thread: that message is kept per thread, so threads never see or overwrite
 * each other's.  The
 * string is owned by the library and stays valid until the next failing call of the same
 * kind (on ctx, or on this thread). */
HELM_API const char* helm_last_error(const helm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HELM_H */
