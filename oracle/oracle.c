/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the matrix-free CSLP-preconditioned
 * Helmholtz solver of Chen, Dwarka & Vuik (arXiv 2308.06085).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this
 * file; only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code with the CUDA library: every step below is written out directly
 * from the paper's equations, in the paper's order, with plain loops and no fusion.
 *
 * Conventions
 *   - Grid: unit-spaced vertex-centred grid with n_d intervals per direction, h the
 *     spacing (Sec. 2.4).  Unknowns:
 *       Dirichlet  : interior nodes 1..n_d-1   -> N_d = n_d - 1 unknowns, node = idx + 1
 *       Sommerfeld : all nodes 0..n_d           -> N_d = n_d + 1 unknowns, node = idx
 *     (ghost-point elimination, Eq. "elimination", makes boundary nodes unknowns).
 *   - Arrays are x-fastest, u(i1,i2,i3) at [i3*N2*N1 + i2*N1 + i1] (Sec. 4.1 storage).
 *   - Complex vectors are interleaved (re, im) doubles.
 *   - Inner product <v, w> = sum conj(v_i) w_i.
 *
 * Readings of the paper taken here (all listed with reasons in the design notes):
 *   - CSLP shift M = -Lap - (beta1 - beta2 i) k^2, with the paper's beta2 = -0.5 by default.
 *   - Ghost elimination per face, independently at edges/corners, with the real k at the node.
 *   - Coarse grids re-discretise M (DCG), same boundary type, k^2 by injection.
 *   - Transfers: full weighting / trilinear with out-of-domain terms taken as 0.
 *   - Coarsest grid: exact dense LU solve (the paper uses GMRES to 1e-11; an exact solve
 *     makes the V-cycle a fixed linear operator both sides can agree on to rounding).
 *   - Outer Krylov: right-preconditioned GMRES(m) with modified Gram-Schmidt and complex
 *     Givens rotations, x0 given; stop on the Arnoldi residual estimate, then confirm
 *     with the explicit residual ||b - A x|| / ||b||.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { BC_DIRICHLET = 0, BC_SOMMERFELD = 1 };

static size_t npts3(int N1, int N2, int N3) { return (size_t)N1 * N2 * N3; }
static size_t at(int i, int j, int k, int N1, int N2) { return ((size_t)k * N2 + j) * N1 + i; }

/* ---------------------------------------------------------------------------------
 * Stencil coefficients at one node (Sec. 3.5, "Matrix-free method", Algorithm 2).
 * Interior: ap = (6 - s k^2 h^2)/h^2, aw = ae = as = an = ad = au = -1/h^2, where
 * s = 1 for the Helmholtz operator A_h and s = beta1 - beta2 i for the CSLP M_h.
 * At a physical boundary the coefficients are reset:
 *   Dirichlet  -- the neighbour outside the unknown set is a known boundary value
 *                 (homogeneous here; inhomogeneous data is lifted into b), so its
 *                 coefficient is dropped.
 *   Sommerfeld -- the ghost value is eliminated with Eq. (elimination):
 *                 u_ghost = u_opposite + 2 h i k u_p, so the opposite neighbour's
 *                 coefficient gains the ghost's, and ap gains ghost_coef * 2 h i k.
 * --------------------------------------------------------------------------------- */
typedef struct { cplx ap, aw, ae, as, an, ad, au; } coefs;

static coefs node_coefs(int i, int j, int k, int N1, int N2, int N3, double h, int bc,
                        double k2p, cplx s) {
  coefs c;
  double ih2 = 1.0 / (h * h);
  c.ap = (6.0 - s * k2p * h * h) * ih2;
  c.aw = c.ae = c.as = c.an = c.ad = c.au = -ih2;
  if (bc == BC_SOMMERFELD) {
    cplx g = 2.0 * h * I * sqrt(k2p); /* u_ghost = u_opposite + g u_p */
    if (i == 0)      { c.ae += c.aw; c.ap += c.aw * g; c.aw = 0; }
    if (i == N1 - 1) { c.aw += c.ae; c.ap += c.ae * g; c.ae = 0; }
    if (j == 0)      { c.an += c.as; c.ap += c.as * g; c.as = 0; }
    if (j == N2 - 1) { c.as += c.an; c.ap += c.an * g; c.an = 0; }
    if (k == 0)      { c.au += c.ad; c.ap += c.ad * g; c.ad = 0; }
    if (k == N3 - 1) { c.ad += c.au; c.ap += c.au * g; c.au = 0; }
  } else {
    if (i == 0) c.aw = 0;
    if (i == N1 - 1) c.ae = 0;
    if (j == 0) c.as = 0;
    if (j == N2 - 1) c.an = 0;
    if (k == 0) c.ad = 0;
    if (k == N3 - 1) c.au = 0;
  }
  return c;
}

/* v = (-Lap_h - s k^2) u   (Algorithm 2; s = 1 gives A_h, s = beta1 - beta2 i gives M_h) */
static void apply_op(int N1, int N2, int N3, double h, int bc, const double* k2, cplx s,
                     const cplx* u, cplx* v) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < N3; ++k)
    for (int j = 0; j < N2; ++j)
      for (int i = 0; i < N1; ++i) {
        size_t p = at(i, j, k, N1, N2);
        coefs c = node_coefs(i, j, k, N1, N2, N3, h, bc, k2[p], s);
        cplx acc = c.ap * u[p];
        if (i > 0) acc += c.aw * u[at(i - 1, j, k, N1, N2)];
        if (i < N1 - 1) acc += c.ae * u[at(i + 1, j, k, N1, N2)];
        if (j > 0) acc += c.as * u[at(i, j - 1, k, N1, N2)];
        if (j < N2 - 1) acc += c.an * u[at(i, j + 1, k, N1, N2)];
        if (k > 0) acc += c.ad * u[at(i, j, k - 1, N1, N2)];
        if (k < N3 - 1) acc += c.au * u[at(i, j, k + 1, N1, N2)];
        v[p] = acc;
      }
}

/* Diagonal of the operator (the reset ap of Algorithm 2). */
static void op_diag(int N1, int N2, int N3, double h, int bc, const double* k2, cplx s, cplx* d) {
  for (int k = 0; k < N3; ++k)
    for (int j = 0; j < N2; ++j)
      for (int i = 0; i < N1; ++i) {
        size_t p = at(i, j, k, N1, N2);
        d[p] = node_coefs(i, j, k, N1, N2, N3, h, bc, k2[p], s).ap;
      }
}

/* One damped-Jacobi sweep (Sec. 3.4.1): u <- u + omega D^{-1} (b - M u). */
static void jacobi_sweep(int N1, int N2, int N3, double h, int bc, const double* k2, cplx s,
                         double omega, const cplx* b, cplx* u, cplx* work_mu, cplx* work_d) {
  size_t n = npts3(N1, N2, N3);
  apply_op(N1, N2, N3, h, bc, k2, s, u, work_mu);
  op_diag(N1, N2, N3, h, bc, k2, s, work_d);
  for (size_t p = 0; p < n; ++p) u[p] = u[p] + omega * (b[p] - work_mu[p]) / work_d[p];
}

/* ---------------------------------------------------------------------------------
 * Inter-grid transfers (Sec. 3.4.2 and 3.4.3).  Node space: fine node 2c <-> coarse
 * node c (0-based; the paper's 1-based 2i-1 <-> i).  `off` converts an unknown index
 * to a node index (1 for Dirichlet, 0 for Sommerfeld).  Fine values outside the
 * unknown set are taken as 0 (Dirichlet boundary values of residuals and errors
 * vanish; at a Sommerfeld boundary there is no node beyond the boundary node).
 * --------------------------------------------------------------------------------- */
static cplx fine_val(const cplx* r, int fi, int fj, int fk, int off, int N1, int N2, int N3) {
  int i = fi - off, j = fj - off, k = fk - off; /* node -> unknown index */
  if (i < 0 || i >= N1 || j < 0 || j >= N2 || k < 0 || k >= N3) return 0;
  return r[at(i, j, k, N1, N2)];
}

/* Full weighting, Eq. (matrix-free restriction): 27 points with weights
 * 8 (centre), 4 (face neighbours), 2 (edge neighbours), 1 (corner neighbours), / 64. */
static void restrict_fw(int Nf1, int Nf2, int Nf3, int bc, const cplx* r, int Nc1, int Nc2,
                        int Nc3, cplx* out) {
  int off = (bc == BC_DIRICHLET) ? 1 : 0;
  for (int K = 0; K < Nc3; ++K)
    for (int J = 0; J < Nc2; ++J)
      for (int ic = 0; ic < Nc1; ++ic) {
        int fi = 2 * (ic + off), fj = 2 * (J + off), fk = 2 * (K + off);
        cplx acc = 0;
        for (int dk = -1; dk <= 1; ++dk)
          for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
              int nz = (di != 0) + (dj != 0) + (dk != 0); /* 0 centre, 1 face, 2 edge, 3 corner */
              double w = (nz == 0) ? 8.0 : (nz == 1) ? 4.0 : (nz == 2) ? 2.0 : 1.0;
              acc += w * fine_val(r, fi + di, fj + dj, fk + dk, off, Nf1, Nf2, Nf3);
            }
        out[at(ic, J, K, Nc1, Nc2)] = acc / 64.0;
      }
}

static cplx coarse_val(const cplx* e, int ci, int cj, int ck, int off, int N1, int N2, int N3) {
  int i = ci - off, j = cj - off, k = ck - off;
  if (i < 0 || i >= N1 || j < 0 || j >= N2 || k < 0 || k >= N3) return 0;
  return e[at(i, j, k, N1, N2)];
}

/* Trilinear interpolation, Eq. (matrix-free prolongation): a fine node that coincides
 * with a coarse node takes its value; one between two coarse nodes along 1, 2 or 3
 * axes takes the mean of the 2, 4 or 8 surrounding coarse values. */
static void prolong_tl(int Nc1, int Nc2, int Nc3, int bc, const cplx* e, int Nf1, int Nf2,
                       int Nf3, cplx* out) {
  int off = (bc == BC_DIRICHLET) ? 1 : 0;
  for (int k = 0; k < Nf3; ++k)
    for (int j = 0; j < Nf2; ++j)
      for (int i = 0; i < Nf1; ++i) {
        int fi = i + off, fj = j + off, fk = k + off;
        int ilo = fi / 2, ihi = (fi + 1) / 2; /* equal when the node is even */
        int jlo = fj / 2, jhi = (fj + 1) / 2;
        int klo = fk / 2, khi = (fk + 1) / 2;
        int ci[2] = {ilo, ihi}, cj[2] = {jlo, jhi}, ck[2] = {klo, khi};
        int ni = (ilo == ihi) ? 1 : 2, nj = (jlo == jhi) ? 1 : 2, nk = (klo == khi) ? 1 : 2;
        cplx acc = 0;
        for (int c = 0; c < nk; ++c)
          for (int b = 0; b < nj; ++b)
            for (int a = 0; a < ni; ++a) acc += coarse_val(e, ci[a], cj[b], ck[c], off, Nc1, Nc2, Nc3);
        out[at(i, j, k, Nf1, Nf2)] = acc / (double)(ni * nj * nk);
      }
}

/* ---------------------------------------------------------------------------------
 * Dense complex LU with partial pivoting (used for the coarsest-grid solve).
 * --------------------------------------------------------------------------------- */
static int lu_factor(int n, cplx* a, int* piv) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = cabs(a[(size_t)c * n + c]);
    for (int r = c + 1; r < n; ++r) {
      double v = cabs(a[(size_t)r * n + c]);
      if (v > best) { best = v; p = r; }
    }
    if (best == 0.0) return -1;
    piv[c] = p;
    if (p != c)
      for (int q = 0; q < n; ++q) {
        cplx t = a[(size_t)c * n + q];
        a[(size_t)c * n + q] = a[(size_t)p * n + q];
        a[(size_t)p * n + q] = t;
      }
    for (int r = c + 1; r < n; ++r) {
      cplx f = a[(size_t)r * n + c] / a[(size_t)c * n + c];
      a[(size_t)r * n + c] = f;
      for (int q = c + 1; q < n; ++q) a[(size_t)r * n + q] -= f * a[(size_t)c * n + q];
    }
  }
  return 0;
}

static void lu_solve(int n, const cplx* a, const int* piv, cplx* x) {
  for (int c = 0; c < n; ++c)
    if (piv[c] != c) { cplx t = x[c]; x[c] = x[piv[c]]; x[piv[c]] = t; }
  for (int r = 0; r < n; ++r)
    for (int q = 0; q < r; ++q) x[r] -= a[(size_t)r * n + q] * x[q];
  for (int r = n - 1; r >= 0; --r) {
    for (int q = r + 1; q < n; ++q) x[r] -= a[(size_t)r * n + q] * x[q];
    x[r] /= a[(size_t)r * n + r];
  }
}

/* ---------------------------------------------------------------------------------
 * Multigrid hierarchy (Sec. 3.4 and 4.2) and the V-cycle (Algorithm 1 applied
 * recursively, one pre- and one post-smoothing sweep per level by default).
 * --------------------------------------------------------------------------------- */
#define MAXLEV 32
typedef struct {
  int n1, n2, n3;   /* intervals */
  int N1, N2, N3;   /* unknowns */
  double h;
  double* k2;
  cplx *b, *u, *r, *t, *d; /* per-level work */
} olevel;

typedef struct {
  int bc, nlev, nu1, nu2;
  int cycle;    /* preconditioner of the Krylov methods: 0 one V-cycle, 1 one F-cycle */
  double coarse_tol; /* 0: exact coarsest solve (LU); > 0: full GMRES to this relative residual */
  double beta1, beta2, omega;
  olevel L[MAXLEV];
  int nc;       /* coarsest unknown count */
  cplx* lu;     /* coarsest M_L, LU factors */
  int* piv;
} octx;

static int unknowns(int n, int bc) { return bc == BC_DIRICHLET ? n - 1 : n + 1; }
static cplx cslp_shift(const octx* c) { return c->beta1 - c->beta2 * I; }

static void level_alloc(olevel* L) {
  size_t n = npts3(L->N1, L->N2, L->N3);
  L->k2 = (double*)calloc(n, sizeof(double));
  L->b = (cplx*)calloc(n, sizeof(cplx));
  L->u = (cplx*)calloc(n, sizeof(cplx));
  L->r = (cplx*)calloc(n, sizeof(cplx));
  L->t = (cplx*)calloc(n, sizeof(cplx));
  L->d = (cplx*)calloc(n, sizeof(cplx));
}

void oracle_destroy(void* vctx) {
  octx* c = (octx*)vctx;
  if (!c) return;
  for (int l = 0; l < c->nlev; ++l) {
    free(c->L[l].k2); free(c->L[l].b); free(c->L[l].u); free(c->L[l].r); free(c->L[l].t); free(c->L[l].d);
  }
  free(c->lu); free(c->piv); free(c);
}

/* Coarsen while every direction has an even interval count whose half is still at
 * least coarsest_n intervals.  k^2 on the coarse grid by injection: a coarse node is a
 * fine node, so it keeps that node's value (DCG re-discretisation, Sec. 3.4.4). */
void* oracle_create(int n1, int n2, int n3, double h, int bc, const double* k2, double beta1,
                    double beta2, double omega, int nu1, int nu2, int coarsest_n) {
  if (n1 < 2 || n2 < 2 || n3 < 2 || h <= 0 || (bc != 0 && bc != 1) || coarsest_n < 1) return NULL;
  octx* c = (octx*)calloc(1, sizeof(octx));
  c->bc = bc; c->beta1 = beta1; c->beta2 = beta2; c->omega = omega; c->nu1 = nu1; c->nu2 = nu2;
  int a = n1, b = n2, d = n3;
  double hl = h;
  int nl = 0;
  for (;;) {
    olevel* L = &c->L[nl];
    L->n1 = a; L->n2 = b; L->n3 = d; L->h = hl;
    L->N1 = unknowns(a, bc); L->N2 = unknowns(b, bc); L->N3 = unknowns(d, bc);
    level_alloc(L);
    ++nl;
    int can = (a % 2 == 0) && (b % 2 == 0) && (d % 2 == 0) && a / 2 >= coarsest_n &&
              b / 2 >= coarsest_n && d / 2 >= coarsest_n && nl < MAXLEV;
    if (!can) break;
    a /= 2; b /= 2; d /= 2; hl *= 2;
  }
  c->nlev = nl;
  memcpy(c->L[0].k2, k2, npts3(c->L[0].N1, c->L[0].N2, c->L[0].N3) * sizeof(double));
  int off = (bc == BC_DIRICHLET) ? 1 : 0;
  for (int l = 1; l < nl; ++l) {
    olevel *F = &c->L[l - 1], *C = &c->L[l];
    for (int K = 0; K < C->N3; ++K)
      for (int J = 0; J < C->N2; ++J)
        for (int I0 = 0; I0 < C->N1; ++I0) {
          int fi = 2 * (I0 + off) - off, fj = 2 * (J + off) - off, fk = 2 * (K + off) - off;
          C->k2[at(I0, J, K, C->N1, C->N2)] = F->k2[at(fi, fj, fk, F->N1, F->N2)];
        }
  }
  /* Coarsest operator assembled column by column (column q = M_L e_q), then LU. */
  olevel* Lc = &c->L[nl - 1];
  int nc = (int)npts3(Lc->N1, Lc->N2, Lc->N3);
  c->nc = nc;
  c->lu = (cplx*)calloc((size_t)nc * nc, sizeof(cplx));
  c->piv = (int*)calloc(nc, sizeof(int));
  cplx* e = (cplx*)calloc(nc, sizeof(cplx));
  cplx* col = (cplx*)calloc(nc, sizeof(cplx));
  for (int q = 0; q < nc; ++q) {
    memset(e, 0, nc * sizeof(cplx));
    e[q] = 1;
    apply_op(Lc->N1, Lc->N2, Lc->N3, Lc->h, bc, Lc->k2, cslp_shift(c), e, col);
    for (int r = 0; r < nc; ++r) c->lu[(size_t)r * nc + q] = col[r];
  }
  free(e); free(col);
  if (lu_factor(nc, c->lu, c->piv) != 0) { oracle_destroy(c); return NULL; }
  return c;
}

int oracle_nlevels(void* vctx) { return ((octx*)vctx)->nlev; }

void oracle_level_info(void* vctx, int l, int* dims6, double* h) {
  olevel* L = &((octx*)vctx)->L[l];
  dims6[0] = L->n1; dims6[1] = L->n2; dims6[2] = L->n3;
  dims6[3] = L->N1; dims6[4] = L->N2; dims6[5] = L->N3;
  *h = L->h;
}

void oracle_level_k2(void* vctx, int l, double* out) {
  olevel* L = &((octx*)vctx)->L[l];
  memcpy(out, L->k2, npts3(L->N1, L->N2, L->N3) * sizeof(double));
}

/* Exact coarsest-grid solve e = M_L^{-1} b (Algorithm 1, step 4, on the last level). */
/* The paper's coarsest-grid solver (Sec. 5): full (unrestarted, unpreconditioned) GMRES on
 * M_L e = b from e = 0, stopped when ||b - M_L e|| / ||b|| <= coarse_tol; modified
 * Gram-Schmidt and complex Givens rotations, as the outer GMRES. */
static void coarse_gmres(octx* c, const cplx* b, cplx* e) {
  olevel* L = &c->L[c->nlev - 1];
  const int n = c->nc;
  const cplx s = cslp_shift(c);
  const int m = n;  /* at most n steps: the Krylov space is then the whole space */
  cplx* V = (cplx*)calloc((size_t)(m + 1) * n, sizeof(cplx));
  cplx* H = (cplx*)calloc((size_t)(m + 1) * m, sizeof(cplx));
  double* cs = (double*)calloc(m, sizeof(double));
  cplx* sn = (cplx*)calloc(m, sizeof(cplx));
  cplx* g = (cplx*)calloc(m + 1, sizeof(cplx));
  cplx* y = (cplx*)calloc(m, sizeof(cplx));
  cplx* w = (cplx*)calloc(n, sizeof(cplx));
  double bn = 0;
  for (int p = 0; p < n; ++p) bn += creal(b[p]) * creal(b[p]) + cimag(b[p]) * cimag(b[p]);
  bn = sqrt(bn);
  memset(e, 0, (size_t)n * sizeof(cplx));
  if (bn == 0.0) goto done;
  for (int p = 0; p < n; ++p) V[p] = b[p] / bn;
  g[0] = bn;
  int k = 0;
  for (int j = 0; j < m; ++j) {
    apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, V + (size_t)j * n, w);
    for (int i = 0; i <= j; ++i) {
      cplx hij = 0;
      for (int p = 0; p < n; ++p) hij += conj(V[(size_t)i * n + p]) * w[p];
      H[(size_t)i * m + j] = hij;
      for (int p = 0; p < n; ++p) w[p] -= hij * V[(size_t)i * n + p];
    }
    double hn = 0;
    for (int p = 0; p < n; ++p) hn += creal(w[p]) * creal(w[p]) + cimag(w[p]) * cimag(w[p]);
    hn = sqrt(hn);
    H[(size_t)(j + 1) * m + j] = hn;
    if (hn != 0.0)
      for (int p = 0; p < n; ++p) V[(size_t)(j + 1) * n + p] = w[p] / hn;
    for (int i = 0; i < j; ++i) {
      cplx a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
      H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
      H[(size_t)(i + 1) * m + j] = -conj(sn[i]) * a + cs[i] * bb;
    }
    cplx a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
    double na = cabs(a), t = sqrt(na * na + cabs(bb) * cabs(bb));
    if (na == 0.0) { cs[j] = 0.0; sn[j] = 1.0; H[(size_t)j * m + j] = bb; }
    else {
      cplx ph = a / na;
      cs[j] = na / t;
      sn[j] = ph * conj(bb) / t;
      H[(size_t)j * m + j] = ph * t;
    }
    H[(size_t)(j + 1) * m + j] = 0;
    g[j + 1] = -conj(sn[j]) * g[j];
    g[j] = cs[j] * g[j];
    k = j + 1;
    if (cabs(g[j + 1]) / bn <= c->coarse_tol || hn == 0.0) break;
  }
  for (int i = k - 1; i >= 0; --i) {
    cplx acc = g[i];
    for (int q = i + 1; q < k; ++q) acc -= H[(size_t)i * m + q] * y[q];
    y[i] = acc / H[(size_t)i * m + i];
  }
  for (int i = 0; i < k; ++i)
    for (int p = 0; p < n; ++p) e[p] += y[i] * V[(size_t)i * n + p];
done:
  free(V); free(H); free(cs); free(sn); free(g); free(y); free(w);
}

static void coarse_solve(octx* c, const cplx* b, cplx* e) {
  if (c->coarse_tol > 0.0) { coarse_gmres(c, b, e); return; }
  memcpy(e, b, (size_t)c->nc * sizeof(cplx));
  lu_solve(c->nc, c->lu, c->piv, e);
}

void oracle_set_coarse_tol(void* vctx, double tol) { ((octx*)vctx)->coarse_tol = tol; }

/* Two-grid cycle (Algorithm 1) applied recursively with a zero initial guess on every
 * level: the V-cycle.  Writes u ~= M_l^{-1} b. */
static void vcycle_level(octx* c, int l, const cplx* b, cplx* u) {
  olevel* L = &c->L[l];
  size_t n = npts3(L->N1, L->N2, L->N3);
  if (l == c->nlev - 1) { coarse_solve(c, b, u); return; }
  cplx s = cslp_shift(c);
  olevel* C = &c->L[l + 1];
  /* 1. nu1 pre-smoothing sweeps from u = 0 */
  memset(u, 0, n * sizeof(cplx));
  for (int it = 0; it < c->nu1; ++it) jacobi_sweep(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, c->omega, b, u, L->t, L->d);
  /* 2. residual r = b - M u */
  apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, u, L->t);
  for (size_t p = 0; p < n; ++p) L->r[p] = b[p] - L->t[p];
  /* 3. restriction of the residual to the coarse grid */
  restrict_fw(L->N1, L->N2, L->N3, c->bc, L->r, C->N1, C->N2, C->N3, C->b);
  /* 4. coarse-grid error: recursion (or the exact solve on the coarsest level) */
  vcycle_level(c, l + 1, C->b, C->u);
  /* 5.-6. prolongation of the error and correction */
  prolong_tl(C->N1, C->N2, C->N3, c->bc, C->u, L->N1, L->N2, L->N3, L->t);
  for (size_t p = 0; p < n; ++p) u[p] += L->t[p];
  /* 7. nu2 post-smoothing sweeps */
  for (int it = 0; it < c->nu2; ++it) jacobi_sweep(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, c->omega, b, u, L->t, L->d);
}

/* V-cycle on level l started from the current u (not from zero): nu1 Jacobi sweeps from u,
 * residual, restriction, zero-start V-cycle below, correction, nu2 sweeps. */
static void vcycle_from(octx* c, int l, const cplx* b, cplx* u) {
  olevel* L = &c->L[l];
  size_t n = npts3(L->N1, L->N2, L->N3);
  if (l == c->nlev - 1) { coarse_solve(c, b, u); return; }
  cplx s = cslp_shift(c);
  olevel* C = &c->L[l + 1];
  for (int it = 0; it < c->nu1; ++it) jacobi_sweep(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, c->omega, b, u, L->t, L->d);
  apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, u, L->t);
  for (size_t p = 0; p < n; ++p) L->r[p] = b[p] - L->t[p];
  restrict_fw(L->N1, L->N2, L->N3, c->bc, L->r, C->N1, C->N2, C->N3, C->b);
  vcycle_level(c, l + 1, C->b, C->u);
  prolong_tl(C->N1, C->N2, C->N3, c->bc, C->u, L->N1, L->N2, L->N3, L->t);
  for (size_t p = 0; p < n; ++p) u[p] += L->t[p];
  for (int it = 0; it < c->nu2; ++it) jacobi_sweep(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, c->omega, b, u, L->t, L->d);
}

/* F-cycle (Sec. 3.4.5): like the V-cycle, but the coarse-grid error of every level is an
 * F-cycle on the next level followed by one more V-cycle there, started from that result.
 * Each level keeps its own right-hand side copy because the recursion revisits levels. */
static void fcycle_level(octx* c, int l, const cplx* b, cplx* u) {
  olevel* L = &c->L[l];
  size_t n = npts3(L->N1, L->N2, L->N3);
  if (l == c->nlev - 1) { coarse_solve(c, b, u); return; }
  cplx s = cslp_shift(c);
  olevel* C = &c->L[l + 1];
  size_t nc = npts3(C->N1, C->N2, C->N3);
  memset(u, 0, n * sizeof(cplx));
  for (int it = 0; it < c->nu1; ++it) jacobi_sweep(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, c->omega, b, u, L->t, L->d);
  apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, u, L->t);
  for (size_t p = 0; p < n; ++p) L->r[p] = b[p] - L->t[p];
  cplx* bc = (cplx*)malloc(nc * sizeof(cplx));
  cplx* ec = (cplx*)malloc(nc * sizeof(cplx));
  restrict_fw(L->N1, L->N2, L->N3, c->bc, L->r, C->N1, C->N2, C->N3, bc);
  fcycle_level(c, l + 1, bc, ec);
  vcycle_from(c, l + 1, bc, ec);
  prolong_tl(C->N1, C->N2, C->N3, c->bc, ec, L->N1, L->N2, L->N3, L->t);
  for (size_t p = 0; p < n; ++p) u[p] += L->t[p];
  for (int it = 0; it < c->nu2; ++it) jacobi_sweep(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, c->omega, b, u, L->t, L->d);
  free(bc);
  free(ec);
}

void oracle_fcycle(void* vctx, const double* b, double* z) {
  octx* c = (octx*)vctx;
  size_t n = npts3(c->L[0].N1, c->L[0].N2, c->L[0].N3);
  cplx* bb = (cplx*)malloc(n * sizeof(cplx));
  memcpy(bb, b, n * sizeof(cplx));
  fcycle_level(c, 0, bb, (cplx*)z);
  free(bb);
}

void oracle_vcycle(void* vctx, const double* b, double* z) {
  octx* c = (octx*)vctx;
  size_t n = npts3(c->L[0].N1, c->L[0].N2, c->L[0].N3);
  cplx* bb = (cplx*)malloc(n * sizeof(cplx));
  memcpy(bb, b, n * sizeof(cplx));
  vcycle_level(c, 0, bb, (cplx*)z);
  free(bb);
}

/* The preconditioner z = M^{-1} b used by the Krylov methods: one V-cycle, or one F-cycle. */
static void precond(octx* c, const cplx* b, cplx* z) {
  if (c->cycle == 1) fcycle_level(c, 0, b, z);
  else vcycle_level(c, 0, b, z);
}

void oracle_set_cycle(void* vctx, int cycle) { ((octx*)vctx)->cycle = cycle; }

/* Plain building blocks exposed for pins and stage-level parity. */
void oracle_apply(int N1, int N2, int N3, double h, int bc, const double* k2, double s_re,
                  double s_im, const double* u, double* v) {
  apply_op(N1, N2, N3, h, bc, k2, s_re + s_im * I, (const cplx*)u, (cplx*)v);
}

void oracle_diag(int N1, int N2, int N3, double h, int bc, const double* k2, double s_re,
                 double s_im, double* d) {
  op_diag(N1, N2, N3, h, bc, k2, s_re + s_im * I, (cplx*)d);
}

void oracle_jacobi(int N1, int N2, int N3, double h, int bc, const double* k2, double s_re,
                   double s_im, double omega, const double* b, double* u) {
  size_t n = npts3(N1, N2, N3);
  cplx* t = (cplx*)malloc(n * sizeof(cplx));
  cplx* d = (cplx*)malloc(n * sizeof(cplx));
  jacobi_sweep(N1, N2, N3, h, bc, k2, s_re + s_im * I, omega, (const cplx*)b, (cplx*)u, t, d);
  free(t); free(d);
}

void oracle_restrict(int Nf1, int Nf2, int Nf3, int bc, const double* r, int Nc1, int Nc2, int Nc3,
                     double* out) {
  restrict_fw(Nf1, Nf2, Nf3, bc, (const cplx*)r, Nc1, Nc2, Nc3, (cplx*)out);
}

void oracle_prolong(int Nc1, int Nc2, int Nc3, int bc, const double* e, int Nf1, int Nf2, int Nf3,
                    double* out) {
  prolong_tl(Nc1, Nc2, Nc3, bc, (const cplx*)e, Nf1, Nf2, Nf3, (cplx*)out);
}

void oracle_coarse_solve(void* vctx, const double* b, double* e) {
  coarse_solve((octx*)vctx, (const cplx*)b, (cplx*)e);
}

/* Level-l "down" stage of the V-cycle: nu1 sweeps from zero, residual, restriction.
 * Writes the coarse right-hand side b_{l+1}. */
void oracle_vcycle_down(void* vctx, int l, const double* b, double* bcoarse) {
  octx* c = (octx*)vctx;
  olevel *L = &c->L[l], *C = &c->L[l + 1];
  size_t n = npts3(L->N1, L->N2, L->N3);
  cplx s = cslp_shift(c);
  cplx* u = (cplx*)calloc(n, sizeof(cplx));
  for (int it = 0; it < c->nu1; ++it) jacobi_sweep(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, c->omega, (const cplx*)b, u, L->t, L->d);
  apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, u, L->t);
  for (size_t p = 0; p < n; ++p) L->r[p] = ((const cplx*)b)[p] - L->t[p];
  restrict_fw(L->N1, L->N2, L->N3, c->bc, L->r, C->N1, C->N2, C->N3, (cplx*)bcoarse);
  free(u);
}

/* Level-l "up" stage: redo the pre-smoothing from zero, add the prolongated coarse
 * error e_{l+1}, then nu2 post-smoothing sweeps.  Writes u_l. */
void oracle_vcycle_up(void* vctx, int l, const double* b, const double* ecoarse, double* uout) {
  octx* c = (octx*)vctx;
  olevel *L = &c->L[l], *C = &c->L[l + 1];
  size_t n = npts3(L->N1, L->N2, L->N3);
  cplx s = cslp_shift(c);
  cplx* u = (cplx*)uout;
  memset(u, 0, n * sizeof(cplx));
  for (int it = 0; it < c->nu1; ++it) jacobi_sweep(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, c->omega, (const cplx*)b, u, L->t, L->d);
  prolong_tl(C->N1, C->N2, C->N3, c->bc, (const cplx*)ecoarse, L->N1, L->N2, L->N3, L->t);
  for (size_t p = 0; p < n; ++p) u[p] += L->t[p];
  for (int it = 0; it < c->nu2; ++it) jacobi_sweep(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, s, c->omega, (const cplx*)b, u, L->t, L->d);
}

/* ---------------------------------------------------------------------------------
 * Right-preconditioned GMRES(m) (Sec. 3.1-3.2): A M^{-1} y = b, x = M^{-1} y, with
 * M^{-1} one V-cycle.  Arnoldi by modified Gram-Schmidt, Hessenberg least squares by
 * complex Givens rotations.  flexible = 1 stores z_j = M^{-1} v_j and updates
 * x += Z y (FGMRES); flexible = 0 updates x += M^{-1}(V y).  flexible = 2 is the paper's own
 * left preconditioning (Sec. 3.2): GMRES on M^{-1} A x = M^{-1} b, Arnoldi vectors
 * w = M^{-1}(A v_j), x += V y, and the paper's GMRES stopping rule (Sec. 5) on the
 * preconditioned residual ||M^{-1}(b - A x)|| / ||M^{-1} b||.  `iters` counts products with
 * A_h inside the Arnoldi process (#Matvec, Sec. 5).  Returns 0 when the explicit relative
 * residual (preconditioned, for flexible = 2) reached tol, 1 when max_iter was hit first,
 * -1 on breakdown to NaN.
 * --------------------------------------------------------------------------------- */
static double vnorm(size_t n, const cplx* x) {
  double s = 0;
  for (size_t p = 0; p < n; ++p) s += creal(x[p]) * creal(x[p]) + cimag(x[p]) * cimag(x[p]);
  return sqrt(s);
}

static cplx vdot(size_t n, const cplx* v, const cplx* w) {
  cplx s = 0;
  for (size_t p = 0; p < n; ++p) s += conj(v[p]) * w[p];
  return s;
}

int oracle_gmres(void* vctx, const double* bin, double* xio, int m, double tol, int max_iter,
                 int flexible, int* iters_out, double* relres_out, double* hist, int hist_len) {
  octx* c = (octx*)vctx;
  olevel* L = &c->L[0];
  size_t n = npts3(L->N1, L->N2, L->N3);
  const cplx* b = (const cplx*)bin;
  cplx* x = (cplx*)xio;
  cplx one = 1.0;
  cplx* V = (cplx*)calloc((size_t)(m + 1) * n, sizeof(cplx));
  cplx* Z = flexible ? (cplx*)calloc((size_t)m * n, sizeof(cplx)) : NULL;
  cplx* w = (cplx*)calloc(n, sizeof(cplx));
  cplx* z = (cplx*)calloc(n, sizeof(cplx));
  cplx* r = (cplx*)calloc(n, sizeof(cplx));
  cplx* H = (cplx*)calloc((size_t)(m + 1) * m, sizeof(cplx)); /* H[i*m + j] */
  double* cs = (double*)calloc(m, sizeof(double));
  cplx* sn = (cplx*)calloc(m, sizeof(cplx));
  cplx* g = (cplx*)calloc(m + 1, sizeof(cplx));
  cplx* y = (cplx*)calloc(m, sizeof(cplx));
  (void)one;
  int iters = 0, status = 1;
  const int left = flexible == 2;
  if (left) flexible = 0;
  double bnorm;
  if (left) {
    precond(c, b, z);
    bnorm = vnorm(n, z);
  } else {
    bnorm = vnorm(n, b);
  }
  if (bnorm == 0.0) bnorm = 1.0;
  /* r = b - A x, and M^{-1} of it when preconditioning from the left */
  apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, 1.0, x, w);
  for (size_t p = 0; p < n; ++p) r[p] = b[p] - w[p];
  if (left) {
    precond(c, r, z);
    memcpy(r, z, n * sizeof(cplx));
  }
  double beta = vnorm(n, r);
  double relres = beta / bnorm;
  for (;;) {
    if (relres <= tol) { status = 0; break; }
    if (iters >= max_iter) { status = 1; break; }
    if (!isfinite(relres)) { status = -1; break; }
    for (size_t p = 0; p < n; ++p) V[p] = r[p] / beta;
    memset(g, 0, (m + 1) * sizeof(cplx));
    g[0] = beta;
    int jend = 0;
    for (int j = 0; j < m; ++j) {
      cplx* vj = V + (size_t)j * n;
      if (left) {
        apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, 1.0, vj, z);  /* z = A v_j */
        precond(c, z, w);                                                /* w = M^{-1} z */
      } else {
        cplx* zj = flexible ? Z + (size_t)j * n : z;
        precond(c, vj, zj);                                      /* z_j = M^{-1} v_j */
        apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, 1.0, zj, w);  /* w = A z_j */
      }
      ++iters;
      for (int i = 0; i <= j; ++i) {                                   /* modified Gram-Schmidt */
        cplx* vi = V + (size_t)i * n;
        cplx hij = vdot(n, vi, w);
        H[(size_t)i * m + j] = hij;
        for (size_t p = 0; p < n; ++p) w[p] -= hij * vi[p];
      }
      double hn = vnorm(n, w);
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn != 0.0) {
        cplx* vn = V + (size_t)(j + 1) * n;
        for (size_t p = 0; p < n; ++p) vn[p] = w[p] / hn;
      }
      /* apply the previous rotations to column j */
      for (int i = 0; i < j; ++i) {
        cplx a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
        H[(size_t)(i + 1) * m + j] = -conj(sn[i]) * a + cs[i] * bb;
      }
      /* new rotation zeroing H[j+1][j] */
      cplx a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
      double na = cabs(a), t = sqrt(na * na + cabs(bb) * cabs(bb));
      if (na == 0.0) { cs[j] = 0.0; sn[j] = 1.0; H[(size_t)j * m + j] = bb; }
      else {
        cplx ph = a / na;
        cs[j] = na / t;
        sn[j] = ph * conj(bb) / t;
        H[(size_t)j * m + j] = ph * t;
      }
      H[(size_t)(j + 1) * m + j] = 0;
      g[j + 1] = -conj(sn[j]) * g[j];
      g[j] = cs[j] * g[j];
      double est = cabs(g[j + 1]) / bnorm;
      if (hist && iters - 1 < hist_len) hist[iters - 1] = est;
      jend = j;
      if (est <= tol || iters >= max_iter || hn == 0.0) break;
    }
    /* back-substitution H(0:jend,0:jend) y = g */
    int k = jend + 1;
    for (int i = k - 1; i >= 0; --i) {
      cplx s = g[i];
      for (int q = i + 1; q < k; ++q) s -= H[(size_t)i * m + q] * y[q];
      y[i] = s / H[(size_t)i * m + i];
    }
    if (left) {
      for (int i = 0; i < k; ++i)
        for (size_t p = 0; p < n; ++p) x[p] += y[i] * V[(size_t)i * n + p];
    } else if (flexible) {
      for (int i = 0; i < k; ++i)
        for (size_t p = 0; p < n; ++p) x[p] += y[i] * Z[(size_t)i * n + p];
    } else {
      memset(w, 0, n * sizeof(cplx));
      for (int i = 0; i < k; ++i)
        for (size_t p = 0; p < n; ++p) w[p] += y[i] * V[(size_t)i * n + p];
      precond(c, w, z);
      for (size_t p = 0; p < n; ++p) x[p] += z[p];
    }
    apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, 1.0, x, w);
    for (size_t p = 0; p < n; ++p) r[p] = b[p] - w[p];
    if (left) {
      precond(c, r, z);
      memcpy(r, z, n * sizeof(cplx));
    }
    beta = vnorm(n, r);
    relres = beta / bnorm;
  }
  *iters_out = iters;
  *relres_out = relres;
  free(V); free(Z); free(w); free(z); free(r); free(H); free(cs); free(sn); free(g); free(y);
  return status;
}

/* ---------------------------------------------------------------------------------
 * Right-hand sides.
 * --------------------------------------------------------------------------------- */
/* Discrete Dirac delta (Sec. 2.4, Eq. "discrete dirac func"): 1/h^3 at the source
 * node, 0 elsewhere.  Sources are given as node coordinates (0..n per direction);
 * a source on a Dirichlet boundary node is not an unknown and is ignored. */
void oracle_rhs_point(int N1, int N2, int N3, int bc, double h, int nsrc, const int* nodes,
                      double* bout) {
  cplx* b = (cplx*)bout;
  int off = (bc == BC_DIRICHLET) ? 1 : 0;
  memset(b, 0, npts3(N1, N2, N3) * sizeof(cplx));
  for (int s = 0; s < nsrc; ++s) {
    int i = nodes[3 * s] - off, j = nodes[3 * s + 1] - off, k = nodes[3 * s + 2] - off;
    if (i < 0 || i >= N1 || j < 0 || j >= N2 || k < 0 || k >= N3) continue;
    b[at(i, j, k, N1, N2)] += 1.0 / (h * h * h);
  }
}

/* Closed-off problem (Sec. 2.1): b = (21 pi^2 - k^2) sin(pi x1) sin(2 pi x2) sin(4 pi x3) - k^2
 * on the unit cube with Dirichlet u = g = 1, n intervals per direction.  The known
 * boundary values are lifted into the right-hand side: each boundary neighbour of an
 * unknown contributes g / h^2. */
void oracle_rhs_closed_off(int n, double kconst, double* bout) {
  cplx* b = (cplx*)bout;
  int N = n - 1;
  double h = 1.0 / n, pi = acos(-1.0), k2 = kconst * kconst;
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        double x = (i + 1) * h, y = (j + 1) * h, z = (k + 1) * h;
        double f = (21.0 * pi * pi - k2) * sin(pi * x) * sin(2 * pi * y) * sin(4 * pi * z) - k2;
        int nb = (i == 0) + (i == N - 1) + (j == 0) + (j == N - 1) + (k == 0) + (k == N - 1);
        b[at(i, j, k, N, N)] = f + nb * 1.0 / (h * h);
      }
}

/* ---------------------------------------------------------------------------------
 * Adjoint state for frequency-domain gradients (not in the paper; its operator and
 * boundary scheme are).  With D = diag(2^-faces) the row scaling that makes D A symmetric
 * (Sommerfeld; D = I for Dirichlet), A^T = D A D^-1, so A^H lambda = g is solved with the
 * forward operator: A nu = D^-1 conj(g), lambda = conj(D nu).
 * --------------------------------------------------------------------------------- */
static int face_count(int i, int j, int k, int N1, int N2, int N3, int bc) {
  if (bc != BC_SOMMERFELD) return 0;
  return (i == 0) + (i == N1 - 1) + (j == 0) + (j == N2 - 1) + (k == 0) + (k == N3 - 1);
}

/* q = D^-1 conj(g) */
void oracle_adjoint_rhs(int N1, int N2, int N3, int bc, const double* gin, double* qout) {
  const cplx* g = (const cplx*)gin;
  cplx* q = (cplx*)qout;
  for (int k = 0; k < N3; ++k)
    for (int j = 0; j < N2; ++j)
      for (int i = 0; i < N1; ++i) {
        size_t p = at(i, j, k, N1, N2);
        q[p] = ldexp(1.0, face_count(i, j, k, N1, N2, N3, bc)) * conj(g[p]);
      }
}

/* lambda = conj(D nu) */
void oracle_adjoint_finish(int N1, int N2, int N3, int bc, const double* nuin, double* lout) {
  const cplx* nu = (const cplx*)nuin;
  cplx* l = (cplx*)lout;
  for (int k = 0; k < N3; ++k)
    for (int j = 0; j < N2; ++j)
      for (int i = 0; i < N1; ++i) {
        size_t p = at(i, j, k, N1, N2);
        l[p] = conj(ldexp(1.0, -face_count(i, j, k, N1, N2, N3, bc)) * nu[p]);
      }
}

/* grad[p] += -Re(conj(lambda_p) (dA_pp / dk2_p) u_p): A depends on k^2_p only through its
 * diagonal entry -k^2_p - i (2 k_p / h) nf_p, whose derivative is -1 - i nf_p / (h k_p). */
void oracle_grad_k2(int N1, int N2, int N3, double h, int bc, const double* k2, const double* uin,
                    const double* lin, double* grad) {
  const cplx* u = (const cplx*)uin;
  const cplx* l = (const cplx*)lin;
  for (int k = 0; k < N3; ++k)
    for (int j = 0; j < N2; ++j)
      for (int i = 0; i < N1; ++i) {
        size_t p = at(i, j, k, N1, N2);
        int nf = face_count(i, j, k, N1, N2, N3, bc);
        cplx da = -1.0 - I * (double)nf / (h * sqrt(k2[p]));
        grad[p] += -creal(conj(l[p]) * da * u[p]);
      }
}

/* ---------------------------------------------------------------------------------
 * Right-preconditioned Bi-CGSTAB (Sec. 3.1; van der Vorst's method with the CSLP V-cycle as
 * M^{-1} on the right): x = x0 + M^{-1} y, stopping on ||b - A x|| / ||b|| (Sec. 5 stopping
 * rule for Bi-CGSTAB and IDR(s)).  The shadow residual is the initial residual.  `iters`
 * counts products with A (two per full step, one when the half step already converged).
 * Returns 0 (converged), 1 (max_iter), -1 (breakdown or non-finite).
 * --------------------------------------------------------------------------------- */
int oracle_bicgstab(void* vctx, const double* bin, double* xio, double tol, int max_iter, int* iters_out,
                    double* relres_out, double* hist, int hist_len) {
  octx* c = (octx*)vctx;
  olevel* L = &c->L[0];
  size_t n = npts3(L->N1, L->N2, L->N3);
  const cplx* b = (const cplx*)bin;
  cplx* x = (cplx*)xio;
  cplx* r = (cplx*)calloc(n, sizeof(cplx));
  cplx* rh = (cplx*)calloc(n, sizeof(cplx));
  cplx* p = (cplx*)calloc(n, sizeof(cplx));
  cplx* v = (cplx*)calloc(n, sizeof(cplx));
  cplx* ph = (cplx*)calloc(n, sizeof(cplx));
  cplx* s = (cplx*)calloc(n, sizeof(cplx));
  cplx* sh = (cplx*)calloc(n, sizeof(cplx));
  cplx* t = (cplx*)calloc(n, sizeof(cplx));
  int iters = 0, status = 1;
  double bnorm = vnorm(n, b);
  if (bnorm == 0.0) bnorm = 1.0;
  apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, 1.0, x, t);
  for (size_t q = 0; q < n; ++q) { r[q] = b[q] - t[q]; rh[q] = r[q]; }
  double relres = vnorm(n, r) / bnorm;
  cplx rho_prev = 1.0, alpha = 1.0, omega = 1.0;
  for (;;) {
    if (relres <= tol) { status = 0; break; }
    if (iters >= max_iter) { status = 1; break; }
    if (!isfinite(relres)) { status = -1; break; }
    cplx rho = vdot(n, rh, r);
    if (rho == 0.0 || omega == 0.0) { status = -1; break; }
    cplx beta = (rho / rho_prev) * (alpha / omega);
    for (size_t q = 0; q < n; ++q) p[q] = r[q] + beta * (p[q] - omega * v[q]);
    precond(c, p, ph);                                      /* p^ = M^{-1} p */
    apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, 1.0, ph, v);  /* v = A p^ */
    ++iters;
    cplx rv = vdot(n, rh, v);
    if (rv == 0.0) { status = -1; break; }
    alpha = rho / rv;
    for (size_t q = 0; q < n; ++q) s[q] = r[q] - alpha * v[q];
    double snorm = vnorm(n, s) / bnorm;
    if (hist && iters - 1 < hist_len) hist[iters - 1] = snorm;
    if (snorm <= tol || iters >= max_iter) {
      for (size_t q = 0; q < n; ++q) { x[q] += alpha * ph[q]; r[q] = s[q]; }
      relres = snorm;
      continue;
    }
    precond(c, s, sh);                                      /* s^ = M^{-1} s */
    apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, 1.0, sh, t);  /* t = A s^ */
    ++iters;
    cplx ts = vdot(n, t, s);
    double tt = vnorm(n, t);
    tt *= tt;
    if (tt == 0.0) { status = -1; break; }
    omega = ts / tt;
    for (size_t q = 0; q < n; ++q) {
      x[q] += alpha * ph[q] + omega * sh[q];
      r[q] = s[q] - omega * t[q];
    }
    relres = vnorm(n, r) / bnorm;
    if (hist && iters - 1 < hist_len) hist[iters - 1] = relres;
    rho_prev = rho;
  }
  /* report the explicit residual */
  apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, 1.0, x, t);
  for (size_t q = 0; q < n; ++q) r[q] = b[q] - t[q];
  double rr = vnorm(n, r) / bnorm;
  if (status == 0 && rr > tol) status = 1;
  *iters_out = iters;
  *relres_out = rr;
  free(r); free(rh); free(p); free(v); free(ph); free(s); free(sh); free(t);
  return status;
}

/* ---------------------------------------------------------------------------------
 * Right-preconditioned IDR(s) (Sec. 3.1; the induced-dimension-reduction method of Sonneveld
 * and van Gijzen that the paper runs as IDR(4)), in its biorthogonal form: the s directions
 * G_i = A U_i of a cycle are built so that P_j^H G_i = 0 for j < i, which makes the small
 * matrix Ms = P^H G lower triangular and keeps f = P^H r up to date by one subtraction per
 * step.  Each cycle takes s steps that remove one component of P^H r each, then one
 * dimension-reduction step r -= omega A M^{-1} r with the minimal-residual omega, enlarged to
 * make the angle between r and A M^{-1} r at least acos(kappa) when it is smaller (kappa = 0
 * keeps the minimal-residual omega).  The preconditioner enters only through U, so A U = G
 * holds whatever M^{-1} does and r stays the recursive residual of x.  P holds s vectors of n
 * complex values (the shadow space; only its span matters).  Stops on ||r|| / ||b|| <= tol
 * after any step (Sec. 5 stopping rule), reports the explicit residual; `iters` counts
 * products with A (s + 1 per full cycle).  Returns 0 converged, 1 max_iter, -1 breakdown.
 * --------------------------------------------------------------------------------- */
#define IDR_SMAX 16
int oracle_idrs(void* vctx, int s, const double* Pin, double kappa, const double* bin, double* xio, double tol,
                int max_iter, int* iters_out, double* relres_out, double* hist, int hist_len) {
  octx* c = (octx*)vctx;
  olevel* L = &c->L[0];
  if (s < 1 || s > IDR_SMAX) return -2;
  size_t n = npts3(L->N1, L->N2, L->N3);
  const cplx* b = (const cplx*)bin;
  const cplx* P = (const cplx*)Pin;
  cplx* x = (cplx*)xio;
  cplx* r = (cplx*)calloc(n, sizeof(cplx));
  cplx* v = (cplx*)calloc(n, sizeof(cplx));
  cplx* vh = (cplx*)calloc(n, sizeof(cplx));
  cplx* t = (cplx*)calloc(n, sizeof(cplx));
  cplx* G = (cplx*)calloc(n * (size_t)s, sizeof(cplx));
  cplx* U = (cplx*)calloc(n * (size_t)s, sizeof(cplx));
  cplx Ms[IDR_SMAX][IDR_SMAX], f[IDR_SMAX], cc[IDR_SMAX];
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) Ms[i][j] = i == j ? 1.0 : 0.0;
  cplx om = 1.0;
  int iters = 0, status = 1, done = 0;
  double bnorm = vnorm(n, b);
  if (bnorm == 0.0) bnorm = 1.0;
  apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, 1.0, x, t);
  for (size_t q = 0; q < n; ++q) r[q] = b[q] - t[q];
  double relres = vnorm(n, r) / bnorm;
  if (relres <= tol) { status = 0; done = 1; }
  while (!done) {
    if (iters >= max_iter) { status = 1; break; }
    for (int i = 0; i < s; ++i) f[i] = vdot(n, P + (size_t)i * n, r);
    for (int k = 0; k < s && !done; ++k) {
      /* Ms[k.., k..] c = f[k..] (lower triangular) */
      for (int i = k; i < s; ++i) {
        cplx acc = f[i];
        for (int j = k; j < i; ++j) acc -= Ms[i][j] * cc[j];
        cc[i] = acc / Ms[i][i];
      }
      /* v = r - G[:, k..] c; new direction U_k = omega M^{-1} v + U[:, k..] c */
      for (size_t q = 0; q < n; ++q) {
        cplx a = r[q];
        for (int i = k; i < s; ++i) a -= cc[i] * G[(size_t)i * n + q];
        v[q] = a;
      }
      precond(c, v, vh);
      for (size_t q = 0; q < n; ++q) {
        cplx a = om * vh[q];
        for (int i = k; i < s; ++i) a += cc[i] * U[(size_t)i * n + q];
        t[q] = a;
      }
      cplx* Uk = U + (size_t)k * n;
      cplx* Gk = G + (size_t)k * n;
      memcpy(Uk, t, n * sizeof(cplx));
      apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, 1.0, Uk, Gk);  /* G_k = A U_k */
      ++iters;
      /* biorthogonalise G_k against P_0 .. P_{k-1}, carrying U_k along */
      for (int i = 0; i < k; ++i) {
        cplx alpha = vdot(n, P + (size_t)i * n, Gk) / Ms[i][i];
        for (size_t q = 0; q < n; ++q) {
          Gk[q] -= alpha * G[(size_t)i * n + q];
          Uk[q] -= alpha * U[(size_t)i * n + q];
        }
      }
      for (int i = k; i < s; ++i) Ms[i][k] = vdot(n, P + (size_t)i * n, Gk);
      if (Ms[k][k] == 0.0) { status = -1; done = 1; break; }
      /* remove the k-th component of P^H r */
      cplx beta = f[k] / Ms[k][k];
      for (size_t q = 0; q < n; ++q) {
        r[q] -= beta * Gk[q];
        x[q] += beta * Uk[q];
      }
      relres = vnorm(n, r) / bnorm;
      if (hist && iters - 1 < hist_len) hist[iters - 1] = relres;
      if (!isfinite(relres)) { status = -1; done = 1; break; }
      if (relres <= tol) { status = 0; done = 1; break; }
      if (iters >= max_iter) { status = 1; done = 1; break; }
      for (int i = k + 1; i < s; ++i) f[i] -= beta * Ms[i][k];
    }
    if (done) break;
    /* dimension reduction: r -= omega A M^{-1} r */
    precond(c, r, vh);
    apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, 1.0, vh, t);
    ++iters;
    cplx tr = vdot(n, t, r);
    double tn = vnorm(n, t), rn = vnorm(n, r);
    if (tn == 0.0) { status = -1; break; }
    om = tr / (tn * tn);
    double rho = cabs(tr) / (tn * rn);
    if (rho < kappa) om *= kappa / rho;
    if (om == 0.0) { status = -1; break; }
    for (size_t q = 0; q < n; ++q) {
      r[q] -= om * t[q];
      x[q] += om * vh[q];
    }
    relres = vnorm(n, r) / bnorm;
    if (hist && iters - 1 < hist_len) hist[iters - 1] = relres;
    if (!isfinite(relres)) { status = -1; break; }
    if (relres <= tol) { status = 0; break; }
  }
  /* report the explicit residual */
  apply_op(L->N1, L->N2, L->N3, L->h, c->bc, L->k2, 1.0, x, t);
  for (size_t q = 0; q < n; ++q) r[q] = b[q] - t[q];
  double rr = vnorm(n, r) / bnorm;
  if (status == 0 && rr > tol) status = 1;
  *iters_out = iters;
  *relres_out = rr;
  free(r); free(v); free(vh); free(t); free(G); free(U);
  return status;
}
