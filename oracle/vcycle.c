/*
 * Oracle (test infrastructure and CPU baseline only): the 4-colour
 * V(nu1, nu2)-cycle of oracle/multigrid.py restated in plain C with OpenMP,
 * so that the method can be timed on the host cores.  Nothing here is part
 * of the product path; it shares no code with the CUDA library.
 *
 * What it computes (the same steps, in the same order, as
 * oracle.multigrid.mg_cycle with order="color4"):
 *   - Gauss-Seidel smoother (Sec. 4.1): colours (i mod 2, j mod 2) visited in
 *     the order (0,0), (1,0), (0,1), (1,1); node k of the colour gets
 *     u_k += (F_k - sum_j A_kj u_j) / A_kk, the sum over row k of the CSR
 *     matrix in its stored order.  Same-colour nodes share no 9-point
 *     stencil, so the nodes of one colour are updated in parallel.
 *   - one smoothing step = a sweep over all DOFs, then eta sweeps over the
 *     vertices of the level's cut cells (Sec. 5.3);
 *   - residual r = F - A u, restriction F_2h = P^T r (Sec. 5.1, R = P^T),
 *     recursion (Alg. 1 applied recursively, Sec. 3.2) from e = 0,
 *     prolongation u += P e;
 *   - the coarsest level solved exactly: dense Cholesky of A restricted to
 *     its DOFs (factored once in vc_set_level).
 *   - vc_solve: cycles from u until ||F - A u||_inf / ||F||_inf <= tol.
 * Operators, masks and P come from the Python oracle's hierarchy
 * (oracle.multigrid.build_hierarchy); each level holds copies.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* the rows of A for a list of nodes, stored contiguously (a node set's
 * sweep then streams through memory) */
typedef struct {
  int cnt;
  int *idx, *p, *i;
  double *x, *diag;
} rows_t;

typedef struct {
  int n, m;                       /* cells per side, nodes (n+1)^2 */
  int *Ap, *Ai;                   /* A in CSR over the m nodes */
  double *Ax, *diag;
  rows_t col[4];                  /* DOFs of each colour, increasing */
  rows_t cut[4];                  /* cut-cell vertices (DOFs) of each colour */
  rows_t all;                     /* every DOF (residual) */
  int *dofs, ndof;
  int *Pp, *Pi;                   /* P from the next coarser level: m rows */
  double *Px;
  int *Tp, *Ti;                   /* P^T: rows over the coarse nodes */
  double *Tx;
  double *u, *F, *r;              /* work vectors (levels >= 1), residual */
  double *L;                      /* coarsest: Cholesky factor, ndof^2 */
} level_t;

typedef struct {
  int nlev;
  level_t* lev;
} hier_t;

static void rows_free(rows_t* r) {
  free(r->idx); free(r->p); free(r->i); free(r->x); free(r->diag);
}

/* rows of the listed nodes (increasing) out of the CSR matrix */
static int rows_take(rows_t* r, const int* list, int cnt, const int* Ap, const int* Ai,
                     const double* Ax, const double* diag) {
  int nnz = 0;
  for (int a = 0; a < cnt; ++a) nnz += Ap[list[a] + 1] - Ap[list[a]];
  r->cnt = cnt;
  r->idx = (int*)malloc(sizeof(int) * (size_t)(cnt + 1));
  r->p = (int*)malloc(sizeof(int) * (size_t)(cnt + 1));
  r->i = (int*)malloc(sizeof(int) * (size_t)(nnz + 1));
  r->x = (double*)malloc(sizeof(double) * (size_t)(nnz + 1));
  r->diag = (double*)malloc(sizeof(double) * (size_t)(cnt + 1));
  if (!r->idx || !r->p || !r->i || !r->x || !r->diag) return -1;
  int q = 0;
  r->p[0] = 0;
  for (int a = 0; a < cnt; ++a) {
    const int k = list[a];
    r->idx[a] = k;
    r->diag[a] = diag[k];
    for (int t = Ap[k]; t < Ap[k + 1]; ++t, ++q) {
      r->i[q] = Ai[t];
      r->x[q] = Ax[t];
    }
    r->p[a + 1] = q;
  }
  return 0;
}

static void* copy(const void* src, size_t bytes) {
  void* p = malloc(bytes ? bytes : 1);
  if (p && bytes) memcpy(p, src, bytes);
  return p;
}

void* vc_create(int nlev) {
  hier_t* h = (hier_t*)calloc(1, sizeof(hier_t));
  if (!h) return NULL;
  h->nlev = nlev;
  h->lev = (level_t*)calloc((size_t)nlev, sizeof(level_t));
  if (!h->lev) {
    free(h);
    return NULL;
  }
  return h;
}

void vc_destroy(void* hp) {
  hier_t* h = (hier_t*)hp;
  if (!h) return;
  for (int l = 0; l < h->nlev; ++l) {
    level_t* v = &h->lev[l];
    free(v->Ap); free(v->Ai); free(v->Ax); free(v->diag);
    for (int c = 0; c < 4; ++c) { rows_free(&v->col[c]); rows_free(&v->cut[c]); }
    rows_free(&v->all);
    free(v->dofs);
    free(v->Pp); free(v->Pi); free(v->Px);
    free(v->Tp); free(v->Ti); free(v->Tx);
    free(v->u); free(v->F); free(v->r); free(v->L);
  }
  free(h->lev);
  free(h);
}

/* Level l: A (CSR, m = (n+1)^2 rows), DOF and cut-node masks (bytes), and,
 * for l < nlev - 1, P from level l + 1 (m rows) and P^T (rows over level
 * l + 1's nodes).  Returns 0, or -1 (allocation) / -2 (the coarsest matrix
 * is not positive definite). */
int vc_set_level(void* hp, int l, int n, const int* Ap, const int* Ai, const double* Ax,
                 const uint8_t* dof, const uint8_t* cutm, const int* Pp, const int* Pi,
                 const double* Px, const int* Tp, const int* Ti, const double* Tx, int mc) {
  hier_t* h = (hier_t*)hp;
  level_t* v = &h->lev[l];
  const int m = (n + 1) * (n + 1);
  v->n = n;
  v->m = m;
  const int nnz = Ap[m];
  v->Ap = (int*)copy(Ap, sizeof(int) * (size_t)(m + 1));
  v->Ai = (int*)copy(Ai, sizeof(int) * (size_t)nnz);
  v->Ax = (double*)copy(Ax, sizeof(double) * (size_t)nnz);
  v->diag = (double*)calloc((size_t)m, sizeof(double));
  v->u = (double*)calloc((size_t)m, sizeof(double));
  v->F = (double*)calloc((size_t)m, sizeof(double));
  v->r = (double*)calloc((size_t)m, sizeof(double));
  v->dofs = (int*)malloc(sizeof(int) * (size_t)m);
  if (!v->Ap || !v->Ai || !v->Ax || !v->diag || !v->u || !v->F || !v->r || !v->dofs) return -1;
  for (int k = 0; k < m; ++k)
    for (int q = Ap[k]; q < Ap[k + 1]; ++q)
      if (Ai[q] == k) v->diag[k] += Ax[q];
  v->ndof = 0;
  {
    int* lists = (int*)malloc(sizeof(int) * (size_t)m * 8 + 8);
    int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (!lists) return -1;
    for (int k = 0; k < m; ++k) {
      if (!dof[k]) continue;
      v->dofs[v->ndof++] = k;
      const int i = k % (n + 1), j = k / (n + 1);
      const int c = (i & 1) + 2 * (j & 1);
      lists[(size_t)c * m + cnt[c]++] = k;
      if (cutm[k]) lists[(size_t)(4 + c) * m + cnt[4 + c]++] = k;
    }
    int rc = rows_take(&v->all, v->dofs, v->ndof, Ap, Ai, Ax, v->diag);
    for (int c = 0; c < 4 && rc == 0; ++c) {
      rc = rows_take(&v->col[c], lists + (size_t)c * m, cnt[c], Ap, Ai, Ax, v->diag);
      if (rc == 0)
        rc = rows_take(&v->cut[c], lists + (size_t)(4 + c) * m, cnt[4 + c], Ap, Ai, Ax, v->diag);
    }
    free(lists);
    if (rc) return -1;
  }
  if (Pp) {
    const int pn = Pp[m];
    v->Pp = (int*)copy(Pp, sizeof(int) * (size_t)(m + 1));
    v->Pi = (int*)copy(Pi, sizeof(int) * (size_t)pn);
    v->Px = (double*)copy(Px, sizeof(double) * (size_t)pn);
    v->Tp = (int*)copy(Tp, sizeof(int) * (size_t)(mc + 1));
    v->Ti = (int*)copy(Ti, sizeof(int) * (size_t)Tp[mc]);
    v->Tx = (double*)copy(Tx, sizeof(double) * (size_t)Tp[mc]);
    if (!v->Pp || !v->Pi || !v->Px || !v->Tp || !v->Ti || !v->Tx) return -1;
  }
  if (l == h->nlev - 1) {
    /* dense Cholesky A_dd = L L^T on the DOFs (textbook, column by column) */
    const int d = v->ndof;
    double* L = (double*)calloc((size_t)d * (size_t)d + 1, sizeof(double));
    int* pos = (int*)malloc(sizeof(int) * (size_t)m);
    if (!L || !pos) { free(L); free(pos); return -1; }
    for (int k = 0; k < m; ++k) pos[k] = -1;
    for (int a = 0; a < d; ++a) pos[v->dofs[a]] = a;
    for (int a = 0; a < d; ++a) {
      const int k = v->dofs[a];
      for (int q = Ap[k]; q < Ap[k + 1]; ++q)
        if (pos[Ai[q]] >= 0) L[(size_t)a * d + pos[Ai[q]]] += Ax[q];
    }
    free(pos);
    for (int j = 0; j < d; ++j) {
      double s = L[(size_t)j * d + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)j * d + k] * L[(size_t)j * d + k];
      if (!(s > 0.0)) { free(L); return -2; }
      const double ljj = sqrt(s);
      L[(size_t)j * d + j] = ljj;
      for (int i = j + 1; i < d; ++i) {
        double t = L[(size_t)i * d + j];
        for (int k = 0; k < j; ++k) t -= L[(size_t)i * d + k] * L[(size_t)j * d + k];
        L[(size_t)i * d + j] = t / ljj;
      }
    }
    v->L = L;
  }
  return 0;
}

/* sum_j A_kj u_j over row a of a node set, in the stored order */
static double row_dot(const rows_t* R, int a, const double* u) {
  double s = 0.0;
  for (int q = R->p[a]; q < R->p[a + 1]; ++q) s += R->x[q] * u[R->i[q]];
  return s;
}

/* one colour-ordered Gauss-Seidel sweep over the DOFs (cut = 0) or the
 * cut-cell vertices (cut = 1) */
static void gs_sweep(const level_t* v, double* u, const double* F, int cut) {
  for (int c = 0; c < 4; ++c) {
    const rows_t* R = cut ? &v->cut[c] : &v->col[c];
    const int cnt = R->cnt;
#pragma omp parallel for schedule(static)
    for (int a = 0; a < cnt; ++a) {
      const int k = R->idx[a];
      u[k] += (F[k] - row_dot(R, a, u)) / R->diag[a];
    }
  }
}

/* r = F - A u on the DOFs; r = F elsewhere (the rows of other nodes are
 * empty) */
static void residual(const level_t* v, const double* u, const double* F, double* r) {
  memcpy(r, F, sizeof(double) * (size_t)v->m);
  const rows_t* R = &v->all;
#pragma omp parallel for schedule(static)
  for (int a = 0; a < R->cnt; ++a) {
    const int k = R->idx[a];
    r[k] = F[k] - row_dot(R, a, u);
  }
}

static void coarsest_solve(const level_t* v, const double* F, double* u) {
  const int d = v->ndof;
  const double* L = v->L;
  double* y = (double*)malloc(sizeof(double) * (size_t)(d + 1));
  if (!y) return;
  for (int i = 0; i < d; ++i) {
    double s = F[v->dofs[i]];
    for (int k = 0; k < i; ++k) s -= L[(size_t)i * d + k] * y[k];
    y[i] = s / L[(size_t)i * d + i];
  }
  for (int i = d - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < d; ++k) s -= L[(size_t)k * d + i] * y[k];
    y[i] = s / L[(size_t)i * d + i];
  }
  memset(u, 0, sizeof(double) * (size_t)v->m);
  for (int i = 0; i < d; ++i) u[v->dofs[i]] = y[i];
  free(y);
}

static void cycle(hier_t* h, int l, double* u, const double* F, int nu1, int nu2, int eta) {
  level_t* v = &h->lev[l];
  if (l == h->nlev - 1) {
    coarsest_solve(v, F, u);
    return;
  }
  for (int s = 0; s < nu1; ++s) {
    gs_sweep(v, u, F, 0);
    for (int e = 0; e < eta; ++e) gs_sweep(v, u, F, 1);
  }
  level_t* w = &h->lev[l + 1];
  residual(v, u, F, v->r);
  /* F_2h = P^T r (rows of P^T over the coarse nodes) */
#pragma omp parallel for schedule(static)
  for (int K = 0; K < w->m; ++K) {
    double s = 0.0;
    for (int q = v->Tp[K]; q < v->Tp[K + 1]; ++q) s += v->Tx[q] * v->r[v->Ti[q]];
    w->F[K] = s;
  }
  memset(w->u, 0, sizeof(double) * (size_t)w->m);
  cycle(h, l + 1, w->u, w->F, nu1, nu2, eta);
  /* u += P e */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < v->m; ++k) {
    double s = 0.0;
    for (int q = v->Pp[k]; q < v->Pp[k + 1]; ++q) s += v->Px[q] * w->u[v->Pi[q]];
    u[k] += s;
  }
  for (int s = 0; s < nu2; ++s) {
    gs_sweep(v, u, F, 0);
    for (int e = 0; e < eta; ++e) gs_sweep(v, u, F, 1);
  }
}

static double rel_residual(hier_t* h, const double* u, const double* F, double Fn) {
  level_t* v = &h->lev[0];
  residual(v, u, F, v->r);
  double rmax = 0.0;
#pragma omp parallel for reduction(max : rmax) schedule(static)
  for (int a = 0; a < v->ndof; ++a) {
    const double x = fabs(v->r[v->dofs[a]]);
    if (x > rmax) rmax = x;
  }
  return rmax / Fn;
}

static void set_threads(int threads) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
}

/* Exactly k cycles from u (in/out) with right-hand side F. */
int vc_cycles(void* hp, const double* F, double* u, int k, int nu1, int nu2, int eta,
              int threads) {
  hier_t* h = (hier_t*)hp;
  set_threads(threads);
  for (int s = 0; s < k; ++s) cycle(h, 0, u, F, nu1, nu2, eta);
  return 0;
}

/* Cycles from u until ||F - A u||_inf / ||F||_inf <= tol over the DOFs (the
 * residual checked after every cycle) or max_cycles; u = 0 off the DOFs on
 * entry.  hist (max_cycles + 1 doubles or NULL) gets the relative residuals.
 * Returns the cycles run, or -1 if tol was not reached. */
int vc_solve(void* hp, const double* F, double* u, double tol, int max_cycles, int nu1, int nu2,
             int eta, int threads, double* hist) {
  hier_t* h = (hier_t*)hp;
  level_t* v = &h->lev[0];
  set_threads(threads);
  double Fn = 0.0;
  for (int a = 0; a < v->ndof; ++a) {
    const double x = fabs(F[v->dofs[a]]);
    if (x > Fn) Fn = x;
  }
  if (Fn == 0.0) {
    memset(u, 0, sizeof(double) * (size_t)v->m);
    if (hist) hist[0] = 0.0;
    return 0;
  }
  double rel = rel_residual(h, u, F, Fn);
  if (hist) hist[0] = rel;
  int k = 0;
  while (rel > tol && k < max_cycles) {
    cycle(h, 0, u, F, nu1, nu2, eta);
    ++k;
    rel = rel_residual(h, u, F, Fn);
    if (hist) hist[k] = rel;
  }
  return rel <= tol ? k : -1;
}

/* Threads an OpenMP parallel region gets with `threads` requested (0: the
 * default). */
int vc_threads(int threads) {
  int n = 1;
#ifdef _OPENMP
  set_threads(threads);
#pragma omp parallel
  {
#pragma omp single
    n = omp_get_num_threads();
  }
#else
  (void)threads;
#endif
  return n;
}
