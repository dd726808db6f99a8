/*
 * csolve.c - the oracle's solve phase in plain C (FP64, OpenMP over rows).
 *
 * TEST INFRASTRUCTURE ONLY: built and called by oracle/csolve.py, which only
 * tests/, __graft_entry__.smoke() and bench.py's CPU legs use.  It shares no
 * code with the CUDA library.  It computes exactly what oracle/solve.py
 * computes, written out again as plain loops so that the oracle runs on many
 * host cores:
 *
 *  - Galerkin product A_{l+1} = P_l^T A_l P_l (Sec. 3 and Sec. 6): the block
 *    pattern of every (coarse row I, coarse column J) that some path
 *    I -R- i -A- j -P- J reaches (no dropping, columns ascending), values
 *    sum_{i, j} R_Ii A_ij P_jJ with R = P^T given explicitly;
 *  - block products y = M x, the residual b - A x, the block-l1 Jacobi sweep
 *    x + M^+ (b - A x) with the blocks M^+ supplied (Sec. 7), restriction
 *    R r and prolongation x + P e (Algorithm tg);
 *  - the block-l1 hybrid Gauss-Seidel sweep (the hybrid member of Sec. 7's
 *    block-l1 smoother family, one processor block per colour class): the
 *    colour classes in increasing (forward) or decreasing (backward) order,
 *    the rows of a class take x_v + M_v^+ (b - A x)_v with x as the classes
 *    before left it, Jacobi-wise inside the class; classes and M_v^+
 *    supplied;
 *  - the coarsest solve with a supplied lower Cholesky factor L of
 *    A_L + (I - E_L E_L^T) (Sec. 3 after Lemma eet_is_diag): L L^T x = b;
 *  - the V-cycle (Algorithm tg applied recursively, one pre- and one post-
 *    sweep from x = 0; with Gauss-Seidel a forward sweep before the coarse
 *    correction and a backward one after it) and CG preconditioned by it
 *    (Sec. 7), stopping when ||r|| <= rtol ||f|| (recurrence residual).
 *
 * Matrices are BSR: rowptr (int64, n_rows+1), colidx (int32), values
 * row-major br x bc per block.  Vectors are interleaved per block row.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int n_rows, n_cols, br, bc;
  const int64_t *rp;
  const int32_t *ci;
  const double *v;
} oc_bsr;

void oc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Galerkin product: symbolic pass (row lengths), then columns and values.
 * ---------------------------------------------------------------------- */

/* Sorted distinct coarse columns of row I into cols (returns their count);
 * mark is an n_cols scratch array of -1 entries (restored on return). */
static int row_pattern(const oc_bsr *R, const oc_bsr *A, const oc_bsr *P, int I, int32_t *mark,
                       int32_t *cols) {
  int m = 0;
  for (int64_t p = R->rp[I]; p < R->rp[I + 1]; ++p) {
    const int i = R->ci[p];
    for (int64_t q = A->rp[i]; q < A->rp[i + 1]; ++q) {
      const int j = A->ci[q];
      for (int64_t s = P->rp[j]; s < P->rp[j + 1]; ++s) {
        const int J = P->ci[s];
        if (mark[J] < 0) {
          mark[J] = 1;
          cols[m++] = J;
        }
      }
    }
  }
  /* insertion sort is enough for the short coarse rows; mark back to -1 */
  for (int a = 1; a < m; ++a) {
    const int32_t x = cols[a];
    int b = a - 1;
    while (b >= 0 && cols[b] > x) {
      cols[b + 1] = cols[b];
      --b;
    }
    cols[b + 1] = x;
  }
  for (int a = 0; a < m; ++a) mark[cols[a]] = -1;
  return m;
}

/* Row lengths of C = R A P into crp[1..nc] (crp[0] = 0 and the prefix sum
 * are left to the caller); returns 0, or -1 if scratch memory ran out. */
int oc_galerkin_rows(int nc_rows, int nc_cols, const int64_t *Rrp, const int32_t *Rci,
                     int nf, const int64_t *Arp, const int32_t *Aci, const int64_t *Prp,
                     const int32_t *Pci, int64_t *crp) {
  oc_bsr R = {nc_rows, nf, 0, 0, Rrp, Rci, 0}, A = {nf, nf, 0, 0, Arp, Aci, 0},
         P = {nf, nc_cols, 0, 0, Prp, Pci, 0};
  int fail = 0;
#pragma omp parallel
  {
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc_cols > 0 ? nc_cols : 1));
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc_cols > 0 ? nc_cols : 1));
    const int ok = mark && cols;
    if (!ok) {
#pragma omp atomic write
      fail = 1;
    } else {
      for (int J = 0; J < nc_cols; ++J) mark[J] = -1;
    }
    /* every thread takes part in the loop (a work-sharing construct), one
     * without scratch memory only skips its rows */
#pragma omp for schedule(dynamic, 64)
    for (int I = 0; I < nc_rows; ++I)
      if (ok) crp[I + 1] = row_pattern(&R, &A, &P, I, mark, cols);
    free(mark);
    free(cols);
  }
  return fail ? -1 : 0;
}

/* Columns and values of C = R A P (kc x kc blocks) given its row pointers
 * crp; R is kc x kf per block, A kf x kf, P kf x kc. */
int oc_galerkin_fill(int nc_rows, int nc_cols, int kf, int kc, const int64_t *Rrp,
                     const int32_t *Rci, const double *Rv, int nf, const int64_t *Arp,
                     const int32_t *Aci, const double *Av, const int64_t *Prp, const int32_t *Pci,
                     const double *Pv, const int64_t *crp, int32_t *cci, double *cv) {
  oc_bsr R = {nc_rows, nf, kc, kf, Rrp, Rci, Rv}, A = {nf, nf, kf, kf, Arp, Aci, Av},
         P = {nf, nc_cols, kf, kc, Prp, Pci, Pv};
  int fail = 0;
#pragma omp parallel
  {
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc_cols > 0 ? nc_cols : 1));
    double *T = (double *)malloc(sizeof(double) * (size_t)(kc * kf));
    const int ok = mark && T;
    if (!ok) {
#pragma omp atomic write
      fail = 1;
    } else {
      for (int J = 0; J < nc_cols; ++J) mark[J] = -1;
    }
#pragma omp for schedule(dynamic, 64)
    for (int I = 0; I < nc_rows; ++I) {
      if (ok) {
        int32_t *cols = cci + crp[I];
        double *out = cv + (size_t)crp[I] * kc * kc;
        const int m = row_pattern(&R, &A, &P, I, mark, cols);
        for (int a = 0; a < m; ++a) mark[cols[a]] = a;
        memset(out, 0, sizeof(double) * (size_t)m * kc * kc);
        for (int64_t p = R.rp[I]; p < R.rp[I + 1]; ++p) {
          const int i = R.ci[p];
          const double *Rb = R.v + (size_t)p * kc * kf;
          for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
            const int j = A.ci[q];
            const double *Ab = A.v + (size_t)q * kf * kf;
            /* T = R_Ii A_ij (kc x kf) */
            for (int r = 0; r < kc; ++r)
              for (int c = 0; c < kf; ++c) {
                double s = 0.0;
                for (int t = 0; t < kf; ++t) s += Rb[r * kf + t] * Ab[t * kf + c];
                T[r * kf + c] = s;
              }
            for (int64_t s2 = P.rp[j]; s2 < P.rp[j + 1]; ++s2) {
              const int J = P.ci[s2];
              const double *Pb = P.v + (size_t)s2 * kf * kc;
              double *C = out + (size_t)mark[J] * kc * kc;
              /* C_IJ += T P_jJ */
              for (int r = 0; r < kc; ++r)
                for (int c = 0; c < kc; ++c) {
                  double s = 0.0;
                  for (int t = 0; t < kf; ++t) s += T[r * kf + t] * Pb[t * kc + c];
                  C[r * kc + c] += s;
                }
            }
          }
        }
        for (int a = 0; a < m; ++a) mark[cols[a]] = -1;
      }
    }
    free(mark);
    free(T);
  }
  return fail ? -1 : 0;
}

/* ------------------------------------------------------------------------
 * Solve phase
 * ---------------------------------------------------------------------- */

/* y = M x (+ y if add) */
static void bsr_apply(const oc_bsr *M, const double *x, double *y, int add) {
  const int br = M->br, bc = M->bc;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < M->n_rows; ++i) {
    double acc[8];
    for (int r = 0; r < br; ++r) acc[r] = add ? y[(size_t)i * br + r] : 0.0;
    for (int64_t p = M->rp[i]; p < M->rp[i + 1]; ++p) {
      const double *B = M->v + (size_t)p * br * bc;
      const double *xj = x + (size_t)M->ci[p] * bc;
      for (int r = 0; r < br; ++r)
        for (int c = 0; c < bc; ++c) acc[r] += B[r * bc + c] * xj[c];
    }
    for (int r = 0; r < br; ++r) y[(size_t)i * br + r] = acc[r];
  }
}

/* out = x + M^+ (b - A x); x == NULL means x = 0 (out = M^+ b) */
static void smooth(const oc_bsr *A, const double *Minv, const double *b, const double *x,
                   double *out) {
  const int k = A->br;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < A->n_rows; ++i) {
    double res[8];
    for (int r = 0; r < k; ++r) res[r] = b[(size_t)i * k + r];
    if (x) {
      for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
        const double *B = A->v + (size_t)p * k * k;
        const double *xj = x + (size_t)A->ci[p] * k;
        for (int r = 0; r < k; ++r)
          for (int c = 0; c < k; ++c) res[r] -= B[r * k + c] * xj[c];
      }
    }
    const double *Mi = Minv + (size_t)i * k * k;
    for (int r = 0; r < k; ++r) {
      double u = 0.0;
      for (int c = 0; c < k; ++c) u += Mi[r * k + c] * res[c];
      out[(size_t)i * k + r] = (x ? x[(size_t)i * k + r] : 0.0) + u;
    }
  }
}

/* One block-l1 hybrid Gauss-Seidel sweep on x (in place): class c holds
 * the rows rows[ptr[c] .. ptr[c+1]); forward visits the classes 0, 1, ...,
 * backward the reverse.  The residuals of a class are all taken before any
 * of its rows changes (Jacobi-wise inside a class), into tmp (n_rows x k,
 * indexed by the position in rows). */
static void gs_sweep(const oc_bsr *A, const double *Minv, int n_cls, const int32_t *ptr,
                     const int32_t *rows, const double *b, double *x, double *tmp, int forward) {
  const int k = A->br;
  for (int s = 0; s < n_cls; ++s) {
    const int c = forward ? s : n_cls - 1 - s;
#pragma omp parallel for schedule(static)
    for (int q = ptr[c]; q < ptr[c + 1]; ++q) {
      const int i = rows[q];
      double *res = tmp + (size_t)q * k;
      for (int r = 0; r < k; ++r) res[r] = b[(size_t)i * k + r];
      for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
        const double *B = A->v + (size_t)p * k * k;
        const double *xj = x + (size_t)A->ci[p] * k;
        for (int r = 0; r < k; ++r)
          for (int cc = 0; cc < k; ++cc) res[r] -= B[r * k + cc] * xj[cc];
      }
    }
#pragma omp parallel for schedule(static)
    for (int q = ptr[c]; q < ptr[c + 1]; ++q) {
      const int i = rows[q];
      const double *Mi = Minv + (size_t)i * k * k;
      const double *res = tmp + (size_t)q * k;
      for (int r = 0; r < k; ++r) {
        double u = 0.0;
        for (int cc = 0; cc < k; ++cc) u += Mi[r * k + cc] * res[cc];
        x[(size_t)i * k + r] += u;
      }
    }
  }
}

/* r = b - A x */
static void residual(const oc_bsr *A, const double *b, const double *x, double *r) {
  const int k = A->br;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < A->n_rows; ++i) {
    double acc[8];
    for (int q = 0; q < k; ++q) acc[q] = b[(size_t)i * k + q];
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      const double *B = A->v + (size_t)p * k * k;
      const double *xj = x + (size_t)A->ci[p] * k;
      for (int q = 0; q < k; ++q)
        for (int c = 0; c < k; ++c) acc[q] -= B[q * k + c] * xj[c];
    }
    for (int q = 0; q < k; ++q) r[(size_t)i * k + q] = acc[q];
  }
}

/* L L^T x = b, L dense lower triangular (row-major n x n) */
static void cholesky_solve(int n, const double *L, const double *b, double *x) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int j = 0; j < i; ++j) s -= L[(size_t)i * n + j] * x[j];
    x[i] = s / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int j = i + 1; j < n; ++j) s -= L[(size_t)j * n + i] * x[j];
    x[i] = s / L[(size_t)i * n + i];
  }
}

typedef struct {
  int n_levels;
  oc_bsr *A, *P, *R;       /* A[0..L-1], P/R[0..L-2] */
  const double **Minv;     /* per level but the coarsest */
  const int *n_cls;        /* colour classes per level (NULL: block-l1 Jacobi) */
  const int32_t *const *cls_ptr, *const *cls_rows; /* class c of level l: rows
                              cls_rows[l][cls_ptr[l][c] .. cls_ptr[l][c+1]) */
  int nc;                  /* coarsest size (scalar) */
  const double *Lc;        /* coarsest Cholesky factor */
  double **b, **x, **t, **e; /* work vectors per level */
} oc_hier;

static void vcycle(const oc_hier *H, int l, const double *b, double *y) {
  if (l == H->n_levels - 1) {
    cholesky_solve(H->nc, H->Lc, b, y);
    return;
  }
  const oc_bsr *A = &H->A[l];
  const size_t n = (size_t)A->n_rows * A->br;
  double *x = H->x[l], *t = H->t[l];
  if (H->n_cls) {                                     /* hybrid Gauss-Seidel */
    const int nc = H->n_cls[l];
    memset(x, 0, n * sizeof(double));
    gs_sweep(A, H->Minv[l], nc, H->cls_ptr[l], H->cls_rows[l], b, x, t, 1);
    residual(A, b, x, t);
    bsr_apply(&H->R[l], t, H->b[l + 1], 0);
    vcycle(H, l + 1, H->b[l + 1], H->e[l + 1]);
    bsr_apply(&H->P[l], H->e[l + 1], x, 1);
    gs_sweep(A, H->Minv[l], nc, H->cls_ptr[l], H->cls_rows[l], b, x, t, 0);
    memcpy(y, x, n * sizeof(double));
    return;
  }
  smooth(A, H->Minv[l], b, NULL, x);                  /* pre-smoothing from 0 */
  residual(A, b, x, t);                               /* t = b - A x */
  bsr_apply(&H->R[l], t, H->b[l + 1], 0);             /* restriction */
  vcycle(H, l + 1, H->b[l + 1], H->e[l + 1]);         /* coarse correction */
  bsr_apply(&H->P[l], H->e[l + 1], x, 1);             /* x += P e */
  smooth(A, H->Minv[l], b, x, t);                     /* post-smoothing */
  memcpy(y, t, n * sizeof(double));
}

static double dot(size_t n, const double *a, const double *b) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Arrays of level l are passed flattened: Arp[l], Aci[l], Av[l] etc.;
 * n_cls NULL selects block-l1 Jacobi, else n_cls[l] colour classes with
 * cls_ptr[l] / cls_rows[l] select hybrid Gauss-Seidel (Minv then holds its
 * blocks).  Returns the iteration count (or -1 on allocation failure); hist
 * receives the relative residual after every iteration (maxit + 1 entries). */
int oc_pcg(int n_levels, const int *nrows, const int *k, const int64_t *const *Arp,
           const int32_t *const *Aci, const double *const *Av, const int64_t *const *Prp,
           const int32_t *const *Pci, const double *const *Pv, const int64_t *const *Rrp,
           const int32_t *const *Rci, const double *const *Rv, const double *const *Minv,
           const int *n_cls, const int32_t *const *cls_ptr, const int32_t *const *cls_rows,
           const double *Lc, const double *f, double *x, double rtol, int maxit, double *hist) {
  oc_hier H;
  H.n_levels = n_levels;
  H.A = (oc_bsr *)calloc((size_t)n_levels, sizeof(oc_bsr));
  H.P = (oc_bsr *)calloc((size_t)n_levels, sizeof(oc_bsr));
  H.R = (oc_bsr *)calloc((size_t)n_levels, sizeof(oc_bsr));
  H.Minv = (const double **)calloc((size_t)n_levels, sizeof(double *));
  H.b = (double **)calloc((size_t)n_levels, sizeof(double *));
  H.x = (double **)calloc((size_t)n_levels, sizeof(double *));
  H.t = (double **)calloc((size_t)n_levels, sizeof(double *));
  H.e = (double **)calloc((size_t)n_levels, sizeof(double *));
  int ok = H.A && H.P && H.R && H.Minv && H.b && H.x && H.t && H.e;
  for (int l = 0; ok && l < n_levels; ++l) {
    H.A[l] = (oc_bsr){nrows[l], nrows[l], k[l], k[l], Arp[l], Aci[l], Av[l]};
    if (l + 1 < n_levels) {
      H.P[l] = (oc_bsr){nrows[l], nrows[l + 1], k[l], k[l + 1], Prp[l], Pci[l], Pv[l]};
      H.R[l] = (oc_bsr){nrows[l + 1], nrows[l], k[l + 1], k[l], Rrp[l], Rci[l], Rv[l]};
      H.Minv[l] = Minv[l];
    }
    const size_t n = (size_t)nrows[l] * k[l] + 1;
    H.b[l] = (double *)malloc(n * sizeof(double));
    H.x[l] = (double *)malloc(n * sizeof(double));
    H.t[l] = (double *)malloc(n * sizeof(double));
    H.e[l] = (double *)malloc(n * sizeof(double));
    ok = ok && H.b[l] && H.x[l] && H.t[l] && H.e[l];
  }
  H.nc = nrows[n_levels - 1] * k[n_levels - 1];
  H.Lc = Lc;
  H.n_cls = n_cls;
  H.cls_ptr = cls_ptr;
  H.cls_rows = cls_rows;
  const size_t n = (size_t)nrows[0] * k[0];
  double *r = (double *)malloc((n + 1) * sizeof(double));
  double *z = (double *)malloc((n + 1) * sizeof(double));
  double *p = (double *)malloc((n + 1) * sizeof(double));
  double *q = (double *)malloc((n + 1) * sizeof(double));
  int it = -1;
  if (ok && r && z && p && q) {
    residual(&H.A[0], f, x, r);
    const double nf = sqrt(dot(n, f, f));
    /* relative residual; for f = 0 the rule ||r|| <= rtol ||f|| asks r = 0 */
    double h = nf > 0 ? sqrt(dot(n, r, r)) / nf : sqrt(dot(n, r, r));
    hist[0] = h;
    it = 0;
    double rho_old = 0.0;
    while ((nf > 0 ? h > rtol : h > 0.0) && it < maxit) {
      vcycle(&H, 0, r, z);
      const double rho = dot(n, r, z);
      const double beta = it == 0 ? 0.0 : rho / rho_old;
#pragma omp parallel for schedule(static)
      for (size_t i = 0; i < n; ++i) p[i] = it == 0 ? z[i] : z[i] + beta * p[i];
      bsr_apply(&H.A[0], p, q, 0);
      const double alpha = rho / dot(n, p, q);
#pragma omp parallel for schedule(static)
      for (size_t i = 0; i < n; ++i) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
      }
      rho_old = rho;
      ++it;
      h = nf > 0 ? sqrt(dot(n, r, r)) / nf : sqrt(dot(n, r, r));
      hist[it] = h;
    }
  }
  free(r);
  free(z);
  free(p);
  free(q);
  for (int l = 0; l < n_levels; ++l) {
    if (H.b) free(H.b[l]);
    if (H.x) free(H.x[l]);
    if (H.t) free(H.t[l]);
    if (H.e) free(H.e[l]);
  }
  free(H.A);
  free(H.P);
  free(H.R);
  free(H.Minv);
  free(H.b);
  free(H.x);
  free(H.t);
  free(H.e);
  return it;
}

/* One V-cycle z = B^{-1} r (same arrays as oc_pcg). */
int oc_vcycle(int n_levels, const int *nrows, const int *k, const int64_t *const *Arp,
              const int32_t *const *Aci, const double *const *Av, const int64_t *const *Prp,
              const int32_t *const *Pci, const double *const *Pv, const int64_t *const *Rrp,
              const int32_t *const *Rci, const double *const *Rv, const double *const *Minv,
              const int *n_cls, const int32_t *const *cls_ptr, const int32_t *const *cls_rows,
              const double *Lc, const double *r, double *z) {
  oc_hier H;
  H.n_levels = n_levels;
  oc_bsr Ab[64], Pb[64], Rb[64];
  const double *Mb[64];
  double *bb[64], *xb[64], *tb[64], *eb[64];
  if (n_levels > 64) return -1;
  H.A = Ab;
  H.P = Pb;
  H.R = Rb;
  H.Minv = Mb;
  H.b = bb;
  H.x = xb;
  H.t = tb;
  H.e = eb;
  int ok = 1;
  for (int l = 0; l < n_levels; ++l) {
    Ab[l] = (oc_bsr){nrows[l], nrows[l], k[l], k[l], Arp[l], Aci[l], Av[l]};
    if (l + 1 < n_levels) {
      Pb[l] = (oc_bsr){nrows[l], nrows[l + 1], k[l], k[l + 1], Prp[l], Pci[l], Pv[l]};
      Rb[l] = (oc_bsr){nrows[l + 1], nrows[l], k[l + 1], k[l], Rrp[l], Rci[l], Rv[l]};
      Mb[l] = Minv[l];
    }
    const size_t n = (size_t)nrows[l] * k[l] + 1;
    bb[l] = (double *)malloc(n * sizeof(double));
    xb[l] = (double *)malloc(n * sizeof(double));
    tb[l] = (double *)malloc(n * sizeof(double));
    eb[l] = (double *)malloc(n * sizeof(double));
    ok = ok && bb[l] && xb[l] && tb[l] && eb[l];
  }
  H.nc = nrows[n_levels - 1] * k[n_levels - 1];
  H.Lc = Lc;
  H.n_cls = n_cls;
  H.cls_ptr = cls_ptr;
  H.cls_rows = cls_rows;
  if (ok) vcycle(&H, 0, r, z);
  for (int l = 0; l < n_levels; ++l) {
    free(bb[l]);
    free(xb[l]);
    free(tb[l]);
    free(eb[l]);
  }
  return ok ? 0 : -1;
}

/* y = A x for one BSR matrix (a single step, for pins). */
void oc_spmv(int n_rows, int n_cols, int br, int bc, const int64_t *rp, const int32_t *ci,
             const double *v, const double *x, double *y) {
  const oc_bsr M = {n_rows, n_cols, br, bc, rp, ci, v};
  bsr_apply(&M, x, y, 0);
}
