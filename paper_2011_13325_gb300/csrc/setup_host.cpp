// Host setup of the hierarchy (the part of the method that precedes the
// solve phase): finest edge matrices (Thm. deng_elast and its Remark),
// Algorithm 1 "successive matching" with the measures mu_D, mu_s, mu_p and
// mu_g (Sec. 5), coarse edge/vertex matrices (Thm. cemats), tentative
// prolongation (Def. pwp / pwp_el) and the auxiliary smoothed prolongation
// (Def. aux_sp, Sec. 6).  The Galerkin products between levels run on the
// device (galerkin.cu).  The readings where the paper is silent (sigma,
// omega, the S / A split, the filtered neighbours, the coarse size) are the
// ones documented with amg_setup_params in include/amg.h.
//
// mu_g is checked, as the paper suggests after Thm. mu1, by a semidefinite
// Cholesky factorisation of sigma * R - L instead of an eigen-solve.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <queue>
#include <array>
#include <chrono>
#include <unordered_map>

#ifdef _OPENMP
#include <omp.h>
#endif
#include <vector>

#include "setup_host.h"

namespace amgsetup {

// ------------------------------------------------------------------ small dense algebra

using Mat = std::vector<double>;  // row-major, size n*n (n <= 6 here unless noted)

static inline int kdim(int d) { return d + d * (d - 1) / 2; }

// Q(t) = [[I, Skew(t)], [0, I]] (Sec. 3, eq. qij_epseps)
static void qmat(int d, const double *t, double *q) {
  const int k = kdim(d);
  for (int i = 0; i < k * k; ++i) q[i] = 0.0;
  for (int i = 0; i < k; ++i) q[i * k + i] = 1.0;
  if (d == 1) return;  // the scalar problem: Q = 1
  if (d == 2) {
    q[0 * k + 2] = -t[1];
    q[1 * k + 2] = t[0];
  } else {
    // Skew(t) r = t x r
    q[0 * k + 4] = -t[2];
    q[0 * k + 5] = t[1];
    q[1 * k + 3] = t[2];
    q[1 * k + 5] = -t[0];
    q[2 * k + 3] = -t[1];
    q[2 * k + 4] = t[0];
  }
}

// C = A B (n x m)(m x p)
static void mm(const double *A, const double *B, double *C, int n, int m, int p) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < p; ++j) {
      double s = 0.0;
      for (int l = 0; l < m; ++l) s += A[i * m + l] * B[l * p + j];
      C[i * p + j] = s;
    }
}

// C = A^T B (A: m x n, B: m x p) -> n x p
static void mtm(const double *A, const double *B, double *C, int m, int n, int p) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < p; ++j) {
      double s = 0.0;
      for (int l = 0; l < m; ++l) s += A[l * n + i] * B[l * p + j];
      C[i * p + j] = s;
    }
}

// S = Skew(t) as a d x (k-d) block
static void skew_block(int d, const double *t, double *S) {
  if (d == 1) return;  // no rotations
  if (d == 2) {
    S[0] = -t[1];
    S[1] = t[0];
  } else {
    S[0] = 0.0;   S[1] = -t[2]; S[2] = t[1];
    S[3] = t[2];  S[4] = 0.0;   S[5] = -t[0];
    S[6] = -t[1]; S[7] = t[0];  S[8] = 0.0;
  }
}

// Q(t1)^T X Q(t2) in closed form: with X = [[A, B], [B^T, C]] (blocks d x d,
// d x r, r x r; r = k - d) and S_i = Skew(t_i),
//   [[A, A S2 + B], [S1^T A + B^T, S1^T A S2 + S1^T B + B^T S2 + C]].
// (B^T here is X's lower-left block; X need not be symmetric.)
static void transport2(int d, const double *t1, const double *t2, const double *X, double *out) {
  const int k = kdim(d), r = k - d;
  double S1[9], S2[9], AS2[18], BL[18];
  skew_block(d, t1, S1);
  skew_block(d, t2, S2);
  // A S2 (d x r)
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < r; ++j) {
      double s = 0.0;
      for (int l = 0; l < d; ++l) s += X[i * k + l] * S2[l * r + j];
      AS2[i * r + j] = s;
    }
  // S1^T A (r x d)
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int l = 0; l < d; ++l) s += S1[l * r + i] * X[l * k + j];
      BL[i * d + j] = s;
    }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) out[i * k + j] = X[i * k + j];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < r; ++j) out[i * k + d + j] = AS2[i * r + j] + X[i * k + d + j];
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < d; ++j) out[(d + i) * k + j] = BL[i * d + j] + X[(d + i) * k + j];
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) {
      double s = X[(d + i) * k + d + j];
      for (int l = 0; l < d; ++l) {
        s += S1[l * r + i] * AS2[l * r + j];      // S1^T A S2
        s += S1[l * r + i] * X[l * k + d + j];    // S1^T B
        s += X[(d + i) * k + l] * S2[l * r + j];  // B^T S2 (lower-left block of X)
      }
      out[(d + i) * k + d + j] = s;
    }
}

// Q^T X Q for the shift t (k x k)
static void transport(int d, const double *t, const double *X, double *out) {
  transport2(d, t, t, X, out);
}

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (Golub & Van
// Loan, Sec. 8.5); w eigenvalues, V eigenvectors in columns.
static void sym_eig(int n, const double *A, double *w, double *V) {
  double a[36];
  for (int i = 0; i < n * n; ++i) a[i] = A[i];
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double m = 0.5 * (a[i * n + j] + a[j * n + i]);
      a[i * n + j] = a[j * n + i] = m;
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int i = 0; i < n * n; ++i) fro += a[i] * a[i];
  for (int sweep = 0; sweep < 60 && fro > 0.0; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += a[p * n + q] * a[p * n + q];
    if (off <= 1e-34 * fro) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[p * n + q];
        if (fabs(apq) <= 1e-300) continue;
        const double th = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int r = 0; r < n; ++r) {
          const double x = a[r * n + p], y = a[r * n + q];
          a[r * n + p] = c * x - s * y;
          a[r * n + q] = s * x + c * y;
        }
        for (int r = 0; r < n; ++r) {
          const double x = a[p * n + r], y = a[q * n + r];
          a[p * n + r] = c * x - s * y;
          a[q * n + r] = s * x + c * y;
        }
        for (int r = 0; r < n; ++r) {
          const double x = V[r * n + p], y = V[r * n + q];
          V[r * n + p] = c * x - s * y;
          V[r * n + q] = s * x + c * y;
        }
      }
  }
  for (int i = 0; i < n; ++i) w[i] = a[i * n + i];
}

static void pinv_sym(int n, const double *A, double *out, double rtol = 1e-12) {
  double w[6], V[36];
  sym_eig(n, A, w, V);
  double wmax = 0.0;
  for (int i = 0; i < n; ++i) wmax = std::max(wmax, fabs(w[i]));
  for (int i = 0; i < n * n; ++i) out[i] = 0.0;
  if (wmax <= 0.0) return;
  for (int m = 0; m < n; ++m) {
    if (!(w[m] > rtol * wmax)) continue;
    const double inv = 1.0 / w[m];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) out[i * n + j] += V[i * n + m] * inv * V[j * n + m];
  }
}

// H(A, B) = A (A + B)^+ B (Lemma mu2), symmetrised
static void harmonic(int n, const double *A, const double *B, double *H) {
  double S[36], P[36], T[36];
  for (int i = 0; i < n * n; ++i) S[i] = A[i] + B[i];
  pinv_sym(n, S, P);
  mm(P, B, T, n, n, n);
  mm(A, T, S, n, n, n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) H[i * n + j] = 0.5 * (S[i * n + j] + S[j * n + i]);
}

// smallest mu with L <= mu R (range of R; +inf if L has energy on ker R)
static double gen_lambda_max(int n, const double *L, const double *R) {
  double wl[6], Vl[36], wr[6], Vr[36];
  sym_eig(n, L, wl, Vl);
  double lmax = 0.0;
  for (int i = 0; i < n; ++i) lmax = std::max(lmax, wl[i]);
  if (lmax <= 0.0) return 0.0;
  sym_eig(n, R, wr, Vr);
  double rmax = 0.0;
  for (int i = 0; i < n; ++i) rmax = std::max(rmax, wr[i]);
  if (rmax <= 0.0) return INFINITY;
  int nr = 0, nk = 0;
  double Sr[36], K[36];
  for (int m = 0; m < n; ++m) {
    if (wr[m] > 1e-10 * rmax) {
      const double s = 1.0 / sqrt(wr[m]);
      for (int i = 0; i < n; ++i) Sr[i * n + nr] = Vr[i * n + m] * s;
      ++nr;
    } else {
      for (int i = 0; i < n; ++i) K[i * n + nk] = Vr[i * n + m];
      ++nk;
    }
  }
  double LS[36], C[36], w[6], V[36];
  if (nk > 0) {
    // K^T L K (n x nk columns stored with stride n)
    double Kc[36], LK[36];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < nk; ++j) Kc[i * nk + j] = K[i * n + j];
    mm(L, Kc, LK, n, n, nk);
    mtm(Kc, LK, C, n, nk, nk);
    sym_eig(nk, C, w, V);
    double leak = -INFINITY;
    for (int i = 0; i < nk; ++i) leak = std::max(leak, w[i]);
    if (leak > 1e-8 * lmax) return INFINITY;
  }
  double Sc[36];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < nr; ++j) Sc[i * nr + j] = Sr[i * n + j];
  mm(L, Sc, LS, n, n, nr);
  mtm(Sc, LS, C, n, nr, nr);
  sym_eig(nr, C, w, V);
  double mu = 0.0;
  for (int i = 0; i < nr; ++i) mu = std::max(mu, w[i]);
  return mu;
}

// Positive-semidefiniteness test of a symmetric N x N matrix M = sigma R - L
// (any N) by Cholesky with diagonal pivoting (the largest remaining diagonal
// first, as for semidefinite matrices in Golub & Van Loan, Sec. 4.2.8): the
// factorisation runs while the largest remaining pivot exceeds
// tol = rtol * max|M_ii|; the remaining Schur complement (the common kernel
// of R and L plus rounding) must then vanish to within tol.  Rows made of
// rounding noise are never used as pivots, so coefficient jumps of many
// orders of magnitude do not spoil the test.
static bool psd_cholesky(int N, std::vector<double> &A, double rtol) {
  // only the lower triangle (i >= l) of A is read and updated
  double scale = 0.0;
  for (int i = 0; i < N; ++i) scale = std::max(scale, fabs(A[(size_t)i * N + i]));
  const double tol = rtol * scale;
  auto at = [&](int i, int l) -> double & { return A[(size_t)i * N + l]; };
  std::vector<double> colj;
  for (int j = 0; j < N; ++j) {
    int p = j;
    for (int i = j + 1; i < N; ++i)
      if (at(i, i) > at(p, p)) p = i;
    if (at(p, p) <= tol) {
      for (int l = j; l < N; ++l)
        for (int i = l; i < N; ++i)
          if (fabs(at(i, l)) > 10.0 * tol) return false;
      return true;
    }
    if (p != j) {  // symmetric exchange of rows/columns j and p (lower triangle)
      std::swap(at(j, j), at(p, p));
      for (int l = 0; l < j; ++l) std::swap(at(j, l), at(p, l));
      for (int i = j + 1; i < p; ++i) std::swap(at(i, j), at(p, i));
      for (int i = p + 1; i < N; ++i) std::swap(at(i, j), at(i, p));
    }
    const double ljj = sqrt(at(j, j));
    at(j, j) = ljj;
    for (int i = j + 1; i < N; ++i) at(i, j) /= ljj;
    colj.resize(N);
    for (int i = j + 1; i < N; ++i) colj[i] = at(i, j);
    for (int i = j + 1; i < N; ++i) {
      const double aij = colj[i];
      if (aij == 0.0) continue;
      double *row = &A[(size_t)i * N];
      for (int l = j + 1; l <= i; ++l) row[l] -= aij * colj[l];
    }
  }
  return true;
}

// ------------------------------------------------------------------ topology

void Topo::build_adj() {
  adj_ptr.assign(n + 1, 0);
  const int m = (int)ei.size();
  for (int e = 0; e < m; ++e) {
    adj_ptr[ei[e] + 1]++;
    adj_ptr[ej[e] + 1]++;
  }
  for (int i = 0; i < n; ++i) adj_ptr[i + 1] += adj_ptr[i];
  adj_nbr.assign(adj_ptr[n], 0);
  adj_edge.assign(adj_ptr[n], 0);
  std::vector<int> fill(adj_ptr.begin(), adj_ptr.end() - 1);
  for (int e = 0; e < m; ++e) {
    adj_nbr[fill[ei[e]]] = ej[e];
    adj_edge[fill[ei[e]]++] = e;
    adj_nbr[fill[ej[e]]] = ei[e];
    adj_edge[fill[ej[e]]++] = e;
  }
  // neighbours sorted by id within each vertex (edge ids follow)
  for (int v = 0; v < n; ++v) {
    std::vector<std::pair<int, int>> t;
    for (int p = adj_ptr[v]; p < adj_ptr[v + 1]; ++p) t.push_back({adj_nbr[p], adj_edge[p]});
    std::sort(t.begin(), t.end());
    for (int p = adj_ptr[v], q = 0; p < adj_ptr[v + 1]; ++p, ++q) {
      adj_nbr[p] = t[q].first;
      adj_edge[p] = t[q].second;
    }
  }
}

int Topo::edge(int a, int b) const {
  const int *s = adj_nbr.data() + adj_ptr[a], *e = adj_nbr.data() + adj_ptr[a + 1];
  const int *it = std::lower_bound(s, e, b);
  if (it == e || *it != b) return -1;
  return adj_edge[adj_ptr[a] + (int)(it - s)];
}

// Thm. deng_elast: E^{ij} = c [[t t^T, 0], [0, 0]], c = mean |(A_ij)_lm|, M = 0
Topo finest_topology(int d, int n, const double *coords, const uint8_t *dirichlet,
                     const int32_t *rp, const int32_t *ci, const double *vals) {
  Topo T;
  T.n = n;
  T.d = d;
  T.k = kdim(d);
  const int k = T.k;
  T.pos.assign(coords, coords + (size_t)n * d);
  T.dir.assign(n, 0);
  for (int i = 0; i < n; ++i) T.dir[i] = dirichlet ? (dirichlet[i] != 0) : 0;
  for (int i = 0; i < n; ++i)
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] > i) {
        T.ei.push_back(i);
        T.ej.push_back(ci[p]);
      }
  const size_t m = T.ei.size();
  T.E.assign(m * k * k, 0.0);
  T.M.assign((size_t)n * k * k, 0.0);
  size_t e = 0;
  for (int i = 0; i < n; ++i)
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] > i) {
        const double *blk = vals + (size_t)p * d * d;
        double c = 0.0;
        for (int q = 0; q < d * d; ++q) c += fabs(blk[q]);
        c /= (double)(d * d);
        double t[3];
        for (int a = 0; a < d; ++a) t[a] = coords[(size_t)ci[p] * d + a] - coords[(size_t)i * d + a];
        double *E = T.E.data() + e * k * k;
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) E[a * k + b] = c * t[a] * t[b];
        ++e;
      }
  T.build_adj();
  T.rot_free = true;  // finest elasticity edges: displacement blocks only, M = 0
  return T;
}

// The scalar problem (Sec. 4 after Def. deng): E^{ij} = |A_ij|, M^i =
// max{0, A_ii - sum_{j != i} |A_ij|} over the full matrix.  Its kernel
// transfers are the identity (k = 1), which the topology expresses with one
// coordinate per vertex (kdim(1) = 1), the first of the mesh.
Topo finest_topology_scalar(int dim, int n, const double *coords, const uint8_t *dirichlet,
                            const int32_t *rp, const int32_t *ci, const double *vals) {
  Topo T;
  T.n = n;
  T.d = 1;
  T.k = 1;
  T.pos.resize(n);
  for (int i = 0; i < n; ++i) T.pos[i] = coords[(size_t)i * dim];
  T.dir.assign(n, 0);
  for (int i = 0; i < n; ++i) T.dir[i] = dirichlet ? (dirichlet[i] != 0) : 0;
  T.M.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double diag = 0.0, off = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      if (ci[p] == i)
        diag += vals[p];
      else
        off += fabs(vals[p]);
      if (ci[p] > i) {
        T.ei.push_back(i);
        T.ej.push_back(ci[p]);
        T.E.push_back(fabs(vals[p]));
      }
    }
    T.M[i] = std::max(0.0, diag - off);
  }
  T.build_adj();
  return T;
}

static void half_shift(const Topo &T, int i, int j, double *t) {  // (x_j - x_i)/2
  for (int a = 0; a < T.d; ++a) t[a] = 0.5 * (T.pos[(size_t)j * T.d + a] - T.pos[(size_t)i * T.d + a]);
}

// D-hat_ii = M^i + sum_j Q^{ij,T} E^{ij} Q^{ij}
static std::vector<double> aux_diagonal(const Topo &T) {
  const int k = T.k;
  std::vector<double> D(T.M);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < T.n; ++i) {
    double t[3], X[36];
    for (int p = T.adj_ptr[i]; p < T.adj_ptr[i + 1]; ++p) {
      half_shift(T, i, T.adj_nbr[p], t);
      transport(T.d, t, T.E.data() + (size_t)T.adj_edge[p] * k * k, X);
      for (int q = 0; q < k * k; ++q) D[(size_t)i * k * k + q] += X[q];
    }
  }
  return D;
}

// Thm. cemats for an agglomeration map (agg = -1 for D).  Every coarse
// matrix is the sum of its fine contributions taken in a fixed order (a
// coarse vertex: its fine vertex matrices by ascending vertex, then its
// Dirichlet-coupled fine edges by ascending edge; a coarse edge: its fine
// edges by ascending edge), so the result does not depend on the threads.
static Topo coarse_topology(const Topo &T, const std::vector<int> &agg, int nc,
                            const std::vector<double> &xc, bool use_dir) {
  const int k = T.k, d = T.d;
  const size_t kk = (size_t)k * k;
  Topo C;
  C.n = nc;
  C.d = d;
  C.k = k;
  C.pos = xc;
  C.dir.assign(nc, 0);
  C.M.assign((size_t)nc * kk, 0.0);
  const long long ne = (long long)T.ei.size();
  // per fine edge: coarse edge key a * nc + b (a < b), or -1 (inside one
  // agglomerate, between Dirichlet vertices, or not kept), or -2 - V (a
  // Dirichlet coupling folded into coarse vertex V)
  std::vector<long long> key(ne);
#pragma omp parallel for schedule(static)
  for (long long e = 0; e < ne; ++e) {
    const int I = agg[T.ei[e]], J = agg[T.ej[e]];
    if (I >= 0 && J >= 0)
      key[e] = I == J ? -1 : (long long)std::min(I, J) * nc + std::max(I, J);
    else if (use_dir && ((I >= 0) != (J >= 0)))
      key[e] = -2 - (long long)(I >= 0 ? I : J);
    else
      key[e] = -1;
  }
  // coarse vertex contributions: fine vertices, then Dirichlet edges
  std::vector<int> vptr(nc + 1, 0), eptr(nc + 1, 0);
  for (int i = 0; i < T.n; ++i)
    if (agg[i] >= 0) ++vptr[agg[i] + 1];
  for (long long e = 0; e < ne; ++e)
    if (key[e] <= -2) ++eptr[-2 - key[e] + 1];
  for (int I = 0; I < nc; ++I) {
    vptr[I + 1] += vptr[I];
    eptr[I + 1] += eptr[I];
  }
  std::vector<int> vlist(vptr[nc]), elist(eptr[nc]);
  {
    std::vector<int> fv(vptr.begin(), vptr.end() - 1), fe(eptr.begin(), eptr.end() - 1);
    for (int i = 0; i < T.n; ++i)
      if (agg[i] >= 0) vlist[fv[agg[i]]++] = i;
    for (long long e = 0; e < ne; ++e)
      if (key[e] <= -2) elist[fe[-2 - key[e]]++] = (int)e;
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (int I = 0; I < nc; ++I) {
    double t[3], X[36];
    double *MI = C.M.data() + (size_t)I * kk;
    for (int p = vptr[I]; p < vptr[I + 1]; ++p) {
      const int i = vlist[p];
      for (int a = 0; a < d; ++a) t[a] = T.pos[(size_t)i * d + a] - xc[(size_t)I * d + a];
      transport(d, t, T.M.data() + (size_t)i * kk, X);
      for (size_t q = 0; q < kk; ++q) MI[q] += X[q];
    }
    for (int p = eptr[I]; p < eptr[I + 1]; ++p) {
      const int e = elist[p], i = T.ei[e], j = T.ej[e];
      const int v = agg[i] >= 0 ? i : j, w = agg[i] >= 0 ? j : i;
      // Q^{v_I -> v_i, T} Q^{ij,T} E Q^{ij} Q^{v_I -> v_i}: one shift (x_i+x_j)/2 - x_I
      for (int q = 0; q < d; ++q)
        t[q] = 0.5 * (T.pos[(size_t)v * d + q] + T.pos[(size_t)w * d + q]) - xc[(size_t)I * d + q];
      transport(d, t, T.E.data() + (size_t)e * kk, X);
      for (size_t q = 0; q < kk; ++q) MI[q] += X[q];
    }
  }
  // coarse edges: fine edges sorted by (coarse key, fine edge)
  std::vector<int> ce;
  for (long long e = 0; e < ne; ++e)
    if (key[e] >= 0) ce.push_back((int)e);
  std::sort(ce.begin(), ce.end(), [&](int a, int b) { return key[a] != key[b] ? key[a] < key[b] : a < b; });
  std::vector<int> cptr;
  for (size_t q = 0; q < ce.size(); ++q)
    if (q == 0 || key[ce[q]] != key[ce[q - 1]]) cptr.push_back((int)q);
  const int nce = (int)cptr.size();
  cptr.push_back((int)ce.size());
  C.ei.resize(nce);
  C.ej.resize(nce);
  C.E.assign((size_t)nce * kk, 0.0);
#pragma omp parallel for schedule(dynamic, 256)
  for (int c = 0; c < nce; ++c) {
    const long long kc = key[ce[cptr[c]]];
    const int a = (int)(kc / nc), b = (int)(kc % nc);
    C.ei[c] = a;
    C.ej[c] = b;
    double t[3], X[36];
    double *Ec = C.E.data() + (size_t)c * kk;
    for (int p = cptr[c]; p < cptr[c + 1]; ++p) {
      const int e = ce[p], i = T.ei[e], j = T.ej[e];
      // Q^{IJ->ij} = Q((x_i + x_j)/2 - (x_I + x_J)/2)
      for (int q = 0; q < d; ++q)
        t[q] = 0.5 * (T.pos[(size_t)i * d + q] + T.pos[(size_t)j * d + q]) -
               0.5 * (xc[(size_t)a * d + q] + xc[(size_t)b * d + q]);
      transport(d, t, T.E.data() + (size_t)e * kk, X);
      if (p == cptr[c])
        for (size_t q = 0; q < kk; ++q) Ec[q] = X[q];
      else
        for (size_t q = 0; q < kk; ++q) Ec[q] += X[q];
    }
  }
  C.build_adj();
  return C;
}

// ------------------------------------------------------------------ measures

static double trace(int k, const double *A) {
  double s = 0.0;
  for (int i = 0; i < k; ++i) s += A[i * k + i];
  return s;
}

// Lemma mu2 (delta-stabilised pair measure)
static double mu_p(const Topo &T, const std::vector<double> &Dh, int i, int j, int delta) {
  const int k = T.k, d = T.d;
  double t[3] = {0.0, 0.0, 0.0}, A[36], B[36], L[36], R[36], X[36], Y[36], H[36];
  half_shift(T, j, i, t);  // Q^{ji} = Q((x_i - x_j)/2)
  transport(d, t, Dh.data() + (size_t)i * k * k, A);
  half_shift(T, i, j, t);  // Q^{ij}
  transport(d, t, Dh.data() + (size_t)j * k * k, B);
  harmonic(k, A, B, L);
  const int eij = T.edge(i, j);
  for (int q = 0; q < k * k; ++q) R[q] = T.E[(size_t)eij * k * k + q];
  if (delta) {
    int p = T.adj_ptr[i], q = T.adj_ptr[j];
    const int pe = T.adj_ptr[i + 1], qe = T.adj_ptr[j + 1];
    while (p < pe && q < qe) {
      const int a = T.adj_nbr[p], b = T.adj_nbr[q];
      if (a < b) {
        ++p;
      } else if (b < a) {
        ++q;
      } else {
        const int l = a;
        half_shift(T, l, i, t);  // Q^{li}
        transport(d, t, T.E.data() + (size_t)T.adj_edge[p] * k * k, X);
        half_shift(T, l, j, t);  // Q^{lj}
        transport(d, t, T.E.data() + (size_t)T.adj_edge[q] * k * k, Y);
        harmonic(k, X, Y, H);
        // pull back with Q^{v_i -> v_l} Q^{ji}: a single shift x_l - (x_i + x_j)/2
        for (int s = 0; s < d; ++s)
          t[s] = T.pos[(size_t)l * d + s] - 0.5 * (T.pos[(size_t)i * d + s] + T.pos[(size_t)j * d + s]);
        transport(d, t, H, X);
        for (int s = 0; s < k * k; ++s) R[s] += 0.5 * delta * X[s];
        ++p;
        ++q;
      }
    }
  }
  return gen_lambda_max(k, L, R);
}

// Thm. mu1: checks mu_g^delta(C) < sigma by a semidefinite Cholesky of
// sigma * Right - Left.  On a level whose edge and vertex matrices have no
// rotation part (the finest elasticity level) both sides vanish on the
// rotation dofs, so the test runs on the displacement dofs only.
static bool mu_g_below(const Topo &T, const std::vector<double> &Dh, std::vector<int> C, int delta,
                       double sigma) {
  std::sort(C.begin(), C.end());
  const int k = T.k, d = T.d, nC = (int)C.size();
  const int b = T.rot_free ? d : k;  // dofs per vertex in the test
  const int N = nC * b;
  double xH[3] = {0, 0, 0};
  for (int v : C)
    for (int a = 0; a < d; ++a) xH[a] += T.pos[(size_t)v * d + a];
  for (int a = 0; a < d; ++a) xH[a] /= nC;
  // sub-block (first b rows / columns) of a k x k matrix
  auto sub = [&](const double *X, double *Y) {
    for (int i = 0; i < b; ++i)
      for (int j = 0; j < b; ++j) Y[i * b + j] = X[i * k + j];
  };
  // DP = D_C P_C (N x k, P_C rows Q^{v_H -> v}) and S = P_C^T D_C P_C
  std::vector<double> DP((size_t)N * k);
  double S[36] = {0}, q[36], Db[36], t[3];
  for (int a = 0; a < nC; ++a) {
    const int v = C[a];
    for (int s2 = 0; s2 < d; ++s2) t[s2] = T.pos[(size_t)v * d + s2] - xH[s2];
    qmat(d, t, q);  // rows 0..b-1 are the dofs kept
    sub(Dh.data() + (size_t)v * k * k, Db);
    double *dp = DP.data() + (size_t)a * b * k;
    mm(Db, q, dp, b, b, k);
    double qt[36];
    mtm(q, dp, qt, b, k, k);
    for (int i = 0; i < k * k; ++i) S[i] += qt[i];
  }
  double Sp[36];
  pinv_sym(k, S, Sp);
  // M = DP S^+ DP^T - D_C = -Left
  std::vector<double> M((size_t)N * N, 0.0);
  std::vector<double> DPS((size_t)N * k);
  mm(DP.data(), Sp, DPS.data(), N, k, k);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j <= i; ++j) {
      double sm = 0.0;
      for (int l = 0; l < k; ++l) sm += DPS[(size_t)i * k + l] * DP[(size_t)j * k + l];
      M[(size_t)i * N + j] = sm;
      M[(size_t)j * N + i] = sm;
    }
  for (int a = 0; a < nC; ++a) {
    sub(Dh.data() + (size_t)C[a] * k * k, Db);
    for (int i = 0; i < b; ++i)
      for (int j = 0; j < b; ++j) M[((size_t)a * b + i) * N + a * b + j] -= Db[i * b + j];
  }
  auto local = [&](int v) -> int {
    auto it = std::lower_bound(C.begin(), C.end(), v);
    return (it != C.end() && *it == v) ? (int)(it - C.begin()) : -1;
  };
  auto add_block = [&](int a, int c, const double *X, double f) {  // X is b x b
    for (int i = 0; i < b; ++i)
      for (int j = 0; j < b; ++j) M[((size_t)a * b + i) * N + c * b + j] += f * X[i * b + j];
  };
  // edge-form blocks of the edge (v, l) in the frames of v and l:
  // Evv = Q^{vl,T} E Q^{vl}, Ell = Q^{lv,T} E Q^{lv}, Evl = Q^{vl,T} E Q^{lv}
  auto edge_blocks = [&](int v, int l, const double *E, double *Evv, double *Ell, double *Evl) {
    if (T.rot_free) {
      sub(E, Evv);
      sub(E, Ell);
      sub(E, Evl);
      return;
    }
    double tv[3], tl[3];
    half_shift(T, v, l, tv);
    half_shift(T, l, v, tl);
    transport(d, tv, E, Evv);
    transport(d, tl, E, Ell);
    transport2(d, tv, tl, E, Evl);
  };
  // Right: M^i, edges inside C (each once), delta/2 Schur complements of outside neighbours
  std::vector<std::array<int, 3>> olist;  // (l, a, edge)
  for (int a = 0; a < nC; ++a) {
    const int v = C[a];
    sub(T.M.data() + (size_t)v * k * k, Db);
    add_block(a, a, Db, sigma);
    for (int p = T.adj_ptr[v]; p < T.adj_ptr[v + 1]; ++p) {
      const int l = T.adj_nbr[p], e = T.adj_edge[p];
      const int c = local(l);
      const double *E = T.E.data() + (size_t)e * k * k;
      if (c >= 0) {
        if (l > v) {
          double Evv[36], Ell[36], Evl[36], EvlT[36];
          edge_blocks(v, l, E, Evv, Ell, Evl);
          add_block(a, a, Evv, sigma);
          add_block(c, c, Ell, sigma);
          add_block(a, c, Evl, -sigma);
          for (int i = 0; i < b; ++i)
            for (int j = 0; j < b; ++j) EvlT[i * b + j] = Evl[j * b + i];
          add_block(c, a, EvlT, -sigma);
        }
      } else if (delta) {
        olist.push_back({l, a, e});
      }
    }
  }
  if (delta) {
    std::sort(olist.begin(), olist.end());
    size_t s0 = 0;
    while (s0 < olist.size()) {
      size_t s1 = s0;
      while (s1 < olist.size() && olist[s1][0] == olist[s0][0]) ++s1;
      const int l = olist[s0][0];
      const int m = (int)(s1 - s0);
      double Kll[36] = {0};
      std::vector<double> KCl((size_t)m * b * b);
      std::vector<int> av(m);
      for (int u = 0; u < m; ++u) {
        const int a = olist[s0 + u][1], e = olist[s0 + u][2], v = C[a];
        const double *E = T.E.data() + (size_t)e * k * k;
        double Evv[36], Ell[36], Evl[36];
        edge_blocks(v, l, E, Evv, Ell, Evl);
        add_block(a, a, Evv, 0.5 * delta * sigma);  // K_CC
        for (int i = 0; i < b * b; ++i) KCl[(size_t)u * b * b + i] = -Evl[i];
        for (int i = 0; i < b * b; ++i) Kll[i] += Ell[i];
        av[u] = a;
      }
      double Kp[36];
      pinv_sym(b, Kll, Kp);
      for (int u = 0; u < m; ++u) {
        double T1[36];
        mm(KCl.data() + (size_t)u * b * b, Kp, T1, b, b, b);
        for (int w = 0; w < m; ++w) {
          double T2[36];
          for (int i = 0; i < b; ++i)
            for (int j = 0; j < b; ++j) {
              double sm = 0.0;
              for (int q2 = 0; q2 < b; ++q2) sm += T1[i * b + q2] * KCl[(size_t)w * b * b + j * b + q2];
              T2[i * b + j] = sm;
            }
          add_block(av[u], av[w], T2, -0.5 * delta * sigma);
        }
      }
      s0 = s1;
    }
  }
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j) {
      const double mm2 = 0.5 * (M[(size_t)i * N + j] + M[(size_t)j * N + i]);
      M[(size_t)i * N + j] = M[(size_t)j * N + i] = mm2;
    }
  return psd_cholesky(N, M, 1e-10);
}

// ------------------------------------------------------------------ Algorithm 1

static std::vector<int> cuthill_mckee(const Topo &T, const std::vector<char> &active) {
  std::vector<int> deg(T.n, 0);
  for (int v = 0; v < T.n; ++v)
    if (active[v])
      for (int p = T.adj_ptr[v]; p < T.adj_ptr[v + 1]; ++p) deg[v] += active[T.adj_nbr[p]] ? 1 : 0;
  std::vector<char> seen(T.n, 0);
  for (int v = 0; v < T.n; ++v) seen[v] = !active[v];
  std::vector<int> order;
  order.reserve(T.n);
  // candidates for a new start, by (degree, id)
  std::vector<int> starts;
  for (int v = 0; v < T.n; ++v)
    if (active[v]) starts.push_back(v);
  std::stable_sort(starts.begin(), starts.end(), [&](int a, int b) { return deg[a] < deg[b]; });
  size_t sp = 0;
  std::vector<int> nb;
  while (true) {
    while (sp < starts.size() && seen[starts[sp]]) ++sp;
    if (sp == starts.size()) break;
    const int s = starts[sp];
    seen[s] = 1;
    size_t head = order.size();
    order.push_back(s);
    while (head < order.size()) {
      const int v = order[head++];
      nb.clear();
      for (int p = T.adj_ptr[v]; p < T.adj_ptr[v + 1]; ++p) {
        const int w = T.adj_nbr[p];
        if (active[w] && !seen[w]) nb.push_back(w);
      }
      std::sort(nb.begin(), nb.end(), [&](int a, int b) {
        return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
      });
      for (int w : nb) {
        seen[w] = 1;
        order.push_back(w);
      }
    }
  }
  return order;
}

struct Coarsening {
  std::vector<int> agg;
  int nc = 0;
  std::vector<double> xc;
  Topo coarse;
  std::vector<char> D;
};

// final_topology = false leaves the coarse edge / vertex matrices of the
// last pass to the caller (positions only).
static Coarsening successive_matching(const Topo &T0, const SetupParams &prm, int passes,
                                      bool final_topology, PairMeasure *pm, std::string &err) {
  const int n = T0.n, k = T0.k, d = T0.d;
  const double sigma = prm.sigma;
  std::vector<double> Dh0 = aux_diagonal(T0);
  Coarsening out;
  out.D = T0.dir;
#pragma omp parallel for schedule(static)
  for (int v = 0; v < n; ++v)
    if (!T0.dir[v]) {
      // mu_D(v) = lambda_max(D-hat_vv, M^v) (eq. mu_d)
      const double m = gen_lambda_max(k, Dh0.data() + (size_t)v * k * k, T0.M.data() + (size_t)v * k * k);
      if (m < sigma) out.D[v] = 1;
    }
  std::vector<char> active(n);
  for (int v = 0; v < n; ++v) active[v] = !out.D[v];
  std::vector<int> order = cuthill_mckee(T0, active);
  std::vector<std::vector<int>> members(n);
  for (int v = 0; v < n; ++v) members[v] = {v};
  Topo cur;  // intermediate topology of passes >= 2
  const Topo *Tc = &T0;
  for (int pass = 1; pass <= passes; ++pass) {
    std::vector<double> Dh = (pass == 1) ? Dh0 : aux_diagonal(*Tc);
    // a device evaluator of mu_p for this pass (elasticity levels; the
    // scalar problem's 1 x 1 measures stay on the host)
    PairMeasure *dev_pm = (pm && !prm.scalar_only && Tc->d >= 2) ? pm : nullptr;
    if (dev_pm && dev_pm->begin_pass(*Tc, Dh, prm.delta) != 0) {
      err = "device pair measure: upload failed";
      dev_pm = nullptr;
    }
    const int m = Tc->n;
    std::vector<double> tmax(m, 0.0);
    for (int v = 0; v < m; ++v) {
      tmax[v] = trace(k, Tc->M.data() + (size_t)v * k * k);
      for (int p = Tc->adj_ptr[v]; p < Tc->adj_ptr[v + 1]; ++p)
        tmax[v] = std::max(tmax[v], trace(k, Tc->E.data() + (size_t)Tc->adj_edge[p] * k * k));
    }
    std::vector<int> rank(m, 0);
    std::vector<char> inT(m, 0);
    for (size_t r = 0; r < order.size(); ++r) {
      rank[order[r]] = (int)r;
      inT[order[r]] = 1;
    }
    std::vector<std::vector<int>> groups;
    std::vector<int> singles;
    struct Cand {
      double mu;
      int rank, cj;
    };
    // candidates of ci among the unmatched neighbours (live[] != 0) with
    // mu_s < sigma, ordered by mu_s, ties by the iteration order (Def. muc,
    // Algorithm 1)
    auto candidates = [&](int ci, const std::vector<char> &live, std::vector<Cand> &cands) {
      cands.clear();
      for (int p = Tc->adj_ptr[ci]; p < Tc->adj_ptr[ci + 1]; ++p) {
        const int cj = Tc->adj_nbr[p];
        if (!live[cj]) continue;
        const double tr = trace(k, Tc->E.data() + (size_t)Tc->adj_edge[p] * k * k);
        if (!(tr > 0.0)) continue;
        const double ms = sqrt(tmax[ci] * tmax[cj]) / tr;
        if (ms < sigma) cands.push_back({ms, rank[cj], cj});
      }
      std::sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &b) {
        return a.mu != b.mu ? a.mu < b.mu : a.rank < b.rank;
      });
    };
    // mu_p and (when needed) the mu_g test of one pair; pure functions of
    // the pass's topology, so they can be evaluated ahead of the greedy loop
    auto evaluate = [&](int ci, int cj, double &mu, int &gok) {
      mu = mu_p(*Tc, Dh, ci, cj, prm.delta);
      gok = 1;
      if (mu < sigma && members[ci].size() + members[cj].size() > 2) {
        std::vector<int> uni(members[ci]);
        uni.insert(uni.end(), members[cj].begin(), members[cj].end());
        gok = mu_g_below(T0, Dh0, uni, prm.delta, sigma) ? 1 : 0;
      }
    };
    // The greedy loop below decides pairs in iteration order; the measures
    // it consults are evaluated ahead of it, in parallel batches.  A dry run
    // of the loop over the rest of a chunk predicts its walk: a pair already
    // evaluated decides as in the loop, a pair not evaluated yet is taken to
    // succeed (the first live candidate usually does) and goes into the
    // batch.  One dry run starts each chunk; wherever the loop meets a pair
    // not evaluated yet (its walk left the prediction there), a new dry run
    // starts at that point.  The decisions are those of evaluating each
    // pair when the loop reaches it.
    // a device evaluator wants large batches (one thread per pair: a batch
    // of a 2,048-vertex chunk occupies a fraction of the device); the chunk
    // only decides how far the look-ahead reaches, not the decisions
    const int chunk = dev_pm ? 32768 : 2048, ahead = 1;
    std::vector<Cand> cands;
    struct Eval {
      double mu;
      int gok;
    };
    std::unordered_map<long long, Eval> done;
    std::vector<std::array<int, 2>> tasks;
    std::vector<Eval> res;
    // batches of at least kDeviceBatch pairs go to the device evaluator of
    // mu_p (if any); the mu_g tests stay on the host
    const size_t kDeviceBatch = 512;
    std::vector<double> dmu;
    auto run_tasks = [&]() {
      res.resize(tasks.size());
      if (dev_pm && tasks.size() >= kDeviceBatch && dev_pm->evaluate(tasks, dmu) == 0) {
#pragma omp parallel for schedule(dynamic, 1)
        for (long long q = 0; q < (long long)tasks.size(); ++q) {
          const int ci = tasks[q][0], cj = tasks[q][1];
          res[q].mu = dmu[q];
          res[q].gok = 1;
          if (dmu[q] < sigma && members[ci].size() + members[cj].size() > 2) {
            std::vector<int> uni(members[ci]);
            uni.insert(uni.end(), members[cj].begin(), members[cj].end());
            res[q].gok = mu_g_below(T0, Dh0, uni, prm.delta, sigma) ? 1 : 0;
          }
        }
      } else {
#pragma omp parallel for schedule(dynamic, 1)
        for (long long q = 0; q < (long long)tasks.size(); ++q)
          evaluate(tasks[q][0], tasks[q][1], res[q].mu, res[q].gok);
      }
      for (size_t q = 0; q < tasks.size(); ++q) done[(long long)tasks[q][0] * m + tasks[q][1]] = res[q];
      tasks.clear();
    };
    // live: inT as the dry run sees it (equal to inT between chunks)
    std::vector<char> live(inT);
    std::vector<int> touched;
    // dry run of the loop from position q0 of a chunk to its end c1 (with
    // first_taken, order[q0] has been taken out by the loop already): every
    // pair it meets that is not evaluated yet goes into tasks
    std::vector<Cand> dcands;
    auto dry_run = [&](size_t q0, size_t c1, bool first_taken) {
      for (size_t q = q0; q < c1; ++q) {
        const int ci = order[q];
        if (!(first_taken && q == q0)) {
          if (!live[ci]) continue;
          live[ci] = 0;
          touched.push_back(ci);
        }
        candidates(ci, live, dcands);
        for (size_t u = 0; u < dcands.size(); ++u) {
          const int cj = dcands[u].cj;
          auto it = done.find((long long)ci * m + cj);
          if (it == done.end()) {  // not evaluated yet: evaluate, take it to succeed
            for (size_t w = u; w < dcands.size() && w < u + (size_t)ahead; ++w)
              if (!done.count((long long)ci * m + dcands[w].cj)) tasks.push_back({ci, dcands[w].cj});
          } else if (!(it->second.mu < sigma && it->second.gok)) {
            continue;
          }
          live[cj] = 0;
          touched.push_back(cj);
          break;
        }
      }
      for (int v : touched) live[v] = 1;
      touched.clear();
    };
    for (size_t c0 = 0; c0 < order.size(); c0 += chunk) {
      const size_t c1 = std::min(order.size(), c0 + chunk);
      done.clear();
      if (!prm.scalar_only) {
        dry_run(c0, c1, false);
        run_tasks();
      }
      for (size_t q = c0; q < c1; ++q) {
        const int ci = order[q];
        if (!inT[ci]) continue;
        inT[ci] = live[ci] = 0;
        candidates(ci, inT, cands);
        bool matched = false;
        if (prm.scalar_only) {
          // mu_s alone: the candidate of minimal mu_s is taken (Sec. 5's
          // comparison and the paper's scalar runs)
          if (!cands.empty()) {
            groups.push_back({ci, cands[0].cj});
            inT[cands[0].cj] = live[cands[0].cj] = 0;
          } else {
            singles.push_back(ci);
          }
          continue;
        }
        for (size_t u = 0; u < cands.size(); ++u) {
          const int cj = cands[u].cj;
          auto it = done.find((long long)ci * m + cj);
          if (it == done.end()) {
            // the walk left the last prediction here: predict the rest of
            // the chunk from this point (it starts with this pair)
            dry_run(q, c1, true);
            if (tasks.empty()) tasks.push_back({ci, cj});
            run_tasks();
            it = done.find((long long)ci * m + cj);
            if (it == done.end()) {
              tasks.push_back({ci, cj});
              run_tasks();
              it = done.find((long long)ci * m + cj);
            }
          }
          const double mu = it->second.mu;
          const int gok = it->second.gok;
          if (mu < sigma && gok) {
            groups.push_back({ci, cj});
            inT[cj] = live[cj] = 0;
            matched = true;
            break;
          }
        }
        if (!matched) singles.push_back(ci);
      }
    }
    for (int s : singles) groups.push_back({s});
    const int mc = (int)groups.size();
    std::vector<std::vector<int>> nm(mc);
    std::vector<int> cagg(m, -1);
    std::vector<double> xc((size_t)mc * d, 0.0);
    for (int g = 0; g < mc; ++g) {
      for (int c : groups[g]) {
        cagg[c] = g;
        nm[g].insert(nm[g].end(), members[c].begin(), members[c].end());
      }
      for (int v : nm[g])
        for (int a = 0; a < d; ++a) xc[(size_t)g * d + a] += T0.pos[(size_t)v * d + a];
      for (int a = 0; a < d; ++a) xc[(size_t)g * d + a] /= (double)nm[g].size();
    }
    if (pass == passes && !final_topology) {
      Topo next;
      next.n = mc;
      next.d = d;
      next.k = k;
      next.pos = xc;
      cur = std::move(next);
    } else {
      Topo next = coarse_topology(*Tc, cagg, mc, xc, pass == 1);
      cur = std::move(next);
    }
    Tc = &cur;
    members = std::move(nm);
    order.resize(mc);
    for (int g = 0; g < mc; ++g) order[g] = mc - 1 - g;
  }
  out.nc = (int)members.size();
  out.agg.assign(n, -1);
  for (int g = 0; g < out.nc; ++g)
    for (int v : members[g]) out.agg[v] = g;
  out.xc = cur.pos;
  out.coarse = std::move(cur);
  return out;
}

// ------------------------------------------------------------------ prolongation

struct RowBlocks {  // one prolongation row: sorted columns, kr x k blocks
  std::vector<int> col;
  std::vector<double> val;
};

static void add_to_row(std::vector<std::pair<int, std::array<double, 36>>> &acc, int J, const double *X,
                       int sz) {
  for (auto &pr : acc)
    if (pr.first == J) {
      for (int i = 0; i < sz; ++i) pr.second[i] += X[i];
      return;
    }
  std::array<double, 36> z;
  z.fill(0.0);
  for (int i = 0; i < sz; ++i) z[i] = X[i];
  acc.push_back({J, z});
}

// Def. aux_sp with the S / A split; returns BSR rows and next-level "bad" flags.
static void smoothed_prolongation(const HostBSR &A, const Topo &T, const Coarsening &cs,
                                  const std::vector<int> &rowmap, const std::vector<char> &bad,
                                  bool first, const SetupParams &prm, HostBSR &P,
                                  std::vector<char> &next_bad) {
  const int d = T.d, k = T.k, kr = first ? d : k;
  const int nrows = A.n_rows;
  const int capS = first ? prm.cap_S_first : prm.cap_S_later;
  std::vector<int> row_of(T.n, -1);
  for (int r = 0; r < nrows; ++r) row_of[rowmap[r]] = r;
  // tentative rows (one block each)
  std::vector<std::array<double, 36>> Pt(nrows);
  std::vector<int> Pcol(nrows, -1);
  for (int r = 0; r < nrows; ++r) {
    const int v = rowmap[r], J = cs.agg[v];
    if (J < 0) continue;
    double t[3], q[36];
    for (int a = 0; a < d; ++a) t[a] = T.pos[(size_t)v * d + a] - cs.xc[(size_t)J * d + a];
    qmat(d, t, q);
    Pcol[r] = J;
    for (int i = 0; i < kr; ++i)
      for (int j = 0; j < k; ++j) Pt[r][i * k + j] = q[i * k + j];
  }
  P.n_rows = nrows;
  P.n_cols = cs.nc;
  P.br = kr;
  P.bc = k;
  P.rowptr.assign(nrows + 1, 0);
  P.colidx.clear();
  P.vals.clear();
  const double om = prm.omega;
  // rows are independent: each is built into its own buffers in parallel,
  // then the buffers are concatenated in row order
  std::vector<std::vector<int>> rcol(nrows);
  std::vector<std::vector<double>> rval(nrows);
#pragma omp parallel for schedule(dynamic, 256)
  for (int r = 0; r < nrows; ++r) {
    const int v = rowmap[r];
    std::vector<std::pair<int, std::array<double, 36>>> acc;
    double Dinv[36];
    if (!cs.D[v]) {
      std::vector<int> touched;
      for (int p = A.rowptr[r]; p < A.rowptr[r + 1]; ++p) {
        const int c = A.colidx[p];
        const int w = rowmap[c];
        if (cs.D[w]) continue;
        const int J = cs.agg[w];
        if (std::find(touched.begin(), touched.end(), J) == touched.end()) touched.push_back(J);
      }
      const bool standard = (int)touched.size() <= capS && !bad[r];
      if (standard) {
        double Arr[36] = {0};
        for (int p = A.rowptr[r]; p < A.rowptr[r + 1]; ++p) {
          const int c = A.colidx[p];
          const double *Ab = A.vals.data() + (size_t)p * kr * kr;
          if (c == r)
            for (int i = 0; i < kr * kr; ++i) Arr[i] = Ab[i];
          if (Pcol[c] < 0) continue;
          double X[36];
          mm(Ab, Pt[c].data(), X, kr, kr, k);
          add_to_row(acc, Pcol[c], X, kr * k);
        }
        pinv_sym(kr, Arr, Dinv);
      } else {
        // filtered neighbours F^i: own agglomerate + top (cap_A - 1) by sum tr E
        std::vector<std::pair<int, double>> wsum;
        for (int p = T.adj_ptr[v]; p < T.adj_ptr[v + 1]; ++p) {
          const int l = T.adj_nbr[p];
          if (cs.D[l]) continue;
          const int J = cs.agg[l];
          const double tr = trace(k, T.E.data() + (size_t)T.adj_edge[p] * k * k);
          bool found = false;
          for (auto &pr : wsum)
            if (pr.first == J) {
              pr.second += tr;
              found = true;
            }
          if (!found) wsum.push_back({J, tr});
        }
        const int own = cs.agg[v];
        std::vector<std::pair<int, double>> others;
        for (auto &pr : wsum)
          if (pr.first != own) others.push_back(pr);
        std::sort(others.begin(), others.end(), [](const std::pair<int, double> &a,
                                                   const std::pair<int, double> &b) {
          return a.second != b.second ? a.second > b.second : a.first < b.first;
        });
        std::vector<int> keep = {own};
        for (int q = 0; q < (int)others.size() && q < prm.cap_A - 1; ++q) keep.push_back(others[q].first);
        double Aii[36] = {0};
        std::vector<std::pair<int, std::array<double, 36>>> offd;
        for (int p = T.adj_ptr[v]; p < T.adj_ptr[v + 1]; ++p) {
          const int l = T.adj_nbr[p];
          if (cs.D[l] || std::find(keep.begin(), keep.end(), cs.agg[l]) == keep.end()) continue;
          const double *E = T.E.data() + (size_t)T.adj_edge[p] * k * k;
          std::array<double, 36> X;
          X.fill(0.0);
          if (first) {
            for (int i = 0; i < d; ++i)
              for (int j = 0; j < d; ++j) {
                Aii[i * d + j] += E[i * k + j];
                X[i * d + j] = -E[i * k + j];
              }
          } else {
            double tv[3], tl[3], Z[36];
            half_shift(T, v, l, tv);
            half_shift(T, l, v, tl);
            transport(d, tv, E, Z);
            for (int i = 0; i < k * k; ++i) Aii[i] += Z[i];
            transport2(d, tv, tl, E, Z);
            for (int i = 0; i < k * k; ++i) X[i] = -Z[i];
          }
          offd.push_back({l, X});
        }
        pinv_sym(kr, Aii, Dinv);
        double X[36];
        if (Pcol[r] >= 0) {
          mm(Aii, Pt[r].data(), X, kr, kr, k);
          add_to_row(acc, Pcol[r], X, kr * k);
        }
        for (auto &pr : offd) {
          const int c = row_of[pr.first];
          if (c < 0 || Pcol[c] < 0) continue;
          mm(pr.second.data(), Pt[c].data(), X, kr, kr, k);
          add_to_row(acc, Pcol[c], X, kr * k);
        }
      }
    }
    std::sort(acc.begin(), acc.end(), [](const std::pair<int, std::array<double, 36>> &a,
                                         const std::pair<int, std::array<double, 36>> &b) {
      return a.first < b.first;
    });
    for (auto &pr : acc) {
      double X[36];
      mm(Dinv, pr.second.data(), X, kr, kr, k);
      rcol[r].push_back(pr.first);
      for (int i = 0; i < kr * k; ++i) {
        const double base = (pr.first == Pcol[r]) ? Pt[r][i] : 0.0;
        rval[r].push_back(base - om * X[i]);
      }
    }
  }
  for (int r = 0; r < nrows; ++r) {
    P.colidx.insert(P.colidx.end(), rcol[r].begin(), rcol[r].end());
    P.vals.insert(P.vals.end(), rval[r].begin(), rval[r].end());
    P.rowptr[r + 1] = (int)P.colidx.size();
  }
  next_bad.assign(cs.nc, 0);
  for (int r = 0; r < nrows; ++r)
    if (bad[r])
      for (int p = P.rowptr[r]; p < P.rowptr[r + 1]; ++p) next_bad[P.colidx[p]] = 1;
}

// ------------------------------------------------------------------ level loop

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int build_levels(const Problem &prob, const SetupParams &prm, LevelSink &sink, std::string &err) {
#ifdef _OPENMP
  // thread count of the OpenMP regions started by this (calling) thread only,
  // restored on return: independent setups may run side by side on threads
  struct ThreadScope {
    int saved;
    explicit ThreadScope(int n) : saved(omp_get_max_threads()) {
      if (n > 0) omp_set_num_threads(n);
    }
    ~ThreadScope() { omp_set_num_threads(saved); }
  } scope(prm.host_threads);
#endif
  const int dim = prob.dim, n_all = prob.n_vertices;
  if (dim != 2 && dim != 3) {
    err = "dim must be 2 or 3";
    return -1;
  }
  const bool scalar = prob.block == 1;
  const int d = scalar ? 1 : dim;  // block size of A_0
  Topo T = scalar ? finest_topology_scalar(dim, n_all, prob.coords, prob.dirichlet, prob.rowptr,
                                           prob.colidx, prob.vals)
                  : finest_topology(d, n_all, prob.coords, prob.dirichlet, prob.rowptr, prob.colidx,
                                    prob.vals);
  // A_0: rows / columns of the free vertices
  std::vector<int> rowmap, newid(n_all, -1);
  for (int v = 0; v < n_all; ++v)
    if (!T.dir[v]) {
      newid[v] = (int)rowmap.size();
      rowmap.push_back(v);
    }
  HostBSR A;
  A.n_rows = A.n_cols = (int)rowmap.size();
  A.br = A.bc = d;
  A.rowptr.assign(A.n_rows + 1, 0);
  for (int r = 0; r < A.n_rows; ++r) {
    const int v = rowmap[r];
    for (int p = prob.rowptr[v]; p < prob.rowptr[v + 1]; ++p) {
      const int w = newid[prob.colidx[p]];
      if (w < 0) continue;
      A.colidx.push_back(w);
      A.vals.insert(A.vals.end(), prob.vals + (size_t)p * d * d, prob.vals + (size_t)(p + 1) * d * d);
    }
    A.rowptr[r + 1] = (int)A.colidx.size();
  }
  if (sink.first(A) != 0) {
    err = "upload of A_0 failed";
    return -1;
  }
  const int n0 = A.n_rows;
  const int cmax = prm.coarse_max > 0 ? prm.coarse_max
                                      : std::min(1000, std::max(64, (int)ceil(n0 / 1e4)));
  std::vector<char> bad_exact(A.n_rows, 0);
  // AMG_SETUP_VERBOSE=1 prints the host time of every setup stage to stderr
  const bool verbose = getenv("AMG_SETUP_VERBOSE") != nullptr;
  int level = 0;
  while (A.n_rows > cmax && level + 1 < prm.max_levels) {
    const bool first = level == 0;
    double t0 = now_s();
    const bool dev = sink.device_stages();
    Coarsening cs = successive_matching(T, prm, first ? prm.passes_first : prm.passes_later, !dev,
                                        dev ? sink.pair_measure() : nullptr, err);
    if (!err.empty()) return -1;
    if (verbose)
      fprintf(stderr, "[amg setup] level %d: %d vertices -> %d agglomerates, matching %.2f s\n",
              level, T.n, cs.nc, now_s() - t0);
    if (cs.nc == 0 || A.n_rows < prm.min_ratio * cs.nc) break;
    if (dev && sink.coarse_topology(level, T, cs.agg, cs.nc, cs.xc, cs.coarse) != 0) {
      err = "device coarse edge / vertex matrices failed";
      return -1;
    }
    std::vector<char> bad(A.n_rows, 0);
    for (int r = 0; r < A.n_rows; ++r) {
      bool couples = false;
      if (first) {
        const int v = rowmap[r];
        for (int p = T.adj_ptr[v]; p < T.adj_ptr[v + 1] && !couples; ++p) couples = cs.D[T.adj_nbr[p]];
      } else {
        for (int p = A.rowptr[r]; p < A.rowptr[r + 1] && !couples; ++p) couples = cs.D[rowmap[A.colidx[p]]];
      }
      bad[r] = bad_exact[r] || couples;
    }
    HostBSR P;
    std::vector<char> next_bad;
    t0 = now_s();
    int handled = 0;
    if (dev && sink.prolongation(level, A, T, cs.agg, cs.D, cs.nc, cs.xc, rowmap, bad, first, prm, P,
                                 next_bad, &handled) != 0) {
      err = "device smoothed prolongation failed";
      return -1;
    }
    if (!handled) smoothed_prolongation(A, T, cs, rowmap, bad, first, prm, P, next_bad);
    if (verbose)
      fprintf(stderr, "[amg setup] level %d: prolongation %.2f s (%zu blocks)\n", level, now_s() - t0,
              P.colidx.size());
    HostBSR Anext;
    if (sink.next(level, P, Anext) != 0) {
      err = "device Galerkin product failed";
      return -1;
    }
    A = std::move(Anext);
    T = std::move(cs.coarse);
    rowmap.resize(cs.nc);
    for (int i = 0; i < cs.nc; ++i) rowmap[i] = i;
    bad_exact = std::move(next_bad);
    ++level;
  }
  return 0;
}

std::vector<int> smallest_last_colouring(int n, const int *rp, const int *ci, int *n_colours) {
  // smallest-last order: a heap of (degree, row) with stale entries skipped
  std::vector<int> deg(n, 0), order;
  order.reserve(n);
  for (int i = 0; i < n; ++i)
    for (int p = rp[i]; p < rp[i + 1]; ++p) deg[i] += ci[p] != i;
  {
    std::priority_queue<std::pair<int, int>, std::vector<std::pair<int, int>>,
                        std::greater<std::pair<int, int>>>
        heap;
    for (int i = 0; i < n; ++i) heap.push({deg[i], i});
    std::vector<char> removed(n, 0);
    while (!heap.empty()) {
      const auto top = heap.top();
      heap.pop();
      const int i = top.second;
      if (removed[i] || top.first != deg[i]) continue;
      removed[i] = 1;
      order.push_back(i);
      for (int p = rp[i]; p < rp[i + 1]; ++p) {
        const int j = ci[p];
        if (j != i && !removed[j]) heap.push({--deg[j], j});
      }
    }
    std::reverse(order.begin(), order.end());
  }
  std::vector<int> colour(n, -1), mark;
  int nc = 0;
  for (int i : order) {
    // colours held by the already coloured neighbours of row i
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      const int cc = colour[ci[p]];
      if (cc >= 0) {
        if (cc >= (int)mark.size()) mark.resize(cc + 1, -1);
        mark[cc] = i;
      }
    }
    int cc = 0;
    while (cc < (int)mark.size() && mark[cc] == i) ++cc;
    colour[i] = cc;
    nc = std::max(nc, cc + 1);
  }
  if (n_colours) *n_colours = nc;
  return colour;
}

}  // namespace amgsetup
