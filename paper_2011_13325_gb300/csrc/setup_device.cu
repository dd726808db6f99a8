// Device stages of the setup: the coarse edge and vertex matrices of Thm.
// cemats and the auxiliary smoothed prolongation of Def. aux_sp (Sec. 6),
// computed for the agglomerates Algorithm 1 found on the host.
//
// Coarse topology.  Kernel transfers compose (Q(a) Q(b) = Q(a + b)), so the
// coarse matrices of the final agglomerates follow from the level's own
// topology in one step: E^{IJ} = sum over the fine edges (i, j) between C_I
// and C_J of Q(s)^T E^{ij} Q(s), s = (x_i + x_j)/2 - (x_I + x_J)/2, and
// M^I = sum_{i in C_I} Q(x_i - x_I)^T M^i Q(x_i - x_I) plus, for every fine
// edge from C_I to a vertex of D, Q(s')^T E^{ij} Q(s') with s' = (x_i +
// x_j)/2 - x_I.  Every coarse matrix sums its contributions in a fixed order
// (vertex matrices by ascending vertex, then edges by ascending edge).  The
// host keeps the bookkeeping (which fine items feed which coarse matrix);
// the device does the transfers.
//
// Smoothed prolongation.  One thread per row of P_l: the row's tentative
// blocks Q(x_v - x_J) (Def. pwp / pwp_el; on the first elasticity level their
// displacement rows), then P_s = P_t - omega D^+ (A P_t) restricted as Def.
// aux_sp reads it: a "standard" row (its A-row touches at most cap_S
// agglomerates, does not couple to D and is kernel-exact) uses the real
// matrix row and D = A_vv; every other row uses the auxiliary matrix row of
// its filtered neighbours F^i (its own agglomerate and the cap_A - 1 others
// with the largest sum of tr E^{il}; on the first elasticity level the d x d
// displacement blocks of the edge matrices), D = its diagonal block.  Two
// passes: row lengths, then columns (ascending) and values.
#include <algorithm>
#include <array>
#include <chrono>

#include "amg_internal.h"
#include "dense_dev.cuh"
#include "setup_host.h"

namespace amg {

// ---------------------------------------------------------------- transfers

// Skew(t) as a D x R block (R = K - D rotation coordinates): Skew(t) r = t x r
// in 3D, (-t_1, t_0)^T in 2D (Sec. 3).
template <int D>
__device__ __forceinline__ void skew_dev(const double *t, double *S) {
  if (D == 2) {
    S[0] = -t[1];
    S[1] = t[0];
  } else {
    S[0] = 0.0;   S[1] = -t[2]; S[2] = t[1];
    S[3] = t[2];  S[4] = 0.0;   S[5] = -t[0];
    S[6] = -t[1]; S[7] = t[0];  S[8] = 0.0;
  }
}

// out = Q(t1)^T X Q(t2), Q(t) = [[I, Skew(t)], [0, I]], X = [[A, B], [C, F]]
// (D x D, D x R, R x D, R x R): [[A, A S2 + B], [S1^T A + C, S1^T A S2 +
// S1^T B + C S2 + F]].
template <int D>
__device__ void transfer_dev(const double *t1, const double *t2, const double *X, double *out) {
  constexpr int K = D == 2 ? 3 : 6, R = K - D;
  double S1[D * R], S2[D * R];
  skew_dev<D>(t1, S1);
  skew_dev<D>(t2, S2);
  double AS2[D * R], S1A[R * D];
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < R; ++j) {
      double s = 0.0;
      for (int l = 0; l < D; ++l) s += X[i * K + l] * S2[l * R + j];
      AS2[i * R + j] = s;
    }
  for (int i = 0; i < R; ++i)
    for (int j = 0; j < D; ++j) {
      double s = 0.0;
      for (int l = 0; l < D; ++l) s += S1[l * R + i] * X[l * K + j];
      S1A[i * D + j] = s;
    }
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) out[i * K + j] = X[i * K + j];
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < R; ++j) out[i * K + D + j] = AS2[i * R + j] + X[i * K + D + j];
  for (int i = 0; i < R; ++i)
    for (int j = 0; j < D; ++j) out[(D + i) * K + j] = S1A[i * D + j] + X[(D + i) * K + j];
  for (int i = 0; i < R; ++i)
    for (int j = 0; j < R; ++j) {
      double s = X[(D + i) * K + D + j];
      for (int l = 0; l < D; ++l) {
        s += S1A[i * D + l] * S2[l * R + j];               // S1^T A S2
        s += S1[l * R + i] * X[l * K + D + j];              // S1^T B
        s += X[(D + i) * K + l] * S2[l * R + j];            // C S2
      }
      out[(D + i) * K + D + j] = s;
    }
}

// M^I of every coarse vertex (one thread per coarse vertex).
template <int D>
__global__ void coarse_vertex_kernel(int nc, const int *__restrict__ vptr, const int *__restrict__ vlist,
                                     const int *__restrict__ eptr, const int *__restrict__ elist,
                                     const int *__restrict__ ei, const int *__restrict__ ej,
                                     const int *__restrict__ agg, const double *__restrict__ pos,
                                     const double *__restrict__ xc, const double *__restrict__ Mf,
                                     const double *__restrict__ Ef, double *__restrict__ Mc) {
  constexpr int K = D == 2 ? 3 : 6, KK = K * K;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  double acc[KK], X[KK], t[D];
  for (int q = 0; q < KK; ++q) acc[q] = 0.0;
  for (int p = vptr[I]; p < vptr[I + 1]; ++p) {
    const int i = vlist[p];
    for (int a = 0; a < D; ++a) t[a] = pos[(size_t)i * D + a] - xc[(size_t)I * D + a];
    transfer_dev<D>(t, t, Mf + (size_t)i * KK, X);
    for (int q = 0; q < KK; ++q) acc[q] += X[q];
  }
  for (int p = eptr[I]; p < eptr[I + 1]; ++p) {
    const int e = elist[p], i = ei[e], j = ej[e];
    const int v = agg[i] >= 0 ? i : j, w = agg[i] >= 0 ? j : i;
    for (int a = 0; a < D; ++a)
      t[a] = 0.5 * (pos[(size_t)v * D + a] + pos[(size_t)w * D + a]) - xc[(size_t)I * D + a];
    transfer_dev<D>(t, t, Ef + (size_t)e * KK, X);
    for (int q = 0; q < KK; ++q) acc[q] += X[q];
  }
  for (int q = 0; q < KK; ++q) Mc[(size_t)I * KK + q] = acc[q];
}

// E^{IJ} of every coarse edge (one thread per coarse edge c = (a, b)).
template <int D>
__global__ void coarse_edge_kernel(int nce, const int *__restrict__ cptr, const int *__restrict__ ce,
                                   const int *__restrict__ ca, const int *__restrict__ cb,
                                   const int *__restrict__ ei, const int *__restrict__ ej,
                                   const double *__restrict__ pos, const double *__restrict__ xc,
                                   const double *__restrict__ Ef, double *__restrict__ Ec) {
  constexpr int K = D == 2 ? 3 : 6, KK = K * K;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nce) return;
  const int a = ca[c], b = cb[c];
  double acc[KK], X[KK], t[D];
  for (int q = 0; q < KK; ++q) acc[q] = 0.0;
  for (int p = cptr[c]; p < cptr[c + 1]; ++p) {
    const int e = ce[p], i = ei[e], j = ej[e];
    for (int q = 0; q < D; ++q)
      t[q] = 0.5 * (pos[(size_t)i * D + q] + pos[(size_t)j * D + q]) -
             0.5 * (xc[(size_t)a * D + q] + xc[(size_t)b * D + q]);
    transfer_dev<D>(t, t, Ef + (size_t)e * KK, X);
    for (int q = 0; q < KK; ++q) acc[q] += X[q];
  }
  for (int q = 0; q < KK; ++q) Ec[(size_t)c * KK + q] = acc[q];
}

// Device buffers freed on scope exit.
struct DevScratch {
  std::vector<void *> ptrs;
  ~DevScratch() {
    for (void *p : ptrs) dfree(p);
  }
  template <typename T>
  cudaError_t put(Ctx *c, T **d, const T *h, size_t n) {
    *d = nullptr;
    cudaError_t e = dalloc((void **)d, (n ? n : 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    ptrs.push_back(*d);
    return n ? cudaMemcpyAsync(*d, h, n * sizeof(T), cudaMemcpyHostToDevice, c->stream) : cudaSuccess;
  }
  template <typename T>
  cudaError_t make(T **d, size_t n) {
    *d = nullptr;
    cudaError_t e = dalloc((void **)d, (n ? n : 1) * sizeof(T));
    if (e == cudaSuccess) ptrs.push_back(*d);
    return e;
  }
};

cudaError_t device_coarse_topology(Ctx *c, const amgsetup::Topo &T, const std::vector<int> &agg, int nc,
                                   const std::vector<double> &xc, amgsetup::Topo &C) {
  const int k = T.k, d = T.d;
  const size_t kk = (size_t)k * k;
  const long long ne = (long long)T.ei.size();
  // bookkeeping (host): which fine items feed which coarse matrix
  std::vector<long long> key(ne);
  for (long long e = 0; e < ne; ++e) {
    const int I = agg[T.ei[e]], J = agg[T.ej[e]];
    if (I >= 0 && J >= 0)
      key[e] = I == J ? -1 : (long long)std::min(I, J) * nc + std::max(I, J);
    else if ((I >= 0) != (J >= 0))
      key[e] = -2 - (long long)(I >= 0 ? I : J);
    else
      key[e] = -1;
  }
  std::vector<int> vptr(nc + 1, 0), eptr(nc + 1, 0);
  for (int i = 0; i < T.n; ++i)
    if (agg[i] >= 0) ++vptr[agg[i] + 1];
  for (long long e = 0; e < ne; ++e)
    if (key[e] <= -2) ++eptr[-2 - key[e] + 1];
  for (int I = 0; I < nc; ++I) {
    vptr[I + 1] += vptr[I];
    eptr[I + 1] += eptr[I];
  }
  std::vector<int> vlist(std::max(vptr[nc], 1)), elist(std::max(eptr[nc], 1));
  {
    std::vector<int> fv(vptr.begin(), vptr.end() - 1), fe(eptr.begin(), eptr.end() - 1);
    for (int i = 0; i < T.n; ++i)
      if (agg[i] >= 0) vlist[fv[agg[i]]++] = i;
    for (long long e = 0; e < ne; ++e)
      if (key[e] <= -2) elist[fe[-2 - key[e]]++] = (int)e;
  }
  // coarse edges: fine edges grouped by coarse pair (a counting sort by the
  // first coarse vertex, then by the second), ascending fine edge inside
  std::vector<int> bya(nc + 1, 0);
  for (long long e = 0; e < ne; ++e)
    if (key[e] >= 0) ++bya[key[e] / nc + 1];
  for (int I = 0; I < nc; ++I) bya[I + 1] += bya[I];
  std::vector<int> sorted(std::max(bya[nc], 1));
  {
    std::vector<int> f(bya.begin(), bya.end() - 1);
    for (long long e = 0; e < ne; ++e)
      if (key[e] >= 0) sorted[f[key[e] / nc]++] = (int)e;
  }
  std::vector<int> ce(std::max(bya[nc], 1)), cptr, ca, cb;
  for (int I = 0; I < nc; ++I) {
    // stable sort of this group by the second coarse vertex
    std::stable_sort(sorted.begin() + bya[I], sorted.begin() + bya[I + 1],
                     [&](int x, int y) { return key[x] < key[y]; });
    for (int q = bya[I]; q < bya[I + 1]; ++q) {
      ce[q] = sorted[q];
      if (q == bya[I] || key[sorted[q]] != key[sorted[q - 1]]) {
        cptr.push_back(q);
        ca.push_back(I);
        cb.push_back((int)(key[sorted[q]] % nc));
      }
    }
  }
  const int nce = (int)ca.size();
  cptr.push_back(bya[nc]);
  // device transfers
  DevScratch s;
  int *d_vptr, *d_vlist, *d_eptr, *d_elist, *d_ei, *d_ej, *d_agg, *d_cptr, *d_ce, *d_ca, *d_cb;
  double *d_pos, *d_xc, *d_M, *d_E, *d_Mc, *d_Ec;
  AMG_CUDA_TRY(s.put(c, &d_vptr, vptr.data(), vptr.size()));
  AMG_CUDA_TRY(s.put(c, &d_vlist, vlist.data(), vlist.size()));
  AMG_CUDA_TRY(s.put(c, &d_eptr, eptr.data(), eptr.size()));
  AMG_CUDA_TRY(s.put(c, &d_elist, elist.data(), elist.size()));
  AMG_CUDA_TRY(s.put(c, &d_ei, T.ei.data(), T.ei.size()));
  AMG_CUDA_TRY(s.put(c, &d_ej, T.ej.data(), T.ej.size()));
  AMG_CUDA_TRY(s.put(c, &d_agg, agg.data(), agg.size()));
  AMG_CUDA_TRY(s.put(c, &d_cptr, cptr.data(), cptr.size()));
  AMG_CUDA_TRY(s.put(c, &d_ce, ce.data(), ce.size()));
  AMG_CUDA_TRY(s.put(c, &d_ca, ca.data(), ca.size()));
  AMG_CUDA_TRY(s.put(c, &d_cb, cb.data(), cb.size()));
  AMG_CUDA_TRY(s.put(c, &d_pos, T.pos.data(), T.pos.size()));
  AMG_CUDA_TRY(s.put(c, &d_xc, xc.data(), xc.size()));
  AMG_CUDA_TRY(s.put(c, &d_M, T.M.data(), T.M.size()));
  AMG_CUDA_TRY(s.put(c, &d_E, T.E.data(), T.E.size()));
  AMG_CUDA_TRY(s.make(&d_Mc, (size_t)nc * kk));
  AMG_CUDA_TRY(s.make(&d_Ec, (size_t)nce * kk));
  if (d == 2) {
    if (nc) coarse_vertex_kernel<2><<<(nc + 127) / 128, 128, 0, c->stream>>>(
        nc, d_vptr, d_vlist, d_eptr, d_elist, d_ei, d_ej, d_agg, d_pos, d_xc, d_M, d_E, d_Mc);
    if (nce) coarse_edge_kernel<2><<<(nce + 127) / 128, 128, 0, c->stream>>>(
        nce, d_cptr, d_ce, d_ca, d_cb, d_ei, d_ej, d_pos, d_xc, d_E, d_Ec);
  } else {
    if (nc) coarse_vertex_kernel<3><<<(nc + 127) / 128, 128, 0, c->stream>>>(
        nc, d_vptr, d_vlist, d_eptr, d_elist, d_ei, d_ej, d_agg, d_pos, d_xc, d_M, d_E, d_Mc);
    if (nce) coarse_edge_kernel<3><<<(nce + 127) / 128, 128, 0, c->stream>>>(
        nce, d_cptr, d_ce, d_ca, d_cb, d_ei, d_ej, d_pos, d_xc, d_E, d_Ec);
  }
  AMG_CUDA_TRY(cudaGetLastError());
  C = amgsetup::Topo();
  C.n = nc;
  C.d = d;
  C.k = k;
  C.pos = xc;
  C.dir.assign(nc, 0);
  C.M.resize((size_t)nc * kk);
  C.E.resize((size_t)nce * kk);
  C.ei = ca;
  C.ej = cb;
  AMG_CUDA_TRY(cudaMemcpyAsync(C.M.data(), d_Mc, C.M.size() * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
  AMG_CUDA_TRY(cudaMemcpyAsync(C.E.data(), d_Ec, C.E.size() * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
  AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  C.build_adj();
  return cudaSuccess;
}

// ---------------------------------------------------------------- prolongation

constexpr int kMaxRowCols = 16;  // coarse columns of one row of P_s (caps <= 16)

struct ProlongArgs {
  int nrows, first, cap_s, cap_a;
  double omega;
  const int *rowptr, *colidx;  // A_l (level rows)
  const double *a;             // A_l blocks, KR x KR
  const int *rowmap, *row_of;  // level row -> topology vertex, vertex -> row (-1)
  const int *adj_ptr, *adj_nbr, *adj_edge;
  const double *E, *pos, *xc;  // topology edge matrices, positions, coarse positions
  const int *agg;              // agglomerate of every vertex (-1 for D)
  const char *dflag, *bad;     // D vertices, rows that are not kernel-exact
};

// The first KR rows of the tentative block of row r: Q(x_v - x_J).
template <int D, int KR>
__device__ __forceinline__ void tentative_dev(const ProlongArgs &g, int v, int J, double *P) {
  constexpr int K = D == 2 ? 3 : 6, R = K - D;
  double t[D], S[D * R];
  for (int a = 0; a < D; ++a) t[a] = g.pos[(size_t)v * D + a] - g.xc[(size_t)J * D + a];
  skew_dev<D>(t, S);
  for (int i = 0; i < KR; ++i)
    for (int j = 0; j < K; ++j) {
      double q = (i == j) ? 1.0 : 0.0;
      if (i < D && j >= D) q = S[i * R + (j - D)];
      P[i * K + j] = q;
    }
}

template <int N>
__device__ void pinv_dev(const double *A, double *out) {
  double a[N * N], v[N * N];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) a[i * N + j] = 0.5 * (A[i * N + j] + A[j * N + i]);
  jacobi_eig<N>(a, v);
  double wmax = 0.0;
  for (int i = 0; i < N; ++i) wmax = fmax(wmax, fabs(a[i * N + i]));
  for (int i = 0; i < N * N; ++i) out[i] = 0.0;
  if (wmax <= 0.0) return;
  for (int m = 0; m < N; ++m) {
    const double w = a[m * N + m];
    if (!(w > 1e-12 * wmax)) continue;
    const double inv = 1.0 / w;
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) out[i * N + j] += v[i * N + m] * inv * v[j * N + m];
  }
}

// acc[col] += X (KR x K), columns kept in the order they first appear
template <int KRK>
__device__ __forceinline__ bool acc_add(int *cols, double (*acc)[KRK], int &m, int J, const double *X) {
  int q = 0;
  while (q < m && cols[q] != J) ++q;
  if (q == m) {
    if (m == kMaxRowCols) return false;
    cols[m] = J;
    for (int i = 0; i < KRK; ++i) acc[m][i] = 0.0;
    ++m;
  }
  for (int i = 0; i < KRK; ++i) acc[q][i] += X[i];
  return true;
}

// One row of P_s: its coarse columns (ascending) and, when vals is given,
// the blocks.  Returns the column count, or -1 past kMaxRowCols.
template <int D, bool FIRST>
__device__ int prolong_row(const ProlongArgs &g, int r, int *out_cols, double *vals) {
  constexpr int K = D == 2 ? 3 : 6, KR = FIRST ? D : K, KRK = KR * K;
  int cols[kMaxRowCols];
  double acc[kMaxRowCols][KRK];
  double Dinv[KR * KR], X[KRK], Pt[KRK];
  int m = 0;
  const int v = g.rowmap[r];
  const int own = g.agg[v];
  if (!g.dflag[v]) {
    int touched[kMaxRowCols + 1];
    int nt = 0;
    for (int p = g.rowptr[r]; p < g.rowptr[r + 1] && nt <= g.cap_s; ++p) {
      const int w = g.rowmap[g.colidx[p]];
      if (g.dflag[w]) continue;
      const int J = g.agg[w];
      int q = 0;
      while (q < nt && touched[q] != J) ++q;
      if (q == nt) touched[nt++] = J;
    }
    const bool standard = nt <= g.cap_s && !g.bad[r];
    if (standard) {
      double Arr[KR * KR];
      for (int i = 0; i < KR * KR; ++i) Arr[i] = 0.0;
      for (int p = g.rowptr[r]; p < g.rowptr[r + 1]; ++p) {
        const int cc = g.colidx[p];
        const double *Ab = g.a + (size_t)p * KR * KR;
        if (cc == r)
          for (int i = 0; i < KR * KR; ++i) Arr[i] = Ab[i];
        const int w = g.rowmap[cc];
        const int J = g.agg[w];
        if (J < 0) continue;
        tentative_dev<D, KR>(g, w, J, Pt);
        for (int i = 0; i < KR; ++i)
          for (int j = 0; j < K; ++j) {
            double s2 = 0.0;
            for (int l = 0; l < KR; ++l) s2 += Ab[i * KR + l] * Pt[l * K + j];
            X[i * K + j] = s2;
          }
        if (!acc_add<KRK>(cols, acc, m, J, X)) return -1;
      }
      pinv_dev<KR>(Arr, Dinv);
    } else {
      // filtered neighbours: own agglomerate + the cap_a - 1 others with the
      // largest sum of tr E^{il} (ties by agglomerate id)
      int wj[64];
      double ww[64];
      int nw = 0;
      for (int p = g.adj_ptr[v]; p < g.adj_ptr[v + 1]; ++p) {
        const int l = g.adj_nbr[p];
        if (g.dflag[l]) continue;
        const int J = g.agg[l];
        const double *E = g.E + (size_t)g.adj_edge[p] * K * K;
        double tr = 0.0;
        for (int i = 0; i < K; ++i) tr += E[i * K + i];
        int q = 0;
        while (q < nw && wj[q] != J) ++q;
        if (q == nw) {
          if (nw == 64) return -1;
          wj[nw] = J;
          ww[nw] = tr;
          ++nw;
        } else {
          ww[q] += tr;
        }
      }
      int keep[kMaxRowCols];
      int nk = 0;
      keep[nk++] = own;
      for (int round = 0; round < g.cap_a - 1; ++round) {
        int best = -1;
        for (int q = 0; q < nw; ++q) {
          if (wj[q] == own) continue;
          bool taken = false;
          for (int u = 1; u < nk; ++u) taken |= keep[u] == wj[q];
          if (taken) continue;
          if (best < 0 || ww[q] > ww[best] || (ww[q] == ww[best] && wj[q] < wj[best])) best = q;
        }
        if (best < 0) break;
        keep[nk++] = wj[best];
      }
      double Aii[KR * KR];
      for (int i = 0; i < KR * KR; ++i) Aii[i] = 0.0;
      double Z[K * K], tv[D], tl[D];
      for (int p = g.adj_ptr[v]; p < g.adj_ptr[v + 1]; ++p) {
        const int l = g.adj_nbr[p];
        if (g.dflag[l]) continue;
        bool kept = false;
        for (int u = 0; u < nk; ++u) kept |= keep[u] == g.agg[l];
        if (!kept) continue;
        const double *E = g.E + (size_t)g.adj_edge[p] * K * K;
        if (FIRST) {
          for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) Aii[i * KR + j] += E[i * K + j];
        } else {
          for (int a = 0; a < D; ++a) tv[a] = 0.5 * (g.pos[(size_t)l * D + a] - g.pos[(size_t)v * D + a]);
          transfer_dev<D>(tv, tv, E, Z);
          for (int i = 0; i < K * K; ++i) Aii[i] += Z[i];
        }
      }
      pinv_dev<KR>(Aii, Dinv);
      if (own >= 0) {
        tentative_dev<D, KR>(g, v, own, Pt);
        for (int i = 0; i < KR; ++i)
          for (int j = 0; j < K; ++j) {
            double s2 = 0.0;
            for (int l = 0; l < KR; ++l) s2 += Aii[i * KR + l] * Pt[l * K + j];
            X[i * K + j] = s2;
          }
        if (!acc_add<KRK>(cols, acc, m, own, X)) return -1;
      }
      for (int p = g.adj_ptr[v]; p < g.adj_ptr[v + 1]; ++p) {
        const int l = g.adj_nbr[p];
        if (g.dflag[l]) continue;
        bool kept = false;
        for (int u = 0; u < nk; ++u) kept |= keep[u] == g.agg[l];
        if (!kept) continue;
        const int cr = g.row_of[l];
        if (cr < 0) continue;
        const int J = g.agg[g.rowmap[cr]];
        if (J < 0) continue;
        const double *E = g.E + (size_t)g.adj_edge[p] * K * K;
        double Xo[KR * KR];
        if (FIRST) {
          for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) Xo[i * KR + j] = -E[i * K + j];
        } else {
          for (int a = 0; a < D; ++a) {
            tv[a] = 0.5 * (g.pos[(size_t)l * D + a] - g.pos[(size_t)v * D + a]);
            tl[a] = -tv[a];
          }
          transfer_dev<D>(tv, tl, E, Z);
          for (int i = 0; i < K * K; ++i) Xo[i] = -Z[i];
        }
        tentative_dev<D, KR>(g, l, J, Pt);
        for (int i = 0; i < KR; ++i)
          for (int j = 0; j < K; ++j) {
            double s2 = 0.0;
            for (int q = 0; q < KR; ++q) s2 += Xo[i * KR + q] * Pt[q * K + j];
            X[i * K + j] = s2;
          }
        if (!acc_add<KRK>(cols, acc, m, J, X)) return -1;
      }
    }
  }
  // ascending columns (insertion sort of an index permutation)
  int ord[kMaxRowCols];
  for (int q = 0; q < m; ++q) ord[q] = q;
  for (int a = 1; a < m; ++a) {
    const int x = ord[a];
    int b = a - 1;
    while (b >= 0 && cols[ord[b]] > cols[x]) {
      ord[b + 1] = ord[b];
      --b;
    }
    ord[b + 1] = x;
  }
  if (out_cols)
    for (int q = 0; q < m; ++q) out_cols[q] = cols[ord[q]];
  if (vals) {
    if (own >= 0 && !g.dflag[v]) tentative_dev<D, KR>(g, v, own, Pt);
    for (int q = 0; q < m; ++q) {
      const double *Y = acc[ord[q]];
      double *out = vals + (size_t)q * KRK;
      for (int i = 0; i < KR; ++i)
        for (int j = 0; j < K; ++j) {
          double s2 = 0.0;
          for (int l = 0; l < KR; ++l) s2 += Dinv[i * KR + l] * Y[l * K + j];
          const double base = (cols[ord[q]] == own && !g.dflag[v]) ? Pt[i * K + j] : 0.0;
          out[i * K + j] = base - g.omega * s2;
        }
    }
  }
  return m;
}

template <int D, bool FIRST>
__global__ void __launch_bounds__(64) prolong_count_kernel(ProlongArgs g, int *cnt, int *overflow) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.nrows) return;
  const int m = prolong_row<D, FIRST>(g, r, nullptr, nullptr);
  if (m < 0) {
    *overflow = 1;
    cnt[r] = 0;
  } else {
    cnt[r] = m;
  }
}

template <int D, bool FIRST>
__global__ void __launch_bounds__(64) prolong_fill_kernel(ProlongArgs g, const int *rowptr, int *colidx,
                                                          double *vals) {
  constexpr int K = D == 2 ? 3 : 6, KR = FIRST ? D : K;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.nrows) return;
  prolong_row<D, FIRST>(g, r, colidx + rowptr[r], vals + (size_t)rowptr[r] * KR * K);
}

// Coarse vertices reached by a row that is not kernel-exact are not
// kernel-exact on the next level.
__global__ void next_bad_kernel(int nrows, const char *bad, const int *rowptr, const int *colidx,
                                char *next_bad) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows || !bad[r]) return;
  for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) next_bad[colidx[p]] = 1;
}

template <int D, bool FIRST>
static cudaError_t prolong_launch(Ctx *c, const ProlongArgs &g, DevBSR &P, int nc, int *overflow_out) {
  constexpr int K = D == 2 ? 3 : 6, KR = FIRST ? D : K;
  const int n = g.nrows;
  int *cnt = nullptr, *total = nullptr, *ovf = nullptr;
  AMG_CUDA_TRY(dalloc((void **)&cnt, (size_t)(n + 1) * sizeof(int)));
  AMG_CUDA_TRY(dalloc((void **)&total, sizeof(int)));
  AMG_CUDA_TRY(dalloc((void **)&ovf, sizeof(int)));
  AMG_CUDA_TRY(cudaMemsetAsync(ovf, 0, sizeof(int), c->stream));
  AMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)(n + 1) * sizeof(int), c->stream));
  if (n) prolong_count_kernel<D, FIRST><<<(n + 63) / 64, 64, 0, c->stream>>>(g, cnt, ovf);
  AMG_CUDA_TRY(cudaGetLastError());
  AMG_CUDA_TRY(scan_exclusive(c, n + 1, cnt, total));
  int nnzb = 0, of = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&nnzb, total, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  AMG_CUDA_TRY(cudaMemcpyAsync(&of, ovf, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  dfree(total);
  dfree(ovf);
  *overflow_out = of;
  if (of) {
    dfree(cnt);
    return cudaSuccess;
  }
  free_bsr(P);
  P.n_rows = n;
  P.n_cols = nc;
  P.br = KR;
  P.bc = K;
  P.nnzb = nnzb;
  P.rowptr = cnt;
  AMG_CUDA_TRY(dalloc((void **)&P.colidx, (size_t)(nnzb > 0 ? nnzb : 1) * sizeof(int)));
  AMG_CUDA_TRY(dalloc((void **)&P.v64, (size_t)(nnzb > 0 ? nnzb : 1) * KR * K * sizeof(double)));
  if (n) prolong_fill_kernel<D, FIRST><<<(n + 63) / 64, 64, 0, c->stream>>>(g, P.rowptr, P.colidx, P.v64);
  return cudaGetLastError();
}

// P_s of `level` into c->levels[level].P (device) and its host copy; the
// next level's kernel-exactness flags into next_bad.  *handled = 0 if a row
// has more coarse columns than the kernel holds (the host then builds P).
cudaError_t device_prolongation(Ctx *c, int level, const amgsetup::Topo &T, const std::vector<int> &agg,
                                const std::vector<char> &dflag, int nc, const std::vector<double> &xc,
                                const std::vector<int> &rowmap, const std::vector<char> &bad, bool first,
                                const amgsetup::SetupParams &prm, amgsetup::HostBSR &Ph,
                                std::vector<char> &next_bad, int *handled) {
  *handled = 0;
  const int cap_s = first ? prm.cap_S_first : prm.cap_S_later;
  if (cap_s > kMaxRowCols - 1 || prm.cap_A > kMaxRowCols || prm.cap_A < 1) return cudaSuccess;
  Level &L = c->levels[level];
  const int nrows = L.A.n_rows;
  std::vector<int> row_of(T.n, -1);
  for (int r = 0; r < nrows; ++r) row_of[rowmap[r]] = r;
  DevScratch s;
  ProlongArgs g;
  g.nrows = nrows;
  g.first = first;
  g.cap_s = cap_s;
  g.cap_a = prm.cap_A;
  g.omega = prm.omega;
  g.rowptr = L.A.rowptr;
  g.colidx = L.A.colidx;
  g.a = L.A.v64;
  int *d_rowmap, *d_row_of, *d_aptr, *d_anbr, *d_aedge, *d_agg;
  double *d_E, *d_pos, *d_xc;
  char *d_dflag, *d_bad, *d_next;
  AMG_CUDA_TRY(s.put(c, &d_rowmap, rowmap.data(), rowmap.size()));
  AMG_CUDA_TRY(s.put(c, &d_row_of, row_of.data(), row_of.size()));
  AMG_CUDA_TRY(s.put(c, &d_aptr, T.adj_ptr.data(), T.adj_ptr.size()));
  AMG_CUDA_TRY(s.put(c, &d_anbr, T.adj_nbr.data(), T.adj_nbr.size()));
  AMG_CUDA_TRY(s.put(c, &d_aedge, T.adj_edge.data(), T.adj_edge.size()));
  AMG_CUDA_TRY(s.put(c, &d_agg, agg.data(), agg.size()));
  AMG_CUDA_TRY(s.put(c, &d_E, T.E.data(), T.E.size()));
  AMG_CUDA_TRY(s.put(c, &d_pos, T.pos.data(), T.pos.size()));
  AMG_CUDA_TRY(s.put(c, &d_xc, xc.data(), xc.size()));
  AMG_CUDA_TRY(s.put(c, &d_dflag, dflag.data(), dflag.size()));
  AMG_CUDA_TRY(s.put(c, &d_bad, bad.data(), bad.size()));
  AMG_CUDA_TRY(s.make(&d_next, (size_t)nc));
  AMG_CUDA_TRY(cudaMemsetAsync(d_next, 0, (size_t)(nc > 0 ? nc : 1), c->stream));
  g.rowmap = d_rowmap;
  g.row_of = d_row_of;
  g.adj_ptr = d_aptr;
  g.adj_nbr = d_anbr;
  g.adj_edge = d_aedge;
  g.E = d_E;
  g.pos = d_pos;
  g.xc = d_xc;
  g.agg = d_agg;
  g.dflag = d_dflag;
  g.bad = d_bad;
  int overflow = 0;
  cudaError_t le;
  if (T.d == 2)
    le = first ? prolong_launch<2, true>(c, g, L.P, nc, &overflow)
               : prolong_launch<2, false>(c, g, L.P, nc, &overflow);
  else
    le = first ? prolong_launch<3, true>(c, g, L.P, nc, &overflow)
               : prolong_launch<3, false>(c, g, L.P, nc, &overflow);
  AMG_CUDA_TRY(le);
  if (overflow) return cudaSuccess;
  const DevBSR &P = L.P;
  if (nrows) next_bad_kernel<<<(nrows + 127) / 128, 128, 0, c->stream>>>(nrows, d_bad, P.rowptr,
                                                                         P.colidx, d_next);
  AMG_CUDA_TRY(cudaGetLastError());
  Ph.n_rows = P.n_rows;
  Ph.n_cols = P.n_cols;
  Ph.br = P.br;
  Ph.bc = P.bc;
  Ph.rowptr.resize(P.n_rows + 1);
  Ph.colidx.resize(P.nnzb);
  Ph.vals.resize((size_t)P.nnzb * P.br * P.bc);
  next_bad.assign(nc, 0);
  AMG_CUDA_TRY(cudaMemcpyAsync(Ph.rowptr.data(), P.rowptr, (P.n_rows + 1) * sizeof(int),
                               cudaMemcpyDeviceToHost, c->stream));
  if (P.nnzb) {
    AMG_CUDA_TRY(cudaMemcpyAsync(Ph.colidx.data(), P.colidx, P.nnzb * sizeof(int), cudaMemcpyDeviceToHost,
                                 c->stream));
    AMG_CUDA_TRY(cudaMemcpyAsync(Ph.vals.data(), P.v64, Ph.vals.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, c->stream));
  }
  if (nc)
    AMG_CUDA_TRY(cudaMemcpyAsync(next_bad.data(), d_next, (size_t)nc, cudaMemcpyDeviceToHost, c->stream));
  AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  *handled = 1;
  return cudaSuccess;
}

// ---------------------------------------------------------------- pair measure

// Eigen-decomposition of the symmetric part of A (w eigenvalues, V columns).
template <int K>
__device__ void sym_eig_dev(const double *A, double *w, double *V) {
  double a[K * K];
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j) a[i * K + j] = 0.5 * (A[i * K + j] + A[j * K + i]);
  jacobi_eig<K>(a, V);
  for (int i = 0; i < K; ++i) w[i] = a[i * K + i];
}

// H(A, B) = A (A + B)^+ B, symmetrised (the harmonic mean of Lemma mu2)
template <int K>
__device__ void harmonic_dev(const double *A, const double *B, double *H) {
  double S[K * K], P[K * K], T[K * K];
  for (int i = 0; i < K * K; ++i) S[i] = A[i] + B[i];
  pinv_dev<K>(S, P);
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j) {
      double s = 0.0;
      for (int l = 0; l < K; ++l) s += P[i * K + l] * B[l * K + j];
      T[i * K + j] = s;
    }
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j) {
      double s = 0.0;
      for (int l = 0; l < K; ++l) s += A[i * K + l] * T[l * K + j];
      S[i * K + j] = s;
    }
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j) H[i * K + j] = 0.5 * (S[i * K + j] + S[j * K + i]);
}

// The smallest mu with L <= mu R on the range of R (eigenvalues of R above
// 1e-10 of its largest); +inf when L has energy (above 1e-8 of its largest
// eigenvalue) on the kernel of R.
template <int K>
__device__ double gen_lambda_max_dev(const double *L, const double *R) {
  double wl[K], Vl[K * K], wr[K], Vr[K * K];
  sym_eig_dev<K>(L, wl, Vl);
  double lmax = 0.0;
  for (int i = 0; i < K; ++i) lmax = fmax(lmax, wl[i]);
  if (lmax <= 0.0) return 0.0;
  sym_eig_dev<K>(R, wr, Vr);
  double rmax = 0.0;
  for (int i = 0; i < K; ++i) rmax = fmax(rmax, wr[i]);
  if (rmax <= 0.0) return INFINITY;
  double Sr[K * K], Kr[K * K];
  int nr = 0, nk = 0;
  for (int m = 0; m < K; ++m) {
    if (wr[m] > 1e-10 * rmax) {
      const double sc = 1.0 / sqrt(wr[m]);
      for (int i = 0; i < K; ++i) Sr[i * K + nr] = Vr[i * K + m] * sc;
      ++nr;
    } else {
      for (int i = 0; i < K; ++i) Kr[i * K + nk] = Vr[i * K + m];
      ++nk;
    }
  }
  // C = B^T L B for the columns B (n x m, stride K), returned m x m (stride K)
  auto project = [&](const double *Bc, int m, double *C) {
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        double s = 0.0;
        for (int i = 0; i < K; ++i) {
          double li = 0.0;
          for (int j = 0; j < K; ++j) li += L[i * K + j] * Bc[j * K + b];
          s += Bc[i * K + a] * li;
        }
        C[a * K + b] = s;
      }
  };
  double C[K * K], Cm[K * K], w[K], V[K * K];
  if (nk > 0) {
    project(Kr, nk, C);
    // eigenvalues of the nk x nk leading block
    for (int i = 0; i < K * K; ++i) Cm[i] = 0.0;
    for (int a = 0; a < nk; ++a)
      for (int b = 0; b < nk; ++b) Cm[a * K + b] = C[a * K + b];
    sym_eig_dev<K>(Cm, w, V);
    double leak = -INFINITY;
    // the padding rows / columns add zero eigenvalues; the leak is the
    // largest eigenvalue of the nk x nk block, which is >= 0 here as L >= 0
    for (int i = 0; i < K; ++i) leak = fmax(leak, w[i]);
    if (leak > 1e-8 * lmax) return INFINITY;
  }
  project(Sr, nr, C);
  for (int i = 0; i < K * K; ++i) Cm[i] = 0.0;
  for (int a = 0; a < nr; ++a)
    for (int b = 0; b < nr; ++b) Cm[a * K + b] = C[a * K + b];
  sym_eig_dev<K>(Cm, w, V);
  double mu = 0.0;
  for (int i = 0; i < K; ++i) mu = fmax(mu, w[i]);
  return mu;
}

struct PairArgs {
  int n, delta;
  const double *pos, *E, *Dh;  // pass topology: positions, edge matrices, D-hat blocks
  const int *adj_ptr, *adj_nbr, *adj_edge;
};

// Lemma mu2: mu_p^delta(v_i, v_j) of one candidate pair (one thread).
template <int D>
__global__ void __launch_bounds__(64) mu_p_kernel(PairArgs g, int n_pairs, const int *__restrict__ pairs,
                                                  double *__restrict__ mu_out) {
  constexpr int K = D == 2 ? 3 : 6, KK = K * K;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_pairs) return;
  const int i = pairs[2 * q], j = pairs[2 * q + 1];
  double t[D], A[KK], B[KK], Lm[KK], R[KK], X[KK], Y[KK], H[KK];
  for (int a = 0; a < D; ++a) t[a] = 0.5 * (g.pos[(size_t)i * D + a] - g.pos[(size_t)j * D + a]);
  transfer_dev<D>(t, t, g.Dh + (size_t)i * KK, A);  // Q^{ji, T} D_ii Q^{ji}
  for (int a = 0; a < D; ++a) t[a] = -t[a];
  transfer_dev<D>(t, t, g.Dh + (size_t)j * KK, B);  // Q^{ij, T} D_jj Q^{ij}
  harmonic_dev<K>(A, B, Lm);
  // the edge (i, j): its slot in i's sorted neighbour list
  int e = -1;
  {
    int lo = g.adj_ptr[i], hi = g.adj_ptr[i + 1];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (g.adj_nbr[mid] < j) lo = mid + 1; else hi = mid;
    }
    if (lo < g.adj_ptr[i + 1] && g.adj_nbr[lo] == j) e = g.adj_edge[lo];
  }
  if (e < 0) {
    mu_out[q] = INFINITY;
    return;
  }
  for (int s = 0; s < KK; ++s) R[s] = g.E[(size_t)e * KK + s];
  if (g.delta) {
    int p = g.adj_ptr[i], r = g.adj_ptr[j];
    const int pe = g.adj_ptr[i + 1], re = g.adj_ptr[j + 1];
    while (p < pe && r < re) {
      const int a = g.adj_nbr[p], b = g.adj_nbr[r];
      if (a < b) {
        ++p;
      } else if (b < a) {
        ++r;
      } else {
        const int l = a;
        for (int s = 0; s < D; ++s) t[s] = 0.5 * (g.pos[(size_t)i * D + s] - g.pos[(size_t)l * D + s]);
        transfer_dev<D>(t, t, g.E + (size_t)g.adj_edge[p] * KK, X);   // Q^{li}
        for (int s = 0; s < D; ++s) t[s] = 0.5 * (g.pos[(size_t)j * D + s] - g.pos[(size_t)l * D + s]);
        transfer_dev<D>(t, t, g.E + (size_t)g.adj_edge[r] * KK, Y);   // Q^{lj}
        harmonic_dev<K>(X, Y, H);
        // pulled back with Q^{v_i -> v_l} Q^{ji}: one shift x_l - (x_i + x_j)/2
        for (int s = 0; s < D; ++s)
          t[s] = g.pos[(size_t)l * D + s] - 0.5 * (g.pos[(size_t)i * D + s] + g.pos[(size_t)j * D + s]);
        transfer_dev<D>(t, t, H, X);
        for (int s = 0; s < KK; ++s) R[s] += 0.5 * g.delta * X[s];
        ++p;
        ++r;
      }
    }
  }
  mu_out[q] = gen_lambda_max_dev<K>(Lm, R);
}

// Device evaluation of mu_p for the batches of one matching pass: the
// pass's topology is uploaded once (begin_pass), every batch of pairs is one
// launch.
struct DevicePairMeasure : amgsetup::PairMeasure {
  Ctx *c;
  DevScratch buf;
  PairArgs g{};
  int d = 0;
  int *d_pairs = nullptr;
  double *d_mu = nullptr;
  size_t cap = 0;
  explicit DevicePairMeasure(Ctx *cc) : c(cc) {}
  int begin_pass(const amgsetup::Topo &T, const std::vector<double> &Dh, int delta) override {
    const auto t0 = std::chrono::steady_clock::now();
    const int rc = begin_pass_impl(T, Dh, delta);
    c->setup_times[5] += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
  }
  int begin_pass_impl(const amgsetup::Topo &T, const std::vector<double> &Dh, int delta) {
    for (void *p : buf.ptrs) dfree(p);
    buf.ptrs.clear();
    d_pairs = nullptr;
    d_mu = nullptr;
    cap = 0;
    d = T.d;
    g.n = T.n;
    g.delta = delta;
    double *pos, *E, *dh;
    int *ap, *an, *ae;
    if (buf.put(c, &pos, T.pos.data(), T.pos.size()) != cudaSuccess ||
        buf.put(c, &E, T.E.data(), T.E.size()) != cudaSuccess ||
        buf.put(c, &dh, Dh.data(), Dh.size()) != cudaSuccess ||
        buf.put(c, &ap, T.adj_ptr.data(), T.adj_ptr.size()) != cudaSuccess ||
        buf.put(c, &an, T.adj_nbr.data(), T.adj_nbr.size()) != cudaSuccess ||
        buf.put(c, &ae, T.adj_edge.data(), T.adj_edge.size()) != cudaSuccess)
      return -1;
    g.pos = pos;
    g.E = E;
    g.Dh = dh;
    g.adj_ptr = ap;
    g.adj_nbr = an;
    g.adj_edge = ae;
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? 0 : -1;
  }
  int evaluate(const std::vector<std::array<int, 2>> &pairs, std::vector<double> &mu) override {
    const auto t0 = std::chrono::steady_clock::now();
    const int rc = evaluate_impl(pairs, mu);
    c->setup_times[5] += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
  }
  int evaluate_impl(const std::vector<std::array<int, 2>> &pairs, std::vector<double> &mu) {
    const size_t n = pairs.size();
    mu.resize(n);
    if (n == 0) return 0;
    if (n > cap) {
      if (d_pairs) dfree(d_pairs);
      if (d_mu) dfree(d_mu);
      d_pairs = nullptr;
      d_mu = nullptr;
      cap = std::max(n, (size_t)4096);
      if (dalloc((void **)&d_pairs, cap * 2 * sizeof(int)) != cudaSuccess ||
          dalloc((void **)&d_mu, cap * sizeof(double)) != cudaSuccess)
        return -1;
    }
    if (cudaMemcpyAsync(d_pairs, pairs.data(), n * 2 * sizeof(int), cudaMemcpyHostToDevice, c->stream) !=
        cudaSuccess)
      return -1;
    const int nb = (int)((n + 63) / 64);
    if (d == 2)
      mu_p_kernel<2><<<nb, 64, 0, c->stream>>>(g, (int)n, d_pairs, d_mu);
    else
      mu_p_kernel<3><<<nb, 64, 0, c->stream>>>(g, (int)n, d_pairs, d_mu);
    if (cudaGetLastError() != cudaSuccess) return -1;
    if (cudaMemcpyAsync(mu.data(), d_mu, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
        cudaSuccess)
      return -1;
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? 0 : -1;
  }
  ~DevicePairMeasure() override {
    if (d_pairs) dfree(d_pairs);
    if (d_mu) dfree(d_mu);
  }
};

amgsetup::PairMeasure *make_device_pair_measure(Ctx *c) { return new DevicePairMeasure(c); }

}  // namespace amg
