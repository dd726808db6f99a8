// Setup kernels of the smoother and the coarsest level (FP64):
//  - block-l1 smoother blocks M_v = A_vv + diag(sum_{c outside v} |a_rc|)
//    (Sec. 7, block version of the l1 smoother) and their pseudo-inverse
//    (Sec. 3 after Lemma eet_is_diag, pseudo smoother: singular diagonal blocks are pseudo-inverted);
//  - the regularised coarsest matrix A_L + (I - E_L E_L^T), E_L spanning the
//    complement of the kernels of the diagonal blocks (Lemma eet_is_diag,
//    Sec. 3 after Lemma eet_is_diag), and its explicit inverse by Gauss-Jordan elimination.
// Small symmetric eigenproblems use the cyclic Jacobi method (Golub & Van
// Loan, "Matrix Computations", Sec. 8.5), written from the mathematics.
#include <math.h>

#include "amg_internal.h"
#include "dense_dev.cuh"

namespace amg {

constexpr double kKernelRtol = 1e-12;

// One thread per block row: assemble M_v, eigen-decompose, pseudo-invert.
// With colour (hybrid Gauss-Seidel) the l1 term sums only the couplings to
// rows of v's own colour class; without it (block-l1 Jacobi), all of them.
template <int K>
__global__ void l1_pinv_kernel(int n, const int *__restrict__ rowptr, const int *__restrict__ colidx,
                               const double *__restrict__ vals, double *__restrict__ minv,
                               float *__restrict__ minv32, const int *__restrict__ colour) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  double a[K * K], e[K * K], l1[K];
  for (int i = 0; i < K * K; ++i) a[i] = 0.0;
  for (int r = 0; r < K; ++r) l1[r] = 0.0;
  for (int p = rowptr[v]; p < rowptr[v + 1]; ++p) {
    const double *blk = vals + (size_t)p * K * K;
    if (colidx[p] == v) {
      for (int i = 0; i < K * K; ++i) a[i] += blk[i];
    } else if (!colour || colour[colidx[p]] == colour[v]) {
      for (int r = 0; r < K; ++r)
        for (int c = 0; c < K; ++c) l1[r] += fabs(blk[r * K + c]);
    }
  }
  for (int r = 0; r < K; ++r) a[r * K + r] += l1[r];
  // symmetrise (A_vv is symmetric up to rounding of the Galerkin product)
  for (int i = 0; i < K; ++i)
    for (int j = i + 1; j < K; ++j) {
      const double m = 0.5 * (a[i * K + j] + a[j * K + i]);
      a[i * K + j] = m;
      a[j * K + i] = m;
    }
  jacobi_eig<K>(a, e);
  double wmax = 0.0;
  for (int i = 0; i < K; ++i) wmax = fmax(wmax, fabs(a[i * K + i]));
  double out[K * K];
  for (int i = 0; i < K * K; ++i) out[i] = 0.0;
  for (int m = 0; m < K; ++m) {
    const double w = a[m * K + m];
    if (wmax > 0.0 && w > kKernelRtol * wmax) {
      const double inv = 1.0 / w;
      for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) out[i * K + j] += e[i * K + m] * inv * e[j * K + m];
    }
  }
  for (int i = 0; i < K * K; ++i) {
    minv[(size_t)v * K * K + i] = out[i];
    if (minv32) minv32[(size_t)v * K * K + i] = (float)out[i];
  }
}

cudaError_t smoother_setup(Ctx *c, int level) {
  Level &L = c->levels[level];
  const int n = L.A.n_rows, k = L.k;
  const size_t sz = (size_t)n * k * k;
  if (!L.minv64) AMG_CUDA_TRY(dalloc((void **)&L.minv64, sz * sizeof(double)));
  if (c->precision != AMG_PREC_FP64 && !L.minv32)
    AMG_CUDA_TRY(dalloc((void **)&L.minv32, sz * sizeof(float)));
  if (n == 0) return cudaSuccess;
  const int g = (n + 127) / 128;
  float *m32 = (c->precision != AMG_PREC_FP64) ? L.minv32 : nullptr;
  const int *col = c->smoother == AMG_SMOOTHER_HYBRID_GS ? L.gs_colour : nullptr;
  if (k == 1)
    l1_pinv_kernel<1><<<g, 128, 0, c->stream>>>(n, L.A.rowptr, L.A.colidx, L.A.v64, L.minv64, m32, col);
  else if (k == 2)
    l1_pinv_kernel<2><<<g, 128, 0, c->stream>>>(n, L.A.rowptr, L.A.colidx, L.A.v64, L.minv64, m32, col);
  else if (k == 3)
    l1_pinv_kernel<3><<<g, 128, 0, c->stream>>>(n, L.A.rowptr, L.A.colidx, L.A.v64, L.minv64, m32, col);
  else if (k == 6)
    l1_pinv_kernel<6><<<g, 128, 0, c->stream>>>(n, L.A.rowptr, L.A.colidx, L.A.v64, L.minv64, m32, col);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// Scatter the BSR coarsest matrix into a dense n*k x n*k array and add the
// projector onto the kernel of each diagonal block (I - E E^T restricted to
// the block).  One thread per block row.
template <int K>
__global__ void coarse_dense_kernel(int n, const int *__restrict__ rowptr,
                                    const int *__restrict__ colidx, const double *__restrict__ vals,
                                    double *__restrict__ dense) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const size_t N = (size_t)n * K;
  double a[K * K], e[K * K];
  for (int i = 0; i < K * K; ++i) a[i] = 0.0;
  for (int p = rowptr[v]; p < rowptr[v + 1]; ++p) {
    const int cidx = colidx[p];
    const double *blk = vals + (size_t)p * K * K;
    for (int r = 0; r < K; ++r)
      for (int q = 0; q < K; ++q) dense[((size_t)v * K + r) * N + (size_t)cidx * K + q] = blk[r * K + q];
    if (cidx == v)
      for (int i = 0; i < K * K; ++i) a[i] = blk[i];
  }
  for (int i = 0; i < K; ++i)
    for (int j = i + 1; j < K; ++j) {
      const double m = 0.5 * (a[i * K + j] + a[j * K + i]);
      a[i * K + j] = m;
      a[j * K + i] = m;
    }
  jacobi_eig<K>(a, e);
  double wmax = 0.0;
  for (int i = 0; i < K; ++i) wmax = fmax(wmax, fabs(a[i * K + i]));
  for (int m = 0; m < K; ++m) {
    const double w = a[m * K + m];
    const bool kernel = (wmax > 0.0) ? (w <= kKernelRtol * wmax) : true;
    if (!kernel) continue;
    for (int r = 0; r < K; ++r)
      for (int q = 0; q < K; ++q)
        dense[((size_t)v * K + r) * N + (size_t)v * K + q] += e[r * K + m] * e[q * K + m];
  }
}

// Gauss-Jordan step k: save pivot row and column, then eliminate.
__global__ void gj_save_kernel(int N, int k, const double *__restrict__ a, double *__restrict__ row,
                               double *__restrict__ col) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  row[i] = a[(size_t)k * N + i];
  col[i] = a[(size_t)i * N + k];
}

__global__ void gj_update_kernel(int N, int k, double *__restrict__ a, const double *__restrict__ row,
                                 const double *__restrict__ col) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)N * N) return;
  const int i = (int)(t / N), j = (int)(t % N);
  const double piv = row[k];
  const double rk = (j == k) ? 1.0 : row[j];  // after the step column k holds the inverse's column
  if (i == k) {
    a[t] = rk / piv;
  } else {
    const double f = col[i] / piv;
    a[t] = ((j == k) ? 0.0 : a[t]) - f * rk;
  }
}

cudaError_t coarse_setup(Ctx *c) {
  Level &L = c->levels.back();
  const int n = L.A.n_rows, k = L.k;
  const int N = n * k;
  c->coarse_n = N;
  dfree(c->cinv);
  c->cinv = nullptr;
  if (N == 0) return cudaSuccess;
  AMG_CUDA_TRY(dalloc((void **)&c->cinv, (size_t)N * N * sizeof(double)));
  AMG_CUDA_TRY(cudaMemsetAsync(c->cinv, 0, (size_t)N * N * sizeof(double), c->stream));
  const int g = (n + 127) / 128;
  if (k == 1)
    coarse_dense_kernel<1><<<g, 128, 0, c->stream>>>(n, L.A.rowptr, L.A.colidx, L.A.v64, c->cinv);
  else if (k == 2)
    coarse_dense_kernel<2><<<g, 128, 0, c->stream>>>(n, L.A.rowptr, L.A.colidx, L.A.v64, c->cinv);
  else if (k == 3)
    coarse_dense_kernel<3><<<g, 128, 0, c->stream>>>(n, L.A.rowptr, L.A.colidx, L.A.v64, c->cinv);
  else if (k == 6)
    coarse_dense_kernel<6><<<g, 128, 0, c->stream>>>(n, L.A.rowptr, L.A.colidx, L.A.v64, c->cinv);
  else
    return cudaErrorInvalidValue;
  AMG_CUDA_TRY(cudaGetLastError());
  double *tmp = nullptr;
  AMG_CUDA_TRY(dalloc((void **)&tmp, 2 * (size_t)N * sizeof(double)));
  const int g1 = (N + 255) / 256;
  const int g2 = (int)(((size_t)N * N + 255) / 256);
  for (int s = 0; s < N; ++s) {
    gj_save_kernel<<<g1, 256, 0, c->stream>>>(N, s, c->cinv, tmp, tmp + N);
    gj_update_kernel<<<g2, 256, 0, c->stream>>>(N, s, c->cinv, tmp, tmp + N);
  }
  cudaError_t e = cudaGetLastError();
  cudaStreamSynchronize(c->stream);
  dfree(tmp);
  return e;
}

}  // namespace amg
