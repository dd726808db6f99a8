// Multi-right-hand-side (NR load cases) forms of the V-cycle and CG kernels,
// for several load cases of one system solved together: vectors are
// interleaved per dof (entry (i*k + r) * NR + j for vertex i, dof r, load
// case j), so every matrix block read serves all NR load cases.  The
// arithmetic of every load case is the same, in the same order, as in the
// single-load-case kernels of bsr_kernels.cu / pcg.cu.
#include "amg_internal.h"
#include "multirhs.h"

namespace amg {

template <typename T>
struct AccM {
  using type = float;
};
template <>
struct AccM<double> {
  using type = double;
};

__device__ __forceinline__ double mld(const double *p) { return __ldg(p); }
__device__ __forceinline__ float mld(const float *p) { return __ldg(p); }
__device__ __forceinline__ double mlds(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float mlds(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float mlds(const __nv_bfloat16 *p) {
  unsigned short u = __ldcs(reinterpret_cast<const unsigned short *>(p));
  return __uint_as_float(((unsigned)u) << 16);
}

// ---------------------------------------------------------------------------
// SELL-32 SpMM (thread per block row)
// ---------------------------------------------------------------------------
template <int BR, int BC, int NR, typename V, typename T, int MODE, typename TO>
__global__ void __launch_bounds__(64) sell_mr_kernel(int n_rows, int n_slices,
                                                     const int *__restrict__ sell_ptr,
                                                     const int *__restrict__ sell_col,
                                                     const V *__restrict__ vals,
                                                     const T *__restrict__ x,
                                                     const T *__restrict__ b,
                                                     const T *__restrict__ minv,
                                                     TO *__restrict__ y) {
  using A = typename AccM<T>::type;
  constexpr int E = BR * BC;
  const int slice = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (slice >= n_slices) return;
  const int t = threadIdx.x & 31;
  const int row = slice * 32 + t;
  const int j0 = sell_ptr[slice], j1 = sell_ptr[slice + 1];
  A acc[BR][NR];
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[r][j] = 0;
  for (int s = j0; s < j1; ++s) {
    const int c = __ldg(sell_col + (size_t)s * 32 + t);
    const V *v = vals + (size_t)s * E * 32 + t;
    A a[E];
#pragma unroll
    for (int e = 0; e < E; ++e) a[e] = (A)mlds(v + e * 32);
    const T *xp = x + (size_t)c * BC * NR;
#pragma unroll
    for (int q = 0; q < BC; ++q) {
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const A xv = (A)mld(xp + q * NR + j);
#pragma unroll
        for (int r = 0; r < BR; ++r) acc[r][j] += a[r * BC + q] * xv;
      }
    }
  }
  if (row >= n_rows) return;
  const size_t o = (size_t)row * BR;
  if (MODE == SPMV_SMOOTH) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      A res[BR];
#pragma unroll
      for (int r = 0; r < BR; ++r) res[r] = (A)b[(o + r) * NR + j] - acc[r][j];
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        A u = 0;
#pragma unroll
        for (int q = 0; q < BR; ++q) u += (A)minv[(o + r) * BR + q] * res[q];
        y[(o + r) * NR + j] = (TO)((A)x[(o + r) * NR + j] + u);
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const size_t i = (o + r) * NR + j;
        if (MODE == SPMV_SET) y[i] = (TO)acc[r][j];
        if (MODE == SPMV_RESID) y[i] = (TO)((A)b[i] - acc[r][j]);
        if (MODE == SPMV_ADD) y[i] = (TO)((A)y[i] + acc[r][j]);
      }
  }
}

// ---------------------------------------------------------------------------
// warp-per-row SpMM (long rows): lane (slot b, row r) streams row r of every
// NB-th block; NR accumulators per lane, shuffle reduction per load case.
// ---------------------------------------------------------------------------
template <int BR, int BC, int NR, typename V, typename T, int MODE, typename TO>
__global__ void __launch_bounds__(256) warp_mr_kernel(int n_rows, const int *__restrict__ rowptr,
                                                      const int *__restrict__ colidx,
                                                      const V *__restrict__ vals,
                                                      const T *__restrict__ x,
                                                      const T *__restrict__ b,
                                                      const T *__restrict__ minv,
                                                      TO *__restrict__ y) {
  using A = typename AccM<T>::type;
  constexpr int NB = 32 / BR;
  const int lane = threadIdx.x & 31;
  const int bl = lane / BR;
  const int r = lane - bl * BR;
  const bool active = bl < NB;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n_rows; row += nwarps) {
    const int s = rowptr[row], e = rowptr[row + 1];
    A acc[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[j] = 0;
    if (active) {
      for (int p = s + bl; p < e; p += NB) {
        const int c = __ldg(colidx + p);
        const V *v = vals + ((size_t)p * BR + r) * BC;
        const T *xp = x + (size_t)c * BC * NR;
#pragma unroll
        for (int q = 0; q < BC; ++q) {
          const A a = (A)mlds(v + q);
#pragma unroll
          for (int j = 0; j < NR; ++j) acc[j] += a * (A)mld(xp + q * NR + j);
        }
      }
    }
#pragma unroll
    for (int sft = 1; sft < NB; sft <<= 1) {
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const A o2 = __shfl_down_sync(0xffffffffu, acc[j], sft * BR);
        if (bl + sft < NB) acc[j] += o2;
      }
    }
    const size_t o = (size_t)row * BR;
    if (MODE == SPMV_SMOOTH) {
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const A res = (lane < BR) ? (A)b[(o + lane) * NR + j] - acc[j] : (A)0;
        A upd = 0;
#pragma unroll
        for (int q = 0; q < BR; ++q) {
          const A rq = __shfl_sync(0xffffffffu, res, q);
          if (lane < BR) upd += (A)minv[(o + lane) * BR + q] * rq;
        }
        if (lane < BR) y[(o + lane) * NR + j] = (TO)((A)x[(o + lane) * NR + j] + upd);
      }
    } else if (lane < BR) {
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const size_t i = (o + lane) * NR + j;
        if (MODE == SPMV_SET) y[i] = (TO)acc[j];
        if (MODE == SPMV_RESID) y[i] = (TO)((A)b[i] - acc[j]);
        if (MODE == SPMV_ADD) y[i] = (TO)((A)y[i] + acc[j]);
      }
    }
  }
}

template <int BR, int BC, int NR, typename V, typename T, typename TO>
static cudaError_t mr_launch_vt(const Ctx *c, const DevBSR &A, const V *bsr_v, const V *sell_v,
                                int mode, const void *x, const void *b, const void *minv, void *y) {
  const T *xx = (const T *)x;
  const T *bb = (const T *)b;
  const T *mm = (const T *)minv;
  TO *yy = (TO *)y;
  if (A.sell_ptr) {
    const int g = (A.n_slices + 1) / 2;
#define AMG_MR_SELL(M_)                                                                  \
  sell_mr_kernel<BR, BC, NR, V, T, M_, TO><<<g, 64, 0, c->stream>>>(                    \
      A.n_rows, A.n_slices, A.sell_ptr, A.sell_col, sell_v, xx, bb, mm, yy)
    switch (mode) {
      case SPMV_SET: AMG_MR_SELL(SPMV_SET); break;
      case SPMV_RESID: AMG_MR_SELL(SPMV_RESID); break;
      case SPMV_ADD: AMG_MR_SELL(SPMV_ADD); break;
      case SPMV_SMOOTH: AMG_MR_SELL(SPMV_SMOOTH); break;
      default: return cudaErrorInvalidValue;
    }
#undef AMG_MR_SELL
  } else {
    long want = ((long)A.n_rows + 7) / 8;
    const long cap = (long)c->num_sms * 8;
    if (want > cap) want = cap;
    const int g = (int)(want < 1 ? 1 : want);
#define AMG_MR_WARP(M_)                                                                    \
  warp_mr_kernel<BR, BC, NR, V, T, M_, TO><<<g, 256, 0, c->stream>>>(A.n_rows, A.rowptr,  \
                                                                     A.colidx, bsr_v, xx, \
                                                                     bb, mm, yy)
    switch (mode) {
      case SPMV_SET: AMG_MR_WARP(SPMV_SET); break;
      case SPMV_RESID: AMG_MR_WARP(SPMV_RESID); break;
      case SPMV_ADD: AMG_MR_WARP(SPMV_ADD); break;
      case SPMV_SMOOTH: AMG_MR_WARP(SPMV_SMOOTH); break;
      default: return cudaErrorInvalidValue;
    }
#undef AMG_MR_WARP
  }
  return cudaGetLastError();
}

template <int BR, int BC, int NR>
static cudaError_t mr_launch_shape(const Ctx *c, const DevBSR &A, int prec, int mode,
                                   const void *x, const void *b, const void *minv, void *y,
                                   bool y_fp64) {
  if (A.n_rows == 0) return cudaSuccess;
  if ((mode == SPMV_SMOOTH) && BR != BC) return cudaErrorInvalidValue;
  if (prec == AMG_PREC_FP64)
    return mr_launch_vt<BR, BC, NR, double, double, double>(c, A, A.v64, A.s64, mode, x, b, minv, y);
  if (prec == AMG_PREC_FP32_VCYCLE) {
    if (y_fp64)
      return mr_launch_vt<BR, BC, NR, float, float, double>(c, A, A.v32, A.s32, mode, x, b, minv, y);
    return mr_launch_vt<BR, BC, NR, float, float, float>(c, A, A.v32, A.s32, mode, x, b, minv, y);
  }
  if (y_fp64)
    return mr_launch_vt<BR, BC, NR, __nv_bfloat16, float, double>(c, A, A.v16, A.s16, mode, x, b, minv, y);
  return mr_launch_vt<BR, BC, NR, __nv_bfloat16, float, float>(c, A, A.v16, A.s16, mode, x, b, minv, y);
}

template <int NR>
static cudaError_t mr_launch_nr(const Ctx *c, const DevBSR &A, int prec, int mode, const void *x,
                                const void *b, const void *minv, void *y, bool y_fp64) {
#define AMG_MR_CASE(R_, C_) \
  if (A.br == R_ && A.bc == C_) return mr_launch_shape<R_, C_, NR>(c, A, prec, mode, x, b, minv, y, y_fp64);
  AMG_MR_CASE(2, 2)
  AMG_MR_CASE(3, 3)
  AMG_MR_CASE(6, 6)
  AMG_MR_CASE(2, 3)
  AMG_MR_CASE(3, 2)
  AMG_MR_CASE(3, 6)
  AMG_MR_CASE(6, 3)
#undef AMG_MR_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_bsr_mr(const Ctx *c, const DevBSR &A, int prec, int nr, int mode, const void *x,
                          const void *b, const void *minv, void *y, bool y_fp64) {
  if (nr == 1) return mr_launch_nr<1>(c, A, prec, mode, x, b, minv, y, y_fp64);
  if (nr == 6) return mr_launch_nr<6>(c, A, prec, mode, x, b, minv, y, y_fp64);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// block-diagonal apply y = M^+ b per vertex (NR load cases); the entry form
// reads the FP64 residual and also stores its V-cycle-precision copy.
// ---------------------------------------------------------------------------
template <int K, int NR, typename T, typename TI>
__global__ void blockdiag_mr_kernel(int n, const T *__restrict__ minv, const TI *__restrict__ bin,
                                    T *__restrict__ bcopy, T *__restrict__ y) {
  using A = typename AccM<T>::type;
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= (size_t)n) return;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    A rb[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const T bv = (T)bin[(v * K + q) * NR + j];
      rb[q] = (A)bv;
      if (bcopy) bcopy[(v * K + q) * NR + j] = bv;
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
      A acc = 0;
#pragma unroll
      for (int q = 0; q < K; ++q) acc += (A)minv[(v * K + i) * K + q] * rb[q];
      y[(v * K + i) * NR + j] = (T)acc;
    }
  }
}

template <int K, int NR>
static cudaError_t blockdiag_mr_k(const Ctx *c, int n, int prec, const void *minv, const void *bin,
                                  bool bin_fp64, void *bcopy, void *y) {
  const int g = (n + 127) / 128;
  if (prec == AMG_PREC_FP64)
    blockdiag_mr_kernel<K, NR, double, double><<<g, 128, 0, c->stream>>>(
        n, (const double *)minv, (const double *)bin, (double *)bcopy, (double *)y);
  else if (bin_fp64)
    blockdiag_mr_kernel<K, NR, float, double><<<g, 128, 0, c->stream>>>(
        n, (const float *)minv, (const double *)bin, (float *)bcopy, (float *)y);
  else
    blockdiag_mr_kernel<K, NR, float, float><<<g, 128, 0, c->stream>>>(
        n, (const float *)minv, (const float *)bin, (float *)bcopy, (float *)y);
  return cudaGetLastError();
}

cudaError_t launch_blockdiag_mr(const Ctx *c, int n, int k, int prec, int nr, const void *minv,
                                const void *bin, bool bin_fp64, void *bcopy, void *y) {
  if (n == 0) return cudaSuccess;
#define AMG_BD(K_, NR_) \
  if (k == K_ && nr == NR_) return blockdiag_mr_k<K_, NR_>(c, n, prec, minv, bin, bin_fp64, bcopy, y);
  AMG_BD(2, 1) AMG_BD(3, 1) AMG_BD(6, 1) AMG_BD(2, 6) AMG_BD(3, 6) AMG_BD(6, 6)
#undef AMG_BD
  return cudaErrorInvalidValue;
}

// coarsest level: Y = Cinv B for NR interleaved columns (one warp per row)
template <int NR, typename T>
__global__ void coarse_gemm_mr_kernel(int n, const double *__restrict__ cinv, const T *__restrict__ b,
                                      T *__restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const double *a = cinv + (size_t)row * n;
  double acc[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = 0.0;
  for (int q = lane; q < n; q += 32) {
    const double av = a[q];
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[j] += av * (double)b[(size_t)q * NR + j];
  }
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    for (int s = 16; s > 0; s >>= 1) acc[j] += __shfl_down_sync(0xffffffffu, acc[j], s);
    if (lane == 0) y[(size_t)row * NR + j] = (T)acc[j];
  }
}

cudaError_t launch_coarse_mr(const Ctx *c, int n, int nr, const double *cinv, const void *b, void *y,
                             int prec) {
  if (n == 0) return cudaSuccess;
  const int g = (n + 7) / 8;
  if (nr == 1) {
    if (prec == AMG_PREC_FP64)
      coarse_gemm_mr_kernel<1, double><<<g, 256, 0, c->stream>>>(n, cinv, (const double *)b, (double *)y);
    else
      coarse_gemm_mr_kernel<1, float><<<g, 256, 0, c->stream>>>(n, cinv, (const float *)b, (float *)y);
  } else if (nr == 6) {
    if (prec == AMG_PREC_FP64)
      coarse_gemm_mr_kernel<6, double><<<g, 256, 0, c->stream>>>(n, cinv, (const double *)b, (double *)y);
    else
      coarse_gemm_mr_kernel<6, float><<<g, 256, 0, c->stream>>>(n, cinv, (const float *)b, (float *)y);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace amg
