// Grouped kernels of the batched solve: one launch per V-cycle / CG step for
// all systems of a batch (item tables in batch_kernels.h).  The arithmetic of
// every load case follows the single-system kernels: block-sparse products
// with FP64 (FP64 operators) or FP32 (FP32 / BF16 operators) accumulation,
// block-l1 Jacobi steps, dense coarsest solve in FP64, FP64 CG scalars.
#include <cuda_bf16.h>

#include "batch_kernels.h"
#include "df_arith.cuh"

namespace amg {

template <typename T>
struct GAcc {
  using type = float;
};
template <>
struct GAcc<double> {
  using type = double;
};

__device__ __forceinline__ double gld(const double *p) { return __ldg(p); }
__device__ __forceinline__ float gld(const float *p) { return __ldg(p); }
// matrix values are read once per product: streaming loads
__device__ __forceinline__ double glds(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float glds(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float glds(const __nv_bfloat16 *p) {
  const unsigned short u = __ldcs(reinterpret_cast<const unsigned short *>(p));
  return __uint_as_float(((unsigned)u) << 16);
}

// the NR load cases of one dof: for NR = 6 they sit 48 (FP64) or 24 (FP32)
// bytes apart from a 16 / 8-byte aligned start, so three vector loads do
template <int NR, typename A>
__device__ __forceinline__ void gld_nr(const double *p, A (&v)[NR]) {
  if constexpr (NR == 6) {
    const double2 a = __ldg((const double2 *)p), b = __ldg((const double2 *)p + 1),
                  c = __ldg((const double2 *)p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
  } else {
#pragma unroll
    for (int j = 0; j < NR; ++j) v[j] = (A)__ldg(p + j);
  }
}
template <int NR, typename A>
__device__ __forceinline__ void gld_nr(const float *p, A (&v)[NR]) {
  if constexpr (NR == 6) {
    const float2 a = __ldg((const float2 *)p), b = __ldg((const float2 *)p + 1),
                 c = __ldg((const float2 *)p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
  } else {
#pragma unroll
    for (int j = 0; j < NR; ++j) v[j] = (A)__ldg(p + j);
  }
}

// item owning block blk: the last item whose first_block <= blk
template <typename Item>
__device__ __forceinline__ int find_item(const Item *__restrict__ items, int n, int blk) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&items[mid].first_block) <= blk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// block-sparse product, LPR lanes per block row: lane (slot b, row r) of a
// row's lane group streams row r of every NB-th block of the row; the slots
// are then summed by shuffles inside the group.
//   SET    y = A x            RESID  y = b - A x
//   ADD    y += A x           SMOOTH y = x + M (b - A x)  (block-l1 Jacobi)
// ---------------------------------------------------------------------------
template <int BR, int BC, int NR, int LPR, typename V, typename T, int MODE, typename TO>
__global__ void __launch_bounds__(256) gspmm_kernel(const SpmmItem *__restrict__ items, int n_items,
                                                    const McgState *__restrict__ st) {
  using A = typename GAcc<T>::type;
  constexpr int RPW = 32 / LPR;  // rows per warp
  constexpr int NB = LPR / BR;   // block slots per row
  const int ii = find_item(items, n_items, blockIdx.x);
  const SpmmItem &I = items[ii];
  if (!st[I.sys].active) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane / LPR, sl = lane - sub * LPR;
  const int bl = sl / BR, r = sl - bl * BR;
  const int row = ((blockIdx.x - I.first_block) * (blockDim.x >> 5) + warp) * RPW + sub;
  const bool valid = row < I.n_rows;
  const T *__restrict__ x = (const T *)I.x;
  A acc[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = 0;
  if (valid && bl < NB) {
    const int s = __ldg(I.rowptr + row), e = __ldg(I.rowptr + row + 1);
    const V *__restrict__ vals = (const V *)I.vals;
    for (int p = s + bl; p < e; p += NB) {
      const int c = __ldg(I.colidx + p);
      const V *v = vals + ((size_t)p * BR + r) * BC;
      const T *xp = x + (size_t)c * BC * NR;
#pragma unroll
      for (int q = 0; q < BC; ++q) {
        const A a = (A)glds(v + q);
        A xv[NR];
        gld_nr<NR>(xp + q * NR, xv);
#pragma unroll
        for (int j = 0; j < NR; ++j) acc[j] += a * xv[j];
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
  // lanes sl < BR of the group hold the row's BR results
  const size_t o = (size_t)row * BR;
  const bool out = valid && sl < BR;
  TO *__restrict__ y = (TO *)I.y;
  const T *__restrict__ b = (const T *)I.b;
  if (MODE == SPMV_SMOOTH) {
    const T *__restrict__ minv = (const T *)I.minv;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const A res = out ? (A)b[(o + sl) * NR + j] - acc[j] : (A)0;
      A upd = 0;
#pragma unroll
      for (int q = 0; q < BR; ++q) {
        const A rq = __shfl_sync(0xffffffffu, res, sub * LPR + q);
        if (out) upd += (A)minv[(o + sl) * BR + q] * rq;
      }
      if (out) y[(o + sl) * NR + j] = (TO)((A)x[(o + sl) * NR + j] + upd);
    }
  } else if (out) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const size_t i = (o + sl) * NR + j;
      if (MODE == SPMV_SET) y[i] = (TO)acc[j];
      if (MODE == SPMV_RESID) y[i] = (TO)((A)b[i] - acc[j]);
      if (MODE == SPMV_ADD) y[i] = (TO)((A)y[i] + acc[j]);
    }
  }
}

// SELL-32 form: one thread per block row; slot j of a slice holds one block
// per lane, element e of the 32 blocks contiguous (coalesced value loads);
// a sorted copy (rectangular operators) names each lane's row in sell_perm
template <int BR, int BC, int NR, typename V, typename T, int MODE, typename TO>
__global__ void __launch_bounds__(128) gsell_kernel(const SpmmItem *__restrict__ items, int n_items,
                                                    const McgState *__restrict__ st) {
  using A = typename GAcc<T>::type;
  constexpr int E = BR * BC;
  const int ii = find_item(items, n_items, blockIdx.x);
  const SpmmItem &I = items[ii];
  if (!st[I.sys].active) return;
  const int slice = (blockIdx.x - I.first_block) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (slice >= I.n_slices) return;  // whole warp
  const int t = threadIdx.x & 31;
  const int row = I.sell_perm ? __ldg(I.sell_perm + slice * 32 + t) : slice * 32 + t;
  const int j0 = __ldg(I.sell_ptr + slice), j1 = __ldg(I.sell_ptr + slice + 1);
  const T *__restrict__ x = (const T *)I.x;
  const V *__restrict__ sv = (const V *)I.svals;
  A acc[BR][NR];
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[r][j] = 0;
  for (int j = j0; j < j1; ++j) {
    const int c = __ldg(I.sell_col + (size_t)j * 32 + t);
    const V *v = sv + (size_t)j * E * 32 + t;
    const T *xp = x + (size_t)c * BC * NR;
#pragma unroll
    for (int q = 0; q < BC; ++q) {
      A xv[NR];
      gld_nr<NR>(xp + q * NR, xv);
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        const A a = (A)glds(v + (r * BC + q) * 32);
#pragma unroll
        for (int jj = 0; jj < NR; ++jj) acc[r][jj] += a * xv[jj];
      }
    }
  }
  if (row >= I.n_rows) return;
  const size_t o = (size_t)row * BR;
  TO *__restrict__ y = (TO *)I.y;
  const T *__restrict__ b = (const T *)I.b;
  if (MODE == SPMV_SMOOTH) {
    const T *__restrict__ minv = (const T *)I.minv;
#pragma unroll
    for (int jj = 0; jj < NR; ++jj) {
      A res[BR];
#pragma unroll
      for (int r = 0; r < BR; ++r) res[r] = (A)b[(o + r) * NR + jj] - acc[r][jj];
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        A u = 0;
#pragma unroll
        for (int q = 0; q < BR; ++q) u += (A)minv[(o + r) * BR + q] * res[q];
        y[(o + r) * NR + jj] = (TO)((A)x[(o + r) * NR + jj] + u);
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int jj = 0; jj < NR; ++jj) {
        const size_t i = (o + r) * NR + jj;
        if (MODE == SPMV_SET) y[i] = (TO)acc[r][jj];
        if (MODE == SPMV_RESID) y[i] = (TO)((A)b[i] - acc[r][jj]);
        if (MODE == SPMV_ADD) y[i] = (TO)((A)y[i] + acc[r][jj]);
      }
  }
}

// The CG product q = A_0 p in double-float arithmetic on the SELL-32 copy
// (thread per block row, rows in order): the values as hi/lo FP32 pairs
// scaled by 2^-df_exp, p as pairs (written by the p update), every product
// exact by two-product, summed by two-sum, the low parts of each block on
// their own and two-summed into the row's low word (as the single-system
// kernel); q in FP64.
template <int BR, int NR>
__global__ void __launch_bounds__(128) gsell_df_kernel(const SpmmItem *__restrict__ items, int n_items,
                                                       const McgState *__restrict__ st) {
  constexpr int E = BR * BR;
  const int ii = find_item(items, n_items, blockIdx.x);
  const SpmmItem &I = items[ii];
  if (!st[I.sys].active) return;
  const int slice = (blockIdx.x - I.first_block) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (slice >= I.n_slices) return;  // whole warp
  const int t = threadIdx.x & 31;
  const int row = slice * 32 + t;
  const int j0 = __ldg(I.sell_ptr + slice), j1 = __ldg(I.sell_ptr + slice + 1);
  const float2 *__restrict__ x = (const float2 *)I.x;
  const float2 *__restrict__ sv = (const float2 *)I.svals;
  float hi[BR][NR], lo[BR][NR], lo2[BR][NR];
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int j = 0; j < NR; ++j) hi[r][j] = lo[r][j] = lo2[r][j] = 0.f;
  for (int j = j0; j < j1; ++j) {
    const int c = __ldg(I.sell_col + (size_t)j * 32 + t);
    const float2 *v = sv + (size_t)j * E * 32 + t;
    const float2 *xp = x + (size_t)c * BR * NR;
    float lt[BR][NR];
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int jj = 0; jj < NR; ++jj) lt[r][jj] = 0.f;
#pragma unroll
    for (int q = 0; q < BR; ++q) {
      float2 xv[NR];
#pragma unroll
      for (int jj = 0; jj < NR; ++jj) xv[jj] = __ldg(xp + q * NR + jj);
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        const float2 a = __ldcs(v + (r * BR + q) * 32);
#pragma unroll
        for (int jj = 0; jj < NR; ++jj) df_mac(hi[r][jj], lt[r][jj], a, xv[jj]);
      }
    }
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int jj = 0; jj < NR; ++jj) two_sum_into(lo[r][jj], lo2[r][jj], lt[r][jj]);
  }
  if (row >= I.n_rows) return;
  double *__restrict__ y = (double *)I.y;
  const size_t o = (size_t)row * BR;
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int jj = 0; jj < NR; ++jj)
      y[(o + r) * NR + jj] = float_to_double_scaled(hi[r][jj], I.df_exp) +
                             (float_to_double_scaled(lo[r][jj], I.df_exp) +
                              float_to_double_scaled(lo2[r][jj], I.df_exp));
}

// Block-lane form for long rows of large blocks: G lanes per block row
// (32 / G rows per warp); lane j of a row's group takes the blocks j, j + G,
// ... whole (BR x BC values) for all NR load cases, and an xor butterfly
// inside the group leaves every sum on every lane of the group.
template <int BR, int BC, int NR, int G, typename V, typename T, int MODE, typename TO>
__global__ void __launch_bounds__(256) gblock_kernel(const SpmmItem *__restrict__ items, int n_items,
                                                     const McgState *__restrict__ st) {
  using A = typename GAcc<T>::type;
  constexpr int E = BR * BC;
  constexpr int RPW = 32 / G;
  const int ii = find_item(items, n_items, blockIdx.x);
  const SpmmItem &I = items[ii];
  if (!st[I.sys].active) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane - grp * G;
  const int row = ((blockIdx.x - I.first_block) * (blockDim.x >> 5) + warp) * RPW + grp;
  const bool valid = row < I.n_rows;
  const T *__restrict__ x = (const T *)I.x;
  A acc[BR][NR];
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[r][j] = 0;
  if (valid) {
    const int s = __ldg(I.rowptr + row), e = __ldg(I.rowptr + row + 1);
    const V *__restrict__ vals = (const V *)I.vals;
    for (int p = s + gl; p < e; p += G) {
      const int c = __ldg(I.colidx + p);
      const V *v = vals + (size_t)p * E;
      const T *xp = x + (size_t)c * BC * NR;
#pragma unroll
      for (int q = 0; q < BC; ++q) {
        A xv[NR];
        gld_nr<NR>(xp + q * NR, xv);
#pragma unroll
        for (int r = 0; r < BR; ++r) {
          const A a = (A)glds(v + r * BC + q);
#pragma unroll
          for (int j = 0; j < NR; ++j) acc[r][j] += a * xv[j];
        }
      }
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int j = 0; j < NR; ++j) acc[r][j] += __shfl_xor_sync(0xffffffffu, acc[r][j], o);
  if (!valid || gl >= BR) return;
  const size_t o = (size_t)row * BR;
  TO *__restrict__ y = (TO *)I.y;
  const T *__restrict__ b = (const T *)I.b;
  if (MODE == SPMV_SMOOTH) {
    const T *__restrict__ minv = (const T *)I.minv;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      A upd = 0;
#pragma unroll
      for (int q = 0; q < BR; ++q) upd += (A)minv[(o + gl) * BR + q] * ((A)b[(o + q) * NR + j] - acc[q][j]);
      y[(o + gl) * NR + j] = (TO)((A)x[(o + gl) * NR + j] + upd);
    }
  } else {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      A mine = 0;  // acc[gl][j] without dynamic register indexing
#pragma unroll
      for (int r = 0; r < BR; ++r)
        if (gl == r) mine = acc[r][j];
      const size_t i = (o + gl) * NR + j;
      if (MODE == SPMV_SET) y[i] = (TO)mine;
      if (MODE == SPMV_RESID) y[i] = (TO)((A)b[i] - mine);
      if (MODE == SPMV_ADD) y[i] = (TO)((A)y[i] + mine);
    }
  }
}

template <int BR, int BC, int NR, int LPR, typename V, typename T, int MODE, typename TO>
static cudaError_t gspmm_go(int wpb, const SpmmItem *items, int n_items, int grid,
                            const McgState *st, cudaStream_t s) {
  if constexpr (LPR == 0)
    gsell_kernel<BR, BC, NR, V, T, MODE, TO><<<grid, wpb * 32, 0, s>>>(items, n_items, st);
  else if constexpr (LPR < 0)
    gblock_kernel<BR, BC, NR, -LPR, V, T, MODE, TO><<<grid, wpb * 32, 0, s>>>(items, n_items, st);
  else
    gspmm_kernel<BR, BC, NR, LPR, V, T, MODE, TO><<<grid, wpb * 32, 0, s>>>(items, n_items, st);
  return cudaGetLastError();
}

template <int BR, int BC, int NR, int LPR>
static cudaError_t gspmm_lpr(const SpmmKey &k, int wpb, const SpmmItem *items, int n_items, int grid,
                             const McgState *st, cudaStream_t s) {
#define G_ARGS wpb, items, n_items, grid, st, s
  // modes by role: square operators RESID / SMOOTH (and SET for the CG
  // product), prolongations ADD, restrictions SET
  if (k.vt == 0) {
    switch (k.mode) {
      case SPMV_SET: return gspmm_go<BR, BC, NR, LPR, double, double, SPMV_SET, double>(G_ARGS);
      case SPMV_RESID:
        if (BR == BC) return gspmm_go<BR, BC, NR, LPR, double, double, SPMV_RESID, double>(G_ARGS);
        break;
      case SPMV_ADD: return gspmm_go<BR, BC, NR, LPR, double, double, SPMV_ADD, double>(G_ARGS);
      case SPMV_SMOOTH:
        if (BR == BC) return gspmm_go<BR, BC, NR, LPR, double, double, SPMV_SMOOTH, double>(G_ARGS);
        break;
    }
    return cudaErrorInvalidValue;
  }
  if (k.vt == 1) {
    switch (k.mode) {
      case SPMV_SET: return gspmm_go<BR, BC, NR, LPR, float, float, SPMV_SET, float>(G_ARGS);
      case SPMV_RESID:
        if (BR == BC) return gspmm_go<BR, BC, NR, LPR, float, float, SPMV_RESID, float>(G_ARGS);
        break;
      case SPMV_ADD: return gspmm_go<BR, BC, NR, LPR, float, float, SPMV_ADD, float>(G_ARGS);
      case SPMV_SMOOTH:
        if (BR != BC) break;
        if (k.to64) return gspmm_go<BR, BC, NR, LPR, float, float, SPMV_SMOOTH, double>(G_ARGS);
        return gspmm_go<BR, BC, NR, LPR, float, float, SPMV_SMOOTH, float>(G_ARGS);
    }
    return cudaErrorInvalidValue;
  }
  if (k.vt == 2) {
    switch (k.mode) {
      case SPMV_SET: return gspmm_go<BR, BC, NR, LPR, __nv_bfloat16, float, SPMV_SET, float>(G_ARGS);
      case SPMV_RESID:
        if (BR == BC)
          return gspmm_go<BR, BC, NR, LPR, __nv_bfloat16, float, SPMV_RESID, float>(G_ARGS);
        break;
      case SPMV_ADD: return gspmm_go<BR, BC, NR, LPR, __nv_bfloat16, float, SPMV_ADD, float>(G_ARGS);
      case SPMV_SMOOTH:
        if (BR != BC) break;
        if (k.to64)
          return gspmm_go<BR, BC, NR, LPR, __nv_bfloat16, float, SPMV_SMOOTH, double>(G_ARGS);
        return gspmm_go<BR, BC, NR, LPR, __nv_bfloat16, float, SPMV_SMOOTH, float>(G_ARGS);
    }
  }
#undef G_ARGS
  return cudaErrorInvalidValue;
}

bool gblock_supported(int br, int bc) { return br == 6 && (bc == 6 || bc == 3); }

bool gsell_supported(int br, int bc) {
  return (br == 3 && bc == 3) || (br == 3 && bc == 6) || (br == 2 && bc == 2) || (br == 2 && bc == 3);
}

template <int BR, int BC, int NR>
static cudaError_t gspmm_shape(const SpmmKey &k, int lpr, int wpb, const SpmmItem *items,
                               int n_items, int grid, const McgState *st, cudaStream_t s) {
  constexpr bool sell_ok = (BR == 3 && BC == 3) || (BR == 3 && BC == 6) || (BR == 2 && BC == 2) ||
                           (BR == 2 && BC == 3);
  if (lpr == 0) {
    if constexpr (sell_ok) return gspmm_lpr<BR, BC, NR, 0>(k, wpb, items, n_items, grid, st, s);
    return cudaErrorInvalidValue;
  }
  constexpr bool block_ok = BR == 6 && (BC == 6 || BC == 3);
  if (lpr < 0) {
    if constexpr (block_ok) {
      if (lpr == -8) return gspmm_lpr<BR, BC, NR, -8>(k, wpb, items, n_items, grid, st, s);
      if (lpr == -16) return gspmm_lpr<BR, BC, NR, -16>(k, wpb, items, n_items, grid, st, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (lpr) {
    case 32: return gspmm_lpr<BR, BC, NR, 32>(k, wpb, items, n_items, grid, st, s);
    case 16: return gspmm_lpr<BR, BC, NR, 16>(k, wpb, items, n_items, grid, st, s);
    case 8: return gspmm_lpr<BR, BC, NR, 8>(k, wpb, items, n_items, grid, st, s);
  }
  return cudaErrorInvalidValue;
}

template <int NR>
static cudaError_t gspmm_nr(const SpmmKey &k, int lpr, int wpb, const SpmmItem *items, int n_items,
                            int grid, const McgState *st, cudaStream_t s) {
#define G_SHAPE(R_, C_) \
  if (k.br == R_ && k.bc == C_) return gspmm_shape<R_, C_, NR>(k, lpr, wpb, items, n_items, grid, st, s);
  G_SHAPE(2, 2)
  G_SHAPE(3, 3)
  G_SHAPE(6, 6)
  G_SHAPE(2, 3)
  G_SHAPE(3, 2)
  G_SHAPE(3, 6)
  G_SHAPE(6, 3)
#undef G_SHAPE
  return cudaErrorInvalidValue;
}

cudaError_t launch_gspmm(const SpmmKey &k, int nr, int lpr, int wpb, const SpmmItem *items,
                         int n_items, int grid, const McgState *st, cudaStream_t s) {
  if (grid <= 0 || n_items <= 0) return cudaSuccess;
  if (wpb < 1 || wpb > 8 || (lpr > 0 && lpr < k.br)) return cudaErrorInvalidValue;
  if (lpr == 0 && wpb > 4) return cudaErrorInvalidValue;
  if (k.vt == 3) {
    // the double-float CG product: SELL-32 copy, square 2x2 / 3x3 blocks
    if (lpr != 0 || k.mode != SPMV_SET || k.br != k.bc) return cudaErrorInvalidValue;
#define G_DF(R_, N_)                                                                    \
  if (k.br == R_ && nr == N_) {                                                         \
    gsell_df_kernel<R_, N_><<<grid, wpb * 32, 0, s>>>(items, n_items, st);              \
    return cudaGetLastError();                                                          \
  }
    G_DF(2, 1)
    G_DF(2, 6)
    G_DF(3, 1)
    G_DF(3, 6)
#undef G_DF
    return cudaErrorInvalidValue;
  }
  if (nr == 6) return gspmm_nr<6>(k, lpr, wpb, items, n_items, grid, st, s);
  if (nr == 1) return gspmm_nr<1>(k, lpr, wpb, items, n_items, grid, st, s);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// block-diagonal apply y = M^+ b per vertex (thread per vertex)
// ---------------------------------------------------------------------------
template <int K, int NR, typename TM, typename TI, typename TO>
__global__ void __launch_bounds__(128) gdiag_kernel(const DiagItem *__restrict__ items, int n_items,
                                                    const McgState *__restrict__ st) {
  using A = typename GAcc<TO>::type;
  const int ii = find_item(items, n_items, blockIdx.x);
  const DiagItem &I = items[ii];
  if (!st[I.sys].active) return;
  const size_t v = (size_t)(blockIdx.x - I.first_block) * blockDim.x + threadIdx.x;
  if (v >= (size_t)I.n) return;
  const TM *__restrict__ minv = (const TM *)I.minv;
  const TI *__restrict__ bin = (const TI *)I.bin;
  TO *__restrict__ bcopy = (TO *)I.bcopy;
  TO *__restrict__ y = (TO *)I.y;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    A rb[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const TO bv = (TO)bin[(v * K + q) * NR + j];
      rb[q] = (A)bv;
      if (bcopy) bcopy[(v * K + q) * NR + j] = bv;
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
      A acc = 0;
#pragma unroll
      for (int q = 0; q < K; ++q) acc += (A)minv[(v * K + i) * K + q] * rb[q];
      y[(v * K + i) * NR + j] = (TO)acc;
    }
  }
}

template <int K, int NR>
static cudaError_t gdiag_k(int kind, const DiagItem *items, int n_items, int grid, const McgState *st,
                           cudaStream_t s) {
  if (kind == 0)
    gdiag_kernel<K, NR, double, double, double><<<grid, 128, 0, s>>>(items, n_items, st);
  else if (kind == 1)
    gdiag_kernel<K, NR, float, double, float><<<grid, 128, 0, s>>>(items, n_items, st);
  else
    gdiag_kernel<K, NR, float, float, float><<<grid, 128, 0, s>>>(items, n_items, st);
  return cudaGetLastError();
}

cudaError_t launch_gdiag(int k, int kind, int nr, const DiagItem *items, int n_items, int grid,
                         const McgState *st, cudaStream_t s) {
  if (grid <= 0 || n_items <= 0) return cudaSuccess;
#define G_DIAG(K_, NR_) \
  if (k == K_ && nr == NR_) return gdiag_k<K_, NR_>(kind, items, n_items, grid, st, s);
  G_DIAG(2, 1) G_DIAG(3, 1) G_DIAG(6, 1) G_DIAG(2, 6) G_DIAG(3, 6) G_DIAG(6, 6)
#undef G_DIAG
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// coarsest level: Y = C^{-1} B (dense FP64 inverse, warp per row, 8 rows per
// block)
// ---------------------------------------------------------------------------
template <int NR, typename T>
__global__ void __launch_bounds__(256) gcoarse_kernel(const CoarseItem *__restrict__ items, int n_items,
                                                      const McgState *__restrict__ st) {
  const int ii = find_item(items, n_items, blockIdx.x);
  const CoarseItem &I = items[ii];
  if (!st[I.sys].active) return;
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x - I.first_block) * 8 + (threadIdx.x >> 5);
  if (row >= I.n) return;  // whole warp
  const double *a = I.cinv + (size_t)row * I.n;
  const T *__restrict__ b = (const T *)I.b;
  double acc[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = 0.0;
  for (int q = lane; q < I.n; q += 32) {
    const double av = __ldg(a + q);
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[j] += av * (double)b[(size_t)q * NR + j];
  }
  T *__restrict__ y = (T *)I.y;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_down_sync(0xffffffffu, acc[j], o);
    if (lane == 0) y[(size_t)row * NR + j] = (T)acc[j];
  }
}

cudaError_t launch_gcoarse(bool fp64, int nr, const CoarseItem *items, int n_items, int grid,
                           const McgState *st, cudaStream_t s) {
  if (grid <= 0 || n_items <= 0) return cudaSuccess;
  if (nr == 6) {
    if (fp64) gcoarse_kernel<6, double><<<grid, 256, 0, s>>>(items, n_items, st);
    else gcoarse_kernel<6, float><<<grid, 256, 0, s>>>(items, n_items, st);
  } else if (nr == 1) {
    if (fp64) gcoarse_kernel<1, double><<<grid, 256, 0, s>>>(items, n_items, st);
    else gcoarse_kernel<1, float><<<grid, 256, 0, s>>>(items, n_items, st);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CG: per-system inner products (partials per block, the last block of a
// system sums them in a fixed order and updates the system's scalars)
//   INIT r.r, f.f      RHO r.z, r.z_old -> beta, rho
//   PQ   p.q -> alpha  RR  r.r
// ---------------------------------------------------------------------------
template <int NR, int PH>
__global__ void __launch_bounds__(256) gdots_kernel(const SysItem *__restrict__ items, int n_items,
                                                    const GSys *__restrict__ gs,
                                                    McgState *__restrict__ st) {
  __shared__ double sh[2 * NR][8];
  __shared__ double tot[2 * NR];
  __shared__ bool last;
  const int ii = find_item(items, n_items, blockIdx.x);
  const int sys = items[ii].sys;
  McgState *S = st + sys;
  if (PH != PH_INIT && !S->active) return;
  const GSys &G = gs[sys];
  const double *a1, *b1, *a2 = nullptr, *b2 = nullptr;
  if (PH == PH_INIT) { a1 = G.r; b1 = G.r; a2 = G.f; b2 = G.f; }
  else if (PH == PH_RHO) { a1 = G.r; b1 = G.z; a2 = G.r; b2 = G.zold; }
  else if (PH == PH_PQ) { a1 = G.p; b1 = G.q; }
  else { a1 = G.r; b1 = G.r; }
  const bool two = a2 != nullptr && (PH == PH_INIT || S->flexible);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int lb = blockIdx.x - items[ii].first_block, nb = G.red_blocks;
  double v1[NR], v2[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) v1[j] = v2[j] = 0.0;
  const size_t n = G.n, stride = (size_t)nb * blockDim.x;
  for (size_t i = (size_t)lb * blockDim.x + threadIdx.x; i < n; i += stride) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      v1[j] += a1[i * NR + j] * b1[i * NR + j];
      if (two) v2[j] += a2[i * NR + j] * b2[i * NR + j];
    }
  }
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    for (int o = 16; o > 0; o >>= 1) {
      v1[j] += __shfl_down_sync(0xffffffffu, v1[j], o);
      v2[j] += __shfl_down_sync(0xffffffffu, v2[j], o);
    }
    if (lane == 0) {
      sh[j][w] = v1[j];
      sh[NR + j][w] = v2[j];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 0; j < 2 * NR; ++j) {
      double s = 0.0;
      for (int k = 0; k < 8; ++k) s += sh[j][k];
      G.partials[(size_t)j * nb + lb] = s;
    }
    __threadfence();
    last = atomicAdd(G.counter, 1u) == (unsigned)nb - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int j = w; j < 2 * NR; j += 8) {
    double a = 0.0;
    for (int b = lane; b < nb; b += 32) a += ((volatile double *)G.partials)[(size_t)j * nb + b];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) tot[j] = a;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  *G.counter = 0u;
  if (PH == PH_INIT) {
    for (int j = 0; j < NR; ++j) {
      S->rr[j] = tot[j];
      S->ff[j] = tot[NR + j];
      S->tol2[j] = S->rtol * S->rtol * tot[NR + j];
      S->it[j] = 0;
      S->status[j] = 0;
      S->rho_old[j] = 0.0;
      S->done[j] = !(tot[j] > S->tol2[j]) || S->maxit <= 0 || !isfinite(tot[j]);
    }
  } else if (PH == PH_RHO) {
    for (int j = 0; j < NR; ++j) {
      if (S->done[j]) continue;
      const double rho = tot[j];
      S->beta[j] = S->it[j] > 0 ? (S->flexible ? (rho - tot[NR + j]) : rho) / S->rho_old[j] : 0.0;
      S->rho[j] = rho;
      S->rho_old[j] = rho;
    }
  } else if (PH == PH_PQ) {
    for (int j = 0; j < NR; ++j) {
      S->pq[j] = tot[j];
      if (S->done[j]) {
        S->alpha[j] = 0.0;
        continue;
      }
      if (!(tot[j] > 0.0) || !isfinite(tot[j])) {
        S->status[j] = AMG_ERR_NOT_SPD;
        S->done[j] = 1;
        S->alpha[j] = 0.0;
      } else {
        S->alpha[j] = S->rho[j] / tot[j];
      }
    }
  } else {
    for (int j = 0; j < NR; ++j)
      if (!S->done[j]) S->rr[j] = tot[j];
  }
}

template <int PH>
static cudaError_t gdots_ph(int nr, const SysItem *items, int n_items, int grid, const GSys *gs,
                            McgState *st, cudaStream_t s) {
  if (nr == 6) gdots_kernel<6, PH><<<grid, 256, 0, s>>>(items, n_items, gs, st);
  else if (nr == 1) gdots_kernel<1, PH><<<grid, 256, 0, s>>>(items, n_items, gs, st);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_gdots(int phase, int nr, const SysItem *items, int n_items, int grid,
                         const GSys *gs, McgState *st, cudaStream_t s) {
  if (grid <= 0 || n_items <= 0) return cudaSuccess;
  switch (phase) {
    case PH_INIT: return gdots_ph<PH_INIT>(nr, items, n_items, grid, gs, st, s);
    case PH_RHO: return gdots_ph<PH_RHO>(nr, items, n_items, grid, gs, st, s);
    case PH_PQ: return gdots_ph<PH_PQ>(nr, items, n_items, grid, gs, st, s);
    case PH_RR: return gdots_ph<PH_RR>(nr, items, n_items, grid, gs, st, s);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// CG vector updates and (un)packing, thread per dof
// ---------------------------------------------------------------------------
// p = z + beta p (first iteration p = z); z_old = z for flexible CG
template <int NR>
__global__ void __launch_bounds__(256) gupdate_p_kernel(const SysItem *__restrict__ items, int n_items,
                                                        const GSys *__restrict__ gs,
                                                        const McgState *__restrict__ st) {
  const int ii = find_item(items, n_items, blockIdx.x);
  const int sys = items[ii].sys;
  const McgState *S = st + sys;
  if (!S->active) return;
  const GSys &G = gs[sys];
  const size_t i = (size_t)(blockIdx.x - items[ii].first_block) * blockDim.x + threadIdx.x;
  if (i >= G.n) return;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    if (S->done[j]) continue;
    const double zi = G.z[i * NR + j];
    const double pi = S->it[j] == 0 ? zi : zi + S->beta[j] * G.p[i * NR + j];
    G.p[i * NR + j] = pi;
    if (G.pdf) G.pdf[i * NR + j] = split_double_float(pi);  // for the double-float CG product
    if (S->flexible) G.zold[i * NR + j] = zi;
  }
}

// x += alpha p ; r -= alpha q
template <int NR>
__global__ void __launch_bounds__(256) gupdate_xr_kernel(const SysItem *__restrict__ items, int n_items,
                                                         const GSys *__restrict__ gs,
                                                         const McgState *__restrict__ st) {
  const int ii = find_item(items, n_items, blockIdx.x);
  const int sys = items[ii].sys;
  const McgState *S = st + sys;
  if (!S->active) return;
  const GSys &G = gs[sys];
  const size_t i = (size_t)(blockIdx.x - items[ii].first_block) * blockDim.x + threadIdx.x;
  if (i >= G.n) return;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    if (S->done[j]) continue;
    const double a = S->alpha[j];
    G.x[i * NR + j] += a * G.p[i * NR + j];
    G.r[i * NR + j] -= a * G.q[i * NR + j];
  }
}

// stacked (load cases one after another) -> interleaved f, x
template <int NR>
__global__ void __launch_bounds__(256) gpack_kernel(const SysItem *__restrict__ items, int n_items,
                                                    const GSys *__restrict__ gs,
                                                    const double *__restrict__ fin,
                                                    const double *__restrict__ uin) {
  const int ii = find_item(items, n_items, blockIdx.x);
  const GSys &G = gs[items[ii].sys];
  const size_t i = (size_t)(blockIdx.x - items[ii].first_block) * blockDim.x + threadIdx.x;
  if (i >= G.n) return;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    G.f[i * NR + j] = fin[G.offset + (size_t)j * G.n + i];
    G.x[i * NR + j] = uin[G.offset + (size_t)j * G.n + i];
  }
}

template <int NR>
__global__ void __launch_bounds__(256) gunpack_kernel(const SysItem *__restrict__ items, int n_items,
                                                      const GSys *__restrict__ gs,
                                                      double *__restrict__ uout) {
  const int ii = find_item(items, n_items, blockIdx.x);
  const GSys &G = gs[items[ii].sys];
  const size_t i = (size_t)(blockIdx.x - items[ii].first_block) * blockDim.x + threadIdx.x;
  if (i >= G.n) return;
#pragma unroll
  for (int j = 0; j < NR; ++j) uout[G.offset + (size_t)j * G.n + i] = G.x[i * NR + j];
}

#define G_NR_LAUNCH(KERNEL, ...)                                              \
  if (grid <= 0 || n_items <= 0) return cudaSuccess;                          \
  if (nr == 6) KERNEL<6><<<grid, 256, 0, s>>>(items, n_items, __VA_ARGS__);   \
  else if (nr == 1) KERNEL<1><<<grid, 256, 0, s>>>(items, n_items, __VA_ARGS__); \
  else return cudaErrorInvalidValue;                                          \
  return cudaGetLastError();

cudaError_t launch_gupdate_p(int nr, const SysItem *items, int n_items, int grid, const GSys *gs,
                             const McgState *st, cudaStream_t s) {
  G_NR_LAUNCH(gupdate_p_kernel, gs, st)
}
cudaError_t launch_gupdate_xr(int nr, const SysItem *items, int n_items, int grid, const GSys *gs,
                              const McgState *st, cudaStream_t s) {
  G_NR_LAUNCH(gupdate_xr_kernel, gs, st)
}
cudaError_t launch_gpack(int nr, const SysItem *items, int n_items, int grid, const GSys *gs,
                         const double *fin, const double *uin, cudaStream_t s) {
  G_NR_LAUNCH(gpack_kernel, gs, fin, uin)
}
cudaError_t launch_gunpack(int nr, const SysItem *items, int n_items, int grid, const GSys *gs,
                           double *uout, cudaStream_t s) {
  G_NR_LAUNCH(gunpack_kernel, gs, uout)
}
#undef G_NR_LAUNCH

// ---------------------------------------------------------------------------
// loop decision (one block): count the iteration of every active load case,
// freeze the converged ones, mark systems with no active load case inactive,
// bound the loop and set the condition of the while node.  init: only the
// activity after the initial residuals.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) gguard_kernel(int ns, McgState *__restrict__ st,
                                                      BatchLoop *__restrict__ loop,
                                                      cudaGraphConditionalHandle h, int init) {
  int any = 0;
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    McgState &S = st[s];
    int act = 0;
    if (init || S.active) {
      for (int j = 0; j < S.nr; ++j) {
        if (S.done[j]) continue;
        if (!init) {
          S.it[j] += 1;
          if (!isfinite(S.rr[j])) {
            S.status[j] = AMG_ERR_NOT_SPD;
            S.done[j] = 1;
          } else if (!(S.rr[j] > S.tol2[j]) || S.it[j] >= S.maxit) {
            S.done[j] = 1;
          }
        }
        act |= !S.done[j];
      }
    }
    S.active = act;
    any |= act;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    if (init) loop->guard = 0;
    else loop->guard += 1;
    cudaGraphSetConditional(h, (any && loop->guard < loop->maxit) ? 1u : 0u);
  }
}

cudaError_t launch_gguard(int ns, McgState *st, BatchLoop *loop, cudaGraphConditionalHandle h,
                          bool init, cudaStream_t s) {
  gguard_kernel<<<1, 1024, 0, s>>>(ns, st, loop, h, init ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace amg
