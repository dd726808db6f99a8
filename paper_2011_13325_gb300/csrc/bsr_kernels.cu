// BSR operator kernels of the V-cycle (Sec. 3 Algorithm tg, Sec. 7 smoother):
// SpMV, residual, prolongation-add and the fused block-l1 Jacobi sweep, plus
// the block-diagonal apply, the coarsest-level dense GEMV and conversions.
//
// Layout: one warp per block row.  Lane (b, r) = (lane / BR, lane % BR)
// streams row r of the b-th block of each group of NB = 32 / BR consecutive
// blocks: a warp step reads NB*BR*BC contiguous values (fully coalesced), the
// x gather reads BC contiguous entries per lane.  Partial sums of lanes with
// the same r are combined with warp shuffles; lanes 0..BR-1 finish the row.
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "amg_internal.h"
#include "bsr_loads.cuh"

namespace amg {

// Staging of a warp's 32 blocks in shared memory (block-lane kernel): the
// blocks of one pass are contiguous in memory, so the warp copies them with
// coalesced word loads and each lane then reads its own block from shared
// memory.  Read straight from global memory, a block that is not 16-byte
// aligned takes several 8-byte loads 32 blocks apart, each touching 32
// sectors for 256 useful bytes; those shapes are staged when their 32 blocks
// fit in 4.5 KB (8 warps per block: at most 36 KB of shared memory).  Blocks
// that are 16-byte aligned (6x6 FP32, read as 16-byte vectors) ran slower
// staged, and so did the warp-row kernel (its lanes already read contiguous
// 24-byte rows; the copy serialises each trip's loads behind the previous
// trip's arithmetic).
template <int E, typename V>
struct LbStage {
  static constexpr int BYTES = E * (int)sizeof(V);
  static constexpr bool ON = (BYTES % 16 != 0) && (32 * BYTES <= 4608);
  using W = typename std::conditional<
      BYTES % 8 == 0, uint2,
      typename std::conditional<BYTES % 4 == 0, unsigned, unsigned short>::type>::type;
};

template <int E>
__device__ __forceinline__ void stage_read(const float *p, float *out) {
  if constexpr (E % 2 == 0) {
#pragma unroll
    for (int i = 0; i < E; i += 2) {
      const float2 v = *reinterpret_cast<const float2 *>(p + i);
      out[i] = v.x;
      out[i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) out[i] = p[i];
  }
}
template <int E>
__device__ __forceinline__ void stage_read(const double *p, double *out) {
#pragma unroll
  for (int i = 0; i < E; ++i) out[i] = p[i];
}
template <int E>
__device__ __forceinline__ void stage_read(const __nv_bfloat16 *p, float *out) {
#pragma unroll
  for (int i = 0; i < E; ++i) out[i] = __bfloat162float(p[i]);
}

template <int BR, int BC, typename V, typename T, int MODE, typename TO = T>
__global__ void __launch_bounds__(256) bsr_warp_kernel(int n_rows, const int *__restrict__ rowptr,
                                                       const int *__restrict__ colidx,
                                                       const V *__restrict__ vals,
                                                       const T *__restrict__ x,
                                                       const T *__restrict__ b,
                                                       const T *__restrict__ minv,
                                                       TO *__restrict__ y) {
  pdl_enter();
  using A = typename AccT<T>::type;
  constexpr int NB = 32 / BR;
  const int lane = threadIdx.x & 31;
  const int bl = lane / BR;
  const int r = lane - bl * BR;
  const bool active = bl < NB;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n_rows; row += nwarps) {
    const int s = rowptr[row], e = rowptr[row + 1];
    A acc = 0;
    if (active) {
      int p = s + bl;
      // two block steps per iteration keep more loads in flight
      for (; p + NB < e; p += 2 * NB) {
        const int c0 = __ldg(colidx + p), c1 = __ldg(colidx + p + NB);
        A a0[BC], a1[BC], x0[BC], x1[BC];
        ldn_stream<BC>(vals + ((size_t)p * BR + r) * BC, a0);
        ldn_stream<BC>(vals + ((size_t)(p + NB) * BR + r) * BC, a1);
        ldn_cached<BC>(x + (size_t)c0 * BC, x0);
        ldn_cached<BC>(x + (size_t)c1 * BC, x1);
#pragma unroll
        for (int q = 0; q < BC; ++q) {
          acc += a0[q] * x0[q];
          acc += a1[q] * x1[q];
        }
      }
      if (p < e) {
        const int c0 = __ldg(colidx + p);
        A a0[BC], x0[BC];
        ldn_stream<BC>(vals + ((size_t)p * BR + r) * BC, a0);
        ldn_cached<BC>(x + (size_t)c0 * BC, x0);
#pragma unroll
        for (int q = 0; q < BC; ++q) acc += a0[q] * x0[q];
      }
    }
#pragma unroll
    for (int sft = 1; sft < NB; sft <<= 1) {
      A o = __shfl_down_sync(0xffffffffu, acc, sft * BR);
      if (bl + sft < NB) acc += o;
    }
    const size_t o = (size_t)row * BR;
    if (MODE == SPMV_SMOOTH) {
      // x_out = x_in + M^+ (b - A x_in) for this vertex (block-l1 Jacobi)
      A res = (lane < BR) ? (A)b[o + lane] - acc : (A)0;
      A upd = 0;
#pragma unroll
      for (int q = 0; q < BR; ++q) {
        A rq = __shfl_sync(0xffffffffu, res, q);
        if (lane < BR) upd += (A)minv[(o + lane) * BR + q] * rq;
      }
      if (lane < BR) y[o + lane] = (TO)((A)x[o + lane] + upd);
    } else if (lane < BR) {
      if (MODE == SPMV_SET) y[o + lane] = (TO)acc;
      if (MODE == SPMV_RESID) y[o + lane] = (TO)((A)b[o + lane] - acc);
      if (MODE == SPMV_ADD) y[o + lane] = (TO)((A)y[o + lane] + acc);
    }
  }
}

// Blocks of `threads` threads of kernel k that are resident on one SM at
// once (from its registers and shared memory; cached per kernel).
template <typename... P>
static int resident_blocks(void (*k)(P...), int threads) {
  static std::mutex mu;
  static std::unordered_map<const void *, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  const auto it = cache.find((const void *)k);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, 0) != cudaSuccess || n < 1) {
    (void)cudaGetLastError();
    n = 1;
  }
  cache[(const void *)k] = n;
  return n;
}

// Grid of a grid-stride kernel with one warp per block row: one block per 8
// rows, at most as many blocks as are resident at once (every block then
// starts at once and the rows are spread evenly; a grid above that would
// run its last blocks on a mostly idle GPU).
template <typename... P>
static int grid_for_rows(const Ctx *c, int n_rows, void (*k)(P...)) {
  long want = ((long)n_rows + 7) / 8;  // 8 warps per 256-thread block
  const long cap = (long)c->num_sms * resident_blocks(k, 256);
  if (want > cap) want = cap;
  return (int)(want < 1 ? 1 : want);
}

template <int BR, int BC, typename V, typename T>
static cudaError_t bsr_mode(const Ctx *c, const DevBSR &A, const V *vals, int mode, const void *x,
                            const void *b, const void *minv, void *y) {
  const T *xx = (const T *)x;
  const T *bb = (const T *)b;
  const T *mm = (const T *)minv;
  T *yy = (T *)y;
#define AMG_WARP_LAUNCH(M_)                                                                    \
  AMG_KLAUNCH(c, bsr_warp_kernel<BR, BC, V, T, M_>,                                            \
              grid_for_rows(c, A.n_rows, bsr_warp_kernel<BR, BC, V, T, M_>), 256, A.n_rows,    \
              A.rowptr, A.colidx, vals, xx, bb, mm, yy)
  switch (mode) {
    case SPMV_SET:
      AMG_WARP_LAUNCH(SPMV_SET);
      break;
    case SPMV_RESID:
      AMG_WARP_LAUNCH(SPMV_RESID);
      break;
    case SPMV_ADD:
      AMG_WARP_LAUNCH(SPMV_ADD);
      break;
    case SPMV_SMOOTH:
      if constexpr (BR == BC) {
        AMG_WARP_LAUNCH(SPMV_SMOOTH);
        break;
      } else {
        return cudaErrorInvalidValue;
      }
    default:
      return cudaErrorInvalidValue;
  }
#undef AMG_WARP_LAUNCH
  return cudaGetLastError();
}

// Row-lane variant: BR lanes per block row (lane r owns scalar row r of the
// block row and streams row r of each of its blocks), 32 / BR block rows per
// warp.  The BR lanes of a block row read its blocks as contiguous
// BR * BC-value chunks; no cross-lane reduction; 30 or 32 of 32 lanes busy.
// Used for operators with long rows and few block rows (coarse levels,
// restriction), where one thread per block row would leave the GPU idle.
template <int BR, int BC, typename V, typename T, int MODE>
__global__ void __launch_bounds__(256) bsr_rowlane_kernel(int n_rows, const int *__restrict__ rowptr,
                                                          const int *__restrict__ colidx,
                                                          const V *__restrict__ vals,
                                                          const T *__restrict__ x,
                                                          const T *__restrict__ b,
                                                          const T *__restrict__ minv,
                                                          T *__restrict__ y) {
  pdl_enter();
  using A = typename AccT<T>::type;
  constexpr int G = 32 / BR;
  const int lane = threadIdx.x & 31;
  const int g = lane / BR;
  const int r = lane - g * BR;
  const int row = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * G + g;
  const bool active = g < G && row < n_rows;
  A acc = 0;
  if (active) {
    const int e = rowptr[row + 1];
    int p = rowptr[row];
    for (; p + 1 < e; p += 2) {
      const int c0 = __ldg(colidx + p), c1 = __ldg(colidx + p + 1);
      const V *v0 = vals + ((size_t)p * BR + r) * BC;
      const V *v1 = v0 + BR * BC;
      A a0[BC], a1[BC];
#pragma unroll
      for (int q = 0; q < BC; ++q) {
        a0[q] = (A)lds(v0 + q);
        a1[q] = (A)lds(v1 + q);
      }
#pragma unroll
      for (int q = 0; q < BC; ++q) {
        acc += a0[q] * (A)ld(x + (size_t)c0 * BC + q);
        acc += a1[q] * (A)ld(x + (size_t)c1 * BC + q);
      }
    }
    if (p < e) {
      const int c0 = __ldg(colidx + p);
      const V *v0 = vals + ((size_t)p * BR + r) * BC;
#pragma unroll
      for (int q = 0; q < BC; ++q) acc += (A)lds(v0 + q) * (A)ld(x + (size_t)c0 * BC + q);
    }
  }
  const size_t o = (size_t)row * BR;
  if (MODE == SPMV_SMOOTH) {
    A res = active ? (A)b[o + r] - acc : (A)0;
    A upd = 0;
#pragma unroll
    for (int q = 0; q < BR; ++q) {
      const A rq = __shfl_sync(0xffffffffu, res, (g < G ? g : 0) * BR + q);
      if (active) upd += (A)minv[(o + r) * BR + q] * rq;
    }
    if (active) y[o + r] = (T)((A)x[o + r] + upd);
  } else if (active) {
    if (MODE == SPMV_SET) y[o + r] = (T)acc;
    if (MODE == SPMV_RESID) y[o + r] = (T)((A)b[o + r] - acc);
    if (MODE == SPMV_ADD) y[o + r] = (T)((A)y[o + r] + acc);
  }
}

template <int BR, int BC, typename V, typename T>
static cudaError_t rowlane_mode(const Ctx *c, const DevBSR &A, const V *vals, int mode,
                                const void *x, const void *b, const void *minv, void *y) {
  constexpr int G = 32 / BR;
  const long warps = ((long)A.n_rows + G - 1) / G;
  const int g = (int)((warps + 7) / 8);
  const T *xx = (const T *)x;
  const T *bb = (const T *)b;
  const T *mm = (const T *)minv;
  T *yy = (T *)y;
#define AMG_RL_LAUNCH(M_)                                                                      \
  AMG_KLAUNCH(c, bsr_rowlane_kernel<BR, BC, V, T, M_>, g, 256, A.n_rows, A.rowptr, A.colidx, \
                                                                 vals, xx, bb, mm, yy)
  switch (mode) {
    case SPMV_SET: AMG_RL_LAUNCH(SPMV_SET); break;
    case SPMV_RESID: AMG_RL_LAUNCH(SPMV_RESID); break;
    case SPMV_ADD: AMG_RL_LAUNCH(SPMV_ADD); break;
    case SPMV_SMOOTH:
      if constexpr (BR == BC) {
        AMG_RL_LAUNCH(SPMV_SMOOTH);
        break;
      } else {
        return cudaErrorInvalidValue;
      }
    default: return cudaErrorInvalidValue;
  }
#undef AMG_RL_LAUNCH
  return cudaGetLastError();
}

// Block-lane variant: one warp per block row; lane j takes the blocks j,
// j + 32, ... of the row whole (all BR x BC values, contiguous, the widest
// aligned loads) and keeps BR partial sums, which a butterfly reduction then
// leaves on every lane.  Meant for long rows of large blocks (6x6 coarse
// levels, restrictions), where one block-row element per lane spends most of
// its loads on x entries that the lanes of the same block share.
template <int E, bool W16>
__device__ __forceinline__ void ldblock(const float *p, float *out) {
  if constexpr (W16 && E % 4 == 0) {
#pragma unroll
    for (int i = 0; i < E; i += 4) {
      const float4 v = __ldcs(reinterpret_cast<const float4 *>(p + i));
      out[i] = v.x;
      out[i + 1] = v.y;
      out[i + 2] = v.z;
      out[i + 3] = v.w;
    }
  } else {
    ldn_stream<E>(p, out);
  }
}
template <int E, bool W16>
__device__ __forceinline__ void ldblock(const double *p, double *out) {
  ldn_stream<E>(p, out);
}
template <int E, bool W16>
__device__ __forceinline__ void ldblock(const __nv_bfloat16 *p, float *out) {
  ldn_stream<E>(p, out);
}

template <int BR, int BC, typename V, typename T, int MODE>
__global__ void __launch_bounds__(256) bsr_lblock_kernel(int n_rows, const int *__restrict__ rowptr,
                                                         const int *__restrict__ colidx,
                                                         const V *__restrict__ vals,
                                                         const T *__restrict__ x,
                                                         const T *__restrict__ b,
                                                         const T *__restrict__ minv,
                                                         T *__restrict__ y) {
  pdl_enter();
  using A = typename AccT<T>::type;
  constexpr int E = BR * BC;
  // a block starts 16-byte aligned when E * sizeof(V) is a multiple of 16
  constexpr bool W16 = (E * sizeof(V)) % 16 == 0;
  using St = LbStage<E, V>;
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n_rows; row += nwarps) {
    const int s = rowptr[row], e = rowptr[row + 1];
    A acc[BR];
#pragma unroll
    for (int r = 0; r < BR; ++r) acc[r] = 0;
    if constexpr (St::ON) {
      using W = typename St::W;
      constexpr int WPB = St::BYTES / (int)sizeof(W);  // words per block
      // one 32-block buffer per warp of the 256-thread block
      __shared__ __align__(16) W stage_w[8 * 32 * WPB];
      W *dst = stage_w + (threadIdx.x >> 5) * 32 * WPB;
      const V *stage = reinterpret_cast<const V *>(dst);
      // passes of 32 blocks (uniform over the warp)
      for (int p0 = s; p0 < e; p0 += 32) {
        const int nb = min(32, e - p0);
        const W *src = reinterpret_cast<const W *>(vals + (size_t)p0 * E);
        for (int k = lane; k < nb * WPB; k += 32) dst[k] = __ldcs(src + k);
        __syncwarp();
        if (lane < nb) {
          const int c = __ldg(colidx + p0 + lane);
          A xv[BC], v[E];
          ldn_cached<BC>(x + (size_t)c * BC, xv);
          stage_read<E>(stage + lane * E, v);
#pragma unroll
          for (int r = 0; r < BR; ++r)
#pragma unroll
            for (int q = 0; q < BC; ++q) acc[r] += v[r * BC + q] * xv[q];
        }
        __syncwarp();
      }
    } else {
      for (int p = s + lane; p < e; p += 32) {
        const int c = __ldg(colidx + p);
        A xv[BC], v[E];
        ldn_cached<BC>(x + (size_t)c * BC, xv);
        ldblock<E, W16>(vals + (size_t)p * E, v);
#pragma unroll
        for (int r = 0; r < BR; ++r)
#pragma unroll
          for (int q = 0; q < BC; ++q) acc[r] += v[r * BC + q] * xv[q];
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < BR; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    const size_t o = (size_t)row * BR;
    if (lane >= BR) continue;
    A mine = 0;  // acc[lane] without dynamic register indexing
#pragma unroll
    for (int r = 0; r < BR; ++r)
      if (lane == r) mine = acc[r];
    if (MODE == SPMV_SMOOTH) {
      A upd = 0;
#pragma unroll
      for (int q = 0; q < BR; ++q) upd += (A)minv[(o + lane) * BR + q] * ((A)b[o + q] - acc[q]);
      y[o + lane] = (T)((A)x[o + lane] + upd);
    } else {
      if (MODE == SPMV_SET) y[o + lane] = (T)mine;
      if (MODE == SPMV_RESID) y[o + lane] = (T)((A)b[o + lane] - mine);
      if (MODE == SPMV_ADD) y[o + lane] = (T)((A)y[o + lane] + mine);
    }
  }
}

template <int BR, int BC, typename V, typename T>
static cudaError_t lblock_mode(const Ctx *c, const DevBSR &A, const V *vals, int mode, const void *x,
                               const void *b, const void *minv, void *y) {
  const T *xx = (const T *)x;
  const T *bb = (const T *)b;
  const T *mm = (const T *)minv;
  T *yy = (T *)y;
#define AMG_LB_LAUNCH(M_)                                                                    \
  AMG_KLAUNCH(c, bsr_lblock_kernel<BR, BC, V, T, M_>,                                        \
              grid_for_rows(c, A.n_rows, bsr_lblock_kernel<BR, BC, V, T, M_>), 256, A.n_rows, \
              A.rowptr, A.colidx, vals, xx, bb, mm, yy)
  switch (mode) {
    case SPMV_SET: AMG_LB_LAUNCH(SPMV_SET); break;
    case SPMV_RESID: AMG_LB_LAUNCH(SPMV_RESID); break;
    case SPMV_ADD: AMG_LB_LAUNCH(SPMV_ADD); break;
    case SPMV_SMOOTH:
      if constexpr (BR == BC) {
        AMG_LB_LAUNCH(SPMV_SMOOTH);
        break;
      } else {
        return cudaErrorInvalidValue;
      }
    default: return cudaErrorInvalidValue;
  }
#undef AMG_LB_LAUNCH
  return cudaGetLastError();
}

// SELL-32 variant: one thread per block row, all lanes of a warp on 32
// consecutive rows.  Every value load of a slot is a coalesced 32-wide row,
// no cross-lane reduction is needed, and every FP64 lane does useful work
// (on sm_103a each FP64 warp instruction occupies the SM's FP64 pipe for
// many cycles, so idle or reducing lanes cost as much as useful ones).
template <int BR, int BC, typename V, typename T, int MODE, typename TO = T>
__global__ void __launch_bounds__(256) sell_kernel(int n_rows, int n_slices,
                                                   const int *__restrict__ sell_ptr,
                                                   const int *__restrict__ sell_col,
                                                   const V *__restrict__ vals,
                                                   const T *__restrict__ x,
                                                   const T *__restrict__ b,
                                                   const T *__restrict__ minv,
                                                   TO *__restrict__ y) {
  pdl_enter();
  using A = typename AccT<T>::type;
  constexpr int E = BR * BC;
  const int slice = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (slice >= n_slices) return;
  const int t = threadIdx.x & 31;
  const int row = slice * 32 + t;
  const int j0 = sell_ptr[slice], j1 = sell_ptr[slice + 1];
  A acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = 0;
#pragma unroll 2
  for (int j = j0; j < j1; ++j) {
    const int c = __ldg(sell_col + (size_t)j * 32 + t);
    const V *v = vals + (size_t)j * E * 32 + t;
    A xv[BC];
#pragma unroll
    for (int q = 0; q < BC; ++q) xv[q] = (A)ld(x + (size_t)c * BC + q);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int q = 0; q < BC; ++q) acc[r] += (A)lds(v + (r * BC + q) * 32) * xv[q];
  }
  if (row >= n_rows) return;
  const size_t o = (size_t)row * BR;
  if (MODE == SPMV_SMOOTH) {
    A res[BR];
#pragma unroll
    for (int r = 0; r < BR; ++r) res[r] = (A)b[o + r] - acc[r];
#pragma unroll
    for (int r = 0; r < BR; ++r) {
      A u = 0;
#pragma unroll
      for (int q = 0; q < BR; ++q) u += (A)minv[(o + r) * BR + q] * res[q];
      y[o + r] = (TO)((A)x[o + r] + u);
    }
  } else {
#pragma unroll
    for (int r = 0; r < BR; ++r) {
      if (MODE == SPMV_SET) y[o + r] = (TO)acc[r];
      if (MODE == SPMV_RESID) y[o + r] = (TO)((A)b[o + r] - acc[r]);
      if (MODE == SPMV_ADD) y[o + r] = (TO)((A)y[o + r] + acc[r]);
    }
  }
}

// The same for a sorted SELL-32 copy (the transfer operators and the square
// operators of the coarse levels): lane t of a slice computes row
// perm[32 * slice + t] (n_rows on a padding lane), so rows of similar length
// share a slice.
template <int BR, int BC, typename V, typename T, int MODE>
__global__ void __launch_bounds__(256) sell_perm_kernel(int n_rows, int n_slices,
                                                        const int *__restrict__ sell_ptr,
                                                        const int *__restrict__ sell_col,
                                                        const int *__restrict__ perm,
                                                        const V *__restrict__ vals,
                                                        const T *__restrict__ x,
                                                        const T *__restrict__ b,
                                                        const T *__restrict__ minv,
                                                        T *__restrict__ y) {
  static_assert(MODE != SPMV_SMOOTH || BR == BC, "smoothing needs a square operator");
  pdl_enter();
  using A = typename AccT<T>::type;
  constexpr int E = BR * BC;
  const int slice = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (slice >= n_slices) return;
  const int t = threadIdx.x & 31;
  const int row = __ldg(perm + slice * 32 + t);
  const int j0 = sell_ptr[slice], j1 = sell_ptr[slice + 1];
  A acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = 0;
  // the rows of transfer operators are short (about five blocks): take the
  // slots four at a time, column indices first, then all their x gathers,
  // so that the dependent loads of four blocks are in flight together
  constexpr int U = 4;
  for (int j = j0; j < j1; j += U) {
    int cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) cc[u] = (j + u < j1) ? __ldg(sell_col + (size_t)(j + u) * 32 + t) : 0;
    A xv[U][BC];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j + u < j1) {
        ldn_cached<BC>(x + (size_t)cc[u] * BC, xv[u]);
      } else {
#pragma unroll
        for (int q = 0; q < BC; ++q) xv[u][q] = (A)0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j + u < j1) {
        const V *v = vals + (size_t)(j + u) * E * 32 + t;
#pragma unroll
        for (int r = 0; r < BR; ++r)
#pragma unroll
          for (int q = 0; q < BC; ++q) acc[r] += (A)lds(v + (r * BC + q) * 32) * xv[u][q];
      }
    }
  }
  if (row >= n_rows) return;
  const size_t o = (size_t)row * BR;
  if (MODE == SPMV_SMOOTH) {
    A res[BR];
#pragma unroll
    for (int r = 0; r < BR; ++r) res[r] = (A)b[o + r] - acc[r];
#pragma unroll
    for (int r = 0; r < BR; ++r) {
      A u = 0;
#pragma unroll
      for (int q = 0; q < BR; ++q) u += (A)minv[(o + r) * BR + q] * res[q];
      y[o + r] = (T)((A)x[o + r] + u);
    }
    return;
  }
#pragma unroll
  for (int r = 0; r < BR; ++r) {
    if (MODE == SPMV_SET) y[o + r] = (T)acc[r];
    if (MODE == SPMV_RESID) y[o + r] = (T)((A)b[o + r] - acc[r]);
    if (MODE == SPMV_ADD) y[o + r] = (T)((A)y[o + r] + acc[r]);
  }
}

// The sorted SELL-32 product with the BR output rows of a slice split over
// BR warps: warp r of a slice computes output row r of its 32 block rows
// from row r of every block (BC contiguous 32-wide rows of a slot).  The BR
// warps of a slice read the same column indices and x entries (the second
// and later from L1) and each a BR-th of the values, so a transfer operator
// with short rows has BR times the warps in flight, each with a BR-th of the
// arithmetic.  Per output entry the sums run in sell_perm_kernel's order, so
// both give the same bits.
template <int BR, int BC, typename V, typename T, int MODE>
__global__ void __launch_bounds__(256) sell_split_kernel(int n_rows, int n_slices,
                                                         const int *__restrict__ sell_ptr,
                                                         const int *__restrict__ sell_col,
                                                         const int *__restrict__ perm,
                                                         const V *__restrict__ vals,
                                                         const T *__restrict__ x,
                                                         const T *__restrict__ b,
                                                         T *__restrict__ y) {
  static_assert(MODE != SPMV_SMOOTH, "the smoothing mode needs every output row of a block row");
  pdl_enter();
  using A = typename AccT<T>::type;
  constexpr int E = BR * BC;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int slice = gw / BR, r = gw - slice * BR;
  if (slice >= n_slices) return;
  const int t = threadIdx.x & 31;
  const int row = __ldg(perm + slice * 32 + t);
  const int j0 = sell_ptr[slice], j1 = sell_ptr[slice + 1];
  A acc = 0;
  constexpr int U = 4;
  for (int j = j0; j < j1; j += U) {
    int cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) cc[u] = (j + u < j1) ? __ldg(sell_col + (size_t)(j + u) * 32 + t) : 0;
    A xv[U][BC];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j + u < j1) {
        ldn_cached<BC>(x + (size_t)cc[u] * BC, xv[u]);
      } else {
#pragma unroll
        for (int q = 0; q < BC; ++q) xv[u][q] = (A)0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j + u < j1) {
        const V *v = vals + (size_t)(j + u) * E * 32 + (size_t)r * BC * 32 + t;
#pragma unroll
        for (int q = 0; q < BC; ++q) acc += (A)lds(v + q * 32) * xv[u][q];
      }
    }
  }
  if (row >= n_rows) return;
  const size_t o = (size_t)row * BR + r;
  if (MODE == SPMV_SET) y[o] = (T)acc;
  if (MODE == SPMV_RESID) y[o] = (T)((A)b[o] - acc);
  if (MODE == SPMV_ADD) y[o] = (T)((A)y[o] + acc);
}

template <int BR, int BC, typename V, typename T>
static cudaError_t sell_mode(const Ctx *c, const DevBSR &A, const V *vals, int mode, const void *x,
                             const void *b, const void *minv, void *y) {
  // 64-thread blocks (two slices each) spread the rows evenly over the SMs
  const int g = (A.n_slices + 1) / 2;
  const T *xx = (const T *)x;
  const T *bb = (const T *)b;
  const T *mm = (const T *)minv;
  T *yy = (T *)y;
  if (A.sell_perm && A.kern == KERN_SELL_SPLIT && mode != SPMV_SMOOTH) {
    // BR warps per slice, 8 warps per block
    const int gs = (int)(((long long)A.n_slices * BR + 7) / 8);
#define AMG_SELL_SPLIT_LAUNCH(M_)                                                                  \
  AMG_KLAUNCH(c, sell_split_kernel<BR, BC, V, T, M_>, gs, 256, A.n_rows, A.n_slices, A.sell_ptr, \
              A.sell_col, A.sell_perm, vals, xx, bb, yy)
    switch (mode) {
      case SPMV_SET: AMG_SELL_SPLIT_LAUNCH(SPMV_SET); break;
      case SPMV_RESID: AMG_SELL_SPLIT_LAUNCH(SPMV_RESID); break;
      case SPMV_ADD: AMG_SELL_SPLIT_LAUNCH(SPMV_ADD); break;
      default: return cudaErrorInvalidValue;
    }
#undef AMG_SELL_SPLIT_LAUNCH
    return cudaGetLastError();
  }
  if (A.sell_perm) {
#define AMG_SELL_PERM_LAUNCH(M_)                                                                 \
  AMG_KLAUNCH(c, sell_perm_kernel<BR, BC, V, T, M_>, g, 64, A.n_rows, A.n_slices, A.sell_ptr, \
              A.sell_col, A.sell_perm, vals, xx, bb, mm, yy)
    switch (mode) {
      case SPMV_SET: AMG_SELL_PERM_LAUNCH(SPMV_SET); break;
      case SPMV_RESID: AMG_SELL_PERM_LAUNCH(SPMV_RESID); break;
      case SPMV_ADD: AMG_SELL_PERM_LAUNCH(SPMV_ADD); break;
      case SPMV_SMOOTH:
        if constexpr (BR == BC) {
          AMG_SELL_PERM_LAUNCH(SPMV_SMOOTH);
          break;
        } else {
          return cudaErrorInvalidValue;
        }
      default: return cudaErrorInvalidValue;
    }
#undef AMG_SELL_PERM_LAUNCH
    return cudaGetLastError();
  }
#define AMG_SELL_LAUNCH(M_)                                                                    \
  AMG_KLAUNCH(c, sell_kernel<BR, BC, V, T, M_>, g, 64, A.n_rows, A.n_slices, A.sell_ptr,   \
                                                          A.sell_col, vals, xx, bb, mm, yy)
  switch (mode) {
    case SPMV_SET: AMG_SELL_LAUNCH(SPMV_SET); break;
    case SPMV_RESID: AMG_SELL_LAUNCH(SPMV_RESID); break;
    case SPMV_ADD: AMG_SELL_LAUNCH(SPMV_ADD); break;
    case SPMV_SMOOTH:
      if constexpr (BR == BC) {
        AMG_SELL_LAUNCH(SPMV_SMOOTH);
        break;
      } else {
        return cudaErrorInvalidValue;
      }
    default: return cudaErrorInvalidValue;
  }
#undef AMG_SELL_LAUNCH
  return cudaGetLastError();
}

template <int BR, int BC>
static cudaError_t bsr_prec(const Ctx *c, const DevBSR &A, int prec, int mode, const void *x,
                            const void *b, const void *minv, void *y) {
  if (A.n_rows == 0) return cudaSuccess;
  if (A.sell_ptr && (A.kern == KERN_SELL || A.kern == KERN_SELL_SPLIT)) {
    if (prec == AMG_PREC_FP64)
      return sell_mode<BR, BC, double, double>(c, A, A.s64, mode, x, b, minv, y);
    if (prec == AMG_PREC_FP32_VCYCLE)
      return sell_mode<BR, BC, float, float>(c, A, A.s32, mode, x, b, minv, y);
    return sell_mode<BR, BC, __nv_bfloat16, float>(c, A, A.s16, mode, x, b, minv, y);
  }
  int kern = (A.kern == KERN_SELL || A.kern == KERN_SELL_SPLIT) ? KERN_WARP_ROWS : A.kern;
  if (c->layout_policy == AMG_LAYOUT_ROW_LANES) kern = KERN_ROW_LANES;
  if (c->layout_policy == AMG_LAYOUT_BLOCK_LANES) kern = KERN_BLOCK_LANES;
  if (kern == KERN_BLOCK_LANES) {
    if (prec == AMG_PREC_FP64)
      return lblock_mode<BR, BC, double, double>(c, A, A.v64, mode, x, b, minv, y);
    if (prec == AMG_PREC_FP32_VCYCLE)
      return lblock_mode<BR, BC, float, float>(c, A, A.v32, mode, x, b, minv, y);
    return lblock_mode<BR, BC, __nv_bfloat16, float>(c, A, A.v16, mode, x, b, minv, y);
  }
  if (kern != KERN_ROW_LANES) {
    if (prec == AMG_PREC_FP64)
      return bsr_mode<BR, BC, double, double>(c, A, A.v64, mode, x, b, minv, y);
    if (prec == AMG_PREC_FP32_VCYCLE)
      return bsr_mode<BR, BC, float, float>(c, A, A.v32, mode, x, b, minv, y);
    return bsr_mode<BR, BC, __nv_bfloat16, float>(c, A, A.v16, mode, x, b, minv, y);
  }
  if (prec == AMG_PREC_FP64)
    return rowlane_mode<BR, BC, double, double>(c, A, A.v64, mode, x, b, minv, y);
  if (prec == AMG_PREC_FP32_VCYCLE)
    return rowlane_mode<BR, BC, float, float>(c, A, A.v32, mode, x, b, minv, y);
  return rowlane_mode<BR, BC, __nv_bfloat16, float>(c, A, A.v16, mode, x, b, minv, y);
}

// Post-smoothing of the finest level in the mixed precisions: FP32
// arithmetic, result written as FP64 for the outer CG (saves a cast pass).
template <int K, typename V>
static cudaError_t smooth_out64_k(const Ctx *c, const DevBSR &A, const V *bsr_vals, const V *sell_vals,
                                  const float *x, const float *b, const float *minv, double *y) {
  if (A.sell_ptr && A.kern == KERN_SELL) {
    AMG_KLAUNCH(c, sell_kernel<K, K, V, float, SPMV_SMOOTH, double>, (A.n_slices + 1) / 2, 64, 
        A.n_rows, A.n_slices, A.sell_ptr, A.sell_col, sell_vals, x, b, minv, y);
  } else {
    AMG_KLAUNCH(c, bsr_warp_kernel<K, K, V, float, SPMV_SMOOTH, double>,
                grid_for_rows(c, A.n_rows, bsr_warp_kernel<K, K, V, float, SPMV_SMOOTH, double>), 256, 
        A.n_rows, A.rowptr, A.colidx, bsr_vals, x, b, minv, y);
  }
  return cudaGetLastError();
}

cudaError_t launch_smooth_out64(const Ctx *c, const DevBSR &A, int prec, const float *x,
                                const float *b, const float *minv, double *y) {
  if (A.n_rows == 0) return cudaSuccess;
  if (A.br != A.bc || prec == AMG_PREC_FP64) return cudaErrorInvalidValue;
  if (prec == AMG_PREC_FP32_VCYCLE) {
    if (A.br == 1) return smooth_out64_k<1, float>(c, A, A.v32, A.s32, x, b, minv, y);
    if (A.br == 2) return smooth_out64_k<2, float>(c, A, A.v32, A.s32, x, b, minv, y);
    if (A.br == 3) return smooth_out64_k<3, float>(c, A, A.v32, A.s32, x, b, minv, y);
  } else {
    if (A.br == 1) return smooth_out64_k<1, __nv_bfloat16>(c, A, A.v16, A.s16, x, b, minv, y);
    if (A.br == 2) return smooth_out64_k<2, __nv_bfloat16>(c, A, A.v16, A.s16, x, b, minv, y);
    if (A.br == 3) return smooth_out64_k<3, __nv_bfloat16>(c, A, A.v16, A.s16, x, b, minv, y);
  }
  return cudaErrorInvalidValue;
}

// Pre-smoothing of the finest level in the mixed precisions: reads the FP64
// CG residual, stores its FP32 copy b and x = M^+ b (FP32).
template <int K>
__global__ void blockdiag_entry_kernel(int n, const float *__restrict__ minv,
                                       const double *__restrict__ r, float *__restrict__ b,
                                       float *__restrict__ x) {
  pdl_enter();
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= (size_t)n) return;
  float rb[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    rb[q] = (float)r[v * K + q];
    b[v * K + q] = rb[q];
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < K; ++q) acc += minv[(v * K + i) * K + q] * rb[q];
    x[v * K + i] = acc;
  }
}

cudaError_t launch_blockdiag_entry(const Ctx *c, int n, int k, const float *minv, const double *r,
                                   float *b, float *x) {
  if (n == 0) return cudaSuccess;
  const int g = (n + 255) / 256;
  if (k == 1)
    AMG_KLAUNCH(c, blockdiag_entry_kernel<1>, g, 256, n, minv, r, b, x);
  else if (k == 2)
    AMG_KLAUNCH(c, blockdiag_entry_kernel<2>, g, 256, n, minv, r, b, x);
  else if (k == 3)
    AMG_KLAUNCH(c, blockdiag_entry_kernel<3>, g, 256, n, minv, r, b, x);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_bsr(const Ctx *c, const DevBSR &A, int prec, int mode, const void *x,
                       const void *b, const void *minv, void *y) {
#define AMG_BSR_CASE(R_, C_) \
  if (A.br == R_ && A.bc == C_) return bsr_prec<R_, C_>(c, A, prec, mode, x, b, minv, y);
  AMG_BSR_CASE(1, 1)
  AMG_BSR_CASE(2, 2)
  AMG_BSR_CASE(3, 3)
  AMG_BSR_CASE(6, 6)
  AMG_BSR_CASE(2, 3)
  AMG_BSR_CASE(3, 2)
  AMG_BSR_CASE(3, 6)
  AMG_BSR_CASE(6, 3)
#undef AMG_BSR_CASE
  return cudaErrorInvalidValue;
}

// y_i = M_i^+ b_i for every vertex (pre-smoothing from a zero guess).
template <int K, typename T>
__global__ void blockdiag_kernel(int n, const T *__restrict__ minv, const T *__restrict__ b,
                                 T *__restrict__ y) {
  pdl_enter();
  using A = typename AccT<T>::type;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * K) return;
  const size_t v = t / K;
  A acc = 0;
#pragma unroll
  for (int q = 0; q < K; ++q) acc += (A)minv[t * K + q] * (A)b[v * K + q];
  y[t] = (T)acc;
}

template <int K>
static cudaError_t blockdiag_k(const Ctx *c, int n, int prec, const void *minv, const void *b,
                               void *y) {
  const size_t tot = (size_t)n * K;
  const int g = (int)((tot + 255) / 256);
  if (tot == 0) return cudaSuccess;
  if (prec == AMG_PREC_FP64)
    AMG_KLAUNCH(c, blockdiag_kernel<K, double>, g, 256, n, (const double *)minv,
                                                          (const double *)b, (double *)y);
  else
    AMG_KLAUNCH(c, blockdiag_kernel<K, float>, g, 256, n, (const float *)minv,
                                                         (const float *)b, (float *)y);
  return cudaGetLastError();
}

cudaError_t launch_blockdiag(const Ctx *c, int n, int k, int prec, const void *minv, const void *b,
                             void *y) {
  if (k == 1) return blockdiag_k<1>(c, n, prec, minv, b, y);
  if (k == 2) return blockdiag_k<2>(c, n, prec, minv, b, y);
  if (k == 3) return blockdiag_k<3>(c, n, prec, minv, b, y);
  if (k == 6) return blockdiag_k<6>(c, n, prec, minv, b, y);
  return cudaErrorInvalidValue;
}

// y = Cinv b (FP64 dense inverse of the regularised coarsest matrix); input
// and output in the V-cycle precision.  Four warps per row, each summing a
// quarter of it with four partial sums per lane, combined in shared memory:
// a row of the inverse (up to ~10 KB) read by one warp alone is a chain of
// dependent trips that leaves the GPU idle (13 us for 1,242 rows).
template <typename T>
__global__ void __launch_bounds__(256) coarse_gemv_kernel(int n, const double *__restrict__ cinv,
                                                          const T *__restrict__ b,
                                                          T *__restrict__ y) {
  pdl_enter();
  __shared__ double part[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // 2 rows x 4 quarters
  const int row = blockIdx.x * 2 + (w >> 2), qtr = w & 3;
  double acc = 0.0;
  if (row < n) {
    const int j0 = (int)((long)n * qtr / 4), j1 = (int)((long)n * (qtr + 1) / 4);
    const double *a = cinv + (size_t)row * n;
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
    int j = j0 + lane;
    for (; j + 96 < j1; j += 128) {
      acc0 += a[j] * (double)b[j];
      acc1 += a[j + 32] * (double)b[j + 32];
      acc2 += a[j + 64] * (double)b[j + 64];
      acc3 += a[j + 96] * (double)b[j + 96];
    }
    for (; j < j1; j += 32) acc0 += a[j] * (double)b[j];
    acc = (acc0 + acc1) + (acc2 + acc3);
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, s);
  }
  if (lane == 0) part[w] = acc;
  __syncthreads();
  if (threadIdx.x < 2) {
    const int r = blockIdx.x * 2 + threadIdx.x;
    const double *pp = part + 4 * threadIdx.x;
    if (r < n) y[r] = (T)((pp[0] + pp[1]) + (pp[2] + pp[3]));
  }
}

cudaError_t launch_coarse_gemv(const Ctx *c, int n, const double *cinv, const void *b, void *y,
                               int prec) {
  if (n == 0) return cudaSuccess;
  const int g = (n + 1) / 2;
  if (prec == AMG_PREC_FP64)
    AMG_KLAUNCH(c, coarse_gemv_kernel<double>, g, 256, n, cinv, (const double *)b, (double *)y);
  else
    AMG_KLAUNCH(c, coarse_gemv_kernel<float>, g, 256, n, cinv, (const float *)b, (float *)y);
  return cudaGetLastError();
}

template <typename S, typename D>
__global__ void convert_kernel(size_t n, const S *__restrict__ s, D *__restrict__ d) {
  pdl_enter();
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = (D)s[i];
}

cudaError_t launch_convert(const Ctx *c, size_t n, const void *src, int src_prec, void *dst,
                           int dst_prec) {
  if (n == 0) return cudaSuccess;
  const int g = (int)((n + 255) / 256);
  const bool s64 = src_prec == AMG_PREC_FP64, d64 = dst_prec == AMG_PREC_FP64;
  if (s64 && !d64)
    AMG_KLAUNCH(c, convert_kernel<double, float>, g, 256, n, (const double *)src, (float *)dst);
  else if (!s64 && d64)
    AMG_KLAUNCH(c, convert_kernel<float, double>, g, 256, n, (const float *)src, (double *)dst);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// FP32 / BF16 copies of a matrix's values (round to nearest).
__global__ void to_f32_kernel(size_t n, const double *__restrict__ s, float *__restrict__ d) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = (float)s[i];
}
__global__ void to_bf16_kernel(size_t n, const double *__restrict__ s, __nv_bfloat16 *__restrict__ d) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = __float2bfloat16_rn((float)s[i]);
}

// ---------------------------------------------------------------------------
// SELL-32 construction from the BSR arrays (device)
// ---------------------------------------------------------------------------

// Row order of a sorted SELL-32 copy: one 256-thread block per window of 256
// rows ranks the window's rows by length, longest first (ties by row index),
// so that the window's 8 slices each hold rows of similar length and little
// padding.  perm[w*256 + rank] = row; lanes past the window's last row get
// n_rows (padding).  Every slot below n_slots is written exactly once.
__global__ void __launch_bounds__(256) sell_sort_kernel(int n_rows, int n_slots,
                                                        const int *__restrict__ rowptr,
                                                        int *__restrict__ perm) {
  __shared__ int len[256];
  const int i = threadIdx.x;
  const int row = blockIdx.x * 256 + i;
  const int l = row < n_rows ? rowptr[row + 1] - rowptr[row] : -1;
  len[i] = l;
  __syncthreads();
  int rank = 0;
  for (int j = 0; j < 256; ++j) {
    const int lj = len[j];
    rank += (lj > l) || (lj == l && j < i);
  }
  const int dst = blockIdx.x * 256 + rank;
  if (dst < n_slots) perm[dst] = l >= 0 ? row : n_rows;
}

// the row held by lane t of a slice (identity order without perm)
__device__ __forceinline__ int sell_lane_row(const int *__restrict__ perm, int slice, int t) {
  return perm ? perm[slice * 32 + t] : slice * 32 + t;
}

__global__ void sell_width_kernel(int n_rows, int n_slices, const int *__restrict__ rowptr,
                                  const int *__restrict__ perm, int *__restrict__ w) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > n_slices) return;
  if (s == n_slices) {
    w[s] = 0;
    return;
  }
  int m = 0;
  for (int t = 0; t < 32; ++t) {
    const int r = sell_lane_row(perm, s, t);
    if (r < n_rows) m = max(m, rowptr[r + 1] - rowptr[r]);
  }
  w[s] = m;
}

template <int E>
__global__ void sell_fill_kernel(int n_rows, int n_slices, const int *__restrict__ rowptr,
                                 const int *__restrict__ colidx, const double *__restrict__ vals,
                                 const int *__restrict__ sell_ptr, const int *__restrict__ perm,
                                 int *__restrict__ sell_col, double *__restrict__ s64) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int slice = g >> 5, t = g & 31;
  if (slice >= n_slices) return;
  const int row = sell_lane_row(perm, slice, t);
  const int rs = row < n_rows ? rowptr[row] : 0;
  const int len = row < n_rows ? rowptr[row + 1] - rs : 0;
  for (int j = sell_ptr[slice]; j < sell_ptr[slice + 1]; ++j) {
    const int jj = j - sell_ptr[slice];
    const bool real = jj < len;
    sell_col[(size_t)j * 32 + t] = real ? colidx[rs + jj] : 0;
    for (int q = 0; q < E; ++q)
      s64[((size_t)j * E + q) * 32 + t] = real ? vals[(size_t)(rs + jj) * E + q] : 0.0;
  }
}

bool want_sell(const Ctx *c, const DevBSR &m, bool coarse_square) {
  // thread-per-row pays off when there are enough rows to fill the GPU with
  // warps (>= 16 warps per SM) and the rows are short; rectangular operators
  // (length-sorted slices, little padding) up to 64 blocks per row, so that
  // the tuner also times the sorted SELL-32 form of the first restriction
  const double avg = m.n_rows ? (double)m.nnzb / m.n_rows : 0.0;
  const bool rect = m.br != m.bc || m.n_rows != m.n_cols;
  if (c->layout_policy == AMG_LAYOUT_WARP_ROWS || c->layout_policy == AMG_LAYOUT_ROW_LANES ||
      c->layout_policy == AMG_LAYOUT_BLOCK_LANES)
    return false;
  if (c->layout_policy == AMG_LAYOUT_SELL_SHORT_ROWS || c->layout_policy == AMG_LAYOUT_SELL_SPLIT)
    return avg <= 32.0;
  // coarse square operators (sorted slices too) up to 96 blocks per row
  return m.n_rows >= 32 * 16 * c->num_sms && avg <= (rect ? 64.0 : coarse_square ? 96.0 : 32.0);
}

cudaError_t build_sell(Ctx *c, DevBSR &m, bool sort_square) {
  const int E = m.br * m.bc;
  dfree(m.sell_ptr);
  dfree(m.sell_col);
  dfree(m.sell_perm);
  dfree(m.s64);
  m.sell_ptr = nullptr;
  m.sell_col = nullptr;
  m.sell_perm = nullptr;
  m.s64 = nullptr;
  m.n_slices = (m.n_rows + 31) / 32;
  // rectangular operators (P_l, R_l) and, when asked, square ones get
  // length-sorted slices
  if ((m.br != m.bc || m.n_rows != m.n_cols || sort_square) && m.n_slices > 0) {
    const int n_slots = m.n_slices * 32;
    AMG_CUDA_TRY(dalloc((void **)&m.sell_perm, (size_t)n_slots * sizeof(int)));
    sell_sort_kernel<<<(n_slots + 255) / 256, 256, 0, c->stream>>>(m.n_rows, n_slots, m.rowptr,
                                                                   m.sell_perm);
    AMG_CUDA_TRY(cudaGetLastError());
  }
  AMG_CUDA_TRY(dalloc((void **)&m.sell_ptr, (size_t)(m.n_slices + 1) * sizeof(int)));
  int *total = nullptr;
  AMG_CUDA_TRY(dalloc((void **)&total, sizeof(int)));
  sell_width_kernel<<<(m.n_slices + 256) / 256, 256, 0, c->stream>>>(m.n_rows, m.n_slices, m.rowptr,
                                                                     m.sell_perm, m.sell_ptr);
  AMG_CUDA_TRY(cudaGetLastError());
  AMG_CUDA_TRY(scan_exclusive(c, m.n_slices + 1, m.sell_ptr, total));
  int slots = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&slots, total, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  dfree(total);
  m.sell_slots = slots;
  AMG_CUDA_TRY(dalloc((void **)&m.sell_col, (size_t)slots * 32 * sizeof(int)));
  AMG_CUDA_TRY(dalloc((void **)&m.s64, (size_t)slots * 32 * E * sizeof(double)));
  const int g = (m.n_slices * 32 + 255) / 256;
#define AMG_FILL(E_)                                                                     \
  if (E == E_)                                                                          \
    sell_fill_kernel<E_><<<g, 256, 0, c->stream>>>(m.n_rows, m.n_slices, m.rowptr,     \
                                                   m.colidx, m.v64, m.sell_ptr,        \
                                                   m.sell_perm, m.sell_col, m.s64);
  AMG_FILL(1) AMG_FILL(4) AMG_FILL(9) AMG_FILL(36) AMG_FILL(6) AMG_FILL(18)
#undef AMG_FILL
  return cudaGetLastError();
}

// Largest |a| of n values, as the bit pattern of a non-negative double
// (non-negative doubles are ordered like their bit patterns).
__global__ void absmax_bits_kernel(size_t n, const double *__restrict__ v,
                                   unsigned long long *__restrict__ out) {
  unsigned long long m = 0ull;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v[i]));
    m = b > m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_down_sync(0xffffffffu, m, o);
    m = w > m ? w : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// a * scale (a power of two, exact) as hi + lo: hi the FP32 rounding, lo the
// FP32 rounding of the exact remainder (48 significant bits together).
__global__ void split_double_float_kernel(size_t n, const double *__restrict__ v, double scale,
                                          float2 *__restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = v[i] * scale;
  const float hi = __double2float_rn(a);
  const float lo = __double2float_rn(a - (double)hi);
  out[i] = make_float2(hi, lo);
}

// The CG operator's double-float copy of a SELL-32 operator: the values
// scaled by 2^-df_exp (max |a| 2^-df_exp < 1) and split into hi + lo.
cudaError_t build_double_float(Ctx *c, DevBSR &m) {
  dfree(m.sdf);
  m.sdf = nullptr;
  m.df_exp = 0;
  if (!m.s64) return cudaSuccess;
  const size_t ns = (size_t)m.sell_slots * 32 * m.br * m.bc;
  unsigned long long *d_max = nullptr;
  AMG_CUDA_TRY(dalloc((void **)&d_max, sizeof(unsigned long long)));
  AMG_CUDA_TRY(cudaMemsetAsync(d_max, 0, sizeof(unsigned long long), c->stream));
  absmax_bits_kernel<<<c->num_sms * 8, 256, 0, c->stream>>>(ns, m.s64, d_max);
  AMG_CUDA_TRY(cudaGetLastError());
  unsigned long long mb = 0ull;
  AMG_CUDA_TRY(cudaMemcpyAsync(&mb, d_max, sizeof(mb), cudaMemcpyDeviceToHost, c->stream));
  AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  dfree(d_max);
  // max |a| in [2^e, 2^(e+1)): df_exp = e + 1 puts every scaled value below 1
  const int e = (int)((mb >> 52) & 0x7FFull) - 1023;
  m.df_exp = mb ? e + 1 : 0;
  AMG_CUDA_TRY(dalloc((void **)&m.sdf, (ns ? ns : 1) * sizeof(float2)));
  if (ns) {
    split_double_float_kernel<<<(unsigned)((ns + 255) / 256), 256, 0, c->stream>>>(
        ns, m.s64, ldexp(1.0, -m.df_exp), m.sdf);
    AMG_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

cudaError_t make_low_precision(Ctx *c, DevBSR &m, int prec) {
  const size_t n = (size_t)m.nnzb * m.br * m.bc;
  if (n == 0) return cudaSuccess;
  const int g = (int)((n + 255) / 256);
  if (prec == AMG_PREC_FP32_VCYCLE) {
    if (!m.v32) AMG_CUDA_TRY(dalloc((void **)&m.v32, n * sizeof(float)));
    to_f32_kernel<<<g, 256, 0, c->stream>>>(n, m.v64, m.v32);
  } else if (prec == AMG_PREC_BF16_STORAGE) {
    if (!m.v16) AMG_CUDA_TRY(dalloc((void **)&m.v16, n * sizeof(__nv_bfloat16)));
    to_bf16_kernel<<<g, 256, 0, c->stream>>>(n, m.v64, m.v16);
  }
  AMG_CUDA_TRY(cudaGetLastError());
  if (m.s64) {
    const size_t ns = (size_t)m.sell_slots * 32 * m.br * m.bc;
    const int gs = (int)((ns + 255) / 256);
    if (prec == AMG_PREC_FP32_VCYCLE) {
      if (!m.s32) AMG_CUDA_TRY(dalloc((void **)&m.s32, ns * sizeof(float)));
      to_f32_kernel<<<gs, 256, 0, c->stream>>>(ns, m.s64, m.s32);
    } else if (prec == AMG_PREC_BF16_STORAGE) {
      if (!m.s16) AMG_CUDA_TRY(dalloc((void **)&m.s16, ns * sizeof(__nv_bfloat16)));
      to_bf16_kernel<<<gs, 256, 0, c->stream>>>(ns, m.s64, m.s16);
    }
  }
  return cudaGetLastError();
}

}  // namespace amg
