// Block-l1 hybrid Gauss-Seidel smoother (AMG_SMOOTHER_HYBRID_GS), the other
// form of the l1 smoothers the paper's Sec. 7 cites, for one device: the
// block rows of a level are coloured so that rows of one colour never couple
// (greedy, rows in index order: each takes the smallest colour none of its
// already coloured neighbours holds), and a sweep visits the colour classes
// in order; every row of a class computes x_v <- x_v + M_v^+ (b - A x)_v with
// the values the classes before it wrote.  A class is what a processor's
// block is to the hybrid smoother of the multi-process setting: its rows are
// updated together, and the l1 term of M_v covers couplings inside the class
// (none for a distance-1 colouring, so M_v = A_vv).  The pre-smoothing sweep
// runs the classes forward, the post-smoothing sweep backward, which keeps
// the V-cycle symmetric.
#include <algorithm>

#include "amg_internal.h"
#include "bsr_loads.cuh"

namespace amg {

// Host greedy colouring of the block graph of A_level, uploaded with the
// rows grouped by colour (ascending row index inside a class).
cudaError_t gs_prepare(Ctx *c, int level) {
  Level &L = c->levels[level];
  const int n = L.A.n_rows;
  std::vector<int> rp(n + 1), ci(L.A.nnzb > 0 ? L.A.nnzb : 1);
  AMG_CUDA_TRY(cudaMemcpyAsync(rp.data(), L.A.rowptr, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost,
                               c->stream));
  if (L.A.nnzb)
    AMG_CUDA_TRY(cudaMemcpyAsync(ci.data(), L.A.colidx, L.A.nnzb * sizeof(int),
                                 cudaMemcpyDeviceToHost, c->stream));
  AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  std::vector<int> colour(n, -1), mark;
  int n_col = 0;
  for (int i = 0; i < n; ++i) {
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
    n_col = std::max(n_col, cc + 1);
  }
  L.gs_ptr.assign(n_col + 1, 0);
  for (int i = 0; i < n; ++i) ++L.gs_ptr[colour[i] + 1];
  for (int k = 0; k < n_col; ++k) L.gs_ptr[k + 1] += L.gs_ptr[k];
  std::vector<int> rows(n > 0 ? n : 1), fill(L.gs_ptr.begin(), L.gs_ptr.end() - 1);
  for (int i = 0; i < n; ++i) rows[fill[colour[i]]++] = i;
  dfree(L.gs_colour);
  dfree(L.gs_rows);
  L.gs_colour = L.gs_rows = nullptr;
  AMG_CUDA_TRY(dalloc((void **)&L.gs_colour, (size_t)(n > 0 ? n : 1) * sizeof(int)));
  AMG_CUDA_TRY(dalloc((void **)&L.gs_rows, (size_t)(n > 0 ? n : 1) * sizeof(int)));
  AMG_CUDA_TRY(cudaMemcpyAsync(L.gs_colour, colour.data(), (size_t)n * sizeof(int),
                               cudaMemcpyHostToDevice, c->stream));
  AMG_CUDA_TRY(cudaMemcpyAsync(L.gs_rows, rows.data(), (size_t)n * sizeof(int),
                               cudaMemcpyHostToDevice, c->stream));
  return cudaStreamSynchronize(c->stream);
}

// One colour class: warp w updates block row rows[w] (lanes = block slot x
// row of the block, two block steps per trip with vector loads, as the
// warp-row SpMV kernel), x in place.  Rows of one class do not couple, so no
// warp reads an x entry another warp of this launch writes (a warp reads its
// own row's entries before it writes them): x is read through the
// read-only path.
template <int K, typename V, typename T>
__global__ void __launch_bounds__(256) gs_colour_kernel(int n, const int *__restrict__ rows,
                                                        const int *__restrict__ rowptr,
                                                        const int *__restrict__ colidx,
                                                        const V *__restrict__ vals,
                                                        const T *__restrict__ minv,
                                                        const T *__restrict__ b, T *x) {
  pdl_enter();
  constexpr int NB = 32 / K;
  const int lane = threadIdx.x & 31;
  const int bl = lane / K, r = lane - bl * K;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= n) return;  // whole warps leave together
  const int row = __ldg(rows + w);
  T acc = 0;
  if (bl < NB) {
    const int e = __ldg(rowptr + row + 1);
    int p = __ldg(rowptr + row) + bl;
    for (; p + NB < e; p += 2 * NB) {
      const int c0 = __ldg(colidx + p), c1 = __ldg(colidx + p + NB);
      T a0[K], a1[K], x0[K], x1[K];
      ldn_stream<K>(vals + ((size_t)p * K + r) * K, a0);
      ldn_stream<K>(vals + ((size_t)(p + NB) * K + r) * K, a1);
      ldn_cached<K>(x + (size_t)c0 * K, x0);
      ldn_cached<K>(x + (size_t)c1 * K, x1);
#pragma unroll
      for (int q = 0; q < K; ++q) {
        acc += a0[q] * x0[q];
        acc += a1[q] * x1[q];
      }
    }
    if (p < e) {
      const int c0 = __ldg(colidx + p);
      T a0[K], x0[K];
      ldn_stream<K>(vals + ((size_t)p * K + r) * K, a0);
      ldn_cached<K>(x + (size_t)c0 * K, x0);
#pragma unroll
      for (int q = 0; q < K; ++q) acc += a0[q] * x0[q];
    }
  }
#pragma unroll
  for (int s = 1; s < NB; s <<= 1) {
    const T o = __shfl_down_sync(0xffffffffu, acc, s * K);
    if (bl + s < NB) acc += o;
  }
  const size_t o = (size_t)row * K;
  const T res = lane < K ? b[o + lane] - acc : (T)0;
  T upd = 0;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const T rq = __shfl_sync(0xffffffffu, res, q);
    if (lane < K) upd += minv[(o + lane) * K + q] * rq;
  }
  if (lane < K) x[o + lane] += upd;
}

// The same update with block lanes, for the long rows of the coarse levels
// (6x6 blocks, 50 to 90 per row): lane j takes the blocks j, j + 32, ... of
// the row whole, all K of its sums at once, and an xor butterfly leaves the
// row's K sums on every lane.  One warp then covers 32 blocks per trip
// instead of 5, which shortens the chain of dependent loads that bounds a
// colour class of few rows.
template <int K, typename V, typename T>
__global__ void __launch_bounds__(256) gs_block_kernel(int n, const int *__restrict__ rows,
                                                       const int *__restrict__ rowptr,
                                                       const int *__restrict__ colidx,
                                                       const V *__restrict__ vals,
                                                       const T *__restrict__ minv,
                                                       const T *__restrict__ b, T *x) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= n) return;  // whole warps leave together
  const int row = __ldg(rows + w);
  const int e = __ldg(rowptr + row + 1);
  T acc[K];
#pragma unroll
  for (int r = 0; r < K; ++r) acc[r] = 0;
  for (int p = __ldg(rowptr + row) + lane; p < e; p += 32) {
    const int cc = __ldg(colidx + p);
    T xv[K], v[K * K];
    ldn_cached<K>(x + (size_t)cc * K, xv);
    ldn_stream<K * K>(vals + (size_t)p * K * K, v);
#pragma unroll
    for (int r = 0; r < K; ++r)
#pragma unroll
      for (int q = 0; q < K; ++q) acc[r] += v[r * K + q] * xv[q];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int r = 0; r < K; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
  if (lane < K) {
    const size_t o = (size_t)row * K;
    T upd = 0;
#pragma unroll
    for (int q = 0; q < K; ++q) upd += minv[(o + lane) * K + q] * (b[o + q] - acc[q]);
    x[o + lane] += upd;
  }
}

template <int K, typename V, typename T>
static cudaError_t gs_sweep_k(const Ctx *c, const Level &L, const V *vals, const T *minv, const T *b,
                              T *x, bool forward) {
  const int nc = (int)L.gs_ptr.size() - 1;
  for (int s = 0; s < nc; ++s) {
    const int k = forward ? s : nc - 1 - s;
    const int n = L.gs_ptr[k + 1] - L.gs_ptr[k];
    if (n == 0) continue;
    if constexpr (K == 6)
      AMG_KLAUNCH(c, gs_block_kernel<K, V, T>, (n + 7) / 8, 256, n,
                  (const int *)(L.gs_rows + L.gs_ptr[k]), (const int *)L.A.rowptr,
                  (const int *)L.A.colidx, vals, minv, b, x);
    else
      AMG_KLAUNCH(c, gs_colour_kernel<K, V, T>, (n + 7) / 8, 256, n,
                  (const int *)(L.gs_rows + L.gs_ptr[k]), (const int *)L.A.rowptr,
                  (const int *)L.A.colidx, vals, minv, b, x);
  }
  return cudaGetLastError();
}

template <int K>
static cudaError_t gs_sweep_prec(const Ctx *c, const Level &L, int prec, const void *b, void *x,
                                 bool forward) {
  if (prec == AMG_PREC_FP64)
    return gs_sweep_k<K, double, double>(c, L, L.A.v64, L.minv64, (const double *)b, (double *)x,
                                         forward);
  if (prec == AMG_PREC_FP32_VCYCLE)
    return gs_sweep_k<K, float, float>(c, L, L.A.v32, L.minv32, (const float *)b, (float *)x, forward);
  return gs_sweep_k<K, __nv_bfloat16, float>(c, L, L.A.v16, L.minv32, (const float *)b, (float *)x,
                                             forward);
}

cudaError_t launch_gs_sweep(const Ctx *c, const Level &L, int prec, const void *b, void *x,
                            bool forward) {
  if (L.A.n_rows == 0) return cudaSuccess;
  switch (L.k) {
    case 1: return gs_sweep_prec<1>(c, L, prec, b, x, forward);
    case 2: return gs_sweep_prec<2>(c, L, prec, b, x, forward);
    case 3: return gs_sweep_prec<3>(c, L, prec, b, x, forward);
    case 6: return gs_sweep_prec<6>(c, L, prec, b, x, forward);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace amg

using namespace amg;

extern "C" int amg_smoother_colouring(amg_ctx *h, int level, int32_t *colour_out, int32_t *n_colours) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  if (c->levels.empty() || c->smoother != AMG_SMOOTHER_HYBRID_GS) {
    c->err = "amg_smoother_colouring: no hierarchy with the hybrid Gauss-Seidel smoother";
    return AMG_ERR_STATE;
  }
  if (level < 0 || level + 1 >= (int)c->levels.size()) {
    c->err = "amg_smoother_colouring: level out of range";
    return AMG_ERR_ARG;
  }
  const Level &L = c->levels[level];
  if (n_colours) *n_colours = (int32_t)L.gs_ptr.size() - 1;
  if (colour_out) {
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(colour_out, L.gs_colour, (size_t)L.A.n_rows * sizeof(int),
                          cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      c->err = std::string("amg_smoother_colouring: ") + cudaGetErrorString(e);
      return AMG_ERR_CUDA;
    }
  }
  c->err.clear();
  return AMG_OK;
}
