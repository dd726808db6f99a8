// Block-l1 hybrid Gauss-Seidel smoother (AMG_SMOOTHER_HYBRID_GS), the other
// form of the l1 smoothers the paper's Sec. 7 cites, for one device: the
// block rows of a level are coloured so that rows of one colour never couple
// (greedy in smallest-last order: each takes the smallest colour none of its
// already coloured neighbours holds), and a sweep visits the colour classes
// in order; every row of a class computes x_v <- x_v + M_v^+ (b - A x)_v with
// the values the classes before it wrote.  A class is what a processor's
// block is to the hybrid smoother of the multi-process setting: its rows are
// updated together, and the l1 term of M_v covers couplings inside the class
// (none for a distance-1 colouring, so M_v = A_vv).  The pre-smoothing sweep
// runs the classes forward, the post-smoothing sweep backward, which keeps
// the V-cycle symmetric.
#include <algorithm>
#include <type_traits>

#include "amg_internal.h"
#include "bsr_loads.cuh"

namespace amg {

// Host greedy colouring of the block graph of A_level in smallest-last
// order (Matula and Beck: repeatedly remove a remaining row of least degree,
// ties by the smallest index; colour in the reverse of the removals, each
// row the smallest colour no already coloured neighbour holds), uploaded
// with the rows grouped by colour (ascending row index inside a class).
// Against rows in index order it halves level 0's classes (8 to 4 on the 3D
// meshes) and cuts the coarse levels' by about a fifth.
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
  int n_col = 0;
  const std::vector<int> colour = amgsetup::smallest_last_colouring(n, rp.data(), ci.data(), &n_col);
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

// Gather of the colour-ordered SELL-32 values: entry (slot, element e, lane)
// takes element e of block map[slot * 32 + lane] (0 where the map is -1).
template <typename V>
__global__ void gs_sell_gather_kernel(size_t n, int E, const int *__restrict__ map,
                                      const V *__restrict__ src, V *__restrict__ dst) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t lane = i & 31, rest = i >> 5;
  const size_t e = rest % (size_t)E, slot = rest / (size_t)E;
  const int blk = map[slot * 32 + lane];
  dst[i] = blk >= 0 ? src[(size_t)blk * E + e] : (V)0.0f;
}

cudaError_t gs_build_sell(Ctx *c, int level, int prec) {
  Level &L = c->levels[level];
  const DevBSR &A = L.A;
  const int n = A.n_rows, E = A.br * A.bc, nc = (int)L.gs_ptr.size() - 1;
  if (n == 0 || nc < 1) return cudaSuccess;
  std::vector<int> rp(n + 1), rows(n);
  AMG_CUDA_TRY(cudaMemcpyAsync(rp.data(), A.rowptr, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost,
                               c->stream));
  AMG_CUDA_TRY(cudaMemcpyAsync(rows.data(), L.gs_rows, n * sizeof(int), cudaMemcpyDeviceToHost,
                               c->stream));
  std::vector<int> ci(A.nnzb > 0 ? A.nnzb : 1);
  if (A.nnzb)
    AMG_CUDA_TRY(cudaMemcpyAsync(ci.data(), A.colidx, A.nnzb * sizeof(int), cudaMemcpyDeviceToHost,
                                 c->stream));
  AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  // slices of 32 rows of one class, rows in the class's (ascending) order
  std::vector<int> slice_ptr(nc + 1, 0), perm, sptr(1, 0);
  for (int k = 0; k < nc; ++k) {
    const int r0 = L.gs_ptr[k], r1 = L.gs_ptr[k + 1];
    for (int q = r0; q < r1; q += 32) {
      int w = 0;
      for (int t = 0; t < 32; ++t) {
        const int row = q + t < r1 ? rows[q + t] : n;
        perm.push_back(row);
        if (row < n) w = std::max(w, rp[row + 1] - rp[row]);
      }
      sptr.push_back(sptr.back() + w);
    }
    slice_ptr[k + 1] = (int)sptr.size() - 1;
  }
  const int ns = (int)sptr.size() - 1;
  const size_t slots = (size_t)sptr.back();
  std::vector<int> col(slots * 32 > 0 ? slots * 32 : 1, 0), map(slots * 32 > 0 ? slots * 32 : 1, -1);
  for (int s = 0; s < ns; ++s)
    for (int t = 0; t < 32; ++t) {
      const int row = perm[(size_t)s * 32 + t];
      if (row >= n) continue;
      const int len = rp[row + 1] - rp[row];
      for (int j = 0; j < len; ++j) {
        const size_t at = ((size_t)sptr[s] + j) * 32 + t;
        col[at] = ci[rp[row] + j];
        map[at] = rp[row] + j;
      }
    }
  // padding slots of a row point at its own first column (value 0)
  for (int s = 0; s < ns; ++s)
    for (int t = 0; t < 32; ++t) {
      const int row = perm[(size_t)s * 32 + t];
      const int len = row < n ? rp[row + 1] - rp[row] : 0;
      const int c0 = row < n && len > 0 ? ci[rp[row]] : 0;
      for (int j = len; j < sptr[s + 1] - sptr[s]; ++j) col[((size_t)sptr[s] + j) * 32 + t] = c0;
    }
  for (void *q : {(void *)L.gs_sell_ptr, (void *)L.gs_sell_col, (void *)L.gs_sell_perm, L.gs_sell_vals})
    dfree(q);
  L.gs_sell_ptr = L.gs_sell_col = L.gs_sell_perm = nullptr;
  L.gs_sell_vals = nullptr;
  L.gs_slice_ptr.clear();
  int *d_map = nullptr;
  const size_t wv = prec == AMG_PREC_FP64 ? 8 : prec == AMG_PREC_FP32_VCYCLE ? 4 : 2;
  AMG_CUDA_TRY(dalloc((void **)&L.gs_sell_ptr, sptr.size() * sizeof(int)));
  AMG_CUDA_TRY(dalloc((void **)&L.gs_sell_col, col.size() * sizeof(int)));
  AMG_CUDA_TRY(dalloc((void **)&L.gs_sell_perm, perm.size() * sizeof(int)));
  AMG_CUDA_TRY(dalloc((void **)&d_map, map.size() * sizeof(int)));
  AMG_CUDA_TRY(dalloc(&L.gs_sell_vals, (slots > 0 ? slots : 1) * 32 * E * wv));
  AMG_CUDA_TRY(cudaMemcpyAsync(L.gs_sell_ptr, sptr.data(), sptr.size() * sizeof(int),
                               cudaMemcpyHostToDevice, c->stream));
  AMG_CUDA_TRY(cudaMemcpyAsync(L.gs_sell_col, col.data(), col.size() * sizeof(int),
                               cudaMemcpyHostToDevice, c->stream));
  AMG_CUDA_TRY(cudaMemcpyAsync(L.gs_sell_perm, perm.data(), perm.size() * sizeof(int),
                               cudaMemcpyHostToDevice, c->stream));
  AMG_CUDA_TRY(cudaMemcpyAsync(d_map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice,
                               c->stream));
  const size_t total = slots * 32 * (size_t)E;
  if (total) {
    const unsigned g = (unsigned)((total + 255) / 256);
    if (prec == AMG_PREC_FP64)
      gs_sell_gather_kernel<double><<<g, 256, 0, c->stream>>>(total, E, d_map, A.v64, (double *)L.gs_sell_vals);
    else if (prec == AMG_PREC_FP32_VCYCLE)
      gs_sell_gather_kernel<float><<<g, 256, 0, c->stream>>>(total, E, d_map, A.v32, (float *)L.gs_sell_vals);
    else
      gs_sell_gather_kernel<__nv_bfloat16><<<g, 256, 0, c->stream>>>(total, E, d_map, A.v16,
                                                                      (__nv_bfloat16 *)L.gs_sell_vals);
    AMG_CUDA_TRY(cudaGetLastError());
  }
  AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  dfree(d_map);
  L.gs_slice_ptr = slice_ptr;
  L.gs_sell_prec = prec;
  return cudaSuccess;
}

// One colour class from the colour-ordered SELL-32 copy: thread per row
// (slice lane), the row's blocks four slots at a time (column indices, then
// their x gathers, then the values), x in place as in the warp kernels.
template <int K, typename V, typename T>
__global__ void __launch_bounds__(64) gs_sell_kernel(int n_rows, int s0, int s1,
                                                     const int *__restrict__ sell_ptr,
                                                     const int *__restrict__ sell_col,
                                                     const int *__restrict__ perm,
                                                     const V *__restrict__ vals,
                                                     const T *__restrict__ minv,
                                                     const T *__restrict__ b, T *x) {
  pdl_enter();
  constexpr int E = K * K;
  const int slice = s0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (slice >= s1) return;  // whole warp
  const int t = threadIdx.x & 31;
  const int row = __ldg(perm + slice * 32 + t);
  const int j0 = __ldg(sell_ptr + slice), j1 = __ldg(sell_ptr + slice + 1);
  T acc[K];
#pragma unroll
  for (int r = 0; r < K; ++r) acc[r] = 0;
  constexpr int U = 4;
  for (int j = j0; j < j1; j += U) {
    int cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) cc[u] = (j + u < j1) ? __ldg(sell_col + (size_t)(j + u) * 32 + t) : 0;
    T xv[U][K];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j + u < j1) {
        ldn_cached<K>(x + (size_t)cc[u] * K, xv[u]);
      } else {
#pragma unroll
        for (int q = 0; q < K; ++q) xv[u][q] = 0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j + u < j1) {
        const V *v = vals + (size_t)(j + u) * E * 32 + t;
#pragma unroll
        for (int r = 0; r < K; ++r)
#pragma unroll
          for (int q = 0; q < K; ++q) acc[r] += (T)lds(v + (r * K + q) * 32) * xv[u][q];
      }
    }
  }
  if (row >= n_rows) return;
  const size_t o = (size_t)row * K;
  T res[K], upd[K];
#pragma unroll
  for (int r = 0; r < K; ++r) res[r] = b[o + r] - acc[r];
#pragma unroll
  for (int r = 0; r < K; ++r) {
    upd[r] = 0;
#pragma unroll
    for (int q = 0; q < K; ++q) upd[r] += minv[(o + r) * K + q] * res[q];
  }
#pragma unroll
  for (int r = 0; r < K; ++r) x[o + r] += upd[r];
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
  // the colour-ordered SELL-32 copy (thread per row), where the level has one
  // in this precision, for the classes with rows enough to fill the GPU
  // with thread-per-row warps (16 per SM; every class under
  // AMG_LAYOUT_SELL_SHORT_ROWS); smaller classes run a warp per row
  bool sell = false;
  if constexpr (K <= 3) {
    const int want = std::is_same<V, double>::value ? AMG_PREC_FP64
                     : std::is_same<V, float>::value ? AMG_PREC_FP32_VCYCLE : AMG_PREC_BF16_STORAGE;
    sell = L.gs_sell_vals && L.gs_sell_prec == want;
  }
  const int sell_min_rows = c->layout_policy == AMG_LAYOUT_SELL_SHORT_ROWS ? 0 : 32 * 16 * c->num_sms;
  for (int s = 0; s < nc; ++s) {
    const int k = forward ? s : nc - 1 - s;
    const int n = L.gs_ptr[k + 1] - L.gs_ptr[k];
    if (n == 0) continue;
    if (sell && n >= sell_min_rows) {
      const int s0 = L.gs_slice_ptr[k], s1 = L.gs_slice_ptr[k + 1];
      AMG_KLAUNCH(c, gs_sell_kernel<K, V, T>, (s1 - s0 + 1) / 2, 64, L.A.n_rows, s0, s1,
                  (const int *)L.gs_sell_ptr, (const int *)L.gs_sell_col, (const int *)L.gs_sell_perm,
                  (const V *)L.gs_sell_vals, minv, b, x);
      continue;
    }
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
