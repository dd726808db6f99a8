// Galerkin coarse operator A_{l+1} = P_l^T A_l P_l (Sec. 6: the coarse
// matrix of the auxiliary smoothed prolongation; Sec. 3 Algorithm tg) as two
// row-wise segmented SpGEMMs on the device:  AP = A_l P_l, then
// A_{l+1} = R_l (AP) with the explicit transpose R_l = P_l^T.
//
// Each product runs in three passes, one warp per output block row:
//   symbolic count: candidate block columns of the row are marked in a
//       per-warp shared-memory bitmap (window over [min, max] column), the
//       number of distinct columns is the popcount;
//   fill: same bitmap, columns emitted in ascending order (every
//       structurally reached block is kept, numerically zero or not);
//   numeric: the terms L_ij * R_jq are added in the order of j (sequential
//       per warp, deterministic), the (q, element) pairs of one j in
//       parallel; positions come from a binary search in the sorted row.
#include "amg_internal.h"

namespace amg {

constexpr int kWarpsPerBlock = 4;
constexpr int kBitmapWords = 1024;  // per warp: 32768 columns per window

__global__ void scan_exclusive_kernel(int n, int *__restrict__ a, int *__restrict__ total) {
  // one block: in-place exclusive scan of a[0..n) ; writes the sum to *total
  __shared__ int sh[1024];
  const int t = threadIdx.x;
  const int chunk = (n + blockDim.x - 1) / blockDim.x;
  const int s = t * chunk, e = min(n, s + chunk);
  int local = 0;
  for (int i = s; i < e; ++i) local += a[i];
  sh[t] = local;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    int v = (t >= off) ? sh[t - off] : 0;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  int run = (t == 0) ? 0 : sh[t - 1];
  for (int i = s; i < e; ++i) {
    const int v = a[i];
    a[i] = run;
    run += v;
  }
  if (t == blockDim.x - 1) *total = sh[t];
}

// Pass 1/2: FILL = false counts distinct columns per row, FILL = true writes
// them in ascending order to out_col[out_rp[row] ...].
template <bool FILL>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) spgemm_symbolic(
    int n_rows, const int *__restrict__ lrp, const int *__restrict__ lci, const int *__restrict__ rrp,
    const int *__restrict__ rci, int *__restrict__ count, const int *__restrict__ out_rp,
    int *__restrict__ out_col) {
  __shared__ unsigned bitmap[kWarpsPerBlock][kBitmapWords];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned *bm = bitmap[w];
  const int row = blockIdx.x * kWarpsPerBlock + w;
  if (row >= n_rows) return;
  const int s = lrp[row], e = lrp[row + 1];
  int lo = 0x7fffffff, hi = -1;
  for (int p = s + lane; p < e; p += 32) {
    const int j = lci[p];
    if (rrp[j + 1] > rrp[j]) {
      lo = min(lo, rci[rrp[j]]);
      hi = max(hi, rci[rrp[j + 1] - 1]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  int written = 0;
  for (int base = lo; base <= hi; base += 32 * kBitmapWords) {
    for (int i = lane; i < kBitmapWords; i += 32) bm[i] = 0u;
    __syncwarp();
    const int top = base + 32 * kBitmapWords;
    for (int p = s + lane; p < e; p += 32) {
      const int j = lci[p];
      for (int q = rrp[j]; q < rrp[j + 1]; ++q) {
        const int col = rci[q];
        if (col >= base && col < top) {
          const int off = col - base;
          atomicOr(&bm[off >> 5], 1u << (off & 31));
        }
      }
    }
    __syncwarp();
    // words this window can hold
    const int nwords = min(kBitmapWords, (hi - base) / 32 + 1);
    if (!FILL) {
      int c = 0;
      for (int i = lane; i < nwords; i += 32) c += __popc(bm[i]);
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      written += c;
    } else {
      // ordered emission: 32 consecutive words per step, prefix of popcounts
      for (int i0 = 0; i0 < nwords; i0 += 32) {
        const int i = i0 + lane;
        const unsigned word = (i < nwords) ? bm[i] : 0u;
        const int c = __popc(word);
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        int pos = out_rp[row] + written + incl - c;
        unsigned wv = word;
        while (wv) {
          const int bit = __ffs(wv) - 1;
          out_col[pos++] = base + i * 32 + bit;
          wv &= wv - 1;
        }
        written += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    __syncwarp();
  }
  if (!FILL && lane == 0) count[row] = written;
}

// Pass 3: C_row += sum_j L_ij R_j,: ; C values zero on entry.
template <int BLR, int BLC, int BRC>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) spgemm_numeric(
    int n_rows, const int *__restrict__ lrp, const int *__restrict__ lci,
    const double *__restrict__ lv, const int *__restrict__ rrp, const int *__restrict__ rci,
    const double *__restrict__ rv, const int *__restrict__ crp, const int *__restrict__ cci,
    double *__restrict__ cv) {
  constexpr int EL = BLR * BRC;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int row = blockIdx.x * kWarpsPerBlock + w;
  if (row >= n_rows) return;
  const int cs = crp[row], ce = crp[row + 1];
  for (int p = lrp[row]; p < lrp[row + 1]; ++p) {
    const int j = lci[p];
    const double *lb = lv + (size_t)p * BLR * BLC;
    const int q0 = rrp[j], nq = rrp[j + 1] - q0;
    for (int t = lane; t < nq * EL; t += 32) {
      const int qq = t / EL, el = t - qq * EL;
      const int r = el / BRC, cc = el - r * BRC;
      const int q = q0 + qq;
      const int col = rci[q];
      // lower_bound of col in the sorted output row
      int lo = cs, hi = ce;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cci[mid] < col) lo = mid + 1; else hi = mid;
      }
      const double *rb = rv + (size_t)q * BLC * BRC;
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < BLC; ++m) acc += lb[r * BLC + m] * rb[m * BRC + cc];
      if (lo < ce && cci[lo] == col) cv[(size_t)lo * EL + el] += acc;
    }
    __syncwarp();
  }
}

cudaError_t scan_exclusive(Ctx *c, int n, int *a, int *total_dev) {
  scan_exclusive_kernel<<<1, 1024, 0, c->stream>>>(n, a, total_dev);
  return cudaGetLastError();
}

template <int BLR, int BLC, int BRC>
static cudaError_t spgemm(Ctx *c, const DevBSR &L, const DevBSR &R, DevBSR &C) {
  C.n_rows = L.n_rows;
  C.n_cols = R.n_cols;
  C.br = BLR;
  C.bc = BRC;
  const int n = L.n_rows;
  AMG_CUDA_TRY(dalloc((void **)&C.rowptr, (size_t)(n + 1) * sizeof(int)));
  int *total = nullptr;
  AMG_CUDA_TRY(dalloc((void **)&total, sizeof(int)));
  AMG_CUDA_TRY(cudaMemsetAsync(C.rowptr, 0, (size_t)(n + 1) * sizeof(int), c->stream));
  const int g = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (n > 0)
    spgemm_symbolic<false><<<g, 32 * kWarpsPerBlock, 0, c->stream>>>(
        n, L.rowptr, L.colidx, R.rowptr, R.colidx, C.rowptr, nullptr, nullptr);
  AMG_CUDA_TRY(cudaGetLastError());
  scan_exclusive_kernel<<<1, 1024, 0, c->stream>>>(n + 1, C.rowptr, total);
  AMG_CUDA_TRY(cudaGetLastError());
  int nnz = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&nnz, total, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  dfree(total);
  C.nnzb = nnz;
  AMG_CUDA_TRY(dalloc((void **)&C.colidx, (size_t)(nnz > 0 ? nnz : 1) * sizeof(int)));
  AMG_CUDA_TRY(dalloc((void **)&C.v64, (size_t)(nnz > 0 ? nnz : 1) * BLR * BRC * sizeof(double)));
  AMG_CUDA_TRY(cudaMemsetAsync(C.v64, 0, (size_t)nnz * BLR * BRC * sizeof(double), c->stream));
  if (n > 0) {
    spgemm_symbolic<true><<<g, 32 * kWarpsPerBlock, 0, c->stream>>>(
        n, L.rowptr, L.colidx, R.rowptr, R.colidx, nullptr, C.rowptr, C.colidx);
    AMG_CUDA_TRY(cudaGetLastError());
    spgemm_numeric<BLR, BLC, BRC><<<g, 32 * kWarpsPerBlock, 0, c->stream>>>(
        n, L.rowptr, L.colidx, L.v64, R.rowptr, R.colidx, R.v64, C.rowptr, C.colidx, C.v64);
    AMG_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

static cudaError_t spgemm_dispatch(Ctx *c, const DevBSR &L, const DevBSR &R, DevBSR &C) {
  if (L.bc != R.br) return cudaErrorInvalidValue;
#define AMG_SPGEMM_CASE(a, b, d) \
  if (L.br == a && L.bc == b && R.bc == d) return spgemm<a, b, d>(c, L, R, C);
  AMG_SPGEMM_CASE(1, 1, 1)
  AMG_SPGEMM_CASE(2, 2, 3)
  AMG_SPGEMM_CASE(3, 2, 3)
  AMG_SPGEMM_CASE(3, 3, 6)
  AMG_SPGEMM_CASE(6, 3, 6)
  AMG_SPGEMM_CASE(3, 3, 3)
  AMG_SPGEMM_CASE(6, 6, 6)
#undef AMG_SPGEMM_CASE
  return cudaErrorInvalidValue;
}

cudaError_t galerkin_device(Ctx *c, int level) {
  Level &F = c->levels[level];
  Level &Cl = c->levels[level + 1];
  DevBSR AP;
  cudaError_t e = spgemm_dispatch(c, F.A, F.P, AP);
  if (e == cudaSuccess) {
    free_bsr(Cl.A);
    e = spgemm_dispatch(c, F.R, AP, Cl.A);
  }
  cudaStreamSynchronize(c->stream);
  free_bsr(AP);
  if (e == cudaSuccess) Cl.k = Cl.A.br;
  return e;
}

}  // namespace amg
