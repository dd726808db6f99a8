// FP64 preconditioned conjugate gradients with one V-cycle as the
// preconditioner (Sec. 7), run entirely on the device: the iteration is a
// CUDA graph whose body (V-cycle + CG updates) sits in a device-side while
// node; the last kernel of every iteration decides whether to continue.
//
// All inner products use a fixed grid and a last-block reduction in index
// order, so every run is bit-reproducible.
#include "amg_internal.h"
#include "df_arith.cuh"

namespace amg {

constexpr int kRedThreads = 256;
// residual replacement of the double-float CG operator: every drop of r.r by
// this factor (r by 10^3) since the last replacement
constexpr double kReplaceDrop = 1e-6;

static int red_grid(const Ctx *c) { return c->num_sms * 8; }  // SpMV + dot kernels
// pure vector reductions: 8 blocks of 256 threads per SM keep enough loads
// in flight for HBM (2 per SM left r.z and the x / r update latency-bound)
static int vec_grid(const Ctx *c) { return c->num_sms * 8; }

// Block-wide sum of NV values; returns the sums in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][kRedThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double x = v[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[i][w] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = 0.0;
      for (int k = 0; k < kRedThreads / 32; ++k) s += sh[i][k];
      v[i] = s;
    }
  }
  __syncthreads();
}

// Store this block's partial sums; the block that arrives last sums all
// partials in index order and returns true (with the totals in tot[]).
template <int NV>
__device__ __forceinline__ bool last_block_total(double (&v)[NV], double *partials,
                                                 unsigned *counter, double (&tot)[NV]) {
  __shared__ bool last;
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) partials[(size_t)i * gridDim.x + blockIdx.x] = v[i];
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    s[i] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      s[i] += ((volatile double *)partials)[(size_t)i * gridDim.x + b];
  }
  block_sum<NV>(s);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) tot[i] = s[i];
    *counter = 0u;
  }
  return true;
}

// Warp-per-row SpMV core (same lane mapping as the V-cycle kernels) used
// by the CG: returns A_row . x in lanes 0..BR-1.
template <int BR>
__device__ __forceinline__ double row_dot(int row, const int *__restrict__ rowptr,
                                          const int *__restrict__ colidx,
                                          const double *__restrict__ vals,
                                          const double *__restrict__ x) {
  constexpr int NB = 32 / BR;
  const int lane = threadIdx.x & 31;
  const int bl = lane / BR, r = lane - bl * BR;
  double acc = 0.0;
  if (bl < NB) {
    const int e = rowptr[row + 1];
    for (int p = rowptr[row] + bl; p < e; p += NB) {
      const int c = __ldg(colidx + p);
      const double *v = vals + ((size_t)p * BR + r) * BR;
#pragma unroll
      for (int q = 0; q < BR; ++q) acc += __ldcs(v + q) * __ldg(x + (size_t)c * BR + q);
    }
  }
#pragma unroll
  for (int s = 1; s < NB; s <<= 1) {
    const double o = __shfl_down_sync(0xffffffffu, acc, s * BR);
    if (bl + s < NB) acc += o;
  }
  return acc;
}

// SELL-32 row product (thread per block row): y[0..BR) = A_row . x
template <int BR>
__device__ __forceinline__ void sell_row(int slice, int t, const int *__restrict__ sptr,
                                         const int *__restrict__ scol,
                                         const double *__restrict__ sv,
                                         const double *__restrict__ x, double (&y)[BR]) {
  constexpr int E = BR * BR;
#pragma unroll
  for (int r = 0; r < BR; ++r) y[r] = 0.0;
  const int j1 = sptr[slice + 1];
#pragma unroll 2
  for (int j = sptr[slice]; j < j1; ++j) {
    const int c = __ldg(scol + (size_t)j * 32 + t);
    const double *v = sv + (size_t)j * E * 32 + t;
    double xv[BR];
#pragma unroll
    for (int q = 0; q < BR; ++q) xv[q] = __ldg(x + (size_t)c * BR + q);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int q = 0; q < BR; ++q) y[r] += __ldcs(v + (r * BR + q) * 32) * xv[q];
  }
}

struct SellView {
  int n_rows, n_slices;
  const int *ptr, *col;
  const double *v;
};

template <int BR>
__global__ void __launch_bounds__(kRedThreads) pcg_init_sell_kernel(
    SellView A, const double *f, const double *x, double *r, PcgState *st, double *partials,
    unsigned *counter, cudaGraphConditionalHandle h, int in_graph) {
  pdl_enter();
  const int t = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  double v[2] = {0.0, 0.0};
  for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < A.n_slices; s += nw) {
    double ax[BR];
    sell_row<BR>(s, t, A.ptr, A.col, A.v, x, ax);
    const int row = s * 32 + t;
    if (row < A.n_rows) {
#pragma unroll
      for (int q = 0; q < BR; ++q) {
        const size_t i = (size_t)row * BR + q;
        const double ri = f[i] - ax[q];
        r[i] = ri;
        v[0] += ri * ri;
        v[1] += f[i] * f[i];
      }
    }
  }
  double tot[2];
  if (last_block_total<2>(v, partials, counter, tot) && threadIdx.x == 0) {
    st->rr = tot[0];
    st->rr_ref = tot[0];
    st->ff = tot[1];
    st->tol2 = st->rtol * st->rtol * tot[1];
    st->it = 0;
    st->status = 0;
    st->rho_old = 0.0;
    st->alpha = 0.0;
    st->beta = 0.0;
    const bool go = (tot[0] > st->tol2) && (st->maxit > 0) && isfinite(tot[0]);
    if (in_graph) cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}

// q = A p and the per-block partial of p.q (64-thread blocks, two slices
// each: fine-grained blocks balance the FP64 pipe load across SMs).  The
// partials are summed, in block order, by the consumer (update_xr).
constexpr int kSellThreads = 64;

template <int BR>
__global__ void __launch_bounds__(kSellThreads) pcg_spmv_dot_sell_kernel(SellView A,
                                                                        const double *p, double *q,
                                                                        double *partials) {
  pdl_enter();
  __shared__ double sh[kSellThreads / 32];
  const int t = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  double v = 0.0;
  if (s < A.n_slices) {
    double ap[BR];
    sell_row<BR>(s, t, A.ptr, A.col, A.v, p, ap);
    const int row = s * 32 + t;
    if (row < A.n_rows) {
#pragma unroll
      for (int c = 0; c < BR; ++c) {
        const size_t i = (size_t)row * BR + c;
        q[i] = ap[c];
        v += p[i] * ap[c];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (t == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int k = 0; k < kSellThreads / 32; ++k) b += sh[k];
    partials[blockIdx.x] = b;
  }
}

// ---------------------------------------------------------------------------
// Double-float CG operator (AMG_CG_DOUBLE_FLOAT): q = A_0 p with every FP64
// value held as an unevaluated sum hi + lo of two FP32 numbers, so that the
// products run on the FP32 pipe (on sm_103a the FP64 pipe retires about two
// FMA per clock per SM, below what HBM feeds for 2x2 / 3x3 FP64 blocks).
// Products are exact by Dekker's two-product (the FMA returns the rounding
// error of a*b), sums by Knuth's two-sum; the cross terms hi*lo' + lo*hi' are
// added to the low word, lo*lo' (below 2^-48 relative) is dropped.
// ---------------------------------------------------------------------------

struct SellDfView {
  int n_rows, n_slices, df_exp;
  const int *ptr, *col;
  const float2 *v;
};

// q = A_0 p in double-float arithmetic (p given as hi/lo pairs in pdf) and
// the per-block partial of p.q in FP64 (64-thread blocks, two slices each,
// thread per block row, as the FP64 kernel above).  Two slots per loop trip
// (48 registers with the compensated low word, 42 warps per SM) hold more
// loads in flight than one slot at 32 registers (64 warps per SM: 487
// against 393 us at 128^3 before the compensation), and forcing the
// compensated kernel into 40 registers cost more (445 against 405 us).
template <int BR>
__global__ void __launch_bounds__(kSellThreads) pcg_spmv_dot_sell_df_kernel(
    SellDfView A, const float2 *__restrict__ pdf, const double *__restrict__ p,
    double *__restrict__ q, double *__restrict__ partials) {
  pdl_enter();
  constexpr int E = BR * BR;
  __shared__ double sh_part[kSellThreads / 32];
  const int t = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  double v = 0.0;
  if (s < A.n_slices) {
    // per output row: hi the two-summed products, lo the low parts of the
    // blocks so far (each block's low parts summed on their own, then
    // two-summed into lo), lo2 lo's rounding errors.  Summing the low parts
    // of a whole row plainly would round at 2^-24 of their running total, an
    // error that rows with strong cancellation (coefficient jumps) amplify
    // beyond the 48-bit storage of the values.
    float hi[BR], lo[BR], lo2[BR];
#pragma unroll
    for (int r = 0; r < BR; ++r) hi[r] = lo[r] = lo2[r] = 0.f;
    const int j1 = A.ptr[s + 1];
#pragma unroll 2
    for (int j = A.ptr[s]; j < j1; ++j) {
      const int c = __ldg(A.col + (size_t)j * 32 + t);
      const float2 *a = A.v + (size_t)j * E * 32 + t;
      float2 xv[BR];
#pragma unroll
      for (int k = 0; k < BR; ++k) xv[k] = __ldg(pdf + (size_t)c * BR + k);
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        float lt = 0.f;
#pragma unroll
        for (int k = 0; k < BR; ++k) df_mac(hi[r], lt, __ldcs(a + (r * BR + k) * 32), xv[k]);
        two_sum_into(lo[r], lo2[r], lt);
      }
    }
    const int row = s * 32 + t;
    if (row < A.n_rows) {
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        const size_t i = (size_t)row * BR + r;
        const double qi = float_to_double_scaled(hi[r], A.df_exp) +
                          (float_to_double_scaled(lo[r], A.df_exp) +
                           float_to_double_scaled(lo2[r], A.df_exp));
        q[i] = qi;
        v += p[i] * qi;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (t == 0) sh_part[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int k = 0; k < kSellThreads / 32; ++k) b += sh_part[k];
    partials[blockIdx.x] = b;
  }
}

// r = f - A x ; rr = r.r ; ff = f.f ; decides whether the loop starts.
template <int BR>
__global__ void __launch_bounds__(kRedThreads) pcg_init_kernel(
    int n_rows, const int *rowptr, const int *colidx, const double *vals, const double *f,
    const double *x, double *r, PcgState *st, double *partials, unsigned *counter,
    cudaGraphConditionalHandle h, int in_graph) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  double v[2] = {0.0, 0.0};
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n_rows; row += nwarps) {
    const double ax = row_dot<BR>(row, rowptr, colidx, vals, x);
    if (lane < BR) {
      const size_t i = (size_t)row * BR + lane;
      const double ri = f[i] - ax;
      r[i] = ri;
      v[0] += ri * ri;
      v[1] += f[i] * f[i];
    }
  }
  double tot[2];
  if (last_block_total<2>(v, partials, counter, tot) && threadIdx.x == 0) {
    st->rr = tot[0];
    st->rr_ref = tot[0];
    st->ff = tot[1];
    st->tol2 = st->rtol * st->rtol * tot[1];
    st->it = 0;
    st->status = 0;
    st->rho_old = 0.0;
    st->alpha = 0.0;
    st->beta = 0.0;
    const bool go = (tot[0] > st->tol2) && (st->maxit > 0) && isfinite(tot[0]);
    if (in_graph) cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}

// rho = r.z (and r.z_old for the flexible beta); beta from the previous rho.
__global__ void __launch_bounds__(kRedThreads) pcg_dot_rz_kernel(size_t n, const double *r,
                                                                  const double *z,
                                                                  const double *zold,
                                                                  PcgState *st, double *partials,
                                                                  unsigned *counter) {
  pdl_enter();
  double v[2] = {0.0, 0.0};
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const bool flex = st->flexible != 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double ri = r[i];
    v[0] += ri * z[i];
    if (flex) v[1] += ri * zold[i];
  }
  double tot[2];
  if (last_block_total<2>(v, partials, counter, tot) && threadIdx.x == 0) {
    const double rho = tot[0];
    double beta = 0.0;
    if (st->it > 0) beta = (st->flexible ? (rho - tot[1]) : rho) / st->rho_old;
    st->rho = rho;
    st->beta = beta;
    st->rho_old = rho;
  }
}

// p = z + beta p ; z_old = z (flexible variant); with pdf, also p as
// double-float pairs for the double-float CG operator
__global__ void pcg_update_p_kernel(size_t n, const double *z, double *p, double *zold,
                                    const PcgState *st, float2 *pdf) {
  pdl_enter();
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double beta = st->beta;
  const double zi = z[i];
  const double pi = (st->it == 0) ? zi : zi + beta * p[i];
  p[i] = pi;
  if (pdf) pdf[i] = split_double_float(pi);
  if (st->flexible) zold[i] = zi;
}

// q = A p ; p.q (last-block total written to *pq_out)
template <int BR>
__global__ void __launch_bounds__(kRedThreads) pcg_spmv_dot_kernel(
    int n_rows, const int *rowptr, const int *colidx, const double *vals, const double *p,
    double *q, PcgState *st, double *partials, unsigned *counter, double *pq_out) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  double v[1] = {0.0};
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n_rows; row += nwarps) {
    const double ap = row_dot<BR>(row, rowptr, colidx, vals, p);
    if (lane < BR) {
      const size_t i = (size_t)row * BR + lane;
      q[i] = ap;
      v[0] += p[i] * ap;
    }
  }
  double tot[1];
  if (last_block_total<1>(v, partials, counter, tot) && threadIdx.x == 0) *pq_out = tot[0];
}

// p.q from the SpMV's per-block partials (one block, fixed order:
// deterministic, no atomics) and alpha = rho / p.q.
constexpr int kFinThreads = 1024;
__global__ void __launch_bounds__(kFinThreads) pcg_alpha_kernel(PcgState *st,
                                                                const double *pq_partials,
                                                                int n_pq) {
  pdl_enter();
  __shared__ double sh[kFinThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double a = 0.0;
  for (int b = threadIdx.x; b < n_pq; b += blockDim.x) a += pq_partials[b];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if (lane == 0) sh[w] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double pq = 0.0;
    for (int k = 0; k < kFinThreads / 32; ++k) pq += sh[k];
    const bool ok = (pq > 0.0) && isfinite(pq);
    st->pq = pq;
    st->alpha = ok ? st->rho / pq : 0.0;
    if (!ok) st->status = AMG_ERR_NOT_SPD;
  }
}

// x += alpha p ; r -= alpha q ; per-block partials of r.r for the guard.
__global__ void __launch_bounds__(kRedThreads) pcg_update_xr_kernel(
    size_t n, double *x, double *r, const double *p, const double *q, const PcgState *st,
    double *rr_partials) {
  pdl_enter();
  __shared__ double sh[kRedThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double alpha = st->alpha;
  double v = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    v += ri * ri;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int k = 0; k < kRedThreads / 32; ++k) b += sh[k];
    rr_partials[blockIdx.x] = b;
  }
}

// Last node of every iteration (one warp): sums the r.r partials (block
// order), counts the iteration and is the only place the loop condition is
// set inside the body.  An independent guard counter bounds the loop, and
// the counter of the last-block reductions is re-armed.
// With verify (the double-float CG operator) the recurrence residual drifts
// from the true one by the operator's rounding, most of it from the early
// iterations, whose terms are largest.  So the guard asks the replacement
// kernel that follows to recompute r = f - A x with the FP64 operator
// whenever r.r has dropped by kReplaceDrop since the last replacement, and
// when it meets the tolerance; the loop decision is then taken on the true
// residual.
__global__ void pcg_guard_kernel(PcgState *st, const double *rr_partials, int n_rr,
                                 unsigned *counter, cudaGraphConditionalHandle h, int in_graph,
                                 int verify) {
  pdl_enter();
  double v = 0.0;
  for (int b = threadIdx.x; b < n_rr; b += 32) v += rr_partials[b];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (threadIdx.x != 0) return;
  st->rr = v;
  st->it += 1;
  st->guard += 1;
  *counter = 0u;
  if (!isfinite(v) && st->status == 0) st->status = AMG_ERR_NOT_SPD;
  const bool ok = isfinite(v) && (st->status == 0);
  const bool more = (st->it < st->maxit) && (st->guard < st->maxit);
  const bool go = (v > st->tol2) && ok && more;
  st->replace = (verify && ok && (v <= st->tol2 || (more && v <= kReplaceDrop * st->rr_ref))) ? 1 : 0;
  if (in_graph && !st->replace) cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Residual replacement (van der Vorst and Ye's strategy, applied where the
// recurrence residual meets the tolerance): r = f - A_0 x with the FP64
// operator, r.r by a last-block total, and the loop decision on it.  Every
// block returns at once unless the guard asked for it.
template <int BR>
__global__ void __launch_bounds__(kRedThreads) pcg_replace_kernel(
    SellView A, const double *f, const double *x, double *r, PcgState *st, double *partials,
    unsigned *counter, cudaGraphConditionalHandle h, int in_graph) {
  pdl_enter();
  if (!st->replace) return;
  const int t = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  double v[1] = {0.0};
  for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < A.n_slices; s += nw) {
    double ax[BR];
    sell_row<BR>(s, t, A.ptr, A.col, A.v, x, ax);
    const int row = s * 32 + t;
    if (row < A.n_rows) {
#pragma unroll
      for (int q = 0; q < BR; ++q) {
        const size_t i = (size_t)row * BR + q;
        const double ri = f[i] - ax[q];
        r[i] = ri;
        v[0] += ri * ri;
      }
    }
  }
  double tot[1];
  if (last_block_total<1>(v, partials, counter, tot) && threadIdx.x == 0) {
    st->rr = tot[0];
    st->rr_ref = tot[0];
    st->replace = 0;
    st->replaced += 1;
    if (!isfinite(tot[0]) && st->status == 0) st->status = AMG_ERR_NOT_SPD;
    const bool go = (tot[0] > st->tol2) && isfinite(tot[0]) && (st->it < st->maxit) &&
                    (st->status == 0) && (st->guard < st->maxit);
    if (in_graph) cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}

cudaError_t pcg_alloc(Ctx *c) {
  free_pcg(c);
  const size_t n = (size_t)c->levels[0].A.n_rows * c->levels[0].k;
  const size_t bytes = (n ? n : 1) * sizeof(double);
  double **bufs[] = {&c->f, &c->x, &c->r, &c->z, &c->zold, &c->p, &c->q};
  for (double **b : bufs) {
    AMG_CUDA_TRY(dalloc((void **)b, bytes));
    AMG_CUDA_TRY(cudaMemsetAsync(*b, 0, bytes, c->stream));
  }
  if (c->levels[0].A.sdf) AMG_CUDA_TRY(dalloc((void **)&c->pdf, (n ? n : 1) * sizeof(float2)));
  AMG_CUDA_TRY(dalloc((void **)&c->st, sizeof(PcgState)));
  AMG_CUDA_TRY(cudaMallocHost((void **)&c->st_host, sizeof(PcgState)));
  const int n_slices = (c->levels[0].A.n_rows + 31) / 32;
  const size_t npart = 4 * (size_t)red_grid(c) + (size_t)(n_slices + 1) / 2 + 2 * (size_t)vec_grid(c);
  AMG_CUDA_TRY(dalloc((void **)&c->partials, npart * sizeof(double)));
  AMG_CUDA_TRY(dalloc((void **)&c->counter, sizeof(unsigned)));
  AMG_CUDA_TRY(cudaMemsetAsync(c->counter, 0, sizeof(unsigned), c->stream));
  return cudaStreamSynchronize(c->stream);
}

// The double-float CG operator runs where A_0 has its double-float copy
// (SELL-32, rows in order) and the context asks for it.
static bool use_double_float(const Ctx *c) {
  const DevBSR &A = c->levels[0].A;
  const bool want = c->cg_op == AMG_CG_DOUBLE_FLOAT ||
                    (c->cg_op == AMG_CG_AUTO && c->precision != AMG_PREC_FP64);
  return want && A.sdf && A.sell_ptr && !A.sell_perm && c->pdf;
}

static SellView sell_view(const DevBSR &A) {
  return SellView{A.n_rows, A.n_slices, A.sell_ptr, A.sell_col, A.s64};
}

template <int BR>
static cudaError_t launch_init(Ctx *c, cudaGraphConditionalHandle h, int in_graph) {
  const Level &L0 = c->levels[0];
  if (L0.A.sell_ptr && !L0.A.sell_perm)
    AMG_KLAUNCH(c, pcg_init_sell_kernel<BR>, red_grid(c), kRedThreads, 
        sell_view(L0.A), c->f, c->x, c->r, c->st, c->partials, c->counter, h, in_graph);
  else
    AMG_KLAUNCH(c, pcg_init_kernel<BR>, red_grid(c), kRedThreads, 
        L0.A.n_rows, L0.A.rowptr, L0.A.colidx, L0.A.v64, c->f, c->x, c->r, c->st, c->partials,
        c->counter, h, in_graph);
  return cudaGetLastError();
}

template <int BR>
static cudaError_t launch_body(Ctx *c, cudaGraphConditionalHandle h, int in_graph) {
  const Level &L0 = c->levels[0];
  const size_t n = (size_t)L0.A.n_rows * BR;
  const int g = red_grid(c), gv = vec_grid(c);
  // partial buffers: [0, 4g) last-block reductions, then p.q, then r.r
  double *pq_part = c->partials + 4 * (size_t)g;
  int n_pq;
  AMG_CUDA_TRY(vcycle_launch(c, c->r, c->z));
  AMG_KLAUNCH(c, pcg_dot_rz_kernel, gv, kRedThreads, n, c->r, c->z, c->zold, c->st, c->partials,
                                                       c->counter);
  const bool df = use_double_float(c);
  AMG_KLAUNCH(c, pcg_update_p_kernel, (unsigned)((n + 255) / 256), 256, n, c->z, c->p, c->zold,
                                                                          c->st, df ? c->pdf : nullptr);
  if (df) {
    n_pq = (L0.A.n_slices + 1) / 2;
    const SellDfView A{L0.A.n_rows, L0.A.n_slices, L0.A.df_exp, L0.A.sell_ptr, L0.A.sell_col,
                       L0.A.sdf};
    AMG_KLAUNCH(c, pcg_spmv_dot_sell_df_kernel<BR>, n_pq, kSellThreads, A, (const float2 *)c->pdf,
                (const double *)c->p, c->q, pq_part);
  } else if (L0.A.sell_ptr && !L0.A.sell_perm) {
    n_pq = (L0.A.n_slices + 1) / 2;
    AMG_KLAUNCH(c, pcg_spmv_dot_sell_kernel<BR>, n_pq, kSellThreads, sell_view(L0.A), c->p,
                                                                       c->q, pq_part);
  } else {
    // warp-per-row SpMV + dot with a last-block total: its block partial
    // array holds the single total (n_pq = 1)
    n_pq = 1;
    AMG_KLAUNCH(c, pcg_spmv_dot_kernel<BR>, g, kRedThreads, L0.A.n_rows, L0.A.rowptr,
                                                              L0.A.colidx, L0.A.v64, c->p, c->q,
                                                              c->st, c->partials, c->counter,
                                                              pq_part);
  }
  double *rr_part = pq_part + (size_t)(L0.A.n_slices + 1) / 2 + 1;
  AMG_KLAUNCH(c, pcg_alpha_kernel, 1, kFinThreads, c->st, pq_part, n_pq);
  AMG_KLAUNCH(c, pcg_update_xr_kernel, gv, kRedThreads, n, c->x, c->r, c->p, c->q, c->st,
                                                          rr_part);
  AMG_KLAUNCH(c, pcg_guard_kernel, 1, 32, c->st, rr_part, gv, c->counter, h, in_graph, df ? 1 : 0);
  if (df)
    AMG_KLAUNCH(c, pcg_replace_kernel<BR>, g, kRedThreads, sell_view(L0.A), (const double *)c->f,
                (const double *)c->x, c->r, c->st, c->partials, c->counter, h, in_graph);
  return cudaGetLastError();
}

static cudaError_t capture_init(Ctx *c, int k, cudaGraphConditionalHandle h) {
  return k == 1 ? launch_init<1>(c, h, 1) : k == 2 ? launch_init<2>(c, h, 1)
         : k == 3 ? launch_init<3>(c, h, 1) : cudaErrorInvalidValue;
}

static cudaError_t capture_body(Ctx *c, int k, cudaGraphConditionalHandle h) {
  return k == 1 ? launch_body<1>(c, h, 1) : k == 2 ? launch_body<2>(c, h, 1)
         : k == 3 ? launch_body<3>(c, h, 1) : cudaErrorInvalidValue;
}

static bool host_go(const PcgState &s) {
  return s.rr > s.tol2 && isfinite(s.rr) && s.it < s.maxit && s.status == 0 && s.guard < s.maxit;
}

// Host-driven PCG: the same kernels launched one by one, the loop condition
// read back after every iteration (no graph; used for per-kernel profiling).
cudaError_t pcg_host_loop(Ctx *c) {
  const int k = c->levels[0].k;
  if (k != 1 && k != 2 && k != 3) return cudaErrorInvalidValue;
  AMG_CUDA_TRY(k == 1 ? launch_init<1>(c, 0, 0) : k == 2 ? launch_init<2>(c, 0, 0) : launch_init<3>(c, 0, 0));
  AMG_CUDA_TRY(cudaMemcpyAsync(c->st_host, c->st, sizeof(PcgState), cudaMemcpyDeviceToHost,
                               c->stream));
  AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  bool go = c->st_host->rr > c->st_host->tol2 && c->st_host->maxit > 0 && isfinite(c->st_host->rr);
  while (go) {
    AMG_CUDA_TRY(k == 1 ? launch_body<1>(c, 0, 0) : k == 2 ? launch_body<2>(c, 0, 0)
                        : launch_body<3>(c, 0, 0));
    AMG_CUDA_TRY(cudaMemcpyAsync(c->st_host, c->st, sizeof(PcgState), cudaMemcpyDeviceToHost,
                                 c->stream));
    AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
    go = host_go(*c->st_host);
  }
  return cudaSuccess;
}

cudaError_t pcg_build_graph(Ctx *c) {
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  if (c->graph_def) {
    cudaGraphDestroy(c->graph_def);
    c->graph_def = nullptr;
  }
  const int k = c->levels[0].k;
  cudaGraph_t g = nullptr;
  AMG_CUDA_TRY(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  AMG_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
  AMG_CUDA_TRY(cudaStreamBeginCaptureToGraph(c->stream, g, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
  cudaError_t e = capture_init(c, k, h);
  cudaGraph_t cap = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(c->stream, &cap);
  if (e != cudaSuccess) return e;
  if (e2 != cudaSuccess) return e2;
  size_t nn = 0;
  AMG_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn), sinks;
  AMG_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &nn));
  for (auto nd : nodes) {
    size_t nd_out = 0;
    AMG_CUDA_TRY(cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nd_out));
    if (nd_out == 0) sinks.push_back(nd);
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  AMG_CUDA_TRY(cudaGraphAddNode(&cnode, g, sinks.data(), nullptr, sinks.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  AMG_CUDA_TRY(cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
  e = capture_body(c, k, h);
  e2 = cudaStreamEndCapture(c->stream, &body);
  if (e != cudaSuccess) return e;
  if (e2 != cudaSuccess) return e2;
  AMG_CUDA_TRY(cudaGraphInstantiate(&c->graph, g, 0));
  c->graph_def = g;
  return cudaSuccess;
}

}  // namespace amg

using namespace amg;

extern "C" int amg_pcg_launches(const amg_ctx *h, int32_t *per_iteration, int32_t *fixed) {
  if (!h) return AMG_ERR_ARG;
  const Ctx *c = &h->c;
  if (c->levels.empty()) return AMG_ERR_STATE;
  const int nl = (int)c->levels.size();
  int vc = 5 * (nl - 1) + 1;                              // V-cycle kernels
  if (nl == 1 && c->precision != AMG_PREC_FP64) vc += 2;  // FP64 <-> FP32 casts
  if (c->smoother == AMG_SMOOTHER_HYBRID_GS && nl > 1) {
    // per level: one kernel per colour class and sweep instead of the two
    // Jacobi kernels (the zero start and the result copy are memory nodes)
    vc = 1;
    for (int l = 0; l + 1 < nl; ++l) vc += 3 + 2 * ((int)c->levels[l].gs_ptr.size() - 1);
    if (c->precision != AMG_PREC_FP64) vc += 2;  // FP64 <-> FP32 casts of level 0
  }
  // r.z, p update, q = A p with p.q, alpha, x / r update with r.r, loop
  // decision (and the residual replacement kernel with the double-float
  // operator, which returns at once except at convergence)
  if (per_iteration) *per_iteration = vc + 6 + (use_double_float(c) ? 1 : 0);
  if (fixed) *fixed = 1;
  return AMG_OK;
}

namespace amg {

// Mean device time (us) of reps launches of fn on c's stream, after one warm
// launch, by CUDA events on that stream.
template <typename F>
static cudaError_t time_kernel(Ctx *c, int reps, F fn, double *us) {
  cudaEvent_t e0, e1;
  AMG_CUDA_TRY(cudaEventCreate(&e0));
  AMG_CUDA_TRY(cudaEventCreate(&e1));
  cudaError_t e = fn();
  if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = fn();
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *us = 1e3 * ms / reps;
  return e;
}

template <int BR>
static cudaError_t profile_pcg_k(Ctx *c, int reps, double *us, double *bytes) {
  const Level &L0 = c->levels[0];
  const DevBSR &A = L0.A;
  const size_t n = (size_t)A.n_rows * BR;
  const int g = red_grid(c), gv = vec_grid(c);
  double *pq_part = c->partials + 4 * (size_t)g;
  double *rr_part = pq_part + (size_t)(A.n_slices + 1) / 2 + 1;
  const bool df = use_double_float(c);
  const bool sell = A.sell_ptr && !A.sell_perm;
  const int flex = c->precision != AMG_PREC_FP64 ? 1 : 0;
  const int n_pq = sell ? (A.n_slices + 1) / 2 : 1;
  // a consistent CG state: iteration 1 (beta used), flexible as in a solve
  PcgState h = *c->st_host;
  h.it = 1;
  h.maxit = 1 << 30;
  h.guard = 0;
  h.status = 0;
  h.flexible = flex;
  h.beta = 0.5;
  h.rho_old = 1.0;
  h.alpha = 0.5;
  h.tol2 = 0.0;
  AMG_CUDA_TRY(cudaMemcpyAsync(c->st, &h, sizeof(PcgState), cudaMemcpyHostToDevice, c->stream));
  AMG_CUDA_TRY(cudaMemcpyAsync(c->z, c->r, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  const double N8 = 8.0 * (double)n;
  AMG_CUDA_TRY(time_kernel(c, reps, [&] {
    launch_k(c, pcg_dot_rz_kernel, gv, kRedThreads, n, (const double *)c->r, (const double *)c->z,
             (const double *)c->zold, c->st, c->partials, c->counter);
    return cudaGetLastError(); }, &us[0]));
  bytes[0] = N8 * (2 + flex);
  AMG_CUDA_TRY(time_kernel(c, reps, [&] {
    launch_k(c, pcg_update_p_kernel, (unsigned)((n + 255) / 256), 256, n, (const double *)c->z, c->p,
             c->zold, (const PcgState *)c->st, df ? c->pdf : nullptr);
    return cudaGetLastError(); }, &us[1]));
  bytes[1] = N8 * (3 + flex + (df ? 1 : 0));
  const double abytes = (double)A.nnzb * (BR * BR * 8.0 + 4.0) + 4.0 * (A.n_rows + 1);
  AMG_CUDA_TRY(time_kernel(c, reps, [&] {
    if (df) {
      const SellDfView V{A.n_rows, A.n_slices, A.df_exp, A.sell_ptr, A.sell_col, A.sdf};
      launch_k(c, pcg_spmv_dot_sell_df_kernel<BR>, n_pq, kSellThreads, V, (const float2 *)c->pdf,
               (const double *)c->p, c->q, pq_part);
    } else if (sell) {
      launch_k(c, pcg_spmv_dot_sell_kernel<BR>, n_pq, kSellThreads, sell_view(A),
               (const double *)c->p, c->q, pq_part);
    } else {
      launch_k(c, pcg_spmv_dot_kernel<BR>, g, kRedThreads, A.n_rows, (const int *)A.rowptr,
               (const int *)A.colidx, (const double *)A.v64, (const double *)c->p, c->q, c->st,
               c->partials, c->counter, pq_part);
    }
    return cudaGetLastError(); }, &us[2]));
  bytes[2] = abytes + N8 * (df ? 3 : 2);
  AMG_CUDA_TRY(time_kernel(c, reps, [&] {
    launch_k(c, pcg_alpha_kernel, 1, kFinThreads, c->st, (const double *)pq_part, n_pq);
    return cudaGetLastError(); }, &us[3]));
  bytes[3] = 8.0 * n_pq;
  AMG_CUDA_TRY(time_kernel(c, reps, [&] {
    launch_k(c, pcg_update_xr_kernel, gv, kRedThreads, n, c->x, c->r, (const double *)c->p,
             (const double *)c->q, (const PcgState *)c->st, rr_part);
    return cudaGetLastError(); }, &us[4]));
  bytes[4] = N8 * 6;
  AMG_CUDA_TRY(time_kernel(c, reps, [&] {
    launch_k(c, pcg_guard_kernel, 1, 32, c->st, (const double *)rr_part, gv, c->counter,
             (cudaGraphConditionalHandle)0, 0, 0);
    return cudaGetLastError(); }, &us[5]));
  bytes[5] = 8.0 * gv;
  return cudaStreamSynchronize(c->stream);
}

__global__ void split_vector_kernel(size_t n, const double *__restrict__ p, float2 *__restrict__ pdf) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pdf[i] = split_double_float(p[i]);
}

// q = A_0 p by the CG operator's kernel (p.q partials to the reduction scratch).
template <int BR>
static cudaError_t cg_operator_k(Ctx *c, const double *p, double *q) {
  const DevBSR &A = c->levels[0].A;
  const size_t n = (size_t)A.n_rows * BR;
  const int g = red_grid(c);
  double *pq_part = c->partials + 4 * (size_t)g;
  if (use_double_float(c)) {
    split_vector_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, p, c->pdf);
    AMG_CUDA_TRY(cudaGetLastError());
    const SellDfView V{A.n_rows, A.n_slices, A.df_exp, A.sell_ptr, A.sell_col, A.sdf};
    AMG_KLAUNCH(c, pcg_spmv_dot_sell_df_kernel<BR>, (A.n_slices + 1) / 2, kSellThreads, V,
                (const float2 *)c->pdf, p, q, pq_part);
  } else if (A.sell_ptr && !A.sell_perm) {
    AMG_KLAUNCH(c, pcg_spmv_dot_sell_kernel<BR>, (A.n_slices + 1) / 2, kSellThreads, sell_view(A),
                p, q, pq_part);
  } else {
    AMG_KLAUNCH(c, pcg_spmv_dot_kernel<BR>, g, kRedThreads, A.n_rows, (const int *)A.rowptr,
                (const int *)A.colidx, (const double *)A.v64, p, q, c->st, c->partials, c->counter,
                pq_part);
  }
  return cudaStreamSynchronize(c->stream);
}

}  // namespace amg

extern "C" int amg_cg_operator(amg_ctx *h, const double *p, double *q) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  if (c->levels.empty() || !c->st) {
    c->err = "amg_cg_operator: no hierarchy uploaded";
    return AMG_ERR_STATE;
  }
  const int k = c->levels[0].k;
  if (!p || !q || (k != 1 && k != 2 && k != 3)) {
    c->err = "amg_cg_operator: NULL vector or A_0 block size other than 1, 2 or 3";
    return AMG_ERR_ARG;
  }
  cudaError_t e = cudaSetDevice(c->device);
  if (e == cudaSuccess)
    e = k == 1 ? cg_operator_k<1>(c, p, q) : k == 2 ? cg_operator_k<2>(c, p, q) : cg_operator_k<3>(c, p, q);
  if (e != cudaSuccess) {
    c->err = std::string("amg_cg_operator: ") + cudaGetErrorString(e);
    return AMG_ERR_CUDA;
  }
  c->err.clear();
  return AMG_OK;
}

extern "C" int amg_profile_pcg(amg_ctx *h, int reps, int32_t *kind, double *us, double *bytes,
                               int max_entries, int32_t *n_entries) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  if (reps < 1 || max_entries < 0) {
    c->err = "amg_profile_pcg: reps < 1 or max_entries < 0";
    return AMG_ERR_ARG;
  }
  if (c->levels.empty() || !c->st) {
    c->err = "amg_profile_pcg: no hierarchy uploaded";
    return AMG_ERR_STATE;
  }
  const int k = c->levels[0].k;
  if (k != 1 && k != 2 && k != 3) {
    c->err = "amg_profile_pcg: A_0 block size";
    return AMG_ERR_ARG;
  }
  cudaError_t e = cudaSetDevice(c->device);
  double t[6] = {0}, b[6] = {0};
  if (e == cudaSuccess)
    e = k == 1 ? profile_pcg_k<1>(c, reps, t, b)
        : k == 2 ? profile_pcg_k<2>(c, reps, t, b) : profile_pcg_k<3>(c, reps, t, b);
  if (e != cudaSuccess) {
    c->err = std::string("amg_profile_pcg: ") + cudaGetErrorString(e);
    return AMG_ERR_CUDA;
  }
  for (int i = 0; i < 6 && i < max_entries; ++i) {
    if (kind) kind[i] = i;
    if (us) us[i] = t[i];
    if (bytes) bytes[i] = b[i];
  }
  if (n_entries) *n_entries = 6;
  c->err.clear();
  return AMG_OK;
}
