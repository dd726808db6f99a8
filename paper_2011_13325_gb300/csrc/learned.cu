// Learned smoother of the finest level (an extension: the paper has no
// learned component).  A per-vertex MLP 13 -> 64 -> 64 -> 6 maps features of
// a vertex (its diagonal block, the sum of its finest-level edge matrices'
// displacement part c^{ij} t t^T of Thm. deng_elast, its degree) to a lower
// triangular factor L; the smoother block is B_v = (L L^T + 1e-6 I) / tr A_vv,
// SPD by construction, damped by omega = 4 / (3 * 1.05 * lambda) with lambda
// from 30 Lanczos steps on B A (the smoother x += omega B r is convergent iff
// omega lambda_max(BA) < 2).  Training targets are the vv blocks of the
// inverses of the patch matrices A_{N(v),N(v)} (v and its neighbours), times
// tr A_vv, computed here by a dense FP64 Cholesky per vertex.  The network
// keeps FP32 master weights (Adam) and computes with a BF16 copy of them,
// FP32 activations and FP32 accumulation.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "amg_internal.h"

namespace amg {

constexpr int MLP_IN = 13, MLP_H = 64, MLP_OUT = 6;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H,
              OFF_B2 = OFF_W2 + MLP_H * MLP_H, OFF_W3 = OFF_B2 + MLP_H,
              OFF_B3 = OFF_W3 + MLP_OUT * MLP_H, MLP_PARAMS = OFF_B3 + MLP_OUT;
static_assert(MLP_PARAMS == 5446, "parameter count");
constexpr float LEARN_EPS = 1e-6f;
constexpr double DEGREE_SCALE = 14.0;
constexpr int TILE = 32;       // samples per tile of the MLP kernels
constexpr int MLP_THREADS = 256;
constexpr int MAX_PATCH = 16;  // vertices of a patch (degree <= 15)
constexpr int PN = 3 * MAX_PATCH, PLD = PN + 1;
constexpr int LANCZOS_STEPS = 30;
constexpr double LANCZOS_SAFETY = 1.05, OMEGA_NUM = 4.0 / 3.0;

// ---------------------------------------------------------------------------
// features: A_vv (6 unique) / tr, sum_j c^{vj} t t^T (6 unique) / (tr * mean
// |t|^2), degree / 14.  Unique order (0,0) (1,1) (2,2) (0,1) (0,2) (1,2).
// ---------------------------------------------------------------------------
__global__ void features_kernel(int n, const int *__restrict__ rowptr, const int *__restrict__ colidx,
                                const double *__restrict__ vals, const double *__restrict__ coords,
                                float *__restrict__ X, double *__restrict__ tr_out, int *__restrict__ err) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  double D[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double l2 = 0.0;
  int deg = 0;
  bool diag = false;
  const double x0 = coords[3 * (size_t)v], x1 = coords[3 * (size_t)v + 1], x2 = coords[3 * (size_t)v + 2];
  for (int q = rowptr[v]; q < rowptr[v + 1]; ++q) {
    const int j = colidx[q];
    const double *a = vals + (size_t)q * 9;
    if (j == v) {
      for (int e = 0; e < 9; ++e) D[e] = a[e];
      diag = true;
      continue;
    }
    double c = 0.0;
    for (int e = 0; e < 9; ++e) c += fabs(a[e]);
    c /= 9.0;
    const double t[3] = {coords[3 * (size_t)j] - x0, coords[3 * (size_t)j + 1] - x1,
                         coords[3 * (size_t)j + 2] - x2};
    for (int r = 0; r < 3; ++r)
      for (int s = 0; s < 3; ++s) S[r * 3 + s] += c * t[r] * t[s];
    l2 += t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    ++deg;
  }
  const double tr = D[0] + D[4] + D[8];
  if (!diag || !(tr > 0.0)) atomicAdd(err, 1);
  const double hs = deg ? l2 / deg : 1.0;
  const int uq[6] = {0, 4, 8, 1, 2, 5};
  float *xo = X + (size_t)v * MLP_IN;
  for (int k = 0; k < 6; ++k) {
    xo[k] = (float)(D[uq[k]] / tr);
    xo[6 + k] = (float)(S[uq[k]] / (tr * hs));
  }
  xo[12] = (float)(deg / DEGREE_SCALE);
  if (tr_out) tr_out[v] = tr;
}

// ---------------------------------------------------------------------------
// patch targets: one warp per vertex v; the patch matrix (neighbours in row
// order, v last) in shared memory, Cholesky A = L L^T in place; with v last
// [A^{-1}]_vv = (L_vv L_vv^T)^{-1}.  Output T_v * tr A_vv (row-major 3x3).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(64) patch_target_kernel(int n, const int *__restrict__ rowptr,
                                                          const int *__restrict__ colidx,
                                                          const double *__restrict__ vals,
                                                          float *__restrict__ T32, double *__restrict__ T64,
                                                          int *__restrict__ err) {
  __shared__ double Dsh[2][PN * PLD];
  __shared__ int nbs[2][MAX_PATCH];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = blockIdx.x * 2 + warp;
  if (v >= n) return;  // whole warp
  double *D = Dsh[warp];
  int *nb = nbs[warp];
  const int s = rowptr[v], e = rowptr[v + 1];
  int deg = 0;
  for (int q = s; q < e; ++q) deg += colidx[q] != v;
  const int m = deg + 1;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  if (m > MAX_PATCH) {
    if (lane == 0) {
      atomicAdd(err, 1);
      for (int k = 0; k < 9; ++k) {
        if (T64) T64[(size_t)v * 9 + k] = nan;
        if (T32) T32[(size_t)v * 9 + k] = (float)nan;
      }
    }
    return;
  }
  if (lane == 0) {
    int a = 0;
    for (int q = s; q < e; ++q)
      if (colidx[q] != v) nb[a++] = colidx[q];
    nb[a] = v;
  }
  const int N = 3 * m;
  for (int i = lane; i < N * PLD; i += 32) D[i] = 0.0;
  __syncwarp();
  for (int a = 0; a < m; ++a) {
    const int r = nb[a];
    for (int q = rowptr[r] + lane; q < rowptr[r + 1]; q += 32) {
      const int c = colidx[q];
      int b = -1;
      for (int t = 0; t < m; ++t)
        if (nb[t] == c) b = t;
      if (b < 0) continue;
      const double *blk = vals + (size_t)q * 9;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) D[(3 * a + i) * PLD + 3 * b + j] = blk[i * 3 + j];
    }
  }
  __syncwarp();
  const double trv = D[(N - 3) * PLD + N - 3] + D[(N - 2) * PLD + N - 2] + D[(N - 1) * PLD + N - 1];
  bool ok = true;
  for (int j = 0; j < N; ++j) {
    const double djj = D[j * PLD + j];
    if (!(djj > 0.0)) {  // same value on every lane: uniform exit
      ok = false;
      break;
    }
    const double piv = sqrt(djj);
    __syncwarp();
    for (int i = j + 1 + lane; i < N; i += 32) D[i * PLD + j] /= piv;
    __syncwarp();
    if (lane == 0) D[j * PLD + j] = piv;
    for (int i = j + 1 + lane; i < N; i += 32) {
      const double lij = D[i * PLD + j];
      for (int k = j + 1; k <= i; ++k) D[i * PLD + k] -= lij * D[k * PLD + j];
    }
    __syncwarp();
  }
  if (lane != 0) return;
  double T[9];
  if (ok) {
    const int o = N - 3;
    const double l00 = D[o * PLD + o], l10 = D[(o + 1) * PLD + o], l11 = D[(o + 1) * PLD + o + 1],
                 l20 = D[(o + 2) * PLD + o], l21 = D[(o + 2) * PLD + o + 1],
                 l22 = D[(o + 2) * PLD + o + 2];
    // Li = L_vv^{-1} (lower), T = Li^T Li
    const double i00 = 1.0 / l00, i11 = 1.0 / l11, i22 = 1.0 / l22;
    const double i10 = -l10 * i00 * i11, i21 = -l21 * i11 * i22;
    const double i20 = -(l20 * i00 + l21 * i10) * i22;
    const double Li[9] = {i00, 0.0, 0.0, i10, i11, 0.0, i20, i21, i22};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double t = 0.0;
        for (int k = 0; k < 3; ++k) t += Li[k * 3 + a] * Li[k * 3 + b];
        T[a * 3 + b] = t * trv;
      }
  } else {
    atomicAdd(err, 1);
    for (int k = 0; k < 9; ++k) T[k] = nan;
  }
  for (int k = 0; k < 9; ++k) {
    if (T64) T64[(size_t)v * 9 + k] = T[k];
    if (T32) T32[(size_t)v * 9 + k] = (float)T[k];
  }
}

// ---------------------------------------------------------------------------
// MLP: tiles of 32 samples, 256 threads, weights (BF16 in memory) in shared
// memory as FP32 (W2 rows padded to 65 floats: conflict-free row and column
// reads).  MODE 0: forward (outputs L, or the normalised blocks); MODE 1:
// forward + backward, per-block gradient partials.
// ---------------------------------------------------------------------------
struct MlpShared {
  float w1[MLP_H * MLP_IN], b1[MLP_H], w2[MLP_H * 65], b2[MLP_H], w3[MLP_OUT * MLP_H], b3[MLP_OUT];
  float xs[TILE * MLP_IN], ha[TILE * 65], hb[TILE * 65], o[TILE * MLP_OUT];
  double loss[MLP_THREADS / 32];
};

__device__ __forceinline__ void tril_from(const float *o, float L[9]) {
  L[0] = o[0]; L[1] = 0.f; L[2] = 0.f;
  L[3] = o[1]; L[4] = o[2]; L[5] = 0.f;
  L[6] = o[3]; L[7] = o[4]; L[8] = o[5];
}

template <int MODE>
__global__ void __launch_bounds__(MLP_THREADS) mlp_kernel(
    long n, const int *__restrict__ perm, const float *__restrict__ X, const float *__restrict__ Tgt,
    const __nv_bfloat16 *__restrict__ w16, float scale, float *__restrict__ out6,
    const double *__restrict__ tr, double *__restrict__ Bn, float *__restrict__ partials,
    double *__restrict__ lpart) {
  __shared__ MlpShared sm;
  const int t = threadIdx.x;
  for (int p = t; p < MLP_PARAMS; p += MLP_THREADS) {
    const float w = __bfloat162float(w16[p]);
    if (p < OFF_B1) sm.w1[p - OFF_W1] = w;
    else if (p < OFF_W2) sm.b1[p - OFF_B1] = w;
    else if (p < OFF_B2) {
      const int q = p - OFF_W2;
      sm.w2[(q >> 6) * 65 + (q & 63)] = w;
    } else if (p < OFF_W3) sm.b2[p - OFF_B2] = w;
    else if (p < OFF_B3) sm.w3[p - OFF_W3] = w;
    else sm.b3[p - OFF_B3] = w;
  }
  // gradient accumulators of the parameters this thread owns
  float gw1[4] = {0.f, 0.f, 0.f, 0.f}, gw2[16], gw3[2] = {0.f, 0.f}, gb1 = 0.f, gb2 = 0.f, gb3 = 0.f;
#pragma unroll
  for (int k = 0; k < 16; ++k) gw2[k] = 0.f;
  double lacc = 0.0;
  __syncthreads();
  const long tiles = (n + TILE - 1) / TILE;
  for (long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long base = tile * TILE;
    const int cnt = (int)min((long)TILE, n - base);
    for (int i = t; i < TILE * MLP_IN; i += MLP_THREADS) {
      const int s = i / MLP_IN, f = i - s * MLP_IN;
      float xv = 0.f;
      if (s < cnt) {
        const long id = perm ? (long)perm[base + s] : base + s;
        xv = X[id * MLP_IN + f];
      }
      sm.xs[i] = xv;
    }
    __syncthreads();
    for (int i = t; i < TILE * MLP_H; i += MLP_THREADS) {
      const int s = i >> 6, h = i & 63;
      float a = sm.b1[h];
#pragma unroll
      for (int f = 0; f < MLP_IN; ++f) a += sm.w1[h * MLP_IN + f] * sm.xs[s * MLP_IN + f];
      sm.ha[s * 65 + h] = fmaxf(a, 0.f);
    }
    __syncthreads();
    for (int i = t; i < TILE * MLP_H; i += MLP_THREADS) {
      const int s = i >> 6, h = i & 63;
      float a = sm.b2[h];
#pragma unroll 16
      for (int g = 0; g < MLP_H; ++g) a += sm.w2[h * 65 + g] * sm.ha[s * 65 + g];
      sm.hb[s * 65 + h] = fmaxf(a, 0.f);
    }
    __syncthreads();
    if (t < TILE * MLP_OUT) {
      const int s = t / MLP_OUT, o = t - s * MLP_OUT;
      float a = sm.b3[o];
#pragma unroll 16
      for (int h = 0; h < MLP_H; ++h) a += sm.w3[o * MLP_H + h] * sm.hb[s * 65 + h];
      sm.o[t] = a;
    }
    __syncthreads();
    if (MODE == 0) {
      if (t < cnt) {
        const long id = base + t;
        const float *o = sm.o + t * MLP_OUT;
        if (out6)
          for (int k = 0; k < MLP_OUT; ++k) out6[id * MLP_OUT + k] = o[k];
        if (Bn) {
          float L[9];
          tril_from(o, L);
          const double inv = 1.0 / tr[id];
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              float sab = (a == b) ? LEARN_EPS : 0.f;
              for (int c = 0; c < 3; ++c) sab += L[a * 3 + c] * L[b * 3 + c];
              Bn[id * 9 + a * 3 + b] = (double)sab * inv;
            }
        }
      }
      __syncthreads();
      continue;
    }
    // loss and d loss / d outputs (thread per sample)
    if (t < TILE) {
      float dO[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      double ls = 0.0;
      if (t < cnt) {
        const long id = perm ? (long)perm[base + t] : base + t;
        float L[9], dS[9];
        tril_from(sm.o + t * MLP_OUT, L);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            float sab = (a == b) ? LEARN_EPS : 0.f;
            for (int c = 0; c < 3; ++c) sab += L[a * 3 + c] * L[b * 3 + c];
            const float g = sab - Tgt[id * 9 + a * 3 + b];
            ls += (double)g * g;
            dS[a * 3 + b] = 2.f * g * scale;
          }
        // d/dL_ab of sum dS_cd S_cd = ((dS + dS^T) L)_ab, lower entries only
        const int ta[6] = {0, 1, 1, 2, 2, 2}, tb[6] = {0, 0, 1, 0, 1, 2};
        for (int k = 0; k < 6; ++k) {
          float d = 0.f;
          for (int c = 0; c < 3; ++c) d += (dS[ta[k] * 3 + c] + dS[c * 3 + ta[k]]) * L[c * 3 + tb[k]];
          dO[k] = d;
        }
      }
      for (int k = 0; k < 6; ++k) sm.o[t * MLP_OUT + k] = dO[k];
      for (int o = 16; o > 0; o >>= 1) ls += __shfl_down_sync(0xffffffffu, ls, o);
      if (t == 0) lacc += ls;
    }
    __syncthreads();
    // W3, b3
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int i = t + r * MLP_THREADS;
      if (i < MLP_OUT * MLP_H) {
        const int o = i >> 6, h = i & 63;
        float a = 0.f;
        for (int s = 0; s < TILE; ++s) a += sm.o[s * MLP_OUT + o] * sm.hb[s * 65 + h];
        gw3[r] += a;
      }
    }
    if (t < MLP_OUT)
      for (int s = 0; s < TILE; ++s) gb3 += sm.o[s * MLP_OUT + t];
    __syncthreads();
    // dH2 (in place of H2): ReLU mask from the stored activation
    for (int i = t; i < TILE * MLP_H; i += MLP_THREADS) {
      const int s = i >> 6, h = i & 63;
      float d = 0.f;
#pragma unroll
      for (int o = 0; o < MLP_OUT; ++o) d += sm.w3[o * MLP_H + h] * sm.o[s * MLP_OUT + o];
      sm.hb[s * 65 + h] = sm.hb[s * 65 + h] > 0.f ? d : 0.f;
    }
    __syncthreads();
    {  // W2 rows h = hq*16 + k, column g; b2
      const int g = t & 63, hq = t >> 6;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int h = hq * 16 + k;
        float a = 0.f;
        for (int s = 0; s < TILE; ++s) a += sm.hb[s * 65 + h] * sm.ha[s * 65 + g];
        gw2[k] += a;
      }
      if (t < MLP_H)
        for (int s = 0; s < TILE; ++s) gb2 += sm.hb[s * 65 + t];
    }
    __syncthreads();
    // dH1 (in place of H1)
    for (int i = t; i < TILE * MLP_H; i += MLP_THREADS) {
      const int s = i >> 6, g = i & 63;
      float d = 0.f;
#pragma unroll 16
      for (int h = 0; h < MLP_H; ++h) d += sm.w2[h * 65 + g] * sm.hb[s * 65 + h];
      sm.ha[s * 65 + g] = sm.ha[s * 65 + g] > 0.f ? d : 0.f;
    }
    __syncthreads();
    // W1, b1
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = t + r * MLP_THREADS;
      if (i < MLP_H * MLP_IN) {
        const int g = i / MLP_IN, f = i - g * MLP_IN;
        float a = 0.f;
        for (int s = 0; s < TILE; ++s) a += sm.ha[s * 65 + g] * sm.xs[s * MLP_IN + f];
        gw1[r] += a;
      }
    }
    if (t < MLP_H)
      for (int s = 0; s < TILE; ++s) gb1 += sm.ha[s * 65 + t];
    __syncthreads();
  }
  if (MODE == 0) return;
  float *P = partials + (size_t)blockIdx.x * MLP_PARAMS;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = t + r * MLP_THREADS;
    if (i < MLP_H * MLP_IN) P[OFF_W1 + i] = gw1[r];
  }
  if (t < MLP_H) P[OFF_B1 + t] = gb1;
  {
    const int g = t & 63, hq = t >> 6;
#pragma unroll
    for (int k = 0; k < 16; ++k) P[OFF_W2 + (hq * 16 + k) * MLP_H + g] = gw2[k];
  }
  if (t < MLP_H) P[OFF_B2 + t] = gb2;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int i = t + r * MLP_THREADS;
    if (i < MLP_OUT * MLP_H) P[OFF_W3 + i] = gw3[r];
  }
  if (t < MLP_OUT) P[OFF_B3 + t] = gb3;
  if (t == 0) lpart[blockIdx.x] = lacc;
}

// Sum of the per-block partials in block order (deterministic), then either
// the plain gradient or one Adam step on the FP32 master weights and their
// BF16 working copy.
__global__ void mlp_reduce_kernel(int nblk, const float *__restrict__ partials,
                                  const double *__restrict__ lpart, float loss_scale,
                                  float *__restrict__ grad, double *__restrict__ loss_out, int adam,
                                  float *__restrict__ master, __nv_bfloat16 *__restrict__ w16,
                                  float *__restrict__ m1, float *__restrict__ m2, float lr, float bc1,
                                  float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss_out) {
    double l = 0.0;
    for (int b = 0; b < nblk; ++b) l += lpart[b];
    *loss_out = l * loss_scale;
  }
  if (p >= MLP_PARAMS) return;
  float g = 0.f;
  for (int b = 0; b < nblk; ++b) g += partials[(size_t)b * MLP_PARAMS + p];
  if (grad) grad[p] = g;
  if (!adam) return;
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  const float a = beta1 * m1[p] + (1.f - beta1) * g;
  const float b = beta2 * m2[p] + (1.f - beta2) * g * g;
  m1[p] = a;
  m2[p] = b;
  const float w = master[p] - lr * (a / bc1) / (sqrtf(b / bc2) + eps);
  master[p] = w;
  w16[p] = __float2bfloat16_rn(w);
}

__global__ void to_bf16_kernel(int n, const float *__restrict__ src, __nv_bfloat16 *__restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// ---------------------------------------------------------------------------
// Lanczos helpers and installation of the damped blocks
// ---------------------------------------------------------------------------
__global__ void dot_partial_kernel(size_t n, const double *__restrict__ a, const double *__restrict__ b,
                                   double *__restrict__ part) {
  __shared__ double sh[8];
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// w = w - alpha v - beta v_old
__global__ void lanczos_update_kernel(size_t n, double *__restrict__ w, const double *__restrict__ v,
                                      const double *__restrict__ vo, double alpha, double beta) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] -= alpha * v[i] + beta * vo[i];
}

__global__ void scale_kernel(size_t n, double *__restrict__ x, double s) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= s;
}

__global__ void install_kernel(size_t n, const double *__restrict__ Bn, double w, double *__restrict__ m64,
                               float *__restrict__ m32) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = w * Bn[i];
  m64[i] = v;
  if (m32) m32[i] = (float)v;
}

// splitmix64: the generator of the initial weights, the sample orders and
// the Lanczos start vector (host)
static uint64_t splitmix64(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static double uniform01(uint64_t &s) { return ((splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
static double normal01(uint64_t &s) {  // Box-Muller
  const double u1 = uniform01(s), u2 = uniform01(s);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// largest eigenvalue of the symmetric tridiagonal (a, b) by bisection on
// the Sturm sequence counts
static double tridiag_max_eig(const std::vector<double> &a, const std::vector<double> &b) {
  const int n = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < n ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  auto count_below = [&](double x) {  // eigenvalues < x
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < n; ++i) {
      d = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0.0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * fmax(fabs(hi), fabs(lo)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= n) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace amg

using namespace amg;

struct amg_mlp {
  int device = 0;
  float *master = nullptr, *m1 = nullptr, *m2 = nullptr, *partials = nullptr, *grad = nullptr;
  __nv_bfloat16 *w16 = nullptr;
  double *lpart = nullptr, *loss = nullptr;
  int *perm = nullptr;
  long perm_n = 0;
  int max_blocks = 0;
  long steps = 0;
  cudaStream_t stream = nullptr;
  std::string err;
};

static int mfail(amg_mlp *m, int code, const std::string &msg) {
  m->err = msg;
  return code;
}

#define MCUDA(m, expr, where)                                                                  \
  do {                                                                                         \
    cudaError_t _e = (expr);                                                                   \
    if (_e != cudaSuccess) return mfail(m, AMG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(_e)); \
  } while (0)

static void mlp_free(amg_mlp *m) {
  dfree(m->master);
  dfree(m->m1);
  dfree(m->m2);
  dfree(m->partials);
  dfree(m->grad);
  dfree(m->w16);
  dfree(m->lpart);
  dfree(m->loss);
  dfree(m->perm);
  if (m->stream) cudaStreamDestroy(m->stream);
}

// master -> BF16 working copy, Adam state cleared
static cudaError_t mlp_reset(amg_mlp *m) {
  to_bf16_kernel<<<(MLP_PARAMS + 255) / 256, 256, 0, m->stream>>>(MLP_PARAMS, m->master, m->w16);
  AMG_CUDA_TRY(cudaGetLastError());
  AMG_CUDA_TRY(cudaMemsetAsync(m->m1, 0, MLP_PARAMS * sizeof(float), m->stream));
  AMG_CUDA_TRY(cudaMemsetAsync(m->m2, 0, MLP_PARAMS * sizeof(float), m->stream));
  m->steps = 0;
  return cudaStreamSynchronize(m->stream);
}

// forward + backward over n samples (in perm order if perm), gradient of
// scale * sum of sample losses; optionally one Adam step
static cudaError_t mlp_step(amg_mlp *m, long n, const int *perm, const float *X, const float *T, float scale,
                            float *grad, double *loss_out, bool adam, float lr) {
  const long tiles = (n + TILE - 1) / TILE;
  const int nblk = (int)(tiles < m->max_blocks ? tiles : m->max_blocks);
  if (nblk < 1) return cudaErrorInvalidValue;
  mlp_kernel<1><<<nblk, MLP_THREADS, 0, m->stream>>>(n, perm, X, T, m->w16, scale, nullptr, nullptr,
                                                     nullptr, m->partials, m->lpart);
  AMG_CUDA_TRY(cudaGetLastError());
  float bc1 = 1.f, bc2 = 1.f;
  if (adam) {
    m->steps += 1;
    bc1 = 1.f - powf(0.9f, (float)m->steps);
    bc2 = 1.f - powf(0.999f, (float)m->steps);
  }
  mlp_reduce_kernel<<<(MLP_PARAMS + 255) / 256, 256, 0, m->stream>>>(
      nblk, m->partials, m->lpart, scale, grad, loss_out, adam ? 1 : 0, m->master, m->w16, m->m1, m->m2,
      lr, bc1, bc2);
  return cudaGetLastError();
}

extern "C" {

int amg_mlp_create(amg_mlp **out, int device, uint64_t seed) {
  if (!out) return AMG_ERR_ARG;
  *out = nullptr;
  amg_mlp *m = new amg_mlp();
  m->device = device;
  int sms = 0;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  m->max_blocks = 4 * (sms > 0 ? sms : 1);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = dalloc((void **)&m->master, MLP_PARAMS * sizeof(float));
  if (e == cudaSuccess) e = dalloc((void **)&m->m1, MLP_PARAMS * sizeof(float));
  if (e == cudaSuccess) e = dalloc((void **)&m->m2, MLP_PARAMS * sizeof(float));
  if (e == cudaSuccess) e = dalloc((void **)&m->grad, MLP_PARAMS * sizeof(float));
  if (e == cudaSuccess) e = dalloc((void **)&m->w16, MLP_PARAMS * sizeof(__nv_bfloat16));
  if (e == cudaSuccess)
    e = dalloc((void **)&m->partials, (size_t)m->max_blocks * MLP_PARAMS * sizeof(float));
  if (e == cudaSuccess) e = dalloc((void **)&m->lpart, (size_t)m->max_blocks * sizeof(double));
  if (e == cudaSuccess) e = dalloc((void **)&m->loss, sizeof(double));
  if (e == cudaSuccess) {
    // He-normal weights, zero biases
    std::vector<float> p(MLP_PARAMS, 0.f);
    uint64_t s = seed;
    for (int i = 0; i < MLP_H * MLP_IN; ++i) p[OFF_W1 + i] = (float)(normal01(s) * sqrt(2.0 / MLP_IN));
    for (int i = 0; i < MLP_H * MLP_H; ++i) p[OFF_W2 + i] = (float)(normal01(s) * sqrt(2.0 / MLP_H));
    for (int i = 0; i < MLP_OUT * MLP_H; ++i) p[OFF_W3 + i] = (float)(normal01(s) * sqrt(2.0 / MLP_H));
    e = cudaMemcpy(m->master, p.data(), MLP_PARAMS * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = mlp_reset(m);
  if (e != cudaSuccess) {
    mlp_free(m);
    delete m;
    return AMG_ERR_CUDA;
  }
  *out = m;
  return AMG_OK;
}

void amg_mlp_destroy(amg_mlp *m) {
  if (!m) return;
  cudaSetDevice(m->device);
  if (m->stream) cudaStreamSynchronize(m->stream);
  mlp_free(m);
  delete m;
}

const char *amg_mlp_last_error(const amg_mlp *m) { return m ? m->err.c_str() : "NULL network"; }

int amg_mlp_n_params(void) { return MLP_PARAMS; }

int amg_mlp_get_params(amg_mlp *m, float *params, int working) {
  if (!m || !params) return AMG_ERR_ARG;
  MCUDA(m, cudaSetDevice(m->device), "cudaSetDevice");
  if (!working) {
    MCUDA(m, cudaMemcpy(params, m->master, MLP_PARAMS * sizeof(float), cudaMemcpyDeviceToHost), "params");
    return AMG_OK;
  }
  std::vector<__nv_bfloat16> w(MLP_PARAMS);
  MCUDA(m, cudaMemcpy(w.data(), m->w16, MLP_PARAMS * sizeof(__nv_bfloat16), cudaMemcpyDeviceToHost),
        "params");
  for (int i = 0; i < MLP_PARAMS; ++i) {
    uint16_t u;
    memcpy(&u, &w[i], 2);
    const uint32_t bits = (uint32_t)u << 16;
    memcpy(&params[i], &bits, 4);
  }
  return AMG_OK;
}

int amg_mlp_set_params(amg_mlp *m, const float *params) {
  if (!m || !params) return AMG_ERR_ARG;
  MCUDA(m, cudaSetDevice(m->device), "cudaSetDevice");
  MCUDA(m, cudaMemcpy(m->master, params, MLP_PARAMS * sizeof(float), cudaMemcpyHostToDevice), "params");
  MCUDA(m, mlp_reset(m), "params");
  m->err.clear();
  return AMG_OK;
}

int amg_mlp_loss_grad(amg_mlp *m, const float *X_dev, const float *T_dev, int64_t n, double *loss,
                      float *grad_host) {
  if (!m || !X_dev || !T_dev || n < 1) return AMG_ERR_ARG;
  MCUDA(m, cudaSetDevice(m->device), "cudaSetDevice");
  MCUDA(m, mlp_step(m, (long)n, nullptr, X_dev, T_dev, (float)(1.0 / (double)n), m->grad, m->loss, false,
                    0.f),
        "mlp forward/backward");
  if (grad_host)
    MCUDA(m, cudaMemcpyAsync(grad_host, m->grad, MLP_PARAMS * sizeof(float), cudaMemcpyDeviceToHost,
                             m->stream),
          "gradient");
  double l = 0.0;
  MCUDA(m, cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream), "loss");
  MCUDA(m, cudaStreamSynchronize(m->stream), "mlp sync");
  if (loss) *loss = l;
  m->err.clear();
  return AMG_OK;
}

int amg_mlp_train(amg_mlp *m, const float *X_dev, const float *T_dev, int64_t n, int epochs, int batch,
                  float lr, uint64_t seed, double *epoch_loss) {
  if (!m || !X_dev || !T_dev || n < 1 || epochs < 0 || batch < TILE || !(lr > 0.f)) return AMG_ERR_ARG;
  if (n > 0x7fffffff) return mfail(m, AMG_ERR_ARG, "at most 2^31-1 samples");
  MCUDA(m, cudaSetDevice(m->device), "cudaSetDevice");
  if (m->perm_n < n) {
    dfree(m->perm);
    m->perm = nullptr;
    MCUDA(m, dalloc((void **)&m->perm, (size_t)n * sizeof(int)), "order buffer");
    m->perm_n = n;
  }
  std::vector<int> perm((size_t)n);
  for (long i = 0; i < n; ++i) perm[i] = (int)i;
  const long nsteps = (n + batch - 1) / batch;
  std::vector<double> losses((size_t)nsteps);
  double *dloss = nullptr;
  MCUDA(m, dalloc((void **)&dloss, (size_t)nsteps * sizeof(double)), "loss buffer");
  uint64_t s = seed;
  for (int ep = 0; ep < epochs; ++ep) {
    for (long i = n - 1; i > 0; --i) {  // Fisher-Yates
      const long j = (long)(splitmix64(s) % (uint64_t)(i + 1));
      const int t = perm[i];
      perm[i] = perm[j];
      perm[j] = t;
    }
    cudaError_t e = cudaMemcpyAsync(m->perm, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice,
                                    m->stream);
    for (long st = 0; st < nsteps && e == cudaSuccess; ++st) {
      const long b0 = st * batch, cnt = (n - b0 < batch) ? n - b0 : batch;
      e = mlp_step(m, cnt, m->perm + b0, X_dev, T_dev, (float)(1.0 / (double)cnt), nullptr, dloss + st,
                   true, lr);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(losses.data(), dloss, (size_t)nsteps * sizeof(double), cudaMemcpyDeviceToHost,
                          m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
      dfree(dloss);
      return mfail(m, AMG_ERR_CUDA, std::string("training: ") + cudaGetErrorString(e));
    }
    if (epoch_loss) {
      double tot = 0.0;
      for (long st = 0; st < nsteps; ++st) {
        const long b0 = st * batch, cnt = (n - b0 < batch) ? n - b0 : batch;
        tot += losses[st] * cnt;
      }
      epoch_loss[ep] = tot / (double)n;
    }
  }
  dfree(dloss);
  m->err.clear();
  return AMG_OK;
}

int amg_mlp_infer(amg_mlp *m, const float *X_dev, int64_t n, float *out_dev) {
  if (!m || !X_dev || !out_dev || n < 1) return AMG_ERR_ARG;
  MCUDA(m, cudaSetDevice(m->device), "cudaSetDevice");
  const long tiles = (n + TILE - 1) / TILE;
  const int nblk = (int)(tiles < 64L * m->max_blocks ? tiles : 64L * m->max_blocks);
  mlp_kernel<0><<<nblk, MLP_THREADS, 0, m->stream>>>((long)n, nullptr, X_dev, nullptr, m->w16, 0.f, out_dev,
                                                     nullptr, nullptr, nullptr, nullptr);
  MCUDA(m, cudaGetLastError(), "mlp inference");
  MCUDA(m, cudaStreamSynchronize(m->stream), "mlp inference");
  m->err.clear();
  return AMG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// context side: features, targets, installation of the learned blocks
// ---------------------------------------------------------------------------
static int cfail(Ctx *c, int code, const std::string &msg) {
  c->err = msg;
  return code;
}

#define CCUDA(c, expr, where)                                                                  \
  do {                                                                                         \
    cudaError_t _e = (expr);                                                                   \
    if (_e != cudaSuccess) return cfail(c, AMG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(_e)); \
  } while (0)

static int check_fine(Ctx *c, const char *where) {
  if (c->levels.empty()) return cfail(c, AMG_ERR_STATE, std::string(where) + ": no hierarchy uploaded");
  if (c->levels[0].k != 3)
    return cfail(c, AMG_ERR_ARG, std::string(where) + ": defined for 3D elasticity (3x3 blocks)");
  return AMG_OK;
}

static int features_dev(Ctx *c, const double *coords_host, float *X_dev, double *tr_dev) {
  const Level &L = c->levels[0];
  const int n = L.A.n_rows;
  double *xd = nullptr;
  int *err = nullptr;
  cudaError_t e = dalloc((void **)&xd, (size_t)n * 3 * sizeof(double));
  if (e == cudaSuccess) e = dalloc((void **)&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(xd, coords_host, (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && n > 0) {
    features_kernel<<<(n + 127) / 128, 128, 0, c->stream>>>(n, L.A.rowptr, L.A.colidx, L.A.v64, xd, X_dev,
                                                            tr_dev, err);
    e = cudaGetLastError();
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(xd);
  dfree(err);
  if (e != cudaSuccess) return cfail(c, AMG_ERR_CUDA, std::string("features: ") + cudaGetErrorString(e));
  if (herr) return cfail(c, AMG_ERR_ARG, "features: a vertex without positive diagonal block");
  return AMG_OK;
}

// Lanczos on B A in the A-inner product; returns the largest Ritz value
static int lanczos(Ctx *c, const double *Bn, double *lam_out) {
  const Level &L = c->levels[0];
  const size_t n = (size_t)L.A.n_rows * 3;
  double *buf = nullptr, *part = nullptr;
  const int nb = 256;
  CCUDA(c, dalloc((void **)&buf, 5 * n * sizeof(double)), "lanczos buffers");
  CCUDA(c, dalloc((void **)&part, nb * sizeof(double)), "lanczos buffers");
  double *v = buf, *u = buf + n, *vo = buf + 2 * n, *w = buf + 3 * n, *z = buf + 4 * n;
  std::vector<double> hv(n), hp(nb);
  uint64_t s = 0x5EEDULL;
  for (size_t i = 0; i < n; ++i) hv[i] = normal01(s);
  cudaError_t e = cudaMemcpyAsync(v, hv.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(vo, 0, n * sizeof(double), c->stream);
  auto dot = [&](const double *a, const double *b, double *r) -> cudaError_t {
    dot_partial_kernel<<<nb, 256, 0, c->stream>>>(n, a, b, part);
    AMG_CUDA_TRY(cudaGetLastError());
    AMG_CUDA_TRY(cudaMemcpyAsync(hp.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
    double t = 0.0;
    for (int i = 0; i < nb; ++i) t += hp[i];
    *r = t;
    return cudaSuccess;
  };
  const unsigned ge = (unsigned)((n + 255) / 256);
  std::vector<double> al, be;
  double nrm2 = 0.0, beta = 0.0;
  if (e == cudaSuccess) e = launch_bsr(c, L.A, AMG_PREC_FP64, SPMV_SET, v, nullptr, nullptr, u);
  if (e == cudaSuccess) e = dot(v, u, &nrm2);
  if (e == cudaSuccess && !(nrm2 > 0.0)) e = cudaErrorInvalidValue;
  if (e == cudaSuccess) {
    scale_kernel<<<ge, 256, 0, c->stream>>>(n, v, 1.0 / sqrt(nrm2));
    scale_kernel<<<ge, 256, 0, c->stream>>>(n, u, 1.0 / sqrt(nrm2));
    e = cudaGetLastError();
  }
  for (int k = 0; k < LANCZOS_STEPS && e == cudaSuccess; ++k) {
    double alpha = 0.0, wz = 0.0;
    e = launch_blockdiag(c, L.A.n_rows, 3, AMG_PREC_FP64, Bn, u, w);  // w = B A v
    if (e == cudaSuccess) e = dot(w, u, &alpha);                      // <BAv, v>_A
    if (e != cudaSuccess) break;
    lanczos_update_kernel<<<ge, 256, 0, c->stream>>>(n, w, v, vo, alpha, beta);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_bsr(c, L.A, AMG_PREC_FP64, SPMV_SET, w, nullptr, nullptr, z);
    if (e == cudaSuccess) e = dot(w, z, &wz);
    if (e != cudaSuccess) break;
    const double beta_new = sqrt(wz > 0.0 ? wz : 0.0);
    al.push_back(alpha);
    if (k == LANCZOS_STEPS - 1 || beta_new <= 1e-14 * fabs(alpha)) break;
    be.push_back(beta_new);
    // v_old <- v, v <- w / beta, u <- z / beta (rotate the buffers)
    double *t0 = vo;
    vo = v;
    v = w;
    w = t0;
    double *t1 = u;
    u = z;
    z = t1;
    scale_kernel<<<ge, 256, 0, c->stream>>>(n, v, 1.0 / beta_new);
    scale_kernel<<<ge, 256, 0, c->stream>>>(n, u, 1.0 / beta_new);
    e = cudaGetLastError();
    beta = beta_new;
  }
  dfree(buf);
  dfree(part);
  if (e != cudaSuccess) return cfail(c, AMG_ERR_CUDA, std::string("lanczos: ") + cudaGetErrorString(e));
  be.resize(al.size() > 0 ? al.size() - 1 : 0);
  *lam_out = tridiag_max_eig(al, be);
  return AMG_OK;
}

extern "C" {

int amg_learned_features(amg_ctx *h, const double *coords_host, float *X_dev, double *tr_dev) {
  if (!h || !coords_host || !X_dev) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_fine(c, "amg_learned_features");
  if (s) return s;
  CCUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  s = features_dev(c, coords_host, X_dev, tr_dev);
  if (s == AMG_OK) c->err.clear();
  return s;
}

int amg_learned_targets(amg_ctx *h, float *T32_dev, double *T64_dev) {
  if (!h || (!T32_dev && !T64_dev)) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_fine(c, "amg_learned_targets");
  if (s) return s;
  CCUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  const Level &L = c->levels[0];
  const int n = L.A.n_rows;
  int *err = nullptr;
  CCUDA(c, dalloc((void **)&err, sizeof(int)), "targets");
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess && n > 0) {
    patch_target_kernel<<<(n + 1) / 2, 64, 0, c->stream>>>(n, L.A.rowptr, L.A.colidx, L.A.v64, T32_dev,
                                                           T64_dev, err);
    e = cudaGetLastError();
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(err);
  if (e != cudaSuccess) return cfail(c, AMG_ERR_CUDA, std::string("targets: ") + cudaGetErrorString(e));
  if (herr)
    return cfail(c, AMG_ERR_ARG, "targets: " + std::to_string(herr) +
                                     " vertices with more than 15 neighbours or a singular patch");
  c->err.clear();
  return AMG_OK;
}

int amg_set_learned_smoother(amg_ctx *h, amg_mlp *m, const double *coords_host, double *lambda_out,
                             double *omega_out) {
  if (!h || !m || !coords_host) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_fine(c, "amg_set_learned_smoother");
  if (s) return s;
  if (c->levels.size() < 2) return cfail(c, AMG_ERR_STATE, "amg_set_learned_smoother: one-level hierarchy");
  if (c->smoother == AMG_SMOOTHER_HYBRID_GS)
    return cfail(c, AMG_ERR_STATE, "amg_set_learned_smoother: the context uses the hybrid Gauss-Seidel smoother");
  if (m->device != c->device) return cfail(c, AMG_ERR_ARG, "network and context on different devices");
  CCUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  Level &L = c->levels[0];
  const int n = L.A.n_rows;
  float *X = nullptr;
  double *tr = nullptr, *Bn = nullptr;
  CCUDA(c, dalloc((void **)&X, (size_t)n * MLP_IN * sizeof(float)), "learned buffers");
  cudaError_t e = dalloc((void **)&tr, (size_t)n * sizeof(double));
  if (e == cudaSuccess) e = dalloc((void **)&Bn, (size_t)n * 9 * sizeof(double));
  if (e != cudaSuccess) {
    dfree(X);
    dfree(tr);
    return cfail(c, AMG_ERR_CUDA, "learned buffers");
  }
  s = features_dev(c, coords_host, X, tr);
  double lam = 0.0;
  if (s == AMG_OK) {
    // the network's stream waits for the features (synchronised above)
    const long tiles = ((long)n + TILE - 1) / TILE;
    const int nblk = (int)(tiles < 64L * m->max_blocks ? tiles : 64L * m->max_blocks);
    mlp_kernel<0><<<nblk, MLP_THREADS, 0, c->stream>>>((long)n, nullptr, X, nullptr, m->w16, 0.f, nullptr,
                                                       tr, Bn, nullptr, nullptr);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) s = cfail(c, AMG_ERR_CUDA, std::string("mlp inference: ") + cudaGetErrorString(e));
  }
  if (s == AMG_OK) s = lanczos(c, Bn, &lam);
  if (s == AMG_OK && !(lam > 0.0)) s = cfail(c, AMG_ERR_NOT_SPD, "learned smoother: lambda_max(BA) <= 0");
  double w = 0.0;
  if (s == AMG_OK) {
    w = OMEGA_NUM / (LANCZOS_SAFETY * lam);
    const size_t nn = (size_t)n * 9;
    install_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(
        nn, Bn, w, L.minv64, c->precision != AMG_PREC_FP64 ? L.minv32 : nullptr);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) s = cfail(c, AMG_ERR_CUDA, std::string("install: ") + cudaGetErrorString(e));
  }
  dfree(X);
  dfree(tr);
  dfree(Bn);
  if (s != AMG_OK) return s;
  c->smoother = AMG_SMOOTHER_LEARNED;
  if (lambda_out) *lambda_out = lam;
  if (omega_out) *omega_out = w;
  c->err.clear();
  return AMG_OK;
}

int amg_reset_smoother(amg_ctx *h) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  if (c->levels.empty()) return cfail(c, AMG_ERR_STATE, "amg_reset_smoother: no hierarchy uploaded");
  CCUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (c->levels.size() > 1) {
    CCUDA(c, smoother_setup(c, 0), "smoother setup");
    CCUDA(c, cudaStreamSynchronize(c->stream), "smoother setup");
  }
  if (c->smoother == AMG_SMOOTHER_LEARNED) c->smoother = AMG_SMOOTHER_L1_JACOBI;
  c->err.clear();
  return AMG_OK;
}

}  // extern "C"
