// Load helpers of the block-sparse kernels (BSR, SELL-32 and the Gauss-Seidel
// sweeps): accumulation type per vector type, single loads (cached for
// vectors, streamed for matrix values that are read once), and runs of n
// consecutive values with 8- or 16-byte vector loads where they align.
#pragma once

#include <cuda_bf16.h>

namespace amg {

template <typename T>
struct AccT {
  using type = float;
};
template <>
struct AccT<double> {
  using type = double;
};

__device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p) {
  return __bfloat162float(__ldg(p));
}
// streamed matrix values: read once, keep them out of L1
__device__ __forceinline__ double lds(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float lds(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float lds(const __nv_bfloat16 *p) {
  unsigned short u = __ldcs(reinterpret_cast<const unsigned short *>(p));
  return __uint_as_float(((unsigned)u) << 16);
}

// n consecutive values starting at p, streamed (values) or cached (vectors),
// with the widest loads the alignment allows: a block row of BC values is
// 2-element aligned whenever BC is even.
template <int N, typename A>
__device__ __forceinline__ void ldn_stream(const double *p, A *out) {
  if (N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      const double2 v = __ldcs(reinterpret_cast<const double2 *>(p + i));
      out[i] = (A)v.x;
      out[i + 1] = (A)v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = (A)__ldcs(p + i);
  }
}
template <int N, typename A>
__device__ __forceinline__ void ldn_stream(const float *p, A *out) {
  if (N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      const float2 v = __ldcs(reinterpret_cast<const float2 *>(p + i));
      out[i] = (A)v.x;
      out[i + 1] = (A)v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = (A)__ldcs(p + i);
  }
}
template <int N, typename A>
__device__ __forceinline__ void ldn_stream(const __nv_bfloat16 *p, A *out) {
  if (N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      const unsigned u = __ldcs(reinterpret_cast<const unsigned *>(p + i));
      out[i] = (A)__uint_as_float(u << 16);
      out[i + 1] = (A)__uint_as_float(u & 0xffff0000u);
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = (A)lds(p + i);
  }
}
template <int N, typename A>
__device__ __forceinline__ void ldn_cached(const double *p, A *out) {
  if (N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      const double2 v = __ldg(reinterpret_cast<const double2 *>(p + i));
      out[i] = (A)v.x;
      out[i + 1] = (A)v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = (A)__ldg(p + i);
  }
}
template <int N, typename A>
__device__ __forceinline__ void ldn_cached(const float *p, A *out) {
  if (N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      const float2 v = __ldg(reinterpret_cast<const float2 *>(p + i));
      out[i] = (A)v.x;
      out[i + 1] = (A)v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = (A)__ldg(p + i);
  }
}

}  // namespace amg
