// Arithmetic-throughput probe: the FP64 and FP32 FMA rates of the device,
// measured live so that ALU-bound kernels (FP64 sparse products on sm_103a,
// whose FP64 pipe is narrow) are reported against a measured peak.
#include "amg_internal.h"

namespace amg {

template <typename T>
__global__ void fma_probe_kernel(T *out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static cudaError_t probe_one(Ctx *c, int iters, double *gflops) {
  const int blocks = c->num_sms * 8, threads = 256;
  T *out = nullptr;
  AMG_CUDA_TRY(dalloc((void **)&out, (size_t)blocks * threads * sizeof(T)));
  fma_probe_kernel<T><<<blocks, threads, 0, c->stream>>>(out, 64, (T)0.999, (T)0.001);
  AMG_CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
  fma_probe_kernel<T><<<blocks, threads, 0, c->stream>>>(out, iters, (T)0.999, (T)0.001);
  AMG_CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
  AMG_CUDA_TRY(cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  AMG_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  dfree(out);
  *gflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e6);
  return cudaGetLastError();
}

cudaError_t probe_fma(Ctx *c, double *fp64, double *fp32) {
  AMG_CUDA_TRY(probe_one<double>(c, 2048, fp64));
  return probe_one<float>(c, 16384, fp32);
}

}  // namespace amg
