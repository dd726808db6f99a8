// amg_vcycle_static: the V-cycle of amg_vcycle with its work vectors in a
// fixed, file-scope device array instead of buffers of the context, for
// callers that must not allocate device memory while they run it.
//
// Callers that cannot allocate: code that runs where a framework's caching
// allocator already holds all free device memory (a cudaMalloc would fail or
// force the framework to release its cache), and code with a memory budget
// fixed before it starts (real-time or embedded use).  The hierarchy must
// have been uploaded before (amg_upload_hierarchy / amg_setup allocate).
//
// The first call on a device is the set-up: it looks up the array's device
// address (cudaGetSymbolAddress, with that device current).  With lazy module
// loading (the CUDA default) that lookup also loads this file's device module,
// and the driver reserves the array's 16 MiB then.  Make that first call
// while 16 MiB are free; every later call on the device allocates nothing.
#include <mutex>

#include "amg_internal.h"

namespace amg {

// Work vectors of every level (b, x, t, y per level, each 256-byte aligned).
// Every GPU that loads the library holds this array until the process exits.
constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_vcycle_scratch[kStaticScratchBytes];

// Device address of g_vcycle_scratch per device, looked up once per device
// with that device current (the host-side symbol is only a stand-in).
static std::mutex g_scratch_mutex;
static void *g_scratch_ptr[64] = {nullptr};

static cudaError_t scratch_address(int device, void **out) {
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[device]) {
    int cur = -1;
    AMG_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != device) AMG_CUDA_TRY(cudaSetDevice(device));
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_vcycle_scratch);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Bytes of scratch the V-cycle of this hierarchy needs.
static size_t scratch_bytes(const Ctx *c) {
  const size_t w = c->precision == AMG_PREC_FP64 ? sizeof(double) : sizeof(float);
  size_t total = 0;
  for (const Level &L : c->levels) total += 4 * align256((size_t)L.A.n_rows * L.k * w);
  return total;
}

// Same steps and kernels as the context V-cycle (Algorithm tg applied
// recursively), on the vectors bx[l] / xx[l] / tx[l] / yx[l].
static cudaError_t vcycle_static_level(Ctx *c, int l, void *const *bx, void *const *xx,
                                       void *const *tx, void *const *yx, const void *b, void *y,
                                       const double *r64, double *z64) {
  const int prec = mat_prec(c, l);
  Level &L = c->levels[l];
  if (l == (int)c->levels.size() - 1) return launch_coarse_gemv(c, c->coarse_n, c->cinv, b, y, prec);
  const void *mi = prec == AMG_PREC_FP64 ? (const void *)L.minv64 : (const void *)L.minv32;
  if (r64)
    AMG_CUDA_TRY(launch_blockdiag_entry(c, L.A.n_rows, L.k, L.minv32, r64, (float *)b, (float *)xx[l]));
  else
    AMG_CUDA_TRY(launch_blockdiag(c, L.A.n_rows, L.k, prec, mi, b, xx[l]));
  AMG_CUDA_TRY(launch_bsr(c, L.A, prec, SPMV_RESID, xx[l], b, nullptr, tx[l]));
  AMG_CUDA_TRY(launch_bsr(c, L.R, prec, SPMV_SET, tx[l], nullptr, nullptr, bx[l + 1]));
  AMG_CUDA_TRY(vcycle_static_level(c, l + 1, bx, xx, tx, yx, bx[l + 1], yx[l + 1], nullptr, nullptr));
  AMG_CUDA_TRY(launch_bsr(c, L.P, prec, SPMV_ADD, yx[l + 1], nullptr, nullptr, xx[l]));
  if (z64)
    return launch_smooth_out64(c, L.A, prec, (const float *)xx[l], (const float *)b, L.minv32, z64);
  return launch_bsr(c, L.A, prec, SPMV_SMOOTH, xx[l], b, mi, y);
}

}  // namespace amg

using namespace amg;

extern "C" int amg_vcycle_static(amg_ctx *h, const double *r_dev, double *z_dev) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  if (c->levels.empty()) {
    c->err = "amg_vcycle_static: no hierarchy uploaded";
    return AMG_ERR_STATE;
  }
  if (!r_dev || !z_dev) {
    c->err = "amg_vcycle_static: NULL vector";
    return AMG_ERR_ARG;
  }
  if (c->smoother == AMG_SMOOTHER_HYBRID_GS) {
    c->err = "amg_vcycle_static: runs the block-l1 Jacobi and learned smoothers only";
    return AMG_ERR_ARG;
  }
  const int nl = (int)c->levels.size();
  if (nl > 32) {
    c->err = "amg_vcycle_static: more than 32 levels";
    return AMG_ERR_ARG;
  }
  const size_t need = scratch_bytes(c);
  if (need > kStaticScratchBytes) {
    c->err = "amg_vcycle_static: the V-cycle needs " + std::to_string(need) +
             " bytes of work vectors, more than the fixed " +
             std::to_string(kStaticScratchBytes) + "-byte device array";
    return AMG_ERR_ARG;
  }
  void *base = nullptr;
  cudaError_t e = scratch_address(c->device, &base);
  if (e != cudaSuccess) {
    c->err = std::string("amg_vcycle_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return AMG_ERR_CUDA;
  }
  // carve the level vectors out of the array (nothing in them has to start
  // at zero: every vector is written before it is read in one V-cycle)
  void *bx[32], *xx[32], *tx[32], *yx[32];
  const size_t w = c->precision == AMG_PREC_FP64 ? sizeof(double) : sizeof(float);
  unsigned char *cur = (unsigned char *)base;
  for (int l = 0; l < nl; ++l) {
    const size_t bytes = align256((size_t)c->levels[l].A.n_rows * c->levels[l].k * w);
    bx[l] = cur;
    cur += bytes;
    xx[l] = cur;
    cur += bytes;
    tx[l] = cur;
    cur += bytes;
    yx[l] = cur;
    cur += bytes;
  }
  if (c->precision == AMG_PREC_FP64)
    e = vcycle_static_level(c, 0, bx, xx, tx, yx, r_dev, z_dev, nullptr, nullptr);
  else if (nl == 1) {
    const size_t n = (size_t)c->levels[0].A.n_rows * c->levels[0].k;
    e = launch_convert(c, n, r_dev, AMG_PREC_FP64, bx[0], AMG_PREC_FP32_VCYCLE);
    if (e == cudaSuccess) e = launch_coarse_gemv(c, c->coarse_n, c->cinv, bx[0], yx[0], mat_prec(c, 0));
    if (e == cudaSuccess) e = launch_convert(c, n, yx[0], AMG_PREC_FP32_VCYCLE, z_dev, AMG_PREC_FP64);
  } else {
    e = vcycle_static_level(c, 0, bx, xx, tx, yx, bx[0], yx[0], r_dev, z_dev);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    c->err = std::string("amg_vcycle_static: ") + cudaGetErrorString(e);
    return AMG_ERR_CUDA;
  }
  c->err.clear();
  return AMG_OK;
}
