// Batched solve: many independent systems (each an amg_ctx with its own
// hierarchy), each with NR load cases, solved by one launch of one CUDA
// graph.  Every system is an independent branch of the graph: its own
// device-side while loop (conditional node) runs FP64 PCG (Sec. 7) on its NR
// load cases at once, preconditioned by the multi-load-case V-cycle, so the
// uneven systems proceed concurrently and finish independently.  Load cases
// that converge are frozen (their iteration count stops) while the others
// continue.
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "amg_internal.h"
#include "multirhs.h"

namespace amg {

constexpr int kMaxNR = 8;

struct McgState {  // per system
  double rr[kMaxNR], ff[kMaxNR], tol2[kMaxNR], rho[kMaxNR], rho_old[kMaxNR], alpha[kMaxNR],
      beta[kMaxNR], pq[kMaxNR];
  int it[kMaxNR], done[kMaxNR], status[kMaxNR];
  double rtol;
  int maxit, flexible, guard, nr;
};

struct SysBuf {
  Ctx *c = nullptr;       // the system's context (hierarchy, stream ignored)
  size_t n = 0;           // dofs of A_0
  size_t offset = 0;      // offset of the system's load cases in the stacked f / u
  double *f = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *zold = nullptr, *p = nullptr,
         *q = nullptr;
  std::vector<void *> lb, lx, lt, ly;  // V-cycle level vectors (n_l * NR)
  McgState *st = nullptr;
  double *partials = nullptr;
  unsigned *counter = nullptr;
  int red_grid = 1;
};

struct Batch {
  int device = 0, nr = 1, precision = 0, num_sms = 0;
  cudaStream_t stream = nullptr;
  std::vector<SysBuf> sys;
  size_t total = 0;  // stacked length of f / u
  double *fin = nullptr, *uio = nullptr;
  McgState *st_host = nullptr;
  cudaGraph_t graph_def = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err;
};

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// rhs-major (NR vectors of n) <-> interleaved (n x NR)
template <int NR>
__global__ void pack_kernel(size_t n, const double *__restrict__ src, double *__restrict__ dst) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int j = 0; j < NR; ++j) dst[i * NR + j] = src[(size_t)j * n + i];
}
template <int NR>
__global__ void unpack_kernel(size_t n, const double *__restrict__ src, double *__restrict__ dst) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int j = 0; j < NR; ++j) dst[(size_t)j * n + i] = src[i * NR + j];
}

enum McgPhase { PH_INIT = 0, PH_RHO = 1, PH_PQ = 2, PH_RR = 3 };

// Per-load-case inner products with a last-block total (index order:
// deterministic), then the phase's scalar update of the CG state.
//   INIT: rr = r.r, ff = f.f      RHO: r.z, r.z_old -> beta, rho
//   PQ:   p.q -> alpha            RR:  r.r (loop decision in the guard)
template <int NR, int PH>
__global__ void __launch_bounds__(256) mcg_dots_kernel(size_t n, const double *a1, const double *b1,
                                                       const double *a2, const double *b2,
                                                       McgState *st, double *partials,
                                                       unsigned *counter,
                                                       cudaGraphConditionalHandle h) {
  __shared__ double sh[2 * NR][8];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double v1[NR], v2[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) v1[j] = v2[j] = 0.0;
  const bool two = (PH == PH_INIT) || (PH == PH_RHO && true);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      v1[j] += a1[i * NR + j] * b1[i * NR + j];
      if (two && a2) v2[j] += a2[i * NR + j] * b2[i * NR + j];
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
      partials[(size_t)j * gridDim.x + blockIdx.x] = s;
    }
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double t1[NR], t2[NR];
  for (int j = 0; j < NR; ++j) {
    t1[j] = t2[j] = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      t1[j] += ((volatile double *)partials)[(size_t)j * gridDim.x + b];
      t2[j] += ((volatile double *)partials)[(size_t)(NR + j) * gridDim.x + b];
    }
  }
  *counter = 0u;
  if (PH == PH_INIT) {
    bool any = false;
    for (int j = 0; j < NR; ++j) {
      st->rr[j] = t1[j];
      st->ff[j] = t2[j];
      st->tol2[j] = st->rtol * st->rtol * t2[j];
      st->it[j] = 0;
      st->status[j] = 0;
      st->rho_old[j] = 0.0;
      st->done[j] = !(t1[j] > st->tol2[j]) || st->maxit <= 0 || !isfinite(t1[j]);
      any = any || !st->done[j];
    }
    st->guard = 0;
    cudaGraphSetConditional(h, any ? 1u : 0u);
  } else if (PH == PH_RHO) {
    for (int j = 0; j < NR; ++j) {
      if (st->done[j]) continue;
      const double rho = t1[j];
      st->beta[j] = st->it[j] > 0 ? (st->flexible ? (rho - t2[j]) : rho) / st->rho_old[j] : 0.0;
      st->rho[j] = rho;
      st->rho_old[j] = rho;
    }
  } else if (PH == PH_PQ) {
    for (int j = 0; j < NR; ++j) {
      st->pq[j] = t1[j];
      if (st->done[j]) {
        st->alpha[j] = 0.0;
        continue;
      }
      if (!(t1[j] > 0.0) || !isfinite(t1[j])) {
        st->status[j] = AMG_ERR_NOT_SPD;
        st->done[j] = 1;
        st->alpha[j] = 0.0;
      } else {
        st->alpha[j] = st->rho[j] / t1[j];
      }
    }
  } else {  // PH_RR
    for (int j = 0; j < NR; ++j)
      if (!st->done[j]) st->rr[j] = t1[j];
  }
}

// p = z + beta p (first iteration: p = z) for the active load cases
template <int NR>
__global__ void mcg_update_p_kernel(size_t n, const double *z, double *p, double *zold,
                                    const McgState *st) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    if (st->done[j]) continue;
    const double zi = z[i * NR + j];
    p[i * NR + j] = st->it[j] == 0 ? zi : zi + st->beta[j] * p[i * NR + j];
    if (st->flexible) zold[i * NR + j] = zi;
  }
}

// x += alpha p ; r -= alpha q for the active load cases
template <int NR>
__global__ void mcg_update_xr_kernel(size_t n, double *x, double *r, const double *p,
                                     const double *q, const McgState *st) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    if (st->done[j]) continue;
    const double a = st->alpha[j];
    x[i * NR + j] += a * p[i * NR + j];
    r[i * NR + j] -= a * q[i * NR + j];
  }
}

// Last node of every iteration (one thread): counts iterations of the active
// load cases, marks the converged ones, bounds the loop, sets the condition.
__global__ void mcg_guard_kernel(McgState *st, unsigned *counter, cudaGraphConditionalHandle h) {
  *counter = 0u;
  st->guard += 1;
  bool any = false;
  for (int j = 0; j < st->nr; ++j) {
    if (st->done[j]) continue;
    st->it[j] += 1;
    if (!isfinite(st->rr[j])) {
      st->status[j] = AMG_ERR_NOT_SPD;
      st->done[j] = 1;
    } else if (!(st->rr[j] > st->tol2[j]) || st->it[j] >= st->maxit) {
      st->done[j] = 1;
    }
    any = any || !st->done[j];
  }
  cudaGraphSetConditional(h, (any && st->guard < st->maxit) ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// multi-load-case V-cycle of one system
// ---------------------------------------------------------------------------

static cudaError_t vcycle_mr_level(const Batch *B, const SysBuf &S, int l, const void *b, void *y,
                                   const double *r64, double *z64) {
  Ctx *c = S.c;
  const int prec = c->precision, nr = B->nr;
  Level &L = c->levels[l];
  if (l == (int)c->levels.size() - 1) {
    if (!r64 || prec == AMG_PREC_FP64) return launch_coarse_mr(c, c->coarse_n, nr, c->cinv, b, y, prec);
    // one-level hierarchy in low precision: cast in, coarsest solve, cast out
    const size_t m = (size_t)c->coarse_n * nr;
    AMG_CUDA_TRY(launch_convert(c, m, r64, AMG_PREC_FP64, (void *)b, AMG_PREC_FP32_VCYCLE));
    AMG_CUDA_TRY(launch_coarse_mr(c, c->coarse_n, nr, c->cinv, b, y, prec));
    return launch_convert(c, m, y, AMG_PREC_FP32_VCYCLE, z64, AMG_PREC_FP64);
  }
  const void *mi = prec == AMG_PREC_FP64 ? (const void *)L.minv64 : (const void *)L.minv32;
  void *x = S.lx[l], *t = S.lt[l];
  if (r64)  // finest level: the FP64 CG residual, cast copy kept in b
    AMG_CUDA_TRY(launch_blockdiag_mr(c, L.A.n_rows, L.k, prec, nr, mi, r64, true,
                                     prec == AMG_PREC_FP64 ? nullptr : (void *)b, x));
  else
    AMG_CUDA_TRY(launch_blockdiag_mr(c, L.A.n_rows, L.k, prec, nr, mi, b, false, nullptr, x));
  const void *bb = (r64 && prec == AMG_PREC_FP64) ? (const void *)r64 : b;
  AMG_CUDA_TRY(launch_bsr_mr(c, L.A, prec, nr, SPMV_RESID, x, bb, nullptr, t, false));
  AMG_CUDA_TRY(launch_bsr_mr(c, L.R, prec, nr, SPMV_SET, t, nullptr, nullptr, S.lb[l + 1], false));
  AMG_CUDA_TRY(vcycle_mr_level(B, S, l + 1, S.lb[l + 1], S.ly[l + 1], nullptr, nullptr));
  AMG_CUDA_TRY(launch_bsr_mr(c, L.P, prec, nr, SPMV_ADD, S.ly[l + 1], nullptr, nullptr, x, false));
  if (z64) return launch_bsr_mr(c, L.A, prec, nr, SPMV_SMOOTH, x, bb, mi, z64, prec != AMG_PREC_FP64);
  return launch_bsr_mr(c, L.A, prec, nr, SPMV_SMOOTH, x, bb, mi, y, false);
}

template <int NR>
static cudaError_t capture_system(Batch *B, SysBuf &S, cudaGraph_t g) {
  Ctx *c = S.c;
  cudaStream_t s = B->stream;
  const Level &L0 = c->levels[0];
  const size_t n = S.n;
  const int gv = S.red_grid;
  const unsigned ge = (unsigned)((n + 255) / 256);
  cudaGraphConditionalHandle h;
  AMG_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
  // init branch: pack f, u; r = f - A x; rr, ff; loop decision
  AMG_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaStream_t cs = c->stream;
  c->stream = s;  // the system's launches go to the capturing stream
  cudaError_t e = cudaSuccess;
  pack_kernel<NR><<<ge, 256, 0, s>>>(n, B->fin + S.offset, S.f);
  pack_kernel<NR><<<ge, 256, 0, s>>>(n, B->uio + S.offset, S.x);
  if (e == cudaSuccess)
    e = launch_bsr_mr(c, L0.A, AMG_PREC_FP64, NR, SPMV_RESID, S.x, S.f, nullptr, S.r, false);
  mcg_dots_kernel<NR, PH_INIT><<<gv, 256, 0, s>>>(n, S.r, S.r, S.f, S.f, S.st, S.partials, S.counter, h);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaGraph_t cap = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  cudaStreamCaptureStatus status;
  cudaError_t e2 = cudaStreamGetCaptureInfo(s, &status, nullptr, nullptr, &deps, nullptr, &ndeps);
  std::vector<cudaGraphNode_t> sinks(deps, deps + ndeps);
  cudaError_t e3 = cudaStreamEndCapture(s, &cap);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = e3;
  if (e != cudaSuccess) {
    c->stream = cs;
    return e;
  }
  // while node with the iteration body
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  e = cudaGraphAddNode(&cnode, g, sinks.data(), nullptr, sinks.size(), &cp);
  if (e != cudaSuccess) {
    c->stream = cs;
    return e;
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  AMG_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const bool fp64 = c->precision == AMG_PREC_FP64;
  e = vcycle_mr_level(B, S, 0, fp64 ? (void *)S.r : S.lb[0], fp64 ? (void *)S.z : S.ly[0], S.r, S.z);
  mcg_dots_kernel<NR, PH_RHO><<<gv, 256, 0, s>>>(n, S.r, S.z, S.r, S.zold, S.st, S.partials, S.counter, h);
  mcg_update_p_kernel<NR><<<ge, 256, 0, s>>>(n, S.z, S.p, S.zold, S.st);
  if (e == cudaSuccess)
    e = launch_bsr_mr(c, L0.A, AMG_PREC_FP64, NR, SPMV_SET, S.p, nullptr, nullptr, S.q, false);
  mcg_dots_kernel<NR, PH_PQ><<<gv, 256, 0, s>>>(n, S.p, S.q, nullptr, nullptr, S.st, S.partials, S.counter, h);
  mcg_update_xr_kernel<NR><<<ge, 256, 0, s>>>(n, S.x, S.r, S.p, S.q, S.st);
  mcg_dots_kernel<NR, PH_RR><<<gv, 256, 0, s>>>(n, S.r, S.r, nullptr, nullptr, S.st, S.partials, S.counter, h);
  mcg_guard_kernel<<<1, 1, 0, s>>>(S.st, S.counter, h);
  if (e == cudaSuccess) e = cudaGetLastError();
  e2 = cudaStreamEndCapture(s, &body);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    c->stream = cs;
    return e;
  }
  // after the loop: unpack the solution (a third capture, depending on cnode)
  AMG_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, g, &cnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  unpack_kernel<NR><<<ge, 256, 0, s>>>(n, S.x, B->uio + S.offset);
  e = cudaGetLastError();
  e2 = cudaStreamEndCapture(s, &cap);
  c->stream = cs;
  if (e == cudaSuccess) e = e2;
  return e;
}

static void free_batch(Batch *B) {
  if (B->graph) cudaGraphExecDestroy(B->graph);
  if (B->graph_def) cudaGraphDestroy(B->graph_def);
  for (SysBuf &S : B->sys) {
    double *d[] = {S.f, S.x, S.r, S.z, S.zold, S.p, S.q, S.partials};
    for (double *p : d) dfree(p);
    for (auto *v : {&S.lb, &S.lx, &S.lt, &S.ly})
      for (void *p : *v) dfree(p);
    dfree(S.st);
    dfree(S.counter);
  }
  dfree(B->fin);
  dfree(B->uio);
  if (B->st_host) cudaFreeHost(B->st_host);
  if (B->ev0) cudaEventDestroy(B->ev0);
  if (B->ev1) cudaEventDestroy(B->ev1);
  if (B->stream) cudaStreamDestroy(B->stream);
}

}  // namespace amg

using namespace amg;

struct amg_batch {
  Batch b;
};

static int bfail(Batch *B, int code, const std::string &m) {
  B->err = m;
  return code;
}

#define BCUDA(B, expr, where)                                                              \
  do {                                                                                     \
    cudaError_t _e = (expr);                                                               \
    if (_e != cudaSuccess) return bfail(B, AMG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(_e)); \
  } while (0)

extern "C" {

int amg_batch_create(amg_batch **out, amg_ctx *const *systems, int n_systems, int nrhs) {
  if (!out || !systems || n_systems < 1 || (nrhs != 1 && nrhs != 6)) return AMG_ERR_ARG;
  *out = nullptr;
  amg_batch *hb = new amg_batch();
  Batch *B = &hb->b;
  B->nr = nrhs;
  for (int s = 0; s < n_systems; ++s) {
    if (!systems[s] || systems[s]->c.levels.empty() ||
        (systems[s]->c.levels[0].k != 2 && systems[s]->c.levels[0].k != 3)) {
      delete hb;
      return AMG_ERR_STATE;
    }
    if (s > 0 && (systems[s]->c.device != systems[0]->c.device ||
                  systems[s]->c.precision != systems[0]->c.precision)) {
      delete hb;
      return AMG_ERR_ARG;
    }
  }
  Ctx *c0 = &systems[0]->c;
  B->device = c0->device;
  B->precision = c0->precision;
  B->num_sms = c0->num_sms;
  int rc = AMG_OK;
  auto fail_out = [&](int code) {
    free_batch(B);
    delete hb;
    return code;
  };
  if (cudaSetDevice(B->device) != cudaSuccess) return fail_out(AMG_ERR_CUDA);
  if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&B->ev0) != cudaSuccess || cudaEventCreate(&B->ev1) != cudaSuccess ||
      cudaMallocHost((void **)&B->st_host, sizeof(McgState) * n_systems) != cudaSuccess)
    return fail_out(AMG_ERR_CUDA);
  B->sys.resize(n_systems);
  size_t off = 0;
  for (int s = 0; s < n_systems; ++s) {
    SysBuf &S = B->sys[s];
    S.c = &systems[s]->c;
    S.n = (size_t)S.c->levels[0].A.n_rows * S.c->levels[0].k;
    S.offset = off;
    off += S.n * nrhs;
    const size_t bytes = S.n * nrhs * sizeof(double);
    double **d[] = {&S.f, &S.x, &S.r, &S.z, &S.zold, &S.p, &S.q};
    for (double **p : d)
      if (dalloc((void **)p, bytes) != cudaSuccess || cudaMemset(*p, 0, bytes) != cudaSuccess)
        return fail_out(AMG_ERR_CUDA);
    const size_t w = B->precision == AMG_PREC_FP64 ? sizeof(double) : sizeof(float);
    for (const Level &L : S.c->levels) {
      const size_t lb = (size_t)L.A.n_rows * L.k * nrhs * w;
      for (auto *v : {&S.lb, &S.lx, &S.lt, &S.ly}) {
        void *p = nullptr;
        if (dalloc(&p, lb) != cudaSuccess || cudaMemset(p, 0, lb) != cudaSuccess)
          return fail_out(AMG_ERR_CUDA);
        v->push_back(p);
      }
    }
    long gv = (long)((S.n * nrhs + 2047) / 2048);
    if (gv > B->num_sms) gv = B->num_sms;
    S.red_grid = (int)(gv < 1 ? 1 : gv);
    if (dalloc((void **)&S.st, sizeof(McgState)) != cudaSuccess ||
        dalloc((void **)&S.partials, 2 * kMaxNR * (size_t)S.red_grid * sizeof(double)) != cudaSuccess ||
        dalloc((void **)&S.counter, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(S.counter, 0, sizeof(unsigned)) != cudaSuccess)
      return fail_out(AMG_ERR_CUDA);
  }
  B->total = off;
  if (dalloc((void **)&B->fin, off * sizeof(double)) != cudaSuccess ||
      dalloc((void **)&B->uio, off * sizeof(double)) != cudaSuccess)
    return fail_out(AMG_ERR_CUDA);
  // one graph: one independent branch per system
  cudaError_t e = cudaGraphCreate(&B->graph_def, 0);
  for (int s = 0; s < n_systems && e == cudaSuccess; ++s)
    e = (nrhs == 6) ? capture_system<6>(B, B->sys[s], B->graph_def)
                    : capture_system<1>(B, B->sys[s], B->graph_def);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&B->graph, B->graph_def, 0);
  if (e != cudaSuccess) return fail_out(AMG_ERR_CUDA);
  (void)rc;
  *out = hb;
  return AMG_OK;
}

void amg_batch_destroy(amg_batch *hb) {
  if (!hb) return;
  cudaSetDevice(hb->b.device);
  cudaStreamSynchronize(hb->b.stream);
  free_batch(&hb->b);
  delete hb;
}

const char *amg_batch_last_error(const amg_batch *hb) { return hb ? hb->b.err.c_str() : "NULL batch"; }

int amg_batch_layout(const amg_batch *hb, int s, int64_t *offset, int64_t *n_dofs, int64_t *total) {
  if (!hb) return AMG_ERR_ARG;
  const Batch *B = &hb->b;
  if (total) *total = (int64_t)B->total;
  if (s < 0 || s >= (int)B->sys.size()) return AMG_ERR_ARG;
  if (offset) *offset = (int64_t)B->sys[s].offset;
  if (n_dofs) *n_dofs = (int64_t)B->sys[s].n;
  return AMG_OK;
}

int amg_batch_pcg_solve(amg_batch *hb, const double *f_dev, double *u_dev, double rtol, int maxit,
                        int *iters_out, double *relres_out, float *ms_out) {
  if (!hb) return AMG_ERR_ARG;
  Batch *B = &hb->b;
  if (!f_dev || !u_dev || !(rtol >= 0.0) || maxit < 0) return bfail(B, AMG_ERR_ARG, "bad arguments");
  BCUDA(B, cudaSetDevice(B->device), "cudaSetDevice");
  const int ns = (int)B->sys.size();
  for (int s = 0; s < ns; ++s) {
    McgState &h = B->st_host[s];
    memset(&h, 0, sizeof(McgState));
    h.rtol = rtol;
    h.maxit = maxit;
    h.nr = B->nr;
    h.flexible = B->precision != AMG_PREC_FP64;
    BCUDA(B, cudaMemcpyAsync(B->sys[s].st, &h, sizeof(McgState), cudaMemcpyHostToDevice, B->stream),
          "state");
  }
  BCUDA(B, cudaMemcpyAsync(B->fin, f_dev, B->total * sizeof(double), cudaMemcpyDeviceToDevice, B->stream),
        "copy f");
  BCUDA(B, cudaMemcpyAsync(B->uio, u_dev, B->total * sizeof(double), cudaMemcpyDeviceToDevice, B->stream),
        "copy u");
  BCUDA(B, cudaEventRecord(B->ev0, B->stream), "event");
  BCUDA(B, cudaGraphLaunch(B->graph, B->stream), "batch graph launch");
  BCUDA(B, cudaEventRecord(B->ev1, B->stream), "event");
  BCUDA(B, cudaMemcpyAsync(u_dev, B->uio, B->total * sizeof(double), cudaMemcpyDeviceToDevice, B->stream),
        "copy u back");
  for (int s = 0; s < ns; ++s)
    BCUDA(B, cudaMemcpyAsync(&B->st_host[s], B->sys[s].st, sizeof(McgState), cudaMemcpyDeviceToHost,
                             B->stream), "state");
  BCUDA(B, cudaStreamSynchronize(B->stream), "batch sync");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, B->ev0, B->ev1);
  if (ms_out) *ms_out = ms;
  int worst = AMG_OK;
  for (int s = 0; s < ns; ++s) {
    const McgState &h = B->st_host[s];
    for (int j = 0; j < B->nr; ++j) {
      if (iters_out) iters_out[s * B->nr + j] = h.it[j];
      if (relres_out) relres_out[s * B->nr + j] = h.ff[j] > 0 ? sqrt(h.rr[j] / h.ff[j]) : sqrt(h.rr[j]);
      if (h.status[j] == AMG_ERR_NOT_SPD && worst == AMG_OK) worst = AMG_ERR_NOT_SPD;
      if (h.rr[j] > h.tol2[j] && worst == AMG_OK) worst = AMG_ERR_NO_CONVERGENCE;
    }
  }
  if (worst != AMG_OK) return bfail(B, worst, "some load case did not reach rtol");
  B->err.clear();
  return AMG_OK;
}

}  // extern "C"
