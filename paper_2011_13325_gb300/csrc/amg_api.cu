// C ABI of libamg: context, hierarchy upload, single V-cycle steps, V-cycle,
// PCG.  See include/amg.h for the contract of every entry point.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

#include "amg_internal.h"
#include "setup_host.h"

namespace amg {

cudaError_t dalloc(void **p, size_t bytes) {
  *p = nullptr;
  return cudaMalloc(p, bytes > 0 ? bytes : 16);
}

void dfree(void *p) {
  if (p) cudaFree(p);
}

void free_bsr(DevBSR &m) {
  dfree(m.rowptr);
  dfree(m.colidx);
  dfree(m.v64);
  dfree(m.v32);
  dfree(m.v16);
  dfree(m.sell_ptr);
  dfree(m.sell_col);
  dfree(m.sell_perm);
  dfree(m.s64);
  dfree(m.s32);
  dfree(m.s16);
  dfree(m.sdf);
  m = DevBSR();
}

void free_levels(Ctx *c) {
  for (Level &L : c->levels) {
    free_bsr(L.A);
    free_bsr(L.P);
    free_bsr(L.R);
    void *ptrs[] = {L.minv64, L.minv32, L.b64, L.x64, L.t64, L.y64, L.b32, L.x32, L.t32, L.y32,
                    L.gs_colour, L.gs_rows, L.gs_sell_ptr, L.gs_sell_col, L.gs_sell_perm,
                    L.gs_sell_vals};
    for (void *p : ptrs) dfree(p);
  }
  c->levels.clear();
  dfree(c->cinv);
  c->cinv = nullptr;
  c->coarse_n = 0;
}

void free_pcg(Ctx *c) {
  double *bufs[] = {c->f, c->x, c->r, c->z, c->zold, c->p, c->q, c->partials};
  for (double *b : bufs) dfree(b);
  c->f = c->x = c->r = c->z = c->zold = c->p = c->q = c->partials = nullptr;
  dfree(c->st);
  c->st = nullptr;
  dfree(c->counter);
  c->counter = nullptr;
  dfree(c->pdf);
  c->pdf = nullptr;
  if (c->st_host) cudaFreeHost(c->st_host);
  c->st_host = nullptr;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->graph_def) cudaGraphDestroy(c->graph_def);
  c->graph = nullptr;
  c->graph_def = nullptr;
}

// ---------------------------------------------------------------------------
// V-cycle (Algorithm tg applied recursively)
// ---------------------------------------------------------------------------

static void *vb(Level &L, int prec, char which) {
  const bool d = prec == AMG_PREC_FP64;
  switch (which) {
    case 'b': return d ? (void *)L.b64 : (void *)L.b32;
    case 'x': return d ? (void *)L.x64 : (void *)L.x32;
    case 't': return d ? (void *)L.t64 : (void *)L.t32;
    default: return d ? (void *)L.y64 : (void *)L.y32;
  }
}

static const void *minv_of(const Level &L, int prec) {
  return prec == AMG_PREC_FP64 ? (const void *)L.minv64 : (const void *)L.minv32;
}

// Solve on level l: input b (level buffer or external), output y.  In the
// mixed precisions the finest level reads the FP64 residual r64 and writes
// the FP64 result z64 directly (casts fused into its first / last kernel).
static cudaError_t vcycle_level(Ctx *c, int l, const void *b, void *y, const double *r64 = nullptr,
                                double *z64 = nullptr) {
  const int prec = mat_prec(c, l);
  Level &L = c->levels[l];
  if (l == (int)c->levels.size() - 1) return launch_coarse_gemv(c, c->coarse_n, c->cinv, b, y, prec);
  Level &Cn = c->levels[l + 1];
  void *x = vb(L, prec, 'x');
  void *t = vb(L, prec, 't');
  const void *mi = minv_of(L, prec);
  if (c->smoother == AMG_SMOOTHER_HYBRID_GS) {
    const size_t n = (size_t)L.A.n_rows * L.k;
    const size_t w = prec == AMG_PREC_FP64 ? sizeof(double) : sizeof(float);
    if (r64) AMG_CUDA_TRY(launch_convert(c, n, r64, AMG_PREC_FP64, (void *)b, AMG_PREC_FP32_VCYCLE));
    // forward sweep from x = 0
    AMG_CUDA_TRY(cudaMemsetAsync(x, 0, n * w, c->stream));
    AMG_CUDA_TRY(launch_gs_sweep(c, L, prec, b, x, true));
    AMG_CUDA_TRY(launch_bsr(c, L.A, prec, SPMV_RESID, x, b, nullptr, t));
    AMG_CUDA_TRY(launch_bsr(c, L.R, prec, SPMV_SET, t, nullptr, nullptr, vb(Cn, prec, 'b')));
    AMG_CUDA_TRY(vcycle_level(c, l + 1, vb(Cn, prec, 'b'), vb(Cn, prec, 'y')));
    AMG_CUDA_TRY(launch_bsr(c, L.P, prec, SPMV_ADD, vb(Cn, prec, 'y'), nullptr, nullptr, x));
    // backward sweep (the adjoint of the forward one)
    AMG_CUDA_TRY(launch_gs_sweep(c, L, prec, b, x, false));
    if (z64) return launch_convert(c, n, x, AMG_PREC_FP32_VCYCLE, z64, AMG_PREC_FP64);
    return cudaMemcpyAsync(y, x, n * w, cudaMemcpyDeviceToDevice, c->stream);
  }
  // pre-smoothing from x = 0: x = M^+ b
  if (r64)
    AMG_CUDA_TRY(launch_blockdiag_entry(c, L.A.n_rows, L.k, L.minv32, r64, (float *)b, (float *)x));
  else
    AMG_CUDA_TRY(launch_blockdiag(c, L.A.n_rows, L.k, prec, mi, b, x));
  // residual t = b - A x
  AMG_CUDA_TRY(launch_bsr(c, L.A, prec, SPMV_RESID, x, b, nullptr, t));
  // restriction b_{l+1} = R t
  AMG_CUDA_TRY(launch_bsr(c, L.R, prec, SPMV_SET, t, nullptr, nullptr, vb(Cn, prec, 'b')));
  // coarse-grid correction
  AMG_CUDA_TRY(vcycle_level(c, l + 1, vb(Cn, prec, 'b'), vb(Cn, prec, 'y')));
  // prolongation x += P e
  AMG_CUDA_TRY(launch_bsr(c, L.P, prec, SPMV_ADD, vb(Cn, prec, 'y'), nullptr, nullptr, x));
  // post-smoothing y = x + M^+ (b - A x)
  if (z64)
    return launch_smooth_out64(c, L.A, prec, (const float *)x, (const float *)b, L.minv32, z64);
  return launch_bsr(c, L.A, prec, SPMV_SMOOTH, x, b, mi, y);
}

// One timed entry of amg_profile_vcycle: the kernel launch fn, repeated.
template <typename F>
static cudaError_t time_launch(Ctx *c, int reps, F fn, double *us) {
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

// Algorithmic bytes of one application of m: values + column indices + row
// pointers, the input vector once, the output once (twice when updated).
static double op_bytes(const DevBSR &m, int prec, double wv, int out_rw) {
  const double w = prec == AMG_PREC_FP64 ? 8.0 : prec == AMG_PREC_FP32_VCYCLE ? 4.0 : 2.0;
  return (double)m.nnzb * (m.br * m.bc * w + 4.0) + 4.0 * (m.n_rows + 1) +
         (double)m.n_cols * m.bc * wv + out_rw * (double)m.n_rows * m.br * wv;
}

cudaError_t vcycle_launch(Ctx *c, const double *r, double *z) {
  if (c->precision == AMG_PREC_FP64) return vcycle_level(c, 0, r, z);
  Level &L0 = c->levels[0];
  const size_t n = (size_t)L0.A.n_rows * L0.k;
  if (c->levels.size() == 1) {  // single level: the coarsest solve is FP64 anyway
    AMG_CUDA_TRY(launch_convert(c, n, r, AMG_PREC_FP64, L0.b32, AMG_PREC_FP32_VCYCLE));
    AMG_CUDA_TRY(vcycle_level(c, 0, L0.b32, L0.y32));
    return launch_convert(c, n, L0.y32, AMG_PREC_FP32_VCYCLE, z, AMG_PREC_FP64);
  }
  return vcycle_level(c, 0, L0.b32, L0.y32, r, z);
}

}  // namespace amg

using namespace amg;

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

static int fail(Ctx *c, int code, const std::string &msg) {
  c->err = msg;
  return code;
}

static int cuda_fail(Ctx *c, cudaError_t e, const char *where) {
  c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return AMG_ERR_CUDA;
}

#define CUDA_OR_FAIL(c, expr, where)              \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) return cuda_fail(c, _e, where); \
  } while (0)

static bool block_ok(int b) { return b == 1 || b == 2 || b == 3 || b == 6; }

static int validate_bsr(Ctx *c, const amg_bsr &m, const char *name) {
  char buf[256];
  if (m.n_rows < 0 || m.n_cols < 0 || m.nnzb < 0 || !block_ok(m.br) || !block_ok(m.bc)) {
    snprintf(buf, sizeof buf, "%s: bad sizes (n_rows %d n_cols %d br %d bc %d nnzb %lld)", name,
             m.n_rows, m.n_cols, m.br, m.bc, (long long)m.nnzb);
    return fail(c, AMG_ERR_ARG, buf);
  }
  if (!m.rowptr || (m.nnzb > 0 && (!m.colidx || !m.vals))) {
    snprintf(buf, sizeof buf, "%s: NULL array", name);
    return fail(c, AMG_ERR_ARG, buf);
  }
  if (m.rowptr[0] != 0 || (int64_t)m.rowptr[m.n_rows] != m.nnzb) {
    snprintf(buf, sizeof buf, "%s: rowptr[0] must be 0 and rowptr[n_rows] == nnzb", name);
    return fail(c, AMG_ERR_ARG, buf);
  }
  for (int i = 0; i < m.n_rows; ++i) {
    if (m.rowptr[i + 1] < m.rowptr[i]) {
      snprintf(buf, sizeof buf, "%s: rowptr decreases at row %d", name, i);
      return fail(c, AMG_ERR_ARG, buf);
    }
    for (int p = m.rowptr[i]; p < m.rowptr[i + 1]; ++p) {
      const int col = m.colidx[p];
      if (col < 0 || col >= m.n_cols || (p > m.rowptr[i] && col <= m.colidx[p - 1])) {
        snprintf(buf, sizeof buf, "%s: colidx out of range or unsorted in row %d", name, i);
        return fail(c, AMG_ERR_ARG, buf);
      }
    }
  }
  const size_t nv = (size_t)m.nnzb * m.br * m.bc;
  for (size_t i = 0; i < nv; ++i)
    if (!isfinite(m.vals[i])) {
      snprintf(buf, sizeof buf, "%s: non-finite value at %zu", name, i);
      return fail(c, AMG_ERR_ARG, buf);
    }
  return AMG_OK;
}

static cudaError_t upload_bsr(Ctx *c, DevBSR &d, int n_rows, int n_cols, int br, int bc,
                              int64_t nnzb, const int32_t *rp, const int32_t *ci,
                              const double *v) {
  free_bsr(d);
  d.n_rows = n_rows;
  d.n_cols = n_cols;
  d.br = br;
  d.bc = bc;
  d.nnzb = nnzb;
  AMG_CUDA_TRY(dalloc((void **)&d.rowptr, (size_t)(n_rows + 1) * sizeof(int)));
  AMG_CUDA_TRY(dalloc((void **)&d.colidx, (size_t)nnzb * sizeof(int)));
  AMG_CUDA_TRY(dalloc((void **)&d.v64, (size_t)nnzb * br * bc * sizeof(double)));
  AMG_CUDA_TRY(cudaMemcpyAsync(d.rowptr, rp, (size_t)(n_rows + 1) * sizeof(int),
                               cudaMemcpyHostToDevice, c->stream));
  if (nnzb > 0) {
    AMG_CUDA_TRY(cudaMemcpyAsync(d.colidx, ci, (size_t)nnzb * sizeof(int), cudaMemcpyHostToDevice,
                                 c->stream));
    AMG_CUDA_TRY(cudaMemcpyAsync(d.v64, v, (size_t)nnzb * br * bc * sizeof(double),
                                 cudaMemcpyHostToDevice, c->stream));
  }
  return cudaStreamSynchronize(c->stream);
}

// R = P^T with sorted columns (counting sort by block column, stable in the
// row index), block values transposed.
static cudaError_t upload_transpose(Ctx *c, DevBSR &R, const amg_bsr &P) {
  const int nr = P.n_cols, nc = P.n_rows, br = P.bc, bc = P.br;
  std::vector<int32_t> rp(nr + 1, 0), ci((size_t)P.nnzb);
  std::vector<double> v((size_t)P.nnzb * br * bc);
  for (int64_t p = 0; p < P.nnzb; ++p) rp[P.colidx[p] + 1]++;
  for (int i = 0; i < nr; ++i) rp[i + 1] += rp[i];
  std::vector<int32_t> fill(rp.begin(), rp.end() - 1);
  for (int i = 0; i < P.n_rows; ++i)
    for (int p = P.rowptr[i]; p < P.rowptr[i + 1]; ++p) {
      const int J = P.colidx[p];
      const int q = fill[J]++;
      ci[q] = i;
      const double *src = P.vals + (size_t)p * P.br * P.bc;
      double *dst = v.data() + (size_t)q * br * bc;
      for (int a = 0; a < P.br; ++a)
        for (int b = 0; b < P.bc; ++b) dst[b * bc + a] = src[a * P.bc + b];
    }
  return upload_bsr(c, R, nr, nc, br, bc, P.nnzb, rp.data(), ci.data(), v.data());
}

static cudaError_t alloc_level_vectors(Ctx *c, Level &L) {
  const size_t n = (size_t)L.A.n_rows * L.k;
  const size_t nb = (n ? n : 1);
  double **d[] = {&L.b64, &L.x64, &L.t64, &L.y64};
  for (double **p : d) {
    AMG_CUDA_TRY(dalloc((void **)p, nb * sizeof(double)));
    AMG_CUDA_TRY(cudaMemsetAsync(*p, 0, nb * sizeof(double), c->stream));
  }
  if (c->precision != AMG_PREC_FP64) {
    float **f[] = {&L.b32, &L.x32, &L.t32, &L.y32};
    for (float **p : f) {
      AMG_CUDA_TRY(dalloc((void **)p, nb * sizeof(float)));
      AMG_CUDA_TRY(cudaMemsetAsync(*p, 0, nb * sizeof(float), c->stream));
    }
  }
  return cudaSuccess;
}

static int check_ready(Ctx *c) {
  if (c->levels.empty()) return fail(c, AMG_ERR_STATE, "no hierarchy uploaded");
  return AMG_OK;
}

static int check_level(Ctx *c, int level, bool need_next) {
  int s = check_ready(c);
  if (s) return s;
  const int nl = (int)c->levels.size();
  if (level < 0 || level >= nl || (need_next && level >= nl - 1))
    return fail(c, AMG_ERR_ARG, "level out of range");
  return AMG_OK;
}

static int finish(Ctx *c, const char *where) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  c->err.clear();
  return AMG_OK;
}

// Kernel tuner of the upload (AMG_LAYOUT_AUTO): every V-cycle operator (but
// a square one with a SELL-32 copy) is applied with the warp-row, row-lane
// and block-lane kernels and, where it has one, its SELL-32 copy (one warm
// launch, then three timed) in the V-cycle precision, and keeps the
// fastest.  The kernels differ only in the order of the sums.
// Optional tuning cache: with AMG_TUNE_CACHE naming a file, choices found
// there (key: level, operator, rows, stored blocks, precision) are reused
// without timing and new ones are appended, so that a later process (e.g. one
// run under a profiler, where event timings are distorted) applies the same
// kernels.
static std::string tune_key(int l, char op, const DevBSR &m, int prec) {
  char k[128];
  snprintf(k, sizeof k, "L%d%c_%d_%lld_%dx%d_p%d", l, op, m.n_rows, (long long)m.nnzb, m.br, m.bc, prec);
  return k;
}

static std::vector<std::pair<std::string, int>> load_tune_cache(const char *path) {
  std::vector<std::pair<std::string, int>> out;
  FILE *f = path ? fopen(path, "r") : nullptr;
  if (!f) return out;
  char key[128];
  int k = 0;
  while (fscanf(f, "%127s %d", key, &k) == 2)
    if (k >= KERN_WARP_ROWS && k <= KERN_SELL_SPLIT) out.emplace_back(key, k);
  fclose(f);
  return out;
}

static cudaError_t tune_operators(Ctx *c) {
  if (c->layout_policy != AMG_LAYOUT_AUTO) return cudaSuccess;
  const char *cache_path = getenv("AMG_TUNE_CACHE");
  const auto cache = load_tune_cache(cache_path);
  std::vector<std::pair<std::string, int>> fresh;
  // (operator, its mode in the V-cycle): A residual, P prolongation-add,
  // R restriction
  std::vector<std::pair<DevBSR *, int>> ops;
  std::vector<int> op_prec;
  std::vector<std::string> keys;
  size_t nx = 0, ny = 0;
  for (int l = 0; l + 1 < (int)c->levels.size(); ++l) {
    Level &L = c->levels[l];
    const std::pair<DevBSR *, int> cand[3] = {{&L.A, SPMV_RESID}, {&L.P, SPMV_ADD}, {&L.R, SPMV_SET}};
    const char names[3] = {'A', 'P', 'R'};
    for (int i = 0; i < 3; ++i) {
      DevBSR *m = cand[i].first;
      // A_0 with a SELL-32 copy keeps it (it is also the CG operator, whose
      // kernels use that copy)
      if (!m->nnzb || (l == 0 && m == &L.A && m->sell_ptr)) continue;
      const std::string key = tune_key(l, names[i], *m, mat_prec(c, l));
      bool hit = false;
      for (const auto &kv : cache)
        if (kv.first == key && ((kv.second != KERN_SELL && kv.second != KERN_SELL_SPLIT) || m->sell_ptr) &&
            (kv.second != KERN_SELL_SPLIT || m->sell_perm)) {
          m->kern = kv.second;
          hit = true;
        }
      if (hit) continue;
      ops.push_back(cand[i]);
      op_prec.push_back(mat_prec(c, l));
      keys.push_back(key);
      nx = std::max(nx, (size_t)m->n_cols * m->bc);
      ny = std::max(ny, (size_t)m->n_rows * m->br);
    }
  }
  if (ops.empty()) return cudaSuccess;
  void *x = nullptr, *y = nullptr, *b = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = dalloc(&x, nx * sizeof(double));
  if (e == cudaSuccess) e = dalloc(&y, ny * sizeof(double));
  if (e == cudaSuccess) e = dalloc(&b, ny * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, nx * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(y, 0, ny * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b, 0, ny * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int kerns[5] = {KERN_SELL, KERN_SELL_SPLIT, KERN_WARP_ROWS, KERN_ROW_LANES, KERN_BLOCK_LANES};
  for (size_t i = 0; i < ops.size() && e == cudaSuccess; ++i) {
    DevBSR &m = *ops[i].first;
    const int mode = ops[i].second, prec = op_prec[i];
    float best = 1e30f;
    int pick = m.sell_ptr ? KERN_SELL : KERN_WARP_ROWS;
    for (int k : kerns) {
      if (k == KERN_SELL && !m.sell_ptr) continue;
      // the split form: sorted copies of rectangular operators (which never
      // run the smoothing mode)
      if (k == KERN_SELL_SPLIT && !(m.sell_ptr && m.sell_perm && (m.br != m.bc || m.n_rows != m.n_cols)))
        continue;
      m.kern = k;
      // the operator's own V-cycle mode; best of two timed triples
      e = launch_bsr(c, m, prec, mode, x, b, nullptr, y);
      for (int trial = 0; trial < 2 && e == cudaSuccess; ++trial) {
        e = cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_bsr(c, m, prec, mode, x, b, nullptr, y);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) {
          best = ms;
          pick = k;
        }
      }
    }
    m.kern = pick;
    fresh.emplace_back(keys[i], pick);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dfree(x);
  dfree(y);
  dfree(b);
  if (e == cudaSuccess && cache_path && !fresh.empty()) {
    FILE *f = fopen(cache_path, "a");
    if (f) {
      for (const auto &kv : fresh) fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
      fclose(f);
    }
  }
  return e;
}

// Smoothers, level vectors, low-precision copies, coarsest inverse, CG buffers.
static int finalize_hierarchy(Ctx *c) {
  for (int l = 0; l < (int)c->levels.size(); ++l) {
    Level &L = c->levels[l];
    const int precision = mat_prec(c, l);
    if (l + 1 < (int)c->levels.size() && c->smoother == AMG_SMOOTHER_HYBRID_GS)
      CUDA_OR_FAIL(c, gs_prepare(c, l), "colouring");
    if (l + 1 < (int)c->levels.size()) CUDA_OR_FAIL(c, smoother_setup(c, l), "smoother setup");
    CUDA_OR_FAIL(c, alloc_level_vectors(c, L), "level vectors");
    DevBSR *ops[] = {&L.A, &L.P, &L.R};
    for (DevBSR *m : ops)
      if (m->nnzb && want_sell(c, *m, m == &L.A && l > 0)) {
        CUDA_OR_FAIL(c, build_sell(c, *m, m == &L.A && l > 0), "sell layout");
        if (c->layout_policy == AMG_LAYOUT_SELL_SPLIT && m->sell_perm && m != &L.A) m->kern = KERN_SELL_SPLIT;
      }
    // the CG operator's double-float copy of A_0 (rows in order, 2x2 / 3x3)
    if (l == 0 && L.A.s64 && !L.A.sell_perm && (L.k == 1 || L.k == 2 || L.k == 3))
      CUDA_OR_FAIL(c, build_double_float(c, L.A), "double-float A_0");
    if (precision != AMG_PREC_FP64) {
      CUDA_OR_FAIL(c, make_low_precision(c, L.A, precision), "low precision A");
      if (L.P.nnzb) CUDA_OR_FAIL(c, make_low_precision(c, L.P, precision), "low precision P");
      if (L.R.nnzb) CUDA_OR_FAIL(c, make_low_precision(c, L.R, precision), "low precision R");
    }
    // hybrid Gauss-Seidel on a level 0 with a SELL-32 copy: A_0 again as
    // SELL-32 slices in colour order, so a class's sweep is one thread per row
    if (l == 0 && l + 1 < (int)c->levels.size() && c->smoother == AMG_SMOOTHER_HYBRID_GS &&
        L.A.sell_ptr && L.k <= 3)
      CUDA_OR_FAIL(c, gs_build_sell(c, l, precision), "colour-ordered sell layout");
  }
  CUDA_OR_FAIL(c, tune_operators(c), "kernel tuner");
  CUDA_OR_FAIL(c, coarse_setup(c), "coarse setup");
  CUDA_OR_FAIL(c, pcg_alloc(c), "pcg buffers");
  return finish(c, "upload");
}

// Level sink of the host setup: uploads A_0, then per level P_l, R_l and the
// device Galerkin product, handing A_{l+1} back to the host.
static double wall_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

namespace amg {
amgsetup::PairMeasure *make_device_pair_measure(Ctx *c);
cudaError_t device_coarse_topology(Ctx *c, const amgsetup::Topo &T, const std::vector<int> &agg, int nc,
                                   const std::vector<double> &xc, amgsetup::Topo &C);
cudaError_t device_prolongation(Ctx *c, int level, const amgsetup::Topo &T, const std::vector<int> &agg,
                                const std::vector<char> &dflag, int nc, const std::vector<double> &xc,
                                const std::vector<int> &rowmap, const std::vector<char> &bad, bool first,
                                const amgsetup::SetupParams &prm, amgsetup::HostBSR &Ph,
                                std::vector<char> &next_bad, int *handled);
}  // namespace amg

struct DeviceSink : amgsetup::LevelSink {
  Ctx *c;
  double device_s = 0.0, device_setup_s = 0.0;
  bool device = true, keep = false, device_pm = false;
  std::vector<char> p_on_device;  // per level: P_l already built on the device
  amgsetup::PairMeasure *pm = nullptr;
  explicit DeviceSink(Ctx *cc) : c(cc) {}
  ~DeviceSink() override { delete pm; }
  bool device_stages() const override { return device; }
  amgsetup::PairMeasure *pair_measure() override {
    if (!device_pm) return nullptr;
    if (!pm) pm = make_device_pair_measure(c);
    return pm;
  }
  int coarse_topology(int level, const amgsetup::Topo &T, const std::vector<int> &agg, int nc,
                      const std::vector<double> &xc, amgsetup::Topo &out) override {
    const double t0 = wall_s();
    const cudaError_t e = device_coarse_topology(c, T, agg, nc, xc, out);
    device_setup_s += wall_s() - t0;
    if (e != cudaSuccess) return -1;
    if (keep) {
      if ((int)c->topo.size() < level + 2) c->topo.resize(level + 2);
      c->topo[level + 1] = out;
    }
    return 0;
  }
  int prolongation(int level, const amgsetup::HostBSR &A, const amgsetup::Topo &T,
                   const std::vector<int> &agg, const std::vector<char> &D, int nc,
                   const std::vector<double> &xc, const std::vector<int> &rowmap,
                   const std::vector<char> &bad, bool first, const amgsetup::SetupParams &prm,
                   amgsetup::HostBSR &P, std::vector<char> &next_bad, int *handled) override {
    (void)A;
    const double t0 = wall_s();
    if ((int)c->levels.size() < level + 2) c->levels.resize(level + 2);
    const cudaError_t e = device_prolongation(c, level, T, agg, D, nc, xc, rowmap, bad, first, prm, P,
                                              next_bad, handled);
    device_setup_s += wall_s() - t0;
    if (e != cudaSuccess) return -1;
    if ((int)p_on_device.size() < level + 1) p_on_device.resize(level + 1, 0);
    p_on_device[level] = *handled ? 1 : 0;
    return 0;
  }
  int first(const amgsetup::HostBSR &A) override {
    c->levels.clear();
    c->levels.resize(1);
    if (upload_bsr(c, c->levels[0].A, A.n_rows, A.n_cols, A.br, A.bc, (int64_t)A.colidx.size(),
                   A.rowptr.data(), A.colidx.data(), A.vals.data()) != cudaSuccess)
      return -1;
    c->levels[0].k = A.br;
    return 0;
  }
  int next(int level, const amgsetup::HostBSR &P, amgsetup::HostBSR &An) override {
    const double t0 = wall_s();
    const int rc = next_impl(level, P, An);
    device_s += wall_s() - t0;
    return rc;
  }
  int next_impl(int level, const amgsetup::HostBSR &P, amgsetup::HostBSR &An) {
    c->levels.resize(level + 2);
    Level &L = c->levels[level];
    amg_bsr pv = {P.n_rows, P.n_cols, P.br, P.bc, (int64_t)P.colidx.size(), P.rowptr.data(),
                  P.colidx.data(), P.vals.data()};
    const bool on_dev = level < (int)p_on_device.size() && p_on_device[level];
    if (!on_dev && upload_bsr(c, L.P, P.n_rows, P.n_cols, P.br, P.bc, pv.nnzb, P.rowptr.data(),
                              P.colidx.data(), P.vals.data()) != cudaSuccess)
      return -1;
    if (upload_transpose(c, L.R, pv) != cudaSuccess) return -1;
    if (galerkin_device(c, level) != cudaSuccess) return -1;
    const DevBSR &A = c->levels[level + 1].A;
    An.n_rows = A.n_rows;
    An.n_cols = A.n_cols;
    An.br = A.br;
    An.bc = A.bc;
    An.rowptr.resize(A.n_rows + 1);
    An.colidx.resize(A.nnzb);
    An.vals.resize((size_t)A.nnzb * A.br * A.bc);
    if (cudaMemcpy(An.rowptr.data(), A.rowptr, (A.n_rows + 1) * sizeof(int),
                   cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(An.colidx.data(), A.colidx, A.nnzb * sizeof(int), cudaMemcpyDeviceToHost) !=
            cudaSuccess ||
        cudaMemcpy(An.vals.data(), A.v64, An.vals.size() * sizeof(double),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
      return -1;
    return 0;
  }
};

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------

extern "C" {

int amg_create(amg_ctx **out, int device, void *cuda_stream) {
  if (!out) return AMG_ERR_ARG;
  *out = nullptr;
  amg_ctx *h = new amg_ctx();
  Ctx *c = &h->c;
  c->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      c->stream = (cudaStream_t)cuda_stream;
    } else {
      e = cudaStreamCreate(&c->stream);  // blocking: ordered with the legacy default stream
      c->own_stream = true;
    }
  }
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
  if (e != cudaSuccess) {
    delete h;
    return AMG_ERR_CUDA;
  }
  *out = h;
  return AMG_OK;
}

void amg_destroy(amg_ctx *h) {
  if (!h) return;
  Ctx *c = &h->c;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  free_pcg(c);
  free_levels(c);
  if (c->hbuf) cudaFreeHost(c->hbuf);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete h;
}

const char *amg_last_error(const amg_ctx *h) { return h ? h->c.err.c_str() : "NULL context"; }

int amg_profile_vcycle(amg_ctx *h, int reps, int32_t *level, int32_t *kind, double *us, double *bytes,
                       int max_entries, int32_t *n_entries) {
  if (!h || reps < 1 || max_entries < 0) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  if (c->levels.empty()) return fail(c, AMG_ERR_STATE, "amg_profile_vcycle: no hierarchy uploaded");
  CUDA_OR_FAIL(c, cudaSetDevice(c->device), "cudaSetDevice");
  const double wv = c->precision == AMG_PREC_FP64 ? 8.0 : 4.0;
  const int nl = (int)c->levels.size();
  int n = 0;
  auto put = [&](int l, int k, double t, double b) {
    if (n < max_entries) {
      if (level) level[n] = l;
      if (kind) kind[n] = k;
      if (us) us[n] = t;
      if (bytes) bytes[n] = b;
    }
    ++n;
  };
  for (int l = 0; l < nl; ++l) {
    Level &L = c->levels[l];
    const int prec = mat_prec(c, l);
    const double N = (double)L.A.n_rows * L.k;
    double t = 0.0;
    void *b = vb(L, prec, 'b'), *x = vb(L, prec, 'x'), *tt = vb(L, prec, 't'), *y = vb(L, prec, 'y');
    if (l == nl - 1) {
      CUDA_OR_FAIL(c, time_launch(c, reps, [&] { return launch_coarse_gemv(c, c->coarse_n, c->cinv, b, y, prec); }, &t),
                   "profile");
      put(l, 5, t, (double)c->coarse_n * c->coarse_n * 8.0 + 2.0 * c->coarse_n * wv);
      break;
    }
    Level &Cn = c->levels[l + 1];
    const void *mi = minv_of(L, prec);
    const bool entry = l == 0 && prec != AMG_PREC_FP64;  // FP64 residual in, FP64 z out
    const bool gs = c->smoother == AMG_SMOOTHER_HYBRID_GS;
    // a hybrid Gauss-Seidel sweep reads every block and writes x once
    const double gs_bytes = op_bytes(L.A, prec, wv, 1) + N * L.k * wv + N * wv;
    if (gs) {
      CUDA_OR_FAIL(c, time_launch(c, reps, [&] {
        cudaError_t e = cudaMemsetAsync(x, 0, (size_t)N * (size_t)wv, c->stream);
        return e == cudaSuccess ? launch_gs_sweep(c, L, prec, b, x, true) : e; }, &t), "profile");
      put(l, 0, t, gs_bytes);
    } else if (entry)
      CUDA_OR_FAIL(c, time_launch(c, reps, [&] {
        return launch_blockdiag_entry(c, L.A.n_rows, L.k, L.minv32, c->r, (float *)b, (float *)x); }, &t), "profile");
    else
      CUDA_OR_FAIL(c, time_launch(c, reps, [&] { return launch_blockdiag(c, L.A.n_rows, L.k, prec, mi, b, x); }, &t),
                   "profile");
    if (!gs) put(l, 0, t, N * L.k * wv + N * (entry ? 8.0 + 2 * wv : 2 * wv));
    CUDA_OR_FAIL(c, time_launch(c, reps, [&] { return launch_bsr(c, L.A, prec, SPMV_RESID, x, b, nullptr, tt); }, &t),
                 "profile");
    put(l, 1, t, op_bytes(L.A, prec, wv, 1) + N * wv);
    CUDA_OR_FAIL(c, time_launch(c, reps, [&] {
      return launch_bsr(c, L.R, prec, SPMV_SET, tt, nullptr, nullptr, vb(Cn, prec, 'b')); }, &t), "profile");
    put(l, 2, t, op_bytes(L.R, prec, wv, 1));
    CUDA_OR_FAIL(c, time_launch(c, reps, [&] {
      return launch_bsr(c, L.P, prec, SPMV_ADD, vb(Cn, prec, 'y'), nullptr, nullptr, x); }, &t), "profile");
    put(l, 3, t, op_bytes(L.P, prec, wv, 2));
    if (gs) {
      CUDA_OR_FAIL(c, time_launch(c, reps, [&] { return launch_gs_sweep(c, L, prec, b, x, false); }, &t),
                   "profile");
      put(l, 4, t, gs_bytes);
      continue;
    }
    if (entry)
      CUDA_OR_FAIL(c, time_launch(c, reps, [&] {
        return launch_smooth_out64(c, L.A, prec, (const float *)x, (const float *)b, L.minv32, c->z); }, &t),
                   "profile");
    else
      CUDA_OR_FAIL(c, time_launch(c, reps, [&] { return launch_bsr(c, L.A, prec, SPMV_SMOOTH, x, b, mi, y); }, &t),
                   "profile");
    put(l, 4, t, op_bytes(L.A, prec, wv, 0) + N * L.k * wv + N * wv + N * (entry ? 8.0 : wv));
  }
  if (n_entries) *n_entries = n;
  return finish(c, "profile");
}

const char *amg_describe(amg_ctx *h) {
  if (!h) return "";
  Ctx *c = &h->c;
  static const char *kname[3] = {"warp rows", "row lanes", "block lanes"};
  std::string d;
  char line[256];
  for (int l = 0; l < (int)c->levels.size(); ++l) {
    const Level &L = c->levels[l];
    const char *nm[3] = {"A", "P", "R"};
    const DevBSR *ops[3] = {&L.A, &L.P, &L.R};
    for (int i = 0; i < 3; ++i) {
      const DevBSR &m = *ops[i];
      if (!m.nnzb) continue;
      char k[96];
      if (m.sell_ptr && (m.kern == KERN_SELL || m.kern == KERN_SELL_SPLIT))
        snprintf(k, sizeof k, "SELL-32 (%s,%s %.0f%% of the slots filled)",
                 m.kern == KERN_SELL_SPLIT ? "warp per output row of a slice" : "thread per block row",
                 m.sell_perm ? " rows sorted by length," : "",
                 100.0 * (double)m.nnzb / (32.0 * (double)m.sell_slots));
      else
        snprintf(k, sizeof k, "%s", kname[m.kern >= 0 && m.kern < 3 ? m.kern : 0]);
      snprintf(line, sizeof line, "level %d %s: %d x %d blocks of %dx%d, %lld stored, %s\n", l, nm[i],
               m.n_rows, m.n_cols, m.br, m.bc, (long long)m.nnzb, k);
      d += line;
    }
  }
  if (!c->levels.empty()) {
    const DevBSR &A = c->levels[0].A;
    const bool df = (c->cg_op == AMG_CG_DOUBLE_FLOAT ||
                     (c->cg_op == AMG_CG_AUTO && c->precision != AMG_PREC_FP64)) &&
                    A.sdf && A.sell_ptr && !A.sell_perm;
    snprintf(line, sizeof line, "CG operator q = A_0 p: %s\n",
             df ? "double-float pairs on the FP32 pipe, SELL-32 (pcg_spmv_dot_sell_df_kernel)"
                : (A.sell_ptr && !A.sell_perm ? "FP64, SELL-32 (pcg_spmv_dot_sell_kernel)"
                                              : "FP64, warp rows (pcg_spmv_dot_kernel)"));
    d += line;
  }
  c->desc = d;
  return c->desc.c_str();
}

int amg_upload_hierarchy(amg_ctx *h, const amg_hierarchy *hier, int precision, int smoother) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  if (!hier || hier->n_levels < 1 || (hier->n_levels > 1 && !hier->P))
    return fail(c, AMG_ERR_ARG, "hierarchy: need n_levels >= 1 and P for n_levels > 1");
  if (precision < AMG_PREC_FP64 || precision > AMG_PREC_BF16_COARSE)
    return fail(c, AMG_ERR_ARG, "unknown precision");
  if (smoother != AMG_SMOOTHER_L1_JACOBI && smoother != AMG_SMOOTHER_HYBRID_GS)
    return fail(c, AMG_ERR_ARG, "unknown smoother");
  const amg_bsr &A0 = hier->A0;
  int s = validate_bsr(c, A0, "A0");
  if (s) return s;
  if (A0.br != A0.bc || A0.n_rows != A0.n_cols || (A0.br != 1 && A0.br != 2 && A0.br != 3))
    return fail(c, AMG_ERR_ARG, "A0 must be square with 1x1, 2x2 or 3x3 blocks");
  // every row of A0 needs a diagonal block with positive diagonal entries
  for (int i = 0; i < A0.n_rows; ++i) {
    const double *blk = nullptr;
    for (int p = A0.rowptr[i]; p < A0.rowptr[i + 1]; ++p)
      if (A0.colidx[p] == i) blk = A0.vals + (size_t)p * A0.br * A0.bc;
    bool ok = blk != nullptr;
    for (int r = 0; ok && r < A0.br; ++r) ok = blk[r * A0.bc + r] > 0.0;
    if (!ok) {
      char buf[128];
      snprintf(buf, sizeof buf, "A0: row %d has no positive diagonal block", i);
      return fail(c, AMG_ERR_NOT_SPD, buf);
    }
  }
  int rows = A0.n_rows, k = A0.br;
  for (int l = 0; l + 1 < hier->n_levels; ++l) {
    char name[32];
    snprintf(name, sizeof name, "P[%d]", l);
    s = validate_bsr(c, hier->P[l], name);
    if (s) return s;
    const amg_bsr &P = hier->P[l];
    if (P.n_rows != rows || P.br != k || (l > 0 && P.bc != k) || (l == 0 && P.bc < P.br))
      return fail(c, AMG_ERR_ARG, std::string(name) + ": dimensions do not match the level above");
    rows = P.n_cols;
    k = P.bc;
  }
  CUDA_OR_FAIL(c, cudaSetDevice(c->device), "cudaSetDevice");
  cudaStreamSynchronize(c->stream);
  free_pcg(c);
  free_levels(c);
  c->precision = precision;
  c->smoother = smoother;
  c->levels.resize(hier->n_levels);
  CUDA_OR_FAIL(c, upload_bsr(c, c->levels[0].A, A0.n_rows, A0.n_cols, A0.br, A0.bc, A0.nnzb,
                             A0.rowptr, A0.colidx, A0.vals), "upload A0");
  c->levels[0].k = A0.br;
  for (int l = 0; l + 1 < hier->n_levels; ++l) {
    const amg_bsr &P = hier->P[l];
    Level &L = c->levels[l];
    CUDA_OR_FAIL(c, upload_bsr(c, L.P, P.n_rows, P.n_cols, P.br, P.bc, P.nnzb, P.rowptr,
                               P.colidx, P.vals), "upload P");
    CUDA_OR_FAIL(c, upload_transpose(c, L.R, P), "upload R");
    CUDA_OR_FAIL(c, galerkin_device(c, l), "galerkin");
  }
  return finalize_hierarchy(c);
}

int amg_galerkin(amg_ctx *h, int level, amg_bsr_out *out) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_level(c, level, true);
  if (s) return s;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    cudaGraphDestroy(c->graph_def);
    c->graph = nullptr;
    c->graph_def = nullptr;
  }
  CUDA_OR_FAIL(c, galerkin_device(c, level), "galerkin");
  Level &Cl = c->levels[level + 1];
  if (want_sell(c, Cl.A, true)) CUDA_OR_FAIL(c, build_sell(c, Cl.A, true), "sell layout");
  if (c->precision != AMG_PREC_FP64)
    CUDA_OR_FAIL(c, make_low_precision(c, Cl.A, mat_prec(c, level + 1)), "low precision A");
  if (out) {
    if (!out->rowptr || (Cl.A.nnzb > 0 && (!out->colidx || !out->vals)))
      return fail(c, AMG_ERR_ARG, "amg_galerkin: NULL output array");
    out->n_rows = Cl.A.n_rows;
    out->n_cols = Cl.A.n_cols;
    out->br = Cl.A.br;
    out->bc = Cl.A.bc;
    out->nnzb = Cl.A.nnzb;
    return amg_download_matrix(h, level + 1, out->rowptr, out->colidx, out->vals);
  }
  return finish(c, "galerkin");
}

int amg_level_info(const amg_ctx *h, int level, int32_t *n_rows, int32_t *block, int64_t *nnzb_A,
                   int64_t *nnzb_P, int32_t *n_levels) {
  if (!h) return AMG_ERR_ARG;
  const Ctx *c = &h->c;
  if (n_levels) *n_levels = (int32_t)c->levels.size();
  if (c->levels.empty()) return AMG_ERR_STATE;
  if (level < 0 || level >= (int)c->levels.size()) return AMG_ERR_ARG;
  const Level &L = c->levels[level];
  if (n_rows) *n_rows = L.A.n_rows;
  if (block) *block = L.k;
  if (nnzb_A) *nnzb_A = L.A.nnzb;
  if (nnzb_P) *nnzb_P = L.P.nnzb;
  return AMG_OK;
}

int amg_download_matrix(amg_ctx *h, int level, int32_t *rowptr, int32_t *colidx, double *vals) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_level(c, level, false);
  if (s) return s;
  const DevBSR &A = c->levels[level].A;
  if (!rowptr || (A.nnzb > 0 && (!colidx || !vals)))
    return fail(c, AMG_ERR_ARG, "NULL output array");
  CUDA_OR_FAIL(c, cudaMemcpyAsync(rowptr, A.rowptr, (size_t)(A.n_rows + 1) * sizeof(int),
                                  cudaMemcpyDeviceToHost, c->stream), "download rowptr");
  if (A.nnzb > 0) {
    CUDA_OR_FAIL(c, cudaMemcpyAsync(colidx, A.colidx, (size_t)A.nnzb * sizeof(int),
                                    cudaMemcpyDeviceToHost, c->stream), "download colidx");
    CUDA_OR_FAIL(c, cudaMemcpyAsync(vals, A.v64, (size_t)A.nnzb * A.br * A.bc * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream), "download vals");
  }
  return finish(c, "download matrix");
}

int amg_download_smoother(amg_ctx *h, int level, double *minv) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_level(c, level, true);
  if (s) return s;
  if (!minv) return fail(c, AMG_ERR_ARG, "NULL output");
  const Level &L = c->levels[level];
  CUDA_OR_FAIL(c, cudaMemcpyAsync(minv, L.minv64, (size_t)L.A.n_rows * L.k * L.k * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream), "download smoother");
  return finish(c, "download smoother");
}

int amg_download_coarse_inverse(amg_ctx *h, double *cinv) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_ready(c);
  if (s) return s;
  if (!cinv) return fail(c, AMG_ERR_ARG, "NULL output");
  CUDA_OR_FAIL(c, cudaMemcpyAsync(cinv, c->cinv, (size_t)c->coarse_n * c->coarse_n * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream), "download coarse inverse");
  return finish(c, "download coarse inverse");
}

int amg_spmv(amg_ctx *h, int level, const double *x, double *y) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_level(c, level, false);
  if (s) return s;
  if (!x || !y) return fail(c, AMG_ERR_ARG, "NULL vector");
  CUDA_OR_FAIL(c, launch_bsr(c, c->levels[level].A, AMG_PREC_FP64, SPMV_SET, x, nullptr, nullptr, y),
               "spmv");
  return finish(c, "spmv");
}

int amg_residual(amg_ctx *h, int level, const double *b, const double *x, double *r) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_level(c, level, false);
  if (s) return s;
  if (!b || !x || !r) return fail(c, AMG_ERR_ARG, "NULL vector");
  CUDA_OR_FAIL(c, launch_bsr(c, c->levels[level].A, AMG_PREC_FP64, SPMV_RESID, x, b, nullptr, r),
               "residual");
  return finish(c, "residual");
}

int amg_smooth(amg_ctx *h, int level, const double *b, const double *x_in, double *x_out) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_level(c, level, true);
  if (s) return s;
  if (!b || !x_out || x_in == x_out) return fail(c, AMG_ERR_ARG, "bad vectors");
  Level &L = c->levels[level];
  if (!x_in)
    CUDA_OR_FAIL(c, launch_blockdiag(c, L.A.n_rows, L.k, AMG_PREC_FP64, L.minv64, b, x_out),
                 "smooth");
  else
    CUDA_OR_FAIL(c, launch_bsr(c, L.A, AMG_PREC_FP64, SPMV_SMOOTH, x_in, b, L.minv64, x_out),
                 "smooth");
  return finish(c, "smooth");
}

int amg_restrict(amg_ctx *h, int level, const double *r, double *bc) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_level(c, level, true);
  if (s) return s;
  if (!r || !bc) return fail(c, AMG_ERR_ARG, "NULL vector");
  CUDA_OR_FAIL(c, launch_bsr(c, c->levels[level].R, AMG_PREC_FP64, SPMV_SET, r, nullptr, nullptr, bc),
               "restrict");
  return finish(c, "restrict");
}

int amg_prolong_add(amg_ctx *h, int level, const double *ec, double *x) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_level(c, level, true);
  if (s) return s;
  if (!ec || !x) return fail(c, AMG_ERR_ARG, "NULL vector");
  CUDA_OR_FAIL(c, launch_bsr(c, c->levels[level].P, AMG_PREC_FP64, SPMV_ADD, ec, nullptr, nullptr, x),
               "prolong");
  return finish(c, "prolong");
}

int amg_coarse_solve(amg_ctx *h, const double *b, double *x) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_ready(c);
  if (s) return s;
  if (!b || !x) return fail(c, AMG_ERR_ARG, "NULL vector");
  CUDA_OR_FAIL(c, launch_coarse_gemv(c, c->coarse_n, c->cinv, b, x, AMG_PREC_FP64), "coarse solve");
  return finish(c, "coarse solve");
}

int amg_vcycle(amg_ctx *h, const double *r, double *z, int nrhs) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_ready(c);
  if (s) return s;
  if (!r || !z || nrhs < 1) return fail(c, AMG_ERR_ARG, "bad vectors / nrhs");
  const size_t n = (size_t)c->levels[0].A.n_rows * c->levels[0].k;
  for (int i = 0; i < nrhs; ++i)
    CUDA_OR_FAIL(c, vcycle_launch(c, r + i * n, z + i * n), "vcycle");
  return finish(c, "vcycle");
}

// Build the PCG graph; if the capture or instantiation refuses the
// programmatic launches, rebuild it with plain launches.
static cudaError_t ensure_pcg_graph(Ctx *c) {
  if (!c->pcg_graph || c->graph) return cudaSuccess;
  cudaError_t e = pcg_build_graph(c);
  if (e == cudaSuccess || !c->pdl) return e;
  (void)cudaGetLastError();
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->graph_def) cudaGraphDestroy(c->graph_def);
  c->graph = nullptr;
  c->graph_def = nullptr;
  c->pdl = false;
  return pcg_build_graph(c);
}

static int pcg_one(Ctx *c, double rtol, int maxit, int *iters, double *relres) {
  c->st_host->rtol = rtol;
  c->st_host->maxit = maxit;
  c->st_host->flexible = (c->precision != AMG_PREC_FP64) ? 1 : 0;
  c->st_host->it = 0;
  c->st_host->status = 0;
  c->st_host->guard = 0;
  c->st_host->replace = 0;
  c->st_host->replaced = 0;
  CUDA_OR_FAIL(c, cudaMemcpyAsync(c->st, c->st_host, sizeof(PcgState), cudaMemcpyHostToDevice,
                                  c->stream), "pcg state");
  CUDA_OR_FAIL(c, cudaEventRecord(c->ev0, c->stream), "event");
  if (c->pcg_graph) {
    CUDA_OR_FAIL(c, cudaGraphLaunch(c->graph, c->stream), "pcg graph launch");
    CUDA_OR_FAIL(c, cudaEventRecord(c->ev1, c->stream), "event");
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->st_host, c->st, sizeof(PcgState), cudaMemcpyDeviceToHost,
                                    c->stream), "pcg state");
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream), "pcg sync");
  } else {
    CUDA_OR_FAIL(c, pcg_host_loop(c), "pcg host loop");
    CUDA_OR_FAIL(c, cudaEventRecord(c->ev1, c->stream), "event");
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream), "pcg sync");
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->last_ms += ms;
  const PcgState &st = *c->st_host;
  if (iters) *iters = st.it;
  if (relres) *relres = st.ff > 0 ? sqrt(st.rr / st.ff) : sqrt(st.rr);
  if (st.status == AMG_ERR_NOT_SPD) return fail(c, AMG_ERR_NOT_SPD, "CG breakdown: p^T A p <= 0 or non-finite");
  if (st.rr > st.tol2) return fail(c, AMG_ERR_NO_CONVERGENCE, "maxit reached before rtol");
  return AMG_OK;
}

int amg_pcg_solve(amg_ctx *h, const double *f, double *u, int nrhs, double rtol, int maxit,
                  int *iters, double *relres) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_ready(c);
  if (s) return s;
  if (!f || !u || nrhs < 1 || !(rtol >= 0.0) || maxit < 0)
    return fail(c, AMG_ERR_ARG, "bad arguments");
  if (c->levels[0].k < 1 || c->levels[0].k > 3) return fail(c, AMG_ERR_ARG, "A0 block size");
  CUDA_OR_FAIL(c, ensure_pcg_graph(c), "pcg graph");
  const size_t n = (size_t)c->levels[0].A.n_rows * c->levels[0].k;
  c->last_ms = 0.f;
  int worst = AMG_OK;
  for (int i = 0; i < nrhs; ++i) {
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->f, f + i * n, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                    c->stream), "copy f");
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->x, u + i * n, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                    c->stream), "copy u");
    s = pcg_one(c, rtol, maxit, iters ? iters + i : nullptr, relres ? relres + i : nullptr);
    CUDA_OR_FAIL(c, cudaMemcpyAsync(u + i * n, c->x, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                    c->stream), "copy u back");
    if (s != AMG_OK && worst == AMG_OK) worst = s;
  }
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream), "pcg sync");
  if (worst != AMG_OK) return worst;
  c->err.clear();
  return AMG_OK;
}

int amg_pcg_solve_host(amg_ctx *h, const double *f, double *u, int nrhs, double rtol, int maxit,
                       int *iters, double *relres) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_ready(c);
  if (s) return s;
  if (!f || !u || nrhs < 1 || !(rtol >= 0.0) || maxit < 0)
    return fail(c, AMG_ERR_ARG, "bad arguments");
  CUDA_OR_FAIL(c, ensure_pcg_graph(c), "pcg graph");
  const size_t n = (size_t)c->levels[0].A.n_rows * c->levels[0].k;
  c->last_ms = 0.f;
  int worst = AMG_OK;
  for (int i = 0; i < nrhs; ++i) {
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->f, f + i * n, n * sizeof(double), cudaMemcpyHostToDevice,
                                    c->stream), "copy f");
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->x, u + i * n, n * sizeof(double), cudaMemcpyHostToDevice,
                                    c->stream), "copy u");
    s = pcg_one(c, rtol, maxit, iters ? iters + i : nullptr, relres ? relres + i : nullptr);
    CUDA_OR_FAIL(c, cudaMemcpyAsync(u + i * n, c->x, n * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream), "copy u back");
    if (s != AMG_OK && worst == AMG_OK) worst = s;
  }
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream), "pcg sync");
  if (worst != AMG_OK) return worst;
  c->err.clear();
  return AMG_OK;
}

int amg_setup_times(const amg_ctx *h, double *times4) {
  if (!h || !times4) return AMG_ERR_ARG;
  for (int i = 0; i < 4; ++i) times4[i] = h->c.setup_times[i];
  return AMG_OK;
}

int amg_setup_device_split(const amg_ctx *h, double *galerkin_s, double *topology_prolongation_s,
                           double *pair_measure_s) {
  if (!h) return AMG_ERR_ARG;
  if (galerkin_s) *galerkin_s = h->c.setup_times[1] - h->c.setup_times[4];
  if (topology_prolongation_s) *topology_prolongation_s = h->c.setup_times[4];
  if (pair_measure_s) *pair_measure_s = h->c.setup_times[5];
  return AMG_OK;
}

int amg_download_topology(amg_ctx *h, int level, int32_t *n_vertices, int64_t *n_edges, int32_t *k,
                          int32_t *ei, int32_t *ej, double *E, double *M, double *pos) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  if (level < 1 || level >= (int)c->topo.size() || c->topo[level].n == 0)
    return fail(c, AMG_ERR_STATE, "amg_download_topology: no kept topology of that level (amg_setup "
                                  "with keep_topology and the device stages)");
  const amgsetup::Topo &T = c->topo[level];
  const size_t kk = (size_t)T.k * T.k;
  if (n_vertices) *n_vertices = T.n;
  if (n_edges) *n_edges = (int64_t)T.ei.size();
  if (k) *k = T.k;
  if (ei) std::copy(T.ei.begin(), T.ei.end(), ei);
  if (ej) std::copy(T.ej.begin(), T.ej.end(), ej);
  if (E) std::copy(T.E.begin(), T.E.begin() + T.ei.size() * kk, E);
  if (M) std::copy(T.M.begin(), T.M.begin() + (size_t)T.n * kk, M);
  if (pos) std::copy(T.pos.begin(), T.pos.end(), pos);
  c->err.clear();
  return AMG_OK;
}

int amg_probe_fma_rate(amg_ctx *h, double *fp64_gflops, double *fp32_gflops) {
  if (!h || !fp64_gflops || !fp32_gflops) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  CUDA_OR_FAIL(c, probe_fma(c, fp64_gflops, fp32_gflops), "fma probe");
  return finish(c, "fma probe");
}

int amg_set_layout_policy(amg_ctx *h, int policy) {
  if (!h) return AMG_ERR_ARG;
  if (policy < AMG_LAYOUT_AUTO || policy > AMG_LAYOUT_SELL_SPLIT)
    return fail(&h->c, AMG_ERR_ARG, "unknown layout policy");
  h->c.layout_policy = policy;
  return AMG_OK;
}

int amg_set_launch_overlap(amg_ctx *h, int enable) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream), "sync");
  c->pdl = enable != 0;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->graph_def) cudaGraphDestroy(c->graph_def);
  c->graph = nullptr;
  c->graph_def = nullptr;
  c->err.clear();
  return AMG_OK;
}

int amg_set_cg_operator(amg_ctx *h, int mode) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  if (mode != AMG_CG_FP64 && mode != AMG_CG_DOUBLE_FLOAT && mode != AMG_CG_AUTO)
    return fail(c, AMG_ERR_ARG, "unknown CG operator mode");
  if (mode != c->cg_op) {
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream), "sync");
    c->cg_op = mode;
    // the PCG graph holds the operator's kernel: rebuilt at the next solve
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph_def) cudaGraphDestroy(c->graph_def);
    c->graph = nullptr;
    c->graph_def = nullptr;
  }
  c->err.clear();
  return AMG_OK;
}

int amg_set_pcg_graph(amg_ctx *h, int enable) {
  if (!h) return AMG_ERR_ARG;
  h->c.pcg_graph = enable != 0;
  return AMG_OK;
}

int amg_last_solve_ms(const amg_ctx *h, float *ms) {
  if (!h || !ms) return AMG_ERR_ARG;
  *ms = h->c.last_ms;
  return AMG_OK;
}

void amg_default_setup_params(amg_setup_params *p) {
  if (!p) return;
  const amgsetup::SetupParams d;
  p->sigma = d.sigma;
  p->delta = d.delta;
  p->passes_first = d.passes_first;
  p->passes_later = d.passes_later;
  p->omega = d.omega;
  p->cap_S_first = d.cap_S_first;
  p->cap_S_later = d.cap_S_later;
  p->cap_A = d.cap_A;
  p->coarse_max = d.coarse_max;
  p->min_ratio = d.min_ratio;
  p->max_levels = d.max_levels;
  p->host_threads = d.host_threads;
  p->device_setup = 1;
  p->keep_topology = 0;
  p->scalar_only = 0;
  p->device_pair_measure = 0;
}

int amg_setup(amg_ctx *h, const amg_problem *prob, const amg_setup_params *params, int precision,
              int smoother) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  if (!prob || (prob->dim != 2 && prob->dim != 3) || prob->n_vertices < 1 || !prob->coords)
    return fail(c, AMG_ERR_ARG, "amg_setup: bad problem");
  if (precision < AMG_PREC_FP64 || precision > AMG_PREC_BF16_COARSE)
    return fail(c, AMG_ERR_ARG, "unknown precision");
  if (smoother != AMG_SMOOTHER_L1_JACOBI && smoother != AMG_SMOOTHER_HYBRID_GS)
    return fail(c, AMG_ERR_ARG, "unknown smoother");
  const amg_bsr &A = prob->A_full;
  int s = validate_bsr(c, A, "A_full");
  if (s) return s;
  const int blk = prob->block ? prob->block : prob->dim;
  if (blk != 1 && blk != prob->dim) return fail(c, AMG_ERR_ARG, "amg_setup: block must be 0, 1 or dim");
  if (A.n_rows != prob->n_vertices || A.n_cols != A.n_rows || A.br != blk || A.bc != blk)
    return fail(c, AMG_ERR_ARG, "A_full must be n_vertices x n_vertices with block x block blocks");
  amgsetup::SetupParams prm;
  if (params) {
    prm.sigma = params->sigma;
    prm.delta = params->delta;
    prm.passes_first = params->passes_first;
    prm.passes_later = params->passes_later;
    prm.omega = params->omega;
    prm.cap_S_first = params->cap_S_first;
    prm.cap_S_later = params->cap_S_later;
    prm.cap_A = params->cap_A;
    prm.coarse_max = params->coarse_max;
    prm.min_ratio = params->min_ratio;
    prm.max_levels = params->max_levels;
    prm.host_threads = params->host_threads;
    prm.scalar_only = params->scalar_only != 0;
  }
  if (!(prm.sigma > 0) || prm.passes_first < 1 || prm.passes_later < 1 || prm.cap_A < 1 ||
      prm.max_levels < 1 || prm.host_threads < 0)
    return fail(c, AMG_ERR_ARG, "amg_setup: bad parameters");
  CUDA_OR_FAIL(c, cudaSetDevice(c->device), "cudaSetDevice");
  cudaStreamSynchronize(c->stream);
  free_pcg(c);
  free_levels(c);
  c->precision = precision;
  c->smoother = smoother;
  amgsetup::Problem pb;
  pb.dim = prob->dim;
  pb.block = blk;
  pb.n_vertices = prob->n_vertices;
  pb.coords = prob->coords;
  pb.dirichlet = prob->dirichlet;
  pb.rowptr = A.rowptr;
  pb.colidx = A.colidx;
  pb.vals = A.vals;
  DeviceSink sink(c);
  sink.device = (!params || params->device_setup != 0) && blk != 1;
  sink.keep = params && params->keep_topology != 0;
  sink.device_pm = params && params->device_pair_measure != 0;
  c->topo.clear();
  c->setup_times[5] = 0.0;
  std::string err;
  const double t0 = wall_s();
  if (amgsetup::build_levels(pb, prm, sink, err) != 0) {
    free_levels(c);
    return fail(c, AMG_ERR_CUDA, "amg_setup: " + err);
  }
  const double t1 = wall_s();
  const int rc = finalize_hierarchy(c);
  const double t2 = wall_s();
  c->setup_times[0] = (t1 - t0) - sink.device_s - sink.device_setup_s;
  c->setup_times[1] = sink.device_s + sink.device_setup_s;
  c->setup_times[2] = t2 - t1;
  c->setup_times[3] = t2 - t0;
  c->setup_times[4] = sink.device_setup_s;
  return rc;
}

int amg_prolongation_info(const amg_ctx *h, int level, int32_t *n_rows, int32_t *n_cols,
                          int32_t *br, int32_t *bc, int64_t *nnzb) {
  if (!h) return AMG_ERR_ARG;
  const Ctx *c = &h->c;
  if (level < 0 || level + 1 >= (int)c->levels.size()) return AMG_ERR_ARG;
  const DevBSR &P = c->levels[level].P;
  if (n_rows) *n_rows = P.n_rows;
  if (n_cols) *n_cols = P.n_cols;
  if (br) *br = P.br;
  if (bc) *bc = P.bc;
  if (nnzb) *nnzb = P.nnzb;
  return AMG_OK;
}

int amg_download_prolongation(amg_ctx *h, int level, int32_t *rowptr, int32_t *colidx,
                              double *vals) {
  if (!h) return AMG_ERR_ARG;
  Ctx *c = &h->c;
  int s = check_level(c, level, true);
  if (s) return s;
  const DevBSR &P = c->levels[level].P;
  if (!rowptr || (P.nnzb > 0 && (!colidx || !vals))) return fail(c, AMG_ERR_ARG, "NULL output array");
  CUDA_OR_FAIL(c, cudaMemcpyAsync(rowptr, P.rowptr, (size_t)(P.n_rows + 1) * sizeof(int),
                                  cudaMemcpyDeviceToHost, c->stream), "download P");
  if (P.nnzb > 0) {
    CUDA_OR_FAIL(c, cudaMemcpyAsync(colidx, P.colidx, (size_t)P.nnzb * sizeof(int),
                                    cudaMemcpyDeviceToHost, c->stream), "download P");
    CUDA_OR_FAIL(c, cudaMemcpyAsync(vals, P.v64, (size_t)P.nnzb * P.br * P.bc * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream), "download P");
  }
  return finish(c, "download P");
}

}  // extern "C"
