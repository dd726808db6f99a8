// Batched solve: many independent systems (each an amg_ctx with its own
// hierarchy), each with NR load cases, solved by one launch of one CUDA
// graph.  The systems advance in lockstep: every step of the V-cycle (per
// level) and of CG (Sec. 7) is ONE grouped launch over all systems
// (batch_kernels.cu), inside one device-side while loop.  Systems and load
// cases that have converged are frozen: their blocks return at once and their
// iteration counts stop.  The block-sparse tile of every grouped product
// (lanes per block row, warps per block) is picked at creation by timing the
// candidates on the batch's own operators.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "amg_internal.h"
#include "batch_kernels.h"

namespace amg {

enum StageKind { ST_SPMM, ST_DIAG, ST_COARSE, ST_DOTS, ST_UPD_P, ST_UPD_XR, ST_PACK, ST_UNPACK, ST_GUARD };

struct SpmmOp {
  const DevBSR *A;
  const void *vals, *x, *b, *minv;
  void *y;
  int sys;
  const void *svals;  // SELL-32 values in the operator's precision (NULL: none)
};

struct Stage {
  int kind = ST_SPMM;
  std::string name;
  // products
  SpmmKey key{};
  int lpr = 32, wpb = 8;
  std::vector<SpmmOp> ops;
  // block diagonal
  int k = 0, dkind = 0;
  // coarsest
  bool c64 = true;
  // inner products
  int phase = 0;
  bool init = false;
  // item tables (host) and where they sit in the device buffer
  std::vector<SpmmItem> sp;
  std::vector<DiagItem> dg;
  std::vector<CoarseItem> co;
  std::vector<SysItem> si;
  size_t off = 0;
  int n_items = 0, grid = 0;
  float us = 0.f;  // tuned time of one launch
};

struct SysVec {
  std::vector<void *> lb, lx, lt, ly;  // V-cycle level vectors (n_l * NR)
};

struct Batch {
  int device = 0, nr = 1, precision = 0, num_sms = 0;
  bool df = false;  // CG product q = A_0 p in double-float arithmetic
  cudaStream_t stream = nullptr;
  std::vector<Ctx *> ctx;
  std::vector<GSys> gsh;  // host copy of the per-system descriptors
  std::vector<SysVec> vec;
  GSys *gs = nullptr;
  McgState *st = nullptr, *st_host = nullptr;
  BatchLoop *loop = nullptr, *loop_host = nullptr;
  unsigned char *items = nullptr;
  size_t items_bytes = 0;
  std::vector<Stage> init, body, tail;
  size_t total = 0;  // stacked length of f / u
  double *fin = nullptr, *uio = nullptr;
  cudaGraph_t graph_def = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err, describe;
};

static int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// item tables
// ---------------------------------------------------------------------------
static void build_spmm_items(Stage &S) {
  S.sp.clear();
  const int g = S.lpr < 0 ? -S.lpr : S.lpr;  // lanes per row (block lanes: -g)
  const int rpb = g ? S.wpb * (32 / g) : 0;
  int first = 0;
  for (const SpmmOp &o : S.ops) {
    SpmmItem it{};
    it.rowptr = o.A->rowptr;
    it.colidx = o.A->colidx;
    it.vals = o.vals;
    it.x = o.x;
    it.b = o.b;
    it.minv = o.minv;
    it.y = o.y;
    it.n_rows = o.A->n_rows;
    it.sys = o.sys;
    it.first_block = first;
    it.sell_ptr = o.A->sell_ptr;
    it.sell_col = o.A->sell_col;
    it.sell_perm = o.A->sell_perm;
    it.svals = o.svals;
    it.n_slices = o.A->n_slices;
    it.df_exp = o.A->df_exp;
    first += S.lpr ? cdiv(o.A->n_rows, rpb) : cdiv(o.A->n_slices, S.wpb);
    S.sp.push_back(it);
  }
  S.n_items = (int)S.sp.size();
  S.grid = first;
}

static size_t item_bytes(const Stage &S) {
  switch (S.kind) {
    case ST_SPMM: return S.sp.size() * sizeof(SpmmItem);
    case ST_DIAG: return S.dg.size() * sizeof(DiagItem);
    case ST_COARSE: return S.co.size() * sizeof(CoarseItem);
    case ST_GUARD: return 0;
    default: return S.si.size() * sizeof(SysItem);
  }
}

static const void *item_host(const Stage &S) {
  switch (S.kind) {
    case ST_SPMM: return S.sp.data();
    case ST_DIAG: return S.dg.data();
    case ST_COARSE: return S.co.data();
    case ST_GUARD: return nullptr;
    default: return S.si.data();
  }
}

// products of one logical step, split into one stage per block shape
static void add_spmm(std::vector<Stage> &out, const std::string &name, const std::vector<SpmmOp> &ops,
                     int mode, int vt, int to64) {
  std::vector<std::pair<int, int>> shapes;
  for (const SpmmOp &o : ops) {
    const std::pair<int, int> sh(o.A->br, o.A->bc);
    if (std::find(shapes.begin(), shapes.end(), sh) == shapes.end()) shapes.push_back(sh);
  }
  for (const auto &sh : shapes) {
    Stage S;
    S.kind = ST_SPMM;
    S.name = name + " " + std::to_string(sh.first) + "x" + std::to_string(sh.second);
    S.key = SpmmKey{sh.first, sh.second, vt, mode, to64};
    for (const SpmmOp &o : ops)
      if (o.A->br == sh.first && o.A->bc == sh.second && o.A->n_rows > 0) S.ops.push_back(o);
    if (S.ops.empty()) continue;
    build_spmm_items(S);
    out.push_back(std::move(S));
  }
}

static Stage sys_stage(const Batch *B, int kind, const std::string &name, bool reduction) {
  Stage S;
  S.kind = kind;
  S.name = name;
  int first = 0;
  for (int s = 0; s < (int)B->gsh.size(); ++s) {
    S.si.push_back(SysItem{s, first});
    first += reduction ? B->gsh[s].red_blocks : cdiv((long)B->gsh[s].n, 256);
  }
  S.n_items = (int)S.si.size();
  S.grid = first;
  return S;
}

static const void *vals_of(const DevBSR &A, int prec) {
  return prec == AMG_PREC_FP64 ? (const void *)A.v64
                               : prec == AMG_PREC_FP32_VCYCLE ? (const void *)A.v32 : (const void *)A.v16;
}
static const void *svals_of(const DevBSR &A, int prec) {
  if (!A.sell_ptr) return nullptr;
  return prec == AMG_PREC_FP64 ? (const void *)A.s64
                               : prec == AMG_PREC_FP32_VCYCLE ? (const void *)A.s32 : (const void *)A.s16;
}

// the stages of init (r = f - A x), body (one PCG iteration with the
// V-cycle) and tail (unpack)
static void build_stages(Batch *B) {
  const int ns = (int)B->ctx.size(), prec = B->precision;
  const bool f64 = prec == AMG_PREC_FP64;
  // init
  B->init.push_back(sys_stage(B, ST_PACK, "pack f, u", false));
  {
    std::vector<SpmmOp> ops;
    for (int s = 0; s < ns; ++s) {
      const DevBSR &A = B->ctx[s]->levels[0].A;
      ops.push_back(SpmmOp{&A, A.v64, B->gsh[s].x, B->gsh[s].f, nullptr, B->gsh[s].r, s, svals_of(A, 0)});
    }
    add_spmm(B->init, "r = f - A_0 x", ops, SPMV_RESID, 0, 0);
  }
  {
    Stage S = sys_stage(B, ST_DOTS, "r.r, f.f", true);
    S.phase = PH_INIT;
    B->init.push_back(std::move(S));
  }
  {
    Stage S;
    S.kind = ST_GUARD;
    S.name = "loop decision (initial)";
    S.init = true;
    B->init.push_back(std::move(S));
  }
  // body: V-cycle, lockstep over levels
  int lmax = 0;
  for (Ctx *c : B->ctx) lmax = std::max(lmax, (int)c->levels.size());
  auto bvec = [&](int s, int l) -> const void * {  // right-hand side of level l
    if (l > 0) return B->vec[s].lb[l];
    return f64 ? (const void *)B->gsh[s].r : B->vec[s].lb[0];
  };
  const char *pn = f64 ? "" : " (low precision)";
  for (int l = 0; l < lmax; ++l) {
    const std::string ls = "level " + std::to_string(l);
    // x_l = M_l^+ b_l (level 0 reads the FP64 residual, keeps its cast copy)
    std::vector<std::pair<int, DiagItem>> dg;
    std::vector<SpmmOp> resid, restr;
    std::vector<CoarseItem> crs64, crs32;
    for (int s = 0; s < ns; ++s) {
      Ctx *c = B->ctx[s];
      const int Ls = (int)c->levels.size();
      if (l < Ls - 1) {
        const Level &L = c->levels[l];
        DiagItem d{};
        d.minv = f64 ? (const void *)L.minv64 : (const void *)L.minv32;
        d.bin = l == 0 ? (const void *)B->gsh[s].r : B->vec[s].lb[l];
        d.bcopy = (l == 0 && !f64) ? B->vec[s].lb[0] : nullptr;
        d.y = B->vec[s].lx[l];
        d.n = L.A.n_rows;
        d.sys = s;
        dg.push_back({L.k, d});
        resid.push_back(SpmmOp{&L.A, vals_of(L.A, prec), B->vec[s].lx[l], bvec(s, l), nullptr,
                               B->vec[s].lt[l], s, svals_of(L.A, prec)});
        restr.push_back(SpmmOp{&L.R, vals_of(L.R, prec), B->vec[s].lt[l], nullptr, nullptr,
                               B->vec[s].lb[l + 1], s, svals_of(L.R, prec)});
      } else if (l == Ls - 1) {
        CoarseItem ci{};
        ci.cinv = c->cinv;
        ci.n = c->coarse_n;
        ci.sys = s;
        if (Ls == 1) {  // one-level hierarchy: the coarsest solve is the V-cycle
          ci.b = B->gsh[s].r;
          ci.y = B->gsh[s].z;
          crs64.push_back(ci);
        } else {
          ci.b = B->vec[s].lb[l];
          ci.y = B->vec[s].ly[l];
          (f64 ? crs64 : crs32).push_back(ci);
        }
      }
    }
    for (int k : {2, 3, 6}) {
      Stage S;
      S.kind = ST_DIAG;
      S.k = k;
      S.dkind = f64 ? 0 : (l == 0 ? 1 : 2);
      S.name = ls + " x = M^+ b " + std::to_string(k) + "x" + std::to_string(k) + pn;
      int first = 0;
      for (auto &pr : dg)
        if (pr.first == k) {
          DiagItem d = pr.second;
          d.first_block = first;
          first += cdiv(d.n, 128);
          S.dg.push_back(d);
        }
      if (S.dg.empty()) continue;
      S.n_items = (int)S.dg.size();
      S.grid = first;
      B->body.push_back(std::move(S));
    }
    add_spmm(B->body, ls + " t = b - A x" + pn, resid, SPMV_RESID, prec, 0);
    add_spmm(B->body, ls + " b_c = R t" + pn, restr, SPMV_SET, prec, 0);
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<CoarseItem> &cv = pass == 0 ? crs64 : crs32;
      if (cv.empty()) continue;
      Stage S;
      S.kind = ST_COARSE;
      S.c64 = pass == 0;
      S.name = ls + " coarsest y = C^-1 b" + (pass == 0 ? "" : pn);
      int first = 0;
      for (CoarseItem ci : cv) {
        ci.first_block = first;
        first += cdiv(ci.n, 8);
        S.co.push_back(ci);
      }
      S.n_items = (int)S.co.size();
      S.grid = first;
      B->body.push_back(std::move(S));
    }
  }
  for (int l = lmax - 2; l >= 0; --l) {
    const std::string ls = "level " + std::to_string(l);
    std::vector<SpmmOp> prol, smooth;
    for (int s = 0; s < ns; ++s) {
      Ctx *c = B->ctx[s];
      if (l >= (int)c->levels.size() - 1) continue;
      const Level &L = c->levels[l];
      prol.push_back(SpmmOp{&L.P, vals_of(L.P, prec), B->vec[s].ly[l + 1], nullptr, nullptr,
                            B->vec[s].lx[l], s, svals_of(L.P, prec)});
      smooth.push_back(SpmmOp{&L.A, vals_of(L.A, prec), B->vec[s].lx[l], bvec(s, l),
                              f64 ? (const void *)L.minv64 : (const void *)L.minv32,
                              l == 0 ? (void *)B->gsh[s].z : B->vec[s].ly[l], s,
                              svals_of(L.A, prec)});
    }
    add_spmm(B->body, ls + " x += P y_c" + pn, prol, SPMV_ADD, prec, 0);
    add_spmm(B->body, ls + " y = x + M^+(b - A x)" + pn, smooth, SPMV_SMOOTH, prec,
             (l == 0 && !f64) ? 1 : 0);
  }
  // body: CG
  {
    Stage S = sys_stage(B, ST_DOTS, "rho = r.z", true);
    S.phase = PH_RHO;
    B->body.push_back(std::move(S));
  }
  B->body.push_back(sys_stage(B, ST_UPD_P, "p = z + beta p", false));
  {
    std::vector<SpmmOp> ops;
    for (int s = 0; s < ns; ++s) {
      const DevBSR &A = B->ctx[s]->levels[0].A;
      if (B->df)
        ops.push_back(SpmmOp{&A, A.v64, B->gsh[s].pdf, nullptr, nullptr, B->gsh[s].q, s, A.sdf});
      else
        ops.push_back(SpmmOp{&A, A.v64, B->gsh[s].p, nullptr, nullptr, B->gsh[s].q, s, svals_of(A, 0)});
    }
    if (B->df)
      add_spmm(B->body, "q = A_0 p (double-float)", ops, SPMV_SET, 3, 0);
    else
      add_spmm(B->body, "q = A_0 p", ops, SPMV_SET, 0, 0);
  }
  {
    Stage S = sys_stage(B, ST_DOTS, "p.q -> alpha", true);
    S.phase = PH_PQ;
    B->body.push_back(std::move(S));
  }
  B->body.push_back(sys_stage(B, ST_UPD_XR, "x += alpha p, r -= alpha q", false));
  {
    Stage S = sys_stage(B, ST_DOTS, "r.r", true);
    S.phase = PH_RR;
    B->body.push_back(std::move(S));
  }
  {
    Stage S;
    S.kind = ST_GUARD;
    S.name = "loop decision";
    B->body.push_back(std::move(S));
  }
  B->tail.push_back(sys_stage(B, ST_UNPACK, "unpack u", false));
}

static cudaError_t launch_stage(Batch *B, const Stage &S, cudaGraphConditionalHandle h) {
  const void *it = B->items + S.off;
  cudaStream_t s = B->stream;
  switch (S.kind) {
    case ST_SPMM:
      return launch_gspmm(S.key, B->nr, S.lpr, S.wpb, (const SpmmItem *)it, S.n_items, S.grid, B->st, s);
    case ST_DIAG:
      return launch_gdiag(S.k, S.dkind, B->nr, (const DiagItem *)it, S.n_items, S.grid, B->st, s);
    case ST_COARSE:
      return launch_gcoarse(S.c64, B->nr, (const CoarseItem *)it, S.n_items, S.grid, B->st, s);
    case ST_DOTS:
      return launch_gdots(S.phase, B->nr, (const SysItem *)it, S.n_items, S.grid, B->gs, B->st, s);
    case ST_UPD_P:
      return launch_gupdate_p(B->nr, (const SysItem *)it, S.n_items, S.grid, B->gs, B->st, s);
    case ST_UPD_XR:
      return launch_gupdate_xr(B->nr, (const SysItem *)it, S.n_items, S.grid, B->gs, B->st, s);
    case ST_PACK:
      return launch_gpack(B->nr, (const SysItem *)it, S.n_items, S.grid, B->gs, B->fin, B->uio, s);
    case ST_UNPACK:
      return launch_gunpack(B->nr, (const SysItem *)it, S.n_items, S.grid, B->gs, B->uio, s);
    case ST_GUARD:
      return launch_gguard((int)B->ctx.size(), B->st, B->loop, h, S.init, s);
  }
  return cudaErrorInvalidValue;
}

// lay the item tables out in one device buffer (16-byte aligned each)
static cudaError_t upload_items(Batch *B) {
  size_t off = 0;
  for (auto *v : {&B->init, &B->body, &B->tail})
    for (Stage &S : *v) {
      S.off = off;
      off += (item_bytes(S) + 15) & ~size_t(15);
    }
  if (off > B->items_bytes) {
    dfree(B->items);
    B->items = nullptr;
    AMG_CUDA_TRY(dalloc((void **)&B->items, off ? off : 16));
    B->items_bytes = off;
  }
  for (auto *v : {&B->init, &B->body, &B->tail})
    for (Stage &S : *v)
      if (item_bytes(S))
        AMG_CUDA_TRY(cudaMemcpyAsync(B->items + S.off, item_host(S), item_bytes(S),
                                     cudaMemcpyHostToDevice, B->stream));
  return cudaStreamSynchronize(B->stream);
}

// Autotuner: every product stage is timed with each tile (lanes per block
// row 32 / 16 / 8, warps per block 8 / 4) on the batch's own operators and
// vectors (the work vectors hold no data between solves; every system is
// marked active), and keeps the fastest.  The loop-decision kernel is never
// launched here, so no conditional handle is needed.
static cudaError_t autotune(Batch *B) {
  for (int s = 0; s < (int)B->ctx.size(); ++s) {
    B->st_host[s] = McgState{};
    B->st_host[s].active = 1;
    B->st_host[s].nr = B->nr;
  }
  AMG_CUDA_TRY(cudaMemcpyAsync(B->st, B->st_host, sizeof(McgState) * B->ctx.size(),
                               cudaMemcpyHostToDevice, B->stream));
  // candidates: (lanes per row, warps per block); (0, s): SELL-32, s slices
  // per block, when every operator of the stage has its SELL copy
  // (-g, w): block lanes, g lanes per block row, for 6x6 / 6x3 blocks
  const int cand[12][2] = {{32, 8}, {32, 4}, {16, 8}, {16, 4}, {8, 8}, {8, 4},
                           {0, 4},  {0, 2},  {-8, 8}, {-8, 4}, {-16, 8}, {-16, 4}};
  for (auto *v : {&B->init, &B->body})
    for (Stage &S : *v) {
      if (S.kind != ST_SPMM) continue;
      bool sell = gsell_supported(S.key.br, S.key.bc);
      for (const SpmmOp &o : S.ops) sell = sell && o.svals && o.A->sell_ptr;
      float best = 1e30f;
      int bl = 32, bw = 8;
      for (const auto &cw : cand) {
        const int lpr = cw[0], wpb = cw[1];
        if (lpr > 0 && lpr < S.key.br) continue;
        if (lpr == 0 && !sell) continue;
        if (S.key.vt == 3 && lpr != 0) continue;  // the double-float product: SELL-32 only
        if (lpr < 0 && !gblock_supported(S.key.br, S.key.bc)) continue;
        {
          S.lpr = lpr;
          S.wpb = wpb;
          build_spmm_items(S);
          AMG_CUDA_TRY(cudaMemcpyAsync(B->items + S.off, S.sp.data(), item_bytes(S),
                                       cudaMemcpyHostToDevice, B->stream));
          AMG_CUDA_TRY(launch_stage(B, S, 0));
          AMG_CUDA_TRY(cudaEventRecord(B->ev0, B->stream));
          for (int r = 0; r < 3; ++r) AMG_CUDA_TRY(launch_stage(B, S, 0));
          AMG_CUDA_TRY(cudaEventRecord(B->ev1, B->stream));
          AMG_CUDA_TRY(cudaEventSynchronize(B->ev1));
          float ms = 0.f;
          AMG_CUDA_TRY(cudaEventElapsedTime(&ms, B->ev0, B->ev1));
          if (ms < best) {
            best = ms;
            bl = lpr;
            bw = wpb;
          }
        }
      }
      S.lpr = bl;
      S.wpb = bw;
      S.us = best * 1e3f / 3.f;
      build_spmm_items(S);
      AMG_CUDA_TRY(cudaMemcpyAsync(B->items + S.off, S.sp.data(), item_bytes(S), cudaMemcpyHostToDevice,
                                   B->stream));
    }
  return cudaStreamSynchronize(B->stream);
}

static cudaError_t capture(Batch *B) {
  cudaStream_t s = B->stream;
  AMG_CUDA_TRY(cudaGraphCreate(&B->graph_def, 0));
  cudaGraph_t g = B->graph_def;
  cudaGraphConditionalHandle h;
  AMG_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
  AMG_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (const Stage &S : B->init)
    if (e == cudaSuccess) e = launch_stage(B, S, h);
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  cudaStreamCaptureStatus status;
  cudaError_t e2 = cudaStreamGetCaptureInfo(s, &status, nullptr, nullptr, &deps, nullptr, &ndeps);
  std::vector<cudaGraphNode_t> sinks(deps, deps + ndeps);
  cudaGraph_t cap = nullptr;
  cudaError_t e3 = cudaStreamEndCapture(s, &cap);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = e3;
  AMG_CUDA_TRY(e);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  AMG_CUDA_TRY(cudaGraphAddNode(&cnode, g, sinks.data(), nullptr, sinks.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  AMG_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  for (const Stage &S : B->body)
    if (e == cudaSuccess) e = launch_stage(B, S, h);
  e2 = cudaStreamEndCapture(s, &body);
  if (e == cudaSuccess) e = e2;
  AMG_CUDA_TRY(e);
  AMG_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, g, &cnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  for (const Stage &S : B->tail)
    if (e == cudaSuccess) e = launch_stage(B, S, h);
  e2 = cudaStreamEndCapture(s, &cap);
  if (e == cudaSuccess) e = e2;
  AMG_CUDA_TRY(e);
  return cudaGraphInstantiate(&B->graph, B->graph_def, 0);
}

static void free_batch(Batch *B) {
  if (B->graph) cudaGraphExecDestroy(B->graph);
  if (B->graph_def) cudaGraphDestroy(B->graph_def);
  for (GSys &G : B->gsh) {
    double *d[] = {G.f, G.x, G.r, G.z, G.zold, G.p, G.q, G.partials};
    for (double *p : d) dfree(p);
    dfree(G.pdf);
    dfree(G.counter);
  }
  for (SysVec &V : B->vec)
    for (auto *v : {&V.lb, &V.lx, &V.lt, &V.ly})
      for (void *p : *v) dfree(p);
  dfree(B->gs);
  dfree(B->st);
  dfree(B->loop);
  dfree(B->items);
  dfree(B->fin);
  dfree(B->uio);
  if (B->st_host) cudaFreeHost(B->st_host);
  if (B->loop_host) cudaFreeHost(B->loop_host);
  if (B->ev0) cudaEventDestroy(B->ev0);
  if (B->ev1) cudaEventDestroy(B->ev1);
  if (B->stream) cudaStreamDestroy(B->stream);
}

static std::string describe(const Batch *B) {
  std::string d;
  char line[320];
  for (auto *v : {&B->init, &B->body, &B->tail}) {
    const char *part = v == &B->init ? "init" : v == &B->body ? "iteration" : "tail";
    for (const Stage &S : *v) {
      if (S.kind == ST_SPMM && S.lpr == 0)
        snprintf(line, sizeof line, "%s: %s: %d systems, %d blocks, SELL-32 thread/row, %d slices/block, %.1f us\n",
                 part, S.name.c_str(), S.n_items, S.grid, S.wpb, S.us);
      else if (S.kind == ST_SPMM && S.lpr < 0)
        snprintf(line, sizeof line, "%s: %s: %d systems, %d blocks, block lanes %d lanes/row, %d warps/block, %.1f us\n",
                 part, S.name.c_str(), S.n_items, S.grid, -S.lpr, S.wpb, S.us);
      else if (S.kind == ST_SPMM)
        snprintf(line, sizeof line, "%s: %s: %d systems, %d blocks, %d lanes/row, %d warps/block, %.1f us\n",
                 part, S.name.c_str(), S.n_items, S.grid, S.lpr, S.wpb, S.us);
      else
        snprintf(line, sizeof line, "%s: %s: %d systems, %d blocks\n", part, S.name.c_str(), S.n_items,
                 S.grid);
      d += line;
    }
  }
  return d;
}

// SELL-32 copies of every system's A_0 and P_0 (candidates of the tuner;
// they also serve the system's own single-system kernels), and, for the
// double-float CG product, A_0's double-float copy.  The CG product runs in
// double-float arithmetic when the contexts ask for it (amg_set_cg_operator
// before the batch is created: AMG_CG_DOUBLE_FLOAT, or AMG_CG_AUTO with a
// mixed-precision V-cycle) and every A_0 has a SELL-32 copy with its rows in
// order.
static cudaError_t ensure_sell(Batch *B) {
  for (Ctx *c : B->ctx) {
    DevBSR *ops[2] = {&c->levels[0].A, c->levels.size() > 1 ? &c->levels[0].P : nullptr};
    for (DevBSR *m : ops) {
      if (!m || !m->nnzb || m->sell_ptr || !gsell_supported(m->br, m->bc)) continue;
      AMG_CUDA_TRY(build_sell(c, *m));
      if (c->precision != AMG_PREC_FP64) AMG_CUDA_TRY(make_low_precision(c, *m, c->precision));
      AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
  }
  const Ctx *c0 = B->ctx[0];
  bool df = c0->cg_op == AMG_CG_DOUBLE_FLOAT || (c0->cg_op == AMG_CG_AUTO && c0->precision != AMG_PREC_FP64);
  for (Ctx *c : B->ctx) {
    const DevBSR &A = c->levels[0].A;
    df = df && c->cg_op == c0->cg_op && A.sell_ptr && !A.sell_perm && A.br == A.bc && (A.br == 2 || A.br == 3);
  }
  B->df = df;
  if (df)
    for (Ctx *c : B->ctx)
      if (!c->levels[0].A.sdf) {
        AMG_CUDA_TRY(build_double_float(c, c->levels[0].A));
        AMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
      }
  return cudaSuccess;
}

static cudaError_t create_buffers(Batch *B) {
  const int ns = (int)B->ctx.size(), nr = B->nr;
  AMG_CUDA_TRY(cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking));
  AMG_CUDA_TRY(cudaEventCreate(&B->ev0));
  AMG_CUDA_TRY(cudaEventCreate(&B->ev1));
  AMG_CUDA_TRY(cudaMallocHost((void **)&B->st_host, sizeof(McgState) * ns));
  AMG_CUDA_TRY(cudaMallocHost((void **)&B->loop_host, sizeof(BatchLoop)));
  B->gsh.resize(ns);
  B->vec.resize(ns);
  size_t off = 0;
  const size_t w = B->precision == AMG_PREC_FP64 ? sizeof(double) : sizeof(float);
  for (int s = 0; s < ns; ++s) {
    GSys &G = B->gsh[s];
    memset(&G, 0, sizeof(GSys));
    const Ctx *c = B->ctx[s];
    G.n = (size_t)c->levels[0].A.n_rows * c->levels[0].k;
    G.offset = off;
    off += G.n * nr;
    const size_t bytes = G.n * nr * sizeof(double);
    double **d[] = {&G.f, &G.x, &G.r, &G.z, &G.zold, &G.p, &G.q};
    for (double **p : d) {
      AMG_CUDA_TRY(dalloc((void **)p, bytes));
      AMG_CUDA_TRY(cudaMemset(*p, 0, bytes));
    }
    if (B->df) {
      AMG_CUDA_TRY(dalloc((void **)&G.pdf, G.n * nr * sizeof(float2)));
      AMG_CUDA_TRY(cudaMemset(G.pdf, 0, G.n * nr * sizeof(float2)));
    }
    for (const Level &L : c->levels) {
      const size_t lb = (size_t)L.A.n_rows * L.k * nr * w;
      for (auto *v : {&B->vec[s].lb, &B->vec[s].lx, &B->vec[s].lt, &B->vec[s].ly}) {
        void *p = nullptr;
        AMG_CUDA_TRY(dalloc(&p, lb));
        v->push_back(p);
        AMG_CUDA_TRY(cudaMemset(p, 0, lb));
      }
    }
    G.red_blocks = std::max(1, std::min(32, cdiv((long)(G.n * nr), 8192)));
    AMG_CUDA_TRY(dalloc((void **)&G.partials, 2 * kBatchMaxNR * (size_t)G.red_blocks * sizeof(double)));
    AMG_CUDA_TRY(dalloc((void **)&G.counter, sizeof(unsigned)));
    AMG_CUDA_TRY(cudaMemset(G.counter, 0, sizeof(unsigned)));
  }
  B->total = off;
  AMG_CUDA_TRY(dalloc((void **)&B->fin, off * sizeof(double)));
  AMG_CUDA_TRY(dalloc((void **)&B->uio, off * sizeof(double)));
  AMG_CUDA_TRY(dalloc((void **)&B->gs, sizeof(GSys) * ns));
  AMG_CUDA_TRY(cudaMemcpy(B->gs, B->gsh.data(), sizeof(GSys) * ns, cudaMemcpyHostToDevice));
  AMG_CUDA_TRY(dalloc((void **)&B->st, sizeof(McgState) * ns));
  AMG_CUDA_TRY(dalloc((void **)&B->loop, sizeof(BatchLoop)));
  return cudaSuccess;
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

#define BCUDA(B, expr, where)                                                                  \
  do {                                                                                         \
    cudaError_t _e = (expr);                                                                   \
    if (_e != cudaSuccess)                                                                     \
      return bfail(B, AMG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(_e));      \
  } while (0)

// One batched solve: copy f / u in, launch the graph, copy u out, read the
// per-system states.  host_io: f / u are host buffers and the events bracket
// the copies too (end-to-end time); else device buffers and only the graph.
static int batch_run(amg_batch *hb, const double *f, double *u, double rtol, int maxit,
                     int *iters_out, double *relres_out, float *ms_out, bool host_io) {
  if (!hb) return AMG_ERR_ARG;
  Batch *B = &hb->b;
  if (!f || !u || !(rtol >= 0.0) || maxit < 0) return bfail(B, AMG_ERR_ARG, "bad arguments");
  BCUDA(B, cudaSetDevice(B->device), "cudaSetDevice");
  const cudaMemcpyKind kin = host_io ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind kout = host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const size_t bytes = B->total * sizeof(double);
  const int ns = (int)B->ctx.size();
  for (int s = 0; s < ns; ++s) {
    McgState &h = B->st_host[s];
    memset(&h, 0, sizeof(McgState));
    h.rtol = rtol;
    h.maxit = maxit;
    h.nr = B->nr;
    h.flexible = B->precision != AMG_PREC_FP64;
    h.active = 1;
  }
  B->loop_host->guard = 0;
  B->loop_host->maxit = maxit;
  BCUDA(B, cudaMemcpyAsync(B->st, B->st_host, sizeof(McgState) * ns, cudaMemcpyHostToDevice, B->stream),
        "state");
  BCUDA(B, cudaMemcpyAsync(B->loop, B->loop_host, sizeof(BatchLoop), cudaMemcpyHostToDevice, B->stream),
        "state");
  if (host_io) BCUDA(B, cudaEventRecord(B->ev0, B->stream), "event");
  BCUDA(B, cudaMemcpyAsync(B->fin, f, bytes, kin, B->stream), "copy f");
  BCUDA(B, cudaMemcpyAsync(B->uio, u, bytes, kin, B->stream), "copy u");
  if (!host_io) BCUDA(B, cudaEventRecord(B->ev0, B->stream), "event");
  BCUDA(B, cudaGraphLaunch(B->graph, B->stream), "batch graph launch");
  if (!host_io) BCUDA(B, cudaEventRecord(B->ev1, B->stream), "event");
  BCUDA(B, cudaMemcpyAsync(u, B->uio, bytes, kout, B->stream), "copy u back");
  if (host_io) BCUDA(B, cudaEventRecord(B->ev1, B->stream), "event");
  BCUDA(B, cudaMemcpyAsync(B->st_host, B->st, sizeof(McgState) * ns, cudaMemcpyDeviceToHost, B->stream),
        "state");
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

extern "C" {

int amg_batch_create(amg_batch **out, amg_ctx *const *systems, int n_systems, int nrhs) {
  if (!out || !systems || n_systems < 1 || (nrhs != 1 && nrhs != 6)) return AMG_ERR_ARG;
  *out = nullptr;
  for (int s = 0; s < n_systems; ++s) {
    if (!systems[s] || systems[s]->c.levels.empty() ||
        (systems[s]->c.levels[0].k != 2 && systems[s]->c.levels[0].k != 3))
      return AMG_ERR_STATE;
    if (s > 0 && (systems[s]->c.device != systems[0]->c.device ||
                  systems[s]->c.precision != systems[0]->c.precision))
      return AMG_ERR_ARG;
    // the grouped V-cycle runs the block-l1 Jacobi (or learned) smoother only
    if (systems[s]->c.smoother == AMG_SMOOTHER_HYBRID_GS) return AMG_ERR_ARG;
    // and one storage precision on every level
    if (systems[s]->c.precision == AMG_PREC_BF16_COARSE) return AMG_ERR_ARG;
  }
  amg_batch *hb = new amg_batch();
  Batch *B = &hb->b;
  B->nr = nrhs;
  for (int s = 0; s < n_systems; ++s) B->ctx.push_back(&systems[s]->c);
  B->device = B->ctx[0]->device;
  B->precision = B->ctx[0]->precision;
  B->num_sms = B->ctx[0]->num_sms;
  cudaError_t e = cudaSetDevice(B->device);
  if (e == cudaSuccess) e = ensure_sell(B);
  if (e == cudaSuccess) e = create_buffers(B);
  if (e == cudaSuccess) {
    build_stages(B);
    e = upload_items(B);
  }
  if (e == cudaSuccess) e = autotune(B);
  if (e == cudaSuccess) e = capture(B);
  if (e != cudaSuccess) {
    free_batch(B);
    delete hb;
    return AMG_ERR_CUDA;
  }
  B->describe = describe(B);
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

const char *amg_batch_describe(const amg_batch *hb) { return hb ? hb->b.describe.c_str() : ""; }

int amg_batch_launches(const amg_batch *hb, int32_t *per_iteration, int32_t *fixed) {
  if (!hb) return AMG_ERR_ARG;
  if (per_iteration) *per_iteration = (int32_t)hb->b.body.size();
  if (fixed) *fixed = (int32_t)(hb->b.init.size() + hb->b.tail.size());
  return AMG_OK;
}

int amg_batch_layout(const amg_batch *hb, int s, int64_t *offset, int64_t *n_dofs, int64_t *total) {
  if (!hb) return AMG_ERR_ARG;
  const Batch *B = &hb->b;
  if (total) *total = (int64_t)B->total;
  if (s < 0 || s >= (int)B->gsh.size()) return AMG_ERR_ARG;
  if (offset) *offset = (int64_t)B->gsh[s].offset;
  if (n_dofs) *n_dofs = (int64_t)B->gsh[s].n;
  return AMG_OK;
}

int amg_batch_pcg_solve(amg_batch *hb, const double *f_dev, double *u_dev, double rtol, int maxit,
                        int *iters_out, double *relres_out, float *ms_out) {
  return batch_run(hb, f_dev, u_dev, rtol, maxit, iters_out, relres_out, ms_out, false);
}

int amg_batch_pcg_solve_host(amg_batch *hb, const double *f_host, double *u_host, double rtol,
                             int maxit, int *iters_out, double *relres_out, float *ms_out) {
  return batch_run(hb, f_host, u_host, rtol, maxit, iters_out, relres_out, ms_out, true);
}

}  // extern "C"
