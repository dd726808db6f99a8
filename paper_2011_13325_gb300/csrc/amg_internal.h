// Internal declarations of libamg (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/amg.h"
#include "setup_host.h"

namespace amg {

// Device block-sparse-row matrix.  Values exist in FP64 always; FP32 / BF16
// copies only for the mixed-precision V-cycles.
enum BsrKernel {
  KERN_WARP_ROWS = 0,
  KERN_ROW_LANES = 1,
  KERN_BLOCK_LANES = 2,
  KERN_SELL = 3,
  KERN_SELL_SPLIT = 4  // sorted SELL-32, one warp per output row of a slice (rectangular operators)
};

struct DevBSR {
  int n_rows = 0, n_cols = 0, br = 0, bc = 0;
  int64_t nnzb = 0;
  int *rowptr = nullptr;
  int *colidx = nullptr;
  double *v64 = nullptr;
  float *v32 = nullptr;
  __nv_bfloat16 *v16 = nullptr;
  // SELL-32 copy for operators with many short rows (thread per block row):
  // slice s holds rows 32s..32s+31 in slots sell_ptr[s]..sell_ptr[s+1]-1;
  // slot j of lane t: column sell_col[j*32 + t], element q of its block at
  // s??[(j*br*bc + q)*32 + t] (every element of a slot is one coalesced
  // 32-wide row); padding slots have column 0 and zero values.
  // Rectangular operators (P_l, R_l, whose row lengths vary) have sorted
  // slices: inside each window of 256 rows the rows are ordered by length,
  // longest first, and lane t of slice s holds row sell_perm[32s + t]
  // (n_rows on a padding lane); sell_perm is null where lane t of slice s
  // holds row 32s + t (square operators, whose CG kernels assume that).
  // kernel choice (set by the upload's tuner under AMG_LAYOUT_AUTO); the
  // SELL-32 copy is used when present unless the tuner picked a BSR kernel
  int kern = KERN_SELL;  // KERN_WARP_ROWS / KERN_ROW_LANES / KERN_BLOCK_LANES / KERN_SELL(_SPLIT)
  int n_slices = 0;
  int64_t sell_slots = 0;
  int *sell_ptr = nullptr;
  int *sell_col = nullptr;
  int *sell_perm = nullptr;
  double *s64 = nullptr;
  float *s32 = nullptr;
  __nv_bfloat16 *s16 = nullptr;
  // double-float copy of the SELL-32 values (A_0 only, for the CG operator):
  // value a is held as a * 2^-df_exp = hi + lo, two FP32 numbers (hi the
  // value rounded to FP32, lo the rounded remainder), stored as one float2
  // per element in the SELL-32 order of s64 (8 bytes, as the FP64 copy)
  float2 *sdf = nullptr;
  int df_exp = 0;
};

struct Level {
  DevBSR A, P, R;          // P, R: to / from level l+1 (empty on the coarsest)
  int k = 0;               // block size of A_l
  double *minv64 = nullptr;  // smoother blocks M_v^+ (n * k * k)
  float *minv32 = nullptr;
  // V-cycle work vectors (n * k), FP64 and FP32 sets
  double *b64 = nullptr, *x64 = nullptr, *t64 = nullptr, *y64 = nullptr;
  float *b32 = nullptr, *x32 = nullptr, *t32 = nullptr, *y32 = nullptr;
  // hybrid Gauss-Seidel: colour of every block row (device), the rows ordered
  // by colour then index (device), and the class offsets (host, n_colours+1)
  int *gs_colour = nullptr;
  int *gs_rows = nullptr;
  std::vector<int> gs_ptr;
  // level 0 with a SELL-32 copy: A's rows in colour order as SELL-32 slices
  // (every class padded to whole slices; class k owns the slices
  // gs_slice_ptr[k] .. gs_slice_ptr[k+1]), values in the level's storage
  // precision, gs_sell_perm the row of every slice lane (n_rows on padding)
  int *gs_sell_ptr = nullptr, *gs_sell_col = nullptr, *gs_sell_perm = nullptr;
  void *gs_sell_vals = nullptr;
  int gs_sell_prec = -1;
  std::vector<int> gs_slice_ptr;
};

// Scalars of the device-resident PCG iteration.
struct PcgState {
  double rr, ff, tol2, rho, rho_old, alpha, beta, pq, rtol;
  int it, maxit, status, flexible, guard;
  int replace;     // 1: recompute the residual as f - A x (FP64 operator)
  int replaced;    // residual replacements of this solve
  double rr_ref;   // r.r at the start or the last replacement
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  std::string err;
  std::string desc;  // amg_describe text
  std::vector<Level> levels;
  int precision = AMG_PREC_FP64;
  int smoother = AMG_SMOOTHER_L1_JACOBI;
  // coarsest level: explicit FP64 inverse of A_L + (I - E E^T)
  int coarse_n = 0;
  double *cinv = nullptr;
  // PCG buffers (finest level, FP64)
  double *f = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *zold = nullptr, *p = nullptr,
         *q = nullptr;
  PcgState *st = nullptr;       // device
  PcgState *st_host = nullptr;  // pinned
  double *partials = nullptr;   // reduction scratch
  unsigned *counter = nullptr;  // last-block counter
  int layout_policy = 0;        // AMG_LAYOUT_*: which operators get the SELL-32 copy
  bool pcg_graph = true;        // false: host-driven loop (same kernels, for profiling)
  bool pdl = true;              // programmatic dependent launch of the solve kernels
  cudaGraphExec_t graph = nullptr;
  cudaGraph_t graph_def = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  float last_ms = 0.f;
  // host setup, device stages (Galerkin, transfers, coarse topology,
  // prolongation), finalize, total, and the coarse topology + prolongation
  // part of the device stages (s)
  // [5]: device evaluation of the pair measure mu_p (inside the host part)
  double setup_times[6] = {0, 0, 0, 0, 0, 0};
  // coarse topologies built by the device stages of amg_setup (kept when
  // asked for, level l >= 1 at index l)
  std::vector<amgsetup::Topo> topo;
  double *hbuf = nullptr;        // pinned staging for host solves
  size_t hbuf_len = 0;
  int cg_op = AMG_CG_AUTO;       // arithmetic of the CG operator q = A_0 p
  float2 *pdf = nullptr;         // p split into double-float pairs (CG operator input)
};


// Programmatic dependent launch of the solve-phase kernels: such a kernel
// starts with pdl_enter(), which waits until the previous grid of the stream
// has completed with its writes visible (griddepcontrol.wait).  The
// predecessor triggers the launch implicitly as its blocks exit (no explicit
// early trigger: waiting blocks of the next grid would take SM slots from a
// predecessor with several waves), so the next launch overlaps only the
// predecessor's drain.  A no-op for a kernel launched without the
// attribute.  pdl_enter() must be the first statement (a block that
// returned before it would let a successor run early).
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

// Launch on c's stream, with programmatic stream serialization if c->pdl.
template <typename... P, typename... A>
inline cudaError_t launch_k(const Ctx *c, void (*k)(P...), dim3 g, dim3 b, A &&... a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = c->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = c->pdl ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<A &&>(a)...);
}
#define AMG_KLAUNCH(...)                          \
  do {                                            \
    const cudaError_t _le = launch_k(__VA_ARGS__); \
    if (_le != cudaSuccess) return _le;           \
  } while (0)

// Device allocation helpers (all internal buffers are owned by the context).
cudaError_t dalloc(void **p, size_t bytes);
void dfree(void *p);
void free_bsr(DevBSR &m);
void free_levels(Ctx *c);
void free_pcg(Ctx *c);

// launches (stream-ordered, no synchronisation)
enum SpmvMode { SPMV_SET = 0, SPMV_RESID = 1, SPMV_ADD = 2, SPMV_SMOOTH = 3 };

// y = op(A) on FP64 / FP32 / BF16 values with FP64 or FP32 vectors.
cudaError_t launch_bsr(const Ctx *c, const DevBSR &A, int prec, int mode, const void *x,
                       const void *b, const void *minv, void *y);
cudaError_t launch_blockdiag(const Ctx *c, int n, int k, int prec, const void *minv,
                             const void *b, void *y);
cudaError_t launch_smooth_out64(const Ctx *c, const DevBSR &A, int prec, const float *x,
                                const float *b, const float *minv, double *y);
cudaError_t launch_blockdiag_entry(const Ctx *c, int n, int k, const float *minv, const double *r,
                                   float *b, float *x);
cudaError_t launch_coarse_gemv(const Ctx *c, int n, const double *cinv, const void *b, void *y,
                               int prec);
cudaError_t launch_convert(const Ctx *c, size_t n, const void *src, int src_prec, void *dst,
                           int dst_prec);

// setup kernels
cudaError_t galerkin_device(Ctx *c, int level);
cudaError_t smoother_setup(Ctx *c, int level);
// hybrid Gauss-Seidel: colouring of level l (host greedy, uploaded), and one
// sweep over the colour classes (forward or backward) updating x in place
cudaError_t gs_prepare(Ctx *c, int level);
// Colour-ordered SELL-32 copy of level `level`'s A for the Gauss-Seidel
// sweeps (after the level's low-precision copies exist).
cudaError_t gs_build_sell(Ctx *c, int level, int prec);
cudaError_t launch_gs_sweep(const Ctx *c, const Level &L, int prec, const void *b, void *x,
                            bool forward);
cudaError_t coarse_setup(Ctx *c);
// Storage precision of level l's matrices (and the precision its kernels run
// in): the V-cycle precision, except AMG_PREC_BF16_COARSE, which keeps level
// 0 in FP32 and stores the coarser levels in BF16.
inline int mat_prec(const Ctx *c, int l) {
  if (c->precision != AMG_PREC_BF16_COARSE) return c->precision;
  return l == 0 ? AMG_PREC_FP32_VCYCLE : AMG_PREC_BF16_STORAGE;
}
cudaError_t make_low_precision(Ctx *c, DevBSR &m, int prec);
// sort_square: length-sorted slices for a square operator too (coarse
// levels; A_0 keeps its rows in order, which the CG kernels assume)
cudaError_t build_sell(Ctx *c, DevBSR &m, bool sort_square = false);
cudaError_t build_double_float(Ctx *c, DevBSR &m);
bool want_sell(const Ctx *c, const DevBSR &m, bool coarse_square = false);
cudaError_t scan_exclusive(Ctx *c, int n, int *a, int *total_dev);

// V-cycle on device buffers (FP64 in / out), stream-ordered.
cudaError_t vcycle_launch(Ctx *c, const double *r, double *z);

cudaError_t probe_fma(Ctx *c, double *fp64_gflops, double *fp32_gflops);

// PCG graph
cudaError_t pcg_build_graph(Ctx *c);
cudaError_t pcg_alloc(Ctx *c);
// host-driven PCG (no graph): returns the device status in *st_host
cudaError_t pcg_host_loop(Ctx *c);

}  // namespace amg

struct amg_ctx {
  amg::Ctx c;
};

#define AMG_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return _e;                        \
  } while (0)
