// Grouped kernels of the batched solve (internal to libamg).
//
// A grouped launch runs one step of the V-cycle or of CG for every system of
// a batch at once: its grid is the concatenation of the systems' blocks, and
// an item table (one item per system, with the first block it owns) tells a
// block which system and which operands it works on.  Vectors carry NR load
// cases interleaved per dof: entry (i * k + r) * NR + j for vertex i, dof r,
// load case j, so every matrix block read serves all NR load cases.
#pragma once

#include "amg_internal.h"

namespace amg {

constexpr int kBatchMaxNR = 8;

// CG state of one system (device-resident; NR load cases)
struct McgState {
  double rr[kBatchMaxNR], ff[kBatchMaxNR], tol2[kBatchMaxNR], rho[kBatchMaxNR],
      rho_old[kBatchMaxNR], alpha[kBatchMaxNR], beta[kBatchMaxNR], pq[kBatchMaxNR];
  int it[kBatchMaxNR], done[kBatchMaxNR], status[kBatchMaxNR];
  double rtol;
  int maxit, flexible, nr, active;
};

struct BatchLoop {  // whole-batch loop bound
  int guard, maxit;
};

// per-system CG vectors (FP64, interleaved) and reduction scratch
struct GSys {
  size_t n;       // dofs of A_0
  size_t offset;  // offset of the system's load cases in the stacked f / u
  double *f, *x, *r, *z, *zold, *p, *q;
  float2 *pdf;  // p as double-float pairs (the double-float CG operator), else null
  double *partials;
  unsigned *counter;
  int red_blocks;
};

struct SpmmItem {
  const int *rowptr, *colidx;
  const void *vals, *x, *b, *minv;
  void *y;
  int n_rows, sys, first_block;
  // SELL-32 copy of the operator (thread per block row), if present;
  // sell_perm: row of each slice lane of a sorted copy (null: row 32s + t)
  const int *sell_ptr, *sell_col, *sell_perm;
  const void *svals;
  int n_slices;
  int df_exp;  // double-float copy: values scaled by 2^-df_exp
};
struct DiagItem {
  const void *minv, *bin;
  void *bcopy, *y;
  int n, sys, first_block;
};
struct CoarseItem {
  const double *cinv;
  const void *b;
  void *y;
  int n, sys, first_block;
};
struct SysItem {
  int sys, first_block;
};

// value type of the operator: 0 FP64, 1 FP32, 2 BF16 (vectors FP32 for 1, 2),
// 3 double-float pairs (the CG product q = A_0 p: SELL-32 copy only, x the
// pairs of p, FP64 output)
struct SpmmKey {
  int br, bc, vt, mode, to64;  // to64: FP64 output from an FP32 / BF16 operator
};

// lanes per row (32, 16 or 8) and warps per block (tile / schedule choice);
// lpr = 0: the SELL-32 copy, one thread per block row, wpb slices per block
// (block shapes with gsell_supported only)
bool gsell_supported(int br, int bc);
// lpr = -8 / -16: block lanes, 8 or 16 lanes per block row, one whole block
// per lane (6x6 and 6x3 blocks only)
bool gblock_supported(int br, int bc);
cudaError_t launch_gspmm(const SpmmKey &k, int nr, int lpr, int wpb, const SpmmItem *items,
                         int n_items, int grid, const McgState *st, cudaStream_t s);
// kind: 0 FP64; 1 FP64 input -> FP32 (+ FP32 copy of the input); 2 FP32
cudaError_t launch_gdiag(int k, int kind, int nr, const DiagItem *items, int n_items, int grid,
                         const McgState *st, cudaStream_t s);
cudaError_t launch_gcoarse(bool fp64, int nr, const CoarseItem *items, int n_items, int grid,
                           const McgState *st, cudaStream_t s);

enum McgPhase { PH_INIT = 0, PH_RHO = 1, PH_PQ = 2, PH_RR = 3 };
cudaError_t launch_gdots(int phase, int nr, const SysItem *items, int n_items, int grid,
                         const GSys *gs, McgState *st, cudaStream_t s);
cudaError_t launch_gupdate_p(int nr, const SysItem *items, int n_items, int grid, const GSys *gs,
                             const McgState *st, cudaStream_t s);
cudaError_t launch_gupdate_xr(int nr, const SysItem *items, int n_items, int grid, const GSys *gs,
                              const McgState *st, cudaStream_t s);
cudaError_t launch_gpack(int nr, const SysItem *items, int n_items, int grid, const GSys *gs,
                         const double *fin, const double *uin, cudaStream_t s);
cudaError_t launch_gunpack(int nr, const SysItem *items, int n_items, int grid, const GSys *gs,
                           double *uout, cudaStream_t s);
cudaError_t launch_gguard(int ns, McgState *st, BatchLoop *loop, cudaGraphConditionalHandle h,
                          bool init, cudaStream_t s);

}  // namespace amg
