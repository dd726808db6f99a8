// Multi-load-case launchers (internal to libamg); see multirhs.cu.
#pragma once

#include "amg_internal.h"

namespace amg {

// y = op(A) x on NR interleaved load cases (nr = 1 or 6); y_fp64 writes an
// FP64 result from an FP32 / BF16 operator (finest-level post-smoothing).
cudaError_t launch_bsr_mr(const Ctx *c, const DevBSR &A, int prec, int nr, int mode, const void *x,
                          const void *b, const void *minv, void *y, bool y_fp64);
// y = M^+ b per vertex; bin may be FP64 (bin_fp64) and is then also stored
// in the V-cycle precision into bcopy (if not NULL).
cudaError_t launch_blockdiag_mr(const Ctx *c, int n, int k, int prec, int nr, const void *minv,
                                const void *bin, bool bin_fp64, void *bcopy, void *y);
cudaError_t launch_coarse_mr(const Ctx *c, int n, int nr, const double *cinv, const void *b, void *y,
                             int prec);

}  // namespace amg
