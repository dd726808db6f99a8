// Small dense symmetric eigenproblems on the device (setup kernels): the
// cyclic Jacobi method (Golub & Van Loan, "Matrix Computations", Sec. 8.5),
// written from the mathematics.
#pragma once

#include <math.h>

namespace amg {

// Cyclic Jacobi: on return a holds the eigenvalues on its diagonal and v the
// eigenvectors as columns (a, v row-major K x K).
template <int K>
__device__ void jacobi_eig(double *a, double *v) {
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j) v[i * K + j] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int i = 0; i < K * K; ++i) fro += a[i] * a[i];
  if (fro == 0.0) return;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < K; ++p)
      for (int q = p + 1; q < K; ++q) off += a[p * K + q] * a[p * K + q];
    if (off <= 1e-34 * fro) break;
    for (int p = 0; p < K; ++p) {
      for (int q = p + 1; q < K; ++q) {
        const double apq = a[p * K + q];
        if (fabs(apq) <= 1e-300) continue;
        const double theta = (a[q * K + q] - a[p * K + p]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
        const double cs = 1.0 / sqrt(1.0 + t * t);
        const double sn = t * cs;
        // A <- J^T A J with J the rotation in the (p, q) plane
        for (int k = 0; k < K; ++k) {
          const double akp = a[k * K + p], akq = a[k * K + q];
          a[k * K + p] = cs * akp - sn * akq;
          a[k * K + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < K; ++k) {
          const double apk = a[p * K + k], aqk = a[q * K + k];
          a[p * K + k] = cs * apk - sn * aqk;
          a[q * K + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < K; ++k) {
          const double vkp = v[k * K + p], vkq = v[k * K + q];
          v[k * K + p] = cs * vkp - sn * vkq;
          v[k * K + q] = sn * vkp + cs * vkq;
        }
      }
    }
  }
}


}  // namespace amg
