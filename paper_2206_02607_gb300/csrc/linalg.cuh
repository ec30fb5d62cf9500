// Small dense linear algebra shared by the step kernels: the r x r normal
// equations (J^T J) delta = -J^T rho of one Gauss-Newton iteration (paper App. C),
// solved in FP64.
#pragma once

#include <math.h>

#include "../../include/crom.h"

namespace crom {

// Warp-parallel FP64 Cholesky solve of A x = b, r <= 32, with A = a[i*(r+1)+j] in
// shared memory and b in column r (right-looking factorisation: lane i owns row i).
// Status: NONFINITE when A or b holds a NaN/Inf, SINGULAR when a pivot is
// <= 1e-14 * max diag(A); on success x_k is left in a[k*(r+1)+r].  invd: r
// doubles of shared scratch.  All 32 lanes of the warp must call it.
__device__ __forceinline__ int chol_solve_warp(double* A, double* invd, int r, int lane) {
  const int R = r + 1;
  bool bad = false;
  for (int e = lane; e < r * R; e += 32) bad |= !isfinite(A[e]);
  if (__any_sync(0xffffffffu, bad)) return CROM_ERR_NONFINITE;
  double dmax = 0.0;
  for (int a = 0; a < r; ++a) dmax = fmax(dmax, A[a * R + a]);
  const double tol = 1e-14 * dmax;
  for (int j = 0; j < r; ++j) {
    const double d = A[j * R + j];
    if (!(d > tol)) return CROM_ERR_SINGULAR;
    // one reciprocal square root instead of a square root and a division: FP64 is
    // a slow pipe on this GPU, and each of these is a sequence of FP64 instructions
    const double inv = rsqrt(d);
    const double ljj = d * inv;
    __syncwarp();
    if (lane == 0) {
      A[j * R + j] = ljj;
      invd[j] = inv;
    }
    if (lane > j && lane < r) A[lane * R + j] *= inv;
    __syncwarp();
    if (lane > j && lane < r) {
      const double lij = A[lane * R + j];
      for (int k = j + 1; k <= lane; ++k) A[lane * R + k] -= lij * A[k * R + j];
    }
    __syncwarp();
  }
  for (int k = 0; k < r; ++k) {  // L y = b
    const double yk = A[k * R + r] * invd[k];
    __syncwarp();
    if (lane == 0) A[k * R + r] = yk;
    if (lane > k && lane < r) A[lane * R + r] -= A[lane * R + k] * yk;
    __syncwarp();
  }
  for (int k = r - 1; k >= 0; --k) {  // L^T x = y
    const double xk = A[k * R + r] * invd[k];
    __syncwarp();
    if (lane == 0) A[k * R + r] = xk;
    if (lane < k) A[lane * R + r] -= A[k * R + lane] * xk;
    __syncwarp();
  }
  return CROM_OK;
}

}  // namespace crom
