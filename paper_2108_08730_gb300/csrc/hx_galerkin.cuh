// Galerkin coarse operators and stored-coefficient stencils (see hx_galerkin.cu).
#pragma once

#include <cuda_runtime.h>

#include "hx_internal.h"

namespace hx {

// coarse_coef[k][I] = (R A P)[I, I + offset k] with A the on-the-fly operator
// `fine` (its shift included); nc = coarse grid ((n+1)/2 per axis).
template <typename T>
cudaError_t launch_galerkin_onfly(const OpDesc<T>& fine, void* coarse_coef, const int nc[3],
                                  cudaStream_t s);
// the same with A given by stored coefficients fine_coef[k][i] on grid nf
template <typename T>
cudaError_t launch_galerkin_stored(const void* fine_coef, const int nf[3], void* coarse_coef,
                                   const int nc[3], cudaStream_t s);
// stencil modes of hx_internal.h (kApply, kResidual, kJacobi, kJacobi0) with
// stored coefficients coef[k][i] on grid n, R fields of n[0]*n[1]*n[2] each
template <typename T>
cudaError_t launch_stored_stencil(const void* coef, const int n[3], int mode, const void* x,
                                  const void* b, void* y, int R, double omega_j, cudaStream_t s);
// the on-the-fly operator of `op`, one thread per row (for small grids); same
// modes, R fields of op.nx*op.ny*op.nz each
template <typename T>
cudaError_t launch_direct_stencil(const OpDesc<T>& op, int mode, const void* x, const void* b, void* y,
                                  int R, double omega_j, cudaStream_t s);

}  // namespace hx
