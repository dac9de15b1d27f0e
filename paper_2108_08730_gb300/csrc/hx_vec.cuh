// Batched vector kernels of the solver (declarations).
//
// Fields are [R][N] interleaved complex of type T (float -> complex64,
// double -> complex128).  Per-RHS scalars live on the device as double2
// (complex) or double arrays of length R, so the Krylov loop never needs the
// host except for convergence checks.
#pragma once

#include <cuda_runtime.h>

namespace hx {

// Deterministic reductions: every RHS is reduced over the same fixed blocks in
// the same order, so a result does not depend on how many RHS share the batch.
int reduce_blocks(long long N);
// out[r] = sum_i conj(a[r,i]) b[r,i]   (partials: >= R * reduce_blocks(N) double2)
template <typename T>
cudaError_t launch_dot(const void* a, const void* b, long long N, int R, double2* partials,
                       double2* out, cudaStream_t s);
// out[r] = sum_i |a[r,i]|^2
template <typename T>
cudaError_t launch_norm2(const void* a, long long N, int R, double2* partials, double* out,
                         cudaStream_t s);

// BiCGStab (right preconditioned) updates with per-RHS scalars sc (see kernel)
template <typename T>
cudaError_t launch_bicg_p(void* p, const void* r, const void* v, const double2* beta,
                          const double2* omega, long long N, int R, cudaStream_t s);
template <typename T>
cudaError_t launch_bicg_s(void* sv, const void* r, const void* v, const double2* alpha, long long N,
                          int R, cudaStream_t s);
template <typename T>
cudaError_t launch_bicg_xr(void* x, void* r, const void* sv, const void* phat, const void* shat,
                           const void* t, const double2* alpha, const double2* omega, long long N,
                           int R, cudaStream_t s);

// Multigrid transfers between a fine level (nf) and its coarse level (nc):
// coarse = full weighting of fine;  fine += trilinear(coarse).
template <typename T>
cudaError_t launch_restrict(const void* fine, const int nf[3], void* coarse, const int nc[3], int R,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_prolong_add(void* fine, const int nf[3], const void* coarse, const int nc[3],
                               int R, cudaStream_t s);
cudaError_t launch_inject_velocity(const float* vf, const int nf[3], float* vc, const int nc[3],
                                   cudaStream_t s);

// r32[r,i] = (complex64)(r64[r,i] * scale[r]);  x64[r,i] += scale[r] * d32[r,i]
cudaError_t launch_cast_scale(const double2* r64, float2* r32, const double* scale, long long N,
                              int R, cudaStream_t s);
cudaError_t launch_axpy_mixed(double2* x64, const float2* d32, const double* scale, long long N,
                              int R, cudaStream_t s);
// x64[r,i] += scale[r] * d64[r,i]
cudaError_t launch_axpy_c128(double2* x64, const double2* d64, const double* scale, long long N,
                             int R, cudaStream_t s);
// y = x (copy) for complex T fields
template <typename T>
cudaError_t launch_copy(void* y, const void* x, long long n_complex, cudaStream_t s);

// Point sources: r[rhs][idx] += w * amp  for each of n entries.
struct SourceEntry {
  long long idx;
  int rhs;
  double re, im;
};
template <typename T>
cudaError_t launch_add_sources(void* r, long long N, const SourceEntry* e, int n, cudaStream_t s);

// Per-RHS scalar steps of BiCGStab (one thread per RHS).
//   beta step : beta = (rho_new / rho) (alpha / omega); rho = rho_new
//   alpha step: alpha = rho / rv        (rv = (rhat, v))
//   omega step: omega = ts / tt         (ts = (t, s), tt = |t|^2)
// Inactive RHS (active[r] == 0) get zero alpha/omega/beta, so the vector
// updates leave them unchanged.  A zero denominator deactivates the RHS and
// sets breakdown[r] = 1.
cudaError_t launch_scal_beta(double2* beta, double2* rho, const double2* rho_new,
                             const double2* alpha, const double2* omega, const int* active,
                             int* breakdown, int R, cudaStream_t s);
cudaError_t launch_scal_alpha(double2* alpha, const double2* rho, const double2* rv, int* active,
                              int* breakdown, int R, cudaStream_t s);
cudaError_t launch_scal_omega(double2* omega, const double2* ts, const double* tt, int* active,
                              int* breakdown, int R, cudaStream_t s);

}  // namespace hx

namespace hx {
// out[r][i] = sum_j M[i][j] b[r][j]  (dense n x n complex matrix, row-major)
template <typename T>
cudaError_t launch_dense_matvec(const void* M, const void* b, void* out, long long n, int R,
                                cudaStream_t s);
}  // namespace hx
