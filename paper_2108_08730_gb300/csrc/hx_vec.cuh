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
// out[r] = sum_i |a[r,i]|^2   (partials: >= R * reduce_blocks(N) double2)
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
// Multigrid transfers between a fine level (nf) and its coarse level (nc):
// coarse = full weighting of fine;  fine += trilinear(coarse).  fpitch: x-row
// pitch of the fine field (0: nf[0]); the coarse field is unpadded.
template <typename T>
cudaError_t launch_restrict(const void* fine, const int nf[3], void* coarse, const int nc[3], int R,
                            cudaStream_t s, long long fpitch = 0);
template <typename T>
cudaError_t launch_prolong_add(void* fine, const int nf[3], const void* coarse, const int nc[3],
                               int R, cudaStream_t s, long long fpitch = 0);
// Coarse-level velocity from the next finer level (coarse node X over fine
// node 2X): mode 0 injection, mode 1 full-weighting average of 1/v^2.
cudaError_t launch_coarse_velocity(const float* vf, const int nf[3], float* vc, const int nc[3], int mode,
                                   cudaStream_t s);

// r32[r,i] = (complex64)(r64[r,i] * scale[r]);  x64[r,i] += scale[r] * d32[r,i]
// (N points per field in rows of nx; the complex64 fields use x-row pitch p32,
// 0 = nx, and their padding is not touched)
cudaError_t launch_cast_scale(const double2* r64, float2* r32, const double* scale, long long N,
                              int R, cudaStream_t s, int nx, long long p32 = 0);
cudaError_t launch_axpy_mixed(double2* x64, const float2* d32, const double* scale, long long N,
                              int R, cudaStream_t s, int nx, long long p32 = 0);
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

// Per-RHS scalars of BiCGStab on the device (arrays of length R) and the
// reductions that produce them.  Each reduction is one launch: every block
// writes its partial sum, and the last block of each RHS to arrive (a
// per-RHS arrival counter) adds the partials in block order, stores the sum
// and takes the scalar step, then resets the counter.  The block partition and
// both summation orders are fixed, so the result does not depend on timing or
// on how many RHS share the batch.
//   kRedBeta : rho_new = (rhat, r);  beta = (rho_new / rho)(alpha / omega), rho = rho_new
//   kRedAlpha: rv = (rhat, v);       alpha = rho / rv
//   kRedOmega: ts = (t, s), tt = |t|^2 (one pass over t);  omega = ts / tt
//   kRedNorm : rn2 = |a|^2
//   kRedBetaNorm (launch_bicg_xr_reduce only): kRedBeta of the updated r, and rn2 = |r|^2
// (x, y) = sum_i conj(x_i) y_i.  Inactive RHS (active[r] == 0) get zero
// alpha / omega / beta, so the vector updates leave them unchanged; a zero
// denominator deactivates the RHS and sets brk[r] = 1.
struct BicgScalars {
  double2 *rho, *rho_new, *alpha, *omega, *beta, *rv, *ts;
  double *tt, *rn2;
  int *active, *brk;
  unsigned* count;   // R arrival counters, zero between launches
  double kappa;      // omega safeguard (0: plain minimal-residual omega)
};
enum { kRedBeta = 0, kRedAlpha = 1, kRedOmega = 2, kRedNorm = 3, kRedBetaNorm = 4 };
// partials: >= 2 * R * reduce_blocks(N) double2; b is unused for kRedNorm
template <typename T>
cudaError_t launch_bicg_reduce(int kind, const void* a, const void* b, long long N, int R, double2* partials,
                               const BicgScalars& sc, cudaStream_t s);
// The last update of a BiCGStab iteration fused with the next iteration's
// first reduction: x += alpha phat + omega shat, r = s - omega t, then
// kRedBetaNorm over the new r (with rhat).
template <typename T>
cudaError_t launch_bicg_xr_reduce(void* x, void* r, const void* sv, const void* phat, const void* shat,
                                  const void* t, const void* rhat, long long N, int R, double2* partials,
                                  const BicgScalars& sc, cudaStream_t s);

}  // namespace hx

namespace hx {
// out[r][i] = sum_j M[i][j] b[r][j]  (dense n x n complex matrix, row-major)
template <typename T>
cudaError_t launch_dense_matvec(const void* M, const void* b, void* out, long long n, int R,
                                cudaStream_t s);
}  // namespace hx
