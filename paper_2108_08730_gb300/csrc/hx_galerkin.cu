// Galerkin coarse operators of the multigrid preconditioner and the kernels
// that apply stored 27-point operators on the coarse levels.
//
// Not in the paper.  A_c = R A P with R full weighting and P trilinear
// interpolation on vertex-centred grids (R = P^T / 8): with a 27-point fine
// operator the coarse operator is again 27-point.  The fine operator of level
// 0 is formed on the fly (the adaptive row of Eqs. 4-8 with the shifted mass);
// deeper levels take the stored coefficients of the level above.  Coefficients
// are stored offset-major, coef[k][i] for offset k = (dk+1)*9 + (dj+1)*3 +
// (di+1), so a warp reads each offset's coefficients coalesced.
#include "hx_complex.cuh"
#include "hx_galerkin.cuh"
#include "hx_internal.h"
#include "hx_launch.cuh"
#include "hx_row.cuh"

namespace hx {
namespace {

// trilinear weight of fine offset r (relative to 2I, in [-2, 2]) for coarse
// offset D in {-1, 0, 1}
__device__ __forceinline__ float pw1(int r, int D) {
  const int d = r - 2 * D;
  return d == 0 ? 1.f : (d == 1 || d == -1 ? 0.5f : 0.f);
}

template <typename T, bool ONFLY>
__global__ void __launch_bounds__(128)
galerkin_k(OpDesc<T> op, const typename CT<T>::type* __restrict__ cf, int fx, int fy, int fz,
           typename CT<T>::type* __restrict__ cc, int cx, int cy, int cz) {
  pdl_enter();
  using C = typename CT<T>::type;
  const long long Nc = (long long)cx * cy * cz, Nf = (long long)fx * fy * fz;
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < Nc;
       I += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(I % cx), Y = (int)((I / cx) % cy), Z = (int)(I / ((long long)cx * cy));
    C acc[27];
#pragma unroll
    for (int k = 0; k < 27; ++k) acc[k] = czero<C>();
    for (int s = 0; s < 27; ++s) {
      const int sx = s % 3 - 1, sy = (s / 3) % 3 - 1, sz = s / 9 - 1;
      const int ix = 2 * X + sx, iy = 2 * Y + sy, iz = 2 * Z + sz;
      if (ix < 0 || ix >= fx || iy < 0 || iy >= fy || iz < 0 || iz >= fz) continue;
      const T wr = (T)1 / (T)(8 << (abs(sx) + abs(sy) + abs(sz)));
      C a[27];
      if (ONFLY) {
        fine_row<T>(op, ix, iy, iz, a);
      } else {
        const long long i = ix + (long long)fx * (iy + (long long)fy * iz);
#pragma unroll
        for (int k = 0; k < 27; ++k) a[k] = cf[(long long)k * Nf + i];
      }
#pragma unroll
      for (int k = 0; k < 27; ++k) {
        const int oi = k % 3 - 1, oj = (k / 3) % 3 - 1, ok = k / 9 - 1;
        const int jx = ix + oi, jy = iy + oj, jz = iz + ok;
        if (jx < 0 || jx >= fx || jy < 0 || jy >= fy || jz < 0 || jz >= fz) continue;
        const C c = cscale(wr, a[k]);
        const int rx = sx + oi, ry = sy + oj, rz = sz + ok;   // in [-2, 2]
#pragma unroll
        for (int q = 0; q < 27; ++q) {
          const int Dx = q % 3 - 1, Dy = (q / 3) % 3 - 1, Dz = q / 9 - 1;
          const float p = pw1(rx, Dx) * pw1(ry, Dy) * pw1(rz, Dz);
          if (p != 0.f) {
            const int Jx = X + Dx, Jy = Y + Dy, Jz = Z + Dz;
            if (Jx >= 0 && Jx < cx && Jy >= 0 && Jy < cy && Jz >= 0 && Jz < cz)
              acc[q] = cfmar((T)p, c, acc[q]);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 27; ++k) cc[(long long)k * Nc + I] = acc[k];
  }
}

// y = A x / b - A x / x + w D^-1 (b - A x) / w D^-1 b with stored coefficients
template <typename T, int MODE>
__global__ void __launch_bounds__(256)
stored_stencil_k(const typename CT<T>::type* __restrict__ coef, int nx, int ny, int nz,
                 const typename CT<T>::type* __restrict__ x, const typename CT<T>::type* __restrict__ b,
                 typename CT<T>::type* __restrict__ y, int R, T omega_j) {
  pdl_enter();
  using C = typename CT<T>::type;
  const long long N = (long long)nx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long long)nx * ny));
    const C dg = coef[13 * N + i];
    const C dinv = cscale(omega_j, crcp(dg));
    if (MODE == kJacobi0) {
      for (int r = 0; r < R; ++r) y[(long long)r * N + i] = cmul(dinv, b[(long long)r * N + i]);
      continue;
    }
    for (int r = 0; r < R; ++r) {
      const C* xr = x + (long long)r * N;
      C acc = czero<C>();
#pragma unroll
      for (int k = 0; k < 27; ++k) {
        const int di = k % 3 - 1, dj = (k / 3) % 3 - 1, dk = k / 9 - 1;
        const int jx = ix + di, jy = iy + dj, jz = iz + dk;
        if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
        acc = cfma(coef[(long long)k * N + i], xr[i + di + (long long)nx * (dj + (long long)ny * dk)], acc);
      }
      const long long o = (long long)r * N + i;
      C res = acc;
      if (MODE == kResidual) res = csub(b[o], acc);
      if (MODE == kJacobi) res = cfma(dinv, csub(b[o], acc), xr[i]);
      y[o] = res;
    }
  }
}

// Small grids (coarse multigrid levels): one thread per row, the 27
// coefficients formed on the fly (the same row as the tiled kernel) and the
// neighbours read through the read-only cache.  A z-marching tiled kernel is
// latency-bound when a level has only a few tiles.
template <typename T, int MODE, bool MED>
__global__ void __launch_bounds__(128)
direct_stencil_k(OpDesc<T> op, const typename CT<T>::type* __restrict__ x,
                 const typename CT<T>::type* __restrict__ b, typename CT<T>::type* __restrict__ y,
                 int R, T omega_j) {
  pdl_enter();
  using C = typename CT<T>::type;
  const long long N = (long long)op.nx * op.ny * op.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % op.nx), iy = (int)((i / op.nx) % op.ny), iz = (int)(i / ((long long)op.nx * op.ny));
    C a[27];
    fine_row<T, MED>(op, ix, iy, iz, a);
    const C dinv = cscale(omega_j, crcp(a[13]));
    for (int r = 0; r < R; ++r) {
      const long long o = (long long)r * N + i;
      if (MODE == kJacobi0) {
        y[o] = cmul(dinv, __ldg(b + o));
        continue;
      }
      const C* xr = x + (long long)r * N;
      C acc = czero<C>();
#pragma unroll
      for (int k = 0; k < 27; ++k) {
        const int di = k % 3 - 1, dj = (k / 3) % 3 - 1, dk = k / 9 - 1;
        const int jx = ix + di, jy = iy + dj, jz = iz + dk;
        if (jx < 0 || jx >= op.nx || jy < 0 || jy >= op.ny || jz < 0 || jz >= op.nz) continue;
        acc = cfma(a[k], __ldg(xr + i + di + (long long)op.nx * (dj + (long long)op.ny * dk)), acc);
      }
      C res = acc;
      if (MODE == kResidual) res = b ? csub(__ldg(b + o), acc) : cmk(-acc.x, -acc.y);
      if (MODE == kJacobi) res = cfma(dinv, csub(__ldg(b + o), acc), __ldg(xr + i));
      y[o] = res;
    }
  }
}

unsigned blocks_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

}  // namespace

template <typename T>
cudaError_t launch_galerkin_onfly(const OpDesc<T>& fine, void* coarse_coef, const int nc[3],
                                  cudaStream_t s) {
  using C = typename CT<T>::type;
  const long long Nc = (long long)nc[0] * nc[1] * nc[2];
  (void)launch_k(galerkin_k<T, true>, blocks_for(Nc, 128, 152 * 64), 128, 0, s,
      fine, nullptr, fine.nx, fine.ny, fine.nz, (C*)coarse_coef, nc[0], nc[1], nc[2]);
  count_launch(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_galerkin_stored(const void* fine_coef, const int nf[3], void* coarse_coef,
                                   const int nc[3], cudaStream_t s) {
  using C = typename CT<T>::type;
  const long long Nc = (long long)nc[0] * nc[1] * nc[2];
  OpDesc<T> dummy{};
  (void)launch_k(galerkin_k<T, false>, blocks_for(Nc, 128, 152 * 64), 128, 0, s,
      dummy, (const C*)fine_coef, nf[0], nf[1], nf[2], (C*)coarse_coef, nc[0], nc[1], nc[2]);
  count_launch(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stored_stencil(const void* coef, const int n[3], int mode, const void* x,
                                  const void* b, void* y, int R, double omega_j, cudaStream_t s) {
  using C = typename CT<T>::type;
  const long long N = (long long)n[0] * n[1] * n[2];
  const unsigned g = blocks_for(N, 256, 152 * 16);
  switch (mode) {
    case kApply:
      (void)launch_k(stored_stencil_k<T, kApply>, g, 256, 0, s, (const C*)coef, n[0], n[1], n[2], (const C*)x,
                                                    (const C*)b, (C*)y, R, (T)omega_j);
      break;
    case kResidual:
      (void)launch_k(stored_stencil_k<T, kResidual>, g, 256, 0, s, (const C*)coef, n[0], n[1], n[2], (const C*)x,
                                                       (const C*)b, (C*)y, R, (T)omega_j);
      break;
    case kJacobi:
      (void)launch_k(stored_stencil_k<T, kJacobi>, g, 256, 0, s, (const C*)coef, n[0], n[1], n[2], (const C*)x,
                                                     (const C*)b, (C*)y, R, (T)omega_j);
      break;
    case kJacobi0:
      (void)launch_k(stored_stencil_k<T, kJacobi0>, g, 256, 0, s, (const C*)coef, n[0], n[1], n[2], (const C*)x,
                                                      (const C*)b, (C*)y, R, (T)omega_j);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  count_launch(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_direct_stencil(const OpDesc<T>& op, int mode, const void* x, const void* b, void* y,
                                  int R, double omega_j, cudaStream_t s) {
  using C = typename CT<T>::type;
  const long long N = (long long)op.nx * op.ny * op.nz;
  const unsigned g = blocks_for(N, 128, 152 * 32);
  const T om = (T)omega_j;
  const bool med = op.buoy || op.invq;
#define HX_DIRECT(M)                                                                                    \
  (med ? launch_k(direct_stencil_k<T, M, true>, g, 128, 0, s, op, (const C*)x, (const C*)b, (C*)y, R, om) \
       : launch_k(direct_stencil_k<T, M, false>, g, 128, 0, s, op, (const C*)x, (const C*)b, (C*)y, R, om))
  switch (mode) {
    case kApply: (void)HX_DIRECT(kApply); break;
    case kResidual: (void)HX_DIRECT(kResidual); break;
    case kJacobi: (void)HX_DIRECT(kJacobi); break;
    case kJacobi0: (void)HX_DIRECT(kJacobi0); break;
    default: return cudaErrorInvalidValue;
  }
#undef HX_DIRECT
  count_launch(1);
  return cudaGetLastError();
}
template cudaError_t launch_direct_stencil<float>(const OpDesc<float>&, int, const void*, const void*, void*,
                                                  int, double, cudaStream_t);
template cudaError_t launch_direct_stencil<double>(const OpDesc<double>&, int, const void*, const void*, void*,
                                                   int, double, cudaStream_t);

#define HX_GAL_INST(T)                                                                             \
  template cudaError_t launch_galerkin_onfly<T>(const OpDesc<T>&, void*, const int*, cudaStream_t); \
  template cudaError_t launch_galerkin_stored<T>(const void*, const int*, void*, const int*,       \
                                                 cudaStream_t);                                    \
  template cudaError_t launch_stored_stencil<T>(const void*, const int*, int, const void*,         \
                                                const void*, void*, int, double, cudaStream_t);
HX_GAL_INST(float)
HX_GAL_INST(double)

}  // namespace hx
