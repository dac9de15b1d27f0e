// Matrix-free application of the adaptive 27-point operator [M + S] (Eq. 3).
//
// Each row is formed on the fly (Eqs. 4-8, GA weight selection of Section
// 3.1): the row's 1/G = f h / v indexes the weight table, whose derived
// entries are linearly interpolated; the stiffness is sum_d T_d[delta_d p]
// (stretched second difference along d, averaged over the transverse 3x3
// plane); the mass is the second form of Eq. 8 (kappa at the collocation
// point) with omega^2 optionally shifted to (1 + i beta) omega^2.
//
// Kernel layout (GB300): a CTA owns a TX x TY column tile and a z-range and
// marches along z.  Each step stages one x/y plane (tile + 1-node halo) of RB
// right-hand sides into a 3-plane shared-memory ring, so every x value is read
// from global memory once per CTA.  Per column and plane the in-plane class
// sums (centre, 4 in-plane faces, 4 in-plane corners) are computed once and
// kept in registers for the three z-steps that need them; an interior row
// (xi = 1 on all three axes) is then 4 class coefficients times 4 class sums.
// Rows in the PML use the general factored form with complex per-axis
// coefficients read from the ring.  Coefficients are formed once per point and
// reused across the RB right-hand sides.
#include "hx_complex.cuh"
#include "hx_internal.h"

namespace hx {
namespace {

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

template <typename T>
struct PointW {
  T w[11];   // interpolated derived table entries (see kTabW)
  T m;       // omega^2 / v^2
};

template <typename T>
__device__ __forceinline__ PointW<T> point_weights(const OpDesc<T>& op, float vv) {
  PointW<T> p;
  const T vt = (T)vv;
  T u = op.u_scale / vt;
  const T umax = (T)(op.n_g - 1);
  u = u < (T)0 ? (T)0 : (u > umax ? umax : u);
  int i0 = (int)u;
  if (i0 > op.n_g - 2) i0 = op.n_g - 2;
  const T t = u - (T)i0;
  const T* a = op.tab + (size_t)i0 * kTabW;
#pragma unroll
  for (int k = 0; k < 11; ++k) {
    const T lo = ldg(a + k), hi = ldg(a + kTabW + k);
    p.w[k] = fma(t, hi - lo, lo);
  }
  p.m = op.omega2 / (vt * vt);
  return p;
}

template <int TX, int TY, int RB, typename C>
struct Ring {
  C v[3][RB][TY + 2][TX + 2];
};

template <typename T, int MODE, bool SHIFT, int RB, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
stencil_kernel(OpDesc<T> op, const typename CT<T>::type* __restrict__ x,
               const typename CT<T>::type* __restrict__ b, typename CT<T>::type* __restrict__ y,
               int nrhs, long long rstride, int zchunk, T omega_j) {
  using C = typename CT<T>::type;
  __shared__ Ring<TX, TY, RB, C> ring;

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int gx0 = blockIdx.x * TX, gy0 = blockIdx.y * TY;
  const int ix = gx0 + tx, iy = gy0 + ty;
  const int nzc = (op.nz + zchunk - 1) / zchunk;
  const int zc = blockIdx.z % nzc, rblk = blockIdx.z / nzc;
  const int r0 = rblk * RB;
  const int rcount = min(RB, nrhs - r0);
  const int z0 = zc * zchunk, z1 = min(op.nz, z0 + zchunk);
  const bool active = ix < op.nx && iy < op.ny;
  const long long plane = (long long)op.nx * op.ny;

  auto load_plane = [&](int z, int slot) {
    for (int e = ty * TX + tx; e < (TY + 2) * (TX + 2); e += TX * TY) {
      const int ly = e / (TX + 2), lx = e - ly * (TX + 2);
      const int gx = gx0 + lx - 1, gy = gy0 + ly - 1;
      const bool ok = z >= 0 && z < op.nz && gx >= 0 && gx < op.nx && gy >= 0 && gy < op.ny;
      const long long off = (long long)z * plane + (long long)gy * op.nx + gx;
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        C val = czero<C>();
        if (ok && r < rcount) val = x[(long long)(r0 + r) * rstride + off];
        ring.v[slot][r][ly][lx] = val;
      }
    }
  };

  // in-plane class sums of column (tx, ty) in a slot: centre, faces, corners
  C cs[3][RB], es[3][RB], ks[3][RB];   // window index 0: z-1, 1: z, 2: z+1
  auto plane_sums = [&](int slot, int w) {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const auto& P = ring.v[slot][r];
      cs[w][r] = P[ty + 1][tx + 1];
      es[w][r] = cadd(cadd(P[ty + 1][tx], P[ty + 1][tx + 2]), cadd(P[ty][tx + 1], P[ty + 2][tx + 1]));
      ks[w][r] = cadd(cadd(P[ty][tx], P[ty][tx + 2]), cadd(P[ty + 2][tx], P[ty + 2][tx + 2]));
    }
  };

  // prologue: planes z0-1 and z0
  load_plane(z0 - 1, 0);
  load_plane(z0, 1);
  __syncthreads();
  plane_sums(0, 0);
  plane_sums(1, 1);

  const bool plain_xy = ix >= op.plain_lo[0] && ix <= op.plain_hi[0] && iy >= op.plain_lo[1] &&
                        iy <= op.plain_hi[1];

  for (int z = z0; z < z1; ++z) {
    const int s_m = (z - z0) % 3, s_0 = (z - z0 + 1) % 3, s_p = (z - z0 + 2) % 3;
    __syncthreads();               // everyone is done with the slot of plane z-2
    load_plane(z + 1, s_p);
    __syncthreads();
    plane_sums(s_p, 2);

    if (active) {
      const long long off = (long long)z * plane + (long long)iy * op.nx + ix;
      const PointW<T> pw = point_weights(op, __ldg(op.v + off));
      const T m = pw.m;
      const bool plain = plain_xy && z >= op.plain_lo[2] && z <= op.plain_hi[2];
      C out[RB];
      C diag;
      if (plain) {
        // interior row: class coefficients (stiffness real; mass m (1 + i beta))
        T a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = fma(m, pw.w[4 + k], pw.w[k] * op.inv_h2);
        diag = cmk(a[0], SHIFT ? op.beta * m * pw.w[4] : (T)0);
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const C c0 = cs[1][r];
          const C f6 = cadd(es[1][r], cadd(cs[0][r], cs[2][r]));
          const C e12 = cadd(ks[1][r], cadd(es[0][r], es[2][r]));
          const C c8 = cadd(ks[0][r], ks[2][r]);
          C acc = cscale(a[0], c0);
          acc = cfmar(a[1], f6, acc);
          acc = cfmar(a[2], e12, acc);
          acc = cfmar(a[3], c8, acc);
          if (SHIFT) {
            C ms = cscale(pw.w[4], c0);
            ms = cfmar(pw.w[5], f6, ms);
            ms = cfmar(pw.w[6], e12, ms);
            ms = cfmar(pw.w[7], c8, ms);
            acc = cadd(acc, cscale_i(op.beta * m, ms));
          }
          out[r] = acc;
        }
      } else {
        // PML row: general form sum_d up_d (F_d+ - F_d0) + dn_d (F_d- - F_d0)
        const T t0 = pw.w[8], t1 = pw.w[9], t2 = pw.w[10];
        const int idx[3] = {ix, iy, z};
        C up[3], dn[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T* q = op.axis[d] + 4 * (size_t)idx[d];
          up[d] = cmk(ldg(q), ldg(q + 1));
          dn[d] = cmk(ldg(q + 2), ldg(q + 3));
        }
        const C mc = cmk(m, SHIFT ? op.beta * m : (T)0);   // m (1 + i beta)
        C sdiag = cadd(cadd(up[0], dn[0]), cadd(cadd(up[1], dn[1]), cadd(up[2], dn[2])));
        diag = cfma(mc, cmk(pw.w[4], (T)0), cscale(-t0, sdiag));
        const int sl[3] = {s_m, s_0, s_p};
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          auto Q = [&](int dk, int dj, int di) -> C {
            return ring.v[sl[dk + 1]][r][ty + 1 + dj][tx + 1 + di];
          };
          C F[3][3];   // F[axis][s+1]
#pragma unroll
          for (int s = -1; s <= 1; ++s) {
            // x: transverse plane (dk, dj) at di = s
            C fx = cscale(t0, Q(0, 0, s));
            fx = cfmar(t1, cadd(cadd(Q(0, -1, s), Q(0, 1, s)), cadd(Q(-1, 0, s), Q(1, 0, s))), fx);
            fx = cfmar(t2, cadd(cadd(Q(-1, -1, s), Q(-1, 1, s)), cadd(Q(1, -1, s), Q(1, 1, s))), fx);
            F[0][s + 1] = fx;
            C fy = cscale(t0, Q(0, s, 0));
            fy = cfmar(t1, cadd(cadd(Q(0, s, -1), Q(0, s, 1)), cadd(Q(-1, s, 0), Q(1, s, 0))), fy);
            fy = cfmar(t2, cadd(cadd(Q(-1, s, -1), Q(-1, s, 1)), cadd(Q(1, s, -1), Q(1, s, 1))), fy);
            F[1][s + 1] = fy;
            C fz = cscale(t0, Q(s, 0, 0));
            fz = cfmar(t1, cadd(cadd(Q(s, 0, -1), Q(s, 0, 1)), cadd(Q(s, -1, 0), Q(s, 1, 0))), fz);
            fz = cfmar(t2, cadd(cadd(Q(s, -1, -1), Q(s, -1, 1)), cadd(Q(s, 1, -1), Q(s, 1, 1))), fz);
            F[2][s + 1] = fz;
          }
          C acc = czero<C>();
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            acc = cfma(up[d], csub(F[d][2], F[d][1]), acc);
            acc = cfma(dn[d], csub(F[d][0], F[d][1]), acc);
          }
          const C c0 = cs[1][r];
          const C f6 = cadd(es[1][r], cadd(cs[0][r], cs[2][r]));
          const C e12 = cadd(ks[1][r], cadd(es[0][r], es[2][r]));
          const C c8 = cadd(ks[0][r], ks[2][r]);
          C ms = cscale(pw.w[4], c0);
          ms = cfmar(pw.w[5], f6, ms);
          ms = cfmar(pw.w[6], e12, ms);
          ms = cfmar(pw.w[7], c8, ms);
          out[r] = cfma(mc, ms, acc);
        }
      }
      C dinv = czero<C>();
      if (MODE == kJacobi) dinv = crcp(diag);
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        if (r < rcount) {
          const long long o = (long long)(r0 + r) * rstride + off;
          C res = out[r];
          if (MODE == kResidual) res = b ? csub(b[o], res) : cmk(-res.x, -res.y);
          if (MODE == kJacobi) res = cfma(cscale(omega_j, dinv), csub(b[o], res), cs[1][r]);
          y[o] = res;
        }
      }
    }
    // shift the register window
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      cs[0][r] = cs[1][r]; es[0][r] = es[1][r]; ks[0][r] = ks[1][r];
      cs[1][r] = cs[2][r]; es[1][r] = es[2][r]; ks[1][r] = ks[2][r];
    }
  }
}

// First damped-Jacobi sweep from a zero guess: y = omega_j D^{-1} b, with D
// the row's diagonal coefficient (no neighbour reads).
template <typename T, bool SHIFT>
__global__ void jacobi0_kernel(OpDesc<T> op, const typename CT<T>::type* __restrict__ b,
                               typename CT<T>::type* __restrict__ y, int nrhs, long long rstride,
                               T omega_j) {
  using C = typename CT<T>::type;
  const long long N = (long long)op.nx * op.ny * op.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % op.nx);
    const int iy = (int)((i / op.nx) % op.ny);
    const int iz = (int)(i / ((long long)op.nx * op.ny));
    const PointW<T> pw = point_weights(op, __ldg(op.v + i));
    const int id[3] = {ix, iy, iz};
    C sdiag = czero<C>();
    for (int d = 0; d < 3; ++d) {
      const T* q = op.axis[d] + 4 * (size_t)id[d];
      sdiag = cadd(sdiag, cmk(ldg(q) + ldg(q + 2), ldg(q + 1) + ldg(q + 3)));
    }
    const C mc = cmk(pw.m, SHIFT ? op.beta * pw.m : (T)0);
    const C diag = cfma(mc, cmk(pw.w[4], (T)0), cscale(-pw.w[8], sdiag));
    const C f = cscale(omega_j, crcp(diag));
    for (int r = 0; r < nrhs; ++r) y[(long long)r * rstride + i] = cmul(f, b[(long long)r * rstride + i]);
  }
}

// One thread per row: the 27 coefficients in (dk, dj, di) order, FP64.
__global__ void row_coef_kernel(OpDesc<double> op, double2* __restrict__ coef) {
  const long long N = (long long)op.nx * op.ny * op.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % op.nx);
    const int iy = (int)((i / op.nx) % op.ny);
    const int iz = (int)(i / ((long long)op.nx * op.ny));
    const PointW<double> pw = point_weights(op, op.v[i]);
    const double tw[3] = {pw.w[8], pw.w[9], pw.w[10]};
    const double2 mc = make_double2(pw.m, op.beta * pw.m);
    const int id[3] = {ix, iy, iz};
    const int n[3] = {op.nx, op.ny, op.nz};
    double2 D[3][3];   // D[axis][s+1]
    for (int d = 0; d < 3; ++d) {
      const double* q = op.axis[d] + 4 * (size_t)id[d];
      const double2 up = make_double2(q[0], q[1]), dn = make_double2(q[2], q[3]);
      D[d][2] = up;
      D[d][0] = dn;
      D[d][1] = make_double2(-(up.x + dn.x), -(up.y + dn.y));
    }
    int k = 0;
    for (int dk = -1; dk <= 1; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di, ++k) {
          const int o[3] = {di, dj, dk};
          bool inside = true;
          for (int d = 0; d < 3; ++d) inside = inside && id[d] + o[d] >= 0 && id[d] + o[d] < n[d];
          double2 c = make_double2(0.0, 0.0);
          if (inside) {
            c = cfmar(tw[abs(dj) + abs(dk)], D[0][di + 1], c);
            c = cfmar(tw[abs(di) + abs(dk)], D[1][dj + 1], c);
            c = cfmar(tw[abs(di) + abs(dj)], D[2][dk + 1], c);
            c = cfma(mc, make_double2(pw.w[4 + abs(di) + abs(dj) + abs(dk)], 0.0), c);
          }
          coef[i * 27 + k] = c;
        }
  }
}

int pick_zchunk(int nz, int ntiles_xy, int nrb) {
  const int target = 152 * 8;
  int nzc = (target + ntiles_xy * nrb - 1) / (ntiles_xy * nrb);
  nzc = nzc < 1 ? 1 : nzc;
  int zc = (nz + nzc - 1) / nzc;
  return zc < 4 ? 4 : zc;
}

template <typename T, int MODE, bool SHIFT, int RB>
cudaError_t launch_t(const OpDesc<T>& op, const void* x, const void* b, void* y, int nrhs,
                     long long rstride, double omega_j, cudaStream_t s) {
  constexpr int TX = 32, TY = 8;
  using C = typename CT<T>::type;
  const int bx = (op.nx + TX - 1) / TX, by = (op.ny + TY - 1) / TY;
  const int nrb = (nrhs + RB - 1) / RB;
  const int zchunk = pick_zchunk(op.nz, bx * by, nrb);
  const int nzc = (op.nz + zchunk - 1) / zchunk;
  const long long gz = (long long)nzc * nrb;
  if (gz > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid(bx, by, (unsigned)gz), block(TX, TY);
  stencil_kernel<T, MODE, SHIFT, RB, TX, TY><<<grid, block, 0, s>>>(
      op, (const C*)x, (const C*)b, (C*)y, nrhs, rstride, zchunk, (T)omega_j);
  count_launch(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_j0(const OpDesc<T>& op, const void* b, void* y, int nrhs, long long rstride,
                      double omega_j, cudaStream_t s) {
  using C = typename CT<T>::type;
  const long long N = (long long)op.nx * op.ny * op.nz;
  long long blocks = (N + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (op.beta != 0)
    jacobi0_kernel<T, true><<<(unsigned)blocks, 256, 0, s>>>(op, (const C*)b, (C*)y, nrhs, rstride, (T)omega_j);
  else
    jacobi0_kernel<T, false><<<(unsigned)blocks, 256, 0, s>>>(op, (const C*)b, (C*)y, nrhs, rstride, (T)omega_j);
  count_launch(1);
  return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t launch_m(const OpDesc<T>& op, const void* x, const void* b, void* y, int nrhs,
                     long long rstride, double omega_j, cudaStream_t s) {
  constexpr int RB = sizeof(T) == 4 ? 4 : 2;
  if (nrhs == 1) {
    return op.beta != 0 ? launch_t<T, MODE, true, 1>(op, x, b, y, nrhs, rstride, omega_j, s)
                        : launch_t<T, MODE, false, 1>(op, x, b, y, nrhs, rstride, omega_j, s);
  }
  return op.beta != 0 ? launch_t<T, MODE, true, RB>(op, x, b, y, nrhs, rstride, omega_j, s)
                      : launch_t<T, MODE, false, RB>(op, x, b, y, nrhs, rstride, omega_j, s);
}

}  // namespace

template <typename T>
cudaError_t launch_stencil(const OpDesc<T>& op, int mode, const void* x, const void* b, void* y,
                           int nrhs, long long rstride, double omega_j, cudaStream_t s) {
  switch (mode) {
    case kApply: return launch_m<T, kApply>(op, x, b, y, nrhs, rstride, omega_j, s);
    case kResidual: return launch_m<T, kResidual>(op, x, b, y, nrhs, rstride, omega_j, s);
    case kJacobi: return launch_m<T, kJacobi>(op, x, b, y, nrhs, rstride, omega_j, s);
    case kJacobi0: return launch_j0<T>(op, b, y, nrhs, rstride, omega_j, s);
  }
  return cudaErrorInvalidValue;
}

template cudaError_t launch_stencil<float>(const OpDesc<float>&, int, const void*, const void*,
                                           void*, int, long long, double, cudaStream_t);
template cudaError_t launch_stencil<double>(const OpDesc<double>&, int, const void*, const void*,
                                            void*, int, long long, double, cudaStream_t);

cudaError_t launch_row_coefficients(const OpDesc<double>& op, double* coef, cudaStream_t s) {
  const long long N = (long long)op.nx * op.ny * op.nz;
  long long blocks = (N + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  row_coef_kernel<<<(unsigned)blocks, 256, 0, s>>>(op, (double2*)coef);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace hx
