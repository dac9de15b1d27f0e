// Matrix-free application of the adaptive 27-point operator [M + S] (Eq. 3).
//
// Each row is formed on the fly (Eqs. 4-8, GA weight selection of Section
// 3.1): the row's 1/G = f h / v indexes the weight table, whose derived
// entries are linearly interpolated; the stiffness is sum_d T_d[delta_d p]
// (stretched second difference along d, averaged over the transverse 3x3
// plane); the mass is the second form of Eq. 8 (kappa at the collocation
// point) with omega^2 optionally shifted to (1 + i beta) omega^2.
//
// Kernel layout (GB300):
//  * a CTA owns a TX x TY column tile, RB right-hand sides and a z-range, and
//    marches along z;
//  * x planes (tile + 1-node halo, RB fields) stream into an NSLOT-plane
//    shared-memory ring with cp.async (8/16-byte copies, zero-filled outside
//    the grid), NSLOT - 3 planes ahead of the one being consumed, so global
//    latency overlaps compute; one barrier per z-step;
//  * per column and plane the in-plane class sums (centre, 4 in-plane faces,
//    4 in-plane corners) are computed once and kept in registers for the three
//    z-steps that need them: an interior row is 4 class coefficients times 4
//    class sums; a row whose only complex stretching is along z adds the
//    z-terms from the same registers; rows in the x/y PML use the general
//    factored form read from the ring;
//  * the table of derived weights is staged in shared memory;
//  * RHS blocks are the fastest grid index, so neighbouring CTAs re-read the
//    same velocity tile from L2 rather than HBM.
#include <cuda_pipeline_primitives.h>

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
__device__ __forceinline__ PointW<T> point_weights(const OpDesc<T>& op, const T* tab, float vv) {
  PointW<T> p;
  const T vt = (T)vv;
  const T iv = (T)1 / vt;
  T u = op.u_scale * iv;
  const T umax = (T)(op.n_g - 1);
  u = u < (T)0 ? (T)0 : (u > umax ? umax : u);
  int i0 = (int)u;
  if (i0 > op.n_g - 2) i0 = op.n_g - 2;
  const T t = u - (T)i0;
  const T* a = tab + (size_t)i0 * kTabW;
#pragma unroll
  for (int k = 0; k < 11; ++k) {
    const T lo = a[k], hi = a[kTabW + k];
    p.w[k] = fma(t, hi - lo, lo);
  }
  p.m = op.omega2 * iv * iv;
  return p;
}

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes, bool ok) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(ok ? 8 : 0));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(ok ? 16 : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

constexpr int kTX = 32, kTY = 8, kNSlot = 6, kDist = kNSlot - 3;

template <typename T, int RB>
__host__ __device__ constexpr size_t ring_bytes() {
  return (size_t)kNSlot * RB * (kTY + 2) * (kTX + 2) * sizeof(typename CT<T>::type);
}

template <typename T, int MODE, bool SHIFT, int RB>
__global__ void __launch_bounds__(kTX * kTY, sizeof(T) == 4 ? 3 : 2)
stencil_kernel(OpDesc<T> op, const typename CT<T>::type* __restrict__ x,
               const typename CT<T>::type* __restrict__ b, typename CT<T>::type* __restrict__ y,
               int nrhs, long long rstride, int zchunk, T omega_j, int tab_in_smem) {
  using C = typename CT<T>::type;
  constexpr int TX = kTX, TY = kTY, PW = TX + 2, PH = TY + 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* ring = reinterpret_cast<C*>(smem_raw);                        // [NSLOT][RB][PH][PW]
  T* tab_s = reinterpret_cast<T*>(smem_raw + ring_bytes<T, RB>());
  auto R = [&](int slot, int r, int ly, int lx) -> C& {
    return ring[((slot * RB + r) * PH + ly) * PW + lx];
  };

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int gx0 = blockIdx.x * TX, gy0 = blockIdx.y * TY;
  const int ix = gx0 + tx, iy = gy0 + ty;
  const int nrb = (nrhs + RB - 1) / RB;
  const int rblk = blockIdx.z % nrb, zc = blockIdx.z / nrb;
  const int r0 = rblk * RB;
  const int rcount = min(RB, nrhs - r0);
  const int z0 = zc * zchunk, z1 = min(op.nz, z0 + zchunk);
  const bool active = ix < op.nx && iy < op.ny;
  const long long plane = (long long)op.nx * op.ny;

  // stage the derived table (or read it from global memory when too large)
  const T* tab = op.tab;
  if (tab_in_smem) {
    for (int i = tid; i < op.n_g * kTabW; i += TX * TY) tab_s[i] = op.tab[i];
    tab = tab_s;
  }

  // issue the asynchronous copies of plane z (all RB fields) into slot
  auto issue_plane = [&](int z) {
    if (z < z0 - 1 || z > z1) return;                     // not needed by this CTA
    const int slot = (z - z0 + 1) % kNSlot;
    const bool zin = z >= 0 && z < op.nz;
    for (int e = tid; e < PH * PW; e += TX * TY) {
      const int ly = e / PW, lx = e - ly * PW;
      const int gx = gx0 + lx - 1, gy = gy0 + ly - 1;
      const bool ok = zin && gx >= 0 && gx < op.nx && gy >= 0 && gy < op.ny;
      const long long off = ok ? (long long)z * plane + (long long)gy * op.nx + gx : 0;
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const bool okr = ok && r < rcount;
        const C* src = x + (okr ? (long long)(r0 + r) * rstride + off : 0);
        cp_async(&R(slot, r, ly, lx), src, (int)sizeof(C), okr);
      }
    }
  };

  // in-plane class sums of column (tx, ty): centre, 4 faces, 4 corners
  C cs[3][RB], es[3][RB], ks[3][RB];   // window: 0 -> z-1, 1 -> z, 2 -> z+1
  auto plane_sums = [&](int z, int w) {
    const int slot = (z - z0 + 1) % kNSlot;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      cs[w][r] = R(slot, r, ty + 1, tx + 1);
      es[w][r] = cadd(cadd(R(slot, r, ty + 1, tx), R(slot, r, ty + 1, tx + 2)),
                      cadd(R(slot, r, ty, tx + 1), R(slot, r, ty + 2, tx + 1)));
      ks[w][r] = cadd(cadd(R(slot, r, ty, tx), R(slot, r, ty, tx + 2)),
                      cadd(R(slot, r, ty + 2, tx), R(slot, r, ty + 2, tx + 2)));
    }
  };

  // prologue: planes z0-1 .. z0+kDist in flight, one commit group per plane
  for (int k = -1; k <= kDist; ++k) {
    issue_plane(z0 + k);
    cp_commit();
  }
  cp_wait<kDist>();                // planes z0-1 and z0 have landed
  __syncthreads();
  plane_sums(z0 - 1, 0);
  plane_sums(z0, 1);

  const bool plain_x = ix >= op.plain_lo[0] && ix <= op.plain_hi[0];
  const bool plain_y = iy >= op.plain_lo[1] && iy <= op.plain_hi[1];
  const bool plain_xy = plain_x && plain_y;
  float v_next = active && z0 < z1 ? __ldg(op.v + (long long)z0 * plane + (long long)iy * op.nx + ix) : 1.f;

  for (int z = z0; z < z1; ++z) {
    cp_wait<kDist - 1>();          // plane z+1 has landed (own copies)
    __syncthreads();               // ... for every thread; step z-1 finished everywhere
    issue_plane(z + kDist + 1);    // into the slot of plane z-2
    cp_commit();
    plane_sums(z + 1, 2);

    const float vv = v_next;
    if (active && z + 1 < z1) v_next = __ldg(op.v + (long long)(z + 1) * plane + (long long)iy * op.nx + ix);

    if (active) {
      const long long off = (long long)z * plane + (long long)iy * op.nx + ix;
      const PointW<T> pw = point_weights(op, tab, vv);
      const T m = pw.m;
      const bool plain_z = z >= op.plain_lo[2] && z <= op.plain_hi[2];
      if (plain_xy) {
        // interior-like row: class form, plus z-stretching corrections
        T a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = fma(m, pw.w[4 + k], pw.w[k] * op.inv_h2);
        C diag = cmk(a[0], SHIFT ? op.beta * m * pw.w[4] : (T)0);
        C duz = czero<C>(), ddz = czero<C>();
        if (!plain_z) {
          const T* q = op.axis[2] + 4 * (size_t)z;
          duz = cmk(ldg(q) - op.inv_h2, ldg(q + 1));
          ddz = cmk(ldg(q + 2) - op.inv_h2, ldg(q + 3));
          diag = csub(diag, cscale(pw.w[8], cadd(duz, ddz)));
        }
        C dinv = czero<C>();
        if (MODE == kJacobi) dinv = cscale(omega_j, crcp(diag));
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
          if (!plain_z) {
            // F_z(s) = t0 c(z+s) + t1 faces(z+s) + t2 corners(z+s)
            const T t0 = pw.w[8], t1 = pw.w[9], t2 = pw.w[10];
            const C fzm = cfmar(t2, ks[0][r], cfmar(t1, es[0][r], cscale(t0, cs[0][r])));
            const C fz0 = cfmar(t2, ks[1][r], cfmar(t1, es[1][r], cscale(t0, cs[1][r])));
            const C fzp = cfmar(t2, ks[2][r], cfmar(t1, es[2][r], cscale(t0, cs[2][r])));
            acc = cfma(duz, csub(fzp, fz0), acc);
            acc = cfma(ddz, csub(fzm, fz0), acc);
          }
          if (r < rcount) {
            const long long o = (long long)(r0 + r) * rstride + off;
            C res = acc;
            if (MODE == kResidual) res = b ? csub(b[o], res) : cmk(-res.x, -res.y);
            if (MODE == kJacobi) res = cfma(dinv, csub(b[o], res), c0);
            y[o] = res;
          }
        }
      } else {
        // x/y PML row: general form sum_d up_d (F_d+ - F_d0) + dn_d (F_d- - F_d0)
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
        const C sdiag = cadd(cadd(up[0], dn[0]), cadd(cadd(up[1], dn[1]), cadd(up[2], dn[2])));
        const C diag = cfma(mc, cmk(pw.w[4], (T)0), cscale(-t0, sdiag));
        C dinv = czero<C>();
        if (MODE == kJacobi) dinv = cscale(omega_j, crcp(diag));
        // Streams the three z-planes of the 27-point neighbourhood: Fx[i]
        // accumulates the transverse (y,z) average of the column at x-offset
        // i-1, Fy[j] that of the row at y-offset j-1; the z-term and the mass
        // are added plane by plane.
        const C dz_m = dn[2], dz_p = up[2], dz_0 = cmk(-(up[2].x + dn[2].x), -(up[2].y + dn[2].y));
#pragma unroll 1
        for (int r = 0; r < rcount; ++r) {
          C Fx[3] = {czero<C>(), czero<C>(), czero<C>()};
          C Fy[3] = {czero<C>(), czero<C>(), czero<C>()};
          C acc = czero<C>(), ms = czero<C>(), xc = czero<C>();
#pragma unroll 1
          for (int dk = -1; dk <= 1; ++dk) {
            const int slot = (z - z0 + 1 + dk) % kNSlot;
            C q[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
              for (int i = 0; i < 3; ++i) q[j][i] = R(slot, r, ty + j, tx + i);
            const bool off_plane = dk != 0;
            const T ta = off_plane ? t1 : t0;      // transverse weight at in-plane offset 0
            const T tb = off_plane ? t2 : t1;      // ... at in-plane offset 1
#pragma unroll
            for (int i = 0; i < 3; ++i) Fx[i] = cfmar(tb, cadd(q[0][i], q[2][i]), cfmar(ta, q[1][i], Fx[i]));
#pragma unroll
            for (int j = 0; j < 3; ++j) Fy[j] = cfmar(tb, cadd(q[j][0], q[j][2]), cfmar(ta, q[j][1], Fy[j]));
            const C faces = cadd(cadd(q[1][0], q[1][2]), cadd(q[0][1], q[2][1]));
            const C corners = cadd(cadd(q[0][0], q[0][2]), cadd(q[2][0], q[2][2]));
            const C tp = cfmar(t2, corners, cfmar(t1, faces, cscale(t0, q[1][1])));
            const C dzk = dk < 0 ? dz_m : (dk > 0 ? dz_p : dz_0);
            acc = cfma(dzk, tp, acc);
            const T mw0 = off_plane ? pw.w[5] : pw.w[4];
            const T mw1 = off_plane ? pw.w[6] : pw.w[5];
            const T mw2 = off_plane ? pw.w[7] : pw.w[6];
            ms = cfmar(mw2, corners, cfmar(mw1, faces, cfmar(mw0, q[1][1], ms)));
            if (!off_plane) xc = q[1][1];
          }
          acc = cfma(up[0], csub(Fx[2], Fx[1]), acc);
          acc = cfma(dn[0], csub(Fx[0], Fx[1]), acc);
          acc = cfma(up[1], csub(Fy[2], Fy[1]), acc);
          acc = cfma(dn[1], csub(Fy[0], Fy[1]), acc);
          acc = cfma(mc, ms, acc);
          const long long o = (long long)(r0 + r) * rstride + off;
          C res = acc;
          if (MODE == kResidual) res = b ? csub(b[o], res) : cmk(-res.x, -res.y);
          if (MODE == kJacobi) res = cfma(dinv, csub(b[o], res), xc);
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
  cp_wait<0>();
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
    const PointW<T> pw = point_weights(op, op.tab, __ldg(op.v + i));
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
    const PointW<double> pw = point_weights(op, op.tab, op.v[i]);
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

int pick_zchunk(int nz, int ntiles_xy, int nrb, int ctas_per_sm) {
  const int target = 152 * ctas_per_sm * 2;
  int nzc = (target + ntiles_xy * nrb - 1) / (ntiles_xy * nrb);
  nzc = nzc < 1 ? 1 : nzc;
  int zc = (nz + nzc - 1) / nzc;
  return zc < 8 ? 8 : zc;
}

template <typename T, int MODE, bool SHIFT, int RB>
cudaError_t launch_t(const OpDesc<T>& op, const void* x, const void* b, void* y, int nrhs,
                     long long rstride, double omega_j, cudaStream_t s) {
  using C = typename CT<T>::type;
  const int bx = (op.nx + kTX - 1) / kTX, by = (op.ny + kTY - 1) / kTY;
  const int nrb = (nrhs + RB - 1) / RB;
  const size_t tab_bytes = (size_t)op.n_g * kTabW * sizeof(T);
  const int tab_in_smem = tab_bytes <= 48 * 1024 ? 1 : 0;
  const size_t smem = ring_bytes<T, RB>() + (tab_in_smem ? tab_bytes : 0);
  auto kern = stencil_kernel<T, MODE, SHIFT, RB>;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(ring_bytes<T, RB>() + 48 * 1024));
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  const int zchunk = pick_zchunk(op.nz, bx * by, nrb, sizeof(T) == 4 ? 3 : 2);
  const int nzc = (op.nz + zchunk - 1) / zchunk;
  const long long gz = (long long)nzc * nrb;
  if (gz > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid(bx, by, (unsigned)gz), block(kTX, kTY);
  kern<<<grid, block, smem, s>>>(op, (const C*)x, (const C*)b, (C*)y, nrhs, rstride, zchunk, (T)omega_j,
                                 tab_in_smem);
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
  constexpr int RB = sizeof(T) == 4 ? 2 : 1;
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
