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
#include "hx_galerkin.cuh"
#include "hx_launch.cuh"
#include "hx_row.cuh"
#include "hx_zmarch.cuh"

namespace hx {
namespace {

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

template <typename T>
struct PointW {
  T w[11];   // interpolated derived table entries (see kTabW)
  T m;       // omega^2 / v^2
};

// 4-wide read-only loads of table entries (a node is 12 entries = 3 x 4)
__device__ __forceinline__ void ld4(const float* p, float* o) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double* o) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

// Table position of a row: node i0 and fraction t of 1/G = f h / v.
template <typename T>
struct TabPos {
  const T* a;   // node i0 (node i0 + 1 follows at a + kTabW)
  T t;
  T m;          // omega^2 / v^2
};

template <typename T>
__device__ __forceinline__ TabPos<T> tab_pos(const OpDesc<T>& op, const T* tab, float vv) {
  TabPos<T> q;
  const T vt = (T)vv;
  const T iv = (T)1 / vt;
  T u = op.u_scale * iv;
  const T umax = (T)(op.n_g - 1);
  u = u < (T)0 ? (T)0 : (u > umax ? umax : u);
  int i0 = (int)u;
  if (i0 > op.n_g - 2) i0 = op.n_g - 2;
  q.t = u - (T)i0;
  q.a = tab + (size_t)i0 * kTabW;
  q.m = op.omega2 * iv * iv;
  return q;
}

// entries [4g, 4g+4) of the interpolated row weights
template <typename T>
__device__ __forceinline__ void tab_lerp4(const TabPos<T>& q, int g, T* w) {
  T lo[4], hi[4];
  ld4(q.a + 4 * g, lo);
  ld4(q.a + kTabW + 4 * g, hi);
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = fma(q.t, hi[k] - lo[k], lo[k]);
}

template <typename T>
__device__ __forceinline__ PointW<T> point_weights(const OpDesc<T>& op, const T* tab, float vv) {
  PointW<T> p;
  const TabPos<T> q = tab_pos(op, tab, vv);
  T w12[12];
  tab_lerp4(q, 0, w12);
  tab_lerp4(q, 1, w12 + 4);
  tab_lerp4(q, 2, w12 + 8);
#pragma unroll
  for (int k = 0; k < 11; ++k) p.w[k] = w12[k];
  p.m = q.m;
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

constexpr int kTX = 16, kTY = 16, kNSlot = 6, kDist = kNSlot - 3;
constexpr int kPW = kTX + 2, kPH = kTY + 2, kPlane = kPW * kPH;   // ring plane (tile + halo)
constexpr int kLoadIters = (kPlane + kTX * kTY - 1) / (kTX * kTY);

template <typename T, int RB>
__host__ __device__ constexpr size_t ring_bytes() {
  return (size_t)kNSlot * RB * kPlane * sizeof(typename CT<T>::type);
}

__device__ __forceinline__ int next_slot(int s) { return s + 1 == kNSlot ? 0 : s + 1; }

template <typename T, int MODE, bool SHIFT, int RB>
__global__ void __launch_bounds__(kTX * kTY, sizeof(T) == 4 ? 3 : 2)
stencil_kernel(OpDesc<T> op, const typename CT<T>::type* __restrict__ x,
               const typename CT<T>::type* __restrict__ b, typename CT<T>::type* __restrict__ y,
               int nrhs, long long rstride, int zchunk, T omega_j) {
  pdl_enter();
  using C = typename CT<T>::type;
  constexpr int TX = kTX, TY = kTY, PW = kPW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* ring = reinterpret_cast<C*>(smem_raw);                        // [NSLOT][RB][PH][PW]
  // this thread's 3x3 window in (slot, rhs) plane: element (dy, dx) at [dy * PW + dx]
  auto P = [&](int slot, int r) -> const C* { return ring + (slot * RB + r) * kPlane + threadIdx.y * PW + threadIdx.x; };

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
  const T* tab = op.tab;

  // loader descriptors, fixed for the CTA: the ring elements this thread
  // copies, their offsets inside a z-plane, and whether they lie in the grid
  int ld_s[kLoadIters];
  int ld_g[kLoadIters];
  bool ld_ok[kLoadIters];
#pragma unroll
  for (int k = 0; k < kLoadIters; ++k) {
    const int e = tid + k * TX * TY;
    const int ly = e / PW, lx = e - ly * PW;
    const int gx = gx0 + lx - 1, gy = gy0 + ly - 1;
    ld_s[k] = e < kPlane ? e : -1;
    ld_ok[k] = e < kPlane && gx >= 0 && gx < op.nx && gy >= 0 && gy < op.ny;
    ld_g[k] = ld_ok[k] ? gy * op.nx + gx : 0;
  }
  // issue the asynchronous copies of plane z (all RB fields) into slot
  auto issue_plane = [&](int z, int slot) {
    if (z < z0 - 1 || z > z1) return;                     // not needed by this CTA
    const bool zin = z >= 0 && z < op.nz;
    const long long zoff = zin ? (long long)z * plane : 0;
#pragma unroll
    for (int k = 0; k < kLoadIters; ++k) {
      if (ld_s[k] < 0) continue;
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const bool ok = zin && ld_ok[k] && r < rcount;
        const C* src = x + (ok ? (long long)(r0 + r) * rstride + zoff + ld_g[k] : 0);
        cp_async(ring + (slot * RB + r) * kPlane + ld_s[k], src, (int)sizeof(C), ok);
      }
    }
  };

  // in-plane class sums of column (tx, ty): centre, 4 faces, 4 corners
  C cs[3][RB], es[3][RB], ks[3][RB];   // window: 0 -> z-1, 1 -> z, 2 -> z+1
  auto plane_sums = [&](int slot, int w) {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const C* q = P(slot, r);
      cs[w][r] = q[PW + 1];
      es[w][r] = cadd(cadd(q[PW], q[PW + 2]), cadd(q[1], q[2 * PW + 1]));
      ks[w][r] = cadd(cadd(q[0], q[2]), cadd(q[2 * PW], q[2 * PW + 2]));
    }
  };

  // prologue: planes z0-1 .. z0+kDist in flight (slots 0..kDist+1), one
  // commit group per plane
#pragma unroll
  for (int k = -1; k <= kDist; ++k) {
    issue_plane(z0 + k, k + 1);
    cp_commit();
  }
  cp_wait<kDist>();                // planes z0-1 and z0 have landed
  __syncthreads();
  // rolling slots of planes z-1, z, z+1 and of the plane issued next
  int s_m = 0, s_0 = 1, s_p = 2, s_issue = kDist + 2;
  plane_sums(s_m, 0);
  plane_sums(s_0, 1);

  const bool plain_x = ix >= op.plain_lo[0] && ix <= op.plain_hi[0];
  const bool plain_y = iy >= op.plain_lo[1] && iy <= op.plain_hi[1];
  const bool plain_xy = plain_x && plain_y;
  float v_next = active && z0 < z1 ? __ldg(op.v + (long long)z0 * plane + (long long)iy * op.nx + ix) : 1.f;

  for (int z = z0; z < z1; ++z) {
    cp_wait<kDist - 1>();          // plane z+1 has landed (own copies)
    __syncthreads();               // ... for every thread; step z-1 finished everywhere
    issue_plane(z + kDist + 1, s_issue);   // into the slot of plane z-2
    cp_commit();
    plane_sums(s_p, 2);

    const float vv = v_next;
    if (active && z + 1 < z1) v_next = __ldg(op.v + (long long)(z + 1) * plane + (long long)iy * op.nx + ix);

    if (active) {
      const long long off = (long long)z * plane + (long long)iy * op.nx + ix;
      // interpolated row weights: wv[0..3] stiffness class coefficients x h^2,
      // wv[4..7] mass weights, wv[8..10] transverse weights (PML rows only)
      const TabPos<T> tq = tab_pos(op, tab, vv);
      T wv[12];
      tab_lerp4(tq, 0, wv);
      tab_lerp4(tq, 1, wv + 4);
      const T m = tq.m;
      const bool plain_z = z >= op.plain_lo[2] && z <= op.plain_hi[2];
      if (plain_x || plain_y) {
        // At most one of x, y stretched: the interior class form plus, for each
        // stretched axis d, (up_d - 1/h^2)(F_d+ - F_d0) + (dn_d - 1/h^2)(F_d- - F_d0)
        // with F_d(s) the transverse average at offset s along d (z from the
        // register window, x or y from the ring).
        T a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = fma(m, wv[4 + k], wv[k] * op.inv_h2);
        C diag = cmk(a[0], SHIFT ? op.beta * m * wv[4] : (T)0);
        C duz = czero<C>(), ddz = czero<C>(), dua = czero<C>(), dda = czero<C>();
        if (!plain_z || !plain_xy) tab_lerp4(tq, 2, wv + 8);
        if (!plain_z) {
          const T* q = op.axis[2] + 4 * (size_t)z;
          duz = cmk(ldg(q) - op.inv_h2, ldg(q + 1));
          ddz = cmk(ldg(q + 2) - op.inv_h2, ldg(q + 3));
          diag = csub(diag, cscale(wv[8], cadd(duz, ddz)));
        }
        // the stretched in-plane axis (if any): x when !plain_x, else y
        const int ax = plain_x ? 1 : 0;
        if (!plain_xy) {
          const T* q = (ax == 0 ? op.axis[0] + 4 * (size_t)ix : op.axis[1] + 4 * (size_t)iy);
          dua = cmk(ldg(q) - op.inv_h2, ldg(q + 1));
          dda = cmk(ldg(q + 2) - op.inv_h2, ldg(q + 3));
          diag = csub(diag, cscale(wv[8], cadd(dua, dda)));
        }
        // ring offsets of the line along the stretched axis and its transverse pair
        const int stx = ax == 0 ? 1 : 0, sty = 1 - stx;      // step along the axis
        const int ptx = sty, pty = stx;                      // step to the pair
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
            C ms = cscale(wv[4], c0);
            ms = cfmar(wv[5], f6, ms);
            ms = cfmar(wv[6], e12, ms);
            ms = cfmar(wv[7], c8, ms);
            acc = cadd(acc, cscale_i(op.beta * m, ms));
          }
          if (!plain_z) {
            // F_z(s) = t0 c(z+s) + t1 faces(z+s) + t2 corners(z+s)
            const T t0 = wv[8], t1 = wv[9], t2 = wv[10];
            const C fzm = cfmar(t2, ks[0][r], cfmar(t1, es[0][r], cscale(t0, cs[0][r])));
            const C fz0 = cfmar(t2, ks[1][r], cfmar(t1, es[1][r], cscale(t0, cs[1][r])));
            const C fzp = cfmar(t2, ks[2][r], cfmar(t1, es[2][r], cscale(t0, cs[2][r])));
            acc = cfma(duz, csub(fzp, fz0), acc);
            acc = cfma(ddz, csub(fzm, fz0), acc);
          }
          if (!plain_xy) {
            const T t0 = wv[8], t1 = wv[9], t2 = wv[10];
            C Fm = czero<C>(), F0 = czero<C>(), Fp = czero<C>();
#pragma unroll
            for (int dk = -1; dk <= 1; ++dk) {
              const C* q = P(dk < 0 ? s_m : (dk > 0 ? s_p : s_0), r);
              const T ta = dk != 0 ? t1 : t0, tb = dk != 0 ? t2 : t1;
#pragma unroll
              for (int s = -1; s <= 1; ++s) {
                const int c = (1 + s * sty) * PW + 1 + s * stx;   // line element at offset s
                const int pr = pty * PW + ptx;                    // its transverse pair
                const C f = cfmar(tb, cadd(q[c - pr], q[c + pr]), cscale(ta, q[c]));
                if (s < 0) Fm = cadd(Fm, f);
                else if (s == 0) F0 = cadd(F0, f);
                else Fp = cadd(Fp, f);
              }
            }
            acc = cfma(dua, csub(Fp, F0), acc);
            acc = cfma(dda, csub(Fm, F0), acc);
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
        tab_lerp4(tq, 2, wv + 8);
        const T t0 = wv[8], t1 = wv[9], t2 = wv[10];
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
        const C diag = cfma(mc, cmk(wv[4], (T)0), cscale(-t0, sdiag));
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
            const C* qp = P(dk < 0 ? s_m : (dk > 0 ? s_p : s_0), r);
            C q[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
              for (int i = 0; i < 3; ++i) q[j][i] = qp[j * PW + i];
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
            const T mw0 = off_plane ? wv[5] : wv[4];
            const T mw1 = off_plane ? wv[6] : wv[5];
            const T mw2 = off_plane ? wv[7] : wv[6];
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
    s_m = next_slot(s_m);
    s_0 = next_slot(s_0);
    s_p = next_slot(s_p);
    s_issue = next_slot(s_issue);
  }
  cp_wait<0>();
}

// First damped-Jacobi sweep from a zero guess: y = omega_j D^{-1} b, with D
// the row's diagonal coefficient (no neighbour reads).
template <typename T, bool SHIFT>
__global__ void jacobi0_kernel(OpDesc<T> op, const typename CT<T>::type* __restrict__ b,
                               typename CT<T>::type* __restrict__ y, int nrhs, long long rstride,
                               T omega_j) {
  pdl_enter();
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

// One thread per row: the 27 coefficients in (dk, dj, di) order, FP64
// (entries whose neighbour lies outside the grid are 0).
template <bool MED>
__global__ void row_coef_kernel(OpDesc<double> op, double2* __restrict__ coef) {
  pdl_enter();
  const long long N = (long long)op.nx * op.ny * op.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % op.nx);
    const int iy = (int)((i / op.nx) % op.ny);
    const int iz = (int)(i / ((long long)op.nx * op.ny));
    double2 c[27];
    fine_row<double, MED>(op, ix, iy, iz, c);
    for (int k = 0; k < 27; ++k) {
      const int di = k % 3 - 1, dj = (k / 3) % 3 - 1, dk = k / 9 - 1;
      const bool inside = ix + di >= 0 && ix + di < op.nx && iy + dj >= 0 && iy + dj < op.ny &&
                          iz + dk >= 0 && iz + dk < op.nz;
      coef[i * 27 + k] = inside ? c[k] : make_double2(0.0, 0.0);
    }
  }
}

// z-range per CTA: minimise (waves of CTAs) x (z-steps per CTA + ring
// prologue), with waves counted against the resident-CTA slots of 152 SMs.
int pick_zchunk(int nz, int ntiles_xy, int nrb, int ctas_per_sm) {
  const long long slots = 152LL * ctas_per_sm;
  int best = nz;
  double best_cost = 1e300;
  for (int zc = nz; zc >= 4; --zc) {
    const long long nzc = (nz + zc - 1) / zc;
    if ((nz + nzc - 1) / nzc != zc) continue;          // same split as a larger zc
    const long long ctas = (long long)ntiles_xy * nrb * nzc;
    if (nzc * nrb > 65535) break;
    const long long waves = (ctas + slots - 1) / slots;
    const double cost = (double)waves * (zc + kDist + 2);
    if (cost < best_cost * 0.999) {
      best_cost = cost;
      best = zc;
    }
  }
  return best;
}

template <typename T, int MODE, bool SHIFT, int RB>
cudaError_t launch_t(const OpDesc<T>& op, const void* x, const void* b, void* y, int nrhs,
                     long long rstride, double omega_j, cudaStream_t s) {
  using C = typename CT<T>::type;
  const int bx = (op.nx + kTX - 1) / kTX, by = (op.ny + kTY - 1) / kTY;
  const int nrb = (nrhs + RB - 1) / RB;
  // the weight table is read through the read-only cache (staging it per CTA
  // cost more L2 traffic than the field itself on small grids)
  const size_t smem = ring_bytes<T, RB>();
  auto kern = stencil_kernel<T, MODE, SHIFT, RB>;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (smem > 48 * 1024 && (dev < 0 || dev >= 64 || !attr_set[dev])) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  const int zchunk = pick_zchunk(op.nz, bx * by, nrb, sizeof(T) == 4 ? 3 : 2);
  const int nzc = (op.nz + zchunk - 1) / zchunk;
  const long long gz = (long long)nzc * nrb;
  if (gz > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid(bx, by, (unsigned)gz), block(kTX, kTY);
  (void)launch_k(kern, grid, block, smem, s, op, (const C*)x, (const C*)b, (C*)y, nrhs, rstride, zchunk, (T)omega_j);
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
    (void)launch_k(jacobi0_kernel<T, true>, (unsigned)blocks, 256, 0, s, op, (const C*)b, (C*)y, nrhs, rstride, (T)omega_j);
  else
    (void)launch_k(jacobi0_kernel<T, false>, (unsigned)blocks, 256, 0, s, op, (const C*)b, (C*)y, nrhs, rstride, (T)omega_j);
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
  // operator variants and heterogeneous media: the one-thread-per-row kernel
  // (fields back to back)
  if (op.gam || op.mass1 || op.buoy || op.invq) {
    if (rstride != (long long)op.nx * op.ny * op.nz) return cudaErrorInvalidValue;
    return launch_direct_stencil<T>(op, mode, x, b, y, nrhs, omega_j, s);
  }
  if (sizeof(T) == 4) {
    // complex64: the two z-marching kernels.  Configuration ids 0-2 select
    // the cp.async kernel (any row pitch), ids 3.. the tensor-copy kernel
    // (even pitch, 16-byte aligned x and b); -1 lets an even pitch take the
    // tensor-copy kernel.  The first Jacobi sweep of padded fields is the
    // pitched per-row kernel of hx_zmarch.cu.
    const OpDesc<float>& of = reinterpret_cast<const OpDesc<float>&>(op);
    const long long pitch = field_pitch(op);
    if (rstride != pitch * op.ny * op.nz) return cudaErrorInvalidValue;
    int dev = 0;
    cudaGetDevice(&dev);
    const bool even = (pitch & 1) == 0;
    if (mode == kJacobi0 && pitch != op.nx)
      return even ? launch_zmarch(of, kJacobi0, -1, x, b, y, nrhs, pitch, omega_j, nullptr, s)
                  : cudaErrorInvalidValue;
    if (mode != kJacobi0) {
      const bool want_cp = op.cfg32 >= 0 && op.cfg32 < kZmCfgBase;
      if (even && !want_cp && ((uintptr_t)x & 15) == 0 && ((uintptr_t)b & 15) == 0)
        return launch_zmarch(of, mode, op.cfg32 >= kZmCfgBase ? op.cfg32 - kZmCfgBase : -1, x, b, y, nrhs, pitch,
                             omega_j, zm_error_flag(dev), s);
      // the cp.async kernel's row copies need a 16-byte aligned x
      if (((uintptr_t)x & 15) == 0)
        return launch_stencil32(of, mode, want_cp ? op.cfg32 : st32_default_config(nrhs), x, b, y, nrhs, rstride,
                                omega_j, s);
    }
    if (pitch != op.nx) return cudaErrorInvalidValue;
  }
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
  if (op.buoy || op.invq)
    (void)launch_k(row_coef_kernel<true>, (unsigned)blocks, 256, 0, s, op, (double2*)coef);
  else
    (void)launch_k(row_coef_kernel<false>, (unsigned)blocks, 256, 0, s, op, (double2*)coef);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace hx
