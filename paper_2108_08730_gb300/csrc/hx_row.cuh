// One row of the operator on the fly, one thread per row: the 27 complex
// coefficients in offset order k = (dk+1)*9 + (dj+1)*3 + (di+1).  Used by the
// one-thread-per-row kernels (coarse levels, Galerkin products, row
// coefficients) and by every launch of an operator variant.
//
// Row (Eqs. 4-8): sum_d T_d[delta_d] with the stretched second differences
// delta_d of the PML (axis arrays up/dn) and the transverse weights
// (t0, t1, t2), plus the consistent mass w_class * m (1 + i shift).  Weights
// come from the table at 1/G = f h / v: the row's own v (GA), or the mean of
// the table rows of the in-grid stencil points (GAm, Section 3.1; the table
// entries are linear in the seven weights, so this is the table row of the
// mean weights).  m = omega^2 / v^2 at the collocation point (second mass form
// of Eq. 8) or at each stencil point (first form).
//
// Heterogeneous medium (Eq. 2): with buoyancy b every second difference of
// T_d[delta_d] is the conservative form on its own stencil line, b at a half
// node the mean of its two nodes (b at the node when the other lies outside
// the grid), and the mass is omega^2 b / c*^2 with c* = v (1 - i/(2Q)).
#pragma once

#include "hx_complex.cuh"
#include "hx_internal.h"

namespace hx {

// the 11 interpolated table entries at velocity vt
template <typename T>
__device__ __forceinline__ void table_row(const OpDesc<T>& op, T vt, T w[11]) {
  const T iv = (T)1 / vt;
  T u = op.u_scale * iv;
  const T umax = (T)(op.n_g - 1);
  u = u < (T)0 ? (T)0 : (u > umax ? umax : u);
  int i0 = (int)u;
  if (i0 > op.n_g - 2) i0 = op.n_g - 2;
  const T t = u - (T)i0;
  const T* a = op.tab + (size_t)i0 * kTabW;
#pragma unroll
  for (int k = 0; k < 11; ++k) w[k] = fma(t, __ldg(a + kTabW + k) - __ldg(a + k), __ldg(a + k));
}

// fine_row with buoyancy and / or attenuation; w: the row's 11 table entries
template <typename T>
__device__ __forceinline__ void medium_row(const OpDesc<T>& op, int ix, int iy, int iz, const T w[11],
                                           typename CT<T>::type c[27]) {
  using C = typename CT<T>::type;
  const long long sy = op.nx, sz = (long long)op.nx * op.ny;
  // b over the 3 x 3 x 3 block (0 outside the grid) and the in-grid flags
  T bb[27];
  bool in[27];
#pragma unroll
  for (int s = 0; s < 27; ++s) {
    const int jx = ix + s % 3 - 1, jy = iy + (s / 3) % 3 - 1, jz = iz + s / 9 - 1;
    in[s] = jx >= 0 && jx < op.nx && jy >= 0 && jy < op.ny && jz >= 0 && jz < op.nz;
    bb[s] = !in[s] ? (T)0 : (op.buoy ? (T)__ldg(op.buoy + jx + sy * jy + sz * jz) : (T)1);
  }
  auto half = [&](int p, int q) { return in[q] ? (T)0.5 * (bb[p] + bb[q]) : bb[p]; };
  const T tw[3] = {w[8], w[9], w[10]};
  const int id[3] = {ix, iy, iz};
  C up[3], dn[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T* q = op.axis[d] + 4 * (size_t)id[d];
    up[d] = cmk(__ldg(q), __ldg(q + 1));
    dn[d] = cmk(__ldg(q + 2), __ldg(q + 3));
  }
  // omega^2 b / c*^2 (1 + i shift) at block point s
  auto mass = [&](int s) {
    const int jx = ix + s % 3 - 1, jy = iy + (s / 3) % 3 - 1, jz = iz + s / 9 - 1;
    const long long j = jx + sy * jy + sz * jz;
    const T ivj = (T)1 / (T)__ldg(op.v + j);
    C mj = cmk(op.omega2 * ivj * ivj * bb[s], (T)0);
    if (op.invq) {
      // 1 / (1 - i q/2)^2 = conj(z) / |z|^2 with z = (1 - q^2/4) - i q
      const T q = (T)__ldg(op.invq + j);
      const C z = cmk((T)1 - (T)0.25 * q * q, -q);
      const T n2 = z.x * z.x + z.y * z.y;
      mj = cmul(mj, cmk(z.x / n2, -z.y / n2));
    }
    return cmul(mj, cmk((T)1, op.beta));
  };
  const C m0 = mass(13);
#pragma unroll 1
  for (int k = 0; k < 27; ++k) {
    const int di = k % 3 - 1, dj = (k / 3) % 3 - 1, dk = k / 9 - 1;
    auto at = [](int a, int b2, int c2) { return (c2 + 1) * 9 + (b2 + 1) * 3 + (a + 1); };
    const int o[3] = {di, dj, dk};
    C v = czero<C>();
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // the line along d through the stencil point with offsets o on the other axes
      int pa[3] = {o[0], o[1], o[2]};
      pa[d] = 0;
      int qp[3] = {pa[0], pa[1], pa[2]}, qm[3] = {pa[0], pa[1], pa[2]};
      qp[d] = 1;
      qm[d] = -1;
      const int p = at(pa[0], pa[1], pa[2]);
      const T bp = half(p, at(qp[0], qp[1], qp[2])), bm = half(p, at(qm[0], qm[1], qm[2]));
      const C dd = o[d] == 1 ? cscale(bp, up[d])
                             : (o[d] == -1 ? cscale(bm, dn[d]) : cmk(-(bp * up[d].x + bm * dn[d].x),
                                                                     -(bp * up[d].y + bm * dn[d].y)));
      const int t = abs(o[(d + 1) % 3]) + abs(o[(d + 2) % 3]);
      v = cfmar(tw[t], dd, v);
    }
    const C mk = op.mass1 && in[k] ? mass(k) : m0;
    c[k] = cfma(mk, cmk(w[4 + abs(di) + abs(dj) + abs(dk)], (T)0), v);
  }
}

// MED: the heterogeneous-medium row (op.buoy / op.invq set); a separate
// instantiation, so the common kernels carry none of its code or state
template <typename T, bool MED = false>
__device__ __forceinline__ void fine_row(const OpDesc<T>& op, int ix, int iy, int iz,
                                         typename CT<T>::type c[27]) {
  using C = typename CT<T>::type;
  const long long i = ix + (long long)op.nx * (iy + (long long)op.ny * iz);
  const long long sy = op.nx, sz = (long long)op.nx * op.ny;
  const T vt = (T)__ldg(op.v + i);
  T w[11];
  if (!op.gam) {
    table_row(op, vt, w);
  } else {
#pragma unroll
    for (int k = 0; k < 11; ++k) w[k] = (T)0;
    int cnt = 0;
    for (int s = 0; s < 27; ++s) {
      const int jx = ix + s % 3 - 1, jy = iy + (s / 3) % 3 - 1, jz = iz + s / 9 - 1;
      if (jx < 0 || jx >= op.nx || jy < 0 || jy >= op.ny || jz < 0 || jz >= op.nz) continue;
      T wj[11];
      table_row(op, (T)__ldg(op.v + jx + sy * jy + sz * jz), wj);
#pragma unroll
      for (int k = 0; k < 11; ++k) w[k] += wj[k];
      ++cnt;
    }
    const T inv = (T)1 / (T)cnt;
#pragma unroll
    for (int k = 0; k < 11; ++k) w[k] *= inv;
  }
  const T iv = (T)1 / vt;
  const T m = op.omega2 * iv * iv;
  const T tw[3] = {w[8], w[9], w[10]};
  if constexpr (MED) {
    medium_row(op, ix, iy, iz, w, c);
    return;
  }
  const int id[3] = {ix, iy, iz};
  C D[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T* q = op.axis[d] + 4 * (size_t)id[d];
    const C up = cmk(__ldg(q), __ldg(q + 1)), dn = cmk(__ldg(q + 2), __ldg(q + 3));
    D[d][2] = up;
    D[d][0] = dn;
    D[d][1] = cmk(-(up.x + dn.x), -(up.y + dn.y));
  }
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const int di = k % 3 - 1, dj = (k / 3) % 3 - 1, dk = k / 9 - 1;
    C v = cscale(tw[abs(dj) + abs(dk)], D[0][di + 1]);
    v = cfmar(tw[abs(di) + abs(dk)], D[1][dj + 1], v);
    v = cfmar(tw[abs(di) + abs(dj)], D[2][dk + 1], v);
    T mk = m;
    if (op.mass1) {
      const int jx = ix + di, jy = iy + dj, jz = iz + dk;
      if (jx >= 0 && jx < op.nx && jy >= 0 && jy < op.ny && jz >= 0 && jz < op.nz) {
        const T ivj = (T)1 / (T)__ldg(op.v + jx + sy * jy + sz * jz);
        mk = op.omega2 * ivj * ivj;
      }
    }
    c[k] = cfma(cmk(mk, op.beta * mk), cmk(w[4 + abs(di) + abs(dj) + abs(dk)], (T)0), v);
  }
}

}  // namespace hx
