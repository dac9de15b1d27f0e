// Complex64 z-marching kernel of the adaptive 27-point operator [M + S]
// (Eq. 3; rows of Eqs. 4-8 with the GA weight selection of Section 3.1).
//
// Same operator, modes and results as the generic kernel in hx_stencil.cu
// (which keeps the complex128 path); this one is arranged for instruction
// economy, because the complex64 apply is issue- and latency-bound long
// before it is bandwidth-bound:
//  * a CTA owns a 32 x TY column tile, RB right-hand sides and a z-range and
//    marches along z; x planes (tile + 1-node halo, RB fields) stream into an
//    NSLOT-plane shared-memory ring with 8-byte cp.async (zero fill outside
//    the grid, source pointers precomputed per thread), D planes ahead of the
//    one being consumed, one barrier per z-step;
//  * complex additions and real-times-complex products use the packed
//    FP32x2 instructions of sm_100+ (add/sub/mul/fma .f32x2);
//  * a warp covers 32 consecutive x; each thread owns YB consecutive y rows
//    of its column;
//  * per column and plane the in-plane class sums (centre, 4 faces, 4
//    corners) live in registers for the three z-steps that use them; the z
//    loop is unrolled by three so this window rotates without moves;
//  * 1/v comes from the approximate reciprocal (the table coordinate and
//    omega^2/v^2 tolerate its 1-ulp error), and with few fields per CTA the
//    table entries of the next plane are fetched one step ahead;
//  * rows whose only complex stretching is along z stay on the register
//    path; rows in the x/y PML read their 27 neighbours from the ring.
#include <algorithm>
#include <vector>

#include "hx_complex.cuh"
#include "hx_internal.h"
#include "hx_launch.cuh"

namespace hx {
namespace {

// ------------------------------------------------------------ FP32x2 helpers
// HX_PACKED_F32X2 = 1 issues the packed FP32x2 instructions of sm_100+ through
// inline PTX; 0 leaves plain float arithmetic to the compiler.
#ifndef HX_PACKED_F32X2
#define HX_PACKED_F32X2 1
#endif
#if HX_PACKED_F32X2
#define HX_P2(op)                                                                              \
  float2 r;                                                                                    \
  asm("{.reg .b64 a,b,d;\n\tmov.b64 a,{%2,%3};\n\tmov.b64 b,{%4,%5};\n\t" op               \
      ".rn.f32x2 d,a,b;\n\tmov.b64 {%0,%1},d;}"                                                \
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                      \
  return r;
__device__ __forceinline__ float2 padd(float2 a, float2 b) { HX_P2("add") }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { HX_P2("sub") }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { HX_P2("mul") }
#undef HX_P2
// a * b + c, elementwise
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{.reg .b64 a,b,c,d;\n\tmov.b64 a,{%2,%3};\n\tmov.b64 b,{%4,%5};\n\tmov.b64 c,{%6,%7};\n\t"
      "fma.rn.f32x2 d,a,b,c;\n\tmov.b64 {%0,%1},d;}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}
#else
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
#endif
__device__ __forceinline__ float2 dup(float s) { return make_float2(s, s); }
// complex a * b + acc (both complex), scalar FMAs
__device__ __forceinline__ float2 cfmac(float2 a, float2 b, float2 acc) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 crcpf(float2 a) {
  const float d = __frcp_rn(fmaf(a.x, a.x, a.y * a.y));
  return make_float2(a.x * d, -a.y * d);
}
__device__ __forceinline__ float rcp_approx(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

// ------------------------------------------------------------ async copies
__device__ __forceinline__ void cp_commit32() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait32() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int V>
struct I {
  static constexpr int value = V;
};

// ------------------------------------------------------------ configuration
// HX_ST32_PREFETCH = 0 turns the one-plane-ahead table fetch off;
// HX_ST32_MINB sets the resident CTAs per SM the register budget is cut for;
// HX_ST32_ZMAX > 0 caps the z-chunk of a CTA.
#ifndef HX_ST32_PREFETCH
#define HX_ST32_PREFETCH 1
#endif
#ifndef HX_ST32_MINB
#define HX_ST32_MINB 2
#endif
#ifndef HX_ST32_ZMAX
#define HX_ST32_ZMAX 0
#endif
constexpr int kW = 32;              // tile extent in x: one warp
constexpr int kNW = 8;              // warps per CTA
constexpr int kThr = kW * kNW;
constexpr int kPW = kW + 2;         // ring row pitch (tile + halo)

// YB rows per thread, RB right-hand sides per CTA.
template <int YB, int RB>
struct Cfg {
  static constexpr int TY = kNW * YB;                  // tile extent in y
  static constexpr int PH = TY + 2;                    // ring rows (tile + halo)
  static constexpr int PLANE = PH * kPW;               // complex64 per field plane
  static constexpr int LI = (PLANE + kThr - 1) / kThr; // loader elements per thread
  static constexpr int SLOTB = PLANE * RB * 8;         // bytes per ring slot
  static constexpr int D = SLOTB <= 6144 ? 5 : 4;      // planes in flight beyond the window
  static constexpr int NSLOT = D + 3;
  static constexpr int SMEM = NSLOT * SLOTB;
  static constexpr int MINB = HX_ST32_MINB;            // resident CTAs per SM
  // with RB >= 4 the table lookup is amortised over the fields and its
  // registers are better spent on the class-sum window
  static constexpr bool PREFETCH = HX_ST32_PREFETCH && RB <= 2;
};

// One CTA's work: the 32 x TY column tile (tbx, tby), RHS block and z-chunk
// packed in tbz (RHS block fastest), of the operator op.  ring: the CTA's
// dynamic shared memory ([NSLOT][RB][PH][kPW] complex64).
template <int MODE, int YB, int RB>
__device__ __forceinline__ void st32_tile(const OpDesc<float>& op, const float2* __restrict__ x,
                                          const float2* __restrict__ b, float2* __restrict__ y,
                                          int nrhs, long long rstride, int zchunk, int zmul,
                                          float omega_j, int tbx, int tby, int tbz, float2* ring) {
  using K = Cfg<YB, RB>;
  constexpr unsigned SLOTB = K::SLOTB, RINGB = K::NSLOT * K::SLOTB;
  const int tid = threadIdx.x, tx = tid & 31, w = tid >> 5;
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const int gx0 = tbx * kW - op.xshift, gy0 = tby * K::TY;   // gx0 may be negative (tile 0)
  const int ix = gx0 + tx, iyb = gy0 + w * YB;
  const int nrb = (nrhs + RB - 1) / RB;
  const int rblk = tbz % nrb, zc = tbz / nrb;
  const int r0 = rblk * RB, rcount = min(RB, nrhs - r0);
  // Tiles holding no x/y-PML row march zmul times longer z-chunks: their
  // planes cost about half as much, so all CTAs of a launch end together.
  int zlen = zchunk;
  if (zmul > 1) {
    const int xa = max(gx0, 0), xb = min(gx0 + kW - 1, nx - 1), yb = min(gy0 + K::TY - 1, ny - 1);
    if (xa >= op.plain_lo[0] && xb <= op.plain_hi[0] && gy0 >= op.plain_lo[1] && yb <= op.plain_hi[1])
      zlen = zchunk * zmul;
  }
  const int z0 = zc * zlen, z1 = min(nz, z0 + zlen);
  if (z0 >= nz) return;                                // a chunk index past a long-chunk tile's end
  // fields: x-row pitch op.pitch (0: nx); the velocity is unpadded
  const long long fpitch = op.pitch > 0 ? op.pitch : nx;
  const long long plane = fpitch * ny, vplane = (long long)nx * ny;
  const bool shift = op.beta != 0.f;

  // ---- loader.  This thread copies elements tid + k kThr of every plane
  // tile (8-byte cp.async, zero fill outside the grid); ld_p[k] walks plane
  // by plane through field r0 (x itself for elements outside the grid, which
  // never advance).
  const unsigned ld_s = (unsigned)__cvta_generic_to_shared(ring) + 8u * tid;
  const float2* ld_p[K::LI];
  bool ld_in[K::LI];
  const bool ld_last = tid + (K::LI - 1) * kThr < K::PLANE;   // does the last element exist
  {
    const float2* xr = x + (long long)r0 * rstride + (long long)(z0 - 1) * plane;
#pragma unroll
    for (int k = 0; k < K::LI; ++k) {
      const int e = tid + k * kThr;
      const int ly = e / kPW, lx = e - ly * kPW;
      const int gx = gx0 + lx - 1, gy = gy0 + ly - 1;
      ld_in[k] = e < K::PLANE && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
      ld_p[k] = ld_in[k] ? xr + (gy * fpitch + gx) : x;
    }
  }
  // copies of plane z (all RB fields) into the slot at byte offset so; planes
  // are issued in increasing z, once each, from z0 - 1 to z1
  auto issue = [&](int z, unsigned so) {
    if (z > z1) return;                                // not needed by this CTA
    const unsigned dst = ld_s + so;
    const bool zin = z >= 0 && z < nz;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
#pragma unroll
      for (int k = 0; k < K::LI; ++k) {
        if (k == K::LI - 1 && !ld_last) continue;
        const bool ok = zin && ld_in[k] && (r == 0 || r < rcount);
        const float2* src = ok ? ld_p[k] + (r == 0 ? 0 : r * rstride) : x;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst + r * (K::PLANE * 8) + k * (kThr * 8)),
                     "l"(src), "r"(ok ? 8 : 0) : "memory");
      }
    }
#pragma unroll
    for (int k = 0; k < K::LI; ++k)
      if (ld_in[k]) ld_p[k] += plane;
  };

  // register window of in-plane class sums: [window slot][row][rhs]
  float2 cs[3][YB][RB], es[3][YB][RB], ks[3][YB][RB];
  const float2* thr = ring + (w * YB) * kPW + tx;      // top-left of this thread's window
  auto slotp = [&](unsigned so) { return reinterpret_cast<const float2*>(reinterpret_cast<const char*>(thr) + so); };
  auto sums = [&](unsigned so, auto wtag) {
    constexpr int WS = decltype(wtag)::value;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const float2* q = slotp(so) + r * K::PLANE;
      float2 M[YB + 2], H[YB + 2];
#pragma unroll
      for (int rr = 0; rr < YB + 2; ++rr) {
        M[rr] = q[rr * kPW + 1];
        H[rr] = padd(q[rr * kPW], q[rr * kPW + 2]);
      }
#pragma unroll
      for (int j = 0; j < YB; ++j) {
        cs[WS][j][r] = M[j + 1];
        es[WS][j][r] = padd(H[j + 1], padd(M[j], M[j + 2]));
        ks[WS][j][r] = padd(H[j], H[j + 2]);
      }
    }
  };

  // prologue: planes z0-1 .. z0+D in flight (slots 0 .. D+1), one group each
#pragma unroll
  for (int k = -1; k <= K::D; ++k) {
    issue(z0 + k, (unsigned)(k + 1) * SLOTB);
    cp_commit32();
  }
  cp_wait32<K::D>();                                   // planes z0-1 and z0 landed
  __syncthreads();
  sums(0u, I<0>{});
  sums(SLOTB, I<1>{});
  // byte offsets of the slots of planes z-1, z, z+1 and of the next issue
  unsigned o_m = 0, o_0 = SLOTB, o_p = 2 * SLOTB, o_i = (K::D + 2) * SLOTB;

  const bool xin = ix >= 0 && ix < nx;
  const bool plain_x = ix >= op.plain_lo[0] && ix <= op.plain_hi[0];
  const float umax = (float)(op.n_g - 1);
  const float ih2 = op.inv_h2;
  const unsigned zlo = (unsigned)op.plain_lo[2], zspan = (unsigned)(op.plain_hi[2] - op.plain_lo[2]);
  // Table entries of a row (stiffness class coefficients x h^2 and mass
  // weights at nodes i0 and i0 + 1, the fraction tf, omega^2 / v^2); with
  // PREFETCH they are fetched one plane ahead so the lookup latency overlaps
  // the previous plane's arithmetic.
  struct Tab {
    float4 ls, hs, lm, hm;
    float tf, m;
    int i0;
  };
  auto tab_fetch = [&](float vv, Tab& t) {
    const float iv = rcp_approx(vv);
    const float u = fminf(fmaxf(op.u_scale * iv, 0.f), umax);
    t.i0 = min((int)u, op.n_g - 2);
    t.tf = u - (float)t.i0;
    t.m = op.omega2 * iv * iv;
    const float* tq = op.tab + t.i0 * kTabW;
    t.ls = ldg4(tq);
    t.hs = ldg4(tq + kTabW);
    t.lm = ldg4(tq + 4);
    t.hm = ldg4(tq + kTabW + 4);
  };
  bool act[YB], plain_xy[YB];
  Tab tnext[YB];                                       // entries of plane z (PREFETCH)
  float v1[YB];                                        // v at plane z + 1 (PREFETCH) or z
  const float* vp[YB];                                 // v at the plane after v1's
  long long yo[YB];                                    // element offset of (ix, iy, z) in field r0
  // b of a single RHS is fetched one plane ahead, so its latency is not
  // exposed after the per-plane barrier (Jacobi and residual sweeps)
  constexpr bool BPF = MODE != kApply && RB == 1;
  float2 bnx[YB];                                      // b at plane z (BPF)
#pragma unroll
  for (int j = 0; j < YB; ++j) {
    const int iy = iyb + j;
    act[j] = xin && iy < ny;
    // the general form is exact for every row: a warp holding any x/y PML
    // row runs it on all lanes rather than running both forms
    plain_xy[j] = !__any_sync(0xffffffffu, act[j] && !(plain_x && iy >= op.plain_lo[1] && iy <= op.plain_hi[1]));
    const long long ov = (long long)z0 * vplane + (long long)(act[j] ? iy * nx + ix : 0);
    const long long o = (long long)z0 * plane + (long long)(act[j] ? iy * fpitch + ix : 0);
    if (K::PREFETCH) {
      tab_fetch(act[j] && z0 < z1 ? __ldg(op.v + ov) : 1.5e3f, tnext[j]);
      v1[j] = act[j] && z0 + 1 < z1 ? __ldg(op.v + ov + vplane) : 1.5e3f;
      vp[j] = op.v + ov + 2 * vplane;
    } else {
      v1[j] = act[j] && z0 < z1 ? __ldg(op.v + ov) : 1.5e3f;
      vp[j] = op.v + ov + vplane;
    }
    yo[j] = o + (long long)r0 * rstride;
    bnx[j] = BPF && b && act[j] && z0 < z1 ? b[yo[j]] : make_float2(0.f, 0.f);
  }

  auto step = [&](auto ptag, int z) {
    constexpr int P = decltype(ptag)::value;
    constexpr int W0 = P % 3, W1 = (P + 1) % 3, W2 = (P + 2) % 3;   // planes z-1, z, z+1
    cp_wait32<K::D - 1>();                             // plane z+1 landed (own copies)
    __syncthreads();                                   // ... everyone's; step z-1 done
    issue(z + K::D + 1, o_i);                          // into the slot of plane z-2
    cp_commit32();
    sums(o_p, I<W2>{});
    const bool plain_z = (unsigned)z - zlo <= zspan;
#pragma unroll
    for (int j = 0; j < YB; ++j) {
      Tab t;
      if (K::PREFETCH) {
        t = tnext[j];
        if (act[j] && z + 1 < z1) tab_fetch(v1[j], tnext[j]);
      } else {
        tab_fetch(v1[j], t);                           // v1 holds v at plane z here
      }
      v1[j] = act[j] && z + (K::PREFETCH ? 2 : 1) < z1 ? __ldg(vp[j]) : 1.5e3f;
      vp[j] += vplane;
      const long long off = yo[j];
      yo[j] += plane;
      float2 bcur = make_float2(0.f, 0.f);
      if (BPF) {
        bcur = bnx[j];
        if (b && act[j] && z + 1 < z1) bnx[j] = b[off + plane];
      }
      if (!act[j]) continue;
      const float tf = t.tf, m = t.m;
      const float* tq = op.tab + t.i0 * kTabW;
      const float4 lo_s = t.ls, hi_s = t.hs, lo_m = t.lm, hi_m = t.hm;
      const float2 ts = dup(tf);
      // stiffness class coefficients x h^2 (centre, face, edge, corner), mass weights
      const float2 s01 = pfma(ts, psub(make_float2(hi_s.x, hi_s.y), make_float2(lo_s.x, lo_s.y)), make_float2(lo_s.x, lo_s.y));
      const float2 s23 = pfma(ts, psub(make_float2(hi_s.z, hi_s.w), make_float2(lo_s.z, lo_s.w)), make_float2(lo_s.z, lo_s.w));
      const float2 m01 = pfma(ts, psub(make_float2(hi_m.x, hi_m.y), make_float2(lo_m.x, lo_m.y)), make_float2(lo_m.x, lo_m.y));
      const float2 m23 = pfma(ts, psub(make_float2(hi_m.z, hi_m.w), make_float2(lo_m.z, lo_m.w)), make_float2(lo_m.z, lo_m.w));
      const float bm = op.beta * m;
      if (plain_xy[j]) {
        // interior form: 4 real class coefficients times 4 class sums
        const float2 a01 = pfma(dup(m), m01, pmul(dup(ih2), s01));
        const float2 a23 = pfma(dup(m), m23, pmul(dup(ih2), s23));
        const float2 A0 = dup(a01.x), A1 = dup(a01.y), A2 = dup(a23.x), A3 = dup(a23.y);
        float2 diag = make_float2(a01.x, shift ? bm * m01.x : 0.f);
        float2 duz = make_float2(0.f, 0.f), ddz = duz;
        float t0 = 0.f, t1 = 0.f, t2 = 0.f;
        if (!plain_z) {
          const float4 lo_t = ldg4(tq + 8), hi_t = ldg4(tq + kTabW + 8);
          t0 = fmaf(tf, hi_t.x - lo_t.x, lo_t.x);
          t1 = fmaf(tf, hi_t.y - lo_t.y, lo_t.y);
          t2 = fmaf(tf, hi_t.z - lo_t.z, lo_t.z);
          const float4 az = ldg4(op.axis[2] + 4 * (size_t)z);
          duz = make_float2(az.x - ih2, az.y);
          ddz = make_float2(az.z - ih2, az.w);
          diag = make_float2(diag.x - t0 * (duz.x + ddz.x), diag.y - t0 * (duz.y + ddz.y));
        }
        float2 dinv = make_float2(0.f, 0.f);
        if (MODE == kJacobi) {
          dinv = crcpf(diag);
          dinv = make_float2(omega_j * dinv.x, omega_j * dinv.y);
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const float2 c0 = cs[W1][j][r];
          const float2 f6 = padd(es[W1][j][r], padd(cs[W0][j][r], cs[W2][j][r]));
          const float2 e12 = padd(ks[W1][j][r], padd(es[W0][j][r], es[W2][j][r]));
          const float2 c8 = padd(ks[W0][j][r], ks[W2][j][r]);
          float2 acc = pfma(A3, c8, pfma(A2, e12, pfma(A1, f6, pmul(A0, c0))));
          if (shift) {
            const float2 ms = pfma(dup(m23.y), c8, pfma(dup(m23.x), e12, pfma(dup(m01.y), f6, pmul(dup(m01.x), c0))));
            acc = make_float2(fmaf(-bm, ms.y, acc.x), fmaf(bm, ms.x, acc.y));
          }
          if (!plain_z) {
            // complex z-stretching: (up_z - 1/h^2)(F_z+ - F_z0) + (dn_z - 1/h^2)(F_z- - F_z0)
            const float2 T0 = dup(t0), T1 = dup(t1), T2 = dup(t2);
            const float2 fzm = pfma(T2, ks[W0][j][r], pfma(T1, es[W0][j][r], pmul(T0, cs[W0][j][r])));
            const float2 fz0 = pfma(T2, ks[W1][j][r], pfma(T1, es[W1][j][r], pmul(T0, c0)));
            const float2 fzp = pfma(T2, ks[W2][j][r], pfma(T1, es[W2][j][r], pmul(T0, cs[W2][j][r])));
            acc = cfmac(duz, psub(fzp, fz0), acc);
            acc = cfmac(ddz, psub(fzm, fz0), acc);
          }
          if (r == 0 || r < rcount) {
            const long long o = off + (r == 0 ? 0 : r * rstride);
            float2 res = acc;
            if (MODE == kResidual) res = b ? psub(BPF ? bcur : b[o], acc) : make_float2(-acc.x, -acc.y);
            if (MODE == kJacobi) res = cfmac(dinv, psub(BPF ? bcur : b[o], acc), c0);
            y[o] = res;
          }
        }
      } else {
        // x/y PML row: sum_d up_d (F_d+ - F_d0) + dn_d (F_d- - F_d0) + m (1 + i beta) mass
        const int iy = iyb + j;
        const float4 lo_t = ldg4(tq + 8), hi_t = ldg4(tq + kTabW + 8);
        const float t0 = fmaf(tf, hi_t.x - lo_t.x, lo_t.x);
        const float t1 = fmaf(tf, hi_t.y - lo_t.y, lo_t.y);
        const float t2 = fmaf(tf, hi_t.z - lo_t.z, lo_t.z);
        const float2 mc = make_float2(m, shift ? bm : 0.f);
        const float4 ax = ldg4(op.axis[0] + 4 * (size_t)ix);
        const float4 ay = ldg4(op.axis[1] + 4 * (size_t)iy);
        const float4 az = ldg4(op.axis[2] + 4 * (size_t)z);
#pragma unroll 1
        for (int r = 0; r < rcount; ++r) {
          float2 Fx[3], Fy[3], Fz[3];
          float2 ms = make_float2(0.f, 0.f), xc = ms;
#pragma unroll
          for (int i = 0; i < 3; ++i) Fx[i] = Fy[i] = ms;
#pragma unroll
          for (int dk = 0; dk < 3; ++dk) {
            const float2* q = slotp(dk == 0 ? o_m : (dk == 1 ? o_0 : o_p)) + r * K::PLANE + j * kPW;
            float2 v[3][3];
#pragma unroll
            for (int jj = 0; jj < 3; ++jj)
#pragma unroll
              for (int ii = 0; ii < 3; ++ii) v[jj][ii] = q[jj * kPW + ii];
            const float2 Ta = dup(dk == 1 ? t0 : t1), Tb = dup(dk == 1 ? t1 : t2);
            float2 vs[3], hs[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              vs[i] = padd(v[0][i], v[2][i]);
              hs[i] = padd(v[i][0], v[i][2]);
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              Fx[i] = pfma(Tb, vs[i], pfma(Ta, v[1][i], Fx[i]));
              Fy[i] = pfma(Tb, hs[i], pfma(Ta, v[i][1], Fy[i]));
            }
            const float2 faces = padd(hs[1], vs[1]), corners = padd(vs[0], vs[2]);
            Fz[dk] = pfma(dup(t2), corners, pfma(dup(t1), faces, pmul(dup(t0), v[1][1])));
            const float w0 = dk == 1 ? m01.x : m01.y, w1 = dk == 1 ? m01.y : m23.x,
                        w2 = dk == 1 ? m23.x : m23.y;
            ms = pfma(dup(w2), corners, pfma(dup(w1), faces, pfma(dup(w0), v[1][1], ms)));
            if (dk == 1) xc = v[1][1];
          }
          float2 acc = cmulc(mc, ms);
          acc = cfmac(make_float2(ax.x, ax.y), Fx[2], cfmac(make_float2(ax.z, ax.w), Fx[0],
                      cfmac(make_float2(-(ax.x + ax.z), -(ax.y + ax.w)), Fx[1], acc)));
          acc = cfmac(make_float2(ay.x, ay.y), Fy[2], cfmac(make_float2(ay.z, ay.w), Fy[0],
                      cfmac(make_float2(-(ay.x + ay.z), -(ay.y + ay.w)), Fy[1], acc)));
          acc = cfmac(make_float2(az.x, az.y), Fz[2], cfmac(make_float2(az.z, az.w), Fz[0],
                      cfmac(make_float2(-(az.x + az.z), -(az.y + az.w)), Fz[1], acc)));
          const long long o = off + r * rstride;
          float2 res = acc;
          if (MODE == kResidual) res = b ? psub(BPF ? bcur : b[o], acc) : make_float2(-acc.x, -acc.y);
          if (MODE == kJacobi) {
            const float sdx = ax.x + ax.z + ay.x + ay.z + az.x + az.z;
            const float sdy = ax.y + ax.w + ay.y + ay.w + az.y + az.w;
            const float2 diag = make_float2(fmaf(mc.x, m01.x, -t0 * sdx), fmaf(mc.y, m01.x, -t0 * sdy));
            float2 dinv = crcpf(diag);
            dinv = make_float2(omega_j * dinv.x, omega_j * dinv.y);
            res = cfmac(dinv, psub(BPF ? bcur : b[o], acc), xc);
          }
          y[o] = res;
        }
      }
    }
    // rotate the ring: plane z-1's slot takes the next issue, z+2 lands after z+1
    o_i = o_m;
    o_m = o_0;
    o_0 = o_p;
    o_p = o_p + SLOTB == RINGB ? 0u : o_p + SLOTB;
  };

  for (int z = z0; z < z1; z += 3) {
    step(I<0>{}, z);
    if (z + 1 >= z1) break;
    step(I<1>{}, z + 1);
    if (z + 2 >= z1) break;
    step(I<2>{}, z + 2);
  }
  cp_wait32<0>();
}

template <int MODE, int YB, int RB>
__global__ void __launch_bounds__(kThr, Cfg<YB, RB>::MINB)
st32_kernel(const OpDesc<float> op, const float2* __restrict__ x, const float2* __restrict__ b,
            float2* __restrict__ y, int nrhs, long long rstride, int zchunk, int zmul, float omega_j) {
  pdl_enter();
  extern __shared__ __align__(16) float2 ring[];       // [NSLOT][RB][PH][kPW]
  st32_tile<MODE, YB, RB>(op, x, b, y, nrhs, rstride, zchunk, zmul, omega_j, blockIdx.x, blockIdx.y,
                          blockIdx.z, ring);
}

// Persistent form over a list of problems of different sizes: each CTA takes
// work items (problem, tile x, tile y, RHS block + z-chunk) from a shared
// counter until the list is exhausted; every item is one st32_tile.
template <int YB, int RB>
__global__ void __launch_bounds__(kThr, Cfg<YB, RB>::MINB)
st32_group_kernel(const GroupProb* __restrict__ probs, const GroupItem* __restrict__ items, int nitems,
                  int* __restrict__ counter) {
  pdl_enter();
  extern __shared__ __align__(16) float2 ring[];
  __shared__ int next;
  __shared__ GroupProb P;                              // the current item's problem
  int cur = -1;
  for (;;) {
    __syncthreads();                                   // the previous item is done with the ring and P
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    __syncthreads();
    const int k = next;
    if (k >= nitems) break;
    const GroupItem it = items[k];
    if (it.prob != cur) {
      if (threadIdx.x == 0) P = probs[it.prob];
      __syncthreads();
      cur = it.prob;
    }
    st32_tile<kApply, YB, RB>(P.op, (const float2*)P.x, nullptr, (float2*)P.y, P.nrhs, P.rstride, P.zchunk, 1,
                              0.f, it.bx, it.by, it.bz, ring);
  }
}

// z-range per CTA: minimise (waves of CTAs) x (z-steps per CTA + ring
// prologue), with waves counted against the resident-CTA slots of the SMs.
int pick_zchunk32(int nz, long long ntiles_xy, int nrb, int slots, int prologue) {
  int best = nz;
  double best_cost = 1e300;
  for (int zc = nz; zc >= 3; --zc) {
    const long long nzc = (nz + zc - 1) / zc;
    if ((nz + nzc - 1) / nzc != zc) continue;          // same split as a larger zc
    if (nzc * nrb > 65535) break;
    const long long ctas = ntiles_xy * nrb * nzc;
    const long long waves = (ctas + slots - 1) / slots;
    const double cost = (double)waves * (zc + prologue);
    if (cost < best_cost * 0.999) {
      best_cost = cost;
      best = zc;
    }
  }
  return best;
}

// The same with tiles of two costs: n_gen tiles holding x/y-PML rows (about
// twice the per-plane cost) march zg planes per CTA, the n_cln others zmul zg;
// minimise waves x the longest CTA (in interior-plane units).  Returns zg.
int pick_zchunk32_bal(int nz, long long n_gen, long long n_cln, int nrb, int slots, int prologue, int zmul) {
  int best = nz;
  double best_cost = 1e300;
  for (int zg = nz; zg >= 3; --zg) {
    const long long nzg = (nz + zg - 1) / zg;
    if ((nz + nzg - 1) / nzg != zg) continue;
    if (nzg * nrb > 65535) break;
    const long long zc = std::min<long long>((long long)zmul * zg, nz), nzc = (nz + zc - 1) / zc;
    const long long ctas = (n_gen * nzg + n_cln * nzc) * nrb;
    const long long waves = (ctas + slots - 1) / slots;
    const double t = std::max(2.0 * zg, (double)zc) + prologue;
    const double cost = (double)waves * t;
    if (cost < best_cost * 0.999) {
      best_cost = cost;
      best = zg;
    }
  }
  return best;
}

int g_num_sms = 0;

template <int MODE, int YB, int RB>
cudaError_t launch_cfg(const OpDesc<float>& op, const void* x, const void* b, void* y, int nrhs,
                       long long rstride, double omega_j, cudaStream_t s) {
  using K = Cfg<YB, RB>;
  auto kern = st32_kernel<MODE, YB, RB>;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  if (g_num_sms <= 0) {
    if (cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) g_num_sms = 152;
  }
  const int bx = (op.nx + kW - 1) / kW, by = (op.ny + K::TY - 1) / K::TY;
  const int nrb = (nrhs + RB - 1) / RB;
  // tiles holding x/y-PML rows (the same test as in st32_tile)
  long long gen_x = 0, gen_y = 0;
  for (int t = 0; t < bx; ++t) {
    const int xa = std::max(t * kW - op.xshift, 0), xb = std::min(t * kW - op.xshift + kW - 1, op.nx - 1);
    gen_x += xa < op.plain_lo[0] || xb > op.plain_hi[0];
  }
  for (int t = 0; t < by; ++t) {
    const int ya = t * K::TY, yb = std::min(ya + K::TY - 1, op.ny - 1);
    gen_y += ya < op.plain_lo[1] || yb > op.plain_hi[1];
  }
  const long long n_cln = (long long)(bx - gen_x) * (by - gen_y), n_gen = (long long)bx * by - n_cln;
  const long long slots = (long long)g_num_sms * K::MINB;
  int zchunk = pick_zchunk32(op.nz, (long long)bx * by, nrb, (int)slots, K::D + 2);
  const long long waves = ((op.nz + zchunk - 1) / zchunk * nrb * bx * by + slots - 1) / slots;
  // with a few waves the longest CTA sets the time: balance the two tile
  // kinds; with more waves the CTA scheduler balances by itself
  const int zmul = n_gen > 0 && n_cln > 0 && waves <= 2 ? 2 : 1;
  if (zmul > 1) zchunk = pick_zchunk32_bal(op.nz, n_gen, n_cln, nrb, (int)slots, K::D + 2, zmul);
  if (HX_ST32_ZMAX > 0 && zchunk > HX_ST32_ZMAX) zchunk = (op.nz + (op.nz + HX_ST32_ZMAX - 1) / HX_ST32_ZMAX - 1) / ((op.nz + HX_ST32_ZMAX - 1) / HX_ST32_ZMAX);
  const long long gz = (long long)((op.nz + zchunk - 1) / zchunk) * nrb;
  if (gz > 65535) return cudaErrorInvalidConfiguration;
  (void)launch_k(kern, dim3(bx, by, (unsigned)gz), kThr, K::SMEM, s, op, (const float2*)x, (const float2*)b,
                 (float2*)y, nrhs, rstride, zchunk, zmul, (float)omega_j);
  count_launch(1);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_mode(const OpDesc<float>& op, int cfg, const void* x, const void* b, void* y,
                        int nrhs, long long rstride, double omega_j, cudaStream_t s) {
  switch (cfg) {
    case 0: return launch_cfg<MODE, 1, 1>(op, x, b, y, nrhs, rstride, omega_j, s);
    case 1: return launch_cfg<MODE, 1, 2>(op, x, b, y, nrhs, rstride, omega_j, s);
    case 2: return launch_cfg<MODE, 1, 4>(op, x, b, y, nrhs, rstride, omega_j, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// Kernel configurations (rows per thread YB, RHS per CTA RB):
//   0: (1,1)  1: (1,2)  2: (1,4)
int st32_num_configs() { return 3; }

int st32_default_config(int nrhs) { return nrhs == 1 ? 0 : (nrhs == 2 ? 1 : 2); }

int st32_config_rhs(int cfg) { return cfg == 0 ? 1 : (cfg == 1 ? 2 : 4); }

namespace {
template <int YB, int RB>
cudaError_t launch_group_cfg(const GroupProb* probs_dev, const GroupItem* items_dev, int nitems, int* counter,
                             cudaStream_t s) {
  using K = Cfg<YB, RB>;
  auto kern = st32_group_kernel<YB, RB>;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  if (g_num_sms <= 0) {
    if (cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) g_num_sms = 152;
  }
  const int grid = std::min(nitems, g_num_sms * K::MINB);
  (void)launch_k(kern, grid, kThr, K::SMEM, s, probs_dev, items_dev, nitems, counter);
  count_launch(1);
  return cudaGetLastError();
}
}  // namespace

void st32_group_plan(GroupProb* probs, int n, int cfg, std::vector<GroupItem>& items) {
  if (g_num_sms <= 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) g_num_sms = 152;
  }
  const int RB = st32_config_rhs(cfg);
  const int TY = kNW;                                   // every configuration has one row per thread
  // target z-planes per item: about eight items per resident CTA slot overall
  double work = 0;
  for (int i = 0; i < n; ++i) {
    const GroupProb& P = probs[i];
    work += (double)((P.op.nx + kW - 1) / kW) * ((P.op.ny + TY - 1) / TY) * ((P.nrhs + RB - 1) / RB) * P.op.nz;
  }
  const int zt = std::max(6, (int)(work / (8.0 * 2 * g_num_sms)));
  items.clear();
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  // largest problems first, so the last items to start are small ones
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)probs[a].op.nx * probs[a].op.ny * probs[a].op.nz * probs[a].nrhs >
           (double)probs[b].op.nx * probs[b].op.ny * probs[b].op.nz * probs[b].nrhs;
  });
  for (int i : order) {
    GroupProb& P = probs[i];
    const int nzc = (P.op.nz + zt - 1) / zt;
    P.zchunk = (P.op.nz + nzc - 1) / nzc;
    const int bx = (P.op.nx + kW - 1) / kW, by = (P.op.ny + TY - 1) / TY, nrb = (P.nrhs + RB - 1) / RB;
    for (int zc = 0; zc < nzc; ++zc)
      for (int y = 0; y < by; ++y)
        for (int x = 0; x < bx; ++x)
          for (int r = 0; r < nrb; ++r) items.push_back({i, x, y, zc * nrb + r});
  }
}

cudaError_t launch_stencil32_group(int cfg, const GroupProb* probs_dev, const GroupItem* items_dev, int nitems,
                                   int* counter_dev, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counter_dev, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  switch (cfg) {
    case 0: return launch_group_cfg<1, 1>(probs_dev, items_dev, nitems, counter_dev, s);
    case 1: return launch_group_cfg<1, 2>(probs_dev, items_dev, nitems, counter_dev, s);
    case 2: return launch_group_cfg<1, 4>(probs_dev, items_dev, nitems, counter_dev, s);
  }
  return cudaErrorInvalidValue;
}

int st32_xshift(const OpDesc<float>& op) {
  const int ntiles = (op.nx + kW - 1) / kW, smax = ntiles * kW - op.nx;
  if (op.plain_lo[0] > op.plain_hi[0]) return 0;   // every column stretched
  int best = 0, best_n = ntiles + 1;
  for (int sh = 0; sh <= smax; ++sh) {
    int n = 0;
    for (int t = 0; t < ntiles; ++t) {
      const int lo = std::max(t * kW - sh, 0), hi = std::min(t * kW - sh + kW - 1, op.nx - 1);
      if (lo < op.plain_lo[0] || hi > op.plain_hi[0]) ++n;
    }
    if (n < best_n) {
      best_n = n;
      best = sh;
    }
  }
  return best;
}

cudaError_t launch_stencil32(const OpDesc<float>& op_in, int mode, int cfg, const void* x, const void* b,
                             void* y, int nrhs, long long rstride, double omega_j, cudaStream_t s) {
  OpDesc<float> op = op_in;
  op.xshift = st32_xshift(op);
  switch (mode) {
    case kApply: return launch_mode<kApply>(op, cfg, x, b, y, nrhs, rstride, omega_j, s);
    case kResidual: return launch_mode<kResidual>(op, cfg, x, b, y, nrhs, rstride, omega_j, s);
    case kJacobi: return launch_mode<kJacobi>(op, cfg, x, b, y, nrhs, rstride, omega_j, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hx
