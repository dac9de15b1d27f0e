// Device code of the TMA z-marching complex64 operator kernel (template; each
// mode is instantiated in its own translation unit, hx_zmarch_<mode>.cu).
//
// Operator (Eq. 3; rows of Eqs. 4-8, GA weights of Section 3.1): an interior
// row (no x/y stretching) is 4 real class coefficients times 4 class sums of
// its 26 neighbours (centre, 6 faces, 12 edges, 8 corners):
//   y(p) = A0 c(p) + A1 [e(p) + c(p-1) + c(p+1)] + A2 [k(p) + e(p-1) + e(p+1)]
//        + A3 [k(p-1) + k(p+1)]
// with c, e, k the in-plane centre, 4-face and 4-corner sums of plane p at the
// row's column and A_k = s_k / h^2 + m wm_k (s_k the stiffness class
// coefficients x h^2, wm_k the per-point mass weights, m = omega^2 / v^2); the
// complex shift of the preconditioner adds i beta m wm_k.  Rows stretched
// along z only add (up_z - 1/h^2)(F(p+1) - F(p)) + (dn_z - 1/h^2)(F(p-1) - F(p))
// with F = t0 c + t1 e + t2 k (the transverse average of Eq. 4).
//
// GB300 layout of the work:
//  * Interior CTAs (rows with no x/y stretching): a 32 x TY column tile, RB
//    right-hand sides and a z-range.  Each z-plane of the tile (halo and all
//    RB fields included: a 36 x (TY+2) x 1 x RB box) is ONE TMA copy
//    (cp.async.bulk.tensor) issued by one thread into a ring slot and
//    completed on that slot's mbarrier; the b plane of the sweeps is a second
//    box.  Out-of-grid halo elements are zero-filled by the copy.
//  * Every plane is consumed once: its in-plane sums are scattered into the
//    three rows it feeds (p-1 finished and stored, p accumulated, p+1
//    started), so a row keeps 1 complex accumulator per RHS instead of a
//    3-plane window of sums; that is what lets 8 RHS share a CTA's row
//    coefficients.
//  * A second kernel, launched first, takes the rows in the x/y PML (the
//    "frame"), one thread per (column, z-range, RHS), in the general factored
//    form: the thread marches up its column with three planes' 3 x 3
//    neighbourhoods in registers and the next one in flight; columns are
//    packed densely, so no lane of a 32-wide tile idles on a 10-node PML
//    band, and it uses no shared memory.
//  * Packed FP32x2 arithmetic (__fadd2_rn / __ffma2_rn) for complex values
//    times real coefficients.
//  * Every wait on an mbarrier is bounded (about one second of globaltimer);
//    a CTA whose wait runs out sets *err, lets its copies in flight land
//    (again bounded) and returns.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "hx_internal.h"
#include "hx_launch.cuh"

namespace hx {

constexpr int kZXW = 36;          // x box width: 32 columns + 1 halo + 1 alignment on each side
constexpr int kZFrameThreads = 128;   // threads per CTA of the frame kernel

template <int TY, int RB, bool HASB>
struct ZK {
  static constexpr int XH = TY + 2;
  static constexpr int XBOX = kZXW * XH * RB;     // complex64 in the x box
  static constexpr int BBOX = HASB ? 32 * TY * RB : 0;
  // byte offset of the b box in a slot: a tensor copy's shared-memory
  // destination must be 128-byte aligned (slots are multiples of 128 bytes)
  static constexpr int BOFF = (XBOX * 8 + 127) / 128 * 128;
  static constexpr int SLOT = (BOFF + BBOX * 8 + 127) / 128 * 128;
  // Ring: D planes in flight beyond the one consumed, that plane, and the two
  // before it (the b and centre values of the row being finished, and the
  // z-PML terms).  D is as deep as shared memory allows, up to 6 planes:
  // within half an SM's 228 KB when registers allow two CTAs per SM (8 warps
  // per CTA), else within the 227 KB of one CTA.
  static constexpr int THREADS = 32 * TY;
  static constexpr int D2 = (113 * 1024) / SLOT - 3;          // two CTAs per SM
  static constexpr bool TWO = TY <= 8 && D2 >= 2;
  static constexpr int D1 = (227 * 1024 - 64) / SLOT - 3;     // one CTA per SM
  static constexpr int D = TWO ? (D2 < 6 ? D2 : 6) : (D1 < 6 ? D1 : 6);
  static constexpr int NSLOT = D + 3;
  static constexpr int SMEM = NSLOT * SLOT + 8 * NSLOT;
  static constexpr int MINB = TWO ? 2 : 1;   // registers: <= 128 per thread with two CTAs
  static_assert(D >= 1, "ring does not fit in shared memory");
};

struct ZParams {
  OpDesc<float> op;
  const float2* x;
  const float2* b;          // may be null (residual with b = 0)
  float2* y;
  long long pitch, plane, rstride;   // x-row pitch, z-plane and field strides (elements)
  int nrhs, zchunk, nzc, nrb;
  int xs, ys, ntx, nty;     // interior tiles: origin (xs even) and counts
  int xlo, xhi, ylo, yhi;   // rows with no x/y stretching: [xlo, xhi] x [ylo, yhi] (may be empty)
  long long fcols;          // frame columns (x or y in the PML)
  int nfc;                  // frame-kernel CTAs per (frame z-chunk, RHS)
  int fzchunk, fnzc;        // frame kernel: planes per thread, z-chunks
  float omega_j;
  int* err;
};

namespace zm {

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 dup(float s) { return make_float2(s, s); }
// Compiler-only fence: keeps the loads of the next RHS (or plane) from being
// hoisted above it, which bounds the registers a thread holds at once (the
// warps of the SM hide the shared-memory latency instead).
__device__ __forceinline__ void sched_fence() { asm volatile("" ::: "memory"); }
// acc + c v, complex c and v
__device__ __forceinline__ float2 cmac(float2 c, float2 v, float2 acc) {
  return make_float2(fmaf(c.x, v.x, fmaf(-c.y, v.y, acc.x)), fmaf(c.x, v.y, fmaf(c.y, v.x, acc.y)));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 crcp(float2 a) {
  const float d = __frcp_rn(fmaf(a.x, a.x, a.y * a.y));
  return make_float2(a.x * d, -a.y * d);
}
__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
// 1/v for the table coordinate and omega^2 / v^2, which tolerate the
// approximate reciprocal's 1-ulp error (one MUFU instruction)
__device__ __forceinline__ float rcp_fast(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float lerp(float t, float lo, float hi) { return fmaf(t, hi - lo, lo); }

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned a, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned a, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned a, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Wait for phase `parity` of the mbarrier at a; false after about a second.
__device__ __forceinline__ bool mbar_wait(unsigned a, unsigned parity) {
  if (mbar_try_wait(a, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (;;) {
    if (mbar_try_wait(a, parity)) return true;
    if (globaltimer() - t0 > 1000000000ull) return false;
  }
}
// One 4-D tile of the tensor map into shared memory at dst (128-byte
// aligned), completing on the mbarrier at bar.  c0 (x) must be even: 8-byte
// elements, 16-byte rule.
__device__ __forceinline__ void tma_load4(unsigned dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// Table position and raw entries of a row.
struct Tab {
  float4 ls, hs, lm, hm;   // stiffness class coefficients x h^2 and mass weights at nodes i0, i0 + 1
  float tf, m;             // fraction, omega^2 / v^2
  int i0;
};
__device__ __forceinline__ void tab_fetch(const OpDesc<float>& op, float vv, Tab& t) {
  const float iv = rcp_fast(vv);
  const float u = fminf(fmaxf(op.u_scale * iv, 0.f), (float)(op.n_g - 1));
  t.i0 = min((int)u, op.n_g - 2);
  t.tf = u - (float)t.i0;
  t.m = op.omega2 * iv * iv;
  const float* q = op.tab + t.i0 * kTabW;
  t.ls = ldg4(q);
  t.hs = ldg4(q + kTabW);
  t.lm = ldg4(q + 4);
  t.hm = ldg4(q + kTabW + 4);
}

// Row coefficients A_k (real) and B_k = beta m wm_k (shift), each held as a
// (c, c) pair: the packed products with a complex class sum then need no
// per-use broadcast.
struct Row {
  float2 a0, a1, a2, a3;
  float2 b0, b1, b2, b3;
};
template <bool SHIFT>
__device__ __forceinline__ void row_form(const OpDesc<float>& op, const Tab& t, Row& R) {
  const float ih2 = op.inv_h2, m = t.m, tf = t.tf;
  const float w1 = lerp(tf, t.lm.x, t.hm.x), w2 = lerp(tf, t.lm.y, t.hm.y), w3 = lerp(tf, t.lm.z, t.hm.z),
              w4 = lerp(tf, t.lm.w, t.hm.w);
  R.a0 = dup(fmaf(lerp(tf, t.ls.x, t.hs.x), ih2, m * w1));
  R.a1 = dup(fmaf(lerp(tf, t.ls.y, t.hs.y), ih2, m * w2));
  R.a2 = dup(fmaf(lerp(tf, t.ls.z, t.hs.z), ih2, m * w3));
  R.a3 = dup(fmaf(lerp(tf, t.ls.w, t.hs.w), ih2, m * w4));
  if (SHIFT) {
    const float bm = op.beta * m;
    R.b0 = dup(bm * w1);
    R.b1 = dup(bm * w2);
    R.b2 = dup(bm * w3);
    R.b3 = dup(bm * w4);
  }
}

// z-stretching of row p (a z-PML row): transverse weights t0..t2 and the
// corrections up_z - 1/h^2, dn_z - 1/h^2 of its stretched second difference.
struct ZRow {
  float t0, t1, t2;
  float2 du, dd;
};
__device__ __forceinline__ ZRow zrow(const OpDesc<float>& op, float vv, int p) {
  ZRow z;
  const float iv = rcp_fast(vv);
  const float u = fminf(fmaxf(op.u_scale * iv, 0.f), (float)(op.n_g - 1));
  const int i0 = min((int)u, op.n_g - 2);
  const float tf = u - (float)i0;
  const float* q = op.tab + i0 * kTabW + 8;
  const float4 lo = ldg4(q), hi = ldg4(q + kTabW);
  z.t0 = lerp(tf, lo.x, hi.x);
  z.t1 = lerp(tf, lo.y, hi.y);
  z.t2 = lerp(tf, lo.z, hi.z);
  const float4 az = ldg4(op.axis[2] + 4 * (size_t)p);
  z.du = make_float2(az.x - op.inv_h2, az.y);
  z.dd = make_float2(az.z - op.inv_h2, az.w);
  return z;
}

// ---------------------------------------------------------------- interior
template <int MODE, int TY, int RB, bool SHIFT>
__device__ __forceinline__ void interior(const ZParams& P, const CUtensorMap* xmap, const CUtensorMap* bmap,
                                         int cta, unsigned char* smem) {
  using K = ZK<TY, RB, MODE != kApply>;
  constexpr int NS = K::NSLOT, D = K::D;
  const OpDesc<float>& op = P.op;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int t = cta;
  const int rblk = t % P.nrb;
  t /= P.nrb;
  const int tbx = t % P.ntx;
  t /= P.ntx;
  const int tby = t % P.nty;
  const int zc = t / P.nty;
  const int gx0 = P.xs + 32 * tbx, gy0 = P.ys + TY * tby;
  const int ix = gx0 + lane, iy = gy0 + w;
  const bool act = ix >= P.xlo && ix <= P.xhi && iy <= P.yhi;
  const int r0 = rblk * RB, rcount = min(RB, P.nrhs - r0);
  const int z0 = zc * P.zchunk, z1 = min(op.nz, z0 + P.zchunk);
  const bool has_b = MODE != kApply && P.b != nullptr;
  const unsigned ring = smem_u32(smem), bars = ring + NS * K::SLOT;
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) mbar_init(bars + 8 * k, 1);
    fence_mbar_init();
  }
  __syncthreads();
  constexpr unsigned XB = K::XBOX * 8, BB = K::BBOX * 8, BO = K::BOFF;
  // plane q (z0 - 1 <= q <= z1) goes to slot (q - z0 + 1) % NS
  auto issue = [&](int q) {
    const int sl = (q - z0 + 1) % NS;
    const unsigned dst = ring + sl * K::SLOT, bar = bars + 8 * sl;
    const bool need_b = has_b && q >= z0 && q < z1;
    mbar_expect_tx(bar, XB + (need_b ? BB : 0u));
    tma_load4(dst, xmap, gx0 - 2, gy0 - 1, q, r0, bar);
    if (need_b) tma_load4(dst + BO, bmap, gx0, gy0, q, r0, bar);
  };
  if (tid == 0)
    for (int q = z0 - 1; q <= min(z1, z0 - 1 + D); ++q) issue(q);

  const int zlo = op.plain_lo[2], zhi = op.plain_hi[2];
  const long long vplane = (long long)op.nx * op.ny;
  const float* vp = op.v + (act ? (long long)iy * op.nx + ix : 0);
  auto vload = [&](int p) { return act && p < z1 ? __ldg(vp + p * vplane) : 1500.f; };
  float vn = vload(z0);                                // v of the row formed at the next step
  Row rw[3];
  float2 acc[3][RB];                                   // per row slot and RHS
  float2* yb = P.y + (long long)r0 * P.rstride + (act ? (long long)iy * P.pitch + ix : 0);
  // this thread's window in a slot: x box element (lane + 1, w) and b box element (lane, w)
  const int xoff = w * kZXW + lane + 1, boff = w * 32 + lane;
  auto slot_x = [&](int j) { return reinterpret_cast<const float2*>(smem + (j % NS) * K::SLOT) + xoff; };
  // in-plane centre, 4-face and 4-corner sums of field r of the plane in slot X
  auto sums = [&](const float2* X, int r, float2& c, float2& e, float2& k) {
    const float2* s = X + r * (K::XH * kZXW);
    const float2 L0 = s[0], M0 = s[1], R0 = s[2];
    const float2 L1 = s[kZXW], M1 = s[kZXW + 1], R1 = s[kZXW + 2];
    const float2 L2 = s[2 * kZXW], M2 = s[2 * kZXW + 1], R2 = s[2 * kZXW + 2];
    c = M1;
    e = f2add(f2add(L1, R1), f2add(M0, M2));
    k = f2add(f2add(L0, R0), f2add(L2, R2));
  };
  bool bad = false;
  int qfail = z1;

  // FULL: rows q - 1, q and q + 1 all in this CTA's range and row q - 1 outside
  // the z-PML (the common step, compiled without those branches)
  auto step = [&](auto ptag, auto ftag, int q) {
    constexpr int PP = decltype(ptag)::value;
    constexpr bool FULL = decltype(ftag)::value;
    constexpr int SP = (PP + 2) % 3, SC = PP, SN = (PP + 1) % 3;   // row slots of q - 1, q, q + 1
    const int j = q - z0 + 1;
    const bool do_prev = FULL || q - 1 >= z0, do_cur = FULL || (q >= z0 && q < z1),
               do_next = FULL || q + 1 < z1;
    // row q + 1's table entries are requested before the wait for plane q
    Tab tb;
    if (do_next) tab_fetch(op, vn, tb);
    vn = vload(q + 2);
    const bool ok = mbar_wait(bars + 8 * (j % NS), (unsigned)(j / NS) & 1u);
    bad = bad || !ok;
    if (do_next) row_form<SHIFT>(op, tb, rw[SN]);
    if (ok) {
      const float2* X = slot_x(j);
      // row q - 1 is completed by this plane and stored in the same pass.  A
      // z-PML row adds its z-stretching terms from the plane sums of q - 2,
      // q - 1 and q, recomputed out of the ring (which keeps plane q - 2).
      const bool zp = !FULL && do_prev && (q - 1 < zlo || q - 1 > zhi);
      ZRow Z;
      if (zp) Z = zrow(op, vload(q - 1), q - 1);
      const float2* Xp = slot_x(j - 1);
      const float2* Bp = reinterpret_cast<const float2*>(smem + ((j - 1) % NS) * K::SLOT + BO) + boff;
      float2 dinv = make_float2(0.f, 0.f);
      if (MODE == kJacobi && do_prev) {
        const Row& R = rw[SP];
        float2 diag = make_float2(R.a0.x, SHIFT ? R.b0.x : 0.f);
        if (zp) diag = make_float2(diag.x - Z.t0 * (Z.du.x + Z.dd.x), diag.y - Z.t0 * (Z.du.y + Z.dd.y));
        dinv = crcp(diag);
        dinv = make_float2(P.omega_j * dinv.x, P.omega_j * dinv.y);
      }
      float2* yo = yb + (long long)(q - 1) * P.plane;
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        float2 c, e, k;
        sums(X, r, c, e, k);
        // with the shift the class coefficients are A_k + i B_k: the B part
        // multiplies the sums rotated by i (one accumulator per row and RHS)
        float2 ic, ie, ik;
        if (SHIFT) {
          ic = make_float2(-c.y, c.x);
          ie = make_float2(-e.y, e.x);
          ik = make_float2(-k.y, k.x);
        }
        if (do_prev) {
          const Row& R = rw[SP];
          float2 a = f2fma(R.a3, k, f2fma(R.a2, e, f2fma(R.a1, c, acc[SP][r])));
          if (SHIFT) a = f2fma(R.b3, ik, f2fma(R.b2, ie, f2fma(R.b1, ic, a)));
          if (zp) {
            float2 c2, e2, k2;
            sums(slot_x(j - 2), r, c2, e2, k2);
            const float2 Fm = f2fma(dup(Z.t2), k2, f2fma(dup(Z.t1), e2, f2mul(dup(Z.t0), c2)));
            sched_fence();
            sums(Xp, r, c2, e2, k2);
            const float2 F0 = f2fma(dup(Z.t2), k2, f2fma(dup(Z.t1), e2, f2mul(dup(Z.t0), c2)));
            const float2 Fp = f2fma(dup(Z.t2), k, f2fma(dup(Z.t1), e, f2mul(dup(Z.t0), c)));
            a = cmac(Z.du, f2sub(Fp, F0), cmac(Z.dd, f2sub(Fm, F0), a));
          }
          float2 res = a;
          if (MODE == kResidual) res = has_b ? f2sub(Bp[r * (TY * 32)], a) : make_float2(-a.x, -a.y);
          if (MODE == kJacobi) {
            const float2 rr = has_b ? f2sub(Bp[r * (TY * 32)], a) : make_float2(-a.x, -a.y);
            res = cmac(dinv, rr, Xp[r * (K::XH * kZXW) + kZXW + 1]);
          }
          if (act && (r == 0 || r < rcount)) yo[r * P.rstride] = res;
        }
        if (do_cur) {
          const Row& R = rw[SC];
          acc[SC][r] = f2fma(R.a2, k, f2fma(R.a1, e, f2fma(R.a0, c, acc[SC][r])));
          if (SHIFT) acc[SC][r] = f2fma(R.b2, ik, f2fma(R.b1, ie, f2fma(R.b0, ic, acc[SC][r])));
        }
        if (do_next) {
          const Row& R = rw[SN];
          acc[SN][r] = f2fma(R.a3, k, f2fma(R.a2, e, f2mul(R.a1, c)));
          if (SHIFT) acc[SN][r] = f2fma(R.b3, ik, f2fma(R.b2, ie, f2fma(R.b1, ic, acc[SN][r])));
        }
        sched_fence();
      }
    }
    // every thread is done with plane q - 2's slot; refill it
    if (__syncthreads_or(bad)) {
      qfail = q;
      return false;
    }
    if (tid == 0 && q + D + 1 <= z1) issue(q + D + 1);
    return true;
  };

  auto full = [&](int q) { return q - 1 >= z0 && q + 1 < z1 && q - 1 >= zlo && q - 1 <= zhi; };
  auto run_step = [&](auto ptag, int q) {
    return full(q) ? step(ptag, std::true_type{}, q) : step(ptag, std::false_type{}, q);
  };
  bool run = true;
  for (int q = z0 - 1; run && q <= z1; q += 3) {
    run = run_step(std::integral_constant<int, 0>{}, q);
    if (!run || q + 1 > z1) break;
    run = run_step(std::integral_constant<int, 1>{}, q + 1);
    if (!run || q + 2 > z1) break;
    run = run_step(std::integral_constant<int, 2>{}, q + 2);
  }
  if (!run) {
    // a wait ran out: record it, and let the copies still in flight (planes
    // qfail .. qfail + D, issued before the failing step) land before the
    // CTA's shared memory is released, each wait bounded as well
    if (tid == 0) {
      if (P.err) atomicExch(P.err, 1);
      for (int q = qfail; q <= min(z1, qfail + D); ++q) {
        const int j = q - z0 + 1;
        (void)mbar_wait(bars + 8 * (j % NS), (unsigned)(j / NS) & 1u);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- frame
// Column c of the frame (rows with x or y in the PML) -> (ix, iy).
__device__ __forceinline__ void frame_column(const ZParams& P, long long c, int& ix, int& iy) {
  const int nx = P.op.nx;
  const long long na = (long long)P.ylo * nx;
  if (c < na) {
    iy = (int)(c / nx);
    ix = (int)(c - (long long)iy * nx);
    return;
  }
  c -= na;
  const long long nb = (long long)(P.op.ny - 1 - P.yhi) * nx;
  if (c < nb) {
    const int q = (int)(c / nx);
    iy = P.yhi + 1 + q;
    ix = (int)(c - (long long)q * nx);
    return;
  }
  c -= nb;
  const int wx = P.xlo + (nx - 1 - P.xhi);
  const int q = (int)(c / wx), kx = (int)(c - (long long)q * wx);
  iy = P.ylo + q;
  ix = kx < P.xlo ? kx : P.xhi + 1 + (kx - P.xlo);
}

// General row (any stretching): sum_d up_d (F_d+ - F_d0) + dn_d (F_d- - F_d0)
// + m (1 + i beta) mass, F_d the transverse averages (t0, t1, t2) of the
// planes normal to d.  One thread per (frame column, z-range, RHS): it marches
// up its column with the 3 x 3 neighbourhoods of planes z - 1, z, z + 1 in
// registers while plane z + 2 is in flight, so each plane is read once per
// column instead of once per row it feeds.  Neighbourhood element 3 dj + di is
// (ix + di - 1, iy + dj - 1); out-of-grid elements are zero.
template <int MODE, bool SHIFT>
__device__ __forceinline__ void frame(const ZParams& P, int fcta) {
  const OpDesc<float>& op = P.op;
  int t = fcta;
  const int r = t % P.nrhs;
  t /= P.nrhs;
  const int zc = t % P.fnzc;
  const long long c = (long long)(t / P.fnzc) * kZFrameThreads + threadIdx.x;
  if (c >= P.fcols) return;
  int ix, iy;
  frame_column(P, c, ix, iy);
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const int z0 = zc * P.fzchunk, z1 = min(nz, z0 + P.fzchunk);
  const bool has_b = MODE != kApply && P.b != nullptr;
  const float4 ax = ldg4(op.axis[0] + 4 * (size_t)ix), ay = ldg4(op.axis[1] + 4 * (size_t)iy);
  unsigned in9 = 0;   // bit 3 dj + di: that neighbour lies inside the grid
#pragma unroll
  for (int dj = 0; dj < 3; ++dj)
#pragma unroll
    for (int di = 0; di < 3; ++di)
      if ((dj != 0 || iy > 0) && (dj != 2 || iy < ny - 1) && (di != 0 || ix > 0) && (di != 2 || ix < nx - 1))
        in9 |= 1u << (3 * dj + di);
  const long long roff = (long long)r * P.rstride + (long long)iy * P.pitch + ix;
  const float* vc = op.v + (long long)iy * nx + ix;
  const long long vplane = (long long)nx * ny;

  // columns away from the grid's x/y faces read their neighbourhoods unchecked
  const bool face = in9 != 0x1ffu;
  auto load = [&](float2(&a)[9], int q) {
    if (q < 0 || q >= nz) {
#pragma unroll
      for (int k = 0; k < 9; ++k) a[k] = make_float2(0.f, 0.f);
      return;
    }
    const float2* p = P.x + roff + (long long)q * P.plane;
    if (!face) {
#pragma unroll
      for (int dj = 0; dj < 3; ++dj)
#pragma unroll
        for (int di = 0; di < 3; ++di) a[3 * dj + di] = __ldg(p + (dj - 1) * P.pitch + (di - 1));
    } else {
#pragma unroll
      for (int dj = 0; dj < 3; ++dj)
#pragma unroll
        for (int di = 0; di < 3; ++di)
          a[3 * dj + di] = ((in9 >> (3 * dj + di)) & 1u) ? __ldg(p + (dj - 1) * P.pitch + (di - 1))
                                                          : make_float2(0.f, 0.f);
    }
  };

  // row z from the neighbourhoods of planes z - 1 (Am), z (A0) and z + 1 (Ap)
  auto row = [&](const float2(&Am)[9], const float2(&A0)[9], const float2(&Ap)[9], int z, float vv) {
    const long long oo = roff + (long long)z * P.plane;
    const float2 bz = has_b ? __ldg(P.b + oo) : make_float2(0.f, 0.f);
    const float iv = rcp_fast(vv);
    const float u = fminf(fmaxf(op.u_scale * iv, 0.f), (float)(op.n_g - 1));
    const int i0 = min((int)u, op.n_g - 2);
    const float tf = u - (float)i0;
    const float m = op.omega2 * iv * iv;
    const float* tq = op.tab + i0 * kTabW;
    const float4 lm = ldg4(tq + 4), hm = ldg4(tq + kTabW + 4), lt = ldg4(tq + 8), ht = ldg4(tq + kTabW + 8);
    const float w1 = lerp(tf, lm.x, hm.x), w2 = lerp(tf, lm.y, hm.y), w3 = lerp(tf, lm.z, hm.z),
                w4 = lerp(tf, lm.w, hm.w);
    const float t0 = lerp(tf, lt.x, ht.x), t1 = lerp(tf, lt.y, ht.y), t2 = lerp(tf, lt.z, ht.z);
    const float4 az = ldg4(op.axis[2] + 4 * (size_t)z);
    const float2 mc = make_float2(m, SHIFT ? op.beta * m : 0.f);
    float2 Fx[3], Fy[3], Fz[3];
    float2 ms = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 3; ++i) Fx[i] = Fy[i] = ms;
    auto plane = [&](const float2(&a)[9], int dk) {
      // weights of this plane in the transverse averages normal to x and y
      const float2 Ta = dup(dk == 1 ? t0 : t1), Tb = dup(dk == 1 ? t1 : t2);
      float2 vs[3], hs[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        vs[i] = f2add(a[i], a[6 + i]);           // column i: y-neighbours
        hs[i] = f2add(a[3 * i], a[3 * i + 2]);   // row i: x-neighbours
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        Fx[i] = f2fma(Tb, vs[i], f2fma(Ta, a[3 + i], Fx[i]));
        Fy[i] = f2fma(Tb, hs[i], f2fma(Ta, a[3 * i + 1], Fy[i]));
      }
      const float2 faces = f2add(hs[1], vs[1]), corners = f2add(vs[0], vs[2]);
      Fz[dk] = f2fma(dup(t2), corners, f2fma(dup(t1), faces, f2mul(dup(t0), a[4])));
      // consistent mass (second form of Eq. 8): centre / faces / edges / corners
      const float m0 = dk == 1 ? w1 : w2, m1 = dk == 1 ? w2 : w3, m2 = dk == 1 ? w3 : w4;
      ms = f2fma(dup(m2), corners, f2fma(dup(m1), faces, f2fma(dup(m0), a[4], ms)));
    };
    plane(Am, 0);
    plane(A0, 1);
    plane(Ap, 2);
    float2 acc = cmul(mc, ms);
    acc = cmac(make_float2(ax.x, ax.y), Fx[2], cmac(make_float2(ax.z, ax.w), Fx[0],
               cmac(make_float2(-(ax.x + ax.z), -(ax.y + ax.w)), Fx[1], acc)));
    acc = cmac(make_float2(ay.x, ay.y), Fy[2], cmac(make_float2(ay.z, ay.w), Fy[0],
               cmac(make_float2(-(ay.x + ay.z), -(ay.y + ay.w)), Fy[1], acc)));
    acc = cmac(make_float2(az.x, az.y), Fz[2], cmac(make_float2(az.z, az.w), Fz[0],
               cmac(make_float2(-(az.x + az.z), -(az.y + az.w)), Fz[1], acc)));
    float2 res = acc;
    if (MODE == kResidual) res = f2sub(bz, acc);
    if (MODE == kJacobi) {
      const float sdx = ax.x + ax.z + ay.x + ay.z + az.x + az.z;
      const float sdy = ax.y + ax.w + ay.y + ay.w + az.y + az.w;
      float2 dinv = crcp(make_float2(fmaf(mc.x, w1, -t0 * sdx), fmaf(mc.y, w1, -t0 * sdy)));
      dinv = make_float2(P.omega_j * dinv.x, P.omega_j * dinv.y);
      res = cmac(dinv, f2sub(bz, acc), A0[4]);
    }
    P.y[oo] = res;
  };

  // the window rotates through four register sets: (W0, W1, W2) hold planes
  // z - 1, z, z + 1 while plane z + 2 is loaded into W3, and so on
  float2 W0[9], W1[9], W2[9], W3[9];
  load(W0, z0 - 1);
  load(W1, z0);
  load(W2, z0 + 1);
  float vv = __ldg(vc + z0 * vplane);
  auto it = [&](float2(&Am)[9], float2(&A0)[9], float2(&Ap)[9], float2(&An)[9], int z) {
    float vn = 1500.f;
    if (z + 1 < z1) {
      load(An, z + 2);
      vn = __ldg(vc + (z + 1) * vplane);
    }
    row(Am, A0, Ap, z, vv);
    vv = vn;
  };
#pragma unroll 1
  for (int z = z0; z < z1; z += 4) {
    it(W0, W1, W2, W3, z);
    if (z + 1 >= z1) break;
    it(W1, W2, W3, W0, z + 1);
    if (z + 2 >= z1) break;
    it(W2, W3, W0, W1, z + 2);
    if (z + 3 >= z1) break;
    it(W3, W0, W1, W2, z + 3);
  }
}

// The two kernels of a launch: the frame rows (no shared memory, so they run
// at high occupancy with their own register budget), then the interior tiles.
// They write disjoint rows; the interior kernel is launched after the frame
// kernel on the same stream (dependent launch hides the gap).
template <int MODE, bool SHIFT>
__global__ void __launch_bounds__(kZFrameThreads, 3) zm_frame_kernel(const ZParams P) {
  pdl_enter();
  frame<MODE, SHIFT>(P, blockIdx.x);
}

template <int MODE, int TY, int RB, bool SHIFT>
__global__ void __launch_bounds__(32 * TY, (ZK<TY, RB, MODE != kApply>::MINB))
zm_kernel(const ZParams P, const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap bmap) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char zsmem[];
  interior<MODE, TY, RB, SHIFT>(P, &xmap, &bmap, blockIdx.x, zsmem);
}

}  // namespace zm

// Host side of one mode (hx_zmarch_<mode>.cu): launches config (TY, RB).
// frame: CTAs of the frame kernel (0: none); interior: CTAs of the interior
// kernel (0: none).
template <int MODE, int TY, int RB>
cudaError_t zm_launch_mode(const ZParams& P, bool shift, const CUtensorMap& xmap, const CUtensorMap& bmap,
                           int frame, int interior, cudaStream_t s) {
  using K = ZK<TY, RB, MODE != kApply>;
  if (frame > 0) {
    auto fk = shift ? zm::zm_frame_kernel<MODE, true> : zm::zm_frame_kernel<MODE, false>;
    cudaError_t e = launch_k(fk, dim3((unsigned)frame), dim3(kZFrameThreads), 0, s, P);
    count_launch(1);
    if (e != cudaSuccess) return e;
  }
  if (interior <= 0) return cudaSuccess;
  auto kern = shift ? zm::zm_kernel<MODE, TY, RB, true> : zm::zm_kernel<MODE, TY, RB, false>;
  static bool attr_set[2][64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[shift][dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[shift][dev] = true;
  }
  count_launch(1);
  return launch_k(kern, dim3((unsigned)interior), dim3(K::THREADS), (size_t)K::SMEM, s, P, xmap, bmap);
}

}  // namespace hx
