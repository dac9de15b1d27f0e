// Complex64 z-marching kernel of the adaptive 27-point operator [M + S]
// (Eq. 3; rows of Eqs. 4-8 with the GA weight selection of Section 3.1).
//
// Same operator, modes and results as the generic kernel in hx_stencil.cu
// (which keeps the complex128 path); this one is arranged for instruction
// economy and latency hiding, because the complex64 apply is issue- and
// latency-bound long before it is bandwidth-bound:
//  * a CTA owns a 32 x TY column tile, RB right-hand sides and a z-range;
//    one producer warp streams the x planes (tile + 1-node halo, RB fields)
//    into an NSLOT-plane shared-memory ring, NC consumer warps compute;
//  * the producer copies each tile row with one cp.async.bulk (the
//    16-byte-aligned inner part of the row) plus at most two 8-byte cp.async
//    for unaligned ends, all completing on the slot's "full" mbarrier; the
//    consumers release a slot on its "empty" mbarrier, so consumer warps
//    never meet at a CTA-wide barrier inside the z loop;
//  * the ring row pitch has the parity of nx and each (plane, field) is
//    stored at a parity offset c0 in {1, 2}: every element then sits at a
//    shared address congruent to its global address mod 16, which is what
//    lets one bulk copy serve a row whatever the row's alignment;
//  * complex additions and real-times-complex products use the packed
//    FP32x2 instructions of sm_100+ (add/sub/mul/fma .f32x2);
//  * a warp covers 32 consecutive x; each thread owns YB consecutive y rows
//    of its column, so the in-plane sums of neighbouring rows share their
//    horizontal pair sums;
//  * per column and plane the in-plane class sums (centre, 4 faces, 4
//    corners) live in registers for the three z-steps that use them; the z
//    loop is unrolled by three so this window rotates without moves;
//  * 1/v comes from the approximate reciprocal (the table coordinate and
//    omega^2/v^2 tolerate its 1-ulp error);
//  * rows whose only complex stretching is along z stay on the register
//    path; rows in the x/y PML read their 27 neighbours from the ring.
// Every mbarrier wait is bounded: on expiry the kernel sets a device flag
// (read by the host as HX_ERR_TIMEOUT) and the waiting warp leaves its loop.
#include "hx_complex.cuh"
#include "hx_internal.h"

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
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
// the async arrive of the executing thread fires when all of its prior
// cp.async copies have landed; it counts as one of the barrier's arrivals
__device__ __forceinline__ void cp_arrive_noinc(unsigned bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void cp8(unsigned dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
// bytes (a multiple of 16) from a 16-byte aligned global address to a
// 16-byte aligned shared address, completing on bar
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Set by a bounded wait that ran out (never in correct operation).
__device__ int g_st32_timeout;
constexpr int kWaitLimit = 1 << 22;
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (int it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(&g_st32_timeout, 1);
  return false;
}

template <int V>
struct I {
  static constexpr int value = V;
};

// ------------------------------------------------------------ configuration
constexpr int kW = 32;              // tile extent in x: one warp
constexpr int kPWmax = 38;          // ring row pitch: 37 (odd nx) or 38 (even nx)

// YB rows per thread, RB right-hand sides per CTA; the register window grows
// with YB * RB, so the larger configurations run fewer consumer warps (NC)
// with more registers each.
template <int YB, int RB>
struct Cfg {
  static constexpr int NC = YB * RB <= 1 ? 8 : 4;       // consumer warps per CTA
  static constexpr int THR = 32 * (NC + 1);            // + one producer warp
  static constexpr int MINB = YB * RB <= 1 ? 2 : (YB * RB <= 2 ? 3 : 2);   // resident CTAs per SM
  static constexpr int TY = NC * YB;                   // tile extent in y
  static constexpr int PH = TY + 2;                    // ring rows (tile + halo)
  static constexpr int FPLANE = (PH * kPWmax + 1) & ~1;   // complex64 per field plane (even)
  static constexpr int SLOTE = FPLANE * RB;            // complex64 per ring slot
  // NSLOT must be even: a (slot, field) plane's parity offset c0 depends on
  // z only through z & 1, so an even slot count gives every reuse of a slot
  // the offset of its previous fill, and the out-of-grid halo positions that
  // no copy writes keep the zeros stored at start-up
  static constexpr int NSLOT = 8;
  static constexpr int D = NSLOT - 3;                  // planes in flight beyond the window
  static constexpr int BAR_BYTES = 256;                // 2 NSLOT mbarriers, padded
  static constexpr int SMEM = BAR_BYTES + NSLOT * SLOTE * 8;
  static_assert(NSLOT % 2 == 0, "slot reuse must keep the parity offset");
};

template <int MODE, int YB, int RB>
__global__ void __launch_bounds__(Cfg<YB, RB>::THR, Cfg<YB, RB>::MINB)
st32_kernel(const OpDesc<float> op, const float2* __restrict__ x, const float2* __restrict__ b,
            float2* __restrict__ y, int nrhs, long long rstride, int zchunk, float omega_j) {
  using K = Cfg<YB, RB>;
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(smem);
  const unsigned full0 = sbase, empty0 = sbase + 8 * K::NSLOT;    // mbarriers
  const unsigned ring0 = sbase + K::BAR_BYTES;                     // ring of NSLOT slots
  constexpr unsigned SLOTB = K::SLOTE * 8, FPB = K::FPLANE * 8;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const int PW = 37 + ((nx & 1) ^ 1);                  // row pitch, parity of nx
  const int gx0 = blockIdx.x * kW, gy0 = blockIdx.y * K::TY;
  const int nrb = (nrhs + RB - 1) / RB;
  const int rblk = blockIdx.z % nrb, zc = blockIdx.z / nrb;
  const int r0 = rblk * RB, rcount = min(RB, nrhs - r0);
  const int z0 = zc * zchunk, z1 = min(nz, z0 + zchunk);
  const int np = z1 - z0 + 2;                          // planes z0-1 .. z1
  const long long plane = (long long)nx * ny;
  // parity of the global element index of tile element (row 0, col 0) of
  // plane z, field r0 + r is  g0par ^ (z & ppar) ^ rpar[r];  the element is
  // stored at offset c0 = 2 - parity inside its (slot, field) plane
  const int g0par = ((gy0 - 1) * nx + gx0 - 1) & 1;
  const int ppar = (int)(plane & 1);
  int rpar[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) rpar[r] = (int)((((long long)(r0 + r)) * rstride) & 1);

  // zero the ring (rows outside the grid are never written afterwards), set
  // up the barriers: full = 32 producer-lane arrivals (+ bulk bytes),
  // empty = one arrival per consumer warp
  for (int i = tid; i < K::NSLOT * K::SLOTE; i += K::THR)
    asm volatile("st.shared.v2.f32 [%0], {%1, %1};" ::"r"(ring0 + 8u * i), "f"(0.f) : "memory");
  if (tid < K::NSLOT) {
    mbar_init(full0 + 8 * tid, 32);
    mbar_init(empty0 + 8 * tid, K::NC);
  }
  fence_async_smem();
  __syncthreads();

  if (warp == K::NC) {
    // ------------------------------------------------------------ producer
    const int j = lane;                                // tile row copied by this lane
    const int gy = gy0 - 1 + j;
    const bool row_ok = j < K::PH && gy >= 0 && gy < ny;
    const int xa = max(gx0 - 1, 0), xb = min(gx0 + kW, nx - 1);   // row segment in the grid
    const int lxa = xa - (gx0 - 1);                    // its first tile column
    int s = 0, ph = 0;                                 // slot and its fill parity
    for (int p = 0; p < np; ++p) {
      const int z = z0 - 1 + p;
      if (p >= K::NSLOT && !mbar_wait(empty0 + 8 * s, ph ^ 1)) break;
      const unsigned full = full0 + 8 * s, slot = ring0 + s * SLOTB;
      if (z < 0 || z >= nz) {
        for (int i = lane; i < K::SLOTE; i += 32)
          asm volatile("st.shared.v2.f32 [%0], {%1, %1};" ::"r"(slot + 8u * i), "f"(0.f) : "memory");
        fence_async_smem();
        mbar_arrive(full);
      } else if (!row_ok) {
        mbar_arrive(full);
      } else {
        const int zp = z & ppar;
        unsigned bytes = 0;
        long long ga[RB], gb[RB];
        unsigned da[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const long long g = (long long)(r0 + r) * rstride + (long long)z * plane + (long long)gy * nx + xa;
          const long long ge = g + (xb - xa + 1);       // exclusive end
          ga[r] = (g + 1) & ~1LL;
          gb[r] = ge & ~1LL;
          const int c0 = 2 - (g0par ^ zp ^ rpar[r]);
          da[r] = slot + r * FPB + 8u * (c0 + j * PW + lxa + (int)(ga[r] - g));
          if (r < rcount && gb[r] > ga[r]) bytes += (unsigned)(gb[r] - ga[r]) * 8u;
        }
        if (bytes) mbar_expect_tx(full, bytes);
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          if (r >= rcount) continue;
          if (gb[r] > ga[r]) bulk_g2s(da[r], x + ga[r], (unsigned)(gb[r] - ga[r]) * 8u, full);
          const long long g = (long long)(r0 + r) * rstride + (long long)z * plane + (long long)gy * nx + xa;
          const long long ge = g + (xb - xa + 1);
          if (g & 1) cp8(da[r] - 8u * (unsigned)(ga[r] - g), x + g);                 // first element
          if ((ge & 1) && ge - 1 >= ga[r]) cp8(da[r] + 8u * (unsigned)(gb[r] - ga[r]), x + gb[r]);   // last
        }
        cp_arrive_noinc(full);
      }
      if (++s == K::NSLOT) { s = 0; ph ^= 1; }
    }
    // let the last fills land before the warp leaves
    for (int q = 0; q < K::NSLOT && q < np; ++q) {
      if (--s < 0) { s = K::NSLOT - 1; ph ^= 1; }
      if (!mbar_wait(full0 + 8 * s, ph)) break;
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  const int tx = lane, w = warp;
  const int ix = gx0 + tx, iyb = gy0 + w * YB;
  const bool shift = op.beta != 0.f;
  // shared byte offset of this thread's 3 x (YB + 2) window in a field plane
  const unsigned thr = 8u * (unsigned)((w * YB) * PW + tx);
  const unsigned rowb = 8u * PW;
  // byte offset (from smem) of this thread's window in field plane (slot, r) of plane z
  auto fbase = [&](int slot, int r, int z) -> unsigned {
    return K::BAR_BYTES + slot * SLOTB + r * FPB + 8u * (unsigned)(2 - (g0par ^ (z & ppar) ^ rpar[r])) + thr;
  };
  auto lds2 = [&](unsigned off) { return *reinterpret_cast<const float2*>(smem + off); };

  float2 cs[3][YB][RB], es[3][YB][RB], ks[3][YB][RB];
  auto sums = [&](int slot, int z, auto wtag) {
    constexpr int WS = decltype(wtag)::value;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const unsigned q = fbase(slot, r, z);
      float2 M[YB + 2], H[YB + 2];
#pragma unroll
      for (int rr = 0; rr < YB + 2; ++rr) {
        const unsigned qa = q + rr * rowb;
        M[rr] = lds2(qa + 8);
        H[rr] = padd(lds2(qa), lds2(qa + 16));
      }
#pragma unroll
      for (int j = 0; j < YB; ++j) {
        cs[WS][j][r] = M[j + 1];
        es[WS][j][r] = padd(H[j + 1], padd(M[j], M[j + 2]));
        ks[WS][j][r] = padd(H[j], H[j + 2]);
      }
    }
  };

  bool ok = mbar_wait(full0, 0) && mbar_wait(full0 + 8, 0);   // planes z0-1, z0
  sums(0, z0 - 1, I<0>{});
  sums(1, z0, I<1>{});
  // slots of planes z-1, z and of the next plane to wait for (z+1), its parity
  int s_m = 0, s_0 = 1, s_w = 2, ph_w = 0;
  if (s_w == K::NSLOT) { s_w = 0; ph_w = 1; }

  const bool xin = ix < nx;
  const bool plain_x = ix >= op.plain_lo[0] && ix <= op.plain_hi[0];
  bool act[YB], plain_xy[YB];
  float vnext[YB];
  const float* vp[YB];                                 // v at (ix, iy, z + 1)
  long long yo[YB];                                    // element offset of (ix, iy, z) in field r0
#pragma unroll
  for (int j = 0; j < YB; ++j) {
    const int iy = iyb + j;
    act[j] = xin && iy < ny;
    plain_xy[j] = plain_x && iy >= op.plain_lo[1] && iy <= op.plain_hi[1];
    const long long o = (long long)z0 * plane + (long long)(act[j] ? iy * nx + ix : 0);
    vnext[j] = act[j] && z0 < z1 ? __ldg(op.v + o) : 1.f;
    vp[j] = op.v + o + plane;
    yo[j] = o + (long long)r0 * rstride;
  }
  const float umax = (float)(op.n_g - 1);
  const float ih2 = op.inv_h2;
  const unsigned zlo = (unsigned)op.plain_lo[2], zspan = (unsigned)(op.plain_hi[2] - op.plain_lo[2]);

  auto step = [&](auto ptag, int z) {
    constexpr int P = decltype(ptag)::value;
    constexpr int W0 = P % 3, W1 = (P + 1) % 3, W2 = (P + 2) % 3;   // planes z-1, z, z+1
    ok = ok && mbar_wait(full0 + 8 * s_w, ph_w);        // plane z+1 landed
    sums(s_w, z + 1, I<W2>{});
    const bool plain_z = (unsigned)z - zlo <= zspan;
#pragma unroll
    for (int j = 0; j < YB; ++j) {
      const float vv = vnext[j];
      if (act[j] && z + 1 < z1) vnext[j] = __ldg(vp[j]);
      vp[j] += plane;
      const long long off = yo[j];
      yo[j] += plane;
      if (!act[j]) continue;
      // table position of 1/G = f h / v and the interpolated derived weights
      const float iv = rcp_approx(vv);
      const float u = fminf(fmaxf(op.u_scale * iv, 0.f), umax);
      const int i0 = min((int)u, op.n_g - 2);
      const float tf = u - (float)i0;
      const float* tq = op.tab + i0 * kTabW;
      const float m = op.omega2 * iv * iv;
      const float4 lo_s = ldg4(tq), hi_s = ldg4(tq + kTabW);
      const float4 lo_m = ldg4(tq + 4), hi_m = ldg4(tq + kTabW + 4);
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
            if (MODE == kResidual) res = b ? psub(b[o], acc) : make_float2(-acc.x, -acc.y);
            if (MODE == kJacobi) res = cfmac(dinv, psub(b[o], acc), c0);
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
            const unsigned q = fbase(dk == 0 ? s_m : (dk == 1 ? s_0 : s_w), r, z - 1 + dk) + j * rowb;
            float2 v[3][3];
#pragma unroll
            for (int jj = 0; jj < 3; ++jj)
#pragma unroll
              for (int ii = 0; ii < 3; ++ii) v[jj][ii] = lds2(q + jj * rowb + 8 * ii);
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
          if (MODE == kResidual) res = b ? psub(b[o], acc) : make_float2(-acc.x, -acc.y);
          if (MODE == kJacobi) {
            const float sdx = ax.x + ax.z + ay.x + ay.z + az.x + az.z;
            const float sdy = ax.y + ax.w + ay.y + ay.w + az.y + az.w;
            const float2 diag = make_float2(fmaf(mc.x, m01.x, -t0 * sdx), fmaf(mc.y, m01.x, -t0 * sdy));
            float2 dinv = crcpf(diag);
            dinv = make_float2(omega_j * dinv.x, omega_j * dinv.y);
            res = cfmac(dinv, psub(b[o], acc), xc);
          }
          y[o] = res;
        }
      }
    }
    // plane z-1 is done for this warp: release its slot to the producer
    __syncwarp();
    if (tx == 0) mbar_arrive(empty0 + 8 * s_m);
    s_m = s_0;
    s_0 = s_w;
    if (++s_w == K::NSLOT) { s_w = 0; ph_w ^= 1; }
  };

  for (int z = z0; z < z1 && ok; z += 3) {
    step(I<0>{}, z);
    if (z + 1 >= z1 || !ok) break;
    step(I<1>{}, z + 1);
    if (z + 2 >= z1 || !ok) break;
    step(I<2>{}, z + 2);
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
  const int zchunk = pick_zchunk32(op.nz, (long long)bx * by, nrb, g_num_sms * K::MINB, K::D + 2);
  const long long gz = (long long)((op.nz + zchunk - 1) / zchunk) * nrb;
  if (gz > 65535) return cudaErrorInvalidConfiguration;
  kern<<<dim3(bx, by, (unsigned)gz), K::THR, K::SMEM, s>>>(op, (const float2*)x, (const float2*)b,
                                                          (float2*)y, nrhs, rstride, zchunk,
                                                          (float)omega_j);
  count_launch(1);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_mode(const OpDesc<float>& op, int cfg, const void* x, const void* b, void* y,
                        int nrhs, long long rstride, double omega_j, cudaStream_t s) {
  switch (cfg) {
    case 0: return launch_cfg<MODE, 2, 1>(op, x, b, y, nrhs, rstride, omega_j, s);
    case 1: return launch_cfg<MODE, 1, 2>(op, x, b, y, nrhs, rstride, omega_j, s);
    case 2: return launch_cfg<MODE, 2, 2>(op, x, b, y, nrhs, rstride, omega_j, s);
    case 3: return launch_cfg<MODE, 1, 4>(op, x, b, y, nrhs, rstride, omega_j, s);
    case 4: return launch_cfg<MODE, 1, 1>(op, x, b, y, nrhs, rstride, omega_j, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// Kernel configurations (rows per thread YB, RHS per CTA RB):
//   0: (2,1)  1: (1,2)  2: (2,2)  3: (1,4)  4: (1,1)
int st32_num_configs() { return 5; }

int st32_take_timeout() {
  int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_st32_timeout, sizeof(int)) != cudaSuccess) return 0;
  if (v) cudaMemcpyToSymbol(g_st32_timeout, &zero, sizeof(int));
  return v;
}

int st32_default_config(int nrhs) { return nrhs == 1 ? 0 : (nrhs == 2 ? 2 : 3); }

cudaError_t launch_stencil32(const OpDesc<float>& op, int mode, int cfg, const void* x, const void* b,
                             void* y, int nrhs, long long rstride, double omega_j, cudaStream_t s) {
  switch (mode) {
    case kApply: return launch_mode<kApply>(op, cfg, x, b, y, nrhs, rstride, omega_j, s);
    case kResidual: return launch_mode<kResidual>(op, cfg, x, b, y, nrhs, rstride, omega_j, s);
    case kJacobi: return launch_mode<kJacobi>(op, cfg, x, b, y, nrhs, rstride, omega_j, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hx
