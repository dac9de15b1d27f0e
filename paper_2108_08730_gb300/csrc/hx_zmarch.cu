// Host side of the TMA z-marching complex64 operator kernel (device code in
// hx_zmarch_kernel.cuh, one translation unit per mode) and the first damped
// Jacobi sweep y = omega D^-1 b in the same pitched layout.
//
// The tensor maps are encoded per launch with cuTensorMapEncodeTiled, reached
// through the runtime's driver entry point (the library does not link
// libcuda): a 4-D view (x, y, z, rhs) of the field with 8-byte elements, row
// stride pitch * 8 bytes (pitch even: the 16-byte stride rule), zero fill
// outside the grid.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "hx_complex.cuh"
#include "hx_launch.cuh"
#include "hx_zmarch.cuh"
#include "hx_zmarch_kernel.cuh"

namespace hx {

// per-mode launchers (hx_zmarch_apply.cu, hx_zmarch_residual.cu, hx_zmarch_jacobi.cu)
cudaError_t zm_launch_apply(int cfg, const ZParams& P, bool shift, const CUtensorMap& xm, const CUtensorMap& bm,
                            int frame, int interior, cudaStream_t s);
cudaError_t zm_launch_residual(int cfg, const ZParams& P, bool shift, const CUtensorMap& xm,
                               const CUtensorMap& bm, int frame, int interior, cudaStream_t s);
cudaError_t zm_launch_jacobi(int cfg, const ZParams& P, bool shift, const CUtensorMap& xm, const CUtensorMap& bm,
                             int frame, int interior, cudaStream_t s);

namespace {

constexpr ZCfgInfo kZCfg[] = {{8, 1}, {8, 2}, {8, 4}, {8, 8}, {16, 2}, {16, 4}};
constexpr int kNZCfg = sizeof(kZCfg) / sizeof(kZCfg[0]);

template <int TY, int RB>
constexpr int smem_of(bool hasb) {
  return hasb ? ZK<TY, RB, true>::SMEM : ZK<TY, RB, false>::SMEM;
}
int cfg_smem(int cfg, bool hasb) {
  switch (cfg) {
    case 0: return smem_of<8, 1>(hasb);
    case 1: return smem_of<8, 2>(hasb);
    case 2: return smem_of<8, 4>(hasb);
    case 3: return smem_of<8, 8>(hasb);
    case 4: return smem_of<16, 2>(hasb);
    case 5: return smem_of<16, 4>(hasb);
  }
  return 0;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool encode_field(CUtensorMap* m, const void* base, const OpDesc<float>& op, int nrhs, long long pitch, int bw,
                  int bh, int rb) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t gdim[4] = {(cuuint64_t)op.nx, (cuuint64_t)op.ny, (cuuint64_t)op.nz, (cuuint64_t)nrhs};
  const cuuint64_t gstr[3] = {(cuuint64_t)pitch * 8, (cuuint64_t)pitch * op.ny * 8,
                              (cuuint64_t)pitch * op.ny * op.nz * 8};
  const cuuint32_t box[4] = {(cuuint32_t)bw, (cuuint32_t)bh, 1u, (cuuint32_t)rb};
  const cuuint32_t es[4] = {1u, 1u, 1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, const_cast<void*>(base), gdim, gstr, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  static int n = 0;
  if (n <= 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  }
  return n;
}

// First damped-Jacobi sweep from x = 0 in the pitched layout: y = omega D^-1 b,
// D the row's diagonal (general form: m (1 + i beta) wm1 - t0 sum_d (up_d + dn_d)).
__global__ void zm_jacobi0_k(const OpDesc<float> op, const float2* __restrict__ b, float2* __restrict__ y,
                             int nrhs, long long pitch, float omega_j) {
  pdl_enter();
  const long long N = (long long)op.nx * op.ny * op.nz;
  const long long plane = pitch * op.ny, rstride = plane * op.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % op.nx);
    const int iy = (int)((i / op.nx) % op.ny);
    const int iz = (int)(i / ((long long)op.nx * op.ny));
    const float iv = __frcp_rn(__ldg(op.v + i));
    const float u = fminf(fmaxf(op.u_scale * iv, 0.f), (float)(op.n_g - 1));
    const int i0 = min((int)u, op.n_g - 2);
    const float tf = u - (float)i0;
    const float m = op.omega2 * iv * iv;
    const float* tq = op.tab + i0 * kTabW;
    const float w1 = fmaf(tf, __ldg(tq + kTabW + 4) - __ldg(tq + 4), __ldg(tq + 4));
    const float t0 = fmaf(tf, __ldg(tq + kTabW + 8) - __ldg(tq + 8), __ldg(tq + 8));
    float sr = 0.f, si = 0.f;
    const int id[3] = {ix, iy, iz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(op.axis[d] + 4 * (size_t)id[d]));
      sr += a.x + a.z;
      si += a.y + a.w;
    }
    const float dr = fmaf(m, w1, -t0 * sr), di = fmaf(op.beta * m, w1, -t0 * si);
    const float q = omega_j * __frcp_rn(fmaf(dr, dr, di * di));
    const float fr = dr * q, fi = -di * q;
    const long long o = (long long)iz * plane + (long long)iy * pitch + ix;
    for (int r = 0; r < nrhs; ++r) {
      const float2 bb = b[r * rstride + o];
      y[r * rstride + o] = make_float2(fmaf(fr, bb.x, -fi * bb.y), fmaf(fr, bb.y, fi * bb.x));
    }
  }
}

}  // namespace

// bounded-wait error flag, one per device (its address looked up once per
// device with that device current)
static __device__ int g_zm_err;
namespace {
int* g_zm_err_addr[64] = {};
std::mutex g_zm_err_mu;
}  // namespace

int* zm_error_flag(int device) {
  if (device < 0 || device >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_zm_err_mu);
  if (!g_zm_err_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_zm_err) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_zm_err_addr[device] = (int*)p;
  }
  return g_zm_err_addr[device];
}

int zm_take_error(int device) {
  int* p = zm_error_flag(device);
  if (!p) return 0;
  int v = 0;
  if (cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
  if (v) {
    const int z = 0;
    cudaMemcpy(p, &z, sizeof(int), cudaMemcpyHostToDevice);
  }
  return v;
}

int cfg32_count() { return kZmCfgBase + kNZCfg; }

int zm_num_configs() { return kNZCfg; }
ZCfgInfo zm_config(int cfg) { return cfg >= 0 && cfg < kNZCfg ? kZCfg[cfg] : ZCfgInfo{0, 0}; }
int zm_default_config(int nrhs, int mode) {
  if (nrhs <= 1) return 0;
  if (nrhs == 2) return 1;
  if (nrhs <= 4) return 2;
  return mode == kApply ? 3 : 2;
}

cudaError_t launch_zmarch(const OpDesc<float>& op, int mode, int cfg, const void* x, const void* b, void* y,
                          int nrhs, long long pitch, double omega_j, int* err, cudaStream_t s) {
  if (nrhs < 1 || pitch < op.nx || (pitch & 1)) return cudaErrorInvalidValue;
  if (mode == kJacobi0) {
    const long long N = (long long)op.nx * op.ny * op.nz;
    const long long blocks = std::min<long long>((N + 255) / 256, (long long)num_sms() * 16);
    (void)launch_k(zm_jacobi0_k, dim3((unsigned)blocks), dim3(256), 0, s, op, (const float2*)b, (float2*)y, nrhs,
                   pitch, (float)omega_j);
    count_launch(1);
    return cudaGetLastError();
  }
  if (((uintptr_t)x & 15) || (b && ((uintptr_t)b & 15))) return cudaErrorInvalidValue;
  if (cfg < 0 || cfg >= kNZCfg) cfg = zm_default_config(nrhs, mode);
  const ZCfgInfo C = kZCfg[cfg];
  ZParams P{};
  P.op = op;
  P.x = (const float2*)x;
  P.b = (const float2*)b;
  P.y = (float2*)y;
  P.pitch = pitch;
  P.plane = pitch * op.ny;
  P.rstride = P.plane * op.nz;
  P.nrhs = nrhs;
  P.omega_j = (float)omega_j;
  P.err = err;
  int xlo = op.plain_lo[0], xhi = op.plain_hi[0], ylo = op.plain_lo[1], yhi = op.plain_hi[1];
  if (xlo > xhi) xlo = op.nx, xhi = op.nx - 1;   // no unstretched column: all frame
  if (ylo > yhi) ylo = op.ny, yhi = op.ny - 1;
  P.xlo = xlo;
  P.xhi = xhi;
  P.ylo = ylo;
  P.yhi = yhi;
  P.xs = xlo & ~1;
  P.ys = ylo;
  const bool interior = xlo <= xhi && ylo <= yhi;
  P.ntx = interior ? (xhi + 1 - P.xs + 31) / 32 : 0;
  P.nty = interior ? (yhi + 1 - ylo + C.ty - 1) / C.ty : 0;
  P.fcols = (long long)op.nx * op.ny - (interior ? (long long)(xhi - xlo + 1) * (yhi - ylo + 1) : 0);
  P.nrb = (nrhs + C.rb - 1) / C.rb;
  const int threads = 32 * C.ty;
  P.nfc = (int)((P.fcols + kZFrameThreads - 1) / kZFrameThreads);
  // z-range per CTA: minimise waves x (planes per CTA + halo planes + the
  // planes in flight at the start), waves against the resident-CTA slots
  const bool hasb = mode != kApply;
  const int smem = cfg_smem(cfg, hasb);
  // resident CTAs per SM: shared memory, and registers (128 per thread at most
  // two 256-thread CTAs; the 512-thread configurations run one)
  const int per_sm = std::max(1, std::min((228 * 1024) / (smem + 1024), C.ty <= 8 ? 2 : 1));
  const long long slots = (long long)num_sms() * per_sm;
  const long long cols = (long long)P.ntx * P.nty;
  int best = op.nz;
  double best_cost = 1e300;
  for (int zc = op.nz; zc >= 4; --zc) {
    const long long nzc = (op.nz + zc - 1) / zc;
    if ((op.nz + nzc - 1) / nzc != zc) continue;
    const long long ctas = cols * P.nrb * nzc;
    if (ctas > (1LL << 30)) break;
    const long long waves = (ctas + slots - 1) / slots;
    const double cost = (double)waves * (zc + 8);
    if (cost < best_cost * 0.999) {
      best_cost = cost;
      best = zc;
    }
  }
  P.zchunk = best;
  P.nzc = (op.nz + best - 1) / best;
  // frame kernel: one thread per (column, z-range, RHS) marching up its
  // column; z-range length by the same waves x (planes + halo) cost against
  // its resident CTAs (three 128-thread CTAs per SM: registers)
  {
    const long long fslots = (long long)num_sms() * 3;
    const long long per_z = (long long)P.nfc * nrhs;
    int fbest = op.nz;
    double fcost = 1e300;
    for (int fz = op.nz; fz >= 1 && per_z > 0; --fz) {
      const long long nzc = (op.nz + fz - 1) / fz;
      if ((op.nz + nzc - 1) / nzc != fz) continue;
      const long long ctas = per_z * nzc;
      if (ctas > (1LL << 30)) break;
      const double cost = (double)((ctas + fslots - 1) / fslots) * (fz + 2);
      if (cost < fcost * 0.999) {
        fcost = cost;
        fbest = fz;
      }
    }
    P.fzchunk = fbest;
    P.fnzc = (op.nz + fbest - 1) / fbest;
  }
  const long long nframe = (long long)P.nfc * P.fnzc * nrhs;
  const long long ninter = (long long)P.ntx * P.nty * P.nzc * P.nrb;
  if (nframe + ninter <= 0) return cudaSuccess;
  if (nframe > (1LL << 31) - 1 || ninter > (1LL << 31) - 1) return cudaErrorInvalidConfiguration;
  CUtensorMap xm, bm;
  if (!encode_field(&xm, x, op, nrhs, pitch, kZXW, C.ty + 2, C.rb) ||
      !encode_field(&bm, b ? b : x, op, nrhs, pitch, 32, C.ty, C.rb))
    return cudaErrorInvalidValue;
  const bool shift = op.beta != 0.f;
  cudaError_t e = cudaErrorInvalidValue;
  switch (mode) {
    case kApply: e = zm_launch_apply(cfg, P, shift, xm, bm, (int)nframe, (int)ninter, s); break;
    case kResidual: e = zm_launch_residual(cfg, P, shift, xm, bm, (int)nframe, (int)ninter, s); break;
    case kJacobi: e = zm_launch_jacobi(cfg, P, shift, xm, bm, (int)nframe, (int)ninter, s); break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace hx
