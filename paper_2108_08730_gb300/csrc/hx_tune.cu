// Autotuner of the complex64 operator kernel: times every configuration
// (RHS per CTA, rows per CTA) of the z-marching kernel serving the layout and
// records the fastest per (grid size, nrhs) in the context; launches on that
// context then use it.  Not part of the paper's method (its solver is a
// sparse direct factorisation); it only chooses between launch shapes that
// compute the same operator.
#include <cstdio>
#include <cstring>
#include <vector>

#include "hx_context.h"
#include "hx_internal.h"
#include "hx_zmarch.cuh"

namespace hx {

int ctx_cfg32(const hx_ctx* ctx, int nx, int ny, int nz, int nrhs, bool sweep) {
  if (ctx->st32_cfg >= 0) return ctx->st32_cfg;
  auto it = ctx->tuned.find(tune_key(nx, ny, nz, nrhs) + (sweep ? "s" : ""));
  return it == ctx->tuned.end() ? -1 : it->second;
}

}  // namespace hx

using namespace hx;

namespace {
// RHS per CTA of a configuration: ids < kZmCfgBase are the cp.async kernel
// (hx_stencil32.cu), the others the TMA kernel (hx_zmarch.cu)
int cfg_rhs(int cfg) { return cfg < kZmCfgBase ? st32_config_rhs(cfg) : zm_config(cfg - kZmCfgBase).rb; }
}  // namespace

extern "C" int hx_kernel_config_info(int cfg, int* rows_per_thread, int* rhs_per_cta) {
  const int n = cfg32_count();
  if (cfg >= 0 && cfg < n) {
    if (rows_per_thread) *rows_per_thread = 1;
    if (rhs_per_cta) *rhs_per_cta = cfg_rhs(cfg);
  }
  return n;
}

extern "C" int hx_set_kernel_config(hx_ctx* ctx, int cfg) {
  if (!ctx) return HX_ERR_ARG;
  if (cfg < -1 || cfg >= cfg32_count()) return fail(ctx, HX_ERR_ARG, "unknown kernel configuration");
  ctx->st32_cfg = cfg;
  return HX_OK;
}

namespace hx {

// Times every configuration of the complex64 apply that serves the layout
// (row pitch `pitch`: even -> both kernels' configurations, odd -> the
// cp.async kernel's) on level lv with buffers x, y (nrhs fields of that
// layout, caller-owned) and records the fastest in ctx.  Configurations with
// at least twice nrhs RHS per CTA are skipped (their extra RHS are empty).
// ms_out is indexed by configuration id (1e300 for those not timed).
// Synchronises s.
int tune_cfg32(hx_ctx* ctx, const Level& lv, const float* v_dev, int nrhs, const void* x, void* y,
               long long pitch, int ncalls, cudaStream_t s, int* best_cfg, double* ms_out, int ms_cap) {
  const long long rstride = pitch * lv.n[1] * lv.n[2];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int n = cfg32_count();
  const bool tma = (pitch & 1) == 0;
  std::vector<double> ms(n, 1e300), ms_sweep(n, 1e300);
  // y = A x (the Krylov operator), and the damped-Jacobi sweep of the shifted
  // operator (the smoother; x serves as its b), timed and chosen apart
  OpDesc<float> da = make_desc<float>(ctx, lv, v_dev, 0.0), dj = make_desc<float>(ctx, lv, v_dev, 0.5);
  da.pitch = dj.pitch = pitch;
  int best = -1, best_sweep = -1;
  for (int c = 0; c < (tma ? n : kZmCfgBase) && e == cudaSuccess; ++c) {
    if (cfg_rhs(c) > 1 && cfg_rhs(c) >= 2 * nrhs) continue;
    for (int sweep = 0; sweep < 2 && e == cudaSuccess; ++sweep) {
      OpDesc<float>& d = sweep ? dj : da;
      d.cfg32 = c;
      const int mode = sweep ? kJacobi : kApply;
      const void* b = sweep ? x : nullptr;
      e = launch_stencil<float>(d, mode, x, b, y, nrhs, rstride, 0.6, s);   // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      for (int k = 0; k < ncalls && e == cudaSuccess; ++k) e = launch_stencil<float>(d, mode, x, b, y, nrhs, rstride, 0.6, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float t = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e != cudaSuccess) break;
      std::vector<double>& m = sweep ? ms_sweep : ms;
      int& bst = sweep ? best_sweep : best;
      m[c] = t / ncalls;
      if (bst < 0 || m[c] < m[bst]) bst = c;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
  if (best < 0 || best_sweep < 0) return fail(ctx, HX_ERR_STATE, "autotune: no configuration timed");
  ctx->tuned[tune_key(lv.n[0], lv.n[1], lv.n[2], nrhs) + "s"] = best_sweep;
  ctx->tuned[tune_key(lv.n[0], lv.n[1], lv.n[2], nrhs)] = best;
  if (best_cfg) *best_cfg = best;
  for (int c = 0; c < n && c < ms_cap && ms_out; ++c) ms_out[c] = ms[c];
  return HX_OK;
}

}  // namespace hx

extern "C" int hx_autotune(hx_ctx* ctx, const hx_grid* grid, const float* v_dev, int nrhs, int ncalls,
                           int* best_cfg, double* ms_out, int ms_cap, void* stream) {
  if (!ctx) return HX_ERR_ARG;
  int st = check_grid(ctx, grid);
  if (st) return st;
  if (!ctx->tab64) return fail(ctx, HX_ERR_STATE, "no weight table set (hx_set_table)");
  if (!v_dev || nrhs < 1 || ncalls < 1) return fail(ctx, HX_ERR_ARG, "need v_dev, nrhs >= 1, ncalls >= 1");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone)
    return fail(ctx, HX_ERR_STATE, "hx_autotune cannot run while the stream is being captured");
  Level* lv = nullptr;
  const int nl[3] = {grid->nx, grid->ny, grid->nz};
  if ((st = get_level(ctx, grid, nl, grid->h, &lv))) return st;
  const long long N = (long long)grid->nx * grid->ny * grid->nz;
  const size_t fb = (size_t)nrhs * N * 8;
  void *x = nullptr, *y = nullptr;
  cudaError_t e = cudaMalloc(&x, fb);
  if (e == cudaSuccess) e = cudaMalloc(&y, fb);
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, fb, s);
  if (e == cudaSuccess) st = tune_cfg32(ctx, *lv, v_dev, nrhs, x, y, grid->nx, ncalls, s, best_cfg, ms_out, ms_cap);
  if (x) cudaFree(x);
  if (y) cudaFree(y);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune buffers");
  return st;
}
