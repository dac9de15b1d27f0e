// hx_measure_fp64_peak: the FP64 fused multiply-add throughput of this GPU.
//
// The complex128 kernels of the plain FP64 solve (and the FP64 residual of
// the mixed form) run on the FP64 units, whose rate on GB300 is a small
// fraction of the FP32 rate; their roofline is this measured number, not the
// HBM bandwidth.  Each thread runs kChains independent FMA recurrences
// a <- a m + c (|m| < 1, so the values stay bounded), enough warps per SM to
// keep the FP64 pipes busy, and the launch is timed with CUDA events after a
// warm-up launch.  2 flops per FMA.
#include <algorithm>

#include "hx_context.h"
#include "hx_internal.h"

namespace hx {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fp64_fma_k(double* __restrict__ sink, int iters, double m, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0) sink[blockIdx.x] = s;   // never true; keeps the chains live
}

}  // namespace
}  // namespace hx

using namespace hx;

extern "C" int hx_measure_fp64_peak(hx_ctx* ctx, double* gflops, void* stream) {
  if (!ctx || !gflops) return ctx ? fail(ctx, HX_ERR_ARG, "null gflops") : HX_ERR_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device)) != cudaSuccess)
    return cuda_fail(ctx, e, "SM count");
  const int blocks = sms * 8;
  const int iters = 4096;
  double* sink = nullptr;
  if ((e = cudaMalloc(&sink, blocks * sizeof(double))) != cudaSuccess) return cuda_fail(ctx, e, "sink");
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  double best_ms = 1e300;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up
    e = cudaEventRecord(a, s);
    fp64_fma_k<<<blocks, kThreads, 0, s>>>(sink, iters, 0.999999, 1e-6);
    count_launch(1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && rep > 0) best_ms = std::min(best_ms, (double)ms);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "FP64 peak kernel");
  const double fmas = (double)blocks * kThreads * kChains * iters;
  *gflops = 2.0 * fmas / (best_ms * 1e-3) / 1e9;
  return HX_OK;
}
