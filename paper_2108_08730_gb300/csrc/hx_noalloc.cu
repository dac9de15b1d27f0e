// hx_assemble_csr_noalloc: hx_assemble_csr without any device allocation.
//
// Who needs it: code that may not call cudaMalloc/cudaFree at the point where
// it wants the matrix -- for example a caller whose device memory is entirely
// owned by another allocator (a framework's caching pool that has reserved the
// GPU), a caller that must not trigger the implicit device-wide
// synchronisation cudaFree performs, or a caller running under a memory
// budget that forbids new allocations after start-up.  hx_assemble_csr needs
// a temporary device buffer for the 27 coefficients of every row; this variant
// uses a fixed array compiled into the library instead.
//
// The scratch lives in file-scope __device__ arrays, so every GPU that loads
// the library holds them (about 8.7 MB) until the process exits.  Host code
// cannot pass the arrays' names to a kernel (in host code they only stand in
// for the symbols), so the first call on each device looks up their device
// addresses with cudaGetSymbolAddress while that device is current, and
// later calls reuse them (which assumes the device's primary context is not
// torn down and recreated, e.g. by cudaDeviceReset, while the process runs).
//
// All calls share the device arrays and one host staging copy of them.  Two
// calls whose work overlapped -- on the same GPU or on different GPUs, from
// any host threads or streams -- would overwrite each other's scratch and
// return each other's coefficients, so every call holds one process-wide
// lock from the first upload to the last read of the staging copy (the call
// synchronises its stream before it lets go).  Calls are therefore
// serialised; the lock does not cover other processes, which load their own
// copy of the library and its arrays.
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>

#include "hx_context.h"
#include "hx_internal.h"

namespace hx {
namespace {

constexpr long long kNoAllocMaxPoints = HX_NOALLOC_MAX_POINTS;   // 27^3 grid points
constexpr int kNoAllocMaxAxis = HX_NOALLOC_MAX_POINTS / 9;        // nodes per axis

// Device scratch: every row's 27 complex coefficients, and the per-axis PML
// coefficients (up.re, up.im, dn.re, dn.im) of the three axes.
static __device__ __align__(256) double2 g_row_coef[kNoAllocMaxPoints * 27];
static __device__ __align__(256) double g_axis_coef[3][kNoAllocMaxAxis * 4];

// Host staging of the same sizes (file scope, never freed).
static double2 h_row_coef[kNoAllocMaxPoints * 27];
static double h_axis_coef[3][kNoAllocMaxAxis * 4];

constexpr int kMaxDevices = 64;
struct DeviceScratch {
  bool ready = false;
  double2* row = nullptr;
  double* axis = nullptr;
};
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

// Device addresses of the scratch arrays on `device` (which must be current).
// The caller holds g_scratch_mu.
int scratch_for(hx_ctx* ctx, int device, DeviceScratch* out) {
  if (device < 0 || device >= kMaxDevices) return fail(ctx, HX_ERR_ARG, "device index out of range");
  DeviceScratch& s = g_scratch[device];
  if (!s.ready) {
    void* a = nullptr;
    void* b = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&a, g_row_coef);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(row scratch)");
    e = cudaGetSymbolAddress(&b, g_axis_coef);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(axis scratch)");
    s.row = (double2*)a;
    s.axis = (double*)b;
    s.ready = true;
  }
  *out = s;
  return HX_OK;
}

}  // namespace
}  // namespace hx

using namespace hx;

extern "C" int hx_assemble_csr_noalloc(hx_ctx* ctx, const hx_grid* grid, const float* v_dev,
                                       double shift_beta, int64_t* rowptr, int32_t* col, double* val,
                                       int64_t nnz_cap, int64_t* nnz_out, void* stream) {
  if (!ctx) return HX_ERR_ARG;
  int st = check_grid(ctx, grid);
  if (st) return st;
  if (!ctx->tab64) return fail(ctx, HX_ERR_STATE, "no weight table set (hx_set_table)");
  if (!v_dev || !rowptr || !col || !val || !nnz_out) return fail(ctx, HX_ERR_ARG, "null buffer");
  if (!std::isfinite(shift_beta)) return fail(ctx, HX_ERR_ARG, "shift_beta must be finite");
  const int n[3] = {grid->nx, grid->ny, grid->nz};
  const long long N = (long long)n[0] * n[1] * n[2];
  if (N > kNoAllocMaxPoints)
    return fail(ctx, HX_ERR_ARG,
                "hx_assemble_csr_noalloc: grid has more than HX_NOALLOC_MAX_POINTS (19683) points; "
                "use hx_assemble_csr");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  // held until the CSR is filled from the host staging copy (see the top of
  // this file): no other call may touch the scratch or the staging meanwhile
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  cudaStream_t s = (cudaStream_t)stream;
  // on every exit, error paths included, the work this call enqueued has
  // finished before the lock is released (destroyed before `lock`)
  struct Drain {
    cudaStream_t s;
    ~Drain() { cudaStreamSynchronize(s); }
  } drain{s};
  DeviceScratch sc;
  if ((st = scratch_for(ctx, ctx->device, &sc))) return st;

  // per-axis PML coefficients 1/(xi(i) xi(i +- 1/2) h^2), same reading as the
  // operator (gamma0 (d/L)^2 damping, xi = 1 + i gamma/omega)
  const double omega = 2.0 * M_PI * grid->f;
  const double ih2 = 1.0 / (grid->h * grid->h);
  OpDesc<double> d;
  d.nx = n[0];
  d.ny = n[1];
  d.nz = n[2];
  d.v = v_dev;
  d.tab = ctx->tab64;
  d.n_g = ctx->n_g;
  d.u_scale = grid->f * grid->h / ctx->d_inv_g;
  d.omega2 = omega * omega;
  d.beta = shift_beta;
  d.inv_h2 = ih2;
  d.gam = ctx->op_weights == HX_WEIGHTS_GAM;
  d.mass1 = ctx->op_mass_form == 1;
  d.buoy = ctx->med_buoy;
  d.invq = ctx->med_invq;
  for (int a = 0; a < 3; ++a) {
    const Profile1D prof = Profile1D::from_grid(n[a], grid->h, grid->npml[2 * a], grid->npml[2 * a + 1],
                                                grid->v_ref, grid->r_coef);
    for (int i = 0; i < n[a]; ++i) {
      auto xi = [&](double x) { return std::complex<double>(1.0, prof.gamma(x) / omega); };
      const std::complex<double> xn = xi(i * grid->h), xp = xi((i + 0.5) * grid->h),
                                 xm = xi((i - 0.5) * grid->h);
      const std::complex<double> up = 1.0 / (xn * xp) * ih2, dn = 1.0 / (xn * xm) * ih2;
      h_axis_coef[a][4 * i + 0] = up.real();
      h_axis_coef[a][4 * i + 1] = up.imag();
      h_axis_coef[a][4 * i + 2] = dn.real();
      h_axis_coef[a][4 * i + 3] = dn.imag();
    }
    e = cudaMemcpyAsync(sc.axis + (size_t)a * kNoAllocMaxAxis * 4, h_axis_coef[a],
                        4 * sizeof(double) * n[a], cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "axis coefficient upload");
    d.axis[a] = sc.axis + (size_t)a * kNoAllocMaxAxis * 4;
    d.plain_lo[a] = 1;   // not used by the coefficient kernel
    d.plain_hi[a] = 0;
  }
  // every one of the N*27 scratch entries read below is written by the kernel
  // (zeros for neighbours outside the grid), so nothing needs clearing
  e = launch_row_coefficients(d, (double*)sc.row, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_row_coef, sc.row, (size_t)N * 27 * sizeof(double2), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "coefficients");

  int64_t nnz = 0;
  rowptr[0] = 0;
  for (long long i = 0; i < N; ++i) {
    const int ix = (int)(i % n[0]), iy = (int)((i / n[0]) % n[1]), iz = (int)(i / ((long long)n[0] * n[1]));
    int k = 0;
    for (int dk = -1; dk <= 1; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di, ++k) {
          if (ix + di < 0 || ix + di >= n[0] || iy + dj < 0 || iy + dj >= n[1] || iz + dk < 0 ||
              iz + dk >= n[2])
            continue;
          if (nnz >= nnz_cap) return fail(ctx, HX_ERR_ARG, "nnz_cap too small");
          col[nnz] = (int32_t)(i + di + (long long)n[0] * (dj + (long long)n[1] * dk));
          val[2 * nnz] = h_row_coef[i * 27 + k].x;
          val[2 * nnz + 1] = h_row_coef[i * 27 + k].y;
          ++nnz;
        }
    rowptr[i + 1] = nnz;
  }
  *nnz_out = nnz;
  return HX_OK;
}
