// hx_solve: batched Krylov solve of [M + S] p = s (Eq. 3) for point sources.
//
// Not the paper's solver (it factorises with a sparse direct method); the
// engineering choice here is
//   * BiCGStab, right-preconditioned, one independent recurrence per RHS with
//     all per-RHS scalars on the device;
//   * preconditioner: one V-cycle of the complex-shifted operator
//     (omega^2 -> (1 + i beta) omega^2) rediscretised with the same adaptive
//     27-point stencil on vertex-centred grids coarsened by 2, velocity
//     injected, same physical PML profile, damped-Jacobi smoothing, full
//     weighting and trilinear prolongation;
//   * mixed precision: the Krylov solve and the V-cycle in complex64, wrapped
//     by FP64 iterative refinement (FP64 residual s - A x, FP64 update of x),
//     or everything in complex128 for the plain FP64 form.
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hx_complex.cuh"
#include "hx_context.h"
#include "hx_galerkin.cuh"
#include "hx_internal.h"
#include "hx_trace.h"
#include "hx_launch.cuh"
#include "hx_vec.cuh"

namespace hx {
namespace {

constexpr int kMaxLev = 12;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t b) {
    if (p && bytes >= b) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, b);
    if (e == cudaSuccess) bytes = b;
    return e;
  }
};

struct SolverImpl : Solver {
  int prec = 32;   // inner precision
  int R = 0;
  int nlev = 0;
  int n[kMaxLev][3];
  long long N[kMaxLev];
  // fine-level Krylov / multigrid fields of the inner precision: x-row pitch
  // (complex64: nx rounded up to 4, so rows are 32-byte aligned and the TMA
  // kernel loads plane tiles; complex128: nx) and elements per field
  long long pitch0 = 0, NP = 0;
  std::string op_key;
  std::unique_ptr<Level> lvl[kMaxLev];  // preconditioner levels (capped PML)
  std::unique_ptr<Level> lvlA;          // the true fine-level operator
  DevBuf vlev[kMaxLev];                 // coarse velocities (level >= 1)
  DevBuf mb[kMaxLev], me[kMaxLev], mw[kMaxLev];
  DevBuf acoef[kMaxLev];                // Galerkin coarse operators [27][N_l] (level >= 1)
  bool galerkin = false;
  // Krylov vectors (inner precision), R * NP complex each (padding kept zero)
  DevBuf r, rhat, p, v, s, t, x, ph, sh, tmp;
  DevBuf r64;                           // FP64 residual (mixed mode)
  DevBuf sc;                            // per-RHS scalars
  DevBuf part;                          // reduction partials
  DevBuf srcs;                          // source entries
  // exact solve of the coarsest level: dense inverse of its shifted operator
  DevBuf cinv;                          // [Nc][Nc] complex (inner precision)
  bool have_cinv = false;
  std::string cinv_key;                 // operator parameters it was built for
  std::vector<float> cinv_v;            // coarsest velocity it was built for
  std::vector<double> h_rn2, h_bn2;
  std::vector<int> h_active;
  // scalar slots inside sc
  double2 *rho, *rho_new, *alpha, *omega, *beta, *rv, *ts;
  double *tt, *rn2, *bn2, *scale;
  int *active, *brk;
  unsigned* count;                      // arrival counters of the reductions
  double kappa = 0;
  BicgScalars scalars() const {
    return BicgScalars{rho, rho_new, alpha, omega, beta, rv, ts, tt, rn2, active, brk, count, kappa};
  }
  // pinned host mirrors read at convergence checks
  double* pin_rn2 = nullptr;
  int* pin_act = nullptr;
  int* pin_act_up = nullptr;
  // graph of one block of Krylov iterations (rebuilt once per hx_solve call)
  cudaGraphExec_t gexec = nullptr;
  bool graph_ready = false;
  int graph_k = 0;
  long long graph_kernels = 0;
  std::vector<hx_ctx::ProfPending> graph_prof;

  ~SolverImpl() override {
    if (gexec) cudaGraphExecDestroy(gexec);
    for (auto& e : graph_prof) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    if (pin_rn2) cudaFreeHost(pin_rn2);
    if (pin_act) cudaFreeHost(pin_act);
    if (pin_act_up) cudaFreeHost(pin_act_up);
  }
};

#define HX_CK(expr)                                          \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #expr); \
  } while (0)

// Largest coarsest level solved exactly through a dense inverse.
constexpr long long kMaxDense = 512;
// Coarse levels up to this size use the one-thread-per-row stencil kernel.
constexpr long long kDirectMaxPoints = 300000;

int plan_levels(const int n0[3], int requested, int out[kMaxLev][3]) {
  out[0][0] = n0[0];
  out[0][1] = n0[1];
  out[0][2] = n0[2];
  int L = 1;
  while (L < kMaxLev) {
    if (requested > 0 && L >= requested) break;
    int c[3];
    for (int d = 0; d < 3; ++d) c[d] = (out[L - 1][d] + 1) / 2;
    if (c[0] < 2 || c[1] < 2 || c[2] < 2) break;
    // automatic: coarsen until the coarsest grid is small enough for the
    // dense exact solve (smoothing alone cannot converge there: damped Jacobi
    // amplifies the shifted operator's propagating modes)
    if (requested <= 0 && (long long)out[L - 1][0] * out[L - 1][1] * out[L - 1][2] <= kMaxDense) break;
    for (int d = 0; d < 3; ++d) out[L][d] = c[d];
    ++L;
  }
  return L;
}

__global__ void minmax_k(const float* __restrict__ v, long long N, float* part) {
  pdl_enter();
  float lo = 3.0e38f, hi = -3.0e38f, bad = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const float a = v[i];
    if (!(a > 0.f) || !(a < 3.0e38f)) bad = 1.f;
    lo = fminf(lo, a);
    hi = fmaxf(hi, a);
  }
  __shared__ float sl[256], sh[256], sb[256];
  sl[threadIdx.x] = lo;
  sh[threadIdx.x] = hi;
  sb[threadIdx.x] = bad;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sl[threadIdx.x] = fminf(sl[threadIdx.x], sl[threadIdx.x + o]);
      sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + o]);
      sb[threadIdx.x] = fmaxf(sb[threadIdx.x], sb[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = sl[0];
    part[3 * blockIdx.x + 1] = sh[0];
    part[3 * blockIdx.x + 2] = sb[0];
  }
}

__global__ void init_scalars_k(double2* rho, double2* alpha, double2* omega, int* brk, int R) {
  pdl_enter();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  rho[r] = make_double2(1.0, 0.0);
  alpha[r] = make_double2(1.0, 0.0);
  omega[r] = make_double2(1.0, 0.0);
  brk[r] = 0;
}

class Run {
 public:
  Run(hx_ctx* c, SolverImpl* s, const hx_grid* g, const float* v0, const hx_solve_opts& o,
      cudaStream_t st)
      : ctx(c), S(s), grid(g), v_fine(v0), opt(o), stream(st), t0(std::chrono::steady_clock::now()) {}

  // opts.time_limit_s ran out or opts.cancel was set (checked where the host
  // synchronises anyway)
  bool past_deadline() const {
    return cancelled() || (opt.time_limit_s > 0 && std::chrono::duration<double>(
                                                       std::chrono::steady_clock::now() - t0)
                                                           .count() > opt.time_limit_s);
  }
  bool cancelled() const { return opt.cancel && __atomic_load_n(opt.cancel, __ATOMIC_RELAXED) != 0; }

  template <typename T>
  OpDesc<T> desc(int l, double beta) const {
    OpDesc<T> d = make_desc<T>(ctx, *S->lvl[l], l == 0 ? v_fine : (const float*)S->vlev[l].p, beta, true);
    d.cfg32 = ctx_cfg32(ctx, S->n[l][0], S->n[l][1], S->n[l][2], S->R, true);
    if (l == 0) d.pitch = S->pitch0;
    return d;
  }

  // Stencil launch on level l; fine-level launches are timed by the profiler
  // with their algorithmic bytes (streams read/written once, v once).
  template <typename T>
  cudaError_t stencil(int l, const OpDesc<T>& op, int mode, const void* x, const void* b, void* y,
                      double om) {
    const long long N = S->N[l];
    if (l > 0 && S->galerkin)
      return launch_stored_stencil<T>(S->acoef[l].p, S->n[l], mode, x, b, y, S->R, om, stream);
    if (l > 0 && N <= kDirectMaxPoints)   // coarse level: a few tiles only
      return launch_direct_stencil<T>(op, mode, x, b, y, S->R, om, stream);
    const bool timed = l == 0 && mode != kJacobi0;
    cudaEvent_t a = timed ? prof_begin(ctx, stream) : nullptr;
    cudaError_t e = launch_stencil(op, mode, x, b, y, S->R, l == 0 ? S->NP : N, om, stream);
    if (timed) {
      const int kind = mode == kApply ? (sizeof(T) == 4 ? HX_PROF_APPLY32 : HX_PROF_APPLY64)
                                      : (sizeof(T) == 4 ? HX_PROF_SMOOTH32 : HX_PROF_SMOOTH64);
      const int streams = (mode == kApply || (mode == kResidual && !b)) ? 2 : 3;
      prof_end(ctx, kind, a, (double)streams * 2 * sizeof(T) * N * S->R + 4.0 * N, stream);
    }
    return e;
  }

  // One V-cycle on level l for rhs b; the result is left in e (w is the
  // level's second work buffer).  The Jacobi sweeps ping-pong between e and
  // w; the starting buffer is chosen by the parity of the sweep count so that
  // the last sweep writes e, which keeps every launch's pointers fixed from
  // one Krylov iteration to the next (a requirement of graph replay).
  template <typename T>
  int vcycle(int l, const void* b, void* e, void* w) {
    const OpDesc<T> op = desc<T>(l, opt.shift_beta);
    const long long N = S->N[l];
    const int R = S->R;
    const bool coarsest = l == S->nlev - 1;
    if (coarsest && S->have_cinv) {
      HX_CK(launch_dense_matvec<T>(S->cinv.p, b, e, N, R, stream));
      return HX_OK;
    }
    const int nu1 = l > 0 && opt.nu_coarse > 0 ? opt.nu_coarse : opt.nu_pre;
    const int nu2 = l > 0 && opt.nu_coarse > 0 ? opt.nu_coarse : opt.nu_post;
    const int pre = coarsest ? opt.coarse_sweeps : nu1;
    const int swaps = (pre - 1) + (coarsest ? 0 : nu2);
    void* cur = swaps % 2 == 0 ? e : w;
    void* oth = swaps % 2 == 0 ? w : e;
    HX_CK(stencil<T>(l, op, kJacobi0, nullptr, b, cur, opt.omega_jacobi));
    for (int k = 1; k < pre; ++k) {
      HX_CK(stencil<T>(l, op, kJacobi, cur, b, oth, opt.omega_jacobi));
      std::swap(cur, oth);
    }
    if (!coarsest) {
      HX_CK(stencil<T>(l, op, kResidual, cur, b, oth, 0.0));
      HX_CK(launch_restrict<T>(oth, S->n[l], S->mb[l + 1].p, S->n[l + 1], R, stream, l == 0 ? S->pitch0 : 0));
      int st = vcycle<T>(l + 1, S->mb[l + 1].p, S->me[l + 1].p, S->mw[l + 1].p);
      if (st) return st;
      HX_CK(launch_prolong_add<T>(cur, S->n[l], S->me[l + 1].p, S->n[l + 1], R, stream, l == 0 ? S->pitch0 : 0));
      for (int k = 0; k < nu2; ++k) {
        HX_CK(stencil<T>(l, op, kJacobi, cur, b, oth, opt.omega_jacobi));
        std::swap(cur, oth);
      }
    }
    return cur == e ? HX_OK : fail(ctx, HX_ERR_STATE, "V-cycle buffer parity");
  }

  // One BiCGStab iteration (all RHS), launches only.  On entry rho_new and
  // beta of this iteration are already on the device (the previous
  // iteration's last kernel, or the reduction before the first iteration).
  template <typename T>
  int bicg_iteration(const OpDesc<T>& A) {
    const int R = S->R;
    const long long N = S->NP;
    double2* part = (double2*)S->part.p;
    const BicgScalars sc = S->scalars();
    HX_CK(launch_bicg_p<T>(S->p.p, S->r.p, S->v.p, S->beta, S->omega, N, R, stream));
    int st = vcycle<T>(0, S->p.p, S->ph.p, S->tmp.p);
    if (st) return st;
    HX_CK(stencil<T>(0, A, kApply, S->ph.p, nullptr, S->v.p, 0.0));
    HX_CK(launch_bicg_reduce<T>(kRedAlpha, S->rhat.p, S->v.p, N, R, part, sc, stream));
    HX_CK(launch_bicg_s<T>(S->s.p, S->r.p, S->v.p, S->alpha, N, R, stream));
    st = vcycle<T>(0, S->s.p, S->sh.p, S->tmp.p);
    if (st) return st;
    HX_CK(stencil<T>(0, A, kApply, S->sh.p, nullptr, S->t.p, 0.0));
    HX_CK(launch_bicg_reduce<T>(kRedOmega, S->t.p, S->s.p, N, R, part, sc, stream));
    HX_CK(launch_bicg_xr_reduce<T>(S->x.p, S->r.p, S->s.p, S->ph.p, S->sh.p, S->t.p, S->rhat.p, N, R, part, sc,
                                   stream));
    return HX_OK;
  }

  // k iterations followed by the residual norms (left by the last iteration)
  // and active flags copied to pinned host memory: the unit replayed between
  // host convergence checks.
  template <typename T>
  int bicg_block(const OpDesc<T>& A, int k) {
    for (int j = 0; j < k; ++j) {
      int st = bicg_iteration<T>(A);
      if (st) return st;
    }
    const int R = S->R;
    HX_CK(cudaMemcpyAsync(S->pin_rn2, S->rn2, R * sizeof(double), cudaMemcpyDeviceToHost, stream));
    HX_CK(cudaMemcpyAsync(S->pin_act, S->active, R * sizeof(int), cudaMemcpyDeviceToHost, stream));
    return HX_OK;
  }

  // Capture bicg_block as a CUDA graph (instantiated once per hx_solve call,
  // updated in place when the topology is unchanged).  Returns false when
  // capture is unavailable; the caller then launches directly.
  template <typename T>
  bool capture_block(const OpDesc<T>& A, int k) {
    if (S->graph_ready && S->graph_k == k) return true;
    if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    const size_t p0 = ctx->prof_pending.size();
    const long long c0 = launch_count();
    const int st = bicg_block<T>(A, k);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(stream, &g);
    // kernels captured, not run: count them per replay instead
    S->graph_kernels = launch_count() - c0;
    count_launch(-(int)S->graph_kernels);
    // event pairs recorded inside the graph belong to it, not to the pending list
    for (auto& e : S->graph_prof) {
      ctx->prof_pool.push_back(e.a);
      ctx->prof_pool.push_back(e.b);
    }
    S->graph_prof.assign(ctx->prof_pending.begin() + p0, ctx->prof_pending.end());
    ctx->prof_pending.resize(p0);
    if (st || ec != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return false;
    }
    bool ok = false;
    if (S->gexec) {
      cudaGraphExecUpdateResultInfo info;
      ok = cudaGraphExecUpdate(S->gexec, g, &info) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        cudaGraphExecDestroy(S->gexec);
        S->gexec = nullptr;
      }
    }
    if (!ok) ok = cudaGraphInstantiate(&S->gexec, g, 0) == cudaSuccess;
    cudaGraphDestroy(g);
    if (!ok) {
      cudaGetLastError();
      S->gexec = nullptr;
      return false;
    }
    S->graph_ready = true;
    S->graph_k = k;
    return true;
  }

  void collect_graph_prof() {
    if (!ctx->prof_on) return;
    for (auto& p : S->graph_prof) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        ctx->prof[p.kind].launches += 1;
        ctx->prof[p.kind].ms += ms;
        ctx->prof[p.kind].bytes += p.bytes;
      }
    }
  }

  // Right-preconditioned BiCGStab on A x = b with x0 = 0.  The RHS b is in
  // S->r on entry (it becomes the residual); the solution is left in S->x.
  // Per-RHS tolerance `tol` relative to ||b||; active_in: host flags.
  template <typename T>
  int bicgstab(double tol, int max_iter, const std::vector<int>& active_in, int* iters) {
    const int R = S->R;
    const long long N = S->NP;
    const size_t fb = (size_t)R * N * 2 * sizeof(T);
    OpDesc<T> A = make_desc<T>(ctx, *S->lvlA, v_fine, 0.0);   // the true operator
    A.cfg32 = ctx_cfg32(ctx, S->n[0][0], S->n[0][1], S->n[0][2], R);
    A.pitch = S->pitch0;
    void* r = S->r.p;
    void* rhat = S->rhat.p;
    void* p = S->p.p;
    void* v = S->v.p;
    void* sv = S->s.p;
    void* t = S->t.p;
    void* x = S->x.p;
    void* ph = S->ph.p;
    void* sh = S->sh.p;
    void* tmp = S->tmp.p;
    HX_CK(launch_norm2<T>(r, N, R, (double2*)S->part.p, S->bn2, stream));
    HX_CK(cudaMemcpyAsync(rhat, r, fb, cudaMemcpyDeviceToDevice, stream));
    HX_CK(cudaMemsetAsync(x, 0, fb, stream));
    HX_CK(cudaMemsetAsync(p, 0, fb, stream));
    HX_CK(cudaMemsetAsync(v, 0, fb, stream));
    (void)launch_k(init_scalars_k, (R + 127) / 128, 128, 0, stream, S->rho, S->alpha, S->omega, S->brk, R);
    count_launch(1);
    HX_CK(cudaGetLastError());
    S->h_active = active_in;
    HX_CK(cudaMemcpyAsync(S->h_bn2.data(), S->bn2, R * sizeof(double), cudaMemcpyDeviceToHost, stream));
    HX_CK(cudaStreamSynchronize(stream));
    for (int k = 0; k < R; ++k)
      if (!(S->h_bn2[k] > 0)) S->h_active[k] = 0;
    HX_CK(cudaMemcpyAsync(S->active, S->h_active.data(), R * sizeof(int), cudaMemcpyHostToDevice, stream));
    // rho_new = (rhat, r) and the first beta step (p = r whatever beta is, since p = v = 0)
    HX_CK(launch_bicg_reduce<T>(kRedBeta, rhat, r, N, R, (double2*)S->part.p, S->scalars(), stream));
    (void)p; (void)v; (void)sv; (void)t; (void)ph; (void)sh; (void)tmp;
    int it = 0;
    bool any = false;
    for (int k = 0; k < R; ++k) any = any || S->h_active[k];
    const int kblk = opt.check_every;
    // graph replay is skipped while the profiler times individual launches
    const bool graphed = opt.use_graphs && !ctx->prof_on && capture_block<T>(A, kblk);
    while (any && it < max_iter && !past_deadline()) {
      if (graphed) {
        HX_CK(cudaGraphLaunch(S->gexec, stream));
        count_launch(S->graph_kernels);
      } else {
        int st = bicg_block<T>(A, kblk);
        if (st) return st;
      }
      it += kblk;
      HX_CK(cudaStreamSynchronize(stream));
      if (graphed) collect_graph_prof();
      any = false;
      for (int k = 0; k < R; ++k) {
        const double rn2 = S->pin_rn2[k];
        if (!std::isfinite(rn2)) return fail(ctx, HX_ERR_NUMERIC, "non-finite Krylov residual");
        if (S->h_active[k] && (!S->pin_act[k] || rn2 <= tol * tol * S->h_bn2[k])) S->h_active[k] = 0;
        any = any || S->h_active[k];
      }
      for (int k = 0; k < R; ++k) S->pin_act_up[k] = S->h_active[k];
      HX_CK(cudaMemcpyAsync(S->active, S->pin_act_up, R * sizeof(int), cudaMemcpyHostToDevice, stream));
    }
    *iters = it;
    return HX_OK;
  }

  hx_ctx* ctx;
  SolverImpl* S;
  const hx_grid* grid;
  const float* v_fine;
  hx_solve_opts opt;
  cudaStream_t stream;
  std::chrono::steady_clock::time_point t0;
};

}  // namespace
}  // namespace hx

using namespace hx;

extern "C" void hx_solve_default_opts(hx_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->mode = HX_SOLVE_MIXED;
  o->tol = 1e-10;
  o->inner_tol = 1e-4;
  o->max_outer = 12;
  o->max_iter = 2000;
  o->shift_beta = 1.0;
  o->mg_levels = 0;
  // three sweeps on either side: measured against 2 + 2 (and 4 + 4, which
  // diverged on two large models) on the workloads of this library
  o->nu_pre = 3;
  o->nu_post = 3;
  o->coarse_sweeps = 4;
  o->omega_jacobi = 0.6;
  o->source_spread = 0;
  o->initial_guess = 0;
  o->check_every = 2;
  o->coarse_galerkin = 0;
  o->pml_cap = -15.0;   // automatic: min(1, 15 omega / gamma0), see hx_solve_opts
  o->use_graphs = 1;
  o->autotune = 1;
  o->time_limit_s = 0.0;
  o->cancel = nullptr;
  o->nu_coarse = 2;
  o->bicg_kappa = 0.0;
  o->coarse_velocity = 0;
}

namespace {

int validate_velocity(hx_ctx* ctx, const hx_grid* g, const float* v, cudaStream_t s, float* vmin,
                      float* vmax) {
  const long long N = (long long)g->nx * g->ny * g->nz;
  const int nb = 304;
  float* part = nullptr;
  cudaError_t e = cudaMalloc(&part, 3 * nb * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "validation buffer");
  (void)launch_k(minmax_k, nb, 256, 0, s, v, N, part);
  count_launch(1);
  std::vector<float> h(3 * nb);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, h.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(part);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "velocity validation");
  float lo = 3e38f, hi = -3e38f, bad = 0;
  for (int i = 0; i < nb; ++i) {
    lo = std::min(lo, h[3 * i]);
    hi = std::max(hi, h[3 * i + 1]);
    bad = std::max(bad, h[3 * i + 2]);
  }
  if (bad > 0) return fail(ctx, HX_ERR_ARG, "velocity must be finite and > 0 everywhere");
  *vmin = lo;
  *vmax = hi;
  return HX_OK;
}

// Dense inverse of the coarsest level's shifted operator (FP64 Gauss-Jordan
// with partial pivoting on the host), uploaded in the inner precision.  The
// coarsest grid has at most kMaxDense nodes; the inverse is rebuilt only when
// the operator parameters or the coarsest (injected) velocity change.
int setup_coarse_inverse(hx_ctx* ctx, SolverImpl* S, const float* /*v_fine*/, double beta,
                         const std::string& okey, cudaStream_t s) {
  const int L = S->nlev - 1;
  const long long Nc = S->N[L];
  if (L == 0 || Nc > kMaxDense) {
    S->have_cinv = false;
    return HX_OK;
  }
  // h[i*54 + 2k (+1)]: coefficient k of row i of the coarsest operator, FP64
  std::vector<double> h((size_t)Nc * 54);
  cudaError_t e = cudaSuccess;
  std::vector<float> vc;
  if (S->galerkin) {
    // stored Galerkin operator [27][Nc] in the inner precision
    const size_t cs = S->prec == 64 ? 16 : 8;
    std::vector<unsigned char> raw((size_t)27 * Nc * cs);
    e = cudaMemcpyAsync(raw.data(), S->acoef[L].p, raw.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "coarsest operator");
    for (long long i = 0; i < Nc; ++i)
      for (int k = 0; k < 27; ++k) {
        const size_t q = (size_t)k * Nc + i;
        if (cs == 16) {
          h[i * 54 + 2 * k] = ((const double*)raw.data())[2 * q];
          h[i * 54 + 2 * k + 1] = ((const double*)raw.data())[2 * q + 1];
        } else {
          h[i * 54 + 2 * k] = ((const float*)raw.data())[2 * q];
          h[i * 54 + 2 * k + 1] = ((const float*)raw.data())[2 * q + 1];
        }
      }
    vc.assign((const float*)h.data(), (const float*)(h.data() + h.size()));   // cache key: the operator
  } else {
    vc.resize(Nc);
    const float* vdev = (const float*)S->vlev[L].p;
    e = cudaMemcpyAsync(vc.data(), vdev, Nc * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "coarsest velocity");
  }
  char kb[64];
  std::snprintf(kb, sizeof(kb), " b%.17g p%d g%d", beta, S->prec, S->galerkin ? 1 : 0);
  const std::string key = okey + kb;
  if (S->have_cinv && key == S->cinv_key && vc == S->cinv_v) return HX_OK;
  S->have_cinv = false;
  if (!S->galerkin) {
    double* coef = nullptr;
    e = cudaMalloc(&coef, (size_t)Nc * 54 * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "coarse coefficients");
    e = launch_row_coefficients(make_desc<double>(ctx, *S->lvl[L], (const float*)S->vlev[L].p, beta, true), coef, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), coef, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(coef);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "coarse coefficients");
  }
  typedef std::complex<double> cd;
  const int n = (int)Nc;
  const int nx = S->n[L][0], ny = S->n[L][1], nz = S->n[L][2];
  std::vector<cd> M((size_t)n * n, cd(0, 0)), I((size_t)n * n, cd(0, 0));
  for (int i = 0; i < n; ++i) {
    const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
    int k = 0;
    for (int dk = -1; dk <= 1; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di, ++k) {
          if (ix + di < 0 || ix + di >= nx || iy + dj < 0 || iy + dj >= ny || iz + dk < 0 || iz + dk >= nz)
            continue;
          const int j = i + di + nx * (dj + ny * dk);
          M[(size_t)i * n + j] = cd(h[(size_t)i * 54 + 2 * k], h[(size_t)i * 54 + 2 * k + 1]);
        }
    I[(size_t)i * n + i] = cd(1, 0);
  }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    double best = std::abs(M[(size_t)c * n + c]);
    for (int r = c + 1; r < n; ++r) {
      const double a = std::abs(M[(size_t)r * n + c]);
      if (a > best) { best = a; piv = r; }
    }
    if (!(best > 0)) return HX_OK;   // singular: fall back to smoothing on that level
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        std::swap(M[(size_t)c * n + j], M[(size_t)piv * n + j]);
        std::swap(I[(size_t)c * n + j], I[(size_t)piv * n + j]);
      }
    const cd inv = 1.0 / M[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) {
      M[(size_t)c * n + j] *= inv;
      I[(size_t)c * n + j] *= inv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const cd f = M[(size_t)r * n + c];
      if (f == cd(0, 0)) continue;
      for (int j = 0; j < n; ++j) {
        M[(size_t)r * n + j] -= f * M[(size_t)c * n + j];
        I[(size_t)r * n + j] -= f * I[(size_t)c * n + j];
      }
    }
  }
  const size_t cs = S->prec == 64 ? 16 : 8;
  e = S->cinv.alloc((size_t)n * n * cs);
  if (e == cudaSuccess) {
    if (S->prec == 64) {
      e = cudaMemcpy(S->cinv.p, I.data(), (size_t)n * n * 16, cudaMemcpyHostToDevice);
    } else {
      std::vector<float> f32((size_t)n * n * 2);
      for (size_t q = 0; q < (size_t)n * n; ++q) {
        f32[2 * q] = (float)I[q].real();
        f32[2 * q + 1] = (float)I[q].imag();
      }
      e = cudaMemcpy(S->cinv.p, f32.data(), f32.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "coarse inverse upload");
  S->have_cinv = true;
  S->cinv_key = key;
  S->cinv_v = vc;
  return HX_OK;
}

}  // namespace

extern "C" int hx_solve(hx_ctx* ctx, const hx_grid* grid, const float* v_dev, const hx_source* src,
                        int nsrc, int nrhs, void* wavefield_dev, const hx_solve_opts* opts_in,
                        hx_solve_report* report, void* stream_v) {
  if (!ctx) return HX_ERR_ARG;
  TraceRange trace_solve("hx_solve");
  TraceRange trace_setup("hx_solve setup");
  auto t_start = std::chrono::steady_clock::now();
  hx_solve_opts opt;
  if (opts_in) opt = *opts_in; else hx_solve_default_opts(&opt);
  if (report) std::memset(report, 0, sizeof(*report));
  auto finish = [&](int st) {
    if (report) report->status = st;
    return st;
  };
  int st = check_grid(ctx, grid);
  if (st) return finish(st);
  if (!ctx->tab64) return finish(fail(ctx, HX_ERR_STATE, "no weight table set (hx_set_table)"));
  if (!v_dev || !wavefield_dev || !src || nsrc < 1 || nrhs < 1 || nrhs > 65535)
    return finish(fail(ctx, HX_ERR_ARG, "need v, wavefield, sources and 1 <= nrhs <= 65535"));
  if (opt.mode != HX_SOLVE_MIXED && opt.mode != HX_SOLVE_FP64)
    return finish(fail(ctx, HX_ERR_ARG, "unknown mode"));
  if (!(opt.tol > 0) || !(opt.inner_tol > 0 && opt.inner_tol < 1) || opt.max_iter < 1 ||
      opt.max_outer < 1 || opt.nu_pre < 1 || opt.nu_post < 0 || opt.coarse_sweeps < 1 ||
      !(opt.omega_jacobi > 0 && opt.omega_jacobi < 2) || !(opt.shift_beta >= 0) ||
      opt.check_every < 1 || opt.coarse_galerkin < 0 || opt.coarse_galerkin > 1 ||
      !std::isfinite(opt.pml_cap) || opt.use_graphs < 0 || opt.use_graphs > 1 ||
      opt.autotune < 0 || opt.autotune > 1 || !(opt.time_limit_s >= 0) || opt.mg_levels < 0 || opt.nu_coarse < 0 ||
      !(opt.bicg_kappa >= 0 && opt.bicg_kappa < 1) || opt.coarse_velocity < 0 || opt.coarse_velocity > 1 ||
      opt.mg_levels > kMaxLev)
    return finish(fail(ctx, HX_ERR_ARG, "invalid solve options"));
  std::vector<int> has_src(nrhs, 0);
  for (int k = 0; k < nsrc; ++k) {
    const hx_source& q = src[k];
    if (q.ix < 0 || q.ix >= grid->nx || q.iy < 0 || q.iy >= grid->ny || q.iz < 0 || q.iz >= grid->nz ||
        q.rhs < 0 || q.rhs >= nrhs || !std::isfinite(q.amp_re) || !std::isfinite(q.amp_im))
      return finish(fail(ctx, HX_ERR_ARG, "source outside the grid, bad rhs index or amplitude"));
    has_src[q.rhs] = 1;
  }
  for (int k = 0; k < nrhs; ++k)
    if (!has_src[k]) return finish(fail(ctx, HX_ERR_ARG, "every rhs needs at least one source"));
  cudaSetDevice(ctx->device);
  // The solve runs on the context's own non-blocking stream (graph capture is
  // not possible on the legacy default stream), ordered after the caller's
  // stream on entry; the caller's stream waits for it on every exit.
  const cudaStream_t user_stream = (cudaStream_t)stream_v;
  if (!ctx->work_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->work_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->order_ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->order_ev[1], cudaEventDisableTiming);
    if (e != cudaSuccess) return finish(cuda_fail(ctx, e, "work stream"));
  }
  cudaStream_t stream = ctx->work_stream;
  cudaEventRecord(ctx->order_ev[0], user_stream);
  cudaStreamWaitEvent(stream, ctx->order_ev[0], 0);
  struct Rejoin {
    hx_ctx* c;
    cudaStream_t user, work;
    ~Rejoin() {
      cudaEventRecord(c->order_ev[1], work);
      cudaStreamWaitEvent(user, c->order_ev[1], 0);
    }
  } rejoin{ctx, user_stream, stream};
  float vmin = 0, vmax = 0;
  if ((st = validate_velocity(ctx, grid, v_dev, stream, &vmin, &vmax))) return finish(st);
  const double inv_g_max = (ctx->n_g - 1) * ctx->d_inv_g;
  if (grid->f * grid->h / vmin > inv_g_max * (1 + 1e-12))
    return finish(fail(ctx, HX_ERR_ARG, "G = v/(f h) below the table's range somewhere (grid too coarse)"));

  // ---- workspace (cached per grid size, nrhs, precision)
  const int prec = opt.mode == HX_SOLVE_FP64 ? 64 : 32;
  const int n0[3] = {grid->nx, grid->ny, grid->nz};
  int lv_n[kMaxLev][3];
  const int nlev = plan_levels(n0, opt.mg_levels, lv_n);
  char key[256];
  const bool variant = ctx->op_weights != HX_WEIGHTS_GA || ctx->op_mass_form != 2 || ctx->med_buoy || ctx->med_invq;
  std::snprintf(key, sizeof(key), "%d %d %d r%d p%d L%d v%d", grid->nx, grid->ny, grid->nz, nrhs, prec, nlev,
                variant ? 1 : 0);
  SolverImpl* S = nullptr;
  {
    auto it = ctx->solvers.find(key);
    if (it != ctx->solvers.end()) {
      S = static_cast<SolverImpl*>(it->second.get());
      ctx->solver_lru.remove(key);
      ctx->solver_lru.push_front(key);
    } else {
      while (!ctx->solvers.empty() && (int)ctx->solvers.size() >= ctx->max_solvers) {
        ctx->solvers.erase(ctx->solver_lru.back());
        ctx->solver_lru.pop_back();
      }
      auto up = std::make_unique<SolverImpl>();
      S = up.get();
      S->prec = prec;
      S->R = nrhs;
      S->nlev = nlev;
      for (int l = 0; l < nlev; ++l) {
        for (int d = 0; d < 3; ++d) S->n[l][d] = lv_n[l][d];
        S->N[l] = (long long)lv_n[l][0] * lv_n[l][1] * lv_n[l][2];
      }
      const size_t cs = prec == 64 ? 16 : 8;
      // operator variants and media run on the one-thread-per-row kernel,
      // which takes unpadded fields
      S->pitch0 = prec == 64 || variant ? grid->nx : (grid->nx + 3) / 4 * 4;
      S->NP = S->pitch0 * grid->ny * grid->nz;
      const size_t fb = (size_t)nrhs * S->NP * cs;
      cudaError_t e = cudaSuccess;
      DevBuf* vecs[] = {&S->r, &S->rhat, &S->p, &S->v, &S->s, &S->t, &S->x, &S->ph, &S->sh, &S->tmp};
      for (DevBuf* b : vecs) {
        if (e == cudaSuccess) e = b->alloc(fb);
        // the row padding is read as zeros by the vector kernels and never written
        if (e == cudaSuccess) e = cudaMemsetAsync(b->p, 0, fb, stream);
      }
      if (e == cudaSuccess) e = S->r64.alloc((size_t)nrhs * S->N[0] * 16);
      for (int l = 1; l < nlev && e == cudaSuccess; ++l) {
        const size_t lb = (size_t)nrhs * S->N[l] * cs;
        e = S->vlev[l].alloc(S->N[l] * sizeof(float));
        if (e == cudaSuccess) e = S->mb[l].alloc(lb);
        if (e == cudaSuccess) e = S->me[l].alloc(lb);
        if (e == cudaSuccess) e = S->mw[l].alloc(lb);
      }
      if (e == cudaSuccess) e = S->sc.alloc((size_t)nrhs * (7 * 16 + 4 * 8 + 3 * 4) + 64);
      if (e == cudaSuccess) e = S->part.alloc((size_t)2 * nrhs * reduce_blocks(std::max(S->N[0], S->NP)) * 16);
      if (e != cudaSuccess) return finish(cuda_fail(ctx, e, "solver workspace"));
      char* q = (char*)S->sc.p;
      auto take = [&](size_t bytes) { char* r = q; q += bytes; return r; };
      S->rho = (double2*)take(nrhs * 16);
      S->rho_new = (double2*)take(nrhs * 16);
      S->alpha = (double2*)take(nrhs * 16);
      S->omega = (double2*)take(nrhs * 16);
      S->beta = (double2*)take(nrhs * 16);
      S->rv = (double2*)take(nrhs * 16);
      S->ts = (double2*)take(nrhs * 16);
      S->tt = (double*)take(nrhs * 8);
      S->rn2 = (double*)take(nrhs * 8);
      S->bn2 = (double*)take(nrhs * 8);
      S->scale = (double*)take(nrhs * 8);
      S->active = (int*)take(nrhs * 4);
      S->brk = (int*)take(nrhs * 4);
      S->count = (unsigned*)take(nrhs * 4);
      e = cudaMemsetAsync(S->count, 0, nrhs * 4, stream);
      if (e != cudaSuccess) return finish(cuda_fail(ctx, e, "solver workspace"));
      S->h_rn2.resize(nrhs);
      if (cudaHostAlloc(&S->pin_rn2, nrhs * sizeof(double), cudaHostAllocDefault) != cudaSuccess ||
          cudaHostAlloc(&S->pin_act, nrhs * sizeof(int), cudaHostAllocDefault) != cudaSuccess ||
          cudaHostAlloc(&S->pin_act_up, nrhs * sizeof(int), cudaHostAllocDefault) != cudaSuccess)
        return finish(fail(ctx, HX_ERR_OOM, "pinned host buffers"));
      S->h_bn2.resize(nrhs);
      S->h_active.resize(nrhs);
      ctx->solvers[key] = std::move(up);
      ctx->solver_lru.push_front(key);
    }
  }
  // ---- the preconditioner's PML cap: fixed, or (pml_cap < 0) tighter the more
  // strongly the grid's PML damps: min(1, |pml_cap| omega / gamma0), gamma0
  // the largest damping of the grid's PML faces
  double pml_cap = opt.pml_cap;
  if (pml_cap < 0) {
    const double omega = 2.0 * M_PI * grid->f;
    double ratio = 0;
    for (int k = 0; k < 6; ++k)
      if (grid->npml[k] > 0)
        ratio = std::max(ratio, 3.0 * grid->v_ref / (2.0 * grid->npml[k] * grid->h) * std::log(1.0 / grid->r_coef) /
                                    omega);
    pml_cap = ratio > 0 ? std::min(1.0, -opt.pml_cap / ratio) : 1.0;
  }
  // ---- operator levels (PML arrays depend on h, f, npml, v_ref, r_coef)
  char okey[320];
  std::snprintf(okey, sizeof(okey), "%.17g %.17g %d %d %d %d %d %d %.17g %.17g cap%.17g", grid->h, grid->f,
                grid->npml[0], grid->npml[1], grid->npml[2], grid->npml[3], grid->npml[4], grid->npml[5],
                grid->v_ref, grid->r_coef, pml_cap);
  if (S->op_key != okey) {
    // private copies, so LRU eviction in the shared cache cannot free them:
    // lvlA = the true fine operator (Krylov apply, FP64 residual); lvl[l] =
    // the preconditioner's levels with the PML damping capped at pml_cap.
    auto own_copy = [&](const int* nl, double hl, double cap, std::unique_ptr<Level>* dst) -> int {
      Level* tmp = nullptr;
      int s2 = get_level(ctx, grid, nl, hl, &tmp, cap);
      if (s2) return s2;
      auto own = std::make_unique<Level>();
      for (int d = 0; d < 3; ++d) {
        own->n[d] = tmp->n[d];
        own->lo[d] = tmp->lo[d];
        own->hi[d] = tmp->hi[d];
        const size_t nb64 = 4 * (size_t)tmp->n[d] * sizeof(double), nb32 = nb64 / 2;
        cudaError_t e = cudaMalloc(&own->ax64[d], nb64);
        if (e == cudaSuccess) e = cudaMalloc(&own->ax32[d], nb32);
        if (e == cudaSuccess) e = cudaMemcpy(own->ax64[d], tmp->ax64[d], nb64, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(own->ax32[d], tmp->ax32[d], nb32, cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "level copy");
      }
      own->h = tmp->h;
      own->f = tmp->f;
      *dst = std::move(own);
      return HX_OK;
    };
    if ((st = own_copy(S->n[0], grid->h, 0.0, &S->lvlA))) return finish(st);
    for (int l = 0; l < S->nlev; ++l)
      if ((st = own_copy(S->n[l], grid->h * (double)(1 << l), pml_cap, &S->lvl[l]))) return finish(st);
    S->op_key = okey;
  }
  // coarse velocities, level by level (injection or averaged slowness squared)
  for (int l = 1; l < S->nlev; ++l) {
    const float* vf = l == 1 ? v_dev : (const float*)S->vlev[l - 1].p;
    cudaError_t e = launch_coarse_velocity(vf, S->n[l - 1], (float*)S->vlev[l].p, S->n[l], opt.coarse_velocity,
                                           stream);
    if (e != cudaSuccess) return finish(cuda_fail(ctx, e, "coarse velocity"));
  }
  // Galerkin coarse operators R A P of the shifted operator (inner precision)
  S->galerkin = opt.coarse_galerkin != 0 && S->nlev > 1;
  S->kappa = opt.bicg_kappa;
  if (S->galerkin) {
    const size_t cs = prec == 64 ? 16 : 8;
    for (int l = 1; l < S->nlev; ++l) {
      cudaError_t e = S->acoef[l].alloc((size_t)27 * S->N[l] * cs);
      if (e == cudaSuccess) {
        if (l == 1)
          e = prec == 64 ? launch_galerkin_onfly<double>(make_desc<double>(ctx, *S->lvl[0], v_dev, opt.shift_beta, true),
                                                         S->acoef[1].p, S->n[1], stream)
                         : launch_galerkin_onfly<float>(make_desc<float>(ctx, *S->lvl[0], v_dev, opt.shift_beta, true),
                                                        S->acoef[1].p, S->n[1], stream);
        else
          e = prec == 64 ? launch_galerkin_stored<double>(S->acoef[l - 1].p, S->n[l - 1], S->acoef[l].p, S->n[l], stream)
                         : launch_galerkin_stored<float>(S->acoef[l - 1].p, S->n[l - 1], S->acoef[l].p, S->n[l], stream);
      }
      if (e != cudaSuccess) return finish(cuda_fail(ctx, e, "Galerkin coarse operator"));
    }
  }
  if ((st = setup_coarse_inverse(ctx, S, v_dev, opt.shift_beta, okey, stream))) return finish(st);
  // ---- sources (grid delta or consistent-mass spread), FP64 amplitudes / h^3
  std::vector<SourceEntry> ent;
  const long long N = S->N[0];
  const double ih3 = 1.0 / (grid->h * grid->h * grid->h);
  for (int k = 0; k < nsrc; ++k) {
    const hx_source& q = src[k];
    const long long idx = q.ix + (long long)grid->nx * (q.iy + (long long)grid->ny * q.iz);
    if (!opt.source_spread) {
      ent.push_back({idx, q.rhs, q.amp_re * ih3, q.amp_im * ih3});
      continue;
    }
    float vs = 0;
    cudaError_t e = cudaMemcpy(&vs, v_dev + idx, sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return finish(cuda_fail(ctx, e, "source velocity"));
    double u = grid->f * grid->h / (double)vs / ctx->d_inv_g;
    u = std::min(std::max(u, 0.0), (double)(ctx->n_g - 1));
    int i0 = std::min((int)u, ctx->n_g - 2);
    const double tf = u - i0;
    double wm[4];
    for (int c = 0; c < 4; ++c)
      wm[c] = (1 - tf) * ctx->table[7 * i0 + 3 + c] + tf * ctx->table[7 * (i0 + 1) + 3 + c];
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int x = q.ix + dx, y = q.iy + dy, z = q.iz + dz;
          if (x < 0 || x >= grid->nx || y < 0 || y >= grid->ny || z < 0 || z >= grid->nz) continue;
          const double w = wm[std::abs(dx) + std::abs(dy) + std::abs(dz)] * ih3;
          ent.push_back({x + (long long)grid->nx * (y + (long long)grid->ny * z), q.rhs, q.amp_re * w, q.amp_im * w});
        }
  }
  {
    cudaError_t e = S->srcs.alloc(ent.size() * sizeof(SourceEntry));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(S->srcs.p, ent.data(), ent.size() * sizeof(SourceEntry), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return finish(cuda_fail(ctx, e, "source upload"));
  }
  const SourceEntry* dsrc = (const SourceEntry*)S->srcs.p;
  const int nent = (int)ent.size();
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return finish(cuda_fail(ctx, e, "setup"));
  // complex64 kernel configuration of the fine level, tuned once per grid
  // size and nrhs (the Krylov buffers serve as scratch before the solve)
  if (prec == 32 && opt.autotune && (long long)N * nrhs >= (1LL << 18) &&
      ctx->st32_cfg < 0 && !ctx->tuned.count(tune_key(grid->nx, grid->ny, grid->nz, nrhs))) {
    if ((e = cudaMemsetAsync(S->p.p, 0, (size_t)nrhs * S->NP * 8, stream)))
      return finish(cuda_fail(ctx, e, "autotune scratch"));
    if ((st = tune_cfg32(ctx, *S->lvlA, v_dev, nrhs, S->p.p, S->v.p, S->pitch0, 2, stream, nullptr, nullptr, 0)))
      return finish(st);
  }
  auto t_setup = std::chrono::steady_clock::now();
  trace_setup.end();

  S->graph_ready = false;   // kernel parameters may differ from the last call
  Run run(ctx, S, grid, v_dev, opt, stream);
  const int R = nrhs;
  double2* x64 = (double2*)wavefield_dev;
  const size_t f64 = (size_t)R * N * 16;
  int inner_total = 0, outer = 0;
  double worst = 0;
  st = HX_OK;
  std::vector<double> sn2(R), rn2(R);
  const OpDesc<double> A64 = make_desc<double>(ctx, *S->lvlA, v_dev, 0.0);
  // Residual r64 = s - A x64 (FP64) and its per-RHS squared norms.
  double2* r64 = (double2*)S->r64.p;
  if (!opt.initial_guess) {
    if ((e = cudaMemsetAsync(x64, 0, f64, stream))) return finish(cuda_fail(ctx, e, "x init"));
  }
  auto residual = [&](bool x_is_zero) -> int {
    cudaError_t ee;
    if (x_is_zero) ee = cudaMemsetAsync(r64, 0, f64, stream);
    else {
      cudaEvent_t ev = prof_begin(ctx, stream);
      ee = launch_stencil(A64, kResidual, x64, nullptr, r64, R, N, 0.0, stream);
      prof_end(ctx, HX_PROF_APPLY64, ev, 2.0 * 16 * N * R + 4.0 * N, stream);
    }
    if (ee == cudaSuccess) ee = launch_add_sources<double>(r64, N, dsrc, nent, stream);
    if (ee == cudaSuccess) ee = launch_norm2<double>(r64, N, R, (double2*)S->part.p, S->rn2, stream);
    if (ee == cudaSuccess) ee = cudaMemcpyAsync(rn2.data(), S->rn2, R * sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (ee == cudaSuccess) ee = cudaStreamSynchronize(stream);
    if (ee != cudaSuccess) return cuda_fail(ctx, ee, "FP64 residual");
    for (int k = 0; k < R; ++k)
      if (!std::isfinite(rn2[k])) return fail(ctx, HX_ERR_NUMERIC, "non-finite FP64 residual");
    return HX_OK;
  };
  // ||s||^2 from the source field alone
  if ((st = residual(true))) return finish(st);
  sn2 = rn2;
  if (opt.initial_guess && (st = residual(false))) return finish(st);

  auto worst_rel = [&]() {
    double w = 0;
    for (int k = 0; k < R; ++k) w = std::max(w, std::sqrt(rn2[k] / sn2[k]));
    return w;
  };
  worst = worst_rel();
  if (prec == 64) {
    // plain FP64 form: BiCGStab<double> on A d = r64 (= s, or s - A x0)
    std::vector<int> act(R);
    for (int k = 0; k < R; ++k) act[k] = std::sqrt(rn2[k] / sn2[k]) > opt.tol;
    std::vector<double> sc(R);
    for (int k = 0; k < R; ++k) sc[k] = rn2[k] > 0 ? std::sqrt(sn2[k] / rn2[k]) : 1.0;
    if ((e = cudaMemcpyAsync(S->r.p, r64, f64, cudaMemcpyDeviceToDevice, stream)))
      return finish(cuda_fail(ctx, e, "rhs copy"));
    int its = 0;
    // tolerance relative to ||s|| expressed relative to the Krylov RHS
    double itol = opt.tol;
    for (int k = 0; k < R; ++k) itol = std::min(itol, opt.tol * sc[k]);
    if ((st = run.bicgstab<double>(itol, opt.max_iter, act, &its))) return finish(st);
    inner_total += its;
    for (int k = 0; k < R; ++k) sc[k] = 1.0;
    if ((e = cudaMemcpyAsync(S->scale, sc.data(), R * sizeof(double), cudaMemcpyHostToDevice, stream)) ||
        (e = launch_axpy_c128(x64, (const double2*)S->x.p, S->scale, N, R, stream)))
      return finish(cuda_fail(ctx, e, "update"));
    if ((st = residual(false))) return finish(st);
    worst = worst_rel();
    outer = 1;
  } else {
    while (outer < opt.max_outer && worst > opt.tol && !run.past_deadline()) {
      TraceRange trace_step("refinement step");
      // inner complex64 solve of A d = r / ||r||
      std::vector<double> sc(R);
      std::vector<int> act(R);
      for (int k = 0; k < R; ++k) {
        const bool a = std::sqrt(rn2[k] / sn2[k]) > opt.tol;
        act[k] = a;
        sc[k] = a ? 1.0 / std::sqrt(rn2[k]) : 0.0;
      }
      if ((e = cudaMemcpyAsync(S->scale, sc.data(), R * sizeof(double), cudaMemcpyHostToDevice, stream)) ||
          (e = launch_cast_scale(r64, (float2*)S->r.p, S->scale, N, R, stream, grid->nx, S->pitch0)))
        return finish(cuda_fail(ctx, e, "cast"));
      int its = 0;
      if ((st = run.bicgstab<float>(opt.inner_tol, opt.max_iter, act, &its))) return finish(st);
      inner_total += its;
      for (int k = 0; k < R; ++k) sc[k] = act[k] ? std::sqrt(rn2[k]) : 0.0;
      if ((e = cudaMemcpyAsync(S->scale, sc.data(), R * sizeof(double), cudaMemcpyHostToDevice, stream)) ||
          (e = launch_axpy_mixed(x64, (const float2*)S->x.p, S->scale, N, R, stream, grid->nx, S->pitch0)))
        return finish(cuda_fail(ctx, e, "update"));
      ++outer;
      if ((st = residual(false))) return finish(st);
      worst = worst_rel();
    }
  }
  prof_collect(ctx);
  auto t_end = std::chrono::steady_clock::now();
  // a TMA-kernel CTA whose bounded wait for a plane ran out
  if (zm_take_error(ctx->device)) {
    if (report) report->rel_residual = worst;
    return finish(fail(ctx, HX_ERR_TIMEOUT, "a stencil kernel's bounded wait for its plane copies ran out"));
  }
  if (report) {
    report->outer_iters = outer;
    report->inner_iters = inner_total;
    report->mg_levels = S->nlev;
    report->rel_residual = worst;
    report->setup_ms = std::chrono::duration<double, std::milli>(t_setup - t_start).count();
    report->solve_ms = std::chrono::duration<double, std::milli>(t_end - t_setup).count();
  }
  if (worst > opt.tol && run.cancelled()) return finish(fail(ctx, HX_ERR_CANCELLED, "cancelled"));
  if (worst > opt.tol) return finish(fail(ctx, HX_ERR_NOT_CONVERGED, "tolerance not reached"));
  return finish(HX_OK);
}
