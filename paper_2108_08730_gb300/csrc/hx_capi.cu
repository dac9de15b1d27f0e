// C-ABI entry points: context, weight table, operator apply / coefficients.
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "hx_context.h"
#include "hx_galerkin.cuh"
#include "hx_internal.h"

namespace hx {

Profile1D Profile1D::from_grid(int n, double h, int npml_lo, int npml_hi, double v_ref,
                               double r_coef) {
  auto g0 = [&](int np) { return np <= 0 ? 0.0 : 3.0 * v_ref / (2.0 * np * h) * std::log(1.0 / r_coef); };
  return Profile1D{npml_lo * h, (n - 1 - npml_hi) * h, npml_lo * h, npml_hi * h, g0(npml_lo),
                   g0(npml_hi)};
}

double Profile1D::gamma(double x) const {
  double g = 0.0;
  if (len_lo > 0) {
    const double d = x_lo - x > 0 ? x_lo - x : 0.0;
    g += g0_lo * (d / len_lo) * (d / len_lo);
  }
  if (len_hi > 0) {
    const double d = x - x_hi > 0 ? x - x_hi : 0.0;
    g += g0_hi * (d / len_hi) * (d / len_hi);
  }
  return g;
}

Level::~Level() {
  for (int d = 0; d < 3; ++d) {
    if (ax64[d]) cudaFree(ax64[d]);
    if (ax32[d]) cudaFree(ax32[d]);
  }
}

int fail(hx_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(hx_ctx* ctx, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(ctx, e == cudaErrorMemoryAllocation ? HX_ERR_OOM : HX_ERR_CUDA, m);
}

int check_grid(hx_ctx* ctx, const hx_grid* g) {
  if (!g) return fail(ctx, HX_ERR_ARG, "grid is NULL");
  const int n[3] = {g->nx, g->ny, g->nz};
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 3) return fail(ctx, HX_ERR_ARG, "each grid dimension must be >= 3");
    const int lo = g->npml[2 * d], hi = g->npml[2 * d + 1];
    if (lo < 0 || hi < 0 || 2 * lo >= n[d] || 2 * hi >= n[d])
      return fail(ctx, HX_ERR_ARG, "npml must satisfy 0 <= npml < n/2 on every face");
  }
  if ((double)g->nx * g->ny * g->nz > 4.0e9) return fail(ctx, HX_ERR_ARG, "grid too large");
  if (!(g->h > 0) || !std::isfinite(g->h)) return fail(ctx, HX_ERR_ARG, "h must be > 0");
  if (!(g->f > 0) || !std::isfinite(g->f)) return fail(ctx, HX_ERR_ARG, "f must be > 0");
  if (!(g->v_ref > 0) || !std::isfinite(g->v_ref)) return fail(ctx, HX_ERR_ARG, "v_ref must be > 0");
  if (!(g->r_coef > 0 && g->r_coef < 1)) return fail(ctx, HX_ERR_ARG, "r_coef must be in (0, 1)");
  return HX_OK;
}

int get_level(hx_ctx* ctx, const hx_grid* g, const int nl[3], double hl, Level** out, double gamma_cap) {
  char key[512];
  std::snprintf(key, sizeof(key), "%d %d %d %.17g %.17g %d %d %d %d %d %d %.17g %.17g | %d %d %d %.17g c%.17g",
                g->nx, g->ny, g->nz, g->h, g->f, g->npml[0], g->npml[1], g->npml[2], g->npml[3],
                g->npml[4], g->npml[5], g->v_ref, g->r_coef, nl[0], nl[1], nl[2], hl, gamma_cap);
  auto it = ctx->levels.find(key);
  if (it != ctx->levels.end()) {
    ctx->lru.remove(key);
    ctx->lru.push_front(key);
    *out = it->second.get();
    return HX_OK;
  }
  while (ctx->levels.size() >= 64) {
    ctx->levels.erase(ctx->lru.back());
    ctx->lru.pop_back();
  }
  auto lv = std::make_unique<Level>();
  const int nf[3] = {g->nx, g->ny, g->nz};
  const double omega = 2.0 * M_PI * g->f;
  lv->h = hl;
  lv->f = g->f;
  for (int d = 0; d < 3; ++d) {
    lv->n[d] = nl[d];
    Profile1D prof =
        Profile1D::from_grid(nf[d], g->h, g->npml[2 * d], g->npml[2 * d + 1], g->v_ref, g->r_coef);
    if (gamma_cap > 0) {
      prof.g0_lo = std::min(prof.g0_lo, gamma_cap * omega);
      prof.g0_hi = std::min(prof.g0_hi, gamma_cap * omega);
    }
    std::vector<double> a64(4 * (size_t)nl[d]);
    std::vector<float> a32(4 * (size_t)nl[d]);
    const double ih2 = 1.0 / (hl * hl);
    int lo = -1, hi = -2;
    for (int i = 0; i < nl[d]; ++i) {
      // xi = 1 + i gamma / omega at the node and the two half nodes
      auto xi = [&](double x) { return std::complex<double>(1.0, prof.gamma(x) / omega); };
      const std::complex<double> xn = xi(i * hl), xp = xi((i + 0.5) * hl), xm = xi((i - 0.5) * hl);
      const std::complex<double> up = 1.0 / (xn * xp) * ih2, dn = 1.0 / (xn * xm) * ih2;
      a64[4 * i + 0] = up.real();
      a64[4 * i + 1] = up.imag();
      a64[4 * i + 2] = dn.real();
      a64[4 * i + 3] = dn.imag();
      for (int k = 0; k < 4; ++k) a32[4 * i + k] = (float)a64[4 * i + k];
      const bool plain = up.imag() == 0.0 && dn.imag() == 0.0 && up.real() == ih2 && dn.real() == ih2;
      if (plain) {
        if (lo < 0) lo = i;
        hi = i;
      }
    }
    // the plain nodes must be contiguous for the range test in the kernels
    for (int i = (lo < 0 ? 0 : lo); i <= hi; ++i) {
      if (!(a64[4 * i + 1] == 0.0 && a64[4 * i + 3] == 0.0)) return fail(ctx, HX_ERR_ARG, "PML layout");
    }
    lv->lo[d] = lo < 0 ? 1 : lo;
    lv->hi[d] = lo < 0 ? 0 : hi;
    cudaError_t e = cudaMalloc(&lv->ax64[d], a64.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&lv->ax32[d], a32.size() * sizeof(float));
    if (e == cudaSuccess)
      e = cudaMemcpy(lv->ax64[d], a64.data(), a64.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(lv->ax32[d], a32.data(), a32.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "PML coefficient upload");
  }
  *out = lv.get();
  ctx->levels[key] = std::move(lv);
  ctx->lru.push_front(key);
  return HX_OK;
}

template <typename T>
OpDesc<T> make_desc(const hx_ctx* ctx, const Level& lv, const float* v, double beta, bool precond) {
  OpDesc<T> d;
  d.nx = lv.n[0];
  d.ny = lv.n[1];
  d.nz = lv.n[2];
  d.v = v;
  const bool pt = precond && ctx->ptab64;
  if (pt) d.tab = sizeof(T) == 8 ? (const T*)ctx->ptab64 : (const T*)ctx->ptab32;
  else d.tab = sizeof(T) == 8 ? (const T*)ctx->tab64 : (const T*)ctx->tab32;
  d.n_g = pt ? ctx->pn_g : ctx->n_g;
  d.u_scale = (T)(lv.f * lv.h / (pt ? ctx->pd_inv_g : ctx->d_inv_g));
  d.omega2 = (T)((2.0 * M_PI * lv.f) * (2.0 * M_PI * lv.f));
  d.beta = (T)beta;
  d.inv_h2 = (T)(1.0 / (lv.h * lv.h));
  for (int a = 0; a < 3; ++a) {
    d.axis[a] = sizeof(T) == 8 ? (const T*)lv.ax64[a] : (const T*)lv.ax32[a];
    d.plain_lo[a] = lv.lo[a];
    d.plain_hi[a] = lv.hi[a];
  }
  d.cfg32 = ctx->st32_cfg;   // call sites that know nrhs refine this (ctx_cfg32)
  if (!precond) {
    d.gam = ctx->op_weights == HX_WEIGHTS_GAM;
    d.mass1 = ctx->op_mass_form == 1;
    d.buoy = ctx->med_buoy;
    d.invq = ctx->med_invq;
  }
  return d;
}

template OpDesc<float> make_desc<float>(const hx_ctx*, const Level&, const float*, double, bool);
template OpDesc<double> make_desc<double>(const hx_ctx*, const Level&, const float*, double, bool);

namespace {
std::atomic<long long> g_launches{0};
}
long long launch_count() { return g_launches.load(); }
void count_launch(int n) { g_launches += n; }
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("HX_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

cudaEvent_t prof_begin(hx_ctx* ctx, cudaStream_t s) {
  if (!ctx->prof_on) return nullptr;
  cudaEvent_t e;
  if (!ctx->prof_pool.empty()) {
    e = ctx->prof_pool.back();
    ctx->prof_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    return nullptr;
  }
  cudaEventRecord(e, s);
  return e;
}

void prof_end(hx_ctx* ctx, int kind, cudaEvent_t a, double bytes, cudaStream_t s) {
  if (!ctx->prof_on || !a) return;
  cudaEvent_t e;
  if (!ctx->prof_pool.empty()) {
    e = ctx->prof_pool.back();
    ctx->prof_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    ctx->prof_pool.push_back(a);
    return;
  }
  cudaEventRecord(e, s);
  ctx->prof_pending.push_back({kind, a, e, bytes});
}

void prof_collect(hx_ctx* ctx) {
  for (auto& p : ctx->prof_pending) {
    float ms = 0;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      ctx->prof[p.kind].launches += 1;
      ctx->prof[p.kind].ms += ms;
      ctx->prof[p.kind].bytes += p.bytes;
    }
    ctx->prof_pool.push_back(p.a);
    ctx->prof_pool.push_back(p.b);
  }
  ctx->prof_pending.clear();
}

}  // namespace hx

hx_ctx::~hx_ctx() {
  if (grp_ev) cudaEventSynchronize(grp_ev);
  if (grp_dev) cudaFree(grp_dev);
  if (grp_host) cudaFreeHost(grp_host);
  if (grp_ev) cudaEventDestroy(grp_ev);
  for (auto& p : prof_pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : prof_pool) cudaEventDestroy(e);
  solvers.clear();
  levels.clear();
  if (work_stream) cudaStreamDestroy(work_stream);
  for (auto e : order_ev)
    if (e) cudaEventDestroy(e);
  if (ptab64 && ptab64 != tab64) cudaFree(ptab64);
  if (ptab32 && ptab32 != tab32) cudaFree(ptab32);
  if (tab64) cudaFree(tab64);
  if (tab32) cudaFree(tab32);
}

using namespace hx;

extern "C" {

int hx_build_weight_table(const double* theta_deg, int n_theta, const double* phi_deg, int n_phi,
                          double inv_g_max, double d_inv_g, double lambda, double* table_out,
                          int capacity, int* n_g_out) {
  std::string err;
  return build_weight_table(theta_deg, n_theta, phi_deg, n_phi, inv_g_max, d_inv_g, lambda,
                            table_out, capacity, n_g_out, &err);
}

int hx_fit_joint_weights(const double* inv_g, int n, const double* theta_deg, int n_theta,
                         const double* phi_deg, int n_phi, double* w7_out) {
  std::string err;
  return fit_joint_weights(inv_g, n, theta_deg, n_theta, phi_deg, n_phi, w7_out, &err);
}

int hx_ctx_create(hx_ctx** out, int device) {
  if (!out) return HX_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return HX_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return HX_ERR_CUDA;
  hx_ctx* c = new (std::nothrow) hx_ctx();
  if (!c) return HX_ERR_OOM;
  c->device = device;
  *out = c;
  return HX_OK;
}

void hx_ctx_destroy(hx_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  delete ctx;
}

const char* hx_last_error(const hx_ctx* ctx) {
  if (!ctx) return "no context";
  return ctx->err.c_str();
}

namespace {
// Derived device tables (FP64 and FP32) of a weight table [n_g][7].
cudaError_t upload_table(const double* table, int n_g, double** t64, float** t32) {
  std::vector<double> d64((size_t)n_g * kTabW, 0.0);
  std::vector<float> d32((size_t)n_g * kTabW, 0.f);
  for (int i = 0; i < n_g; ++i) {
    const double* w = table + 7 * (size_t)i;
    const double ws2 = w[1], ws3 = w[2];
    const double t0 = w[0] + 2.0 * ws2 / 3.0 + 0.5 * ws3;
    double* o = &d64[(size_t)i * kTabW];
    o[0] = -6.0 * t0;
    o[1] = t0 - ws2 / 3.0;
    o[2] = ws2 / 6.0 - ws3 / 4.0;
    o[3] = 3.0 * ws3 / 8.0;
    for (int k = 0; k < 4; ++k) o[4 + k] = w[3 + k];
    o[8] = t0;
    o[9] = ws2 / 12.0;
    o[10] = ws3 / 8.0;
    for (int k = 0; k < kTabW; ++k) d32[(size_t)i * kTabW + k] = (float)o[k];
  }
  *t64 = nullptr;
  *t32 = nullptr;
  cudaError_t e = cudaMalloc(t64, d64.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(t32, d32.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(*t64, d64.data(), d64.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(*t32, d32.data(), d32.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (*t64) cudaFree(*t64);
    if (*t32) cudaFree(*t32);
    *t64 = nullptr;
    *t32 = nullptr;
  }
  return e;
}
}  // namespace

int hx_set_operator_form(hx_ctx* ctx, int weights, int mass_form) {
  if (!ctx) return HX_ERR_ARG;
  if (weights != HX_WEIGHTS_GA && weights != HX_WEIGHTS_GAM) return fail(ctx, HX_ERR_ARG, "unknown weights");
  if (mass_form != 1 && mass_form != 2) return fail(ctx, HX_ERR_ARG, "mass_form must be 1 or 2");
  ctx->op_weights = weights;
  ctx->op_mass_form = mass_form;
  return HX_OK;
}

int hx_set_medium(hx_ctx* ctx, const float* buoyancy_dev, const float* inv_q_dev) {
  if (!ctx) return HX_ERR_ARG;
  ctx->med_buoy = buoyancy_dev;
  ctx->med_invq = inv_q_dev;
  return HX_OK;
}

int hx_set_table_ex(hx_ctx* ctx, const double* table, int n_g, double d_inv_g, int which) {
  if (!ctx) return HX_ERR_ARG;
  if (which < HX_TABLE_BOTH || which > HX_TABLE_PRECONDITIONER) return fail(ctx, HX_ERR_ARG, "unknown table role");
  if (!table || n_g < 2 || !(d_inv_g > 0)) return fail(ctx, HX_ERR_ARG, "need table, n_g >= 2, d_inv_g > 0");
  for (int i = 0; i < 7 * n_g; ++i)
    if (!std::isfinite(table[i])) return fail(ctx, HX_ERR_ARG, "table has non-finite entries");
  if (which == HX_TABLE_PRECONDITIONER && !ctx->tab64)
    return fail(ctx, HX_ERR_STATE, "set the operator table first");
  cudaSetDevice(ctx->device);
  double* t64 = nullptr;
  float* t32 = nullptr;
  cudaError_t e = upload_table(table, n_g, &t64, &t32);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "table upload");
  auto drop_precond = [&]() {
    if (ctx->ptab64) cudaFree(ctx->ptab64);
    if (ctx->ptab32) cudaFree(ctx->ptab32);
    ctx->ptab64 = nullptr;
    ctx->ptab32 = nullptr;
  };
  if (which == HX_TABLE_PRECONDITIONER) {
    drop_precond();
    ctx->ptab64 = t64;
    ctx->ptab32 = t32;
    ctx->pn_g = n_g;
    ctx->pd_inv_g = d_inv_g;
  } else {
    if (which == HX_TABLE_OPERATOR && !ctx->ptab64 && ctx->tab64) {
      // the preconditioner keeps the table it used so far
      ctx->ptab64 = ctx->tab64;
      ctx->ptab32 = ctx->tab32;
      ctx->pn_g = ctx->n_g;
      ctx->pd_inv_g = ctx->d_inv_g;
    } else {
      if (which == HX_TABLE_BOTH) drop_precond();
      if (ctx->tab64 && ctx->tab64 != ctx->ptab64) cudaFree(ctx->tab64);
      if (ctx->tab32 && ctx->tab32 != ctx->ptab32) cudaFree(ctx->tab32);
    }
    ctx->tab64 = t64;
    ctx->tab32 = t32;
    ctx->table.assign(table, table + 7 * (size_t)n_g);
    ctx->n_g = n_g;
    ctx->d_inv_g = d_inv_g;
  }
  ctx->solvers.clear();
  ctx->solver_lru.clear();
  return HX_OK;
}

int hx_set_table(hx_ctx* ctx, const double* table, int n_g, double d_inv_g) {
  return hx_set_table_ex(ctx, table, n_g, d_inv_g, HX_TABLE_BOTH);
}

int hx_apply_operator(hx_ctx* ctx, const hx_grid* grid, const float* v_dev, double shift_beta,
                      const void* x_dev, void* y_dev, int nrhs, int precision, void* stream) {
  if (!ctx) return HX_ERR_ARG;
  int st = check_grid(ctx, grid);
  if (st) return st;
  if (!ctx->tab64) return fail(ctx, HX_ERR_STATE, "no weight table set (hx_set_table)");
  if (!v_dev || !x_dev || !y_dev || nrhs < 1) return fail(ctx, HX_ERR_ARG, "null buffer or nrhs < 1");
  if (x_dev == y_dev) return fail(ctx, HX_ERR_ARG, "x and y must not overlap");
  const bool direct = (precision & HX_APPLY_DIRECT) != 0;
  precision &= ~HX_APPLY_DIRECT;
  if (precision != 32 && precision != 64) return fail(ctx, HX_ERR_ARG, "precision must be 32 or 64");
  if (!std::isfinite(shift_beta)) return fail(ctx, HX_ERR_ARG, "shift_beta must be finite");
  cudaSetDevice(ctx->device);
  Level* lv = nullptr;
  const int nl[3] = {grid->nx, grid->ny, grid->nz};
  if ((st = get_level(ctx, grid, nl, grid->h, &lv))) return st;
  const long long N = (long long)grid->nx * grid->ny * grid->nz;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (precision == 32) {
    OpDesc<float> d = make_desc<float>(ctx, *lv, v_dev, shift_beta);
    d.cfg32 = ctx_cfg32(ctx, grid->nx, grid->ny, grid->nz, nrhs);
    e = direct ? launch_direct_stencil<float>(d, kApply, x_dev, nullptr, y_dev, nrhs, 0.0, s)
               : launch_stencil(d, kApply, x_dev, nullptr, y_dev, nrhs, N, 0.0, s);
  } else {
    const OpDesc<double> d = make_desc<double>(ctx, *lv, v_dev, shift_beta);
    e = direct ? launch_direct_stencil<double>(d, kApply, x_dev, nullptr, y_dev, nrhs, 0.0, s)
               : launch_stencil(d, kApply, x_dev, nullptr, y_dev, nrhs, N, 0.0, s);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "apply launch");
  return HX_OK;
}

int hx_stencil_sweep(hx_ctx* ctx, const hx_grid* grid, const float* v_dev, double shift_beta,
                     int kind, const void* x_dev, const void* b_dev, void* y_dev, int nrhs,
                     int precision, double omega, void* stream) {
  if (!ctx) return HX_ERR_ARG;
  int st = check_grid(ctx, grid);
  if (st) return st;
  if (!ctx->tab64) return fail(ctx, HX_ERR_STATE, "no weight table set (hx_set_table)");
  if (kind != HX_SWEEP_RESIDUAL && kind != HX_SWEEP_JACOBI) return fail(ctx, HX_ERR_ARG, "unknown sweep kind");
  if (!v_dev || !x_dev || !y_dev || nrhs < 1 || (kind == HX_SWEEP_JACOBI && !b_dev))
    return fail(ctx, HX_ERR_ARG, "null buffer or nrhs < 1");
  if (x_dev == y_dev || b_dev == y_dev) return fail(ctx, HX_ERR_ARG, "y must overlap neither x nor b");
  if (precision != 32 && precision != 64) return fail(ctx, HX_ERR_ARG, "precision must be 32 or 64");
  if (!std::isfinite(shift_beta) || !std::isfinite(omega)) return fail(ctx, HX_ERR_ARG, "non-finite parameter");
  cudaSetDevice(ctx->device);
  Level* lv = nullptr;
  const int nl[3] = {grid->nx, grid->ny, grid->nz};
  if ((st = get_level(ctx, grid, nl, grid->h, &lv))) return st;
  const long long N = (long long)grid->nx * grid->ny * grid->nz;
  const int mode = kind == HX_SWEEP_RESIDUAL ? kResidual : kJacobi;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (precision == 32) {
    OpDesc<float> d = make_desc<float>(ctx, *lv, v_dev, shift_beta);
    d.cfg32 = ctx_cfg32(ctx, grid->nx, grid->ny, grid->nz, nrhs, true);
    e = launch_stencil(d, mode, x_dev, b_dev, y_dev, nrhs, N, omega, s);
  } else {
    const OpDesc<double> d = make_desc<double>(ctx, *lv, v_dev, shift_beta);
    e = launch_stencil(d, mode, x_dev, b_dev, y_dev, nrhs, N, omega, s);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sweep launch");
  return HX_OK;
}

int hx_stencil_pitched(hx_ctx* ctx, const hx_grid* grid, const float* v_dev, double shift_beta, int kind,
                       const void* x_dev, const void* b_dev, void* y_dev, int nrhs, int64_t pitch, double omega,
                       void* stream) {
  if (!ctx) return HX_ERR_ARG;
  int st = check_grid(ctx, grid);
  if (st) return st;
  if (!ctx->tab64) return fail(ctx, HX_ERR_STATE, "no weight table set (hx_set_table)");
  if (kind != 0 && kind != HX_SWEEP_RESIDUAL && kind != HX_SWEEP_JACOBI)
    return fail(ctx, HX_ERR_ARG, "unknown kind (0 = apply, HX_SWEEP_RESIDUAL, HX_SWEEP_JACOBI)");
  if (!v_dev || !x_dev || !y_dev || nrhs < 1 || (kind == HX_SWEEP_JACOBI && !b_dev))
    return fail(ctx, HX_ERR_ARG, "null buffer or nrhs < 1");
  if (x_dev == y_dev || (b_dev && b_dev == y_dev)) return fail(ctx, HX_ERR_ARG, "y must overlap neither x nor b");
  if (pitch < grid->nx || (pitch != grid->nx && (pitch & 1)))
    return fail(ctx, HX_ERR_ARG, "pitch must be nx or an even number >= nx");
  if (((uintptr_t)x_dev & 15) || ((uintptr_t)b_dev & 15) || ((uintptr_t)y_dev & 7))
    return fail(ctx, HX_ERR_ARG, "x and b must be 16-byte aligned, y 8-byte aligned");
  if (!std::isfinite(shift_beta) || !std::isfinite(omega)) return fail(ctx, HX_ERR_ARG, "non-finite parameter");
  cudaSetDevice(ctx->device);
  Level* lv = nullptr;
  const int nl[3] = {grid->nx, grid->ny, grid->nz};
  if ((st = get_level(ctx, grid, nl, grid->h, &lv))) return st;
  const int mode = kind == 0 ? kApply : (kind == HX_SWEEP_RESIDUAL ? kResidual : kJacobi);
  OpDesc<float> d = make_desc<float>(ctx, *lv, v_dev, shift_beta);
  d.cfg32 = ctx_cfg32(ctx, grid->nx, grid->ny, grid->nz, nrhs, kind != 0);
  d.pitch = pitch;
  const cudaError_t e = launch_stencil(d, mode, x_dev, kind == 0 ? nullptr : b_dev, y_dev, nrhs,
                                       (long long)pitch * grid->ny * grid->nz, omega, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stencil launch");
  return HX_OK;
}

int hx_apply_batched(hx_ctx* ctx, const hx_apply_item* items, int n, double shift_beta, void* stream) {
  if (!ctx) return HX_ERR_ARG;
  if (!items || n < 1 || n > (1 << 20)) return fail(ctx, HX_ERR_ARG, "need 1 <= n <= 2^20 items");
  if (!ctx->tab64) return fail(ctx, HX_ERR_STATE, "no weight table set (hx_set_table)");
  if (!std::isfinite(shift_beta)) return fail(ctx, HX_ERR_ARG, "shift_beta must be finite");
  if (ctx->op_weights != HX_WEIGHTS_GA || ctx->op_mass_form != 2 || ctx->med_buoy || ctx->med_invq)
    return fail(ctx, HX_ERR_STATE,
                "hx_apply_batched applies the GA operator with the second mass form and b = 1, no Q only");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<GroupProb> probs(n);
  int min_rhs = 1 << 30;
  for (int i = 0; i < n; ++i) {
    const hx_apply_item& it = items[i];
    int st = check_grid(ctx, &it.grid);
    if (st) return st;
    if (!it.v_dev || !it.x_dev || !it.y_dev || it.nrhs < 1) return fail(ctx, HX_ERR_ARG, "null buffer or nrhs < 1");
    if (it.x_dev == it.y_dev) return fail(ctx, HX_ERR_ARG, "x and y must not overlap");
    if (((uintptr_t)it.x_dev & 15) != 0) return fail(ctx, HX_ERR_ARG, "x_dev must be 16-byte aligned");
    Level* lv = nullptr;
    const int nl[3] = {it.grid.nx, it.grid.ny, it.grid.nz};
    if ((st = get_level(ctx, &it.grid, nl, it.grid.h, &lv))) return st;
    probs[i].op = make_desc<float>(ctx, *lv, it.v_dev, shift_beta);
    probs[i].op.xshift = st32_xshift(probs[i].op);
    probs[i].x = it.x_dev;
    probs[i].y = it.y_dev;
    probs[i].nrhs = it.nrhs;
    probs[i].rstride = (long long)it.grid.nx * it.grid.ny * it.grid.nz;
    min_rhs = std::min(min_rhs, it.nrhs);
  }
  const int cfg = ctx->st32_cfg >= 0 ? ctx->st32_cfg : st32_default_config(min_rhs);
  std::vector<GroupItem> plan;
  st32_group_plan(probs.data(), n, cfg, plan);
  if (plan.size() > (size_t)(1u << 30)) return fail(ctx, HX_ERR_ARG, "too many work items");
  const size_t pb = ((n * sizeof(GroupProb) + 255) / 256) * 256;
  const size_t bytes = pb + plan.size() * sizeof(GroupItem) + 256;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  if (ctx->grp_dev_bytes < bytes || ctx->grp_host_bytes < bytes) {
    if (capturing) return fail(ctx, HX_ERR_STATE, "hx_apply_batched: call once outside stream capture to size its buffers");
    if (ctx->grp_ev) cudaEventSynchronize(ctx->grp_ev);
    if (ctx->grp_dev) cudaFree(ctx->grp_dev);
    if (ctx->grp_host) cudaFreeHost(ctx->grp_host);
    ctx->grp_dev = ctx->grp_host = nullptr;
    ctx->grp_dev_bytes = ctx->grp_host_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->grp_dev, 2 * bytes);
    if (e == cudaSuccess) e = cudaHostAlloc(&ctx->grp_host, 2 * bytes, cudaHostAllocDefault);
    if (e == cudaSuccess && !ctx->grp_ev) e = cudaEventCreateWithFlags(&ctx->grp_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batched apply buffers");
    ctx->grp_dev_bytes = ctx->grp_host_bytes = 2 * bytes;
  } else if (!capturing && ctx->grp_ev) {
    cudaEventSynchronize(ctx->grp_ev);                // the previous call's upload has been read
  }
  unsigned char* h = (unsigned char*)ctx->grp_host;
  std::memcpy(h, probs.data(), n * sizeof(GroupProb));
  std::memcpy(h + pb, plan.data(), plan.size() * sizeof(GroupItem));
  unsigned char* d = (unsigned char*)ctx->grp_dev;
  int* counter = (int*)(d + bytes - 256);
  cudaError_t e = cudaMemcpyAsync(d, h, bytes - 256, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !capturing) e = cudaEventRecord(ctx->grp_ev, s);
  if (e == cudaSuccess)
    e = launch_stencil32_group(cfg, (const GroupProb*)d, (const GroupItem*)(d + pb), (int)plan.size(), counter, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batched apply launch");
  return HX_OK;
}

int hx_profile(hx_ctx* ctx, int enable) {
  if (!ctx) return HX_ERR_ARG;
  prof_collect(ctx);
  for (auto& p : ctx->prof) p = hx_ctx::ProfStat();
  ctx->prof_on = enable != 0;
  ctx->prof_launch_base = launch_count();
  return HX_OK;
}

int hx_profile_read(hx_ctx* ctx, int kind, int64_t* launches, double* total_ms, double* algo_bytes) {
  if (!ctx || kind < -1 || kind >= HX_PROF_KINDS) return fail(ctx, HX_ERR_ARG, "bad profile kind");
  prof_collect(ctx);
  if (kind == -1) {
    if (launches) *launches = launch_count() - ctx->prof_launch_base;
    if (total_ms) *total_ms = 0;
    if (algo_bytes) *algo_bytes = 0;
    return HX_OK;
  }
  if (launches) *launches = ctx->prof[kind].launches;
  if (total_ms) *total_ms = ctx->prof[kind].ms;
  if (algo_bytes) *algo_bytes = ctx->prof[kind].bytes;
  return HX_OK;
}

int hx_row_coefficients(hx_ctx* ctx, const hx_grid* grid, const float* v_dev, double shift_beta,
                        double* coef_dev, void* stream) {
  if (!ctx) return HX_ERR_ARG;
  int st = check_grid(ctx, grid);
  if (st) return st;
  if (!ctx->tab64) return fail(ctx, HX_ERR_STATE, "no weight table set (hx_set_table)");
  if (!v_dev || !coef_dev) return fail(ctx, HX_ERR_ARG, "null buffer");
  cudaSetDevice(ctx->device);
  Level* lv = nullptr;
  const int nl[3] = {grid->nx, grid->ny, grid->nz};
  if ((st = get_level(ctx, grid, nl, grid->h, &lv))) return st;
  cudaError_t e = launch_row_coefficients(make_desc<double>(ctx, *lv, v_dev, shift_beta), coef_dev,
                                          (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "row coefficient launch");
  return HX_OK;
}

int hx_assemble_csr(hx_ctx* ctx, const hx_grid* grid, const float* v_dev, double shift_beta,
                    int64_t* rowptr, int32_t* col, double* val, int64_t nnz_cap, int64_t* nnz_out,
                    void* stream) {
  if (!ctx) return HX_ERR_ARG;
  int st = check_grid(ctx, grid);
  if (st) return st;
  if (!rowptr || !col || !val || !nnz_out) return fail(ctx, HX_ERR_ARG, "null host buffer");
  const long long N = (long long)grid->nx * grid->ny * grid->nz;
  if (N > (1LL << 31) / 27) return fail(ctx, HX_ERR_ARG, "grid too large for 32-bit CSR columns");
  cudaSetDevice(ctx->device);
  double* coef = nullptr;
  cudaError_t e = cudaMalloc(&coef, (size_t)N * 27 * 2 * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "coefficient buffer");
  st = hx_row_coefficients(ctx, grid, v_dev, shift_beta, coef, stream);
  std::vector<double> h;
  if (!st) {
    h.resize((size_t)N * 54);
    e = cudaMemcpyAsync(h.data(), coef, h.size() * sizeof(double), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "coefficient download");
  }
  cudaFree(coef);
  if (st) return st;
  const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
  int64_t nnz = 0;
  rowptr[0] = 0;
  for (long long i = 0; i < N; ++i) {
    const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long long)nx * ny));
    int k = 0;
    for (int dk = -1; dk <= 1; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di, ++k) {
          if (ix + di < 0 || ix + di >= nx || iy + dj < 0 || iy + dj >= ny || iz + dk < 0 || iz + dk >= nz)
            continue;
          if (nnz >= nnz_cap) return fail(ctx, HX_ERR_ARG, "nnz_cap too small");
          col[nnz] = (int32_t)(i + di + (long long)nx * (dj + (long long)ny * dk));
          val[2 * nnz] = h[(size_t)i * 54 + 2 * k];
          val[2 * nnz + 1] = h[(size_t)i * 54 + 2 * k + 1];
          ++nnz;
        }
    rowptr[i + 1] = nnz;
  }
  *nnz_out = nnz;
  return HX_OK;
}

}  // extern "C"
