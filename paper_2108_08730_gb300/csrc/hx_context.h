// Context object behind the opaque hx_ctx handle.
#pragma once

#include <cuda_runtime.h>

#include <list>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "hx_internal.h"

namespace hx {

// Physical PML profile of one axis (the reading documented in hx27.h).
struct Profile1D {
  double x_lo, x_hi, len_lo, len_hi, g0_lo, g0_hi;
  static Profile1D from_grid(int n, double h, int npml_lo, int npml_hi, double v_ref,
                             double r_coef);
  double gamma(double x) const;
};

// Operator data of one grid level: per-axis PML coefficients on the device.
struct Level {
  int n[3] = {0, 0, 0};
  double h = 0, f = 0;
  double* ax64[3] = {nullptr, nullptr, nullptr};
  float* ax32[3] = {nullptr, nullptr, nullptr};
  int lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
  ~Level();
};

// Solver workspaces (defined by the solver translation unit).
struct Solver {
  virtual ~Solver() = default;
};

}  // namespace hx

struct hx_ctx {
  int device = 0;
  std::string err;
  // weight table
  int n_g = 0;
  double d_inv_g = 0;
  std::vector<double> table;    // host copy [n_g][7]
  double* tab64 = nullptr;      // derived [n_g][kTabW]
  float* tab32 = nullptr;
  // preconditioner table (hx_set_table_ex); NULL: the operator's table
  double* ptab64 = nullptr;
  float* ptab32 = nullptr;
  int pn_g = 0;
  double pd_inv_g = 0;
  int st32_cfg = -1;            // forced complex64 kernel configuration (-1: automatic)
  int op_weights = 0;           // HX_WEIGHTS_GA / HX_WEIGHTS_GAM (hx_set_operator_form)
  int op_mass_form = 2;         // 2 or 1 (hx_set_operator_form)
  const float* med_buoy = nullptr;   // hx_set_medium: caller-owned device arrays
  const float* med_invq = nullptr;
  std::map<std::string, int> tuned;   // hx_autotune choices by grid size and nrhs
  // cached levels, keyed by their defining parameters
  std::map<std::string, std::unique_ptr<hx::Level>> levels;
  std::list<std::string> lru;
  std::map<std::string, std::unique_ptr<hx::Solver>> solvers;
  std::list<std::string> solver_lru;
  int max_solvers = 8;          // solver workspaces kept (least recently used go first)
  // stream the solver runs on, and the events ordering it with the caller's
  cudaStream_t work_stream = nullptr;
  cudaEvent_t order_ev[2] = {nullptr, nullptr};
  // profiler (hx_profile): per-class launch count, time, algorithmic bytes
  bool prof_on = false;
  long long prof_launch_base = 0;
  struct ProfStat {
    long long launches = 0;
    double ms = 0, bytes = 0;
  } prof[4];
  struct ProfPending {
    int kind;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<ProfPending> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  // hx_apply_batched: device copy of the plan, pinned staging, and the event
  // after which the staging may be rewritten
  void* grp_dev = nullptr;
  size_t grp_dev_bytes = 0;
  void* grp_host = nullptr;
  size_t grp_host_bytes = 0;
  cudaEvent_t grp_ev = nullptr;

  ~hx_ctx();
};

namespace hx {

int fail(hx_ctx* ctx, int code, const std::string& msg);
inline std::string tune_key(int nx, int ny, int nz, int nrhs) {
  return std::to_string(nx) + "x" + std::to_string(ny) + "x" + std::to_string(nz) + "r" + std::to_string(nrhs);
}
// complex64 kernel configuration for a launch on ctx (forced, tuned, or -1);
// sweep: a residual / Jacobi sweep (tuned apart from y = A x)
int ctx_cfg32(const hx_ctx* ctx, int nx, int ny, int nz, int nrhs, bool sweep = false);
// autotuner core (hx_tune.cu): times the configurations on level lv with
// caller-owned buffers and records the fastest for (level size, nrhs)
int tune_cfg32(hx_ctx* ctx, const Level& lv, const float* v_dev, int nrhs, const void* x, void* y,
               long long pitch, int ncalls, cudaStream_t s, int* best_cfg, double* ms_out, int ms_cap);
int cuda_fail(hx_ctx* ctx, cudaError_t e, const char* where);
int check_grid(hx_ctx* ctx, const hx_grid* g);
// Level for grid g evaluated at spacing h_level with n_level nodes per axis
// (level 0: the grid itself).  Returned pointer is owned by ctx.
// gamma_cap > 0 caps the PML damping at gamma <= gamma_cap * omega (used by the
// multigrid preconditioner); 0 = the grid's own profile.
int get_level(hx_ctx* ctx, const hx_grid* g, const int n_level[3], double h_level, Level** out,
              double gamma_cap = 0.0);
template <typename T>
OpDesc<T> make_desc(const hx_ctx* ctx, const Level& lv, const float* v, double beta, bool precond = false);

// Profiler helpers: open/close an event pair around a launch of class `kind`
// (no-ops when profiling is off); collect() folds finished pairs into the
// counters (call after the stream is synchronised).
cudaEvent_t prof_begin(hx_ctx* ctx, cudaStream_t s);
void prof_end(hx_ctx* ctx, int kind, cudaEvent_t a, double bytes, cudaStream_t s);
void prof_collect(hx_ctx* ctx);


}  // namespace hx
