// Internal declarations shared by the translation units of libhx27.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hx27.h"

namespace hx {

// Derived per-table-node quantities (all linear in the 7 weights, so
// interpolating them equals deriving them from the interpolated weights):
//   0..3  stiffness class coefficients times h^2 of an interior row
//         (centre, face, edge, corner): -6 t0, t0 - ws2/3, ws2/6 - ws3/4, 3 ws3/8
//   4..7  per-point mass weights wm1..wm4
//   8..10 transverse-average weights t0 = ws1 + 2ws2/3 + ws3/2, t1 = ws2/12,
//         t2 = ws3/8 of the stiffness  S = sum_d T_d[delta_d p]
constexpr int kTabW = 12;

int build_weight_table(const double* theta_deg, int n_theta, const double* phi_deg, int n_phi,
                       double inv_g_max, double d_inv_g, double lambda, double* out, int capacity,
                       int* n_g_out, std::string* err);

int fit_joint_weights(const double* inv_g, int n, const double* theta_deg, int n_theta, const double* phi_deg,
                      int n_phi, double* w7, std::string* err);

// Per-level operator description handed to the kernels (device pointers).
template <typename T>
struct OpDesc {
  int nx, ny, nz;
  const float* v;          // velocity [nz][ny][nx]
  const T* tab;            // [n_g][kTabW]
  int n_g;
  T u_scale;               // f h / d_inv_g  ->  table coordinate u = u_scale / v
  T omega2;                // omega^2
  T beta;                  // CSL shift
  T inv_h2;                // 1 / h^2
  const T* axis[3];        // per axis: [n][4] = (up.re, up.im, dn.re, dn.im)
  int plain_lo[3], plain_hi[3];  // nodes whose up = dn = 1/h^2 exactly
  int cfg32 = -1;          // complex64 kernel configuration (-1: automatic)
  // operator variants (Section 3.1 GAm weights, first mass form of Eq. 8);
  // descriptors with either set run on the one-thread-per-row kernels
  int xshift = 0;          // complex64 kernel: x-tile origin at -xshift (st32_xshift)
  int gam = 0;             // 1: row weights = mean over the in-grid stencil points
  int mass1 = 0;           // 1: mass term with omega^2 / v_j^2 at each stencil point
  // heterogeneous medium (Eq. 2): buoyancy b = 1/rho and 1/Q per node of this
  // grid, or null (b = 1, no attenuation); set only on the operator itself
  const float* buoy = nullptr;
  const float* invq = nullptr;
  // x-row pitch (elements) of the complex fields this descriptor is launched
  // on; 0 = nx (fields back to back).  An even pitch (16-byte rows) selects
  // the TMA complex64 kernel (hx_zmarch.cu).
  long long pitch = 0;
};

enum StencilMode { kApply = 0, kResidual = 1, kJacobi = 2, kJacobi0 = 3 };

// Launch y = A x (kApply), y = b - A x (kResidual; b == nullptr means b = 0),
// y = x + omega_j D^{-1} (b - A x) (kJacobi) or y = omega_j D^{-1} b
// (kJacobi0, the first sweep from x = 0; x is not read) for nrhs fields of
// stride `rstride` elements.  Returns a cudaError_t.
template <typename T>
cudaError_t launch_stencil(const OpDesc<T>& op, int mode, const void* x, const void* b, void* y,
                           int nrhs, long long rstride, double omega_j, cudaStream_t s);

// Complex64 z-marching kernel (hx_stencil32.cu) for kApply / kResidual /
// kJacobi; cfg selects rows-per-thread and RHS-per-CTA (st32_num_configs()).
int st32_num_configs();
cudaError_t launch_stencil32(const OpDesc<float>& op, int mode, int cfg, const void* x, const void* b,
                             void* y, int nrhs, long long rstride, double omega_j, cudaStream_t s);
// Origin shift of the complex64 kernel's 32-wide x-tiles: the shift in
// [0, 32 ceil(nx/32) - nx] (so the tile count is unchanged) that leaves the
// fewest tiles holding x-PML columns; such tiles take the general PML form.
int st32_xshift(const OpDesc<float>& op);
// Automatic choice of the complex64 configuration for nrhs fields.
int st32_default_config(int nrhs);

// Grouped complex64 apply (one persistent launch over problems of different
// sizes): per-problem descriptor and work item of the persistent kernel.
struct GroupProb {
  OpDesc<float> op;
  const void* x;      // complex64 [nrhs][nz][ny][nx]
  void* y;
  int nrhs, zchunk;   // zchunk: set by st32_group_plan
  long long rstride;
};
struct GroupItem {
  int prob, bx, by, bz;   // problem, tile x, tile y, z-chunk * RHS blocks + RHS block
};
int st32_config_rhs(int cfg);
// Chooses each problem's z-chunk and lists the work items (largest problems first).
void st32_group_plan(GroupProb* probs, int n, int cfg, std::vector<GroupItem>& items);
// probs_dev / items_dev: device copies of the plan; counter_dev: one int of
// device scratch (reset here).  Configurations as for launch_stencil32.
cudaError_t launch_stencil32_group(int cfg, const GroupProb* probs_dev, const GroupItem* items_dev, int nitems,
                                   int* counter_dev, cudaStream_t s);

cudaError_t launch_row_coefficients(const OpDesc<double>& op, double* coef, cudaStream_t s);

// Complex64 launch configurations visible through the C ABI: ids 0..2 are the
// cp.async z-marching kernel (any nx; RHS per CTA 1, 2, 4), ids 3.. the TMA
// kernel (even row pitch; hx_zmarch.cu's list shifted by kZmCfgBase).
constexpr int kZmCfgBase = 3;
int cfg32_count();
// Row pitch a descriptor's fields use (op.pitch, or nx).
template <typename T>
inline long long field_pitch(const OpDesc<T>& op) { return op.pitch > 0 ? op.pitch : op.nx; }
// Device flag set by a TMA-kernel CTA whose bounded wait ran out (read and
// cleared by zm_take_error; 0 when none).
int zm_take_error(int device);
int* zm_error_flag(int device);

// Kernels launched by the library in this process (every launcher counts).
long long launch_count();
void count_launch(int n);

}  // namespace hx
