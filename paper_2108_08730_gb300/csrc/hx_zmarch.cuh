// Complex64 z-marching operator kernel on TMA-loaded planes (hx_zmarch.cu).
//
// Fields in this kernel's layout are complex64 [nrhs][nz][ny][pitch] with an
// even x-row pitch >= nx (16-byte rows), so a tile of a z-plane, halo
// included, is one cp.async.bulk.tensor copy.  hx_solve keeps its fine-level
// complex64 fields in that layout; public calls use it when nx is even or when
// the caller passes padded rows.
#pragma once

#include "hx_internal.h"

namespace hx {

// Launch configurations: rows per CTA (TY, one warp per row) x RHS per CTA.
struct ZCfgInfo {
  int ty, rb;
};
int zm_num_configs();
ZCfgInfo zm_config(int cfg);
int zm_default_config(int nrhs, int mode);

// y = A x (kApply), y = b - A x (kResidual; b may be null: y = -A x),
// y = x + omega_j D^-1 (b - A x) (kJacobi), y = omega_j D^-1 b (kJacobi0; x
// unused) for nrhs fields of row pitch `pitch` (even, >= nx; field stride
// pitch * ny * nz).  x, b: 16-byte aligned; y may not overlap x or b.
// err: device int set to 1 by a CTA whose bounded wait for a plane ran out
// (it then stops early); may be null.  cfg < 0: automatic.
cudaError_t launch_zmarch(const OpDesc<float>& op, int mode, int cfg, const void* x, const void* b, void* y,
                          int nrhs, long long pitch, double omega_j, int* err, cudaStream_t s);

}  // namespace hx
