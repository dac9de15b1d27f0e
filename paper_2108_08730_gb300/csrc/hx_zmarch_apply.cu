// Instantiations of the TMA z-marching kernel for mode kApply (see
// hx_zmarch_kernel.cuh); one translation unit per mode keeps the build parallel.
#include "hx_zmarch_kernel.cuh"

namespace hx {

cudaError_t zm_launch_apply(int cfg, const ZParams& P, bool shift, const CUtensorMap& xm, const CUtensorMap& bm,
                         int frame, int interior, cudaStream_t s) {
  switch (cfg) {
    case 0: return zm_launch_mode<kApply, 8, 1>(P, shift, xm, bm, frame, interior, s);
    case 1: return zm_launch_mode<kApply, 8, 2>(P, shift, xm, bm, frame, interior, s);
    case 2: return zm_launch_mode<kApply, 8, 4>(P, shift, xm, bm, frame, interior, s);
    case 3: return zm_launch_mode<kApply, 8, 8>(P, shift, xm, bm, frame, interior, s);
    case 4: return zm_launch_mode<kApply, 16, 2>(P, shift, xm, bm, frame, interior, s);
    case 5: return zm_launch_mode<kApply, 16, 4>(P, shift, xm, bm, frame, interior, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hx
