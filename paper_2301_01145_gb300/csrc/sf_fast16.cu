// sf_fast16.cu -- instantiation of the register fast path for L = 512 (E = 16).
#include "sf_fast.cuh"

namespace sfg {

int sf_fast_launch_e16(const FastLaunch &fl, const IOArgs<float> &io, int *launches) {
  const bool pad = fl.h_prob->ax[0].kind == AK_U;  // all axes unbounded (doubled) or all periodic
  return pad ? fast_launch_all<16, true>(fl, io, launches) : fast_launch_all<16, false>(fl, io, launches);
}

}  // namespace sfg
