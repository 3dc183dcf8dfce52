// sf_fast8.cu -- instantiation of the register fast path for L = 256 (E = 8).
#include "sf_fast.cuh"

namespace sfg {

int sf_fast_launch_e8(const FastLaunch &fl, const IOArgs<float> &io, int *launches) {
  const bool pad = fl.h_prob->ax[0].kind == AK_U;  // all axes unbounded (doubled) or all periodic
  return pad ? fast_launch_all<8, true>(fl, io, launches) : fast_launch_all<8, false>(fl, io, launches);
}

}  // namespace sfg
