// sf_engine_f64.cu -- the general engine's kernels in FP64 (see sf_engine.cuh).
#define SF_ENGINE_INSTANTIATE
#include "sf_engine.cuh"

namespace sfg {
SF_ENGINE_EXPLICIT_EXEC(double)
SF_ENGINE_EXPLICIT_PASS(double)
}  // namespace sfg
