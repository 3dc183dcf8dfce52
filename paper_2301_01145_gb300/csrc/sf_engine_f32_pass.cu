// sf_engine_f32_pass.cu -- the general engine's per-pass kernel in FP32 (see sf_engine.cuh).
#define SF_ENGINE_INSTANTIATE
#include "sf_engine.cuh"

namespace sfg {
SF_ENGINE_EXPLICIT_PASS(float)
}  // namespace sfg
