// sf_engine_f32_exec.cu -- the general engine's persistent executor in FP32 (see sf_engine.cuh).
#define SF_ENGINE_INSTANTIATE
#include "sf_engine.cuh"

namespace sfg {
SF_ENGINE_EXPLICIT_EXEC(float)
}  // namespace sfg
