// sf_engine.cuh -- host entry points of the general engine's two kernels
// (k_pass: one launch per pass; k_exec: the persistent executor, sf_kernels.cuh).
//
// The kernels are instantiated in translation units of their own
// (sf_engine_f32_exec.cu, sf_engine_f32_pass.cu, sf_engine_f64.cu), so that
// the library builds in parallel; the host runtime (sf_api.cu) launches them
// only through these functions.
#pragma once

#include "sf_kernels.cuh"

namespace sfg {

// raise the dynamic shared-memory limit of each kernel to the engine's budget
template <typename T> cudaError_t engine_set_attrs_exec();
template <typename T> cudaError_t engine_set_attrs_pass();
template <typename T> cudaError_t engine_set_attrs() {
  const cudaError_t e = engine_set_attrs_exec<T>();
  return e != cudaSuccess ? e : engine_set_attrs_pass<T>();
}
// resident CTAs per SM of the persistent executor with smem bytes of dynamic shared memory
template <typename T> cudaError_t engine_exec_occupancy(int *per_sm, size_t smem);
// the persistent executor over a whole pass list
template <typename T>
cudaError_t engine_launch_exec(int grid, size_t smem, cudaStream_t st, const Prob<T> *probs, const Pass<T> *passes,
                               const int *pass_start, int npass, unsigned *done, ExecCtl *ctl, unsigned *sticky,
                               unsigned long long timeout_ns, const IOArgs<T> &io);
// one pass (its tiles as the grid)
template <typename T>
cudaError_t engine_launch_pass(int ntiles, size_t smem, cudaStream_t st, const Prob<T> *probs, const Pass<T> *passes,
                               int pass_idx, const IOArgs<T> &io);

// definitions, compiled only where SF_ENGINE_INSTANTIATE is set
#ifdef SF_ENGINE_INSTANTIATE
template <typename T> cudaError_t engine_set_attrs_exec() {
  return cudaFuncSetAttribute(k_exec<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}
template <typename T> cudaError_t engine_set_attrs_pass() {
  return cudaFuncSetAttribute(k_pass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}
template <typename T> cudaError_t engine_exec_occupancy(int *per_sm, size_t smem) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_exec<T>, SF_THREADS, smem);
}
template <typename T>
cudaError_t engine_launch_exec(int grid, size_t smem, cudaStream_t st, const Prob<T> *probs, const Pass<T> *passes,
                               const int *pass_start, int npass, unsigned *done, ExecCtl *ctl, unsigned *sticky,
                               unsigned long long timeout_ns, const IOArgs<T> &io) {
  k_exec<T><<<grid, SF_THREADS, smem, st>>>(probs, passes, pass_start, npass, done, ctl, sticky, timeout_ns, io);
  return cudaGetLastError();
}
template <typename T>
cudaError_t engine_launch_pass(int ntiles, size_t smem, cudaStream_t st, const Prob<T> *probs, const Pass<T> *passes,
                               int pass_idx, const IOArgs<T> &io) {
  k_pass<T><<<ntiles, SF_THREADS, smem, st>>>(probs, passes, pass_idx, io);
  return cudaGetLastError();
}
// the persistent executor and the per-pass kernel of one precision, for
// translation units of their own
#define SF_ENGINE_EXPLICIT_EXEC(T)                                                                                    \
  template cudaError_t engine_set_attrs_exec<T>();                                                                    \
  template cudaError_t engine_exec_occupancy<T>(int *, size_t);                                                       \
  template cudaError_t engine_launch_exec<T>(int, size_t, cudaStream_t, const Prob<T> *, const Pass<T> *, const int *, \
                                             int, unsigned *, ExecCtl *, unsigned *, unsigned long long,              \
                                             const IOArgs<T> &);
#define SF_ENGINE_EXPLICIT_PASS(T)                                                                                    \
  template cudaError_t engine_set_attrs_pass<T>();                                                                    \
  template cudaError_t engine_launch_pass<T>(int, size_t, cudaStream_t, const Prob<T> *, const Pass<T> *, int,         \
                                             const IOArgs<T> &);
#endif

}  // namespace sfg
