// Step kernels instantiated for iterates of type float and matrix values of type __nv_bfloat16.
#include "iter_launch.cuh"

namespace pdlp {
cudaError_t launch_iter_bf16(int which, int lanes, const IterRaw& r, cudaStream_t s) {
  return launch_iter_t<float, __nv_bfloat16, true>(which, lanes, r, s);
}
}  // namespace pdlp
