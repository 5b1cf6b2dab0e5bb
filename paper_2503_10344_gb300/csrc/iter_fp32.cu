// Step kernels instantiated for iterates of type float and matrix values of type float.
#include "iter_launch.cuh"

namespace pdlp {
cudaError_t launch_iter_fp32(int which, int lanes, const IterRaw& r, cudaStream_t s) {
  return launch_iter_t<float, float, false>(which, lanes, r, s);
}
}  // namespace pdlp
