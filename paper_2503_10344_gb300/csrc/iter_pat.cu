// Step kernels instantiated for iterates of type float and matrix values of type Pattern.
#include "iter_launch.cuh"

namespace pdlp {
cudaError_t launch_iter_pat(int which, int lanes, const IterRaw& r, cudaStream_t s) {
  return launch_iter_t<float, Pattern, true>(which, lanes, r, s);
}
}  // namespace pdlp
