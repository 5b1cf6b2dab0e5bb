// Step kernels instantiated for iterates of type double and matrix values of type double.
#include "iter_launch.cuh"

namespace pdlp {
cudaError_t launch_iter_fp64(int which, int lanes, const IterRaw& r, cudaStream_t s) {
  return launch_iter_t<double, double, false>(which, lanes, r, s);
}
}  // namespace pdlp
