// Halpern-variant step kernels instantiated for iterates of type double and matrix values
// of type double (a unit of its own so that the library's units compile in parallel).
#include "iter_launch.cuh"

namespace pdlp {
cudaError_t launch_iter_fp64_h(int which, int lanes, const IterRaw& r, cudaStream_t s) {
  return launch_iter_t<double, double, false, true>(which, lanes, r, s);
}
}  // namespace pdlp
