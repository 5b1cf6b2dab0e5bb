// Halpern-variant step kernels instantiated for iterates of type float and matrix values
// of type float (a unit of its own so that the library's units compile in parallel).
#include "iter_launch.cuh"

namespace pdlp {
cudaError_t launch_iter_fp32_h(int which, int lanes, const IterRaw& r, cudaStream_t s) {
  return launch_iter_t<float, float, false, true>(which, lanes, r, s);
}
}  // namespace pdlp
