// Halpern-variant step kernels instantiated for iterates of type float and matrix values
// of type Pattern (a unit of its own so that the library's units compile in parallel).
#include "iter_launch.cuh"

namespace pdlp {
cudaError_t launch_iter_pat_h(int which, int lanes, const IterRaw& r, cudaStream_t s) {
  return launch_iter_t<float, Pattern, true, true>(which, lanes, r, s);
}
}  // namespace pdlp
