// Step kernels instantiated for iterates of type double and matrix values of type double.
#include "iter_launch.cuh"

namespace pdlp {
cudaError_t launch_iter_fp64(int which, int lanes, const IterRaw& r, cudaStream_t s) {
  return launch_iter_t<double, double, false>(which, lanes, r, s);
}
cudaError_t launch_persist_fp64(int lanes_a, int lanes_t, const IterRaw& r, int max_attempts,
                                  int grid, int* grid_out, cudaStream_t s) {
  return launch_persist_t<double, double, false>(lanes_a, lanes_t, r, max_attempts, grid, grid_out, s);
}
}  // namespace pdlp
