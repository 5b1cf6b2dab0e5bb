// Step kernels instantiated for iterates of type float and matrix values of type Pattern.
#include "iter_launch.cuh"

namespace pdlp {
cudaError_t launch_iter_pat(int which, int lanes, const IterRaw& r, cudaStream_t s) {
  return launch_iter_t<float, Pattern, true>(which, lanes, r, s);
}
cudaError_t launch_persist_pat(int lanes_a, int lanes_t, const IterRaw& r, int max_attempts,
                                  int grid, int* grid_out, cudaStream_t s) {
  return launch_persist_t<float, Pattern, true>(lanes_a, lanes_t, r, max_attempts, grid, grid_out, s);
}
cudaError_t tile_resident_pat(int form, int* primal_blocks, int* dual_blocks) {
  const cudaError_t e = tile_resident<Pattern, true, false>(form, primal_blocks);
  return e != cudaSuccess ? e : tile_resident<Pattern, true, true>(form, dual_blocks);
}
}  // namespace pdlp
