// Step kernels instantiated for iterates of type float and matrix values of type __nv_bfloat16.
#include "iter_launch.cuh"

namespace pdlp {
cudaError_t launch_iter_bf16(int which, int lanes, const IterRaw& r, cudaStream_t s) {
  return launch_iter_t<float, __nv_bfloat16, true>(which, lanes, r, s);
}
cudaError_t launch_persist_bf16(int lanes_a, int lanes_t, const IterRaw& r, int max_attempts,
                                  int grid, int* grid_out, cudaStream_t s) {
  return launch_persist_t<float, __nv_bfloat16, true>(lanes_a, lanes_t, r, max_attempts, grid, grid_out, s);
}
cudaError_t tile_resident_bf16(int form, int* primal_blocks, int* dual_blocks) {
  const cudaError_t e = tile_resident<__nv_bfloat16, true, false>(form, primal_blocks);
  return e != cudaSuccess ? e : tile_resident<__nv_bfloat16, true, true>(form, dual_blocks);
}
}  // namespace pdlp
