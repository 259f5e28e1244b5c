// tde_sweep_m8.cu -- the sweep kernels of the 8-lane tile shape (288 threads per
// CTA, registers sized for 3 CTAs per SM), every direction and scheme variant.
#include "tde_sweep.cuh"

namespace tde {
cudaError_t sweep_launch_m8(const SweepArgs &a, int D, bool last, dim3 grid, size_t smem, cudaStream_t s) {
  return sweep_launch_shape<8, 288, 3>(a, D, last, grid, smem, s);
}
}  // namespace tde
