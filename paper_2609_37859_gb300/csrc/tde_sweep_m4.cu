// tde_sweep_m4.cu -- the sweep kernels of the 4-lane tile shape (160 threads per
// CTA, registers sized for 5 CTAs per SM), every direction and scheme variant.
#include "tde_sweep.cuh"

namespace tde {
cudaError_t sweep_launch_m4(const SweepArgs &a, int D, bool last, dim3 grid, size_t smem, cudaStream_t s) {
  return sweep_launch_shape<4, 160, 5>(a, D, last, grid, smem, s);
}
}  // namespace tde
