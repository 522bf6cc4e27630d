// One variant of the persistent GMRES(m) kernel (FP32 inner precision, 3D, V streamed through bulk-copy stages),
// compiled on its own so that the variants build in parallel.
#include "gmres_kernel.cuh"

namespace mlg {

cudaError_t launch_gmres_f3b(const KParams& kp, int grid, cudaStream_t s) {
  return launch_t<float, 3, kMaxM, 256, kVBulk>(kp, grid, s);
}

int max_blocks_f3b(int* bs) { return max_blocks_t<float, 3, kMaxM, 256, kVBulk>(bs); }

}  // namespace mlg
