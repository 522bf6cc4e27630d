// One variant of the persistent GMRES(m) kernel (FP64, 3D, V streamed through bulk-copy stages),
// compiled on its own so that the variants build in parallel.
#include "gmres_kernel.cuh"

namespace mlg {

cudaError_t launch_gmres_d3b(const KParams& kp, int grid, cudaStream_t s) {
  return launch_t<double, 3, kMaxM, 256, kVBulk>(kp, grid, s);
}

int max_blocks_d3b(int* bs) { return max_blocks_t<double, 3, kMaxM, 256, kVBulk>(bs); }

}  // namespace mlg
