// One variant of the persistent GMRES(m) kernel (FP64, 3D, V in HBM loaded by the passes),
// compiled on its own so that the variants build in parallel.
#include "gmres_kernel.cuh"

namespace mlg {

cudaError_t launch_gmres_d3d(const KParams& kp, int grid, cudaStream_t s) {
  return launch_t<double, 3, kMaxM, 256, kVDirect>(kp, grid, s);
}

int max_blocks_d3d(int* bs) { return max_blocks_t<double, 3, kMaxM, 256, kVDirect>(bs); }

}  // namespace mlg
