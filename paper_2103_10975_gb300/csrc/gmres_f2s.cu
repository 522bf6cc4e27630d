// One variant of the persistent GMRES(m) kernel (FP32 inner precision, 2D, V slices in shared memory),
// compiled on its own so that the variants build in parallel.
#include "gmres_kernel.cuh"

namespace mlg {

cudaError_t launch_gmres_f2s(const KParams& kp, int grid, cudaStream_t s) {
  return launch_t<float, 2, kMaxM, 256, kVShared>(kp, grid, s);
}

int max_blocks_f2s(int* bs) { return max_blocks_t<float, 2, kMaxM, 256, kVShared>(bs); }

}  // namespace mlg
