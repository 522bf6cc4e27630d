// The shared-slice variant (FP32 inner precision, 2D, V slices in shared
// memory) instantiated for restart lengths m <= 32: four buckets of j instead
// of eight, so less code for the instruction cache and a smaller shared state
// (1.8% less time per Arnoldi step than the m <= 64 instantiation at 256^2,
// GMRES(30), 128 CTAs).  Compiled on its own so the variants build in parallel.
#include "gmres_kernel.cuh"

namespace mlg {

cudaError_t launch_gmres_f2s32(const KParams& kp, int grid, cudaStream_t s) {
  return launch_t<float, 2, kSmallM, 256, kVShared>(kp, grid, s);
}

}  // namespace mlg
