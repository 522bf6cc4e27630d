// The compact variant with V slices in shared memory: FP32 inner precision,
// 2D operator, restart length m <= 47, two co-resident CTAs per SM, each with
// a slice of V next to its smaller shared state (grids whose slices fit at
// twice the CTA count, e.g. 256^2 at 256 CTAs).  Compiled on its own so the
// variants build in parallel.
#include "gmres_kernel.cuh"

namespace mlg {

cudaError_t launch_gmres_f2cs(const KParams& kp, int grid, cudaStream_t s) {
  return launch_t<float, 2, kCompactM2, 256, kVShared, 2>(kp, grid, s);
}

}  // namespace mlg
