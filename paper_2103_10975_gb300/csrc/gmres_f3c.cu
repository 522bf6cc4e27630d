// The compact variant for the 3D variable-coefficient operator: FP32 inner
// precision, V streamed through bulk-copy stages, two co-resident CTAs per
// SM (at most 128 registers per thread); restart lengths up to the bucket
// limit 55 whose stage of m rows fits next to the 3D shared state (all of
// them on GB300, the triangle R being in global memory).  Compiled on its own
// so the variants build in parallel.
#include "gmres_kernel.cuh"

namespace mlg {

cudaError_t launch_gmres_f3c(const KParams& kp, int grid, cudaStream_t s) {
  return launch_t<float, 3, kCompactM3, 256, kVBulk, 2>(kp, grid, s);
}

int max_blocks_f3c(int* bs, int extra) {
  return max_blocks_t<float, 3, kCompactM3, 256, kVBulk, 2>(bs, extra);
}

int own_bytes_f3c() { return (int)smem_own_bytes<float, kCompactM3, 256>(); }

}  // namespace mlg
