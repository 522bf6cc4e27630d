// The compact variant of the persistent GMRES(m) kernel: FP32 inner precision,
// 2D operator, V streamed through bulk-copy stages, restart length m <= 47,
// compiled for two co-resident CTAs per SM (at most 128 registers per thread,
// smaller shared state), so twice the warps hide the latency of the stencil
// loads and of the stages.  Compiled on its own so the variants build in
// parallel.
#include "gmres_kernel.cuh"

namespace mlg {

cudaError_t launch_gmres_f2c(const KParams& kp, int grid, cudaStream_t s) {
  return launch_t<float, 2, kCompactM2, 256, kVBulk, 2>(kp, grid, s);
}

int max_blocks_f2c(int* bs, int extra) {
  return max_blocks_t<float, 2, kCompactM2, 256, kVBulk, 2>(bs, extra);
}

int own_bytes_f2c() { return (int)smem_own_bytes<float, kCompactM2, 256>(); }

}  // namespace mlg
