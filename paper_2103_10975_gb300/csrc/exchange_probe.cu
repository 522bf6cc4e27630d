// Latency floor of the persistent solver's Arnoldi step: the same cooperative
// launch, one CTA of 256 threads per SM, and per step the same two group
// exchanges as gmres_persistent (the CTA's partial sums of j+2 slots, the
// group barrier, the gather of the j+2 sums in the same fixed order), with the
// passes over the grid and the scalar recurrences left out.  Timing the real
// kernel against it shows what share of a step the exchanges take.
#include "../../include/mlgmres.h"
#include "gmres_kernel.cuh"

namespace mlg {
namespace {

constexpr int kBS = 256;
constexpr int kLW = kMaxM + 2;
using ProbeSmem = Smem<float, kMaxM, kBS>;
// dynamic shared memory per CTA: more than half an SM's, so that (like the
// solver) exactly one CTA lands on each SM
constexpr int kProbeSmem = 160 * 1024;
static_assert(sizeof(ProbeSmem) <= kProbeSmem, "probe state exceeds its shared memory");

__global__ void __launch_bounds__(kBS, 1)
    exchange_floor_kernel(int m, int steps, double* part, int ps, GroupBarrier gb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ProbeSmem& sm = *reinterpret_cast<ProbeSmem*>(smem_raw);
  const int lb = blockIdx.x, nb = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long epoch = 0;
  int red = 0;
  auto P = [&]() { return (float*)(part + (long long)(red & 1) * kLW * ps); };
  int j = 0;
  for (int s = 0; s < steps; s++) {
    const int L = j + 2;
    // what a pass leaves behind: every warp's partial of each slot
    for (int k = lane; k < L; k += 32) sm.red[warp][k] = (float)(k + warp);
    // X exchange (warp 1 is free during it, as when it rotates a column)
    finish_and_sync_side<kLW, kBS, float>(L, P(), lb, sm.red, ps, gb, epoch, &sm.flag,
                                          NoSide());
    gather<kBS, float, float, true>(P(), L, nb, sm.tot, sm.coef, ps);
    if (!sm.flag) break;
    red++;
    for (int k = lane; k < L; k += 32) sm.red[warp][k] = (float)(k - warp);
    // Y exchange
    if (!finish_and_sync<kLW, kBS, float>(L, P(), lb, sm.red, ps, gb, epoch, &sm.flag, NoSide()))
      break;
    gather<kBS, float, float>(P(), L, nb, sm.tot, sm.coef, ps);
    red++;
    j = j + 1 == m ? 0 : j + 1;
  }
}

}  // namespace
}  // namespace mlg

extern "C" mlgmres_status mlgmres_exchange_floor(int ctas, int m, int steps, float* us_per_step) {
  using namespace mlg;
  if (!us_per_step || m < 1 || m > kMaxM || steps < 1 || ctas < 1 || ctas > kPartStride)
    return MLGMRES_ERR_ARG;
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MLGMRES_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MLGMRES_ERR_CUDA;
  if (cudaFuncSetAttribute(exchange_floor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kProbeSmem) != cudaSuccess)
    return MLGMRES_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, exchange_floor_kernel, kBS,
                                                    kProbeSmem) != cudaSuccess)
    return MLGMRES_ERR_CUDA;
  if (ctas > per * nsm) return MLGMRES_ERR_ARG;
  double* part = nullptr;
  unsigned long long* ctr = nullptr;
  int* err = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mlgmres_status st = MLGMRES_OK;
  float ms = 0.f;
  int herr = 0;
  GroupBarrier gb;
  if (cudaMalloc(&part, sizeof(double) * part_doubles(ctas)) != cudaSuccess ||
      cudaMalloc(&ctr, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&err, sizeof(int)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = MLGMRES_ERR_CUDA;
    goto done;
  }
  gb.ctr = ctr;
  gb.err = err;
  gb.nblocks = (unsigned)ctas;
  gb.timeout_ns = 2000000000ull;
  for (int rep = 0; rep < 2 && st == MLGMRES_OK; rep++) {  // the first launch warms up
    if (cudaMemset(ctr, 0, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(err, 0, sizeof(int)) != cudaSuccess) {
      st = MLGMRES_ERR_CUDA;
      break;
    }
    int pm = m, ps_ = ctas, nsteps = steps;
    void* args[] = {(void*)&pm, (void*)&nsteps, (void*)&part, (void*)&ps_, (void*)&gb};
    cudaEventRecord(e0, 0);
    note_launches(1);
    if (cudaLaunchCooperativeKernel((const void*)exchange_floor_kernel, dim3(ctas), dim3(kBS),
                                    args, kProbeSmem, 0) != cudaSuccess) {
      st = MLGMRES_ERR_CUDA;
      break;
    }
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess ||
        cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      st = MLGMRES_ERR_CUDA;
      break;
    }
    if (herr != kErrNone) st = MLGMRES_ERR_TIMEOUT;
    cudaEventElapsedTime(&ms, e0, e1);
  }
  if (st == MLGMRES_OK) *us_per_step = 1000.f * ms / (float)steps;
done:
  cudaFree(part);
  cudaFree(ctr);
  cudaFree(err);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}
