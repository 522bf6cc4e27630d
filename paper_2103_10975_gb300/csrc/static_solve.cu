// mlgmres_solve_static: the persistent GMRES(m) solve without any device
// allocation, for callers that cannot allocate device memory themselves or
// through this library -- for example code running inside a memory pool that
// owns all of the GPU's free memory, or a process whose allocator must not be
// entered while it solves.  Its workspace is one fixed array compiled into the
// library (kStaticBytes, held by every GPU that loads the library until the
// process exits).
#include <mutex>
#include <string.h>

#include "../../include/mlgmres.h"
#include "solver.h"

namespace mlg {

// Largest problem the fixed workspace holds: a 2D grid of up to 256 x 256
// points with m <= 32, in FP32-refined precision.
constexpr int kStaticMaxN = 256 * 256;
constexpr int kStaticMaxM = 32;
constexpr long long kStaticLdv = kStaticMaxN;  // a multiple of 64
constexpr size_t kStaticBasis = sizeof(float) * (size_t)vrows_p(kStaticMaxM + 1) * kStaticLdv;
constexpr size_t kStaticWork = 2 * sizeof(float) * (size_t)kStaticLdv;
constexpr size_t kStaticPart = sizeof(double) * part_doubles(kPartStride);
constexpr size_t kStaticMisc = 4096;  // barrier counter, error flag, result, launch tables
constexpr size_t kStaticBytes = kStaticBasis + kStaticWork + kStaticPart + kStaticMisc;

// The fixed workspace.  In host code this name is only a stand-in for the
// symbol; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

namespace {

constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;  // host threads calling for the first time on a device

// Device address of the workspace on the current device (looked up once per
// device, the first time that device calls mlgmres_solve_static).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = (unsigned char*)p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace mlg

using namespace mlg;

extern "C" mlgmres_status mlgmres_solve_static(int n, int m, double rtol, long long max_iters,
                                               const double* b_dev, double* x_dev, void* stream,
                                               mlgmres_result* res) {
  if (res) memset(res, 0, sizeof(*res));
  if (n < 1 || (long long)n * n > kStaticMaxN || m < 1 || m > kStaticMaxM)
    return MLGMRES_ERR_ARG;  // larger than the fixed workspace
  if (!(rtol > 0.0 && rtol < 1.0) || max_iters <= 0 || !b_dev || !x_dev || b_dev == x_dev)
    return MLGMRES_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return MLGMRES_ERR_CUDA;

  // carve the fixed workspace
  unsigned char* p = base;
  float* V = (float*)p;
  p += kStaticBasis;
  float* W0 = (float*)p;
  float* W1 = W0 + kStaticLdv;
  p += kStaticWork;
  double* part = (double*)p;
  p += kStaticPart;
  unsigned long long* bar = (unsigned long long*)p;
  int* err = (int*)(p + 8);
  DevResult* dres = (DevResult*)(p + 64);
  int* cfg = (int*)(p + 256);                 // group_first[2], task_first[2], task_order[1]
  SolveTask* task = (SolveTask*)(p + 512);
  GroupWork* work = (GroupWork*)(p + 1024);

  const int N = n * n;
  int bs = 0;
  const int maxb = gmres_max_blocks(true, 2, m, &bs);
  if (maxb < 1) return MLGMRES_ERR_CUDA;
  long long want = (N + 511) / 512;
  int blocks = (int)(want < 1 ? 1 : (want > maxb ? maxb : want));
  if (blocks > kPartStride) blocks = kPartStride;

  int hcfg[5] = {0, blocks, 0, 1, 0};
  SolveTask t;
  t.n = n;
  t.N = N;
  t.b = b_dev;
  t.x = x_dev;
  t.x_alt = nullptr;
  t.kappa = nullptr;
  t.res = dres;
  t.hist = nullptr;
  t.hist_cap = 0;
  t.zero_x = 0;
  GroupWork w;
  w.V = V;
  w.ldv = kStaticLdv;
  w.W0 = W0;
  w.W1 = W1;
  w.part = part;
  w.pstride = kPartStride;
  w.Rg = nullptr;
  w.bar.ctr = bar;
  w.bar.err = err;
  w.bar.nblocks = (unsigned)blocks;
  w.bar.timeout_ns = 2000000000ull;
  // the guess is zero; the counter and flag must start at zero on every call
  if (cudaMemsetAsync(x_dev, 0, sizeof(double) * N, s) != cudaSuccess ||
      cudaMemsetAsync(bar, 0, 64, s) != cudaSuccess ||
      cudaMemcpyAsync(cfg, hcfg, sizeof(hcfg), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(task, &t, sizeof(t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(work, &w, sizeof(w), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return MLGMRES_ERR_CUDA;
  KParams kp;
  kp.m = m;
  kp.rtol = rtol;
  kp.max_iters = max_iters;
  kp.arnoldi_steps = 0;
  kp.vsmem = 0;
  kp.bulk_stages = 0;
  kp.bulk_cap = 0;
  kp.vmode = kVDirect;
  kp.compact = 0;
  kp.ngroups = 1;
  kp.group_first = cfg;
  kp.task_first = cfg + 2;
  kp.task_order = cfg + 4;
  kp.tasks = task;
  kp.work = work;
  if (launch_gmres(kp, true, 2, blocks, s) != cudaSuccess) return MLGMRES_ERR_CUDA;
  DevResult r;
  if (cudaMemcpyAsync(&r, dres, sizeof(r), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MLGMRES_ERR_CUDA;
  mlgmres_status st;
  switch (r.status) {
    case 0: st = MLGMRES_OK; break;
    case 1: st = MLGMRES_NOT_CONVERGED; break;
    case kErrTimeout: st = MLGMRES_ERR_TIMEOUT; break;
    case kErrNonfinite: st = MLGMRES_ERR_NONFINITE; break;
    default: st = MLGMRES_ERR_CUDA; break;
  }
  if (res) {
    res->iters = r.iters;
    res->cycles = r.cycles;
    res->status = st;
    res->guess_used = MLGMRES_GUESS_ZERO;
    res->bnorm = r.bnorm;
    res->relres_true = r.relres_true;
    res->relres_first_cycle = r.relres_first_cycle;
    res->relres_guess = r.relres_guess;
    res->relres_learned = -1.0;
  }
  return st;
}
