// Host side of the persistent GMRES(m) solver (the kernel and its passes are
// in gmres_kernel.cuh): variant dispatch, shared-memory budgets, and the FP64
// operator and basis-conversion kernels used for inspection.
#include "gmres_kernel.cuh"

namespace mlg {

// Variant table: 256-thread CTAs (the register budget of 255 per thread keeps the
// V column and the dot accumulators of a pass in registers); the passes are
// instantiated per bucket of j, so one variant per precision and dimension,
// each in its own translation unit (gmres_{f,d}{2,3}.cu).
cudaError_t launch_gmres_f2(const KParams& kp, int grid, cudaStream_t s);
cudaError_t launch_gmres_f3(const KParams& kp, int grid, cudaStream_t s);
cudaError_t launch_gmres_d2(const KParams& kp, int grid, cudaStream_t s);
cudaError_t launch_gmres_d3(const KParams& kp, int grid, cudaStream_t s);
int max_blocks_f2(int* bs);
int max_blocks_f3(int* bs);
int max_blocks_d2(int* bs);
int max_blocks_d3(int* bs);

cudaError_t launch_gmres(const KParams& kp, bool fp32, int dim, int grid, cudaStream_t s) {
  if (fp32) return dim == 2 ? launch_gmres_f2(kp, grid, s) : launch_gmres_f3(kp, grid, s);
  return dim == 2 ? launch_gmres_d2(kp, grid, s) : launch_gmres_d3(kp, grid, s);
}

int gmres_max_blocks(bool fp32, int dim, int m, int* bs) {
  (void)m;
  if (fp32) return dim == 2 ? max_blocks_f2(bs) : max_blocks_f3(bs);
  return dim == 2 ? max_blocks_d2(bs) : max_blocks_d3(bs);
}

bool gmres_stages_fit(int m, int P) {
  return P >= 0 && P <= kMaxStages && 4LL * 8 * P * m * 32 <= gmres_vsmem_budget(true);
}

int gmres_bulk_stages(bool fp32, int m) {
  // two stages measured fastest on GB300 at 1024^2 and 2048^2 (m = 40) and
  // 192^3 (m = 50): 662 against 880 (three) and 860 (direct) us per step at 2048^2
  if (!fp32) return 0;
  return gmres_stages_fit(m, 2) ? 2 : 0;
}

int gmres_vsmem_budget(bool fp32) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int own = fp32 ? (int)smem_own_bytes<float, kMaxM, 256>()
                       : (int)smem_own_bytes<double, kMaxM, 256>();
  const int left = optin - own - 1024;
  return left > 0 ? left : 0;
}

// FP64 A u, one thread per point.
template <int DIM>
__global__ void apply_kernel(int n, int N, const float* kappa, const double* u, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double h = 2.0 / (n + 1);
  out[i] = stencil<double, DIM>(u, i, n, kappa, u[i]) / (h * h);
}

cudaError_t launch_apply(int dim, int n, const float* kappa, const double* u, double* out,
                         cudaStream_t s) {
  const int N = dim == 2 ? n * n : n * n * n;
  const int bs = 256, gr = (N + bs - 1) / bs;
  note_launches(1);
  if (dim == 2)
    apply_kernel<2><<<gr, bs, 0, s>>>(n, N, kappa, u, out);
  else
    apply_kernel<3><<<gr, bs, 0, s>>>(n, N, kappa, u, out);
  return cudaGetLastError();
}

template <typename T>
__global__ void basis_to_f64(const T* V, int vrows, int rows, int N, double* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)rows * N) return;
  const int r = (int)(i / N), c = (int)(i % N);
  out[i] = (double)V[vix(r, c, vrows)];
}

cudaError_t launch_basis_to_f64(bool fp32, const void* V, int vrows, int rows, int N,
                                double* out, cudaStream_t s) {
  const long long tot = (long long)rows * N;
  const int bs = 256;
  const unsigned gr = (unsigned)((tot + bs - 1) / bs);
  note_launches(1);
  if (fp32)
    basis_to_f64<float><<<gr, bs, 0, s>>>((const float*)V, vrows, rows, N, out);
  else
    basis_to_f64<double><<<gr, bs, 0, s>>>((const double*)V, vrows, rows, N, out);
  return cudaGetLastError();
}

}  // namespace mlg
