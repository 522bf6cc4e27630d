// Host side of the persistent GMRES(m) solver (the kernel and its passes are
// in gmres_kernel.cuh): variant dispatch, shared-memory budgets, and the FP64
// operator and basis-conversion kernels used for inspection.
#include "gmres_kernel.cuh"

namespace mlg {

// Variant table: 256-thread CTAs (the register budget of 255 per thread keeps the
// V column and the dot accumulators of a pass in registers); the passes are
// instantiated per bucket of j; one variant per precision, dimension and
// placement of V, each in its own translation unit (gmres_<variant>.cu).
#define MLG_VARIANT(tag)                                                \
  cudaError_t launch_gmres_##tag(const KParams& kp, int grid, cudaStream_t s); \
  int max_blocks_##tag(int* bs);
MLG_VARIANT(f2d)
MLG_VARIANT(f2s)
MLG_VARIANT(f2b)
MLG_VARIANT(f3d)
MLG_VARIANT(f3b)
MLG_VARIANT(d2d)
MLG_VARIANT(d2s)
MLG_VARIANT(d2b)
MLG_VARIANT(d3d)
MLG_VARIANT(d3b)
#undef MLG_VARIANT
cudaError_t launch_gmres_f2c(const KParams& kp, int grid, cudaStream_t s);
int max_blocks_f2c(int* bs, int extra);
int own_bytes_f2c();
cudaError_t launch_gmres_f3c(const KParams& kp, int grid, cudaStream_t s);
cudaError_t launch_gmres_f2cs(const KParams& kp, int grid, cudaStream_t s);
cudaError_t launch_gmres_f2s32(const KParams& kp, int grid, cudaStream_t s);
int max_blocks_f3c(int* bs, int extra);
int own_bytes_f3c();



int gmres_compact_cap(int dim, int m, int P) {
  if (P <= 0) return 0;
  int dev = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const int own = dim == 2 ? own_bytes_f2c() : own_bytes_f3c();
  const long long budget = (long long)per_sm / 2 - 1024 - own;  // per CTA
  const long long row = 32LL * 4;
  const long long share = budget / 8 / 128 * 128;
  // a stage: m rows of V and the X pass's w'/kappa windows
  const long long stage = (long long)vrows_p(m) * row + (dim == 2 ? Aux<float, 2>::kXBytes
                                                                   : Aux<float, 3>::kXBytes);
  const long long want = (long long)P * stage;
  const long long cap = want < share ? want : share;
  return cap >= stage ? (int)cap : 0;
}

bool gmres_compact_ok(bool fp32, int dim, int m) {
  // and one stage of m rows must fit in a warp's share (m <= 55 in 3D on GB300)
  return fp32 && (dim == 2 ? m < kCompactM2 : m < kCompactM3) && gmres_compact_cap(dim, m, 1) > 0;
}

int gmres_compact_vsmem_budget() {
  int dev = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const int left = per_sm / 2 - 1024 - own_bytes_f2c();
  return left > 0 ? left : 0;
}

int gmres_compact_max_blocks(int dim, int m) {
  int bs = 0;
  const int extra = 8 * gmres_compact_cap(dim, m, kMaxStages);
  return dim == 2 ? max_blocks_f2c(&bs, extra) : max_blocks_f3c(&bs, extra);
}

cudaError_t launch_gmres(const KParams& kp, bool fp32, int dim, int grid, cudaStream_t s) {
  if (dim == 3 && kp.vmode == kVShared) return cudaErrorInvalidValue;
  if (kp.compact) {
    if (!gmres_compact_ok(fp32, dim, kp.m) || kp.vmode == kVDirect ||
        (dim == 3 && kp.vmode == kVShared))
      return cudaErrorInvalidValue;
    if (dim == 2 && kp.vmode == kVShared) return launch_gmres_f2cs(kp, grid, s);
    return dim == 2 ? launch_gmres_f2c(kp, grid, s) : launch_gmres_f3c(kp, grid, s);
  }
  if (fp32) {
    if (dim == 2) {
      if (kp.vmode == kVShared)
        return kp.m <= kSmallM ? launch_gmres_f2s32(kp, grid, s) : launch_gmres_f2s(kp, grid, s);
      if (kp.vmode == kVBulk) return launch_gmres_f2b(kp, grid, s);
      return launch_gmres_f2d(kp, grid, s);
    }
    if (kp.vmode == kVBulk) return launch_gmres_f3b(kp, grid, s);
    return launch_gmres_f3d(kp, grid, s);
  }
  if (dim == 2) {
    if (kp.vmode == kVShared) return launch_gmres_d2s(kp, grid, s);
    if (kp.vmode == kVBulk) return launch_gmres_d2b(kp, grid, s);
    return launch_gmres_d2d(kp, grid, s);
  }
  if (kp.vmode == kVBulk) return launch_gmres_d3b(kp, grid, s);
  return launch_gmres_d3d(kp, grid, s);
}

// The co-resident limit of the direct variant (every variant runs one 256-thread
// CTA per SM: 255 registers per thread).
int gmres_max_blocks(bool fp32, int dim, int m, int* bs) {
  (void)m;
  if (fp32) return dim == 2 ? max_blocks_f2d(bs) : max_blocks_f3d(bs);
  return dim == 2 ? max_blocks_d2d(bs) : max_blocks_d3d(bs);
}

int gmres_bulk_cap(bool fp32, int m, int P) {
  if (P <= 0) return 0;
  const long long row = 32LL * (fp32 ? 4 : 8);                                  // bytes
  const long long share = (long long)gmres_vsmem_budget(fp32) / 8 / 128 * 128;  // per warp
  // a stage: m rows of V and the X pass's w'/kappa windows (the 3D size, the
  // larger of the two dimensions)
  const long long stage =
      (long long)vrows_p(m) * row + (fp32 ? Aux<float, 3>::kXBytes : Aux<double, 3>::kXBytes);
  const long long want = (long long)P * stage;
  const long long cap = want < share ? want : share;
  return cap >= stage ? (int)cap : 0;
}

int gmres_bulk_stages(bool fp32, int m) {
  return gmres_bulk_cap(fp32, m, kMaxStages) > 0 ? kMaxStages : 0;
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

__global__ void kappa_faces_kernel(int n, int N, const float* __restrict__ kappa,
                                   float* __restrict__ faces, long long fstride) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int nn = n * n;
  const int ix = i % n, iy = (i / n) % n, iz = i / nn;
  const double kc = kappa[i];
  // the harmonic mean in FP64, rounded once to FP32
  auto hm = [&](int j) {
    const double kn = kappa[j];
    return (float)(2.0 * kc * kn / (kc + kn));
  };
  faces[i] = ix < n - 1 ? hm(i + 1) : 0.f;
  faces[fstride + i] = iy < n - 1 ? hm(i + n) : 0.f;
  faces[2 * fstride + i] = iz < n - 1 ? hm(i + nn) : 0.f;
  const int walls = (ix == 0) + (ix == n - 1) + (iy == 0) + (iy == n - 1) + (iz == 0) + (iz == n - 1);
  faces[3 * fstride + i] = (float)(kc * walls);
}

cudaError_t launch_kappa_faces(int n, const float* kappa, float* faces, long long fstride,
                               cudaStream_t s) {
  const int N = n * n * n;
  const int bs = 256, gr = (N + bs - 1) / bs;
  note_launches(1);
  kappa_faces_kernel<<<gr, bs, 0, s>>>(n, N, kappa, faces, fstride);
  return cudaGetLastError();
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
