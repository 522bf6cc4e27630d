// Small vector kernels around the solver: the input normalisation of the
// learned guess (s = rms(b), u = b/s, x0 = s y), replay-ring stores and the
// dot products of the spread check (Sec. 2.2).
#include <atomic>

#include "misc.h"

namespace mlg {

static std::atomic<long long> g_launches{0};
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// sum of squares of b into *out (one CTA, fixed order: deterministic).
__global__ void sumsq_kernel(const double* __restrict__ b, int N, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += b[i] * b[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) *out = s;
  }
}

// u = b / s with s = sqrt(sumsq / N) (s = 1 when b = 0)
__global__ void normalise_kernel(const double* __restrict__ b, int N, const double* sumsq,
                                 float* __restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = sqrt(*sumsq / N);
  if (!(s > 0.0)) s = 1.0;
  u[i] = (float)(b[i] / s);
}

// x = scale s y
__global__ void denormalise_kernel(const float* __restrict__ y, int N, const double* sumsq,
                                   double scale, double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = sqrt(*sumsq / N);
  if (!(s > 0.0)) s = 1.0;
  x[i] = scale * s * (double)y[i];
}

// One damped-Jacobi sweep on the 2D operator: out = in + omega/d (b - A in),
// d = 4/h^2 the diagonal of A.  s2 = 1/h^2 and f = omega/(4 s2) come from the
// host (the same IEEE divisions, once per launch instead of three FP64
// divisions per point on a GPU whose FP64 pipe is narrow).
__global__ void jacobi_kernel(int n, const double* __restrict__ b, const double* __restrict__ xin,
                              double* __restrict__ xout, double s2, double f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * n) return;
  const int ix = i % n, iy = i / n;
  const double c = xin[i];
  const double l = ix > 0 ? xin[i - 1] : 0.0;
  const double r = ix < n - 1 ? xin[i + 1] : 0.0;
  const double d = iy > 0 ? xin[i - n] : 0.0;
  const double t = iy < n - 1 ? xin[i + n] : 0.0;
  const double ax = s2 * (((c - l) + (c - r)) + ((c - d) + (c - t)));
  xout[i] = c + f * (b[i] - ax);
}

// 3D: A u = (1/h^2) sum_faces k_f (u_c - u_nb), k_f the harmonic mean of the
// two cells' kappa (kappa_c on a wall face, u = 0 beyond it; kappa = NULL
// means 1); the diagonal is (1/h^2) sum_faces k_f.  s2 = 1/h^2 from the host.
__global__ void jacobi3d_kernel(int n, const float* __restrict__ kappa,
                                const double* __restrict__ b, const double* __restrict__ xin,
                                double* __restrict__ xout, double omega, double s2) {
  const long long N = (long long)n * n * n;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
  const long long nn = (long long)n * n;
  const long long off[6] = {-1, 1, -(long long)n, (long long)n, -nn, nn};
  const bool has[6] = {ix > 0, ix < n - 1, iy > 0, iy < n - 1, iz > 0, iz < n - 1};
  const double c = xin[i];
  const double kc = kappa ? (double)kappa[i] : 1.0;
  double au = 0.0, diag = 0.0;
  for (int f = 0; f < 6; f++) {
    double kf = kc, unb = 0.0;
    if (has[f]) {
      const double kn = kappa ? (double)kappa[i + off[f]] : 1.0;
      kf = 2.0 * kc * kn / (kc + kn);
      unb = xin[i + off[f]];
    }
    au += kf * (c - unb);
    diag += kf;
  }
  xout[i] = c + omega * (b[i] - s2 * au) / (s2 * diag);
}

// ring pair: u = b/s, t = x/s
__global__ void store_pair_kernel(const double* __restrict__ b, const double* __restrict__ x,
                                  int N, const double* sumsq, float* __restrict__ u,
                                  float* __restrict__ t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = sqrt(*sumsq / N);
  if (!(s > 0.0)) s = 1.0;
  u[i] = (float)(b[i] / s);
  t[i] = (float)(x[i] / s);
}

// out[2c] = <x, t_c>, out[2c+1] = <t_c, t_c> for the listed ring slots;
// out[2*count] = <x, x>.  One CTA per slot (+1 for ||x||), fixed order.
__global__ void spread_dots_kernel(const double* __restrict__ x, const float* __restrict__ ring,
                                   long long stride, const int* __restrict__ slots, int count,
                                   int N, double* out) {
  __shared__ double red[2][32];
  const int c = blockIdx.x;
  double a = 0.0, bb = 0.0;
  if (c < count) {
    const float* tc = ring + (long long)slots[c] * stride;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const double tv = tc[i];
      a += x[i] * tv;
      bb += tv * tv;
    }
  } else {
    for (int i = threadIdx.x; i < N; i += blockDim.x) a += x[i] * x[i];
  }
  a = warp_sum(a);
  bb = warp_sum(bb);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = bb;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool in = threadIdx.x < (int)(blockDim.x >> 5);
    a = warp_sum(in ? red[0][threadIdx.x] : 0.0);
    bb = warp_sum(in ? red[1][threadIdx.x] : 0.0);
    if (threadIdx.x == 0) {
      if (c < count) {
        out[2 * c] = a;
        out[2 * c + 1] = bb;
      } else {
        out[2 * count] = a;
      }
    }
  }
}

static unsigned blocks_for(int N) { return (unsigned)((N + 255) / 256); }

cudaError_t launch_sumsq(const double* b, int N, double* out, cudaStream_t s) {
  sumsq_kernel<<<1, 1024, 0, s>>>(b, N, out);
  note_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_normalise(const double* b, int N, const double* sumsq, float* u,
                             cudaStream_t s) {
  normalise_kernel<<<blocks_for(N), 256, 0, s>>>(b, N, sumsq, u);
  note_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_jacobi(int dim, int n, const float* kappa, const double* b, const double* xin,
                          double* xout, double omega, cudaStream_t s) {
  const double h = 2.0 / (n + 1);
  const double s2 = 1.0 / (h * h);
  if (dim == 3)
    jacobi3d_kernel<<<blocks_for(n * n * n), 256, 0, s>>>(n, kappa, b, xin, xout, omega, s2);
  else
    jacobi_kernel<<<blocks_for(n * n), 256, 0, s>>>(n, b, xin, xout, s2, omega / (4.0 * s2));
  note_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_denormalise(const float* y, int N, const double* sumsq, double scale,
                               double* x, cudaStream_t s) {
  denormalise_kernel<<<blocks_for(N), 256, 0, s>>>(y, N, sumsq, scale, x);
  note_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_store_pair(const double* b, const double* x, int N, const double* sumsq,
                              float* u, float* t, cudaStream_t s) {
  store_pair_kernel<<<blocks_for(N), 256, 0, s>>>(b, x, N, sumsq, u, t);
  note_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_spread_dots(const double* x, const float* ring, long long stride,
                               const int* slots, int count, int N, double* out, cudaStream_t s) {
  spread_dots_kernel<<<count + 1, 512, 0, s>>>(x, ring, stride, slots, count, N, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace mlg
