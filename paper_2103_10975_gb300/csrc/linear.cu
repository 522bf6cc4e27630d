// The single fully connected layer of the paper's simplified model (Sec. 3.1):
// y = T u with a dense N x N matrix T, trained online like the network (MSE on
// normalised pairs, Adam).  It exists to study the spectrum of A T: the guess
// is x0 = c s T(b/s) = c T b, so r0 = (I - c A T) b and ||r0|| <= ||I - c A T|| ||b||.
// It trains by plain gradient descent (step lr), so T stays 0 outside the span
// of the training inputs.
#include <math.h>

#include "common.cuh"
#include "linear.h"

namespace mlg {

namespace {

unsigned nblk(long long count, int bs) { return (unsigned)((count + bs - 1) / bs); }

// y[b][i] = sum_j T[i][j] u[b][j]: one warp per (b, i), lanes stride over j
__global__ void lin_fwd(int B, int N, const float* __restrict__ T, const float* __restrict__ u,
                        float* __restrict__ y) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (long long)B * N) return;
  const int b = (int)(w / N), i = (int)(w % N);
  const float* row = T + (long long)i * N;
  const float* ub = u + (long long)b * N;
  float acc = 0.f;
  for (int j = lane; j < N; j += 32) acc += row[j] * ub[j];
  acc = warp_sum(acc);
  if (lane == 0) y[(long long)b * N + i] = acc;
}

// gy = 2 (y - ts t) scale; per-CTA partial sums of (y - ts t)^2
__global__ void lin_mse(long long total, float scale, float ts, const float* __restrict__ y,
                        const float* __restrict__ t, float* __restrict__ gy,
                        float* __restrict__ part) {
  __shared__ float red[32];
  float acc = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - ts * t[i];
    gy[i] = 2.f * d * scale;
    acc += d * d;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    acc = warp_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
  }
}

__global__ void lin_loss(const float* __restrict__ part, int nparts, float scale,
                         float* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nparts; i++) s += part[i];
    *loss = (float)(s * scale);
  }
}

// G[i][j] = sum_b gy[b][i] u[b][j]
__global__ void lin_grad(int B, int N, const float* __restrict__ gy, const float* __restrict__ u,
                         float* __restrict__ G) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= (long long)N * N) return;
  const int i = (int)(k / N), j = (int)(k % N);
  float acc = 0.f;
  for (int b = 0; b < B; b++) acc += gy[(long long)b * N + i] * u[(long long)b * N + j];
  G[k] = acc;
}

// plain gradient descent T -= lr G: T changes only along the training inputs'
// span (Adam's per-entry normalisation would move every entry by about lr per
// step, also those no training pair constrains, and A amplifies that noise)
__global__ void lin_sgd(long long count, float* __restrict__ theta, const float* __restrict__ g,
                        float lr) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= count) return;
  theta[i] -= lr * g[i];
}

}  // namespace

#define LIN_CK(x)                         \
  do {                                    \
    cudaError_t e_ = (x);                 \
    if (e_ != cudaSuccess) return e_;     \
  } while (0)

cudaError_t lin_create(Lin& L, int N, int bmax) {
  L.N = N;
  L.bmax = bmax;
  const long long nn = (long long)N * N;
  LIN_CK(cudaMalloc(&L.T, sizeof(float) * nn));
  LIN_CK(cudaMalloc(&L.grad, sizeof(float) * nn));
  LIN_CK(cudaMemset(L.T, 0, sizeof(float) * nn));  // T = 0: A T starts with a zero spectrum
  LIN_CK(cudaMemset(L.grad, 0, sizeof(float) * nn));
  LIN_CK(cudaMalloc(&L.bu, sizeof(float) * (long long)bmax * N));
  LIN_CK(cudaMalloc(&L.bt, sizeof(float) * (long long)bmax * N));
  LIN_CK(cudaMalloc(&L.by, sizeof(float) * (long long)bmax * N));
  LIN_CK(cudaMalloc(&L.gy, sizeof(float) * (long long)bmax * N));
  LIN_CK(cudaMalloc(&L.part, sizeof(float) * 256));
  return cudaDeviceSynchronize();
}

void lin_destroy(Lin& L) {
  cudaFree(L.T);
  cudaFree(L.grad);
  cudaFree(L.bu);
  cudaFree(L.bt);
  cudaFree(L.by);
  cudaFree(L.gy);
  cudaFree(L.part);
  L = Lin();
}

cudaError_t lin_forward(Lin& L, int B, const float* u, float* y, cudaStream_t s) {
  const long long warps = (long long)B * L.N;
  lin_fwd<<<nblk(warps * 32, 256), 256, 0, s>>>(B, L.N, L.T, u, y);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t lin_backward(Lin& L, int B, const float* u, const float* y, const float* t,
                         float tscale, float* loss_dev, cudaStream_t s) {
  const long long tot = (long long)B * L.N;
  lin_mse<<<256, 256, 0, s>>>(tot, 1.f / (float)tot, tscale, y, t, L.gy, L.part);
  lin_loss<<<1, 32, 0, s>>>(L.part, 256, 1.f / (float)tot, loss_dev);
  lin_grad<<<nblk((long long)L.N * L.N, 256), 256, 0, s>>>(B, L.N, L.gy, u, L.grad);
  note_launches(3);
  return cudaGetLastError();
}

cudaError_t lin_step(Lin& L, float lr, cudaStream_t s) {
  const long long nn = (long long)L.N * L.N;
  lin_sgd<<<nblk(nn, 256), 256, 0, s>>>(nn, L.T, L.grad, lr);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t lin_train_batch(Lin& L, int B, const float* ring_u, const float* ring_t,
                            long long stride, const int* pick, float tscale, float lr,
                            float* loss_dev, cudaStream_t s) {
  const long long N = L.N;
  for (int i = 0; i < B; i++) {
    LIN_CK(cudaMemcpyAsync(L.bu + i * N, ring_u + (long long)pick[i] * stride,
                           sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
    LIN_CK(cudaMemcpyAsync(L.bt + i * N, ring_t + (long long)pick[i] * stride,
                           sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
  }
  LIN_CK(lin_forward(L, B, L.bu, L.by, s));
  LIN_CK(lin_backward(L, B, L.bu, L.by, L.bt, tscale, loss_dev, s));
  return lin_step(L, lr, s);
}

}  // namespace mlg
