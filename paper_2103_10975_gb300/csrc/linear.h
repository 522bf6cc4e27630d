// Dense linear initial-guess model y = T u (the simplified model of Sec. 3.1);
// see linear.cu.
#pragma once
#include <cuda_runtime.h>

namespace mlg {

struct Lin {
  int N = 0;                 // grid points (T is N x N, row-major, FP32)
  int bmax = 0;              // largest minibatch
  float* T = nullptr;
  float* grad = nullptr;
  float* bu = nullptr;       // gathered minibatch (bmax x N each)
  float* bt = nullptr;
  float* by = nullptr;
  float* gy = nullptr;
  float* part = nullptr;
};

cudaError_t lin_create(Lin& L, int N, int bmax);
void lin_destroy(Lin& L);
cudaError_t lin_forward(Lin& L, int B, const float* u, float* y, cudaStream_t s);
// MSE 1/(B N) sum ||T u_b - ts t_b||^2 into *loss_dev and its gradient into L.grad.
cudaError_t lin_backward(Lin& L, int B, const float* u, const float* y, const float* t,
                         float tscale, float* loss_dev, cudaStream_t s);
// T -= lr * grad (plain gradient descent)
cudaError_t lin_step(Lin& L, float lr, cudaStream_t s);
cudaError_t lin_train_batch(Lin& L, int B, const float* ring_u, const float* ring_t,
                            long long stride, const int* pick, float tscale, float lr,
                            float* loss_dev, cudaStream_t s);

}  // namespace mlg
