// The initial-guess network N(b) (Sec. 2.1): a variation of FluidNet's pressure
// model -- multi-resolution average-pool pyramid, one convolution per level,
// bilinear upsampling and summation -- followed by a dilated residual block
// and an output convolution, trained online with Adam on the MSE loss
// (Sec. 2.3).  The same network in 3D (dim = 3, for the variable-coefficient
// workload) uses 3x3x3 kernels, 2x2x2 pooling down to 8^3 and trilinear
// upsampling; weights are then [out][in][kz][ky][kx].
//
//   a0  = relu(conv3x3(u, W_in) + b_in)                 1 -> 32
//   p_0 = a0, p_l = avgpool2(p_{l-1}) while the side stays >= 8
//   z_l = relu(conv3x3(p_l, W_l) + b_l)                 32 -> 32 per level
//   s   = sum_l upsample(z_l)   (bilinear, half-pixel centres)
//   t   = s + relu(conv3x3_dil2(s, W_d) + b_d)          32 -> 32
//   y   = conv3x3(t, W_out) + b_out                     32 -> 1
//
// Parameters live in one flat FP32 array in the order
// in.w, in.b, level0.w, level0.b, ..., dil.w, dil.b, out.w, out.b with weights
// [out][in][ky][kx].  The 32 -> 32 convolutions run as implicit GEMMs on the
// tensor cores with BF16 operands and FP32 accumulation.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mlg {

constexpr int kC = 32;      // channels
constexpr int kMaxLevels = 12;
constexpr int kMaxExtra = 4;  // residual blocks the network may grow (Sec. 2.1)

// Device-side state of a training phase, so that one Adam step is the same
// sequence of launches every time (a CUDA graph replays it): the step counter
// and bias corrections of Adam, the minibatch's offset into the phase's picks,
// and the target scale.
struct TrainCtr {
  long long adam_t;   // Adam steps taken (t of the next step is adam_t + 1)
  int iter;           // Adam steps taken in the current phase
  int pick_off;       // iter * B for the step in progress
  float c1, c2;       // 1 - b1^t, 1 - b2^t of the step in progress
  float tscale;       // 1 / c: targets of the phase are t / c
};

struct Net {
  int n = 0;                // grid side
  int dim = 2;              // 2: 3x3 kernels, 2x2 pooling; 3: 3x3x3, 2x2x2
  int taps = 9;             // 3^dim
  int L = 0;                // pyramid levels
  int side[kMaxLevels];     // level sides
  int bmax = 0;             // largest batch
  long long nparams = 0;
  long long off_w[kMaxLevels + 3];  // offsets of each conv's weights (0 in, 1..L levels, L+1 dil, L+2 out)
  long long off_b[kMaxLevels + 3];
  // adaptive growth: residual blocks appended before the output layer,
  // t <- t + relu(conv_dil2(t) + b); parameters after out.b (res1, res2, ...)
  int extra_max = 0;
  int extra_active = 0;
  long long off_rw[kMaxExtra] = {};
  long long off_rb[kMaxExtra] = {};
  __nv_bfloat16* te[kMaxExtra] = {};         // relu part of extra block r
  __nv_bfloat16* tt[kMaxExtra] = {};         // output of extra block r
  float* master = nullptr;  // FP32 parameters
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  __nv_bfloat16* wq = nullptr;  // BF16 copies of the 32->32 weights, [conv][tap][ci][co]
                                // (B operand of the data gradient)
  __nv_bfloat16* wqT = nullptr; // [conv][tap][co][ci] (B operand of the forward pass)
  long long* offs_dev = nullptr;  // device copy of the 32->32 weight offsets
  // activations, channels last (NHWC / NDHWC) with 32 channels, BF16 (masks are recovered from
  // post-ReLU values: relu(x) > 0 <=> x > 0)
  __nv_bfloat16* a0 = nullptr;               // bmax x n^2 x 32
  __nv_bfloat16* pool[kMaxLevels] = {};      // levels 1..L-1
  __nv_bfloat16* z[kMaxLevels] = {};         // levels 0..L-1
  __nv_bfloat16* s = nullptr;                // sum of the levels
  __nv_bfloat16* e = nullptr;                // relu(dilated conv)
  __nv_bfloat16* t = nullptr;                // s + e
  // gradients of activations (FP32 for accumulation, BF16 copies as GEMM operands)
  float* g_t = nullptr;                      // bmax x n^2 x 32
  float* g_s = nullptr;
  float* g_lvl = nullptr;                    // scratch, bmax x n^2 x 32
  float* g_pool = nullptr;                   // pooled accumulation, bmax x n^2 x 32
  __nv_bfloat16* g_bf = nullptr;             // bf16 operand scratch
  float* wgrad_part = nullptr;               // split-K partials of weight gradients
  float* gy = nullptr;                       // bmax x n^2
  float* loss_part = nullptr;
  float* bu = nullptr;                       // gathered minibatch inputs, bmax x n^2
  float* bt = nullptr;                       // gathered minibatch targets
  float* by = nullptr;                       // minibatch outputs
  long long lvl_off[kMaxLevels];             // offsets of level l inside g_pool (per sample)
  // transposed linear upsampling n -> side[l], per axis, as sparse rows:
  // coarse j takes sum over k in [up_ptr[j], up_ptr[j+1]) of up_w[k] * fine[up_idx[k]]
  int* up_ptr[kMaxLevels] = {};
  int* up_idx[kMaxLevels] = {};
  float* up_w[kMaxLevels] = {};
  long long pyr = 0;                         // sum of level sizes (pixels) per sample
  int wparts = 0;                            // CTAs of the weight-gradient kernels
  TrainCtr* ctr = nullptr;                   // device state of the training phase
};

// Tensor-core 32 -> 32 convolution (dim 2: 3x3, dim 3: 3x3x3; mode 0:
// relu(conv + b) -> zo; 1: e = relu(conv + b) -> zo and resid + e -> to;
// 2: conv (+ addend) -> fo in FP32).  wop is [tap][n][k].
cudaError_t launch_conv32_mma(int dim, int mode, int B, int H, const __nv_bfloat16* in,
                              const __nv_bfloat16* wop, const float* bias, int dil, int sign,
                              __nv_bfloat16* zo, __nv_bfloat16* to, const __nv_bfloat16* resid,
                              float* fo, const float* addend, cudaStream_t s);
// The same convolution on the fifth-generation tensor cores (tcgen05.mma into
// tensor memory, operands by TMA), for 2D and 3D grids with at least 128 points
// per row (the environment variable MLGMRES_TC_MIN_ROW lowers the threshold).
bool conv32_tc_applies(int dim, int H);
cudaError_t launch_conv32_tc(int dim, int mode, int B, int H, const __nv_bfloat16* in,
                             const __nv_bfloat16* wop, const float* bias, int dil, int sign,
                             __nv_bfloat16* zo, __nv_bfloat16* to, const __nv_bfloat16* resid,
                             float* fo, const float* addend, cudaStream_t s);
// One-time set-up of the tcgen05 convolution (shared-memory limits, its error
// flag) and of the mma.sync convolution (shared-memory limits); net_create
// calls them so that no forward pass allocates or sets attributes (which a
// graph capture of a training step could not contain).
cudaError_t conv32_tc_setup();
cudaError_t conv32_mma_setup();
// 1 if a tcgen05 convolution tile timed out waiting for its MMAs (0 otherwise).
int conv32_tc_error();
// Tensor-core weight gradient partials of a 32 -> 32 convolution (nparts CTAs):
// part[cta][(tap*32 + k)*32 + o] and the bias sums at 1024 T + o.  Grids whose
// rows qualify for the tcgen05 convolution (conv32_tc_applies) take
// launch_wgrad_tc (tcgen05.mma with the pixels as the reduction dimension).
cudaError_t launch_wgrad_mma(int dim, int B, int H, const __nv_bfloat16* in,
                             const __nv_bfloat16* g, int dil, float* part, int stride, int nparts,
                             cudaStream_t s);
cudaError_t launch_wgrad_tc(int dim, int B, int H, const __nv_bfloat16* in,
                            const __nv_bfloat16* g, int dil, float* part, int stride, int nparts,
                            cudaStream_t s);

// infer_only: allocate what forward passes need (parameters, BF16 operand
// copies, activations) and no gradient, Adam or minibatch buffers; such a
// network takes its weights from another one (net_copy_params).
cudaError_t net_create(Net& net, int n, int bmax, unsigned long long seed, int dim = 2,
                       int extra_max = 0, bool infer_only = false);
// dst.master = src (FP32 parameters, dst.nparams of them) and dst's BF16
// operand copies re-derived, on stream s.
cudaError_t net_copy_params(Net& dst, const float* src, cudaStream_t s);
void net_destroy(Net& net);
// Re-derive the BF16 operand copies from the FP32 master parameters.
cudaError_t net_sync_weights(Net& net, cudaStream_t s);
// y = N(u) for B samples (u, y: B x n^2 FP32).
cudaError_t net_forward(Net& net, int B, const float* u, float* y, cudaStream_t s);
// After net_forward on the same inputs: loss = 1/(B N) sum ||y - tscale t||^2
// into *loss_dev and all parameter gradients into net.grad.
cudaError_t net_backward(Net& net, int B, const float* u, const float* y, const float* target,
                         float tscale, float* loss_dev, cudaStream_t s);
// Resets Adam (moments and the step counter), on stream s.
cudaError_t net_adam_reset(Net& net, cudaStream_t s);
// One minibatch step with every per-step input in device memory: advances
// ctr (t, iter), gathers ring slots picks[pick_off .. pick_off + B) (stride
// floats apart) of inputs u and targets t, runs forward, backward (targets
// scaled by ctr->tscale) and Adam with lr.  *loss_dev gets the loss.  The
// launches do not depend on the step, so a graph capture replays it.
cudaError_t net_train_step_dev(Net& net, int B, const float* ring_u, const float* ring_t,
                               long long stride, const int* picks, TrainCtr* ctr, float lr,
                               float* loss_dev, cudaStream_t s);

}  // namespace mlg
