// Internal state behind an mlgmres_t handle.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/mlgmres.h"
#include "linear.h"
#include "nn.h"
#include "solver.h"

struct mlgmres {
  mlgmres_grid grid;
  mlgmres_options opt;
  int N = 0;
  int dev = 0;
  int nsm = 0;
  bool fp32 = false;
  int blocks = 0;       // solver CTAs for a single solve
  int max_blocks = 0;   // co-resident limit of the kernel variant
  int bs = 0;
  int vsmem = 0;        // shared-memory bytes for the V slice of a single solve
  int tuned_stages = -1;  // bulk-copy stages chosen by mlgmres_autotune (-1 = none)
  int tuned_compact = 0;  // 1: the autotuner chose the two-CTAs-per-SM bulk variant

  // ---- solver workspace (one group for single solves) ----
  long long ldv = 0;
  void* V = nullptr;
  void* W0 = nullptr;
  void* W1 = nullptr;
  void* W0_alloc = nullptr;  // W0's allocation (W0 may start past a zero pad)
  float* faces = nullptr;    // FP32 face coefficients (single 3D FP32 solves with kappa)
  long long fstride = 0;     // their array stride
  double* part = nullptr;
  double* Rg = nullptr;      // compact variants' triangles R (rg_blocks of them)
  int rg_blocks = 0;
  unsigned long long* bar = nullptr;  // per group: counter
  int* err = nullptr;                 // per group: error flag
  mlg::DevResult* dres = nullptr;     // device results
  mlg::DevResult* hres = nullptr;     // pinned host copy
  int* dcfg = nullptr;                // group_first | task_first | task_order
  mlg::SolveTask* dtasks = nullptr;
  mlg::GroupWork* dwork = nullptr;
  mlg::SolveTask* htasks = nullptr;   // pinned staging
  int* hcfg = nullptr;                // pinned staging
  mlg::GroupWork* hwork = nullptr;    // pinned staging
  int cfg_cap = 0;                    // capacity (tasks) of the config buffers
  int group_cap = 0;                  // capacity (groups) of the group buffers
  // batched solves: one-CTA groups with their own bases
  int batch_groups = 0;
  bool batch_compact = false;         // batches may launch the compact variant
  void* Vb = nullptr;
  void* Wb = nullptr;                 // 2 work vectors per group
  double* partb = nullptr;

  // ---- guess state ----
  double* x_prev = nullptr;
  bool have_prev = false;
  double* x_alt = nullptr;            // learned guess
  float* u_in = nullptr;              // normalised input b/s (FP32)
  float* y_out = nullptr;             // network output (FP32)
  double* scal = nullptr;             // device scalars (rms etc.)

  // ---- learned guess / training ----
  mlg::Net net;
  mlg::Lin lin;                       // the dense linear model (opt.model = LINEAR)
  bool linear = false;
  bool net_ready = false;             // the guess holds trained parameters
  int train_calls = 0;
  // replay ring: normalised (b/s, x/s) pairs, FP32, N each
  float* ring_u = nullptr;
  float* ring_t = nullptr;
  int ring_count = 0;
  int ring_head = 0;                  // next slot to write
  std::vector<int> fresh;             // C_t: slots of the candidates admitted since the last
                                      // training phase (warm-up pairs are not candidates)
  int cand_n = 0;                     // Algorithm 1's N: under-performing steps since the
                                      // last training phase (admitted or not)
  std::vector<double> E_hist, T_hist;
  std::vector<double> ring_c;         // rms(x)/rms(b) of each stored pair
  double c_train = 1.0;               // target scale used by the last training phase
  double mp_last_phase = 0.0;         // M_p(E_k) at the previous training phase (growth)
  double* x_tmp = nullptr;            // smoothing ping-pong buffer
  long long solves = 0;
  double* ddots = nullptr;            // device dots for the spread check
  double* hdots = nullptr;            // pinned
  unsigned long long rng_state = 0;
  // training phases run beside the solves (Sec. 2.3, training in real time):
  // the guess reads only `inf`, an inference copy of the network with its own
  // activations; a phase reads a snapshot of the ring taken at its start and
  // ends by copying its parameters to `snap`, which a later solve copies into
  // `inf` once the phase has completed
  mlg::Net inf;
  float* snap = nullptr;
  float* ring_u_snap = nullptr;
  float* ring_t_snap = nullptr;
  cudaEvent_t train_done = nullptr;   // the latest phase (and its parameter snapshot) completed
  cudaEvent_t ring_copied = nullptr;  // the latest phase's ring snapshot completed
  cudaStream_t phase_stream = nullptr;  // stream of the latest phase
  bool phase_enqueued = false;        // some phase was enqueued (the events are meaningful)
  bool snap_pending = false;          // the latest phase's parameters are not in `inf` yet
  double snap_c = 1.0;                // target scale c of that phase
  int snap_extra = 0;                 // residual blocks of that phase
  double c_guess = 1.0;               // c of the parameters `inf` holds
  int phase_waits = 0;                // phases that had to wait for the previous one
  // A phase is thousands of launches (train_iters Adam steps of ~60 kernels);
  // enqueued one by one they fill the launch queue and block the caller.  One
  // Adam step is captured once as a CUDA graph (its per-step inputs -- picks,
  // step counter, target scale -- live in device memory) and a phase launches
  // that graph train_iters times.
  struct StepGraph {
    int B = 0, extra = 0;               // minibatch size and grown blocks it was captured for
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;              // kernels per replay
  };
  std::vector<StepGraph> graphs;
  cudaStream_t cap_stream = nullptr;  // capture stream (no work ever runs on it)
  int* picks_dev = nullptr;           // the phase's minibatch picks, train_iters x batch
  int* picks_host = nullptr;          // pinned staging of the picks
  float* tscale_host = nullptr;       // pinned staging of the phase's target scale
  cudaStream_t train_stream = nullptr;  // training phases started by solve (retrain_after)
  float* loss_dev = nullptr;

  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
  std::string last_error;
};
