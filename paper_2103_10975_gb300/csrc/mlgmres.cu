// C ABI of the library: handle life cycle, guess selection, the persistent
// solve, the online data-collection gate (Sec. 2.2, Algorithm 1) and the
// training phase (Sec. 2.3).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "handle.h"
#include "schedule.h"
#include "misc.h"

using namespace mlg;

namespace {

constexpr int kBatchCap = 4096;  // most systems per mlgmres_solve_batch call

struct Fail {
  mlgmres_status st;
};

std::string fmt_cuda(const char* what, cudaError_t e) {
  return std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

#define CK(call)                                                  \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) {                                      \
      h->last_error = fmt_cuda(#call, e_);                        \
      throw Fail{e_ == cudaErrorMemoryAllocation ? MLGMRES_ERR_OOM \
                                                 : MLGMRES_ERR_CUDA}; \
    }                                                             \
  } while (0)

#define ARG(cond, msg)              \
  do {                              \
    if (!(cond)) {                  \
      h->last_error = (msg);        \
      throw Fail{MLGMRES_ERR_ARG};  \
    }                               \
  } while (0)

long long grid_points(int dim, int n) {
  return dim == 2 ? (long long)n * n : (long long)n * n * n;
}

unsigned long long splitmix_next(unsigned long long& st) {
  st += 0x9E3779B97F4A7C15ull;
  unsigned long long z = st;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int auto_blocks(const mlgmres* h, int N) {
  // about 512 grid points per CTA (two per thread): measured on GB300 at 256^2,
  // 128 CTAs take 18 us per Arnoldi step against 26 us with 64 and 43 us with 32;
  // never more CTAs than can be co-resident
  long long want = (N + 511) / 512;
  if (want < 1) want = 1;
  if (want > h->max_blocks) want = h->max_blocks;
  if (want > kPartStride) want = kPartStride;
  return (int)want;
}

void check_options(mlgmres* h, const mlgmres_options* o) {
  ARG(o->m >= 1 && o->m <= kMaxM, "m must be in 1..64");
  ARG(o->rtol > 0.0 && o->rtol < 1.0, "rtol must be in (0, 1)");
  ARG(o->max_iters > 0, "max_iters must be positive");
  ARG(o->precision == MLGMRES_FP64 || o->precision == MLGMRES_FP32_REFINE, "bad precision");
  ARG(o->guess >= MLGMRES_GUESS_ZERO && o->guess <= MLGMRES_GUESS_USER, "bad guess mode");
  ARG(o->fallback == MLGMRES_GUESS_ZERO || o->fallback == MLGMRES_GUESS_PREV, "bad fallback");
  ARG(o->replay_cap >= 1 && o->replay_cap <= 4096, "replay_cap must be in 1..4096");
  ARG(o->warmup_steps >= 0, "warmup_steps must be >= 0");
  ARG(o->window_p >= 1, "window_p must be >= 1");
  ARG(o->ortho_theta >= 0.0 && o->ortho_theta <= 1.0, "ortho_theta must be in [0, 1]");
  ARG(o->train_iters >= 0, "train_iters must be >= 0");
  ARG(o->batch >= 1 && o->batch <= 64, "batch must be in 1..64");
  ARG(o->lr > 0.0f, "lr must be positive");
  ARG(o->grid_blocks >= 0, "grid_blocks must be >= 0");
  ARG(o->batch_slots >= 0 && o->batch_slots <= 4096, "batch_slots must be in 0..4096");
  ARG(o->barrier_timeout_s > 0.0 && o->barrier_timeout_s <= 60.0,
      "barrier_timeout_s must be in (0, 60]");
  ARG(o->fault_inject == 0 || o->fault_inject == 1, "fault_inject must be 0 or 1");
  ARG(o->guess_smooth >= 0 && o->guess_smooth <= 1000, "guess_smooth must be in 0..1000");
  ARG(o->guess_omega > 0.0f && o->guess_omega <= 1.0f, "guess_omega must be in (0, 1]");
  ARG(o->guess_select == 0 || o->guess_select == 1, "guess_select must be 0 or 1");
  ARG(o->v_stages == -1 || o->v_stages == 0 || (o->v_stages >= 2 && o->v_stages <= 16),
      "v_stages must be -1, 0 or 2..16");
  ARG(o->v_stages <= 0 ||
          gmres_bulk_cap(o->precision == MLGMRES_FP32_REFINE, o->m, o->v_stages) > 0,
      "v_stages: no stage of m rows fits in shared memory");
  ARG(o->retrain_after >= 0, "retrain_after must be >= 0");
  ARG(o->grow_blocks >= 0 && o->grow_blocks <= kMaxExtra, "grow_blocks must be in 0..4");
  ARG(o->grow_tol >= 0.0 && o->grow_tol <= 1.0, "grow_tol must be in [0, 1]");
  ARG(o->model == MLGMRES_MODEL_CONV || o->model == MLGMRES_MODEL_LINEAR, "bad model");
  ARG(o->compact >= -1 && o->compact <= 1, "compact must be -1, 0 or 1");
  ARG(o->model == MLGMRES_MODEL_CONV || o->grow_blocks == 0,
      "grow_blocks applies to the convolutional model only");
  ARG(o->overlap_train == 0 || o->overlap_train == 1, "overlap_train must be 0 or 1");
}

// Bulk-copy stages the passes use for an FP32 basis in HBM.
int effective_stages(const mlgmres* h) {
  if (h->opt.v_stages >= 0) return h->opt.v_stages;
  if (h->tuned_stages >= 0) return h->tuned_stages;
  return gmres_bulk_stages(h->fp32, h->opt.m);
}

// Allocates the network, its replay ring and the learned-guess buffers (2D
// and 3D networks; once per handle).
void ensure_net(mlgmres* h) {
  if (h->net.master || h->lin.T) return;
  const mlgmres_options* opt = &h->opt;
  CK(cudaMalloc(&h->u_in, sizeof(float) * h->ldv));
  CK(cudaMalloc(&h->y_out, sizeof(float) * h->ldv));
  CK(cudaMalloc(&h->ring_u, sizeof(float) * h->ldv * opt->replay_cap));
  CK(cudaMalloc(&h->ring_t, sizeof(float) * h->ldv * opt->replay_cap));
  CK(cudaMalloc(&h->ddots, sizeof(double) * (2 * opt->replay_cap + 1)));
  CK(cudaMallocHost(&h->hdots, sizeof(double) * (2 * opt->replay_cap + 1)));
  CK(cudaMalloc(&h->ring_u_snap, sizeof(float) * h->ldv * opt->replay_cap));
  CK(cudaMalloc(&h->ring_t_snap, sizeof(float) * h->ldv * opt->replay_cap));
  CK(cudaMalloc(&h->loss_dev, sizeof(float) * 4));
  if (opt->model == MLGMRES_MODEL_LINEAR) {
    ARG(h->N <= 4096, "the linear model needs N <= 4096");
    h->linear = true;
    CK(lin_create(h->lin, h->N, opt->batch));
  } else {
    ARG(32LL * opt->batch * h->N < (1LL << 31),
        "the network indexes its activations in 32 bits: 32 * batch * n^dim must be < 2^31");
    CK(net_create(h->net, h->grid.n, opt->batch, opt->seed, h->grid.dim, opt->grow_blocks));
    // the inference copy starts from the same initial parameters (same seed)
    CK(net_create(h->inf, h->grid.n, 1, opt->seed, h->grid.dim, opt->grow_blocks, true));
    CK(cudaMalloc(&h->snap, sizeof(float) * h->net.nparams));
    const size_t np = (size_t)std::max(1, opt->train_iters) * opt->batch;
    CK(cudaMalloc(&h->picks_dev, sizeof(int) * np));
    CK(cudaMallocHost(&h->picks_host, sizeof(int) * np));
    CK(cudaMallocHost(&h->tscale_host, sizeof(float)));
    CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  }
}

// cudaEventQuery's "not ready" is a state, not a failure: keep it out of the
// error that the next launch check reads
cudaError_t query_event(cudaEvent_t e) {
  const cudaError_t q = cudaEventQuery(e);
  if (q == cudaErrorNotReady && cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
  return q;
}

// Moves the parameters of the latest training phase into the guess's network,
// on stream s.  With overlap_train (and for another stream than the phase's)
// only once the phase has completed: a solve issued while it runs keeps the
// previous parameters and never waits.  Otherwise s waits for the phase.
void take_snapshot(mlgmres* h, cudaStream_t s) {
  if (!h->snap_pending) return;
  const bool same = s == h->phase_stream;
  if (h->linear || h->opt.overlap_train == 0 || same) {
    if (!same) CK(cudaStreamWaitEvent(s, h->train_done, 0));
  } else {
    const cudaError_t q = query_event(h->train_done);
    if (q == cudaErrorNotReady) return;
    CK(q);
  }
  if (!h->linear) {
    CK(net_copy_params(h->inf, h->snap, s));
    h->inf.extra_active = h->snap_extra;
  }
  h->c_guess = h->snap_c;
  h->snap_pending = false;
  h->net_ready = true;
}

// Forward pass of the handle's model on `batch` normalised inputs (the
// training copy of the network).
void model_forward(mlgmres* h, int batch, const float* u, float* y, cudaStream_t s) {
  if (h->linear)
    CK(lin_forward(h->lin, batch, u, y, s));
  else
    CK(net_forward(h->net, batch, u, y, s));
}

// Forward pass of the guess: the inference copy of the network (one sample).
void guess_forward(mlgmres* h, const float* u, float* y, cudaStream_t s) {
  if (h->linear)
    CK(lin_forward(h->lin, 1, u, y, s));
  else
    CK(net_forward(h->inf, 1, u, y, s));
}

// Streams that touch the training copy of the network (inspection entry
// points) first wait for the latest phase.
void wait_phase(mlgmres* h, cudaStream_t s) {
  if (h->phase_enqueued && s != h->phase_stream) CK(cudaStreamWaitEvent(s, h->train_done, 0));
}

long long model_params(const mlgmres* h) {
  return h->linear ? (long long)h->lin.N * h->lin.N : h->net.nparams;
}
float* model_master(mlgmres* h) { return h->linear ? h->lin.T : h->net.master; }
float* model_grad(mlgmres* h) { return h->linear ? h->lin.grad : h->net.grad; }

// The learned guess x0 = c s N(b/s) (s = rms(b), c the target scale of the
// training phase whose parameters the guess holds), then opt.guess_smooth
// damped-Jacobi sweeps; returns the buffer (x_alt or x_tmp) that holds it.
double* learned_guess(mlgmres* h, const double* b, cudaStream_t s) {
  const int N = h->N;
  CK(launch_sumsq(b, N, h->scal, s));
  CK(launch_normalise(b, N, h->scal, h->u_in, s));
  guess_forward(h, h->u_in, h->y_out, s);
  double* cur = h->x_alt;
  double* oth = h->x_tmp;
  CK(launch_denormalise(h->y_out, N, h->scal, h->c_guess, cur, s));
  for (int k = 0; k < h->opt.guess_smooth; k++) {
    CK(launch_jacobi(h->grid.dim, h->grid.n, h->grid.kappa_dev, b, cur, oth,
                     (double)h->opt.guess_omega, s));
    std::swap(cur, oth);
  }
  return cur;
}

// Whether single solves launch the compact bulk-copy variant.
int use_compact(const mlgmres* h) {
  if (h->opt.compact == 0) return 0;
  if (h->opt.compact == 1) return 1;
  return h->tuned_compact;
}

// Shared-memory bytes of a single solve's V slice at `blocks` CTAs (0 if the
// slice does not fit).
int single_vsmem(const mlgmres* h, int blocks, bool compact = false) {
  const long long chunk = (((long long)h->N + blocks - 1) / blocks + 31) / 32 * 32;
  const long long need = chunk * vrows_p(h->opt.m + 1) * (h->fp32 ? 4 : 8);
  const int budget = compact ? (h->grid.dim == 2 ? gmres_compact_vsmem_budget() : 0)
                             : gmres_vsmem_budget(h->fp32);
  return need <= budget ? (int)need : 0;
}

// Run the persistent kernel for `count` tasks already staged in h->htasks,
// with the group layout staged in h->hcfg / h->hwork.
void run_solver(mlgmres* h, int ngroups, int ntasks, int grid, int arnoldi_steps,
                cudaStream_t s, int vsmem = 0, long long max_iters = -1, int stages = -1,
                int compact = 0) {
  const size_t cfg_bytes = sizeof(int) * (size_t)(2 * (ngroups + 1) + ntasks);
  CK(cudaMemcpyAsync(h->dcfg, h->hcfg, cfg_bytes, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->dtasks, h->htasks, sizeof(SolveTask) * ntasks, cudaMemcpyHostToDevice,
                     s));
  CK(cudaMemcpyAsync(h->dwork, h->hwork, sizeof(GroupWork) * ngroups, cudaMemcpyHostToDevice,
                     s));
  CK(cudaMemsetAsync(h->bar, 0, sizeof(unsigned long long) * ngroups, s));
  CK(cudaMemsetAsync(h->err, 0, sizeof(int) * ngroups, s));
  KParams kp;
  kp.m = h->opt.m;
  kp.rtol = h->opt.rtol;
  kp.max_iters = max_iters > 0 ? max_iters : h->opt.max_iters;
  kp.arnoldi_steps = arnoldi_steps;
  kp.vsmem = arnoldi_steps > 0 ? 0 : vsmem;
  kp.bulk_stages = stages >= 0 ? stages : effective_stages(h);
  kp.bulk_cap = gmres_bulk_cap(h->fp32, h->opt.m, kp.bulk_stages);
  if (kp.bulk_cap == 0) kp.bulk_stages = 0;
  // placement of V: shared-memory slices when every task's slice fits (2D),
  // else bulk-copy stages, else direct loads
  kp.vmode = kVDirect;
  if (kp.vsmem > 0 && h->grid.dim == 2) kp.vmode = kVShared;
  else if (kp.bulk_stages > 0) kp.vmode = kVBulk;
  // the compact (two CTAs per SM) bulk variant, when chosen
  kp.compact = 0;
  if (compact && gmres_compact_ok(h->fp32, h->grid.dim, h->opt.m)) {
    if (kp.vmode == kVBulk) {
      const int cap = gmres_compact_cap(h->grid.dim, h->opt.m, kp.bulk_stages);
      if (cap > 0) {
        kp.compact = 1;
        kp.bulk_cap = cap;
      }
    } else if (kp.vmode == kVShared && kp.vsmem <= gmres_compact_vsmem_budget()) {
      kp.compact = 1;  // V slices in shared memory, two CTAs per SM
    }
  }
  ARG(!kp.compact || (h->Rg && grid <= h->rg_blocks), "compact variant: grid exceeds its R workspace");
  // face coefficients from the current kappa (one pass over the grid)
  if (ntasks == 1 && h->htasks[0].faces)
    CK(launch_kappa_faces(h->grid.n, h->grid.kappa_dev, h->faces, h->fstride, s));
  kp.ngroups = ngroups;
  kp.group_first = h->dcfg;
  kp.task_first = h->dcfg + (ngroups + 1);
  kp.task_order = h->dcfg + 2 * (ngroups + 1);
  kp.tasks = h->dtasks;
  kp.work = h->dwork;
  CK(launch_gmres(kp, h->fp32, h->grid.dim, grid, s));
}

GroupWork single_group_work(mlgmres* h, int nblocks) {
  GroupWork w;
  w.V = h->V;
  w.ldv = h->ldv;
  w.W0 = h->W0;
  w.W1 = h->W1;
  w.part = h->part;
  w.pstride = kPartStride;
  w.Rg = h->Rg;
  w.bar.ctr = h->bar;
  w.bar.err = h->err;
  // fault_inject = 1 makes the barrier wait for a CTA that is never launched
  w.bar.nblocks = (unsigned)(nblocks + (h->opt.fault_inject == 1 ? 1 : 0));
  w.bar.timeout_ns = (unsigned long long)(h->opt.barrier_timeout_s * 1e9);
  return w;
}

void stage_single(mlgmres* h, const SolveTask& t, int nblocks) {
  h->hcfg[0] = 0;
  h->hcfg[1] = nblocks;
  h->hcfg[2] = 0;
  h->hcfg[3] = 1;
  h->hcfg[4] = 0;
  h->htasks[0] = t;
  // the handle's own 3D grid: the FP32 passes use its face coefficients
  if (h->faces && t.kappa == h->grid.kappa_dev && t.n == h->grid.n) {
    h->htasks[0].faces = h->faces;
    h->htasks[0].fstride = h->fstride;
  }
  h->hwork[0] = single_group_work(h, nblocks);
}

mlgmres_status to_status(int s) {
  switch (s) {
    case 0: return MLGMRES_OK;
    case 1: return MLGMRES_NOT_CONVERGED;
    case kErrTimeout: return MLGMRES_ERR_TIMEOUT;
    case kErrNonfinite: return MLGMRES_ERR_NONFINITE;
    default: return MLGMRES_ERR_CUDA;
  }
}

void fill_result(const DevResult& d, mlgmres_result* r) {
  r->iters = d.iters;
  r->cycles = d.cycles;
  r->status = to_status(d.status);
  r->bnorm = d.bnorm;
  r->relres_true = d.relres_true;
  r->relres_first_cycle = d.relres_first_cycle;
  r->relres_guess = d.relres_guess;
  r->relres_learned = d.relres_alt;
}

// Algorithm 1: decide whether the pair (b, x) of the solve just finished joins
// the replay ring, and store it.  Runs after every LEARNED-mode solve.
int gate_and_store(mlgmres* h, const double* b, const double* x, const mlgmres_result& r,
                   cudaStream_t s) {
  const int p = h->opt.window_p;
  const double E = r.relres_first_cycle;
  const double T = h->opt.deterministic_tos ? (double)r.iters : (double)r.tos_ms;
  h->E_hist.push_back(E);
  h->T_hist.push_back(T);
  h->solves++;
  bool admit = false;
  const bool warm = h->solves <= h->opt.warmup_steps;
  if (warm) {
    admit = true;  // warm-up: every pair joins the training set X_t directly (Sec. 2.3)
  } else {
    auto mean_last = [p](const std::vector<double>& v) {
      const size_t k = std::min<size_t>((size_t)p, v.size());
      double acc = 0.0;
      for (size_t i = v.size() - k; i < v.size(); i++) acc += v[i];
      return acc / (double)k;
    };
    const bool good = (E < mean_last(h->E_hist)) && (T < mean_last(h->T_hist));
    if (!good) {
      // an under-performing step: Algorithm 1 counts it towards f_r (N = N + 1)
      // whether or not it passes the spread check
      h->cand_n++;
      admit = true;
      const int cnt = (int)h->fresh.size();
      if (cnt > 0) {  // spread check against C_t
        CK(cudaMemcpyAsync(h->scal + 8, h->fresh.data(), sizeof(int) * cnt,
                           cudaMemcpyHostToDevice, s));
        // slots live in the int view of scal[8...]
        CK(launch_spread_dots(x, h->ring_t, h->ldv, (const int*)(h->scal + 8), cnt, h->N,
                              h->ddots, s));
        CK(cudaMemcpyAsync(h->hdots, h->ddots, sizeof(double) * (2 * cnt + 1),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const double xx = h->hdots[2 * cnt];
        for (int c = 0; c < cnt; c++) {
          const double den = sqrt(xx * h->hdots[2 * c + 1]);
          const double cosv = den > 0.0 ? fabs(h->hdots[2 * c]) / den : 1.0;
          if (cosv > h->opt.ortho_theta) { admit = false; break; }
        }
      }
    }
  }
  if (!admit) return 0;
  const int slot = h->ring_head;
  h->ring_head = (h->ring_head + 1) % h->opt.replay_cap;
  if (h->ring_count < h->opt.replay_cap) h->ring_count++;
  h->fresh.erase(std::remove(h->fresh.begin(), h->fresh.end(), slot), h->fresh.end());
  // a running phase reads its own copy of the ring; the store waits until that
  // copy has been taken
  if (h->phase_enqueued && s != h->phase_stream) CK(cudaStreamWaitEvent(s, h->ring_copied, 0));
  CK(launch_sumsq(b, h->N, h->scal + 1, s));
  CK(launch_sumsq(x, h->N, h->scal + 2, s));
  CK(launch_store_pair(b, x, h->N, h->scal + 1, h->ring_u + (long long)slot * h->ldv,
                       h->ring_t + (long long)slot * h->ldv, s));
  CK(cudaMemcpyAsync(h->hdots, h->scal + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  {
    const double bb = h->hdots[0], xx = h->hdots[1];
    const double ci = bb > 0.0 ? sqrt(xx / bb) : 1.0;
    if ((int)h->ring_c.size() < h->opt.replay_cap) h->ring_c.resize(h->opt.replay_cap, 0.0);
    h->ring_c[slot] = (std::isfinite(ci) && ci > 0.0) ? ci : 1.0;
  }
  // C_t holds the candidates admitted since the last training phase; the
  // warm-up pairs are part of X_t, so C_t starts empty after them (Algorithm 1)
  if (!warm) h->fresh.push_back(slot);
  return 1;
}

// The graph of one Adam step of the network for minibatch size B at the
// current depth, captured on first use (its launches, counted once at
// capture, are counted again at every replay).
const mlgmres::StepGraph& step_graph(mlgmres* h, int B) {
  for (const auto& g : h->graphs)
    if (g.B == B && g.extra == h->net.extra_active) return g;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
  const long long l0 = launches_so_far();
  const cudaError_t e = net_train_step_dev(h->net, B, h->ring_u_snap, h->ring_t_snap, h->ldv,
                                           h->picks_dev, h->net.ctr, h->opt.lr, h->loss_dev,
                                           h->cap_stream);
  const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
  const long long k = launches_so_far() - l0;
  note_launches(-k);
  CK(e);
  CK(e2);
  mlgmres::StepGraph g;
  g.B = B;
  g.extra = h->net.extra_active;
  g.kernels = k;
  const cudaError_t e3 = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(e3);
  h->graphs.push_back(g);
  return h->graphs.back();
}

// One training phase (Sec. 2.3) on stream s; see mlgmres_train_step.
void train_phase(mlgmres* h, cudaStream_t s, float* loss_host) {
  if (loss_host) *loss_host = -1.0f;
  if (h->ring_count == 0 || h->solves < h->opt.warmup_steps || h->opt.train_iters == 0) return;
  // one phase at a time: if the previous phase is still running, the caller
  // waits for it here (its ring and parameter snapshots are reused below)
  if (h->phase_enqueued) {
    const cudaError_t q = query_event(h->train_done);
    if (q == cudaErrorNotReady) {
      h->phase_waits++;
      CK(cudaEventSynchronize(h->train_done));
    } else {
      CK(q);
    }
  }
  // the ring was written on the solve streams; the handle's solves synchronise
  // before returning, so everything they enqueued is complete here.  The
  // phase trains on a copy of it, so that solves issued while it runs can
  // store new pairs.
  CK(cudaMemcpyAsync(h->ring_u_snap, h->ring_u, sizeof(float) * h->ldv * h->ring_count,
                     cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->ring_t_snap, h->ring_t, sizeof(float) * h->ldv * h->ring_count,
                     cudaMemcpyDeviceToDevice, s));
  CK(cudaEventRecord(h->ring_copied, s));
  // adaptive depth (Sec. 2.1): append a residual block when M_p(E_k) has not
  // improved by grow_tol since the previous training phase
  if (h->net.extra_max > 0 && !h->E_hist.empty()) {
    const size_t k = std::min<size_t>((size_t)h->opt.window_p, h->E_hist.size());
    double mp = 0.0;
    for (size_t i = h->E_hist.size() - k; i < h->E_hist.size(); i++) mp += h->E_hist[i];
    mp /= (double)k;
    if (h->mp_last_phase > 0.0 && mp >= (1.0 - h->opt.grow_tol) * h->mp_last_phase &&
        h->net.extra_active < h->net.extra_max)
      h->net.extra_active++;
    h->mp_last_phase = mp;
  }
  const int B = std::min(h->opt.batch, std::max(1, h->ring_count));
  // unit-scale targets: t / c with c the mean rms(x)/rms(b) over the ring
  double csum = 0.0;
  for (int i = 0; i < h->ring_count; i++) csum += h->ring_c[i];
  h->c_train = csum > 0.0 ? csum / h->ring_count : 1.0;
  const float tscale = (float)(1.0 / h->c_train);
  // every minibatch: the candidates admitted since the last phase (C_t, up
  // to B), then uniform samples of the ring
  const int iters = h->opt.train_iters;
  std::vector<int> picks((size_t)iters * B);
  for (int it = 0; it < iters; it++) {
    int* pick = picks.data() + (size_t)it * B;
    int k = 0;
    for (int f : h->fresh) {
      if (k >= B) break;
      pick[k++] = f;
    }
    while (k < B) pick[k++] = (int)(splitmix_next(h->rng_state) % (unsigned long long)h->ring_count);
  }
  if (h->linear) {
    for (int it = 0; it < iters; it++)
      CK(lin_train_batch(h->lin, B, h->ring_u_snap, h->ring_t_snap, h->ldv,
                         picks.data() + (size_t)it * B, tscale, h->opt.lr, h->loss_dev, s));
  } else {
    // the phase's inputs to device memory (the pinned staging is free: the
    // previous phase has completed), then train_iters replays of the step
    const mlgmres::StepGraph& g = step_graph(h, B);
    memcpy(h->picks_host, picks.data(), sizeof(int) * picks.size());
    *h->tscale_host = tscale;
    CK(cudaMemcpyAsync(h->picks_dev, h->picks_host, sizeof(int) * picks.size(),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(&h->net.ctr->tscale, h->tscale_host, sizeof(float),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(&h->net.ctr->iter, 0, sizeof(int), s));
    for (int it = 0; it < iters; it++) {
      CK(cudaGraphLaunch(g.exec, s));
      note_launches(g.kernels);
    }
    // the parameters the guess will take once the phase has completed
    CK(cudaMemcpyAsync(h->snap, h->net.master, sizeof(float) * h->net.nparams,
                       cudaMemcpyDeviceToDevice, s));
  }
  CK(cudaEventRecord(h->train_done, s));
  h->phase_enqueued = true;
  h->phase_stream = s;
  h->snap_pending = true;
  h->snap_c = h->c_train;
  h->snap_extra = h->net.extra_active;
  h->train_calls++;
  h->fresh.clear();
  h->cand_n = 0;
  if (loss_host) {
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(loss_host, h->loss_dev, sizeof(float), cudaMemcpyDeviceToHost));
  }
}

}  // namespace

extern "C" {

void mlgmres_default_options(mlgmres_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->m = 30;
  o->rtol = 1e-10;
  o->max_iters = 10000000;
  o->precision = MLGMRES_FP64;
  o->guess = MLGMRES_GUESS_ZERO;
  o->fallback = MLGMRES_GUESS_ZERO;
  o->replay_cap = 64;
  o->warmup_steps = 50;
  o->window_p = 10;
  o->ortho_theta = 0.9;
  o->deterministic_tos = 0;
  o->train_iters = 32;
  o->batch = 8;
  o->lr = 1e-3f;
  o->seed = 1;
  o->grid_blocks = 0;
  o->batch_slots = 0;
  o->barrier_timeout_s = 2.0;
  o->guess_smooth = 8;
  o->guess_select = 0;
  o->guess_omega = 0.8f;
  o->fault_inject = 0;
  o->v_stages = -1;
  o->retrain_after = 0;
  o->grow_blocks = 0;
  o->grow_tol = 0.02;
  o->compact = -1;
  o->model = MLGMRES_MODEL_CONV;
  o->overlap_train = 1;
}

mlgmres_status mlgmres_create(const mlgmres_grid* grid, const mlgmres_options* opt,
                              mlgmres_t* out) {
  if (!out) return MLGMRES_ERR_ARG;
  *out = nullptr;
  if (!grid || !opt) return MLGMRES_ERR_ARG;
  mlgmres* h = new mlgmres();
  try {
    ARG(grid->dim == 2 || grid->dim == 3, "dim must be 2 or 3");
    ARG(grid->n >= 1, "n must be >= 1");
    ARG(grid_points(grid->dim, grid->n) < (1ll << 30), "grid too large");
    ARG(grid->dim == 3 || grid->kappa_dev == nullptr, "kappa is for 3D grids only");
    check_options(h, opt);
    h->grid = *grid;
    h->opt = *opt;
    h->N = (int)grid_points(grid->dim, grid->n);
    h->fp32 = opt->precision == MLGMRES_FP32_REFINE;
    CK(cudaGetDevice(&h->dev));
    CK(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev));
    h->max_blocks = gmres_max_blocks(h->fp32, grid->dim, opt->m, &h->bs);
    CK(cudaGetLastError());
    ARG(h->max_blocks >= 1, "solver kernel cannot be resident");
    const bool force_compact =
        opt->compact == 1 && gmres_compact_ok(h->fp32, grid->dim, opt->m);
    const int maxb = force_compact ? std::max(h->max_blocks, gmres_compact_max_blocks(grid->dim, opt->m))
                                   : h->max_blocks;
    h->blocks = opt->grid_blocks > 0 ? std::min(opt->grid_blocks, maxb) : auto_blocks(h, h->N);
    h->blocks = std::min(h->blocks, kPartStride);
    h->ldv = ((long long)h->N + 63) / 64 * 64;
    // V slice in shared memory when it fits (the compact variant streams V)
    h->vsmem = single_vsmem(h, h->blocks, force_compact);
    const size_t es = h->fp32 ? sizeof(float) : sizeof(double);
    CK(cudaMalloc(&h->V, es * (size_t)vrows_p(opt->m + 1) * h->ldv));
    if (grid->dim == 3 && grid->kappa_dev && h->fp32) {
      // the FP32 passes read the operator's face coefficients instead of
      // forming harmonic means per point; w' and the coefficient arrays get
      // zero pads of n^2 + 64 points at both ends, so that no stencil window
      // of a bulk-copy stage is ever clipped (every stage takes the fast path)
      const long long pad = ((long long)h->grid.n * h->grid.n + 64 + 63) / 64 * 64;
      h->fstride = h->ldv + 2 * pad;
      CK(cudaMalloc(&h->W0_alloc, es * (size_t)h->fstride));
      CK(cudaMemset(h->W0_alloc, 0, es * (size_t)h->fstride));
      h->W0 = (char*)h->W0_alloc + es * pad;
      float* f = nullptr;
      CK(cudaMalloc(&f, sizeof(float) * 4 * (size_t)h->fstride));
      CK(cudaMemset(f, 0, sizeof(float) * 4 * (size_t)h->fstride));
      h->faces = f + pad;
    } else {
      CK(cudaMalloc(&h->W0_alloc, es * (size_t)h->ldv));
      h->W0 = h->W0_alloc;
    }
    CK(cudaMalloc(&h->W1, es * (size_t)h->ldv));
    CK(cudaMalloc(&h->part, sizeof(double) * part_doubles(kPartStride)));
    if (opt->compact != 0 && gmres_compact_ok(h->fp32, grid->dim, opt->m)) {
      // the compact variants keep each CTA's triangle R in HBM (L2-resident),
      // which leaves room for a second bulk-copy stage per warp
      h->rg_blocks = 2 * h->nsm;
      CK(cudaMalloc(&h->Rg, sizeof(double) * kRgDoubles * (size_t)h->rg_blocks));
    }
    h->group_cap = 1;
    h->cfg_cap = 1;
    if (opt->batch_slots > 0) {
      // batches may run the compact variant (two CTAs per SM) when V streams
      // from HBM: reserve workspaces for that many groups
      h->batch_compact = opt->compact != 0 && gmres_compact_ok(h->fp32, grid->dim, opt->m);
      const int bmax = h->batch_compact
                           ? std::max(h->max_blocks, gmres_compact_max_blocks(grid->dim, opt->m))
                           : h->max_blocks;
      h->batch_groups = std::min(opt->batch_slots, bmax);
      h->group_cap = std::max(h->group_cap, h->batch_groups);
      h->cfg_cap = kBatchCap;
      const size_t G = (size_t)h->batch_groups;
      CK(cudaMalloc(&h->Vb, es * G * (size_t)vrows_p(opt->m + 1) * h->ldv));
      CK(cudaMalloc(&h->Wb, es * G * 2 * (size_t)h->ldv));
      CK(cudaMalloc(&h->partb, sizeof(double) * G * part_doubles(1)));
    }
    CK(cudaMalloc(&h->bar, sizeof(unsigned long long) * h->group_cap));
    CK(cudaMalloc(&h->err, sizeof(int) * h->group_cap));
    CK(cudaMalloc(&h->dres, sizeof(DevResult) * h->cfg_cap));
    CK(cudaMallocHost(&h->hres, sizeof(DevResult) * h->cfg_cap));
    CK(cudaMalloc(&h->dcfg, sizeof(int) * (2 * (h->group_cap + 1) + h->cfg_cap)));
    CK(cudaMallocHost(&h->hcfg, sizeof(int) * (2 * (h->group_cap + 1) + h->cfg_cap)));
    CK(cudaMalloc(&h->dtasks, sizeof(SolveTask) * h->cfg_cap));
    CK(cudaMallocHost(&h->htasks, sizeof(SolveTask) * h->cfg_cap));
    CK(cudaMalloc(&h->dwork, sizeof(GroupWork) * h->group_cap));
    CK(cudaMallocHost(&h->hwork, sizeof(GroupWork) * h->group_cap));
    CK(cudaMalloc(&h->x_prev, sizeof(double) * h->ldv));
    CK(cudaMalloc(&h->x_alt, sizeof(double) * h->ldv));
    CK(cudaMalloc(&h->x_tmp, sizeof(double) * h->ldv));
    CK(cudaMalloc(&h->scal, sizeof(double) * (8 + 4096)));
    CK(cudaEventCreate(&h->ev0));
    CK(cudaEventCreate(&h->ev1));
    CK(cudaEventCreate(&h->ev2));
    CK(cudaEventCreateWithFlags(&h->train_done, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ring_copied, cudaEventDisableTiming));
    if (opt->guess == MLGMRES_GUESS_LEARNED && opt->retrain_after > 0) {
      // the phases the solves start run at the lowest stream priority, so that
      // the solver's CTAs are dispatched first when both wait for SMs
      int least = 0, greatest = 0;
      CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
      CK(cudaStreamCreateWithPriority(&h->train_stream, cudaStreamNonBlocking, least));
    }
    h->rng_state = opt->seed;
    // learned-guess machinery: at create for the LEARNED mode, else on the
    // first call of an nn_* inspection entry point
    if (opt->guess == MLGMRES_GUESS_LEARNED) ensure_net(h);
    CK(cudaDeviceSynchronize());
  } catch (const Fail& f) {
    fprintf(stderr, "mlgmres_create: %s\n", h->last_error.c_str());
    mlgmres_destroy(h);
    return f.st;
  }
  *out = h;
  return MLGMRES_OK;
}

void mlgmres_destroy(mlgmres_t h) {
  if (!h) return;
  cudaDeviceSynchronize();  // no phase may still use the workspace freed below
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  cudaFree(h->picks_dev);
  cudaFreeHost(h->picks_host);
  cudaFreeHost(h->tscale_host);
  cudaFree(h->Vb);
  cudaFree(h->Wb);
  cudaFree(h->partb);
  cudaFree(h->V);
  cudaFree(h->W0_alloc);
  if (h->faces) cudaFree(h->faces - (h->fstride - h->ldv) / 2);
  cudaFree(h->W1);
  cudaFree(h->part);
  cudaFree(h->Rg);
  cudaFree(h->bar);
  cudaFree(h->err);
  cudaFree(h->dres);
  cudaFreeHost(h->hres);
  cudaFree(h->dcfg);
  cudaFreeHost(h->hcfg);
  cudaFree(h->dtasks);
  cudaFreeHost(h->htasks);
  cudaFree(h->dwork);
  cudaFreeHost(h->hwork);
  cudaFree(h->x_prev);
  cudaFree(h->x_alt);
  cudaFree(h->x_tmp);
  cudaFree(h->u_in);
  cudaFree(h->y_out);
  cudaFree(h->scal);
  cudaFree(h->ring_u);
  cudaFree(h->ring_t);
  cudaFree(h->ddots);
  cudaFreeHost(h->hdots);
  cudaFree(h->loss_dev);
  cudaFree(h->ring_u_snap);
  cudaFree(h->ring_t_snap);
  cudaFree(h->snap);
  net_destroy(h->inf);
  net_destroy(h->net);
  lin_destroy(h->lin);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->ev2) cudaEventDestroy(h->ev2);
  if (h->train_done) cudaEventDestroy(h->train_done);
  if (h->ring_copied) cudaEventDestroy(h->ring_copied);
  if (h->train_stream) cudaStreamDestroy(h->train_stream);
  delete h;
}

const char* mlgmres_last_error(mlgmres_t h) { return h ? h->last_error.c_str() : "null handle"; }

mlgmres_status mlgmres_solve(mlgmres_t h, const double* b, double* x, void* stream,
                             mlgmres_result* res_out) {
  if (!h) return MLGMRES_ERR_ARG;
  h->last_error.clear();
  try {
    ARG(b && x, "b and x must be device pointers");
    ARG(b != x, "b and x must not alias");
    cudaStream_t s = (cudaStream_t)stream;
    mlgmres_result r;
    memset(&r, 0, sizeof(r));
    r.relres_learned = -1.0;
    const int N = h->N;
    const int mode = h->opt.guess;
    const double* x_alt = nullptr;
    int fallback = mode == MLGMRES_GUESS_LEARNED ? h->opt.fallback : mode;
    // guess in x
    if (fallback == MLGMRES_GUESS_ZERO || (fallback == MLGMRES_GUESS_PREV && !h->have_prev)) {
      CK(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
      r.guess_used = MLGMRES_GUESS_ZERO;
    } else if (fallback == MLGMRES_GUESS_PREV) {
      CK(cudaMemcpyAsync(x, h->x_prev, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      r.guess_used = MLGMRES_GUESS_PREV;
    } else {
      r.guess_used = MLGMRES_GUESS_USER;
    }
    if (mode == MLGMRES_GUESS_LEARNED) take_snapshot(h, s);
    if (mode == MLGMRES_GUESS_LEARNED && h->net_ready) {
      CK(cudaEventRecord(h->ev2, s));
      x_alt = learned_guess(h, b, s);
    }
    // one persistent launch from the guess in xs (optionally competing with
    // alt by initial residual), capped at maxit Arnoldi steps
    auto run_one = [&](double* xs, const double* alt, long long maxit) {
      SolveTask t;
      t.n = h->grid.n;
      t.N = N;
      t.b = b;
      t.x = xs;
      t.x_alt = alt;
      t.kappa = h->grid.kappa_dev;
      t.res = h->dres;
      t.hist = nullptr;
      t.hist_cap = 0;
      t.zero_x = 0;
      stage_single(h, t, h->blocks);
      run_solver(h, 1, 1, h->blocks, 0, s, h->vsmem, maxit, -1, use_compact(h));
      CK(cudaMemcpyAsync(h->hres, h->dres, sizeof(DevResult), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      return h->hres[0];
    };
    CK(cudaEventRecord(h->ev0, s));
    DevResult fin;
    long long extra_iters = 0;
    int extra_cycles = 0;
    if (x_alt && h->opt.guess_select == 0) {
      // E_k selection: one GMRES(m) cycle from each candidate, keep the one
      // with the smaller true residual after it and continue from there
      const long long cyc = std::min<long long>(h->opt.m, h->opt.max_iters);
      double* xa = const_cast<double*>(x_alt);
      const DevResult ra = run_one(xa, nullptr, cyc);
      const DevResult rb = run_one(x, nullptr, cyc);
      const bool learned = std::isfinite(ra.relres_true) && ra.status != kErrTimeout &&
                           (!std::isfinite(rb.relres_true) || ra.relres_true < rb.relres_true);
      const DevResult& w = learned ? ra : rb;
      const DevResult& l = learned ? rb : ra;
      if (learned) CK(cudaMemcpyAsync(x, xa, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      extra_iters = l.iters;
      extra_cycles = l.cycles;
      r.relres_learned = ra.relres_guess;
      if (learned) r.guess_used = MLGMRES_GUESS_LEARNED;
      if (w.status == 0 || w.status == kErrTimeout || w.status == kErrNonfinite ||
          w.iters + l.iters >= h->opt.max_iters) {
        fin = w;
      } else {
        fin = run_one(x, nullptr, h->opt.max_iters - w.iters - l.iters);
        fin.iters += w.iters;
        fin.cycles += w.cycles;
        fin.relres_first_cycle = w.relres_true;  // E_k of the chosen guess
        fin.relres_guess = w.relres_guess;
      }
    } else {
      fin = run_one(x, x_alt, h->opt.max_iters);
      if (fin.used_alt) r.guess_used = MLGMRES_GUESS_LEARNED;
      if (x_alt) r.relres_learned = fin.relres_alt;
    }
    CK(cudaEventRecord(h->ev1, s));
    CK(cudaMemcpyAsync(h->x_prev, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    h->have_prev = true;
    const int guess_used = r.guess_used;
    const double relres_learned = r.relres_learned;
    fill_result(fin, &r);
    r.iters += extra_iters;
    r.cycles += extra_cycles;
    r.guess_used = guess_used;
    r.relres_learned = relres_learned;
    if (x_alt) CK(cudaEventElapsedTime(&r.guess_ms, h->ev2, h->ev0));
    CK(cudaEventElapsedTime(&r.tos_ms, h->ev0, h->ev1));
    if (mode == MLGMRES_GUESS_LEARNED && r.status != MLGMRES_ERR_TIMEOUT)
      r.admitted = gate_and_store(h, b, x, r, s);
    // Algorithm 1's trigger: retrain once f_r under-performing steps were seen
    // since the previous phase (the first phase at tau0 takes the warm-up pairs)
    r.trained = 0;
    if (h->opt.guess == MLGMRES_GUESS_LEARNED && h->opt.retrain_after > 0 &&
        h->solves >= h->opt.warmup_steps &&
        (h->cand_n >= h->opt.retrain_after || h->train_calls == 0)) {
      const int before = h->train_calls;
      train_phase(h, h->train_stream, nullptr);
      r.trained = h->train_calls > before ? 1 : 0;
    }
    if (res_out) *res_out = r;
    if (r.status == MLGMRES_ERR_TIMEOUT) h->last_error = "device barrier wait timed out";
    if (r.status == MLGMRES_ERR_NONFINITE) h->last_error = "non-finite residual";
    return (mlgmres_status)r.status;
  } catch (const Fail& f) {
    return f.st;
  }
}

mlgmres_status mlgmres_solve_batch(mlgmres_t h, int count, const mlgmres_grid* grids,
                                   const double* const* b, double* const* x, void* stream,
                                   mlgmres_result* out) {
  if (!h) return MLGMRES_ERR_ARG;
  h->last_error.clear();
  try {
    ARG(h->batch_groups > 0, "the handle was created with batch_slots = 0");
    ARG(count >= 1 && count <= kBatchCap, "count must be in 1..4096");
    ARG(grids && b && x && out, "null argument");
    for (int i = 0; i < count; i++) {
      ARG(grids[i].dim == h->grid.dim, "every grid must have the handle's dim");
      ARG(grids[i].n >= 1 && grids[i].n <= h->grid.n, "grid side out of range");
      ARG(grids[i].dim == 3 || grids[i].kappa_dev == nullptr, "kappa is for 3D grids only");
      ARG(b[i] && x[i] && b[i] != x[i], "b and x must be distinct device pointers");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int dim = h->grid.dim;
    // CTA groups in proportion to the systems' cost (see schedule.cu)
    std::vector<int> sides(count), gctas, gof, order;
    for (int i = 0; i < count; i++) sides[i] = grids[i].n;
    const size_t es0 = h->fp32 ? sizeof(float) : sizeof(double);
    // shared-memory bytes of the largest CTA slice of V under a plan (0: does not fit)
    auto slice_need = [&](const std::vector<int>& gc, const std::vector<int>& go) {
      long long need = 0;
      for (int i = 0; i < count; i++) {
        const long long N = grid_points(dim, grids[i].n);
        const long long k = gc[go[i]];
        const long long chunk = ((N + k - 1) / k + 31) / 32 * 32;
        need = std::max(need, chunk * vrows_p(h->opt.m + 1) * (long long)es0);
      }
      return need <= gmres_vsmem_budget(h->fp32) ? (int)need : 0;
    };
    // one CTA per SM first; if the basis streams from HBM anyway, the compact
    // variant (two CTAs per SM) gets all the reserved CTAs
    int G = plan_batch(dim, count, sides.data(), std::min(h->batch_groups, h->max_blocks), gctas,
                       gof, order);
    const int vsmem = slice_need(gctas, gof);
    const bool compact = vsmem == 0 && h->batch_compact && h->batch_groups > h->max_blocks;
    if (compact) G = plan_batch(dim, count, sides.data(), h->batch_groups, gctas, gof, order);
    ARG(G >= 1 && G <= h->batch_groups, "batch schedule failed");
    int* gf = h->hcfg;
    int* tf = h->hcfg + (G + 1);
    int* to = h->hcfg + 2 * (G + 1);
    int pos = 0, cta = 0;
    for (int g = 0; g < G; g++) {
      gf[g] = cta;
      cta += gctas[g];
      tf[g] = pos;
      for (int i : order)
        if (gof[i] == g) to[pos++] = i;
    }
    gf[G] = cta;
    tf[G] = pos;
    const int grid_ctas = cta;
    const size_t es = h->fp32 ? sizeof(float) : sizeof(double);
    for (int i = 0; i < count; i++) {
      SolveTask t;
      t.n = grids[i].n;
      t.N = (int)grid_points(dim, grids[i].n);
      t.b = b[i];
      t.x = x[i];
      t.x_alt = nullptr;
      t.kappa = grids[i].kappa_dev;
      t.res = h->dres + i;
      t.hist = nullptr;
      t.hist_cap = 0;
      t.zero_x = h->opt.guess == MLGMRES_GUESS_USER ? 0 : 1;
      h->htasks[i] = t;
    }
    long long part_off = 0;
    for (int g = 0; g < G; g++) {
      GroupWork w;
      w.V = (char*)h->Vb + es * (size_t)g * vrows_p(h->opt.m + 1) * h->ldv;
      w.ldv = h->ldv;
      w.W0 = (char*)h->Wb + es * (size_t)g * 2 * h->ldv;
      w.W1 = (char*)w.W0 + es * h->ldv;
      w.part = h->partb + part_off;
      part_off += part_doubles(gctas[g]);
      w.pstride = gctas[g];
      w.Rg = h->Rg;
      w.bar.ctr = h->bar + g;
      w.bar.err = h->err + g;
      w.bar.nblocks = (unsigned)gctas[g];
      w.bar.timeout_ns = (unsigned long long)(h->opt.barrier_timeout_s * 1e9);
      h->hwork[g] = w;
    }
    CK(cudaEventRecord(h->ev0, s));
    run_solver(h, G, count, grid_ctas, 0, s, vsmem, -1, -1,
               (compact || (vsmem == 0 && h->batch_compact)) ? 1 : 0);
    CK(cudaEventRecord(h->ev1, s));
    CK(cudaMemcpyAsync(h->hres, h->dres, sizeof(DevResult) * count, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    int worst = MLGMRES_OK;
    for (int i = 0; i < count; i++) {
      memset(&out[i], 0, sizeof(out[i]));
      fill_result(h->hres[i], &out[i]);
      out[i].guess_used = h->opt.guess == MLGMRES_GUESS_USER ? MLGMRES_GUESS_USER : MLGMRES_GUESS_ZERO;
      out[i].relres_learned = -1.0;
      out[i].tos_ms = ms;
      const int st = out[i].status;
      if (st < 0 && (worst >= 0 || st < worst)) worst = st;
      else if (worst == MLGMRES_OK && st == MLGMRES_NOT_CONVERGED) worst = st;
    }
    return (mlgmres_status)worst;
  } catch (const Fail& f) {
    return f.st;
  }
}

mlgmres_status mlgmres_train_step(mlgmres_t h, void* side_stream, float* loss_host) {
  if (!h) return MLGMRES_ERR_ARG;
  h->last_error.clear();
  try {
    if (!h->net.master && !h->lin.T) {  // no learned guess on this handle: nothing to train
      if (loss_host) *loss_host = -1.0f;
      return MLGMRES_OK;
    }
    train_phase(h, (cudaStream_t)side_stream, loss_host);
    return MLGMRES_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

namespace {
struct TuneKey {
  int dev, dim, n, m, fp32;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, dim, n, m, fp32) < std::tie(o.dev, o.dim, o.n, o.m, o.fp32);
  }
};
struct TuneVal {
  int blocks, stages, compact;
  float us;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;
}  // namespace

mlgmres_status mlgmres_autotune(mlgmres_t h, const double* b, int steps, int retune, void* stream,
                                mlgmres_tuning* out) {
  if (!h) return MLGMRES_ERR_ARG;
  h->last_error.clear();
  double* xs = nullptr;
  try {
    ARG(b != nullptr, "null b");
    ARG(steps >= 0, "steps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (steps == 0) steps = 2 * h->opt.m;
    const TuneKey key{h->dev, h->grid.dim, h->grid.n, h->opt.m, h->fp32 ? 1 : 0};
    mlgmres_tuning t;
    memset(&t, 0, sizeof(t));
    auto apply = [&](int blocks, int stages, int compact) {
      if (h->opt.grid_blocks == 0) {
        h->blocks = blocks;
        h->vsmem = single_vsmem(h, blocks, compact != 0);
      }
      h->tuned_stages = stages;
      h->tuned_compact = compact && h->opt.grid_blocks == 0 ? 1 : 0;
    };
    if (!retune) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        apply(it->second.blocks, it->second.stages, it->second.compact);
        t.compact = h->tuned_compact;
        t.grid_blocks = h->blocks;
        t.v_stages = it->second.stages;
        t.us_per_step = it->second.us;
        t.from_cache = 1;
        if (out) *out = t;
        return MLGMRES_OK;
      }
    }
    wait_phase(h, s);
    CK(cudaMalloc(&xs, sizeof(double) * (size_t)h->N));
    // candidate CTA counts around one per 512 points, and the co-resident limit
    std::vector<int> blocks;
    const int cap = std::min(h->max_blocks, kPartStride);
    if (h->opt.grid_blocks > 0) {
      blocks.push_back(h->blocks);
    } else {
      const int base = auto_blocks(h, h->N);
      for (int c : {base / 2, base, base * 2, cap}) {
        c = std::max(1, std::min(c, cap));
        if (std::find(blocks.begin(), blocks.end(), c) == blocks.end()) blocks.push_back(c);
      }
    }
    int best_b = h->blocks, best_p = -1, best_c = 0;
    float best_us = INFINITY;
    // the compact variant (two CTAs per SM) as well, where it applies
    std::vector<std::pair<int, int>> shapes;  // (CTAs, compact)
    for (int nb : blocks) shapes.push_back({nb, 0});
    if (h->opt.compact == 1) shapes.clear();
    if (h->opt.grid_blocks == 0 && h->opt.v_stages != 0 && h->opt.compact != 0 &&
        gmres_compact_ok(h->fp32, h->grid.dim, h->opt.m)) {
      const int cmax = std::min(gmres_compact_max_blocks(h->grid.dim, h->opt.m), kPartStride);
      std::vector<int> cs = {cap, std::min(2 * cap, cmax)};
      const int two = std::min(2 * auto_blocks(h, h->N), cmax);
      if (std::find(cs.begin(), cs.end(), two) == cs.end()) cs.push_back(two);
      for (int c : cs)
        if (c > 0) shapes.push_back({c, 1});
    }
    for (auto [nb, compact] : shapes) {
      const int vs = single_vsmem(h, nb, compact != 0);
      // 2D passes keep V in shared memory when the slice fits
      const bool shared = h->grid.dim == 2 && vs > 0;
      std::vector<int> stages;
      if (shared) {
        stages.push_back(-1);
      } else if (compact) {
        for (int P : {2, 4, 8, 16})
          if (gmres_compact_cap(h->grid.dim, h->opt.m, P) > 0 && (h->opt.v_stages < 0 || P == h->opt.v_stages))
            stages.push_back(P);
      } else if (h->opt.v_stages >= 0) {
        stages.push_back(h->opt.v_stages);
      } else {
        for (int P : {0, 2, 4, 8, 16})
          if (P == 0 || gmres_bulk_cap(h->fp32, h->opt.m, P) > 0) stages.push_back(P);
      }
      for (int P : stages) {
        if (t.candidates >= 32) break;
        SolveTask tk;
        tk.n = h->grid.n;
        tk.N = h->N;
        tk.b = b;
        tk.x = xs;
        tk.x_alt = nullptr;
        tk.kappa = h->grid.kappa_dev;
        tk.res = h->dres;
        tk.hist = nullptr;
        tk.hist_cap = 0;
        tk.zero_x = 1;
        float ms = 0.f;
        for (int rep = 0; rep < 2; rep++) {  // the first run warms up
          stage_single(h, tk, nb);
          CK(cudaEventRecord(h->ev0, s));
          run_solver(h, 1, 1, nb, 0, s, vs, steps, P < 0 ? 0 : P, compact);
          CK(cudaEventRecord(h->ev1, s));
          CK(cudaMemcpyAsync(h->hres, h->dres, sizeof(DevResult), cudaMemcpyDeviceToHost, s));
          CK(cudaStreamSynchronize(s));
          CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        }
        const DevResult r = h->hres[0];
        ARG(r.status == 0 || r.status == 1, "autotune: a timed solve failed");
        const float us = r.iters > 0 ? 1000.f * ms / (float)r.iters : INFINITY;
        t.cand_blocks[t.candidates] = nb;
        t.cand_stages[t.candidates] = P;
        t.cand_us_per_step[t.candidates] = us;
        t.cand_compact[t.candidates] = compact;
        t.candidates++;
        if (us < best_us) {
          best_us = us;
          best_b = nb;
          best_p = P;
          best_c = compact;
        }
      }
    }
    CK(cudaFree(xs));
    xs = nullptr;
    apply(best_b, best_p, best_c);
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = TuneVal{best_b, best_p, best_c, best_us};
    }
    t.grid_blocks = h->blocks;
    t.v_stages = best_p;
    t.us_per_step = best_us;
    t.compact = h->tuned_compact;
    if (out) *out = t;
    return MLGMRES_OK;
  } catch (const Fail& f) {
    if (xs) cudaFree(xs);
    return f.st;
  }
}

mlgmres_status mlgmres_apply(mlgmres_t h, const double* u, double* out, void* stream) {
  if (!h) return MLGMRES_ERR_ARG;
  h->last_error.clear();
  try {
    ARG(u && out && u != out, "u and out must be distinct device pointers");
    cudaStream_t s = (cudaStream_t)stream;
    CK(launch_apply(h->grid.dim, h->grid.n, h->grid.kappa_dev, u, out, s));
    CK(cudaStreamSynchronize(s));
    return MLGMRES_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

mlgmres_status mlgmres_arnoldi(mlgmres_t h, const double* v0, int steps, double* H_host,
                               double* V_dev, int* done, void* stream) {
  if (!h) return MLGMRES_ERR_ARG;
  h->last_error.clear();
  try {
    ARG(v0 && H_host && V_dev && done, "null argument");
    ARG(steps >= 1 && steps <= h->opt.m, "steps must be in 1..m");
    cudaStream_t s = (cudaStream_t)stream;
    double* Hd = nullptr;
    CK(cudaMallocAsync(&Hd, sizeof(double) * (steps + 1) * steps, s));
    CK(cudaMemsetAsync(Hd, 0, sizeof(double) * (steps + 1) * steps, s));
    SolveTask t;
    t.n = h->grid.n;
    t.N = h->N;
    t.b = v0;
    t.x = nullptr;
    t.x_alt = nullptr;
    t.kappa = h->grid.kappa_dev;
    t.res = h->dres;
    t.hist = Hd;
    t.hist_cap = (long long)(steps + 1) * steps;
    t.zero_x = 0;
    stage_single(h, t, h->blocks);
    run_solver(h, 1, 1, h->blocks, steps, s);
    CK(cudaMemcpyAsync(h->hres, h->dres, sizeof(DevResult), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(H_host, Hd, sizeof(double) * (steps + 1) * steps, cudaMemcpyDeviceToHost,
                       s));
    CK(cudaStreamSynchronize(s));
    const int k = h->hres[0].status;
    ARG(k >= 1, "Arnoldi run failed (barrier timeout or zero start vector)");
    *done = k;
    CK(launch_basis_to_f64(h->fp32, h->V, h->opt.m + 1, k + 1, h->N, V_dev, s));
    CK(cudaFreeAsync(Hd, s));
    CK(cudaStreamSynchronize(s));
    return MLGMRES_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

mlgmres_status mlgmres_nn_param_count(mlgmres_t h, long long* count) {
  if (!h || !count) return MLGMRES_ERR_ARG;
  try {
    ensure_net(h);
  } catch (const Fail& f) {
    return f.st;
  }
  *count = model_params(h);
  return MLGMRES_OK;
}

mlgmres_status mlgmres_nn_get_params(mlgmres_t h, float* p, long long count) {
  if (!h) return MLGMRES_ERR_ARG;
  try {
    ensure_net(h);
    ARG(p && count == model_params(h), "bad parameter buffer");
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(p, model_master(h), sizeof(float) * count, cudaMemcpyDeviceToHost));
    return MLGMRES_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

mlgmres_status mlgmres_nn_set_params(mlgmres_t h, const float* p, long long count) {
  if (!h) return MLGMRES_ERR_ARG;
  try {
    ensure_net(h);
    ARG(p && count == model_params(h), "bad parameter buffer");
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(model_master(h), p, sizeof(float) * count, cudaMemcpyHostToDevice));
    if (!h->linear) {
      CK(net_adam_reset(h->net, 0));
      CK(net_sync_weights(h->net, 0));
      // the guess uses the parameters just set (they supersede a pending phase's)
      CK(net_copy_params(h->inf, h->net.master, 0));
      h->snap_pending = false;
    }
    CK(cudaDeviceSynchronize());
    return MLGMRES_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

mlgmres_status mlgmres_nn_forward(mlgmres_t h, int batch, const float* u, float* y,
                                  void* stream) {
  if (!h) return MLGMRES_ERR_ARG;
  try {
    ensure_net(h);
    ARG(u && y, "bad arguments");
    ARG(batch >= 1 && batch <= h->opt.batch, "batch must be in 1..opt.batch");
    cudaStream_t s = (cudaStream_t)stream;
    wait_phase(h, s);
    model_forward(h, batch, u, y, s);
    CK(cudaStreamSynchronize(s));
    return MLGMRES_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

mlgmres_status mlgmres_nn_loss_grad(mlgmres_t h, int batch, const float* u, const float* t,
                                    float* loss_host, float* grad_host, void* stream) {
  if (!h) return MLGMRES_ERR_ARG;
  try {
    ensure_net(h);
    ARG(u && t && loss_host && grad_host, "bad arguments");
    ARG(batch >= 1 && batch <= h->opt.batch, "batch must be in 1..opt.batch");
    cudaStream_t s = (cudaStream_t)stream;
    wait_phase(h, s);
    float* y = nullptr;
    CK(cudaMallocAsync(&y, sizeof(float) * (size_t)batch * h->N, s));
    model_forward(h, batch, u, y, s);
    if (h->linear)
      CK(lin_backward(h->lin, batch, u, y, t, 1.0f, h->loss_dev, s));
    else
      CK(net_backward(h->net, batch, u, y, t, 1.0f, h->loss_dev, s));
    CK(cudaMemcpyAsync(loss_host, h->loss_dev, sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(grad_host, model_grad(h), sizeof(float) * model_params(h),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaFreeAsync(y, s));
    CK(cudaStreamSynchronize(s));
    return MLGMRES_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

mlgmres_status mlgmres_guess(mlgmres_t h, const double* b, double* x, void* stream) {
  if (!h) return MLGMRES_ERR_ARG;
  h->last_error.clear();
  try {
    ARG(b && x && b != x, "b and x must be distinct device pointers");
    ensure_net(h);
    cudaStream_t s = (cudaStream_t)stream;
    // the guess of the latest phase: wait for it to complete
    if (h->phase_enqueued) CK(cudaEventSynchronize(h->train_done));
    take_snapshot(h, s);
    const double* g = learned_guess(h, b, s);
    CK(cudaMemcpyAsync(x, g, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return MLGMRES_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

mlgmres_status mlgmres_smooth(mlgmres_t h, const double* b, double* x, int sweeps,
                              void* stream) {
  if (!h) return MLGMRES_ERR_ARG;
  h->last_error.clear();
  try {
    ARG(b && x && b != x, "b and x must be distinct device pointers");
    ARG(sweeps >= 0 && sweeps <= 1000, "sweeps must be in 0..1000");
    cudaStream_t s = (cudaStream_t)stream;
    double* cur = x;
    double* oth = h->x_tmp;
    for (int k = 0; k < sweeps; k++) {
      CK(launch_jacobi(h->grid.dim, h->grid.n, h->grid.kappa_dev, b, cur, oth,
                       (double)h->opt.guess_omega, s));
      std::swap(cur, oth);
    }
    if (cur != x) CK(cudaMemcpyAsync(x, cur, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return MLGMRES_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

mlgmres_status mlgmres_nn_blocks(mlgmres_t h, int set_to, int* active) {
  if (!h || !active) return MLGMRES_ERR_ARG;
  h->last_error.clear();
  try {
    ARG(set_to >= -1, "set_to must be >= -1");
    ensure_net(h);
    if (set_to >= 0) {
      CK(cudaDeviceSynchronize());  // no training phase may be using the old depth
      h->net.extra_active = std::min(set_to, h->net.extra_max);
      h->inf.extra_active = h->net.extra_active;
    }
    *active = h->net.extra_active;
    return MLGMRES_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

mlgmres_status mlgmres_kernel_launches(long long* count) {
  if (!count) return MLGMRES_ERR_ARG;
  *count = launches_so_far();
  return MLGMRES_OK;
}

mlgmres_status mlgmres_replay_size(mlgmres_t h, int* count) {
  if (!h || !count) return MLGMRES_ERR_ARG;
  *count = h->ring_count;
  return MLGMRES_OK;
}

}  // extern "C"
