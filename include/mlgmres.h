/*
 * mlgmres.h - C ABI of the GB300 (sm_103a) MLGMRES library.
 *
 * MLGMRES (arXiv 2103.10975) solves a time series of linear systems A x_t = b_t
 * (Sec. 2: a time-dependent simulation is a sequence of such problems, one per
 * time step) with restarted GMRES(k) (Sec. 1.2), started from an initial guess
 * that a small network N(b) proposes and that is trained online on the
 * (b, x) pairs the solver itself produces (Sec. 2, Algorithm 1, Sec. 2.3).
 *
 * A is the discrete Laplacian with zero-Dirichlet walls on [-1,1]^d (Sec. 1.4
 * and the benchmark of Sec. 3), written as the SPD operator
 *   2D: (A u)_ij = (4 u_ij - u_{i-1,j} - u_{i+1,j} - u_{i,j-1} - u_{i,j+1}) / h^2
 *   3D: (A u)_c  = sum_faces kappa_f (u_c - u_nb) / h^2, kappa_f the harmonic
 *       mean of the two cell coefficients, kappa_c on a wall face (u_nb = 0),
 * h = 2/(n+1), n interior points per axis, row-major with x fastest
 * (2D index iy*n + ix; 3D index (iz*n + iy)*n + ix).
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are device pointers owned by the caller; the library
 *    never frees them.  Pointers named *_host are host memory.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Calls return after the work they enqueue has finished unless a
 *    comment says otherwise.
 *  - Errors are returned as mlgmres_status; no exception or abort crosses the
 *    ABI.  mlgmres_last_error() gives a text for the last failing call.
 *  - The library allocates all of its workspace (Krylov basis, Hessenberg
 *    state, network weights, Adam state, replay buffer) in mlgmres_create;
 *    solves allocate no device memory.  (A handle whose guess mode is not
 *    LEARNED allocates the network only on its first mlgmres_nn_* call.)
 *  - A handle is not thread safe; use one handle per host thread.
 */
#ifndef MLGMRES_H
#define MLGMRES_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlgmres* mlgmres_t;

typedef enum {
  MLGMRES_OK = 0,
  MLGMRES_NOT_CONVERGED = 1,  /* iteration cap reached; x holds the last iterate */
  MLGMRES_ERR_ARG = -1,       /* invalid argument (null pointer, bad size, bad option) */
  MLGMRES_ERR_CUDA = -2,      /* a CUDA runtime call failed (text in last_error) */
  MLGMRES_ERR_OOM = -3,       /* device allocation failed in create */
  MLGMRES_ERR_TIMEOUT = -4,   /* a device-side barrier wait exceeded its limit */
  MLGMRES_ERR_NONFINITE = -5  /* a residual or norm became NaN/Inf */
} mlgmres_status;

/* Model of the learned guess. */
enum {
  MLGMRES_MODEL_CONV = 0,
  MLGMRES_MODEL_LINEAR = 1
};

/* Arithmetic of the Arnoldi cycles. */
enum {
  MLGMRES_FP64 = 0,        /* everything in FP64 */
  MLGMRES_FP32_REFINE = 1  /* FP32 Krylov basis, SpMV and sweeps; FP64 true residual at
                              every restart, FP64 solution accumulation and FP64
                              Hessenberg / Givens least squares */
};

/* Initial-guess policy (Sec. 1.3: the guess x0 sets r0 = A x0 - b and with it
 * the whole Krylov space; Sec. 2.2: x0 = N(b) once the network is trained). */
enum {
  MLGMRES_GUESS_ZERO = 0,    /* x0 = 0 */
  MLGMRES_GUESS_PREV = 1,    /* x0 = solution of the previous solve on this handle */
  MLGMRES_GUESS_LEARNED = 2, /* x0 = c s N(b/s), s = rms(b); kept only if its residual
                                (after the first cycle, see guess_select) is finite and
                                below the fallback's */
  MLGMRES_GUESS_USER = 3     /* x0 = the caller's x_dev contents */
};

/* Problem geometry.  dim = 2 or 3; n = interior points per axis (square / cubic
 * grids); kappa_dev = n^3 cell coefficients (3D only; NULL = constant 1).  The
 * kappa array must stay valid for the handle's lifetime; it is read at the start
 * of every solve (the FP32 cycles of a single solve use face coefficients formed
 * from it then, the harmonic means in FP64 rounded once to FP32), so it may
 * change between solves. */
typedef struct {
  int dim;
  int n;
  const float* kappa_dev;
} mlgmres_grid;

typedef struct {
  int m;                     /* restart length k of GMRES(k), 1..64 */
  double rtol;               /* stop when ||b - A x|| <= rtol ||b|| (true FP64 residual) */
  long long max_iters;       /* cap on Arnoldi steps per solve (> 0) */
  int precision;             /* MLGMRES_FP64 | MLGMRES_FP32_REFINE */
  int guess;                 /* MLGMRES_GUESS_* */
  int fallback;              /* ZERO or PREV: the guess used before the network is trained
                                and whenever the learned guess loses */
  int replay_cap;            /* capacity of the (b, x) replay ring, pairs */
  int warmup_steps;          /* tau0: solves whose pairs are always kept (Sec. 2.3) */
  int window_p;              /* p of the moving average M_p (Sec. 2.2) */
  double ortho_theta;        /* admit a candidate if |cos(x_n, x_c)| <= theta for all
                                x_c in C_t (Sec. 2.2 spread check) */
  int deterministic_tos;     /* 1: the gate uses iteration counts in place of wall-clock TOS */
  int train_iters;           /* Adam steps per mlgmres_train_step */
  int batch;                 /* minibatch size; the network's activations index points in
                                32 bits, so 32 * batch * n^dim must stay below 2^31 (else
                                MLGMRES_ERR_ARG when the network is created) */
  float lr;                  /* Adam learning rate */
  unsigned long long seed;   /* network initialisation and minibatch sampling */
  int grid_blocks;           /* solver CTAs; 0 = pick from the problem size */
  int batch_slots;           /* CTAs (and at most as many basis workspaces for the handle's
                                grid) reserved for mlgmres_solve_batch (0 = none); at most
                                the number of co-resident CTAs is used */
  double barrier_timeout_s;  /* limit of every device-side wait (> 0) */
  int guess_smooth;          /* damped-Jacobi sweeps applied to the learned guess before it is
                                scored (0 = the network output as it is).  The sweeps remove
                                the white rounding noise of the BF16 network output, which A
                                amplifies by up to its condition number in the residual */
  float guess_omega;         /* damping of those sweeps (0 < omega <= 1) */
  int guess_select;          /* how the learned guess competes with the fallback:
                                0 = by E_k (Sec. 2.2): one GMRES(m) cycle from each, the
                                    smaller true residual after it wins and the solve
                                    continues from there (the losing cycle counts in
                                    iters);
                                1 = by the initial residual ||b - A x0|| */
  int fault_inject;          /* test hook, 0 in normal use.  1: the solver's CTA-group
                                barrier waits for one CTA more than is launched, so its
                                first wait runs out after barrier_timeout_s and the solve
                                returns MLGMRES_ERR_TIMEOUT (exercises the bounded-wait
                                path without faulting the GPU) */
  int v_stages;              /* basis held in HBM: most shared-memory stages per warp
                                through which the passes stream V with bulk copies (2..16;
                                a pass uses as many as fit in the warp's share of shared
                                memory for its j rows), or 0 for direct loads; -1 =
                                automatic (the autotuned value if mlgmres_autotune ran,
                                else 16) */
  int retrain_after;         /* f_r of Algorithm 1 (Sec. 2.2): when > 0, mlgmres_solve itself
                                starts a training phase (as mlgmres_train_step, on a stream
                                of the handle) at tau0 and then once f_r under-performing
                                steps (steps that fail the M_p test, whether or not their
                                pair passes the spread check: Algorithm 1's counter N) have
                                been seen since the previous phase; 0 = the caller decides
                                when to call mlgmres_train_step (fixed cadence) */
  int grow_blocks;           /* adaptive depth (Sec. 2.1): up to this many residual blocks
                                (0..4) are appended before the output layer, one at a
                                training phase whose M_p(E_k) has stagnated (0 = fixed
                                depth) */
  double grow_tol;           /* stagnation: M_p(E_k) at a training phase is above
                                (1 - grow_tol) times its value at the previous phase */
  int compact;               /* the two-CTAs-per-SM variants (at most 128 registers, smaller
                                shared state) for FP32 grids: 2D with m <= 47 (V slices in
                                shared memory when they fit, else streamed), 3D with m <= 55
                                (streamed): -1 = if the autotuner chose it, 0 = never, 1 =
                                always (where it applies) */
  int model;                 /* MLGMRES_MODEL_CONV: the multi-scale network of Sec. 2.1;
                                MLGMRES_MODEL_LINEAR: one dense layer x0 = c s T (b/s) =
                                c T b (the simplified model of Sec. 3.1, for studying the
                                spectrum of A T; N <= 4096, T starts at 0 and trains by
                                plain gradient descent with step lr; the nn_* entry
                                points then see T, row-major, as the parameters) */
  int overlap_train;         /* 1: training phases run beside the solves (Sec. 2.3 trains in
                                real time while the simulation goes on): the guess is formed
                                by an inference copy of the network, and a solve takes the
                                parameters of the latest phase only once that phase has
                                completed -- it never waits for one that is still running
                                (unless the phase runs on the solve's own stream); 0: every
                                solve waits for the latest phase first (deterministic, the
                                linear model always does) */
} mlgmres_options;

typedef struct {
  long long iters;           /* Arnoldi steps (matrix-vector products in cycles) */
  int cycles;                /* restart cycles */
  int status;                /* mlgmres_status of this solve */
  int guess_used;            /* MLGMRES_GUESS_* actually used */
  int admitted;              /* 1 if the (b, x) pair entered the replay ring */
  double bnorm;              /* ||b|| */
  double relres_true;        /* ||b - A x|| / ||b||, FP64, at exit */
  double relres_first_cycle; /* E_k: true relative residual after the first cycle (Sec. 2.2) */
  double relres_guess;       /* ||b - A x0|| / ||b|| of the guess used */
  double relres_learned;     /* initial relative residual of the learned candidate (-1 if
                                none was formed) */
  float tos_ms;              /* device time of the solve kernel (TOS, Sec. 2.2) */
  float guess_ms;            /* device time of the learned-guess forward pass and smoothing */
  int trained;               /* 1 if this solve started a training phase (retrain_after) */
} mlgmres_result;

/* Fills *opt with the defaults: m = 30, rtol = 1e-10, max_iters = 10^7, FP64,
 * guess ZERO, fallback ZERO, replay_cap 64, warmup 50, p = 10, theta = 0.9,
 * deterministic_tos 0, train_iters 32, batch 8, lr 1e-3, seed 1,
 * grid_blocks 0, batch_slots 0, barrier_timeout_s 2, guess_smooth 8, guess_omega 0.8,
 * guess_select 0, fault_inject 0, v_stages -1, retrain_after 0, grow_blocks 0,
 * grow_tol 0.02, compact -1, model CONV, overlap_train 1. */
void mlgmres_default_options(mlgmres_options* opt);

/* Creates a solver for one grid and allocates all workspace on the current
 * CUDA device.  Returns ERR_ARG for an invalid grid or option, ERR_OOM if the
 * workspace does not fit, ERR_CUDA on other CUDA errors; *out is NULL then. */
mlgmres_status mlgmres_create(const mlgmres_grid* grid, const mlgmres_options* opt,
                              mlgmres_t* out);

/* Solves A x = b (GMRES(m), Sec. 1.2) to the handle's rtol.
 * b_dev: N doubles (input).  x_dev: N doubles (output; input too in guess mode
 * USER).  Both must be 8-byte aligned and must not overlap.  When the handle's
 * guess mode is LEARNED the (b, x) pair then passes Algorithm 1's gate and may
 * enter the replay ring (res->admitted).  On NOT_CONVERGED x holds the last
 * iterate and res->relres_true its residual.  b = 0 gives x = 0, iters = 0, OK.
 * res may be NULL. */
mlgmres_status mlgmres_solve(mlgmres_t h, const double* b_dev, double* x_dev, void* stream,
                             mlgmres_result* res);

/* Solves `count` (1..4096) independent systems, each on its own grid
 * (grids[i].dim must equal the handle's dim, grids[i].n must not exceed the
 * handle's n; 3D grids may carry their own kappa), in one persistent launch.
 * The handle must have been created with batch_slots > 0.  Its CTAs are split
 * into groups by mlgmres_batch_plan: a system whose n^(dim+2) cost estimate
 * exceeds the ideal per-CTA share gets a group of several CTAs, the rest of
 * the CTAs form one-CTA groups, and every group works through its list of
 * systems largest first.  b_dev[i], x_dev[i]: device
 * arrays of grids[i].n^dim doubles; b_dev and x_dev themselves are HOST arrays
 * of device pointers.  Guesses are ZERO (USER when the handle's mode is USER);
 * no pair is collected.  out: `count` results (host); tos_ms of each is the
 * whole launch.  Returns the worst status. */
mlgmres_status mlgmres_solve_batch(mlgmres_t h, int count, const mlgmres_grid* grids,
                                   const double* const* b_dev, double* const* x_dev,
                                   void* stream, mlgmres_result* out);

/* One training phase (Sec. 2.3): opt.train_iters Adam steps on the MSE loss
 * ||N(b/s) - x/(c s)||^2 over minibatches drawn from the replay ring (c is the
 * mean of rms(x)/rms(b) over the ring, so the targets have unit scale; the
 * guess is then x0 = c s N(b/s)), each batch
 * holding every candidate pair admitted since the previous call (C_t of
 * Algorithm 1, up to opt.batch) and uniform samples of the rest.  The phase
 * trains on a copy of the ring taken at its start, so solves issued while it
 * runs may store new pairs.  Runs on side_stream and returns once enqueued.
 * With opt.overlap_train = 1 the solves do not wait for it: each takes the
 * phase's parameters once the phase has completed (solves issued on another
 * stream while it runs keep the previous ones); with 0 the next solve waits
 * for it.  If the previous phase is still running, this call first waits for
 * it on the host (one phase at a time).  loss_host (may be NULL) receives the
 * mean loss of the last minibatch after the phase completes (this
 * synchronises). Does nothing and returns OK while the ring is empty or
 * before tau0 solves. */
mlgmres_status mlgmres_train_step(mlgmres_t h, void* side_stream, float* loss_host);

/* Text of the last error on this handle ("" if none); valid until the next call. */
const char* mlgmres_last_error(mlgmres_t h);

/* Frees the handle and all its workspace.  NULL is ignored. */
void mlgmres_destroy(mlgmres_t h);

/* ---- inspection entry points (used by tests; same conventions) ---------- */

/* out = A u in FP64 on the handle's grid (u_dev, out_dev: N doubles). */
mlgmres_status mlgmres_apply(mlgmres_t h, const double* u_dev, double* out_dev, void* stream);

/* Runs `steps` (<= m) Arnoldi steps from v0 with the handle's precision and
 * Gram-Schmidt (classical, twice), without restarts or Givens, and copies the
 * Hessenberg matrix to H_host ((steps+1) x steps, column-major, leading
 * dimension steps+1) and the basis to V_dev ((steps+1) x N doubles, row per
 * vector).  Returns the number of steps done (breakdown may stop it early)
 * through *done. */
mlgmres_status mlgmres_arnoldi(mlgmres_t h, const double* v0_dev, int steps, double* H_host,
                               double* V_dev, int* done, void* stream);

/* The network of Sec. 2.1 exists in 2D (3x3 kernels, 2x2 average pooling,
 * bilinear upsampling) and, for dim = 3 handles, in 3D (3x3x3 kernels, 2x2x2
 * pooling, trilinear upsampling); inputs are n^dim values per sample.
 * Number of network parameters (FP32 master copy). */
mlgmres_status mlgmres_nn_param_count(mlgmres_t h, long long* count);

/* Copies the FP32 master parameters out / in, in the order
 * in.w, in.b, level[0].w, level[0].b, ..., dil.w, dil.b, out.w, out.b (then
 * res1.w, res1.b, ... when opt.grow_blocks > 0)
 * (weights as [out][in][ky][kx], 3D [out][in][kz][ky][kx]).  Setting them also
 * resets Adam's moments. */
mlgmres_status mlgmres_nn_get_params(mlgmres_t h, float* params_host, long long count);
mlgmres_status mlgmres_nn_set_params(mlgmres_t h, const float* params_host, long long count);

/* Network output for `batch` normalised inputs: y_dev[b] = N(u_dev[b]) (FP32,
 * batch x N each), computed with the BF16 inference weights. */
mlgmres_status mlgmres_nn_forward(mlgmres_t h, int batch, const float* u_dev, float* y_dev,
                                  void* stream);

/* Mean-squared loss 1/(B N) sum_b ||N(u_b) - t_b||^2 and its gradient with
 * respect to every parameter (grad_host: param_count floats, same order as
 * get_params), at the current weights; does not update anything. */
mlgmres_status mlgmres_nn_loss_grad(mlgmres_t h, int batch, const float* u_dev,
                                    const float* t_dev, float* loss_host, float* grad_host,
                                    void* stream);

/* The network's initial guess for b alone (the x0 = N(b) step of Sec. 2.2,
 * as mlgmres_solve forms it in guess mode LEARNED): x_dev = c s N(b/s) with
 * s = rms(b) and c the target scale of the last training phase, after
 * opt.guess_smooth damped-Jacobi sweeps.  Runs no GMRES and records nothing.
 * b_dev, x_dev: N doubles each, distinct.  An untrained network gives its
 * initial output. */
mlgmres_status mlgmres_guess(mlgmres_t h, const double* b_dev, double* x_dev, void* stream);

/* The damped-Jacobi sweeps that follow the network in the learned guess:
 * `sweeps` times x <- x + omega D^-1 (b - A x), D the diagonal of A (4/h^2 in
 * 2D; the sum of the face coefficients over h^2 in 3D) and omega the handle's
 * guess_omega, on x_dev in place (input: the starting x; output: the result).
 * b_dev, x_dev: N doubles each, distinct.  sweeps in 0..1000.  Not a step of
 * the paper: it is how the library removes the BF16 rounding noise of the
 * network's output, exposed so that its effect can be measured on its own. */
mlgmres_status mlgmres_smooth(mlgmres_t h, const double* b_dev, double* x_dev, int sweeps,
                              void* stream);

/* Residual blocks appended so far by the adaptive growth (opt.grow_blocks).
 * set_to >= 0 sets the count (clamped to opt.grow_blocks; for tests and for
 * callers that choose the depth themselves), -1 only queries.  *active
 * receives the count after the call.  Parameters of every possible block are
 * always part of the parameter array (after out.b: res1.w, res1.b, ...). */
mlgmres_status mlgmres_nn_blocks(mlgmres_t h, int set_to, int* active);

/* Pairs currently in the replay ring. */
mlgmres_status mlgmres_replay_size(mlgmres_t h, int* count);

/* Latency floor of the solver's Arnoldi step (the paper has no counterpart: a
 * profiling probe).  One persistent cooperative launch of `ctas` CTAs (256
 * threads, one per SM, like mlgmres_solve's kernel) runs `steps` steps with j
 * cycling 0..m-1 and does in each only the step's two group exchanges -- the
 * per-CTA partial sums of j+2 slots, the group barrier and the gather of the
 * j+2 sums, with the solver's own code -- and no pass over a grid and no
 * scalar recurrence.  *us_per_step receives the device time per step of the
 * second of two launches (CUDA events on the legacy default stream).  Allocates
 * and frees its own partial-sum and barrier buffers and synchronises.
 * ERR_ARG for ctas outside 1..min(co-resident CTAs, 1024), m outside 1..64,
 * steps < 1 or a NULL output; ERR_TIMEOUT if a barrier wait ran out (2 s). */
mlgmres_status mlgmres_exchange_floor(int ctas, int m, int steps, float* us_per_step);

/* Number of CUDA kernels this library has launched in this process so far (all
 * handles).  Used to count the kernels inside a timed region. */
mlgmres_status mlgmres_kernel_launches(long long* count);

/* ---- solving without allocating ------------------------------------------ */

/* The paper has no counterpart to this entry point.
 *
 * Solves A x = b on a 2D n x n grid like mlgmres_solve with guess ZERO and
 * FP32-refined precision, but allocates no device memory at all: no handle is
 * created, and the Krylov basis, work vectors, partial sums and barrier state
 * live in one fixed array compiled into the library (about 10 MB, held on every
 * GPU that loads the library until the process exits).  It is meant for
 * callers that cannot call cudaMalloc -- a code whose memory pool has already
 * taken all free device memory, a host thread that must not enter an
 * allocator while it solves, or a plug-in that is not allowed to own device
 * memory.
 *   n, m:            n*n <= 65536 (grids up to 256 x 256) and 1 <= m <= 32;
 *                    larger sizes return MLGMRES_ERR_ARG.
 *   rtol, max_iters: as in mlgmres_options.
 *   b_dev, x_dev:    caller-owned device arrays of n*n doubles (b input, x output).
 *   res:             may be NULL.
 * The first call on a device looks up the array's device address for that
 * device (and loads the module holding the array).
 * Every call uses the same array and it keeps the last call's contents (the
 * barrier state is cleared at the start of each call): calls that overlap on
 * the GPU -- from two streams or two threads -- race with each other and must
 * be serialised by the caller.  Synchronises the stream before returning. */
mlgmres_status mlgmres_solve_static(int n, int m, double rtol, long long max_iters,
                                    const double* b_dev, double* x_dev, void* stream,
                                    mlgmres_result* res);

/* Result of mlgmres_autotune. */
typedef struct {
  int grid_blocks;        /* chosen CTA count for single solves */
  int v_stages;           /* chosen bulk-copy stages (0 = direct loads; -1 = not applicable:
                             FP64, or V in shared memory) */
  float us_per_step;      /* device time per Arnoldi step at the choice */
  int candidates;         /* configurations timed (<= 32) */
  int cand_blocks[32];
  int cand_stages[32];
  float cand_us_per_step[32];
  int from_cache;         /* 1: taken from the process-wide cache, nothing was timed */
  int compact;            /* 1: the chosen shape is a compact variant (two CTAs of at most
                             128 registers per SM; see mlgmres_options.compact) */
  int cand_compact[32];
} mlgmres_tuning;

/* Autotuner (the paper has no counterpart).  Times capped solves of `steps`
 * Arnoldi steps (0 = 2m) of A x = b_dev from x0 = 0, with the handle's
 * precision and m, for candidate launch shapes -- CTA counts around one per
 * 512 grid points (x1/2, x1, x2, and the co-resident maximum) and, for an FP32
 * basis held in HBM, 0/2/4/8/16 bulk-copy stages, and for FP32 grids the compact
 * variants at one and two CTAs per SM -- and keeps the fastest per
 * step for this handle's later solves (options grid_blocks and v_stages set
 * explicitly at create still win).  Results are cached per process by
 * (device, dim, n, m, precision); a cached shape is reused without timing
 * unless `retune` is 1.  Writes into an internal scratch vector (allocated
 * here and freed before returning), records no (b, x) pair, synchronises
 * `stream`.  out may be NULL.  ERR_ARG on a NULL handle or b_dev, steps < 0. */
mlgmres_status mlgmres_autotune(mlgmres_t h, const double* b_dev, int steps, int retune,
                                void* stream, mlgmres_tuning* out);

/* The batch schedule mlgmres_solve_batch uses, computed on the host only (no
 * device work; the paper has no counterpart: it solves one system at a time).
 * Splits `ctas` CTAs into groups and assigns each of the `count` systems of
 * sides n[0..count-1] (dim 2 or 3) to one group.  Cost of a system: N n^2
 * (Arnoldi steps grow like n^2, each moves O(N) values).  Systems whose cost
 * exceeds total / ctas get a dedicated group of ceil(cost / (total / ctas))
 * CTAs (at most one per 512 points, and one CTA is kept back while systems
 * remain); the remaining CTAs become one-CTA groups (no more than systems
 * left); the remaining systems, largest first, go to the group on which they
 * would finish earliest.  Outputs (host arrays): *groups = G;
 * group_ctas[0..G-1] (room for `ctas` ints) sum to at most ctas;
 * group_of[0..count-1] in 0..G-1.  ERR_ARG on a bad dim, count < 1, ctas < 1,
 * a side < 1 or a NULL pointer. */
mlgmres_status mlgmres_batch_plan(int dim, int count, const int* n, int ctas, int* groups,
                                  int* group_ctas, int* group_of);

#ifdef __cplusplus
}
#endif

#endif /* MLGMRES_H */
