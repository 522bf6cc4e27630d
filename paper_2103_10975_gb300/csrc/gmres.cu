// Persistent restarted GMRES(m) for the discrete Poisson operator (Sec. 1.2,
// Sec. 1.4, Sec. 3 of arXiv 2103.10975), one cooperative launch per solve or
// per batch of solves.
//
// Each CTA group (all CTAs for a single solve) owns one system at a time; the
// grid points are split into contiguous per-CTA ranges.  One Arnoldi step j is
// three fused passes separated by group barriers:
//   A: w = A v_j (matrix-free stencil on the unnormalised previous vector,
//      scaled by 1/h_{j,j-1} -- lazy normalisation), store v_j, and
//      h1 = V_{0..j}^T w, ||w||^2 partial sums.
//   B: w -= V h1 and h2 = V^T w in the same pass over V (each thread keeps its
//      column of V in registers between the update and the dots).
//   C: w -= V h2 and ||w||^2.
// (classical Gram-Schmidt applied twice.)  After each barrier every CTA sums
// the per-CTA partials in the same fixed order, so all CTAs hold bit-identical
// coefficients and run the Givens update of the Hessenberg least-squares
// problem redundantly in shared memory (FP64) with no extra synchronisation.
// At a cycle end the back-substitution y = H^{-1} g runs in shared memory,
// x += V y is accumulated in FP64 and the true residual b - A x is recomputed
// in FP64 (the restart of GMRES(k)).  The FP32 variant stores V and w in FP32
// and so runs every cycle as one step of mixed-precision iterative refinement.
#include <math.h>

#include "solver.h"

namespace mlg {

// ---------------------------------------------------------------- stencils --
// Sum over faces of kappa_f (u_c - u_nb), unscaled; neighbours outside the grid
// are 0 (zero Dirichlet).  Writing the 2D/3D Laplacian as a sum of differences
// keeps the rounding error relative to |A u| instead of |u|.
template <typename T>
__device__ __forceinline__ T stencil2d(const T* __restrict__ u, int i, int n, T uc) {
  const int ix = i % n;
  const int iy = i / n;
  const T l = ix > 0 ? ldcg(u + i - 1) : T(0);
  const T r = ix < n - 1 ? ldcg(u + i + 1) : T(0);
  const T d = iy > 0 ? ldcg(u + i - n) : T(0);
  const T t = iy < n - 1 ? ldcg(u + i + n) : T(0);
  return ((uc - l) + (uc - r)) + ((uc - d) + (uc - t));
}

template <typename T>
__device__ __forceinline__ T face(T kc, T knb) { return T(2) * kc * knb / (kc + knb); }

template <typename T>
__device__ __forceinline__ T stencil3d(const T* __restrict__ u, int i, int n,
                                       const float* __restrict__ kappa, T uc) {
  const int ix = i % n;
  const int t = i / n;
  const int iy = t % n;
  const int iz = t / n;
  const int nn = n * n;
  const int off[6] = {-1, 1, -n, n, -nn, nn};
  const bool has[6] = {ix > 0, ix < n - 1, iy > 0, iy < n - 1, iz > 0, iz < n - 1};
  T acc = T(0);
  if (kappa) {
    const T kc = (T)__ldg(kappa + i);
#pragma unroll
    for (int f = 0; f < 6; f++) {
      if (has[f]) {
        const T knb = (T)__ldg(kappa + i + off[f]);
        acc += face(kc, knb) * (uc - ldcg(u + i + off[f]));
      } else {
        acc += kc * uc;
      }
    }
  } else {
#pragma unroll
    for (int f = 0; f < 6; f++) acc += has[f] ? (uc - ldcg(u + i + off[f])) : uc;
  }
  return acc;
}

template <typename T, int DIM>
__device__ __forceinline__ T stencil(const T* __restrict__ u, int i, int n,
                                     const float* __restrict__ kappa, T uc) {
  if constexpr (DIM == 2)
    return stencil2d<T>(u, i, n, uc);
  else
    return stencil3d<T>(u, i, n, kappa, uc);
}

// ----------------------------------------------------------- shared state --
template <int MAXM, int BS>
struct Smem {
  double red[BS / 32][MAXM + 2];
  double tot[MAXM + 2];
  double H[(MAXM + 1) * MAXM];  // column-major, leading dimension MAXM+1
  double cs[MAXM], sn[MAXM], g[MAXM + 1], y[MAXM];
  double hn, anorm, bnorm, beta;
  int ctl;
  int flag;
};

// Warp partial of slot k (lane 0 stores it); block_finish then adds the warp
// partials of slots 0..L-1 and writes the CTA's sums to part[k*kPartStride + lb].
template <int LMAX>
__device__ __forceinline__ void warp_slot(double (*red)[LMAX], int k, double v) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
}

template <int LMAX, int BS>
__device__ __forceinline__ void block_finish(int L, double* part, int lb, double (*red)[LMAX]) {
  __syncthreads();
  for (int k = threadIdx.x; k < L; k += BS) {
    double s = 0.0;
    for (int w = 0; w < BS / 32; w++) s += red[w][k];
    part[(long long)k * kPartStride + lb] = s;
  }
}

// Sum of the group's partials for k < L, identical in every CTA.
template <int BS>
__device__ __forceinline__ void gather(const double* part, int L, int nb, double* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = warp; k < L; k += BS / 32) {
    double s = 0.0;
    for (int g = lane; g < nb; g += 32) s += ldcg(part + (long long)k * kPartStride + g);
    s = warp_sum(s);
    if (lane == 0) tot[k] = s;
  }
  __syncthreads();
}

// --------------------------------------------------------------- one solve --
template <typename T, int DIM, int MAXM, int BS>
__device__ void solve_one(const KParams& kp, const SolveTask& tk, const GroupWork& w, int lb,
                          int nb, unsigned long long& epoch, Smem<MAXM, BS>& sm) {
  constexpr int LD = MAXM + 1;
  constexpr int LMAX = MAXM + 2;
  const int tid = threadIdx.x;
  const int n = tk.n;
  const int N = tk.N;
  const int m = kp.m;
  const bool arnoldi = kp.arnoldi_steps > 0;
  int chunk = (N + nb - 1) / nb;
  chunk = (chunk + 3) & ~3;
  const int lo = min(N, lb * chunk);
  const int hi = min(N, lo + chunk);
  T* __restrict__ V = (T*)w.V;
  const long long ldv = w.ldv;
  T* bufs[2] = {(T*)w.W0, (T*)w.W1};
  const double h = 2.0 / (n + 1);
  const double s2 = 1.0 / (h * h);
  const float* kappa = tk.kappa;
  int red = 0;
  auto part = [&]() { return w.part + (long long)(red & 1) * LMAX * kPartStride; };
  const bool leader = (lb == 0 && tid == 0);

  long long iters = 0;
  int cycles = 0;
  int status = 1;
  double relres = 0.0, relres_first = -1.0, relres_guess = -1.0, relres_alt = -1.0;
  int used_alt = 0;
  int cur = 0;
  double bnorm = 0.0;
  bool ok = true;

  // ---- phase 0: ||b||, and the residuals of both guesses when an alternative
  // (learned) guess competes with the fallback already in x.
  if (!arnoldi) {
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
    const bool alt = tk.x_alt != nullptr;
    for (int i = lo + tid; i < hi; i += BS) {
      const double bi = tk.b[i];
      v0 += bi * bi;
      if (alt) {
        const double xc = ldcg(tk.x + i);
        const double r0 = bi - s2 * stencil<double, DIM>(tk.x, i, n, kappa, xc);
        const double ac = ldcg(tk.x_alt + i);
        const double r1 = bi - s2 * stencil<double, DIM>(tk.x_alt, i, n, kappa, ac);
        v1 += r0 * r0;
        v2 += r1 * r1;
      }
    }
    warp_slot<LMAX>(sm.red, 0, v0);
    if (alt) {
      warp_slot<LMAX>(sm.red, 1, v1);
      warp_slot<LMAX>(sm.red, 2, v2);
    }
    block_finish<LMAX, BS>(alt ? 3 : 1, part(), lb, sm.red);
    ok = group_sync(w.bar, epoch, &sm.flag);
    if (!ok) goto abort;
    gather<BS>(part(), alt ? 3 : 1, nb, sm.tot);
    red++;
    bnorm = sqrt(sm.tot[0]);
    if (bnorm == 0.0) {  // A x = 0 has the unique solution 0
      for (int i = lo + tid; i < hi; i += BS) tk.x[i] = 0.0;
      status = 0;
      relres = 0.0;
      relres_guess = 0.0;
      relres_first = 0.0;
      goto finish;
    }
    if (alt) {
      const double rx = sqrt(sm.tot[1]), ra = sqrt(sm.tot[2]);
      relres_alt = ra / bnorm;
      if (isfinite(ra) && ra < rx) {
        used_alt = 1;
        for (int i = lo + tid; i < hi; i += BS) tk.x[i] = tk.x_alt[i];
        ok = group_sync(w.bar, epoch, &sm.flag);
        if (!ok) goto abort;
      }
    }
  }

  for (;;) {
    // ---- restart: P = r = b - A x (FP64), beta = ||r||
    {
      double v0 = 0.0;
      T* P = bufs[cur];
      for (int i = lo + tid; i < hi; i += BS) {
        double ri;
        if (arnoldi) {
          ri = tk.b[i];
        } else {
          const double xc = ldcg(tk.x + i);
          ri = tk.b[i] - s2 * stencil<double, DIM>(tk.x, i, n, kappa, xc);
        }
        P[i] = (T)ri;
        v0 += ri * ri;
      }
      warp_slot<LMAX>(sm.red, 0, v0);
      block_finish<LMAX, BS>(1, part(), lb, sm.red);
      ok = group_sync(w.bar, epoch, &sm.flag);
      if (!ok) goto abort;
      gather<BS>(part(), 1, nb, sm.tot);
      red++;
    }
    const double beta = sqrt(sm.tot[0]);
    if (arnoldi) {
      bnorm = beta;
    } else {
      relres = beta / bnorm;
      if (cycles == 0) relres_guess = relres;
      if (cycles == 1) relres_first = relres;
      if (!isfinite(relres)) { status = kErrNonfinite; break; }
      if (relres <= kp.rtol) { status = 0; break; }
      if (iters >= kp.max_iters) { status = 1; break; }
    }
    if (beta == 0.0) { status = 0; break; }
    double hn = beta;  // norm of the unnormalised vector in bufs[cur]
    if (tid == 0) {
      for (int k = 0; k <= MAXM; k++) sm.g[k] = 0.0;
      sm.g[0] = beta;
    }
    int kcols = 0;
    const int jmax = arnoldi ? kp.arnoldi_steps : m;
    for (int j = 0; j < jmax; j++) {
      T* P = bufs[cur];
      T* Q = bufs[cur ^ 1];
      // ---- phase A: v_j = P/hn, w = A v_j, h1 = V^T w, ||w||^2
      {
        T acc[MAXM];
#pragma unroll
        for (int k = 0; k < MAXM; k++) acc[k] = T(0);
        T accA = T(0);
        const T inv = (T)(1.0 / hn);
        const T sc = (T)(s2 / hn);
        for (int i = lo + tid; i < hi; i += BS) {
          const T pc = ldcg(P + i);
          const T q = stencil<T, DIM>(P, i, n, kappa, pc) * sc;
          const T vj = pc * inv;
          V[(long long)j * ldv + i] = vj;
          Q[i] = q;
          accA += q * q;
#pragma unroll
          for (int k = 0; k < MAXM; k++) {
            if (k < j)
              acc[k] += V[(long long)k * ldv + i] * q;
            else if (k == j)
              acc[k] += vj * q;
          }
        }
#pragma unroll
        for (int k = 0; k < MAXM; k++)
          if (k <= j) warp_slot<LMAX>(sm.red, k, (double)acc[k]);
        warp_slot<LMAX>(sm.red, j + 1, (double)accA);  // slot j+1 carries ||w||^2
        block_finish<LMAX, BS>(j + 2, part(), lb, sm.red);
        ok = group_sync(w.bar, epoch, &sm.flag);
        if (!ok) goto abort;
        gather<BS>(part(), j + 2, nb, sm.tot);
        red++;
        if (tid <= j) sm.H[tid + j * LD] = sm.tot[tid];
        if (tid == 0) sm.anorm = sqrt(sm.tot[j + 1]);
      }
      // ---- phase B: w -= V h1, h2 = V^T w
      {
        T acc[MAXM];
#pragma unroll
        for (int k = 0; k < MAXM; k++) acc[k] = T(0);
        for (int i = lo + tid; i < hi; i += BS) {
          T q = Q[i];
          T col[MAXM];
#pragma unroll
          for (int k = 0; k < MAXM; k++) {
            if (k <= j) {
              col[k] = V[(long long)k * ldv + i];
              q -= (T)sm.tot[k] * col[k];
            }
          }
          Q[i] = q;
#pragma unroll
          for (int k = 0; k < MAXM; k++)
            if (k <= j) acc[k] += col[k] * q;
        }
#pragma unroll
        for (int k = 0; k < MAXM; k++)
          if (k <= j) warp_slot<LMAX>(sm.red, k, (double)acc[k]);
        block_finish<LMAX, BS>(j + 1, part(), lb, sm.red);
        ok = group_sync(w.bar, epoch, &sm.flag);
        if (!ok) goto abort;
        gather<BS>(part(), j + 1, nb, sm.tot);
        red++;
        if (tid <= j) sm.H[tid + j * LD] += sm.tot[tid];
      }
      // ---- phase C: w -= V h2, ||w||^2
      {
        T accN = T(0);
        for (int i = lo + tid; i < hi; i += BS) {
          T q = Q[i];
#pragma unroll
          for (int k = 0; k < MAXM; k++)
            if (k <= j) q -= (T)sm.tot[k] * V[(long long)k * ldv + i];
          Q[i] = q;
          accN += q * q;
        }
        warp_slot<LMAX>(sm.red, 0, (double)accN);
        block_finish<LMAX, BS>(1, part(), lb, sm.red);
        ok = group_sync(w.bar, epoch, &sm.flag);
        if (!ok) goto abort;
        gather<BS>(part(), 1, nb, sm.tot);
        red++;
      }
      // ---- Hessenberg column j, Givens rotation, convergence test
      hn = sqrt(sm.tot[0]);
      iters++;
      kcols = j + 1;
      if (tid == 0) {
        double* hc = sm.H + j * LD;
        hc[j + 1] = hn;
        int stop = 0;
        if (arnoldi) {
          if (lb == 0 && tk.hist)  // unrotated column j, leading dimension jmax+1
            for (int k = 0; k <= j + 1; k++) tk.hist[(long long)j * (jmax + 1) + k] = hc[k];
          if (!(hn > 1e-14 * sm.anorm)) stop = 1;
        } else {
          for (int i = 0; i < j; i++) {
            const double t = sm.cs[i] * hc[i] + sm.sn[i] * hc[i + 1];
            hc[i + 1] = -sm.sn[i] * hc[i] + sm.cs[i] * hc[i + 1];
            hc[i] = t;
          }
          const double rho = hypot(hc[j], hn);
          if (rho == 0.0) {
            sm.cs[j] = 1.0;
            sm.sn[j] = 0.0;
          } else {
            sm.cs[j] = hc[j] / rho;
            sm.sn[j] = hn / rho;
          }
          hc[j] = rho;
          hc[j + 1] = 0.0;
          sm.g[j + 1] = -sm.sn[j] * sm.g[j];
          sm.g[j] = sm.cs[j] * sm.g[j];
          const double res = fabs(sm.g[j + 1]);
          if (lb == 0 && tk.hist && iters <= tk.hist_cap) tk.hist[iters - 1] = res / bnorm;
          if (!isfinite(res) || !isfinite(hn)) stop = 2;
          else if (res <= kp.rtol * bnorm || !(hn > 1e-14 * sm.anorm) || iters >= kp.max_iters)
            stop = 1;
        }
        sm.ctl = stop;
      }
      __syncthreads();
      const int stop = sm.ctl;
      if (stop == 2) { status = kErrNonfinite; goto finish_x; }
      cur ^= 1;
      if (stop) break;
    }
    if (arnoldi) {
      // store the last basis vector too, so V_{k+1} is complete
      const T inv = (T)(1.0 / hn);
      const T* P = bufs[cur];
      for (int i = lo + tid; i < hi; i += BS) V[(long long)kcols * ldv + i] = ldcg(P + i) * inv;
      status = kcols;  // steps done
      break;
    }
    // ---- cycle end: y = H^{-1} g (upper triangular), x += V y
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      for (int i = kcols - 1; i >= 0; i--) {
        const double yi = sm.g[i] / sm.H[i + i * LD];
        for (int l = lane; l < i; l += 32) sm.g[l] -= sm.H[l + i * LD] * yi;
        if (lane == 0) sm.y[i] = yi;
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = lo + tid; i < hi; i += BS) {
      double d = 0.0;
      for (int k = 0; k < kcols; k++) d += sm.y[k] * (double)V[(long long)k * ldv + i];
      tk.x[i] += d;
    }
    cycles++;
    ok = group_sync(w.bar, epoch, &sm.flag);
    if (!ok) goto abort;
  }
  goto finish;

finish_x:
  // non-finite Hessenberg data: keep x as it is
  goto finish;

abort:
  status = *(volatile int*)w.bar.err;
  if (status == 0) status = kErrTimeout;

finish:
  if (leader) {
    DevResult r;
    r.iters = iters;
    r.cycles = cycles;
    r.status = status;
    r.used_alt = used_alt;
    r.pad = 0;
    r.bnorm = bnorm;
    r.relres_true = relres;
    r.relres_first_cycle = relres_first < 0.0 ? relres : relres_first;
    r.relres_guess = relres_guess;
    r.relres_alt = relres_alt;
    *tk.res = r;
  }
}

template <typename T, int DIM, int MAXM, int BS>
__global__ void __launch_bounds__(BS, 1) gmres_persistent(KParams kp) {
  __shared__ Smem<MAXM, BS> sm;
  int g = 0;
  while (g + 1 < kp.ngroups && (int)blockIdx.x >= kp.group_first[g + 1]) g++;
  const int lb = blockIdx.x - kp.group_first[g];
  const int nb = kp.group_first[g + 1] - kp.group_first[g];
  const GroupWork w = kp.work[g];
  unsigned long long epoch = 0;
  for (int t = kp.task_first[g]; t < kp.task_first[g + 1]; t++) {
    const SolveTask tk = kp.tasks[kp.task_order[t]];
    solve_one<T, DIM, MAXM, BS>(kp, tk, w, lb, nb, epoch, sm);
    if (*(volatile int*)w.bar.err != kErrNone) break;
    // all CTAs finish with this task's data before the next task starts
    if (!group_sync(w.bar, epoch, &sm.flag)) break;
  }
}

// ------------------------------------------------------------- host side --
template <typename T, int DIM, int MAXM, int BS>
static cudaError_t launch_t(const KParams& kp, int grid, cudaStream_t s) {
  void* args[] = {(void*)&kp};
  note_launches(1);
  return cudaLaunchCooperativeKernel((const void*)gmres_persistent<T, DIM, MAXM, BS>, dim3(grid),
                                     dim3(BS), args, 0, s);
}

template <typename T, int DIM, int MAXM, int BS>
static int max_blocks_t(int* bs) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gmres_persistent<T, DIM, MAXM, BS>, BS, 0);
  *bs = BS;
  return per * nsm;
}

// Variant table: 256-thread CTAs (the register budget of 255 per thread keeps the
// V column and the dot accumulators of a CGS2 sweep in registers).
#define MLG_DISPATCH(FN, ...)                                                              \
  if (fp32) {                                                                              \
    if (dim == 2) {                                                                        \
      if (m <= 32) return FN<float, 2, 32, 256>(__VA_ARGS__);                              \
      return FN<float, 2, 64, 256>(__VA_ARGS__);                                           \
    } else {                                                                               \
      if (m <= 32) return FN<float, 3, 32, 256>(__VA_ARGS__);                              \
      return FN<float, 3, 64, 256>(__VA_ARGS__);                                           \
    }                                                                                      \
  } else {                                                                                 \
    if (dim == 2) {                                                                        \
      if (m <= 32) return FN<double, 2, 32, 256>(__VA_ARGS__);                             \
      return FN<double, 2, 64, 256>(__VA_ARGS__);                                          \
    } else {                                                                               \
      if (m <= 32) return FN<double, 3, 32, 256>(__VA_ARGS__);                             \
      return FN<double, 3, 64, 256>(__VA_ARGS__);                                          \
    }                                                                                      \
  }

cudaError_t launch_gmres(const KParams& kp, bool fp32, int dim, int grid, cudaStream_t s) {
  const int m = kp.arnoldi_steps > 0 ? kp.arnoldi_steps : kp.m;
  MLG_DISPATCH(launch_t, kp, grid, s);
}

int gmres_max_blocks(bool fp32, int dim, int m, int* bs) { MLG_DISPATCH(max_blocks_t, bs); }

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
__global__ void basis_to_f64(const T* V, long long ldv, int rows, int N, double* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)rows * N) return;
  const int r = (int)(i / N), c = (int)(i % N);
  out[i] = (double)V[r * ldv + c];
}

cudaError_t launch_basis_to_f64(bool fp32, const void* V, long long ldv, int rows, int N,
                                double* out, cudaStream_t s) {
  const long long tot = (long long)rows * N;
  const int bs = 256;
  const unsigned gr = (unsigned)((tot + bs - 1) / bs);
  note_launches(1);
  if (fp32)
    basis_to_f64<float><<<gr, bs, 0, s>>>((const float*)V, ldv, rows, N, out);
  else
    basis_to_f64<double><<<gr, bs, 0, s>>>((const double*)V, ldv, rows, N, out);
  return cudaGetLastError();
}

}  // namespace mlg
