/*
 * FP64 CPU oracle for restarted GMRES(m) on the discrete Poisson operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg load this file's library.  It shares no code,
 * header or constant with the CUDA path; it is deliberately plain: one pass per
 * vector operation, modified Gram-Schmidt, textbook Givens rotations, no
 * blocking or fusion.
 *
 * Operator (the discrete Laplacian with zero-Dirichlet walls, Sec. 1.4 and the
 * benchmark description of Sec. 3), sign chosen so that A is SPD:
 *   2D:  (A u)_{ij} = (4 u_ij - u_{i-1,j} - u_{i+1,j} - u_{i,j-1} - u_{i,j+1}) / h^2
 *   3D:  (A u)_c    = sum over the 6 faces f of kappa_f (u_c - u_nb) / h^2,
 *        kappa_f = 2 k_c k_nb / (k_c + k_nb) inside, kappa_f = k_c on a wall face
 *        (where u_nb = 0).
 *   h = 2/(n+1) on [-1,1]; missing neighbours are 0.
 *
 * GMRES(k) (Sec. 1.2: restarted GMRES starts each cycle from the last iterate):
 *   r = b - A x, beta = ||r||, v0 = r/beta, g = beta e1
 *   for j = 0..m-1: w = A v_j; MGS against v_0..v_j; h_{j+1,j} = ||w||;
 *     rotate column j by the stored rotations, form rotation j, update g;
 *     stop the cycle when |g_{j+1}| <= rtol ||b|| or on breakdown;
 *     v_{j+1} = w / h_{j+1,j}
 *   solve H y = g (upper triangular), x += V y, recompute the true residual.
 * The tolerance is relative to ||b||, so a good initial guess is not penalised.
 * E_k (Sec. 2.2, the residual at the end of the first restart cycle) is the
 * true relative residual after cycle 1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  long iters;
  int cycles;
  int status; /* 0 = converged, 1 = iteration cap reached, -1 = bad argument, -3 = no memory */
  double bnorm;
  double relres_true;        /* ||b - A x|| / ||b|| at exit */
  double relres_first_cycle; /* E_k: true relative residual after the first cycle */
  double relres_guess;       /* ||b - A x0|| / ||b|| */
} oracle_stats;

static int g_threads = 1;

static double dot(long N, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) num_threads(g_threads) if (g_threads > 1)
  for (long i = 0; i < N; i++) s += a[i] * b[i];
  return s;
}

static void axpy(long N, double alpha, const double* x, double* y) {
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1)
  for (long i = 0; i < N; i++) y[i] += alpha * x[i];
}

static void scale_into(long N, double alpha, const double* x, double* y) {
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1)
  for (long i = 0; i < N; i++) y[i] = alpha * x[i];
}

void oracle_apply_2d(int n, const double* u, double* out) {
  const double h = 2.0 / (n + 1);
  const double s = 1.0 / (h * h);
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1)
  for (int iy = 0; iy < n; iy++) {
    for (int ix = 0; ix < n; ix++) {
      const long c = (long)iy * n + ix;
      double left = ix > 0 ? u[c - 1] : 0.0;
      double right = ix < n - 1 ? u[c + 1] : 0.0;
      double down = iy > 0 ? u[c - n] : 0.0;
      double up = iy < n - 1 ? u[c + n] : 0.0;
      out[c] = s * (4.0 * u[c] - left - right - down - up);
    }
  }
}

static double face_coef(double kc, double knb) { return 2.0 * kc * knb / (kc + knb); }

void oracle_apply_3d(int n, const double* kappa, const double* u, double* out) {
  const double h = 2.0 / (n + 1);
  const double s = 1.0 / (h * h);
  const long nn = (long)n * n;
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1)
  for (int iz = 0; iz < n; iz++) {
    for (int iy = 0; iy < n; iy++) {
      for (int ix = 0; ix < n; ix++) {
        const long c = (long)iz * nn + (long)iy * n + ix;
        const double kc = kappa ? kappa[c] : 1.0;
        const double uc = u[c];
        double acc = 0.0;
        /* each of the 6 faces: (neighbour exists?, neighbour index) */
        const int has[6] = {ix > 0, ix < n - 1, iy > 0, iy < n - 1, iz > 0, iz < n - 1};
        const long off[6] = {-1, 1, -(long)n, (long)n, -nn, nn};
        for (int f = 0; f < 6; f++) {
          if (has[f]) {
            const long nb = c + off[f];
            const double knb = kappa ? kappa[nb] : 1.0;
            acc += face_coef(kc, knb) * (uc - u[nb]);
          } else {
            acc += kc * uc; /* wall face: u_nb = 0, kappa_f = kappa_c */
          }
        }
        out[c] = s * acc;
      }
    }
  }
}

static void apply_op(int dim, int n, const double* kappa, const double* u, double* out) {
  if (dim == 2)
    oracle_apply_2d(n, u, out);
  else
    oracle_apply_3d(n, kappa, u, out);
}

static long grid_size(int dim, int n) { return dim == 2 ? (long)n * n : (long)n * n * n; }

/* One MGS Arnoldi step: w = A v_j orthogonalised against v_0..v_j.
 * H is column-major with leading dimension m+1 (entry (i,j) at H[i + j*(m+1)]);
 * column j receives h_{0..j,j} and h_{j+1,j} = ||w||.  Returns ||A v_j||. */
static double mgs_step(int dim, int n, const double* kappa, long N, int m, int j, double* V,
                       double* H, double* w) {
  apply_op(dim, n, kappa, V + (long)j * N, w);
  const double anorm = sqrt(dot(N, w, w));
  for (int i = 0; i <= j; i++) {
    const double hij = dot(N, w, V + (long)i * N);
    H[i + (long)j * (m + 1)] = hij;
    axpy(N, -hij, V + (long)i * N, w);
  }
  H[j + 1 + (long)j * (m + 1)] = sqrt(dot(N, w, w));
  return anorm;
}

/* Arnoldi relation check helper: runs up to m MGS steps from v0 (normalised
 * here) and returns V ((m+1) x N, row per vector) and H ((m+1) x m, column-major
 * with leading dimension m+1).  Returns the number of completed steps. */
int oracle_arnoldi(int dim, int n, const double* kappa, const double* v0, int m, double* V,
                   double* H, int nthreads) {
  g_threads = nthreads > 0 ? nthreads : 1;
  const long N = grid_size(dim, n);
  double* w = (double*)malloc(sizeof(double) * N);
  if (!w) return -3;
  memset(H, 0, sizeof(double) * (size_t)(m + 1) * m);
  const double beta = sqrt(dot(N, v0, v0));
  scale_into(N, 1.0 / beta, v0, V);
  int done = 0;
  for (int j = 0; j < m; j++) {
    const double anorm = mgs_step(dim, n, kappa, N, m, j, V, H, w);
    done = j + 1;
    const double hn = H[j + 1 + (long)j * (m + 1)];
    if (hn <= 1e-14 * anorm) break;
    scale_into(N, 1.0 / hn, w, V + (long)(j + 1) * N);
  }
  free(w);
  return done;
}

int oracle_gmres(int dim, int n, const double* kappa, const double* b, double* x, int m,
                 double rtol, long max_iters, int nthreads, oracle_stats* st, double* hist,
                 long hist_cap) {
  memset(st, 0, sizeof(*st));
  if ((dim != 2 && dim != 3) || n < 1 || m < 1 || !(rtol > 0.0) || max_iters < 0) {
    st->status = -1;
    return -1;
  }
  g_threads = nthreads > 0 ? nthreads : 1;
  const long N = grid_size(dim, n);
  double* V = (double*)malloc(sizeof(double) * (size_t)(m + 1) * N);
  double* w = (double*)malloc(sizeof(double) * N);
  double* r = (double*)malloc(sizeof(double) * N);
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double* cs = (double*)calloc(m + 1, sizeof(double));
  double* sn = (double*)calloc(m + 1, sizeof(double));
  double* g = (double*)calloc(m + 1, sizeof(double));
  double* y = (double*)calloc(m + 1, sizeof(double));
  if (!V || !w || !r || !H || !cs || !sn || !g || !y) {
    free(V); free(w); free(r); free(H); free(cs); free(sn); free(g); free(y);
    st->status = -3;
    return -3;
  }
  const double bnorm = sqrt(dot(N, b, b));
  st->bnorm = bnorm;
  if (bnorm == 0.0) { /* A x = 0 has the unique solution x = 0 */
    memset(x, 0, sizeof(double) * N);
    st->status = 0;
    goto done;
  }
  for (;;) {
    /* true residual r = b - A x */
    apply_op(dim, n, kappa, x, r);
    for (long i = 0; i < N; i++) r[i] = b[i] - r[i];
    const double beta = sqrt(dot(N, r, r));
    const double relres = beta / bnorm;
    st->relres_true = relres;
    if (st->cycles == 0) st->relres_guess = relres;
    if (st->cycles == 1) st->relres_first_cycle = relres;
    if (relres <= rtol) { st->status = 0; break; }
    if (st->iters >= max_iters) { st->status = 1; break; }

    scale_into(N, 1.0 / beta, r, V);
    memset(g, 0, sizeof(double) * (m + 1));
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m; j++) {
      const double anorm = mgs_step(dim, n, kappa, N, m, j, V, H, w);
      double* hc = H + (long)j * (m + 1);
      const double hnext = hc[j + 1];
      for (int i = 0; i < j; i++) { /* previous rotations */
        const double t = cs[i] * hc[i] + sn[i] * hc[i + 1];
        hc[i + 1] = -sn[i] * hc[i] + cs[i] * hc[i + 1];
        hc[i] = t;
      }
      const double rho = hypot(hc[j], hc[j + 1]);
      if (rho == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
      else { cs[j] = hc[j] / rho; sn[j] = hc[j + 1] / rho; }
      hc[j] = rho;
      hc[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      st->iters++;
      k = j + 1;
      if (hist && st->iters <= hist_cap) hist[st->iters - 1] = fabs(g[j + 1]) / bnorm;
      if (fabs(g[j + 1]) <= rtol * bnorm || hnext <= 1e-14 * anorm || st->iters >= max_iters)
        break;
      scale_into(N, 1.0 / hnext, w, V + (long)(j + 1) * N);
    }
    /* back substitution H(0:k,0:k) y = g(0:k) */
    for (int i = k - 1; i >= 0; i--) {
      double s = g[i];
      for (int l = i + 1; l < k; l++) s -= H[i + (long)l * (m + 1)] * y[l];
      y[i] = s / H[i + (long)i * (m + 1)];
    }
    for (int i = 0; i < k; i++) axpy(N, y[i], V + (long)i * N, x);
    st->cycles++;
  }
  if (st->cycles == 0) st->relres_first_cycle = st->relres_true;
done:
  free(V); free(w); free(r); free(H); free(cs); free(sn); free(g); free(y);
  return st->status;
}
