// Host/device structures of the persistent GMRES(m) solver.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace mlg {

constexpr int kMaxM = 64;          // largest supported restart length
// bucket limits of the compact (2 CTAs per SM) variants: m <= 47 (2D), m <= 55 (3D)
constexpr int kCompactM2 = 48;
constexpr int kCompactM3 = 56;
// restart lengths up to which the FP32 2D shared-slice variant runs its m <= 32
// instantiation (fewer buckets of j, less code)
constexpr int kSmallM = 32;
// Where a launch keeps the basis V (one kernel variant each):
constexpr int kVDirect = 0;  // HBM, loaded into registers by the passes
constexpr int kVShared = 1;  // each CTA's slice in shared memory (2D)
constexpr int kVBulk = 2;    // HBM, streamed through per-warp bulk-copy stages
constexpr int kPartStride = 1024;  // max CTAs per group (partials row length)
// doubles in a group's partial-sum area (two alternating sets)
constexpr long long part_doubles(int pstride) { return 2LL * (kMaxM + 2) * pstride; }
// Rows a tile of the basis occupies for `rows` vectors: V stores basis vectors
// in pairs, so the count is rounded up to even (see gmres_kernel.cuh).
__host__ __device__ constexpr int vrows_p(int rows) { return (rows + 1) & ~1; }

// Per-system result written by the solver (mirrors mlgmres_result's numeric part).
struct DevResult {
  long long iters;
  int cycles;
  int status;      // 0 OK, 1 NOT_CONVERGED, kErrTimeout, kErrNonfinite
  int used_alt;    // 1 if the alternative (learned) guess replaced x
  int pad;
  double bnorm;
  double relres_true;
  double relres_first_cycle;
  double relres_guess;
  double relres_alt;  // residual of the alternative guess, -1 if none
};

// One linear system A x = b.
struct SolveTask {
  int n;                 // interior points per axis
  int N;                 // n^dim
  const double* b;       // rhs (or the start vector in Arnoldi mode)
  double* x;             // guess in, solution out
  const double* x_alt;   // optional competing guess (learned), may be null
  const float* kappa;    // 3D cell coefficients, may be null
  // FP32 face coefficients of the 3D operator (or null: formed from kappa per
  // point): four arrays fx, fy, fz, fb at faces + a * fstride, each padded
  // with zeros far enough past both ends that no stencil window is clipped;
  // set only with a work vector W0 padded the same way (single 3D solves)
  const float* faces = nullptr;
  long long fstride = 0;
  DevResult* res;
  double* hist;          // optional |g_{j+1}|/||b|| per step (Arnoldi mode: H)
  long long hist_cap;
  int zero_x;            // 1: the solve starts from x = 0 (written by the kernel)
};

// Workspace of one CTA group.
struct GroupWork {
  void* V;            // basis, tile-major (m+1 vectors per 32-point tile), ldv points
  long long ldv;
  void* W0;           // two work vectors (ping-pong), ldv each
  void* W1;
  double* part;       // 2 x (kMaxM+2) x pstride partial sums
  int pstride;        // row length of part (>= the group's CTA count)
  double* Rg;         // compact variants: (m+1) x m FP64 triangle per CTA, indexed
                      // by blockIdx.x (the others keep R in shared memory)
  GroupBarrier bar;
};

// Doubles of the per-CTA triangle R of the compact variants.
constexpr long long kRgDoubles = (long long)(kCompactM3 + 1) * kCompactM3;

struct KParams {
  int m;
  double rtol;
  long long max_iters;
  int arnoldi_steps;        // > 0: run that many Arnoldi steps only (inspection mode)
  int vsmem;                // bytes of shared memory for a CTA's slice of V (0 = V in HBM)
  int bulk_stages;          // most bulk-copy stages per warp when V is in HBM (0 = off)
  int bulk_cap;             // bytes of staging area per warp (>= m 32-point rows)
  int vmode;                // kVDirect | kVShared | kVBulk (the kernel variant launched)
  int compact;              // 1: the two-CTAs-per-SM bulk variant (FP32, m below its limit)
  int ngroups;
  const int* group_first;   // ngroups+1 CTA ranges
  const int* task_first;    // ngroups+1 ranges into task_order
  const int* task_order;    // task indices, grouped
  const SolveTask* tasks;
  const GroupWork* work;    // ngroups
};

// Launch the persistent cooperative solver.  `fp32` selects the FP32 inner
// precision; dim is 2 or 3.  Returns the CUDA error of the launch.
cudaError_t launch_gmres(const KParams& kp, bool fp32, int dim, int grid_blocks, cudaStream_t s);

// Largest co-resident grid for the chosen kernel variant (blocks), and its CTA size.
int gmres_max_blocks(bool fp32, int dim, int m, int* block_threads);

// Shared-memory bytes a CTA may use for its slice of V (so that slice + the
// solver's own state fit the per-CTA limit); 0 if none.
int gmres_vsmem_budget(bool fp32);

// Most bulk-copy stages per warp (kMaxStages) for a basis in HBM.  A pass uses
// as many as fit in a warp's staging area for its rows.
int gmres_bulk_stages(bool fp32, int m);

// Bytes of staging area per warp for at most P stages of m rows each: the
// warp's share of the shared memory left next to the solver's state, capped
// at P m rows; 0 if not even one stage of m rows fits.
int gmres_bulk_cap(bool fp32, int m, int P);

// The compact variants (FP32 bulk-copy, two CTAs per SM; m < kCompactM2 in
// 2D, m < kCompactM3 in 3D): whether one applies, its co-resident CTA count,
// and its staging bytes per warp for at most P stages (0 if none fits).
bool gmres_compact_ok(bool fp32, int dim, int m);
int gmres_compact_max_blocks(int dim, int m);
int gmres_compact_cap(int dim, int m, int P);
// Shared-memory bytes a compact 2D CTA may use for its slice of V.
int gmres_compact_vsmem_budget();

// FP64 operator application out = A u (2D or 3D) on one grid.
// The FP32 face coefficients of the 3D variable-coefficient operator (see
// SolveTask::faces): fx/fy/fz(i) = harmonic mean of kappa_i and its +x/+y/+z
// neighbour (0 on the domain's upper walls), fb(i) = kappa_i times the number
// of the point's wall faces.
cudaError_t launch_kappa_faces(int n, const float* kappa, float* faces, long long fstride,
                               cudaStream_t s);
cudaError_t launch_apply(int dim, int n, const float* kappa, const double* u, double* out,
                         cudaStream_t s);

// Convert the first `rows` vectors of a tile-major basis holding `vrows`
// vectors per tile (element type fp32 ? float : double) to row-major doubles.
cudaError_t launch_basis_to_f64(bool fp32, const void* V, int vrows, int rows, int N,
                                double* out, cudaStream_t s);

}  // namespace mlg
