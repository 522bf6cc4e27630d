// Persistent restarted GMRES(m) for the discrete Poisson operator (Sec. 1.2,
// Sec. 1.4, Sec. 3 of arXiv 2103.10975), one cooperative launch per solve or
// per batch of solves.
//
// Each CTA group (all CTAs for a single solve, or one CTA per system of a
// batch) owns one system at a time; its grid points are split into contiguous
// per-CTA ranges of whole 32-point tiles.  One Arnoldi step is classical
// Gram-Schmidt applied twice, arranged as two fused passes over the CTA's
// points with one group barrier each (see solve_one):
//   X: v_j (lazy normalisation of the previous step's vector), z = A v_j
//      obtained from the SpMV of the unnormalised vector through the Arnoldi
//      relation, and the dots h1 = V^T z;
//   Y: w' = z - V h1 with the dots h2 = V^T w' in the same pass.
// After each barrier every CTA sums the per-CTA partials in the same fixed
// order, so all CTAs hold bit-identical coefficients and run the scalar
// recurrences (Pythagorean norm, Hessenberg column, Givens rotation) redundantly
// in shared memory with no extra synchronisation.  At a cycle end the
// back-substitution y = R^{-1} g runs in shared memory, x += V y is accumulated
// in FP64 and the true residual b - A x is recomputed in FP64 (the restart of
// GMRES(k)).  The FP32 variant stores V and the work vectors in FP32 and so
// runs every cycle as one step of mixed-precision iterative refinement.
#pragma once
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
// The FP32 inner operator takes the fast reciprocal-based division (about 2 ulp,
// two instructions) instead of the IEEE division sequence: six per point in 3D
// were a third of the X pass's instructions.  Its rounding is of the order of
// the FP32 arithmetic around it; the FP64 restart residual keeps the exact face.
template <>
__device__ __forceinline__ float face<float>(float kc, float knb) {
  return __fdividef(2.f * kc * knb, kc + knb);
}

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

// Two values side by side: two basis vectors at one point, or the coefficients
// of two basis vectors (one load each).
template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

// ------------------------------------------------------------ basis layout --
// V is stored tile-major in pairs of basis vectors: for every tile of 32
// consecutive grid points, the values of vectors 2q and 2q+1 at a point sit
// side by side (one 8-byte FP32 or 16-byte FP64 word), and the pair rows
// q = 0, 1, ... of the tile follow each other.  A warp's column block of V (all
// k for its 32 points) is one contiguous run of vrows_p(rows) * 32 elements,
// and one vector load gives a point two basis values, which the passes consume
// with one paired FMA (half the load and FMA instructions of one value each).
__host__ __device__ __forceinline__ long long vbase(int i, int rows) {
  return ((long long)(i >> 5) * vrows_p(rows) << 5) + ((i & 31) << 1);
}
// offset of basis vector k from a point's vbase
__host__ __device__ __forceinline__ int vko(int k) { return ((k >> 1) << 6) + (k & 1); }
__host__ __device__ __forceinline__ long long vix(int k, int i, int rows) {
  return vbase(i, rows) + vko(k);
}

// Paired FMA: (a.x b.x + c.x, a.y b.y + c.y); one instruction for FP32.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  return __ffma2_rn(a, b, c);
}
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
template <typename T2>
__device__ __forceinline__ T2 dup2(decltype(T2::x) v) {
  T2 r;
  r.x = v;
  r.y = v;
  return r;
}

// Stores v_j in a column: with the zero slot of v_{j+1} when j is even.
template <typename T>
__device__ __forceinline__ void store_vj(T* vc, int j, T vj) {
  if (j & 1) {
    vc[vko(j)] = vj;
  } else {
    typename Vec2<T>::type p;
    p.x = vj;
    p.y = T(0);
    *reinterpret_cast<typename Vec2<T>::type*>(vc + vko(j)) = p;
  }
}

// ----------------------------------------------------------- shared state --
constexpr int kMaxStages = 16;  // bulk-copy stages per warp (upper bound)

// Where the Givens triangle R ((MAXM + 1) x MAXM FP64) lives: in the shared
// state, or, for the compact variants (two CTAs per SM, instantiated with the
// bucket limits kCompactM2 / kCompactM3), in a global buffer with one region per
// CTA of the launch, which leaves their warps room for a second bulk-copy stage
// (R is written by the Givens warp once per step and read once per cycle).
template <int MAXM>
__host__ __device__ constexpr bool compact_bucket() {
  return MAXM == kCompactM2 || MAXM == kCompactM3;
}
template <int MAXM>
__host__ __device__ constexpr bool r_in_shared() { return !compact_bucket<MAXM>(); }
template <int MAXM>
__host__ __device__ constexpr size_t r_doubles() { return (size_t)(MAXM + 1) * MAXM; }

template <typename T, int MAXM, int BS>
struct Smem {
  T red[BS / 32][MAXM + 2];      // per-warp partials in the working precision
  double redd[BS / 32][4];       // per-warp partials of the FP64 residual norms
  double tot[MAXM + 2];
  double hcol[MAXM + 2];         // the column being rotated, in FP64 (Givens warp)
  // the same columns after the Givens rotations, each above the diagonal divided
  // by its diagonal entry; the compact variants keep them in global memory (Rg)
  double R[r_in_shared<MAXM>() ? (MAXM + 1) * MAXM : 1];
  double cs[MAXM], sn[MAXM], g[MAXM + 1], y[MAXM];
  float2 yf[MAXM];               // y_k as hi + lo floats (FP32 variants' V y)
  double rinv[MAXM];             // 1 / R(c,c), formed with rotation c (the back-
                                 // substitution then multiplies: no FP64 division)
  T HuT[(MAXM + 1) * MAXM];      // Hessenberg as built (Arnoldi relation), ld MAXM+1
  alignas(16) T coef[MAXM + 2];  // gather output in the working precision
  // per basis vector k: h2v[k] = h2_k, the pending second-pass coefficient of
  // w', and cv[k] = c_k, the coefficient turning A w' into A v_j; the passes
  // read them in pairs (k = 2q, 2q+1), as they read V
  alignas(16) T h2v[MAXM + 2];
  alignas(16) T cv[MAXM + 2];
  // the latest column's two projections, from which the Givens warp forms
  // the FP64 column (FP64 work kept off the step's critical path)
  T h1c[MAXM + 2], h2h[MAXM + 2];
  T anorm2T;                     // ||z||^2 of the latest column
  T invT;                        // 1 / hn in the working precision
  T hn2T;                        // ||w'||^2 - ||h2||^2 in the working precision
  int ctl, stop, flag, fallback;
  // bulk-copy stage barriers, one set per warp; kept here rather than after
  // the staging buffers because a CTA's slice of V may occupy that space for
  // other systems of the same launch
  unsigned long long bbar[BS / 32][kMaxStages];
  double* Rg;  // this CTA's R in global memory (the variants that keep it there)
};

// Shared state rounded up to 128 bytes (the staging buffers that follow it are
// bulk-copy destinations).
template <typename T, int MAXM, int BS>
__host__ __device__ constexpr size_t smem_own_bytes() {
  return (sizeof(Smem<T, MAXM, BS>) + 127) / 128 * 128;
}

// Warp partial of slot k (lane 0 stores it); block_finish then adds the warp
// partials of slots 0..L-1 and writes the CTA's sums to part[k*kPartStride + lb].
// All of it runs in the element type R (FP32 for the FP32 variant: the FP64
// pipe of this GPU is ~1/64 of FP32 and would otherwise dominate).
template <int LW, typename R, typename V>
__device__ __forceinline__ void warp_slot(R (*red)[LW], int k, V v) {
  R x = (R)v;
  x = warp_sum(x);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = x;
}

// Sums acc[k] over the warp for all k < MAXM at once (butterfly transpose
// reduction: 31 shuffles per 32 slots instead of 5 per slot); lane l ends with
// the warp total of slot l (+32 for the second half when MAXM = 64), which it
// stores to red[warp][slot] for slot < L.
template <int LMAX, int MAXM, typename T>
__device__ __forceinline__ void warp_slots(T (*red)[LMAX], T (&acc)[MAXM], int L) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < MAXM / 32; g++) {
    T v[32];
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = acc[g * 32 + i];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const bool up = (lane & off) != 0;
#pragma unroll
      for (int i = 0; i < off; i++) {
        const T send = up ? v[i] : v[i + off];
        const T keep = up ? v[i + off] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
    const int slot = g * 32 + lane;
    if (slot < L) red[warp][slot] = v[0];
  }
}

// warp_slots for an accumulator array of K <= MAXM entries (padded to 32).
template <int LMAX, int K, typename T>
__device__ __forceinline__ void warp_slots_k(T (*red)[LMAX], const T (&acc)[K], int L) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < (K + 31) / 32; g++) {
    T v[32];
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = (g * 32 + i < K) ? acc[g * 32 + i] : T(0);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const bool up = (lane & off) != 0;
#pragma unroll
      for (int i = 0; i < off; i++) {
        const T send = up ? v[i] : v[i + off];
        const T keep = up ? v[i + off] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
    const int slot = g * 32 + lane;
    if (slot < L) red[warp][slot] = v[0];
  }
}

template <int LW, int BS, typename R>
__device__ __forceinline__ void block_finish(int L, R* part, int lb, R (*red)[LW], int ps) {
  __syncthreads();
  for (int k = threadIdx.x; k < L; k += BS) {
    R s = R(0);
#pragma unroll
    for (int w = 0; w < BS / 32; w++) s += red[w][k];
    part[(long long)k * ps + lb] = s;
  }
}

// block_finish and the group barrier in one: after one CTA barrier, warp 0
// adds the warp partials, stores the CTA's sums, and (its lanes' stores ordered
// by __syncwarp before lane 0's release) arrives and waits at the group
// barrier, while warp 1 runs `side`; a second CTA barrier ends it.  Saves the
// CTA barrier that separates the two when they are done one after the other.
template <int LW, int BS, typename R, typename Side>
__device__ __forceinline__ bool finish_and_sync(int L, R* part, int lb, R (*red)[LW], int ps,
                                                const GroupBarrier& gb, unsigned long long& epoch,
                                                int* s_flag, Side side) {
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    for (int k = lane; k < L; k += 32) {
      R s = R(0);
#pragma unroll
      for (int w = 0; w < BS / 32; w++) s += red[w][k];
      part[(long long)k * ps + lb] = s;
    }
    __syncwarp();
    if (lane == 0)
      *s_flag = gb.nblocks == 1 ? (*(volatile int*)gb.err == kErrNone)
                                : group_arrive_wait(gb, epoch);
  } else if (warp == 1) {
    side();
  }
  __syncthreads();
  return *s_flag != 0;
}

// finish_and_sync for an exchange whose `side` work may outlast the group
// barrier: warp 1 runs `side` and skips the barrier that releases the other
// warps once thread 0 has passed the group barrier (a named barrier over the
// other BS - 32 threads), so that `side` also overlaps the gather that follows
// (gather with SKIP1, whose closing CTA barrier warp 1 joins when `side` is
// done).  *s_flag is valid for every thread after that gather.
template <int LW, int BS, typename R, typename Side>
__device__ __forceinline__ void finish_and_sync_side(int L, R* part, int lb, R (*red)[LW], int ps,
                                                     const GroupBarrier& gb,
                                                     unsigned long long& epoch, int* s_flag,
                                                     Side side) {
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 1) {
    side();
    return;
  }
  if (warp == 0) {
    for (int k = lane; k < L; k += 32) {
      R s = R(0);
#pragma unroll
      for (int w = 0; w < BS / 32; w++) s += red[w][k];
      part[(long long)k * ps + lb] = s;
    }
    __syncwarp();
    if (lane == 0)
      *s_flag = gb.nblocks == 1 ? (*(volatile int*)gb.err == kErrNone)
                                : group_arrive_wait(gb, epoch);
  }
  asm volatile("bar.sync 1, %0;" ::"r"(BS - 32) : "memory");
}

// Sum of the group's partials for k < L, identical in every CTA (same order);
// tot gets the sums in FP64, coef the same values in the working precision.
// Each warp takes up to four slots at a time, four partials per lane each, so
// that sixteen loads per lane are in flight together.  SKIP1: warp 1 takes no
// slots (it is still on finish_and_sync_side's `side` work).
template <int BS, typename R, typename T, bool SKIP1 = false>
__device__ __forceinline__ void gather(const R* part, int L, int nb, double* tot, T* coef,
                                       int ps) {
  constexpr int NW = BS / 32 - (SKIP1 ? 1 : 0);
  // slots per warp and round: 4, or 5 without warp 1, so that one round covers
  // 32 slots either way (a second round is a second L2 round trip)
  constexpr int Q = SKIP1 ? 5 : 4;
  const int lane = threadIdx.x & 31, warp0 = threadIdx.x >> 5;
  // (warp 1 under SKIP1 starts past every slot)
  const int warp = SKIP1 ? (warp0 == 1 ? (1 << 20) : (warp0 == 0 ? 0 : warp0 - 1)) : warp0;
  for (int k0 = warp; k0 < L; k0 += Q * NW) {
    R s[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) s[q] = R(0);
    // 128 partials per round, all loads of a lane issued before any is used
    for (int g0 = 0; g0 < nb; g0 += 128) {
      R v[Q][4];
#pragma unroll
      for (int q = 0; q < Q; q++) {
        const int k = k0 + q * NW;
#pragma unroll
        for (int r = 0; r < 4; r++) {
          const int g = g0 + r * 32 + lane;
          v[q][r] = (k < L && g < nb) ? ldcg(part + (long long)k * ps + g) : R(0);
        }
      }
#pragma unroll
      for (int q = 0; q < Q; q++) s[q] += (v[q][0] + v[q][1]) + (v[q][2] + v[q][3]);
    }
#pragma unroll
    for (int q = 0; q < Q; q++) s[q] = warp_sum(s[q]);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < Q; q++) {
        const int k = k0 + q * NW;
        if (k < L) {
          // FP32 partials: coef only (an FP64 conversion is a long-latency
          // operation on this GPU; consumers convert where they need FP64)
          if constexpr (sizeof(R) == 8) tot[k] = (double)s[q];
          coef[k] = (T)s[q];
        }
      }
    }
  }
  __syncthreads();
}

// Double-float accumulation (error-free transformations, Dekker 1971 and
// Knuth's TwoSum): (s, c) += (y.x + y.y) v with the head s and tail c floats.
// The _rn intrinsics keep the compiler from contracting the steps into FMAs.
__device__ __forceinline__ void df_fma(float& s, float& c, float2 y, float v) {
  const float p = __fmul_rn(y.x, v);
  float e = __fmaf_rn(y.x, v, -p);  // y.x v - p, exactly
  e = __fmaf_rn(y.y, v, e);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));  // s + p - t
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}
// The value of two (head, tail) pairs in FP64: the heads joined by TwoSum in
// FP32, so that only two conversions and one FP64 addition remain.
__device__ __forceinline__ double df_value(float s0, float c0, float s1, float c1) {
  const float t = __fadd_rn(s0, s1);
  const float z = __fsub_rn(t, s0);
  const float err = __fadd_rn(__fsub_rn(s0, __fsub_rn(t, z)), __fsub_rn(s1, z));
  const float c = __fadd_rn(__fadd_rn(c0, c1), err);
  return (double)t + (double)c;
}

// Givens update of Hessenberg column c (Hu -> R): apply rotations 0..c-1, form
// rotation c, update g, and return the stop code (0 go on, 1 end the cycle,
// 2 non-finite).  One warp.  Applying rotation i to the running entry ri_i and
// the untouched h_{i+1} gives R(i,c) = cs_i ri_i + sn_i h_{i+1} and
// ri_{i+1} = -sn_i ri_i + cs_i h_{i+1}: an affine recurrence in ri, so the maps
// x -> a_i x + b_i are composed by an inclusive warp scan (composition is
// associative), 32 rotations per round.  The dependent FP64 chain is five scan
// steps per round instead of one FMA per rotation (an FP64 operation has a
// latency of about 70 cycles on this GPU).
template <typename T, int MAXM, int BS>
__device__ int givens_column(Smem<T, MAXM, BS>& sm, int c, double rtol_bnorm, long long it,
                             long long max_iters, int m, double* hist, long long hist_cap,
                             double bnorm) {
  constexpr int LD = MAXM + 1;
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  double* hc = sm.hcol;
  double* rc = (r_in_shared<MAXM>() ? sm.R : sm.Rg) + c * LD;
  // column c in FP64: h1 + h2 (exact sum of two FP32 values) and hn below
  for (int i = lane; i <= c + 1; i += 32)
    hc[i] = i <= c ? (double)sm.h1c[i] + (double)sm.h2h[i] : (double)sm.HuT[c + 1 + c * LD];
  __syncwarp();
  const double h0 = hc[0];
  double ca = 1.0, cb = 0.0;  // composition of the maps of the earlier rounds
  double ri = h0;             // ri_base entering a round, ri_c after the last
  for (int base = 0; base < c; base += 32) {
    const int i = base + lane;
    const bool in = i < c;
    const double csi = in ? sm.cs[i] : 0.0, sni = in ? sm.sn[i] : 0.0;
    const double hi = in ? hc[i + 1] : 0.0;
    double a = in ? -sni : 1.0;  // identity past the last rotation
    double b = csi * hi;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const double pa = __shfl_up_sync(kAll, a, off);
      const double pb = __shfl_up_sync(kAll, b, off);
      if (lane >= off) {  // this lane's map after the earlier lane's
        b = fma(a, pb, b);
        a *= pa;
      }
    }
    const double fa = a * ca, fb = fma(a, cb, b);  // after the earlier rounds
    const double next = fma(fa, h0, fb);           // ri_{i+1}
    double prev = __shfl_up_sync(kAll, next, 1);   // ri_i
    if (lane == 0) prev = ri;
    if (in) rc[i] = fma(csi, prev, sni * hi);
    ca = __shfl_sync(kAll, fa, 31);
    cb = __shfl_sync(kAll, fb, 31);
    ri = __shfl_sync(kAll, next, min(c - 1 - base, 31));
  }
  __syncwarp();
  int stop = 0;
  if (lane == 0) {
    const double hsub = hc[c + 1];
    const double r2 = fma(ri, ri, hsub * hsub);
    double rho;
    if (r2 > 1e-300 && r2 < 1e300) {
      // one reciprocal square root instead of a square root and a division
      // (each a long dependent chain on this GPU's FP64 pipe)
      const double inv = rsqrt(r2);
      sm.cs[c] = ri * inv;
      sm.sn[c] = hsub * inv;
      rho = r2 * inv;
      sm.rinv[c] = inv;  // 1 / rho
    } else {
      rho = sqrt(r2);
      sm.cs[c] = rho == 0.0 ? 1.0 : ri / rho;
      sm.sn[c] = rho == 0.0 ? 0.0 : hsub / rho;
      // a zero column (the Krylov space is exhausted) contributes y_c = 0,
      // the least-squares solution of smallest norm
      sm.rinv[c] = rho == 0.0 ? 0.0 : 1.0 / rho;
    }
    rc[c] = rho;
    rc[c + 1] = 0.0;
    const double gc = sm.g[c];
    sm.g[c + 1] = -sm.sn[c] * gc;
    sm.g[c] = sm.cs[c] * gc;
    const double res = fabs(sm.g[c + 1]);
    if (hist && it <= hist_cap) hist[it - 1] = res / bnorm;
    if (!isfinite(res) || !isfinite(hsub))
      stop = 2;
    else if (res <= rtol_bnorm || !(hsub * hsub > 1e-28 * (double)sm.anorm2T) || it >= max_iters ||
             c + 1 >= m)
      stop = 1;
    sm.stop = stop;
  }
  __syncwarp();
  // R(i,c) / R(c,c) for i < c: the form the back-substitution uses
  const double ic = sm.rinv[c];
  for (int i = lane; i < c; i += 32) rc[i] *= ic;
  __syncwarp();
  return stop;
}

// ------------------------------------------------- bulk-copy staging of V --
// When V lives in HBM, every warp streams its 32-point tiles' column blocks
// (rows 0..r-1 of a tile are one contiguous run in the tile-major layout) into
// shared memory with cp.async.bulk, P tiles ahead, each stage completed on its
// own mbarrier.  The loads in flight no longer depend on the registers a
// thread can hold.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_addr(bar)), "r"(phase) : "memory");
  return ok != 0;
}
// Bounded wait for a stage; on expiry raises *err and returns false.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned phase, int* err,
                                          unsigned long long timeout_ns) {
  if (mbar_test(bar, phase)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_test(bar, phase)) {
    if (globaltimer_ns() - t0 > timeout_ns) {
      atomicCAS(err, kErrNone, kErrTimeout);
      return false;
    }
  }
  return true;
}

struct BulkPipe {
  unsigned char* stage;        // [warp][cap] staging area of each warp
  unsigned long long* bar;     // [warp][kMaxStages]
  int P;                       // most stages per warp
  int cap;                     // bytes of staging area per warp (>= m 32-point rows)
  int* err;
  unsigned long long timeout_ns;
};

// ------------------------------------------------------------ the passes --
// Grid points per thread per loop trip for an accumulator bucket of K slots:
// small buckets take several points so that enough loads are in flight.
template <typename T, int K>
struct PointsPerTrip {
  static constexpr int value = sizeof(T) == 4 ? (K <= 8 ? 4 : (K <= 24 ? 2 : 1)) : (K <= 8 ? 2 : 1);
};

// X pass for step j < K over this CTA's points [lo, hi): v_j = (w' - V h2)/hn,
// z = (A w' - sum_i c_i v_i)/hn, then per-warp partials of h1 = V^T z (slots
// 0..j) and ||z||^2 (slot j+1) into sm.red.
template <typename T, int DIM, int MAXM, int BS, int K>
__device__ __forceinline__ void x_pass(Smem<T, MAXM, BS>& sm, int lo, int hi, int j, int n,
                                       const T* __restrict__ WP, T* __restrict__ Z,
                                       T* __restrict__ V, int rows, int voff,
                                       const float* __restrict__ kappa, T s2t) {
  constexpr int LMAX = MAXM + 2;
  constexpr int U = PointsPerTrip<T, K>::value;
  const int tid = threadIdx.x;
  T acc[K];
#pragma unroll
  for (int k = 0; k < K; k++) acc[k] = T(0);
  T accZ = T(0);
  const T inv = sm.invT;
  const T cj = sm.cv[j];
  for (int i0 = lo + tid; i0 < hi; i0 += U * BS) {
    int ii[U];
    bool ok_[U];
    T wp[U], znum[U], vnum[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      ii[u] = i0 + u * BS;
      ok_[u] = ii[u] < hi;
      wp[u] = ok_[u] ? ldcg(WP + ii[u]) : T(0);
    }
    long long vb[U];
#pragma unroll
    for (int u = 0; u < U; u++) vb[u] = vbase(ii[u] - voff, rows);
    T col[U][K];
#pragma unroll
    for (int k = 0; k < K; k++) {
      if (k < j) {
#pragma unroll
        for (int u = 0; u < U; u++) col[u][k] = ok_[u] ? V[vb[u] + vko(k)] : T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++)
      znum[u] = ok_[u] ? s2t * stencil<T, DIM>(WP, ii[u], n, kappa, wp[u]) : T(0);
    // sum_k h2_k v_k and sum_k c_k v_k with even and odd k apart, in the order
    // of the paired passes (x_proj), so that every placement of V rounds alike
    T sv[U][2], sz[U][2];
#pragma unroll
    for (int u = 0; u < U; u++) sv[u][0] = sv[u][1] = sz[u][0] = sz[u][1] = T(0);
#pragma unroll
    for (int k = 0; k < K; k++) {
      if (k < j) {
        const T h2k = sm.h2v[k], ck = sm.cv[k];
#pragma unroll
        for (int u = 0; u < U; u++) {
          sv[u][k & 1] = fma(h2k, col[u][k], sv[u][k & 1]);
          sz[u][k & 1] = fma(ck, col[u][k], sz[u][k & 1]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      vnum[u] = wp[u] - (sv[u][0] + sv[u][1]);
      znum[u] -= sz[u][0] + sz[u][1];
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const T vj = vnum[u] * inv;
      const T z = (znum[u] - cj * vj) * inv;
      if (ok_[u]) {
        store_vj(V + vb[u], j, vj);
        Z[ii[u]] = z;
      }
      accZ += z * z;
#pragma unroll
      for (int k = 0; k < K; k++) {
        if (k < j)
          acc[k] += col[u][k] * z;
        else if (k == j)
          acc[k] += vj * z;
      }
    }
  }
  warp_slots_k<LMAX, K, T>(sm.red, acc, j + 1);
  warp_slot<LMAX>(sm.red, j + 1, accZ);
}

// Y pass for step j < K: w' = z - V h1 (stored), per-warp partials of
// h2 = V^T w' (slots 0..j) and ||w'||^2 (slot j+1).
template <typename T, int MAXM, int BS, int K>
__device__ __forceinline__ void y_pass(Smem<T, MAXM, BS>& sm, int lo, int hi, int j,
                                       T* __restrict__ WP, const T* __restrict__ Z,
                                       const T* __restrict__ V, int rows, int voff) {
  constexpr int LMAX = MAXM + 2;
  constexpr int U = PointsPerTrip<T, K>::value;
  const int tid = threadIdx.x;
  T acc[K];
#pragma unroll
  for (int k = 0; k < K; k++) acc[k] = T(0);
  T accN = T(0);
  for (int i0 = lo + tid; i0 < hi; i0 += U * BS) {
    int ii[U];
    bool ok_[U];
    T q[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      ii[u] = i0 + u * BS;
      ok_[u] = ii[u] < hi;
      q[u] = ok_[u] ? Z[ii[u]] : T(0);
    }
    long long vb[U];
#pragma unroll
    for (int u = 0; u < U; u++) vb[u] = vbase(ii[u] - voff, rows);
    T col[U][K];
#pragma unroll
    for (int k = 0; k < K; k++) {
      if (k <= j) {
#pragma unroll
        for (int u = 0; u < U; u++) col[u][k] = ok_[u] ? V[vb[u] + vko(k)] : T(0);
      }
    }
    // sum_k h1_k v_k, even and odd k apart (the order of y_proj)
    T sq[U][2];
#pragma unroll
    for (int u = 0; u < U; u++) sq[u][0] = sq[u][1] = T(0);
#pragma unroll
    for (int k = 0; k < K; k++) {
      if (k <= j) {
        const T hk = sm.coef[k];
#pragma unroll
        for (int u = 0; u < U; u++) sq[u][k & 1] = fma(hk, col[u][k], sq[u][k & 1]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) q[u] -= sq[u][0] + sq[u][1];
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (ok_[u]) WP[ii[u]] = q[u];
      accN += q[u] * q[u];
#pragma unroll
      for (int k = 0; k < K; k++)
        if (k <= j) acc[k] += col[u][k] * q[u];
    }
  }
  warp_slots_k<LMAX, K, T>(sm.red, acc, j + 1);
  warp_slot<LMAX>(sm.red, j + 1, accN);
}

// ---------------------------------------- one point's column, in pairs --
// vc points at a point's column of V (pair layout: vector k at vc[vko(k)]),
// in shared memory (a CTA slice or a bulk-copy stage).  Even and odd k are
// accumulated apart, two basis values per load and per paired FMA.  Every
// pair read is whole: the X pass of an even step j stores (v_j, 0) as one
// pair, so the slot of vector j+1 holds zero until step j+1 writes it, and a
// pair that reaches one vector past the vectors in use adds nothing.

// X pass: (sum_{k<j} h2_k v_k, sum_{k<j} c_k v_k) over the pairs that hold
// vectors 0..j-1 (for odd j the last one also holds the zero slot of v_j).
// W4: FP32 coefficients by 16-byte loads (faster in the one-CTA-per-SM
// shared-slice passes and the 3D passes; the 2D bulk-copy pass runs 0.5% faster
// with 8-byte loads, and the compact shared-slice variant spills with them).
template <typename T, int MAXM, int BS, int K, bool W4 = true>
__device__ __forceinline__ void x_proj(const Smem<T, MAXM, BS>& sm, const T* vc, int j, T& sv,
                                       T& sz) {
  using T2 = typename Vec2<T>::type;
  const int np = (j + 1) >> 1;
  T2 av = dup2<T2>(T(0)), az = dup2<T2>(T(0));
  if constexpr (sizeof(T) == 4 && W4) {
    // FP32: the coefficients of pairs 2p and 2p+1 in one 16-byte load each,
    // issued for the whole bucket (h2v and cv are initialised to their end);
    // only the V loads and the FMAs depend on j, in the same order as below
    float4 h[K / 4], c[K / 4];
#pragma unroll
    for (int p = 0; p < K / 4; p++) {
      h[p] = reinterpret_cast<const float4*>(sm.h2v)[p];
      c[p] = reinterpret_cast<const float4*>(sm.cv)[p];
    }
#pragma unroll
    for (int q = 0; q < K / 2; q++) {
      if (q < np) {
        const T2 v = *reinterpret_cast<const T2*>(vc + (q << 6));
        const float4 hq = h[q >> 1], cq = c[q >> 1];
        av = fma2((q & 1) ? make_float2(hq.z, hq.w) : make_float2(hq.x, hq.y), v, av);
        az = fma2((q & 1) ? make_float2(cq.z, cq.w) : make_float2(cq.x, cq.y), v, az);
      }
    }
  } else {
    const T2* h2 = reinterpret_cast<const T2*>(sm.h2v);
    const T2* cc = reinterpret_cast<const T2*>(sm.cv);
#pragma unroll
    for (int q = 0; q < K / 2; q++) {
      if (q < np) {
        const T2 v = *reinterpret_cast<const T2*>(vc + (q << 6));
        av = fma2(h2[q], v, av);
        az = fma2(cc[q], v, az);
      }
    }
  }
  sv = av.x + av.y;
  sz = az.x + az.y;
}

// X pass dots, after v_j is stored in the column: acc_k += v_k z for k <= j
// (for even j the last pair is (v_j, 0)).  acc holds slots 2q, 2q+1 in acc[q].
template <typename T, int K>
__device__ __forceinline__ void x_dots(typename Vec2<T>::type (&acc)[K / 2], const T* vc, int j,
                                       T z) {
  using T2 = typename Vec2<T>::type;
  const T2 zz = dup2<T2>(z);
  const int np = (j >> 1) + 1;
#pragma unroll
  for (int q = 0; q < K / 2; q++)
    if (q < np) acc[q] = fma2(*reinterpret_cast<const T2*>(vc + (q << 6)), zz, acc[q]);
}

// Y pass: sum_{k<=j} h1_k v_k (h1 in sm.coef; for even j the last pair's
// second value is the zero slot of v_{j+1}).
template <typename T, int MAXM, int BS, int K, bool W4 = true>
__device__ __forceinline__ T y_proj(const Smem<T, MAXM, BS>& sm, const T* vc, int j) {
  using T2 = typename Vec2<T>::type;
  const int np = (j >> 1) + 1;
  T2 a = dup2<T2>(T(0));
  if constexpr (sizeof(T) == 4 && W4) {
    // FP32: h1 of pairs 2p and 2p+1 in one 16-byte load (as in x_proj)
    float4 h[K / 4];
#pragma unroll
    for (int p = 0; p < K / 4; p++) h[p] = reinterpret_cast<const float4*>(sm.coef)[p];
#pragma unroll
    for (int q = 0; q < K / 2; q++) {
      if (q < np) {
        const float4 hq = h[q >> 1];
        a = fma2((q & 1) ? make_float2(hq.z, hq.w) : make_float2(hq.x, hq.y),
                 *reinterpret_cast<const T2*>(vc + (q << 6)), a);
      }
    }
  } else {
    const T2* h1 = reinterpret_cast<const T2*>(sm.coef);
#pragma unroll
    for (int q = 0; q < K / 2; q++)
      if (q < np) a = fma2(h1[q], *reinterpret_cast<const T2*>(vc + (q << 6)), a);
  }
  return a.x + a.y;
}

// Y pass dots: acc_k += v_k w' for k <= j.
template <typename T, int K>
__device__ __forceinline__ void y_dots(typename Vec2<T>::type (&acc)[K / 2], const T* vc, int j,
                                       T w) {
  using T2 = typename Vec2<T>::type;
  const T2 ww = dup2<T2>(w);
  const int np = (j >> 1) + 1;
#pragma unroll
  for (int q = 0; q < K / 2; q++)
    if (q < np) acc[q] = fma2(*reinterpret_cast<const T2*>(vc + (q << 6)), ww, acc[q]);
}

// warp_slots_k for accumulators held in pairs (slots 2q, 2q+1 in acc[q]).
template <int LMAX, int K, typename T>
__device__ __forceinline__ void warp_slots_k2(T (*red)[LMAX],
                                              const typename Vec2<T>::type (&acc)[K / 2], int L) {
  T a[K];
#pragma unroll
  for (int k = 0; k < K; k++) a[k] = (k & 1) ? acc[k >> 1].y : acc[k >> 1].x;
  warp_slots_k<LMAX, K, T>(red, a, L);
}

// X and Y passes with the CTA's slice of V in shared memory (2D): the same
// arithmetic as x_pass / y_pass, but a point's V column is read from shared
// memory twice (update, then dots) instead of being held in registers, so
// registers only carry the accumulators; U points per trip keep the
// stencil's global loads in flight together.
// What a thread carries between the passes of the shared-slice 2D variant for
// its first U = 2 points: w' at each point and its four neighbours, loaded
// right after the Y barrier so that the loads are in flight while the CTA
// gathers h2 and runs the scalar recurrences; and z from the X pass, which the
// Y pass of the same step needs at the same points (no reload through L2).
template <typename T>
struct XCarry {
  T c[2], l[2], r[2], d[2], t[2];
  T z[2];
  bool pre;  // the w' values are those the next X pass needs
};

template <typename T, int BS>
__device__ __forceinline__ void prefetch_x2d(XCarry<T>& cy, const T* __restrict__ WP, int lo,
                                             int hi, int n) {
#pragma unroll
  for (int u = 0; u < 2; u++) {
    const int i = lo + (int)threadIdx.x + u * BS;
    const bool ok = i < hi;
    const int ix = i % n, iy = i / n;
    cy.c[u] = ok ? ldcg(WP + i) : T(0);
    cy.l[u] = ok && ix > 0 ? ldcg(WP + i - 1) : T(0);
    cy.r[u] = ok && ix < n - 1 ? ldcg(WP + i + 1) : T(0);
    cy.d[u] = ok && iy > 0 ? ldcg(WP + i - n) : T(0);
    cy.t[u] = ok && iy < n - 1 ? ldcg(WP + i + n) : T(0);
  }
  cy.pre = true;
}

template <typename T, int DIM, int MAXM, int BS, int K>
__device__ __forceinline__ void x_pass_sm(Smem<T, MAXM, BS>& sm, int lo, int hi, int j, int n,
                                          const T* __restrict__ WP, T* __restrict__ Z,
                                          T* __restrict__ Vs, int rows,
                                          const float* __restrict__ kappa, T s2t,
                                          XCarry<T>& cy) {
  static_assert(DIM == 2, "shared-memory slices are a 2D variant");
  constexpr int LMAX = MAXM + 2;
  using T2 = typename Vec2<T>::type;
  const int tid = threadIdx.x;
  T2 acc[K / 2];
#pragma unroll
  for (int q = 0; q < K / 2; q++) acc[q] = dup2<T2>(T(0));
  T accZ = T(0);
  const T inv = sm.invT;
  const T cj = sm.cv[j];
  // FP32, m <= 32: h2 and c in registers for all of the thread's points (at
  // larger bucket limits they spill)
  constexpr bool creg = sizeof(T) == 4 && MAXM <= kSmallM;
  float4 h2r[creg ? K / 4 : 1], ccr[creg ? K / 4 : 1];
  if constexpr (creg) {
#pragma unroll
    for (int p = 0; p < K / 4; p++) {
      h2r[p] = reinterpret_cast<const float4*>(sm.h2v)[p];
      ccr[p] = reinterpret_cast<const float4*>(sm.cv)[p];
    }
  }
  // one point per trip, the loop not unrolled: the body sits in the
  // instruction stream once (the step's code is what bounds it at this size)
  int t = 0;
#pragma unroll 1
  for (int i = lo + tid; i < hi; i += BS, t++) {
    T wp, znum;
    if (t < 2 && cy.pre) {
      // the same differences, in the same order, as stencil2d
      const bool s1 = t == 1;
      const T uc = s1 ? cy.c[1] : cy.c[0];
      const T l = s1 ? cy.l[1] : cy.l[0], r = s1 ? cy.r[1] : cy.r[0];
      const T d = s1 ? cy.d[1] : cy.d[0], tp = s1 ? cy.t[1] : cy.t[0];
      wp = uc;
      znum = s2t * (((uc - l) + (uc - r)) + ((uc - d) + (uc - tp)));
    } else {
      wp = ldcg(WP + i);
      znum = s2t * stencil<T, DIM>(WP, i, n, kappa, wp);
    }
    const T* vc = Vs + vbase(i - lo, rows);
    T sv, sz;
    if constexpr (creg) {
      const int np = (j + 1) >> 1;
      float2 av = make_float2(0.f, 0.f), az = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < K / 2; q++) {
        if (q < np) {
          const float2 v = *reinterpret_cast<const float2*>(vc + (q << 6));
          const float4 hq = h2r[q >> 1], cq = ccr[q >> 1];
          av = fma2((q & 1) ? make_float2(hq.z, hq.w) : make_float2(hq.x, hq.y), v, av);
          az = fma2((q & 1) ? make_float2(cq.z, cq.w) : make_float2(cq.x, cq.y), v, az);
        }
      }
      sv = av.x + av.y;
      sz = az.x + az.y;
    } else {
      x_proj<T, MAXM, BS, K, !compact_bucket<MAXM>()>(sm, vc, j, sv, sz);
    }
    const T vj = (wp - sv) * inv;
    const T z = ((znum - sz) - cj * vj) * inv;
    store_vj(Vs + vbase(i - lo, rows), j, vj);
    Z[i] = z;
    if (t == 0) cy.z[0] = z;
    if (t == 1) cy.z[1] = z;
    accZ += z * z;
    x_dots<T, K>(acc, vc, j, z);
  }
  warp_slots_k2<LMAX, K, T>(sm.red, acc, j + 1);
  warp_slot<LMAX>(sm.red, j + 1, accZ);
}

template <typename T, int MAXM, int BS, int K>
__device__ __forceinline__ void y_pass_sm(Smem<T, MAXM, BS>& sm, int lo, int hi, int j,
                                          T* __restrict__ WP, const T* __restrict__ Z,
                                          const T* __restrict__ Vs, int rows,
                                          const XCarry<T>& cy) {
  constexpr int LMAX = MAXM + 2;
  using T2 = typename Vec2<T>::type;
  const int tid = threadIdx.x;
  T2 acc[K / 2];
#pragma unroll
  for (int q = 0; q < K / 2; q++) acc[q] = dup2<T2>(T(0));
  T accN = T(0);
  // FP32, one CTA per SM: h1 in registers for all of the thread's points (one
  // set of 16-byte loads per pass instead of one per point)
  constexpr bool hreg = sizeof(T) == 4 && !compact_bucket<MAXM>();
  float4 h1r[hreg ? K / 4 : 1];
  if constexpr (hreg) {
#pragma unroll
    for (int p = 0; p < K / 4; p++) h1r[p] = reinterpret_cast<const float4*>(sm.coef)[p];
  }
  int t = 0;
#pragma unroll 1
  for (int i = lo + tid; i < hi; i += BS, t++) {
    // z of the thread's first two points is in cy (the X pass kept it)
    const T q = t == 0 ? cy.z[0] : (t == 1 ? cy.z[1] : Z[i]);
    const T* vc = Vs + vbase(i - lo, rows);
    T qv;
    if constexpr (hreg) {
      const int np = (j >> 1) + 1;
      float2 a = make_float2(0.f, 0.f);
#pragma unroll
      for (int qq = 0; qq < K / 2; qq++) {
        if (qq < np) {
          const float4 hq = h1r[qq >> 1];
          a = fma2((qq & 1) ? make_float2(hq.z, hq.w) : make_float2(hq.x, hq.y),
                   *reinterpret_cast<const float2*>(vc + (qq << 6)), a);
        }
      }
      qv = q - (a.x + a.y);
    } else {
      qv = q - y_proj<T, MAXM, BS, K, !compact_bucket<MAXM>()>(sm, vc, j);
    }
    WP[i] = qv;
    accN += qv * qv;
    y_dots<T, K>(acc, vc, j, qv);
  }
  warp_slots_k2<LMAX, K, T>(sm.red, acc, j + 1);
  warp_slot<LMAX>(sm.red, j + 1, accN);
}

// Besides the tile's V rows, every stage carries the other values the pass
// needs, so that no load of a pass waits outside the bulk-copy pipeline:
//   X pass: w' over [i0 - 4, i0 + 36) (the tile and its +-1 neighbours) and
//           the rows of the tile's neighbours across the grid (+-n; in 3D also
//           +-n^2), 36 values each from a 16-byte aligned start; in 3D with
//           kappa (when kappa is 16-byte aligned and N a multiple of 4) the
//           same windows of kappa;
//   Y pass: z over the tile.
// Copies are clipped to the arrays (w' and z to ldv, kappa to N); the clipped
// parts are never read (the stencil's boundary tests exclude them).
template <typename T, int DIM>
struct Aux {
  static constexpr int kRows = DIM == 3 ? 4 : 2;  // -n, +n (, -n^2, +n^2)
  static constexpr int kCen = 40, kRow = 36;
  static constexpr int kW = kCen + kRows * kRow;  // elements of T (w')
  static constexpr int kK = DIM == 3 ? kW : 0;    // floats (kappa)
  // 3D with face coefficients instead of kappa (floats): fx over [i0-4, i0+36),
  // fy, fz and fb over the tile [i0, i0+32), fy of the row -n and fz of the
  // row -n^2 (36 values each from a 16-byte aligned start)
  static constexpr int kFx = 0, kFy = 40, kFyM = 72, kFz = 108, kFzM = 140, kFb = 176;
  static constexpr int kF = DIM == 3 ? 208 : 0;
  static constexpr int kXBytes = kW * (int)sizeof(T) + (kK > kF ? kK : kF) * 4;
  static constexpr int kYBytes = 32 * (int)sizeof(T);
};

// Per-warp ring of bulk-copy stages for one pass: the pair rows holding the
// first `vrows` rows of V per tile are copied, in a V part with room for
// `vroom` rows, followed by `abytes` of auxiliary values; as many stages as
// fit in the warp's share of the staging buffer (up to pp.P), so that small j
// keep more tiles in flight.
struct BulkRing {
  unsigned char* st;          // the warp's staging area
  unsigned long long* bars;   // the warp's stage barriers
  unsigned vcopy;             // V bytes copied per stage (whole pair rows)
  unsigned vbytes;            // V part of a stage (vroom rows, rounded to pairs)
  unsigned bytes;             // bytes per stage (V part + auxiliary part)
  int P;                      // stages in use for this pass
};

template <typename T>
__device__ __forceinline__ BulkRing bulk_ring(const BulkPipe& pp, int vrows, int vroom,
                                              int abytes) {
  BulkRing r;
  const int warp = threadIdx.x >> 5;
  r.st = pp.stage + (size_t)warp * pp.cap;
  r.bars = pp.bar + warp * kMaxStages;
  r.vcopy = (unsigned)vrows_p(vrows) * 32u * (unsigned)sizeof(T);
  r.vbytes = (unsigned)vrows_p(vroom) * 32u * (unsigned)sizeof(T);
  r.bytes = r.vbytes + (unsigned)abytes;
  const int fit = pp.cap / (int)r.bytes;
  r.P = max(1, min(pp.P, fit));
  return r;
}

// a multiple of a (a power of two) at or below v, for negative v as well
__device__ __forceinline__ int floor_to(int v, int a) { return v & ~(a - 1); }

// Adds `bytes` to the stage's expected transaction count (no arrival).
__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Copies the part of the run src[want, want + cnt) that lies in [0, limit) to
// dst + (its start - want) elements, registering its bytes on the stage's
// barrier first.  want, cnt and limit are multiples of 16 / sizeof(E).
template <typename E>
__device__ __forceinline__ void stage_run(E* dst, const E* src, int want, int cnt,
                                          long long limit, unsigned long long* bar) {
  const long long lo = want < 0 ? 0 : want;
  const long long hi = (long long)want + cnt < limit ? (long long)want + cnt : limit;
  if (hi <= lo) return;
  const unsigned bytes = (unsigned)(hi - lo) * (unsigned)sizeof(E);
  mbar_expect(bar, bytes);
  bulk_g2s(dst + (lo - want), src + lo, bytes, bar);
}

struct AuxSrc {  // what the X pass's stages copy besides V
  const void* wp;       // w' (elements of T)
  const float* kap;     // kappa (3D), or null when it is not staged
  const float* fc;      // face coefficients (3D, FP32; w' padded), or null
  long long fs;         // their array stride
  int n;
  long long N, ldv;
};

// Lane 0 issues stage q: tile lo/32 + warp + NW q.  X pass (aux != null):
// the tile's first pair rows of V (r.vcopy bytes; `rows` rows per tile) and the
// w'/kappa windows; Y pass: V rows and z.  Each
// copy registers its bytes before it is issued; the single arrival comes last,
// so the stage's phase cannot complete early.
template <int NW, typename T, int DIM>
__device__ __forceinline__ void bulk_issue_stage(const BulkRing& r, const T* V, int lo, int rows,
                                                 int q, int sidx, const AuxSrc* aux, const T* Zsrc,
                                                 long long ldv) {
  using A = Aux<T, DIM>;
  constexpr int ALN = 16 / (int)sizeof(T);
  const int i0 = lo + (int)((threadIdx.x >> 5) + NW * q) * 32;
  unsigned char* st = r.st + (size_t)sidx * r.bytes;
  T* at = reinterpret_cast<T*>(st + r.vbytes);
  unsigned long long* bar = &r.bars[sidx];
  // Fast path: no copy needs clipping (every window lies inside its array; the
  // z window of the Y pass always does, since ldv is a multiple of 64 >= N).
  // One arrive.expect_tx registers all of the stage's bytes before the copies
  // are issued (the phase completes only when they have landed), instead of
  // one expect_tx per copy and the clipping arithmetic of each.
  {
    const long long dmax = aux ? (DIM == 3 ? (long long)aux->n * aux->n : aux->n) : 0;
    const long long lim = aux ? (aux->kap && aux->N < ldv ? aux->N : ldv) : ldv;
    // (with face coefficients, w' and the coefficients are padded: never clipped)
    if (!aux || aux->fc ||
        ((long long)i0 - dmax - 16 >= 0 && (long long)i0 + dmax + 40 <= lim)) {
      const bool fcs = aux && A::kF > 0 && aux->fc;
      const bool kap = aux && A::kK > 0 && aux->kap && !fcs;
      const unsigned abytes =
          aux ? (unsigned)(A::kW * (int)sizeof(T) + (kap ? A::kW * 4 : 0) + (fcs ? A::kF * 4 : 0))
              : 32u * sizeof(T);
      mbar_expect_tx(bar, r.vcopy + abytes);
      if (r.vcopy) bulk_g2s(st, V + vbase(i0, rows), r.vcopy, bar);
      if (!aux) {
        bulk_g2s(at, Zsrc + i0, 32u * sizeof(T), bar);
        return;
      }
      const T* wp = reinterpret_cast<const T*>(aux->wp);
      const int n = aux->n, nn = n * n;
      bulk_g2s(at, wp + (i0 - 4), A::kCen * (unsigned)sizeof(T), bar);
#pragma unroll
      for (int k = 0; k < A::kRows; k++) {
        const int d = k == 0 ? -n : (k == 1 ? n : (k == 2 ? -nn : nn));
        bulk_g2s(at + A::kCen + k * A::kRow, wp + floor_to(i0 + d, ALN),
                 A::kRow * (unsigned)sizeof(T), bar);
      }
      if (kap) {
        float* ak = reinterpret_cast<float*>(at + A::kW);
        bulk_g2s(ak, aux->kap + (i0 - 4), A::kCen * 4u, bar);
#pragma unroll
        for (int k = 0; k < A::kRows; k++) {
          const int d = k == 0 ? -n : (k == 1 ? n : (k == 2 ? -nn : nn));
          bulk_g2s(ak + A::kCen + k * A::kRow, aux->kap + floor_to(i0 + d, 4), A::kRow * 4u, bar);
        }
      }
      if (fcs) {
        float* af = reinterpret_cast<float*>(at + A::kW);
        const float* fx = aux->fc;
        const float* fy = fx + aux->fs;
        const float* fz = fy + aux->fs;
        const float* fb = fz + aux->fs;
        bulk_g2s(af + A::kFx, fx + (i0 - 4), 160u, bar);
        bulk_g2s(af + A::kFy, fy + i0, 128u, bar);
        bulk_g2s(af + A::kFyM, fy + floor_to(i0 - n, 4), 144u, bar);
        bulk_g2s(af + A::kFz, fz + i0, 128u, bar);
        bulk_g2s(af + A::kFzM, fz + floor_to(i0 - nn, 4), 144u, bar);
        bulk_g2s(af + A::kFb, fb + i0, 128u, bar);
      }
      return;
    }
  }
  // Near the ends of the arrays: each copy clipped, and registered on its own.
  if (r.vcopy) {
    mbar_expect(bar, r.vcopy);
    bulk_g2s(st, V + vbase(i0, rows), r.vcopy, bar);
  }
  if (aux) {
    const T* wp = reinterpret_cast<const T*>(aux->wp);
    const int n = aux->n, nn = n * n;
    stage_run<T>(at, wp, i0 - 4, A::kCen, ldv, bar);
#pragma unroll
    for (int k = 0; k < A::kRows; k++) {
      const int d = k == 0 ? -n : (k == 1 ? n : (k == 2 ? -nn : nn));
      stage_run<T>(at + A::kCen + k * A::kRow, wp, floor_to(i0 + d, ALN), A::kRow, ldv, bar);
    }
    if (A::kK > 0 && aux->kap) {
      float* ak = reinterpret_cast<float*>(at + A::kW);
      stage_run<float>(ak, aux->kap, i0 - 4, A::kCen, aux->N, bar);
#pragma unroll
      for (int k = 0; k < A::kRows; k++) {
        const int d = k == 0 ? -n : (k == 1 ? n : (k == 2 ? -nn : nn));
        stage_run<float>(ak + A::kCen + k * A::kRow, aux->kap, floor_to(i0 + d, 4), A::kRow,
                         aux->N, bar);
      }
    }
  } else {
    stage_run<T>(at, Zsrc, i0, 32, ldv, bar);
  }
  mbar_arrive(bar);
}

// Waits (bounded) for the copies this warp issued for trips q+1 .. last, so
// that none is left in flight when a pass is abandoned.
__device__ __forceinline__ void bulk_drain(const BulkRing& r, const BulkPipe& pp, int q, int nq,
                                           unsigned& phase) {
  for (int t = q + 1; t < nq && t < q + r.P; t++) {
    const int sidx = t % r.P;
    if (mbar_wait(&r.bars[sidx], (phase >> sidx) & 1u, pp.err, pp.timeout_ns))
      phase ^= 1u << sidx;
  }
}

// The 3D operator at point i = i0 + lane from a stage's w' windows and face
// coefficient windows: fb u_c + sum over the six faces of f (u_c - u_nb), in
// the face order of stencil3d (-x, +x, -y, +y, -z, +z).  A wall face has
// f = 0 here (its kappa_c u_c is in fb) and its u_nb is a zero pad or a finite
// value of w', so no coordinate tests are needed.
template <typename T>
__device__ __forceinline__ T stencil_faces(const T* aw, const float* af, int i0, int lane, int n) {
  using A = Aux<T, 3>;
  constexpr int ALN = 16 / (int)sizeof(T);
  const int nn = n * n;
  const T uc = aw[4 + lane];
  auto wrow = [&](int k, int d) {
    return aw[A::kCen + k * A::kRow + (i0 + d - floor_to(i0 + d, ALN)) + lane];
  };
  const T wl = aw[3 + lane], wr = aw[5 + lane];
  const T wd = wrow(0, -n), wt = wrow(1, n), wb = wrow(2, -nn), wf = wrow(3, nn);
  const T fxl = (T)af[A::kFx + 3 + lane], fxr = (T)af[A::kFx + 4 + lane];
  const T fyd = (T)af[A::kFyM + (i0 - n - floor_to(i0 - n, 4)) + lane];
  const T fyt = (T)af[A::kFy + lane];
  const T fzb = (T)af[A::kFzM + (i0 - nn - floor_to(i0 - nn, 4)) + lane];
  const T fzf = (T)af[A::kFz + lane];
  T acc = (T)af[A::kFb + lane] * uc;
  acc += fxl * (uc - wl);
  acc += fxr * (uc - wr);
  acc += fyd * (uc - wd);
  acc += fyt * (uc - wt);
  acc += fzb * (uc - wb);
  acc += fzf * (uc - wf);
  return acc;
}

// The stencil of stencil<T, DIM> at point i = i0 + lane from a stage's w'
// windows (and kappa windows when staged; else kappa from global memory):
// the same differences, faces and order.
template <typename T, int DIM>
__device__ __forceinline__ T stencil_staged(const T* aw, const float* ak,
                                            const float* __restrict__ kappa, int i, int i0,
                                            int lane, int n, int ix, int iy, int iz) {
  using A = Aux<T, DIM>;
  constexpr int ALN = 16 / (int)sizeof(T);
  const T uc = aw[4 + lane];
  // neighbour f (-1, +1, -n, +n, -n^2, +n^2): its w' in the stage, and its kappa
  auto wnb = [&](int f) -> T {
    if (f < 2) return aw[4 + lane + (f == 0 ? -1 : 1)];
    const int k = f - 2, nn = n * n;
    const int d = k == 0 ? -n : (k == 1 ? n : (k == 2 ? -nn : nn));
    return aw[A::kCen + k * A::kRow + (i0 + d - floor_to(i0 + d, ALN)) + lane];
  };
  if constexpr (DIM == 2) {
    const T l = ix > 0 ? wnb(0) : T(0);
    const T r = ix < n - 1 ? wnb(1) : T(0);
    const T d = iy > 0 ? wnb(2) : T(0);
    const T t = iy < n - 1 ? wnb(3) : T(0);
    return ((uc - l) + (uc - r)) + ((uc - d) + (uc - t));
  } else {
    const int nn = n * n;
    T acc = T(0);
    if (kappa) {
      auto knbf = [&](int f) -> T {
        const int off = f == 0 ? -1 : (f == 1 ? 1 : (f == 2 ? -n : (f == 3 ? n : (f == 4 ? -nn : nn))));
        if (!ak) return (T)__ldg(kappa + i + off);
        if (f < 2) return (T)ak[4 + lane + off];
        const int k = f - 2;
        return (T)ak[A::kCen + k * A::kRow + (i0 + off - floor_to(i0 + off, 4)) + lane];
      };
      const T kc = ak ? (T)ak[4 + lane] : (T)__ldg(kappa + i);
#pragma unroll
      for (int f = 0; f < 6; f++) {
        const bool has = f == 0 ? ix > 0 : f == 1 ? ix < n - 1 : f == 2 ? iy > 0
                       : f == 3 ? iy < n - 1 : f == 4 ? iz > 0 : iz < n - 1;
        if (has)
          acc += face(kc, knbf(f)) * (uc - wnb(f));
        else
          acc += kc * uc;
      }
    } else {
#pragma unroll
      for (int f = 0; f < 6; f++) {
        const bool has = f == 0 ? ix > 0 : f == 1 ? ix < n - 1 : f == 2 ? iy > 0
                       : f == 3 ? iy < n - 1 : f == 4 ? iz > 0 : iz < n - 1;
        acc += has ? (uc - wnb(f)) : uc;
      }
    }
    return acc;
  }
}

// X pass with V in HBM, staged per warp through the bulk-copy ring together
// with the w' (and kappa) windows.  The V column of a point is read from the
// stage twice (update, then dots) instead of being held in registers.
template <typename T, int DIM, int MAXM, int BS, int K>
__device__ __forceinline__ void x_pass_bulk(Smem<T, MAXM, BS>& sm, int lo, int hi, int j,
                                            int n, const T* __restrict__ WP,
                                            T* __restrict__ Z, T* __restrict__ V,
                                            int rows, const float* __restrict__ kappa,
                                            T s2t, const BulkPipe& pp, unsigned& phase,
                                            const AuxSrc& aux) {
  using A = Aux<T, DIM>;
  using T2 = typename Vec2<T>::type;
  constexpr int LMAX = MAXM + 2;
  constexpr int NW = BS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T2 acc[K / 2];
#pragma unroll
  for (int q = 0; q < K / 2; q++) acc[q] = dup2<T2>(T(0));
  T accZ = T(0);
  const T inv = sm.invT;
  const T cj = sm.cv[j];
  const int ntile = (hi - lo + 31) >> 5;
  const int nq = ntile > warp ? (ntile - warp + NW - 1) / NW : 0;
  // rows 0..j-1 copied; room for the pair holding v_j, which the pass writes
  const BulkRing r = bulk_ring<T>(pp, j, j + 1, A::kXBytes);
  // w' (and z, V) were written through the generic proxy; the copies read
  // through the async proxy
  asm volatile("fence.proxy.async.global;" ::: "memory");
  if (lane == 0)
    for (int q = 0; q < r.P && q < nq; q++)
      bulk_issue_stage<NW, T, DIM>(r, V, lo, rows, q, q, &aux, nullptr, aux.ldv);
  bool good = true;
  // grid coordinates of this lane's point, advanced by NW * 32 points per trip
  // (integer divisions once per pass instead of once per point)
  int px = 0, py = 0, pz = 0;
  {
    const int i = lo + warp * 32 + lane;
    px = i % n;
    const int t = i / n;
    py = DIM == 3 ? t % n : t;
    pz = DIM == 3 ? t / n : 0;
  }
  int q = 0;
  // stage slot of trip q (q mod P, kept as a running index: no division)
  for (int sidx = 0; q < nq; q++, sidx = sidx + 1 == r.P ? 0 : sidx + 1) {
    const int i0 = lo + (warp + NW * q) * 32;
    const int i = i0 + lane;
    const bool ok = i < hi;
    if (!mbar_wait(&r.bars[sidx], (phase >> sidx) & 1u, pp.err, pp.timeout_ns)) {
      good = false;
      break;
    }
    phase ^= 1u << sidx;
    const unsigned char* stb = r.st + (size_t)sidx * r.bytes;
    const T* sc = reinterpret_cast<const T*>(stb) + 2 * lane;  // the lane's column (pair layout)
    const T* aw = reinterpret_cast<const T*>(stb + r.vbytes);
    const float* ak = (A::kK > 0 && aux.kap) ? reinterpret_cast<const float*>(aw + A::kW) : nullptr;
    const float* af = (A::kF > 0 && aux.fc) ? reinterpret_cast<const float*>(aw + A::kW) : nullptr;
    const T wp = ok ? aw[4 + lane] : T(0);
    // (2D: the division per point measured faster than the incremental form)
    if constexpr (DIM == 2) {
      px = i % n;
      py = i / n;
    }
    T znum = T(0);
    if constexpr (DIM == 3) {
      if (af)
        znum = ok ? s2t * stencil_faces<T>(aw, af, i0, lane, n) : T(0);
      else
        znum = ok ? s2t * stencil_staged<T, DIM>(aw, ak, kappa, i, i0, lane, n, px, py, pz) : T(0);
    } else {
      znum = ok ? s2t * stencil_staged<T, DIM>(aw, ak, kappa, i, i0, lane, n, px, py, pz) : T(0);
    }
    if (DIM == 3 && !af) {
      px += NW * 32;  // the next trip's point
      while (px >= n) {
        px -= n;
        if (++py == n) {
          py = 0;
          ++pz;
        }
      }
    }
    T sv = T(0), sz = T(0);
    if (ok) x_proj<T, MAXM, BS, K, DIM == 3>(sm, sc, j, sv, sz);
    const T vj = (wp - sv) * inv;
    const T z = ((znum - sz) - cj * vj) * inv;
    if (ok) {
      store_vj(V + vbase(i, rows), j, vj);
      // and into the stage, whose V part has room for the pair of v_j
      store_vj(const_cast<T*>(sc), j, vj);
      Z[i] = z;
      // points past the end of a ragged last tile hold stale values: skipped
      x_dots<T, K>(acc, sc, j, z);
      accZ += z * z;
    }
    __syncwarp();
    if (lane == 0 && q + r.P < nq)
      bulk_issue_stage<NW, T, DIM>(r, V, lo, rows, q + r.P, sidx, &aux, nullptr, aux.ldv);
  }
  if (!good) bulk_drain(r, pp, q, nq, phase);
  // the V_j and z stores above are read by later bulk copies (async proxy)
  asm volatile("fence.proxy.async.global;" ::: "memory");
  warp_slots_k2<LMAX, K, T>(sm.red, acc, j + 1);
  warp_slot<LMAX>(sm.red, j + 1, accZ);
}

// Y pass with V in HBM through the bulk-copy ring (V rows and z per stage).
template <typename T, int DIM, int MAXM, int BS, int K>
__device__ __forceinline__ void y_pass_bulk(Smem<T, MAXM, BS>& sm, int lo, int hi, int j,
                                            T* __restrict__ WP, const T* __restrict__ Z,
                                            const T* __restrict__ V, int rows,
                                            const BulkPipe& pp, unsigned& phase, long long ldv) {
  using A = Aux<T, DIM>;
  using T2 = typename Vec2<T>::type;
  constexpr int LMAX = MAXM + 2;
  constexpr int NW = BS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T2 acc[K / 2];
#pragma unroll
  for (int q = 0; q < K / 2; q++) acc[q] = dup2<T2>(T(0));
  T accN = T(0);
  const int ntile = (hi - lo + 31) >> 5;
  const int nq = ntile > warp ? (ntile - warp + NW - 1) / NW : 0;
  const BulkRing r = bulk_ring<T>(pp, j + 1, j + 1, A::kYBytes);
  if (lane == 0)
    for (int q = 0; q < r.P && q < nq; q++)
      bulk_issue_stage<NW, T, DIM>(r, V, lo, rows, q, q, nullptr, Z, ldv);
  bool good = true;
  int q = 0;
  // stage slot of trip q (q mod P, kept as a running index: no division)
  for (int sidx = 0; q < nq; q++, sidx = sidx + 1 == r.P ? 0 : sidx + 1) {
    const int i = lo + (warp + NW * q) * 32 + lane;
    const bool ok = i < hi;
    if (!mbar_wait(&r.bars[sidx], (phase >> sidx) & 1u, pp.err, pp.timeout_ns)) {
      good = false;
      break;
    }
    phase ^= 1u << sidx;
    const unsigned char* stb = r.st + (size_t)sidx * r.bytes;
    const T* sc = reinterpret_cast<const T*>(stb) + 2 * lane;  // the lane's column (pair layout)
    if (ok) {
      const T qv = reinterpret_cast<const T*>(stb + r.vbytes)[lane] -
                   y_proj<T, MAXM, BS, K, DIM == 3>(sm, sc, j);
      WP[i] = qv;
      accN += qv * qv;
      y_dots<T, K>(acc, sc, j, qv);
    }
    __syncwarp();
    if (lane == 0 && q + r.P < nq)
      bulk_issue_stage<NW, T, DIM>(r, V, lo, rows, q + r.P, sidx, nullptr, Z, ldv);
  }
  if (!good) bulk_drain(r, pp, q, nq, phase);
  warp_slots_k2<LMAX, K, T>(sm.red, acc, j + 1);
  warp_slot<LMAX>(sm.red, j + 1, accN);
}

// Bucket dispatch: the pass instantiated for the smallest multiple of 8 above j.
#define MLG_BUCKETS(CALL)                           \
  switch (j >> 3) {                                 \
    case 0: CALL(8); break;                         \
    case 1: CALL(16); break;                        \
    case 2: CALL(24); break;                        \
    case 3: CALL(32); break;                        \
    case 4: CALL(40); break;                        \
    case 5: if constexpr (MAXM >= 48) { CALL(48); } break; \
    case 6: if constexpr (MAXM >= 56) { CALL(56); } break; \
    default: if constexpr (MAXM >= 64) { CALL(64); } break; \
  }

// --------------------------------------------------------------- one solve --
// Arnoldi step j of a cycle (CGS2 with two group barriers).  Entering it, the
// work vector W holds w', the previous step's vector after its first
// projection (w'_0 = r), h2 = V^T w' are its still unapplied second-pass
// coefficients, hn = ||w' - V h2|| (Pythagoras) and c are the coefficients
// that turn A w' into A v_j through the Arnoldi relation
// A v_k = sum_i Hu(i,k) v_i:
//   X: v_j = (w' - V h2)/hn,  z = (A w' - sum_i c_i v_i)/hn  (= A v_j),
//      h1 = V_{0..j}^T z, ||z||^2                                 -> barrier
//   Y: w'_{j+1} = z - V h1, h2 = V_{0..j}^T w'_{j+1}, ||w'_{j+1}||^2 -> barrier
//   Hu(:,j) = h1 + h2, Hu(j+1,j) = hn_{j+1} = sqrt(||w'||^2 - ||h2||^2)
// When the Pythagorean difference cancels (||h2||^2 > ||w'||^2 / 2) an
// explicit pass applies h2 and measures the norm instead.  The Givens update
// of column j runs on thread 0 while the CTA already starts the next X pass;
// if it ends the cycle, that speculative pass is discarded.
template <typename T, int DIM, int MAXM, int BS, int VM>
__device__ void solve_one(const KParams& kp, const SolveTask& tk, const GroupWork& w, int lb,
                          int nb, unsigned long long& epoch, unsigned& bphase,
                          Smem<T, MAXM, BS>& sm) {
  constexpr int LD = MAXM + 1;
  constexpr int LMAX = MAXM + 2;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int n = tk.n;
  const int N = tk.N;
  const int m = kp.m;
  const bool arnoldi = kp.arnoldi_steps > 0;
  int chunk = (N + nb - 1) / nb;
  chunk = (chunk + 31) & ~31;  // whole tiles of the basis layout
  const int lo = min(N, lb * chunk);
  const int hi = min(N, lo + chunk);
  const int rows = m + 1;  // basis vectors per tile (V holds m+1 vectors)
  // V lives in shared memory when this CTA's slice fits the reserved space
  // (latency of a shared load instead of an L2 round trip); else in HBM.
  // (only the FP32 2D variant has slices small enough to be worth it; each
  // placement of V is its own kernel variant, so every pass uses the right
  // address space and registers are allocated per variant)
  const bool vshared = VM == kVShared;
  T* __restrict__ Vg = (T*)w.V;
  T* __restrict__ Vs = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(&sm) +
                                            smem_own_bytes<T, MAXM, BS>());
  T* __restrict__ V = vshared ? Vs : Vg;  // cycle-end and fallback passes
  const int voff = vshared ? lo : 0;
  // bulk-copy staging of V (FP32, V in HBM): stages follow the shared state
  const bool bulk = VM == kVBulk;
  (void)bulk;
  BulkPipe pipe;
  pipe.stage = reinterpret_cast<unsigned char*>(&sm) + smem_own_bytes<T, MAXM, BS>();
  pipe.P = kp.bulk_stages;
  pipe.cap = kp.bulk_cap;
  pipe.bar = &sm.bbar[0][0];
  pipe.err = w.bar.err;
  pipe.timeout_ns = w.bar.timeout_ns;
  T* __restrict__ WP = (T*)w.W0;  // w' (read by neighbours in X, rewritten in Y)
  T* __restrict__ Z = (T*)w.W1;   // z = A v_j, own rows only
  // what the bulk-copy stages carry besides V (kappa only when its copies can
  // be 16-byte aligned: aligned base, N a multiple of 4)
  AuxSrc auxs;
  auxs.wp = WP;
  auxs.kap = (tk.kappa && ((unsigned long long)tk.kappa & 15ull) == 0 && (N & 3) == 0)
                 ? tk.kappa
                 : nullptr;
  // face coefficients: the FP32 3D passes only (the FP64 ones keep FP64 faces)
  auxs.fc = (DIM == 3 && sizeof(T) == 4) ? tk.faces : nullptr;
  auxs.fs = tk.fstride;
  auxs.n = n;
  auxs.N = N;
  auxs.ldv = w.ldv;
  (void)auxs;
  const double h = 2.0 / (n + 1);
  const double s2 = 1.0 / (h * h);
  const T s2t = (T)s2;
  const float* kappa = tk.kappa;
  int red = 0;
  const int ps = w.pstride;
  auto part = [&]() { return w.part + (long long)(red & 1) * LMAX * ps; };
  const bool leader = (lb == 0 && tid == 0);

  long long iters = 0;
  int cycles = 0;
  int status = 1;
  double relres = 0.0, relres_first = -1.0, relres_guess = -1.0, relres_alt = -1.0;
  int used_alt = 0;
  double bnorm = 0.0;
  bool ok = true;

  if (VM == kVShared && (long long)chunk * vrows_p(rows) * (long long)sizeof(T) > kp.vsmem) {
    status = kErrConfig;  // the slice would overrun the shared-memory reservation
    goto finish;
  }
  // a warp's staging area must hold one stage of m rows and the X pass's windows
  if (VM == kVBulk &&
      kp.bulk_cap < vrows_p(m) * 32 * (int)sizeof(T) + Aux<T, DIM>::kXBytes) {
    status = kErrConfig;
    goto finish;
  }

  // ---- phase 0: ||b||, and the residuals of both guesses when an alternative
  // (learned) guess competes with the fallback already in x.
  if (!arnoldi) {
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
    const bool alt = tk.x_alt != nullptr;
    for (int i = lo + tid; i < hi; i += BS) {
      const double bi = tk.b[i];
      v0 += bi * bi;
      if (tk.zero_x) tk.x[i] = 0.0;
      if (alt) {
        const double xc = ldcg(tk.x + i);
        const double r0 = bi - s2 * stencil<double, DIM>(tk.x, i, n, kappa, xc);
        const double ac = ldcg(tk.x_alt + i);
        const double r1 = bi - s2 * stencil<double, DIM>(tk.x_alt, i, n, kappa, ac);
        v1 += r0 * r0;
        v2 += r1 * r1;
      }
    }
    warp_slot<4>(sm.redd, 0, v0);
    if (alt) {
      warp_slot<4>(sm.redd, 1, v1);
      warp_slot<4>(sm.redd, 2, v2);
    }
    block_finish<4, BS, double>(alt ? 3 : 1, part(), lb, sm.redd, ps);
    ok = group_sync(w.bar, epoch, &sm.flag);
    if (!ok) goto abort;
    gather<BS, double, T>(part(), alt ? 3 : 1, nb, sm.tot, sm.coef, ps);
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
    // ---- restart: w'_0 = r = b - A x (FP64), beta = ||r||
    {
      double v0 = 0.0;
      for (int i = lo + tid; i < hi; i += BS) {
        double ri;
        if (arnoldi) {
          ri = tk.b[i];
        } else {
          const double xc = ldcg(tk.x + i);
          ri = tk.b[i] - s2 * stencil<double, DIM>(tk.x, i, n, kappa, xc);
        }
        WP[i] = (T)ri;
        v0 += ri * ri;
      }
      for (int k = tid; k < LMAX; k += BS) {
        sm.h2v[k] = T(0);
        sm.cv[k] = T(0);
      }
      warp_slot<4>(sm.redd, 0, v0);
      block_finish<4, BS, double>(1, part(), lb, sm.redd, ps);
      ok = group_sync(w.bar, epoch, &sm.flag);
      if (!ok) goto abort;
      gather<BS, double, T>(part(), 1, nb, sm.tot, sm.coef, ps);
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
    if (tid == 0) {
      for (int k = 0; k <= MAXM; k++) sm.g[k] = 0.0;
      sm.g[0] = beta;
      sm.invT = (T)(1.0 / beta);
      sm.stop = 0;
    }
    __syncthreads();
    const double rtol_bnorm = kp.rtol * bnorm;
    double* hist = (lb == 0) ? tk.hist : nullptr;
    int kcols = 0;
    const int jmax = arnoldi ? kp.arnoldi_steps : m;
    XCarry<T> cy;  // shared-slice variant: values carried between its passes
    cy.pre = false;
    for (int j = 0;; j++) {
      // ---- X: v_j and z = A v_j, h1 = V^T z; warp 1 rotates column j-1
      // while thread 0 waits at the group barrier
      {
#define MLG_X(KK) x_pass<T, DIM, MAXM, BS, KK>(sm, lo, hi, j, n, WP, Z, Vg, rows, 0, kappa, s2t)
#define MLG_XS(KK) x_pass_sm<T, DIM, MAXM, BS, KK>(sm, lo, hi, j, n, WP, Z, Vs, rows, kappa, s2t, cy)
#define MLG_XB(KK)                                                                       \
  x_pass_bulk<T, DIM, MAXM, BS, KK>(sm, lo, hi, j, n, WP, Z, Vg, rows, kappa, s2t, pipe, bphase, \
                                    auxs)
        if constexpr (VM == kVShared) {
          MLG_BUCKETS(MLG_XS)
        } else if constexpr (VM == kVBulk) {
          MLG_BUCKETS(MLG_XB)
        } else {
          MLG_BUCKETS(MLG_X)
        }
#undef MLG_X
#undef MLG_XS
#undef MLG_XB
        if (arnoldi && j == jmax) { kcols = j; break; }
        auto givens_prev = [&]() {
          if (j > 0 && !arnoldi)
            givens_column<T, MAXM, BS>(sm, j - 1, rtol_bnorm, iters, kp.max_iters, m, hist,
                                       tk.hist_cap, bnorm);
        };
        // the Givens rotation of column j-1 (warp 1) overlaps the barrier and
        // the gather; its stop code is read after the gather
        finish_and_sync_side<LMAX, BS, T>(min(j + 2, LMAX), (T*)part(), lb, sm.red, ps, w.bar,
                                          epoch, &sm.flag, givens_prev);
        gather<BS, T, T, true>((const T*)part(), j + 2, nb, sm.tot, sm.coef, ps);
        if (!sm.flag) goto abort;
        const int stop = sm.stop;
        if (stop == 2) { status = kErrNonfinite; goto finish; }
        if (stop == 1) { kcols = j; break; }
        red++;
        if (tid <= j) sm.h1c[tid] = sm.coef[tid];
        if (tid == 0) sm.anorm2T = sm.coef[j + 1];
      }
      // ---- Y: w'_{j+1} = z - V h1, h2 = V^T w'_{j+1}, ||w'_{j+1}||^2
      {
#define MLG_Y(KK) y_pass<T, MAXM, BS, KK>(sm, lo, hi, j, WP, Z, Vg, rows, 0)
#define MLG_YS(KK) y_pass_sm<T, MAXM, BS, KK>(sm, lo, hi, j, WP, Z, Vs, rows, cy)
#define MLG_YB(KK) \
  y_pass_bulk<T, DIM, MAXM, BS, KK>(sm, lo, hi, j, WP, Z, Vg, rows, pipe, bphase, w.ldv)
        if constexpr (VM == kVShared) {
          MLG_BUCKETS(MLG_YS)
        } else if constexpr (VM == kVBulk) {
          MLG_BUCKETS(MLG_YB)
        } else {
          MLG_BUCKETS(MLG_Y)
        }
#undef MLG_Y
#undef MLG_YS
#undef MLG_YB
        ok = finish_and_sync<LMAX, BS, T>(j + 2, (T*)part(), lb, sm.red, ps, w.bar, epoch,
                                          &sm.flag, NoSide());
        if (!ok) goto abort;
        // w' is final everywhere: the next X pass's loads go out before the gather
        if constexpr (VM == kVShared) prefetch_x2d<T, BS>(cy, WP, lo, hi, n);
        gather<BS, T, T>((const T*)part(), j + 2, nb, sm.tot, sm.coef, ps);
        red++;
      }
      iters++;
      // ---- column j of Hu; hn_{j+1} = sqrt(||w'||^2 - ||h2||^2), in the working
      // precision (both terms come from reductions in that precision)
      if (tid <= j) {
        const T h2 = sm.coef[tid];
        sm.HuT[tid + j * LD] = sm.h1c[tid] + h2;  // correctly rounded sum
        sm.h2v[tid] = h2;
        sm.h2h[tid] = h2;
      }
      // hn_{j+1} from hn2T: 1/hn for the next X pass and the subdiagonal of Hu;
      // c_{j+1} = Hu(j+1,j) h2_j, the new vector's own coefficient
      auto set_norm = [&]() {
        const T h2v = sm.hn2T > T(0) ? sm.hn2T : T(0);
        const T hnT = sqrt(h2v);
        sm.invT = T(1) / hnT;
        sm.HuT[j + 1 + j * LD] = hnT;  // (the Givens warp reads it in FP64)
        sm.cv[j + 1] = hnT * sm.coef[j];
      };
      // the norm runs on the last warp while the c_i rows (below) leave it idle
      // (rows 4w .. 4w+3 per warp w: the last warp's rows exceed j for small j),
      // else on warp 0
      const int nwarp = j < 4 * (BS / 32 - 1) ? BS / 32 - 1 : 0;
      if ((tid >> 5) == nwarp) {
        T q = T(0);
        for (int k = lane; k <= j; k += 32) q += sm.coef[k] * sm.coef[k];
        q = warp_sum(q);
        if (lane == 0) {
          const T wn2 = sm.coef[j + 1];
          const T hn2 = wn2 - q;
          const bool fb = !(hn2 > T(0.5) * wn2);
          sm.fallback = fb;
          sm.hn2T = hn2;
          if (!fb) set_norm();
        }
      }
      // c_i = sum_{k >= i-1} Hu(i,k) h2_k (i <= j) for the next X pass, in the same
      // phase as the norm: columns k < j of Hu are unchanged since the last step,
      // column j is h1 + h2 and h2 is the gather's output (no read of what this
      // phase writes); eight lanes per row, each a strided part of the sum,
      // added in a fixed order
      for (int i0 = 0; i0 <= j && ((tid >> 5) != nwarp || nwarp == 0); i0 += BS / 8) {
        const int i = i0 + (tid >> 3);
        const int sub = tid & 7;
        const int ir = min(i, j);
        const int k0 = (ir > 0 ? ir - 1 : 0) + sub;
        T c = T(0);
        // all loads of a lane issued together (indices clamped into the column range)
#pragma unroll
        for (int t = 0; t < (MAXM + 7) / 8; t++) {
          const int k = k0 + 8 * t;
          const int kk = min(k, j);
          const T hik = kk == j ? sm.h1c[ir] + sm.coef[ir] : sm.HuT[ir + kk * LD];
          const T prod = hik * sm.coef[kk];
          if (i <= j && k <= j) c += prod;
        }
        c += __shfl_xor_sync(0xffffffffu, c, 4);
        c += __shfl_xor_sync(0xffffffffu, c, 2);
        c += __shfl_xor_sync(0xffffffffu, c, 1);
        if (sub == 0 && i <= j) sm.cv[i] = c;
      }
      __syncthreads();
      if (sm.fallback) {
        // cancellation: apply h2 explicitly and measure ||w''||
        T accN = T(0);
        for (int i = lo + tid; i < hi; i += BS) {
          T q = WP[i];
#pragma unroll
          for (int k = 0; k < MAXM; k++)
            if (k <= j) q -= sm.h2v[k] * V[vix(k, i - voff, rows)];
          WP[i] = q;
          accN += q * q;
        }
        warp_slot<LMAX>(sm.red, 0, accN);
        block_finish<LMAX, BS, T>(1, (T*)part(), lb, sm.red, ps);
        ok = group_sync(w.bar, epoch, &sm.flag);
        if (!ok) goto abort;
        gather<BS, T, T>((const T*)part(), 1, nb, sm.tot, sm.coef, ps);
        red++;
        if (tid == 0) {
          sm.hn2T = sm.coef[0];
          const T h2v = sm.hn2T > T(0) ? sm.hn2T : T(0);
          const T hnT = sqrt(h2v);
          sm.invT = T(1) / hnT;
          sm.HuT[j + 1 + j * LD] = hnT;
        }
        // w' now carries the second projection: no pending coefficients, and
        // A w' is the next X pass's stencil itself
        if (tid <= j + 1) {
          sm.h2v[tid] = T(0);
          sm.cv[tid] = T(0);
        }
        cy.pre = false;  // w' changed at this CTA's points
        __syncthreads();
      }
      if (arnoldi && tid == 0) {
        // column j is complete (the CTA barrier above ordered its entries)
        const double hnext = (double)sm.HuT[j + 1 + j * LD];
        if (hist)
          for (int k = 0; k <= j + 1; k++)
            hist[(long long)j * (jmax + 1) + k] =
                k <= j ? (double)sm.h1c[k] + (double)sm.h2h[k] : hnext;
        sm.stop = !(hnext * hnext > 1e-28 * (double)sm.anorm2T) ? 1 : 0;
        // read by every thread after the next X pass's group exchange
      }
      if (!arnoldi && j + 1 >= m) {
        // last column of the cycle: rotate it now (no further X pass)
        if (tid < 32)
          givens_column<T, MAXM, BS>(sm, j, rtol_bnorm, iters, kp.max_iters, m, hist,
                                     tk.hist_cap, bnorm);
        __syncthreads();
        if (sm.stop == 2) { status = kErrNonfinite; goto finish; }
        kcols = j + 1;
        break;
      }
    }
    if (arnoldi) {
      status = kcols;  // steps done; V_0..V_kcols written by the X passes
      break;
    }
    // ---- cycle end: y = R^{-1} g (upper triangular), x += V y.  The Givens
    // warp stored each column of R divided by its diagonal entry, so starting
    // from u = g the recurrence u_l -= (R(l,i) / R(i,i)) u_i (l < i, i
    // descending) leaves u_i = R(i,i) y_i: one FP64 FMA per column on the
    // dependent chain, with u_i broadcast by a shuffle (the divisions by the
    // diagonal are multiplications by 1/R(i,i), done at the end in parallel).
    if (threadIdx.x < 32) {
      constexpr int UR = (MAXM + 31) / 32;  // rows of u per lane
      double u[UR];
#pragma unroll
      for (int r = 0; r < UR; r++) u[r] = lane + 32 * r < kcols ? sm.g[lane + 32 * r] : 0.0;
#pragma unroll 4
      for (int i = kcols - 1; i > 0; i--) {
        double src = u[0];
#pragma unroll
        for (int r = 1; r < UR; r++)
          if ((i >> 5) == r) src = u[r];
        const double ui = __shfl_sync(0xffffffffu, src, i & 31);
#pragma unroll
        for (int r = 0; r < UR; r++) {
          const int l = lane + 32 * r;
          if (l < i) u[r] = fma(-(r_in_shared<MAXM>() ? sm.R : sm.Rg)[l + i * LD], ui, u[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < UR; r++) {
        const int l = lane + 32 * r;
        if (l < kcols) {
          const double yv = u[r] * sm.rinv[l];
          sm.y[l] = yv;
          if constexpr (sizeof(T) == 4) {
            // y_l as a sum of two floats (head + tail) for the double-float V y
            const float yh = (float)yv;
            sm.yf[l] = make_float2(yh, (float)(yv - (double)yh));
          }
        }
      }
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
      // V y in double-float arithmetic: with V in FP32 and y_k = yh_k + yl_k,
      // each product is split exactly by an FMA (TwoProduct) and accumulated
      // with TwoSum into a (head, tail) pair of floats, as in the Dot2
      // algorithm of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005):
      // about 2^-44 relative accuracy at FP32 instruction rates, where one
      // FP64 FMA and one conversion per basis vector and point run at this
      // GPU's FP64 rate (1/64 of FP32).  The sum is added to x in FP64.
      // Two points per trip and even / odd k apart: four independent pairs.
      for (int i0 = lo + tid; i0 < hi; i0 += 2 * BS) {
        const int i1 = i0 + BS;
        const bool two = i1 < hi;
        const long long vb0 = vbase(i0 - voff, rows);
        const long long vb1 = two ? vbase(i1 - voff, rows) : vb0;
        float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f, s2_ = 0.f, c2 = 0.f, s3 = 0.f, c3 = 0.f;
        int k = 0;
        for (; k + 1 < kcols; k += 2) {  // k even: vectors k, k+1 in one load
          const float2 ya = sm.yf[k], yb = sm.yf[k + 1];
          const float2 v0 = *reinterpret_cast<const float2*>(V + vb0 + vko(k));
          const float2 v1 = *reinterpret_cast<const float2*>(V + vb1 + vko(k));
          df_fma(s0, c0, ya, v0.x);
          df_fma(s1, c1, yb, v0.y);
          df_fma(s2_, c2, ya, v1.x);
          df_fma(s3, c3, yb, v1.y);
        }
        if (k < kcols) {
          const float2 ya = sm.yf[k];
          df_fma(s0, c0, ya, (float)V[vb0 + vko(k)]);
          df_fma(s2_, c2, ya, (float)V[vb1 + vko(k)]);
        }
        tk.x[i0] += df_value(s0, c0, s1, c1);
        if (two) tk.x[i1] += df_value(s2_, c2, s3, c3);
      }
    } else {
      // two points per trip and even / odd k apart: four independent FP64 chains
      // (a dependent FP64 operation costs ~70 cycles on this GPU)
      for (int i0 = lo + tid; i0 < hi; i0 += 2 * BS) {
        const int i1 = i0 + BS;
        const bool two = i1 < hi;
        const long long vb0 = vbase(i0 - voff, rows);
        const long long vb1 = two ? vbase(i1 - voff, rows) : vb0;
        double d0 = 0.0, e0 = 0.0, d1 = 0.0, e1 = 0.0;
        int k = 0;
        for (; k + 1 < kcols; k += 2) {
          const double ya = sm.y[k], yb = sm.y[k + 1];
          d0 = fma(ya, (double)V[vb0 + vko(k)], d0);
          e0 = fma(yb, (double)V[vb0 + vko(k + 1)], e0);
          d1 = fma(ya, (double)V[vb1 + vko(k)], d1);
          e1 = fma(yb, (double)V[vb1 + vko(k + 1)], e1);
        }
        if (k < kcols) {
          d0 = fma(sm.y[k], (double)V[vb0 + vko(k)], d0);
          d1 = fma(sm.y[k], (double)V[vb1 + vko(k)], d1);
        }
        tk.x[i0] += d0 + e0;
        if (two) tk.x[i1] += d1 + e1;
      }
    }
    cycles++;
    ok = group_sync(w.bar, epoch, &sm.flag);
    if (!ok) goto abort;
  }
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

template <typename T, int DIM, int MAXM, int BS, int VM, int MINB = 1>
__global__ void __launch_bounds__(BS, MINB) gmres_persistent(KParams kp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T, MAXM, BS>& sm = *reinterpret_cast<Smem<T, MAXM, BS>*>(smem_raw);
  int g = 0;
  while (g + 1 < kp.ngroups && (int)blockIdx.x >= kp.group_first[g + 1]) g++;
  const int lb = blockIdx.x - kp.group_first[g];
  const int nb = kp.group_first[g + 1] - kp.group_first[g];
  const GroupWork w = kp.work[g];
  unsigned long long epoch = 0;
  unsigned bphase = 0;  // parity of each bulk-copy stage of this thread's warp
  static_assert(r_in_shared<MAXM>() == (MINB == 1), "R placement follows the variant");
  if (!r_in_shared<MAXM>() && threadIdx.x == 0)
    sm.Rg = w.Rg + (size_t)blockIdx.x * r_doubles<MAXM>();
  if (VM == kVBulk) {
    for (int i = threadIdx.x; i < (BS / 32) * kMaxStages; i += BS)
      mbar_init(&sm.bbar[0][0] + i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
  }
  for (int t = kp.task_first[g]; t < kp.task_first[g + 1]; t++) {
    const SolveTask tk = kp.tasks[kp.task_order[t]];
    solve_one<T, DIM, MAXM, BS, VM>(kp, tk, w, lb, nb, epoch, bphase, sm);
    if (*(volatile int*)w.bar.err != kErrNone) break;
    // all CTAs finish with this task's data before the next task starts
    if (!group_sync(w.bar, epoch, &sm.flag)) break;
  }
}

// ------------------------------------------------------------- host side --
// The shared state lives in dynamic shared memory (about 90 KB for m <= 64),
// followed by the CTA's slice of V (VM = kVShared) or the warps' bulk-copy
// stages (VM = kVBulk).
template <typename T, int DIM, int MAXM, int BS, int VM, int MINB = 1>
cudaError_t prepare_t(int extra = 0) {
  return cudaFuncSetAttribute(gmres_persistent<T, DIM, MAXM, BS, VM, MINB>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_own_bytes<T, MAXM, BS>() + extra);
}

template <typename T, int DIM, int MAXM, int BS, int VM, int MINB = 1>
cudaError_t launch_t(const KParams& kp, int grid, cudaStream_t s) {
  if (kp.m > MAXM) return cudaErrorInvalidValue;
  int extra = 0;
  if (VM == kVShared) extra = kp.vsmem;
  if (VM == kVBulk) extra = (BS / 32) * kp.bulk_cap;
  cudaError_t e = prepare_t<T, DIM, MAXM, BS, VM, MINB>(extra);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&kp};
  note_launches(1);
  return cudaLaunchCooperativeKernel((const void*)gmres_persistent<T, DIM, MAXM, BS, VM, MINB>,
                                     dim3(grid), dim3(BS), args,
                                     smem_own_bytes<T, MAXM, BS>() + extra,
                                     s);
}

// Co-resident CTAs of the variant with `extra` bytes of dynamic shared memory
// beyond its own state.
template <typename T, int DIM, int MAXM, int BS, int VM, int MINB = 1>
int max_blocks_t(int* bs, int extra = 0) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (prepare_t<T, DIM, MAXM, BS, VM, MINB>(extra) != cudaSuccess) return 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gmres_persistent<T, DIM, MAXM, BS, VM, MINB>,
                                                BS,
                                                smem_own_bytes<T, MAXM, BS>() +
                                                    extra);
  *bs = BS;
  return per * nsm;
}

}  // namespace mlg
