// Device-side building blocks shared by the solver kernels: warp / block
// reductions, L2-coherent loads, and the bounded grid barrier.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mlg {

// Host-side count of kernels this library has launched (all handles); the
// launch sites call note_launches() right after each launch.
void note_launches(long long k);
long long launches_so_far();

constexpr int kErrNone = 0;
constexpr int kErrTimeout = -4;
constexpr int kErrNonfinite = -5;
constexpr int kErrConfig = -6;  // launch parameters inconsistent with a task (reported as ERR_CUDA)

// Loads of data that another CTA wrote before a grid barrier go through L2
// (ld.global.cg) so a stale L1 line can never be read.
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier over a group of `nblocks` co-resident CTAs sharing the monotonically
// increasing counter *ctr (zeroed before the launch).  Every wait is bounded:
// after timeout_ns the waiting CTA raises *err = kErrTimeout and every CTA
// leaves its wait as soon as it sees a raised *err.  Returns false when the
// group must abandon the solve.  `epoch` is the caller's count of barriers
// passed (only thread 0's copy is used).
struct GroupBarrier {
  unsigned long long* ctr;
  int* err;
  unsigned nblocks;
  unsigned long long timeout_ns;
};

// Thread 0's half of the group barrier: arrive (release) and wait (acquire,
// bounded); returns 0 on a timeout or a raised error flag.
__device__ __forceinline__ int group_arrive_wait(const GroupBarrier& gb, unsigned long long& epoch) {
  epoch += 1;
  const unsigned long long target = epoch * (unsigned long long)gb.nblocks;
  red_release_add_u64(gb.ctr, 1ull);
  int ok = 1;
  if (ld_acquire_u64(gb.ctr) < target) {
    const unsigned long long t0 = globaltimer_ns();
    unsigned it = 0;
    while (ld_acquire_u64(gb.ctr) < target) {
      // the error flag and the clock every eighth poll: a poll is one load
      if ((++it & 7u) != 0) continue;
      if (*(volatile int*)gb.err != kErrNone) { ok = 0; break; }
      if (globaltimer_ns() - t0 > gb.timeout_ns) {
        atomicCAS(gb.err, kErrNone, kErrTimeout);
        ok = 0;
        break;
      }
    }
  }
  if (ok && *(volatile int*)gb.err != kErrNone) ok = 0;
  return ok;
}

// side() runs on warp 1 while thread 0 waits at the barrier (work that would
// otherwise sit on the critical path between two barriers).
template <typename Side>
__device__ __forceinline__ bool group_sync_with(const GroupBarrier& gb,
                                                unsigned long long& epoch, int* s_flag,
                                                Side side) {
  __syncthreads();
  if ((threadIdx.x >> 5) == 1) side();
  if (gb.nblocks == 1) {  // a one-CTA group only needs the CTA barrier
    if (threadIdx.x == 0) *s_flag = (*(volatile int*)gb.err == kErrNone);
    __syncthreads();
    return *s_flag != 0;
  }
  if (threadIdx.x == 0) {
    // the CTA's writes are ordered before this release by the CTA barrier
    // above; the acquire loads order the other CTAs' writes before the CTA
    // barrier that ends the wait (release/acquire at gpu scope, cumulative
    // through bar.sync), so no separate fences are needed
    *s_flag = group_arrive_wait(gb, epoch);
  }
  __syncthreads();
  return *s_flag != 0;
}

struct NoSide {
  __device__ void operator()() const {}
};

__device__ __forceinline__ bool group_sync(const GroupBarrier& gb, unsigned long long& epoch,
                                           int* s_flag) {
  return group_sync_with(gb, epoch, s_flag, NoSide());
}

}  // namespace mlg
