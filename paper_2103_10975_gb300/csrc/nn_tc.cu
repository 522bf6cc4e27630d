// 32 -> 32 channel 3x3 convolutions of the 2D network on the fifth-generation
// tensor cores (tcgen05): the same implicit GEMM as conv32_mma
//   out[p][n] = sum_{tap,k} in[p + sign*dil*off(tap)][k] * Wop[tap][n][k],
// M = 128 pixels of one grid row per tile, N = 32 output channels,
// K = 9 taps x 32 input channels (18 MMAs of K = 16), accumulated in tensor
// memory (32 columns) by one thread's tcgen05.mma, completion signalled to an
// mbarrier by tcgen05.commit, and read back by every warp with tcgen05.ld
// (warp w owns TMEM lanes 32w..32w+31, i.e. pixels 32w..32w+31 of the tile).
// Operands sit in shared memory in the no-swizzle K-major layout (core
// matrices of 8 rows x 16 bytes).  The A operand is not materialised per tap:
// the three input rows a tile needs are staged once, each as 4 column blocks
// (8 channels each) of 132 pixel rows 16 bytes apart (so 8-row groups are 128
// bytes apart, the stride offset, and column blocks 2176 bytes apart, the
// leading-dimension offset); a tap's operand is then the same rows shifted by
// its x offset, i.e. a descriptor whose start address moves by 16 bytes per
// pixel.  The weights use 128 / 512-byte offsets.
// The rows arrive by TMA: a tensor map over the channels-last activation (4D:
// channels, x, y, batch) and one box of 8 channels x 132 pixels per column
// block, zero-filled outside the grid.  Each CTA runs a stream of tiles with
// specialised warps that meet only at mbarriers: a producer warp keeps three
// stages of rows in flight, an MMA warp turns each stage into one of two
// accumulators in tensor memory, and four epilogue warps read an accumulator,
// hand it back and store the tile while the next tiles' copies and MMAs run.
#include <cstdlib>
#include <mutex>
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "nn.h"

namespace mlg {

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kTcM = 128;                    // pixels per tile (TMEM lanes)
constexpr int kRows = kTcM + 4;              // staged pixels per input row (dilation <= 2)
constexpr int kBox = kRows * 16;             // one tensor copy: 8 channels x kRows pixels
constexpr int kLboA = 17 * 128;              // bytes between 8-channel column blocks (a copy
                                             // destination, 128-byte aligned, >= kBox)
constexpr int kRowBytes = 4 * kLboA;         // one staged input row
constexpr int kWBytes = kC * kC * 2;         // one tap's B operand: 2 KB
// per dimension: input rows per tile (3 in 2D; 3 x 3 in 3D), taps, stages in
// flight, bytes of a stage, bytes a stage's copies deliver, shared memory
template <int D>
struct TcGeo {
  static constexpr int kRowsPerTile = D == 3 ? 9 : 3;
  static constexpr int kTaps = D == 3 ? 27 : 9;
  static constexpr int kStages = D == 3 ? 2 : 3;
  static constexpr int kStageBytes = kRowsPerTile * kRowBytes;
  static constexpr int kStageTx = kRowsPerTile * 4 * kBox;
  static constexpr int kSmem = kStages * kStageBytes + kTaps * kWBytes + 128;
  static_assert(kStageBytes % 128 == 0, "stages must keep 128-byte alignment");
  static_assert(kSmem <= 227 * 1024, "shared memory of one CTA");
};
static_assert(kLboA >= kBox && kLboA % 128 == 0,
              "copy destinations must be 128-byte aligned and hold a box");

__device__ __forceinline__ unsigned saddr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor (no swizzle): start address, leading-
// dimension byte offset (between 8-element K blocks) and stride byte offset
// (between 8-row groups)
__device__ __forceinline__ unsigned long long mdesc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr >> 4) & 0x3FFFu) |
         ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor: D F32, A and B BF16, both K-major, N = 32, M = 128
constexpr unsigned kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) |
                            ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(unsigned tmem, unsigned long long a, unsigned long long b,
                                       unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ bool mbar_test_tc(unsigned bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(bar), "r"(phase) : "memory");
  return ok != 0;
}

enum { kRelu = 0, kResid = 1, kF32 = 2 };

// A tile's coordinates: batch b, plane z (3D), grid row y, first pixel x0 of its 128.
template <int D>
__device__ __forceinline__ void tile_coords(long long tIdx, int H, int tpr, int& b, int& z,
                                            int& y, int& x0) {
  const int tx = (int)(tIdx % tpr);
  const long long r = tIdx / tpr;
  y = (int)(r % H);
  if (D == 3) {
    z = (int)((r / H) % H);
    b = (int)(r / ((long long)H * H));
  } else {
    z = 0;
    b = (int)(r / H);
  }
  x0 = tx * kTcM;
}

// Bounded mbarrier wait (2 s); false on expiry.
__device__ __forceinline__ bool mbar_wait_tc(unsigned bar, unsigned phase) {
  if (mbar_test_tc(bar, phase)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_test_tc(bar, phase))
    if (globaltimer_ns() - t0 > 2000000000ull) return false;
  return true;
}

// The input rows of tile (b, z, y, x0) into stage buffer `as`: per row (3 in
// 2D: y - sd, y, y + sd; 9 in 3D: those of planes z - sd, z, z + sd, where sd
// = sign * dil) 4 tensor copies, each a box of 8 channels x kRows pixels
// starting at pixel x0 - dil; pixels, rows and planes outside the grid arrive
// as zeros.  The stage's mbarrier expects all their bytes.
template <int D>
__device__ __forceinline__ void issue_rows(const CUtensorMap* tmap, unsigned as, unsigned bar,
                                           int b, int z, int y, int x0, int dil, int sign) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(TcGeo<D>::kStageTx)
               : "memory");
  for (int r = 0; r < TcGeo<D>::kRowsPerTile; r++) {
    const int ty = r % 3, tz = r / 3;
    const int yy = y + sign * dil * (ty - 1);
    for (int kc = 0; kc < 4; kc++) {
      const unsigned dst = as + r * kRowBytes + kc * kLboA;
      if (D == 3) {
        const int zz = z + sign * dil * (tz - 1);
        asm volatile(
            "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
            "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(8 * kc), "r"(x0 - dil), "r"(yy),
            "r"(zz), "r"(b), "r"(bar)
            : "memory");
      } else {
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
            "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(8 * kc), "r"(x0 - dil), "r"(yy),
            "r"(b), "r"(bar)
            : "memory");
      }
    }
  }
}

// The 2 x taps MMAs of one tile (18 in 2D, 54 in 3D): A from stage buffer
// `as`, B the staged weights, D the accumulator at TMEM column offset `col`;
// tcgen05.commit then arrives on `bar` when they (and every earlier MMA of this
// thread) have completed.
template <int D>
__device__ __forceinline__ void issue_mmas(unsigned tmem, unsigned as, unsigned ws, int dil,
                                           int sign, unsigned bar) {
  for (int t = 0; t < TcGeo<D>::kTaps; t++) {
    // tap ((tz,) ty, tx): pixel p reads staged row t / 3 = (tz * 3 +) ty, pixel
    // p + dil + sign*dil*(tx-1)
    const int row0 = dil + sign * dil * (t % 3 - 1);
    for (int h = 0; h < 2; h++)
      tc_mma(tmem, mdesc(as + (t / 3) * kRowBytes + row0 * 16 + h * 2 * kLboA, kLboA, 128),
             mdesc(ws + t * kWBytes + h * 256, 128, 512), (t | h) ? 1u : 0u);
  }
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// Warp roles of conv32_tc (192 threads): warp 0 issues the TMA copies of the
// input rows, warp 1 issues the MMAs, warps 2..5 run the epilogue (warp w reads
// TMEM lanes 32 (w % 4) .. +31, the pixels of its quarter of the tile).
constexpr int kTcThreads = 192;

template <int D, int MODE>
__global__ void __launch_bounds__(kTcThreads) conv32_tc(const __grid_constant__ CUtensorMap tmap,
                                                        int B, int H, const bf16* __restrict__ wop,
                                                        const float* __restrict__ bias, int dil,
                                                        int sign, bf16* __restrict__ zo,
                                                        bf16* __restrict__ to,
                                                        const bf16* __restrict__ resid,
                                                        float* __restrict__ fo,
                                                        const float* __restrict__ addend,
                                                        int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  using G = TcGeo<D>;
  constexpr int kStages = G::kStages;
  constexpr int kStageBytes = G::kStageBytes;
  unsigned char* As = tc_smem;                                  // kStages stages of input rows
  unsigned char* Ws = tc_smem + kStages * kStageBytes;          // taps x 2 KB
  unsigned long long* full = reinterpret_cast<unsigned long long*>(Ws + G::kTaps * kWBytes);
  unsigned long long* empty = full + kStages;   // the MMAs of a stage have completed
  unsigned long long* tfull = empty + kStages;  // an accumulator holds a finished tile
  unsigned long long* tempty = tfull + 2;       // the epilogue has read an accumulator
  unsigned long long* drain = tempty + 2;       // the MMA warp's last MMAs (teardown)
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(drain + 1);
  int* prog = reinterpret_cast<int*>(tmem_slot + 1);  // [0] copies issued, [1] stages consumed
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // B operand (weights) of all taps: (n, k) at (n/8)*512 + (k/8)*128 + (n%8)*16 + (k%8)*2
  for (int idx = threadIdx.x; idx < G::kTaps * kC * 4; idx += blockDim.x) {
    const int kc = idx & 3, n = (idx >> 2) & 31, t = idx >> 7;
    const uint4 v = *reinterpret_cast<const uint4*>(wop + (t * kC + n) * kC + kc * 8);
    *reinterpret_cast<uint4*>(Ws + t * kWBytes + (n >> 3) * 512 + kc * 128 + (n & 7) * 16) = v;
  }
  // the weights were written through the generic proxy, the MMAs read through the async one
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(full + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(empty + i)) : "memory");
    }
    for (int i = 0; i < 2; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(tfull + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(saddr(tempty + i)) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(drain)) : "memory");
    prog[0] = prog[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
                     saddr(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;
  const unsigned as0 = saddr(As), ws = saddr(Ws);

  const int tpr = (H + kTcM - 1) / kTcM;
  const long long ntiles = (long long)B * H * tpr * (D == 3 ? H : 1);
  // this CTA's tiles: blockIdx.x + k * gridDim.x, k < K
  const long long K = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (warp == 0) {
    // ---- producer: rows of tile k into stage k % kStages once its MMAs are done
    if (lane == 0) {
      for (long long k = 0; k < K; k++) {
        const int st = (int)(k % kStages);
        const long long use = k / kStages;
        if (use > 0 && !mbar_wait_tc(saddr(empty + st), (unsigned)((use - 1) & 1))) {
          atomicExch(err, 1);
          break;
        }
        int b, z, y, x0;
        tile_coords<D>(blockIdx.x + k * gridDim.x, H, tpr, b, z, y, x0);
        issue_rows<D>(&tmap, as0 + (unsigned)st * kStageBytes, saddr(full + st), b, z, y, x0,
                      dil, sign);
        prog[0] = (int)(k + 1);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issue: tile k from stage k % kStages into accumulator k % 2
    if (lane == 0) {
      long long k = 0;
      for (; k < K; k++) {
        const int st = (int)(k % kStages), a = (int)(k & 1);
        if (!mbar_wait_tc(saddr(full + st), (unsigned)((k / kStages) & 1))) break;
        prog[1] = (int)(k + 1);
        if (k >= 2 && !mbar_wait_tc(saddr(tempty + a), (unsigned)(((k >> 1) - 1) & 1))) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        issue_mmas<D>(tmem + 32u * a, as0 + (unsigned)st * kStageBytes, ws, dil, sign,
                      saddr(empty + st));
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                saddr(tfull + a))
            : "memory");
      }
      if (k < K) atomicExch(err, 1);
      // every MMA issued has completed before the teardown frees tensor memory
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              saddr(drain))
          : "memory");
      mbar_wait_tc(saddr(drain), 0u);
    }
  } else {
    // ---- epilogue: accumulator k % 2 to the outputs of tile k
    const int lq = warp & 3;  // TMEM lane quarter of this warp
    float bv[kC];
#pragma unroll
    for (int o = 0; o < kC; o++) bv[o] = (MODE != kF32 && bias) ? bias[o] : 0.f;
    for (long long k = 0; k < K; k++) {
      const int ab = (int)(k & 1);
      // a warp-uniform decision: tcgen05.ld below needs the whole warp
      const bool okw = __all_sync(0xffffffffu, mbar_wait_tc(saddr(tfull + ab),
                                                             (unsigned)((k >> 1) & 1)));
      if (!okw) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned r[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
          "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
            "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
            "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
            "=r"(r[31])
          : "r"(tmem + ((unsigned)(lq * 32) << 16) + (unsigned)(32 * ab)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      // the accumulator may take the next tile's MMAs while this warp stores
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(tempty + ab))
                     : "memory");
      int b, z, y, x0;
      tile_coords<D>(blockIdx.x + k * gridDim.x, H, tpr, b, z, y, x0);
      const int p = lq * 32 + lane;
      const int x = x0 + p;
      if (x < H) {
        const long long pix = D == 3 ? (((long long)b * H + z) * H + y) * H + x
                                     : ((long long)b * H + y) * H + x;
        float v[kC];
#pragma unroll
        for (int o = 0; o < kC; o++) v[o] = __uint_as_float(r[o]) + bv[o];
        if (MODE == kF32) {
          float4* dst = reinterpret_cast<float4*>(fo + pix * kC);
          const float4* add = addend ? reinterpret_cast<const float4*>(addend + pix * kC) : nullptr;
#pragma unroll
          for (int q = 0; q < 8; q++) {
            float4 w = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            if (add) {
              const float4 a = add[q];
              w.x += a.x; w.y += a.y; w.z += a.z; w.w += a.w;
            }
            dst[q] = w;
          }
        } else {
#pragma unroll
          for (int o = 0; o < kC; o++) v[o] = fmaxf(v[o], 0.f);
          uint4* zd = reinterpret_cast<uint4*>(zo + pix * kC);
          const uint4* rs = MODE == kResid ? reinterpret_cast<const uint4*>(resid + pix * kC)
                                           : nullptr;
          uint4* td = MODE == kResid ? reinterpret_cast<uint4*>(to + pix * kC) : nullptr;
#pragma unroll
          for (int q = 0; q < 4; q++) {
            uint4 pz, pt;
            __nv_bfloat162* hz = reinterpret_cast<__nv_bfloat162*>(&pz);
            __nv_bfloat162* ht = reinterpret_cast<__nv_bfloat162*>(&pt);
            uint4 rv = make_uint4(0u, 0u, 0u, 0u);
            if (MODE == kResid) rv = rs[q];
            const __nv_bfloat162* hr = reinterpret_cast<const __nv_bfloat162*>(&rv);
#pragma unroll
            for (int e = 0; e < 4; e++) {
              const float a0 = v[8 * q + 2 * e], a1 = v[8 * q + 2 * e + 1];
              hz[e] = __floats2bfloat162_rn(a0, a1);
              if (MODE == kResid) {
                const float2 sr = __bfloat1622float2(hr[e]);
                ht[e] = __floats2bfloat162_rn(sr.x + a0, sr.y + a1);
              }
            }
            zd[q] = pz;
            if (MODE == kResid) td[q] = pt;
          }
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // copies still in flight (only after a wait ran out) land before the CTA
    // leaves (bounded waits)
    for (int k = prog[1]; k < prog[0]; k++)
      mbar_wait_tc(saddr(full + k % kStages), (unsigned)((k / kStages) & 1));
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
  }
}

// ---------------------------------------------- weight gradient (tcgen05) --
// part[cta][(tap*32 + k)*32 + o] = sum_p in[p + dil*off(tap)][k] g[p][o], and
// the bias partials sum_p g[p][o] at T*1024 + o (T = 9 taps in 2D, 27 in 3D;
// a 3D launch covers the nine taps of one plane offset tz, taps 9 tz + 3 ty +
// tx, and the tz = 0 launch writes the bias partials).  The pixels are the
// reduction dimension: per x offset tx of a tap, D_tx[m][o] += A[m][q] B[q][o]
// over the 128 pixels q of each tile, M = 128 rows m = ty*32 + k (the three
// taps (ty, tx) times the 32 input channels, and in rows 96..127 a row of
// ones, which makes D_tx[96][o] the sum of g), N = 32 output channels, one
// accumulator in tensor memory per tx, kept over all of the CTA's tiles.
// Both operands are MN-major in the no-swizzle layout (core matrices of 8 K
// rows x 16 bytes of M or N): the staged rows are [8-channel block][pixel][8]
// with blocks kLboA bytes apart (the stride offset, between 8-row M or N
// groups) and 8-pixel groups 128 bytes apart (the leading offset, along K).
// Staged rows follow each other 4 blocks apart, so the taps ty = 0, 1, 2 of
// one tx and the row of ones are M groups 0-3, 4-7, 8-11, 12-15 of a single
// operand, and the tap's x offset moves its start address by 16 bytes per
// pixel.  Warp roles as in conv32_tc: a producer warp (TMA), an MMA warp, four
// epilogue warps that read the accumulators once, at the end.
constexpr int kWgRows = 5;  // per stage: input rows y - dil, y, y + dil, ones, g's row
constexpr int kWgStageBytes = kWgRows * kRowBytes;
constexpr int kWgStages = 2;
constexpr int kWgSmem = kWgStages * kWgStageBytes + 128;
constexpr int kWgTx = 16 * kBox;  // 3 input rows and g's row, 4 boxes each
// D F32, A and B BF16 and MN-major, N = 32, M = 128
constexpr unsigned kIdescWg = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                              ((32u >> 3) << 17) | ((128u >> 4) << 24);
static_assert(kWgStageBytes % 128 == 0, "stages must keep 128-byte alignment");

__device__ __forceinline__ void tc_mma_wg(unsigned tmem, unsigned long long a,
                                          unsigned long long b, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdescWg), "r"(acc)
      : "memory");
}

// One box of a row: (channel c, pixel x, row y, plane z (3D), batch b).
template <int D>
__device__ __forceinline__ void tma_row(const CUtensorMap* tmap, unsigned dst, int c, int x,
                                        int y, int z, int b, unsigned bar) {
  if (D == 3)
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(c), "r"(x), "r"(y), "r"(z), "r"(b),
        "r"(bar)
        : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(c), "r"(x), "r"(y), "r"(b), "r"(bar)
        : "memory");
}

template <int D>
__global__ void __launch_bounds__(kTcThreads) wgrad_tc(const __grid_constant__ CUtensorMap tin,
                                                       const __grid_constant__ CUtensorMap tg,
                                                       int B, int H, int dil, int tz,
                                                       float* __restrict__ part, int stride,
                                                       int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char wg_smem[];
  unsigned long long* full = reinterpret_cast<unsigned long long*>(wg_smem + kWgStages * kWgStageBytes);
  unsigned long long* empty = full + kWgStages;  // the MMAs of a stage have completed
  unsigned long long* done = empty + kWgStages;  // every MMA of the CTA has completed
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(done + 1);
  int* prog = reinterpret_cast<int*>(tmem_slot + 1);  // [0] stages issued, [1] consumed
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the row of ones of each stage (BF16 1.0), written once; the copies never touch it
  for (int st = 0; st < kWgStages; st++) {
    unsigned* ones = reinterpret_cast<unsigned*>(wg_smem + st * kWgStageBytes + 3 * kRowBytes);
    for (int i = threadIdx.x; i < kRowBytes / 4; i += blockDim.x) ones[i] = 0x3F803F80u;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int i = 0; i < kWgStages; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(full + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(empty + i)) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(done)) : "memory");
    prog[0] = prog[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
                     saddr(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;
  const unsigned as0 = saddr(wg_smem);
  const int tpr = (H + kTcM - 1) / kTcM;
  const long long ntiles = (long long)B * H * tpr * (D == 3 ? H : 1);
  const long long K = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (warp == 0) {
    // ---- producer: the rows of tile k into stage k % kWgStages once its MMAs are done
    if (lane == 0) {
      for (long long k = 0; k < K; k++) {
        const int st = (int)(k % kWgStages);
        const long long use = k / kWgStages;
        if (use > 0 && !mbar_wait_tc(saddr(empty + st), (unsigned)((use - 1) & 1))) {
          atomicExch(err, 1);
          break;
        }
        int b, z, y, x0;
        tile_coords<D>(blockIdx.x + k * gridDim.x, H, tpr, b, z, y, x0);
        const unsigned as = as0 + (unsigned)st * kWgStageBytes;
        const unsigned bar = saddr(full + st);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(kWgTx)
                     : "memory");
        // (3D: the input rows of plane z + dil (tz - 1), zeros outside the grid)
        for (int ty = 0; ty < 3; ty++)
          for (int kc = 0; kc < 4; kc++)
            tma_row<D>(&tin, as + ty * kRowBytes + kc * kLboA, 8 * kc, x0 - dil,
                       y + dil * (ty - 1), z + dil * (tz - 1), b, bar);
        for (int kc = 0; kc < 4; kc++)
          tma_row<D>(&tg, as + 4 * kRowBytes + kc * kLboA, 8 * kc, x0, y, z, b, bar);
        prog[0] = (int)(k + 1);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issue: 8 K-steps of 16 pixels x 3 taps x per tile, into accumulator tx
    if (lane == 0) {
      long long k = 0;
      for (; k < K; k++) {
        const int st = (int)(k % kWgStages);
        if (!mbar_wait_tc(saddr(full + st), (unsigned)((k / kWgStages) & 1))) break;
        prog[1] = (int)(k + 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned as = as0 + (unsigned)st * kWgStageBytes;
        for (int ks = 0; ks < kTcM / 16; ks++) {
          const unsigned q = (unsigned)ks * 16u * 16u;  // the K-step's first pixel, in bytes
          const unsigned long long bdesc = mdesc(as + 4 * kRowBytes + q, 128, kLboA);
          for (int tx = 0; tx < 3; tx++)
            tc_mma_wg(tmem + 32u * tx, mdesc(as + (unsigned)(dil * tx) * 16u + q, 128, kLboA),
                      bdesc, (k | ks) ? 1u : 0u);
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                saddr(empty + st))
            : "memory");
      }
      if (k < K) atomicExch(err, 1);
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              saddr(done))
          : "memory");
    }
  } else {
    // ---- epilogue: the three accumulators (and the bias sums) into the partial
    const int lq = warp & 3;  // TMEM lane quarter: rows 32 lq .. 32 lq + 31
    constexpr int T = D == 3 ? 27 : 9;
    float* dst = part + (long long)blockIdx.x * stride;
    float* dw = dst + (D == 3 ? (long long)tz * 9 * kC * kC : 0);
    const bool okw = __all_sync(0xffffffffu, mbar_wait_tc(saddr(done), 0u));
    if (!okw) {
      if (lane == 0) atomicExch(err, 1);
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int tx = 0; tx < 3; tx++) {
        unsigned r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
              "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
              "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
              "=r"(r[31])
            : "r"(tmem + ((unsigned)(lq * 32) << 16) + 32u * tx));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // (a CTA without tiles wrote no accumulator: its partial is zero)
        float v[kC];
#pragma unroll
        for (int o = 0; o < kC; o++) v[o] = K > 0 ? __uint_as_float(r[o]) : 0.f;
        if (lq < 3) {
          const int tap = lq * 3 + tx, kin = lane;
          float4* d4 = reinterpret_cast<float4*>(dw + (long long)(tap * kC + kin) * kC);
#pragma unroll
          for (int q4 = 0; q4 < 8; q4++)
            d4[q4] = make_float4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
        } else if (tx == 0 && lane == 0 && (D == 2 || tz == 0)) {
#pragma unroll
          for (int o = 0; o < kC; o++) dst[T * kC * kC + o] = v[o];
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // copies still in flight (only after a wait ran out) land before the CTA
    // leaves, and every MMA issued has completed (bounded waits)
    for (int k = prog[1]; k < prog[0]; k++)
      mbar_wait_tc(saddr(full + k % kWgStages), (unsigned)((k / kWgStages) & 1));
    mbar_wait_tc(saddr(done), 0u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
  }
}

int* g_tc_err = nullptr;  // set by a tile whose MMAs did not complete in time

// Rows of at least this many points go to the tcgen05 kernel (128, a full
// tile; the environment variable MLGMRES_TC_MIN_ROW lowers it, so that tests
// run the kernel on small grids, whose rows fill part of a tile).
int tc_min_row() {
  const char* e = getenv("MLGMRES_TC_MIN_ROW");
  if (e && *e) {
    const int v = atoi(e);
    if (v >= 1) return v;
  }
  return kTcM;
}

}  // namespace

bool conv32_tc_applies(int dim, int H) { return (dim == 2 || dim == 3) && H >= tc_min_row(); }

namespace {

// cuTensorMapEncodeTiled, looked up through the runtime (the library does not
// link the driver library itself)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;

template <int D>
void set_tc_smem() {
  cudaFuncSetAttribute(conv32_tc<D, kRelu>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       TcGeo<D>::kSmem);
  cudaFuncSetAttribute(conv32_tc<D, kResid>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       TcGeo<D>::kSmem);
  cudaFuncSetAttribute(conv32_tc<D, kF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       TcGeo<D>::kSmem);
}

template <int D>
void launch_tc(int mode, int grid, cudaStream_t s, const CUtensorMap& tm, int B, int H,
               const bf16* wop, const float* bias, int dil, int sign, bf16* zo, bf16* to,
               const bf16* resid, float* fo, const float* addend) {
  constexpr int sm = TcGeo<D>::kSmem;
  if (mode == kRelu)
    conv32_tc<D, kRelu><<<grid, kTcThreads, sm, s>>>(tm, B, H, wop, bias, dil, sign, zo, to,
                                                     resid, fo, addend, g_tc_err);
  else if (mode == kResid)
    conv32_tc<D, kResid><<<grid, kTcThreads, sm, s>>>(tm, B, H, wop, bias, dil, sign, zo, to,
                                                      resid, fo, addend, g_tc_err);
  else
    conv32_tc<D, kF32><<<grid, kTcThreads, sm, s>>>(tm, B, H, wop, bias, dil, sign, zo, to,
                                                    resid, fo, addend, g_tc_err);
}

}  // namespace

cudaError_t conv32_tc_setup() {
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (g_tc_err) return cudaSuccess;
  set_tc_smem<2>();
  set_tc_smem<3>();
  cudaFuncSetAttribute(wgrad_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
  cudaFuncSetAttribute(wgrad_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  int* flag = nullptr;
  e = cudaMalloc(&flag, sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemset(flag, 0, sizeof(int));
  if (e != cudaSuccess) return e;
  g_tc_err = flag;
  return cudaSuccess;
}

cudaError_t launch_conv32_tc(int dim, int mode, int B, int H, const __nv_bfloat16* in,
                             const __nv_bfloat16* wop, const float* bias, int dil, int sign,
                             __nv_bfloat16* zo, __nv_bfloat16* to, const __nv_bfloat16* resid,
                             float* fo, const float* addend, cudaStream_t s) {
  if (!g_tc_err) {
    const cudaError_t e = conv32_tc_setup();
    if (e != cudaSuccess) return e;
  }
  if ((dim != 2 && dim != 3) || dil < 1 || dil > 2 || ((unsigned long long)in & 15ull))
    return cudaErrorInvalidValue;
  // the input activation, channels last: [B]([H])[H][H][32] BF16, as a tensor of
  // rank dim + 2 (channels innermost); a copy box is 8 channels x kRows pixels of
  // one row
  CUtensorMap tm;
  const cuuint64_t row = (cuuint64_t)kC * 2;  // bytes per pixel
  const cuuint64_t h = (cuuint64_t)H;
  const cuuint64_t dims[5] = {(cuuint64_t)kC, h, h, dim == 3 ? h : (cuuint64_t)B, (cuuint64_t)B};
  const cuuint64_t strides[4] = {row, row * h, row * h * h, row * h * h * h};
  const cuuint32_t box[5] = {8, (cuuint32_t)kRows, 1, 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (g_encode(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)(dim + 2), (void*)in, dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
      CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long ntiles = (long long)B * H * ((H + kTcM - 1) / kTcM);
  if (dim == 3) ntiles *= H;
  // CTAs that fit an SM (shared memory: two in 2D, one in 3D); each runs a
  // stream of tiles
  const long long per_sm = dim == 3 ? 1 : 2;
  const int grid = (int)(ntiles < per_sm * nsm ? ntiles : per_sm * nsm);
  if (dim == 3)
    launch_tc<3>(mode, grid, s, tm, B, H, wop, bias, dil, sign, zo, to, resid, fo, addend);
  else
    launch_tc<2>(mode, grid, s, tm, B, H, wop, bias, dil, sign, zo, to, resid, fo, addend);
  note_launches(1);
  return cudaGetLastError();
}

// A tensor map over a channels-last activation, [B][H][H][32] (2D) or
// [B][H][H][H][32] (3D), BF16: boxes of 8 channels x kRows pixels of one row.
static bool encode_rows(CUtensorMap* tm, const __nv_bfloat16* p, int dim, int B, int H) {
  const cuuint64_t row = (cuuint64_t)kC * 2;
  const cuuint64_t h = (cuuint64_t)H;
  const cuuint64_t dims[5] = {(cuuint64_t)kC, h, h, dim == 3 ? h : (cuuint64_t)B, (cuuint64_t)B};
  const cuuint64_t strides[4] = {row, row * h, row * h * h, row * h * h * h};
  const cuuint32_t box[5] = {8, (cuuint32_t)kRows, 1, 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)(dim + 2), (void*)p, dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

cudaError_t launch_wgrad_tc(int dim, int B, int H, const __nv_bfloat16* in,
                            const __nv_bfloat16* g, int dil, float* part, int stride, int nparts,
                            cudaStream_t s) {
  if (!g_tc_err) {
    const cudaError_t e = conv32_tc_setup();
    if (e != cudaSuccess) return e;
  }
  const int T = dim == 3 ? 27 : 9;
  if ((dim != 2 && dim != 3) || dil < 1 || dil > 2 || nparts < 1 ||
      stride < T * kC * kC + kC || ((unsigned long long)in & 15ull) ||
      ((unsigned long long)g & 15ull) || ((unsigned long long)part & 15ull) || (stride & 3))
    return cudaErrorInvalidValue;
  CUtensorMap tin, tg;
  if (!encode_rows(&tin, in, dim, B, H) || !encode_rows(&tg, g, dim, B, H))
    return cudaErrorInvalidValue;
  // every one of the nparts CTAs writes its partial (zeros without tiles); in 3D
  // one launch per plane offset tz of the taps
  if (dim == 2) {
    wgrad_tc<2><<<nparts, kTcThreads, kWgSmem, s>>>(tin, tg, B, H, dil, 1, part, stride,
                                                     g_tc_err);
    note_launches(1);
  } else {
    for (int tz = 0; tz < 3; tz++)
      wgrad_tc<3><<<nparts, kTcThreads, kWgSmem, s>>>(tin, tg, B, H, dil, tz, part, stride,
                                                       g_tc_err);
    note_launches(3);
  }
  return cudaGetLastError();
}

int conv32_tc_error() {
  int v = 0;
  if (g_tc_err) cudaMemcpy(&v, g_tc_err, sizeof(int), cudaMemcpyDeviceToHost);
  return v;
}

}  // namespace mlg
