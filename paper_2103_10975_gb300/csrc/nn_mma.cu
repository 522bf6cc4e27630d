// Tensor-core (mma.sync m16n8k16, BF16 operands, FP32 accumulation) kernels
// for the 32 -> 32 channel 3x3 (2D) and 3x3x3 (3D) convolutions of the
// initial-guess network, as implicit GEMMs over channels-last activations:
//   conv32_mma : out[p][n] = sum_{tap,k} in[p + sign*dil*off(tap)][k] * Wop[tap][n][k]
//                (forward: Wop = transposed-tap copy; data gradient: sign = -1
//                with the other copy), M = pixels, N = 32, K = T * 32 (T = 9 or 27)
//   wgrad_mma  : part[cta][(tap*32 + k)*32 + o] = sum_p in[p + dil*off(tap)][k] g[p][o]
//                M = 32 output channels, N = 288 (the 9 taps of one kz plane x input
//                channel; 3D runs it once per plane), K = pixels
// A CTA owns 64 consecutive pixels of one grid row at a time; the 3 (2D) or 9
// (3D) input rows it needs (with a dil-wide halo, zero outside the grid) are
// staged in shared memory with an 80-byte pixel stride, which keeps ldmatrix
// conflict-free.
#include <mutex>
#include <cuda_bf16.h>

#include "common.cuh"
#include "nn.h"

namespace mlg {

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kTileP = 64;          // pixels per tile
constexpr int kPix = 40;            // bf16 per staged pixel (32 + 8 pad)
constexpr int kMaxDil = 2;
constexpr int kTileW = kTileP + 2 * kMaxDil;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Stage the input rows a tile of row (b, z, y), columns x0 .. x0+63, reads:
// rows y + s*dil*(ty-1) (and planes z + s*dil*(tz-1) in 3D), columns
// x0 - dil .. x0 + 63 + dil, into tile[r][c][kPix], r = tz*3 + ty (zero
// outside the grid).  zoff selects one plane offset only (wgrad, 3D).
template <int D>
__device__ __forceinline__ void stage_rows(bf16* tile, const bf16* __restrict__ in, int b, int n,
                                           int z, int y, int x0, int dil, int s, int nplanes,
                                           int zoff) {
  const int cols = kTileP + 2 * dil;
  const int rows = 3 * nplanes;
  for (int idx = threadIdx.x; idx < rows * cols * 4; idx += blockDim.x) {
    const int q = idx & 3;
    const int c = (idx >> 2) % cols;
    const int r = (idx >> 2) / cols;
    const int ty = r % 3, tz = r / 3;
    const int yy = y + s * dil * (ty - 1);
    const int zz = D == 3 ? z + s * dil * ((nplanes == 3 ? tz : zoff) - 1) : 0;
    const int xx = x0 - dil + c;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (yy >= 0 && yy < n && xx >= 0 && xx < n && (D == 2 || (zz >= 0 && zz < n))) {
      const long long pix = D == 3 ? (((long long)b * n + zz) * n + yy) * n + xx
                                   : ((long long)b * n + yy) * n + xx;
      v = *reinterpret_cast<const uint4*>(in + pix * kC + q * 8);
    }
    *reinterpret_cast<uint4*>(tile + (r * kTileW + c) * kPix + q * 8) = v;
  }
}

// row index (b, z, y) of a grid with rows = B n^(D-1)
template <int D>
__device__ __forceinline__ void decode_row(long long row, int n, int& b, int& z, int& y) {
  // row indices stay below 2^31 (the network's size check): 32-bit division
  const unsigned un = (unsigned)n, r = (unsigned)row;
  y = (int)(r % un);
  const unsigned r2 = r / un;
  z = D == 3 ? (int)(r2 % un) : 0;
  b = D == 3 ? (int)(r2 / un) : (int)r2;
}

enum { kRelu = 0, kResid = 1, kF32 = 2 };

template <int D>
constexpr int conv_smem_bytes() {
  return (int)sizeof(bf16) * ((D == 3 ? 27 : 9) * kC * kPix + (D == 3 ? 9 : 3) * kTileW * kPix);
}

template <int MODE, int D>
__global__ void __launch_bounds__(128) conv32_mma(int B, int H, const bf16* __restrict__ in,
                                                  const bf16* __restrict__ wop,
                                                  const float* __restrict__ bias, int dil,
                                                  int sign, bf16* __restrict__ zo,
                                                  bf16* __restrict__ to,
                                                  const bf16* __restrict__ resid,
                                                  float* __restrict__ fo,
                                                  const float* __restrict__ addend) {
  constexpr int T = D == 3 ? 27 : 9;
  extern __shared__ __align__(16) unsigned char nn_smem[];
  bf16* ws = reinterpret_cast<bf16*>(nn_smem);   // [tap][n][k]
  bf16* tile = ws + T * kC * kPix;               // [r][c][k]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int idx = threadIdx.x; idx < T * kC * 4; idx += blockDim.x) {
    const int q = idx & 3, row = idx >> 2;  // row = tap*32 + n
    *reinterpret_cast<uint4*>(ws + row * kPix + q * 8) =
        *reinterpret_cast<const uint4*>(wop + row * kC + q * 8);
  }
  float bv[4][2];
#pragma unroll
  for (int nt = 0; nt < 4; nt++) {
    const int o = nt * 8 + 2 * (lane & 3);
    bv[nt][0] = (MODE != kF32 && bias) ? bias[o] : 0.f;
    bv[nt][1] = (MODE != kF32 && bias) ? bias[o + 1] : 0.f;
  }
  const int tpr = (H + kTileP - 1) / kTileP;  // tiles per row
  long long nrows = (long long)B * H;
  if (D == 3) nrows *= H;
  const long long ntiles = nrows * tpr;
  for (long long tIdx = blockIdx.x; tIdx < ntiles; tIdx += gridDim.x) {
    const int tx = (int)(tIdx % tpr);
    int b, z, y;
    decode_row<D>(tIdx / tpr, H, b, z, y);
    const int x0 = tx * kTileP;
    __syncthreads();  // previous tile's readers are done (and ws is staged)
    stage_rows<D>(tile, in, b, H, z, y, x0, dil, sign, D == 3 ? 3 : 1, 1);
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; nt++)
#pragma unroll
      for (int e = 0; e < 4; e++) acc[nt][e] = 0.f;
    // A row address of this lane (ldmatrix x4: matrix q = lane/8, row lane%8)
    const int arow = warp * 16 + ((lane >> 3) & 1) * 8 + (lane & 7);
    const int acol = (lane >> 4) * 8;
#pragma unroll 9
    for (int t = 0; t < T; t++) {
      const int r = t / 3, txx = t % 3;  // r = tz*3 + ty
      const int c = arow + dil + sign * dil * (txx - 1);
      const bf16* abase = tile + (r * kTileW + c) * kPix + acol;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        unsigned a[4];
        ldsm_x4(a, abase + h * 16);
        unsigned bb[2][4];
#pragma unroll
        for (int pr = 0; pr < 2; pr++) {
          // n-tiles 2pr, 2pr+1: matrix q -> n = (2pr + q/2)*8 + lane%8, k = (q%2)*8 + 16h
          const int n = (2 * pr + (lane >> 4)) * 8 + (lane & 7);
          const int k = ((lane >> 3) & 1) * 8 + 16 * h;
          ldsm_x4(bb[pr], ws + (t * kC + n) * kPix + k);
        }
        mma16816(acc[0], a, bb[0][0], bb[0][1]);
        mma16816(acc[1], a, bb[0][2], bb[0][3]);
        mma16816(acc[2], a, bb[1][0], bb[1][1]);
        mma16816(acc[3], a, bb[1][2], bb[1][3]);
      }
    }
    // epilogue: rows lane/4 and lane/4 + 8 of this warp's 16 pixels
#pragma unroll
    for (int half = 0; half < 2; half++) {
      const int p = warp * 16 + (lane >> 2) + half * 8;
      const int x = x0 + p;
      if (x >= H) continue;
      const long long pix = D == 3 ? (((long long)b * H + z) * H + y) * H + x
                                   : ((long long)b * H + y) * H + x;
#pragma unroll
      for (int nt = 0; nt < 4; nt++) {
        const int o = nt * 8 + 2 * (lane & 3);
        float v0 = acc[nt][half * 2 + 0] + bv[nt][0];
        float v1 = acc[nt][half * 2 + 1] + bv[nt][1];
        if (MODE == kRelu) {
          *reinterpret_cast<__nv_bfloat162*>(zo + pix * kC + o) =
              __floats2bfloat162_rn(fmaxf(v0, 0.f), fmaxf(v1, 0.f));
        } else if (MODE == kResid) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
          *reinterpret_cast<__nv_bfloat162*>(zo + pix * kC + o) = __floats2bfloat162_rn(v0, v1);
          const float2 sv = __bfloat1622float2(
              *reinterpret_cast<const __nv_bfloat162*>(resid + pix * kC + o));
          *reinterpret_cast<__nv_bfloat162*>(to + pix * kC + o) =
              __floats2bfloat162_rn(sv.x + v0, sv.y + v1);
        } else {
          if (addend) {
            const float2 ad = *reinterpret_cast<const float2*>(addend + pix * kC + o);
            v0 += ad.x;
            v1 += ad.y;
          }
          *reinterpret_cast<float2*>(fo + pix * kC + o) = make_float2(v0, v1);
        }
      }
    }
  }
}

// Weight gradient: every CTA accumulates, over its tiles, the 32 x 288 product
// g^T * im2col(in) of the 9 taps of plane tz (3D; all 9 taps in 2D) in
// registers (warp w owns n-tiles 9w .. 9w+8 of the 36) and the bias sums, then
// writes them as its partial (layout (tap*32 + k)*32 + o, tap = tz*9 + local
// tap in 3D; bias at T*1024 + o, written by the tz = 0 launch).
template <int D>
__global__ void __launch_bounds__(128) wgrad_mma(int B, int H, const bf16* __restrict__ in,
                                                 const bf16* __restrict__ g, int dil, int tz,
                                                 float* __restrict__ part, int stride) {
  constexpr int T = D == 3 ? 27 : 9;
  __shared__ __align__(16) bf16 tile[3 * kTileW * kPix];
  __shared__ __align__(16) bf16 gt[kTileP * kPix];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float acc[2][9][4];
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int j = 0; j < 9; j++)
#pragma unroll
      for (int e = 0; e < 4; e++) acc[mt][j][e] = 0.f;
  float bsum = 0.f;  // thread t < 32: bias sum of channel t
  const int tpr = (H + kTileP - 1) / kTileP;
  long long nrows = (long long)B * H;
  if (D == 3) nrows *= H;
  const long long ntiles = nrows * tpr;
  for (long long tIdx = blockIdx.x; tIdx < ntiles; tIdx += gridDim.x) {
    const int tx = (int)(tIdx % tpr);
    int b, z, y;
    decode_row<D>(tIdx / tpr, H, b, z, y);
    const int x0 = tx * kTileP;
    __syncthreads();
    stage_rows<D>(tile, in, b, H, z, y, x0, dil, 1, 1, tz);
    for (int idx = threadIdx.x; idx < kTileP * 4; idx += blockDim.x) {
      const int q = idx & 3, p = idx >> 2;
      const int x = x0 + p;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (x < H) {
        const long long pix = D == 3 ? (((long long)b * H + z) * H + y) * H + x
                                     : ((long long)b * H + y) * H + x;
        v = *reinterpret_cast<const uint4*>(g + pix * kC + q * 8);
      }
      *reinterpret_cast<uint4*>(gt + p * kPix + q * 8) = v;
    }
    __syncthreads();
    if (threadIdx.x < kC) {
      for (int p = 0; p < kTileP; p++) bsum += __bfloat162float(gt[p * kPix + threadIdx.x]);
    }
#pragma unroll
    for (int ks = 0; ks < kTileP / 16; ks++) {  // 16 pixels per step
      // A = g^T (o x p): transposed 8x8 tiles from gt rows p
      unsigned a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; mt++) {
        // matrices: q0 (o 0-7, p 0-7), q1 (o 8-15, p 0-7), q2 (o 0-7, p 8-15), q3 (o 8-15, p 8-15)
        const int q = lane >> 3;
        const int p = ks * 16 + (q >> 1) * 8 + (lane & 7);
        const int o = mt * 16 + (q & 1) * 8;
        ldsm_x4_t(a[mt], gt + p * kPix + o);
      }
#pragma unroll
      for (int jp = 0; jp < 9; jp += 2) {
        // n-tiles nt = 9*warp + jp (+1): n = tap*32 + k, tap = nt/4, k block = nt%4
        unsigned bb[4];
        const int q = lane >> 3;
        const int ntq = 9 * warp + jp + (q >> 1);
        const int ntc = ntq < 36 ? ntq : 35;
        const int tap = ntc >> 2, kb = ntc & 3;
        const int ty = tap / 3, txx = tap % 3;
        const int p = ks * 16 + (q & 1) * 8 + (lane & 7);
        const int c = p + dil + dil * (txx - 1);
        ldsm_x4_t(bb, tile + (ty * kTileW + c) * kPix + kb * 8);
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
          mma16816(acc[mt][jp], a[mt], bb[0], bb[1]);
          if (jp + 1 < 9) mma16816(acc[mt][jp + 1], a[mt], bb[2], bb[3]);
        }
      }
    }
  }
  // write the partial: c0,c1 -> (o = row, n = col, col+1), c2,c3 -> o + 8
  float* dst = part + (long long)blockIdx.x * stride;
  float* dw = dst + (D == 3 ? (long long)tz * 9 * kC * kC : 0);
#pragma unroll
  for (int mt = 0; mt < 2; mt++) {
#pragma unroll
    for (int j = 0; j < 9; j++) {
      const int nt = 9 * warp + j;
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int o = mt * 16 + (lane >> 2) + (e >> 1) * 8;
        const int n = nt * 8 + 2 * (lane & 3) + (e & 1);
        dw[(long long)n * kC + o] = acc[mt][j][e];
      }
    }
  }
  if (threadIdx.x < kC && (D == 2 || tz == 0)) dst[T * kC * kC + threadIdx.x] = bsum;
}

}  // namespace

template <int D>
static cudaError_t conv_launch(int mode, int B, int H, const __nv_bfloat16* in,
                               const __nv_bfloat16* wop, const float* bias, int dil, int sign,
                               __nv_bfloat16* zo, __nv_bfloat16* to, const __nv_bfloat16* resid,
                               float* fo, const float* addend, cudaStream_t s) {
  constexpr int smem = conv_smem_bytes<D>();
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long ntiles = (long long)B * H * ((H + kTileP - 1) / kTileP);
  if (D == 3) ntiles *= H;
  const int grid = (int)(ntiles < 8LL * nsm ? ntiles : 8LL * nsm);
  if (mode == kRelu)
    conv32_mma<kRelu, D><<<grid, 128, smem, s>>>(B, H, in, wop, bias, dil, sign, zo, to, resid,
                                                  fo, addend);
  else if (mode == kResid)
    conv32_mma<kResid, D><<<grid, 128, smem, s>>>(B, H, in, wop, bias, dil, sign, zo, to, resid,
                                                   fo, addend);
  else
    conv32_mma<kF32, D><<<grid, 128, smem, s>>>(B, H, in, wop, bias, dil, sign, zo, to, resid,
                                                 fo, addend);
  note_launches(1);
  return cudaGetLastError();
}

// The 3D variants need more than the default 48 KB of dynamic shared memory;
// net_create calls this once, before any launch (and before a graph capture).
cudaError_t conv32_mma_setup() {
  static std::mutex mu;
  static bool done = false;
  std::lock_guard<std::mutex> lk(mu);
  if (done) return cudaSuccess;
  constexpr int s2 = conv_smem_bytes<2>(), s3 = conv_smem_bytes<3>();
  cudaError_t e = cudaSuccess;
  for (const void* f : {(const void*)conv32_mma<kRelu, 2>, (const void*)conv32_mma<kResid, 2>,
                        (const void*)conv32_mma<kF32, 2>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, s2);
  for (const void* f : {(const void*)conv32_mma<kRelu, 3>, (const void*)conv32_mma<kResid, 3>,
                        (const void*)conv32_mma<kF32, 3>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, s3);
  done = e == cudaSuccess;
  return e;
}

cudaError_t launch_conv32_mma(int dim, int mode, int B, int H, const __nv_bfloat16* in,
                              const __nv_bfloat16* wop, const float* bias, int dil, int sign,
                              __nv_bfloat16* zo, __nv_bfloat16* to, const __nv_bfloat16* resid,
                              float* fo, const float* addend, cudaStream_t s) {
  if (dil < 1 || dil > kMaxDil || (dim != 2 && dim != 3)) return cudaErrorInvalidValue;
  // full-resolution levels go to the tcgen05 kernel (tensor memory accumulators)
  if (conv32_tc_applies(dim, H))
    return launch_conv32_tc(dim, mode, B, H, in, wop, bias, dil, sign, zo, to, resid, fo, addend,
                            s);
  return dim == 3 ? conv_launch<3>(mode, B, H, in, wop, bias, dil, sign, zo, to, resid, fo,
                                   addend, s)
                  : conv_launch<2>(mode, B, H, in, wop, bias, dil, sign, zo, to, resid, fo,
                                   addend, s);
}

cudaError_t launch_wgrad_mma(int dim, int B, int H, const __nv_bfloat16* in,
                             const __nv_bfloat16* g, int dil, float* part, int stride, int nparts,
                             cudaStream_t s) {
  if (dil < 1 || dil > kMaxDil || (dim != 2 && dim != 3)) return cudaErrorInvalidValue;
  if (conv32_tc_applies(dim, H))
    return launch_wgrad_tc(dim, B, H, in, g, dil, part, stride, nparts, s);
  if (dim == 2) {
    wgrad_mma<2><<<nparts, 128, 0, s>>>(B, H, in, g, dil, 1, part, stride);
    note_launches(1);
  } else {
    for (int tz = 0; tz < 3; tz++) wgrad_mma<3><<<nparts, 128, 0, s>>>(B, H, in, g, dil, tz, part, stride);
    note_launches(3);
  }
  return cudaGetLastError();
}

}  // namespace mlg
