// Initial-guess network N(b): forward, backward and Adam on the GPU.
// Architecture and parameter order are documented in nn.h; activations are
// NHWC with 32 channels in BF16, accumulation in FP32.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "nn.h"

namespace mlg {

namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void load32(const bf16* p, float* v) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int i = 0; i < 4; i++) {
    uint4 u = q[i];
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int j = 0; j < 4; j++) {
      float2 f = __bfloat1622float2(h[j]);
      v[i * 8 + 2 * j] = f.x;
      v[i * 8 + 2 * j + 1] = f.y;
    }
  }
}

__device__ __forceinline__ void store32(bf16* p, const float* v) {
  uint4* q = reinterpret_cast<uint4*>(p);
#pragma unroll
  for (int i = 0; i < 4; i++) {
    uint4 u;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int j = 0; j < 4; j++) h[j] = __floats2bfloat162_rn(v[i * 8 + 2 * j], v[i * 8 + 2 * j + 1]);
    q[i] = u;
  }
}

// --------------------------------------------------------------- geometry --
// Grid points of a cubic grid of side n: p = ((b n + z) n + y) n + x in 3D,
// (b n + y) n + x in 2D.  Tap t of a 3^D stencil: kz = t / 9 (3D), ky = (t / 3) % 3,
// kx = t % 3, offsets k - 1 (times the dilation).
template <int D>
struct Geo {
  static constexpr int T = D == 3 ? 27 : 9;
  // Point indices stay below 2^31 (net_create checks 32 B_max n^D), so the
  // arithmetic is 32-bit: a 64-bit division is a long software sequence.
  __device__ static void decode(long long p, int n, int& b, int& z, int& y, int& x) {
    const unsigned un = (unsigned)n;
    unsigned r = (unsigned)p;
    x = (int)(r % un);
    r /= un;
    y = (int)(r % un);
    r /= un;
    if (D == 3) {
      z = (int)(r % un);
      r /= un;
    } else {
      z = 0;
    }
    b = (int)r;
  }
  // index of (b, z + dz, y + dy, x + dx), or -1 outside the grid
  __device__ static long long nb(int b, int z, int y, int x, int dz, int dy, int dx, int n) {
    const int zz = z + dz, yy = y + dy, xx = x + dx;
    if (yy < 0 || yy >= n || xx < 0 || xx >= n) return -1;
    if (D == 3 && (zz < 0 || zz >= n)) return -1;
    return D == 3 ? (long long)(((b * n + zz) * n + yy) * n + xx) : (long long)((b * n + yy) * n + xx);
  }
  __device__ static void tap(int t, int& dz, int& dy, int& dx) {
    dz = D == 3 ? t / 9 - 1 : 0;
    dy = (t / 3) % 3 - 1;
    dx = t % 3 - 1;
  }
  __host__ __device__ static long long pts(int n) {
    return D == 3 ? (long long)n * n * n : (long long)n * n;
  }
};

// ---------------------------------------------------------------- forward --

// a0[p][c] = relu(b[c] + sum_tap w[c][tap] u[p + off_tap])
template <int D>
__global__ void conv_in_fwd(int B, int n, const float* __restrict__ u,
                            const float* __restrict__ w, const float* __restrict__ bias,
                            bf16* __restrict__ a0) {
  constexpr int T = Geo<D>::T;
  __shared__ float ws[kC * T + kC];
  for (int i = threadIdx.x; i < kC * T; i += blockDim.x) ws[i] = w[i];
  for (int i = threadIdx.x; i < kC; i += blockDim.x) ws[kC * T + i] = bias[i];
  __syncthreads();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= B * Geo<D>::pts(n)) return;
  int b, z, y, x;
  Geo<D>::decode(p, n, b, z, y, x);
  float tp[T];
#pragma unroll
  for (int t = 0; t < T; t++) {
    int dz, dy, dx;
    Geo<D>::tap(t, dz, dy, dx);
    const long long q = Geo<D>::nb(b, z, y, x, dz, dy, dx, n);
    tp[t] = q >= 0 ? u[q] : 0.f;
  }
  float v[kC];
#pragma unroll
  for (int c = 0; c < kC; c++) {
    float acc = ws[kC * T + c];
#pragma unroll
    for (int t = 0; t < T; t++) acc += ws[c * T + t] * tp[t];
    v[c] = fmaxf(acc, 0.f);
  }
  store32(a0 + p * kC, v);
}

// out = mean of each 2^D block of in (side s -> s/2), channels last
template <int D>
__global__ void pool2_fwd(int B, int s, const bf16* __restrict__ in, bf16* __restrict__ out) {
  const int so = s / 2;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= B * Geo<D>::pts(so) * kC) return;
  const int c = (int)(i % kC);
  int b, z, y, x;
  Geo<D>::decode(i / kC, so, b, z, y, x);
  float v = 0.f;
#pragma unroll
  for (int k = 0; k < (1 << D); k++) {
    const long long q = Geo<D>::nb(b, 2 * z, 2 * y, 2 * x, (k >> 2) & 1, (k >> 1) & 1, k & 1, s);
    v += __bfloat162float(in[q * kC + c]);
  }
  out[i] = __float2bfloat16(v * (1.f / (1 << D)));
}

// Half-pixel linear source position of output index i (m source points, n out).
__device__ __forceinline__ void bilin(int i, int m, int n, int& i0, int& i1, float& lam) {
  float src = ((float)i + 0.5f) * (float)m / (float)n - 0.5f;
  if (src < 0.f) src = 0.f;
  i0 = (int)floorf(src);
  if (i0 > m - 1) i0 = m - 1;
  i1 = min(i0 + 1, m - 1);
  lam = src - (float)i0;
}

struct Levels {
  const bf16* z[kMaxLevels];
  int side[kMaxLevels];
  int L;
};

// s[p][c] = sum_l upsample(z_l)[p][c]  (bilinear in 2D, trilinear in 3D);
// four threads per point, eight channels (16 bytes) each, so the
// interpolation weights are computed once per 8 channels
template <int D>
__global__ void upsum_fwd(int B, int n, Levels lv, bf16* __restrict__ s) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= B * Geo<D>::pts(n) * 4) return;
  const int cg = (int)(i & 3);
  const long long p = i >> 2;
  int b, z, y, x;
  Geo<D>::decode(p, n, b, z, y, x);
  float acc[8];
  {
    const uint4 v = *reinterpret_cast<const uint4*>(lv.z[0] + p * kC + cg * 8);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const float2 f = __bfloat1622float2(h[q]);
      acc[2 * q] = f.x;
      acc[2 * q + 1] = f.y;
    }
  }
  for (int l = 1; l < lv.L; l++) {
    const int m = lv.side[l];
    int z0 = 0, z1 = 0, y0, y1, x0, x1;
    float lz = 0.f, ly, lx;
    if (D == 3) bilin(z, m, n, z0, z1, lz);
    bilin(y, m, n, y0, y1, ly);
    bilin(x, m, n, x0, x1, lx);
#pragma unroll
    for (int k = 0; k < (1 << D); k++) {
      const int zz = (k >> 2) & 1 ? z1 : z0, yy = (k >> 1) & 1 ? y1 : y0, xx = k & 1 ? x1 : x0;
      const float wz = D == 3 ? ((k >> 2) & 1 ? lz : 1.f - lz) : 1.f;
      const float w = wz * ((k >> 1) & 1 ? ly : 1.f - ly) * (k & 1 ? lx : 1.f - lx);
      const long long q = Geo<D>::nb(b, zz, yy, xx, 0, 0, 0, m);
      const uint4 v = *reinterpret_cast<const uint4*>(lv.z[l] + q * kC + cg * 8);
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
      for (int qq = 0; qq < 4; qq++) {
        const float2 f = __bfloat1622float2(h[qq]);
        acc[2 * qq] += w * f.x;
        acc[2 * qq + 1] += w * f.y;
      }
    }
  }
  uint4 o;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
  for (int q = 0; q < 4; q++) h[q] = __floats2bfloat162_rn(acc[2 * q], acc[2 * q + 1]);
  *reinterpret_cast<uint4*>(s + p * kC + cg * 8) = o;
}

// y[p] = b + sum_tap sum_c w[c][tap] t[p + off_tap][c]
template <int D>
__global__ void conv_out_fwd(int B, int n, const bf16* __restrict__ t,
                             const float* __restrict__ w, const float* __restrict__ bias,
                             float* __restrict__ y) {
  constexpr int T = Geo<D>::T;
  __shared__ float ws[kC * T];
  for (int i = threadIdx.x; i < kC * T; i += blockDim.x) ws[i] = w[i];
  __syncthreads();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= B * Geo<D>::pts(n)) return;
  int b, z, yy0, xx0;
  Geo<D>::decode(p, n, b, z, yy0, xx0);
  float acc = bias[0];
  for (int tp = 0; tp < T; tp++) {
    int dz, dy, dx;
    Geo<D>::tap(tp, dz, dy, dx);
    const long long q = Geo<D>::nb(b, z, yy0, xx0, dz, dy, dx, n);
    if (q < 0) continue;
    float v[kC];
    load32(t + q * kC, v);
#pragma unroll
    for (int c = 0; c < kC; c++) acc += ws[c * T + tp] * v[c];
  }
  y[p] = acc;
}

// --------------------------------------------------------------- backward --

// gy = 2 (y - ts t) / (B N); per-CTA partial sums of (y - ts t)^2 (ts from
// tsp when given: the target scale of a training phase, in device memory)
__global__ void mse_grad(long long total, float scale, float ts, const float* __restrict__ tsp,
                         const float* __restrict__ y, const float* __restrict__ t,
                         float* __restrict__ gy, float* __restrict__ part) {
  __shared__ float red[32];
  if (tsp) ts = *tsp;
  float acc = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - ts * t[i];
    gy[i] = 2.f * d * scale;
    acc += d * d;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    acc = warp_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
  }
}

__global__ void loss_finish(const float* __restrict__ part, int nparts, float scale,
                            float* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nparts; i++) s += part[i];
    *loss = (float)(s * scale);
  }
}

// g_t[p][c] = sum_tap w[c][tap] gy[p - off_tap]
// Segments of the 1-channel <-> 32-channel kernels: R rows x W points of one
// (b, z) plane (W = min(n, 256), R = max(1, 256 / n)), with the 1-channel field
// of the segment and its one-point halo staged in shared memory, zero outside
// the grid, so each tap is one shared-memory read at a fixed offset.
constexpr int kSeg = 256;
constexpr int kW1Threads = 512;

template <int D>
__host__ __device__ constexpr int w1_planes() { return D == 3 ? 3 : 1; }

__host__ __device__ inline int w1_w(int n) { return n < kSeg ? n : kSeg; }
__host__ __device__ inline int w1_r(int n) { return n < kSeg ? kSeg / n : 1; }

template <int D>
int w1_stage_floats(int n) { return w1_planes<D>() * (w1_r(n) + 2) * (w1_w(n) + 2); }

// sf[pz][r][cx] = f at (plane pl + pz - 1 (3D), row y0 + r - 1, column x0 + cx - 1)
template <int D, int NT>
__device__ __forceinline__ void w1_stage(float* sf, const float* __restrict__ f, int n, int pl,
                                         int y0, int x0, int W, int R) {
  const int TW = W + 2, TP = (R + 2) * TW;
  for (int i = threadIdx.x; i < w1_planes<D>() * TP; i += NT) {
    const int pz = D == 3 ? i / TP : 1, r = (i % TP) / TW, cx = (i % TP) % TW;
    const int gy = y0 + r - 1, gx = x0 + cx - 1;
    bool ok = gy >= 0 && gy < n && gx >= 0 && gx < n;
    int gpl = pl;
    if (D == 3) {
      const int gz = pl % n + pz - 1;
      ok = ok && gz >= 0 && gz < n;
      gpl = pl + pz - 1;
    }
    sf[i] = ok ? f[((long long)gpl * n + gy) * n + gx] : 0.f;
  }
}

// gt[p][c] = sum_tap w[c][tap] gy[p - off_tap] (transpose of the 32 -> 1 output
// conv) and, when gbf is given, gbf[p][c] = bf16(mask[p][c] > 0 ? gt : 0) for
// the masked consumer that follows.  Segments as above (gy staged); lane =
// channel (coalesced 128-byte rows), each warp U points of the segment.
template <int D>
__global__ void __launch_bounds__(kW1Threads) conv_out_bwd_data(int B, int n,
                                                               const float* __restrict__ gy,
                                                               const float* __restrict__ w,
                                                               float* __restrict__ gt,
                                                               const bf16* __restrict__ mask,
                                                               bf16* __restrict__ gbf) {
  constexpr int T = Geo<D>::T;
  constexpr int NW = kW1Threads / 32;
  constexpr int U = kSeg / NW;
  extern __shared__ float sf[];
  const int W = w1_w(n), R = w1_r(n);
  const int TW = W + 2, TP = (R + 2) * TW;
  const int xsegs = (n + W - 1) / W, ysegs = (n + R - 1) / R;
  const int nseg = B * (D == 3 ? n : 1) * ysegs * xsegs;
  const int c = threadIdx.x & 31, wp = threadIdx.x >> 5;
  float wc[T];
#pragma unroll
  for (int tp = 0; tp < T; tp++) wc[tp] = w[c * T + tp];
  const int ry0 = (wp * U) / W, xl0 = (wp * U) % W;
  const int center = D == 3 ? TP : 0;
  for (int sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    const int xs = sg % xsegs, t2 = sg / xsegs;
    const int ys = t2 % ysegs, pl = t2 / ysegs;
    const int x0 = xs * W, y0 = ys * R;
    __syncthreads();
    w1_stage<D, kW1Threads>(sf, gy, n, pl, y0, x0, W, R);
    __syncthreads();
    int ry = ry0, xl = xl0;
#pragma unroll 4
    for (int k = 0; k < U; k++) {
      const int y = y0 + ry, x = x0 + xl;
      if (ry < R && y < n && x < n) {
        const int base = center + (ry + 1) * TW + xl + 1;
        float acc = 0.f;
#pragma unroll
        for (int tp = 0; tp < T; tp++) {
          int dz, dy, dx;
          Geo<D>::tap(tp, dz, dy, dx);
          acc += wc[tp] * sf[base - (dz * TP + dy * TW + dx)];
        }
        const long long p = ((long long)pl * n + y) * n + x;
        gt[p * kC + c] = acc;
        if (gbf)
          gbf[p * kC + c] = __float2bfloat16(__bfloat162float(mask[p * kC + c]) > 0.f ? acc : 0.f);
      }
      if (++xl == W) {
        xl = 0;
        ++ry;
      }
    }
  }
}

// Per-CTA partial weight gradients of a 1-channel <-> 32-channel 3^D conv:
//   part[cta][c*T + tap] and the biases at part[cta][32 T + c].
// MODE 0 (output conv):  dW[c][tap] = sum_p gy[p] t[p + off][c]
//                                   = sum_q t[q][c] gy[q - off],  db = sum_q gy[q]
// MODE 1 (input conv):   dW[c][tap] = sum_p g32[p][c] u[p + off], db[c] = sum_p g32[p][c],
//                        with g32 taken as 0 where m32 <= 0 (the ReLU of a0)
// The grid is cut into segments of R rows x W points of one (b, z) plane
// (W = min(n, 256), R = max(1, 256 / n)).  Lane = channel: every 32-channel row
// is read once, coalesced, U rows per warp in flight; the 1-channel field (gy
// or u) of the segment and its halo is staged in shared memory, zero outside
// the grid, so each tap is one shared-memory read at a fixed offset.  The 16
// warp sums are added in a fixed order.
template <int D>
int conv1_wgrad_smem(int n) {
  constexpr int T = Geo<D>::T;
  const int stage = w1_stage_floats<D>(n);
  const int red = (kW1Threads / 32) * 32 * (T + 1);
  return (int)sizeof(float) * (stage > red ? stage : red);
}

template <int MODE, int D>
__global__ void __launch_bounds__(kW1Threads, D == 3 ? 1 : 2) conv1_wgrad(
    int B, int n, const float* __restrict__ g1, const bf16* __restrict__ x32,
    const float* __restrict__ g32, const bf16* __restrict__ m32, const float* __restrict__ u,
    float* __restrict__ part, int stride) {
  constexpr int T = Geo<D>::T;
  constexpr int NW = kW1Threads / 32;
  constexpr int U = kSeg / NW;             // points per warp and segment
  constexpr int sgn = MODE == 0 ? -1 : 1;  // MODE 0 reads gy at q - off, MODE 1 u at p + off
  extern __shared__ float sf[];
  const int W = w1_w(n), R = w1_r(n);
  const int TW = W + 2, TP = (R + 2) * TW;
  const int xsegs = (n + W - 1) / W, ysegs = (n + R - 1) / R;
  const int nplanes = B * (D == 3 ? n : 1);  // (b, z) planes
  const int nseg = nplanes * ysegs * xsegs;
  const int c = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float* __restrict__ f = MODE == 0 ? g1 : u;
  float acc[T];
#pragma unroll
  for (int t = 0; t < T; t++) acc[t] = 0.f;
  float accb = 0.f;
  for (int sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    const int xs = sg % xsegs, t2 = sg / xsegs;
    const int ys = t2 % ysegs, pl = t2 / ysegs;  // pl = b (2D) or b n + z (3D)
    const int x0 = xs * W, y0 = ys * R;
    // this warp's rows first (their loads overlap the staging below)
    // (the warp's U points run along x from (ry0, xl0), wrapping to the next row)
    const int ry0 = (w * U) / W, xl0 = (w * U) % W;
    float val[U];
    {
      int ry = ry0, xl = xl0;
#pragma unroll
      for (int k = 0; k < U; k++) {
        const int x = x0 + xl, y = y0 + ry;
        float v = 0.f;
        if (ry < R && y < n && x < n) {
          const long long p = ((long long)pl * n + y) * n + x;
          if (MODE == 0)
            v = __bfloat162float(x32[p * kC + c]);
          else
            v = __bfloat162float(m32[p * kC + c]) > 0.f ? g32[p * kC + c] : 0.f;
        }
        val[k] = v;
        if (++xl == W) {
          xl = 0;
          ++ry;
        }
      }
    }
    __syncthreads();  // the previous segment's readers are done with sf
    w1_stage<D, kW1Threads>(sf, f, n, pl, y0, x0, W, R);
    __syncthreads();
    const int center = D == 3 ? TP : 0;
    int ry = ry0, xl = xl0;
#pragma unroll
    for (int k = 0; k < U; k++) {
      if (ry < R && y0 + ry < n && x0 + xl < n) {
        const int base = center + (ry + 1) * TW + xl + 1;
#pragma unroll
        for (int t = 0; t < T; t++) {
          int dz, dy, dx;
          Geo<D>::tap(t, dz, dy, dx);
          acc[t] += val[k] * sf[base + sgn * (dz * TP + dy * TW + dx)];
        }
        accb += MODE == 0 ? sf[base] : val[k];
      }
      if (++xl == W) {
        xl = 0;
        ++ry;
      }
    }
  }
  // fixed-order sum of the 16 warps' partials
  __syncthreads();
  float* red = sf;  // [NW][32 (T + 1)]
#pragma unroll
  for (int t = 0; t < T; t++) red[w * 32 * (T + 1) + c * (T + 1) + t] = acc[t];
  red[w * 32 * (T + 1) + c * (T + 1) + T] = accb;
  __syncthreads();
  for (int t = threadIdx.x; t < kC * T + kC; t += kW1Threads) {
    // t < 32 T: weight c*T + tap; t >= 32 T: bias of channel t - 32 T (MODE 0: one bias)
    const int cc = t < kC * T ? t / T : t - kC * T;
    const int k = t < kC * T ? t % T : T;
    float v = 0.f;
    if (!(MODE == 0 && k == T && cc != 0))
      for (int ww = 0; ww < NW; ww++) v += red[ww * 32 * (T + 1) + cc * (T + 1) + k];
    part[(long long)blockIdx.x * stride + t] = v;
  }
}

// out = bf16(g * (mask > 0)), eight elements per thread (count is a multiple
// of 32: whole channel rows; the buffers are 32-byte aligned)
__global__ void mask_to_bf16(long long count, const float* __restrict__ g,
                             const bf16* __restrict__ mask, bf16* __restrict__ out) {
  const long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * 8;
  if (i >= count) return;
  const float4 a = *reinterpret_cast<const float4*>(g + i);
  const float4 b = *reinterpret_cast<const float4*>(g + i + 4);
  const uint4 mv = *reinterpret_cast<const uint4*>(mask + i);
  const bf16* m = reinterpret_cast<const bf16*>(&mv);
  const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  uint4 o;
  bf16* ob = reinterpret_cast<bf16*>(&o);
#pragma unroll
  for (int k = 0; k < 8; k++) ob[k] = __float2bfloat16(__bfloat162float(m[k]) > 0.f ? v[k] : 0.f);
  *reinterpret_cast<uint4*>(out + i) = o;
}

// grad[dst_w[i]] = sum over CTAs of part[cta][i] for the weight layout used by
// the partial kernels; the mapping to the parameter layout [o][k][tap] is done
// here so the parameters keep the documented order (T taps).
//   kind 0 (32->32): part index (tap*32 + k)*32 + o  -> param (o*32 + k)*T + tap; bias 1024 T + o
//   kind 1/2 (1-ch): part index c*T + tap (+ 32 T + c bias) -> same order
__global__ void __launch_bounds__(256) reduce_wgrad(const float* __restrict__ part, int nparts,
                                                    int stride, int kind, int T,
                                                    float* __restrict__ gw,
                                                    float* __restrict__ gb) {
  // 32 outputs per CTA (lane = output), the CTA partials split over the 8 warps
  // (coalesced rows), four independent sums per lane so that four loads are in
  // flight, all added in a fixed order (FP32: the FP64 pipe of this GPU is slow)
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const int nw = kind == 0 ? T * kC * kC : T * kC;
  const int nb = kind == 0 ? kC : (kind == 1 ? kC : 1);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  if (i < nw + nb) {
    int c = w;
    for (; c + 24 < nparts; c += 32) {
      s0 += part[(long long)c * stride + i];
      s1 += part[(long long)(c + 8) * stride + i];
      s2 += part[(long long)(c + 16) * stride + i];
      s3 += part[(long long)(c + 24) * stride + i];
    }
    for (; c < nparts; c += 8) s0 += part[(long long)c * stride + i];
  }
  red[w][lane] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  if (w != 0 || i >= nw + nb) return;
  float t = 0.f;
#pragma unroll
  for (int k = 0; k < 8; k++) t += red[k][lane];
  if (i < nw) {
    if (kind == 0) {
      const int tp = i / (kC * kC), k = (i / kC) % kC, o = i % kC;
      gw[(o * kC + k) * T + tp] = (float)t;
    } else {
      gw[i] = (float)t;
    }
  } else {
    gb[i - nw] = (float)t;
  }
}

// Transpose of the linear upsampling from m to n along one axis of a tensor
// viewed as (outer, n, inner) -> (outer, m, inner):
//   out[o][j][c] = sum_x U[x][j] in[o][x][c],  U[x][j] = the weight of coarse j
// in fine x's half-pixel interpolation, read from the level's sparse rows
// (built once on the host with the same arithmetic as bilin).  The
// D-dimensional transpose is D such passes, one per axis.

// With outbf (the last axis): outbf = bf16(mask > 0 ? out : 0) instead of out.
__global__ void upsample_bwd_axis(long long outer, int n, int m, long long inner,
                                  const int* __restrict__ ptr, const int* __restrict__ idx,
                                  const float* __restrict__ wt, const float* __restrict__ in,
                                  float* __restrict__ out, const bf16* __restrict__ mask,
                                  bf16* __restrict__ outbf) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= outer * m * inner) return;
  // element indices stay below 2^31 (network size check): 32-bit division
  const unsigned ui = (unsigned)id, uin = (unsigned)inner;
  const unsigned c = ui % uin;
  const unsigned p = ui / uin;
  const int j = (int)(p % (unsigned)m);
  const unsigned o = p / (unsigned)m;
  float acc = 0.f;
  for (int k = ptr[j]; k < ptr[j + 1]; k++)
    acc += wt[k] * in[((long long)o * n + idx[k]) * inner + c];
  if (outbf)
    outbf[id] = __float2bfloat16(__bfloat162float(mask[id]) > 0.f ? acc : 0.f);
  else
    out[id] = acc;
}

// The x-axis pass of every coarse level's transposed upsampling at once:
//   out_l[r][j][c] = sum_x U_l[x][j] in[r][x][c]   (levels l = 1 .. L-1)
// for each row r of the fine grid (x is the innermost axis in 2D and 3D).  One
// CTA per row: its n x 32 values are read from HBM once and from L1 for the
// other levels (the per-level pass reads the whole fine gradient per level).
// Same sums, in the same order, as upsample_bwd_axis.
struct UpXLevels {
  int nlev;
  int m[kMaxLevels];
  const int* ptr[kMaxLevels];
  const int* idx[kMaxLevels];
  const float* wt[kMaxLevels];
  long long off[kMaxLevels];  // out_l = out + off[l], rows of m_l x 32
};

constexpr int kXLevelsMaxN = 384;  // the staged row (n x 32 floats) stays within 48 KB

__global__ void __launch_bounds__(256) upsample_bwd_x_levels(int n, UpXLevels lv,
                                                             const float* __restrict__ in,
                                                             float* __restrict__ out) {
  extern __shared__ float row[];  // the fine row, n x 32
  const long long r = blockIdx.x;
  const int c = threadIdx.x & 31, w = threadIdx.x >> 5;
  {
    const float4* src = reinterpret_cast<const float4*>(in + r * n * kC);
    float4* dst = reinterpret_cast<float4*>(row);
    for (int i = threadIdx.x; i < n * kC / 4; i += 256) dst[i] = src[i];
  }
  __syncthreads();
  for (int l = 1; l < lv.nlev; l++) {
    const int m = lv.m[l];
    const int* __restrict__ ptr = lv.ptr[l];
    const int* __restrict__ idx = lv.idx[l];
    const float* __restrict__ wt = lv.wt[l];
    float* __restrict__ o = out + lv.off[l] + r * m * kC;
    for (int j = w; j < m; j += 8) {
      float acc = 0.f;
      for (int k = ptr[j]; k < ptr[j + 1]; k++) acc += wt[k] * row[idx[k] * kC + c];
      o[j * kC + c] = acc;
    }
  }
}

// fine[p][c] += coarse[p / 2][c] / 2^D (fine side s, coarse side s/2)
template <int D>
__global__ void pool2_bwd_add(int B, int s, const float* __restrict__ coarse,
                              float* __restrict__ fine) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= B * Geo<D>::pts(s) * kC) return;
  const int c = (int)(idx % kC);
  int b, z, y, x;
  Geo<D>::decode(idx / kC, s, b, z, y, x);
  const int so = s / 2;
  if (y / 2 >= so || x / 2 >= so || (D == 3 && z / 2 >= so)) return;
  const long long q = Geo<D>::nb(b, z / 2, y / 2, x / 2, 0, 0, 0, so);
  fine[idx] += (1.f / (1 << D)) * coarse[q * kC + c];
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// theta -= lr * (m / c1) / (sqrt(v / c2) + eps), c1 = 1 - b1^t, c2 = 1 - b2^t
// (c1, c2 of the step in progress, from the phase's device state)
__global__ void adam_kernel(long long count, float* __restrict__ theta,
                            const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, const TrainCtr* __restrict__ ctr) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float c1 = ctr->c1, c2 = ctr->c2;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Start of one Adam step of a phase: t = adam_t + 1 with its bias corrections,
// and the offset of this step's minibatch in the phase's picks.
__global__ void step_begin(TrainCtr* ctr, int B) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const long long t = ctr->adam_t + 1;
    ctr->adam_t = t;
    ctr->c1 = 1.f - powf(0.9f, (float)t);
    ctr->c2 = 1.f - powf(0.999f, (float)t);
    ctr->pick_off = ctr->iter * B;
    ctr->iter = ctr->iter + 1;
  }
}

// bu[b] = ring_u[picks[pick_off + b]], bt[b] = ring_t[...] for b < B (N each,
// ring slots `stride` floats apart)
__global__ void gather_pairs(int B, long long N, const float* __restrict__ ring_u,
                             const float* __restrict__ ring_t, long long stride,
                             const int* __restrict__ picks, const TrainCtr* __restrict__ ctr,
                             float* __restrict__ bu, float* __restrict__ bt) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)B * N) return;
  const int b = (int)(i / N);
  const long long p = i - (long long)b * N;
  const long long src = (long long)picks[ctr->pick_off + b] * stride + p;
  bu[i] = ring_u[src];
  bt[i] = ring_t[src];
}

// wq[conv][tap][k][o] = W[o][k][tap], wqT[conv][tap][o][k] = W[o][k][tap] (BF16)
__global__ void sync_weights_kernel(int nconv, int T, const float* __restrict__ master,
                                    const long long* __restrict__ offs, bf16* __restrict__ wq,
                                    bf16* __restrict__ wqT) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long per = (long long)T * kC * kC;
  if (i >= nconv * per) return;
  const int cv = (int)((unsigned)i / (unsigned)per);
  const int r = (int)((unsigned)i % (unsigned)per);
  const int o = r / (kC * T), k = (r / T) % kC, tp = r % T;
  const bf16 v = __float2bfloat16(master[offs[cv] + r]);
  wq[(long long)cv * per + (tp * kC + k) * kC + o] = v;
  wqT[(long long)cv * per + (tp * kC + o) * kC + k] = v;
}

unsigned nblk(long long count, int bs) { return (unsigned)((count + bs - 1) / bs); }

unsigned long long sm64(unsigned long long& st) {
  st += 0x9E3779B97F4A7C15ull;
  unsigned long long z = st;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

#define NN_CK(x)                          \
  do {                                    \
    cudaError_t e_ = (x);                 \
    if (e_ != cudaSuccess) return e_;     \
  } while (0)

cudaError_t net_create(Net& net, int n, int bmax, unsigned long long seed, int dim,
                       int extra_max, bool infer_only) {
  if (dim != 2 && dim != 3) return cudaErrorInvalidValue;
  if (extra_max < 0 || extra_max > kMaxExtra) return cudaErrorInvalidValue;
  // the kernels index points and point-channel elements in 32 bits
  if (n < 1 || bmax < 1 ||
      (long long)bmax * (dim == 3 ? (long long)n * n * n : (long long)n * n) * kC >= (1LL << 31))
    return cudaErrorInvalidValue;
  NN_CK(conv32_tc_setup());
  NN_CK(conv32_mma_setup());
  net.extra_max = extra_max;
  net.extra_active = 0;
  net.n = n;
  net.dim = dim;
  net.taps = dim == 3 ? 27 : 9;
  const int T = net.taps;
  net.bmax = bmax;
  net.L = 0;
  int s = n;
  net.side[net.L++] = s;
  while (s / 2 >= 8 && net.L < kMaxLevels) {
    s /= 2;
    net.side[net.L++] = s;
  }
  const int L = net.L;
  const long long per = (long long)T * kC * kC;
  long long off = 0;
  net.off_w[0] = off; off += kC * T;
  net.off_b[0] = off; off += kC;
  for (int l = 0; l < L; l++) {
    net.off_w[1 + l] = off; off += per;
    net.off_b[1 + l] = off; off += kC;
  }
  net.off_w[L + 1] = off; off += per;
  net.off_b[L + 1] = off; off += kC;
  net.off_w[L + 2] = off; off += kC * T;
  net.off_b[L + 2] = off; off += 1;
  for (int r = 0; r < extra_max; r++) {
    net.off_rw[r] = off; off += per;
    net.off_rb[r] = off; off += kC;
  }
  net.nparams = off;

  // He-uniform initialisation from splitmix64: U[-a, a], a = sqrt(6 / fan_in);
  // the output layer uses a = sqrt(3 / fan_in); biases start at 0.
  std::vector<float> p((size_t)net.nparams, 0.f);
  unsigned long long st = seed ^ 0x6A09E667F3BCC909ull;
  auto fill = [&](long long o, long long cnt, int fan_in, float gain) {
    const double a = sqrt(gain / fan_in);
    for (long long i = 0; i < cnt; i++) {
      const double u = (double)(sm64(st) >> 11) * (1.0 / 9007199254740992.0);
      p[(size_t)(o + i)] = (float)((2.0 * u - 1.0) * a);
    }
  };
  fill(net.off_w[0], kC * T, T, 6.f);
  for (int l = 0; l < L; l++) fill(net.off_w[1 + l], per, T * kC, 6.f);
  fill(net.off_w[L + 1], per, T * kC, 6.f);
  fill(net.off_w[L + 2], kC * T, T * kC, 3.f);
  // a grown block starts close to the identity (small weights, zero bias) so
  // the guess changes little when it is appended, yet its gradient is not zero
  for (int r = 0; r < extra_max; r++) fill(net.off_rw[r], per, T * kC, 0.06f);

  const long long np = net.nparams;
  NN_CK(cudaMalloc(&net.master, sizeof(float) * np));
  NN_CK(cudaMemcpy(net.master, p.data(), sizeof(float) * np, cudaMemcpyHostToDevice));
  if (!infer_only) {
    NN_CK(cudaMalloc(&net.grad, sizeof(float) * np));
    NN_CK(cudaMalloc(&net.adam_m, sizeof(float) * np));
    NN_CK(cudaMalloc(&net.adam_v, sizeof(float) * np));
    NN_CK(cudaMemset(net.grad, 0, sizeof(float) * np));
    NN_CK(cudaMemset(net.adam_m, 0, sizeof(float) * np));
    NN_CK(cudaMemset(net.adam_v, 0, sizeof(float) * np));
  }
  const int nconv = L + 1 + extra_max;  // the 32 -> 32 convolutions
  NN_CK(cudaMalloc(&net.wq, sizeof(bf16) * per * nconv));
  NN_CK(cudaMalloc(&net.wqT, sizeof(bf16) * per * nconv));
  long long offs[kMaxLevels + 1 + kMaxExtra];
  for (int c = 0; c < L + 1; c++) offs[c] = net.off_w[1 + c];
  for (int r = 0; r < extra_max; r++) offs[L + 1 + r] = net.off_rw[r];
  NN_CK(cudaMalloc(&net.offs_dev, sizeof(offs)));
  NN_CK(cudaMemcpy(net.offs_dev, offs, sizeof(long long) * nconv, cudaMemcpyHostToDevice));

  auto pts = [dim](int side) {
    return dim == 3 ? (long long)side * side * side : (long long)side * side;
  };
  const long long full = (long long)bmax * pts(n) * kC;
  NN_CK(cudaMalloc(&net.a0, sizeof(bf16) * full));
  net.pyr = 0;
  for (int l = 0; l < L; l++) {
    const long long sz = (long long)bmax * pts(net.side[l]) * kC;
    if (l > 0) NN_CK(cudaMalloc(&net.pool[l], sizeof(bf16) * sz));
    NN_CK(cudaMalloc(&net.z[l], sizeof(bf16) * sz));
    net.lvl_off[l] = net.pyr;
    net.pyr += sz;
  }
  for (int l = 1; l < L; l++) {
    const int m = net.side[l];
    std::vector<std::vector<std::pair<int, float>>> rows(m);
    for (int x = 0; x < n; x++) {
      float src = ((float)x + 0.5f) * (float)m / (float)n - 0.5f;  // as bilin
      if (src < 0.f) src = 0.f;
      int i0 = (int)floorf(src);
      if (i0 > m - 1) i0 = m - 1;
      const int i1 = i0 + 1 < m - 1 ? i0 + 1 : m - 1;
      const float lam = src - (float)i0;
      if (i0 == i1) {
        rows[i0].push_back({x, (1.f - lam) + lam});
      } else {
        rows[i0].push_back({x, 1.f - lam});
        rows[i1].push_back({x, lam});
      }
    }
    std::vector<int> ptr(m + 1, 0), idx;
    std::vector<float> wt;
    for (int j = 0; j < m; j++) {
      for (auto& e : rows[j]) {
        idx.push_back(e.first);
        wt.push_back(e.second);
      }
      ptr[j + 1] = (int)idx.size();
    }
    NN_CK(cudaMalloc(&net.up_ptr[l], sizeof(int) * (m + 1)));
    NN_CK(cudaMalloc(&net.up_idx[l], sizeof(int) * idx.size()));
    NN_CK(cudaMalloc(&net.up_w[l], sizeof(float) * wt.size()));
    NN_CK(cudaMemcpy(net.up_ptr[l], ptr.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice));
    NN_CK(cudaMemcpy(net.up_idx[l], idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice));
    NN_CK(cudaMemcpy(net.up_w[l], wt.data(), sizeof(float) * wt.size(), cudaMemcpyHostToDevice));
  }
  NN_CK(cudaMalloc(&net.s, sizeof(bf16) * full));
  NN_CK(cudaMalloc(&net.e, sizeof(bf16) * full));
  NN_CK(cudaMalloc(&net.t, sizeof(bf16) * full));
  for (int r = 0; r < extra_max; r++) {
    NN_CK(cudaMalloc(&net.te[r], sizeof(bf16) * full));
    NN_CK(cudaMalloc(&net.tt[r], sizeof(bf16) * full));
  }
  if (infer_only) {  // forward passes only: no gradient, Adam or minibatch buffers
    NN_CK(net_sync_weights(net, 0));
    return cudaDeviceSynchronize();
  }
  NN_CK(cudaMalloc(&net.g_t, sizeof(float) * full));
  NN_CK(cudaMalloc(&net.g_s, sizeof(float) * full));
  NN_CK(cudaMalloc(&net.g_lvl, sizeof(float) * full));
  NN_CK(cudaMalloc(&net.g_pool, sizeof(float) * net.pyr));
  NN_CK(cudaMalloc(&net.g_bf, sizeof(bf16) * full));
  int dev = 0, nsm = 0;
  NN_CK(cudaGetDevice(&dev));
  NN_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  net.wparts = 2 * nsm;
  // the 1-channel weight gradients take more than the default 48 KB of
  // dynamic shared memory in 3D (their fixed-order reduction buffer)
  if (dim == 3) {
    NN_CK(cudaFuncSetAttribute(conv1_wgrad<0, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               conv1_wgrad_smem<3>(n)));
    NN_CK(cudaFuncSetAttribute(conv1_wgrad<1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               conv1_wgrad_smem<3>(n)));
  } else {
    NN_CK(cudaFuncSetAttribute(conv1_wgrad<0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               conv1_wgrad_smem<2>(n)));
    NN_CK(cudaFuncSetAttribute(conv1_wgrad<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               conv1_wgrad_smem<2>(n)));
  }
  NN_CK(cudaMalloc(&net.wgrad_part, sizeof(float) * (long long)net.wparts * (per + kC)));
  const long long pix = (long long)bmax * pts(n);
  NN_CK(cudaMalloc(&net.gy, sizeof(float) * pix));
  NN_CK(cudaMalloc(&net.loss_part, sizeof(float) * 1024));
  NN_CK(cudaMalloc(&net.bu, sizeof(float) * pix));
  NN_CK(cudaMalloc(&net.bt, sizeof(float) * pix));
  NN_CK(cudaMalloc(&net.by, sizeof(float) * pix));
  NN_CK(cudaMalloc(&net.ctr, sizeof(TrainCtr)));
  {
    TrainCtr c0{};
    c0.tscale = 1.f;
    NN_CK(cudaMemcpy(net.ctr, &c0, sizeof(c0), cudaMemcpyHostToDevice));
  }
  NN_CK(net_sync_weights(net, 0));
  return cudaDeviceSynchronize();
}

void net_destroy(Net& net) {
  cudaFree(net.master);
  cudaFree(net.grad);
  cudaFree(net.adam_m);
  cudaFree(net.adam_v);
  cudaFree(net.wq);
  cudaFree(net.wqT);
  cudaFree(net.offs_dev);
  cudaFree(net.a0);
  for (int l = 0; l < kMaxLevels; l++) {
    cudaFree(net.pool[l]);
    cudaFree(net.z[l]);
    cudaFree(net.up_ptr[l]);
    cudaFree(net.up_idx[l]);
    cudaFree(net.up_w[l]);
  }
  cudaFree(net.s);
  cudaFree(net.e);
  cudaFree(net.t);
  for (int r = 0; r < kMaxExtra; r++) {
    cudaFree(net.te[r]);
    cudaFree(net.tt[r]);
  }
  cudaFree(net.g_t);
  cudaFree(net.g_s);
  cudaFree(net.g_lvl);
  cudaFree(net.g_pool);
  cudaFree(net.g_bf);
  cudaFree(net.wgrad_part);
  cudaFree(net.gy);
  cudaFree(net.loss_part);
  cudaFree(net.bu);
  cudaFree(net.bt);
  cudaFree(net.by);
  cudaFree(net.ctr);
  net = Net();
}

cudaError_t net_copy_params(Net& dst, const float* src, cudaStream_t s) {
  NN_CK(cudaMemcpyAsync(dst.master, src, sizeof(float) * dst.nparams, cudaMemcpyDeviceToDevice,
                        s));
  return net_sync_weights(dst, s);
}

cudaError_t net_sync_weights(Net& net, cudaStream_t s) {
  const int nconv = net.L + 1 + net.extra_max;
  const long long tot = (long long)nconv * net.taps * kC * kC;
  sync_weights_kernel<<<nblk(tot, 256), 256, 0, s>>>(nconv, net.taps, net.master, net.offs_dev,
                                                    net.wq, net.wqT);
  note_launches(1);
  return cudaGetLastError();
}

namespace {

template <int D>
cudaError_t forward_t(Net& net, int B, const float* u, float* y, cudaStream_t s) {
  const int n = net.n, L = net.L;
  const long long pix = B * Geo<D>::pts(n);
  const long long per = (long long)Geo<D>::T * kC * kC;
  conv_in_fwd<D><<<nblk(pix, 256), 256, 0, s>>>(B, n, u, net.master + net.off_w[0],
                                                 net.master + net.off_b[0], net.a0);
  note_launches(1);
  for (int l = 1; l < L; l++) {
    const int sp = net.side[l - 1];
    const bf16* src = l == 1 ? net.a0 : net.pool[l - 1];
    const long long cnt = B * Geo<D>::pts(net.side[l]) * kC;
    pool2_fwd<D><<<nblk(cnt, 256), 256, 0, s>>>(B, sp, src, net.pool[l]);
    note_launches(1);
  }
  for (int l = 0; l < L; l++) {
    NN_CK(launch_conv32_mma(D, 0, B, net.side[l], l == 0 ? net.a0 : net.pool[l],
                            net.wqT + per * l, net.master + net.off_b[1 + l], 1, 1, net.z[l],
                            nullptr, nullptr, nullptr, nullptr, s));
  }
  Levels lv;
  lv.L = L;
  for (int l = 0; l < L; l++) {
    lv.z[l] = net.z[l];
    lv.side[l] = net.side[l];
  }
  upsum_fwd<D><<<nblk(pix * 4, 256), 256, 0, s>>>(B, n, lv, net.s);
  note_launches(1);
  NN_CK(launch_conv32_mma(D, 1, B, n, net.s, net.wqT + per * L, net.master + net.off_b[L + 1], 2,
                          1, net.e, net.t, net.s, nullptr, nullptr, s));
  const bf16* cur = net.t;
  for (int r = 0; r < net.extra_active; r++) {  // grown residual blocks
    NN_CK(launch_conv32_mma(D, 1, B, n, cur, net.wqT + per * (L + 1 + r),
                            net.master + net.off_rb[r], 2, 1, net.te[r], net.tt[r], cur, nullptr,
                            nullptr, s));
    cur = net.tt[r];
  }
  conv_out_fwd<D><<<nblk(pix, 256), 256, 0, s>>>(B, n, cur, net.master + net.off_w[L + 2],
                                                  net.master + net.off_b[L + 2], y);
  note_launches(1);
  return cudaGetLastError();
}

template <int D>
cudaError_t backward_t(Net& net, int B, const float* u, const float* y, const float* target,
                       float tscale, const float* tscale_dev, float* loss_dev, cudaStream_t s) {
  constexpr int T = Geo<D>::T;
  const int n = net.n, L = net.L;
  const long long pix = B * Geo<D>::pts(n);
  const long long full = pix * kC;
  const long long per = (long long)T * kC * kC;
  const int P = net.wparts;
  const int stride = (int)(per + kC);
  // loss and dL/dy
  const int lparts = 256;
  mse_grad<<<lparts, 256, 0, s>>>(pix, 1.f / (float)pix, tscale, tscale_dev, y, target, net.gy,
                                  net.loss_part);
  note_launches(1);
  loss_finish<<<1, 32, 0, s>>>(net.loss_part, lparts, 1.f / (float)pix, loss_dev);
  note_launches(1);
  // output conv
  const bf16* tfin = net.extra_active > 0 ? net.tt[net.extra_active - 1] : net.t;
  // the 1-channel weight gradients: 32 (T + 1) outputs per CTA (short stride)
  const int P1 = P, stride1 = kC * (T + 1);
  const int smem1 = conv1_wgrad_smem<D>(n);
  conv1_wgrad<0, D><<<P1, kW1Threads, smem1, s>>>(B, n, net.gy, tfin, nullptr, nullptr, nullptr,
                                                  net.wgrad_part, stride1);
  note_launches(1);
  reduce_wgrad<<<nblk(T * kC + 1, 32), 256, 0, s>>>(net.wgrad_part, P1, stride1, 2, T,
                                                     net.grad + net.off_w[L + 2],
                                                     net.grad + net.off_b[L + 2]);
  note_launches(1);
  // the first masked use of g_t (the last grown block's, else the residual
  // block's) is written by the same kernel
  const bf16* mask0 = net.extra_active > 0 ? net.te[net.extra_active - 1] : net.e;
  conv_out_bwd_data<D><<<2 * P, kW1Threads, sizeof(float) * w1_stage_floats<D>(n), s>>>(
      B, n, net.gy, net.master + net.off_w[L + 2], net.g_t, mask0, net.g_bf);
  note_launches(1);
  // grown residual blocks, last first: t_out = t_in + relu(conv_d2(t_in));
  // blocks not appended yet get a zero gradient (Adam then leaves them as they are)
  for (int r = net.extra_active; r < net.extra_max; r++)
    NN_CK(cudaMemsetAsync(net.grad + net.off_rw[r], 0, sizeof(float) * (per + kC), s));
  {
    float* gcur = net.g_t;
    float* gnext = net.g_s;
    for (int r = net.extra_active - 1; r >= 0; r--) {
      const bf16* tin = r == 0 ? net.t : net.tt[r - 1];
      if (r != net.extra_active - 1) {  // (the first one came with g_t)
        mask_to_bf16<<<nblk((full) / 8, 256), 256, 0, s>>>(full, gcur, net.te[r], net.g_bf);
        note_launches(1);
      }
      NN_CK(launch_wgrad_mma(D, B, n, tin, net.g_bf, 2, net.wgrad_part, stride, P, s));
      reduce_wgrad<<<nblk(per + kC, 32), 256, 0, s>>>(net.wgrad_part, P, stride, 0, T,
                                                       net.grad + net.off_rw[r],
                                                       net.grad + net.off_rb[r]);
      note_launches(1);
      NN_CK(launch_conv32_mma(D, 2, B, n, net.g_bf, net.wq + per * (L + 1 + r), nullptr, 2, -1,
                              nullptr, nullptr, nullptr, gnext, gcur, s));
      std::swap(gcur, gnext);
    }
    if (gcur != net.g_t)
      NN_CK(cudaMemcpyAsync(net.g_t, gcur, sizeof(float) * full, cudaMemcpyDeviceToDevice, s));
  }
  // dilated residual block: t = s + e, e = relu(conv_d2(s))
  if (net.extra_active > 0) {
    mask_to_bf16<<<nblk((full) / 8, 256), 256, 0, s>>>(full, net.g_t, net.e, net.g_bf);
    note_launches(1);
  }
  NN_CK(launch_wgrad_mma(D, B, n, net.s, net.g_bf, 2, net.wgrad_part, stride, P, s));
  reduce_wgrad<<<nblk(per + kC, 32), 256, 0, s>>>(net.wgrad_part, P, stride, 0, T,
                                                   net.grad + net.off_w[L + 1],
                                                   net.grad + net.off_b[L + 1]);
  note_launches(1);
  NN_CK(launch_conv32_mma(D, 2, B, n, net.g_bf, net.wq + per * L, nullptr, 2, -1, nullptr,
                          nullptr, nullptr, net.g_s, net.g_t, s));
  // pyramid levels; first the x-axis pass of every coarse level's transposed
  // upsampling, from one read of the fine gradient (g_s) into g_t (free here:
  // the residual block's gradient is already in g_s)
  long long xoff[kMaxLevels] = {};
  const bool fused_x = L > 1 && n <= kXLevelsMaxN;
  if (fused_x) {
    UpXLevels lv;
    lv.nlev = L;
    const long long rows = B * Geo<D>::pts(n) / n;
    long long off = 0;
    for (int l = 1; l < L; l++) {
      lv.m[l] = net.side[l];
      lv.ptr[l] = net.up_ptr[l];
      lv.idx[l] = net.up_idx[l];
      lv.wt[l] = net.up_w[l];
      lv.off[l] = xoff[l] = off;
      off += rows * net.side[l] * kC;
    }
    upsample_bwd_x_levels<<<(unsigned)rows, 256, sizeof(float) * n * kC, s>>>(n, lv, net.g_s,
                                                                               net.g_t);
    note_launches(1);
  }
  for (int l = 0; l < L; l++) {
    const int sd = net.side[l];
    const long long lp = B * Geo<D>::pts(sd);
    const float* gz = net.g_s;
    if (l > 0) {
      // transposed upsampling, one axis at a time (x, y, then z); g_t and
      // g_lvl are free here (the residual block's gradient is already in g_s)
      const long long nn = n, m = sd;
      const int* up = net.up_ptr[l];
      const int* ui = net.up_idx[l];
      const float* uw = net.up_w[l];
      const float* gx = net.g_t + xoff[l];  // this level's x-axis pass (above)
      if (!fused_x) {  // (rows too long to stage: the level's own x-axis pass)
        upsample_bwd_axis<<<nblk(B * Geo<D>::pts(n) / n * m * kC, 256), 256, 0, s>>>(
            B * Geo<D>::pts(n) / n, n, sd, kC, up, ui, uw, net.g_s, net.g_t, nullptr, nullptr);
        note_launches(1);
        gx = net.g_t;
      }
      if (D == 2) {
        upsample_bwd_axis<<<nblk(B * m * m * kC, 256), 256, 0, s>>>(
            B, n, sd, m * kC, up, ui, uw, gx, nullptr, net.z[l], net.g_bf);
        note_launches(1);
        gz = nullptr;  // masked BF16 gradient already in g_bf
      } else {
        upsample_bwd_axis<<<nblk(B * nn * m * m * kC, 256), 256, 0, s>>>(
            B * nn, n, sd, m * kC, up, ui, uw, gx, net.g_lvl, nullptr, nullptr);
        upsample_bwd_axis<<<nblk(B * m * m * m * kC, 256), 256, 0, s>>>(
            B, n, sd, m * m * kC, up, ui, uw, net.g_lvl, nullptr, net.z[l], net.g_bf);
        note_launches(2);
        gz = nullptr;
      }
    }
    if (gz) {
      mask_to_bf16<<<nblk((lp * kC) / 8, 256), 256, 0, s>>>(lp * kC, gz, net.z[l], net.g_bf);
      note_launches(1);
    }
    const bf16* in = l == 0 ? net.a0 : net.pool[l];
    NN_CK(launch_wgrad_mma(D, B, sd, in, net.g_bf, 1, net.wgrad_part, stride, P, s));
    reduce_wgrad<<<nblk(per + kC, 32), 256, 0, s>>>(net.wgrad_part, P, stride, 0, T,
                                                     net.grad + net.off_w[1 + l],
                                                     net.grad + net.off_b[1 + l]);
    note_launches(1);
    NN_CK(launch_conv32_mma(D, 2, B, sd, net.g_bf, net.wq + per * l, nullptr, 1, -1, nullptr,
                            nullptr, nullptr, net.g_pool + net.lvl_off[l], nullptr, s));
  }
  // pooling chain: the gradient of p_{l-1} collects 1/2^D of p_l's
  for (int l = L - 1; l >= 1; l--) {
    const int sf = net.side[l - 1];
    const long long cnt = B * Geo<D>::pts(sf) * kC;
    pool2_bwd_add<D><<<nblk(cnt, 256), 256, 0, s>>>(B, sf, net.g_pool + net.lvl_off[l],
                                                    net.g_pool + net.lvl_off[l - 1]);
    note_launches(1);
  }
  // input conv
  // (the ReLU mask of a0 is applied inside the weight-gradient kernel)
  conv1_wgrad<1, D><<<P1, kW1Threads, smem1, s>>>(B, n, nullptr, nullptr,
                                                  net.g_pool + net.lvl_off[0], net.a0, u,
                                                  net.wgrad_part, stride1);
  note_launches(1);
  reduce_wgrad<<<nblk(T * kC + kC, 32), 256, 0, s>>>(net.wgrad_part, P1, stride1, 1, T,
                                                      net.grad + net.off_w[0],
                                                      net.grad + net.off_b[0]);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t net_forward(Net& net, int B, const float* u, float* y, cudaStream_t s) {
  return net.dim == 3 ? forward_t<3>(net, B, u, y, s) : forward_t<2>(net, B, u, y, s);
}

cudaError_t net_backward(Net& net, int B, const float* u, const float* y, const float* target,
                         float tscale, float* loss_dev, cudaStream_t s) {
  return net.dim == 3 ? backward_t<3>(net, B, u, y, target, tscale, nullptr, loss_dev, s)
                      : backward_t<2>(net, B, u, y, target, tscale, nullptr, loss_dev, s);
}

cudaError_t net_adam_reset(Net& net, cudaStream_t s) {
  NN_CK(cudaMemsetAsync(net.adam_m, 0, sizeof(float) * net.nparams, s));
  NN_CK(cudaMemsetAsync(net.adam_v, 0, sizeof(float) * net.nparams, s));
  return cudaMemsetAsync(&net.ctr->adam_t, 0, sizeof(long long), s);
}

cudaError_t net_train_step_dev(Net& net, int B, const float* ring_u, const float* ring_t,
                               long long stride, const int* picks, TrainCtr* ctr, float lr,
                               float* loss_dev, cudaStream_t s) {
  const long long N = net.dim == 3 ? (long long)net.n * net.n * net.n : (long long)net.n * net.n;
  step_begin<<<1, 32, 0, s>>>(ctr, B);
  gather_pairs<<<nblk((long long)B * N, 256), 256, 0, s>>>(B, N, ring_u, ring_t, stride, picks,
                                                           ctr, net.bu, net.bt);
  note_launches(2);
  NN_CK(cudaGetLastError());
  NN_CK(net_forward(net, B, net.bu, net.by, s));
  NN_CK(net.dim == 3
            ? backward_t<3>(net, B, net.bu, net.by, net.bt, 1.f, &ctr->tscale, loss_dev, s)
            : backward_t<2>(net, B, net.bu, net.by, net.bt, 1.f, &ctr->tscale, loss_dev, s));
  adam_kernel<<<nblk(net.nparams, 256), 256, 0, s>>>(net.nparams, net.master, net.grad,
                                                     net.adam_m, net.adam_v, lr, ctr);
  note_launches(1);
  NN_CK(cudaGetLastError());
  return net_sync_weights(net, s);
}

}  // namespace mlg
