// unet.cu - U-Net kernels (forward FP32 and BF16 tensor cores, backward,
// Adam) and the gkb_unet_* entry points.
//
// Layout: activations NHWC FP32; parameters flat FP32, per layer the weights
// w[ky][kx][cin][cout] then the bias. A convolution input can be the channel
// concatenation of two tensors, the first one read at half resolution with
// bilinear doubling folded into the fetch (pixel-centre alignment: fine pixel
// 2k takes 3/4 of coarse k and 1/4 of k - 1, fine 2k + 1 takes 3/4 of k and
// 1/4 of k + 1, neighbours clamped at the edge).
#include <cuda_bf16.h>
#include <math.h>

#include <cmath>

#include <algorithm>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "../../include/gkb.h"
#include "prof.h"
#include "unet.cuh"

namespace gkb {

struct In2 {
  const float* p0;  // first input (channels [0, c0))
  int c0;
  int up0;          // 1: p0 has half the resolution (nearest upsampling)
  const float* p1;  // second input (channels [c0, c0 + c1)), full resolution
  int c1;
};

constexpr int UT = 256;  // threads per block of the FP32 kernels

// coarse row (or column) pair of a fine index under bilinear doubling
__device__ __forceinline__ void up_pair(int f, int m, int& k, int& k2) {
  k = f >> 1;
  k2 = (f & 1) ? min(k + 1, m - 1) : max(k - 1, 0);
}

// 3/4 x 3/4, 3/4 x 1/4, 1/4 x 3/4 and 1/4 x 1/4 of the four coarse values
__device__ __forceinline__ float bilin(float a, float b, float c, float d) {
  return fmaf(0.0625f, d, fmaf(0.1875f, c, fmaf(0.1875f, b, 0.5625f * a)));
}

// channel ci of the (concatenated) input at full-resolution pixel (yy, xx)
__device__ __forceinline__ float in_val(const In2& in, int b, int yy, int xx, int h, int wd, int ci) {
  if (ci < in.c0) {
    if (!in.up0) return __ldg(in.p0 + (((long long)b * h + yy) * wd + xx) * in.c0 + ci);
    const int h0 = h >> 1, w0 = wd >> 1;
    int k, k2, l, l2;
    up_pair(yy, h0, k, k2);
    up_pair(xx, w0, l, l2);
    const float* base = in.p0 + (long long)b * h0 * w0 * in.c0 + ci;
    return bilin(__ldg(base + ((long long)k * w0 + l) * in.c0), __ldg(base + ((long long)k * w0 + l2) * in.c0),
                 __ldg(base + ((long long)k2 * w0 + l) * in.c0), __ldg(base + ((long long)k2 * w0 + l2) * in.c0));
  }
  return __ldg(in.p1 + (((long long)b * h + yy) * wd + xx) * in.c1 + (ci - in.c0));
}

__device__ __forceinline__ void px_decode(long long p, int h, int w, int& b, int& y, int& x) {
  x = (int)(p % w);
  const long long q = p / w;
  y = (int)(q % h);
  b = (int)(q / h);
}

// ---------------------------------------------------------------------------
// FP32 forward convolution: one thread per pixel, all CO outputs in registers
// ---------------------------------------------------------------------------
template <int CO>
__global__ void __launch_bounds__(UT) k_conv_fwd(In2 in, const float* __restrict__ w, const float* __restrict__ bias,
                                                  float* __restrict__ out, int n, int h, int wd, int relu) {
  extern __shared__ float ws[];  // [9][cin][CO]
  const int cin = in.c0 + in.c1;
  for (int t = threadIdx.x; t < 9 * cin * CO; t += blockDim.x) ws[t] = w[t];
  __syncthreads();
  const long long npx = (long long)n * h * wd;
  const int h0 = h >> in.up0, w0 = wd >> in.up0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npx; p += (long long)gridDim.x * blockDim.x) {
    int b, y, x;
    px_decode(p, h, wd, b, y, x);
    float acc[CO];
#pragma unroll
    for (int o = 0; o < CO; ++o) acc[o] = __ldg(bias + o);
    for (int ky = 0; ky < 3; ++ky) {
      const int yy = y + ky - 1;
      if (yy < 0 || yy >= h) continue;
      for (int kx = 0; kx < 3; ++kx) {
        const int xx = x + kx - 1;
        if (xx < 0 || xx >= wd) continue;
        const float* wt = ws + (ky * 3 + kx) * cin * CO;
        if (!in.up0) {
          const float* s0 = in.p0 + (((long long)b * h + yy) * wd + xx) * in.c0;
          for (int ci = 0; ci < in.c0; ++ci) {
            const float v = __ldg(s0 + ci);
#pragma unroll
            for (int o = 0; o < CO; ++o) acc[o] = fmaf(v, wt[ci * CO + o], acc[o]);
          }
        } else {
          int k, k2, l, l2;
          up_pair(yy, h0, k, k2);
          up_pair(xx, w0, l, l2);
          const float* base = in.p0 + (long long)b * h0 * w0 * in.c0;
          const float* q00 = base + ((long long)k * w0 + l) * in.c0;
          const float* q01 = base + ((long long)k * w0 + l2) * in.c0;
          const float* q10 = base + ((long long)k2 * w0 + l) * in.c0;
          const float* q11 = base + ((long long)k2 * w0 + l2) * in.c0;
          for (int ci = 0; ci < in.c0; ++ci) {
            const float v = bilin(__ldg(q00 + ci), __ldg(q01 + ci), __ldg(q10 + ci), __ldg(q11 + ci));
#pragma unroll
            for (int o = 0; o < CO; ++o) acc[o] = fmaf(v, wt[ci * CO + o], acc[o]);
          }
        }
        if (in.c1) {
          const float* s1 = in.p1 + (((long long)b * h + yy) * wd + xx) * in.c1;
          const float* wt1 = wt + in.c0 * CO;
          for (int ci = 0; ci < in.c1; ++ci) {
            const float v = __ldg(s1 + ci);
#pragma unroll
            for (int o = 0; o < CO; ++o) acc[o] = fmaf(v, wt1[ci * CO + o], acc[o]);
          }
        }
      }
    }
    float* op = out + p * CO;
#pragma unroll
    for (int o = 0; o < CO; ++o) op[o] = relu ? fmaxf(acc[o], 0.f) : acc[o];
  }
}

// ---------------------------------------------------------------------------
// BF16 tensor-core forward convolution (mma.sync m16n8k16, FP32 accumulate)
// Block: 8 warps, tile of TR = 8 rows x TC = 32 columns of output pixels; warp
// w owns row w as two M tiles of 16 pixels; N = output channels in tiles of
// 8; K = 9 taps x input channels in steps of 16. The input tile with a
// one-pixel halo and all nine taps of transposed weights are staged once in
// shared memory as BF16, every pixel's (and output channel's) K vector padded
// by 8 elements so that the fragment loads of a warp hit distinct banks.
// ---------------------------------------------------------------------------
constexpr int TR = 8, TC = 32, TCT = 256;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// four consecutive channels [ci, ci + 4) of the (concatenated) input at
// full-resolution pixel (yy, xx); the group lies inside one of the two
// inputs whenever c0 is a multiple of 4 (vector loads), else per channel
__device__ __forceinline__ float4 in_val4(const In2& in, int b, int yy, int xx, int h, int wd, int ci, int cin) {
  if ((in.c0 & 3) == 0 && ci + 4 <= cin) {
    if (ci < in.c0 && !in.up0 && (in.c0 & 3) == 0)
      return __ldg(reinterpret_cast<const float4*>(in.p0 + (((long long)b * h + yy) * wd + xx) * in.c0 + ci));
    if (ci >= in.c0 && (in.c1 & 3) == 0)
      return __ldg(reinterpret_cast<const float4*>(in.p1 + (((long long)b * h + yy) * wd + xx) * in.c1 + (ci - in.c0)));
  }
  float4 v;
  v.x = ci + 0 < cin ? in_val(in, b, yy, xx, h, wd, ci + 0) : 0.f;
  v.y = ci + 1 < cin ? in_val(in, b, yy, xx, h, wd, ci + 1) : 0.f;
  v.z = ci + 2 < cin ? in_val(in, b, yy, xx, h, wd, ci + 2) : 0.f;
  v.w = ci + 3 < cin ? in_val(in, b, yy, xx, h, wd, ci + 3) : 0.f;
  return v;
}

template <int CIP, int COP>
struct TcSmem {
  static constexpr int KS = CIP + 8;                     // padded K stride (elements)
  static constexpr int XS = (TR + 2) * (TC + 2) * KS;    // input tile
  static constexpr int WS = 9 * COP * KS;                // weights [tap][co][ci]
  static constexpr size_t bytes = (size_t)(XS + WS) * sizeof(__nv_bfloat16);
};

// CIP: input channels padded to a multiple of 16; COP: output channels padded to a multiple of 8
template <int CIP, int COP>
__global__ void __launch_bounds__(TCT) k_conv_fwd_tc(In2 in, const __nv_bfloat16* __restrict__ wbf /*[9][cin][cout]*/,
                                                     const float* __restrict__ bias, float* __restrict__ out, int cout,
                                                     int n, int h, int wd, int relu) {
  using SM = TcSmem<CIP, COP>;
  constexpr int KS = SM::KS;
  extern __shared__ __align__(16) __nv_bfloat16 tc_smem[];
  __nv_bfloat16* xs = tc_smem;
  __nv_bfloat16* wt = tc_smem + SM::XS;
  const int cin = in.c0 + in.c1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int x0 = blockIdx.x * TC, y0 = blockIdx.y * TR, b = blockIdx.z;
  // input tile with halo, four channels per item (zero outside the image and
  // in the channel padding)
  constexpr int G4 = CIP / 4;
  for (int t = tid; t < (TR + 2) * (TC + 2) * G4; t += TCT) {
    const int g4 = t % G4, px = t / G4;
    const int ty = px / (TC + 2), tx = px - ty * (TC + 2);
    const int yy = y0 + ty - 1, xx = x0 + tx - 1;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (yy >= 0 && yy < h && xx >= 0 && xx < wd && 4 * g4 < cin) v = in_val4(in, b, yy, xx, h, wd, 4 * g4, cin);
    __nv_bfloat16* d = xs + px * KS + 4 * g4;
    d[0] = __float2bfloat16(v.x);
    d[1] = __float2bfloat16(v.y);
    d[2] = __float2bfloat16(v.z);
    d[3] = __float2bfloat16(v.w);
  }
  // all nine taps of the weights, transposed to [tap][co][ci] (zero padded)
  for (int t = tid; t < 9 * COP * CIP; t += TCT) {
    const int co = t % COP, ci = (t / COP) % CIP, tap = t / (COP * CIP);
    wt[(tap * COP + co) * KS + ci] =
        (ci < cin && co < cout) ? wbf[((long long)tap * cin + ci) * cout + co] : __float2bfloat16(0.f);
  }
  __syncthreads();
  const int g = lane >> 2, tq = lane & 3;
  constexpr int NT = COP / 8;
  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.f;
  const int row = warp;  // output row within the tile
#pragma unroll 1
  for (int tap = 0; tap < 9; ++tap) {
    const int ky = tap / 3, kx = tap - 3 * ky;
    const __nv_bfloat16* wtap = wt + tap * COP * KS;
#pragma unroll
    for (int k0 = 0; k0 < CIP; k0 += 16) {
      uint32_t bb[NT][2];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        // B[k][n] = w[tap][k0 + k][nt*8 + n], staged as wt[tap][nt*8 + n][k0 + k]
        const __nv_bfloat16* bcol = wtap + (nt * 8 + g) * KS + k0;
        bb[nt][0] = *reinterpret_cast<const uint32_t*>(bcol + 2 * tq);
        bb[nt][1] = *reinterpret_cast<const uint32_t*>(bcol + 2 * tq + 8);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        // A[m][k] = xs[row + ky][mt*16 + m + kx][k0 + k]
        const __nv_bfloat16* arow0 = xs + ((row + ky) * (TC + 2) + (mt * 16 + g + kx)) * KS + k0;
        const __nv_bfloat16* arow1 = arow0 + 8 * KS;
        uint32_t a[4];
        a[0] = *reinterpret_cast<const uint32_t*>(arow0 + 2 * tq);
        a[1] = *reinterpret_cast<const uint32_t*>(arow1 + 2 * tq);
        a[2] = *reinterpret_cast<const uint32_t*>(arow0 + 2 * tq + 8);
        a[3] = *reinterpret_cast<const uint32_t*>(arow1 + 2 * tq + 8);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[mt][nt], a, bb[nt]);
      }
    }
  }
  // D[m][n]: rows g and g + 8, columns 2 tq and 2 tq + 1 of each n tile
  const int yy = y0 + row;
  if (yy >= h) return;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int xx = x0 + mt * 16 + g + 8 * half;
      if (xx >= wd) continue;
      float* op = out + (((long long)b * h + yy) * wd + xx) * cout;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int co = nt * 8 + 2 * tq + e;
          if (co < cout) {
            const float v = acc[mt][nt][2 * half + e] + __ldg(bias + co);
            op[co] = relu ? fmaxf(v, 0.f) : v;
          }
        }
    }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------

// d_in[p, ci] = sum_{tap, co} dout[p - (tap - 1), co] w[tap][ci][co], split into
// d0 (channels < c0, full resolution) and d1 (the rest)
template <int CIN, int CO>
__global__ void __launch_bounds__(UT) k_conv_bwd_data(const float* __restrict__ dout, const float* __restrict__ w, int c0,
                                                       float* __restrict__ d0, float* __restrict__ d1, int n, int h, int wd) {
  extern __shared__ float ws[];
  for (int t = threadIdx.x; t < 9 * CIN * CO; t += blockDim.x) ws[t] = w[t];
  __syncthreads();
  const long long npx = (long long)n * h * wd;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npx; p += (long long)gridDim.x * blockDim.x) {
    int b, y, x;
    px_decode(p, h, wd, b, y, x);
    float acc[CIN];
#pragma unroll
    for (int c = 0; c < CIN; ++c) acc[c] = 0.f;
    for (int ky = 0; ky < 3; ++ky) {
      const int yy = y - (ky - 1);
      if (yy < 0 || yy >= h) continue;
      for (int kx = 0; kx < 3; ++kx) {
        const int xx = x - (kx - 1);
        if (xx < 0 || xx >= wd) continue;
        const float* dp = dout + (((long long)b * h + yy) * wd + xx) * CO;
        const float* wt = ws + (ky * 3 + kx) * CIN * CO;
#pragma unroll 4
        for (int o = 0; o < CO; ++o) {
          const float dv = __ldg(dp + o);
#pragma unroll
          for (int c = 0; c < CIN; ++c) acc[c] = fmaf(dv, wt[c * CO + o], acc[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < CIN; ++c) {
      if (c < c0) d0[p * c0 + c] = acc[c];
      else d1[p * (CIN - c0) + (c - c0)] = acc[c];
    }
  }
}

// partial[blk][t], t < 9 cin co: sum over this block's pixels of
// in[p + tap, ci] * dpre[p, co]; t in [9 cin co, 9 cin co + co): sum of dpre
constexpr int WP = 8;   // pixels staged per step
template <int ITEMS>
__global__ void __launch_bounds__(UT) k_conv_bwd_w(In2 in, const float* __restrict__ dpre, int co,
                                                    float* __restrict__ partial, int n, int h, int wd) {
  extern __shared__ float sm[];
  const int cin = in.c0 + in.c1;
  const int nw = 9 * cin * co, ntot = nw + co;
  float* patch = sm;                      // [WP][9][cin]
  float* dsh = sm + WP * 9 * cin;         // [WP][co]
  float acc[ITEMS];
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) acc[k] = 0.f;
  const long long npx = (long long)n * h * wd;
  for (long long base = (long long)blockIdx.x * WP; base < npx; base += (long long)gridDim.x * WP) {
    __syncthreads();
    for (int t = threadIdx.x; t < WP * 9 * cin; t += blockDim.x) {
      const int ci = t % cin, tap = (t / cin) % 9, pi = t / (9 * cin);
      const long long p = base + pi;
      float v = 0.f;
      if (p < npx) {
        int b, y, x;
        px_decode(p, h, wd, b, y, x);
        const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
        if (yy >= 0 && yy < h && xx >= 0 && xx < wd) v = in_val(in, b, yy, xx, h, wd, ci);
      }
      patch[t] = v;
    }
    for (int t = threadIdx.x; t < WP * co; t += blockDim.x) {
      const long long p = base + t / co;
      dsh[t] = (p < npx) ? __ldg(dpre + p * co + (t % co)) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const int t = threadIdx.x + k * UT;
      if (t < nw) {
        const int o = t % co, ci = (t / co) % cin, tap = t / (co * cin);
        float s = 0.f;
#pragma unroll
        for (int pi = 0; pi < WP; ++pi) s = fmaf(patch[(pi * 9 + tap) * cin + ci], dsh[pi * co + o], s);
        acc[k] += s;
      } else if (t < ntot) {
        const int o = t - nw;
        float s = 0.f;
#pragma unroll
        for (int pi = 0; pi < WP; ++pi) s += dsh[pi * co + o];
        acc[k] += s;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int t = threadIdx.x + k * UT;
    if (t < ntot) partial[(long long)blockIdx.x * ntot + t] = acc[k];
  }
}

// out[t] = sum over blocks of partial[blk][t], fixed order (deterministic)
__global__ void k_reduce_rows(const float* __restrict__ partial, int nblk, int ntot, float* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntot) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(long long)b * ntot + t];
  out[t] = (float)s;
}

__global__ void k_relu_mask(float* __restrict__ d, const float* __restrict__ y, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    if (!(y[t] > 0.f)) d[t] = 0.f;
}

// 2x2 mean pooling (NHWC), h and w of the input
__global__ void k_pool(const float* __restrict__ x, float* __restrict__ y, int n, int h, int w, int c) {
  const long long tot = (long long)n * (h / 2) * (w / 2) * c;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(t % c);
    const long long p = t / c;
    int b, yy, xx;
    px_decode(p, h / 2, w / 2, b, yy, xx);
    const float* s = x + (((long long)b * h + 2 * yy) * w + 2 * xx) * c + ch;
    y[t] = 0.25f * (s[0] + s[c] + s[(long long)w * c] + s[(long long)w * c + c]);
  }
}

// dx (h, w) += pool adjoint of dy (h/2, w/2)
__global__ void k_pool_bwd_add(const float* __restrict__ dy, float* __restrict__ dx, int n, int h, int w, int c) {
  const long long tot = (long long)n * h * w * c;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(t % c);
    const long long p = t / c;
    int b, y, x;
    px_decode(p, h, w, b, y, x);
    dx[t] += 0.25f * dy[(((long long)b * (h / 2) + y / 2) * (w / 2) + x / 2) * c + ch];
  }
}

// weights with which coarse index k (of m) feeds fine indices 2k-1 .. 2k+2
// under bilinear doubling (the clamped edge adds the outer quarter back)
__device__ __forceinline__ void up_adj_weights(int k, int m, float (&wgt)[4]) {
  wgt[0] = k >= 1 ? 0.25f : 0.f;
  wgt[1] = k == 0 ? 1.f : 0.75f;
  wgt[2] = k == m - 1 ? 1.f : 0.75f;
  wgt[3] = k + 1 <= m - 1 ? 0.25f : 0.f;
}

// d (h/2, w/2) = adjoint of bilinear doubling applied to dfull (h, w)
__global__ void k_up_bwd(const float* __restrict__ dfull, float* __restrict__ d, int n, int h, int w, int c) {
  const int h0 = h / 2, w0 = w / 2;
  const long long tot = (long long)n * h0 * w0 * c;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(t % c);
    const long long p = t / c;
    int b, k, l;
    px_decode(p, h0, w0, b, k, l);
    float wy[4], wx[4];
    up_adj_weights(k, h0, wy);
    up_adj_weights(l, w0, wx);
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (wy[a] == 0.f) continue;
      const int fy = 2 * k - 1 + a;
      const float* row = dfull + (((long long)b * h + fy) * w) * c + ch;
      float r = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (wx[e] != 0.f) r = fmaf(wx[e], row[(long long)(2 * l - 1 + e) * c], r);
      acc = fmaf(wy[a], r, acc);
    }
    d[t] = acc;
  }
}

// dy = scale (y - tscale t) (scale = 2 / batch), and the sum of (y - tscale t)^2
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
                                             long long n, float scale, float tscale, RedBuf red, double* out) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - tscale * t[i];
    dy[i] = scale * d;
    acc += (double)d * (double)d;
  }
  double v[1] = {acc};
  grid_reduce<1>(v, red, FIN_STORE, out);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16(a[i]);
}

// He-normal initial weights (std sqrt(2 / (9 cin))), zero biases, from a
// counter-based hash of (seed, index) and the Box-Muller transform
__global__ void k_init_params(float* p, long long off, long long nw, int cin, int cout, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nw + cout; i += (long long)gridDim.x * blockDim.x) {
    if (i >= nw) { p[off + i] = 0.f; continue; }
    unsigned long long z = (seed + (unsigned long long)(off + i)) * 0x9E3779B97F4A7C15ull;
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull; z ^= z >> 27; z *= 0x94D049BB133111EBull; z ^= z >> 31;
    const double u1 = ((z >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    unsigned long long z2 = z * 0x9E3779B97F4A7C15ull + 1442695040888963407ull;
    z2 ^= z2 >> 31;
    const double u2 = (z2 >> 11) * (1.0 / 9007199254740992.0);
    const double nrm = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    p[off + i] = (float)(nrm * sqrt(2.0 / (9.0 * cin)));
  }
}

static unsigned grid_for(long long n, int per = UT) {
  long long b = (n + per - 1) / per;
  if (b > 4096) b = 4096;
  return (unsigned)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

void Unet::init(int cin, int k1, int k2, int cout, unsigned long long seed, cudaStream_t s) {
  c_in = cin; c1 = k1; c2 = k2; c_out = cout; stream = s;
  if (!(cin >= 1 && cin <= 16 && k1 == 16 && k2 == 32 && cout >= 1 && cout <= 3))
    throw Error{GKB_ERR_INVALID_ARG, "supported U-Net: 1..16 inputs, 16/32 channels, 1..3 outputs"};
  const int shapes[9][2] = {{cin, k1}, {k1, k1}, {k1, k2}, {k2, k2}, {k2, k2}, {k2, k2}, {2 * k2, k2}, {k2 + k1, k1}, {k1, cout}};
  layers.clear();
  long long off = 0;
  for (auto& sh : shapes) {
    layers.push_back(ConvLayer{sh[0], sh[1], off});
    off += 9LL * sh[0] * sh[1] + sh[1];
  }
  nparams = off;
  params.alloc(nparams);
  grads.alloc(nparams);
  adam_m.alloc(nparams);
  adam_v.alloc(nparams);
  params_bf16.alloc(nparams);
  for (const ConvLayer& L : layers) {
    k_init_params<<<grid_for(L.nw() + L.cout), UT, 0, s>>>(params.p, L.off, L.nw(), L.cin, L.cout, seed);
    GKB_CUDA(cudaGetLastError());
  }
  red_partial.alloc(4096 * 4 + 64);
  red_ticket.alloc(1);
  loss_dev.alloc(4);
  wpart.alloc((size_t)304 * (9 * 64 * 32 + 32));
  // the largest FP32 convolution needs 9 * 64 * 32 floats of shared memory
  const int big = 9 * 64 * 32 * 4;
  GKB_CUDA(cudaFuncSetAttribute(k_conv_fwd<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  // the tensor-core convolutions stage all nine weight taps (up to 80 KB)
  GKB_CUDA(cudaFuncSetAttribute(k_conv_fwd_tc<16, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcSmem<16, 8>::bytes));
  GKB_CUDA(cudaFuncSetAttribute(k_conv_fwd_tc<16, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcSmem<16, 16>::bytes));
  GKB_CUDA(cudaFuncSetAttribute(k_conv_fwd_tc<16, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcSmem<16, 32>::bytes));
  GKB_CUDA(cudaFuncSetAttribute(k_conv_fwd_tc<32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcSmem<32, 32>::bytes));
  GKB_CUDA(cudaFuncSetAttribute(k_conv_fwd_tc<48, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcSmem<48, 16>::bytes));
  GKB_CUDA(cudaFuncSetAttribute(k_conv_fwd_tc<64, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcSmem<64, 32>::bytes));
  GKB_CUDA(cudaFuncSetAttribute(k_conv_bwd_data<64, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  bf16_stale = true;
  adam_t = 0;
}

void Unet::ensure(UnetAct& A, int n, int h, int w) const {
  if (h % 4 || w % 4 || n < 1 || h < 4 || w < 4) throw Error{GKB_ERR_INVALID_ARG, "U-Net images need sides divisible by 4"};
  if (n == A.n && h == A.h && w == A.w) return;
  const long long P = (long long)n * h * w, P2 = P / 4, P4 = P / 16;
  A.a1.alloc(P * c1); A.s1.alloc(P * c1); A.e1.alloc(P * c1); A.y.alloc(P * c_out);
  A.p1.alloc(P2 * c1); A.b1.alloc(P2 * c2); A.s2.alloc(P2 * c2); A.d1.alloc(P2 * c2);
  A.p2.alloc(P4 * c2); A.c1a.alloc(P4 * c2); A.c2a.alloc(P4 * c2);
  A.n = n; A.h = h; A.w = w;
}

void Unet::refresh_bf16(cudaStream_t s) {
  ProfScope ps_(GKB_KC_UNET, s, nparams);
  k_to_bf16<<<grid_for(nparams), UT, 0, s>>>(params.p, params_bf16.p, nparams);
  GKB_CUDA(cudaGetLastError());
  bf16_stale = false;
}

static void conv_fwd(const Unet& U, int li, In2 in, float* out, int n, int h, int w, int relu, bool tc,
                     cudaStream_t s) {
  const ConvLayer& L = U.layers[li];
  const float* wp = U.params.p + L.off;
  const float* bp = wp + L.nw();
  const long long P = (long long)n * h * w;
  ProfScope ps_(GKB_KC_UNET, s, P);
  if (tc) {
    const __nv_bfloat16* wb = U.params_bf16.p + L.off;
    dim3 grid((w + TC - 1) / TC, (h + TR - 1) / TR, n);
    const int cin = L.cin;
#define GKB_TC(CI, CO) \
  k_conv_fwd_tc<CI, CO><<<grid, TCT, TcSmem<CI, CO>::bytes, s>>>(in, wb, bp, out, L.cout, n, h, w, relu)
    if (cin <= 16 && L.cout <= 8) GKB_TC(16, 8);
    else if (cin <= 16 && L.cout <= 16) GKB_TC(16, 16);
    else if (cin <= 16) GKB_TC(16, 32);
    else if (cin <= 32) GKB_TC(32, 32);
    else if (cin <= 48) GKB_TC(48, 16);
    else GKB_TC(64, 32);
#undef GKB_TC
  } else {
    const size_t sm = 9ull * L.cin * L.cout * sizeof(float);
    if (L.cout == 32) k_conv_fwd<32><<<grid_for(P), UT, sm, s>>>(in, wp, bp, out, n, h, w, relu);
    else if (L.cout == 16) k_conv_fwd<16><<<grid_for(P), UT, sm, s>>>(in, wp, bp, out, n, h, w, relu);
    else if (L.cout == 1) k_conv_fwd<1><<<grid_for(P), UT, sm, s>>>(in, wp, bp, out, n, h, w, relu);
    else if (L.cout == 2) k_conv_fwd<2><<<grid_for(P), UT, sm, s>>>(in, wp, bp, out, n, h, w, relu);
    else if (L.cout == 3) k_conv_fwd<3><<<grid_for(P), UT, sm, s>>>(in, wp, bp, out, n, h, w, relu);
    else throw Error{GKB_ERR_INVALID_ARG, "unsupported convolution shape in forward"};
  }
  GKB_CUDA(cudaGetLastError());
}

const float* Unet::forward(UnetAct& A, const float* x, int n, int h, int w, bool tc, cudaStream_t s) {
  ensure(A, n, h, w);
  if (tc && bf16_stale) refresh_bf16(s);
  const int h2 = h / 2, w2 = w / 2, h4 = h / 4, w4 = w / 4;
  conv_fwd(*this, 0, In2{x, c_in, 0, nullptr, 0}, A.a1.p, n, h, w, 1, tc, s);
  conv_fwd(*this, 1, In2{A.a1.p, c1, 0, nullptr, 0}, A.s1.p, n, h, w, 1, tc, s);
  { ProfScope ps_(GKB_KC_UNET, s); k_pool<<<grid_for((long long)n * h2 * w2 * c1), UT, 0, s>>>(A.s1.p, A.p1.p, n, h, w, c1); }
  conv_fwd(*this, 2, In2{A.p1.p, c1, 0, nullptr, 0}, A.b1.p, n, h2, w2, 1, tc, s);
  conv_fwd(*this, 3, In2{A.b1.p, c2, 0, nullptr, 0}, A.s2.p, n, h2, w2, 1, tc, s);
  { ProfScope ps_(GKB_KC_UNET, s); k_pool<<<grid_for((long long)n * h4 * w4 * c2), UT, 0, s>>>(A.s2.p, A.p2.p, n, h2, w2, c2); }
  conv_fwd(*this, 4, In2{A.p2.p, c2, 0, nullptr, 0}, A.c1a.p, n, h4, w4, 1, tc, s);
  conv_fwd(*this, 5, In2{A.c1a.p, c2, 0, nullptr, 0}, A.c2a.p, n, h4, w4, 1, tc, s);
  conv_fwd(*this, 6, In2{A.c2a.p, c2, 1, A.s2.p, c2}, A.d1.p, n, h2, w2, 1, tc, s);
  conv_fwd(*this, 7, In2{A.d1.p, c2, 1, A.s1.p, c1}, A.e1.p, n, h, w, 1, tc, s);
  conv_fwd(*this, 8, In2{A.e1.p, c1, 0, nullptr, 0}, A.y.p, n, h, w, 0, tc, s);
  return A.y.p;
}

// weight gradient of layer li into grads (two deterministic passes)
static void conv_bwd_w(Unet& U, int li, In2 in, const float* dpre, int n, int h, int w) {
  const ConvLayer& L = U.layers[li];
  const int ntot = (int)(L.nw() + L.cout);
  const int items = (ntot + UT - 1) / UT;
  const long long P = (long long)n * h * w;
  long long nblk = (P + WP - 1) / WP;
  if (nblk > 304) nblk = 304;
  const size_t sm = (size_t)(WP * 9 * L.cin + WP * L.cout) * sizeof(float);
  cudaStream_t s = U.stream;
  ProfScope ps_(GKB_KC_UNET, s, P);
  if (items <= 2) k_conv_bwd_w<2><<<(unsigned)nblk, UT, sm, s>>>(in, dpre, L.cout, U.wpart.p, n, h, w);
  else if (items <= 9) k_conv_bwd_w<9><<<(unsigned)nblk, UT, sm, s>>>(in, dpre, L.cout, U.wpart.p, n, h, w);
  else if (items <= 19) k_conv_bwd_w<19><<<(unsigned)nblk, UT, sm, s>>>(in, dpre, L.cout, U.wpart.p, n, h, w);
  else if (items <= 37) k_conv_bwd_w<37><<<(unsigned)nblk, UT, sm, s>>>(in, dpre, L.cout, U.wpart.p, n, h, w);
  else k_conv_bwd_w<73><<<(unsigned)nblk, UT, sm, s>>>(in, dpre, L.cout, U.wpart.p, n, h, w);
  k_reduce_rows<<<(ntot + 255) / 256, 256, 0, s>>>(U.wpart.p, (int)nblk, ntot, U.grads.p + L.off);
  GKB_CUDA(cudaGetLastError());
}

// d_in of layer li (all input channels), split at c0 into d0 / d1
static void conv_bwd_data(Unet& U, int li, const float* dpre, int c0, float* d0, float* d1, int n, int h, int w) {
  const ConvLayer& L = U.layers[li];
  const long long P = (long long)n * h * w;
  const size_t sm = 9ull * L.cin * L.cout * sizeof(float);
  const float* wp = U.params.p + L.off;
  cudaStream_t s = U.stream;
  ProfScope ps_(GKB_KC_UNET, s, P);
  const unsigned g = grid_for(P);
  if (L.cin == 16 && L.cout == 16) k_conv_bwd_data<16, 16><<<g, UT, sm, s>>>(dpre, wp, c0, d0, d1, n, h, w);
  else if (L.cin == 16 && L.cout == 32) k_conv_bwd_data<16, 32><<<g, UT, sm, s>>>(dpre, wp, c0, d0, d1, n, h, w);
  else if (L.cin == 32 && L.cout == 32) k_conv_bwd_data<32, 32><<<g, UT, sm, s>>>(dpre, wp, c0, d0, d1, n, h, w);
  else if (L.cin == 64 && L.cout == 32) k_conv_bwd_data<64, 32><<<g, UT, sm, s>>>(dpre, wp, c0, d0, d1, n, h, w);
  else if (L.cin == 48 && L.cout == 16) k_conv_bwd_data<48, 16><<<g, UT, sm, s>>>(dpre, wp, c0, d0, d1, n, h, w);
  else if (L.cin == 16 && L.cout == 1) k_conv_bwd_data<16, 1><<<g, UT, sm, s>>>(dpre, wp, c0, d0, d1, n, h, w);
  else if (L.cin == 16 && L.cout == 2) k_conv_bwd_data<16, 2><<<g, UT, sm, s>>>(dpre, wp, c0, d0, d1, n, h, w);
  else if (L.cin == 16 && L.cout == 3) k_conv_bwd_data<16, 3><<<g, UT, sm, s>>>(dpre, wp, c0, d0, d1, n, h, w);
  else throw Error{GKB_ERR_INVALID_ARG, "unsupported convolution shape in backward"};
  GKB_CUDA(cudaGetLastError());
}

double Unet::loss_grad(const float* x, const float* t, int n, int h, int w) {
  cudaStream_t s = stream;
  forward(act, x, n, h, w, false, s);
  if (n != gn || h != gh || w != gw) {
    const long long P = (long long)n * h * w, P2 = P / 4, P4 = P / 16;
    g_full0.alloc(P * c2); g_full1.alloc(P * c2); g_e.alloc(P * c1);
    g_half0.alloc(P2 * c2); g_half1.alloc(P2 * c2);
    g_q0.alloc(P4 * c2); g_q1.alloc(P4 * c2);
    gn = n; gh = h; gw = w;
  }
  float *a1 = act.a1.p, *s1 = act.s1.p, *p1 = act.p1.p, *b1 = act.b1.p, *s2 = act.s2.p, *p2 = act.p2.p;
  float *c1a = act.c1a.p, *c2a = act.c2a.p, *d1 = act.d1.p, *e1 = act.e1.p, *y = act.y.p;
  const int h2 = h / 2, w2 = w / 2, h4 = h / 4, w4 = w / 4;
  const long long P = (long long)n * h * w, P2 = P / 4, P4 = P / 16;
  RedBuf red{red_partial.p, red_ticket.p};
  // dy = y - t (into g_e with c_out channels: g_e holds P * c1 >= P * c_out)
  float* dy = g_e.p;
  {
    ProfScope ps_(GKB_KC_UNET, s);
    k_mse<<<grid_for(P * c_out), 256, 0, s>>>(y, t, dy, P * c_out, 2.f / (float)n, target_scale, red, loss_dev.p);
  }
  // out layer (no ReLU): input e1
  conv_bwd_w(*this, 8, In2{e1, c1, 0, nullptr, 0}, dy, n, h, w);
  float* de1 = g_full1.p;  // P * c1
  conv_bwd_data(*this, 8, dy, c1, de1, nullptr, n, h, w);
  k_relu_mask<<<grid_for(P * c1), UT, 0, s>>>(de1, e1, P * c1);
  // e1 = relu(conv([up(d1), s1]))
  conv_bwd_w(*this, 7, In2{d1, c2, 1, s1, c1}, de1, n, h, w);
  float* du1 = g_full0.p;     // P * c2 (gradient of up(d1))
  float* ds1 = g_e.p;         // P * c1 (dy no longer needed)
  conv_bwd_data(*this, 7, de1, c2, du1, ds1, n, h, w);
  float* dd1 = g_half0.p;     // P2 * c2
  k_up_bwd<<<grid_for(P2 * c2), UT, 0, s>>>(du1, dd1, n, h, w, c2);
  k_relu_mask<<<grid_for(P2 * c2), UT, 0, s>>>(dd1, d1, P2 * c2);
  // d1 = relu(conv([up(c2a), s2]))
  conv_bwd_w(*this, 6, In2{c2a, c2, 1, s2, c2}, dd1, n, h2, w2);
  float* du2 = g_full1.p;     // P2 * c2 (reuse)
  float* ds2 = g_half1.p;     // P2 * c2
  conv_bwd_data(*this, 6, dd1, c2, du2, ds2, n, h2, w2);
  float* dc2 = g_q0.p;        // P4 * c2
  k_up_bwd<<<grid_for(P4 * c2), UT, 0, s>>>(du2, dc2, n, h2, w2, c2);
  k_relu_mask<<<grid_for(P4 * c2), UT, 0, s>>>(dc2, c2a, P4 * c2);
  conv_bwd_w(*this, 5, In2{c1a, c2, 0, nullptr, 0}, dc2, n, h4, w4);
  float* dc1 = g_q1.p;
  conv_bwd_data(*this, 5, dc2, c2, dc1, nullptr, n, h4, w4);
  k_relu_mask<<<grid_for(P4 * c2), UT, 0, s>>>(dc1, c1a, P4 * c2);
  conv_bwd_w(*this, 4, In2{p2, c2, 0, nullptr, 0}, dc1, n, h4, w4);
  float* dp2 = g_q0.p;
  conv_bwd_data(*this, 4, dc1, c2, dp2, nullptr, n, h4, w4);
  k_pool_bwd_add<<<grid_for(P2 * c2), UT, 0, s>>>(dp2, ds2, n, h2, w2, c2);
  k_relu_mask<<<grid_for(P2 * c2), UT, 0, s>>>(ds2, s2, P2 * c2);
  conv_bwd_w(*this, 3, In2{b1, c2, 0, nullptr, 0}, ds2, n, h2, w2);
  float* db1 = g_half0.p;
  conv_bwd_data(*this, 3, ds2, c2, db1, nullptr, n, h2, w2);
  k_relu_mask<<<grid_for(P2 * c2), UT, 0, s>>>(db1, b1, P2 * c2);
  conv_bwd_w(*this, 2, In2{p1, c1, 0, nullptr, 0}, db1, n, h2, w2);
  float* dp1 = g_half1.p;     // P2 * c1
  conv_bwd_data(*this, 2, db1, c1, dp1, nullptr, n, h2, w2);
  k_pool_bwd_add<<<grid_for(P * c1), UT, 0, s>>>(dp1, ds1, n, h, w, c1);
  k_relu_mask<<<grid_for(P * c1), UT, 0, s>>>(ds1, s1, P * c1);
  conv_bwd_w(*this, 1, In2{a1, c1, 0, nullptr, 0}, ds1, n, h, w);
  float* da1 = g_full1.p;
  conv_bwd_data(*this, 1, ds1, c1, da1, nullptr, n, h, w);
  k_relu_mask<<<grid_for(P * c1), UT, 0, s>>>(da1, a1, P * c1);
  conv_bwd_w(*this, 0, In2{x, c_in, 0, nullptr, 0}, da1, n, h, w);
  GKB_CUDA(cudaGetLastError());
  double loss = 0.0;
  GKB_CUDA(cudaMemcpyAsync(&loss, loss_dev.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  return loss / n;
}

void Unet::adam(float lr, float beta1, float beta2, float eps) {
  adam_t += 1;
  const float c1f = (float)(1.0 / (1.0 - pow((double)beta1, (double)adam_t)));
  const float c2f = (float)(1.0 / (1.0 - pow((double)beta2, (double)adam_t)));
  ProfScope ps_(GKB_KC_UNET, stream, nparams);
  k_adam<<<grid_for(nparams), UT, 0, stream>>>(params.p, grads.p, adam_m.p, adam_v.p, nparams, lr, beta1, beta2, eps, c1f, c2f);
  GKB_CUDA(cudaGetLastError());
  bf16_stale = true;
}

void Unet::train(const float* x_img, const float* t_img, long long count, int h, int w, int batch, int steps, float lr,
                 unsigned long long seed, double* losses) {
  if (count < 1 || batch < 1 || batch > count || steps < 0 || !(lr > 0))
    throw Error{GKB_ERR_INVALID_ARG, "training needs 1 <= batch <= count, steps >= 0 and lr > 0"};
  const long long xs = (long long)h * w * c_in, ts = (long long)h * w * c_out;
  if (xb.n != (size_t)(batch * xs)) xb.alloc((size_t)batch * xs);
  if (tb.n != (size_t)(batch * ts)) tb.alloc((size_t)batch * ts);
  std::vector<long long> order(count);
  for (long long i = 0; i < count; ++i) order[i] = i;
  std::mt19937_64 rng(seed);
  long long pos = count;  // forces a shuffle before the first batch
  for (int it = 0; it < steps; ++it) {
    for (int b = 0; b < batch; ++b) {
      if (pos == count) {
        std::shuffle(order.begin(), order.end(), rng);
        pos = 0;
      }
      const long long k = order[pos++];
      GKB_CUDA(cudaMemcpyAsync(xb.p + b * xs, x_img + k * xs, xs * sizeof(float), cudaMemcpyDeviceToDevice, stream));
      GKB_CUDA(cudaMemcpyAsync(tb.p + b * ts, t_img + k * ts, ts * sizeof(float), cudaMemcpyDeviceToDevice, stream));
    }
    const double l = loss_grad(xb.p, tb.p, batch, h, w);
    if (losses) losses[it] = l;
    adam(lr, 0.9f, 0.999f, 1e-8f);
  }
  GKB_CUDA(cudaStreamSynchronize(stream));
}

// ---------------------------------------------------------------------------
// the network as a coarse correction on a 2D MAC level
// ---------------------------------------------------------------------------

// image (ny, nx, 3): west u face and south v face of each cell scaled by
// sqrt(nx ny / ||b||^2), and log viscosity
template <typename T>
__global__ void k_mac_to_img(Lvl L, const T* __restrict__ b, const double* __restrict__ nrm, float* __restrict__ img) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= L.n[0] || j >= L.n[1]) return;
  const double nr2 = nrm[0];
  const double sc = nr2 > 0.0 ? sqrt((double)L.n[0] * L.n[1] / nr2) : 0.0;
  const long long c = cix(L, i, j, 0);
  float* o = img + ((long long)j * L.n[0] + i) * 3;
  o[0] = face_active<0>(L, i, j, 0) ? (float)((double)b[L.off[0] + c] * sc) : 0.f;
  o[1] = face_active<1>(L, i, j, 0) ? (float)((double)b[L.off[1] + c] * sc) : 0.f;
  const T* mu = MuPtr<T>::get(L);
  o[2] = (float)log(mu ? (double)mu[c] : L.mu0);
}

// x on every face of the level: the network output scaled back, zero on the
// faces that are not unknowns and on east / north boundary faces
template <typename T>
__global__ void k_img_to_mac(Lvl L, const float* __restrict__ y, const double* __restrict__ nrm, float inv_tscale,
                             T* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > L.n[0] || j > L.n[1]) return;
  const double nr2 = nrm[0];
  const double sc = nr2 > 0.0 ? sqrt(nr2 / ((double)L.n[0] * L.n[1])) * inv_tscale : 0.0;
  const long long c = cix(L, i, j, 0);
  const bool in = i < L.n[0] && j < L.n[1];
  if (j < L.n[1]) {  // u face (i, j), i <= nx
    const bool a = in && face_active<0>(L, i, j, 0);
    x[L.off[0] + c] = a ? (T)((double)y[((long long)j * L.n[0] + i) * 2 + 0] * sc) : (T)0;
  }
  if (i < L.n[0]) {  // v face (i, j), j <= ny
    const bool a = in && face_active<1>(L, i, j, 0);
    x[L.off[1] + c] = a ? (T)((double)y[((long long)j * L.n[0] + i) * 2 + 1] * sc) : (T)0;
  }
}

// (xs - xk) on the west u / south v face of every cell, scaled like k_mac_to_img
__global__ void k_err_to_img(Lvl L, const double* __restrict__ xs, const double* __restrict__ xk,
                             const double* __restrict__ nrm, float* __restrict__ img) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= L.n[0] || j >= L.n[1]) return;
  const double nr2 = nrm[0];
  const double sc = nr2 > 0.0 ? sqrt((double)L.n[0] * L.n[1] / nr2) : 0.0;
  const long long c = cix(L, i, j, 0);
  float* o = img + ((long long)j * L.n[0] + i) * 2;
  const long long cu = L.off[0] + c, cv = L.off[1] + c;
  o[0] = face_active<0>(L, i, j, 0) ? (float)((xs[cu] - xk[cu]) * sc) : 0.f;
  o[1] = face_active<1>(L, i, j, 0) ? (float)((xs[cv] - xk[cv]) * sc) : 0.f;
}

template <typename T>
void mac_to_img(const Lvl& L, const T* b, const double* nrm, float* img, cudaStream_t s) {
  ProfScope ps_(GKB_KC_UNET, s, (long long)L.n[0] * L.n[1]);
  k_mac_to_img<T><<<dim3((L.n[0] + 31) / 32, (L.n[1] + 7) / 8), dim3(32, 8), 0, s>>>(L, b, nrm, img);
  GKB_CUDA(cudaGetLastError());
}
template void mac_to_img<double>(const Lvl&, const double*, const double*, float*, cudaStream_t);
template void mac_to_img<float>(const Lvl&, const float*, const double*, float*, cudaStream_t);

void err_to_img(const Lvl& L, const double* xs, const double* xk, const double* nrm, float* img, cudaStream_t s) {
  ProfScope ps_(GKB_KC_UNET, s, (long long)L.n[0] * L.n[1]);
  k_err_to_img<<<dim3((L.n[0] + 31) / 32, (L.n[1] + 7) / 8), dim3(32, 8), 0, s>>>(L, xs, xk, nrm, img);
  GKB_CUDA(cudaGetLastError());
}

// x *= omega, omega = d[0] / d[1] when d[1] > 0, else 0
template <typename T>
__global__ void k_scale_step(T* __restrict__ x, long long n, const double* __restrict__ d) {
  const double den = d[1];
  const T w = (T)(den > 0.0 && isfinite(den) && isfinite(d[0]) ? d[0] / den : 0.0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    x[t] *= w;
}

template <typename T>
void unet_correct(Unet& U, UnetAct& A, const Lvl& L, const T* b, T* x, T* q, float* img_in, double* nrm,
                  const RedBuf& red, cudaStream_t s) {
  if (L.dim != 2) throw Error{GKB_ERR_INVALID_ARG, "the learned correction is 2D only"};
  Ops<T>::dot(L.nvel, b, b, red, FIN_STORE, nrm, s);
  const dim3 blk(32, 8);
  mac_to_img<T>(L, b, nrm, img_in, s);
  const float* y = U.forward(A, img_in, 1, L.n[1], L.n[0], true, s);
  {
    ProfScope ps_(GKB_KC_UNET, s, (long long)L.n[0] * L.n[1]);
    k_img_to_mac<T><<<dim3((L.n[0] + 32) / 32, (L.n[1] + 8) / 8), blk, 0, s>>>(L, y, nrm, 1.f / U.target_scale, x);
  }
  // energy-optimal step along the network's direction
  Ops<T>::apply(L, 1, x, q, s);
  Ops<T>::dot2(L.nvel, b, x, q, red, FIN_STORE, nrm + 4, s);
  {
    ProfScope ps_(GKB_KC_UNET, s, L.nvel);
    k_scale_step<T><<<grid_for(L.nvel), UT, 0, s>>>(x, L.nvel, nrm + 4);
  }
  GKB_CUDA(cudaGetLastError());
}

template void unet_correct<double>(Unet&, UnetAct&, const Lvl&, const double*, double*, double*, float*, double*,
                                   const RedBuf&, cudaStream_t);
template void unet_correct<float>(Unet&, UnetAct&, const Lvl&, const float*, float*, float*, float*, double*,
                                  const RedBuf&, cudaStream_t);

}  // namespace gkb

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

namespace {

template <class F>
int unet_guard(gkb_unet h, F&& fn) {
  if (!h) return GKB_ERR_INVALID_ARG;
  try {
    if (cudaSetDevice(h->device) != cudaSuccess) {
      (void)cudaGetLastError();
      return GKB_ERR_CUDA;
    }
    return fn();
  } catch (const gkb::Error& e) {
    h->last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    h->last_error = "host allocation failed";
    return GKB_ERR_OOM;
  } catch (...) {
    h->last_error = "unexpected internal error";
    return GKB_ERR_CUDA;
  }
}

bool dev_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int gkb_unet_create(gkb_unet* out, int c_in, int c1, int c2, int c_out, unsigned long long seed, void* stream) {
  if (!out) return GKB_ERR_INVALID_ARG;
  *out = nullptr;
  gkb_unet h = new (std::nothrow) gkb_unet_ctx();
  if (!h) return GKB_ERR_OOM;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete h;
    return GKB_ERR_CUDA;
  }
  int rc = unet_guard(h, [&] {
    h->u.init(c_in, c1, c2, c_out, seed, (cudaStream_t)stream);
    gkb::check_cuda(cudaStreamSynchronize((cudaStream_t)stream), "init");
    return GKB_OK;
  });
  if (rc != GKB_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return GKB_OK;
}

int gkb_unet_num_params(gkb_unet h, int64_t* n) {
  return unet_guard(h, [&] {
    if (!n) return GKB_ERR_INVALID_ARG;
    *n = h->u.nparams;
    return GKB_OK;
  });
}

int gkb_unet_get_params(gkb_unet h, float* params) {
  return unet_guard(h, [&] {
    if (!params) return GKB_ERR_INVALID_ARG;
    gkb::check_cuda(cudaMemcpyAsync(params, h->u.params.p, h->u.nparams * sizeof(float), cudaMemcpyDefault, h->u.stream), "copy");
    gkb::check_cuda(cudaStreamSynchronize(h->u.stream), "sync");
    return GKB_OK;
  });
}

int gkb_unet_set_params(gkb_unet h, const float* params) {
  return unet_guard(h, [&] {
    if (!params) return GKB_ERR_INVALID_ARG;
    gkb::check_cuda(cudaMemcpyAsync(h->u.params.p, params, h->u.nparams * sizeof(float), cudaMemcpyDefault, h->u.stream), "copy");
    gkb::check_cuda(cudaStreamSynchronize(h->u.stream), "sync");
    h->u.bf16_stale = true;
    return GKB_OK;
  });
}

int gkb_unet_forward(gkb_unet h, const float* x, int n, int hh, int w, float* y, int tensor_cores) {
  return unet_guard(h, [&] {
    if (!x || !y || !dev_ptr(x) || !dev_ptr(y)) throw gkb::Error{GKB_ERR_INVALID_ARG, "x and y must be device arrays"};
    const float* out = h->u.forward(h->u.act, x, n, hh, w, tensor_cores != 0, h->u.stream);
    gkb::check_cuda(cudaMemcpyAsync(y, out, (size_t)n * hh * w * h->u.c_out * sizeof(float), cudaMemcpyDeviceToDevice,
                                    h->u.stream), "copy");
    gkb::check_cuda(cudaStreamSynchronize(h->u.stream), "sync");
    return GKB_OK;
  });
}

int gkb_unet_loss_grad(gkb_unet h, const float* x, const float* target, int n, int hh, int w, double* loss, float* grad) {
  return unet_guard(h, [&] {
    if (!x || !target || !dev_ptr(x) || !dev_ptr(target)) throw gkb::Error{GKB_ERR_INVALID_ARG, "x and target must be device arrays"};
    const double l = h->u.loss_grad(x, target, n, hh, w);
    if (loss) *loss = l;
    if (grad) {
      gkb::check_cuda(cudaMemcpyAsync(grad, h->u.grads.p, h->u.nparams * sizeof(float), cudaMemcpyDefault, h->u.stream), "copy");
      gkb::check_cuda(cudaStreamSynchronize(h->u.stream), "sync");
    }
    return GKB_OK;
  });
}

int gkb_unet_adam_step(gkb_unet h, float lr, float beta1, float beta2, float eps) {
  return unet_guard(h, [&] {
    h->u.adam(lr, beta1, beta2, eps);
    gkb::check_cuda(cudaStreamSynchronize(h->u.stream), "sync");
    return GKB_OK;
  });
}

int gkb_unet_train(gkb_unet h, const float* x_img, const float* t_img, int64_t count, int hh, int w, int batch,
                   int steps, float lr, unsigned long long seed, double* losses) {
  return unet_guard(h, [&] {
    if (!x_img || !t_img || !dev_ptr(x_img) || !dev_ptr(t_img))
      throw gkb::Error{GKB_ERR_INVALID_ARG, "x_img and t_img must be device arrays"};
    h->u.ensure(h->u.act, batch < 1 ? 1 : batch, hh, w);
    h->u.train(x_img, t_img, count, hh, w, batch, steps, lr, seed, losses);
    return GKB_OK;
  });
}

int gkb_unet_set_target_scale(gkb_unet h, float s) {
  return unet_guard(h, [&] {
    if (!(s > 0) || !std::isfinite(s)) throw gkb::Error{GKB_ERR_INVALID_ARG, "target scale must be positive"};
    h->u.target_scale = s;
    return GKB_OK;
  });
}

int gkb_unet_get_target_scale(gkb_unet h, float* s) {
  return unet_guard(h, [&] {
    if (!s) return GKB_ERR_INVALID_ARG;
    *s = h->u.target_scale;
    return GKB_OK;
  });
}

const char* gkb_unet_last_error(gkb_unet h) { return h ? h->last_error.c_str() : "invalid handle"; }

int gkb_unet_destroy(gkb_unet h) {
  if (!h) return GKB_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  delete h;
  return GKB_OK;
}

}  // extern "C"
