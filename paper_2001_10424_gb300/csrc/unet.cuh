// unet.cuh - the learned preconditioner: a 3-level convolutional U-Net with
// forward, backward and Adam kernels (training and inference on the device).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "reduce.cuh"
#include "solver.cuh"

namespace gkb {

// one convolution: weights [3][3][cin][cout] then bias[cout] in the flat
// parameter vector, starting at `off`
struct ConvLayer {
  int cin, cout;
  long long off;
  long long nw() const { return 9LL * cin * cout; }
};

struct Unet {
  int c_in = 3, c1 = 16, c2 = 32, c_out = 2;
  std::vector<ConvLayer> layers;
  long long nparams = 0;
  cudaStream_t stream = nullptr;
  DevBuf<float> params, grads, adam_m, adam_v;
  DevBuf<__nv_bfloat16> params_bf16;  // tensor-core copy of the weights
  bool bf16_stale = true;
  long long adam_t = 0;
  // activations of the last forward (NHWC), sized for (n, h, w)
  int an = 0, ah = 0, aw = 0;
  DevBuf<float> a1, s1, p1, b1, s2, p2, c1a, c2a, d1, e1, y;
  // backward scratch
  DevBuf<float> g_full0, g_full1, g_half0, g_half1, g_q0, g_q1, g_e;
  DevBuf<float> wpart;                  // per-block partial weight gradients
  DevBuf<double> red_partial;
  DevBuf<unsigned int> red_ticket;
  DevBuf<double> loss_dev;

  void init(int cin, int k1, int k2, int cout, unsigned long long seed, cudaStream_t s);
  void ensure(int n, int h, int w);
  // y = N(x) for NHWC x (n, h, w, c_in); returns the output buffer (n, h, w, c_out)
  const float* forward(const float* x, int n, int h, int w, bool tensor_cores);
  // loss = (1/n) sum over the samples of ||N(x) - t||^2; gradient into grads
  double loss_grad(const float* x, const float* t, int n, int h, int w);
  void adam(float lr, float beta1, float beta2, float eps);
};

}  // namespace gkb
