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

// activations of one forward pass (NHWC), sized for (n, h, w); a solver
// owns its own so that the buffers its captured graphs read never move
struct UnetAct {
  int n = 0, h = 0, w = 0;
  DevBuf<float> a1, s1, p1, b1, s2, p2, c1a, c2a, d1, e1, y;
};

struct Unet {
  int c_in = 3, c1 = 16, c2 = 32, c_out = 2;
  std::vector<ConvLayer> layers;
  long long nparams = 0;
  cudaStream_t stream = nullptr;
  DevBuf<float> params, grads, adam_m, adam_v;
  DevBuf<__nv_bfloat16> params_bf16;  // tensor-core copy of the weights (fixed address)
  bool bf16_stale = true;
  long long adam_t = 0;
  float target_scale = 1.f;           // the network is trained on target_scale * e^
  UnetAct act;                        // activations of the entry points' own calls
  // backward scratch
  int gn = 0, gh = 0, gw = 0;
  DevBuf<float> g_full0, g_full1, g_half0, g_half1, g_q0, g_q1, g_e;
  DevBuf<float> wpart;                  // per-block partial weight gradients
  DevBuf<double> red_partial;
  DevBuf<unsigned int> red_ticket;
  DevBuf<double> loss_dev;
  DevBuf<float> xb, tb;                 // training minibatch

  void init(int cin, int k1, int k2, int cout, unsigned long long seed, cudaStream_t s);
  // size the activations of A for (n, h, w) (no-op when unchanged)
  void ensure(UnetAct& A, int n, int h, int w) const;
  void refresh_bf16(cudaStream_t s);
  // y = N(x) for NHWC x (n, h, w, c_in); returns A.y (n, h, w, c_out)
  const float* forward(UnetAct& A, const float* x, int n, int h, int w, bool tensor_cores, cudaStream_t s);
  // loss = (1/n) sum over the samples of ||N(x) - target_scale t||^2; gradient into grads
  double loss_grad(const float* x, const float* t, int n, int h, int w);
  void adam(float lr, float beta1, float beta2, float eps);
  // `steps` Adam steps on minibatches of `batch` pairs drawn without
  // replacement (reshuffled every pass) from count pairs (x_img, t_img)
  void train(const float* x_img, const float* t_img, long long count, int h, int w, int batch, int steps, float lr,
             unsigned long long seed, double* losses);
};

// image (ny, nx, 3) of a 2D level vector b: the west u face and the south v
// face of every cell scaled by sqrt(nx ny / nrm[0]) (0 when nrm[0] = 0), and
// log viscosity
template <typename T>
void mac_to_img(const Lvl& L, const T* b, const double* nrm, float* img, cudaStream_t s);
// image (ny, nx, 2) of (xs - xk) scaled by sqrt(nx ny / nrm[0]), same faces
void err_to_img(const Lvl& L, const double* xs, const double* xk, const double* nrm, float* img, cudaStream_t s);

// Learned coarse correction on a 2D level: z = (||b|| / sqrt(nx ny)) /
// target_scale * N(b^, log mu) with b^ = b sqrt(nx ny) / ||b|| (z = 0 for b = 0),
// through the images img_in (ny, nx, 3) / A.y (ny, nx, 2), then scaled by the
// energy-optimal step: x = omega z, omega = (b, z) / (z, M z) (0 unless
// (z, M z) > 0), so that the correction never increases the M-norm error of
// the level system. q: level-sized scratch (M z); nrm: device double[8].
template <typename T>
void unet_correct(Unet& U, UnetAct& A, const Lvl& L, const T* b, T* x, T* q, float* img_in, double* nrm,
                  const RedBuf& red, cudaStream_t s);

}  // namespace gkb

// the network behind the C ABI handle
struct gkb_unet_ctx {
  gkb::Unet u;
  int device = 0;
  std::string last_error = "no error";
};
