// lockstep.cuh - lock-step batched solve (lockstep.cu): one CUDA graph in
// which every step of the solve is one launch over all problems of a batch.
#pragma once
#include <cuda_runtime.h>

#include "../../include/gkb.h"

namespace gkb {

struct Solver;

// true when the batch can run in lock-step: 2D, constant viscosity, the
// Laplacian viscous form, N = n_scale I, GMG-PCG inner solves, and the same
// precision, smoother degree and iteration limits in every problem
bool lockstep_eligible(Solver* const* S, int count);

class Lockstep {
 public:
  // captures the batch's graph on the private capture streams of S[0]
  Lockstep(Solver* const* S, int count, cudaStream_t cap1, cudaStream_t cap2, cudaStream_t cap3);
  ~Lockstep();
  Lockstep(const Lockstep&) = delete;
  Lockstep& operator=(const Lockstep&) = delete;
  // one launch of the whole batched solve on stream s (inputs and states
  // staged by each handle beforehand)
  void launch(cudaStream_t s);
  // kernel launches of the last solve, by kernel class (synchronises s)
  void launch_counts(cudaStream_t s, long long out[GKB_KC_COUNT]);

 private:
  struct Impl;
  Impl* I = nullptr;
};

}  // namespace gkb
