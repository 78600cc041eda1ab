// reduce.cuh - deterministic grid-wide reductions with a fused finaliser.
//
// Every block reduces its values (warp shuffles, then shared memory) and
// writes one partial per value; the last block to arrive (atomic ticket)
// sums the partials in a fixed order and runs the finaliser, which updates
// the solver scalars on the device. The order of every addition depends only
// on the launch shape, so results are bitwise reproducible run to run.
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"
#include "state.cuh"

namespace gkb {

struct RedBuf {
  double* partial;        // >= max blocks * 4 doubles
  unsigned int* ticket;   // one counter, zero between launches
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// All threads of every block of the problem's grid B must call this exactly
// once.
template <int NV>
__device__ void grid_reduce(double (&v)[NV], RedBuf red, int fin, void* st, const Blk& B) {
  __shared__ double sh[NV][32];
  __shared__ bool am_last;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const int lane = tid & 31, warp = tid >> 5, nwarp = (nthr + 31) >> 5;
  const unsigned bid = B.x + B.nx * (B.y + B.ny * B.z);
  const unsigned nblk = B.nx * B.ny * B.nz;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = warp_sum(v[i]);
    if (lane == 0) sh[i][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = warp_sum(lane < nwarp ? sh[i][lane] : 0.0);
      if (lane == 0) red.partial[(size_t)bid * NV + i] = s;
    }
  }
  if (tid == 0) {
    __threadfence();
    unsigned t = atomicAdd(red.ticket, 1u);
    am_last = (t == nblk - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double tot[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = 0.0;
    for (unsigned b = tid; b < nblk; b += nthr) s += __ldcg(red.partial + (size_t)b * NV + i);
    tot[i] = s;
  }
  __syncthreads();  // sh reuse
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = warp_sum(tot[i]);
    if (lane == 0) sh[i][warp] = s;
  }
  __syncthreads();
  if (tid == 0) {
    double fin_v[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = 0.0;
      for (int w = 0; w < nwarp; ++w) s += sh[i][w];
      fin_v[i] = s;
    }
    finalize(fin, fin_v, st);
    *red.ticket = 0u;
  }
}

// the same over the launch's own grid
template <int NV>
__device__ __forceinline__ void grid_reduce(double (&v)[NV], RedBuf red, int fin, void* st) {
  grid_reduce<NV>(v, red, fin, st, native_blk());
}

}  // namespace gkb
