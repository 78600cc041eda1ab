// FP32 instantiation of the MAC stencil / multigrid / BLAS-1 kernels.
#define KT float
#include "kernels_inst.cuh"
