// FP64 instantiation of the MAC stencil / multigrid / BLAS-1 kernels.
#define KT double
#include "kernels_inst.cuh"
#if GKB_PART == 0 || GKB_PART == 5
namespace gkb {
long long blas_blocks(long long len) {
  long long b = (len + 256LL * 8 - 1) / (256LL * 8);
  if (b > 1216) b = 1216;
  return b < 1 ? 1 : b;
}
}  // namespace gkb
#endif
