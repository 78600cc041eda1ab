// noalloc.cu - gkb_apply_noalloc: the operator product of gkb_apply without
// a handle and without any device allocation.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// another allocator (a framework's caching allocator or a fixed arena that
// forbids raw allocations), and latency-critical loops where cudaMalloc and
// cudaFree would synchronise the device. gkb_apply needs a handle whose
// gkb_set_problem allocates the padded work arrays; this entry point keeps
// those two padded arrays in one file-scope device array instead, so a call
// allocates nothing. The array is part of the module: every GPU that loads
// the library holds it until the process exits.
#include <mutex>

#include "../../include/gkb.h"
#include "common.cuh"
#include "ops.h"
#include "solver.cuh"

namespace {

// two padded work arrays of GKB_NOALLOC_MAX_ELEMS doubles each
__device__ __align__(256) double g_noalloc_scratch[2 * (size_t)GKB_NOALLOC_MAX_ELEMS];

std::mutex g_noalloc_mutex;
double* g_noalloc_addr[64] = {};

// host-side address of the scratch array on the current device (looked up
// once per device and process; the symbol's name on the host is not a device
// address). A cudaDeviceReset reloads the module, possibly elsewhere, so the
// cached address does not survive one.
int noalloc_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    (void)cudaGetLastError();
    return GKB_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return GKB_ERR_CUDA;
    }
    g_noalloc_addr[dev] = (double*)p;
  }
  *out = g_noalloc_addr[dev];
  return GKB_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int gkb_apply_noalloc(const gkb_grid* grid, double mu0, double gamma, double n_scale, int op,
                                 const double* x, double* y, void* stream) {
  if (!grid || !x || !y) return GKB_ERR_INVALID_ARG;
  if (grid->dim != 2 && grid->dim != 3) return GKB_ERR_INVALID_ARG;
  for (int a = 0; a < grid->dim; ++a)
    if (grid->n[a] < 2) return GKB_ERR_INVALID_ARG;
  for (int s = 0; s < 2 * grid->dim; ++s)
    if (grid->bc[s] != GKB_BC_DIRICHLET && grid->bc[s] != GKB_BC_NATURAL) return GKB_ERR_INVALID_ARG;
  if (!(grid->h > 0) || !(mu0 > 0) || !(gamma >= 0)) return GKB_ERR_INVALID_ARG;
  if (op != GKB_OP_W && op != GKB_OP_A && op != GKB_OP_AT && op != GKB_OP_M) return GKB_ERR_INVALID_ARG;
  if (!on_device(x) || !on_device(y)) return GKB_ERR_INVALID_ARG;
  const int dim = grid->dim;
  int nat[6] = {0, 0, 0, 0, 0, 0};
  for (int s = 0; s < 2 * dim; ++s) nat[s] = grid->bc[s] == GKB_BC_NATURAL;
  int n3[3] = {grid->n[0], grid->n[1], dim == 3 ? grid->n[2] : 1};
  const double ns = (n_scale > 0) ? n_scale : pow(grid->h, dim);
  gkb::Lvl L = gkb::make_level(dim, n3, grid->h, nat, gamma / ns);
  L.mu0 = mu0;
  gkb::finish_level(L);
  // both padded arrays must fit the static scratch
  if (L.nvel > (long long)GKB_NOALLOC_MAX_ELEMS || L.ncell > (long long)GKB_NOALLOC_MAX_ELEMS)
    return GKB_ERR_INVALID_ARG;
  double* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != GKB_OK) return rc;
  double* in = scratch;
  double* out = scratch + (size_t)GKB_NOALLOC_MAX_ELEMS;
  cudaStream_t s = (cudaStream_t)stream;
  const bool in_cells = (op == GKB_OP_A), out_cells = (op == GKB_OP_AT);
  // the previous call's contents remain in the array: clear the input's
  // padding, which the operator kernels read as zero
  if (cudaMemsetAsync(in, 0, (in_cells ? L.ncell : L.nvel) * sizeof(double), s) != cudaSuccess) {
    (void)cudaGetLastError();
    return GKB_ERR_CUDA;
  }
  if (in_cells) gkb::pack_cells(L, x, in, s);
  else gkb::pack_velocity(L, x, in, s);
  switch (op) {
    case GKB_OP_W: gkb::Ops<double>::apply(L, 0, in, out, s); break;
    case GKB_OP_M: gkb::Ops<double>::apply(L, 1, in, out, s); break;
    case GKB_OP_A: gkb::Ops<double>::grad(L, in, out, 1.0, s); break;
    default: gkb::Ops<double>::negdiv(L, in, out, 1.0, s); break;
  }
  if (out_cells) gkb::unpack_cells(L, out, y, s);
  else gkb::unpack_velocity(L, out, y, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return GKB_ERR_CUDA;
  }
  return GKB_OK;
}
