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
// once per device; the symbol's name on the host is not a device address)
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

// compact ordering (include/gkb.h) <-> padded layout of one level
struct Box {
  int lo[3][3], ext[3][3];
  long long base[3], m;
};

Box make_box(const gkb::Lvl& L) {
  Box b{};
  long long off = 0;
  for (int c = 0; c < L.dim; ++c) {
    for (int a = 0; a < 3; ++a) {
      if (a >= L.dim) { b.lo[c][a] = 0; b.ext[c][a] = 1; continue; }
      if (a == c) {
        const int lo = L.nat[2 * a] ? 0 : 1, hi = L.nat[2 * a + 1] ? L.n[a] : L.n[a] - 1;
        b.lo[c][a] = lo;
        b.ext[c][a] = hi - lo + 1;
      } else {
        b.lo[c][a] = 0;
        b.ext[c][a] = L.n[a];
      }
    }
    b.base[c] = off;
    off += (long long)b.ext[c][0] * b.ext[c][1] * b.ext[c][2];
  }
  b.m = off;
  return b;
}

__device__ long long box_padded(const gkb::Lvl& L, const Box& b, long long t) {
  int c = 0;
  if (L.dim == 3 && t >= b.base[2]) c = 2;
  else if (t >= b.base[1]) c = 1;
  const long long l = t - b.base[c];
  const long long row = l / b.ext[c][0];
  const int i = (int)(l - row * b.ext[c][0]) + b.lo[c][0];
  const long long pl = row / b.ext[c][1];
  const int j = (int)(row - pl * b.ext[c][1]) + b.lo[c][1];
  const int k = (int)pl + b.lo[c][2];
  return L.off[c] + gkb::cix(L, i, j, k);
}

__device__ long long cell_padded(const gkb::Lvl& L, long long t) {
  const long long row = t / L.n[0];
  const int i = (int)(t - row * L.n[0]);
  const int k = (int)(row / L.n[1]);
  const int j = (int)(row - (long long)k * L.n[1]);
  return gkb::cix(L, i, j, k);
}

// dir 0: compact src -> padded dst; dir 1: padded src -> compact dst
__global__ void k_na_vel(gkb::Lvl L, Box b, int dir, const double* __restrict__ src, double* __restrict__ dst) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < b.m; t += (long long)gridDim.x * blockDim.x) {
    const long long p = box_padded(L, b, t);
    if (dir == 0) dst[p] = src[t];
    else dst[t] = src[p];
  }
}

__global__ void k_na_cell(gkb::Lvl L, int dir, const double* __restrict__ src, double* __restrict__ dst) {
  const long long n = (long long)L.n[0] * L.n[1] * L.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long p = cell_padded(L, t);
    if (dir == 0) dst[p] = src[t];
    else dst[t] = src[p];
  }
}

unsigned blocks_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 4096) b = 4096;
  return (unsigned)(b < 1 ? 1 : b);
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
  const Box b = make_box(L);
  const long long ncells = (long long)n3[0] * n3[1] * n3[2];
  const bool in_cells = (op == GKB_OP_A), out_cells = (op == GKB_OP_AT);
  // the previous call's contents remain in the array: clear the input's
  // padding, which the operator kernels read as zero
  if (cudaMemsetAsync(in, 0, (in_cells ? L.ncell : L.nvel) * sizeof(double), s) != cudaSuccess) {
    (void)cudaGetLastError();
    return GKB_ERR_CUDA;
  }
  if (in_cells) k_na_cell<<<blocks_for(ncells), 256, 0, s>>>(L, 0, x, in);
  else k_na_vel<<<blocks_for(b.m), 256, 0, s>>>(L, b, 0, x, in);
  switch (op) {
    case GKB_OP_W: gkb::Ops<double>::apply(L, 0, in, out, s); break;
    case GKB_OP_M: gkb::Ops<double>::apply(L, 1, in, out, s); break;
    case GKB_OP_A: gkb::Ops<double>::grad(L, in, out, 1.0, s); break;
    default: gkb::Ops<double>::negdiv(L, in, out, 1.0, s); break;
  }
  if (out_cells) k_na_cell<<<blocks_for(ncells), 256, 0, s>>>(L, 1, out, y);
  else k_na_vel<<<blocks_for(b.m), 256, 0, s>>>(L, b, 1, out, y);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return GKB_ERR_CUDA;
  }
  return GKB_OK;
}
