// tail.cu - the coarse end of a 2D constant-viscosity V-cycle as one kernel.
//
// Below some level every launch of the V-cycle (smoothing steps, residuals,
// the two restriction passes, the dense coarse solve, prolongation) is a
// chain of dependent memory round trips whose cost does not fall with the
// level's size. Here one thread-block cluster runs all of those steps, each
// over the virtual blocks of the launch it replaces (the same device bodies,
// so every value is computed by the same operations), with a hardware
// cluster barrier between steps instead of a kernel boundary.
//
// The steps write arrays that later steps read inside the same kernel, so
// this unit compiles the bodies with plain coherent loads (never the
// read-only path) and without restrict; the cluster barrier's release /
// acquire orders the global writes of one step before the reads of the next.
#define GKB_LDG(p) (*(p))
#define GKB_RESTRICT
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "kernels_impl.cuh"
#include "solver.cuh"

namespace gkb {

constexpr int TAIL_MAX_LEVELS = 8;
constexpr int TAIL_MAX_DEG = 4;

template <typename T>
struct TailLevel {
  Lvl L;
  T* x;
  T* b;
  T* r;
  T* d;
  const T* table;
  int use2;                    // class-stencil smoother (k_cheb2's body), else the patch walk
  T ca[TAIL_MAX_DEG], cb[TAIL_MAX_DEG];
  Fold2In<T> f[TAIL_MAX_DEG];  // interior stencils scaled by ca[k]
};

template <typename T>
struct TailPlan {
  int nl;       // levels of the tail; the last is the coarsest
  int degree;
  int m;        // coarse unknowns
  const T* Minv;
  const int* idx;
  TailLevel<T> lev[TAIL_MAX_LEVELS];
};

template <typename T>
__global__ void __launch_bounds__(BX* BY) k_vtail(const TailPlan<T>* P) {
  namespace cgx = cooperative_groups;
  cgx::cluster_group cl = cgx::this_cluster();
  const unsigned rank = cl.block_rank(), cs = cl.num_blocks();
  const int nl = P->nl, deg = P->degree;
  // one step: the blocks of a gx x gy launch spread over the cluster, then
  // the cluster barrier (every block of the cluster reaches it once). The
  // bodies were written for one block per launch and may leave their shared
  // tiles in use when they return, hence a block barrier after each.
  auto over = [&](unsigned gx, unsigned gy, auto&& body) {
    for (unsigned vb = rank; vb < gx * gy; vb += cs) {
      const Blk B{vb % gx, vb / gx, 0u, gx, gy, 1u};
      body(B);
      __syncthreads();
    }
    cl.sync();
  };
  auto residual = [&](const TailLevel<T>& V) {
    const Lvl& L = V.L;
    over((L.n[0] + 1 + BX - 1) / BX, (L.n[1] + 1 + BY - 1) / BY, [&](const Blk& B) {
      mac_tile_body<T, false, 0, false>(B, L, 0, V.x, V.b, V.r, RedBuf{nullptr, nullptr}, 0, nullptr, nullptr);
    });
  };
  auto smooth = [&](const TailLevel<T>& V, bool x_zero) {
    const Lvl& L = V.L;
    for (int k = 0; k < deg; ++k) {
      const bool first = (k == 0 && x_zero);
      if (!first) residual(V);
      const T* r = first ? V.b : V.r;
      over((L.n[0] + 1 + BX - 1) / BX, (L.n[1] + 1 + BY - 1) / BY, [&](const Blk& B) {
        if (V.use2) cheb2_body<T>(B, L, r, V.x, V.d, V.ca[k], V.cb[k], first ? 1 : 0, V.table, V.f[k]);
        else cheb_body<T, false>(B, L, r, V.x, V.d, V.ca[k], V.cb[k], first ? 1 : 0, V.table);
      });
    }
  };
  for (int l = 0; l + 1 < nl; ++l) {
    const TailLevel<T>& F = P->lev[l];
    const TailLevel<T>& C = P->lev[l + 1];
    smooth(F, true);
    residual(F);
    const unsigned gx = (C.L.n[0] + 1 + BX - 1) / BX, gy = (C.L.n[1] + 1 + BY - 1) / BY;
    over(gx, gy, [&](const Blk& B) { restrict_flux2d_a_body<T>(B, F.L, C.L, F.r, C.b, C.x); });
    over(gx, gy, [&](const Blk& B) { restrict_flux2d_b_body<T>(B, C.L, C.x, C.b); });
  }
  {  // the dense coarse solve: one warp per row as k_coarse_solve, 8 rows per block
    const TailLevel<T>& C = P->lev[nl - 1];
    const int m = P->m;
    const T* Minv = P->Minv;
    const int* idx = P->idx;
    over((unsigned)((m + BY - 1) / BY), 1u, [&](const Blk& B) {
      const int row = (int)B.x * BY + threadIdx.y, lane = threadIdx.x;
      if (row < m) {  // uniform over the warp
        double acc = 0.0;
        const T* rw = Minv + (size_t)row * m;
        for (int c = lane; c < m; c += 32) acc += (double)rw[c] * (double)C.b[idx[c]];
        acc = warp_sum(acc);
        if (lane == 0) C.x[idx[row]] = (T)acc;
      }
    });
  }
  for (int l = nl - 2; l >= 0; --l) {
    const TailLevel<T>& F = P->lev[l];
    const TailLevel<T>& C = P->lev[l + 1];
    over((C.L.n[0] + 1 + BX - 1) / BX, (C.L.n[1] + 1 + BY - 1) / BY,
         [&](const Blk& B) { prolong_flux2d_body<T>(B, F.L, C.L, C.x, F.x); });
    smooth(F, false);
  }
}

namespace {

// cluster size of k_vtail<T>: 16 blocks where the device allows it, else 8
template <typename T>
int tail_cluster_size() {
  static std::mutex mtx;
  static std::map<int, int> cached;
  int dev = 0;
  GKB_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mtx);
  int& cs = cached[dev];
  if (cs) return cs;
  const void* fn = (const void*)k_vtail<T>;
  cs = 8;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(BX, BY);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n >= 1) cs = 16;
  }
  (void)cudaGetLastError();
  return cs;
}

}  // namespace

template <typename T>
void gmg_tail_setup(Gmg<T>& G, int side, cudaStream_t s) {
  G.tail_level = -1;
  const int nl = (int)G.lev.size();
  if (side <= 0 || nl < 2 || G.lev[0].L.dim != 2 || G.degree > TAIL_MAX_DEG) return;
  int lt = -1;
  for (int l = 1; l < nl; ++l)
    if (std::max(G.lev[l].L.n[0], G.lev[l].L.n[1]) <= side) { lt = l; break; }
  if (lt < 0 || nl - lt > TAIL_MAX_LEVELS) return;
  TailPlan<T> P{};
  P.nl = nl - lt;
  P.degree = G.degree;
  P.m = G.coarse_m;
  P.Minv = G.coarse_inv.p;
  P.idx = G.coarse_idx.p;
  for (int l = lt; l < nl; ++l) {
    auto& V = G.lev[l];
    if (V.L.mu64 || V.L.mu32) return;  // variable viscosity: not fused
    TailLevel<T>& TL = P.lev[l - lt];
    TL.L = V.L;
    TL.x = V.x.p;
    TL.b = V.b.p;
    TL.r = V.r.p;
    TL.d = V.d.p;
    TL.table = V.table.p;
    if (l == nl - 1) continue;  // the coarsest level is solved, not smoothed: no coefficients
    if ((int)V.ca.size() < G.degree || (int)V.cb.size() < G.degree) return;
    TL.use2 = (!V.fold_in.empty() && V.table.p && cheb2_level(V.L)) ? 1 : 0;
    for (int k = 0; k < G.degree; ++k) {
      TL.ca[k] = (T)V.ca[k];
      TL.cb[k] = (T)V.cb[k];
      if (TL.use2) TL.f[k] = fold2_scaled<T>(V.fold_in.data(), (double)(T)V.ca[k]);
    }
  }
  G.tail_buf.alloc(sizeof(TailPlan<T>));
  GKB_CUDA(cudaMemcpyAsync(G.tail_buf.p, &P, sizeof(P), cudaMemcpyHostToDevice, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  G.tail_cs = tail_cluster_size<T>();
  G.tail_level = lt;
}

template <typename T>
void gmg_tail_launch(const Gmg<T>& G, cudaStream_t s) {
  long long work = 0;
  for (size_t l = G.tail_level; l < G.lev.size(); ++l) work += lvl_unknowns(G.lev[l].L);
  ProfScope ps_(GKB_KC_COARSE, s, work);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = G.tail_cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(G.tail_cs);
  cfg.blockDim = dim3(BX, BY);
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  GKB_CUDA(cudaLaunchKernelEx(&cfg, k_vtail<T>, (const TailPlan<T>*)G.tail_buf.p));
}

template void gmg_tail_setup<float>(Gmg<float>&, int, cudaStream_t);
template void gmg_tail_setup<double>(Gmg<double>&, int, cudaStream_t);
template void gmg_tail_launch<float>(const Gmg<float>&, cudaStream_t);
template void gmg_tail_launch<double>(const Gmg<double>&, cudaStream_t);

}  // namespace gkb
