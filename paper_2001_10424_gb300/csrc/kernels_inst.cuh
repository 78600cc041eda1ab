// kernels_inst.cuh - launch wrappers, instantiated for KT (see kernels_f64.cu).
//
// GKB_PART selects one group of wrappers so that the build can compile the
// heavy stencil and smoother instantiations as separate, parallel units:
// 1 operator products, 2 residuals, 3 Chebyshev steps, 4 patch smoother,
// 5 transfers, coarse solve and BLAS-1, 6 / 7 the variable-viscosity
// Chebyshev / patch smoother; 0 (default) all of them.
#pragma once
#include "kernels_impl.cuh"
#include "prof.h"

#ifndef GKB_PART
#define GKB_PART 0
#endif
#define GKB_IN_PART(k) (GKB_PART == 0 || GKB_PART == (k))

namespace gkb {

#define GKB_VARMU(L) ((sizeof(KT) == 8) ? (L.mu64 != nullptr) : (L.mu32 != nullptr))

#if GKB_IN_PART(1)
template <>
long long Ops<KT>::face_blocks(const Lvl& L) {
  dim3 g = face_grid(L);
  return (long long)g.x * g.y * g.z;
}

template <>
void Ops<KT>::apply(const Lvl& L, int mode, const KT* x, KT* y, cudaStream_t s) {
  ProfScope ps_(GKB_KC_APPLY, s, lvl_unknowns(L));
  RedBuf red{nullptr, nullptr};
  const int wonly = (mode == 0);
  if (mac3_level(L) && !GKB_VARMU(L) && x) k_mac3<KT, 1, false><<<mac3_grid(L), dim3(BX, BY), 0, s>>>(L, wonly, x, nullptr, y, red, 0, nullptr);
  else if (GKB_VARMU(L)) k_mac_tile<KT, true, 1, false><<<face_grid(L), dim3(BX, BY), 0, s>>>(L, wonly, x, nullptr, y, red, 0, nullptr, nullptr);
  else k_mac_tile<KT, false, 1, false><<<face_grid(L), dim3(BX, BY), 0, s>>>(L, wonly, x, nullptr, y, red, 0, nullptr, nullptr);
}

template <>
void Ops<KT>::apply_dot(const Lvl& L, int mode, const KT* x, KT* y, const RedBuf& red, int fin, void* st,
                        cudaStream_t s) {
  ProfScope ps_(GKB_KC_APPLY, s, lvl_unknowns(L));
  const int wonly = (mode == 0);
  if (mac3_level(L) && !GKB_VARMU(L) && x) k_mac3<KT, 1, true><<<mac3_grid(L), dim3(BX, BY), 0, s>>>(L, wonly, x, nullptr, y, red, fin, st);
  else if (GKB_VARMU(L)) k_mac_tile<KT, true, 1, true><<<face_grid(L), dim3(BX, BY), 0, s>>>(L, wonly, x, nullptr, y, red, fin, st, nullptr);
  else k_mac_tile<KT, false, 1, true><<<face_grid(L), dim3(BX, BY), 0, s>>>(L, wonly, x, nullptr, y, red, fin, st, nullptr);
}
#endif

#if GKB_IN_PART(2)
template <>
void Ops<KT>::residual(const Lvl& L, const KT* x, const KT* b, KT* r, cudaStream_t s, const int* pred) {
  ProfScope ps_(GKB_KC_RESIDUAL, s, lvl_unknowns(L));
  RedBuf red{nullptr, nullptr};
  if (mac3_level(L) && !GKB_VARMU(L) && x && !pred) k_mac3<KT, 0, false><<<mac3_grid(L), dim3(BX, BY), 0, s>>>(L, 0, x, b, r, red, 0, nullptr);
  else if (GKB_VARMU(L)) k_mac_tile<KT, true, 0, false><<<face_grid(L), dim3(BX, BY), 0, s>>>(L, 0, x, b, r, red, 0, nullptr, pred);
  else k_mac_tile<KT, false, 0, false><<<face_grid(L), dim3(BX, BY), 0, s>>>(L, 0, x, b, r, red, 0, nullptr, pred);
}
#endif

// variable-viscosity smoother launches, compiled in their own units (6, 7)
void launch_cheb_varmu(const Lvl& L, const KT* r, KT* x, KT* d, KT ca, KT cb, int x_zero, const KT* vtab,
                       cudaStream_t s);
void launch_patch_varmu(const Lvl& L, const KT* r, KT* z, const KT* vtab, cudaStream_t s);

#if GKB_IN_PART(3)
template <>
void Ops<KT>::cheb(const Lvl& L, const KT* r, KT* x, KT* d, KT ca, KT cb, int x_zero, const KT* table,
                   cudaStream_t s, const double* fold_in) {
  ProfScope ps_(GKB_KC_SMOOTH, s, lvl_unknowns(L));
  if (GKB_VARMU(L)) {
    launch_cheb_varmu(L, r, x, d, ca, cb, x_zero, table, s);
  } else if (fold_in && table && cheb3_level(L)) {
    Fold3In<KT> f;
    for (int c = 0; c < 3; ++c)
      for (int q = 0; q < 13; ++q) f.c[c][q] = (KT)fold_in[c * 16 + q];
    if (cheb3s_level(L)) k_cheb3s<KT><<<cheb3s_grid(L), dim3(BX, BY), 0, s>>>(L, r, x, d, ca, cb, x_zero, table, f);
    else k_cheb3<KT><<<cheb3_grid(L), dim3(BX, BY), 0, s>>>(L, r, x, d, ca, cb, x_zero, table, f);
  } else if (fold_in && table && cheb2_level(L)) {
    const Fold2In<KT> f = fold2_scaled<KT>(fold_in, (double)ca);
    k_cheb2<KT><<<face_grid(L), dim3(BX, BY), 0, s>>>(L, r, x, d, ca, cb, x_zero, table, f);
  } else {
    k_cheb<KT, false><<<face_grid(L), dim3(BX, BY), 0, s>>>(L, r, x, d, ca, cb, x_zero, table);
  }
}
#endif

#if GKB_IN_PART(6)
void launch_cheb_varmu(const Lvl& L, const KT* r, KT* x, KT* d, KT ca, KT cb, int x_zero, const KT* vtab,
                       cudaStream_t s) {
  k_cheb<KT, true><<<face_grid(L), dim3(BX, BY), 0, s>>>(L, r, x, d, ca, cb, x_zero, vtab);
}
#endif

#if GKB_IN_PART(7)
void launch_patch_varmu(const Lvl& L, const KT* r, KT* z, const KT* vtab, cudaStream_t s) {
  k_patch<KT, true><<<face_grid(L), dim3(BX, BY), 0, s>>>(L, r, z, vtab);
}
#endif

#if GKB_IN_PART(4)
template <>
void Ops<KT>::patch(const Lvl& L, const KT* r, KT* z, const KT* table, cudaStream_t s) {
  ProfScope ps_(GKB_KC_SMOOTH, s, lvl_unknowns(L));
  if (GKB_VARMU(L)) launch_patch_varmu(L, r, z, table, s);
  else k_patch<KT, false><<<face_grid(L), dim3(BX, BY), 0, s>>>(L, r, z, table);
}

template <>
long long Ops<KT>::patch_table_len(const Lvl& L) {
  // class inverses, the 3D interior stencils, then the 3D class stencils
  if (!GKB_VARMU(L)) return FOLD3_OFF + 48LL * (L.dim == 3 ? FOLD3_CLASSES : FOLD2_CLASSES);
  return (L.dim == 3 ? 3 : 1) * 10 * vtab_plane(L);
}

template <>
long long Ops<KT>::fold_interior_offset(const Lvl& L) {
  if (GKB_VARMU(L)) return -1;
  if (cheb3_level(L)) return FOLD3_OFF + 48LL * FOLD3_INTERIOR;
  if (cheb2_level(L)) return FOLD3_OFF + 48LL * FOLD2_INTERIOR;
  return -1;
}

template <>
void Ops<KT>::patch_table(const Lvl& L, KT* table, cudaStream_t s) {
  ProfScope ps_(GKB_KC_LAYOUT, s, 0);
  if (!GKB_VARMU(L)) {
    k_patch_table<KT><<<1, 256, 0, s>>>(L, table);
    if (L.dim == 3) {
      k_patch_fold<KT><<<1, 32, 0, s>>>(L, table);
      k_fold3_table<KT><<<(FOLD3_CLASSES * 3 + 127) / 128, 128, 0, s>>>(L, table);
    } else {
      k_fold2_table<KT><<<1, 128, 0, s>>>(L, table);
    }
    return;
  }
  // variable viscosity: the per-patch inverses (entries never written stay 0)
  cudaMemsetAsync(table, 0, patch_table_len(L) * sizeof(KT), s);
  const dim3 blk(32, 8);
  const dim3 g((L.n[0] + 1 + 31) / 32, (L.n[1] + 1 + 7) / 8, L.dim == 3 ? L.n[2] + 1 : 1);
  if (L.dim == 2) {
    k_patch_vtab<KT, 2><<<g, blk, 0, s>>>(L, table);
  } else {
    k_patch_vtab<KT, 0><<<g, blk, 0, s>>>(L, table);
    k_patch_vtab<KT, 1><<<g, blk, 0, s>>>(L, table);
    k_patch_vtab<KT, 2><<<g, blk, 0, s>>>(L, table);
  }
}
#endif

#if GKB_IN_PART(5)
template <>
long long Ops<KT>::edge_table_len(const Lvl& L) {
  return (L.dim == 3 ? 3 : 1) * em_plane(L);
}

template <>
void Ops<KT>::edge_table(const Lvl& L, KT* em, cudaStream_t s) {
  ProfScope ps_(GKB_KC_LAYOUT, s);
  const dim3 g((L.n[0] + 1 + 31) / 32, (L.n[1] + 1 + 7) / 8, L.dim == 3 ? L.n[2] + 1 : 1);
  k_edge_mu<KT><<<g, dim3(32, 8), 0, s>>>(L, em);
}

template <>
void Ops<KT>::grad(const Lvl& L, const KT* p, KT* y, KT scale, cudaStream_t s) {
  ProfScope ps_(GKB_KC_LAYOUT, s, lvl_unknowns(L));
  k_grad<KT><<<face_grid(L), dim3(BX, BY), 0, s>>>(L, p, y, scale);
}

template <>
void Ops<KT>::negdiv(const Lvl& L, const KT* x, KT* y, KT scale, cudaStream_t s) {
  ProfScope ps_(GKB_KC_LAYOUT, s, lvl_unknowns(L));
  k_negdiv<KT><<<cell_grid(L), dim3(BX, BY), 0, s>>>(L, x, y, scale);
}

template <>
void Ops<KT>::prolong(const Lvl& Lf, const Lvl& Lc, const KT* xc, KT* xf, KT* slopes, cudaStream_t s) {
  if (Lf.dim == 2) {
    ProfScope ps_(GKB_KC_PROLONG, s, lvl_unknowns(Lf));
    k_prolong_flux2d<KT><<<prolong2d_grid(Lc), dim3(BX, BY), 0, s>>>(Lf, Lc, xc, xf);
    return;
  }
  { ProfScope ps_(GKB_KC_PROLONG, s, 0); k_slopes3d<KT><<<face_grid(Lc), dim3(BX, BY), 0, s>>>(Lc, xc, slopes); }
  ProfScope ps_(GKB_KC_PROLONG, s, lvl_unknowns(Lf));
  k_prolong_flux3d<KT><<<face_grid(Lf), dim3(BX, BY), 0, s>>>(Lf, Lc, xc, slopes, xf);
}

template <>
void Ops<KT>::restrict_(const Lvl& Lf, const Lvl& Lc, const KT* rf, KT* bc, KT* tmp, KT* tmp2, cudaStream_t s) {
  ProfScope ps_(GKB_KC_RESTRICT, s, lvl_unknowns(Lf));
  if (Lf.dim == 2) {
    k_restrict_flux2d_a<KT><<<face_grid(Lc), dim3(BX, BY), 0, s>>>(Lf, Lc, rf, bc, tmp);
    k_restrict_flux2d_b<KT><<<face_grid(Lc), dim3(BX, BY), 0, s>>>(Lc, tmp, bc);
  } else {
    k_restrict_flux3d_a<KT><<<face_grid(Lc), dim3(BX, BY), 0, s>>>(Lf, Lc, rf, bc, tmp, tmp2);
    k_restrict_flux3d_b<KT><<<face_grid(Lc), dim3(BX, BY), 0, s>>>(Lc, tmp, tmp2, bc);
  }
}

template <>
void Ops<KT>::coarse(int m, const KT* Minv, const int* idx, const KT* b, KT* x, cudaStream_t s) {
  ProfScope ps_(GKB_KC_COARSE, s, (long long)m);
  const int warps_per_block = 8;
  k_coarse_solve<KT><<<(m + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(m, Minv, idx, b, x);
}

template <>
void Ops<KT>::dot(long long len, const KT* a, const KT* b, const RedBuf& red, int fin, void* st, cudaStream_t s,
                  const int* pred) {
  ProfScope ps_(GKB_KC_BLAS, s, len);
  k_dot<KT><<<(unsigned)blas_blocks(len), RB, 0, s>>>(len, a, b, red, fin, st, pred);
}

template <>
void Ops<KT>::dot2(long long len, const KT* a, const KT* b, const KT* c, const RedBuf& red, int fin, void* st,
                   cudaStream_t s) {
  ProfScope ps_(GKB_KC_BLAS, s, len);
  k_dot2<KT><<<(unsigned)blas_blocks(len), RB, 0, s>>>(len, a, b, c, red, fin, st);
}

template <>
void Ops<KT>::cg_update(long long len, KT* x, const KT* p, KT* r, const KT* q, const CgState* cg,
                        const RedBuf& red, void* st, cudaStream_t s, int fin) {
  ProfScope ps_(GKB_KC_BLAS, s, len);
  k_cg_update<KT><<<(unsigned)blas_blocks(len), RB, 0, s>>>(len, x, p, r, q, cg, red, st, fin);
}

template <>
void Ops<KT>::cg_dir(long long len, KT* p, const KT* z, const CgState* cg, int first, cudaStream_t s) {
  ProfScope ps_(GKB_KC_BLAS, s, len);
  k_cg_dir<KT><<<(unsigned)blas_blocks(len), RB, 0, s>>>(len, p, z, cg, first);
}

template <>
void Ops<KT>::axpby(long long len, KT a, const KT* x, KT b, KT* y, cudaStream_t s) {
  ProfScope ps_(GKB_KC_BLAS, s, len);
  k_axpby<KT><<<(unsigned)blas_blocks(len), RB, 0, s>>>(len, a, x, b, y);
}
#endif

#undef GKB_VARMU
#undef GKB_IN_PART
}  // namespace gkb
