// Per-dtype launch wrappers (included by vfpi_f32.cu and vfpi_f64.cu only).
#pragma once

#include <algorithm>

#include "vfpi_device.cuh"
#include "vfpi_internal.h"

namespace vfpi {

inline int blocks_for(int64_t n, int nt) { return (int)((n + nt - 1) / nt); }

template <typename T>
DevProblem<T> dev_problem(vfpi_ctx* c, bool adjoint = false) {
  DevProblem<T> P;
  P.n_slices = c->n_slices;
  P.n_pad = c->n_pad;
  P.slice_len = c->d_slice_len;
  P.slice_off = c->d_slice_off;
  P.vals = static_cast<const T*>(c->d_vals);
  P.cols = c->d_cols;
  P.vals6 = static_cast<const T*>(c->d_vals6);
  P.slice_cmin = c->d_slice_cmin;
  P.slice_cmax = c->d_slice_cmax;
  P.uvals = static_cast<const T*>(c->d_uvals);
  P.ucols = c->d_ucols;
  P.uslice_len = c->d_ulen;
  P.uslice_off = c->d_uoff;
  P.lcols = c->d_lcols;
  P.lpos = c->d_lpos;
  P.lslice_len = c->d_llen;
  P.lslice_off = c->d_loff;
  P.b = static_cast<const Vec4<T>*>(c->d_b);
  P.w = static_cast<const Vec4<T>*>(c->d_w);
  P.cslot = c->d_cslot;
  P.n_c = c->n_c;
  P.c_i = c->d_ci;
  P.c_j = c->d_cj;
  P.c_R = static_cast<const T*>(c->d_cR);
  P.c_mu = static_cast<const T*>(c->d_cmu);
  P.c_phi = static_cast<const T*>(c->d_cphi);
  P.c_omega = static_cast<const T*>(c->d_comega);
  P.c_mu2 = static_cast<const T*>(c->d_cmu2);
  P.aniso = c->aniso;
  P.prox = c->opts.operator_ == VFPI_OP_PROXIMAL ? 1 : 0;
  P.lam = static_cast<Vec4<T>*>(c->d_lam);
  P.lam_star = static_cast<Vec4<T>*>(c->d_lam_star);
  P.lam2 = static_cast<Vec4<T>*>(c->d_lam2);
  P.lam_star2 = static_cast<Vec4<T>*>(c->d_lam_star2);
  P.d_list = c->d_dlist;
  P.dstar = static_cast<Vec4<T>*>(c->d_dstar);
  P.v0 = static_cast<Vec4<T>*>(c->d_v0);
  P.v1 = static_cast<Vec4<T>*>(c->d_v1);
  P.r0 = static_cast<Vec4<T>*>(c->d_r0);
  P.r1 = static_cast<Vec4<T>*>(c->d_r1);
  P.adj_ls = static_cast<const Vec4<T>*>(c->d_adj_ls);
  P.adj_gphi = static_cast<T*>(c->d_adj_gphi);
  P.adj_gmu = static_cast<T*>(c->d_adj_gmu);
  if (adjoint) {
    P.b = static_cast<const Vec4<T>*>(c->d_adj_g);
    P.v0 = static_cast<Vec4<T>*>(c->d_adj_u0);
    P.v1 = static_cast<Vec4<T>*>(c->d_adj_u1);
  }
  return P;
}

template <typename T>
cudaError_t Launch<T>::validate_pattern(int N, int n_cols, int sorted, const int32_t* row_ptr,
                                        const int32_t* col_idx, const int32_t* node_scene, int* err,
                                        cudaStream_t s) {
  if (N > 0)
    k_validate_pattern<<<blocks_for(N, 256), 256, 0, s>>>(N, n_cols, sorted, row_ptr, col_idx,
                                                          node_scene, err);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::gather_nodes(vfpi_ctx* c, const int32_t* nodes, int n, void* out) {
  if (n > 0)
    k_gather_nodes<T><<<blocks_for(n, 256), 256, 0, c->stream>>>(
        n, c->N, nodes, c->d_node_map, static_cast<const Vec4<T>*>(c->d_v0), static_cast<T*>(out),
        c->d_err);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::set_halo(vfpi_ctx* c, int first, int n, const void* vals) {
  if (n > 0)
    k_set_halo<T><<<blocks_for(n, 256), 256, 0, c->stream>>>(
        n, (int64_t)c->n_pad + first, static_cast<const T*>(vals), static_cast<Vec4<T>*>(c->d_v0));
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::check_finite(const void* a, int64_t n, int* err, cudaStream_t s) {
  if (n > 0) {
    const int blocks = (int)std::min<int64_t>(blocks_for(n, 256), 152 * 16);
    k_check_finite<T><<<blocks, 256, 0, s>>>(static_cast<const T*>(a), n, err);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::build_layout(vfpi_ctx* c, const int32_t* row_ptr, const int32_t* col_idx,
                                    const void* vals, bool store_cols) {
  cudaStream_t s = c->stream;
  cudaError_t e;
  if (store_cols) {
    if (c->n_slices > 0)
      k_fill_pad_cols<<<blocks_for((int64_t)c->n_slices * 32, 256), 256, 0, s>>>(
          c->n_slices, c->d_slice_len, c->d_slice_off, c->d_cols);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = cudaMemsetAsync(c->d_vals, 0, (size_t)c->n_entries * 288 * sizeof(T), s)) != cudaSuccess)
    return e;
  if (c->N > 0)
    k_scatter_blocks<T><<<blocks_for(c->N, 128), 128, 0, s>>>(
        c->N, row_ptr, col_idx, static_cast<const T*>(vals), c->d_node_map, c->d_slice_len,
        c->d_slice_off, c->d_cols, static_cast<T*>(c->d_vals), store_cols ? 1 : 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (store_cols && c->n_slices > 0)
    k_slice_colrange<<<blocks_for((int64_t)c->n_slices * 32, 256), 256, 0, s>>>(
        c->n_slices, c->d_slice_len, c->d_slice_off, c->d_cols, c->d_slice_cmin, c->d_slice_cmax);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::make_w(vfpi_ctx* c) {
  cudaStream_t s = c->stream;
  const int np = c->n_pad;
  if (np == 0) return cudaSuccess;
  if (c->opts.w_mode == VFPI_W_FROBENIUS) {
    k_row_stats<T><<<blocks_for(np, 128), 128, 0, s>>>(dev_problem<T>(c), c->d_ds);
    k_make_w_frobenius<T><<<blocks_for(np, 256), 256, 0, s>>>(
        np, c->d_ds, c->d_cslot, c->d_ci, c->d_cj, static_cast<Vec4<T>*>(c->d_w));
  } else if (c->opts.w_mode == VFPI_W_SCALAR) {
    k_w_scalar<T><<<blocks_for(np, 256), 256, 0, s>>>(np, (T)c->opts.alpha,
                                                      static_cast<Vec4<T>*>(c->d_w));
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::row_stats(vfpi_ctx* c) {
  if (c->n_pad > 0)
    k_row_stats<T><<<blocks_for(c->n_pad, 128), 128, 0, c->stream>>>(dev_problem<T>(c), c->d_ds);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::split_stats(vfpi_ctx* c, double* out) {
  if (c->n_split > 0)
    k_split_stats<<<blocks_for(6 * (int64_t)c->n_split, 256), 256, 0, c->stream>>>(
        c->n_split, c->d_split_own, c->d_ds, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::split_set_stats(vfpi_ctx* c, const double* partner) {
  cudaStream_t s = c->stream;
  if (c->n_split == 0) return cudaSuccess;
  k_split_set_stats<<<blocks_for(6 * (int64_t)c->n_split, 256), 256, 0, s>>>(
      c->n_split, c->d_split_cs, c->d_split_own, c->d_ci, c->d_cj, partner, c->d_ds);
  // W again from the row statistics (the own rows' are unchanged)
  k_make_w_frobenius<T><<<blocks_for(c->n_pad, 256), 256, 0, s>>>(
      c->n_pad, c->d_ds, c->d_cslot, c->d_ci, c->d_cj, static_cast<Vec4<T>*>(c->d_w));
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::split_vstar(vfpi_ctx* c, void* out) {
  if (c->n_split > 0)
    k_split_vstar<T><<<blocks_for(c->n_split, 256), 256, 0, c->stream>>>(
        c->n_split, c->d_split_cs, c->d_split_own, c->d_cj,
        static_cast<const Vec4<T>*>(c->d_dstar), static_cast<T*>(out));
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::split_finish(vfpi_ctx* c, const void* partner_vstar) {
  if (c->n_split == 0) return cudaSuccess;
  ChebStep<T> ch;   // the step of the sweep this completes
  ch.on = c->opts.chebyshev_ls > 0 ? 1 : 0;
  ch.accel = ch.on && c->shard_l >= c->opts.chebyshev_ls;
  ch.nu = (T)c->shard_cheb.nu;
  ch.u = (T)c->opts.chebyshev_u;
  k_split_finish<T, 256><<<1, 256, 0, c->stream>>>(dev_problem<T>(c), c->n_split, c->d_split_cs,
                                                   c->d_split_own,
                                                   static_cast<const T*>(partner_vstar), ch,
                                                   c->d_sumsq);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::block_sym_check(vfpi_ctx* c) {
  if (c->n_pad > 0)
    k_block_sym_check<T><<<blocks_for(c->n_pad, 128), 128, 0, c->stream>>>(dev_problem<T>(c), c->d_err);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::make_vals6(vfpi_ctx* c) {
  if (c->n_pad > 0)
    k_make_vals6<T><<<blocks_for(c->n_pad, 128), 128, 0, c->stream>>>(dev_problem<T>(c),
                                                                      static_cast<T*>(c->d_vals6));
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::to_internal(vfpi_ctx* c, const void* ext, void* internal) {
  if (c->N > 0)
    k_to_internal<T><<<blocks_for(c->N, 256), 256, 0, c->stream>>>(
        c->N, static_cast<const T*>(ext), c->d_node_map, static_cast<Vec4<T>*>(internal));
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::to_external(vfpi_ctx* c, const void* internal, void* ext) {
  if (c->N > 0)
    k_to_external<T><<<blocks_for(c->N, 256), 256, 0, c->stream>>>(
        c->N, static_cast<const Vec4<T>*>(internal), c->d_node_map, static_cast<T*>(ext));
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::lambda_external(vfpi_ctx* c, const void* lam_int, void* out) {
  if (c->n_c > 0)
    k_lambda_external<T><<<blocks_for(c->n_c, 256), 256, 0, c->stream>>>(
        c->n_c, c->d_cperm, static_cast<const Vec4<T>*>(lam_int), static_cast<T*>(out));
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::contact_vec_internal(vfpi_ctx* c, const void* ext, void* out) {
  if (c->n_c > 0)
    k_contact_vec_internal<T><<<blocks_for(c->n_c, 256), 256, 0, c->stream>>>(
        c->n_c, c->d_cperm, static_cast<const T*>(ext), static_cast<Vec4<T>*>(out));
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::contact_scalar(vfpi_ctx* c, const void* in, void* out, bool to_external) {
  if (c->n_c > 0)
    k_contact_scalar<T><<<blocks_for(c->n_c, 256), 256, 0, c->stream>>>(
        c->n_c, c->d_cperm, static_cast<const T*>(in), static_cast<T*>(out), to_external ? 1 : 0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::integrate(vfpi_ctx* c, double* x_dev) {
  if (c->N > 0)
    k_integrate<T><<<blocks_for(c->N, 256), 256, 0, c->stream>>>(
        c->N, c->h, static_cast<const Vec4<T>*>(c->d_v0), c->d_node_map, x_dev);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::spmv(vfpi_ctx* c, const void* x_int, void* y_int) {
  if (c->n_slices > 0)
    k_spmv<T><<<blocks_for((int64_t)c->n_slices * 32, 256), 256, 0, c->stream>>>(
        dev_problem<T>(c), static_cast<const Vec4<T>*>(x_int), static_cast<Vec4<T>*>(y_int));
  return cudaGetLastError();
}

// Grid-path kernel variants: (threads per CTA, minimum CTAs per SM for the
// register budget, register prefetch of the next chunk).
template <typename T>
static void* grid_kernel(int nt, int minb, int pf, bool adj) {
#define VFPI_GK(NT_, MB_, PF_)                                                          \
  if (nt == NT_ && minb == MB_ && pf == PF_)                                            \
    return adj ? (void*)&k_solve_grid<T, NT_, MB_, PF_ != 0, true>                      \
               : (void*)&k_solve_grid<T, NT_, MB_, PF_ != 0, false>;
  VFPI_GK(64, 1, 0) VFPI_GK(128, 1, 0) VFPI_GK(256, 1, 0) VFPI_GK(512, 1, 0)
  VFPI_GK(256, 3, 0) VFPI_GK(256, 4, 0) VFPI_GK(512, 2, 0) VFPI_GK(128, 8, 0)
  VFPI_GK(256, 2, 1) VFPI_GK(128, 4, 1) VFPI_GK(512, 1, 1) VFPI_GK(256, 2, 0)
#undef VFPI_GK
  return nullptr;
}

// Grid-path and scene kernels on the symmetric-block storage (the forward
// sweep, and the adjoint's, which is the forward product with b := g_v on the
// symmetric A; Barzilai-Borwein steps read the full storage).
template <typename T>
static void* grid_kernel_b6(int nt, int minb, bool adj) {
#define VFPI_GB(NT_, MB_)                                                               \
  if (nt == NT_ && minb == MB_)                                                         \
    return adj ? (void*)&k_solve_grid<T, NT_, MB_, false, true, false, true>            \
               : (void*)&k_solve_grid<T, NT_, MB_, false, false, false, true>;
  VFPI_GB(256, 3) VFPI_GB(256, 2)
#undef VFPI_GB
  return nullptr;
}

template <typename T>
static void* scenes_kernel_b6(int nt, bool adj) {
  switch (nt) {
    case 64: return adj ? (void*)&k_solve_scenes<T, 64, true, true> : (void*)&k_solve_scenes<T, 64, false, true>;
    case 128: return adj ? (void*)&k_solve_scenes<T, 128, true, true> : (void*)&k_solve_scenes<T, 128, false, true>;
    case 256: return adj ? (void*)&k_solve_scenes<T, 256, true, true> : (void*)&k_solve_scenes<T, 256, false, true>;
    case 512: return adj ? (void*)&k_solve_scenes<T, 512, true, true> : (void*)&k_solve_scenes<T, 512, false, true>;
    default: return nullptr;
  }
}

// Grid-path kernels on the symmetric storage.
template <typename T>
static void* grid_kernel_sym(int nt, int minb, bool adj) {
#define VFPI_GS(NT_, MB_)                                                               \
  if (nt == NT_ && minb == MB_)                                                         \
    return adj ? (void*)&k_solve_grid<T, NT_, MB_, false, true, true>                   \
               : (void*)&k_solve_grid<T, NT_, MB_, false, false, true>;
  VFPI_GS(256, 2) VFPI_GS(256, 3) VFPI_GS(256, 4) VFPI_GS(512, 1)
#undef VFPI_GS
  return nullptr;
}

template <typename T>
cudaError_t Launch<T>::sym_nlow(vfpi_ctx* c, const int32_t* row_ptr, const int32_t* col_idx) {
  if (c->N > 0) k_row_nlow<<<blocks_for(c->N, 256), 256, 0, c->stream>>>(c->N, row_ptr, col_idx, c->d_nlow);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::sym_pattern(vfpi_ctx* c) {
  cudaStream_t s = c->stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(c->d_uvals, 0, (size_t)(c->n_uent + 1) * 288 * sizeof(T), s)) != cudaSuccess)
    return e;
  if (c->n_slices > 0)
    k_fill_sym_pad<T><<<blocks_for((int64_t)c->n_slices * 32, 256), 256, 0, s>>>(
        c->n_slices, c->d_ulen, c->d_uoff, c->d_ucols, c->d_llen, c->d_loff, c->d_lcols, c->d_lpos,
        c->n_uent * 288);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (c->N > 0)
    k_build_lower<T><<<blocks_for(c->N, 128), 128, 0, s>>>(
        c->N, c->d_row_ptr, c->d_col_idx, c->d_nlow, c->d_node_map, c->d_ulen, c->d_uoff, c->d_llen,
        c->d_loff, c->d_lcols, c->d_lpos, c->d_err);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::sym_values(vfpi_ctx* c, const void* vals, bool store_cols) {
  cudaStream_t s = c->stream;
  if (c->N > 0) {
    k_sym_check<T><<<blocks_for(c->N, 128), 128, 0, s>>>(c->N, c->d_row_ptr, c->d_col_idx,
                                                         static_cast<const T*>(vals), c->d_err);
    k_scatter_upper<T><<<blocks_for(c->N, 128), 128, 0, s>>>(
        c->N, c->d_row_ptr, c->d_col_idx, static_cast<const T*>(vals), c->d_nlow, c->d_node_map,
        c->d_ulen, c->d_uoff, c->d_ucols, static_cast<T*>(c->d_uvals), store_cols ? 1 : 0);
  }
  return cudaGetLastError();
}

template <typename T>
static void* scenes_kernel(int nt, bool adj) {
  switch (nt) {
    case 64: return adj ? (void*)&k_solve_scenes<T, 64, true> : (void*)&k_solve_scenes<T, 64, false>;
    case 128: return adj ? (void*)&k_solve_scenes<T, 128, true> : (void*)&k_solve_scenes<T, 128, false>;
    case 256: return adj ? (void*)&k_solve_scenes<T, 256, true> : (void*)&k_solve_scenes<T, 256, false>;
    case 512: return adj ? (void*)&k_solve_scenes<T, 512, true> : (void*)&k_solve_scenes<T, 512, false>;
    default: return nullptr;
  }
}

// TMA-staged grid kernels: (threads per CTA, stages per warp); dynamic shared memory.
template <typename T>
static void* tma_kernel(int nt, int nst, bool adj, size_t* smem) {
#define VFPI_TK(NT_, NS_)                                                               \
  if (nt == NT_ && nst == NS_) {                                                        \
    *smem = tma_smem_bytes<T, NT_, NS_>();                                              \
    return adj ? (void*)&k_solve_grid_tma<T, NT_, NS_, true>                            \
               : (void*)&k_solve_grid_tma<T, NT_, NS_, false>;                          \
  }
  VFPI_TK(256, 4) VFPI_TK(128, 4) VFPI_TK(128, 6) VFPI_TK(64, 8) VFPI_TK(256, 2) VFPI_TK(128, 2)
#undef VFPI_TK
  return nullptr;
}

template <typename T>
static void* cluster_kernel(int nt, bool adj) {
  switch (nt) {
    case 128: return adj ? (void*)&k_solve_cluster<T, 128, true> : (void*)&k_solve_cluster<T, 128, false>;
    case 256: return adj ? (void*)&k_solve_cluster<T, 256, true> : (void*)&k_solve_cluster<T, 256, false>;
    case 512: return adj ? (void*)&k_solve_cluster<T, 512, true> : (void*)&k_solve_cluster<T, 512, false>;
    default: return nullptr;
  }
}

// Shared memory per CTA of the cluster kernel (the SM's capacity split over
// cl_per_sm CTAs) and the sliced-ELL entries it holds; cluster occupancy.
template <typename T>
static cudaError_t configure_cluster(vfpi_ctx* c, int dev) {
  int optin = 0, per_sm = 0, resv = 0;
  cudaError_t e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess) return e;
  void* ks[2] = {cluster_kernel<T>(c->nt, false), cluster_kernel<T>(c->nt, true)};
  if (!ks[0] || !ks[1]) return cudaErrorInvalidValue;
  size_t stat = 0;
  for (void* k : ks) {
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, k)) != cudaSuccess) return e;
    stat = std::max(stat, fa.sharedSizeBytes);
  }
  const int64_t share = (int64_t)per_sm / c->cl_per_sm - resv - (int64_t)stat;
  int64_t dyn = std::min<int64_t>(share, (int64_t)optin - (int64_t)stat);
  dyn = dyn / 128 * 128;
  if (dyn < kClusterSmemHead + cluster_entry_bytes<T>()) return cudaErrorInvalidConfiguration;
  c->dyn_smem = (size_t)dyn;
  c->cache_entries = (int)((dyn - kClusterSmemHead) / cluster_entry_bytes<T>());
  int ncl = 0;
  for (int a = 0; a < 2; ++a) {
    if ((e = cudaFuncSetAttribute(ks[a], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn)) != cudaSuccess)
      return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)c->cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)c->cluster);
    cfg.blockDim = dim3((unsigned)c->nt);
    cfg.dynamicSmemBytes = (size_t)dyn;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if ((e = cudaOccupancyMaxActiveClusters(&n, ks[a], &cfg)) != cudaSuccess) return e;
    ncl = a ? std::min(ncl, n) : n;
  }
  if (ncl < 1) return cudaErrorInvalidConfiguration;
  c->max_grid = ncl * c->cluster;
  c->grid = c->cluster * std::max(1, std::min(ncl, c->n_scenes));
  return cudaSuccess;
}

template <typename T>
static void* pick_kernel(vfpi_ctx* c, bool adj, size_t* smem) {
  *smem = 0;
  if (c->path == 2 && c->cluster > 0) {
    // Barzilai-Borwein sweeps run on the CTA-per-scene kernel
    if (!adj && c->bb_rule) return scenes_kernel<T>(c->nt, adj);
    *smem = c->dyn_smem;
    return cluster_kernel<T>(c->nt, adj);
  }
  if (c->path == 1 && c->tma_stages > 0) {
    // Barzilai-Borwein sweeps run on the register-staged kernel
    if (!adj && c->bb_rule) return grid_kernel<T>(256, 2, 0, adj);
    return tma_kernel<T>(c->nt, c->tma_stages, adj, smem);
  }
  if (c->path == 1 && c->sym && c->sym_ok && !(!adj && c->bb_rule))
    return grid_kernel_sym<T>(c->nt, c->minb, adj);
  if (c->b6 && c->bsym_ok && c->d_vals6 && !(!adj && c->bb_rule))
    return c->path == 1 ? grid_kernel_b6<T>(c->nt, c->minb, adj) : scenes_kernel_b6<T>(c->nt, adj);
  return c->path == 1 ? grid_kernel<T>(c->nt, c->minb, c->pf, adj) : scenes_kernel<T>(c->nt, adj);
}

template <typename T>
cudaError_t Launch<T>::configure(vfpi_ctx* c) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if (c->path == 2 && c->cluster > 0) return configure_cluster<T>(c, dev);
  int per_sm = 0;
  for (int adj = 0; adj < 2; ++adj) {  // one grid fits both modes
    size_t smem = 0;
    void* k = pick_kernel<T>(c, adj != 0, &smem);
    if (!k) return cudaErrorInvalidValue;
    if (smem > 0 &&
        (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    int q = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, k, c->nt, smem)) != cudaSuccess) return e;
    if (c->b6) {   // falls back to the full storage if a block stops being symmetric
      int q2 = 0;
      void* kf = c->path == 1 ? grid_kernel<T>(c->nt, c->minb, 0, adj != 0)
                              : scenes_kernel<T>(c->nt, adj != 0);
      if (!kf) return cudaErrorInvalidValue;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q2, kf, c->nt, 0)) != cudaSuccess) return e;
      q = std::min(q, q2);
    }
    if (c->path == 1 && c->sym) {   // falls back to the full storage if A stops being symmetric
      int q2 = 0;
      void* kf = grid_kernel<T>(c->nt, c->minb, 0, adj != 0);
      if (!kf) return cudaErrorInvalidValue;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q2, kf, c->nt, 0)) != cudaSuccess) return e;
      q = std::min(q, q2);
    }
    per_sm = adj ? std::min(per_sm, q) : q;
  }
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  c->max_grid = per_sm * sms;
  if (c->path == 1) {
    // persistent grid: every CTA resident (cooperative launch), no more CTAs
    // than there are warps' worth of slices
    const int need = (c->n_slices + c->nt / 32 - 1) / (c->nt / 32);
    c->grid = std::max(1, std::min(c->max_grid, need));
    if (c->opts.grid_ctas > 0) c->grid = std::min(c->max_grid, c->opts.grid_ctas);
  } else {
    c->grid = std::max(1, std::min(c->max_grid, c->n_scenes));
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t Launch<T>::solve(vfpi_ctx* c, int l_max, double theta_th, bool adjoint) {
  cudaStream_t s = c->stream;
  cudaError_t e;
  SolveCtl ctl;
  ctl.l_max = l_max;
  ctl.theta_th = theta_th;
  ctl.norm_scale = c->d_norm_scale;
  ctl.partials = c->d_partials;
  ctl.bar = c->d_bar;
  ctl.n_scenes = c->n_scenes;
  ctl.order = c->d_order;
  ctl.scene_slice = c->d_scene_slice;
  ctl.scene_d = c->d_scene_d;
  ctl.queue = c->d_queue;
  ctl.iters = c->d_iters;
  ctl.status = c->d_status;
  ctl.theta = c->d_theta;
  ctl.n_d = c->n_d;
  ctl.err = c->d_err;
  ctl.cheb_ls = adjoint ? c->adj_cheb_ls : c->opts.chebyshev_ls;
  ctl.cheb_u = adjoint ? c->adj_cheb_u : c->opts.chebyshev_u;
  ctl.bb_rule = adjoint ? 0 : c->bb_rule;
  ctl.bb_alpha0 = c->bb_alpha0;
  ctl.bb_part = c->d_bbpart;
  ctl.items = c->d_items;
  ctl.cache_entries = c->cache_entries;
  ctl.smem_bytes = (int32_t)c->dyn_smem;
  ctl.theta_rel = (adjoint && c->adj_tol_set && c->adj_rel) ? 1 : 0;
  ctl.th_scene = c->d_thscene;
  ctl.sumsq = c->d_sumsq;
  // a shard's launch is one sweep of a solve the caller drives: its index and
  // weight come from the context, and the iterate buffers keep v^{l-1}
  const bool shard = c->n_halo > 0 && !adjoint;
  ctl.l0 = shard ? c->shard_l : 1;
  ctl.nu0 = shard ? c->shard_cheb.nu : 1.0;
  ctl.swap_end = shard ? 1 : 0;
  // the TMA ring kernel's lagged stop test: forward Alg. 1 sweeps (no
  // Chebyshev weight, which needs the last theta before the next sweep), no
  // D-contacts (their second barrier), more than one sweep
  ctl.lag_stop = (c->path == 1 && c->tma_stages > 0 && !adjoint && !c->bb_rule && !shard &&
                  ctl.cheb_ls <= 0 && c->n_d == 0 && l_max > 1) ? 1 : 0;
  if (ctl.theta_rel && c->path == 1 && c->n_slices > 0) {   // (the per-scene kernels compute theirs)
    k_slice_sumsq<T><<<blocks_for((int64_t)c->n_slices * 32, 256), 256, 0, s>>>(
        c->n_slices, static_cast<const Vec4<T>*>(c->d_adj_g), c->d_slicesq);
    k_scene_threshold<<<c->n_scenes, 256, 0, s>>>(c->d_scene_slice, c->d_slicesq, c->d_norm_scale,
                                                  theta_th, c->d_thscene);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // control words: barrier count/generation, error flag, scene queue
  if ((e = cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned int), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c->d_err, 0, sizeof(int), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c->d_queue, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
  if (c->path == 2 && c->cluster > 0 &&
      (e = cudaMemsetAsync(c->d_items, 0, 8 * (size_t)c->max_grid, s)) != cudaSuccess)
    return e;
  DevProblem<T> P = dev_problem<T>(c, adjoint);
  void* args[] = {&P, &ctl};
  size_t smem = 0;
  void* k = pick_kernel<T>(c, adjoint, &smem);
  if (!k) return cudaErrorInvalidValue;
  // inside a stream capture the events become graph nodes that record on replay
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess) return e;
  const unsigned flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
  if ((e = cudaEventRecordWithFlags(c->ev0, s, flags)) != cudaSuccess) return e;
  const int nt = (c->path == 1 && c->tma_stages > 0 && !adjoint && c->bb_rule) ? 256 : c->nt;
  const bool clustered = c->path == 2 && c->cluster > 0 && !(!adjoint && c->bb_rule);
  if (c->path == 1) {
    e = cudaLaunchCooperativeKernel(k, dim3(c->grid), dim3(nt), args, smem, s);
  } else if (clustered) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)c->cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)c->grid);
    cfg.blockDim = dim3((unsigned)nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelExC(&cfg, k, args);
  } else {
    e = cudaLaunchKernel(k, dim3(std::max(1, std::min(c->grid, c->n_scenes))), dim3(nt), args, 0, s);
  }
  if (e != cudaSuccess) return e;
  c->timed = true;
  return cudaEventRecordWithFlags(c->ev1, s, flags);
}

}  // namespace vfpi
