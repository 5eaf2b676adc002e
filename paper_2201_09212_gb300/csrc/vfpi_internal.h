// Host-side internals of libvfpi: the context and the per-dtype launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/vfpi.h"

namespace vfpi {

struct DevState;  // device pointers, see vfpi_ctx

// Launchers, instantiated for float and double in vfpi_f32.cu / vfpi_f64.cu.
template <typename T>
struct Launch {
  static cudaError_t validate_pattern(int N, int n_cols, int sorted, const int32_t* row_ptr,
                                      const int32_t* col_idx, const int32_t* node_scene, int* err,
                                      cudaStream_t s);
  // sharded scene: v of own nodes out, halo values in
  static cudaError_t gather_nodes(vfpi_ctx* c, const int32_t* nodes, int n, void* out);
  static cudaError_t set_halo(vfpi_ctx* c, int first, int n, const void* vals);
  // split D-contacts (one node in the halo): own endpoints' row statistics
  // out, the partner endpoints' in (then W again), own v* out, the contact step
  static cudaError_t split_stats(vfpi_ctx* c, double* out);
  static cudaError_t split_set_stats(vfpi_ctx* c, const double* partner);
  static cudaError_t split_vstar(vfpi_ctx* c, void* out);
  static cudaError_t split_finish(vfpi_ctx* c, const void* partner_vstar);
  static cudaError_t check_finite(const void* a, int64_t n, int* err, cudaStream_t s);
  static cudaError_t build_layout(vfpi_ctx* c, const int32_t* row_ptr, const int32_t* col_idx,
                                  const void* vals, bool store_cols);
  static cudaError_t make_w(vfpi_ctx* c);
  // symmetric-block storage: check (err bit 128 if a block is not symmetric), build
  static cudaError_t block_sym_check(vfpi_ctx* c);
  static cudaError_t make_vals6(vfpi_ctx* c);
  static cudaError_t row_stats(vfpi_ctx* c);
  static cudaError_t to_internal(vfpi_ctx* c, const void* ext, void* internal);
  static cudaError_t to_external(vfpi_ctx* c, const void* internal, void* ext);
  static cudaError_t lambda_external(vfpi_ctx* c, const void* lam_int, void* out);
  static cudaError_t contact_vec_internal(vfpi_ctx* c, const void* ext, void* out);
  static cudaError_t contact_scalar(vfpi_ctx* c, const void* in, void* out, bool to_external);
  static cudaError_t integrate(vfpi_ctx* c, double* x_dev);
  static cudaError_t spmv(vfpi_ctx* c, const void* x_int, void* y_int);
  static cudaError_t solve(vfpi_ctx* c, int l_max, double theta_th, bool adjoint);
  static cudaError_t configure(vfpi_ctx* c);
  // symmetric storage: diagonal index of each row; padding and the lower
  // entries' positions; symmetry check (error bits 32/64) and upper values
  static cudaError_t sym_nlow(vfpi_ctx* c, const int32_t* row_ptr, const int32_t* col_idx);
  static cudaError_t sym_pattern(vfpi_ctx* c);
  static cudaError_t sym_values(vfpi_ctx* c, const void* vals, bool store_cols);
};

}  // namespace vfpi

// Alg. 3's scalars of a shard's solve, which the caller drives one sweep at a
// time (the host copy of the kernels' per-CTA state).
struct HostChebScalars {
  double nu = 1.0, rho = 0.0, th1 = 0.0, th2 = 0.0;
};

// The opaque context behind vfpi_t.
struct vfpi_ctx {
  int dtype = VFPI_F32;
  size_t esz = 4;
  cudaStream_t stream = nullptr;
  vfpi_opts opts{};
  double h = 0.0;

  // sizes
  int N = 0, nnzb = 0, n_scenes = 1, n_slices = 0, n_pad = 0, n_c = 0, n_d = 0;
  int n_halo = 0;         // shard of a split scene: halo nodes, stored after the n_pad rows
  int n_split = 0;        // shard: D-contacts with one node in the halo (split contacts)
  int split_ready = 0;    // W_FROBENIUS: the split contacts' partner row statistics are set
  int shard_l = 1;        // shard: the index of its next sweep in the solve
  HostChebScalars shard_cheb;   // shard: Alg. 3's rho and the next sweep's weight nu
  int64_t n_entries = 0;  // sum of slice lengths; stored block slots = 32 * n_entries

  // host copies of the layout and contact bookkeeping
  std::vector<int32_t> h_scene_ptr, h_scene_slice, h_node_map, h_slice_len, h_node_scene;
  std::vector<int64_t> h_slice_off;
  std::vector<int32_t> h_cperm;  // internal contact -> caller's index
  std::vector<int32_t> h_ci, h_cj;

  // device memory (owned)
  int32_t *d_slice_len = nullptr;
  int64_t* d_slice_off = nullptr;
  int32_t *d_slice_cmin = nullptr, *d_slice_cmax = nullptr;  // column range of each slice
  // symmetric storage (grid path, built when A = A^T exactly)
  int sym_ok = 0;                           // built and A currently symmetric
  int64_t n_uent = 0, n_lent = 0;           // entries (32 slots each) of the two structures
  int32_t *d_col_idx = nullptr, *d_nlow = nullptr;
  int32_t *d_ulen = nullptr, *d_llen = nullptr;
  int64_t *d_uoff = nullptr, *d_loff = nullptr;
  void* d_uvals = nullptr;
  int32_t *d_ucols = nullptr, *d_lcols = nullptr, *d_lpos = nullptr;
  void* d_vals = nullptr;
  void* d_vals6 = nullptr;   // 6 values per slot (built for the symmetric-block variants)
  int bsym_ok = 0;           // every stored block equals its transpose bit for bit
  int b6 = 0;                // launch variant reads vals6 (when bsym_ok and built)
  int32_t* d_cols = nullptr;
  void *d_b = nullptr, *d_w = nullptr, *d_v0 = nullptr, *d_v1 = nullptr;
  void *d_t0 = nullptr, *d_t1 = nullptr;    // internal temporaries (matvec)
  int32_t* d_cslot = nullptr;
  int32_t* d_node_map = nullptr;
  int32_t* d_row_ptr = nullptr;             // caller's row pointers (value updates)
  double* d_ds = nullptr;                   // per-DOF row statistics for W [n_pad + n_halo][6]
  int32_t *d_split_cs = nullptr, *d_split_own = nullptr;  // [n_split] internal contact, own row
  int32_t *d_ci = nullptr, *d_cj = nullptr, *d_cperm = nullptr, *d_dlist = nullptr;
  void *d_cR = nullptr, *d_cmu = nullptr, *d_cphi = nullptr, *d_comega = nullptr;
  void* d_cmu2 = nullptr;                   // friction along t2 (elliptic cones)
  int aniso = 0;
  void *d_lam = nullptr, *d_lam_star = nullptr;
  void *d_lam2 = nullptr, *d_lam_star2 = nullptr;   // odd sweeps' lambda under the lagged stop test
  void* d_dstar = nullptr;                  // D-contact v* staging [2 n_c]
  int32_t *d_scene_slice = nullptr, *d_scene_d = nullptr, *d_order = nullptr, *d_queue = nullptr;
  double* d_norm_scale = nullptr;
  double* d_partials = nullptr;   // [3][max_grid]
  double* d_sumsq = nullptr;                // the grid kernels' last sum ||dv||^2
  double* d_bbpart = nullptr;               // BB dot-product partials [2][max_grid][3]
  void *d_r0 = nullptr, *d_r1 = nullptr;    // BB residual ping-pong (allocated on use)
  int adj_cheb_ls = 0;                      // Chebyshev acceleration of the adjoint solve
  double adj_cheb_u = 1.0;
  int adj_tol_set = 0, adj_rel = 0, adj_l_max = 0;   // the adjoint's own stop test
  double adj_theta_th = 0.0;
  double *d_slicesq = nullptr, *d_thscene = nullptr;  // relative test: [n_slices], [n_scenes]
  int bb_rule = 0;
  double bb_alpha0 = 0.0;
  unsigned int* d_bar = nullptr;
  int* d_err = nullptr;
  int32_t *d_iters = nullptr, *d_status = nullptr;
  double* d_theta = nullptr;
  // adjoint (allocated on first use): rhs dL/dv, iterates, frozen lambda*, outputs
  void *d_adj_g = nullptr, *d_adj_u0 = nullptr, *d_adj_u1 = nullptr, *d_adj_ls = nullptr;
  void *d_adj_gphi = nullptr, *d_adj_gmu = nullptr;
  int adj_nc = -1;
  void* d_stage = nullptr;
  size_t stage_bytes = 0;

  // launch configuration
  int path = 0;    // 1 grid-wide cooperative kernel, 2 CTA per scene
  int grid = 0;    // CTAs
  int nt = 0;      // threads per CTA
  int minb = 1;    // grid path: minimum CTAs per SM the kernel is compiled for
  int pf = 0;      // grid path: register prefetch of the next chunk
  int tma_stages = 0;  // grid path: > 0 selects the TMA-staged kernel with this ring depth
  int sym = 0;         // grid path: product from the symmetric storage (when sym_ok)
  int cluster = 0;     // scene path: > 0 selects the shared-memory-resident cluster kernel
  int cl_per_sm = 1;   //   with this many CTAs per cluster and CTAs per SM
  size_t dyn_smem = 0; //   shared memory per CTA and the sliced-ELL entries it holds
  int cache_entries = 0;
  int32_t* d_items = nullptr;  // [2 max_grid] work items and poison words of the cluster kernel
  int max_grid = 0;

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // vfpi_advance: a side stream for the positions' upload, which overlaps the
  // solve (created on first use)
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_main = nullptr, ev_aux = nullptr;
  bool timed = false;
  std::string err;
};
