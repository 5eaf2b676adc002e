// C ABI of libvfpi (declared in include/vfpi.h): argument checking, input
// staging, layout set-up, contact bookkeeping and dispatch to the per-dtype
// launchers.  Host code only; every step of the solve runs in the kernels.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>

#include "vfpi_internal.h"

using vfpi::Launch;

namespace {

thread_local std::string g_create_error;

#define VFPI_TRY_CUDA(expr)                                                   \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #expr);                    \
  } while (0)

vfpi_status cuda_fail(vfpi_ctx* c, cudaError_t e, const char* what) {
  cudaGetLastError();
  char buf[512];
  std::snprintf(buf, sizeof buf, "CUDA error %s (%s) in %s", cudaGetErrorName(e),
                cudaGetErrorString(e), what);
  if (c) c->err = buf; else g_create_error = buf;
  return e == cudaErrorMemoryAllocation ? VFPI_ERR_OOM : VFPI_ERR_CUDA;
}

vfpi_status arg_fail(vfpi_ctx* c, vfpi_status st, const std::string& msg) {
  if (c) c->err = msg; else g_create_error = msg;
  return st;
}

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename P>
cudaError_t dalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

// Copy n bytes from caller memory (host or device) into host vector storage.
cudaError_t to_host(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  if (!on_device(src)) {
    std::memcpy(dst, src, bytes);
    return cudaSuccess;
  }
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

// Make the staging buffer at least `bytes` long (waits for earlier users).
cudaError_t ensure_stage(vfpi_ctx* c, size_t bytes) {
  if (bytes <= c->stage_bytes) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  if (c->aux_stream && (e = cudaStreamSynchronize(c->aux_stream)) != cudaSuccess) return e;
  if (c->d_stage) cudaFree(c->d_stage);
  c->d_stage = nullptr;
  c->stage_bytes = 0;
  const size_t want = std::max<size_t>(bytes, 1 << 20);
  if ((e = cudaMalloc(&c->d_stage, want)) != cudaSuccess) return e;
  c->stage_bytes = want;
  return cudaSuccess;
}

// Device view of caller memory: the pointer itself if it is device memory,
// else a copy at byte offset `slot` of the staging buffer (grown if needed;
// growing invalidates earlier views, so multi-view callers size it first).
// The caller may change or free a host array once the call returns: the
// runtime stages pageable memory before cudaMemcpyAsync returns, but reads
// page-locked memory when the stream gets there, so that copy is waited for
// -- unless the stream is being captured, where the copy becomes a graph
// node that reads the caller's buffer at every replay (the graph's contract).
cudaError_t device_view(vfpi_ctx* c, const void* src, size_t bytes, size_t slot, const void** out) {
  cudaPointerAttributes a;
  int type = cudaMemoryTypeUnregistered;
  if (src && cudaPointerGetAttributes(&a, src) == cudaSuccess) type = a.type;
  else cudaGetLastError();
  if (type == cudaMemoryTypeDevice || type == cudaMemoryTypeManaged) {
    *out = src;
    return cudaSuccess;
  }
  cudaError_t e = ensure_stage(c, slot + bytes);
  if (e != cudaSuccess) return e;
  char* dst = static_cast<char*>(c->d_stage) + slot;
  *out = dst;
  if (bytes == 0) return cudaSuccess;
  if ((e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
    return e;
  if (type != cudaMemoryTypeHost) return cudaSuccess;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(c->stream, &cap)) != cudaSuccess) return e;
  return cap == cudaStreamCaptureStatusNone ? cudaStreamSynchronize(c->stream) : cudaSuccess;
}

// The same view without the wait for page-locked sources, queued on stream
// `s`: for a call that waits for its whole step before it returns.  The
// staging buffer must already hold slot + bytes.
cudaError_t device_view_queued(vfpi_ctx* c, const void* src, size_t bytes, size_t slot,
                               cudaStream_t s, const void** out) {
  if (on_device(src)) {
    *out = src;
    return cudaSuccess;
  }
  char* dst = static_cast<char*>(c->d_stage) + slot;
  *out = dst;
  if (bytes == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
}

// Write `bytes` of device data to caller memory (host or device).
cudaError_t to_caller(vfpi_ctx* c, void* dst, const void* dev_src, size_t bytes) {
  if (bytes == 0) return cudaSuccess;
  if (on_device(dst)) return cudaMemcpyAsync(dst, dev_src, bytes, cudaMemcpyDeviceToDevice, c->stream);
  cudaError_t e = cudaMemcpyAsync(dst, dev_src, bytes, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(c->stream);
}

// Where a kernel should write an output bound for caller memory: the caller's
// pointer if it is device memory, else the staging buffer at `slot`.
cudaError_t out_view(vfpi_ctx* c, void* dst, size_t bytes, size_t slot, void** out) {
  if (on_device(dst)) {
    *out = dst;
    return cudaSuccess;
  }
  cudaError_t e = ensure_stage(c, slot + bytes);
  if (e != cudaSuccess) return e;
  *out = static_cast<char*>(c->d_stage) + slot;
  return cudaSuccess;
}

void free_all(vfpi_ctx* c) {
  void* ptrs[] = {c->d_slice_len, c->d_slice_off, c->d_slice_cmin, c->d_slice_cmax, c->d_vals, c->d_cols, c->d_b, c->d_w,
                  c->d_v0, c->d_v1, c->d_t0, c->d_t1, c->d_cslot, c->d_node_map, c->d_row_ptr, c->d_ds,
                  c->d_ci, c->d_cj, c->d_cperm, c->d_dlist, c->d_cR, c->d_cmu, c->d_cphi, c->d_comega, c->d_cmu2,
                  c->d_lam, c->d_lam_star, c->d_lam2, c->d_lam_star2, c->d_dstar, c->d_scene_slice, c->d_scene_d, c->d_order,
                  c->d_queue, c->d_norm_scale, c->d_partials, c->d_bar, c->d_err, c->d_iters,
                  c->d_status, c->d_theta, c->d_adj_g, c->d_adj_u0, c->d_adj_u1,
                  c->d_adj_ls, c->d_adj_gphi, c->d_adj_gmu, c->d_bbpart, c->d_r0, c->d_r1,
                  c->d_stage, c->d_items, c->d_col_idx, c->d_nlow, c->d_ulen, c->d_llen,
                  c->d_uoff, c->d_loff, c->d_uvals, c->d_ucols, c->d_lcols, c->d_lpos,
                  c->d_thscene, c->d_slicesq, c->d_sumsq, c->d_split_cs, c->d_split_own,
                  c->d_vals6};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->ev_main) cudaEventDestroy(c->ev_main);
  if (c->ev_aux) cudaEventDestroy(c->ev_aux);
  if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// kernel_variant -> launch shape: grid path VFPI_VARIANT_DEFAULT..TMA_64_8;
// scene path 0 (CTA-per-scene kernel, block_threads picks its size; the grid
// variants 1..11 are ignored there) or one of the VFPI_VARIANT_CL_* cluster
// shapes.  False for a variant the path does not have.
bool apply_variant(vfpi_ctx* c, int v, int block_threads) {
  static const int grid_table[12][4] = {{256, 3, 0, 0}, {256, 4, 0, 0}, {512, 2, 0, 0}, {128, 8, 0, 0},
                                        {256, 2, 1, 0}, {128, 4, 1, 0}, {512, 1, 1, 0}, {256, 2, 0, 0},
                                        {256, 1, 0, 4}, {128, 1, 0, 4}, {128, 1, 0, 6}, {64, 1, 0, 8}};
  // threads per CTA, CTAs per cluster, CTAs per SM
  static const int cl_table[10][3] = {{256, 1, 1}, {256, 2, 1}, {256, 4, 1}, {256, 8, 1}, {128, 4, 2},
                                      {128, 8, 2}, {256, 4, 2}, {256, 8, 2}, {512, 8, 1}, {128, 8, 4}};
  // symmetric storage: threads per CTA, CTAs/SM register budget
  static const int sym_table[4][2] = {{256, 2}, {256, 3}, {256, 4}, {512, 1}};
  const bool is_cl = v >= VFPI_VARIANT_CL_256_1_1 && v <= VFPI_VARIANT_CL_128_8_4;
  const bool is_sym = v >= VFPI_VARIANT_SYM_256_2 && v <= VFPI_VARIANT_SYM_512_1;
  const bool is_tma2 = v == VFPI_VARIANT_TMA_256_2 || v == VFPI_VARIANT_TMA_128_2;
  const bool is_b6 = v >= VFPI_VARIANT_B6_256_3 && v <= VFPI_VARIANT_B6_SCENES;
  if (v < 0 || (v > VFPI_VARIANT_SYM_512_1 && !is_cl && !is_tma2 && !is_b6)) return false;
  if (c->path == 1 && is_cl) return false;
  if (c->path != 1 && is_tma2) return false;
  if (is_sym && (c->path != 1 || !c->sym_ok)) return false;
  if (is_b6 && (!c->bsym_ok || (c->path == 1) != (v != VFPI_VARIANT_B6_SCENES))) return false;
  c->nt = block_threads ? block_threads : (c->path == 1 ? 256 : 128);
  c->minb = 1;
  c->pf = 0;
  c->tma_stages = 0;
  c->cluster = 0;
  c->cl_per_sm = 1;
  c->sym = 0;
  c->b6 = is_b6 ? 1 : 0;
  if (is_b6) {
    if (v == VFPI_VARIANT_B6_256_3) { c->nt = 256; c->minb = 3; }
    if (v == VFPI_VARIANT_B6_256_2) { c->nt = 256; c->minb = 2; }
  } else if (is_sym) {
    c->nt = sym_table[v - VFPI_VARIANT_SYM_256_2][0];
    c->minb = sym_table[v - VFPI_VARIANT_SYM_256_2][1];
    c->sym = 1;
  } else if (is_tma2) {
    c->nt = v == VFPI_VARIANT_TMA_256_2 ? 256 : 128;
    c->tma_stages = 2;
  } else if (c->path == 1 && (v > 0 || !block_threads)) {
    c->nt = grid_table[v][0];
    c->minb = grid_table[v][1];
    c->pf = grid_table[v][2];
    c->tma_stages = grid_table[v][3];
  } else if (is_cl) {
    const int* t = cl_table[v - VFPI_VARIANT_CL_256_1_1];
    c->nt = t[0];
    c->cluster = t[1];
    c->cl_per_sm = t[2];
  }
  return true;
}

struct Shape {
  int nt, minb, pf, tma_stages, cluster, cl_per_sm, grid_ctas, sym, b6;
};
Shape shape_of(const vfpi_ctx* c) {
  return {c->nt, c->minb, c->pf, c->tma_stages, c->cluster, c->cl_per_sm, c->opts.grid_ctas, c->sym,
          c->b6};
}
void restore_shape(vfpi_ctx* c, const Shape& s) {
  c->nt = s.nt; c->minb = s.minb; c->pf = s.pf; c->tma_stages = s.tma_stages;
  c->cluster = s.cluster; c->cl_per_sm = s.cl_per_sm; c->opts.grid_ctas = s.grid_ctas;
  c->sym = s.sym;
  c->b6 = s.b6;
}


// ---------------------------------------------------------------------------
// dispatch helpers on dtype
// ---------------------------------------------------------------------------

#define DISPATCH(c, call) ((c)->dtype == VFPI_F64 ? Launch<double>::call : Launch<float>::call)

// ---------------------------------------------------------------------------
// contacts
// ---------------------------------------------------------------------------

vfpi_status set_contacts(vfpi_ctx* c, const vfpi_contacts* J) {
  const int n_c = J ? J->n_c : 0;
  if (n_c < 0) return arg_fail(c, VFPI_ERR_INVALID_ARG, "n_c < 0");
  if (n_c > 0 && (!J->node_i || !J->R || !J->mu || !J->phi))
    return arg_fail(c, VFPI_ERR_INVALID_ARG, "contacts: node_i, R, mu and phi are required");
  std::vector<int32_t> ni(n_c), nj(n_c, -1);
  std::vector<double> R(9 * (size_t)n_c), mu(n_c), phi(n_c);
  cudaStream_t s = c->stream;
  VFPI_TRY_CUDA(to_host(ni.data(), J ? J->node_i : nullptr, 4 * (size_t)n_c, s));
  if (J && J->node_j) VFPI_TRY_CUDA(to_host(nj.data(), J->node_j, 4 * (size_t)n_c, s));
  {
    std::vector<unsigned char> raw(c->esz * 11 * (size_t)n_c);
    if (n_c > 0) {
      VFPI_TRY_CUDA(to_host(raw.data(), J->R, c->esz * 9 * (size_t)n_c, s));
      VFPI_TRY_CUDA(to_host(raw.data() + c->esz * 9 * (size_t)n_c, J->mu, c->esz * (size_t)n_c, s));
      VFPI_TRY_CUDA(to_host(raw.data() + c->esz * 10 * (size_t)n_c, J->phi, c->esz * (size_t)n_c, s));
    }
    for (size_t k = 0; k < 11 * (size_t)n_c; ++k) {
      const double v = c->dtype == VFPI_F64 ? reinterpret_cast<const double*>(raw.data())[k]
                                            : (double)reinterpret_cast<const float*>(raw.data())[k];
      if (k < 9 * (size_t)n_c) R[k] = v;
      else if (k < 10 * (size_t)n_c) mu[k - 9 * (size_t)n_c] = v;
      else phi[k - 10 * (size_t)n_c] = v;
    }
  }
  // validation (a shard's D-contact may have one node in the halo: a split contact)
  const int NH = c->N + c->n_halo;
  std::vector<int32_t> owner(NH, -1);
  for (int m = 0; m < n_c; ++m) {
    const int i = ni[m], j = nj[m];
    if (i < 0 || i >= NH || j < -1 || j >= NH || i == j)
      return arg_fail(c, VFPI_ERR_INVALID_ARG, "contact " + std::to_string(m) + ": node index out of range");
    if (i >= c->N && (j < 0 || j >= c->N))
      return arg_fail(c, VFPI_ERR_INVALID_ARG,
                      "contact " + std::to_string(m) + ": a halo node only as one end of a D-contact");
    if (j >= 0 && i < c->N && j < c->N && c->h_node_scene[i] != c->h_node_scene[j])
      return arg_fail(c, VFPI_ERR_INVALID_ARG, "contact " + std::to_string(m) + ": D-contact across scenes");
    for (int q : {i, j}) {
      if (q < 0) continue;
      if (owner[q] >= 0)
        return arg_fail(c, VFPI_ERR_CONTACT_OVERLAP,
                        "node " + std::to_string(q) + " is in contacts " + std::to_string(owner[q]) +
                            " and " + std::to_string(m));
      owner[q] = m;
    }
    const double* r = &R[9 * (size_t)m];
    for (int k = 0; k < 9; ++k)
      if (!std::isfinite(r[k])) return arg_fail(c, VFPI_ERR_NONFINITE, "contact frame not finite");
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const double d = r[3 * a] * r[3 * b] + r[3 * a + 1] * r[3 * b + 1] + r[3 * a + 2] * r[3 * b + 2];
        if (std::fabs(d - (a == b ? 1.0 : 0.0)) > 1e-4)
          return arg_fail(c, VFPI_ERR_INVALID_ARG, "contact " + std::to_string(m) + ": R is not orthonormal");
      }
    const double det = r[0] * (r[4] * r[8] - r[5] * r[7]) - r[1] * (r[3] * r[8] - r[5] * r[6]) +
                       r[2] * (r[3] * r[7] - r[4] * r[6]);
    if (det < 0) return arg_fail(c, VFPI_ERR_INVALID_ARG, "contact " + std::to_string(m) + ": det R < 0");
    if (!std::isfinite(mu[m]) || !std::isfinite(phi[m]))
      return arg_fail(c, VFPI_ERR_NONFINITE, "contact mu/phi not finite");
    if (mu[m] < 0) return arg_fail(c, VFPI_ERR_INVALID_ARG, "contact " + std::to_string(m) + ": mu < 0");
  }
  // internal order: by internal node i (groups contacts by scene, consecutive
  // rows read consecutive records)
  std::vector<int32_t> perm(n_c);
  std::iota(perm.begin(), perm.end(), 0);
  std::sort(perm.begin(), perm.end(), [&](int a, int b) {
    return c->h_node_map[ni[a]] < c->h_node_map[ni[b]];
  });
  c->h_cperm = perm;
  c->h_ci.assign(n_c, -1);
  c->h_cj.assign(n_c, -1);
  std::vector<int32_t> cslot(c->n_pad, -1), dlist;
  std::vector<std::array<int32_t, 3>> split;   // (caller index, internal contact, own row)
  std::vector<int32_t> scene_d(c->n_scenes + 1, 0);
  std::vector<unsigned char> Rint(c->esz * 9 * (size_t)n_c), muint(c->esz * (size_t)n_c),
      phint(c->esz * (size_t)n_c);
  auto put = [&](std::vector<unsigned char>& buf, size_t k, double v) {
    if (c->dtype == VFPI_F64) reinterpret_cast<double*>(buf.data())[k] = v;
    else reinterpret_cast<float*>(buf.data())[k] = (float)v;
  };
  for (int m = 0; m < n_c; ++m) {
    const int e = perm[m];
    const int pi = c->h_node_map[ni[e]];
    const int pj = nj[e] >= 0 ? c->h_node_map[nj[e]] : -1;
    c->h_ci[m] = pi;
    c->h_cj[m] = pj;
    if (pi < c->n_pad) cslot[pi] = m;
    if (pj >= 0) {
      if (pj < c->n_pad) cslot[pj] = m;
      if (pi >= c->n_pad || pj >= c->n_pad) {
        split.push_back({e, m, pi < c->n_pad ? pi : pj});
      } else {
        dlist.push_back(m);
        scene_d[c->h_node_scene[ni[e]] + 1]++;
      }
    }
    for (int q = 0; q < 9; ++q) put(Rint, (size_t)q * n_c + m, R[9 * (size_t)e + q]);
    put(muint, m, mu[e]);
    put(phint, m, phi[e]);
  }
  for (int q = 0; q < c->n_scenes; ++q) scene_d[q + 1] += scene_d[q];
  // split contacts in the caller's order (both shards of a contact list them alike)
  std::sort(split.begin(), split.end());
  std::vector<int32_t> split_cs(split.size()), split_own(split.size());
  for (size_t k = 0; k < split.size(); ++k) {
    split_cs[k] = split[k][1];
    split_own[k] = split[k][2];
  }
  // (re)allocate contact arrays once earlier work on the stream has finished
  VFPI_TRY_CUDA(cudaStreamSynchronize(c->stream));
  c->n_c = n_c;
  c->n_d = (int)dlist.size();
  c->n_split = (int)split.size();
  c->split_ready = 0;
  int32_t* ip[] = {c->d_ci, c->d_cj, c->d_cperm, c->d_dlist, c->d_split_cs, c->d_split_own};
  for (auto p : ip) if (p) cudaFree(p);
  void* vp[] = {c->d_cR, c->d_cmu, c->d_cphi, c->d_comega, c->d_cmu2, c->d_lam, c->d_lam_star,
                c->d_lam2, c->d_lam_star2, c->d_dstar};
  for (auto p : vp) if (p) cudaFree(p);
  VFPI_TRY_CUDA(dalloc(&c->d_ci, 4 * (size_t)n_c));
  VFPI_TRY_CUDA(dalloc(&c->d_cj, 4 * (size_t)n_c));
  VFPI_TRY_CUDA(dalloc(&c->d_cperm, 4 * (size_t)n_c));
  VFPI_TRY_CUDA(dalloc(&c->d_dlist, 4 * dlist.size()));
  VFPI_TRY_CUDA(dalloc(&c->d_split_cs, 4 * split.size()));
  VFPI_TRY_CUDA(dalloc(&c->d_split_own, 4 * split.size()));
  VFPI_TRY_CUDA(dalloc(&c->d_cR, c->esz * 9 * (size_t)n_c));
  VFPI_TRY_CUDA(dalloc(&c->d_cmu, c->esz * (size_t)n_c));
  VFPI_TRY_CUDA(dalloc(&c->d_cphi, c->esz * (size_t)n_c));
  VFPI_TRY_CUDA(dalloc(&c->d_comega, c->esz * (size_t)n_c));
  VFPI_TRY_CUDA(dalloc(&c->d_cmu2, c->esz * (size_t)n_c));
  VFPI_TRY_CUDA(dalloc(&c->d_lam, c->esz * 4 * (size_t)n_c));
  VFPI_TRY_CUDA(dalloc(&c->d_lam_star, c->esz * 4 * (size_t)n_c));
  VFPI_TRY_CUDA(dalloc(&c->d_lam2, c->esz * 4 * (size_t)n_c));
  VFPI_TRY_CUDA(dalloc(&c->d_lam_star2, c->esz * 4 * (size_t)n_c));
  VFPI_TRY_CUDA(dalloc(&c->d_dstar, c->esz * 8 * (size_t)n_c));
  cudaStream_t st = c->stream;
  VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_ci, c->h_ci.data(), 4 * (size_t)n_c, cudaMemcpyHostToDevice, st));
  VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_cj, c->h_cj.data(), 4 * (size_t)n_c, cudaMemcpyHostToDevice, st));
  VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_cperm, perm.data(), 4 * (size_t)n_c, cudaMemcpyHostToDevice, st));
  VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_dlist, dlist.data(), 4 * dlist.size(), cudaMemcpyHostToDevice, st));
  VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_split_cs, split_cs.data(), 4 * split.size(),
                                cudaMemcpyHostToDevice, st));
  VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_split_own, split_own.data(), 4 * split.size(),
                                cudaMemcpyHostToDevice, st));
  VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_cR, Rint.data(), Rint.size(), cudaMemcpyHostToDevice, st));
  VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_cmu, muint.data(), muint.size(), cudaMemcpyHostToDevice, st));
  VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_cmu2, muint.data(), muint.size(), cudaMemcpyHostToDevice, st));
  c->aniso = 0;
  VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_cphi, phint.data(), phint.size(), cudaMemcpyHostToDevice, st));
  VFPI_TRY_CUDA(cudaMemsetAsync(c->d_comega, 0, c->esz * (size_t)n_c, st));
  VFPI_TRY_CUDA(cudaMemsetAsync(c->d_lam, 0, c->esz * 4 * (size_t)n_c, st));
  VFPI_TRY_CUDA(cudaMemsetAsync(c->d_lam_star, 0, c->esz * 4 * (size_t)n_c, st));
  VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_cslot, cslot.data(), 4 * (size_t)c->n_pad, cudaMemcpyHostToDevice, st));
  VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_scene_d, scene_d.data(), 4 * scene_d.size(), cudaMemcpyHostToDevice, st));
  // host vectors must outlive the async copies
  VFPI_TRY_CUDA(cudaStreamSynchronize(st));
  return VFPI_OK;
}

vfpi_status set_w(vfpi_ctx* c) {
  if (c->opts.w_mode == VFPI_W_USER) {
    if (!c->opts.w_user) return arg_fail(c, VFPI_ERR_INVALID_ARG, "w_mode USER needs w_user");
    const size_t bytes = c->esz * 3 * (size_t)c->N;
    std::vector<unsigned char> raw(bytes);
    VFPI_TRY_CUDA(to_host(raw.data(), c->opts.w_user, bytes, c->stream));
    auto wv = [&](size_t k) {
      return c->dtype == VFPI_F64 ? reinterpret_cast<const double*>(raw.data())[k]
                                  : (double)reinterpret_cast<const float*>(raw.data())[k];
    };
    // Prop. 3: the three entries of a contact node (six of a D-contact) are tied
    // (on a shard, over the own endpoint of a split contact: the other shard
    // checks the other one)
    std::vector<int32_t> inv(c->n_pad, -1);
    for (int i = 0; i < c->N; ++i) inv[c->h_node_map[i]] = i;
    for (int m = 0; m < c->n_c; ++m) {
      const int i = inv[c->h_ci[m] < c->n_pad ? c->h_ci[m] : c->h_cj[m]];
      const double w0 = wv(3 * (size_t)i);
      for (int node : {c->h_ci[m], c->h_cj[m]}) {
        if (node < 0 || node >= c->n_pad) continue;
        const int e = inv[node];
        for (int a = 0; a < 3; ++a)
          if (wv(3 * (size_t)e + a) != w0)
            return arg_fail(c, VFPI_ERR_INVALID_ARG, "user W is not tied on contact nodes (Prop. 3)");
      }
    }
    for (size_t k = 0; k < 3 * (size_t)c->N; ++k)
      if (!std::isfinite(wv(k)) || wv(k) <= 0)
        return arg_fail(c, VFPI_ERR_INVALID_ARG, "user W must be positive and finite");
    const void* dv;
    VFPI_TRY_CUDA(device_view(c, c->opts.w_user, bytes, 0, &dv));
    VFPI_TRY_CUDA(cudaMemsetAsync(c->d_w, 0, c->esz * 4 * (size_t)c->n_pad, c->stream));
    VFPI_TRY_CUDA(DISPATCH(c, to_internal(c, dv, c->d_w)));
    return VFPI_OK;
  }
  if (c->opts.w_mode == VFPI_W_SCALAR && !(c->opts.alpha > 0 && std::isfinite(c->opts.alpha)))
    return arg_fail(c, VFPI_ERR_INVALID_ARG, "w_mode SCALAR needs alpha > 0");
  VFPI_TRY_CUDA(DISPATCH(c, make_w(c)));
  return VFPI_OK;
}

vfpi_status read_err(vfpi_ctx* c, int* flags) {
  VFPI_TRY_CUDA(cudaMemcpyAsync(flags, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  VFPI_TRY_CUDA(cudaStreamSynchronize(c->stream));
  return VFPI_OK;
}

// Symmetric storage of A (grid path): on the first call (with the staged
// pattern dcol) size and lay out the upper and lower structures; every call
// checks A = A^T bitwise and scatters the upper values.  A matrix that is not
// symmetric, or too large for 31-bit positions, just leaves sym_ok = 0
// (the solve then reads the full storage, with the same iterates).
vfpi_status set_sym(vfpi_ctx* c, const int32_t* dcol, const void* dv, bool first) {
  if (first) {
    c->sym_ok = 0;
    const int N = c->N;
    VFPI_TRY_CUDA(dalloc(&c->d_col_idx, 4 * (size_t)std::max(c->nnzb, 1)));
    VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_col_idx, dcol, 4 * (size_t)c->nnzb, cudaMemcpyDeviceToDevice, c->stream));
    VFPI_TRY_CUDA(dalloc(&c->d_nlow, 4 * (size_t)std::max(N, 1)));
    VFPI_TRY_CUDA(DISPATCH(c, sym_nlow(c, c->d_row_ptr, c->d_col_idx)));
    std::vector<int32_t> nlow(N), rp(N + 1);
    VFPI_TRY_CUDA(cudaMemcpyAsync(nlow.data(), c->d_nlow, 4 * (size_t)N, cudaMemcpyDeviceToHost, c->stream));
    VFPI_TRY_CUDA(cudaMemcpyAsync(rp.data(), c->d_row_ptr, 4 * ((size_t)N + 1), cudaMemcpyDeviceToHost, c->stream));
    VFPI_TRY_CUDA(cudaStreamSynchronize(c->stream));
    std::vector<int32_t> ulen(c->n_slices, 0), llen(c->n_slices, 0);
    for (int i = 0; i < N; ++i) {
      const int s = c->h_node_map[i] / 32;
      ulen[s] = std::max(ulen[s], rp[i + 1] - rp[i] - nlow[i]);
      llen[s] = std::max(llen[s], nlow[i]);
    }
    std::vector<int64_t> uoff(c->n_slices), loff(c->n_slices);
    int64_t nu = 0, nl = 0;
    for (int s = 0; s < c->n_slices; ++s) {
      uoff[s] = nu;
      loff[s] = nl;
      nu += ulen[s];
      nl += llen[s];
    }
    if ((nu + 1) * 288 >= (int64_t(1) << 31)) return VFPI_OK;   // positions would not fit
    c->n_uent = nu;
    c->n_lent = nl;
    VFPI_TRY_CUDA(dalloc(&c->d_ulen, 4 * (size_t)std::max(c->n_slices, 1)));
    VFPI_TRY_CUDA(dalloc(&c->d_llen, 4 * (size_t)std::max(c->n_slices, 1)));
    VFPI_TRY_CUDA(dalloc(&c->d_uoff, 8 * (size_t)std::max(c->n_slices, 1)));
    VFPI_TRY_CUDA(dalloc(&c->d_loff, 8 * (size_t)std::max(c->n_slices, 1)));
    VFPI_TRY_CUDA(dalloc(&c->d_uvals, c->esz * 288 * (size_t)(nu + 1)));
    VFPI_TRY_CUDA(dalloc(&c->d_ucols, 4 * 32 * (size_t)std::max<int64_t>(nu, 1)));
    VFPI_TRY_CUDA(dalloc(&c->d_lcols, 4 * 32 * (size_t)std::max<int64_t>(nl, 1)));
    VFPI_TRY_CUDA(dalloc(&c->d_lpos, 4 * 32 * (size_t)std::max<int64_t>(nl, 1)));
    VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_ulen, ulen.data(), 4 * (size_t)c->n_slices, cudaMemcpyHostToDevice, c->stream));
    VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_llen, llen.data(), 4 * (size_t)c->n_slices, cudaMemcpyHostToDevice, c->stream));
    VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_uoff, uoff.data(), 8 * (size_t)c->n_slices, cudaMemcpyHostToDevice, c->stream));
    VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_loff, loff.data(), 8 * (size_t)c->n_slices, cudaMemcpyHostToDevice, c->stream));
    VFPI_TRY_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    VFPI_TRY_CUDA(DISPATCH(c, sym_pattern(c)));
    int flags = 0;
    vfpi_status st = read_err(c, &flags);
    if (st != VFPI_OK) return st;
    if (flags) {   // pattern not symmetric: no symmetric storage for this context
      cudaFree(c->d_uvals);
      c->d_uvals = nullptr;
      return VFPI_OK;
    }
  }
  if (!c->d_uvals) return VFPI_OK;
  VFPI_TRY_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  VFPI_TRY_CUDA(DISPATCH(c, sym_values(c, dv, first)));
  int flags = 0;
  vfpi_status st = read_err(c, &flags);
  if (st != VFPI_OK) return st;
  c->sym_ok = flags ? 0 : 1;
  return VFPI_OK;
}

// A's values: checked finite, then scattered into the sliced-ELL layout.  With
// store_cols the pattern (drow, dcol: device copies) is laid out too; without
// it only the values are replaced and the stored pattern is reused.
vfpi_status set_bsym(vfpi_ctx* c);

vfpi_status set_values(vfpi_ctx* c, const int32_t* drow, const int32_t* dcol, const void* vals,
                       bool store_cols, size_t slot) {
  const size_t vbytes = c->esz * 9 * (size_t)c->nnzb;
  const void* dv;
  VFPI_TRY_CUDA(device_view(c, vals, vbytes, slot, &dv));
  VFPI_TRY_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  VFPI_TRY_CUDA(DISPATCH(c, check_finite(dv, 9 * (int64_t)c->nnzb, c->d_err, c->stream)));
  int flags = 0;
  vfpi_status st = read_err(c, &flags);
  if (st != VFPI_OK) return st;
  if (flags) return arg_fail(c, VFPI_ERR_NONFINITE, "A has non-finite values");
  VFPI_TRY_CUDA(DISPATCH(c, build_layout(c, drow, dcol, dv, store_cols)));
  if ((st = set_bsym(c)) != VFPI_OK) return st;
  // (a shard keeps the full storage: its rows see halo columns outside A's square)
  if (c->path == 1 && c->n_halo == 0) return set_sym(c, dcol, dv, store_cols);
  return VFPI_OK;
}

// Symmetric-block storage: whether every stored block equals its transpose
// (checked whenever A is set); vals6 is built when a variant that reads it is
// chosen, and rebuilt with each new A once it exists.
vfpi_status set_bsym(vfpi_ctx* c) {
  c->bsym_ok = 0;
  VFPI_TRY_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  VFPI_TRY_CUDA(DISPATCH(c, block_sym_check(c)));
  int flags = 0;
  vfpi_status st = read_err(c, &flags);
  if (st != VFPI_OK) return st;
  if (flags & 128) return VFPI_OK;
  c->bsym_ok = 1;
  if (c->d_vals6) VFPI_TRY_CUDA(DISPATCH(c, make_vals6(c)));
  return VFPI_OK;
}

vfpi_status ensure_vals6(vfpi_ctx* c) {
  if (!c->b6 || !c->bsym_ok || c->d_vals6) return VFPI_OK;
  VFPI_TRY_CUDA(dalloc(&c->d_vals6, c->esz * 192 * (size_t)std::max<int64_t>(c->n_entries, 1)));
  VFPI_TRY_CUDA(DISPATCH(c, make_vals6(c)));
  return VFPI_OK;
}

vfpi_status set_b(vfpi_ctx* c, const void* b) {
  const size_t bytes = c->esz * 3 * (size_t)c->N;
  const void* db;
  VFPI_TRY_CUDA(device_view(c, b, bytes, 0, &db));
  VFPI_TRY_CUDA(DISPATCH(c, to_internal(c, db, c->d_b)));
  return VFPI_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

void vfpi_default_opts(vfpi_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->dtype = VFPI_F32;
  o->w_mode = VFPI_W_FROBENIUS;
  o->alpha = 0.0;
  o->theta_th = 1e-5;
  o->l_max = 200;
  o->operator_ = VFPI_OP_STRICT;
  o->residual_norm = VFPI_NORM_ABS;
  o->n_scenes = 1;
  o->chebyshev_ls = 0;
  o->chebyshev_u = 1.0;
}

const char* vfpi_status_string(vfpi_status s) {
  switch (s) {
    case VFPI_OK: return "VFPI_OK";
    case VFPI_NOT_CONVERGED: return "VFPI_NOT_CONVERGED";
    case VFPI_ERR_INVALID_ARG: return "VFPI_ERR_INVALID_ARG";
    case VFPI_ERR_NONFINITE: return "VFPI_ERR_NONFINITE";
    case VFPI_ERR_CUDA: return "VFPI_ERR_CUDA";
    case VFPI_ERR_OOM: return "VFPI_ERR_OOM";
    case VFPI_ERR_TIMEOUT: return "VFPI_ERR_TIMEOUT";
    case VFPI_ERR_CONTACT_OVERLAP: return "VFPI_ERR_CONTACT_OVERLAP";
    case VFPI_ERR_UNSUPPORTED: return "VFPI_ERR_UNSUPPORTED";
  }
  return "unknown status";
}

const char* vfpi_last_error(vfpi_t c) { return c ? c->err.c_str() : g_create_error.c_str(); }

void vfpi_destroy(vfpi_t c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_all(c);
  delete c;
}

vfpi_status vfpi_create(const vfpi_bsr* A, const void* b, const vfpi_contacts* Jc, double h,
                        const vfpi_opts* o, void* cuda_stream, vfpi_t* out) {
  g_create_error.clear();
  if (!out) return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!A || !b || !o) return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "A, b and opts are required");
  if (o->dtype != VFPI_F32 && o->dtype != VFPI_F64)
    return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "dtype must be VFPI_F32 or VFPI_F64");
  if (o->operator_ != VFPI_OP_STRICT && o->operator_ != VFPI_OP_PROXIMAL)
    return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "operator_ must be VFPI_OP_STRICT or VFPI_OP_PROXIMAL");
  if (o->l_max < 1) return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "l_max must be >= 1");
  if (o->w_mode < VFPI_W_FROBENIUS || o->w_mode > VFPI_W_USER)
    return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "unknown w_mode");
  if (o->residual_norm != VFPI_NORM_ABS && o->residual_norm != VFPI_NORM_RMS)
    return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "unknown residual_norm");
  if (A->n_nodes < 1 || A->nnzb < A->n_nodes || !A->row_ptr || !A->col_idx || !A->vals)
    return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "A: need n_nodes >= 1, nnzb >= n_nodes and all arrays");
  if ((int64_t)A->n_nodes * 32 > INT32_MAX)
    return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "A: too many nodes");
  if (!(std::isfinite(h))) return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "h must be finite");
  if (o->block_threads && o->block_threads != 64 && o->block_threads != 128 &&
      o->block_threads != 256 && o->block_threads != 512)
    return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "block_threads must be 0, 64, 128, 256 or 512");
  if (o->chebyshev_ls != 0 && (o->chebyshev_ls < 4 || !(o->chebyshev_u > 0 && o->chebyshev_u <= 1)))
    return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "Chebyshev needs l_s >= 4 and 0 < u <= 1");
  if (o->n_halo < 0 || (int64_t)A->n_nodes + o->n_halo > INT32_MAX / 32)
    return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "n_halo must be >= 0 (and the halo not too large)");
  if (o->n_halo > 0) {
    if (o->n_scenes > 1)
      return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "a shard (n_halo > 0) is one scene");
    if (o->force_path == 2)
      return arg_fail(nullptr, VFPI_ERR_UNSUPPORTED, "a shard runs on the grid path");
  }

  vfpi_ctx* c = new (std::nothrow) vfpi_ctx;
  if (!c) return arg_fail(nullptr, VFPI_ERR_OOM, "host allocation failed");
  c->dtype = o->dtype;
  c->esz = o->dtype == VFPI_F64 ? 8 : 4;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->opts = *o;
  c->h = h;
  c->N = A->n_nodes;
  c->nnzb = A->nnzb;
  c->n_scenes = o->n_scenes > 1 ? o->n_scenes : 1;
  c->n_halo = o->n_halo;

  auto fail = [&](vfpi_status st) {
    g_create_error = c->err;
    free_all(c);
    delete c;
    return st;
  };
  auto cuda_err = [&](cudaError_t e, const char* what) { return fail(cuda_fail(c, e, what)); };
#define CREATE_CUDA(expr)                      \
  do {                                         \
    cudaError_t e__ = (expr);                  \
    if (e__ != cudaSuccess) return cuda_err(e__, #expr); \
  } while (0)
#define CREATE_ST(expr)                        \
  do {                                         \
    vfpi_status s__ = (expr);                  \
    if (s__ != VFPI_OK) return fail(s__);      \
  } while (0)

  // scenes
  const int N = c->N;
  c->h_scene_ptr.assign(c->n_scenes + 1, 0);
  if (c->n_scenes > 1) {
    if (!o->scene_ptr) { c->err = "n_scenes > 1 needs scene_ptr"; return fail(VFPI_ERR_INVALID_ARG); }
    CREATE_CUDA(to_host(c->h_scene_ptr.data(), o->scene_ptr, 4 * ((size_t)c->n_scenes + 1), c->stream));
    if (c->h_scene_ptr[0] != 0 || c->h_scene_ptr[c->n_scenes] != N) {
      c->err = "scene_ptr must start at 0 and end at n_nodes";
      return fail(VFPI_ERR_INVALID_ARG);
    }
    for (int q = 0; q < c->n_scenes; ++q)
      if (c->h_scene_ptr[q + 1] <= c->h_scene_ptr[q]) {
        c->err = "scene_ptr must be strictly increasing";
        return fail(VFPI_ERR_INVALID_ARG);
      }
  } else {
    c->h_scene_ptr[1] = N;
  }
  // row pointers on the host: check them; every row's block count decides the
  // internal numbering and the slice lengths
  std::vector<int32_t> row_ptr(N + 1);
  CREATE_CUDA(to_host(row_ptr.data(), A->row_ptr, 4 * ((size_t)N + 1), c->stream));
  if (row_ptr[0] != 0 || row_ptr[N] != A->nnzb) {
    c->err = "row_ptr must start at 0 and end at nnzb";
    return fail(VFPI_ERR_INVALID_ARG);
  }
  for (int i = 0; i < N; ++i) {
    const int len = row_ptr[i + 1] - row_ptr[i];
    if (len < 1 || len > N + c->n_halo) {
      c->err = "row_ptr: every row needs 1..n_nodes (+ n_halo) blocks";
      return fail(VFPI_ERR_INVALID_ARG);
    }
  }
  auto row_len = [&](int i) { return row_ptr[i + 1] - row_ptr[i]; };

  // internal numbering: every scene padded to a multiple of 32 rows.  A slice
  // (32 rows) is padded to its longest row; within a scene whose rows differ
  // in length (the boundary rows of a small lattice), ordering the rows by
  // block count, longest first and otherwise in the given order, gives
  // slices of similar rows.  That order is taken where it stores more than
  // 2 % fewer slots than the given one -- a choice made from the scene's own
  // rows, so a scene gets the same layout alone or in a batch.  The row
  // arithmetic is the same in either order.
  c->h_node_map.resize(N);
  c->h_node_scene.resize(N);
  c->h_scene_slice.assign(c->n_scenes + 1, 0);
  int64_t base = 0;
  std::vector<int32_t> rows_q;
  auto padded_slots = [&](const std::vector<int32_t>& rows) {
    int64_t slots = 0;
    for (size_t k = 0; k < rows.size(); k += 32) {
      int32_t m = 0;
      for (size_t t = k; t < std::min(rows.size(), k + 32); ++t) m = std::max(m, row_len(rows[t]));
      slots += 32 * (int64_t)m;
    }
    return slots;
  };
  for (int q = 0; q < c->n_scenes; ++q) {
    const int s0 = c->h_scene_ptr[q], s1 = c->h_scene_ptr[q + 1];
    c->h_scene_slice[q] = (int32_t)(base / 32);
    rows_q.resize(s1 - s0);
    std::iota(rows_q.begin(), rows_q.end(), s0);
    const int64_t given = padded_slots(rows_q);
    std::stable_sort(rows_q.begin(), rows_q.end(), [&](int a, int b) { return row_len(a) > row_len(b); });
    const int64_t sorted = padded_slots(rows_q);
    const bool use_sorted = sorted * 50 < given * 49;
    for (int k = 0; k < s1 - s0; ++k) {
      const int i = use_sorted ? rows_q[k] : s0 + k;
      c->h_node_map[i] = (int32_t)(base + k);
      c->h_node_scene[i] = q;
    }
    base += (int64_t)round_up(s1 - s0, 32);
  }
  if (base + c->n_halo > INT32_MAX) { c->err = "too many padded rows"; return fail(VFPI_ERR_INVALID_ARG); }
  c->n_pad = (int)base;
  c->n_slices = c->n_pad / 32;
  c->h_scene_slice[c->n_scenes] = c->n_slices;
  // a shard's halo nodes: read by the row products, stored after the padded
  // rows (no slice covers them, so no sweep writes them)
  c->h_node_map.resize((size_t)N + c->n_halo);
  for (int k = 0; k < c->n_halo; ++k) c->h_node_map[(size_t)N + k] = c->n_pad + k;
  c->h_slice_len.assign(c->n_slices, 0);
  for (int i = 0; i < N; ++i) {
    int32_t& sl = c->h_slice_len[c->h_node_map[i] / 32];
    sl = std::max(sl, row_len(i));
  }
  c->h_slice_off.assign(c->n_slices, 0);
  int64_t ent = 0;
  for (int s = 0; s < c->n_slices; ++s) {
    c->h_slice_off[s] = ent;
    ent += c->h_slice_len[s];
  }
  c->n_entries = ent;

  // device allocations (the iterates hold a shard's halo after its rows)
  const size_t vec = c->esz * 4 * ((size_t)c->n_pad + c->n_halo);
  CREATE_CUDA(dalloc(&c->d_slice_len, 4 * (size_t)c->n_slices));
  CREATE_CUDA(dalloc(&c->d_slice_off, 8 * (size_t)c->n_slices));
  CREATE_CUDA(dalloc(&c->d_slice_cmin, 4 * (size_t)std::max(c->n_slices, 1)));
  CREATE_CUDA(dalloc(&c->d_slice_cmax, 4 * (size_t)std::max(c->n_slices, 1)));
  CREATE_CUDA(dalloc(&c->d_vals, c->esz * 288 * (size_t)c->n_entries));
  CREATE_CUDA(dalloc(&c->d_cols, 4 * 32 * (size_t)c->n_entries));
  CREATE_CUDA(dalloc(&c->d_b, vec));
  CREATE_CUDA(dalloc(&c->d_w, vec));
  CREATE_CUDA(dalloc(&c->d_v0, vec));
  CREATE_CUDA(dalloc(&c->d_v1, vec));
  CREATE_CUDA(dalloc(&c->d_t0, vec));
  CREATE_CUDA(dalloc(&c->d_t1, vec));
  CREATE_CUDA(dalloc(&c->d_cslot, 4 * (size_t)c->n_pad));
  CREATE_CUDA(dalloc(&c->d_node_map, 4 * ((size_t)N + c->n_halo)));
  CREATE_CUDA(dalloc(&c->d_sumsq, 8));
  CREATE_CUDA(dalloc(&c->d_row_ptr, 4 * ((size_t)N + 1)));
  CREATE_CUDA(cudaMemcpyAsync(c->d_row_ptr, row_ptr.data(), 4 * ((size_t)N + 1), cudaMemcpyHostToDevice, c->stream));
  CREATE_CUDA(dalloc(&c->d_ds, 8 * 6 * ((size_t)c->n_pad + c->n_halo)));
  CREATE_CUDA(cudaMemsetAsync(c->d_ds, 0, 8 * 6 * ((size_t)c->n_pad + c->n_halo), c->stream));
  CREATE_CUDA(dalloc(&c->d_scene_slice, 4 * ((size_t)c->n_scenes + 1)));
  CREATE_CUDA(dalloc(&c->d_scene_d, 4 * ((size_t)c->n_scenes + 1)));
  CREATE_CUDA(dalloc(&c->d_order, 4 * (size_t)c->n_scenes));
  CREATE_CUDA(dalloc(&c->d_queue, 16));
  CREATE_CUDA(dalloc(&c->d_norm_scale, 8 * (size_t)c->n_scenes));
  CREATE_CUDA(dalloc(&c->d_bar, 16));
  CREATE_CUDA(dalloc(&c->d_err, 16));
  CREATE_CUDA(dalloc(&c->d_iters, 4 * (size_t)c->n_scenes));
  CREATE_CUDA(dalloc(&c->d_status, 4 * (size_t)c->n_scenes));
  CREATE_CUDA(dalloc(&c->d_theta, 8 * (size_t)c->n_scenes));
  CREATE_CUDA(dalloc(&c->d_thscene, 8 * (size_t)c->n_scenes));
  CREATE_CUDA(dalloc(&c->d_slicesq, 8 * (size_t)std::max(c->n_slices, 1)));
  CREATE_CUDA(cudaEventCreate(&c->ev0));
  CREATE_CUDA(cudaEventCreate(&c->ev1));
  cudaStream_t st = c->stream;
  CREATE_CUDA(cudaMemcpyAsync(c->d_slice_len, c->h_slice_len.data(), 4 * (size_t)c->n_slices, cudaMemcpyHostToDevice, st));
  CREATE_CUDA(cudaMemcpyAsync(c->d_slice_off, c->h_slice_off.data(), 8 * (size_t)c->n_slices, cudaMemcpyHostToDevice, st));
  CREATE_CUDA(cudaMemcpyAsync(c->d_node_map, c->h_node_map.data(), 4 * ((size_t)N + c->n_halo),
                              cudaMemcpyHostToDevice, st));
  CREATE_CUDA(cudaMemcpyAsync(c->d_scene_slice, c->h_scene_slice.data(), 4 * ((size_t)c->n_scenes + 1), cudaMemcpyHostToDevice, st));
  // largest scene first; per-scene norm scale
  std::vector<int32_t> order(c->n_scenes);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return c->h_scene_ptr[a + 1] - c->h_scene_ptr[a] > c->h_scene_ptr[b + 1] - c->h_scene_ptr[b];
  });
  std::vector<double> nscale(c->n_scenes, 1.0);
  if (o->residual_norm == VFPI_NORM_RMS)
    for (int q = 0; q < c->n_scenes; ++q)
      nscale[q] = 1.0 / std::sqrt(3.0 * (c->h_scene_ptr[q + 1] - c->h_scene_ptr[q]));
  CREATE_CUDA(cudaMemcpyAsync(c->d_order, order.data(), 4 * (size_t)c->n_scenes, cudaMemcpyHostToDevice, st));
  CREATE_CUDA(cudaMemcpyAsync(c->d_norm_scale, nscale.data(), 8 * (size_t)c->n_scenes, cudaMemcpyHostToDevice, st));
  CREATE_CUDA(cudaMemsetAsync(c->d_v0, 0, vec, st));
  CREATE_CUDA(cudaMemsetAsync(c->d_v1, 0, vec, st));
  CREATE_CUDA(cudaMemsetAsync(c->d_b, 0, vec, st));
  CREATE_CUDA(cudaMemsetAsync(c->d_w, 0, vec, st));
  CREATE_CUDA(cudaMemsetAsync(c->d_t0, 0, vec, st));
  CREATE_CUDA(cudaMemsetAsync(c->d_t1, 0, vec, st));
  CREATE_CUDA(cudaMemsetAsync(c->d_cslot, 0xff, 4 * (size_t)c->n_pad, st));
  CREATE_CUDA(cudaMemsetAsync(c->d_iters, 0, 4 * (size_t)c->n_scenes, st));
  CREATE_CUDA(cudaMemsetAsync(c->d_status, 0, 4 * (size_t)c->n_scenes, st));
  CREATE_CUDA(cudaMemsetAsync(c->d_theta, 0, 8 * (size_t)c->n_scenes, st));

  // stage the pattern (front of the staging buffer), then validate it
  const size_t off_col = 4 * ((size_t)N + 1);
  const size_t off_scene = off_col + 4 * (size_t)c->nnzb;
  const size_t off_vals = round_up(off_scene + 4 * (size_t)N, 256);
  {
    size_t need = off_vals;
    if (!on_device(A->vals)) need += c->esz * 9 * (size_t)c->nnzb;
    CREATE_CUDA(ensure_stage(c, need));
  }
  const int32_t *drow, *dcol, *dscene;
  CREATE_CUDA(device_view(c, A->row_ptr, 4 * ((size_t)N + 1), 0, reinterpret_cast<const void**>(&drow)));
  CREATE_CUDA(device_view(c, A->col_idx, 4 * (size_t)c->nnzb, off_col, reinterpret_cast<const void**>(&dcol)));
  CREATE_CUDA(device_view(c, c->h_node_scene.data(), 4 * (size_t)N, off_scene,
                          reinterpret_cast<const void**>(&dscene)));
  CREATE_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
  CREATE_CUDA(DISPATCH(c, validate_pattern(N, N + c->n_halo, c->n_halo == 0 ? 1 : 0, drow, dcol,
                                           dscene, c->d_err, st)));
  {
    int flags = 0;
    CREATE_ST(read_err(c, &flags));
    if (flags) {
      c->err = std::string("A: invalid block pattern (") + ((flags & 1) ? "column out of range " : "") +
               ((flags & 2) ? (c->n_halo ? "column repeated in a row " : "columns not strictly increasing ")
                            : "") +
               ((flags & 4) ? "block couples two scenes " : "") + ((flags & 16) ? "missing diagonal block" : "") + ")";
      return fail(VFPI_ERR_INVALID_ARG);
    }
  }
  // kernel path (the grid path keeps A in symmetric storage as well, built by set_values)
  c->path = o->force_path ? o->force_path : (c->n_scenes > 1 || c->n_slices <= 64 ? 2 : 1);
  if (c->n_halo > 0) c->path = 1;
  if (c->path != 1 && c->path != 2) { c->err = "force_path must be 0, 1 or 2"; return fail(VFPI_ERR_INVALID_ARG); }
  if (c->path == 1 && c->n_scenes > 1) { c->err = "the grid-wide path solves one scene"; return fail(VFPI_ERR_INVALID_ARG); }
  CREATE_ST(set_values(c, drow, dcol, A->vals, true, off_vals));
  // contacts, b, W
  CREATE_ST(set_contacts(c, Jc));
  {
    const size_t bytes = c->esz * 3 * (size_t)N;
    const void* db;
    CREATE_CUDA(device_view(c, b, bytes, 0, &db));
    CREATE_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
    CREATE_CUDA(DISPATCH(c, check_finite(db, 3 * (int64_t)N, c->d_err, st)));
    int flags = 0;
    CREATE_ST(read_err(c, &flags));
    if (flags) { c->err = "b has non-finite values"; return fail(VFPI_ERR_NONFINITE); }
    CREATE_ST(set_b(c, b));
  }
  CREATE_ST(set_w(c));

  // launch shape
  c->opts.grid_ctas = o->grid_ctas;
  if (!apply_variant(c, o->kernel_variant, o->block_threads)) {
    c->err = "unknown kernel_variant for this path";
    return fail(VFPI_ERR_INVALID_ARG);
  }
  CREATE_ST(ensure_vals6(c));
  if (o->grid_ctas < 0) { c->err = "grid_ctas must be >= 0"; return fail(VFPI_ERR_INVALID_ARG); }
  CREATE_CUDA(DISPATCH(c, configure(c)));
  CREATE_CUDA(dalloc(&c->d_partials, 8 * 3 * (size_t)std::max(c->max_grid, 1)));
  CREATE_CUDA(dalloc(&c->d_bbpart, 8 * 6 * (size_t)std::max(c->max_grid, 1)));
  CREATE_CUDA(dalloc(&c->d_items, 8 * (size_t)std::max(c->max_grid, 1)));
  CREATE_CUDA(cudaStreamSynchronize(st));
  if (c->stage_bytes > (64u << 20)) {  // the copy of a host-side A is no longer needed
    cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_bytes = 0;
  }
  *out = c;
  return VFPI_OK;
#undef CREATE_CUDA
#undef CREATE_ST
}

#define CTX_CHECK(c)                                                            \
  do {                                                                          \
    if (!(c)) return arg_fail(nullptr, VFPI_ERR_INVALID_ARG, "context is NULL"); \
  } while (0)
// calls that need the whole scene (or the sweeps of one launch to meet no
// halo) are not available on a shard
#define NOT_ON_SHARD(c, what)                                                              \
  do {                                                                                     \
    if ((c)->n_halo > 0) return arg_fail(c, VFPI_ERR_UNSUPPORTED, what " is not available on a shard"); \
  } while (0)

vfpi_status vfpi_update(vfpi_t c, const void* A_vals, const void* b, const vfpi_contacts* Jc) {
  CTX_CHECK(c);
  vfpi_status st;
  if (A_vals) {
    if ((st = set_values(c, c->d_row_ptr, nullptr, A_vals, false, 0)) != VFPI_OK) return st;
    c->split_ready = 0;   // the other shards' rows changed too: exchange their statistics again
  }
  if (Jc) {
    if ((st = set_contacts(c, Jc)) != VFPI_OK) return st;
  }
  if (b) {
    const void* db;
    VFPI_TRY_CUDA(device_view(c, b, c->esz * 3 * (size_t)c->N, 0, &db));
    VFPI_TRY_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    VFPI_TRY_CUDA(DISPATCH(c, check_finite(db, 3 * (int64_t)c->N, c->d_err, c->stream)));
    int flags = 0;
    if ((st = read_err(c, &flags)) != VFPI_OK) return st;
    if (flags) return arg_fail(c, VFPI_ERR_NONFINITE, "b has non-finite values");
    VFPI_TRY_CUDA(DISPATCH(c, to_internal(c, db, c->d_b)));
  }
  if (A_vals || Jc) {
    if ((st = set_w(c)) != VFPI_OK) return st;
  }
  return VFPI_OK;
}

vfpi_status vfpi_set_rhs(vfpi_t c, const void* b, const void* phi) {
  CTX_CHECK(c);
  if (b) {
    const void* db;
    VFPI_TRY_CUDA(device_view(c, b, c->esz * 3 * (size_t)c->N, 0, &db));
    VFPI_TRY_CUDA(DISPATCH(c, to_internal(c, db, c->d_b)));
  }
  if (phi && c->n_c > 0) {
    const void* dp;
    VFPI_TRY_CUDA(device_view(c, phi, c->esz * (size_t)c->n_c,
                              round_up(c->esz * 3 * (size_t)c->N, 256), &dp));
    VFPI_TRY_CUDA(DISPATCH(c, contact_scalar(c, dp, c->d_cphi, false)));
  }
  return VFPI_OK;
}

vfpi_status vfpi_set_velocity(vfpi_t c, const void* v) {
  CTX_CHECK(c);
  if (!v) return arg_fail(c, VFPI_ERR_INVALID_ARG, "v is NULL");
  const void* dv;
  VFPI_TRY_CUDA(device_view(c, v, c->esz * 3 * (size_t)c->N, 0, &dv));
  VFPI_TRY_CUDA(DISPATCH(c, to_internal(c, dv, c->d_v0)));
  if (c->n_halo > 0) {   // a shard's solve starts again at sweep 1
    c->shard_l = 1;
    c->shard_cheb = HostChebScalars{};
  }
  return VFPI_OK;
}

static vfpi_status export_vec(vfpi_ctx* c, const void* internal, void* out) {
  const size_t bytes = c->esz * 3 * (size_t)c->N;
  void* dst;
  VFPI_TRY_CUDA(out_view(c, out, bytes, 0, &dst));
  VFPI_TRY_CUDA(DISPATCH(c, to_external(c, internal, dst)));
  if (dst != out) VFPI_TRY_CUDA(to_caller(c, out, dst, bytes));
  return VFPI_OK;
}

vfpi_status vfpi_get_velocity(vfpi_t c, void* v) {
  CTX_CHECK(c);
  if (!v) return arg_fail(c, VFPI_ERR_INVALID_ARG, "v is NULL");
  return export_vec(c, c->d_v0, v);
}

vfpi_status vfpi_get_w(vfpi_t c, void* w) {
  CTX_CHECK(c);
  if (!w) return arg_fail(c, VFPI_ERR_INVALID_ARG, "w is NULL");
  return export_vec(c, c->d_w, w);
}

static vfpi_status export_contact_vec(vfpi_ctx* c, const void* internal, void* out) {
  if (!out) return arg_fail(c, VFPI_ERR_INVALID_ARG, "output is NULL");
  const size_t bytes = c->esz * 3 * (size_t)c->n_c;
  if (bytes == 0) return VFPI_OK;
  void* dst;
  VFPI_TRY_CUDA(out_view(c, out, bytes, 0, &dst));
  VFPI_TRY_CUDA(DISPATCH(c, lambda_external(c, internal, dst)));
  if (dst != out) VFPI_TRY_CUDA(to_caller(c, out, dst, bytes));
  return VFPI_OK;
}

vfpi_status vfpi_get_lambda(vfpi_t c, void* lambda) {
  CTX_CHECK(c);
  return export_contact_vec(c, c->d_lam, lambda);
}

vfpi_status vfpi_get_lambda_star(vfpi_t c, void* lambda_star) {
  CTX_CHECK(c);
  return export_contact_vec(c, c->d_lam_star, lambda_star);
}

vfpi_status vfpi_set_friction(vfpi_t c, const void* mu) {
  CTX_CHECK(c);
  if (!mu) return arg_fail(c, VFPI_ERR_INVALID_ARG, "mu is NULL");
  if (c->n_c == 0) return VFPI_OK;
  const void* dm;
  VFPI_TRY_CUDA(device_view(c, mu, c->esz * (size_t)c->n_c, 0, &dm));
  VFPI_TRY_CUDA(DISPATCH(c, contact_scalar(c, dm, c->d_cmu, false)));
  return VFPI_OK;
}

vfpi_status vfpi_adjoint(vfpi_t c, const void* lambda_star, const void* g_v, void* g_b,
                         void* g_phi, void* g_mu, int32_t* iters_out, double* theta_out) {
  CTX_CHECK(c);
  NOT_ON_SHARD(c, "vfpi_adjoint");
  if (!g_v) return arg_fail(c, VFPI_ERR_INVALID_ARG, "g_v is NULL");
  if (c->aniso)
    return arg_fail(c, VFPI_ERR_UNSUPPORTED, "the adjoint of elliptic friction cones is not built");
  if (c->bb_rule && !lambda_star)
    return arg_fail(c, VFPI_ERR_UNSUPPORTED,
                    "with Barzilai-Borwein steps pass lambda_star of a sweep with the context's W");
  const size_t vec = c->esz * 4 * (size_t)c->n_pad;
  if (!c->d_adj_g) {
    VFPI_TRY_CUDA(dalloc(&c->d_adj_g, vec));
    VFPI_TRY_CUDA(dalloc(&c->d_adj_u0, vec));
    VFPI_TRY_CUDA(dalloc(&c->d_adj_u1, vec));
    VFPI_TRY_CUDA(cudaMemsetAsync(c->d_adj_g, 0, vec, c->stream));
  }
  if (c->adj_nc != c->n_c) {
    VFPI_TRY_CUDA(cudaStreamSynchronize(c->stream));
    for (void* p : {c->d_adj_ls, c->d_adj_gphi, c->d_adj_gmu})
      if (p) cudaFree(p);
    c->d_adj_ls = c->d_adj_gphi = c->d_adj_gmu = nullptr;
    VFPI_TRY_CUDA(dalloc(&c->d_adj_ls, c->esz * 4 * (size_t)c->n_c));
    VFPI_TRY_CUDA(dalloc(&c->d_adj_gphi, c->esz * (size_t)c->n_c));
    VFPI_TRY_CUDA(dalloc(&c->d_adj_gmu, c->esz * (size_t)c->n_c));
    c->adj_nc = c->n_c;
  }
  const size_t vb = c->esz * 3 * (size_t)c->N;
  // frozen active set: the caller's lambda* or the last forward sweep's
  if (lambda_star) {
    const void* dl;
    VFPI_TRY_CUDA(device_view(c, lambda_star, c->esz * 3 * (size_t)c->n_c, 0, &dl));
    VFPI_TRY_CUDA(DISPATCH(c, contact_vec_internal(c, dl, c->d_adj_ls)));
  } else if (c->n_c > 0) {
    VFPI_TRY_CUDA(cudaMemcpyAsync(c->d_adj_ls, c->d_lam_star, c->esz * 4 * (size_t)c->n_c,
                                  cudaMemcpyDeviceToDevice, c->stream));
  }
  const void* dg;
  VFPI_TRY_CUDA(device_view(c, g_v, vb, round_up(c->esz * 3 * (size_t)c->n_c, 256), &dg));
  VFPI_TRY_CUDA(DISPATCH(c, to_internal(c, dg, c->d_adj_g)));
  VFPI_TRY_CUDA(cudaMemsetAsync(c->d_adj_u0, 0, vec, c->stream));
  VFPI_TRY_CUDA(cudaMemsetAsync(c->d_adj_u1, 0, vec, c->stream));
  VFPI_TRY_CUDA(DISPATCH(c, solve(c, c->adj_tol_set ? c->adj_l_max : c->opts.l_max,
                                   c->adj_tol_set ? c->adj_theta_th : c->opts.theta_th, true)));
  vfpi_status run = vfpi_get_status(c, iters_out, theta_out);
  if (run < 0) return run;
  vfpi_status st;
  if (g_b && (st = export_vec(c, c->d_adj_u0, g_b)) != VFPI_OK) return st;
  for (int k = 0; k < 2; ++k) {
    void* out = k == 0 ? g_phi : g_mu;
    if (!out || c->n_c == 0) continue;
    const size_t bytes = c->esz * (size_t)c->n_c;
    void* dst;
    VFPI_TRY_CUDA(out_view(c, out, bytes, 0, &dst));
    VFPI_TRY_CUDA(DISPATCH(c, contact_scalar(c, k == 0 ? c->d_adj_gphi : c->d_adj_gmu, dst, true)));
    if (dst != out) VFPI_TRY_CUDA(to_caller(c, out, dst, bytes));
  }
  return run;
}

vfpi_status vfpi_get_status(vfpi_t c, int32_t* iters_out, double* theta_out) {
  CTX_CHECK(c);
  const int S = c->n_scenes;
  std::vector<int32_t> it(S), stv(S);
  std::vector<double> th(S);
  int err = 0;
  VFPI_TRY_CUDA(cudaMemcpyAsync(it.data(), c->d_iters, 4 * (size_t)S, cudaMemcpyDeviceToHost, c->stream));
  VFPI_TRY_CUDA(cudaMemcpyAsync(stv.data(), c->d_status, 4 * (size_t)S, cudaMemcpyDeviceToHost, c->stream));
  VFPI_TRY_CUDA(cudaMemcpyAsync(th.data(), c->d_theta, 8 * (size_t)S, cudaMemcpyDeviceToHost, c->stream));
  VFPI_TRY_CUDA(cudaMemcpyAsync(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  VFPI_TRY_CUDA(cudaStreamSynchronize(c->stream));
  if (iters_out) std::memcpy(iters_out, it.data(), 4 * (size_t)S);
  if (theta_out) std::memcpy(theta_out, th.data(), 8 * (size_t)S);
  if (err & 1) return arg_fail(c, VFPI_ERR_TIMEOUT, "a grid barrier wait ran out; the iterate is invalid");
  vfpi_status worst = VFPI_OK;
  for (int q = 0; q < S; ++q) {
    if (stv[q] == VFPI_ERR_NONFINITE) {
      return arg_fail(c, VFPI_ERR_NONFINITE, "non-finite residual in scene " + std::to_string(q));
    }
    if (stv[q] == VFPI_NOT_CONVERGED) worst = VFPI_NOT_CONVERGED;
  }
  return worst;
}

vfpi_status vfpi_get_scene_status(vfpi_t c, int32_t* status_out) {
  CTX_CHECK(c);
  if (!status_out) return arg_fail(c, VFPI_ERR_INVALID_ARG, "status_out is required");
  const int S = c->n_scenes;
  std::vector<int32_t> stv(S);
  int err = 0;
  VFPI_TRY_CUDA(cudaMemcpyAsync(stv.data(), c->d_status, 4 * (size_t)S, cudaMemcpyDeviceToHost, c->stream));
  VFPI_TRY_CUDA(cudaMemcpyAsync(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  VFPI_TRY_CUDA(cudaStreamSynchronize(c->stream));
  // a wait that ran out invalidates every scene of that launch
  if (err & 1) std::fill(stv.begin(), stv.end(), (int32_t)VFPI_ERR_TIMEOUT);
  std::memcpy(status_out, stv.data(), 4 * (size_t)S);
  return VFPI_OK;
}

vfpi_status vfpi_solve_async(vfpi_t c) {
  CTX_CHECK(c);
  NOT_ON_SHARD(c, "a multi-sweep solve (use vfpi_shard_sweep)");
  VFPI_TRY_CUDA(DISPATCH(c, solve(c, c->opts.l_max, c->opts.theta_th, false)));
  return VFPI_OK;
}

vfpi_status vfpi_step(vfpi_t c, double* theta_out) {
  CTX_CHECK(c);
  // one sweep: l_max = 1, never "converged" early
  VFPI_TRY_CUDA(DISPATCH(c, solve(c, 1, -1.0, false)));
  if (!theta_out) return VFPI_OK;
  std::vector<double> th(c->n_scenes);
  vfpi_status st = vfpi_get_status(c, nullptr, th.data());
  *theta_out = th[0];
  if (c->n_scenes > 1)
    for (int q = 0; q < c->n_scenes; ++q) theta_out[q] = th[q];
  return st == VFPI_NOT_CONVERGED ? VFPI_OK : st;
}

vfpi_status vfpi_shard_sweep(vfpi_t c, double* sumsq_out) {
  CTX_CHECK(c);
  if (c->path != 1) return arg_fail(c, VFPI_ERR_UNSUPPORTED, "shard sweeps run on the grid path");
  if (c->n_split > 0 && c->opts.w_mode == VFPI_W_FROBENIUS && !c->split_ready)
    return arg_fail(c, VFPI_ERR_INVALID_ARG,
                    "split contacts: set the other endpoints' row statistics first (vfpi_set_split_stats)");
  // one sweep: l_max = 1, never "converged" early; the kernel leaves the
  // sweep's FP64 sum of squares in d_sumsq
  VFPI_TRY_CUDA(DISPATCH(c, solve(c, 1, -1.0, false)));
  if (!sumsq_out) return VFPI_OK;
  double s2 = 0.0;
  VFPI_TRY_CUDA(cudaMemcpyAsync(&s2, c->d_sumsq, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  const vfpi_status st = vfpi_get_status(c, nullptr, nullptr);   // synchronises
  *sumsq_out = s2;
  return st == VFPI_NOT_CONVERGED ? VFPI_OK : st;
}

vfpi_status vfpi_get_nodes(vfpi_t c, const int32_t* nodes, int32_t n, void* out) {
  CTX_CHECK(c);
  if (n < 0 || (n > 0 && (!nodes || !out)))
    return arg_fail(c, VFPI_ERR_INVALID_ARG, "nodes and out are required (n >= 0)");
  if (n == 0) return VFPI_OK;
  // a host list is checked here, so that the gather needs no wait for the
  // device's verdict (the sharded loop calls this every sweep)
  const bool host_nodes = !on_device(nodes);
  if (host_nodes)
    for (int32_t k = 0; k < n; ++k)
      if (nodes[k] < 0 || nodes[k] >= c->N)
        return arg_fail(c, VFPI_ERR_INVALID_ARG, "vfpi_get_nodes: node index out of range");
  const size_t bytes = c->esz * 3 * (size_t)n;
  const size_t slot = round_up(4 * (size_t)n, 256);
  VFPI_TRY_CUDA(ensure_stage(c, slot + bytes));
  const void* dn;
  void* dst;
  VFPI_TRY_CUDA(device_view(c, nodes, 4 * (size_t)n, 0, &dn));
  VFPI_TRY_CUDA(out_view(c, out, bytes, slot, &dst));
  if (!host_nodes) VFPI_TRY_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  VFPI_TRY_CUDA(DISPATCH(c, gather_nodes(c, static_cast<const int32_t*>(dn), n, dst)));
  if (!host_nodes) {
    int flags = 0;
    vfpi_status st = read_err(c, &flags);
    if (st != VFPI_OK) return st;
    if (flags) return arg_fail(c, VFPI_ERR_INVALID_ARG, "vfpi_get_nodes: node index out of range");
  }
  if (dst != out) VFPI_TRY_CUDA(to_caller(c, out, dst, bytes));
  return VFPI_OK;
}

vfpi_status vfpi_set_halo(vfpi_t c, int32_t first, int32_t n, const void* vals) {
  CTX_CHECK(c);
  if (first < 0 || n < 0 || (int64_t)first + n > c->n_halo || (n > 0 && !vals))
    return arg_fail(c, VFPI_ERR_INVALID_ARG, "halo range must lie in [0, n_halo)");
  if (n == 0) return VFPI_OK;
  const void* dv;
  VFPI_TRY_CUDA(device_view(c, vals, c->esz * 3 * (size_t)n, 0, &dv));
  VFPI_TRY_CUDA(DISPATCH(c, set_halo(c, first, n, dv)));
  return VFPI_OK;
}

vfpi_status vfpi_shard_set_theta(vfpi_t c, double theta) {
  CTX_CHECK(c);
  if (c->n_halo == 0) return arg_fail(c, VFPI_ERR_UNSUPPORTED, "vfpi_shard_set_theta is for shards");
  if (!std::isfinite(theta) || theta < 0)
    return arg_fail(c, VFPI_ERR_NONFINITE, "theta must be finite and >= 0");
  const int l = c->shard_l, l_s = c->opts.chebyshev_ls;
  if (l_s > 0) {   // the kernels' recurrence (ChebScalars::advance), same operations
    HostChebScalars& q = c->shard_cheb;
    // eq. (varrho) with the current l: rho = min(theta_{l-1} / theta_{l-2}, 1)
    if (l >= 3) q.rho = q.th2 > 0.0 ? std::fmin(q.th1 / q.th2, 1.0) : 1.0;
    q.th2 = q.th1;
    q.th1 = theta;
    const int ln = l + 1;   // nu of sweep l + 1 (Alg. 3)
    if (ln < l_s) q.nu = 1.0;
    else if (ln == l_s) q.nu = 2.0 / (2.0 - q.rho * q.rho);
    else q.nu = 4.0 / (4.0 - q.rho * q.rho * q.nu);
  }
  c->shard_l = l + 1;
  return VFPI_OK;
}

vfpi_status vfpi_get_shard_info(vfpi_t c, int32_t* info2) {
  CTX_CHECK(c);
  if (!info2) return arg_fail(c, VFPI_ERR_INVALID_ARG, "info is NULL");
  info2[0] = c->n_halo;
  info2[1] = c->n_split;
  return VFPI_OK;
}

vfpi_status vfpi_get_split_stats(vfpi_t c, double* out) {
  CTX_CHECK(c);
  if (c->n_split == 0) return VFPI_OK;
  if (!out) return arg_fail(c, VFPI_ERR_INVALID_ARG, "out is NULL");
  const size_t bytes = 8 * 6 * (size_t)c->n_split;
  void* dst;
  VFPI_TRY_CUDA(out_view(c, out, bytes, 0, &dst));
  // the Frobenius W keeps the statistics of the current A; other modes form them here
  if (c->opts.w_mode != VFPI_W_FROBENIUS) VFPI_TRY_CUDA(DISPATCH(c, row_stats(c)));
  VFPI_TRY_CUDA(DISPATCH(c, split_stats(c, static_cast<double*>(dst))));
  if (dst != out) VFPI_TRY_CUDA(to_caller(c, out, dst, bytes));
  return VFPI_OK;
}

vfpi_status vfpi_set_split_stats(vfpi_t c, const double* partner) {
  CTX_CHECK(c);
  if (c->n_split == 0) return VFPI_OK;
  if (!partner) return arg_fail(c, VFPI_ERR_INVALID_ARG, "partner statistics are required");
  const size_t bytes = 8 * 6 * (size_t)c->n_split;
  std::vector<double> h(6 * (size_t)c->n_split);
  VFPI_TRY_CUDA(to_host(h.data(), partner, bytes, c->stream));
  for (double x : h)
    if (!std::isfinite(x)) return arg_fail(c, VFPI_ERR_NONFINITE, "partner statistics not finite");
  if (c->opts.w_mode != VFPI_W_FROBENIUS) return VFPI_OK;   // W does not use them
  const void* dp;
  VFPI_TRY_CUDA(device_view(c, partner, bytes, 0, &dp));
  VFPI_TRY_CUDA(DISPATCH(c, split_set_stats(c, static_cast<const double*>(dp))));
  c->split_ready = 1;
  return VFPI_OK;
}

vfpi_status vfpi_get_split_vstar(vfpi_t c, void* out) {
  CTX_CHECK(c);
  if (c->n_split == 0) return VFPI_OK;
  if (!out) return arg_fail(c, VFPI_ERR_INVALID_ARG, "out is NULL");
  const size_t bytes = c->esz * 3 * (size_t)c->n_split;
  void* dst;
  VFPI_TRY_CUDA(out_view(c, out, bytes, 0, &dst));
  VFPI_TRY_CUDA(DISPATCH(c, split_vstar(c, dst)));
  if (dst != out) VFPI_TRY_CUDA(to_caller(c, out, dst, bytes));
  return VFPI_OK;
}

vfpi_status vfpi_finish_split(vfpi_t c, const void* partner_vstar, double* sumsq_out) {
  CTX_CHECK(c);
  if (c->n_split > 0) {
    if (!partner_vstar) return arg_fail(c, VFPI_ERR_INVALID_ARG, "partner v* is required");
    const void* dp;
    VFPI_TRY_CUDA(device_view(c, partner_vstar, c->esz * 3 * (size_t)c->n_split, 0, &dp));
    VFPI_TRY_CUDA(DISPATCH(c, split_finish(c, dp)));
  }
  if (!sumsq_out) return VFPI_OK;
  double s2 = 0.0;
  VFPI_TRY_CUDA(cudaMemcpyAsync(&s2, c->d_sumsq, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  const vfpi_status st = vfpi_get_status(c, nullptr, nullptr);   // synchronises
  *sumsq_out = s2;
  return st == VFPI_NOT_CONVERGED ? VFPI_OK : st;
}

vfpi_status vfpi_solve(vfpi_t c, void* v_inout, void* lambda_out, int32_t* iters_out, double* theta_out) {
  CTX_CHECK(c);
  NOT_ON_SHARD(c, "a multi-sweep solve (use vfpi_shard_sweep)");
  vfpi_status st;
  if (v_inout && (st = vfpi_set_velocity(c, v_inout)) != VFPI_OK) return st;
  if ((st = vfpi_solve_async(c)) != VFPI_OK) return st;
  vfpi_status run = vfpi_get_status(c, iters_out, theta_out);
  if (run < 0) return run;
  if (v_inout && (st = vfpi_get_velocity(c, v_inout)) != VFPI_OK) return st;
  if (lambda_out && (st = vfpi_get_lambda(c, lambda_out)) != VFPI_OK) return st;
  return run;
}

vfpi_status vfpi_advance(vfpi_t c, const void* b, const void* phi, const void* v_start,
                         void* v_out, void* lambda_out, double* x, int32_t* iters_out,
                         double* theta_out) {
  CTX_CHECK(c);
  NOT_ON_SHARD(c, "vfpi_advance (use vfpi_shard_sweep)");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  VFPI_TRY_CUDA(cudaStreamIsCapturing(c->stream, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return arg_fail(c, VFPI_ERR_INVALID_ARG,
                    "vfpi_advance waits for its step; inside a stream capture use vfpi_solve_async");
  const size_t vb = c->esz * 3 * (size_t)c->N, pb = c->esz * (size_t)c->n_c;
  const size_t lb = 3 * pb, xb = 8 * 3 * (size_t)c->N;
  // every staging slot is sized first: growing the buffer invalidates views
  size_t top = 0;
  auto slot = [&](size_t bytes) {
    const size_t at = top;
    top += round_up(bytes, 256);
    return at;
  };
  const size_t s_b = slot(vb), s_phi = slot(pb), s_v = slot(vb), s_x = slot(xb);
  const size_t s_vo = slot(vb), s_l = slot(lb);
  VFPI_TRY_CUDA(ensure_stage(c, top));
  cudaStream_t st = c->stream;
  // the positions go up on the side stream, after the stream's earlier work
  // (which may still read the staging buffer), while the solve runs
  double* xdev = x;
  const bool x_staged = x && !on_device(x) && xb > 0;
  if (x_staged) {
    if (!c->aux_stream) {
      VFPI_TRY_CUDA(cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking));
      VFPI_TRY_CUDA(cudaEventCreateWithFlags(&c->ev_main, cudaEventDisableTiming));
      VFPI_TRY_CUDA(cudaEventCreateWithFlags(&c->ev_aux, cudaEventDisableTiming));
    }
    VFPI_TRY_CUDA(cudaEventRecord(c->ev_main, st));
    VFPI_TRY_CUDA(cudaStreamWaitEvent(c->aux_stream, c->ev_main, 0));
    const void* dx;
    VFPI_TRY_CUDA(device_view_queued(c, x, xb, s_x, c->aux_stream, &dx));
    VFPI_TRY_CUDA(cudaEventRecord(c->ev_aux, c->aux_stream));
    xdev = const_cast<double*>(static_cast<const double*>(dx));
  }
  if (b) {
    const void* db;
    VFPI_TRY_CUDA(device_view_queued(c, b, vb, s_b, st, &db));
    VFPI_TRY_CUDA(DISPATCH(c, to_internal(c, db, c->d_b)));
  }
  if (phi && pb > 0) {
    const void* dp;
    VFPI_TRY_CUDA(device_view_queued(c, phi, pb, s_phi, st, &dp));
    VFPI_TRY_CUDA(DISPATCH(c, contact_scalar(c, dp, c->d_cphi, false)));
  }
  if (v_start) {
    const void* dv;
    VFPI_TRY_CUDA(device_view_queued(c, v_start, vb, s_v, st, &dv));
    VFPI_TRY_CUDA(DISPATCH(c, to_internal(c, dv, c->d_v0)));
  }
  VFPI_TRY_CUDA(DISPATCH(c, solve(c, c->opts.l_max, c->opts.theta_th, false)));
  if (v_out) {
    void* dst;
    VFPI_TRY_CUDA(out_view(c, v_out, vb, s_vo, &dst));
    VFPI_TRY_CUDA(DISPATCH(c, to_external(c, c->d_v0, dst)));
    if (dst != v_out) VFPI_TRY_CUDA(cudaMemcpyAsync(v_out, dst, vb, cudaMemcpyDeviceToHost, st));
  }
  if (lambda_out && lb > 0) {
    void* dst;
    VFPI_TRY_CUDA(out_view(c, lambda_out, lb, s_l, &dst));
    VFPI_TRY_CUDA(DISPATCH(c, lambda_external(c, c->d_lam, dst)));
    if (dst != lambda_out)
      VFPI_TRY_CUDA(cudaMemcpyAsync(lambda_out, dst, lb, cudaMemcpyDeviceToHost, st));
  }
  if (x) {
    if (x_staged) VFPI_TRY_CUDA(cudaStreamWaitEvent(st, c->ev_aux, 0));
    VFPI_TRY_CUDA(DISPATCH(c, integrate(c, xdev)));
    if (x_staged) VFPI_TRY_CUDA(cudaMemcpyAsync(x, xdev, xb, cudaMemcpyDeviceToHost, st));
  }
  // the one wait: the status words come back behind everything above
  return vfpi_get_status(c, iters_out, theta_out);
}

vfpi_status vfpi_integrate(vfpi_t c, double* x) {
  CTX_CHECK(c);
  if (!x) return arg_fail(c, VFPI_ERR_INVALID_ARG, "x is NULL");
  const size_t bytes = 8 * 3 * (size_t)c->N;
  if (on_device(x)) {
    VFPI_TRY_CUDA(DISPATCH(c, integrate(c, x)));
    return VFPI_OK;
  }
  const void* dx;
  VFPI_TRY_CUDA(device_view(c, x, bytes, 0, &dx));
  VFPI_TRY_CUDA(DISPATCH(c, integrate(c, const_cast<double*>(static_cast<const double*>(dx)))));
  VFPI_TRY_CUDA(to_caller(c, x, dx, bytes));
  return VFPI_OK;
}

vfpi_status vfpi_matvec(vfpi_t c, const void* x, void* y) {
  CTX_CHECK(c);
  NOT_ON_SHARD(c, "vfpi_matvec");
  if (!x || !y) return arg_fail(c, VFPI_ERR_INVALID_ARG, "x and y are required");
  const void* dx;
  VFPI_TRY_CUDA(device_view(c, x, c->esz * 3 * (size_t)c->N, 0, &dx));
  VFPI_TRY_CUDA(DISPATCH(c, to_internal(c, dx, c->d_t0)));
  VFPI_TRY_CUDA(DISPATCH(c, spmv(c, c->d_t0, c->d_t1)));
  return export_vec(c, c->d_t1, y);
}

vfpi_status vfpi_configure_launch(vfpi_t c, int32_t kernel_variant, int32_t block_threads,
                                  int32_t grid_ctas) {
  CTX_CHECK(c);
  if (block_threads && block_threads != 64 && block_threads != 128 && block_threads != 256 &&
      block_threads != 512)
    return arg_fail(c, VFPI_ERR_INVALID_ARG, "block_threads must be 0, 64, 128, 256 or 512");
  if (grid_ctas < 0) return arg_fail(c, VFPI_ERR_INVALID_ARG, "grid_ctas must be >= 0");
  VFPI_TRY_CUDA(cudaStreamSynchronize(c->stream));
  const Shape saved = shape_of(c);
  if (!apply_variant(c, kernel_variant, block_threads)) {
    restore_shape(c, saved);
    return arg_fail(c, VFPI_ERR_INVALID_ARG, "unknown kernel_variant for this path");
  }
  vfpi_status vst = ensure_vals6(c);
  if (vst != VFPI_OK) {
    restore_shape(c, saved);
    return vst;
  }
  c->opts.grid_ctas = grid_ctas;
  const int old_max = c->max_grid;
  cudaError_t e = DISPATCH(c, configure(c));
  if (e != cudaSuccess) {
    restore_shape(c, saved);
    DISPATCH(c, configure(c));
    return cuda_fail(c, e, "configure");
  }
  if (c->max_grid > old_max) {
    if (c->d_partials) cudaFree(c->d_partials);
    if (c->d_bbpart) cudaFree(c->d_bbpart);
    if (c->d_items) cudaFree(c->d_items);
    c->d_partials = nullptr;
    c->d_bbpart = nullptr;
    c->d_items = nullptr;
    VFPI_TRY_CUDA(dalloc(&c->d_partials, 8 * 3 * (size_t)c->max_grid));
    VFPI_TRY_CUDA(dalloc(&c->d_bbpart, 8 * 6 * (size_t)c->max_grid));
    VFPI_TRY_CUDA(dalloc(&c->d_items, 8 * (size_t)c->max_grid));
  }
  return VFPI_OK;
}

vfpi_status vfpi_last_kernel_ms(vfpi_t c, float* ms) {
  CTX_CHECK(c);
  if (!ms) return arg_fail(c, VFPI_ERR_INVALID_ARG, "ms is NULL");
  if (!c->timed) return arg_fail(c, VFPI_ERR_INVALID_ARG, "no solve launched yet");
  VFPI_TRY_CUDA(cudaEventSynchronize(c->ev1));
  VFPI_TRY_CUDA(cudaEventElapsedTime(ms, c->ev0, c->ev1));
  return VFPI_OK;
}

vfpi_status vfpi_get_layout(vfpi_t c, int64_t* info) {
  CTX_CHECK(c);
  if (!info) return arg_fail(c, VFPI_ERR_INVALID_ARG, "info is NULL");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  info[0] = c->n_pad;
  info[1] = c->n_slices;
  info[2] = 32 * c->n_entries;
  info[3] = c->path;
  info[4] = c->grid;
  info[5] = c->nt;
  info[6] = c->max_grid;
  info[7] = sms;
  return VFPI_OK;
}

vfpi_status vfpi_get_storage(vfpi_t c, int32_t* info) {
  CTX_CHECK(c);
  if (!info) return arg_fail(c, VFPI_ERR_INVALID_ARG, "info is NULL");
  int st = 0;
  if (c->path == 2 && c->cluster > 0) st = 0;
  else if (c->path == 1 && c->tma_stages > 0) st = 0;
  else if (c->path == 1 && c->sym && c->sym_ok) st = 1;
  else if (c->b6 && c->bsym_ok && c->d_vals6) st = 2;
  info[0] = st;
  info[1] = c->bsym_ok;
  info[2] = c->sym_ok;
  info[3] = 0;
  return VFPI_OK;
}

vfpi_status vfpi_set_regularization(vfpi_t c, const void* omega) {
  CTX_CHECK(c);
  if (c->n_c == 0) return VFPI_OK;
  if (!omega) {
    VFPI_TRY_CUDA(cudaMemsetAsync(c->d_comega, 0, c->esz * (size_t)c->n_c, c->stream));
    return VFPI_OK;
  }
  // host check: omega >= 0 and finite (n_c values)
  std::vector<unsigned char> raw(c->esz * (size_t)c->n_c);
  VFPI_TRY_CUDA(to_host(raw.data(), omega, raw.size(), c->stream));
  for (int m = 0; m < c->n_c; ++m) {
    const double x = c->dtype == VFPI_F64 ? reinterpret_cast<const double*>(raw.data())[m]
                                          : (double)reinterpret_cast<const float*>(raw.data())[m];
    if (!(x >= 0) || !std::isfinite(x))
      return arg_fail(c, VFPI_ERR_INVALID_ARG, "omega must be finite and >= 0");
  }
  const void* d;
  VFPI_TRY_CUDA(device_view(c, omega, raw.size(), 0, &d));
  VFPI_TRY_CUDA(DISPATCH(c, contact_scalar(c, d, c->d_comega, false)));
  VFPI_TRY_CUDA(cudaStreamSynchronize(c->stream));
  return VFPI_OK;
}

vfpi_status vfpi_set_anisotropic_friction(vfpi_t c, const void* mu2) {
  CTX_CHECK(c);
  if (!mu2) {
    c->aniso = 0;
    return VFPI_OK;
  }
  if (c->opts.operator_ != VFPI_OP_STRICT)
    return arg_fail(c, VFPI_ERR_UNSUPPORTED, "elliptic friction cones need the strict operator");
  if (c->n_c == 0) return VFPI_OK;
  std::vector<unsigned char> raw(c->esz * (size_t)c->n_c);
  VFPI_TRY_CUDA(to_host(raw.data(), mu2, raw.size(), c->stream));
  for (int m = 0; m < c->n_c; ++m) {
    const double x = c->dtype == VFPI_F64 ? reinterpret_cast<const double*>(raw.data())[m]
                                          : (double)reinterpret_cast<const float*>(raw.data())[m];
    if (!(x >= 0) || !std::isfinite(x))
      return arg_fail(c, VFPI_ERR_INVALID_ARG, "mu2 must be finite and >= 0");
  }
  const void* d;
  VFPI_TRY_CUDA(device_view(c, mu2, raw.size(), 0, &d));
  VFPI_TRY_CUDA(DISPATCH(c, contact_scalar(c, d, c->d_cmu2, false)));
  VFPI_TRY_CUDA(cudaStreamSynchronize(c->stream));
  c->aniso = 1;
  return VFPI_OK;
}

vfpi_status vfpi_set_barzilai_borwein(vfpi_t c, int32_t rule, double alpha0) {
  CTX_CHECK(c);
  if (rule) NOT_ON_SHARD(c, "Barzilai-Borwein");
  if (rule < 0 || rule > 3) return arg_fail(c, VFPI_ERR_INVALID_ARG, "rule must be 0..3");
  if (rule && !(alpha0 > 0 && std::isfinite(alpha0)))
    return arg_fail(c, VFPI_ERR_INVALID_ARG, "alpha0 must be > 0");
  if (rule && c->opts.chebyshev_ls)
    return arg_fail(c, VFPI_ERR_UNSUPPORTED, "Barzilai-Borwein steps and Chebyshev acceleration exclude each other");
  if (rule && !c->d_r0) {
    const size_t vec = c->esz * 4 * (size_t)c->n_pad;
    VFPI_TRY_CUDA(dalloc(&c->d_r0, vec));
    VFPI_TRY_CUDA(dalloc(&c->d_r1, vec));
    VFPI_TRY_CUDA(cudaMemsetAsync(c->d_r0, 0, vec, c->stream));
    VFPI_TRY_CUDA(cudaMemsetAsync(c->d_r1, 0, vec, c->stream));
  }
  c->bb_rule = rule;
  c->bb_alpha0 = alpha0;
  return VFPI_OK;
}

vfpi_status vfpi_set_chebyshev(vfpi_t c, int32_t l_s, double u) {
  CTX_CHECK(c);
  if (l_s != 0 && (l_s < 4 || !(u > 0 && u <= 1)))
    return arg_fail(c, VFPI_ERR_INVALID_ARG, "Chebyshev needs l_s >= 4 and 0 < u <= 1");
  if (l_s && c->bb_rule)
    return arg_fail(c, VFPI_ERR_UNSUPPORTED, "Barzilai-Borwein steps and Chebyshev acceleration exclude each other");
  c->opts.chebyshev_ls = l_s;
  c->opts.chebyshev_u = u;
  return VFPI_OK;
}

vfpi_status vfpi_set_adjoint_chebyshev(vfpi_t c, int32_t l_s, double u) {
  CTX_CHECK(c);
  if (l_s) NOT_ON_SHARD(c, "Chebyshev acceleration");
  if (l_s != 0 && (l_s < 4 || !(u > 0 && u <= 1)))
    return arg_fail(c, VFPI_ERR_INVALID_ARG, "Chebyshev needs l_s >= 4 and 0 < u <= 1");
  c->adj_cheb_ls = l_s;
  c->adj_cheb_u = u;
  return VFPI_OK;
}

vfpi_status vfpi_set_adjoint_tolerance(vfpi_t c, double theta_th, int32_t l_max, int32_t relative) {
  CTX_CHECK(c);
  if (l_max < 1) return arg_fail(c, VFPI_ERR_INVALID_ARG, "l_max must be >= 1");
  if (relative != 0 && relative != 1) return arg_fail(c, VFPI_ERR_INVALID_ARG, "relative must be 0 or 1");
  c->adj_tol_set = 1;
  c->adj_theta_th = theta_th;
  c->adj_l_max = l_max;
  c->adj_rel = relative;
  return VFPI_OK;
}

vfpi_status vfpi_set_tolerance(vfpi_t c, double theta_th, int32_t l_max) {
  CTX_CHECK(c);
  if (l_max < 1) return arg_fail(c, VFPI_ERR_INVALID_ARG, "l_max must be >= 1");
  c->opts.theta_th = theta_th;
  c->opts.l_max = l_max;
  return VFPI_OK;
}

}  // extern "C"
