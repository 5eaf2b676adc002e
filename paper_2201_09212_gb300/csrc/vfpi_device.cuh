// Device code of the V-FPI solver (sm_103a).
//
// Data layout (device, built once per A by the create path):
//   * nodes are renumbered so that every scene starts on a multiple of 32 and
//     32 consecutive internal rows form one "slice" (one warp, one lane per
//     block row);
//   * A is stored sliced-ELL: slice s holds len_s entries per lane (len_s = the
//     longest block row of the slice; shorter rows are padded with zero blocks
//     whose column is the slice's first row).  Entries are grouped in chunks of
//     VW = 16 / sizeof(T) so that each lane reads one 128-bit vector per block
//     component: chunk k of slice s stores the column indices as [32 lanes][VW]
//     and the values as [9 components][32 lanes][VW]; the len_s % VW leftover
//     entries follow as [32 lanes] and [9][32] scalars.  Every warp load is a
//     fully used, contiguous 512-byte (or 128-byte) segment;
//   * vectors (v, b, W) are one 16/32-byte Vec4 per node (x, y, z, pad).
//
// One sweep (Alg. 1 body) is fused into a single pass over the rows: the
// block-row product r = A v - b (eq. pgd1), v* = v - W r, then -- for a node
// carrying an S-contact -- the gather eta = R v* (eq. subp), the one-shot
// strict solve (Alg. 2, eq. operator) with gamma = w_i (Prop. 3), and the
// scatter v^{l+1} = v* + w_i R^T lambda (eq. vup); finally the FP64 partial of
// ||v^{l+1} - v^l||^2.  D-contacts couple two rows and run in a second phase
// after a barrier.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace vfpi {

// status values mirrored from vfpi.h (kept numeric to avoid a C++ dependency)
constexpr int ST_OK = 0;
constexpr int ST_NOT_CONVERGED = 1;
constexpr int ST_NONFINITE = -2;
constexpr int ST_TIMEOUT = -5;

// bounded spin of the grid barrier: polls x sleep >= ~1 s before giving up
constexpr long long kBarrierPolls = 1ll << 24;

template <typename T>
struct alignas(4 * sizeof(T)) Vec4 {
  T x, y, z, w;
};

template <typename T>
struct DevProblem {
  int32_t n_slices;
  int32_t n_pad;                 // padded node count (n_slices * 32)
  const int32_t* slice_len;      // [n_slices] entries per lane
  const int64_t* slice_off;      // [n_slices] offset in entries (1 entry = 32 slots)
  const T* vals;                 // sliced-ELL values
  const T* vals6;                // the same slots, 6 values each, when every block is symmetric
  const int32_t* cols;           // sliced-ELL internal column indices
  const int32_t* slice_cmin;     // [n_slices] smallest / largest column of a slice
  const int32_t* slice_cmax;     //   (padding slots included)
  const Vec4<T>* b;              // [n_pad]
  const Vec4<T>* w;              // [n_pad]
  const int32_t* cslot;          // [n_pad] contact of the node or -1
  int32_t n_c;
  const int32_t* c_i;            // [n_c] internal node i
  const int32_t* c_j;            // [n_c] internal node j or -1 (S-contact)
  const T* c_R;                  // [9][n_c] plane-major rotation entries
  const T* c_mu;                 // [n_c]
  const T* c_phi;                // [n_c]
  const T* c_omega;              // [n_c] regularisation Omega_m = omega_m I (eq. invt)
  const T* c_mu2;                // [n_c] friction along t2 of an elliptic cone
  int prox;                      // ProjectFC: 0 strict, 1 proximal (eq. operator)
  int aniso;                     // elliptic friction cones (strict operator, Prop. 6)
  Vec4<T>* lam;                  // [n_c] lambda of the last sweep (n, t1, t2)
  Vec4<T>* lam_star;             // [n_c] lambda* of the last sweep
  Vec4<T>* lam2;                 // [n_c] the same for odd sweeps under the lagged stop
  Vec4<T>* lam_star2;            //   test (copied to lam / lam_star at the end)
  const Vec4<T>* adj_ls;         // adjoint: frozen lambda* defining the active set
  T* adj_gphi;                   // adjoint: dL/dphi [n_c] (internal order)
  T* adj_gmu;                    // adjoint: dL/dmu  [n_c]
  const int32_t* d_list;         // D-contacts (internal contact ids)
  Vec4<T>* dstar;                // [2 n_c] v* of the two nodes of a D-contact
  Vec4<T>* v0;                   // ping-pong iterates
  Vec4<T>* v1;
  Vec4<T>* r0;                   // Barzilai-Borwein: residuals A v^l - b of the
  Vec4<T>* r1;                   //   current and previous sweep (ping-pong)
  // Symmetric storage (grid path, A = A^T exactly): the blocks with c >= r,
  // sliced like the full storage but each entry lane-contiguous (values
  // [9][32], columns [32]), plus for each row its entries c < r as (column,
  // position of component 0 of block (c, r) in uvals; components 32 apart),
  // chunked like the full storage's columns; padding points at a zero block
  // after the last entry.
  const T* uvals;
  const int32_t* ucols;
  const int32_t* uslice_len;
  const int64_t* uslice_off;
  const int32_t* lcols;
  const int32_t* lpos;
  const int32_t* lslice_len;
  const int64_t* lslice_off;
};

struct SolveCtl {
  int32_t l_max;
  double theta_th;
  const double* norm_scale;      // [n_scenes] 1 or 1/sqrt(n_q)
  double* partials;              // [3][grid] FP64 block partials (grid path; 2 used
                                 //   unless lag_stop)
  unsigned int* bar;             // [1] barrier arrivals, zeroed per launch (grid path)
  int32_t n_scenes;
  const int32_t* order;          // [n_scenes] processing order (largest first)
  const int32_t* scene_slice;    // [n_scenes+1]
  const int32_t* scene_d;        // [n_scenes+1] range in d_list
  int32_t* queue;                // scene work counter (CTA-per-scene path)
  int32_t* iters;                // [n_scenes]
  int32_t* status;               // [n_scenes]
  double* theta;                 // [n_scenes]
  int32_t n_d;                   // total D-contacts (grid path)
  int* err;                      // bit 0: a barrier wait ran out
  int32_t cheb_ls;               // Alg. 3 slow start l_s (0: plain Alg. 1)
  double cheb_u;                 // under-relaxation u
  int32_t bb_rule;               // 0 off; W = alpha_l I with 1 bb1, 2 bb2, 3 alternating
  double bb_alpha0;              // alpha_1
  double* bb_part;               // [2][grid][3] FP64 partials of s.s, s.z, z.z (grid path)
  int32_t* items;                // [grid] work item of each CTA, then [grid / cluster] poison
                                 //   words, zero at launch (cluster path)
  int32_t cache_entries;         // sliced-ELL entries one CTA holds in shared memory (cluster path)
  int32_t smem_bytes;            // dynamic shared memory per CTA (cluster path)
  int32_t theta_rel;             // 1: the adjoint stops at theta < theta_th * ||b|| (same norm)
  const double* th_scene;        // grid path: [1] theta_th * ||b||, computed before the launch
  double* sumsq;                 // grid path: [1] the last sweep's sum ||dv||^2 (before scaling)
  // grid path, a shard's one-sweep launches: the launch's first sweep is sweep
  // l0 of the solve with Chebyshev weight nu0 (else 1 and 1), and swap_end
  // trades the two iterate buffers at the end instead of copying, so that the
  // next launch finds v^{l-1} where Alg. 3 reads it
  int32_t l0;
  double nu0;
  int32_t swap_end;
  // TMA ring kernel: the stop test of sweep l runs while the barrier of sweep
  // l + 1 completes (the sweep after a stop is discarded; same iterates)
  int32_t lag_stop;
};


// alpha_l from the three dot products (Sec. IV.C); the previous value stays
// when the curvature s.z is not positive.
__device__ __forceinline__ double bb_next(int rule, int l, double ss, double sz, double zz,
                                          double prev) {
  const int r = rule == 3 ? ((l & 1) ? 1 : 2) : rule;
  const double a = r == 1 ? ss / sz : (zz > 0.0 ? sz / zz : -1.0);
  return (sz > 0.0 && isfinite(a) && a > 0.0) ? a : prev;
}

// Chebyshev acceleration (Alg. 3): weight of the current sweep and the
// combination v^{l+1} = nu (u (v** - v^l) + v^l - v^{l-1}) + v^{l-1}.
template <typename T>
struct ChebStep {
  int on;       // Alg. 3 active
  int accel;    // l >= l_s: nu from the Chebyshev recurrence (else nu = 1)
  T nu, u;
  int lam_alt = 0;   // lagged stop test: this sweep's lambda goes to lam2 / lam_star2
};

// nu_{l+1} of Alg. 3 from the slow-start index, the estimate rho and nu_l.
__device__ __forceinline__ double cheb_nu(int l, int l_s, double rho, double nu_prev) {
  if (l < l_s) return 1.0;
  if (l == l_s) return 2.0 / (2.0 - rho * rho);
  return 4.0 / (4.0 - rho * rho * nu_prev);
}

// Alg. 3's scalars across sweeps, kept in shared memory (entries 35..38 of a
// kernel's reduction array) and advanced once per sweep by thread 0, the
// thread that forms theta (FP64 divisions are slow on this part, and no other
// thread holds registers for them): after sweep l with residual theta_l, rho
// of eq. (varrho) and the weight nu of sweep l + 1.  reset() before a solve:
// the first sweep's nu is 1.
struct ChebScalars {
  double nu, rho, th1, th2;
  __device__ __forceinline__ void reset() {
    nu = 1.0;
    rho = th1 = th2 = 0.0;
  }
  __device__ __forceinline__ double advance(int l, int l_s, double theta) {
    // eq. (varrho) with the current l: rho = min(theta_{l-1} / theta_{l-2}, 1)
    if (l >= 3) rho = th2 > 0.0 ? fmin(th1 / th2, 1.0) : 1.0;
    th2 = th1;
    th1 = theta;
    nu = cheb_nu(l + 1, l_s, rho, nu);
    return nu;
  }
};

// A kernel's Chebyshev scalars (in its reduction array red[40]), or null when
// the solve is plain Alg. 1; reset by thread 0, the only thread that uses them
// (nu0: the first sweep's weight, 1 unless a shard's launch continues a solve).
__device__ __forceinline__ ChebScalars* cheb_scalars(double* red, int l_s, double nu0 = 1.0) {
  ChebScalars* cs = l_s > 0 ? reinterpret_cast<ChebScalars*>(red + 35) : nullptr;
  if (cs && threadIdx.x == 0) {
    cs->reset();
    cs->nu = nu0;
  }
  return cs;
}

// v** -> v^{l+1}; vp is this row's v^{l-1} (read only when accelerating).
template <typename T>
__device__ __forceinline__ Vec4<T> cheb_combine(const ChebStep<T>& c, const Vec4<T>& vss,
                                                const Vec4<T>& vl, const Vec4<T>* vp_ptr) {
  if (!c.on) return vss;
  Vec4<T> o;
  if (!c.accel) {   // nu = 1: the v^{l-1} terms cancel
    o.x = vl.x + c.u * (vss.x - vl.x);
    o.y = vl.y + c.u * (vss.y - vl.y);
    o.z = vl.z + c.u * (vss.z - vl.z);
  } else {
    const Vec4<T> vp = ldv(vp_ptr);
    o.x = c.nu * (c.u * (vss.x - vl.x) + vl.x - vp.x) + vp.x;
    o.y = c.nu * (c.u * (vss.y - vl.y) + vl.y - vp.y) + vp.y;
    o.z = c.nu * (c.u * (vss.z - vl.z) + vl.z - vp.z) + vp.z;
  }
  o.w = T(0);
  return o;
}

// ---------------------------------------------------------------------------
// loads
// ---------------------------------------------------------------------------

template <typename T>
struct Chunk;
template <>
struct Chunk<float> {
  static constexpr int VW = 4;
  __device__ __forceinline__ static void vals(const float* p, float (&o)[4]) {
    const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
    o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
  }
  __device__ __forceinline__ static void cols(const int32_t* p, int (&o)[4]) {
    const int4 q = __ldcs(reinterpret_cast<const int4*>(p));
    o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
  }
};
template <>
struct Chunk<double> {
  static constexpr int VW = 2;
  __device__ __forceinline__ static void vals(const double* p, double (&o)[2]) {
    const double2 q = __ldcs(reinterpret_cast<const double2*>(p));
    o[0] = q.x; o[1] = q.y;
  }
  __device__ __forceinline__ static void cols(const int32_t* p, int (&o)[2]) {
    const int2 q = __ldcs(reinterpret_cast<const int2*>(p));
    o[0] = q.x; o[1] = q.y;
  }
};

__device__ __forceinline__ Vec4<float> ldv(const Vec4<float>* p) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  return {q.x, q.y, q.z, q.w};
}
__device__ __forceinline__ Vec4<double> ldv(const Vec4<double>* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 c = reinterpret_cast<const double2*>(p)[1];
  return {a.x, a.y, c.x, c.y};
}
__device__ __forceinline__ void stv(Vec4<float>* p, const Vec4<float>& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.x, v.y, v.z, v.w);
}
__device__ __forceinline__ void stv(Vec4<double>* p, const Vec4<double>& v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v.x, v.y);
  reinterpret_cast<double2*>(p)[1] = make_double2(v.z, v.w);
}

// Position of entry e of lane `lane` in a slice with `len` entries at `off`.
// Returns the column index position; *vpos gets the position of component 0
// and *vstride the distance between components.
template <typename T>
__device__ __forceinline__ int64_t slot_pos(int64_t off, int len, int e, int lane, int64_t* vpos,
                                            int* vstride) {
  constexpr int VW = Chunk<T>::VW;
  const int nfull = len / VW;
  if (e < nfull * VW) {
    const int k = e / VW, r = e % VW;
    *vpos = off * 288 + (int64_t)k * (288 * VW) + lane * VW + r;
    *vstride = 32 * VW;
    return off * 32 + (int64_t)k * (32 * VW) + lane * VW + r;
  }
  const int t = e - nfull * VW;
  *vpos = off * 288 + (int64_t)nfull * (288 * VW) + (int64_t)t * 288 + lane;
  *vstride = 32;
  return off * 32 + (int64_t)nfull * (32 * VW) + (int64_t)t * 32 + lane;
}

// ---------------------------------------------------------------------------
// block-row product r = (A v)_row for one lane of a slice
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void row_product(const DevProblem<T>& P, int slice, int lane,
                                            const Vec4<T>* vin, T& a0, T& a1, T& a2) {
  constexpr int VW = Chunk<T>::VW;
  const int len = P.slice_len[slice];
  const int64_t off = P.slice_off[slice];
  const T* __restrict__ vb = P.vals + off * 288;
  const int32_t* __restrict__ cb = P.cols + off * 32;
  a0 = T(0); a1 = T(0); a2 = T(0);
  const int nfull = len / VW;
#pragma unroll 1
  for (int k = 0; k < nfull; ++k) {
    int c[VW];
    T m[9][VW];
    Chunk<T>::cols(cb + (int64_t)k * (32 * VW) + lane * VW, c);
    const T* p = vb + (int64_t)k * (288 * VW) + lane * VW;
#pragma unroll
    for (int q = 0; q < 9; ++q) Chunk<T>::vals(p + q * (32 * VW), m[q]);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const Vec4<T> x = ldv(vin + c[e]);
      a0 = fma(m[0][e], x.x, fma(m[1][e], x.y, fma(m[2][e], x.z, a0)));
      a1 = fma(m[3][e], x.x, fma(m[4][e], x.y, fma(m[5][e], x.z, a1)));
      a2 = fma(m[6][e], x.x, fma(m[7][e], x.y, fma(m[8][e], x.z, a2)));
    }
  }
  const int ntail = len - nfull * VW;
  const T* pt = vb + (int64_t)nfull * (288 * VW) + lane;
  const int32_t* ct = cb + (int64_t)nfull * (32 * VW) + lane;
  for (int t = 0; t < ntail; ++t) {
    const int c = __ldcs(ct + t * 32);
    T m[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) m[q] = __ldcs(pt + t * 288 + q * 32);
    const Vec4<T> x = ldv(vin + c);
    a0 = fma(m[0], x.x, fma(m[1], x.y, fma(m[2], x.z, a0)));
    a1 = fma(m[3], x.x, fma(m[4], x.y, fma(m[5], x.z, a1)));
    a2 = fma(m[6], x.x, fma(m[7], x.y, fma(m[8], x.z, a2)));
  }
}

// Symmetric-block storage: when every stored 3x3 block equals its transpose
// bit for bit (a mass-spring lattice's blocks are multiples of e e^T plus
// diagonal mass), vals6 keeps each slot's (m00, m01, m02, m11, m12, m22) in
// the layout of vals with 6 planes instead of 9 (192 values per slot group
// of 32 rows).  The product rebuilds the 9 entries and runs the same FMAs in
// the same order, so the iterates are bitwise those of the full storage,
// from 24 + 4 instead of 36 + 4 bytes per block.
template <typename T>
__device__ __forceinline__ void expand6(const T (&q)[6], T (&m)[9]) {
  m[0] = q[0]; m[1] = q[1]; m[2] = q[2];
  m[3] = q[1]; m[4] = q[3]; m[5] = q[4];
  m[6] = q[2]; m[7] = q[4]; m[8] = q[5];
}

template <typename T, int UNR = 1>
__device__ __forceinline__ void row_product6(const DevProblem<T>& P, int slice, int lane,
                                             const Vec4<T>* vin, T& a0, T& a1, T& a2) {
  constexpr int VW = Chunk<T>::VW;
  const int len = P.slice_len[slice];
  const int64_t off = P.slice_off[slice];
  const T* __restrict__ vb = P.vals6 + off * 192;
  const int32_t* __restrict__ cb = P.cols + off * 32;
  a0 = T(0); a1 = T(0); a2 = T(0);
  const int nfull = len / VW;
  // UNR = 2: two chunks per iteration, so that the second chunk's loads are in
  // flight during the first one's FMAs (where the register budget allows; the
  // adjoint sweeps keep one chunk: two made the batched adjoint solve 10 %
  // slower)
  auto chunk = [&](int k) {
    int c[VW];
    T q[6][VW];
    Chunk<T>::cols(cb + (int64_t)k * (32 * VW) + lane * VW, c);
    const T* p = vb + (int64_t)k * (192 * VW) + lane * VW;
#pragma unroll
    for (int j = 0; j < 6; ++j) Chunk<T>::vals(p + j * (32 * VW), q[j]);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const Vec4<T> x = ldv(vin + c[e]);
      T qe[6], m[9];
#pragma unroll
      for (int j = 0; j < 6; ++j) qe[j] = q[j][e];
      expand6(qe, m);
      a0 = fma(m[0], x.x, fma(m[1], x.y, fma(m[2], x.z, a0)));
      a1 = fma(m[3], x.x, fma(m[4], x.y, fma(m[5], x.z, a1)));
      a2 = fma(m[6], x.x, fma(m[7], x.y, fma(m[8], x.z, a2)));
    }
  };
  if constexpr (UNR == 2) {
#pragma unroll 2
    for (int k = 0; k < nfull; ++k) chunk(k);
  } else {
#pragma unroll 1
    for (int k = 0; k < nfull; ++k) chunk(k);
  }
  const int ntail = len - nfull * VW;
  const T* pt = vb + (int64_t)nfull * (192 * VW) + lane;
  const int32_t* ct = cb + (int64_t)nfull * (32 * VW) + lane;
  for (int t = 0; t < ntail; ++t) {
    const int c = __ldcs(ct + t * 32);
    T qe[6], m[9];
#pragma unroll
    for (int j = 0; j < 6; ++j) qe[j] = __ldcs(pt + t * 192 + j * 32);
    expand6(qe, m);
    const Vec4<T> x = ldv(vin + c);
    a0 = fma(m[0], x.x, fma(m[1], x.y, fma(m[2], x.z, a0)));
    a1 = fma(m[3], x.x, fma(m[4], x.y, fma(m[5], x.z, a1)));
    a2 = fma(m[6], x.x, fma(m[7], x.y, fma(m[8], x.z, a2)));
  }
}

// Same product with the next chunk's columns and values loaded into registers
// while the current chunk's gathers and FMAs run (twice the bytes in flight
// per warp, same arithmetic in the same order).
template <typename T>
__device__ __forceinline__ void row_product_prefetch(const DevProblem<T>& P, int slice, int lane,
                                                     const Vec4<T>* vin, T& a0, T& a1, T& a2) {
  constexpr int VW = Chunk<T>::VW;
  const int len = P.slice_len[slice];
  const int64_t off = P.slice_off[slice];
  const T* __restrict__ vb = P.vals + off * 288;
  const int32_t* __restrict__ cb = P.cols + off * 32;
  a0 = T(0); a1 = T(0); a2 = T(0);
  const int nfull = len / VW;
  int c[VW];
  T m[9][VW];
  if (nfull > 0) {
    Chunk<T>::cols(cb + lane * VW, c);
#pragma unroll
    for (int q = 0; q < 9; ++q) Chunk<T>::vals(vb + lane * VW + q * (32 * VW), m[q]);
  }
#pragma unroll 1
  for (int k = 0; k < nfull; ++k) {
    int cn[VW];
    T mn[9][VW];
    const bool more = k + 1 < nfull;
    if (more) {
      Chunk<T>::cols(cb + (int64_t)(k + 1) * (32 * VW) + lane * VW, cn);
      const T* p = vb + (int64_t)(k + 1) * (288 * VW) + lane * VW;
#pragma unroll
      for (int q = 0; q < 9; ++q) Chunk<T>::vals(p + q * (32 * VW), mn[q]);
    }
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const Vec4<T> x = ldv(vin + c[e]);
      a0 = fma(m[0][e], x.x, fma(m[1][e], x.y, fma(m[2][e], x.z, a0)));
      a1 = fma(m[3][e], x.x, fma(m[4][e], x.y, fma(m[5][e], x.z, a1)));
      a2 = fma(m[6][e], x.x, fma(m[7][e], x.y, fma(m[8][e], x.z, a2)));
    }
    if (more) {
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        c[e] = cn[e];
#pragma unroll
        for (int q = 0; q < 9; ++q) m[q][e] = mn[q][e];
      }
    }
  }
  const int ntail = len - nfull * VW;
  const T* pt = vb + (int64_t)nfull * (288 * VW) + lane;
  const int32_t* ct = cb + (int64_t)nfull * (32 * VW) + lane;
  for (int t = 0; t < ntail; ++t) {
    const int cc = __ldcs(ct + t * 32);
    T mm[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) mm[q] = __ldcs(pt + t * 288 + q * 32);
    const Vec4<T> x = ldv(vin + cc);
    a0 = fma(mm[0], x.x, fma(mm[1], x.y, fma(mm[2], x.z, a0)));
    a1 = fma(mm[3], x.x, fma(mm[4], x.y, fma(mm[5], x.z, a1)));
    a2 = fma(mm[6], x.x, fma(mm[7], x.y, fma(mm[8], x.z, a2)));
  }
}

// Block-row product from the symmetric storage.  The upper structure keeps
// each entry lane-contiguous -- values [9][32], columns [32] -- so that both
// its owner row and a row reading the block transposed (whose lanes map to
// consecutive rows c) load whole 128-byte lines.  The row's entries c < r
// come first, read back through L2 (their first reader brought them from
// HBM), then its entries c >= r; same order and operations as row_product,
// so the sum is bitwise the same.
template <typename T>
__device__ __forceinline__ void lower_entry(const DevProblem<T>& P, int c, int pos, const Vec4<T>* vin,
                                            T& a0, T& a1, T& a2) {
  const T* b = P.uvals + pos;
  T m[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) m[q] = __ldcg(b + q * 32);
  const Vec4<T> x = ldv(vin + c);
  // (A_rc)_ij = (A_cr)_ji
  a0 = fma(m[0], x.x, fma(m[3], x.y, fma(m[6], x.z, a0)));
  a1 = fma(m[1], x.x, fma(m[4], x.y, fma(m[7], x.z, a1)));
  a2 = fma(m[2], x.x, fma(m[5], x.y, fma(m[8], x.z, a2)));
}

template <typename T>
__device__ __forceinline__ void row_product_sym(const DevProblem<T>& P, int slice, int lane,
                                                const Vec4<T>* vin, T& a0, T& a1, T& a2) {
  constexpr int VW = Chunk<T>::VW;
  a0 = T(0); a1 = T(0); a2 = T(0);
  {
    const int len = P.lslice_len[slice];
    const int64_t off = P.lslice_off[slice];
    const int32_t* __restrict__ cb = P.lcols + off * 32;
    const int32_t* __restrict__ pb = P.lpos + off * 32;
    const int nfull = len / VW;
#pragma unroll 1
    for (int k = 0; k < nfull; ++k) {
      int c[VW], q[VW];
      Chunk<T>::cols(cb + (int64_t)k * (32 * VW) + lane * VW, c);
      Chunk<T>::cols(pb + (int64_t)k * (32 * VW) + lane * VW, q);
#pragma unroll
      for (int e = 0; e < VW; ++e) lower_entry(P, c[e], q[e], vin, a0, a1, a2);
    }
    const int ntail = len - nfull * VW;
    for (int t = 0; t < ntail; ++t) {
      const int64_t o = (int64_t)nfull * (32 * VW) + t * 32 + lane;
      lower_entry(P, __ldcs(cb + o), __ldcs(pb + o), vin, a0, a1, a2);
    }
  }
  const int len = P.uslice_len[slice];
  const int64_t off = P.uslice_off[slice];
  const T* __restrict__ vb = P.uvals + off * 288 + lane;
  const int32_t* __restrict__ cb = P.ucols + off * 32 + lane;
#pragma unroll 2
  for (int e = 0; e < len; ++e) {
    const int c = __ldcs(cb + e * 32);
    T m[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) m[q] = __ldcg(vb + (int64_t)e * 288 + q * 32);   // kept in L2
    const Vec4<T> x = ldv(vin + c);
    a0 = fma(m[0], x.x, fma(m[1], x.y, fma(m[2], x.z, a0)));
    a1 = fma(m[3], x.x, fma(m[4], x.y, fma(m[5], x.z, a1)));
    a2 = fma(m[6], x.x, fma(m[7], x.y, fma(m[8], x.z, a2)));
  }
}

// ---------------------------------------------------------------------------
// one-shot contact solve (Alg. 2, strict operator of eq. operator)
// ---------------------------------------------------------------------------

template <typename T>
struct ContactRec {
  T R[9];
  T mu, phi, omega, mu2;
};

template <typename T>
__device__ __forceinline__ ContactRec<T> load_contact(const DevProblem<T>& P, int cs) {
  ContactRec<T> c;
#pragma unroll
  for (int q = 0; q < 9; ++q) c.R[q] = __ldg(P.c_R + (int64_t)q * P.n_c + cs);
  c.mu = __ldg(P.c_mu + cs);
  c.phi = __ldg(P.c_phi + cs);
  c.omega = __ldg(P.c_omega + cs);
  c.mu2 = __ldg(P.c_mu2 + cs);
  return c;
}

// Nearest point of the ellipse t1^2/a1^2 + t2^2/a2^2 <= 1 to (t1, t2): outside
// it, t_k = a_k^2 t_k / (a_k^2 + nu) with nu > 0 the root of
// sum_k (a_k t_k / (a_k^2 + nu))^2 = 1, bracketed in [0, |a| |t|] and found by
// bisection to the last representable bit (bounded loop).
template <typename T>
__device__ __forceinline__ void ellipse_project(T a1, T a2, T& t1, T& t2) {
  const T A1 = a1 * a1, A2 = a2 * a2;
  if (A1 == T(0) && A2 == T(0)) {   // frictionless
    t1 = t2 = T(0);
    return;
  }
  // inside (multiplied out; a zero semi-axis goes to the bisection, which
  // handles the degenerate segment)
  if (A1 > T(0) && A2 > T(0) && t1 * t1 * A2 + t2 * t2 * A1 <= A1 * A2) return;
  T lo = T(0), hi = sqrt(A1 + A2) * sqrt(t1 * t1 + t2 * t2);
  for (int it = 0; it < 200; ++it) {
    const T mid = T(0.5) * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    const T f1 = a1 * t1 / (A1 + mid), f2 = a2 * t2 / (A2 + mid);
    if (f1 * f1 + f2 * f2 > T(1)) lo = mid; else hi = mid;
  }
  t1 = A1 * t1 / (A1 + hi);
  t2 = A2 * t2 / (A2 + hi);
}

// Given the relative surrogate velocity r = v*_i - v*_j (v*_i for an
// S-contact) and gamma' = gamma + omega (eq. diagonal, eq. invt), compute
// lambda* and lambda = ProjectFC(lambda*) (Alg. 2).
template <typename T>
__device__ __forceinline__ void one_shot(const ContactRec<T>& c, T gamma, T rx, T ry, T rz,
                                         Vec4<T>& ls, Vec4<T>& lam, int prox) {
  // eta = R r  (eq. subp, J_{c,m} v*)
  const T en = c.R[0] * rx + c.R[1] * ry + c.R[2] * rz;
  const T e1 = c.R[3] * rx + c.R[4] * ry + c.R[5] * rz;
  const T e2 = c.R[6] * rx + c.R[7] * ry + c.R[8] * rz;
  // lambda* = -(gamma I)^{-1} (eta + phi e_n)   (Alg. 2)
  ls.x = -(en + c.phi) / gamma;
  ls.y = -e1 / gamma;
  ls.z = -e2 / gamma;
  ls.w = T(0);
  const T rho = sqrt(ls.y * ls.y + ls.z * ls.z);
  lam.w = T(0);
  if (prox == 2) {
    // strict operator, elliptic cone: normal clamp, then the nearest point of
    // the ellipse with semi-axes mu lambda_n, mu2 lambda_n (Prop. 6)
    const T ln = ls.x > T(0) ? ls.x : T(0);
    T t1 = ls.y, t2 = ls.z;
    if (ln > T(0)) ellipse_project(c.mu * ln, c.mu2 * ln, t1, t2);
    else t1 = t2 = T(0);
    lam.x = ln;
    lam.y = t1;
    lam.z = t2;
  } else if (!prox) {
    // strict operator: normal clamp, then projection onto the disk mu*lambda_n
    const T ln = ls.x > T(0) ? ls.x : T(0);
    const T rad = c.mu * ln;
    const T s = (rho <= rad) ? T(1) : rad / rho;
    lam.x = ln;
    lam.y = s * ls.y;
    lam.z = s * ls.z;
  } else {
    // proximal operator: Euclidean projection onto the friction cone
    if (rho <= c.mu * ls.x) {
      lam.x = ls.x; lam.y = ls.y; lam.z = ls.z;
    } else if (c.mu * rho <= -ls.x) {
      lam.x = T(0); lam.y = T(0); lam.z = T(0);
    } else {
      const T ln = (ls.x + c.mu * rho) / (T(1) + c.mu * c.mu);
      const T s = c.mu * ln / rho;
      lam.x = ln;
      lam.y = s * ls.y;
      lam.z = s * ls.z;
    }
  }
}

// R^T lambda
template <typename T>
__device__ __forceinline__ void rt_lambda(const ContactRec<T>& c, const Vec4<T>& l, T& dx, T& dy,
                                          T& dz) {
  dx = c.R[0] * l.x + c.R[3] * l.y + c.R[6] * l.z;
  dy = c.R[1] * l.x + c.R[4] * l.y + c.R[7] * l.z;
  dz = c.R[2] * l.x + c.R[5] * l.y + c.R[8] * l.z;
}

// Adjoint of the contact step at a frozen active set.  With
// S = W J^T P' Gamma'^{-1} J (P' the Jacobian of ProjectFC at the frozen
// lambda*, Gamma' = Gamma + Omega), the transpose iteration on
// u = W (I - S^T) g_bar reads u_new = u* - (1/gamma') W J^T P'^T J u*; for one
// contact, z = R (u*_i - u*_j) and q = P'^T z.  Returns q; also
// dL/dphi = -q_n / gamma' and dL/dmu = z . dProjectFC/dmu.
template <typename T>
__device__ __forceinline__ void adjoint_step(const ContactRec<T>& c, const Vec4<T>& ls, T gamma,
                                             T rx, T ry, T rz, Vec4<T>& q, T& gphi, T& gmu,
                                             int prox) {
  const T zn = c.R[0] * rx + c.R[1] * ry + c.R[2] * rz;
  const T z1 = c.R[3] * rx + c.R[4] * ry + c.R[5] * rz;
  const T z2 = c.R[6] * rx + c.R[7] * ry + c.R[8] * rz;
  q = Vec4<T>{T(0), T(0), T(0), T(0)};
  gmu = T(0);
  const T a = ls.x;
  const T rho = sqrt(ls.y * ls.y + ls.z * ls.z);
  if (!prox) {
    if (a > T(0)) {
      if (rho <= c.mu * a) {            // stick: P' = I
        q.x = zn; q.y = z1; q.z = z2;
      } else {                          // slip
        const T t1 = ls.y / rho, t2 = ls.z / rho;
        const T tz = t1 * z1 + t2 * z2;
        const T kap = c.mu * a / rho;
        q.x = zn + c.mu * tz;
        q.y = kap * (z1 - t1 * tz);
        q.z = kap * (z2 - t2 * tz);
        gmu = a * tz;
      }
    }
  } else {
    if (rho <= c.mu * a) {              // inside the cone: P' = I
      q.x = zn; q.y = z1; q.z = z2;
    } else if (!(c.mu * rho <= -a)) {   // on the cone's surface (polar cone: 0)
      const T t1 = ls.y / rho, t2 = ls.z / rho;
      const T tz = t1 * z1 + t2 * z2;
      const T k = T(1) + c.mu * c.mu;
      const T ln = (a + c.mu * rho) / k;
      const T kap = c.mu * ln / rho;
      // P' = [dln; mu t dln + kap (I - t t^T)] with dln = [1, mu t] / k
      const T w = (zn + c.mu * tz) / k;  // dln . z summed over the rows that carry dln
      q.x = w;
      q.y = c.mu * t1 * w + kap * (z1 - t1 * tz);
      q.z = c.mu * t2 * w + kap * (z2 - t2 * tz);
      const T dln_dmu = (rho * k - T(2) * c.mu * (a + c.mu * rho)) / (k * k);
      gmu = zn * dln_dmu + (ln + c.mu * dln_dmu) * tz;
    }
  }
  gphi = -q.x / gamma;
}

// One row's ||v^{l+1} - v^l||^2 in the iterate's own precision; the rows'
// terms are summed in FP64 in a fixed order (the residual reduction of
// Alg. 1).  In FP32 the rounding of the squares (a few 1e-7 of theta) is far
// below that of the FP32 iterates' difference itself (up to ulp(v) / |dv|
// near convergence); FP64 arithmetic per row measured 12 % of a sweep on a
// latency-bound scene (the FEM block, 215k DOF).
template <typename T>
__device__ __forceinline__ double sqdiff(const Vec4<T>& a, const Vec4<T>& b) {
  const T dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return (double)(dx * dx + dy * dy + dz * dz);
}

// One row of one sweep after its block-row product (a0, a1, a2) = (A v)_row:
// returns the row's contribution to ||dv||^2 (0 for a D-contact node, whose
// update happens in phase 2).  ADJ selects the adjoint sweep (b is then dL/dv
// and the contact step is the frozen linear map).
// (vo, bb, ww, cs) = (v^l, b, W, contact slot) of the row, wherever they were read
// from; out = where v^{l+1} of the row goes (holding v^{l-1}, which Chebyshev reads).
template <typename T, bool ADJ>
__device__ __forceinline__ double finish_row_core(const DevProblem<T>& P, int row, T a0, T a1, T a2,
                                                  const Vec4<T>& vo, const Vec4<T>& bb,
                                                  const Vec4<T>& ww, int cs, Vec4<T>* out,
                                                  const ChebStep<T>& ch) {
  // eq. (pgd1): v* = v - W (A v - b)
  Vec4<T> vn;
  vn.x = vo.x - ww.x * (a0 - bb.x);
  vn.y = vo.y - ww.y * (a1 - bb.y);
  vn.z = vo.z - ww.z * (a2 - bb.z);
  vn.w = T(0);
  if (cs >= 0) {
    const int cj = __ldg(P.c_j + cs);
    if (cj >= 0) {  // D-contact: stage v* and finish in phase 2
      stv(P.dstar + 2 * cs + (row == cj ? 1 : 0), vn);
      return 0.0;
    }
    const ContactRec<T> c = load_contact(P, cs);
    const T gam = ww.x + c.omega;                    // gamma = w_i (Prop. 3), + omega (eq. invt)
    if constexpr (ADJ) {
      Vec4<T> q;
      T gphi, gmu;
      adjoint_step(c, ldv(P.adj_ls + cs), gam, vn.x, vn.y, vn.z, q, gphi, gmu, P.prox);
      T dx, dy, dz;
      rt_lambda(c, q, dx, dy, dz);
      const T f = ww.x / gam;
      vn.x -= f * dx;
      vn.y -= f * dy;
      vn.z -= f * dz;
      P.adj_gphi[cs] = gphi;
      P.adj_gmu[cs] = gmu;
    } else {
      Vec4<T> ls, lam;
      one_shot(c, gam, vn.x, vn.y, vn.z, ls, lam, P.aniso ? 2 : P.prox);
      T dx, dy, dz;
      rt_lambda(c, lam, dx, dy, dz);
      vn.x += ww.x * dx;                               // eq. (vup)
      vn.y += ww.x * dy;
      vn.z += ww.x * dz;
      stv((ch.lam_alt ? P.lam2 : P.lam) + cs, lam);
      stv((ch.lam_alt ? P.lam_star2 : P.lam_star) + cs, ls);
    }
  }
  vn = cheb_combine(ch, vn, vo, out);   // *out holds v^{l-1} (u^{l-1} in the adjoint)
  stv(out, vn);
  return sqdiff(vn, vo);
}

template <typename T, bool ADJ>
__device__ __forceinline__ double finish_row(const DevProblem<T>& P, int row, T a0, T a1, T a2,
                                             const Vec4<T>* vin, Vec4<T>* vout,
                                             const ChebStep<T>& ch) {
  return finish_row_core<T, ADJ>(P, row, a0, a1, a2, ldv(vin + row), ldv(P.b + row),
                                 ldv(P.w + row), __ldg(P.cslot + row), vout + row, ch);
}

template <typename T, bool ADJ, bool PF = false, bool SYM = false, bool B6 = false, int U6 = 1>
__device__ __forceinline__ double sweep_row(const DevProblem<T>& P, int slice, int lane,
                                            const Vec4<T>* vin, Vec4<T>* vout,
                                            const ChebStep<T>& ch) {
  T a0, a1, a2;
  if constexpr (B6) row_product6<T, U6>(P, slice, lane, vin, a0, a1, a2);
  else if constexpr (SYM) row_product_sym(P, slice, lane, vin, a0, a1, a2);
  else if constexpr (PF) row_product_prefetch(P, slice, lane, vin, a0, a1, a2);
  else row_product(P, slice, lane, vin, a0, a1, a2);
  return finish_row<T, ADJ>(P, slice * 32 + lane, a0, a1, a2, vin, vout, ch);
}

// Barzilai-Borwein sweep, phase A: r_l = A v^l - b for this row (stored), and
// the row's share of s.s, s.z, z.z with s = v^l - v^{l-1} (v^{l-1} is still in
// the output buffer) and z = r_l - r_{l-1}.
template <typename T>
__device__ __forceinline__ void bb_residual_row(const DevProblem<T>& P, int slice, int lane,
                                                const Vec4<T>* vin, const Vec4<T>* vold,
                                                Vec4<T>* rcur, const Vec4<T>* rprev, bool first,
                                                double& ss, double& sz, double& zz) {
  T a0, a1, a2;
  row_product(P, slice, lane, vin, a0, a1, a2);
  const int row = slice * 32 + lane;
  const Vec4<T> bb = ldv(P.b + row);
  const Vec4<T> r = {a0 - bb.x, a1 - bb.y, a2 - bb.z, T(0)};
  stv(rcur + row, r);
  if (first) return;
  const Vec4<T> vl = ldv(vin + row), vp = ldv(vold + row), rp = ldv(rprev + row);
  const double s0 = (double)vl.x - vp.x, s1 = (double)vl.y - vp.y, s2 = (double)vl.z - vp.z;
  const double z0 = (double)r.x - rp.x, z1 = (double)r.y - rp.y, z2 = (double)r.z - rp.z;
  ss += s0 * s0 + s1 * s1 + s2 * s2;
  sz += s0 * z0 + s1 * z1 + s2 * z2;
  zz += z0 * z0 + z1 * z1 + z2 * z2;
}

// Phase B: v* = v^l - alpha r_l (eq. pgd1 with W = alpha I), then the contact
// step as in sweep_row with gamma = alpha (+ omega).
template <typename T>
__device__ __forceinline__ double bb_update_row(const DevProblem<T>& P, int slice, int lane,
                                                const Vec4<T>* vin, Vec4<T>* vout,
                                                const Vec4<T>* rcur, T alpha) {
  const int row = slice * 32 + lane;
  const Vec4<T> vo = ldv(vin + row);
  const Vec4<T> r = ldv(rcur + row);
  Vec4<T> vn = {vo.x - alpha * r.x, vo.y - alpha * r.y, vo.z - alpha * r.z, T(0)};
  const int cs = __ldg(P.cslot + row);
  if (cs >= 0) {
    const int cj = __ldg(P.c_j + cs);
    if (cj >= 0) {
      stv(P.dstar + 2 * cs + (row == cj ? 1 : 0), vn);
      return 0.0;
    }
    const ContactRec<T> c = load_contact(P, cs);
    Vec4<T> ls, lam;
    one_shot(c, alpha + c.omega, vn.x, vn.y, vn.z, ls, lam, P.aniso ? 2 : P.prox);
    T dx, dy, dz;
    rt_lambda(c, lam, dx, dy, dz);
    vn.x += alpha * dx;
    vn.y += alpha * dy;
    vn.z += alpha * dz;
    stv(P.lam + cs, lam);
    stv(P.lam_star + cs, ls);
  }
  stv(vout + row, vn);
  return sqdiff(vn, vo);
}

// D-contact step with W = alpha I (gamma = 2 alpha + omega).
template <typename T>
__device__ __forceinline__ double bb_d_contact(const DevProblem<T>& P, int cs, const Vec4<T>* vin,
                                               Vec4<T>* vout, T alpha) {
  const int i = P.c_i[cs], j = P.c_j[cs];
  const Vec4<T> si = ldv(P.dstar + 2 * cs), sj = ldv(P.dstar + 2 * cs + 1);
  const ContactRec<T> c = load_contact(P, cs);
  Vec4<T> ls, lam;
  one_shot(c, alpha + alpha + c.omega, si.x - sj.x, si.y - sj.y, si.z - sj.z, ls, lam,
           P.aniso ? 2 : P.prox);
  T dx, dy, dz;
  rt_lambda(c, lam, dx, dy, dz);
  const Vec4<T> ni = {si.x + alpha * dx, si.y + alpha * dy, si.z + alpha * dz, T(0)};
  const Vec4<T> nj = {sj.x - alpha * dx, sj.y - alpha * dy, sj.z - alpha * dz, T(0)};
  stv(vout + i, ni);
  stv(vout + j, nj);
  stv(P.lam + cs, lam);
  stv(P.lam_star + cs, ls);
  return sqdiff(ni, ldv(vin + i)) + sqdiff(nj, ldv(vin + j));
}

// Alg. 2 for D-contact cs from the v* of its nodes (si at node i, sj at node
// j) and their W: stores lambda and lambda*, returns both nodes' eq. (vup) values.
template <typename T>
__device__ __forceinline__ void d_contact_step(const DevProblem<T>& P, int cs, const Vec4<T>& si,
                                               const Vec4<T>& sj, T wi, T wj, Vec4<T>& ni,
                                               Vec4<T>& nj) {
  const ContactRec<T> c = load_contact(P, cs);
  const T gamma = wi + wj + c.omega;                       // eq. (diagonal), D-contact; eq. (invt)
  Vec4<T> ls, lam;
  one_shot(c, gamma, si.x - sj.x, si.y - sj.y, si.z - sj.z, ls, lam, P.aniso ? 2 : P.prox);
  T dx, dy, dz;
  rt_lambda(c, lam, dx, dy, dz);
  ni = {si.x + wi * dx, si.y + wi * dy, si.z + wi * dz, T(0)};
  nj = {sj.x - wj * dx, sj.y - wj * dy, sj.z - wj * dz, T(0)};
  stv(P.lam + cs, lam);
  stv(P.lam_star + cs, ls);
}

// Phase 2: D-contact d between internal nodes i and j (both rows hold v*).
template <typename T, bool ADJ>
__device__ __forceinline__ double d_contact(const DevProblem<T>& P, int cs, const Vec4<T>* vin,
                                            Vec4<T>* vout, const ChebStep<T>& ch) {
  const int i = P.c_i[cs], j = P.c_j[cs];
  const Vec4<T> si = ldv(P.dstar + 2 * cs), sj = ldv(P.dstar + 2 * cs + 1);
  const T wi = P.w[i].x, wj = P.w[j].x;
  Vec4<T> ni, nj;
  if constexpr (ADJ) {
    const ContactRec<T> c = load_contact(P, cs);
    const T gamma = wi + wj + c.omega;
    Vec4<T> q;
    T gphi, gmu;
    adjoint_step(c, ldv(P.adj_ls + cs), gamma, si.x - sj.x, si.y - sj.y, si.z - sj.z, q, gphi, gmu,
                 P.prox);
    T dx, dy, dz;
    rt_lambda(c, q, dx, dy, dz);
    const T fi = wi / gamma, fj = wj / gamma;
    ni = {si.x - fi * dx, si.y - fi * dy, si.z - fi * dz, T(0)};
    nj = {sj.x + fj * dx, sj.y + fj * dy, sj.z + fj * dz, T(0)};
    P.adj_gphi[cs] = gphi;
    P.adj_gmu[cs] = gmu;
  } else {
    d_contact_step(P, cs, si, sj, wi, wj, ni, nj);
  }
  const Vec4<T> oi = ldv(vin + i), oj = ldv(vin + j);
  ni = cheb_combine(ch, ni, oi, vout + i);
  nj = cheb_combine(ch, nj, oj, vout + j);
  stv(vout + i, ni);
  stv(vout + j, nj);
  return sqdiff(ni, oi) + sqdiff(nj, oj);
}

// ---------------------------------------------------------------------------
// reductions and the bounded grid barrier
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Sum over the block in a fixed order; every thread receives the result.
template <int NT>
__device__ __forceinline__ double block_allreduce(double x, double* red) {
  x = warp_sum(x);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = x;
  __syncthreads();
  if (wid == 0) {
    double y = lane < NT / 32 ? red[lane] : 0.0;
    y = warp_sum(y);
    if (lane == 0) red[32] = y;
  }
  __syncthreads();
  return red[32];
}

// The same sum, and theta = sqrt(sum) * nscale of Alg. 1 formed once (FP64
// square roots are slow on this part) and handed to every thread with the sum,
// with the next sweep's Chebyshev weight (1 when cs is null); red needs 40
// entries.
template <int NT>
__device__ __forceinline__ double block_allreduce_theta(double x, double* red, double nscale,
                                                        ChebScalars* cs, int l, int l_s,
                                                        double* theta, double* nu) {
  x = warp_sum(x);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = x;
  __syncthreads();
  if (wid == 0) {
    double y = lane < NT / 32 ? red[lane] : 0.0;
    y = warp_sum(y);
    if (lane == 0) {
      const double th = sqrt(y) * nscale;
      red[32] = y;
      red[33] = th;
      red[34] = cs ? cs->advance(l, l_s, th) : 1.0;
    }
  }
  __syncthreads();
  *theta = red[33];
  *nu = red[34];
  return red[32];
}

// All CTAs arrive; returns false if the wait ran out (the caller then stops).
// Co-residency of all CTAs is guaranteed by the cooperative launch; the spin
// is bounded anyway so that a fault elsewhere can never hang the GPU.
// One counter that only grows within a launch (zeroed before it): barrier k
// of the launch is passed once it reads k * gridDim.x.  Each CTA arrives with
// a posted reduction (red.release: nothing to wait for, unlike an atomic that
// returns a ticket) that publishes what the CTA wrote before it; the wait
// reads the counter with acquire loads, so a CTA that sees every arrival sees
// every CTA's writes.  `nb` is the CTA's count of barriers passed times
// gridDim.x (the same in every CTA: all take the same barriers).
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int& nb, int* s_ok) {
  __syncthreads();
  nb += gridDim.x;
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    int ok = 0;
    for (long long it = 0; it < kBarrierPolls; ++it) {
      if (ld_acquire_gpu(bar) >= nb) { ok = 1; break; }
      if (it > 64) __nanosleep(32);
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// End of a grid-wide sweep: the CTA's FP64 sum of its threads' partials, the
// grid barrier (as grid_barrier) and the fixed-order sum of every CTA's
// partial -- computed alike by every CTA, so all take the same stop decision
// -- with two block barriers: warp 0 sums the threads' partials, lane 0
// publishes the CTA's sum and arrives and waits, __syncwarp passes its acquire
// on to the warp, which sums the CTAs' partials, and lane 0 forms theta and
// the next Chebyshev weight; the other warps wait at the second block barrier.
// `part` is this sweep's half of the partials (the other half may still be
// read by a CTA that is one barrier behind).
template <int NT>
__device__ __forceinline__ bool sweep_sum_barrier(double acc, double* part, unsigned int* bar,
                                                  unsigned int& nb, double* red, int* s_ok,
                                                  double nscale, ChebScalars* cs, int l, int l_s,
                                                  double* total, double* theta, double* nu) {
  // every thread's partial staged, warp 0 alone adds them (FP64 adds are slow
  // on this part: NT / 32 + 4 of them in one warp instead of 5 in every warp)
  __shared__ double stage[NT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  stage[threadIdx.x] = acc;
  __syncthreads();   // every row of this sweep written, every thread's partial staged
  nb += gridDim.x;
  if (wid == 0) {
    double y = stage[lane];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) y += stage[w * 32 + lane];
    y = warp_sum(y);
    int ok = 0;
    if (lane == 0) {
      part[blockIdx.x] = y;
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
      for (long long it = 0; it < kBarrierPolls; ++it) {
        if (ld_acquire_gpu(bar) >= nb) { ok = 1; break; }
        if (it > 64) __nanosleep(32);
      }
    }
    __syncwarp();
    ok = __shfl_sync(0xffffffffu, ok, 0);
    double s2w = 0.0;
    for (int q = lane; q < (int)gridDim.x; q += 32) s2w += part[q];
    s2w = warp_sum(s2w);
    if (lane == 0) {
      const double th = sqrt(s2w) * nscale;   // theta of Alg. 1, formed once per CTA
      red[32] = s2w;
      red[33] = th;
      red[34] = cs ? cs->advance(l, l_s, th) : 1.0;
      *s_ok = ok;
    }
  }
  __syncthreads();
  *total = red[32];
  *theta = red[33];
  *nu = red[34];
  return *s_ok != 0;
}

// The same end of sweep with the stop test one sweep behind: warp 0 publishes
// the CTA's partial of this sweep and arrives, then -- while the other CTAs
// arrive -- adds the previous sweep's partials (complete since the last
// barrier; `prev` null on the first sweep) in the same fixed order, and only
// then waits.  *total / *theta are the previous sweep's.  Three rotating
// slices of partials: a CTA still adding sweep l - 1's while a faster one
// publishes sweep l + 1's reads another slice.
template <int NT>
__device__ __forceinline__ bool sweep_sum_barrier_lag(double acc, double* part, const double* prev,
                                                      unsigned int* bar, unsigned int& nb,
                                                      double* red, int* s_ok, double nscale,
                                                      double* total, double* theta) {
  __shared__ double stage[NT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  stage[threadIdx.x] = acc;
  __syncthreads();   // every row of this sweep written, every thread's partial staged
  nb += gridDim.x;
  if (wid == 0) {
    double y = stage[lane];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) y += stage[w * 32 + lane];
    y = warp_sum(y);
    if (lane == 0) {
      part[blockIdx.x] = y;
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    }
    double s2w = 0.0;
    if (prev) {
      for (int q = lane; q < (int)gridDim.x; q += 32) s2w += prev[q];
      s2w = warp_sum(s2w);
    }
    int ok = 0;
    if (lane == 0) {
      for (long long it = 0; it < kBarrierPolls; ++it) {
        if (ld_acquire_gpu(bar) >= nb) { ok = 1; break; }
        if (it > 64) __nanosleep(32);
      }
      red[32] = s2w;
      red[33] = sqrt(s2w) * nscale;
      *s_ok = ok;
    }
  }
  __syncthreads();
  *total = red[32];
  *theta = red[33];
  return *s_ok != 0;
}

// Fixed-order sum of a completed sweep's CTA partials (as at the end of
// sweep_sum_barrier) and its theta, for every thread of the CTA.
template <int NT>
__device__ __forceinline__ void grid_partials_theta(const double* part, double* red, double nscale,
                                                    double* total, double* theta) {
  __syncthreads();   // every thread has read the last values handed out in red
  if ((threadIdx.x >> 5) == 0) {
    const int lane = threadIdx.x & 31;
    double s2w = 0.0;
    for (int q = lane; q < (int)gridDim.x; q += 32) s2w += part[q];
    s2w = warp_sum(s2w);
    if (lane == 0) {
      red[32] = s2w;
      red[33] = sqrt(s2w) * nscale;
    }
  }
  __syncthreads();
  *total = red[32];
  *theta = red[33];
}

// End of a grid launch whose last sweep left the latest iterate in v1: each
// warp's rows into v0, or, for a shard (swap_end), the two buffers trade
// places -- v0 the latest, v1 the one before, which Alg. 3 reads next launch
// -- except at the own endpoint of a split D-contact, where v0 still holds
// v^l and v1 v^{l-1} for the second half of the sweep.
template <typename T>
__device__ __forceinline__ void end_of_grid_launch(const DevProblem<T>& P, const SolveCtl& ctl,
                                                   int gw, int nw, int lane) {
  for (int s = gw; s < P.n_slices; s += nw) {
    const int row = s * 32 + lane;
    const Vec4<T> a = ldv(P.v1 + row);
    if (!ctl.swap_end) {
      stv(P.v0 + row, a);
      continue;
    }
    const int cs = __ldg(P.cslot + row);
    if (cs >= 0) {
      const int cj = __ldg(P.c_j + cs);
      if (cj >= 0 && (cj >= P.n_pad || __ldg(P.c_i + cs) >= P.n_pad)) continue;
    }
    const Vec4<T> b = ldv(P.v0 + row);
    stv(P.v0 + row, a);
    stv(P.v1 + row, b);
  }
}

// Stop threshold of a scene's adjoint solve over slices [s0, s1): theta_th, or
// with the relative test theta_th * ||b|| (b = dL/dv, same norm), the sum of
// squares taken in one fixed order by every CTA that reads the scene.  (The
// forward instantiations compare against theta_th directly.)
template <typename T, int NT>
__device__ __forceinline__ double scene_threshold(const DevProblem<T>& P, const SolveCtl& ctl, int s0,
                                                  int s1, double nscale, double* red) {
  if (!ctl.theta_rel) return ctl.theta_th;
  double acc = 0.0;
  for (int i = threadIdx.x; i < (s1 - s0) * 32; i += NT) {
    const Vec4<T> g = ldv(P.b + s0 * 32 + i);
    acc += (double)g.x * g.x + (double)g.y * g.y + (double)g.z * g.z;
  }
  acc = block_allreduce<NT>(acc, red);
  return ctl.theta_th * sqrt(acc) * nscale;
}


// ---------------------------------------------------------------------------
// solve kernels
// ---------------------------------------------------------------------------

// Grid-wide persistent solve of one scene: every warp owns slices
// gw, gw + W, ...; one barrier per sweep (two with D-contacts).  theta is the
// fixed-order sum of the per-CTA partials, computed identically by every CTA,
// so all CTAs take the same stop decision without a further exchange.
template <typename T, int NT, int MINB, bool PF, bool ADJ, bool SYM = false, bool B6 = false>
__global__ void __launch_bounds__(NT, MINB) k_solve_grid(DevProblem<T> P, SolveCtl ctl) {
  __shared__ double red[40];
  __shared__ int s_ok;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (NT / 32);
  int cur = 0, l = 1, st = ST_NOT_CONVERGED;
  unsigned int nbar = 0;   // barriers passed x gridDim.x
  double theta = 0.0, s2 = 0.0, nu = ctl.nu0, bb_alpha = ctl.bb_alpha0;
  const double nscale = ctl.norm_scale[0];
  ChebScalars* const cs = cheb_scalars(red, ctl.cheb_ls, ctl.nu0);
  for (;; ++l) {
    const Vec4<T>* vin = cur ? P.v1 : P.v0;
    Vec4<T>* vout = cur ? P.v0 : P.v1;
    ChebStep<T> ch;
    ch.on = cs ? 1 : 0;   // nu: this sweep's weight, handed out at the end of the last one
    const int lg = ctl.l0 + l - 1;   // the solve's sweep index
    ch.accel = ch.on && lg >= ctl.cheb_ls;
    ch.nu = (T)nu;
    ch.u = (T)ctl.cheb_u;
    double acc = 0.0;
    if (!ADJ && ctl.bb_rule) {
      Vec4<T>* rcur = (l & 1) ? P.r1 : P.r0;
      const Vec4<T>* rprev = (l & 1) ? P.r0 : P.r1;
      double ss = 0.0, sz = 0.0, zz = 0.0;
      for (int s = gw; s < P.n_slices; s += nw)
        bb_residual_row(P, s, lane, vin, vout, rcur, rprev, l == 1, ss, sz, zz);
      if (l > 1) {
        ss = block_allreduce<NT>(ss, red);
        sz = block_allreduce<NT>(sz, red);
        zz = block_allreduce<NT>(zz, red);
        double* bp = ctl.bb_part + (size_t)(l & 1) * 3 * gridDim.x;
        if (threadIdx.x == 0) {
          bp[3 * blockIdx.x] = ss;
          bp[3 * blockIdx.x + 1] = sz;
          bp[3 * blockIdx.x + 2] = zz;
        }
      }
      if (!grid_barrier(ctl.bar, nbar, &s_ok)) { st = ST_TIMEOUT; break; }
      if (l > 1) {
        const double* bp = ctl.bb_part + (size_t)(l & 1) * 3 * gridDim.x;
        double q0 = 0.0, q1 = 0.0, q2 = 0.0;
        for (int q = threadIdx.x; q < (int)gridDim.x; q += NT) {
          q0 += bp[3 * q];
          q1 += bp[3 * q + 1];
          q2 += bp[3 * q + 2];
        }
        q0 = block_allreduce<NT>(q0, red);
        q1 = block_allreduce<NT>(q1, red);
        q2 = block_allreduce<NT>(q2, red);
        bb_alpha = bb_next(ctl.bb_rule, l, q0, q1, q2, bb_alpha);
      }
      for (int s = gw; s < P.n_slices; s += nw)
        acc += bb_update_row(P, s, lane, vin, vout, rcur, (T)bb_alpha);
      if (ctl.n_d > 0) {
        if (!grid_barrier(ctl.bar, nbar, &s_ok)) { st = ST_TIMEOUT; break; }
        for (int d = blockIdx.x * NT + threadIdx.x; d < ctl.n_d; d += gridDim.x * NT)
          acc += bb_d_contact(P, P.d_list[d], vin, vout, (T)bb_alpha);
      }
    } else {
      for (int s = gw; s < P.n_slices; s += nw)
        acc += sweep_row<T, ADJ, PF, SYM, B6, (!ADJ && MINB <= 2 ? 2 : 1)>(P, s, lane, vin, vout, ch);
      if (ctl.n_d > 0) {
        if (!grid_barrier(ctl.bar, nbar, &s_ok)) { st = ST_TIMEOUT; break; }
        for (int d = blockIdx.x * NT + threadIdx.x; d < ctl.n_d; d += gridDim.x * NT)
          acc += d_contact<T, ADJ>(P, P.d_list[d], vin, vout, ch);
      }
    }
    if (!sweep_sum_barrier<NT>(acc, ctl.partials + (l & 1) * gridDim.x, ctl.bar, nbar, red, &s_ok,
                               nscale, cs, lg, ctl.cheb_ls, &s2, &theta, &nu)) {
      st = ST_TIMEOUT;
      break;
    }
    cur ^= 1;
    if (!isfinite(theta)) { st = ST_NONFINITE; break; }
    if (theta < (ADJ && ctl.theta_rel ? ctl.th_scene[0] : ctl.theta_th)) { st = ST_OK; break; }
    if (l >= ctl.l_max) { st = ST_NOT_CONVERGED; break; }
  }
  if (st != ST_TIMEOUT && cur == 1) end_of_grid_launch(P, ctl, gw, nw, lane);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl.iters[0] = l;
    ctl.theta[0] = theta;
    ctl.status[0] = st;
    if (ctl.sumsq) ctl.sumsq[0] = s2;
  }
  if (st == ST_TIMEOUT && threadIdx.x == 0) atomicOr(ctl.err, 1);
}

// ---------------------------------------------------------------------------
// TMA-staged variant of the grid-wide solve
// ---------------------------------------------------------------------------
//
// Each warp keeps a private ring of NST stages in shared memory.  A stage holds
// one chunk of a slice (the VW-entry group of column indices and values, or the
// slice's leftover entries), which the sliced-ELL layout stores as two
// contiguous, 16-byte aligned byte ranges; lane 0 moves them with two 1-D bulk
// copies (cp.async.bulk, the TMA engine) that complete on the stage's mbarrier,
// and refills a stage as soon as the warp has consumed it, so NST - 1 chunks per
// warp are always in flight while the lanes gather v and do the FMAs from
// shared memory.  Every wait is bounded; on a timeout the warp drains its own
// copies (bounded too), flags the error and the kernel stops.

constexpr long long kMbarPolls = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false if the copy did not land within the poll budget
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kMbarPolls; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <typename T>
struct TmaGeom {
  static constexpr int VW = Chunk<T>::VW;
  static constexpr uint32_t kVals = 288u * VW * sizeof(T);   // one chunk's values
  static constexpr uint32_t kCols = 32u * VW * 4u;           // one chunk's column indices
  static constexpr uint32_t kStage = kVals + kCols;          // multiple of 16
};

template <typename T, int NT, int NST>
constexpr size_t tma_smem_bytes() {
  return 128 * (((NT / 32) * NST * 8 + 127) / 128) + (size_t)(NT / 32) * NST * TmaGeom<T>::kStage;
}

// Cursor over one warp's chunk stream: slices gw, gw + nw, ..., each split in
// its full chunks and (if any) its leftover entries.
struct TmaCursor {
  int s, k;
};

template <typename T>
__device__ __forceinline__ bool tma_issue(const DevProblem<T>& P, TmaCursor& cur, int nw, int lane,
                                          unsigned char* stage, uint64_t* bar) {
  using G = TmaGeom<T>;
  while (cur.s < P.n_slices) {
    const int len = P.slice_len[cur.s];
    const int nfull = len / G::VW, ntail = len - nfull * G::VW;
    const int nitems = nfull + (ntail > 0 ? 1 : 0);
    if (cur.k < nitems) {
      const int64_t off = P.slice_off[cur.s];
      const bool full = cur.k < nfull;
      const uint32_t vb = full ? G::kVals : (uint32_t)(ntail * 288 * sizeof(T));
      const uint32_t cb = full ? G::kCols : (uint32_t)(ntail * 128);
      if (lane == 0) {
        const T* vsrc = P.vals + off * 288 + (int64_t)cur.k * (288 * G::VW);
        const int32_t* csrc = P.cols + off * 32 + (int64_t)cur.k * (32 * G::VW);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, vb + cb);
        bulk_g2s(stage, vsrc, vb, bar);
        bulk_g2s(stage + G::kVals, csrc, cb, bar);
      }
      if (++cur.k >= nitems) {
        cur.k = 0;
        cur.s += nw;
      }
      return true;
    }
    cur.k = 0;
    cur.s += nw;
  }
  return false;
}

// The same, run on into the next sweep's stream when this one is all issued
// (the warp's slices and A are the same every sweep).
template <typename T>
__device__ __forceinline__ bool tma_issue_wrap(const DevProblem<T>& P, TmaCursor& cur, int gw,
                                               int nw, int lane, unsigned char* stage,
                                               uint64_t* bar) {
  if (tma_issue(P, cur, nw, lane, stage, bar)) return true;
  if (gw >= P.n_slices) return false;
  cur = TmaCursor{gw, 0};
  return tma_issue(P, cur, nw, lane, stage, bar);
}

template <typename T, int NT, int NST, bool ADJ>
__global__ void __launch_bounds__(NT, 1) k_solve_grid_tma(DevProblem<T> P, SolveCtl ctl) {
  using G = TmaGeom<T>;
  constexpr int NW = NT / 32;
  constexpr int VW = G::VW;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ double red[40];
  __shared__ int s_ok;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * NW + wib, nw = gridDim.x * NW;
  uint64_t* bars = reinterpret_cast<uint64_t*>(dsm) + wib * NST;
  unsigned char* ring = dsm + 128 * ((NW * NST * 8 + 127) / 128) + (size_t)wib * NST * G::kStage;
  if (lane == 0) {
    for (int q = 0; q < NST; ++q) mbar_init(bars + q, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  uint32_t phase = 0;  // bit q: parity of the next completion of stage q
  int cur = 0, l = 1, st = ST_NOT_CONVERGED;
  bool failed = false;
  unsigned int nbar = 0;   // barriers passed x gridDim.x
  double theta = 0.0, s2 = 0.0, nu = ctl.nu0;
  const double nscale = ctl.norm_scale[0];
  ChebScalars* const cs = cheb_scalars(red, ctl.cheb_ls, ctl.nu0);
  // the warp's chunk stream runs on across sweeps: once a sweep's chunks are
  // all issued, the ring's free stages take the next sweep's first ones (A
  // does not change), so each sweep starts with them in flight or landed
  TmaCursor pc{gw, 0};
  int issued = 0, consumed = 0;
  for (int q = 0; q < NST; ++q)
    if (tma_issue_wrap(P, pc, gw, nw, lane, ring + (size_t)(issued % NST) * G::kStage,
                       bars + issued % NST))
      ++issued;
  const bool lag = ctl.lag_stop != 0;
  for (;; ++l) {
    const Vec4<T>* vin = cur ? P.v1 : P.v0;
    Vec4<T>* vout = cur ? P.v0 : P.v1;
    ChebStep<T> ch;
    ch.on = cs ? 1 : 0;   // nu: this sweep's weight, handed out at the end of the last one
    const int lg = ctl.l0 + l - 1;   // the solve's sweep index
    ch.accel = ch.on && lg >= ctl.cheb_ls;
    ch.nu = (T)nu;
    ch.u = (T)ctl.cheb_u;
    ch.lam_alt = lag ? (l & 1) : 0;
    double acc = 0.0;
    for (int s = gw; s < P.n_slices && !failed; s += nw) {
      const int len = P.slice_len[s];
      const int nfull = len / VW, ntail = len - nfull * VW;
      const int nitems = nfull + (ntail > 0 ? 1 : 0);
      T a0 = T(0), a1 = T(0), a2 = T(0);
      for (int k = 0; k < nitems; ++k) {
        const int sg = consumed % NST;
        if (!mbar_wait(bars + sg, (phase >> sg) & 1u)) {
          failed = true;
          break;
        }
        phase ^= 1u << sg;
        const unsigned char* stg = ring + (size_t)sg * G::kStage;
        const T* sv = reinterpret_cast<const T*>(stg);
        const int32_t* sc = reinterpret_cast<const int32_t*>(stg + G::kVals);
        if (k < nfull) {
          int c[VW];
          T m[9][VW];
          if constexpr (VW == 4) {
            const int4 q4 = *reinterpret_cast<const int4*>(sc + lane * 4);
            c[0] = q4.x; c[1] = q4.y; c[2] = q4.z; c[3] = q4.w;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
              const float4 f = *reinterpret_cast<const float4*>(sv + q * 128 + lane * 4);
              m[q][0] = f.x; m[q][1] = f.y; m[q][2] = f.z; m[q][3] = f.w;
            }
          } else {
            const int2 q2 = *reinterpret_cast<const int2*>(sc + lane * 2);
            c[0] = q2.x; c[1] = q2.y;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
              const double2 f = *reinterpret_cast<const double2*>(sv + q * 64 + lane * 2);
              m[q][0] = f.x; m[q][1] = f.y;
            }
          }
#pragma unroll
          for (int e = 0; e < VW; ++e) {
            const Vec4<T> x = ldv(vin + c[e]);
            a0 = fma(m[0][e], x.x, fma(m[1][e], x.y, fma(m[2][e], x.z, a0)));
            a1 = fma(m[3][e], x.x, fma(m[4][e], x.y, fma(m[5][e], x.z, a1)));
            a2 = fma(m[6][e], x.x, fma(m[7][e], x.y, fma(m[8][e], x.z, a2)));
          }
        } else {
          // leftover entries: every gather of v first (they overlap instead of
          // forming a chain), then the FMAs in entry order from shared memory
          Vec4<T> xt[VW - 1];
#pragma unroll
          for (int t = 0; t < VW - 1; ++t)
            if (t < ntail) xt[t] = ldv(vin + sc[t * 32 + lane]);
#pragma unroll
          for (int t = 0; t < VW - 1; ++t) {
            if (t < ntail) {
              const T* mm = sv + t * 288 + lane;
              a0 = fma(mm[0], xt[t].x, fma(mm[32], xt[t].y, fma(mm[64], xt[t].z, a0)));
              a1 = fma(mm[96], xt[t].x, fma(mm[128], xt[t].y, fma(mm[160], xt[t].z, a1)));
              a2 = fma(mm[192], xt[t].x, fma(mm[224], xt[t].y, fma(mm[256], xt[t].z, a2)));
            }
          }
        }
        __syncwarp();
        ++consumed;
        if (tma_issue_wrap(P, pc, gw, nw, lane, ring + (size_t)(issued % NST) * G::kStage,
                           bars + issued % NST))
          ++issued;
      }
      if (failed) break;
      acc += finish_row<T, ADJ>(P, s * 32 + lane, a0, a1, a2, vin, vout, ch);
    }
    if (failed) {
      // let this warp's own copies land (bounded) before the CTA exits
      while (consumed < issued) {
        const int sg = consumed % NST;
        mbar_wait(bars + sg, (phase >> sg) & 1u);
        phase ^= 1u << sg;
        ++consumed;
      }
      atomicOr(ctl.err, 2);
    }
    if (__syncthreads_or(failed ? 1 : 0)) { st = ST_TIMEOUT; break; }
    if (ctl.n_d > 0) {
      if (!grid_barrier(ctl.bar, nbar, &s_ok)) { st = ST_TIMEOUT; break; }
      for (int d = blockIdx.x * NT + threadIdx.x; d < ctl.n_d; d += gridDim.x * NT)
        acc += d_contact<T, ADJ>(P, P.d_list[d], vin, vout, ch);
    }
    if (lag) {
      // stop test of sweep l - 1 (its v is this sweep's input, still intact;
      // its lambda in the other buffers): a stop discards this sweep
      double s2p = 0.0, thp = 0.0;
      if (!sweep_sum_barrier_lag<NT>(acc, ctl.partials + (l % 3) * gridDim.x,
                                     l > 1 ? ctl.partials + ((l - 1) % 3) * gridDim.x : nullptr,
                                     ctl.bar, nbar, red, &s_ok, nscale, &s2p, &thp)) {
        st = ST_TIMEOUT;
        break;
      }
      if (l > 1 && (!isfinite(thp) || thp < ctl.theta_th)) {
        st = isfinite(thp) ? ST_OK : ST_NONFINITE;
        theta = thp;
        s2 = s2p;
        --l;
        break;
      }
      if (l >= ctl.l_max) {   // the last sweep allowed: its own test, its barrier passed
        grid_partials_theta<NT>(ctl.partials + (l % 3) * gridDim.x, red, nscale, &s2, &theta);
        cur ^= 1;
        st = !isfinite(theta) ? ST_NONFINITE : theta < ctl.theta_th ? ST_OK : ST_NOT_CONVERGED;
        break;
      }
      cur ^= 1;
      continue;
    }
    if (!sweep_sum_barrier<NT>(acc, ctl.partials + (l & 1) * gridDim.x, ctl.bar, nbar, red, &s_ok,
                               nscale, cs, lg, ctl.cheb_ls, &s2, &theta, &nu)) {
      st = ST_TIMEOUT;
      break;
    }
    cur ^= 1;
    if (!isfinite(theta)) { st = ST_NONFINITE; break; }
    if (theta < (ADJ && ctl.theta_rel ? ctl.th_scene[0] : ctl.theta_th)) { st = ST_OK; break; }
    if (l >= ctl.l_max) { st = ST_NOT_CONVERGED; break; }
  }
  // copies issued for a sweep that will not run: let them land (bounded)
  // before the CTA exits
  while (consumed < issued) {
    const int sg = consumed % NST;
    mbar_wait(bars + sg, (phase >> sg) & 1u);
    phase ^= 1u << sg;
    ++consumed;
  }
  if (st != ST_TIMEOUT && cur == 1) end_of_grid_launch(P, ctl, gw, nw, lane);
  // lagged stop test: an odd last sweep left its lambda in the second buffers
  // (every CTA is past that sweep's barrier and the next sweep's, if any)
  if (lag && st != ST_TIMEOUT && (l & 1))
    for (int q = blockIdx.x * NT + threadIdx.x; q < P.n_c; q += gridDim.x * NT) {
      stv(P.lam + q, ldv(P.lam2 + q));
      stv(P.lam_star + q, ldv(P.lam_star2 + q));
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl.iters[0] = l;
    ctl.theta[0] = theta;
    ctl.status[0] = st;
    if (ctl.sumsq) ctl.sumsq[0] = s2;
  }
  if (st == ST_TIMEOUT && threadIdx.x == 0) atomicOr(ctl.err, 1);
}

// Persistent CTA-per-scene solve: CTAs pop scenes (largest first) from a
// queue and run the whole V-FPI loop of a scene with block-level syncs only.
template <typename T, int NT, bool ADJ, bool B6 = false>
__global__ void __launch_bounds__(NT) k_solve_scenes(DevProblem<T> P, SolveCtl ctl) {
  __shared__ double red[40];
  __shared__ int s_q;
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(ctl.queue, 1);
    __syncthreads();
    const int q = s_q;
    __syncthreads();
    if (q >= ctl.n_scenes) break;
    const int sc = ctl.order[q];
    const int s0 = ctl.scene_slice[sc], s1 = ctl.scene_slice[sc + 1];
    const int d0 = ctl.scene_d[sc], d1 = ctl.scene_d[sc + 1];
    const double nscale = ctl.norm_scale[sc];
    double th_adj = 0.0;
    if constexpr (ADJ) th_adj = scene_threshold<T, NT>(P, ctl, s0, s1, nscale, red);
    int cur = 0, l = 1, st = ST_NOT_CONVERGED;
    double theta = 0.0, nu = 1.0, bb_alpha = ctl.bb_alpha0;
    ChebScalars* const cs = cheb_scalars(red, ctl.cheb_ls);
    for (;; ++l) {
      const Vec4<T>* vin = cur ? P.v1 : P.v0;
      Vec4<T>* vout = cur ? P.v0 : P.v1;
      ChebStep<T> ch;
      ch.on = cs ? 1 : 0;   // nu: this sweep's weight, handed out at the end of the last one
      ch.accel = ch.on && l >= ctl.cheb_ls;
      ch.nu = (T)nu;
      ch.u = (T)ctl.cheb_u;
      double acc = 0.0;
      if (!ADJ && ctl.bb_rule) {
        Vec4<T>* rcur = (l & 1) ? P.r1 : P.r0;
        const Vec4<T>* rprev = (l & 1) ? P.r0 : P.r1;
        double ss = 0.0, sz = 0.0, zz = 0.0;
        for (int s = s0 + wid; s < s1; s += NT / 32)
          bb_residual_row(P, s, lane, vin, vout, rcur, rprev, l == 1, ss, sz, zz);
        ss = block_allreduce<NT>(ss, red);   // (also orders phase A before phase B)
        sz = block_allreduce<NT>(sz, red);
        zz = block_allreduce<NT>(zz, red);
        if (l > 1) bb_alpha = bb_next(ctl.bb_rule, l, ss, sz, zz, bb_alpha);
        for (int s = s0 + wid; s < s1; s += NT / 32)
          acc += bb_update_row(P, s, lane, vin, vout, rcur, (T)bb_alpha);
        if (d1 > d0) {
          __syncthreads();
          for (int d = d0 + threadIdx.x; d < d1; d += NT)
            acc += bb_d_contact(P, P.d_list[d], vin, vout, (T)bb_alpha);
        }
      } else {
        for (int s = s0 + wid; s < s1; s += NT / 32)
          acc += sweep_row<T, ADJ, false, false, B6, ADJ ? 1 : 2>(P, s, lane, vin, vout, ch);
        if (d1 > d0) {
          __syncthreads();
          for (int d = d0 + threadIdx.x; d < d1; d += NT)
            acc += d_contact<T, ADJ>(P, P.d_list[d], vin, vout, ch);
        }
      }
      block_allreduce_theta<NT>(acc, red, nscale, cs, l, ctl.cheb_ls, &theta, &nu);
      cur ^= 1;
      if (!isfinite(theta)) { st = ST_NONFINITE; break; }
      if (theta < (ADJ ? th_adj : ctl.theta_th)) { st = ST_OK; break; }
      if (l >= ctl.l_max) { st = ST_NOT_CONVERGED; break; }
    }
    if (cur == 1) {
      for (int s = s0 + wid; s < s1; s += NT / 32) {
        const int row = s * 32 + lane;
        stv(P.v0 + row, ldv(P.v1 + row));
      }
    }
    if (threadIdx.x == 0) {
      ctl.iters[sc] = l;
      ctl.theta[sc] = theta;
      ctl.status[sc] = st;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// batched solve with the scene matrices resident in shared memory
// ---------------------------------------------------------------------------
//
// A scene's matrix is re-read by every sweep of Alg. 1 but is at most a few
// MB; streaming it from HBM each sweep (k_solve_scenes) makes the batched
// solve HBM-bound.  Here each CTA copies its share of a scene's sliced-ELL
// entries into shared memory once per solve (1-D bulk copies completing on an
// mbarrier) and every sweep reads them from there.  A scene too large for one
// CTA is split over the CTAs of a thread-block cluster (contiguous slice
// ranges), which meet at the hardware cluster barrier once per sweep (twice
// with D-contacts) and add their FP64 residual partials in a fixed order, so
// every CTA takes the same stop decision.  Smaller scenes go one per CTA.
// The iterates are bitwise those of k_solve_scenes.

__device__ __forceinline__ unsigned cluster_nctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_id_x() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
// all threads of all CTAs of the cluster; release/acquire at cluster scope
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// Block-row product of a slice held in shared memory (same layout and the
// same operations in the same order as row_product).  VS: the gathered
// iterate is the shared-memory copy vsrc[c - cmin] of v (else vsrc = v in
// global memory, cmin = 0).
template <typename T, bool VS>
__device__ __forceinline__ void row_product_smem(const T* vb, const int32_t* cb, int len, int lane,
                                                 const Vec4<T>* vsrc, int cmin, T& a0, T& a1,
                                                 T& a2) {
  constexpr int VW = Chunk<T>::VW;
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  using I = typename std::conditional<sizeof(T) == 4, int4, int2>::type;
  a0 = T(0); a1 = T(0); a2 = T(0);
  const int nfull = len / VW;
#pragma unroll 1
  for (int k = 0; k < nfull; ++k) {
    int c[VW];
    T m[9][VW];
    {
      const I q = *reinterpret_cast<const I*>(cb + k * (32 * VW) + lane * VW);
      const int* qp = reinterpret_cast<const int*>(&q);
#pragma unroll
      for (int e = 0; e < VW; ++e) c[e] = qp[e] - cmin;
    }
    const T* p = vb + k * (288 * VW) + lane * VW;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const V x = *reinterpret_cast<const V*>(p + q * (32 * VW));
      const T* xp = reinterpret_cast<const T*>(&x);
#pragma unroll
      for (int e = 0; e < VW; ++e) m[q][e] = xp[e];
    }
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const Vec4<T> x = ldv(vsrc + c[e]);
      a0 = fma(m[0][e], x.x, fma(m[1][e], x.y, fma(m[2][e], x.z, a0)));
      a1 = fma(m[3][e], x.x, fma(m[4][e], x.y, fma(m[5][e], x.z, a1)));
      a2 = fma(m[6][e], x.x, fma(m[7][e], x.y, fma(m[8][e], x.z, a2)));
    }
  }
  const int ntail = len - nfull * VW;
  const T* pt = vb + nfull * (288 * VW) + lane;
  const int32_t* ct = cb + nfull * (32 * VW) + lane;
  for (int t = 0; t < ntail; ++t) {
    const int c = ct[t * 32] - cmin;
    T m[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) m[q] = pt[t * 288 + q * 32];
    const Vec4<T> x = ldv(vsrc + c);
    a0 = fma(m[0], x.x, fma(m[1], x.y, fma(m[2], x.z, a0)));
    a1 = fma(m[3], x.x, fma(m[4], x.y, fma(m[5], x.z, a1)));
    a2 = fma(m[6], x.x, fma(m[7], x.y, fma(m[8], x.z, a2)));
  }
}

__device__ __forceinline__ Vec4<float> ldv_cg(const Vec4<float>* p) {
  const float4 q = __ldcg(reinterpret_cast<const float4*>(p));
  return {q.x, q.y, q.z, q.w};
}
__device__ __forceinline__ Vec4<double> ldv_cg(const Vec4<double>* p) {
  const double2 a = __ldcg(reinterpret_cast<const double2*>(p));
  const double2 c = __ldcg(reinterpret_cast<const double2*>(p) + 1);
  return {a.x, a.y, c.x, c.y};
}

// Sliced-ELL entries of slices [s0, s1) (slices are stored back to back).
template <typename T>
__device__ __forceinline__ int64_t slice_span(const DevProblem<T>& P, int s0, int s1) {
  return s1 > s0 ? P.slice_off[s1 - 1] + P.slice_len[s1 - 1] - P.slice_off[s0] : 0;
}

// head of the cluster kernel's shared memory: the copy mbarrier [0], the two
// iterate mbarriers [8, 16), residual slots [2][8] doubles [32, 160)
constexpr int kClusterSmemHead = 256;
constexpr uint32_t kBulkPiece = 32768;  // bytes per bulk copy instruction

template <typename T>
__host__ __device__ constexpr int64_t cluster_entry_bytes() { return 288 * (int64_t)sizeof(T) + 128; }

__host__ __device__ constexpr int64_t round128(int64_t x) { return (x + 127) / 128 * 128; }

// Shared memory that staging the rows [r, r + nr) and the iterate's column
// range of R rows takes (v, b, W as Vec4, contact slots as int).
template <typename T>
__host__ __device__ constexpr int64_t cluster_stage_bytes(int64_t R, int64_t nr) {
  return round128(R * (int64_t)sizeof(Vec4<T>)) + 2 * round128(nr * (int64_t)sizeof(Vec4<T>)) +
         round128(nr * 4);
}

// One scene by a group of G CTAs (G = 1: this CTA alone; G = cluster size:
// the whole cluster), this CTA being number g of the group.  Shared memory of
// the CTA for the scene: [mbarrier | v over the CTA's column range | b, W and
// contact slots of its rows | cached sliced-ELL values | their columns]; the
// staging is left out when it would take more than half of it.
template <typename T, int NT, bool ADJ>
__device__ __forceinline__ void cluster_scene(const DevProblem<T>& P, const SolveCtl& ctl, int sc,
                                              int G, int g, double* slot, double* red,
                                              unsigned char* dsm, uint32_t& phase, int& cache_ok,
                                              int* poison) {
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(dsm);
  const int s0 = ctl.scene_slice[sc], s1 = ctl.scene_slice[sc + 1];
  const int ns = s1 - s0;
  const int a = s0 + (int)((int64_t)g * ns / G);
  const int b = s0 + (int)((int64_t)(g + 1) * ns / G);
  const int row0 = a * 32, nr = (b - a) * 32;
  // the range holds the CTA's own rows too (padding rows at a scene's end
  // are nobody's column)
  int cmin = row0, cmax = row0 + nr - 1;
  for (int s = a; s < b; ++s) {
    cmin = min(cmin, P.slice_cmin[s]);
    cmax = max(cmax, P.slice_cmax[s]);
  }
  const int R = b > a ? cmax - cmin + 1 : 0;
  const int64_t stage = cluster_stage_bytes<T>(R, nr);
  const bool st = b > a && 2 * stage <= ctl.smem_bytes;
  unsigned char* p = dsm + kClusterSmemHead;
  Vec4<T>* vsm = reinterpret_cast<Vec4<T>*>(p);
  Vec4<T>* bsm = reinterpret_cast<Vec4<T>*>(p + round128((int64_t)R * sizeof(Vec4<T>)));
  Vec4<T>* wsm = bsm + round128((int64_t)nr * sizeof(Vec4<T>)) / sizeof(Vec4<T>);
  int32_t* csm = reinterpret_cast<int32_t*>(wsm + round128((int64_t)nr * sizeof(Vec4<T>)) / sizeof(Vec4<T>));
  if (st) p += stage;
  T* svals = reinterpret_cast<T*>(p);
  const int64_t cap = (ctl.smem_bytes - (p - dsm)) / cluster_entry_bytes<T>();
  int32_t* scols = reinterpret_cast<int32_t*>(p + cap * 288 * (int64_t)sizeof(T));
  // cached prefix [a, a + kc) of this CTA's slices
  int kc = 0;
  if (cache_ok)
    while (a + kc < b && slice_span(P, a, a + kc + 1) <= cap) ++kc;
  const int64_t e0 = b > a ? P.slice_off[a] : 0;
  const int64_t ec = slice_span(P, a, a + kc);
  if (ec > 0 && threadIdx.x == 0) {
    const uint32_t vbytes = (uint32_t)(ec * 288 * sizeof(T));
    const uint32_t cbytes = (uint32_t)(ec * 128);
    // the buffers were last read by ordinary loads of the previous scene
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(mbar, vbytes + cbytes);
    const unsigned char* vsrc = reinterpret_cast<const unsigned char*>(P.vals + e0 * 288);
    const unsigned char* csrc = reinterpret_cast<const unsigned char*>(P.cols + e0 * 32);
    unsigned char* vdst = reinterpret_cast<unsigned char*>(svals);
    unsigned char* cdst = reinterpret_cast<unsigned char*>(scols);
    for (uint32_t o = 0; o < vbytes; o += kBulkPiece)
      bulk_g2s(vdst + o, vsrc + o, vbytes - o < kBulkPiece ? vbytes - o : kBulkPiece, mbar);
    for (uint32_t o = 0; o < cbytes; o += kBulkPiece)
      bulk_g2s(cdst + o, csrc + o, cbytes - o < kBulkPiece ? cbytes - o : kBulkPiece, mbar);
  }
  if (st)   // b, W (here dL/dv and W in the adjoint) and contact slots stay for the whole solve
    for (int i = threadIdx.x; i < nr; i += NT) {
      bsm[i] = ldv(P.b + row0 + i);
      wsm[i] = ldv(P.w + row0 + i);
      csm[i] = P.cslot[row0 + i];
    }
  if (ec > 0) {
    const bool ok = __syncthreads_and(mbar_wait(mbar, phase) ? 1 : 0) != 0;
    if (ok) {
      phase ^= 1u;
    } else {  // copies did not land: stream this CTA's slices, stop the cluster after this item
      if (threadIdx.x == 0) {
        atomicOr(ctl.err, 1 | 4);
        *poison = 1;
      }
      cache_ok = 0;
      kc = 0;
    }
  }
  const int d0 = ctl.scene_d[sc], d1 = ctl.scene_d[sc + 1];
  const double nscale = ctl.norm_scale[sc];
  double th_adj = 0.0;
  if constexpr (ADJ) th_adj = scene_threshold<T, NT>(P, ctl, s0, s1, nscale, red);
  int cur = 0, l = 1, status = ST_NOT_CONVERGED;
  double theta = 0.0, nu = 1.0;
  ChebScalars* const cs = cheb_scalars(red, ctl.cheb_ls);
  for (;; ++l) {
    const Vec4<T>* vin = cur ? P.v1 : P.v0;
    Vec4<T>* vout = cur ? P.v0 : P.v1;
    ChebStep<T> ch;
    ch.on = cs ? 1 : 0;   // nu: this sweep's weight, handed out at the end of the last one
    ch.accel = ch.on && l >= ctl.cheb_ls;
    ch.nu = (T)nu;
    ch.u = (T)ctl.cheb_u;
    // v^l over this CTA's column range, read from L2 (other CTAs of the
    // cluster wrote parts of it in the previous sweep)
    if (st) {
      for (int i = threadIdx.x; i < R; i += NT) vsm[i] = ldv_cg(vin + cmin + i);
    }
    __syncthreads();
    double acc = 0.0;
    for (int s = a + wid; s < b; s += NT / 32) {
      T a0, a1, a2;
      if (s < a + kc) {
        const int64_t lo = P.slice_off[s] - e0;
        if (st)
          row_product_smem<T, true>(svals + lo * 288, scols + lo * 32, P.slice_len[s], lane, vsm,
                                    cmin, a0, a1, a2);
        else
          row_product_smem<T, false>(svals + lo * 288, scols + lo * 32, P.slice_len[s], lane, vin,
                                     0, a0, a1, a2);
      } else {
        row_product(P, s, lane, vin, a0, a1, a2);
      }
      const int row = s * 32 + lane;
      if (st) {
        const int i = row - row0;
        acc += finish_row_core<T, ADJ>(P, row, a0, a1, a2, vsm[row - cmin], bsm[i], wsm[i], csm[i],
                                       vout + row, ch);
      } else {
        acc += finish_row<T, ADJ>(P, row, a0, a1, a2, vin, vout, ch);
      }
    }
    if (d1 > d0) {
      if (G > 1) cluster_sync(); else __syncthreads();
      for (int d = d0 + g * NT + threadIdx.x; d < d1; d += G * NT)
        acc += d_contact<T, ADJ>(P, P.d_list[d], vin, vout, ch);
    }
    if (G > 1) {
      double part = block_allreduce<NT>(acc, red);
      double* sl = slot + (l & 1) * G;
      if (threadIdx.x == 0) sl[g] = part;
      cluster_sync();
      part = 0.0;
      for (int k = 0; k < G; ++k) part += __ldcg(sl + k);
      theta = sqrt(part) * nscale;
      if (cs) {   // (thread 0 advances, everyone takes nu)
        if (threadIdx.x == 0) red[34] = cs->advance(l, ctl.cheb_ls, theta);
        __syncthreads();
        nu = red[34];
      }
    } else {
      block_allreduce_theta<NT>(acc, red, nscale, cs, l, ctl.cheb_ls, &theta, &nu);
    }
    cur ^= 1;
    if (!isfinite(theta)) { status = ST_NONFINITE; break; }
    if (theta < (ADJ ? th_adj : ctl.theta_th)) { status = ST_OK; break; }
    if (l >= ctl.l_max) { status = ST_NOT_CONVERGED; break; }
  }
  if (cur == 1) {
    for (int s = a + wid; s < b; s += NT / 32) {
      const int row = s * 32 + lane;
      stv(P.v0 + row, ldv(P.v1 + row));
    }
  }
  if (g == 0 && threadIdx.x == 0) {
    ctl.iters[sc] = l;
    ctl.theta[sc] = theta;
    ctl.status[sc] = status;
  }
}

__device__ __forceinline__ uint32_t mapa_u32(uint32_t addr, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
// Stores into another CTA's shared memory that count against that CTA's
// mbarrier (complete_tx): the receiver sees the data once its phase completes.
__device__ __forceinline__ void st_async_row(uint32_t dst, const Vec4<float>& v, uint32_t bar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(dst),
      "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void st_async_row(uint32_t dst, const Vec4<double>& v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(dst),
               "d"(v.x), "d"(v.y), "r"(bar)
               : "memory");
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(
                   dst + 16),
               "d"(v.z), "d"(v.w), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void st_async_f64(uint32_t dst, double x, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(dst),
               "l"(__double_as_longlong(x)), "r"(bar)
               : "memory");
}

// Work split of a scene over a group of G CTAs: member q gets slices
// [a, b) and needs the iterate over columns [cmin, cmax] (its own rows
// included).  tab[q] = {a, b, cmin, cmax}; fits: every member holds its
// whole share -- both iterate buffers, staged rows and all its entries -- in
// shared memory.  Computed by threads q < G, identically in every CTA.
template <typename T>
__device__ __forceinline__ int64_t dsm_bytes(const DevProblem<T>& P, const int* t) {
  const int R = t[1] > t[0] ? t[3] - t[2] + 1 : 0;
  const int64_t nr = 32 * (int64_t)(t[1] - t[0]);
  return 2 * round128(R * (int64_t)sizeof(Vec4<T>)) + 2 * round128(nr * (int64_t)sizeof(Vec4<T>)) +
         round128(nr * 4) + slice_span(P, t[0], t[1]) * cluster_entry_bytes<T>();
}

template <typename T>
__device__ __forceinline__ void plan_scene(const DevProblem<T>& P, const SolveCtl& ctl, int sc, int G,
                                           int (*tab)[4], int* fits) {
  const int q = threadIdx.x;
  if (q < G) {
    const int s0 = ctl.scene_slice[sc], ns = ctl.scene_slice[sc + 1] - s0;
    const int a = s0 + (int)((int64_t)q * ns / G), b = s0 + (int)((int64_t)(q + 1) * ns / G);
    int cmin = a * 32, cmax = b * 32 - 1;
    for (int s = a; s < b; ++s) {
      cmin = min(cmin, P.slice_cmin[s]);
      cmax = max(cmax, P.slice_cmax[s]);
    }
    tab[q][0] = a; tab[q][1] = b; tab[q][2] = cmin; tab[q][3] = cmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    for (int k = 0; k < G; ++k)
      if (kClusterSmemHead + dsm_bytes(P, tab[k]) > ctl.smem_bytes) ok = 0;
    *fits = ok;
  }
  __syncthreads();
}

// One scene held entirely in shared memory by a group of G CTAs (no
// D-contacts).  The iterate lives in two buffers over each CTA's column
// range; a CTA writes v^{l+1} of its rows into its own buffer and pushes each
// row into every other member whose range covers it (st.async counting
// against that member's iterate mbarrier), then sends its FP64 residual
// partial the same way.  A member starts sweep l+1 once its mbarrier has seen
// all rows and partials of sweep l; nothing goes through global memory but
// lambda and the final v.
template <typename T, int NT, bool ADJ>
__device__ __forceinline__ void cluster_scene_dsm(const DevProblem<T>& P, const SolveCtl& ctl, int sc,
                                                  int G, int g, const int (*tab)[4], double* red,
                                                  unsigned char* dsm, uint32_t& phase,
                                                  uint32_t& vphase, int& cache_ok, int* poison) {
  constexpr int V4 = (int)sizeof(Vec4<T>);
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(dsm);
  uint64_t* mbar_v = mbar + 1;
  double* slots = reinterpret_cast<double*>(dsm + 32);
  const int a = tab[g][0], b = tab[g][1], cmin = tab[g][2], cmax = tab[g][3];
  const int row0 = a * 32, nr = (b - a) * 32;
  const int R = b > a ? cmax - cmin + 1 : 0;
  const int64_t vb = round128((int64_t)R * V4);
  Vec4<T>* V0 = reinterpret_cast<Vec4<T>*>(dsm + kClusterSmemHead);
  Vec4<T>* V1 = reinterpret_cast<Vec4<T>*>(dsm + kClusterSmemHead + vb);
  Vec4<T>* bsm = reinterpret_cast<Vec4<T>*>(dsm + kClusterSmemHead + 2 * vb);
  Vec4<T>* wsm = bsm + round128((int64_t)nr * V4) / V4;
  int32_t* csm = reinterpret_cast<int32_t*>(wsm + round128((int64_t)nr * V4) / V4);
  T* svals = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(csm) + round128((int64_t)nr * 4));
  const int64_t ec = slice_span(P, a, b);   // all of the CTA's entries
  int32_t* scols = reinterpret_cast<int32_t*>(svals + ec * 288);
  const int64_t e0 = b > a ? P.slice_off[a] : 0;
  if (ec > 0 && threadIdx.x == 0) {
    const uint32_t vbytes = (uint32_t)(ec * 288 * sizeof(T));
    const uint32_t cbytes = (uint32_t)(ec * 128);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(mbar, vbytes + cbytes);
    const unsigned char* vsrc = reinterpret_cast<const unsigned char*>(P.vals + e0 * 288);
    const unsigned char* csrc = reinterpret_cast<const unsigned char*>(P.cols + e0 * 32);
    unsigned char* vdst = reinterpret_cast<unsigned char*>(svals);
    unsigned char* cdst = reinterpret_cast<unsigned char*>(scols);
    for (uint32_t o = 0; o < vbytes; o += kBulkPiece)
      bulk_g2s(vdst + o, vsrc + o, vbytes - o < kBulkPiece ? vbytes - o : kBulkPiece, mbar);
    for (uint32_t o = 0; o < cbytes; o += kBulkPiece)
      bulk_g2s(cdst + o, csrc + o, cbytes - o < kBulkPiece ? cbytes - o : kBulkPiece, mbar);
  }
  for (int i = threadIdx.x; i < nr; i += NT) {
    bsm[i] = ldv(P.b + row0 + i);
    wsm[i] = ldv(P.w + row0 + i);
    csm[i] = P.cslot[row0 + i];
  }
  for (int i = threadIdx.x; i < R; i += NT) V0[i] = ldv(P.v0 + cmin + i);   // warm start v^1
  // bytes this CTA receives per sweep: the rows of the other members inside
  // its column range, and their partials
  int64_t expect = 8 * (int64_t)(G - 1);
  for (int q = 0; q < G; ++q)
    if (q != g) {
      const int lo = max(tab[q][0] * 32, cmin), hi = min(tab[q][1] * 32 - 1, cmax);
      if (hi >= lo) expect += (int64_t)(hi - lo + 1) * V4;
    }
  const uint32_t base = smem_u32(dsm);
  bool ok = true;
  if (ec > 0) ok = mbar_wait(mbar, phase);
  if (!__syncthreads_and(ok ? 1 : 0)) {   // the matrix did not arrive: give the scene up
    if (threadIdx.x == 0) {
      atomicOr(ctl.err, 1);
      ctl.status[sc] = ST_TIMEOUT;
      *poison = 1;
    }
    cache_ok = 0;
    return;
  }
  if (ec > 0) phase ^= 1u;
  const double nscale = ctl.norm_scale[sc];
  double th_adj = 0.0;
  if constexpr (ADJ)
    th_adj = scene_threshold<T, NT>(P, ctl, ctl.scene_slice[sc], ctl.scene_slice[sc + 1], nscale, red);
  int l = 1, status = ST_NOT_CONVERGED, fin = 0;
  double theta = 0.0, nu = 1.0;
  ChebScalars* const cs = cheb_scalars(red, ctl.cheb_ls);
  for (;; ++l) {
    const int pb = (l - 1) & 1, nb = pb ^ 1;
    const Vec4<T>* Vp = pb ? V1 : V0;
    Vec4<T>* Vn = pb ? V0 : V1;
    if (G > 1 && threadIdx.x == 0) mbar_arrive_expect_tx(mbar_v + nb, (uint32_t)expect);
    ChebStep<T> ch;
    ch.on = cs ? 1 : 0;   // nu: this sweep's weight, handed out at the end of the last one
    ch.accel = ch.on && l >= ctl.cheb_ls;
    ch.nu = (T)nu;
    ch.u = (T)ctl.cheb_u;
    double acc = 0.0;
    for (int s = a + wid; s < b; s += NT / 32) {
      T a0, a1, a2;
      const int64_t lo = P.slice_off[s] - e0;
      row_product_smem<T, true>(svals + lo * 288, scols + lo * 32, P.slice_len[s], lane, Vp, cmin, a0,
                                a1, a2);
      const int row = s * 32 + lane;
      const int i = row - row0;
      Vec4<T>* out = Vn + (row - cmin);
      acc += finish_row_core<T, ADJ>(P, row, a0, a1, a2, Vp[row - cmin], bsm[i], wsm[i], csm[i], out, ch);
      if (G > 1) {
        const Vec4<T> vn = ldv(out);
        for (int q = 0; q < G; ++q) {
          if (q == g || row < tab[q][2] || row > tab[q][3]) continue;
          const int64_t vbq = round128((int64_t)(tab[q][3] - tab[q][2] + 1) * V4);
          const uint32_t off = (uint32_t)(kClusterSmemHead + nb * vbq + (int64_t)(row - tab[q][2]) * V4);
          st_async_row(mapa_u32(base + off, q), vn, mapa_u32(smem_u32(mbar_v + nb), q));
        }
      }
    }
    double part = G > 1 ? block_allreduce<NT>(acc, red)
                        : block_allreduce_theta<NT>(acc, red, nscale, cs, l, ctl.cheb_ls,
                                                    &theta, &nu);
    if (G > 1) {
      if (threadIdx.x == 0) {
        slots[nb * 8 + g] = part;
        for (int q = 0; q < G; ++q)
          if (q != g)
            st_async_f64(mapa_u32(smem_u32(slots + nb * 8 + g), q), part,
                         mapa_u32(smem_u32(mbar_v + nb), q));
      }
      const bool got = mbar_wait(mbar_v + nb, (vphase >> nb) & 1u);
      if (!__syncthreads_and(got ? 1 : 0)) {
        if (threadIdx.x == 0) {
          atomicOr(ctl.err, 1);
          *poison = 1;
        }
        status = ST_TIMEOUT;
        fin = nb;
        break;
      }
      vphase ^= 1u << nb;
      part = 0.0;
      for (int k = 0; k < G; ++k) part += slots[nb * 8 + k];
      theta = sqrt(part) * nscale;
      if (cs) {   // (thread 0 advances, everyone takes nu)
        if (threadIdx.x == 0) red[34] = cs->advance(l, ctl.cheb_ls, theta);
        __syncthreads();
        nu = red[34];
      }
    }
    fin = nb;
    if (!isfinite(theta)) { status = ST_NONFINITE; break; }
    if (theta < (ADJ ? th_adj : ctl.theta_th)) { status = ST_OK; break; }
    if (l >= ctl.l_max) { status = ST_NOT_CONVERGED; break; }
  }
  const Vec4<T>* Vf = fin ? V1 : V0;
  for (int i = threadIdx.x; i < nr; i += NT) stv(P.v0 + row0 + i, Vf[row0 + i - cmin]);
  if (g == 0 && threadIdx.x == 0) {
    ctl.iters[sc] = l;
    ctl.theta[sc] = theta;
    ctl.status[sc] = status;
  }
}

// Persistent clusters pop work items largest scene first: a scene that does
// not fit one CTA's shared memory takes the whole cluster, otherwise each CTA
// of the cluster takes a scene of its own.  A scene runs from shared memory
// alone (cluster_scene_dsm) when every member holds its whole share and it
// has no D-contacts, else through L2 (cluster_scene).  Control flow that
// reaches a cluster barrier depends only on values every CTA of the cluster
// reads alike; a member whose bounded wait ran out marks the cluster's poison
// word, and the whole cluster stops at the next item.
template <typename T, int NT, bool ADJ>
__global__ void __launch_bounds__(NT) k_solve_cluster(DevProblem<T> P, SolveCtl ctl) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ double red[40];
  __shared__ int tab[8][4];
  __shared__ int fits;
  const int C = (int)cluster_nctarank();
  const int g = (int)cluster_ctarank();
  const int cl = (int)cluster_id_x();
  const int n_cl = (int)(gridDim.x / C);
  int32_t* item = ctl.items + (int64_t)cl * C;
  int32_t* poison = ctl.items + (int64_t)n_cl * C + cl;
  double* slot = ctl.partials + (int64_t)cl * 2 * C;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(dsm);
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    mbar_init(mbar + 1, 1);
    mbar_init(mbar + 2, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0, vphase = 0;
  int cache_ok = 1;
  for (;;) {
    if (g == 0 && threadIdx.x == 0) {
      // item word: 2 * queue position + (1 if the whole cluster solves it)
      const int q = atomicAdd(ctl.queue, 1);
      int coop = 0;
      if (q < ctl.n_scenes && C > 1) {
        const int sc = ctl.order[q];
        const int sa = ctl.scene_slice[sc], sb = ctl.scene_slice[sc + 1];
        const int64_t rows = 32 * (int64_t)(sb - sa);
        const int64_t room = ctl.smem_bytes - kClusterSmemHead - cluster_stage_bytes<T>(rows, rows);
        coop = slice_span(P, sa, sb) * cluster_entry_bytes<T>() > room;
      }
      item[0] = 2 * q + coop;
      if (C > 1) {
        const int q2 = (q < ctl.n_scenes && !coop) ? atomicAdd(ctl.queue, C - 1) : ctl.n_scenes;
        for (int k = 1; k < C; ++k) item[k] = coop ? 2 * q + 1 : 2 * (q2 + k - 1);
      }
    }
    cluster_sync();   // (also: every CTA of the cluster has started and set up its mbarriers)
    const int w0 = __ldcg(item);
    if ((w0 >> 1) >= ctl.n_scenes || __ldcg(poison)) break;   // same words for the whole cluster
    const int w = __ldcg(item + g);
    const int q = w >> 1;
    const int G = (w0 & 1) ? C : 1;
    if (G > 1 || q < ctl.n_scenes) {
      const int sc = ctl.order[q];
      plan_scene(P, ctl, sc, G, tab, &fits);
      const bool no_d = ctl.scene_d[sc + 1] == ctl.scene_d[sc];
      if (fits && no_d && cache_ok)
        cluster_scene_dsm<T, NT, ADJ>(P, ctl, sc, G, G > 1 ? g : 0, tab, red, dsm, phase, vphase,
                                      cache_ok, poison);
      else
        cluster_scene<T, NT, ADJ>(P, ctl, sc, G, G > 1 ? g : 0, slot, red, dsm, phase, cache_ok,
                                  poison);
    }
    cluster_sync();   // the item words, residual slots and iterate buffers are reused next
  }
  // a copy that never landed must not outlive the CTA's shared memory
  if (!cache_ok && threadIdx.x == 0) mbar_wait(mbar, phase);
}

// ---------------------------------------------------------------------------
// set-up and conversion kernels
// ---------------------------------------------------------------------------

// Validate the caller's BSR pattern: columns in range, strictly increasing,
// diagonal present, no block across two scenes.  Error bits go to *err.
// Columns in [0, n_cols) (n_cols = N, or N + the halo of a shard); increasing
// (err 2) when `sorted`, else each once per row (a shard keeps the unsplit
// scene's order, whose halo columns may sort below its own); the diagonal
// present; no block coupling two scenes.
static __global__ void k_validate_pattern(int N, int n_cols, int sorted,
                                          const int32_t* __restrict__ row_ptr,
                                          const int32_t* __restrict__ col_idx,
                                          const int32_t* __restrict__ node_scene, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int r0 = row_ptr[i], r1 = row_ptr[i + 1];
  if (r1 < r0) { atomicOr(err, 1); return; }
  bool diag = false;
  int prev = -1;
  for (int p = r0; p < r1; ++p) {
    const int c = col_idx[p];
    if (c < 0 || c >= n_cols) { atomicOr(err, 1); return; }
    if (sorted) {
      if (c <= prev) atomicOr(err, 2);
    } else {
      for (int q = r0; q < p; ++q)
        if (col_idx[q] == c) atomicOr(err, 2);
    }
    if (c == i) diag = true;
    if (c < N && node_scene[c] != node_scene[i]) atomicOr(err, 4);
    prev = c;
  }
  if (!diag) atomicOr(err, 16);
}

// v of own nodes nodes[0..n) (caller's numbering) -> out [3n]; an index out of
// range sets err bit 1 and is skipped.
template <typename T>
__global__ void k_gather_nodes(int n, int N, const int32_t* __restrict__ nodes,
                               const int32_t* __restrict__ node_map, const Vec4<T>* __restrict__ v,
                               T* __restrict__ out, int* err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int i = nodes[k];
  if (i < 0 || i >= N) { atomicOr(err, 1); return; }
  const Vec4<T> q = ldv(v + node_map[i]);
  out[3 * (int64_t)k] = q.x;
  out[3 * (int64_t)k + 1] = q.y;
  out[3 * (int64_t)k + 2] = q.z;
}

// vals [3n] -> v of halo nodes [first, first + n), stored after the padded rows.
template <typename T>
__global__ void k_set_halo(int n, int64_t base, const T* __restrict__ vals, Vec4<T>* __restrict__ v) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  stv(v + base + k, Vec4<T>{vals[3 * (int64_t)k], vals[3 * (int64_t)k + 1], vals[3 * (int64_t)k + 2], T(0)});
}

// Split D-contacts of a shard: one node own, the other a halo node that
// another shard owns.  Both shards hold the contact and take its step of
// Alg. 2 from the same inputs -- their own endpoint's v*, the other endpoint's
// v* received from the other shard, W (tied over the contact's two nodes,
// Prop. 3) -- so they get the same lambda bit for bit, and each applies eq.
// (vup) to its own endpoint.  k = 0..n-1 runs over the split contacts in the
// caller's contact order; cs[k] is the internal contact, own[k] its own row.

// out[6k + q]: the row statistics (a_rr, ||A_r*||^2 of the three DOFs) of the
// own endpoint of split contact k.
static __global__ void k_split_stats(int n, const int32_t* __restrict__ own,
                                     const double* __restrict__ ds, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 6 * n) return;
  out[t] = ds[6 * (int64_t)own[t / 6] + t % 6];
}

// The other endpoint's statistics (from the other shard) into its halo slot of ds.
static __global__ void k_split_set_stats(int n, const int32_t* __restrict__ cs,
                                         const int32_t* __restrict__ own,
                                         const int32_t* __restrict__ c_i,
                                         const int32_t* __restrict__ c_j,
                                         const double* __restrict__ partner,
                                         double* __restrict__ ds) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 6 * n) return;
  const int k = t / 6, m = cs[k];
  const int other = own[k] == c_i[m] ? c_j[m] : c_i[m];
  ds[6 * (int64_t)other + t % 6] = partner[t];
}

// out[3k..3k+2]: v* (eq. pgd1) of the own endpoint of split contact k, as the
// last shard sweep staged it.
template <typename T>
__global__ void k_split_vstar(int n, const int32_t* __restrict__ cs, const int32_t* __restrict__ own,
                              const int32_t* __restrict__ c_j, const Vec4<T>* __restrict__ dstar,
                              T* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int m = cs[k];
  const Vec4<T> q = ldv(dstar + 2 * m + (own[k] == c_j[m] ? 1 : 0));
  out[3 * (int64_t)k] = q.x;
  out[3 * (int64_t)k + 1] = q.y;
  out[3 * (int64_t)k + 2] = q.z;
}

// The step of each split contact from partner[3k..] (the other endpoint's
// v*): the own endpoint's v^{l+1} into v0 (where the sweep left v^l; with
// Alg. 3 combined with v^{l-1} from v1, as the sweep's own rows are), v^l into
// v1, and sumsq[0] += the FP64 sum of their ||v^{l+1} - v^l||^2, taken in a
// fixed order by one CTA.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_split_finish(DevProblem<T> P, int n,
                                                      const int32_t* __restrict__ cs,
                                                      const int32_t* __restrict__ own,
                                                      const T* __restrict__ partner,
                                                      ChebStep<T> ch, double* __restrict__ sumsq) {
  __shared__ double red[40];
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += NT) {
    const int m = cs[k], r = own[k];
    const bool at_j = r == P.c_j[m];
    const Vec4<T> so = ldv(P.dstar + 2 * m + (at_j ? 1 : 0));
    const Vec4<T> sp = {partner[3 * (int64_t)k], partner[3 * (int64_t)k + 1],
                        partner[3 * (int64_t)k + 2], T(0)};
    const T w = P.w[r].x;                      // tied: the same at both nodes
    Vec4<T> ni, nj;
    if (at_j) d_contact_step(P, m, sp, so, w, w, ni, nj);
    else d_contact_step(P, m, so, sp, w, w, ni, nj);
    // v0 holds v^l and v1 v^{l-1} here (the launch left this row): Alg. 3's
    // combination, then the buffers' order of every other row
    const Vec4<T> o = ldv(P.v0 + r);
    const Vec4<T> nn = cheb_combine(ch, at_j ? nj : ni, o, P.v1 + r);
    stv(P.v0 + r, nn);
    stv(P.v1 + r, o);
    acc += sqdiff(nn, o);
  }
  acc = block_allreduce<NT>(acc, red);
  if (threadIdx.x == 0) sumsq[0] += acc;
}

template <typename T>
__global__ void k_check_finite(const T* __restrict__ a, int64_t n, int* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(a[i])) atomicOr(err, 8);
}

// Smallest and largest column of each slice (one warp per slice).
static __global__ void k_slice_colrange(int n_slices, const int32_t* __restrict__ slice_len,
                                        const int64_t* __restrict__ slice_off,
                                        const int32_t* __restrict__ cols, int32_t* __restrict__ cmin,
                                        int32_t* __restrict__ cmax) {
  const int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= n_slices) return;
  const int64_t base = slice_off[s] * 32;
  const int n = slice_len[s] * 32;
  int lo = 0x7fffffff, hi = -1;
  for (int k = lane; k < n; k += 32) {
    const int c = cols[base + k];
    lo = min(lo, c);
    hi = max(hi, c);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (lane == 0) {
    cmin[s] = n > 0 ? lo : s * 32;
    cmax[s] = n > 0 ? hi : s * 32;
  }
}

// Fill every slot with a zero block pointing at its own row.
static __global__ void k_fill_pad_cols(int n_slices, const int32_t* __restrict__ slice_len,
                                       const int64_t* __restrict__ slice_off,
                                       int32_t* __restrict__ cols) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_slices * 32) return;
  const int s = row >> 5;
  const int64_t base = slice_off[s] * 32;
  const int n = slice_len[s] * 32;
  // padding slots keep zero values; their column is the slice's first row
  // (any valid row would do, one shared row makes the dead gathers a broadcast)
  for (int k = row & 31; k < n; k += 32) cols[base + k] = s * 32;
}

// Scatter the caller's blocks into the sliced-ELL layout.
template <typename T>
__global__ void k_scatter_blocks(int N, const int32_t* __restrict__ row_ptr,
                                 const int32_t* __restrict__ col_idx, const T* __restrict__ vals,
                                 const int32_t* __restrict__ node_map,
                                 const int32_t* __restrict__ slice_len,
                                 const int64_t* __restrict__ slice_off, int32_t* __restrict__ cols,
                                 T* __restrict__ svals, int store_cols) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int p = node_map[i];
  const int s = p >> 5, lane = p & 31;
  const int len = slice_len[s];
  const int64_t off = slice_off[s];
  const int r0 = row_ptr[i], r1 = row_ptr[i + 1];
  for (int e = 0; e < r1 - r0; ++e) {
    int64_t vp;
    int vs;
    const int64_t cp = slot_pos<T>(off, len, e, lane, &vp, &vs);
    if (store_cols) cols[cp] = node_map[col_idx[r0 + e]];
    const T* src = vals + (int64_t)(r0 + e) * 9;
#pragma unroll
    for (int q = 0; q < 9; ++q) svals[vp + (int64_t)q * vs] = src[q];
  }
}

// ---- relative stop test of the adjoint: theta_th * ||b|| per scene ----
// (b = dL/dv there; computed before the solve so that the solve kernels
// carry nothing but one load for it)

// FP64 sum of squares of b over each slice (one warp per slice).
template <typename T>
__global__ void k_slice_sumsq(int n_slices, const Vec4<T>* __restrict__ b, double* __restrict__ out) {
  const int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (s >= n_slices) return;
  const Vec4<T> g = ldv(b + s * 32 + (threadIdx.x & 31));
  const double x = warp_sum((double)g.x * g.x + (double)g.y * g.y + (double)g.z * g.z);
  if ((threadIdx.x & 31) == 0) out[s] = x;
}

// One CTA per scene: th[q] = theta_th * sqrt(sum of its slices' sums) * norm scale,
// the slices' sums taken in a fixed order.
static __global__ void k_scene_threshold(const int32_t* __restrict__ scene_slice,
                                         const double* __restrict__ slice_sumsq,
                                         const double* __restrict__ norm_scale, double theta_th,
                                         double* __restrict__ th) {
  __shared__ double red[40];
  const int q = blockIdx.x;
  double acc = 0.0;
  for (int s = scene_slice[q] + threadIdx.x; s < scene_slice[q + 1]; s += 256) acc += slice_sumsq[s];
  acc = block_allreduce<256>(acc, red);
  if (threadIdx.x == 0) th[q] = theta_th * sqrt(acc) * norm_scale[q];
}

// ---- symmetric storage set-up (caller's sorted BSR pattern, one scene) ----

// Index of the diagonal block in each row = the row's number of entries c < r.
static __global__ void k_row_nlow(int N, const int32_t* __restrict__ row_ptr,
                                  const int32_t* __restrict__ col_idx, int32_t* __restrict__ nlow) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int lo = row_ptr[i], hi = row_ptr[i + 1];
  while (lo < hi) {   // first entry with column >= i
    const int mid = (lo + hi) >> 1;
    if (col_idx[mid] < i) lo = mid + 1; else hi = mid;
  }
  nlow[i] = lo - row_ptr[i];
}

__device__ __forceinline__ int find_col(const int32_t* __restrict__ row_ptr,
                                        const int32_t* __restrict__ col_idx, int row, int col) {
  int lo = row_ptr[row], hi = row_ptr[row + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int c = col_idx[mid];
    if (c == col) return mid;
    if (c < col) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// Error bit 32: the pattern is not symmetric; 64: a block differs from the
// transpose of its mirror (bitwise).
template <typename T>
__global__ void k_sym_check(int N, const int32_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ col_idx, const T* __restrict__ vals, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
    const int c = col_idx[e];
    const int f = find_col(row_ptr, col_idx, c, i);
    if (f < 0) { atomicOr(err, 32); return; }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        if (!(vals[(int64_t)e * 9 + 3 * a + b] == vals[(int64_t)f * 9 + 3 * b + a])) {
          atomicOr(err, 64);
          return;
        }
  }
}

// Padding of both structures: upper slots point at the slice's first row
// (their values stay zero); lower slots at that row and the zero block.
template <typename T>
__global__ void k_fill_sym_pad(int n_slices, const int32_t* __restrict__ ulen,
                               const int64_t* __restrict__ uoff, int32_t* __restrict__ ucols,
                               const int32_t* __restrict__ llen, const int64_t* __restrict__ loff,
                               int32_t* __restrict__ lcols, int32_t* __restrict__ lpos, int64_t zero) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_slices * 32) return;
  const int s = row >> 5, lane = row & 31;
  for (int k = lane; k < ulen[s] * 32; k += 32) ucols[uoff[s] * 32 + k] = s * 32;
  for (int k = lane; k < llen[s] * 32; k += 32) {
    lcols[loff[s] * 32 + k] = s * 32;
    lpos[loff[s] * 32 + k] = (int32_t)(zero + (k & 31));
  }
}

// Blocks with c >= r into the upper structure (values; columns too when
// store_cols).
template <typename T>
__global__ void k_scatter_upper(int N, const int32_t* __restrict__ row_ptr,
                                const int32_t* __restrict__ col_idx, const T* __restrict__ vals,
                                const int32_t* __restrict__ nlow, const int32_t* __restrict__ node_map,
                                const int32_t* __restrict__ ulen, const int64_t* __restrict__ uoff,
                                int32_t* __restrict__ ucols, T* __restrict__ uvals, int store_cols) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int p = node_map[i];
  const int s = p >> 5, lane = p & 31;
  const int r0 = row_ptr[i] + nlow[i], r1 = row_ptr[i + 1];
  for (int e = 0; e < r1 - r0; ++e) {
    const int64_t ent = uoff[s] + e;
    if (store_cols) ucols[ent * 32 + lane] = node_map[col_idx[r0 + e]];
    const T* src = vals + (int64_t)(r0 + e) * 9;
#pragma unroll
    for (int q = 0; q < 9; ++q) uvals[ent * 288 + q * 32 + lane] = src[q];
  }
}

// Entries c < r: the column and where block (c, r) sits in the upper values.
template <typename T>
__global__ void k_build_lower(int N, const int32_t* __restrict__ row_ptr,
                              const int32_t* __restrict__ col_idx, const int32_t* __restrict__ nlow,
                              const int32_t* __restrict__ node_map, const int32_t* __restrict__ ulen,
                              const int64_t* __restrict__ uoff, const int32_t* __restrict__ llen,
                              const int64_t* __restrict__ loff, int32_t* __restrict__ lcols,
                              int32_t* __restrict__ lpos, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int p = node_map[i];
  const int s = p >> 5, lane = p & 31;
  for (int j = 0; j < nlow[i]; ++j) {
    const int c = col_idx[row_ptr[i] + j];
    const int f = find_col(row_ptr, col_idx, c, i);
    if (f < 0) { atomicOr(err, 32); return; }
    const int u = f - row_ptr[c] - nlow[c];   // i > c: among row c's entries >= c
    const int pc = node_map[c];
    int64_t vp2;
    int vs2;
    const int64_t cp = slot_pos<T>(loff[s], llen[s], j, lane, &vp2, &vs2);
    lcols[cp] = pc;
    lpos[cp] = (int32_t)((uoff[pc >> 5] + u) * 288 + (pc & 31));
  }
}

// Per DOF: d = a_rr and s = ||A_r*||^2 in FP64 (Sec. IV.C), from the layout.
template <typename T>
__global__ void k_row_stats(DevProblem<T> P, double* __restrict__ ds) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= P.n_pad) return;
  const int s = row >> 5, lane = row & 31;
  const int len = P.slice_len[s];
  const int64_t off = P.slice_off[s];
  double d[3] = {0, 0, 0}, q2[3] = {0, 0, 0};
  for (int e = 0; e < len; ++e) {
    int64_t vp;
    int vs;
    const int64_t cp = slot_pos<T>(off, len, e, lane, &vp, &vs);
    const int c = P.cols[cp];
    T m[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) m[q] = P.vals[vp + (int64_t)q * vs];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      q2[a] += (double)m[3 * a] * m[3 * a] + (double)m[3 * a + 1] * m[3 * a + 1] +
               (double)m[3 * a + 2] * m[3 * a + 2];
      if (c == row) d[a] += (double)m[4 * a];
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ds[6 * (int64_t)row + a] = d[a];
    ds[6 * (int64_t)row + 3 + a] = q2[a];
  }
}

// Symmetric-block storage: err bit 128 unless every stored slot's block equals
// its transpose bit for bit (one thread per slot: slice s = t / 32 rows,
// entry e over the slice's length).
template <typename T>
__global__ void k_block_sym_check(DevProblem<T> P, int* err) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= P.n_pad) return;
  const int s = row >> 5, lane = row & 31;
  const int len = P.slice_len[s];
  const int64_t off = P.slice_off[s];
  for (int e = 0; e < len; ++e) {
    int64_t vp;
    int vs;
    slot_pos<T>(off, len, e, lane, &vp, &vs);
    const T* m = P.vals + vp;
    if (m[1 * vs] != m[3 * vs] || m[2 * vs] != m[6 * vs] || m[5 * vs] != m[7 * vs]) {
      atomicOr(err, 128);
      return;
    }
  }
}

// vals -> vals6 (m00, m01, m02, m11, m12, m22 per slot, the layout of vals
// with 6 planes: slot_pos with 192 in place of 288).
template <typename T>
__global__ void k_make_vals6(DevProblem<T> P, T* __restrict__ vals6) {
  constexpr int VW = Chunk<T>::VW;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= P.n_pad) return;
  const int s = row >> 5, lane = row & 31;
  const int len = P.slice_len[s];
  const int64_t off = P.slice_off[s];
  const int nfull = len / VW;
  for (int e = 0; e < len; ++e) {
    int64_t vp;
    int vs;
    slot_pos<T>(off, len, e, lane, &vp, &vs);
    int64_t qp;
    if (e < nfull * VW) qp = off * 192 + (int64_t)(e / VW) * (192 * VW) + lane * VW + e % VW;
    else qp = off * 192 + (int64_t)nfull * (192 * VW) + (int64_t)(e - nfull * VW) * 192 + lane;
    const T* m = P.vals + vp;
    const int src[6] = {0, 1, 2, 4, 5, 8};
#pragma unroll
    for (int j = 0; j < 6; ++j) vals6[qp + (int64_t)j * vs] = m[(int64_t)src[j] * vs];
  }
}

// W from the row statistics: tied on contact nodes (both nodes of a D-contact
// share one value), w_rr = a_rr / ||A_r*||^2 elsewhere (Sec. IV.C).
template <typename T>
__global__ void k_make_w_frobenius(int n_pad, const double* __restrict__ ds,
                                   const int32_t* __restrict__ cslot, const int32_t* __restrict__ c_i,
                                   const int32_t* __restrict__ c_j, Vec4<T>* __restrict__ w) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_pad) return;
  const double* r = ds + 6 * (int64_t)row;
  Vec4<T> o;
  const int cs = cslot[row];
  if (cs < 0) {
    o.x = r[3] > 0 ? (T)(r[0] / r[3]) : T(0);
    o.y = r[4] > 0 ? (T)(r[1] / r[4]) : T(0);
    o.z = r[5] > 0 ? (T)(r[2] / r[5]) : T(0);
  } else {
    const int i = c_i[cs], j = c_j[cs];
    const double* ri = ds + 6 * (int64_t)i;
    double num = ri[0] + ri[1] + ri[2];
    double den = ri[3] + ri[4] + ri[5];
    if (j >= 0) {
      const double* rj = ds + 6 * (int64_t)j;
      num += rj[0] + rj[1] + rj[2];
      den += rj[3] + rj[4] + rj[5];
    }
    const T wb = (T)(num / den);
    o.x = o.y = o.z = wb;
  }
  o.w = T(0);
  stv(w + row, o);
}

// W = alpha I (pad rows have A = 0 and b = 0, so they stay at v = 0 for any w)
template <typename T>
__global__ void k_w_scalar(int n_pad, T alpha, Vec4<T>* __restrict__ w) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_pad) return;
  stv(w + row, Vec4<T>{alpha, alpha, alpha, T(0)});
}

// caller layout [3N] -> internal Vec4 rows
template <typename T>
__global__ void k_to_internal(int N, const T* __restrict__ ext, const int32_t* __restrict__ node_map,
                              Vec4<T>* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  stv(out + node_map[i], Vec4<T>{ext[3 * (int64_t)i], ext[3 * (int64_t)i + 1],
                                 ext[3 * (int64_t)i + 2], T(0)});
}

template <typename T>
__global__ void k_to_external(int N, const Vec4<T>* __restrict__ in,
                              const int32_t* __restrict__ node_map, T* __restrict__ ext) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const Vec4<T> v = ldv(in + node_map[i]);
  ext[3 * (int64_t)i] = v.x;
  ext[3 * (int64_t)i + 1] = v.y;
  ext[3 * (int64_t)i + 2] = v.z;
}

// contact data in caller order -> internal (sorted) order
template <typename T>
__global__ void k_gather_contacts(int n_c, const int32_t* __restrict__ perm, const T* __restrict__ R,
                                  const T* __restrict__ mu, const T* __restrict__ phi,
                                  T* __restrict__ cR, T* __restrict__ cmu, T* __restrict__ cphi,
                                  int write_R_mu) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_c) return;
  const int e = perm[m];
  if (write_R_mu) {
#pragma unroll
    for (int q = 0; q < 9; ++q) cR[(int64_t)q * n_c + m] = R[9 * (int64_t)e + q];
    cmu[m] = mu[e];
  }
  if (phi) cphi[m] = phi[e];
}

template <typename T>
__global__ void k_lambda_external(int n_c, const int32_t* __restrict__ perm,
                                  const Vec4<T>* __restrict__ lam, T* __restrict__ out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_c) return;
  const Vec4<T> l = ldv(lam + m);
  const int e = perm[m];
  out[3 * (int64_t)e] = l.x;
  out[3 * (int64_t)e + 1] = l.y;
  out[3 * (int64_t)e + 2] = l.z;
}

// per-contact 3-vectors in caller order -> internal Vec4 (contact m takes caller's perm[m])
template <typename T>
__global__ void k_contact_vec_internal(int n_c, const int32_t* __restrict__ perm,
                                       const T* __restrict__ ext, Vec4<T>* __restrict__ out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_c) return;
  const int e = perm[m];
  stv(out + m, Vec4<T>{ext[3 * (int64_t)e], ext[3 * (int64_t)e + 1], ext[3 * (int64_t)e + 2], T(0)});
}

// per-contact scalars: internal -> caller order, or caller -> internal
template <typename T>
__global__ void k_contact_scalar(int n_c, const int32_t* __restrict__ perm, const T* __restrict__ in,
                                 T* __restrict__ out, int to_external) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_c) return;
  if (to_external) out[perm[m]] = in[m];
  else out[m] = in[perm[m]];
}

// x_{k+1} = x_k + h v_hat in FP64 (eq. disc_dyn)
template <typename T>
__global__ void k_integrate(int N, double h, const Vec4<T>* __restrict__ v,
                            const int32_t* __restrict__ node_map, double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const Vec4<T> q = ldv(v + node_map[i]);
  x[3 * (int64_t)i] += h * (double)q.x;
  x[3 * (int64_t)i + 1] += h * (double)q.y;
  x[3 * (int64_t)i + 2] += h * (double)q.z;
}

// y = A x on internal vectors
template <typename T>
__global__ void k_spmv(DevProblem<T> P, const Vec4<T>* __restrict__ x, Vec4<T>* __restrict__ y) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= P.n_slices) return;
  T a0, a1, a2;
  row_product(P, gw, lane, x, a0, a1, a2);
  stv(y + gw * 32 + lane, Vec4<T>{a0, a1, a2, T(0)});
}

}  // namespace vfpi
