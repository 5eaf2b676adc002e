// vfpi_solve_noalloc: a solve that allocates nothing.
//
// Some callers cannot call cudaMalloc at all -- code running under a memory
// manager that owns every device allocation, code inside a plug-in that may
// not touch the CUDA allocator, or a real-time loop that must never block on
// allocation.  For them this entry point solves one small problem straight
// from the caller's device buffers.  Its scratch (two iterates, W, the
// node-to-contact map, row statistics and a status word) lives in the
// file-scope device array below, of fixed size; every GPU that loads this
// library holds that array until the process exits.
//
// It is the CTA-per-scene solve of vfpi_device.cuh, reduced to one CTA that
// reads the caller's block rows in place instead of the re-laid-out copy: the
// same per-row arithmetic in the same order, so for the same input it gives the
// same iterates as vfpi_solve with W_FROBENIUS.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/vfpi.h"

namespace {

constexpr int kMaxNodes = VFPI_NOALLOC_MAX_NODES;
constexpr int kThreads = 256;

// scratch layout (bytes): v0 | v1 | w (float4 per node) | row sums (2 doubles
// per node) | cslot (int per node) | status words
constexpr size_t kVecBytes = 16ull * kMaxNodes;
constexpr size_t kOffV1 = kVecBytes;
constexpr size_t kOffW = 2 * kVecBytes;
constexpr size_t kOffSums = 3 * kVecBytes;
constexpr size_t kOffSlot = kOffSums + 16ull * kMaxNodes;
constexpr size_t kOffStatus = kOffSlot + 4ull * kMaxNodes;
constexpr size_t kScratchBytes = kOffStatus + 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

static_assert(kScratchBytes == 68ull * kMaxNodes + 64, "scratch size stated in include/vfpi.h");

// error bits set by the kernel's input checks
constexpr int kErrIndex = 1;     // a node or column index out of range
constexpr int kErrOverlap = 2;   // a node in two contacts, or a D-contact with i == j
constexpr int kErrRowPtr = 4;    // row_ptr not 0 .. nnzb with 1..n_nodes blocks per row

struct NoallocStatus {
  int32_t iters;
  int32_t status;
  int32_t err;      // kErr* bits
  int32_t pad;
  double theta;
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

__device__ double block_allreduce(double x, double* red) {
  x = warp_sum(x);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = x;
  __syncthreads();
  if (wid == 0) {
    double y = lane < kThreads / 32 ? red[lane] : 0.0;
    y = warp_sum(y);
    if (lane == 0) red[32] = y;
  }
  __syncthreads();
  return red[32];
}

// strict one-shot solve (Alg. 2, eq. operator), same expression order as the
// main kernels
__device__ __forceinline__ void one_shot(const float* R, float mu, float phi, float gamma, float rx,
                                         float ry, float rz, float4& lam) {
  const float en = R[0] * rx + R[1] * ry + R[2] * rz;
  const float e1 = R[3] * rx + R[4] * ry + R[5] * rz;
  const float e2 = R[6] * rx + R[7] * ry + R[8] * rz;
  const float lx = -(en + phi) / gamma, ly = -e1 / gamma, lz = -e2 / gamma;
  const float ln = lx > 0.f ? lx : 0.f;
  const float rho = sqrtf(ly * ly + lz * lz);
  const float rad = mu * ln;
  const float s = (rho <= rad) ? 1.f : rad / rho;
  lam = make_float4(ln, s * ly, s * lz, 0.f);
}

__global__ void __launch_bounds__(kThreads)
k_solve_noalloc(int N, int nnzb, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                const float* __restrict__ vals, const float* __restrict__ b, int n_c,
                const int32_t* __restrict__ node_i, const int32_t* __restrict__ node_j,
                const float* __restrict__ R, const float* __restrict__ mu,
                const float* __restrict__ phi, double theta_th, int l_max, double nscale,
                const float* __restrict__ v_in, float* __restrict__ v_out,
                float* __restrict__ lambda_out, unsigned char* scratch) {
  __shared__ double red[33];
  __shared__ int s_err;
  float4* v0 = reinterpret_cast<float4*>(scratch);
  float4* v1 = reinterpret_cast<float4*>(scratch + kOffV1);
  float4* w = reinterpret_cast<float4*>(scratch + kOffW);
  double2* sums = reinterpret_cast<double2*>(scratch + kOffSums);
  int32_t* cslot = reinterpret_cast<int32_t*>(scratch + kOffSlot);
  NoallocStatus* st = reinterpret_cast<NoallocStatus*>(scratch + kOffStatus);
  const int tid = threadIdx.x;
  if (tid == 0) s_err = 0;
  // the array keeps the previous call's contents: clear the contact map
  for (int i = tid; i < N; i += kThreads) {
    cslot[i] = -1;
    v0[i] = make_float4(v_in[3 * i], v_in[3 * i + 1], v_in[3 * i + 2], 0.f);
  }
  // row pointers first: every later loop over a row's blocks trusts them
  if (tid == 0 && (row_ptr[0] != 0 || row_ptr[N] != nnzb)) atomicOr(&s_err, kErrRowPtr);
  for (int i = tid; i < N; i += kThreads) {
    const int len = row_ptr[i + 1] - row_ptr[i];
    if (len < 1 || len > N) atomicOr(&s_err, kErrRowPtr);
  }
  __syncthreads();
  if (s_err) {
    if (tid == 0) { st->iters = 0; st->status = VFPI_ERR_INVALID_ARG; st->err = s_err; st->theta = 0; }
    return;
  }
  // each node in at most one contact (Prop. 3): claim it, a second claim fails
  for (int m = tid; m < n_c; m += kThreads) {
    const int i = node_i[m], j = node_j ? node_j[m] : -1;
    if (i < 0 || i >= N || j < -1 || j >= N) { atomicOr(&s_err, kErrIndex); continue; }
    if (i == j || atomicCAS(&cslot[i], -1, m) != -1) { atomicOr(&s_err, kErrOverlap); continue; }
    if (j >= 0 && atomicCAS(&cslot[j], -1, m) != -1) atomicOr(&s_err, kErrOverlap);
  }
  __syncthreads();
  if (s_err) {
    if (tid == 0) { st->iters = 0; st->status = VFPI_ERR_INVALID_ARG; st->err = s_err; st->theta = 0; }
    return;
  }
  // W (Sec. IV.C): row statistics in FP64, tied on contact nodes
  for (int i = tid; i < N; i += kThreads) {
    double d[3] = {0, 0, 0}, q2[3] = {0, 0, 0};
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
      const int c = col_idx[p];
      if (c < 0 || c >= N) { atomicOr(&s_err, kErrIndex); continue; }
      const float* m = vals + 9ll * p;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        q2[a] += (double)m[3 * a] * m[3 * a] + (double)m[3 * a + 1] * m[3 * a + 1] +
                 (double)m[3 * a + 2] * m[3 * a + 2];
        if (c == i) d[a] += (double)m[4 * a];
      }
    }
    if (cslot[i] < 0)
      w[i] = make_float4((float)(d[0] / q2[0]), (float)(d[1] / q2[1]), (float)(d[2] / q2[2]), 0.f);
    sums[i] = make_double2(d[0] + d[1] + d[2], q2[0] + q2[1] + q2[2]);
  }
  __syncthreads();
  for (int m = tid; m < n_c; m += kThreads) {
    const int i = node_i[m], j = node_j ? node_j[m] : -1;
    double num = sums[i].x, den = sums[i].y;
    if (j >= 0) { num += sums[j].x; den += sums[j].y; }
    const float wb = (float)(num / den);
    w[i] = make_float4(wb, wb, wb, 0.f);
    if (j >= 0) w[j] = make_float4(wb, wb, wb, 0.f);
  }
  __syncthreads();
  if (s_err) {
    if (tid == 0) { st->iters = 0; st->status = VFPI_ERR_INVALID_ARG; st->err = s_err; st->theta = 0; }
    return;
  }
  int cur = 0, l = 1, status = VFPI_NOT_CONVERGED;
  double theta = 0.0;
  for (;; ++l) {
    const float4* vin = cur ? v1 : v0;
    float4* vout = cur ? v0 : v1;
    double acc = 0.0;
    for (int i = tid; i < N; i += kThreads) {
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
      for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
        const float* m = vals + 9ll * p;
        const float4 x = vin[col_idx[p]];
        a0 = fmaf(m[0], x.x, fmaf(m[1], x.y, fmaf(m[2], x.z, a0)));
        a1 = fmaf(m[3], x.x, fmaf(m[4], x.y, fmaf(m[5], x.z, a1)));
        a2 = fmaf(m[6], x.x, fmaf(m[7], x.y, fmaf(m[8], x.z, a2)));
      }
      const float4 vo = vin[i], ww = w[i];
      // eq. (pgd1)
      float4 vn = make_float4(vo.x - ww.x * (a0 - b[3 * i]), vo.y - ww.y * (a1 - b[3 * i + 1]),
                              vo.z - ww.z * (a2 - b[3 * i + 2]), 0.f);
      const int cs = cslot[i];
      if (cs >= 0) {
        if (node_j && node_j[cs] >= 0) { vout[i] = vn; continue; }   // D-contact: phase 2
        const float* Rm = R + 9ll * cs;
        float4 lam;
        one_shot(Rm, mu[cs], phi[cs], ww.x, vn.x, vn.y, vn.z, lam);  // gamma = w_i (Prop. 3)
        vn.x += ww.x * (Rm[0] * lam.x + Rm[3] * lam.y + Rm[6] * lam.z);   // eq. (vup)
        vn.y += ww.x * (Rm[1] * lam.x + Rm[4] * lam.y + Rm[7] * lam.z);
        vn.z += ww.x * (Rm[2] * lam.x + Rm[5] * lam.y + Rm[8] * lam.z);
        lambda_out[3 * cs] = lam.x;
        lambda_out[3 * cs + 1] = lam.y;
        lambda_out[3 * cs + 2] = lam.z;
      }
      vout[i] = vn;
      const float dx = vn.x - vo.x, dy = vn.y - vo.y, dz = vn.z - vo.z;   // as sqdiff
      acc += (double)(dx * dx + dy * dy + dz * dz);
    }
    if (node_j) {
      __syncthreads();
      for (int m = tid; m < n_c; m += kThreads) {
        const int i = node_i[m], j = node_j[m];
        if (j < 0) continue;
        const float4 si = vout[i], sj = vout[j];
        const float wi = w[i].x, wj = w[j].x;
        const float* Rm = R + 9ll * m;
        float4 lam;
        one_shot(Rm, mu[m], phi[m], wi + wj, si.x - sj.x, si.y - sj.y, si.z - sj.z, lam);
        const float dx = Rm[0] * lam.x + Rm[3] * lam.y + Rm[6] * lam.z;
        const float dy = Rm[1] * lam.x + Rm[4] * lam.y + Rm[7] * lam.z;
        const float dz = Rm[2] * lam.x + Rm[5] * lam.y + Rm[8] * lam.z;
        const float4 ni = make_float4(si.x + wi * dx, si.y + wi * dy, si.z + wi * dz, 0.f);
        const float4 nj = make_float4(sj.x - wj * dx, sj.y - wj * dy, sj.z - wj * dz, 0.f);
        vout[i] = ni;
        vout[j] = nj;
        lambda_out[3 * m] = lam.x;
        lambda_out[3 * m + 1] = lam.y;
        lambda_out[3 * m + 2] = lam.z;
        const float4 oi = vin[i], oj = vin[j];
        const float e0 = ni.x - oi.x, e1 = ni.y - oi.y, e2 = ni.z - oi.z;
        const float f0 = nj.x - oj.x, f1 = nj.y - oj.y, f2 = nj.z - oj.z;
        acc += (double)(e0 * e0 + e1 * e1 + e2 * e2) + (double)(f0 * f0 + f1 * f1 + f2 * f2);
      }
    }
    theta = sqrt(block_allreduce(acc, red)) * nscale;
    cur ^= 1;
    if (!isfinite(theta)) { status = VFPI_ERR_NONFINITE; break; }
    if (theta < theta_th) { status = VFPI_OK; break; }
    if (l >= l_max) { status = VFPI_NOT_CONVERGED; break; }
  }
  const float4* fin = cur ? v1 : v0;
  for (int i = tid; i < N; i += kThreads) {
    const float4 q = fin[i];
    v_out[3 * i] = q.x;
    v_out[3 * i + 1] = q.y;
    v_out[3 * i + 2] = q.z;
  }
  if (tid == 0) {
    st->iters = l;
    st->status = status;
    st->err = 0;
    st->theta = theta;
  }
}

// device address of g_scratch, looked up once per device
std::mutex g_mu;
void* g_addr[128] = {};

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

thread_local char g_msg[256];

vfpi_status fail(vfpi_status s, const char* msg) {
  std::snprintf(g_msg, sizeof g_msg, "%s", msg);
  return s;
}

}  // namespace

extern "C" const char* vfpi_noalloc_last_error(void) { return g_msg; }

extern "C" vfpi_status vfpi_solve_noalloc(const vfpi_bsr* A, const float* b,
                                          const vfpi_contacts* Jc, double theta_th, int32_t l_max,
                                          int32_t residual_norm, const float* v_in, float* v_out,
                                          float* lambda_out, int32_t* iters_out, double* theta_out,
                                          void* cuda_stream) {
  g_msg[0] = 0;
  if (!A || !b || !v_in || !v_out) return fail(VFPI_ERR_INVALID_ARG, "A, b, v_in and v_out are required");
  const int N = A->n_nodes;
  const int n_c = Jc ? Jc->n_c : 0;
  if (N < 1 || N > kMaxNodes)
    return fail(VFPI_ERR_INVALID_ARG, "n_nodes must be 1..VFPI_NOALLOC_MAX_NODES (4096)");
  if (n_c < 0 || n_c > N) return fail(VFPI_ERR_INVALID_ARG, "n_c must be 0..n_nodes");
  if (A->nnzb < N || (int64_t)A->nnzb > (int64_t)N * N)
    return fail(VFPI_ERR_INVALID_ARG, "nnzb must be n_nodes..n_nodes^2 (every row holds 1..n_nodes blocks)");
  if (l_max < 1) return fail(VFPI_ERR_INVALID_ARG, "l_max must be >= 1");
  if (residual_norm != VFPI_NORM_ABS && residual_norm != VFPI_NORM_RMS)
    return fail(VFPI_ERR_INVALID_ARG, "unknown residual_norm");
  if (n_c > 0 && (!Jc->node_i || !Jc->R || !Jc->mu || !Jc->phi || !lambda_out))
    return fail(VFPI_ERR_INVALID_ARG, "contacts need node_i, R, mu, phi and lambda_out");
  const void* need[] = {A->row_ptr, A->col_idx, A->vals, b, v_in, v_out};
  for (const void* p : need)
    if (!on_device(p)) return fail(VFPI_ERR_INVALID_ARG, "every array must be device memory");
  if (n_c > 0) {
    const void* cneed[] = {Jc->node_i, Jc->R, Jc->mu, Jc->phi, lambda_out};
    for (const void* p : cneed)
      if (!on_device(p)) return fail(VFPI_ERR_INVALID_ARG, "every array must be device memory");
    if (Jc->node_j && !on_device(Jc->node_j))
      return fail(VFPI_ERR_INVALID_ARG, "every array must be device memory");
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
    cudaGetLastError();
    return fail(VFPI_ERR_CUDA, "cudaGetDevice failed");
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      // set-up, once per device, with that device current
      cudaError_t e = cudaGetSymbolAddress(&g_addr[dev], g_scratch);
      if (e != cudaSuccess) {
        cudaGetLastError();
        g_addr[dev] = nullptr;
        return fail(VFPI_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
      }
    }
    scratch = g_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const double nscale = residual_norm == VFPI_NORM_RMS ? 1.0 / std::sqrt(3.0 * N) : 1.0;
  k_solve_noalloc<<<1, kThreads, 0, s>>>(
      N, A->nnzb, A->row_ptr, A->col_idx, static_cast<const float*>(A->vals), b, n_c,
      n_c ? Jc->node_i : nullptr, n_c ? Jc->node_j : nullptr,
      n_c ? static_cast<const float*>(Jc->R) : nullptr, n_c ? static_cast<const float*>(Jc->mu) : nullptr,
      n_c ? static_cast<const float*>(Jc->phi) : nullptr, theta_th, l_max, nscale, v_in, v_out,
      lambda_out, static_cast<unsigned char*>(scratch));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(VFPI_ERR_CUDA, cudaGetErrorString(e));
  NoallocStatus h;
  std::memset(&h, 0, sizeof h);
  e = cudaMemcpyAsync(&h, static_cast<unsigned char*>(scratch) + kOffStatus, sizeof h,
                      cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(VFPI_ERR_CUDA, cudaGetErrorString(e));
  }
  if (iters_out) *iters_out = h.iters;
  if (theta_out) *theta_out = h.theta;
  if (h.status == VFPI_ERR_INVALID_ARG) {
    if (h.err & kErrRowPtr)
      return fail(VFPI_ERR_INVALID_ARG, "row_ptr must run from 0 to nnzb with 1..n_nodes blocks per row");
    if (h.err & kErrIndex) return fail(VFPI_ERR_INVALID_ARG, "a node or column index is out of range");
    return fail(VFPI_ERR_CONTACT_OVERLAP, "a node is in two contacts (or a D-contact joins a node to itself)");
  }
  if (h.status == VFPI_ERR_NONFINITE) return fail(VFPI_ERR_NONFINITE, "non-finite residual");
  return static_cast<vfpi_status>(h.status);
}
