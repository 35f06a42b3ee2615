// Standalone truncated SVD of a device matrix (the factorisation of the local
// update, Sec. 2.3.4): one-sided Jacobi in FP64 and the truncation rule
// k = min(chi_max, min{k : sqrt(sum_{j>k} s_j^2) <= tau_rel ||M||_F}), k >= 1,
// dropping s_j <= 1e-13 s_1. Exposed through the C ABI in include/ttfit.h.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/ttfit.h"
#include "common.cuh"
#include "kernels.h"

using namespace ttfit;

namespace {

// scratch layout (in doubles) for an m x n input, r = min(m, n), q = max(m, n):
// X (q r) | Ux (q r) | Vx (r r) | Vw (r r) | Sv (r) | nrm (1) | dinfo (2) | info (4 x u32 = 2) | k (1)
size_t svd_scratch_doubles(int m, int n) {
  const size_t r = std::min(m, n), q = std::max(m, n);
  return 2 * q * r + 2 * r * r + r + 1 + 2 + 2 + 1;
}
size_t svd_info_offset(int m, int n) {
  const size_t r = std::min(m, n), q = std::max(m, n);
  return 2 * q * r + 2 * r * r + r + 3;
}

__global__ void svd_outputs_kernel(int m, int n, int tr, const double* __restrict__ Ux, const double* __restrict__ Vx,
                                   const double* __restrict__ Sv, double* __restrict__ U, double* __restrict__ S,
                                   double* __restrict__ Vt) {
  // X = Ux diag(S) Vx^T with X = M (tr = 0, Ux m x r) or X = M^T (tr = 1, Ux n x r)
  const int r = min(m, n);
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long e = t0; e < (long long)m * r; e += stride) {  // U: m x r row-major
    const int i = (int)(e / r), j = (int)(e % r);
    U[e] = tr ? Vx[(size_t)j * r + i] : Ux[(size_t)j * m + i];
  }
  for (long long e = t0; e < (long long)r * n; e += stride) {  // Vt: r x n row-major
    const int j = (int)(e / n), c = (int)(e % n);
    Vt[e] = tr ? Ux[(size_t)j * n + c] : Vx[(size_t)j * r + c];
  }
  for (long long e = t0; e < r; e += stride) S[e] = Sv[e];
}

cudaError_t svd_run(const double* M, int m, int n, int chi_max, double tau_rel, double* U, double* S, double* Vt,
                    int* k_dev, double* scratch, cudaStream_t st) {
  const int r = std::min(m, n), q = std::max(m, n);
  const bool tr = m < n;
  double* X = scratch;
  double* Ux = X + (size_t)q * r;
  double* Vx = Ux + (size_t)q * r;
  double* Vw = Vx + (size_t)r * r;
  double* Sv = Vw + (size_t)r * r;
  double* nrm = Sv + r;
  double* dinfo = nrm + 1;
  uint32_t* info = (uint32_t*)(dinfo + 2);
  cudaError_t e = cudaMemsetAsync(info, 0, 4 * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  // tall orientation, column-major: M^T column-major is M row-major (tr); else transpose
  if (tr) e = cudaMemcpyAsync(X, M, sizeof(double) * (size_t)m * n, cudaMemcpyDeviceToDevice, st);
  else e = copy_map<double, double>(m, n, M, IdxMap::lin(n), IdxMap::lin(1), X, IdxMap::lin(1), IdxMap::lin(m), 1.0, st);
  if (e != cudaSuccess) return e;
  if ((e = frob_norm<double>(M, (long long)m * n, nrm, info, st)) != cudaSuccess) return e;
  if ((e = jacobi_svd<double, double>(q, r, X, Ux, Sv, Vx, Vw, 60, info, st)) != cudaSuccess) return e;
  if ((e = fix_signs<double>(tr ? r : q, tr ? q : r, r, tr ? Vx : Ux, tr ? r : q, tr ? Ux : Vx, tr ? q : r, st)) !=
      cudaSuccess)
    return e;
  if ((e = truncate_rule<double>(Sv, r, nrm, tau_rel, chi_max, 1e-13, k_dev, dinfo, st)) != cudaSuccess) return e;
  const long long tot = (long long)q * r;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((tot + 255) / 256, 1024));
  ++tl_launches;
  svd_outputs_kernel<<<blocks, 256, 0, st>>>(m, n, tr ? 1 : 0, Ux, Vx, Sv, U, S, Vt);
  return cudaGetLastError();
}

tt_status svd_check(const double* M, int m, int n, int chi_max, double tau_rel, const double* U, const double* S,
                    const double* Vt, const int* k_out) {
  if (!M || !U || !S || !Vt || !k_out) return TT_ERR_INVALID_ARGUMENT;
  if (m < 1 || n < 1 || chi_max < 1 || !(tau_rel >= 0.0)) return TT_ERR_INVALID_ARGUMENT;
  if (std::min(m, n) > 1024) return TT_ERR_INVALID_ARGUMENT;
  return TT_OK;
}

}  // namespace

extern "C" tt_status tt_svd_truncated(const double* M, int m, int n, int chi_max, double tau_rel, double* U,
                                      double* S, double* Vt, int* k_out, void* stream) {
  tt_status s = svd_check(M, m, n, chi_max, tau_rel, U, S, Vt, k_out);
  if (s != TT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nd = svd_scratch_doubles(m, n);
  double* scratch = nullptr;
  if (cudaMalloc(&scratch, nd * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return TT_ERR_OUT_OF_MEMORY;
  }
  int* k_dev = (int*)(scratch + nd - 1);
  cudaError_t e = svd_run(M, m, n, chi_max, tau_rel, U, S, Vt, k_dev, scratch, st);
  int k = 0;
  uint32_t flags[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&k, k_dev, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(flags, scratch + svd_info_offset(m, n), 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(scratch);
  if (e != cudaSuccess) return TT_ERR_CUDA;
  if (flags[0] & (ERRW_NAN | ERRW_NOCONV)) return TT_ERR_NUMERICAL;
  *k_out = k;
  return TT_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant. Its scratch is this file-scope device array: every
// GPU that loads the library holds these 4 MiB until the process exits, and
// every call on a device reuses the same array (so calls that overlap on the
// GPU race). Host code may not use the array's name as a device address; the
// address is looked up per device with cudaGetSymbolAddress and cached.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocDoubles = size_t(1) << 19;  // 4 MiB of FP64 scratch
__device__ __align__(256) double g_svd_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_svd_scratch on the current device (looked up on the
// first call on that device, with that device current).
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_svd_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (double*)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" tt_status tt_svd_truncated_noalloc(const double* M, int m, int n, int chi_max, double tau_rel, double* U,
                                              double* S, double* Vt, int* k_out, void* stream) {
  tt_status s = svd_check(M, m, n, chi_max, tau_rel, U, S, Vt, k_out);
  if (s != TT_OK) return s;
  const size_t nd = svd_scratch_doubles(m, n);
  if (nd > kNoAllocDoubles) return TT_ERR_INVALID_ARGUMENT;  // beyond the fixed scratch
  cudaStream_t st = (cudaStream_t)stream;
  double* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return TT_ERR_CUDA;
  }
  int* k_dev = (int*)(scratch + nd - 1);
  // svd_run clears the error flags it reads; every other scratch word it uses
  // is written before it is read
  cudaError_t e = svd_run(M, m, n, chi_max, tau_rel, U, S, Vt, k_dev, scratch, st);
  int k = 0;
  uint32_t flags[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&k, k_dev, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(flags, scratch + svd_info_offset(m, n), 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return TT_ERR_CUDA;
  if (flags[0] & (ERRW_NAN | ERRW_NOCONV)) return TT_ERR_NUMERICAL;
  *k_out = k;
  return TT_OK;
}
