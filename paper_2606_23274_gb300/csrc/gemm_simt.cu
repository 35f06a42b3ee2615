// CUDA-core GEMM over arbitrary tensor layouts:
//   C[cm(m) + cn(n)] = alpha * sum_k A[am(m) + ak(k)] * B[bn(n) + bk(k)] + beta * C[...]
// Every contraction of the fit (environment diagrams, halves, two-site tensor)
// is one call with the index maps of its operands (Sec. 2.3.3 / 2.3.4 shapes).
// It serves the FP64 path, the double-FP32 (df32) path that reaches FP64-class
// accuracy on the FP32 pipes, and the plain-FP32 baseline; the tensor-core
// path lives in gemm_tc.cu.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace ttfit {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T>
__global__ void __launch_bounds__(NT, 3) gemm_simt_kernel(GemmArgs<T> g, T* __restrict__ ws, int k_per_split) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  __shared__ long long arow[BM], brow[BN];
  __shared__ long long akoff[BK], bkoff[BK];  // k offsets of the current tile (one index-map evaluation each)
  const int tid = threadIdx.x;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = blockIdx.z * k_per_split;
  const int ke = min(g.K, kb + k_per_split);
  if (tid < BM) arow[tid] = (m0 + tid < g.M) ? g.am(m0 + tid) : 0;
  else if (tid < BM + BN) brow[tid - BM] = (n0 + tid - BM < g.N) ? g.bn(n0 + tid - BM) : 0;
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int k0 = kb; k0 < ke; k0 += BK) {
    if (tid < BK) akoff[tid] = (k0 + tid < ke) ? g.ak(k0 + tid) : 0;
    else if (tid < 2 * BK) bkoff[tid - BK] = (k0 + tid - BK < ke) ? g.bk(k0 + tid - BK) : 0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int e = tid + NT * i;
      int r, kk;
      if (g.a_kfast) { r = e >> 4; kk = e & 15; } else { r = e & 63; kk = e >> 6; }
      T v = T(0);
      if (m0 + r < g.M && k0 + kk < ke) v = g.A[arow[r] + akoff[kk]];
      As[kk][r] = v;
      if (g.b_kfast) { r = e >> 4; kk = e & 15; } else { r = e & 63; kk = e >> 6; }
      T w = T(0);
      if (n0 + r < g.N && k0 + kk < ke) w = g.B[brow[r] + bkoff[kk]];
      Bs[kk][r] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = madd(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (ws) {  // split-K partial: dense [split][M][N]
    T* w = ws + (size_t)blockIdx.z * g.M * g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int m = m0 + ty + 16 * i;
      if (m >= g.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int n = n0 + tx + 16 * j;
        if (n < g.N) w[(size_t)m * g.N + n] = acc[i][j];
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
    long long cr = g.cm(m);
    long long cr2 = g.C2 ? g.cm2(m) : 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      long long o = cr + g.cn(n);
      T v = g.alpha * acc[i][j];
      if (g.C2) g.C2[cr2 + g.cn2(n)] = v;
      if (g.beta != T(0)) v += g.beta * g.C[o];
      g.C[o] = v;
    }
  }
}

template <typename T>
__global__ void splitk_reduce_kernel(GemmArgs<T> g, const T* __restrict__ ws, int splits) {
  long long total = (long long)g.M * g.N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    int m = (int)(e / g.N), n = (int)(e % g.N);
    T s = T(0);
    for (int z = 0; z < splits; ++z) s += ws[(size_t)z * total + e];
    long long o = g.cm(m) + g.cn(n);
    T v = g.alpha * s;
    if (g.C2) g.C2[g.cm2(m) + g.cn2(n)] = v;
    if (g.beta != T(0)) v += g.beta * g.C[o];
    g.C[o] = v;
  }
}

template <typename T>
cudaError_t splitk_reduce(const GemmArgs<T>& g, const T* ws, int splits, int sm_count, cudaStream_t st) {
  long long total = (long long)g.M * g.N;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4 * sm_count) blocks = 4 * sm_count;
  if (blocks < 1) blocks = 1;
  ++tl_launches;
  splitk_reduce_kernel<T><<<blocks, 256, 0, st>>>(g, ws, splits);
  return cudaGetLastError();
}
template cudaError_t splitk_reduce<double>(const GemmArgs<double>&, const double*, int, int, cudaStream_t);
template cudaError_t splitk_reduce<float>(const GemmArgs<float>&, const float*, int, int, cudaStream_t);
template cudaError_t splitk_reduce<df32>(const GemmArgs<df32>&, const df32*, int, int, cudaStream_t);

template <typename T>
cudaError_t gemm_simt(const GemmArgs<T>& g, T* ws, size_t ws_elems, int sm_count, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.K <= 0) {  // empty contraction: C = beta * C
    GemmArgs<T> z = g;
    z.alpha = T(0);
    ++tl_launches;
    splitk_reduce_kernel<T><<<256, 256, 0, st>>>(z, nullptr, 0);
    return cudaGetLastError();
  }
  int gm = (g.M + BM - 1) / BM, gn = (g.N + BN - 1) / BN;
  int tiles = gm * gn;
  int splits = 1;
  // split K while the grid covers fewer than two waves of the SMs and each
  // split keeps at least kmin k-steps: a tile's time is bound by its SM's
  // arithmetic rate, which for FP64 is 1/64 of the FP32 rate on this GPU (and
  // a df32 multiply-add takes 15 FP32 instructions), so the small GEMMs of
  // those types split down to one k-tile per CTA
  const int kmin = (std::is_same<T, double>::value || std::is_same<T, df32>::value) ? 16 : 256;
  while (tiles * splits < 2 * sm_count && g.K / (splits * 2) >= kmin &&
         (size_t)(splits * 2) * g.M * g.N <= ws_elems)
    splits *= 2;
  int kps = (g.K + splits - 1) / splits;
  kps = (kps + BK - 1) / BK * BK;
  splits = (g.K + kps - 1) / kps;
  dim3 grid(gn, gm, splits);
  if (splits == 1) {
    ++tl_launches;
    gemm_simt_kernel<T><<<grid, NT, 0, st>>>(g, nullptr, kps);
  } else {
    ++tl_launches;
    gemm_simt_kernel<T><<<grid, NT, 0, st>>>(g, ws, kps);
    long long total = (long long)g.M * g.N;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4 * sm_count) blocks = 4 * sm_count;
    ++tl_launches;
    splitk_reduce_kernel<T><<<blocks, 256, 0, st>>>(g, ws, splits);
  }
  return cudaGetLastError();
}

template cudaError_t gemm_simt<double>(const GemmArgs<double>&, double*, size_t, int, cudaStream_t);
template cudaError_t gemm_simt<float>(const GemmArgs<float>&, float*, size_t, int, cudaStream_t);
template cudaError_t gemm_simt<df32>(const GemmArgs<df32>&, df32*, size_t, int, cudaStream_t);

}  // namespace ttfit
