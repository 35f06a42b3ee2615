// Exact per-site MPO product, the contraction step of the naive algorithm
// (Sec. 2.1, Alg. 1): C_l[(i_a i_b), s, t, (j_a j_b)] =
// sum_u A_l[i_a, s, u, j_a] B_l[i_b, u, t, j_b]. Exposed through the C ABI in
// include/ttfit.h; the compression that follows it in Alg. 1 is tt_mpo_compress.
#include <cuda_runtime.h>
#include <algorithm>
#include <vector>

#include "../../include/ttfit.h"
#include "common.cuh"

using namespace ttfit;

namespace {

// One output core, row-major (a0 b0, s, t, a1 b1); the output is the dominant
// traffic (chi_A chi_B times the inputs), so consecutive threads write
// consecutive j_b and read consecutive entries of B.
template <typename F>
__global__ void __launch_bounds__(256) naive_product_kernel(int a0, int a1, int b0, int b1, int s, int u, int t,
                                                            const F* __restrict__ A, const F* __restrict__ B,
                                                            F* __restrict__ C) {
  const long long cols = (long long)a1 * b1;
  const long long total = (long long)a0 * b0 * s * t * cols;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += stride) {
    const long long row = e / cols;
    const int col = (int)(e - row * cols);
    const int jb = col % b1, ja = col / b1;
    long long r = row;
    const int tt = (int)(r % t);
    r /= t;
    const int ss = (int)(r % s);
    r /= s;
    const int ib = (int)(r % b0);
    const int ia = (int)(r / b0);
    const F* pa = A + (((long long)ia * s + ss) * u) * a1 + ja;
    const F* pb = B + ((long long)ib * u * t + tt) * b1 + jb;
    F acc = F(0);
    for (int uu = 0; uu < u; ++uu) acc += pa[(long long)uu * a1] * pb[(long long)uu * t * b1];
    C[e] = acc;
  }
}

bool desc_ok(const tt_mpo_desc* X) {
  if (!X || X->L < 1 || !X->d_out || !X->d_in || !X->bond || !X->cores) return false;
  if (X->dtype != TT_DTYPE_F64 && X->dtype != TT_DTYPE_F32) return false;
  for (int l = 0; l < X->L; ++l)
    if (!X->cores[l] || X->d_out[l] < 1 || X->d_in[l] < 1 || X->bond[l] < 1) return false;
  return X->bond[X->L] >= 1;
}

}  // namespace

extern "C" tt_status tt_mpo_naive_product(const tt_mpo_desc* A, const tt_mpo_desc* B, const tt_mpo_desc* C,
                                          void* stream) {
  if (!desc_ok(A) || !desc_ok(B) || !desc_ok(C)) return TT_ERR_INVALID_ARGUMENT;
  if (A->dtype != B->dtype || A->dtype != C->dtype) return TT_ERR_INVALID_ARGUMENT;
  const int L = A->L;
  if (B->L != L || C->L != L) return TT_ERR_SHAPE_MISMATCH;
  if (A->bond[0] != 1 || A->bond[L] != 1 || B->bond[0] != 1 || B->bond[L] != 1) return TT_ERR_SHAPE_MISMATCH;
  for (int l = 0; l <= L; ++l)
    if ((long long)C->bond[l] != (long long)A->bond[l] * B->bond[l]) return TT_ERR_SHAPE_MISMATCH;
  for (int l = 0; l < L; ++l)
    if (A->d_in[l] != B->d_out[l] || C->d_out[l] != A->d_out[l] || C->d_in[l] != B->d_in[l])
      return TT_ERR_SHAPE_MISMATCH;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return TT_ERR_CUDA;
  }
  for (int l = 0; l < L; ++l) {
    const int a0 = A->bond[l], a1 = A->bond[l + 1], b0 = B->bond[l], b1 = B->bond[l + 1];
    const int s = A->d_out[l], u = A->d_in[l], t = B->d_in[l];
    const long long total = (long long)a0 * b0 * s * t * a1 * b1;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 8ll * sms));
    ++tl_launches;
    if (A->dtype == TT_DTYPE_F64)
      naive_product_kernel<double><<<blocks, 256, 0, st>>>(a0, a1, b0, b1, s, u, t, (const double*)A->cores[l],
                                                           (const double*)B->cores[l], (double*)C->cores[l]);
    else
      naive_product_kernel<float><<<blocks, 256, 0, st>>>(a0, a1, b0, b1, s, u, t, (const float*)A->cores[l],
                                                          (const float*)B->cores[l], (float*)C->cores[l]);
    if (cudaGetLastError() != cudaSuccess) return TT_ERR_CUDA;
  }
  return TT_OK;
}
