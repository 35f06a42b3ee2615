// Internal launchers of the fit library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include "common.cuh"

namespace ttfit {

template <typename T>
struct GemmArgs {
  int M = 0, N = 0, K = 0;
  const T* A = nullptr;
  IdxMap am, ak;
  bool a_kfast = true;  // consecutive k are adjacent in memory (load k-fastest)
  const T* B = nullptr;
  IdxMap bn, bk;
  bool b_kfast = true;
  T* C = nullptr;
  IdxMap cm, cn;
  T alpha = T(1), beta = T(0);
  // optional second copy of the result in another layout (written with beta = 0)
  T* C2 = nullptr;
  IdxMap cm2, cn2;
};

template <typename T>
cudaError_t gemm_simt(const GemmArgs<T>& g, T* ws, size_t ws_elems, int sm_count, cudaStream_t st);

// C = alpha * sum over `splits` dense [M][N] partials in ws + beta * C (output maps of g)
template <typename T>
cudaError_t splitk_reduce(const GemmArgs<T>& g, const T* ws, int splits, int sm_count, cudaStream_t st);

// Tensor-core (tcgen05, kind::tf32) GEMM; cudaErrorNotSupported when the operand
// layouts cannot be loaded by TMA (A and B K-major, 16-byte aligned rows).
// split = true: 3xTF32 (hi*hi + hi*lo + lo*hi, about FP32 accuracy).
cudaError_t gemm_tf32(const GemmArgs<float>& g, float* ws, size_t ws_elems, int sm_count, uint32_t* errw,
                      cudaStream_t st, bool split = false);

// FP64-class GEMM of double-FP32 operands on the tensor cores (fixed-point
// digit split, exact FP32 accumulation of the leading digit levels), with TF32
// digits (kind::tf32) or BF16 digits (kind::f16, bf16 = true); scratch as
// documented in gemm_tc.cu. cudaErrorNotSupported: use gemm_simt.
constexpr int OZ_DIGITS = 6;
constexpr int OZ_CHUNK = 512;
cudaError_t gemm_oz(const GemmArgs<df32>& g, float* sA, float* sB, size_t slice_elems, int* eA, int* eB,
                    size_t exp_elems, df32* ws, size_t ws_elems, int sm_count, uint32_t* errw, cudaStream_t st,
                    bool bf16 = false);

// out[om(i) + on(j)] = (Tout) (scale * in[im(i) + in_(j)]), i < rows, j < cols
template <typename Tin, typename Tout>
cudaError_t copy_map(int rows, int cols, const Tin* in, IdxMap im, IdxMap in_, Tout* out, IdxMap om, IdxMap on,
                     double scale, cudaStream_t st);

// fill out[i] = scale * N(0,1)_philox(seed, stream, i), i < count
template <typename F>
cudaError_t philox_fill(F* out, long long count, uint64_t seed, uint64_t stream, double scale, cudaStream_t st);

// Householder QR of the q x p column-major matrix X (ld q; overwritten):
// Q is q x r (col-major, ld q), R is r x p (col-major, ld r), r = min(q, p),
// diag(R) >= 0. One CTA. C: arithmetic type, S: storage type.
template <typename C, typename S>
cudaError_t qr_householder(int q, int p, S* X, S* Q, S* R, cudaStream_t st);
// The same factorisation of FP64 storage in double-FP32 arithmetic (about 4x
// the FP64 rate of this GPU, rounding ~1e-14 instead of 1e-16); shapes the
// cluster kernel does not take run in FP64.
cudaError_t qr_householder_df32(int q, int p, double* X, double* Q, double* R, cudaStream_t st);

// One-sided Jacobi SVD of the q x p column-major W (q >= p, ld q; overwritten):
// W = U diag(S) V^T with U (q x p, col-major), S sorted descending, V (p x p,
// col-major). C is the arithmetic type of the rotations, S the storage type;
// the working set is held in shared memory when it fits (<= 200 KB).
// errw |= ERRW_NOCONV when max_sweeps is reached.
template <typename C, typename S>
cudaError_t jacobi_svd(int q, int p, S* W, S* U, S* Sv, S* V, S* Vwork, int max_sweeps, uint32_t* errw,
                       cudaStream_t st);

// ||X||_F of n values (type T) into *out (double), flags non-finite values.
template <typename T>
cudaError_t frob_norm(const T* x, long long n, double* out, uint32_t* errw, cudaStream_t st);

// Truncation rule (Sec. 2.3.4): from sorted S (p values), ||M||_F, writes
// info[0] = k, and dinfo[0] = sum_{j<k} s_j^2, dinfo[1] = sqrt(sum_{j>=k} s_j^2)/||M||_F.
template <typename F>
cudaError_t truncate_rule(const F* S, int p, const double* normM, double tau_over_L, int chi_max,
                          double cutoff, int* info, double* dinfo, cudaStream_t st);

// x_j = sqrt(max(x_j, 0)) (singular values from Gram eigenvalues)
template <typename F>
cudaError_t sqrt_clamp(int n, F* x, cudaStream_t st);

// Gauge update after the factorisation of the m x n two-site matrix
// (U: m x ld_u col-major, S, V: n x ld_v col-major; k from *kdev):
// mode 0 = site forward (C_l = U, C_{l+1} = S V^T), 1 = site backward
// (C_l = U S, C_{l+1} = V^T), 2 = inverse (Psi_l = U S, Psi_{l+1} = S V^T,
// Y_l = 1/S). Writes Cl (m x k row-major), Cr (k x n row-major), Y (k) and
// the environment operands Ut (k x m row-major) and Vt (k x n row-major) in T.
template <typename T, typename F>
cudaError_t gauge_update(int mode, int m, int n, const F* U, int ld_u, const F* S, const F* V, int ld_v,
                         const int* kdev, double* Cl, double* Cr, double* Y, T* Ut, T* Vt, cudaStream_t st);

// Flip singular pairs j < p so that the largest-magnitude entry of U[:, j] is
// positive (U: m x p col-major ld_u; V: n x p col-major ld_v).
template <typename F>
cudaError_t fix_signs(int m, int n, int p, F* U, int ld_u, F* V, int ld_v, cudaStream_t st);

// Alg. 4 from FP64 isometries and P = U^T Theta V (see linalg.cu)
template <typename T>
cudaError_t inverse_gauge_update(int m, int n, int k, const double* U, const double* V, const T* P, double* Cl,
                                 double* Cr, double* Y, cudaStream_t st);

// out (rows x cols, row-major, type T) = diag(y) * in (y == nullptr: plain cast copy)
template <typename T>
cudaError_t scale_rows(int rows, int cols, const double* in, const double* y, T* out, cudaStream_t st);

// out (rows x cols, row-major) = in * diag(y) (y == nullptr: plain copy)
cudaError_t scale_cols(int rows, int cols, const double* in, const double* y, double* out, cudaStream_t st);
// 2^-e scaling around a lower-precision factorisation (e = exponent of max |x|, device int)
template <typename T>
cudaError_t absmax_exponent(const T* x, long long n, int* e, cudaStream_t st);
template <typename Tin, typename Tout>
cudaError_t copy_pow2(long long n, const Tin* in, Tout* out, const int* e, cudaStream_t st);
template <typename F>
cudaError_t unscale_pow2(int p, F* s, double* nrm, const int* e, cudaStream_t st);
// out (cols x rows) = (in diag(y))^T in type T
template <typename T>
cudaError_t scale_cols_t(int rows, int cols, const double* in, const double* y, T* out, cudaStream_t st);

// Inverse of an FP32 upper-triangular R (p x p, ld ldr) for the FP64-class
// randomized update (linalg.cu), scaled by 2^-*eexp (eexp may be null):
// out p x p column-major double-FP32. p <= TRI_INV_MAX.
constexpr int TRI_INV_MAX = 160;
cudaError_t tri_inv(int p, const float* R, int ldr, const int* eexp, df32* out, uint32_t* errw, cudaStream_t st);
// out = in diag(2^-e / s) in double-FP32 (in, out: rows x cols column-major)
cudaError_t scale_cols_inv(int rows, int cols, const float* in, const float* s, const int* eexp, df32* out,
                           cudaStream_t st);
// ERRW_HPFAIL when max |G - I| > tol (G: p x p double-FP32)
cudaError_t ortho_check(int p, const df32* G, double tol, uint32_t* errw, cudaStream_t st);

}  // namespace ttfit
