// Dense factorisations and element-wise kernels of the fit's local update:
// Householder QR, one-sided Jacobi SVD, the truncation rule (Sec. 2.3.4), the
// gauge update of Alg. 3 / Alg. 4, Philox Gaussian fill (Sec. 3.1's Omega),
// layout copies and norms.
#include <algorithm>
#include <cfloat>
#include "common.cuh"
#include "kernels.h"

namespace ttfit {

template <typename C>
__device__ __forceinline__ C block_sum(C v, C* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  C t = (lane < nw) ? red[lane] : C(0);
  t = warp_sum(t);
  return t;
}

// ---------------------------------------------------------------------------
// Householder QR, one CTA. X: q x p column-major (ld q), overwritten by the
// reflectors (unit vectors, rows j..q-1 of column j). Q: q x r, R: r x p.
// ---------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(1024) qr_house_kernel(int q, int p, double* __restrict__ X, double* __restrict__ Q,
                                                        double* __restrict__ R) {
  __shared__ C red[32];
  __shared__ double diag[1024];  // r <= 1024
  const int r = min(q, p);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < r; ++j) {
    double* xj = X + (size_t)j * q;
    C ss = 0;
    for (int i = j + threadIdx.x; i < q; i += blockDim.x) {
      C v = (C)xj[i];
      ss += v * v;
    }
    ss = block_sum(ss, red);
    const C x0 = (C)xj[j];
    const C nrm = sqrt(ss);
    const C alpha = (x0 >= C(0)) ? -nrm : nrm;
    const C v0 = x0 - alpha;
    const C vn2 = ss - x0 * x0 + v0 * v0;
    __syncthreads();
    const bool zero = !(vn2 > C(0));
    const C inv = zero ? C(0) : C(1) / sqrt(vn2);
    for (int i = j + threadIdx.x; i < q; i += blockDim.x) xj[i] = (double)((i == j ? v0 : (C)xj[i]) * inv);
    if (threadIdx.x == 0) diag[j] = zero ? 0.0 : (double)alpha;
    __syncthreads();
    if (!zero) {
      for (int c = j + 1 + warp; c < p; c += nw) {
        double* xc = X + (size_t)c * q;
        C d = 0;
        for (int i = j + lane; i < q; i += 32) d += (C)xj[i] * (C)xc[i];
        d = warp_sum(d);
        for (int i = j + lane; i < q; i += 32) xc[i] = (double)((C)xc[i] - C(2) * d * (C)xj[i]);
      }
    }
    __syncthreads();
  }
  // R (r x p, col-major, ld r)
  for (long long e = threadIdx.x; e < (long long)r * p; e += blockDim.x) {
    int i = (int)(e % r), c = (int)(e / r);
    double v = (i < c) ? X[(size_t)c * q + i] : (i == c ? diag[i] : 0.0);
    R[(size_t)c * r + i] = v;
  }
  // Q = H_0 ... H_{r-1} [I_r; 0]
  for (long long e = threadIdx.x; e < (long long)q * r; e += blockDim.x) {
    int i = (int)(e % q), c = (int)(e / q);
    Q[(size_t)c * q + i] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = r - 1; j >= 0; --j) {
    const double* vj = X + (size_t)j * q;
    for (int c = j + warp; c < r; c += nw) {
      double* qc = Q + (size_t)c * q;
      C d = 0;
      for (int i = j + lane; i < q; i += 32) d += (C)vj[i] * (C)qc[i];
      d = warp_sum(d);
      for (int i = j + lane; i < q; i += 32) qc[i] = (double)((C)qc[i] - C(2) * d * (C)vj[i]);
    }
    __syncthreads();
  }
  // sign convention diag(R) >= 0
  for (int j = warp; j < r; j += nw) {
    if (diag[j] < 0.0) {
      for (int c = j + lane; c < p; c += 32) R[(size_t)c * r + j] = -R[(size_t)c * r + j];
      for (int i = lane; i < q; i += 32) Q[(size_t)j * q + i] = -Q[(size_t)j * q + i];
    }
  }
}

template <typename C>
cudaError_t qr_householder(int q, int p, double* X, double* Q, double* R, cudaStream_t st) {
  if (q <= 0 || p <= 0) return cudaSuccess;
  if (q > 1 << 20 || min(q, p) > 1024) return cudaErrorInvalidValue;
  qr_house_kernel<C><<<1, 1024, 0, st>>>(q, p, X, Q, R);
  return cudaGetLastError();
}
template cudaError_t qr_householder<double>(int, int, double*, double*, double*, cudaStream_t);
template cudaError_t qr_householder<float>(int, int, double*, double*, double*, cudaStream_t);

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi SVD, one CTA, round-robin pair ordering: every
// round applies P/2 disjoint plane rotations that orthogonalise column pairs;
// a sweep is P-1 rounds; it stops after a sweep without rotations.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rr_pair(int round, int k, int P, int& i, int& j) {
  const int n = P - 1;
  if (k == 0) {
    i = 0;
    j = 1 + round % n;
  } else {
    i = 1 + (round + k) % n;
    j = 1 + (round - k + n) % n;
  }
}

template <typename C>
__global__ void __launch_bounds__(1024) jacobi_kernel(int q, int p, double* __restrict__ W, double* __restrict__ V,
                                                      int max_sweeps, double tol, uint32_t* errw,
                                                      double* __restrict__ Uo, double* __restrict__ So,
                                                      double* __restrict__ Vo) {
  __shared__ int rotated;
  __shared__ double nrm[1024];
  __shared__ int rank_[1024];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (long long e = threadIdx.x; e < (long long)p * p; e += blockDim.x) {
    int i = (int)(e % p), c = (int)(e / p);
    V[e] = (i == c) ? 1.0 : 0.0;
  }
  const int P = p + (p & 1);
  int sweep = 0;
  bool done = (p < 2);
  __syncthreads();
  while (!done && sweep < max_sweeps) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < P - 1; ++round) {
      for (int k = warp; k < P / 2; k += nw) {
        int i, j;
        rr_pair(round, k, P, i, j);
        if (i >= p || j >= p) continue;
        if (i > j) { int t = i; i = j; j = t; }
        double* wi = W + (size_t)i * q;
        double* wj = W + (size_t)j * q;
        C a = 0, b = 0, g = 0;
        for (int r = lane; r < q; r += 32) {
          C x = (C)wi[r], y = (C)wj[r];
          a += x * x;
          b += y * y;
          g += x * y;
        }
        a = warp_sum(a);
        b = warp_sum(b);
        g = warp_sum(g);
        if (!(a > C(0) && b > C(0))) continue;
        if (!(fabs((double)g) > tol * sqrt((double)a) * sqrt((double)b))) continue;
        const C zeta = (b - a) / (C(2) * g);
        const C t = (zeta >= C(0) ? C(1) : C(-1)) / (fabs(zeta) + sqrt(C(1) + zeta * zeta));
        const C cs = C(1) / sqrt(C(1) + t * t);
        const C sn = cs * t;
        for (int r = lane; r < q; r += 32) {
          C x = (C)wi[r], y = (C)wj[r];
          wi[r] = (double)(cs * x - sn * y);
          wj[r] = (double)(sn * x + cs * y);
        }
        double* vi = V + (size_t)i * p;
        double* vj = V + (size_t)j * p;
        for (int r = lane; r < p; r += 32) {
          C x = (C)vi[r], y = (C)vj[r];
          vi[r] = (double)(cs * x - sn * y);
          vj[r] = (double)(sn * x + cs * y);
        }
        if (lane == 0) rotated = 1;
      }
      __syncthreads();
    }
    ++sweep;
    done = (rotated == 0);
    __syncthreads();
  }
  if (!done && threadIdx.x == 0 && errw) atomicOr(errw, ERRW_NOCONV);
  // singular values = column norms (FP64), sorted descending, ties by index
  for (int c = warp; c < p; c += nw) {
    const double* wc = W + (size_t)c * q;
    double s = 0;
    for (int r = lane; r < q; r += 32) s += wc[r] * wc[r];
    s = warp_sum(s);
    if (lane == 0) nrm[c] = sqrt(s);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < p; c += blockDim.x) {
    int rk = 0;
    double v = nrm[c];
    for (int d = 0; d < p; ++d) rk += (nrm[d] > v) || (nrm[d] == v && d < c);
    rank_[c] = rk;
    So[rk] = v;
  }
  __syncthreads();
  for (int c = warp; c < p; c += nw) {
    const int rk = rank_[c];
    const double s = nrm[c];
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    for (int r = lane; r < q; r += 32) Uo[(size_t)rk * q + r] = W[(size_t)c * q + r] * inv;
    for (int r = lane; r < p; r += 32) Vo[(size_t)rk * p + r] = V[(size_t)c * p + r];
  }
}

template <typename C>
cudaError_t jacobi_svd(int q, int p, double* W, double* U, double* S, double* V, double* Vwork, int max_sweeps,
                       uint32_t* errw, cudaStream_t st) {
  if (q <= 0 || p <= 0) return cudaSuccess;
  if (p > 1024 || q < p) return cudaErrorInvalidValue;
  const double eps = (sizeof(C) == 8) ? DBL_EPSILON : (double)FLT_EPSILON;
  const double tol = eps * sqrt((double)q);
  jacobi_kernel<C><<<1, 1024, 0, st>>>(q, p, W, Vwork, max_sweeps, tol, errw, U, S, V);
  return cudaGetLastError();
}
template cudaError_t jacobi_svd<double>(int, int, double*, double*, double*, double*, double*, int, uint32_t*,
                                        cudaStream_t);
template cudaError_t jacobi_svd<float>(int, int, double*, double*, double*, double*, double*, int, uint32_t*,
                                       cudaStream_t);

// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024) frob_kernel(const T* __restrict__ x, long long n, double* out, uint32_t* errw) {
  __shared__ double red[32];
  double s = 0;
  bool bad = false;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    double v = (double)x[i];
    bad |= !isfinite(v);
    s += v * v;
  }
  s = block_sum(s, red);
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    *out = sqrt(s);
    if (bad && errw) atomicOr(errw, ERRW_NAN);
  }
}

template <typename T>
cudaError_t frob_norm(const T* x, long long n, double* out, uint32_t* errw, cudaStream_t st) {
  frob_kernel<T><<<1, 1024, 0, st>>>(x, n, out, errw);
  return cudaGetLastError();
}
template cudaError_t frob_norm<double>(const double*, long long, double*, uint32_t*, cudaStream_t);
template cudaError_t frob_norm<float>(const float*, long long, double*, uint32_t*, cudaStream_t);

// ---------------------------------------------------------------------------
__global__ void truncate_kernel(const double* S, int p, const double* normM, double tau_over_L, int chi_max,
                                double cutoff, int* info, double* dinfo) {
  if (threadIdx.x != 0) return;
  const double nM = *normM;
  int k = min(chi_max, p);
  if (tau_over_L > 0.0) {
    const double thr = tau_over_L * nM;
    int kmin = p;
    double tail = 0.0;
    for (int j = p - 1; j >= 1; --j) {
      tail += S[j] * S[j];
      if (sqrt(tail) <= thr) kmin = j;
      else break;
    }
    k = min(k, kmin);
  }
  if (p > 0) {
    int cnt = 0;
    for (int j = 0; j < p; ++j) cnt += S[j] > cutoff * S[0];
    k = min(k, cnt);
  }
  k = max(k, 1);
  double kept = 0.0, disc = 0.0;
  for (int j = 0; j < p; ++j) {
    if (j < k) kept += S[j] * S[j];
    else disc += S[j] * S[j];
  }
  info[0] = k;
  dinfo[0] = kept;
  dinfo[1] = nM > 0.0 ? sqrt(disc) / nM : 0.0;
}

cudaError_t truncate_rule(const double* S, int p, const double* normM, double tau_over_L, int chi_max, double cutoff,
                          int* info, double* dinfo, cudaStream_t st) {
  truncate_kernel<<<1, 32, 0, st>>>(S, p, normM, tau_over_L, chi_max, cutoff, info, dinfo);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
template <typename T>
__global__ void gauge_update_kernel(int mode, int m, int n, const double* __restrict__ U, int ld_u,
                                    const double* __restrict__ S, const double* __restrict__ V, int ld_v,
                                    const int* __restrict__ kdev, double* Cl, double* Cr, double* Y, T* Ut, T* Vt) {
  const int k = *kdev;
  const long long tot_l = (long long)m * k, tot_r = (long long)k * n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot_l; e += stride) {
    const int i = (int)(e / k), j = (int)(e % k);
    const double u = U[(size_t)j * ld_u + i];
    Cl[e] = (mode == 0) ? u : u * S[j];
    Ut[(size_t)j * m + i] = (T)u;
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot_r; e += stride) {
    const int j = (int)(e / n), c = (int)(e % n);
    const double v = V[(size_t)j * ld_v + c];
    Cr[e] = (mode == 1) ? v : S[j] * v;
    Vt[e] = (T)v;
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < k; e += stride)
    Y[e] = (mode == 2) ? (S[e] > 0.0 ? 1.0 / S[e] : 0.0) : 1.0;
}

template <typename T>
cudaError_t gauge_update(int mode, int m, int n, const double* U, int ld_u, const double* S, const double* V, int ld_v,
                         const int* kdev, double* Cl, double* Cr, double* Y, T* Ut, T* Vt, cudaStream_t st) {
  long long tot = (long long)(m > n ? m : n) * 128;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  gauge_update_kernel<T><<<blocks, 256, 0, st>>>(mode, m, n, U, ld_u, S, V, ld_v, kdev, Cl, Cr, Y, Ut, Vt);
  return cudaGetLastError();
}
template cudaError_t gauge_update<double>(int, int, int, const double*, int, const double*, const double*, int,
                                          const int*, double*, double*, double*, double*, double*, cudaStream_t);
template cudaError_t gauge_update<float>(int, int, int, const double*, int, const double*, const double*, int,
                                         const int*, double*, double*, double*, float*, float*, cudaStream_t);

// ---------------------------------------------------------------------------
template <typename Tin, typename Tout>
__global__ void copy_map_kernel(int rows, int cols, const Tin* __restrict__ in, IdxMap im, IdxMap in_,
                                Tout* __restrict__ out, IdxMap om, IdxMap on, double scale) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols), j = (int)(e % cols);
    out[om(i) + on(j)] = (Tout)(scale * (double)in[im(i) + in_(j)]);
  }
}

template <typename Tin, typename Tout>
cudaError_t copy_map(int rows, int cols, const Tin* in, IdxMap im, IdxMap in_, Tout* out, IdxMap om, IdxMap on,
                     double scale, cudaStream_t st) {
  long long tot = (long long)rows * cols;
  if (tot <= 0) return cudaSuccess;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  copy_map_kernel<Tin, Tout><<<blocks, 256, 0, st>>>(rows, cols, in, im, in_, out, om, on, scale);
  return cudaGetLastError();
}
template cudaError_t copy_map<double, double>(int, int, const double*, IdxMap, IdxMap, double*, IdxMap, IdxMap, double,
                                              cudaStream_t);
template cudaError_t copy_map<double, float>(int, int, const double*, IdxMap, IdxMap, float*, IdxMap, IdxMap, double,
                                             cudaStream_t);
template cudaError_t copy_map<float, double>(int, int, const float*, IdxMap, IdxMap, double*, IdxMap, IdxMap, double,
                                             cudaStream_t);
template cudaError_t copy_map<float, float>(int, int, const float*, IdxMap, IdxMap, float*, IdxMap, IdxMap, double,
                                            cudaStream_t);

// ---------------------------------------------------------------------------
__global__ void philox_fill_kernel(double* out, long long count, uint64_t seed, uint64_t stream, double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    out[i] = scale * philox_normal(seed, stream, (uint64_t)i);
}

cudaError_t philox_fill(double* out, long long count, uint64_t seed, uint64_t stream, double scale, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int blocks = (int)((count + 255) / 256);
  if (blocks > 2048) blocks = 2048;
  philox_fill_kernel<<<blocks, 256, 0, st>>>(out, count, seed, stream, scale);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sign convention of singular pair j: the entry of largest magnitude of u_j is
// positive (lowest index on ties); (u_j, v_j) are flipped together.
__global__ void fix_signs_kernel(int m, int n, double* __restrict__ U, int ld_u, double* __restrict__ V, int ld_v) {
  __shared__ double sb[32];
  __shared__ int si[32];
  __shared__ double sgn;
  double* u = U + (size_t)blockIdx.x * ld_u;
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double a = fabs(u[i]);
    if (a > best) {
      best = a;
      bi = i;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  if (lane == 0) {
    sb[warp] = best;
    si[warp] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w)
      if (sb[w] > sb[0] || (sb[w] == sb[0] && si[w] < si[0])) {
        sb[0] = sb[w];
        si[0] = si[w];
      }
    sgn = (si[0] < m && u[si[0]] < 0.0) ? -1.0 : 1.0;
  }
  __syncthreads();
  if (sgn < 0.0) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) u[i] = -u[i];
    double* v = V + (size_t)blockIdx.x * ld_v;
    for (int c = threadIdx.x; c < n; c += blockDim.x) v[c] = -v[c];
  }
}

cudaError_t fix_signs(int m, int n, int p, double* U, int ld_u, double* V, int ld_v, cudaStream_t st) {
  if (p <= 0 || m <= 0) return cudaSuccess;
  fix_signs_kernel<<<p, 256, 0, st>>>(m, n, U, ld_u, V, ld_v);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void scale_cols_kernel(int rows, int cols, const double* __restrict__ in, const double* __restrict__ y,
                                  double* __restrict__ out) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x)
    out[e] = y ? in[e] * y[e % cols] : in[e];
}

cudaError_t scale_cols(int rows, int cols, const double* in, const double* y, double* out, cudaStream_t st) {
  long long tot = (long long)rows * cols;
  if (tot <= 0) return cudaSuccess;
  int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
  scale_cols_kernel<<<blocks, 256, 0, st>>>(rows, cols, in, y, out);
  return cudaGetLastError();
}

}  // namespace ttfit
