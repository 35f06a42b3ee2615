// Dense factorisations and element-wise kernels of the fit's local update:
// Householder QR, one-sided Jacobi SVD, the truncation rule (Sec. 2.3.4), the
// gauge update of Alg. 3 / Alg. 4, Philox Gaussian fill (Sec. 3.1's Omega),
// layout copies and norms.
#include <cooperative_groups.h>
#include <algorithm>
#include <cfloat>
#include <climits>
#include <type_traits>
#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

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
// reflectors (unit vectors, rows j..q-1 of column j). Q: q x r, R: r x p,
// r = min(q, p), diag(R) >= 0. The current reflector sits in shared memory;
// each warp updates two trailing columns at a time, caching their RM rows per
// lane in registers between the dot product and the update (q <= 32 RM).
// All arithmetic is in C (no FP64 in the FP32 instantiation).
// ---------------------------------------------------------------------------
template <typename C, typename S, int RM>
__device__ __forceinline__ void reflect_two(const C* __restrict__ v, int j, int q, S* xa, S* xb) {
  const int lane = threadIdx.x & 31;
  C ra[RM], rb[RM];
  C da = 0, db = 0;
#pragma unroll
  for (int t = 0; t < RM; ++t) {
    const int i = j + lane + 32 * t;
    const bool in = i < q;
    ra[t] = in ? (C)xa[i] : C(0);
    rb[t] = (in && xb) ? (C)xb[i] : C(0);
  }
#pragma unroll
  for (int t = 0; t < RM; ++t) {
    const int i = j + lane + 32 * t;
    const C vi = (i < q) ? v[i] : C(0);
    da += ra[t] * vi;
    db += rb[t] * vi;
  }
  da = warp_sum(da);
  db = warp_sum(db);
#pragma unroll
  for (int t = 0; t < RM; ++t) {
    const int i = j + lane + 32 * t;
    if (i < q) {
      const C vi = v[i];
      xa[i] = (S)(ra[t] - C(2) * da * vi);
      if (xb) xb[i] = (S)(rb[t] - C(2) * db * vi);
    }
  }
}

template <typename C, typename S, int RM>
__global__ void __launch_bounds__(1024) qr_house_kernel(int q, int p, S* __restrict__ X, S* __restrict__ Q,
                                                        S* __restrict__ R) {
  __shared__ C red[32];
  __shared__ C diag[1024];  // r <= 1024
  __shared__ C v[32 * RM];  // current reflector
  const int r = min(q, p);
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < r; ++j) {
    S* xj = X + (size_t)j * q;
    C ss = 0;
    for (int i = threadIdx.x; i < q; i += blockDim.x) {
      const C t = (i >= j) ? (C)xj[i] : C(0);
      v[i] = t;
      ss += t * t;
    }
    ss = block_sum(ss, red);
    const C x0 = v[j];
    const C nrm = sqrt(ss);
    const C alpha = (x0 >= C(0)) ? -nrm : nrm;
    const C v0 = x0 - alpha;
    const C vn2 = ss - x0 * x0 + v0 * v0;
    const bool zero = !(vn2 > C(0));
    const C inv = zero ? C(0) : C(1) / sqrt(vn2);
    __syncthreads();
    for (int i = j + threadIdx.x; i < q; i += blockDim.x) {
      const C t = (i == j ? v0 : v[i]) * inv;
      v[i] = t;
      xj[i] = (S)t;
    }
    if (threadIdx.x == 0) diag[j] = zero ? C(0) : alpha;
    __syncthreads();
    if (!zero) {
      for (int c = j + 1 + 2 * warp; c < p; c += 2 * nw)
        reflect_two<C, S, RM>(v, j, q, X + (size_t)c * q, (c + 1 < p) ? X + (size_t)(c + 1) * q : nullptr);
    }
    __syncthreads();
  }
  // R (r x p, col-major, ld r)
  for (long long e = threadIdx.x; e < (long long)r * p; e += blockDim.x) {
    const int i = (int)(e % r), c = (int)(e / r);
    R[(size_t)c * r + i] = (i < c) ? X[(size_t)c * q + i] : (i == c ? (S)diag[i] : S(0));
  }
  // Q = H_0 ... H_{r-1} [I_r; 0]
  for (long long e = threadIdx.x; e < (long long)q * r; e += blockDim.x) {
    const int i = (int)(e % q), c = (int)(e / q);
    Q[(size_t)c * q + i] = (i == c) ? S(1) : S(0);
  }
  __syncthreads();
  for (int j = r - 1; j >= 0; --j) {
    for (int i = threadIdx.x; i < q; i += blockDim.x) v[i] = (i >= j) ? (C)X[(size_t)j * q + i] : C(0);
    __syncthreads();
    for (int c = j + 2 * warp; c < r; c += 2 * nw)
      reflect_two<C, S, RM>(v, j, q, Q + (size_t)c * q, (c + 1 < r) ? Q + (size_t)(c + 1) * q : nullptr);
    __syncthreads();
  }
  // sign convention diag(R) >= 0
  const int lane = threadIdx.x & 31;
  for (int j = warp; j < r; j += nw) {
    if (diag[j] < C(0)) {
      for (int c = j + lane; c < p; c += 32) R[(size_t)c * r + j] = -R[(size_t)c * r + j];
      for (int i = lane; i < q; i += 32) Q[(size_t)j * q + i] = -Q[(size_t)j * q + i];
    }
  }
}

// ---------------------------------------------------------------------------
// Householder QR on a thread-block cluster of JQ CTAs: CTA k holds rows
// [k rb, (k+1) rb) of X and of Q in shared memory, so the matrix never leaves
// the SMs. Step j: the CTAs exchange their partial |x_j|^2 and the pivot
// (all-to-all through distributed shared memory, cluster barrier), each forms
// the same reflector, exchanges its partial dot products v^T X (second
// barrier) and updates its own rows. Q = H_0 ... H_{r-1} [I; 0] is then formed
// backwards with one exchange per reflector (buffers alternate by step parity,
// so a CTA that runs ahead never overwrites sums another one still reads).
// Same contract and sign convention (diag R >= 0) as qr_house_kernel.
// ---------------------------------------------------------------------------
constexpr int JQ = 8;

template <typename C>
__global__ void __cluster_dims__(JQ, 1, 1) __launch_bounds__(256)
    qr_cluster_kernel(int q, int p, const C* __restrict__ Xg, C* __restrict__ Qg, C* __restrict__ Rg) {
  cg::cluster_group cl = cg::this_cluster();
  const int k = (int)cl.block_rank();
  const int r = min(q, p);
  const int rb = (q + JQ - 1) / JQ;
  const int ld = rb | 1;  // odd column stride: threads reading one row of consecutive columns hit distinct banks
  const int r0 = k * rb, nr = max(0, min(rb, q - r0));  // my rows: r0 .. r0 + nr - 1
  extern __shared__ __align__(16) unsigned char qcs[];
  C* X = (C*)qcs;                          // [p][ld] my rows of X, column-major
  C* Qm = X + (size_t)p * ld;              // [r][ld] my rows of Q, column-major
  C* xw = Qm + (size_t)r * ld;             // [2][JQ][p] exchanged partial dot products
  C* wsum = xw + 2 * (size_t)JQ * p;       // [p] summed dot products of the current step
  C* xs = wsum + p;                        // [JQ] partial squared norms
  C* diag = xs + JQ;                       // [r] alpha of every reflector
  C* x0s = diag + r;                       // [1] pivot of the current step
  __shared__ C red[32];
  for (long long e = threadIdx.x; e < (long long)p * rb; e += blockDim.x) {
    const int i = (int)(e % rb), c = (int)(e / rb);
    X[(size_t)c * ld + i] = i < nr ? Xg[(size_t)c * q + r0 + i] : C(0);
  }
  cl.sync();
  for (int j = 0; j < r; ++j) {
    C* xj = X + (size_t)j * ld;
    const int i0 = max(0, min(nr, j - r0));  // my first row at or below the diagonal
    // (a) partial |x_j[j:]|^2 and the pivot x_jj, to every CTA
    C ss = 0;
    for (int i = i0 + (int)threadIdx.x; i < nr; i += blockDim.x) ss += xj[i] * xj[i];
    ss = block_sum(ss, red);
    if (threadIdx.x < JQ) {
      C* dst = cl.map_shared_rank(xs, (unsigned)threadIdx.x);
      dst[k] = ss;
      if (j >= r0 && j < r0 + nr) *cl.map_shared_rank(x0s, (unsigned)threadIdx.x) = xj[j - r0];
    }
    cl.sync();
    C tot = 0;
    for (int t = 0; t < JQ; ++t) tot += xs[t];
    const C x0 = *x0s;
    const C nrm = sqrt(tot);
    const C alpha = (x0 >= C(0)) ? -nrm : nrm;
    const C v0 = x0 - alpha;
    const C vn2 = tot - x0 * x0 + v0 * v0;
    const bool zero = !(vn2 > C(0));
    const C inv = zero ? C(0) : C(1) / sqrt(vn2);
    if (threadIdx.x == 0) diag[j] = zero ? C(0) : alpha;
    for (int i = i0 + (int)threadIdx.x; i < nr; i += blockDim.x)
      xj[i] = (r0 + i == j ? v0 : xj[i]) * inv;  // the reflector v (unit norm) below the diagonal
    __syncthreads();
    // (b) partial w_c = v^T x_c for c > j (one thread per column), to every CTA
    C* wbuf = xw + (size_t)(j & 1) * JQ * p;
    for (int c = j + 1 + (int)threadIdx.x; c < p; c += blockDim.x) {
      const C* xc = X + (size_t)c * ld;
      C d = 0;
      for (int i = i0; i < nr; ++i) d += xj[i] * xc[i];
#pragma unroll
      for (int t = 0; t < JQ; ++t) cl.map_shared_rank(wbuf, (unsigned)t)[k * p + c] = d;
    }
    cl.sync();
    // (c) x_c -= 2 v w_c on my rows
    for (int c = j + 1 + (int)threadIdx.x; c < p; c += blockDim.x) {
      C w = 0;
      for (int t = 0; t < JQ; ++t) w += wbuf[t * p + c];
      wsum[c] = C(2) * w;
    }
    __syncthreads();
    if (!zero && nr > i0)
      for (long long e = threadIdx.x; e < (long long)(p - j - 1) * (nr - i0); e += blockDim.x) {
        const int i = i0 + (int)(e % (nr - i0)), c = j + 1 + (int)(e / (nr - i0));
        X[(size_t)c * ld + i] -= xj[i] * wsum[c];
      }
    __syncthreads();
  }
  // Q = H_0 ... H_{r-1} [I_r; 0], my rows
  for (long long e = threadIdx.x; e < (long long)r * rb; e += blockDim.x) {
    const int i = (int)(e % rb), c = (int)(e / rb);
    Qm[(size_t)c * ld + i] = (r0 + i == c) ? C(1) : C(0);
  }
  cl.sync();  // every CTA has read the last step's sums before the buffers are reused below
  for (int j = r - 1; j >= 0; --j) {
    const C* vj = X + (size_t)j * ld;
    const int i0 = max(0, min(nr, j - r0));
    C* tbuf = xw + (size_t)(j & 1) * JQ * p;
    for (int c = j + (int)threadIdx.x; c < r; c += blockDim.x) {
      const C* qc = Qm + (size_t)c * ld;
      C d = 0;
      for (int i = i0; i < nr; ++i) d += vj[i] * qc[i];
#pragma unroll
      for (int t = 0; t < JQ; ++t) cl.map_shared_rank(tbuf, (unsigned)t)[k * p + c] = d;
    }
    cl.sync();
    for (int c = j + (int)threadIdx.x; c < r; c += blockDim.x) {
      C t = 0;
      for (int u = 0; u < JQ; ++u) t += tbuf[u * p + c];
      wsum[c] = C(2) * t;
    }
    __syncthreads();
    if (diag[j] != C(0) && nr > i0)
      for (long long e = threadIdx.x; e < (long long)(r - j) * (nr - i0); e += blockDim.x) {
        const int i = i0 + (int)(e % (nr - i0)), c = j + (int)(e / (nr - i0));
        Qm[(size_t)c * ld + i] -= vj[i] * wsum[c];
      }
    __syncthreads();
  }
  // outputs with diag(R) >= 0: row i of R and column i of Q change sign where alpha_i < 0
  for (long long e = threadIdx.x; e < (long long)r * nr; e += blockDim.x) {
    const int i = (int)(e % nr), c = (int)(e / nr);
    Qg[(size_t)c * q + r0 + i] = diag[c] < C(0) ? -Qm[(size_t)c * ld + i] : Qm[(size_t)c * ld + i];
  }
  for (long long e = threadIdx.x; e < (long long)p * nr; e += blockDim.x) {
    const int i = (int)(e % nr), c = (int)(e / nr);
    const int gi = r0 + i;
    if (gi >= r) continue;
    const C val = gi < c ? X[(size_t)c * ld + i] : (gi == c ? diag[gi] : C(0));
    Rg[(size_t)c * r + gi] = diag[gi] < C(0) ? -val : val;
  }
  cl.sync();  // no CTA leaves while another may still write into its shared memory
}

// Blocked variant: panels of QB columns, compact-WY updates.
//
// Per panel every CTA gathers the panel's rows (>= j0) from all CTAs into
// registers (RPT rows x QB columns per thread) and factors it redundantly, so
// all CTAs hold identical reflectors. One block reduction per column gives the
// column's Gram row g_c = a_j^T a_c (rows >= j), from which the reflector
// (alpha, unit v) and v^T a_c = (g_c - alpha a_c[j]) / ||v|| follow; the same
// reduction carries v_i^T v_{j-1} (i < j-1), the strictly upper part of
// G = V^T V. The product of the panel's reflectors (tau = 2, unit v) is
// I - V T V^T with T^{-1} = I/2 + striu(G) (the UT transform of Joffrain,
// Low, Quintana-Orti, van de Geijn and Puglisi, ACM TOMS 32 (2006)), so T is
// never formed: the trailing update A -= V T^T (V^T A) solves a triangular
// system per column instead. V^T A is a sum over the CTAs' rows: each CTA
// forms its partial, and after one cluster barrier pulls those of all CTAs.
// Q is formed backwards panel by panel with Q -= V T (V^T Q). A null column
// gives v = 0, which leaves everything unchanged. Two cluster barriers per
// panel in the factorisation, one in the formation of Q.
constexpr int QB = 16;

// Element helpers of the blocked QR for float, double and df32 arithmetic.
// The df32 square root and reciprocal start from the FP32 result of the high
// word and take one Newton step in df32 arithmetic, which doubles the number
// of correct bits (Dekker, Numer. Math. 18 (1971); Karp and Markstein, ACM
// TOMS 23 (1997)): sqrt(x) = s + (x - s^2) / (2 s), 1/x = r + r (1 - x r).
__device__ __forceinline__ float qsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double qsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ df32 qsqrt(df32 x) {
  if (!(x.hi > 0.0f)) return df32(0.0f, 0.0f);
  const float s = sqrtf(x.hi);
  const df32 e = madd(df32(-s, 0.0f), df32(s, 0.0f), x);  // x - s^2
  return two_sum(s, e.hi * (0.5f / s));
}
// 1/sqrt(x): FP32 from the hardware estimate and one Newton step (r (3 - x r^2) / 2)
__device__ __forceinline__ float qrsqrt(float x) {
  const float r = rsqrtf(x);
  return r * fmaf(-0.5f * x * r, r, 1.5f);
}
__device__ __forceinline__ double qrsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float qrcp(float x) { return 1.0f / x; }
__device__ __forceinline__ double qrcp(double x) { return 1.0 / x; }
__device__ __forceinline__ df32 qrcp(df32 x) {
  const df32 r(1.0f / x.hi, 0.0f);
  const df32 e = madd(-x, r, df32(1.0f, 0.0f));  // 1 - x r
  return madd(r, e, r);
}
__device__ __forceinline__ df32 qrsqrt(df32 x) { return qrcp(qsqrt(x)); }
__device__ __forceinline__ bool qneg(float x) { return x < 0.0f; }
__device__ __forceinline__ bool qneg(double x) { return x < 0.0; }
__device__ __forceinline__ bool qneg(df32 x) { return x.hi < 0.0f; }  // a normalised pair has the sign of hi
__device__ __forceinline__ bool qpos(float x) { return x > 0.0f; }
__device__ __forceinline__ bool qpos(double x) { return x > 0.0; }
__device__ __forceinline__ bool qpos(df32 x) { return x.hi > 0.0f; }
template <typename C>
__device__ __forceinline__ C qshfl_xor(C v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}
template <>
__device__ __forceinline__ df32 qshfl_xor<df32>(df32 v, int m) {
  return df32(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}
template <typename C>
__device__ __forceinline__ C qshfl(C v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
template <>
__device__ __forceinline__ df32 qshfl<df32>(df32 v, int src) {
  return df32(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}

template <typename C>
__device__ __forceinline__ void ld16(const C* __restrict__ src, C (&v)[QB]) {
  if constexpr (std::is_same<C, float>::value) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int t = 0; t < QB / 4; ++t) {
      const float4 x = s4[t];
      v[4 * t] = x.x;
      v[4 * t + 1] = x.y;
      v[4 * t + 2] = x.z;
      v[4 * t + 3] = x.w;
    }
  } else if constexpr (std::is_same<C, double>::value) {
    const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int t = 0; t < QB / 2; ++t) {
      const double2 x = s2[t];
      v[2 * t] = x.x;
      v[2 * t + 1] = x.y;
    }
  } else {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int t = 0; t < QB / 2; ++t) {
      const float4 x = s4[t];
      v[2 * t] = df32(x.x, x.y);
      v[2 * t + 1] = df32(x.z, x.w);
    }
  }
}

template <typename C>
__device__ __forceinline__ void st16(C* __restrict__ dst, const C (&v)[QB]) {
  if constexpr (std::is_same<C, float>::value) {
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int t = 0; t < QB / 4; ++t) d4[t] = make_float4(v[4 * t], v[4 * t + 1], v[4 * t + 2], v[4 * t + 3]);
  } else if constexpr (std::is_same<C, double>::value) {
    double2* d2 = reinterpret_cast<double2*>(dst);
#pragma unroll
    for (int t = 0; t < QB / 2; ++t) d2[t] = make_double2(v[2 * t], v[2 * t + 1]);
  } else {
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int t = 0; t < QB / 2; ++t) d4[t] = make_float4(v[2 * t].hi, v[2 * t].lo, v[2 * t + 1].hi, v[2 * t + 1].lo);
  }
}

// Sum over the warp of 16 slots (reduce-scatter by halving: 8 + 4 + 2 + 1 + 1
// shuffles); lanes 2s and 2s + 1 return the sum of slot s.
template <typename C>
__device__ __forceinline__ C warp_reduce16(C (&v)[QB], int lane) {
#pragma unroll
  for (int h = QB / 2, m = 16; h >= 1; h >>= 1, m >>= 1) {
    const bool hi = (lane & m) != 0;
#pragma unroll
    for (int t = 0; t < h; ++t) {
      const C send = hi ? v[t] : v[t + h];
      const C keep = hi ? v[t + h] : v[t];
      v[t] = keep + qshfl_xor(send, m);
    }
  }
  return v[0] + qshfl_xor(v[0], 1);
}

__host__ __device__ constexpr size_t qr_al4(size_t n) { return (n + 3) & ~(size_t)3; }

// Shared memory layout (elements of C, every region a multiple of 4 long).
struct QrbLayout {
  size_t X, U, P, Qm, Vmy, Wl, Ys, Gm, Gt, diag, red, xrow, total;
  __host__ __device__ QrbLayout(int q, int p) {
    const size_t rb = (q + JQ - 1) / JQ, ld = rb | 1, r = q < p ? q : p, npan = (r + QB - 1) / QB;
    X = 0;
    U = qr_al4((size_t)p * ld);
    P = U;                                   // factorisation: V of the panel, row-major [q - j0][QB]
    Qm = U;                                  // formation of Q: my rows of Q [r][ld], then my rows of V [rb][QB]
    Vmy = U + qr_al4(r * ld);
    const size_t usz = (size_t)q * QB > qr_al4(r * ld) + rb * QB ? (size_t)q * QB : qr_al4(r * ld) + rb * QB;
    Wl = U + qr_al4(usz);                    // [2][p][QB] my partial V^T A (by panel parity)
    Ys = Wl + 2 * (size_t)p * QB;            // [p][QB] T^T W or T W
    Gm = Ys + (size_t)p * QB;                // [npan][QB][QB] G = V^T V per panel (column-major, strict upper)
    Gt = Gm + npan * QB * QB;                // [QB][QB] G of the current panel, row-major
    diag = Gt + QB * QB;                     // [r]
    red = diag + qr_al4(r);                  // [2][8][QB] warp partials (by column parity)
    xrow = red + 2 * 8 * QB;                 // [2][QB] row j0 + j of the panel
    total = xrow + 2 * QB;
  }
};

template <typename S, typename C, int RPT>
__global__ void __cluster_dims__(JQ, 1, 1) __launch_bounds__(256)
    qr_cluster_blocked_kernel(int q, int p, const S* __restrict__ Xg, S* __restrict__ Qg, S* __restrict__ Rg) {
  cg::cluster_group cl = cg::this_cluster();
  const int k = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = min(q, p);
  const int rb = (q + JQ - 1) / JQ;
  const int ld = rb | 1;
  const int r0 = k * rb, nr = max(0, min(rb, q - r0));
  const int npan = (r + QB - 1) / QB;
  extern __shared__ __align__(16) unsigned char qbs[];
  const QrbLayout Lay(q, p);
  C* sm = (C*)qbs;
  C* X = sm + Lay.X;
  C* P = sm + Lay.P;
  C* Wl = sm + Lay.Wl;
  C* Ys = sm + Lay.Ys;
  C* Gm = sm + Lay.Gm;
  C* Gt = sm + Lay.Gt;
  C* diag = sm + Lay.diag;
  C* red = sm + Lay.red;
  C* xrow = sm + Lay.xrow;
  for (int i = tid & 63; i < rb; i += 64)  // 64 rows x 4 column groups, loads unrolled for overlap
#pragma unroll 4
    for (int c = tid >> 6; c < p; c += 4) X[(size_t)c * ld + i] = i < nr ? C(Xg[(size_t)c * q + r0 + i]) : C(0);
  for (int t = tid; t < npan * QB * QB; t += blockDim.x) Gm[t] = C(0);
  for (int pn = 0; pn < npan; ++pn) {
    for (int t = tid; t < QB * QB; t += blockDim.x) Gt[t] = C(0);  // read after the barriers below
    const int j0 = pn * QB, w = min(QB, r - j0), c1 = j0 + w;
    C* G = Gm + (size_t)pn * QB * QB;
    C* W = Wl + (size_t)(pn & 1) * p * QB;
    cl.sync();  // the panel's columns are final in every CTA
    C a[RPT][QB];
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      const int g = j0 + tid + 256 * s;
      if (g < q) {
        const int owner = g / rb;
        const C* src = cl.map_shared_rank(X, (unsigned)owner) + (g - owner * rb);
#pragma unroll
        for (int c = 0; c < QB; ++c) a[s][c] = c < w ? src[(size_t)(j0 + c) * ld] : C(0);
      } else {
#pragma unroll
        for (int c = 0; c < QB; ++c) a[s][c] = C(0);
      }
    }
#pragma unroll
    for (int jj = 0; jj <= QB; ++jj) {
      if (jj > w) break;
      const int buf = jj & 1;
      C rv[QB];
#pragma unroll
      for (int c = 0; c < QB; ++c) rv[c] = C(0);
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        const int g = j0 + tid + 256 * s;
        if (g < q) {
          if (jj < w && g >= j0 + jj) {
#pragma unroll
            for (int c = jj; c < QB; ++c) rv[c] = madd(a[s][jj], a[s][c], rv[c]);
          }
          if (jj >= 2 && g >= j0 + jj - 1) {
#pragma unroll
            for (int ii = 0; ii < jj - 1; ++ii) rv[ii] = madd(a[s][ii], a[s][jj - 1], rv[ii]);
          }
        }
      }
      if (jj < w && tid == jj) {
#pragma unroll
        for (int c = jj; c < QB; ++c) xrow[buf * QB + c] = a[0][c];
      }
      const C sv = warp_reduce16(rv, lane);
      if (!(lane & 1)) red[(buf * 8 + warp) * QB + (lane >> 1)] = sv;
      __syncthreads();
      C tot[QB];
      {  // lane (w8, grp) loads slots 4 grp .. 4 grp + 3 of warp w8; sum over w8, then broadcast
        const int w8 = lane & 7, grp = lane >> 3;
        const C* src = red + (buf * 8 + w8) * QB + grp * 4;
        C v4[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) v4[t] = src[t];
#pragma unroll
        for (int m = 1; m < 8; m <<= 1)
#pragma unroll
          for (int t = 0; t < 4; ++t) v4[t] = v4[t] + qshfl_xor(v4[t], m);
#pragma unroll
        for (int c = 0; c < QB; ++c) tot[c] = qshfl(v4[c & 3], (c >> 2) * 8);
      }
      if (jj >= 2 && tid == 0) {
#pragma unroll
        for (int ii = 0; ii < jj - 1; ++ii) {
          G[(jj - 1) * QB + ii] = tot[ii];
          Gt[ii * QB + (jj - 1)] = tot[ii];
        }
      }
      if (jj == w) break;
      const C ss = tot[jj];
      const C x0 = xrow[buf * QB + jj];
      const C nrm = qsqrt(ss);
      const C alpha = qneg(x0) ? nrm : -nrm;
      const C v0 = x0 - alpha;
      const C vn2 = madd(v0, v0, madd(-x0, x0, ss));
      const bool zero = !qpos(vn2);
      const C inv = zero ? C(0) : qrsqrt(vn2);
      if (tid == 0) diag[j0 + jj] = zero ? C(0) : alpha;
      C dv[QB];
#pragma unroll
      for (int c = jj + 1; c < QB; ++c) dv[c] = C(2) * (madd(-alpha, xrow[buf * QB + c], tot[c]) * inv);
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        const int g = j0 + tid + 256 * s;
        if (g < q && g >= j0 + jj) {
          const C vi = (g == j0 + jj ? v0 : a[s][jj]) * inv;
          a[s][jj] = vi;
#pragma unroll
          for (int c = jj + 1; c < QB; ++c) a[s][c] = madd(-dv[c], vi, a[s][c]);
        }
      }
    }
    // V (zero above its diagonal) for the partial products and the trailing update
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      const int g = j0 + tid + 256 * s;
      if (g < q) {
        C t[QB];
#pragma unroll
        for (int c = 0; c < QB; ++c) t[c] = (c < w && g - j0 >= c) ? a[s][c] : C(0);
        st16(P + (size_t)(g - j0) * QB, t);
      }
    }
    __syncthreads();
    const int i0 = max(0, j0 - r0);
    for (int c = c1 + tid; c < p; c += blockDim.x) {  // my partial W = V^T A, trailing columns
      C acc[QB];
#pragma unroll
      for (int jj = 0; jj < QB; ++jj) acc[jj] = C(0);
      const C* xc = X + (size_t)c * ld;
#pragma unroll 4
      for (int i = i0; i < nr; ++i) {
        C v[QB];
        ld16(P + (size_t)(r0 + i - j0) * QB, v);
        const C x = xc[i];
#pragma unroll
        for (int jj = 0; jj < QB; ++jj) acc[jj] = madd(v[jj], x, acc[jj]);
      }
      st16(W + (size_t)c * QB, acc);
    }
    cl.sync();  // every CTA has gathered the panel and formed its partial W
#pragma unroll
    for (int s = 0; s < RPT; ++s) {  // my rows of the factored panel (R above, v below the diagonal)
      const int g = j0 + tid + 256 * s;
      if (g < q && g >= r0 && g < r0 + nr) {
#pragma unroll
        for (int c = 0; c < QB; ++c)
          if (c < w) X[(size_t)(j0 + c) * ld + (g - r0)] = a[s][c];
      }
    }
    for (int c = c1 + tid; c < p; c += blockDim.x) {  // W summed over the CTAs; y = T^T w
      C wv[QB];
#pragma unroll
      for (int jj = 0; jj < QB; ++jj) wv[jj] = C(0);
#pragma unroll(sizeof(C) == 4 ? 4 : 2)
      for (int t = 0; t < JQ; ++t) {  // several CTAs' partials in flight at once
        C x[QB];
        ld16(cl.map_shared_rank(W, (unsigned)t) + (size_t)c * QB, x);
#pragma unroll
        for (int jj = 0; jj < QB; ++jj) wv[jj] = wv[jj] + x[jj];
      }
      // (I/2 + striu(G)^T) y = w, forward substitution by rows of G (Gt row-major)
#pragma unroll
      for (int b = 0; b < QB; ++b) {
        wv[b] = C(2) * wv[b];
        C g[QB];
        ld16(Gt + b * QB, g);
#pragma unroll
        for (int a2 = b + 1; a2 < QB; ++a2) wv[a2] = madd(-g[a2], wv[b], wv[a2]);
      }
      st16(Ys + (size_t)c * QB, wv);
    }
    __syncthreads();
    for (int i = i0 + (tid & 63); i < nr; i += 64) {  // A(my rows >= j0, c >= c1) -= V y
      C v[QB];
      ld16(P + (size_t)(r0 + i - j0) * QB, v);
      for (int c = c1 + (tid >> 6); c < p; c += 4) {
        C y[QB];
        ld16(Ys + (size_t)c * QB, y);
        C x = X[(size_t)c * ld + i];
#pragma unroll
        for (int jj = 0; jj < QB; ++jj) x = madd(-v[jj], y[jj], x);
        X[(size_t)c * ld + i] = x;
      }
    }
    __syncthreads();
  }
  cl.sync();  // no CTA reads another's partial W of the last panel any more
  C* Qm = sm + Lay.Qm;
  C* Vmy = sm + Lay.Vmy;
  if (Qg != nullptr) {  // R-only calls (Qg == nullptr, uniform over the cluster) skip the formation of Q
  for (int i = tid & 63; i < rb; i += 64)
    for (int c = tid >> 6; c < r; c += 4) Qm[(size_t)c * ld + i] = (r0 + i == c) ? C(1) : C(0);
  for (int pn = npan - 1; pn >= 0; --pn) {
    const int j0 = pn * QB, w = min(QB, r - j0);
    const C* G = Gm + (size_t)pn * QB * QB;
    C* W = Wl + (size_t)(pn & 1) * p * QB;
    const int i0 = max(0, j0 - r0);
    for (int i = tid; i < nr; i += blockDim.x) {  // my rows of V (zero above its diagonal)
      const int g = r0 + i;
      C t[QB];
#pragma unroll
      for (int jj = 0; jj < QB; ++jj) t[jj] = (jj < w && g >= j0 + jj) ? X[(size_t)(j0 + jj) * ld + i] : C(0);
      st16(Vmy + (size_t)i * QB, t);
    }
    __syncthreads();
    for (int c = j0 + tid; c < r; c += blockDim.x) {  // my partial W = V^T Q
      C acc[QB];
#pragma unroll
      for (int jj = 0; jj < QB; ++jj) acc[jj] = C(0);
      const C* qc = Qm + (size_t)c * ld;
#pragma unroll 4
      for (int i = i0; i < nr; ++i) {
        C v[QB];
        ld16(Vmy + (size_t)i * QB, v);
        const C x = qc[i];
#pragma unroll
        for (int jj = 0; jj < QB; ++jj) acc[jj] = madd(v[jj], x, acc[jj]);
      }
      st16(W + (size_t)c * QB, acc);
    }
    cl.sync();
    for (int c = j0 + tid; c < r; c += blockDim.x) {  // y = T w: (I/2 + striu(G)) y = w, back substitution
      C wv[QB];
#pragma unroll
      for (int jj = 0; jj < QB; ++jj) wv[jj] = C(0);
#pragma unroll(sizeof(C) == 4 ? 4 : 2)
      for (int t = 0; t < JQ; ++t) {  // several CTAs' partials in flight at once
        C x[QB];
        ld16(cl.map_shared_rank(W, (unsigned)t) + (size_t)c * QB, x);
#pragma unroll
        for (int jj = 0; jj < QB; ++jj) wv[jj] = wv[jj] + x[jj];
      }
      // (I/2 + striu(G)) y = w, back substitution by columns of G
#pragma unroll
      for (int b = QB - 1; b >= 0; --b) {
        wv[b] = C(2) * wv[b];
        C g[QB];
        ld16(G + b * QB, g);
#pragma unroll
        for (int a2 = 0; a2 < b; ++a2) wv[a2] = madd(-g[a2], wv[b], wv[a2]);
      }
      st16(Ys + (size_t)c * QB, wv);
    }
    __syncthreads();
    for (int i = i0 + (tid & 63); i < nr; i += 64) {
      C v[QB];
      ld16(Vmy + (size_t)i * QB, v);
      for (int c = j0 + (tid >> 6); c < r; c += 4) {
        C y[QB];
        ld16(Ys + (size_t)c * QB, y);
        C x = Qm[(size_t)c * ld + i];
#pragma unroll
        for (int jj = 0; jj < QB; ++jj) x = madd(-v[jj], y[jj], x);
        Qm[(size_t)c * ld + i] = x;
      }
    }
    __syncthreads();
  }
  for (int i = tid & 63; i < nr; i += 64)
#pragma unroll 4
    for (int c = tid >> 6; c < r; c += 4)
      Qg[(size_t)c * q + r0 + i] = (S)(qneg(diag[c]) ? -Qm[(size_t)c * ld + i] : Qm[(size_t)c * ld + i]);
  }
  for (int i = tid & 63; i < nr; i += 64) {
    const int gi = r0 + i;
    if (gi >= r) continue;
    const bool flip = qneg(diag[gi]);
#pragma unroll 4
    for (int c = tid >> 6; c < p; c += 4) {
      const C val = gi < c ? X[(size_t)c * ld + i] : (gi == c ? diag[gi] : C(0));
      Rg[(size_t)c * r + gi] = (S)(flip ? -val : val);
    }
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

template <typename C>
size_t qr_cluster_blocked_smem(int q, int p) {
  return QrbLayout(q, p).total * sizeof(C) + 16;
}

template <typename C>
size_t qr_cluster_smem(int q, int p) {
  const size_t rb = (q + JQ - 1) / JQ, ld = rb | 1, r = std::min(q, p);
  return ((size_t)p * ld + r * ld + 2 * (size_t)JQ * p + p + JQ + r + 1) * sizeof(C) + 16;
}

template <typename C, typename S>
cudaError_t qr_householder(int q, int p, S* X, S* Q, S* R, cudaStream_t st) {
  if (q <= 0 || p <= 0) return cudaSuccess;
  if (min(q, p) > 1024 || q > 1024) return cudaErrorInvalidValue;
  if constexpr (std::is_same<C, S>::value) {  // rows spread over a cluster when the matrix is large enough
    const size_t bsm = qr_cluster_blocked_smem<C>(q, p);
    if (Q == nullptr && !(q >= 128 && p >= 16 && bsm <= 220 * 1024)) return cudaErrorInvalidValue;
    if (q >= 128 && p >= 16 && bsm <= 220 * 1024) {
      auto launch = [&](auto kern) {
        cudaError_t e = ensure_smem((const void*)kern, bsm);
        if (e != cudaSuccess) return e;
        ++tl_launches;
        kern<<<JQ, 256, bsm, st>>>(q, p, X, Q, R);
        return cudaGetLastError();
      };
      if (q <= 256) return launch(qr_cluster_blocked_kernel<C, C, 1>);
      if (q <= 512) return launch(qr_cluster_blocked_kernel<C, C, 2>);
      return launch(qr_cluster_blocked_kernel<C, C, 4>);
    }
    const size_t csm = qr_cluster_smem<C>(q, p);
    if (q >= 128 && p >= 16 && csm <= 200 * 1024) {
      if (csm > 48 * 1024) {
        cudaError_t e =
            ensure_smem((const void*)qr_cluster_kernel<C>, csm);
        if (e != cudaSuccess) return e;
      }
      ++tl_launches;
      qr_cluster_kernel<C><<<JQ, 256, csm, st>>>(q, p, X, Q, R);
      return cudaGetLastError();
    }
  }
  if (Q == nullptr) return cudaErrorInvalidValue;  // only the cluster kernel has an R-only mode
  ++tl_launches;
  if (q <= 128) qr_house_kernel<C, S, 4><<<1, 1024, 0, st>>>(q, p, X, Q, R);
  else if (q <= 256) qr_house_kernel<C, S, 8><<<1, 1024, 0, st>>>(q, p, X, Q, R);
  else if (q <= 512) qr_house_kernel<C, S, 16><<<1, 1024, 0, st>>>(q, p, X, Q, R);
  else if (q <= 1024) qr_house_kernel<C, S, 32><<<1, 1024, 0, st>>>(q, p, X, Q, R);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}
template cudaError_t qr_householder<double, double>(int, int, double*, double*, double*, cudaStream_t);

cudaError_t qr_householder_df32(int q, int p, double* X, double* Q, double* R, cudaStream_t st) {
  if (q <= 0 || p <= 0) return cudaSuccess;
  const size_t bsm = qr_cluster_blocked_smem<df32>(q, p);
  if (q < 128 || p < 16 || q > 1024 || bsm > 220 * 1024) return qr_householder<double, double>(q, p, X, Q, R, st);
  auto launch = [&](auto kern) {
    cudaError_t e = ensure_smem((const void*)kern, bsm);
    if (e != cudaSuccess) return e;
    ++tl_launches;
    kern<<<JQ, 256, bsm, st>>>(q, p, X, Q, R);
    return cudaGetLastError();
  };
  if (q <= 256) return launch(qr_cluster_blocked_kernel<double, df32, 1>);
  if (q <= 512) return launch(qr_cluster_blocked_kernel<double, df32, 2>);
  return launch(qr_cluster_blocked_kernel<double, df32, 4>);
}
template cudaError_t qr_householder<float, float>(int, int, float*, float*, float*, cudaStream_t);

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

// 1/sqrt(x) for x in [1, 2]: the hardware estimate refined by one Newton step
// r <- r + r (1 - x r^2) / 2, so that cs^2 + sn^2 = cs^2 (1 + t^2) is 1 to the
// FP32 rounding. An estimate left unrefined makes every rotation a rotation
// times sqrt(cs^2 + sn^2), and the accumulated right factor drifts away from
// orthonormal over the thousands of rotations of a decomposition.
__device__ __forceinline__ float rot_rsqrt(float x) {
  const float r = rsqrtf(x);
  return fmaf(0.5f * r, fmaf(-x * r, r, 1.f), r);
}

// Jacobi rotation (c, s) that zeroes the (i, j) entry of the 2x2 Gram block
// [[a, g], [g, b]] (Rutishauser's formulas). In FP32 the fast division serves
// for the angle: any rotation this close to the exact one still drives the
// pair towards orthogonality, and convergence is decided on the recomputed
// Gram entries, not on these values.
__device__ __forceinline__ void rotation_params(float a, float b, float g, float& cs, float& sn) {
  const float zeta = __fdividef(b - a, 2.f * g);
  const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  cs = rot_rsqrt(1.f + t * t);
  sn = cs * t;
}
__device__ __forceinline__ void rotation_params(double a, double b, double g, double& cs, double& sn) {
  const double zeta = (b - a) / (2.0 * g);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  cs = 1.0 / sqrt(1.0 + t * t);
  sn = cs * t;
}

template <typename C, typename S, int NPW>
__global__ void __launch_bounds__(1024) jacobi_kernel(int q, int p, S* __restrict__ Wg, S* __restrict__ Vg,
                                                      int max_sweeps, double tol, uint32_t* errw,
                                                      S* __restrict__ Uo, S* __restrict__ So,
                                                      S* __restrict__ Vo, int in_smem) {
  const bool want_v = Vo != nullptr;  // the right rotations are accumulated only when asked for
  extern __shared__ __align__(16) unsigned char jsm[];
  __shared__ int rotated;
  __shared__ C nrm[1024];
  __shared__ int rank_[1024];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  S* W = Wg;
  S* V = Vg;
  if (in_smem) {  // the whole working set (q x p columns and p x p rotations) lives in shared memory
    W = (S*)jsm;
    V = W + (size_t)q * p;
    for (long long e = threadIdx.x; e < (long long)q * p; e += blockDim.x) W[e] = Wg[e];
  }
  if (want_v)
    for (long long e = threadIdx.x; e < (long long)p * p; e += blockDim.x) {
      int i = (int)(e % p), c = (int)(e / p);
      V[e] = (i == c) ? S(1) : S(0);
    }
  const int P = p + (p & 1);
  const C ctol2 = (C)(tol * tol);
  int sweep = 0;
  bool done = (p < 2);
  __syncthreads();
  while (!done && sweep < max_sweeps) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < P - 1; ++round) {
      // this warp's NPW pairs of the round, processed together so that their
      // load / shuffle-reduction / rotation latencies overlap
      int pi[NPW], pj[NPW];
      bool act[NPW];
#pragma unroll
      for (int t = 0; t < NPW; ++t) {
        const int k = warp + t * nw;
        int i = p, j = p;
        if (k < P / 2) rr_pair(round, k, P, i, j);
        act[t] = (i < p && j < p);
        if (i > j) { int x = i; i = j; j = x; }
        pi[t] = act[t] ? i : 0;
        pj[t] = act[t] ? j : 0;
      }
      C a[NPW], b[NPW], g[NPW];
#pragma unroll
      for (int t = 0; t < NPW; ++t) a[t] = b[t] = g[t] = C(0);
      for (int r = lane; r < q; r += 32) {
#pragma unroll
        for (int t = 0; t < NPW; ++t) {
          const C x = (C)W[(size_t)pi[t] * q + r], y = (C)W[(size_t)pj[t] * q + r];
          a[t] += x * x;
          b[t] += y * y;
          g[t] += x * y;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int t = 0; t < NPW; ++t) {
          a[t] += __shfl_xor_sync(0xffffffffu, a[t], o);
          b[t] += __shfl_xor_sync(0xffffffffu, b[t], o);
          g[t] += __shfl_xor_sync(0xffffffffu, g[t], o);
        }
      }
      C cs[NPW], sn[NPW];
      bool rot[NPW];
      bool any = false;
#pragma unroll
      for (int t = 0; t < NPW; ++t) {
        // all in the rotation type C: FP64 arithmetic costs ~56x FP32 on this GPU
        rot[t] = act[t] && a[t] > C(0) && b[t] > C(0) && g[t] * g[t] > ctol2 * a[t] * b[t];
        cs[t] = C(1);
        sn[t] = C(0);
        if (rot[t]) {
          rotation_params(a[t], b[t], g[t], cs[t], sn[t]);
          any = true;
        }
      }
      if (any) {
        for (int r = lane; r < q; r += 32) {
#pragma unroll
          for (int t = 0; t < NPW; ++t) {
            if (!rot[t]) continue;
            S* wi = W + (size_t)pi[t] * q;
            S* wj = W + (size_t)pj[t] * q;
            const C x = (C)wi[r], y = (C)wj[r];
            wi[r] = (S)(cs[t] * x - sn[t] * y);
            wj[r] = (S)(sn[t] * x + cs[t] * y);
          }
        }
        for (int r = lane; want_v && r < p; r += 32) {
#pragma unroll
          for (int t = 0; t < NPW; ++t) {
            if (!rot[t]) continue;
            S* vi = V + (size_t)pi[t] * p;
            S* vj = V + (size_t)pj[t] * p;
            const C x = (C)vi[r], y = (C)vj[r];
            vi[r] = (S)(cs[t] * x - sn[t] * y);
            vj[r] = (S)(sn[t] * x + cs[t] * y);
          }
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
  if (threadIdx.x == 0 && errw) atomicMax((int*)errw + 1, sweep);  // diagnostics: Jacobi sweeps used
  // singular values = column norms, sorted descending, ties by index
  for (int c = warp; c < p; c += nw) {
    const S* wc = W + (size_t)c * q;
    C s = 0;
    for (int r = lane; r < q; r += 32) s += (C)wc[r] * (C)wc[r];
    s = warp_sum(s);
    if (lane == 0) nrm[c] = sqrt(s);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < p; c += blockDim.x) {
    int rk = 0;
    const C v = nrm[c];
    for (int d = 0; d < p; ++d) rk += (nrm[d] > v) || (nrm[d] == v && d < c);
    rank_[c] = rk;
    So[rk] = (S)v;
  }
  __syncthreads();
  for (int c = warp; c < p; c += nw) {
    const int rk = rank_[c];
    const C s = nrm[c];
    const C inv = s > C(0) ? C(1) / s : C(0);
    for (int r = lane; r < q; r += 32) Uo[(size_t)rk * q + r] = (S)((C)W[(size_t)c * q + r] * inv);
    if (want_v)
      for (int r = lane; r < p; r += 32) Vo[(size_t)rk * p + r] = V[(size_t)c * p + r];
  }
}

// ---------------------------------------------------------------------------
// One-sided Jacobi on a thread-block cluster of JC CTAs (JC SMs). The p columns
// (w part: q rows; v part: the accumulated rotations, p rows) are cut into
// 2 JC blocks of b columns that live in the CTAs' shared memory, two blocks per
// CTA. A sweep is a round-robin tournament of the blocks (circle method, 2 JC - 1
// super-rounds): in each super-round a CTA orthogonalises every pair of columns
// between its two blocks (b micro-rounds of b disjoint pairs, one warp per
// pair); in the first super-round it also orthogonalises the columns inside each
// of its blocks. Between super-rounds every CTA pulls its next two blocks from
// the CTAs that hold them (distributed shared memory, double-buffered), behind
// one cluster barrier. Every column meets every other once per sweep, as in the
// cyclic method; the sweep count and the rotation test are those of
// jacobi_kernel. All CTAs run the same number of barriers (the stop decision is
// a cluster-wide OR read by all), so no barrier waits on a CTA that has left.
// ---------------------------------------------------------------------------
constexpr int JC = 8;  // CTAs per cluster (portable size); 16 (opt-in) when 8 CTAs' shared memory is too small

template <typename C>
__device__ __forceinline__ bool jacobi_pair(C* __restrict__ xi, C* __restrict__ xj, int q, int rows, C tol2) {
  const int lane = threadIdx.x & 31;
  C a = 0, b = 0, g = 0;
  for (int r = lane; r < q; r += 32) {
    const C x = xi[r], y = xj[r];
    a += x * x;
    b += y * y;
    g += x * y;
  }
  a = warp_sum(a);
  b = warp_sum(b);
  g = warp_sum(g);
  if (!(a > C(0) && b > C(0) && g * g > tol2 * a * b)) return false;
  C cs, sn;
  rotation_params(a, b, g, cs, sn);
  for (int r = lane; r < rows; r += 32) {
    const C x = xi[r], y = xj[r];
    xi[r] = cs * x - sn * y;
    xj[r] = sn * x + cs * y;
  }
  return true;
}

// The angle of a rotation only steers convergence; its orthogonality comes
// from cs = 1/sqrt(1 + t^2), sn = cs t, which is computed accurately. So t may
// take approximate division and square root (the next sweep corrects a
// slightly wrong angle).
__device__ __forceinline__ void rotation_params_fast(float a, float b, float g, float& cs, float& sn) {
  const float zeta = __fdividef(b - a, 2.f * g);
  const float z2 = fmaf(zeta, zeta, 1.f);
  const float t = __fdividef(copysignf(1.f, zeta), fabsf(zeta) + z2 * rsqrtf(z2));
  cs = rot_rsqrt(fmaf(t, t, 1.f));
  sn = cs * t;
}
__device__ __forceinline__ void rotation_params_fast(double a, double b, double g, double& cs, double& sn) {
  rotation_params(a, b, g, cs, sn);
}

// A column pair with each lane's RPL entries held in registers (rows <= 32 RPL):
// one round of independent loads, the three dot products over the first q rows,
// and the rotated values stored without reloading.
template <typename C, int RPL>
__device__ __forceinline__ bool jacobi_pair_r(C* __restrict__ xi, C* __restrict__ xj, int q, int rows, C tol2) {
  const int lane = threadIdx.x & 31;
  C x[RPL], y[RPL];
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int r = lane + 32 * t;
    x[t] = r < rows ? xi[r] : C(0);
    y[t] = r < rows ? xj[r] : C(0);
  }
  C a = 0, b = 0, g = 0;
#pragma unroll
  for (int t = 0; t < RPL; ++t)
    if (lane + 32 * t < q) {
      a = madd(x[t], x[t], a);
      b = madd(y[t], y[t], b);
      g = madd(x[t], y[t], g);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {  // the three butterflies interleaved: 5 shuffle latencies, not 15
    const C sa = __shfl_xor_sync(0xffffffffu, a, o);
    const C sb = __shfl_xor_sync(0xffffffffu, b, o);
    const C sg = __shfl_xor_sync(0xffffffffu, g, o);
    a += sa;
    b += sb;
    g += sg;
  }
  if (!(a > C(0) && b > C(0) && g * g > tol2 * a * b)) return false;
  C cs, sn;
  rotation_params_fast(a, b, g, cs, sn);
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int r = lane + 32 * t;
    if (r < rows) {
      xi[r] = cs * x[t] - sn * y[t];
      xj[r] = sn * x[t] + cs * y[t];
    }
  }
  return true;
}

template <typename C, int RPL>
__device__ __forceinline__ bool jacobi_pair_any(C* __restrict__ xi, C* __restrict__ xj, int q, int rows, C tol2) {
  if constexpr (RPL > 0) return jacobi_pair_r<C, RPL>(xi, xj, q, rows, tol2);
  else return jacobi_pair<C>(xi, xj, q, rows, tol2);
}

template <typename C, int RPL, int NC>
__global__ void __launch_bounds__(RPL > 0 ? 640 : 1024)
    jacobi_cluster_kernel(int q, int p, int b, const C* __restrict__ Win, int max_sweeps, double tol, uint32_t* errw,
                          C* __restrict__ Uo, C* __restrict__ So, C* __restrict__ Vo) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int P = 2 * NC;
  const bool want_v = Vo != nullptr;
  const int rows = q + (want_v ? p : 0);  // a column: its w part, then its v part
  constexpr int V16 = 16 / (int)sizeof(C);
  const int ld = (rows + V16 - 1) / V16 * V16;            // column stride: every column 16-byte aligned
  extern __shared__ __align__(16) unsigned char jcs[];
  C* buf = (C*)jcs;                                       // [2 buffers][2 slots][b][ld]
  int* ids = (int*)(buf + (size_t)4 * b * ld);            // [2 buffers][2 slots][b] global column or -1
  C* nrm = (C*)(ids + 4 * b + 4);                         // [2 slots][b] final column norms (16-byte aligned)
  __shared__ int flag[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  auto col = [&](int bi, int sl, int k) { return buf + ((size_t)(bi * 2 + sl) * b + k) * ld; };
  auto cid = [&](int bi, int sl, int k) -> int& { return ids[(bi * 2 + sl) * b + k]; };
  const C tol2 = (C)(tol * tol);

  // blocks start at their own positions: CTA c holds positions c and P-1-c
  for (int sl = 0; sl < 2; ++sl) {
    const int blk = sl == 0 ? rank : P - 1 - rank;
    for (int k = 0; k < b; ++k) {
      const int gid = blk * b + k;
      if (threadIdx.x == 0) cid(0, sl, k) = gid < p ? gid : -1;
      C* x = col(0, sl, k);
      for (int r = threadIdx.x; r < ld; r += blockDim.x) {
        C v = C(0);
        if (gid < p && r < rows) v = r < q ? Win[(size_t)gid * q + r] : ((r - q) == gid ? C(1) : C(0));
        x[r] = v;
      }
    }
  }
  if (threadIdx.x < 2) flag[threadIdx.x] = 0;
  cl.sync();

  int cur = 0, sweep = 0;
  bool done = false;
  while (!done && sweep < max_sweeps) {
    bool rot = false;
    for (int sr = 0; sr < P - 1; ++sr) {
      if (sr == 0) {  // pairs inside each block (round robin over the b columns of both slots)
        const int B = b + (b & 1), half = B / 2;
        for (int mr = 0; mr < B - 1; ++mr) {
          for (int w = warp; w < 2 * half; w += nw) {
            const int sl = w / half, k = w % half;
            int i, j;
            rr_pair(mr, k, B, i, j);
            if (i < b && j < b && cid(cur, sl, i) >= 0 && cid(cur, sl, j) >= 0)
              rot |= jacobi_pair_any<C, RPL>(col(cur, sl, i), col(cur, sl, j), q, rows, tol2);
          }
          __syncthreads();
        }
      }
      // pairs between the two blocks: warp w keeps column w of slot 0 and meets
      // column (w + mr) mod b of slot 1 (padding columns are zero and never rotate)
      if (warp < b) {
        C* xi = col(cur, 0, warp);
        int j = warp;
        for (int mr = 0; mr < b; ++mr) {
          rot |= jacobi_pair_any<C, RPL>(xi, col(cur, 1, j), q, rows, tol2);
          j = (j + 1 == b) ? 0 : j + 1;
          __syncthreads();
        }
      } else {
        for (int mr = 0; mr < b; ++mr) __syncthreads();
      }
      // rotate the positions 1..P-1 by one (position 0 stays): pull the next two blocks
      cl.sync();
      const int nb = cur ^ 1;
      {  // both slots in 16-byte words, every remote load issued before the first store
        const uint4* rsrc[2];
        const int* rid[2];
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
          const int x = sl == 0 ? rank : P - 1 - rank;
          const int src = x == 0 ? 0 : (x == 1 ? P - 1 : x - 1);
          const int scta = src < NC ? src : P - 1 - src, ssl = src < NC ? 0 : 1;
          rsrc[sl] = reinterpret_cast<const uint4*>(cl.map_shared_rank(col(cur, ssl, 0), scta));
          rid[sl] = cl.map_shared_rank(&cid(cur, ssl, 0), scta);
        }
        const int n16 = b * ld / V16;  // 16-byte words per slot
        for (int e0 = threadIdx.x; e0 < n16; e0 += 2 * blockDim.x) {
          uint4 v[2][2];
#pragma unroll
          for (int sl = 0; sl < 2; ++sl)
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int e = e0 + u * blockDim.x;
              if (e < n16) v[sl][u] = rsrc[sl][e];
            }
#pragma unroll
          for (int sl = 0; sl < 2; ++sl)
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int e = e0 + u * blockDim.x;
              if (e < n16) reinterpret_cast<uint4*>(col(nb, sl, 0))[e] = v[sl][u];
            }
        }
        if (threadIdx.x < b) {
          cid(nb, 0, threadIdx.x) = rid[0][threadIdx.x];
          cid(nb, 1, threadIdx.x) = rid[1][threadIdx.x];
        }
      }
      cur = nb;
      __syncthreads();
    }
    // the cluster-wide "any rotation" of this sweep decides, identically in every CTA
    const int any = __syncthreads_or(rot ? 1 : 0);
    int* f0 = cl.map_shared_rank(&flag[sweep & 1], 0);
    if (any && threadIdx.x == 0) atomicOr(f0, 1);
    cl.sync();
    done = (*f0 == 0);
    if (rank == 0 && threadIdx.x == 0) flag[(sweep + 1) & 1] = 0;  // next sweep's flag (last read a sweep ago)
    ++sweep;
    cl.sync();
  }
  if (!done && rank == 0 && threadIdx.x == 0 && errw) atomicOr(errw, ERRW_NOCONV);
  if (rank == 0 && threadIdx.x == 0 && errw) atomicMax((int*)errw + 1, sweep);
  // column norms, then every column's rank among all p (descending, ties by column index)
  for (int w = warp; w < 2 * b; w += nw) {
    const int sl = w / b, k = w % b;
    const C* x = col(cur, sl, k);
    C ss = 0;
    for (int r = lane; r < q; r += 32) ss += x[r] * x[r];
    ss = warp_sum(ss);
    if (lane == 0) nrm[w] = cid(cur, sl, k) >= 0 ? sqrt(ss) : C(-1);
  }
  cl.sync();
  for (int w = warp; w < 2 * b; w += nw) {
    const int sl = w / b, k = w % b;
    const int me = cid(cur, sl, k);
    if (me < 0) continue;
    const C v = nrm[w];
    int rk = 0;
    for (int c = 0; c < NC; ++c) {
      const C* rn = cl.map_shared_rank(nrm, c);
      const int* ri = cl.map_shared_rank(&cid(cur, 0, 0), c);
      for (int t = lane; t < 2 * b; t += 32) {
        const int o = ri[t];  // ids of slot 0 then slot 1 are contiguous
        const C u = rn[t];
        rk += (o >= 0) && (u > v || (u == v && o < me));
      }
    }
    rk = warp_sum(rk);
    const C* x = col(cur, sl, k);
    const C inv = v > C(0) ? C(1) / v : C(0);
    for (int r = lane; r < q; r += 32) Uo[(size_t)rk * q + r] = x[r] * inv;
    if (want_v)
      for (int r = lane; r < p; r += 32) Vo[(size_t)rk * p + r] = x[q + r];
    if (lane == 0) So[rk] = v;
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

template <typename C>
size_t jacobi_cluster_smem(int q, int p, bool want_v, int nc) {
  const int b = (p + 2 * nc - 1) / (2 * nc);
  const size_t V16 = 16 / sizeof(C);
  const size_t rows = (size_t)q + (want_v ? p : 0), ld = (rows + V16 - 1) / V16 * V16;
  return 4 * (size_t)b * ld * sizeof(C) + (4 * (size_t)b + 4) * sizeof(int) + 2 * (size_t)b * sizeof(C) + 16;
}

template <typename C, typename S>
cudaError_t jacobi_svd(int q, int p, S* W, S* U, S* Sv, S* V, S* Vwork, int max_sweeps, uint32_t* errw,
                       cudaStream_t st) {
  if (q <= 0 || p <= 0) return cudaSuccess;
  if (p > 1024 || q < p) return cudaErrorInvalidValue;
  // rotate while |w_i . w_j| > 4 eps sqrt(q) |w_i| |w_j|: the rounding error of the
  // computed dot product is about eps sqrt(q) |w_i| |w_j|, so a smaller threshold
  // would keep rotating on noise
  const double eps = (sizeof(C) == 8) ? DBL_EPSILON : (double)FLT_EPSILON;
  const double tol = 4.0 * eps * sqrt((double)q);
  // the cluster kernel spreads the columns over JC SMs when there are enough of them (16, an
  // opt-in cluster size, when a block of columns of 8 CTAs does not fit in shared memory)
  if constexpr (std::is_same<C, S>::value) {
    for (const int nc : {JC, 2 * JC}) {
      const size_t csm = jacobi_cluster_smem<C>(q, p, V != nullptr, nc);
      const int bc = (p + 2 * nc - 1) / (2 * nc), B = bc + (bc & 1);
      if (!(p >= 32 && csm <= 200 * 1024 && 32 * B <= 1024)) continue;
      auto launch = [&](auto kern) -> cudaError_t {
        cudaError_t e = ensure_smem((const void*)kern, csm);
        if (e != cudaSuccess) return e;
        if (nc > 8 && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
                          cudaSuccess)
          return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nc);
        cfg.blockDim = dim3(32 * B);
        cfg.dynamicSmemBytes = csm;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = nc;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (nc > 8) {  // a 16-CTA cluster must fit in one GPC next to nothing else: check it can be placed
          int nclu = 0;
          if (cudaOccupancyMaxActiveClusters(&nclu, kern, &cfg) != cudaSuccess || nclu < 1) {
            cudaGetLastError();
            return cudaErrorNotSupported;
          }
        }
        ++tl_launches;
        e = cudaLaunchKernelEx(&cfg, kern, q, p, bc, (const C*)W, max_sweeps, tol, errw, (C*)U, (C*)Sv, (C*)V);
        return e != cudaSuccess ? e : cudaGetLastError();
      };
      const int rows = q + (V != nullptr ? p : 0);
      cudaError_t e;
      if (nc == JC) {
        if (rows <= 160 && 32 * B <= 640) e = launch(jacobi_cluster_kernel<C, 5, JC>);
        else if (rows <= 288 && 32 * B <= 640) e = launch(jacobi_cluster_kernel<C, 9, JC>);
        else e = launch(jacobi_cluster_kernel<C, 0, JC>);
      } else {
        e = launch(jacobi_cluster_kernel<C, 0, 2 * JC>);
      }
      if (e != cudaErrorNotSupported) return e;  // otherwise the one-CTA kernel below
    }
  }
  const size_t need = ((size_t)q * p + (V ? (size_t)p * p : 0)) * sizeof(S);
  const size_t cap = 200 * 1024;
  const int in_smem = need <= cap ? 1 : 0;
  const int pairs = (p + (p & 1)) / 2;
  auto launch = [&](auto kern) -> cudaError_t {
    if (in_smem) {
      cudaError_t e = ensure_smem((const void*)kern, cap);
      if (e != cudaSuccess) return e;
    }
    ++tl_launches;
    kern<<<1, 1024, in_smem ? need : 0, st>>>(q, p, W, Vwork, max_sweeps, tol, errw, U, Sv, V, in_smem);
    return cudaGetLastError();
  };
  if (pairs <= 32) return launch(jacobi_kernel<C, S, 1>);
  if (pairs <= 64) return launch(jacobi_kernel<C, S, 2>);
  if (pairs <= 96) return launch(jacobi_kernel<C, S, 3>);
  if (pairs <= 128) return launch(jacobi_kernel<C, S, 4>);
  if (pairs <= 256) return launch(jacobi_kernel<C, S, 8>);
  return launch(jacobi_kernel<C, S, 16>);
}
template cudaError_t jacobi_svd<double, double>(int, int, double*, double*, double*, double*, double*, int,
                                                uint32_t*, cudaStream_t);
template cudaError_t jacobi_svd<float, float>(int, int, float*, float*, float*, float*, float*, int, uint32_t*,
                                              cudaStream_t);

// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024) frob_kernel(const T* __restrict__ x, long long n, double* out, uint32_t* errw) {
  __shared__ double red[32];
  T part = 0;  // per-thread partial in the value type (FP32 stays on the FP32 pipes)
  bool bad = false;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const T v = x[i];
    bad |= !isfinite(v);
    part += v * v;
  }
  double s = block_sum((double)part, red);
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    *out = sqrt(s);
    if (bad && errw) atomicOr(errw, ERRW_NAN);
  }
}

// double-FP32 values: the norm is taken of hi + lo in FP64 (small arrays only)
template <>
__global__ void __launch_bounds__(1024) frob_kernel<df32>(const df32* __restrict__ x, long long n, double* out,
                                                           uint32_t* errw) {
  __shared__ double red[32];
  double part = 0;
  bool bad = false;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = (double)x[i];
    bad |= !isfinite(v);
    part += v * v;
  }
  double s = block_sum(part, red);
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    *out = sqrt(s);
    if (bad && errw) atomicOr(errw, ERRW_NAN);
  }
}

template <typename T>
cudaError_t frob_norm(const T* x, long long n, double* out, uint32_t* errw, cudaStream_t st) {
  ++tl_launches;
  frob_kernel<T><<<1, 1024, 0, st>>>(x, n, out, errw);
  return cudaGetLastError();
}
template cudaError_t frob_norm<double>(const double*, long long, double*, uint32_t*, cudaStream_t);
template cudaError_t frob_norm<float>(const float*, long long, double*, uint32_t*, cudaStream_t);
template cudaError_t frob_norm<df32>(const df32*, long long, double*, uint32_t*, cudaStream_t);

// ---------------------------------------------------------------------------
template <typename F>
__global__ void truncate_kernel(const F* S, int p, const double* normM, double tau_over_L, int chi_max,
                                double cutoff, int* info, double* dinfo) {
  if (threadIdx.x != 0) return;
  const double nM = *normM;
  int k = min(chi_max, p);
  if (tau_over_L > 0.0) {
    const double thr = tau_over_L * nM;
    int kmin = p;
    double tail = 0.0;
    for (int j = p - 1; j >= 1; --j) {
      tail += (double)S[j] * (double)S[j];
      if (sqrt(tail) <= thr) kmin = j;
      else break;
    }
    k = min(k, kmin);
  }
  if (p > 0) {
    int cnt = 0;
    for (int j = 0; j < p; ++j) cnt += (double)S[j] > cutoff * (double)S[0];
    k = min(k, cnt);
  }
  k = max(k, 1);
  double kept = 0.0, disc = 0.0;
  for (int j = 0; j < p; ++j) {
    const double sj = (double)S[j];
    if (j < k) kept += sj * sj;
    else disc += sj * sj;
  }
  info[0] = k;
  dinfo[0] = kept;
  dinfo[1] = nM > 0.0 ? sqrt(disc) / nM : 0.0;
}

template <typename F>
cudaError_t truncate_rule(const F* S, int p, const double* normM, double tau_over_L, int chi_max, double cutoff,
                          int* info, double* dinfo, cudaStream_t st) {
  ++tl_launches;
  truncate_kernel<F><<<1, 32, 0, st>>>(S, p, normM, tau_over_L, chi_max, cutoff, info, dinfo);
  return cudaGetLastError();
}
template cudaError_t truncate_rule<double>(const double*, int, const double*, double, int, double, int*, double*,
                                           cudaStream_t);
template cudaError_t truncate_rule<float>(const float*, int, const double*, double, int, double, int*, double*,
                                          cudaStream_t);

// s_j = sqrt(max(lambda_j, 0)): singular values from the eigenvalues of a Gram matrix
template <typename F>
__global__ void sqrt_clamp_kernel(int n, F* x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const F v = x[i];
    x[i] = v > F(0) ? sqrt(v) : F(0);
  }
}
template <typename F>
cudaError_t sqrt_clamp(int n, F* x, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ++tl_launches;
  sqrt_clamp_kernel<F><<<(n + 255) / 256, 256, 0, st>>>(n, x);
  return cudaGetLastError();
}
template cudaError_t sqrt_clamp<double>(int, double*, cudaStream_t);
template cudaError_t sqrt_clamp<float>(int, float*, cudaStream_t);

// ---------------------------------------------------------------------------
template <typename T, typename F>
__global__ void gauge_update_kernel(int mode, int m, int n, const F* __restrict__ U, int ld_u,
                                    const F* __restrict__ S, const F* __restrict__ V, int ld_v,
                                    const int* __restrict__ kdev, double* Cl, double* Cr, double* Y, T* Ut, T* Vt) {
  const int k = *kdev;
  const long long tot_l = (long long)m * k, tot_r = (long long)k * n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot_l; e += stride) {
    const int i = (int)(e / k), j = (int)(e % k);
    const double u = (double)U[(size_t)j * ld_u + i];
    Cl[e] = (mode == 0) ? u : u * (double)S[j];
    Ut[(size_t)j * m + i] = (T)u;
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot_r; e += stride) {
    const int j = (int)(e / n), c = (int)(e % n);
    const double v = (double)V[(size_t)j * ld_v + c];
    Cr[e] = (mode == 1) ? v : (double)S[j] * v;
    Vt[e] = (T)v;
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < k; e += stride)
    Y[e] = (mode == 2) ? ((double)S[e] > 0.0 ? 1.0 / (double)S[e] : 0.0) : 1.0;
}

template <typename T, typename F>
cudaError_t gauge_update(int mode, int m, int n, const F* U, int ld_u, const F* S, const F* V, int ld_v,
                         const int* kdev, double* Cl, double* Cr, double* Y, T* Ut, T* Vt, cudaStream_t st) {
  long long tot = (long long)(m > n ? m : n) * 128;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  ++tl_launches;
  gauge_update_kernel<T, F><<<blocks, 256, 0, st>>>(mode, m, n, U, ld_u, S, V, ld_v, kdev, Cl, Cr, Y, Ut, Vt);
  return cudaGetLastError();
}
template cudaError_t gauge_update<double, double>(int, int, int, const double*, int, const double*, const double*, int,
                                                  const int*, double*, double*, double*, double*, double*, cudaStream_t);
template cudaError_t gauge_update<float, float>(int, int, int, const float*, int, const float*, const float*, int,
                                                const int*, double*, double*, double*, float*, float*, cudaStream_t);
template cudaError_t gauge_update<double, float>(int, int, int, const float*, int, const float*, const float*, int,
                                                 const int*, double*, double*, double*, double*, double*, cudaStream_t);
template cudaError_t gauge_update<df32, float>(int, int, int, const float*, int, const float*, const float*, int,
                                               const int*, double*, double*, double*, df32*, df32*, cudaStream_t);
template cudaError_t gauge_update<df32, double>(int, int, int, const double*, int, const double*, const double*, int,
                                                const int*, double*, double*, double*, df32*, df32*, cudaStream_t);

// ---------------------------------------------------------------------------
template <typename Tin, typename Tout>
__global__ void copy_map_kernel(int rows, int cols, const Tin* __restrict__ in, IdxMap im, IdxMap in_,
                                Tout* __restrict__ out, IdxMap om, IdxMap on, double scale) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols), j = (int)(e % cols);
    const Tin x = in[im(i) + in_(j)];
    out[om(i) + on(j)] = scale == 1.0 ? (Tout)x : (Tout)(scale * (double)x);  // plain copies stay off the FP64 pipe
  }
}

template <typename Tin, typename Tout>
cudaError_t copy_map(int rows, int cols, const Tin* in, IdxMap im, IdxMap in_, Tout* out, IdxMap om, IdxMap on,
                     double scale, cudaStream_t st) {
  long long tot = (long long)rows * cols;
  if (tot <= 0) return cudaSuccess;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  ++tl_launches;
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
template cudaError_t copy_map<float, df32>(int, int, const float*, IdxMap, IdxMap, df32*, IdxMap, IdxMap, double,
                                           cudaStream_t);
template cudaError_t copy_map<double, df32>(int, int, const double*, IdxMap, IdxMap, df32*, IdxMap, IdxMap, double,
                                            cudaStream_t);
template cudaError_t copy_map<df32, double>(int, int, const df32*, IdxMap, IdxMap, double*, IdxMap, IdxMap, double,
                                            cudaStream_t);
template cudaError_t copy_map<df32, float>(int, int, const df32*, IdxMap, IdxMap, float*, IdxMap, IdxMap, double,
                                           cudaStream_t);
template cudaError_t copy_map<df32, df32>(int, int, const df32*, IdxMap, IdxMap, df32*, IdxMap, IdxMap, double,
                                          cudaStream_t);

// ---------------------------------------------------------------------------
template <typename F>
__global__ void philox_fill_kernel(F* out, long long count, uint64_t seed, uint64_t stream, double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    out[i] = (F)(scale * philox_normal(seed, stream, (uint64_t)i));
}

template <typename F>
cudaError_t philox_fill(F* out, long long count, uint64_t seed, uint64_t stream, double scale, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int blocks = (int)((count + 255) / 256);
  if (blocks > 2048) blocks = 2048;
  ++tl_launches;
  philox_fill_kernel<F><<<blocks, 256, 0, st>>>(out, count, seed, stream, scale);
  return cudaGetLastError();
}
template cudaError_t philox_fill<double>(double*, long long, uint64_t, uint64_t, double, cudaStream_t);
template cudaError_t philox_fill<float>(float*, long long, uint64_t, uint64_t, double, cudaStream_t);
template cudaError_t philox_fill<df32>(df32*, long long, uint64_t, uint64_t, double, cudaStream_t);

// ---------------------------------------------------------------------------
// Sign convention of singular pair j: the entry of largest magnitude of u_j is
// positive (lowest index on ties); (u_j, v_j) are flipped together.
template <typename F>
__global__ void fix_signs_kernel(int m, int n, F* __restrict__ U, int ld_u, F* __restrict__ V, int ld_v) {
  __shared__ double sb[32];
  __shared__ int si[32];
  __shared__ double sgn;
  F* u = U + (size_t)blockIdx.x * ld_u;
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double a = fabs((double)u[i]);
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
    sgn = (si[0] < m && (double)u[si[0]] < 0.0) ? -1.0 : 1.0;
  }
  __syncthreads();
  if (sgn < 0.0) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) u[i] = -u[i];
    if (V) {  // V may be absent when only the left factor is wanted
      F* v = V + (size_t)blockIdx.x * ld_v;
      for (int c = threadIdx.x; c < n; c += blockDim.x) v[c] = -v[c];
    }
  }
}

template <typename F>
cudaError_t fix_signs(int m, int n, int p, F* U, int ld_u, F* V, int ld_v, cudaStream_t st) {
  if (p <= 0 || m <= 0) return cudaSuccess;
  ++tl_launches;
  fix_signs_kernel<F><<<p, 256, 0, st>>>(m, n, U, ld_u, V, ld_v);
  return cudaGetLastError();
}
template cudaError_t fix_signs<double>(int, int, int, double*, int, double*, int, cudaStream_t);
template cudaError_t fix_signs<float>(int, int, int, float*, int, float*, int, cudaStream_t);
template cudaError_t fix_signs<df32>(int, int, int, df32*, int, df32*, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Alg. 4 from FP64 isometries U (m x k), V (n x k) (column-major) and the
// projected k x k block P = U^T Theta V: s = diag(P), Psi_l = U s (m x k
// row-major), Psi_{l+1} = s V^T (k x n row-major), Y_l = 1 / s.
template <typename T>
__global__ void inverse_gauge_kernel(int m, int n, int k, const double* __restrict__ U, const double* __restrict__ V,
                                     const T* __restrict__ P, double* Cl, double* Cr, double* Y) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long e = t0; e < (long long)m * k; e += stride) {
    const int i = (int)(e / k), j = (int)(e % k);
    Cl[e] = U[(size_t)j * m + i] * (double)P[(size_t)j * k + j];
  }
  for (long long e = t0; e < (long long)k * n; e += stride) {
    const int j = (int)(e / n), c = (int)(e % n);
    Cr[e] = (double)P[(size_t)j * k + j] * V[(size_t)j * n + c];
  }
  for (long long e = t0; e < k; e += stride) {
    const double sj = (double)P[(size_t)e * k + e];
    Y[e] = sj != 0.0 ? 1.0 / sj : 0.0;
  }
}

template <typename T>
cudaError_t inverse_gauge_update(int m, int n, int k, const double* U, const double* V, const T* P, double* Cl,
                                 double* Cr, double* Y, cudaStream_t st) {
  long long tot = (long long)(m > n ? m : n) * k;
  int blocks = (int)std::min<long long>((tot + 255) / 256, 1024);
  ++tl_launches;
  inverse_gauge_kernel<T><<<std::max(blocks, 1), 256, 0, st>>>(m, n, k, U, V, P, Cl, Cr, Y);
  return cudaGetLastError();
}
template cudaError_t inverse_gauge_update<float>(int, int, int, const double*, const double*, const float*, double*,
                                                 double*, double*, cudaStream_t);
template cudaError_t inverse_gauge_update<double>(int, int, int, const double*, const double*, const double*, double*,
                                                  double*, double*, cudaStream_t);
template cudaError_t inverse_gauge_update<df32>(int, int, int, const double*, const double*, const df32*, double*,
                                                double*, double*, cudaStream_t);

// ---------------------------------------------------------------------------
__global__ void scale_cols_kernel(int rows, int cols, const double* __restrict__ in, const double* __restrict__ y,
                                  double* __restrict__ out) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x)
    out[e] = y ? in[e] * y[e % cols] : in[e];
}

template <typename T>
__global__ void scale_rows_kernel(int rows, int cols, const double* __restrict__ in, const double* __restrict__ y,
                                  T* __restrict__ out) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x)
    out[e] = (T)(y ? in[e] * y[e / cols] : in[e]);
}

template <typename T>
cudaError_t scale_rows(int rows, int cols, const double* in, const double* y, T* out, cudaStream_t st) {
  long long tot = (long long)rows * cols;
  if (tot <= 0) return cudaSuccess;
  int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
  ++tl_launches;
  scale_rows_kernel<T><<<blocks, 256, 0, st>>>(rows, cols, in, y, out);
  return cudaGetLastError();
}
template cudaError_t scale_rows<float>(int, int, const double*, const double*, float*, cudaStream_t);
template cudaError_t scale_rows<double>(int, int, const double*, const double*, double*, cudaStream_t);
template cudaError_t scale_rows<df32>(int, int, const double*, const double*, df32*, cudaStream_t);

cudaError_t scale_cols(int rows, int cols, const double* in, const double* y, double* out, cudaStream_t st) {
  long long tot = (long long)rows * cols;
  if (tot <= 0) return cudaSuccess;
  int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
  ++tl_launches;
  scale_cols_kernel<<<blocks, 256, 0, st>>>(rows, cols, in, y, out);
  return cudaGetLastError();
}

}  // namespace ttfit

// out (cols x rows, row-major) = (in diag(y))^T, in rows x cols row-major FP64 (y = NULL: 1)
namespace ttfit {
template <typename T>
__global__ void scale_cols_t_kernel(int rows, int cols, const double* __restrict__ in, const double* __restrict__ y,
                                    T* __restrict__ out) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / rows), r = (int)(e % rows);  // e indexes out; the read is strided
    out[e] = (T)(y ? in[(size_t)r * cols + c] * y[c] : in[(size_t)r * cols + c]);
  }
}

template <typename T>
cudaError_t scale_cols_t(int rows, int cols, const double* in, const double* y, T* out, cudaStream_t st) {
  long long tot = (long long)rows * cols;
  if (tot <= 0) return cudaSuccess;
  int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
  ++tl_launches;
  scale_cols_t_kernel<T><<<blocks, 256, 0, st>>>(rows, cols, in, y, out);
  return cudaGetLastError();
}
template cudaError_t scale_cols_t<float>(int, int, const double*, const double*, float*, cudaStream_t);
template cudaError_t scale_cols_t<double>(int, int, const double*, const double*, double*, cudaStream_t);
template cudaError_t scale_cols_t<df32>(int, int, const double*, const double*, df32*, cudaStream_t);
}  // namespace ttfit

// ---------------------------------------------------------------------------
// Power-of-two scaling around a lower-precision factorisation. The two-site
// tensor of an early window can be tiny (a random guess overlaps A B by ~1e-15
// on a long chain); its squares underflow FP32 inside the Gram sums. Scaling by
// 2^-e (e the exponent of max |x|) is exact, leaves the singular vectors and
// every relative rule unchanged, and is undone on the singular values.
namespace ttfit {
// frexp exponent of |x| (x = f 2^e, f in [0.5, 1)) from the IEEE bits, integer ops only
__device__ __forceinline__ int exp_of(float x) {
  const int E = (__float_as_int(x) >> 23) & 0xFF;
  return E == 0xFF ? INT_MIN : E - 126;  // Inf / NaN: ignored here (the norm check flags them)
}
__device__ __forceinline__ int exp_of(double x) {
  const int E = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  return E == 0x7FF ? INT_MIN : E - 1022;
}
__device__ __forceinline__ int exp_of(df32 x) { return exp_of(x.hi); }
template <typename T>
__device__ __forceinline__ bool is_zero(T x) {
  return x == T(0);
}
template <>
__device__ __forceinline__ bool is_zero<df32>(df32 x) {
  return x.hi == 0.f;
}

// e = max over nonzero x of the exponent of x (left untouched when every x is 0); e must
// be preset to a very negative value
template <typename T>
__global__ void absmax_exponent_kernel(const T* __restrict__ x, long long n, int* e) {
  int m = INT_MIN;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!is_zero(x[i])) m = max(m, exp_of(x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m != INT_MIN) atomicMax(e, m);
}
template <typename T>
cudaError_t absmax_exponent(const T* x, long long n, int* e, cudaStream_t st) {
  // preset: every byte 0x80, i.e. -2139062144; an all-zero input keeps it, and scaling by
  // 2^(-e) of zeros is still zero
  cudaError_t err = cudaMemsetAsync(e, 0x80, sizeof(int), st);
  if (err != cudaSuccess) return err;
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 152);
  ++tl_launches;
  absmax_exponent_kernel<T><<<blocks, 256, 0, st>>>(x, n, e);
  return cudaGetLastError();
}
template cudaError_t absmax_exponent<double>(const double*, long long, int*, cudaStream_t);
template cudaError_t absmax_exponent<float>(const float*, long long, int*, cudaStream_t);
template cudaError_t absmax_exponent<df32>(const df32*, long long, int*, cudaStream_t);

template <typename Tout, typename Tin>
__device__ __forceinline__ Tout scale_pow2(Tin x, int s);
template <>
__device__ __forceinline__ float scale_pow2<float, float>(float x, int s) { return scalbnf(x, s); }
template <>
__device__ __forceinline__ float scale_pow2<float, double>(double x, int s) { return (float)scalbn(x, s); }
template <>
__device__ __forceinline__ float scale_pow2<float, df32>(df32 x, int s) { return scalbnf(x.hi, s) + scalbnf(x.lo, s); }
template <>
__device__ __forceinline__ double scale_pow2<double, double>(double x, int s) { return scalbn(x, s); }
template <>
__device__ __forceinline__ double scale_pow2<double, df32>(df32 x, int s) { return scalbn((double)x, s); }

template <typename Tin, typename Tout>
__global__ void copy_pow2_kernel(long long n, const Tin* __restrict__ in, Tout* __restrict__ out, const int* e) {
  const int s = -*e;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = scale_pow2<Tout, Tin>(in[i], s);
}
template <typename Tin, typename Tout>
cudaError_t copy_pow2(long long n, const Tin* in, Tout* out, const int* e, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  ++tl_launches;
  copy_pow2_kernel<Tin, Tout><<<blocks, 256, 0, st>>>(n, in, out, e);
  return cudaGetLastError();
}
template cudaError_t copy_pow2<double, double>(long long, const double*, double*, const int*, cudaStream_t);
template cudaError_t copy_pow2<double, float>(long long, const double*, float*, const int*, cudaStream_t);
template cudaError_t copy_pow2<float, float>(long long, const float*, float*, const int*, cudaStream_t);
template cudaError_t copy_pow2<df32, float>(long long, const df32*, float*, const int*, cudaStream_t);
template cudaError_t copy_pow2<df32, double>(long long, const df32*, double*, const int*, cudaStream_t);

// s_i <- s_i 2^e and ||M|| <- ||M|| 2^e: the factorisation of 2^-e M back to M
template <typename F>
__global__ void unscale_pow2_kernel(int p, F* s, double* nrm, const int* e) {
  const int ex = *e;
  for (int i = threadIdx.x; i < p; i += blockDim.x) s[i] = (F)scalbn((double)s[i], ex);
  if (threadIdx.x == 0) *nrm = scalbn(*nrm, ex);
}
template <typename F>
cudaError_t unscale_pow2(int p, F* s, double* nrm, const int* e, cudaStream_t st) {
  ++tl_launches;
  unscale_pow2_kernel<F><<<1, 256, 0, st>>>(p, s, nrm, e);
  return cudaGetLastError();
}
template cudaError_t unscale_pow2<float>(int, float*, double*, const int*, cudaStream_t);
template cudaError_t unscale_pow2<double>(int, double*, double*, const int*, cudaStream_t);
}  // namespace ttfit

namespace ttfit {

// ---------------------------------------------------------------------------
// Inverse of a small upper-triangular factor in FP32, written in double-FP32,
// for the basis of the randomized update (see engine.cu, factorize_rsvd_hp):
// R is the p x p upper-triangular factor of a Householder QR (FP32,
// column-major, ld ldr); out = 2^-e R^-1 with e = *eexp (0 if null). Any
// non-singular right factor keeps the column space of the matrix it
// multiplies, so FP32 accuracy suffices: the range is carried by the
// double-FP32 product that applies it. For the same reason a pivot below
// 2^-24 max |r_ii| (a sketch column in the noise of the others) is raised to
// that floor instead of stopping the factorisation. One CTA; R and X = R^-1
// live in shared memory (2 p^2 floats). Bottom-up by panels of TI_B rows: the
// rows of a panel are finished column by column (one thread per column,
// back substitution inside the panel: x_i = (e_i - acc_i - sum r_il x_l) / r_ii),
// then every row above takes the panel's rank-TI_B update acc_r += sum_i r_ri x_i.
// Only a non-finite or all-zero R sets ERRW_HPFAIL.
// ---------------------------------------------------------------------------
constexpr int TI_B = 8;

__global__ void __launch_bounds__(1024) tri_inv_kernel(int p, const float* __restrict__ R, int ldr, const int* eexp,
                                                       df32* __restrict__ out, uint32_t* errw) {
  extern __shared__ __align__(16) float tis[];
  float* A = tis;           // R, column-major p x p
  float* X = tis + p * p;   // accumulators, then rows of R^-1
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < p * p; e += nt) {
    const int i = e % p, j = e / p;
    A[e] = i <= j ? R[(size_t)j * ldr + i] : 0.f;
    X[e] = 0.f;
  }
  __syncthreads();
  float big = 0.f;  // max |r_ii|, the same in every thread
  bool finite = true;
  for (int i = 0; i < p; ++i) {
    const float d = A[i * p + i];
    finite = finite && isfinite(d);
    big = fmaxf(big, fabsf(d));
  }
  const float floor_ = big * 0x1p-24f;
  const bool bad = !finite || !(big > 0.f);
  for (int i0 = ((p - 1) / TI_B) * TI_B; i0 >= 0; i0 -= TI_B) {
    const int i1 = min(p, i0 + TI_B);  // panel rows i0 .. i1-1
    for (int c = i0 + tid; c < p; c += nt) {  // finish the panel's rows of column c, bottom-up
      float xv[TI_B];
#pragma unroll
      for (int t = TI_B - 1; t >= 0; --t) {
        const int i = i0 + t;
        if (i >= i1 || c < i) {
          xv[t] = 0.f;
          continue;
        }
        float acc = X[c * p + i];
#pragma unroll
        for (int u = t + 1; u < TI_B; ++u)
          if (i0 + u < i1) acc = fmaf(A[(i0 + u) * p + i], xv[u], acc);
        float rii = A[i * p + i];
        if (!(fabsf(rii) >= floor_)) rii = floor_ > 0.f ? floor_ : 1.f;
        xv[t] = ((c == i ? 1.f : 0.f) - acc) / rii;
      }
#pragma unroll
      for (int t = 0; t < TI_B; ++t)
        if (i0 + t < i1) X[c * p + i0 + t] = xv[t];
    }
    __syncthreads();
    const long long cnt = (long long)i0 * (p - i0);  // rows r < i0 of columns c >= i0
    for (long long e = tid; e < cnt; e += nt) {
      const int r = (int)(e % i0), c = i0 + (int)(e / i0);
      float acc = X[c * p + r];
#pragma unroll
      for (int t = 0; t < TI_B; ++t)
        if (i0 + t < i1) acc = fmaf(A[(i0 + t) * p + r], X[c * p + i0 + t], acc);
      X[c * p + r] = acc;
    }
    __syncthreads();
  }
  const int ex = eexp ? *eexp : 0;
  for (int e = tid; e < p * p; e += nt) {
    const int i = e % p, j = e / p;
    out[e] = df32(i <= j ? scalbnf(X[e], -ex) : 0.f, 0.f);
  }
  if (bad && tid == 0 && errw) atomicOr(errw, ERRW_HPFAIL);
}

cudaError_t tri_inv(int p, const float* R, int ldr, const int* eexp, df32* out, uint32_t* errw, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  const size_t smem = 2 * (size_t)p * p * sizeof(float);
  if (p > TRI_INV_MAX || smem > 220 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = ensure_smem((const void*)tri_inv_kernel, smem);
  if (e != cudaSuccess) return e;
  ++tl_launches;
  tri_inv_kernel<<<1, 1024, smem, st>>>(p, R, ldr, eexp, out, errw);
  return cudaGetLastError();
}

// out (rows x cols, column-major, double-FP32) = in (FP32, column-major, ld rows) with
// column j scaled by 2^-e / s_j (0 where s_j = 0); e = *eexp.
__global__ void scale_cols_inv_kernel(int rows, int cols, const float* __restrict__ in, const float* __restrict__ s,
                                      const int* eexp, df32* __restrict__ out) {
  const long long tot = (long long)rows * cols;
  const int ex = eexp ? *eexp : 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / rows);
    const float sj = s[j];
    // 1 / s_j as a double-FP32 reciprocal: r0 = 1/s, r1 = r0 (2 - s r0) rounded split (Newton's method)
    df32 v(0.f, 0.f);
    if (sj != 0.f) {
      const float r0 = 1.f / sj;
      const float res = __fmaf_rn(-sj, r0, 1.f);  // 1 - s r0, exact by FMA
      v = renorm(r0, r0 * res) * df32(in[e], 0.f);
      v = df32(scalbnf(v.hi, -ex), scalbnf(v.lo, -ex));
    }
    out[e] = v;
  }
}

cudaError_t scale_cols_inv(int rows, int cols, const float* in, const float* s, const int* eexp, df32* out,
                           cudaStream_t st) {
  const long long tot = (long long)rows * cols;
  if (tot <= 0) return cudaSuccess;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  ++tl_launches;
  scale_cols_inv_kernel<<<blocks, 256, 0, st>>>(rows, cols, in, s, eexp, out);
  return cudaGetLastError();
}

// max |G - I| of a p x p double-FP32 matrix; sets ERRW_HPFAIL above tol.
__global__ void ortho_check_kernel(int p, const df32* __restrict__ G, double tol, uint32_t* errw) {
  float worst = 0.f;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e % p, j = e / p;
    const df32 d = G[e] - df32(i == j ? 1.f : 0.f, 0.f);
    const float a = fabsf(d.hi);
    worst = (a > worst || !isfinite(a)) ? (isfinite(a) ? a : INFINITY) : worst;
  }
  worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, 16));
  worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, 8));
  worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, 4));
  worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, 2));
  worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, 1));
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x == 0) {
    float w = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) w = fmaxf(w, red[i]);
    if (!(w <= (float)tol) && errw) atomicOr(errw, ERRW_HPFAIL);
  }
}

cudaError_t ortho_check(int p, const df32* G, double tol, uint32_t* errw, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  ++tl_launches;
  ortho_check_kernel<<<1, 1024, 0, st>>>(p, G, tol, errw);
  return cudaGetLastError();
}

}  // namespace ttfit
