// Shared device/host helpers of the fit library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <map>
#include <mutex>
#include <utility>

namespace ttfit {

// Raise (never lower) a kernel's dynamic shared-memory limit on the current
// device. The limit is process-wide per function, and host threads of
// concurrent handles launch the same kernels with different sizes: setting it
// to each launch's own size would let one thread lower it between another
// thread's set and launch (the launch then fails with an invalid argument).
inline cudaError_t ensure_smem(const void* kern, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> cur;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  size_t& have = cur[{dev, kern}];
  if (have >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

// Kernel launches issued by the calling host thread; every launch site
// increments it, and the API entry points attribute the difference to their
// handle.
inline thread_local long long tl_launches = 0;

// Linear index -> memory offset through a mixed radix of up to three levels,
// i = (i0 * n1 + i1) * n2 + i2, offset = i0*s0 + i1*s1 + i2*s2. Every tensor
// permutation used by the contraction chain is a sum of two such maps (rows,
// columns), so one GEMM kernel covers every layout.
struct IdxMap {
  int n1 = 1, n2 = 1;
  long long s0 = 0, s1 = 0, s2 = 0;
  __host__ __device__ __forceinline__ long long operator()(long long i) const {
    if (i >= 0 && i < (1ll << 30)) {  // every index of this library: 32-bit division, several times cheaper
      if (n2 == (1 << 30) && n1 == 1) return i * s2;  // uniform stride
      const unsigned u = (unsigned)i, q2 = (unsigned)n2;
      const unsigned i2 = u % q2, t = u / q2;
      if (n1 == (1 << 30)) return (long long)t * s1 + (long long)i2 * s2;  // two levels
      const unsigned q1 = (unsigned)n1;
      return (long long)(t / q1) * s0 + (long long)(t % q1) * s1 + (long long)i2 * s2;
    }
    long long i2 = i % n2;
    long long t = i / n2;
    long long i1 = t % n1;
    long long i0 = t / n1;
    return i0 * s0 + i1 * s1 + i2 * s2;
  }
  // uniform stride map
  static IdxMap lin(long long s) {
    IdxMap m;
    m.s2 = s;
    m.n2 = 1 << 30;
    return m;
  }
  // two-level map: i = i1 * n2 + i2
  static IdxMap two(int n2, long long s1, long long s2) {
    IdxMap m;
    m.n1 = 1 << 30;
    m.n2 = n2;
    m.s1 = s1;
    m.s2 = s2;
    return m;
  }
  static IdxMap three(int n1, int n2, long long s0, long long s1, long long s2) {
    IdxMap m;
    m.n1 = n1;
    m.n2 = n2;
    m.s0 = s0;
    m.s1 = s1;
    m.s2 = s2;
    return m;
  }
};

// Double-FP32 number: the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2, about 48 significant bits. Its arithmetic runs on the
// FP32 pipes, which on this GPU issue ~60x the FP64 rate: a multiply-add is
// an exact product (Dekker's TwoProduct through one FMA), the cross terms,
// Knuth's TwoSum and a renormalisation, 15 FP32 instructions against one DFMA.
// Conversions from and to double are explicit so that mixed expressions do
// not silently switch pipes.
struct __align__(8) df32 {
  float hi, lo;
  df32() = default;  // trivial, so that it can live in __shared__ arrays
  __host__ __device__ __forceinline__ df32(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ explicit df32(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ __forceinline__ explicit operator float() const { return hi + lo; }
};

// The error-free transformations below use the _rn intrinsics, which the
// compiler never contracts into FMAs (a contraction would change the rounded
// sum that the error terms are computed against).
// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df32 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df32(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
// renormalise (s, t) with |t| small against s (Dekker's fast two-sum)
__device__ __forceinline__ df32 renorm(float s, float t) {
  const float h = __fadd_rn(s, t);
  return df32(h, __fsub_rn(t, __fsub_rn(h, s)));
}
__device__ __forceinline__ df32 operator+(df32 a, df32 b) {
  df32 s = two_sum(a.hi, b.hi);
  return renorm(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df32 operator-(df32 a) { return df32(-a.hi, -a.lo); }
__device__ __forceinline__ df32 operator-(df32 a, df32 b) { return a + (-b); }
__device__ __forceinline__ df32& operator+=(df32& a, df32 b) { return a = a + b; }
__device__ __forceinline__ df32 operator*(df32 a, df32 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // exact rounding error of the leading product
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return renorm(p, e);
}
// a * b + c, the inner step of the GEMM, for every working type
__host__ __device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double madd(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ df32 madd(df32 a, df32 b, df32 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  const df32 s = two_sum(p, c.hi);
  return renorm(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}
__host__ __device__ __forceinline__ bool operator!=(df32 a, df32 b) { return a.hi != b.hi || a.lo != b.lo; }
__host__ __device__ __forceinline__ bool operator==(df32 a, df32 b) { return a.hi == b.hi && a.lo == b.lo; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and the Box-Muller Gaussian of element
// i of stream s: counter (i lo, i hi, s lo, s hi), key (seed lo, seed hi);
// ua = (x0*2^21 + (x1>>11)) 2^-53, ub = (x2*2^21 + (x3>>11)) 2^-53,
// value sqrt(-2 ln(1-ua)) cos(2 pi ub).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                             uint32_t k0, uint32_t k1) {
  const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
  uint32_t lo0 = m0 * c0, hi0 = __umulhi(m0, c0);
  uint32_t lo1 = m1 * c2, hi1 = __umulhi(m1, c2);
  uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
  c0 = n0;
  c1 = lo1;
  c2 = n2;
  c3 = lo0;
}

__device__ __forceinline__ double philox_normal(uint64_t seed, uint64_t stream, uint64_t idx) {
  uint32_t c0 = (uint32_t)idx, c1 = (uint32_t)(idx >> 32), c2 = (uint32_t)stream, c3 = (uint32_t)(stream >> 32);
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    philox_round(c0, c1, c2, c3, k0, k1);
  }
  const double two53 = 1.0 / 9007199254740992.0;
  double ua = (double)(((uint64_t)c0 << 21) + (c1 >> 11)) * two53;
  double ub = (double)(((uint64_t)c2 << 21) + (c3 >> 11)) * two53;
  return sqrt(-2.0 * log1p(-ua)) * cospi(2.0 * ub);
}

inline uint64_t omega_stream(int sweep, int site) {
  return (1ull << 40) | ((uint64_t)sweep << 20) | (uint64_t)site;
}
inline uint64_t init_stream(int site) { return (2ull << 40) | (uint64_t)site; }

// Device error word bits (written by kernels, read by the host after a window).
enum : uint32_t {
  ERRW_NAN = 1u,        // non-finite value in a two-site tensor
  ERRW_NOCONV = 2u,     // Jacobi sweeps hit their limit
  ERRW_BADSHAPE = 4u,   // a kernel saw dimensions outside its compiled limits
  ERRW_TIMEOUT = 8u,    // a bounded mbarrier wait expired
  ERRW_HPFAIL = 16u,    // the FP64-class sketch basis could not be formed (the window falls back to FP32)
};

}  // namespace ttfit
