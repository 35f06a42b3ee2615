// Tensor-core contraction kernel for sm_103a (5th-generation tensor cores).
//
//   C[cm(m) + cn(n)] = alpha * sum_k A[m*lda + k] * B(n, k) + beta * C[...]
//
// A is K-major (k contiguous, rows at stride lda); B is K-major (rows n at
// stride ldb, k contiguous) or MN-major (rows k at stride ldb, n contiguous).
// Operand tiles are moved global -> shared memory by TMA (128-byte swizzle),
// one elected thread issues tcgen05.mma (kind::tf32, FP32 accumulation in
// tensor memory), and four warps drain the 128 x 128 accumulator with
// tcgen05.ld into the output layout given by two index maps (any tensor
// permutation of the fit's contraction chain). Split-K partial sums go to a
// dense FP32 workspace and are reduced by splitk_reduce_kernel.
//
// Every mbarrier wait is bounded; on expiry the kernel sets ERRW_TIMEOUT in
// the device error word, stops issuing work, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <climits>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace ttfit {

namespace tc {

constexpr int BM = 128, BN = 128, BK = 32;  // BK fp32 elements = 128 bytes = one swizzle span
constexpr int TILE_BYTES = BM * BK * 4;     // 16 KB (A); B tile has the same size
// 1-pass TF32: 4 stages of (A, B); split (3xTF32): 3 stages of (A, B, A_lo, B_lo)
template <bool SPLIT>
struct Cfg {
  static constexpr int STAGES = SPLIT ? 3 : 4;
  static constexpr int TILES = SPLIT ? 4 : 2;
  static constexpr int SMEM_BYTES = STAGES * TILES * TILE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
};
constexpr long long WAIT_LIMIT = 1ll << 26;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// shared-memory matrix descriptor, 128-byte swizzle (layout type 2), version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46) | (2ull << 61);
}
// the same with the 64-byte swizzle (layout type 4): K-major rows of 64 bytes, 8-row groups SBO apart
__device__ __forceinline__ uint64_t sdesc64(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46) | (4ull << 61);
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// instruction descriptor: D = F32 (bits 4-5 = 1), A = B = TF32 (format 2 at bits 7-9 and 10-12),
// A K-major (bit 15 = 0), B major per template (bit 16), N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n, bool b_mn_major) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((b_mn_major ? 1u : 0u) << 16) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

// kind::f16 with both operands BF16 (format 1 at bits 7-9 and 10-12), D = F32, both K-major
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <bool B_MN, bool SPLIT>
__global__ void __launch_bounds__(128, 1)
    gemm_tf32_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
                     int K, int k_per_split, float* __restrict__ C, IdxMap cm, IdxMap cn, float alpha, float beta,
                     float* __restrict__ C2, IdxMap cm2, IdxMap cn2, float* __restrict__ ws, uint32_t* errw) {
  constexpr int STAGES = Cfg<SPLIT>::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * TILE_BYTES;
  uint8_t* sAl = smem + 2 * STAGES * TILE_BYTES;  // split only: low parts, same swizzled layout
  uint8_t* sBl = smem + 3 * STAGES * TILE_BYTES;
  uint64_t* bars = (uint64_t*)(smem + STAGES * Cfg<SPLIT>::TILES * TILE_BYTES);
  // bars[0..S-1] full, [S..2S-1] empty, [2S] accumulator ready, [2S+1..3S] split done
  uint32_t* tmem_slot = (uint32_t*)(bars + 3 * STAGES + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb0 = blockIdx.z * k_per_split;
  const int kend = min(K, kb0 + k_per_split);
  const int nk = (kend - kb0 + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(su32(&bars[s]), 1);
      mbar_init(su32(&bars[STAGES + s]), 1);
    }
    mbar_init(su32(&bars[2 * STAGES]), 1);
    for (int s = 0; s < STAGES; ++s) mbar_init(su32(&bars[2 * STAGES + 1 + s]), 2);  // two splitter warps
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  int issued = 0;  // stages loaded by the producer (for the bounded drain on abort)
  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (*abort_flag || !mbar_wait(su32(&bars[STAGES + s]), ph ^ 1)) {
        *abort_flag = 1;
        break;
      }
      const uint32_t full = su32(&bars[s]);
      mbar_expect_tx(full, 2 * TILE_BYTES);
      const int k = kb0 + kb * BK;
      tma_load_2d(su32(sA + s * TILE_BYTES), &tmA, full, k, m0);
      if (B_MN) {
        // four boxes of (32 n) x (BK k): n chunk j at byte offset j * BK * 128
#pragma unroll
        for (int j = 0; j < BN / 32; ++j) tma_load_2d(su32(sB + s * TILE_BYTES + j * BK * 128), &tmB, full, n0 + 32 * j, k);
      } else {
        tma_load_2d(su32(sB + s * TILE_BYTES), &tmB, full, k, n0);
      }
      issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = idesc_tf32(BM, BN, B_MN);
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      const uint32_t ready = SPLIT ? su32(&bars[2 * STAGES + 1 + s]) : su32(&bars[s]);
      if (*abort_flag || !mbar_wait(ready, ph)) {
        *abort_flag = 1;
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_base = su32(sA + s * TILE_BYTES);
      const uint32_t b_base = su32(sB + s * TILE_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / 8; ++kk) {
        // K-major: advance 8 tf32 = 32 bytes inside the swizzle span; SBO = 8 rows x 128 B
        const uint64_t ad = sdesc(a_base + kk * 32, 16, 1024);
        uint64_t bd;
        if (B_MN) bd = sdesc(b_base + kk * 1024, BK * 128, 1024);  // 8 k-rows per step; LBO = n-chunk stride
        else bd = sdesc(b_base + kk * 32, 16, 1024);
        mma_tf32(tmem, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        if (SPLIT) {  // + A_hi B_lo + A_lo B_hi (the tensor core truncates A, B to their TF32 high parts)
          const uint64_t bdl = sdesc(su32(sBl + s * TILE_BYTES) + kk * 32, 16, 1024);
          const uint64_t adl = sdesc(su32(sAl + s * TILE_BYTES) + kk * 32, 16, 1024);
          mma_tf32(tmem, ad, bdl, idesc, 1u);
          mma_tf32(tmem, adl, bd, idesc, 1u);
        }
      }
      mma_commit(su32(&bars[STAGES + s]));  // frees the stage once these MMAs have read it
    }
    if (ok) mma_commit(su32(&bars[2 * STAGES]));
  } else if (SPLIT && warp >= 2) {
    // ---------------- splitters: lo = x - tf32(x) for the A and B tiles of each stage
    const int t = threadIdx.x - 64;  // 0..63
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (*abort_flag || !mbar_wait(su32(&bars[s]), ph)) {
        *abort_flag = 1;
        break;
      }
      const uint4* a = (const uint4*)(sA + s * TILE_BYTES);
      const uint4* b = (const uint4*)(sB + s * TILE_BYTES);
      float4* al = (float4*)(sAl + s * TILE_BYTES);
      float4* bl = (float4*)(sBl + s * TILE_BYTES);
#pragma unroll 4
      for (int i = t; i < TILE_BYTES / 16; i += 64) {
        const uint4 x = a[i], y = b[i];
        float4 xl, yl;
        xl.x = __uint_as_float(x.x) - __uint_as_float(x.x & 0xFFFFE000u);
        xl.y = __uint_as_float(x.y) - __uint_as_float(x.y & 0xFFFFE000u);
        xl.z = __uint_as_float(x.z) - __uint_as_float(x.z & 0xFFFFE000u);
        xl.w = __uint_as_float(x.w) - __uint_as_float(x.w & 0xFFFFE000u);
        yl.x = __uint_as_float(y.x) - __uint_as_float(y.x & 0xFFFFE000u);
        yl.y = __uint_as_float(y.y) - __uint_as_float(y.y & 0xFFFFE000u);
        yl.z = __uint_as_float(y.z) - __uint_as_float(y.z & 0xFFFFE000u);
        yl.w = __uint_as_float(y.w) - __uint_as_float(y.w & 0xFFFFE000u);
        al[i] = xl;
        bl[i] = yl;
      }
      // generic-proxy writes -> visible to the tensor core (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if ((threadIdx.x & 31) == 0) {
        uint64_t st;
        asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(st) : "r"(su32(&bars[2 * STAGES + 1 + s])) : "memory");
      }
    }
  }
  __syncwarp();
  // ---------------- epilogue: all four warps, warp w owns accumulator rows 32w..32w+31
  bool have = false;
  if (nk > 0) have = mbar_wait(su32(&bars[2 * STAGES]), 0) && !*abort_flag;
  have = __syncthreads_and(have);  // uniform: the epilogue below synchronises the CTA
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (have) {
    const int m = m0 + warp * 32 + lane;
    float* wrow = ws ? ws + (size_t)blockIdx.z * M * N + (size_t)m * N : nullptr;
    // A lane holds one accumulator row. Outputs whose consecutive columns are adjacent in memory
    // (the split-K partials, and C when its column map has unit inner stride) are written from a
    // transposed copy in shared memory instead (the pipeline stages are idle by now), so that the
    // lanes of a warp store 32 consecutive columns of one row: one 128-byte segment per store
    float* tbuf = (float*)smem + warp * 32 * 33;
    const bool c_cols = ws != nullptr || cn.s2 == 1;
    const bool c2_cols = C2 && cn2.s2 == 1;
    // output offsets of the tile's rows and columns, evaluated once per CTA
    long long* roff = (long long*)(smem + 4 * 32 * 33 * sizeof(float));
    long long *roff2 = roff + BM, *coff = roff + 2 * BM, *coff2 = roff + 3 * BM;
    {
      const int t = threadIdx.x;
      const bool mr = m0 + t < M, nr = n0 + t < N;
      roff[t] = (!ws && mr) ? cm(m0 + t) : 0;
      roff2[t] = (C2 && mr) ? cm2(m0 + t) : 0;
      coff[t] = (!ws && nr) ? cn(n0 + t) : 0;
      coff2[t] = (C2 && nr) ? cn2(n0 + t) : 0;
    }
    __syncthreads();
    const long long crow = roff[warp * 32 + lane], crow2 = roff2[warp * 32 + lane];
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c, r);
      if (c_cols || c2_cols) {
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 32; ++j) tbuf[lane * 33 + j] = __uint_as_float(r[j]);
        __syncwarp();
        const int n = n0 + c + lane;
        if (n < N) {
          const long long ccol = coff[c + lane], ccol2 = coff2[c + lane];
#pragma unroll 4
          for (int i = 0; i < 32; ++i) {
            const int mi = m0 + warp * 32 + i;
            if (mi >= M) break;
            const float v = tbuf[i * 33 + lane];
            if (ws) {
              ws[((size_t)blockIdx.z * M + mi) * N + n] = v;
              continue;
            }
            const float out = alpha * v;
            if (c2_cols) C2[roff2[warp * 32 + i] + ccol2] = out;
            if (c_cols) {
              const long long o = roff[warp * 32 + i] + ccol;
              C[o] = beta != 0.f ? out + beta * C[o] : out;
            }
          }
        }
      }
      if (m < M && !ws && (!c_cols || (C2 && !c2_cols))) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + c + j;
          if (n < N) {
            const float out = alpha * __uint_as_float(r[j]);
            if (C2 && !c2_cols) C2[crow2 + coff2[c + j]] = out;
            if (!c_cols) {
              const long long o = crow + coff[c + j];
              C[o] = beta != 0.f ? out + beta * C[o] : out;
            }
          }
        }
      }
    }
    (void)wrow;
  } else if (nk > 0 && threadIdx.x == 0 && errw) {
    atomicOr(errw, ERRW_TIMEOUT);
  }
  if (nk == 0 && ws == nullptr) {  // empty K range: C = beta * C
    const int m = m0 + warp * 32 + lane;
    if (m < M)
      for (int j = 0; j < BN; ++j) {
        const int n = n0 + j;
        if (n < N) {
          const long long o = cm(m) + cn(n);
          C[o] = beta != 0.f ? beta * C[o] : 0.f;
          if (C2) C2[cm2(m) + cn2(n)] = 0.f;
        }
      }
  } else if (nk == 0 && ws) {
    const int m = m0 + warp * 32 + lane;
    if (m < M)
      for (int j = 0; j < BN; ++j)
        if (n0 + j < N) ws[(size_t)blockIdx.z * M * N + (size_t)m * N + n0 + j] = 0.f;
  }
  // drain any TMA still in flight after an abort (bounded), then free tensor memory
  if (warp == 0 && lane == 0 && *abort_flag) {
    for (int kb = 0; kb < issued; ++kb) mbar_wait(su32(&bars[kb % STAGES]), (kb / STAGES) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

bool make_map(CUtensorMap* map, const void* ptr, uint64_t inner, uint64_t outer, uint64_t row_stride_elems,
              uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B,
              CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32, int elem_bytes = 4) {
  auto enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_stride_elems * (uint64_t)elem_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(map, dt, 2, (void*)ptr, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

inline bool lin_stride(const IdxMap& m, long long& s) {
  if (m.n1 == 1 && m.n2 == (1 << 30) && m.s0 == 0 && m.s1 == 0) {
    s = m.s2;
    return true;
  }
  return false;
}

// ---------------------------------------------------------------------------
// FP64-class products on the TF32 tensor cores (Ozaki-type fixed-point split).
// Every row of an operand is cut into chunks of OZ_KC columns; a chunk with
// max |x| < 2^e is written as x = 2^e sum_i s_i 2^(-7-8i), i < OZ_S, with
// integer digits |s_i| <= 128 (stored as s_i 2^(-8i), exact in TF32). A
// product of two chunks is then 2^(eA+eB-14) sum over digit pairs (i, j) of
// 2^(-8(i+j)) sum_k sA_i sB_j. Pairs with i + j < OZ_S are kept (the dropped ones
// weigh <= 2^-48 of the largest term). Level 0 (i = j = 0) and level 1 sum
// integers of <= 2^14 (resp. 2^15 in units of 2^-8) over <= 512 terms, so their
// FP32 accumulators in tensor memory are exact (checked on integer inputs: the
// products come out exact); level 2 has an accumulator of its own (rounding
// weighted 2^-16 x 2^-24) and levels >= 3 share the fourth. The epilogue joins
// the four in double-FP32 and scales by the chunk exponents; the chunks of K
// are the split-K partials, summed in double-FP32 by splitk_reduce.
//
// The digits are integers of at most 8 significant bits times a power of two,
// so they are exact in BF16 as well. The same split then runs on kind::f16
// MMAs with BF16 digit planes: 16 digits of K per instruction instead of 8 at
// the same issue cost (the BF16 tensor rate is twice the TF32 one), and half
// the bytes per plane to write, load and stage.
// ---------------------------------------------------------------------------
constexpr int OZ_S = 6;
constexpr int OZ_KC = 512;
constexpr int OZ_TILES = 2 * OZ_S;
// k-blocks of 64 bytes (the 64-byte swizzle span: 16 TF32 or 32 BF16 digits), so that two stages of
// the 12 digit tiles (2 x 96 KB) fit in shared memory and the TMA of one k-block overlaps the MMAs of
// the other; each MMA takes 32 bytes of K
constexpr int OZ_KBYTES = 64;
constexpr int OZ_TILE = BM * OZ_KBYTES;  // 8 KB
constexpr int OZ_STAGES = 2;
constexpr int OZ_SMEM = OZ_STAGES * OZ_TILES * OZ_TILE + 1024 + 256;
constexpr int OZ_EZERO = -1000;  // exponent of an all-zero chunk

// digits of one operand: X [R][K] (row stride ld, K contiguous) -> sl [OZ_S][R][Kp], ex [R][nch]
template <typename T>
__device__ __forceinline__ float2 as_pair(T x);
template <>
__device__ __forceinline__ float2 as_pair<df32>(df32 x) { return make_float2(x.hi, x.lo); }
template <>
__device__ __forceinline__ float2 as_pair<float>(float x) { return make_float2(x, 0.f); }
// a digit in its plane's type (exact in both: at most 8 significant bits)
template <typename D>
__device__ __forceinline__ D as_digit(float d);
template <>
__device__ __forceinline__ float as_digit<float>(float d) { return d; }
template <>
__device__ __forceinline__ __nv_bfloat16 as_digit<__nv_bfloat16>(float d) { return __float2bfloat16_rn(d); }

template <typename T, typename D>
__global__ void oz_slice_kernel(int R, int K, int Kp, const T* __restrict__ X, long long ld, D* __restrict__ sl,
                                int* __restrict__ ex, int nch) {
  const int lane = threadIdx.x & 31;
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (gw >= (long long)R * nch) return;
  const int row = (int)(gw / nch), ch = (int)(gw % nch);
  const int k0 = ch * OZ_KC, k1 = min(K, k0 + OZ_KC), kp1 = min(Kp, k0 + OZ_KC);
  const T* x = X + row * ld;
  int e = INT_MIN;
  for (int k = k0 + lane; k < k1; k += 32) {
    const float h = as_pair<T>(x[k]).x;
    if (h != 0.f) e = max(e, ((__float_as_int(h) >> 23) & 0xFF) - 126);  // |h| < 2^e
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (e == INT_MIN) e = OZ_EZERO;
  if (lane == 0) ex[(long long)row * nch + ch] = e;
  const size_t plane = (size_t)R * Kp;
  for (int k = k0 + lane; k < kp1; k += 32) {
    float d[OZ_S];
    if (k < K) {
      const float2 v = as_pair<T>(x[k]);
      // x 2^(7-e) = th + tl exactly; peel one 8-bit digit per level, carrying the exact remainder
      float th = scalbnf(v.x, 7 - e), tl = scalbnf(v.y, 7 - e);
#pragma unroll
      for (int i = 0; i < OZ_S; ++i) {
        const float si = rintf(th);
        d[i] = scalbnf(si, -8 * i);
        const df32 r = two_sum(__fsub_rn(th, si), tl);  // th - si is exact
        th = __fmul_rn(r.hi, 256.f);
        tl = __fmul_rn(r.lo, 256.f);
      }
    } else {
#pragma unroll
      for (int i = 0; i < OZ_S; ++i) d[i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) sl[i * plane + (size_t)row * Kp + k] = as_digit<D>(d[i]);
  }
}

template <typename D>
__device__ __forceinline__ void oz_mma(uint32_t tmem, uint64_t ad, uint64_t bd, bool acc) {
  if constexpr (sizeof(D) == 2)
    mma_bf16(tmem, ad, bd, idesc_bf16(BM, BN), acc ? 1u : 0u);
  else
    mma_tf32(tmem, ad, bd, idesc_tf32(BM, BN, false), acc ? 1u : 0u);
}

// One 128 x 128 output tile of one K-chunk (blockIdx.z) into the double-FP32
// partial ws[z][M][N]. Warp 0: TMA producer; warp 1: tensor-memory owner and
// MMA issuer; all four warps: epilogue. A stage holds the 2 OZ_S digit tiles of
// a 64-byte k-block (96 KB); two stages alternate, so the loads of one k-block
// run under the 42 MMAs of the other. The four accumulators fill the 512
// tensor-memory columns. D: the digit type (float: kind::tf32, BF16: kind::f16).
template <typename D>
__global__ void __launch_bounds__(128, 1)
    gemm_oz_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
                   int K, const int* __restrict__ eA, const int* __restrict__ eB, int nch, df32* __restrict__ ws,
                   uint32_t* errw) {
  constexpr int KB = OZ_KBYTES / (int)sizeof(D);  // digits of K per k-block
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // [0, 1] full, [2, 3] empty (per stage), [4] accumulators ready
  uint64_t* bars = (uint64_t*)(smem + OZ_STAGES * OZ_TILES * OZ_TILE);
  uint32_t* tmem_slot = (uint32_t*)(bars + 5);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN, z = blockIdx.z;
  const int kb0 = z * OZ_KC, kend = min(K, kb0 + OZ_KC);
  const int nk = (kend - kb0 + KB - 1) / KB;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 5; ++b) mbar_init(su32(&bars[b]), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  int issued = 0;
  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < nk; ++kb) {
      const int st = kb & 1;
      if (*abort_flag || !mbar_wait(su32(&bars[2 + st]), ((kb >> 1) & 1) ^ 1)) {
        *abort_flag = 1;
        break;
      }
      const uint32_t full = su32(&bars[st]);
      mbar_expect_tx(full, OZ_TILES * OZ_TILE);
      const int k = kb0 + kb * KB;
      uint8_t* base = smem + st * OZ_TILES * OZ_TILE;
#pragma unroll
      for (int i = 0; i < OZ_S; ++i) {
        tma_load_2d(su32(base + i * OZ_TILE), &tmA, full, k, i * M + m0);
        tma_load_2d(su32(base + (OZ_S + i) * OZ_TILE), &tmB, full, k, i * N + n0);
      }
      issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {
    bool started[4] = {false, false, false, false};
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int st = kb & 1;
      if (*abort_flag || !mbar_wait(su32(&bars[st]), (kb >> 1) & 1)) {
        *abort_flag = 1;
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint8_t* base = smem + st * OZ_TILES * OZ_TILE;
#pragma unroll
      for (int i = 0; i < OZ_S; ++i)
#pragma unroll
        for (int j = 0; j + i < OZ_S; ++j) {
          const int lev = min(i + j, 3);
          const uint32_t a_base = su32(base + i * OZ_TILE), b_base = su32(base + (OZ_S + j) * OZ_TILE);
#pragma unroll
          for (int kk = 0; kk < OZ_KBYTES / 32; ++kk) {
            oz_mma<D>(tmem + lev * BN, sdesc64(a_base + kk * 32, 16, 512), sdesc64(b_base + kk * 32, 16, 512),
                      started[lev]);
            started[lev] = true;
          }
        }
      mma_commit(su32(&bars[2 + st]));  // frees the stage once these MMAs have read it
    }
    if (ok) mma_commit(su32(&bars[4]));
  }
  __syncwarp();
  bool have = false;
  if (nk > 0) have = mbar_wait(su32(&bars[4]), 0) && !*abort_flag;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int m = m0 + warp * 32 + lane;
  df32* wrow = ws + ((size_t)z * M + (m < M ? m : 0)) * N;
  const int ea = (m < M) ? eA[(size_t)m * nch + z] : OZ_EZERO;
  if (have) {
    // a lane holds one row; the combined values go through a transposed copy in shared memory (the
    // stages are idle by now), so that a warp stores 32 consecutive df32 of one row at a time
    df32* tbuf = (df32*)smem + warp * 32 * 33;
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
      uint32_t r0[32], r1[32], r2[32], r3[32];
      const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16) + c;
      tmem_ld32(base, r0);
      tmem_ld32(base + BN, r1);
      tmem_ld32(base + 2 * BN, r2);
      tmem_ld32(base + 3 * BN, r3);
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const df32 s = two_sum(__uint_as_float(r0[t]), __uint_as_float(r1[t]));
        const df32 u = two_sum(s.hi, __uint_as_float(r2[t]));
        const df32 u2 = two_sum(u.hi, __uint_as_float(r3[t]));
        tbuf[lane * 33 + t] = renorm(u2.hi, __fadd_rn(__fadd_rn(u2.lo, u.lo), s.lo));
      }
      __syncwarp();
      const int n = n0 + c + lane;
      if (n < N) {
        const int eb = eB[(size_t)n * nch + z];
#pragma unroll 4
        for (int i = 0; i < 32; ++i) {
          const int mi = m0 + warp * 32 + i;
          if (mi >= M) break;
          const df32 v = tbuf[i * 33 + lane];
          const int sc = max(eA[(size_t)mi * nch + z] + eb - 14, -2 * 1000);
          ws[((size_t)z * M + mi) * N + n] = df32(scalbnf(v.hi, sc), scalbnf(v.lo, sc));
        }
      }
    }
    (void)ea;
  } else if (nk > 0 && threadIdx.x == 0 && errw) {
    atomicOr(errw, ERRW_TIMEOUT);
  }
  if (nk == 0 && m < M)
    for (int n = n0; n < min(N, n0 + BN); ++n) wrow[n] = df32(0.f, 0.f);
  if (warp == 0 && lane == 0 && *abort_flag)  // drain the loads still in flight (bounded waits)
    for (int kb = 0; kb < issued; ++kb) mbar_wait(su32(&bars[kb & 1]), (kb >> 1) & 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

}  // namespace tc

// Returns cudaErrorNotSupported when the operand layouts cannot be fed by TMA
// (the caller then uses the CUDA-core kernel).
cudaError_t gemm_tf32(const GemmArgs<float>& g, float* ws, size_t ws_elems, int sm_count, uint32_t* errw,
                      cudaStream_t st, bool split) {
  using namespace tc;
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  long long lda, ldb, one;
  if (!lin_stride(g.am, lda) || !lin_stride(g.ak, one) || one != 1) return cudaErrorNotSupported;
  // B must be K-major: an MN-major B with kind::tf32 produced an all-zero
  // accumulator in the self-check, so such layouts go to the CUDA-core kernel.
  bool b_mn = false;
  if (!(lin_stride(g.bk, one) && one == 1 && lin_stride(g.bn, ldb))) return cudaErrorNotSupported;
  // TMA: 16-byte aligned bases and row strides
  if (((uintptr_t)g.A & 15) || ((uintptr_t)g.B & 15) || (lda * 4) % 16 || (ldb * 4) % 16) return cudaErrorNotSupported;
  if (lda < g.K || (!b_mn && ldb < g.K) || (b_mn && ldb < g.N)) return cudaErrorNotSupported;
  if (g.K < 1) return cudaErrorNotSupported;
  CUtensorMap ta, tb;
  if (!make_map(&ta, g.A, (uint64_t)g.K, (uint64_t)g.M, (uint64_t)lda, BK, BM)) return cudaErrorNotSupported;
  if (!b_mn) {
    if (!make_map(&tb, g.B, (uint64_t)g.K, (uint64_t)g.N, (uint64_t)ldb, BK, BN)) return cudaErrorNotSupported;
  } else {
    if (!make_map(&tb, g.B, (uint64_t)g.N, (uint64_t)g.K, (uint64_t)ldb, 32, BK)) return cudaErrorNotSupported;
  }
  cudaError_t ea = split ? ensure_smem((const void*)gemm_tf32_kernel<false, true>, Cfg<true>::SMEM_BYTES)
                         : ensure_smem((const void*)gemm_tf32_kernel<false, false>, Cfg<false>::SMEM_BYTES);
  if (ea != cudaSuccess) return ea;
  const int gm = (g.M + BM - 1) / BM, gn = (g.N + BN - 1) / BN;
  int splits = 1;
  while (gm * gn * splits < sm_count && g.K / (splits * 2) >= 4 * BK && (size_t)(splits * 2) * g.M * g.N <= ws_elems)
    splits *= 2;
  int kps = (g.K + splits - 1) / splits;
  kps = (kps + BK - 1) / BK * BK;
  splits = (g.K + kps - 1) / kps;
  dim3 grid(gn, gm, splits);
  float* wsp = splits > 1 ? ws : nullptr;
  ++tl_launches;
  if (split)
    gemm_tf32_kernel<false, true><<<grid, 128, Cfg<true>::SMEM_BYTES, st>>>(
        ta, tb, g.M, g.N, g.K, kps, g.C, g.cm, g.cn, g.alpha, g.beta, g.C2, g.cm2, g.cn2, wsp, errw);
  else
    gemm_tf32_kernel<false, false><<<grid, 128, Cfg<false>::SMEM_BYTES, st>>>(
        ta, tb, g.M, g.N, g.K, kps, g.C, g.cm, g.cn, g.alpha, g.beta, g.C2, g.cm2, g.cn2, wsp, errw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  return splitk_reduce<float>(g, ws, splits, sm_count, st);
}

// FP64-class GEMM (double-FP32 operands and result) on the tensor cores by the
// fixed-point digit split above: TF32 digit planes on kind::tf32, or BF16
// digit planes on kind::f16 (bf16 = true). Operands must be K-major with
// 16-byte aligned rows after padding, like gemm_tf32. sA, sB: digit planes,
// OZ_S * M * Kp and OZ_S * N * Kp digits, in buffers of slice_elems floats
// each; eA, eB: M * nch and N * nch ints; ws: nch * M * N double-FP32
// partials. Returns cudaErrorNotSupported when a layout or a capacity does not
// fit (the caller then uses the CUDA-core kernel).
cudaError_t gemm_oz(const GemmArgs<df32>& g, float* sA, float* sB, size_t slice_elems, int* eA, int* eB,
                    size_t exp_elems, df32* ws, size_t ws_elems, int sm_count, uint32_t* errw, cudaStream_t st,
                    bool bf16) {
  using namespace tc;
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.K < 1) return cudaErrorNotSupported;
  long long lda, ldb, one;
  if (!lin_stride(g.am, lda) || !lin_stride(g.ak, one) || one != 1) return cudaErrorNotSupported;
  if (!lin_stride(g.bk, one) || one != 1 || !lin_stride(g.bn, ldb)) return cudaErrorNotSupported;
  const int eb = bf16 ? 2 : 4;                         // bytes per digit
  const int Kp = (g.K + 16 / eb - 1) / (16 / eb) * (16 / eb);  // 16-byte rows of digits
  const int nch = (g.K + OZ_KC - 1) / OZ_KC;
  const size_t cap = slice_elems * sizeof(float);
  if ((size_t)OZ_S * g.M * Kp * eb > cap || (size_t)OZ_S * g.N * Kp * eb > cap) return cudaErrorNotSupported;
  if ((size_t)g.M * nch > exp_elems || (size_t)g.N * nch > exp_elems) return cudaErrorNotSupported;
  if ((size_t)nch * g.M * g.N > ws_elems) return cudaErrorNotSupported;
  auto slice = [&](int R, const df32* X, long long ld, float* sl, int* ex) {
    const long long warps = (long long)R * nch;
    const int blocks = (int)((warps * 32 + 255) / 256);
    ++tl_launches;
    if (bf16)
      oz_slice_kernel<df32, __nv_bfloat16><<<blocks, 256, 0, st>>>(R, g.K, Kp, X, ld, (__nv_bfloat16*)sl, ex, nch);
    else
      oz_slice_kernel<df32, float><<<blocks, 256, 0, st>>>(R, g.K, Kp, X, ld, sl, ex, nch);
    return cudaGetLastError();
  };
  cudaError_t e = slice(g.M, g.A, lda, sA, eA);
  if (e != cudaSuccess) return e;
  if ((e = slice(g.N, g.B, ldb, sB, eB)) != cudaSuccess) return e;
  CUtensorMap ta, tb;
  const CUtensorMapDataType dt = bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const uint32_t kb = OZ_KBYTES / eb;
  if (!make_map(&ta, sA, (uint64_t)Kp, (uint64_t)OZ_S * g.M, (uint64_t)Kp, kb, BM, CU_TENSOR_MAP_SWIZZLE_64B, dt, eb))
    return cudaErrorNotSupported;
  if (!make_map(&tb, sB, (uint64_t)Kp, (uint64_t)OZ_S * g.N, (uint64_t)Kp, kb, BN, CU_TENSOR_MAP_SWIZZLE_64B, dt, eb))
    return cudaErrorNotSupported;
  const void* kern = bf16 ? (const void*)gemm_oz_kernel<__nv_bfloat16> : (const void*)gemm_oz_kernel<float>;
  if ((e = ensure_smem(kern, OZ_SMEM)) != cudaSuccess) return e;
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, nch);
  ++tl_launches;
  if (bf16)
    gemm_oz_kernel<__nv_bfloat16><<<grid, 128, OZ_SMEM, st>>>(ta, tb, g.M, g.N, g.K, eA, eB, nch, ws, errw);
  else
    gemm_oz_kernel<float><<<grid, 128, OZ_SMEM, st>>>(ta, tb, g.M, g.N, g.K, eA, eB, nch, ws, errw);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return splitk_reduce<df32>(g, ws, nch, sm_count, st);
}

}  // namespace ttfit
