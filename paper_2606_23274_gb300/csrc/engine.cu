// Host driver of the variational MPO-MPO fit and its C ABI (include/ttfit.h).
//
// Sweep schedule (Alg. 5): right environments R_L..R_3 are precomputed; a
// forward step at window (l, l+1) finishes L_{l-1} from the cached half
// H1_{l-1} = L_{l-2} A_{l-1} B_{l-1} and the new C_{l-1}, builds the fresh half
// H1_l = L_{l-1} A_l B_l, joins it with the cached H2_{l+1} = A_{l+1} B_{l+1} R_{l+2}
// into the two-site tensor (Fig. derivatives (d)), factorises it and applies
// Alg. 3 or Alg. 4. The backward step mirrors this. Each environment is thus
// the paper's three-diagram contraction (Fig. envs) split as "half" (first two
// diagrams, shared with the two-site tensor) and "finish" (third diagram).
#include <cuda_runtime.h>
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <new>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/ttfit.h"
#include "common.cuh"
#include "kernels.h"

using namespace ttfit;

namespace {

struct TTError : std::runtime_error {
  tt_status code;
  TTError(tt_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define CK(...)                                                                                      \
  do {                                                                                               \
    cudaError_t e_ = (__VA_ARGS__);                                                                  \
    if (e_ != cudaSuccess)                                                                           \
      throw TTError(e_ == cudaErrorMemoryAllocation ? TT_ERR_OUT_OF_MEMORY : TT_ERR_CUDA,             \
                    std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));                                \
  } while (0)

// Process-wide cache of device blocks, by device and size (rounded up to 512
// bytes). A handle takes the smallest cached block of at least the size it asks
// for and at most twice that (best fit, so that fits of uneven shapes reuse each
// other's blocks), or allocates a new one; on allocation failure every cached
// block of the device is freed and the allocation retried. Released blocks return
// to the cache (cudaFree would also synchronise the whole device) while the cache
// holds at most a quarter of the device's memory (and at most 64 GiB); beyond
// that a released block is freed. tt_device_cache_release frees the cache. A
// block is released only after the streams that used it have been synchronised
// (the preparation streams, the handle's lanes), so a block handed out again is idle.
struct BlockCache {
  static constexpr size_t kCapMax = size_t(64) << 30;
  std::mutex mu;
  std::vector<std::pair<std::pair<int, size_t>, void*>> free_blocks;
  std::map<int, size_t> cached;  // bytes held per device
  std::map<int, size_t> cap;     // per device: min(kCapMax, total memory / 4)
  void* take(int dev, size_t bytes, size_t* got) {
    std::lock_guard<std::mutex> g(mu);
    size_t best = 0;
    for (size_t i = 0; i < free_blocks.size(); ++i) {
      const auto& fb = free_blocks[i].first;
      if (fb.first == dev && fb.second >= bytes && fb.second <= 2 * bytes &&
          (best == 0 || fb.second < free_blocks[best - 1].first.second))
        best = i + 1;
    }
    if (!best) return nullptr;
    const size_t i = best - 1;
    void* p = free_blocks[i].second;
    *got = free_blocks[i].first.second;
    free_blocks[i] = free_blocks.back();
    free_blocks.pop_back();
    cached[dev] -= *got;
    return p;
  }
  void give(int dev, size_t bytes, void* p) {
    {
      std::lock_guard<std::mutex> g(mu);
      auto it = cap.find(dev);
      if (it == cap.end()) {
        size_t fr = 0, tot = 0;
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(dev);
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
          cudaGetLastError();
          tot = 0;
        }
        cudaSetDevice(cur);
        it = cap.emplace(dev, std::min(kCapMax, tot / 4)).first;
      }
      if (cached[dev] + bytes <= it->second) {
        free_blocks.push_back({{dev, bytes}, p});
        cached[dev] += bytes;
        return;
      }
    }
    cudaFree(p);
  }
  size_t trim(int dev) {  // dev < 0: every device; returns the bytes freed
    std::vector<std::pair<std::pair<int, size_t>, void*>> drop;
    {
      std::lock_guard<std::mutex> g(mu);
      for (size_t i = 0; i < free_blocks.size();)
        if (dev < 0 || free_blocks[i].first.first == dev) {
          drop.push_back(free_blocks[i]);
          cached[free_blocks[i].first.first] -= free_blocks[i].first.second;
          free_blocks[i] = free_blocks.back();
          free_blocks.pop_back();
        } else {
          ++i;
        }
    }
    if (drop.empty()) return 0;
    int cur = 0;
    cudaGetDevice(&cur);
    size_t bytes = 0;
    for (auto& d : drop) {
      cudaSetDevice(d.first.first);
      cudaFree(d.second);
      bytes += d.first.second;
    }
    cudaSetDevice(cur);
    return bytes;
  }
};

BlockCache& block_cache() {
  static BlockCache* c = new BlockCache;  // lives for the process; the driver reclaims device memory at exit
  return *c;
}

// Device allocations owned by a handle (from the block cache).
struct DevPool {
  struct Blk {
    void* p;
    size_t bytes;
    int dev;
  };
  std::vector<Blk> blks;
  uint32_t fault = 0;
  template <typename T>
  T* alloc(size_t n) {
    if (fault & TT_FAULT_ALLOC_FAIL) throw TTError(TT_ERR_OUT_OF_MEMORY, "injected allocation failure");
    if (n == 0) n = 1;
    const size_t bytes = (n * sizeof(T) + 511) & ~(size_t)511;
    int dev = 0;
    cudaGetDevice(&dev);
    size_t got = bytes;
    void* p = block_cache().take(dev, bytes, &got);
    if (!p) {
      cudaError_t e = cudaMalloc(&p, bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        block_cache().trim(dev);
        e = cudaMalloc(&p, bytes);
      }
      if (e != cudaSuccess) {
        cudaGetLastError();
        throw TTError(TT_ERR_OUT_OF_MEMORY, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
      }
    }
    blks.push_back({p, p ? got : bytes, dev});
    return (T*)p;
  }
  void release(void* p) {
    for (auto& b : blks)
      if (b.p == p) {
        block_cache().give(b.dev, b.bytes, b.p);
        b.p = nullptr;
      }
  }
  ~DevPool() {
    for (auto& b : blks)
      if (b.p) block_cache().give(b.dev, b.bytes, b.p);
  }
};

struct Dims {
  int L = 0;
  std::vector<int> ds, du, dt;  // per site: A out, A in (= B out), B in
  std::vector<int> a, b, c;     // bonds 0..L of A, B, C (current)
  std::vector<int> cb;          // capacity of C bonds (buffer sizes)
};

}  // namespace

// Working state of one sweep lane: the stream it runs on, its events and
// timers, the scratch of the chain and of the factorisation, and the pinned
// host mirrors of its device flags. The handle owns one; a segment-parallel
// fit owns one more per segment, so that segments run concurrently.
struct Work {
  cudaStream_t st = nullptr;
  bool own_stream = false;
  cudaEvent_t ev[10] = {};     // window stages (0..4), gauge update (5, 6), lane join (7), connection finish (8, 9)
  bool gauge_pending = false;  // ev[5], ev[6] recorded but not yet read
  bool connect_pending = false;  // ev[8], ev[9] recorded but not yet read
  double stage_ms[5] = {0, 0, 0, 0, 0};
  double flops = 0;
  // the chain contractions as issued: tensor-core MMA flops (split passes, digit pairs and tile
  // padding included) and CUDA-core flops
  double tc_flops = 0, cc_flops = 0;
  void *X1 = nullptr, *Zs = nullptr, *Th = nullptr, *gws = nullptr;
  size_t gws_elems = 0;
  // factorisation workspace (FP64-sized)
  double *fX = nullptr, *fQ = nullptr, *fR = nullptr, *fU = nullptr, *fV = nullptr, *fVw = nullptr, *fS = nullptr;
  double *fUM = nullptr, *fVM = nullptr, *fOm = nullptr, *fY = nullptr, *fBt = nullptr, *fQ2 = nullptr, *fR2 = nullptr;
  double *pU = nullptr, *pV = nullptr, *pG = nullptr, *pT = nullptr, *pP = nullptr;  // FP64 polish
  // digit planes, chunk exponents and partials of the tensor-core FP64-class GEMM (DF32 chains)
  float *ozA = nullptr, *ozB = nullptr;
  int *ozEA = nullptr, *ozEB = nullptr;
  df32* ozWs = nullptr;
  size_t oz_slice = 0, oz_exp = 0, oz_ws = 0;
  size_t fsz = 0;
  bool hp = false;      // the last factorisation used the FP64-class sketch basis (factors in df32)
  bool hp_off = false;  // fall back to the all-FP32 factorisation for the current window
  long long hp_fallbacks = 0;  // windows that fell back (diagnostic)
  double* dnorm = nullptr;
  int* dk = nullptr;
  double* ddinfo = nullptr;
  uint32_t* errw = nullptr;
  int* hk = nullptr;  // pinned host mirrors
  double* hdinfo = nullptr;
  uint32_t* herrw = nullptr;
};

struct tt_fit {
  // configuration
  int L = 0, chi_max = 0, gauge = 0, update = 0, oversample = 10, precision = 0, init = 0;
  double tol = 0, cutoff = 1e-13, conv_tol = 0;
  bool cutoff_user = false;  // sv_cutoff given by the caller (else it follows the precision)
  uint64_t seed = 0;
  uint32_t fault = 0;
  int sm_count = 0;
  int device = 0;
  Dims D;
  DevPool pool;
  // prepared inputs, FP64 natural layout
  std::vector<double*> A64, B64;
  // C (site gauge: C_l; inverse gauge: Psi_l), natural layout, FP64; Y per bond
  std::vector<double*> C64, Y;
  std::vector<std::vector<double>> lam;  // singular values of the last update per bond
  // contraction tensors in the working type (float or double)
  std::vector<void*> Aop, Anat, Bl, Br, Lenv, Renv, H1, H2, H1t, H2t, Ut, Vt;
  double* dn2 = nullptr;  // per window: ||C||^2 of the last polished update (FP64)
  Work w0;                                 // the handle's own lane (its stream is the caller's)
  std::vector<std::unique_ptr<Work>> wseg;  // one lane per segment (segment-parallel fit)
  // segment-parallel fit (Alg. 6): 0-based inclusive site ranges
  std::vector<std::pair<int, int>> segs;
  int phases_done = 0;
  // state
  int sweeps_done = 0;
  bool forward = true, converged = false, poisoned = false;
  double last_n2 = -1.0, delta = INFINITY, max_disc = 0.0;
  double cur_n2 = -1.0;  // ||C||^2 after the latest phase (segment-parallel fit)
  bool fault_nan_pending = false, fault_noconv_pending = false;
  std::string last_error;
  long long launches = 0, tc_launches = 0;  // monotonic since creation
  long long sweep_launches = 0;              // launches of the last tt_fit_sweep call
  bool have_times = false;
  bool use_f32 = false;   // chain type: float (FP32 / TF32 precisions), df32 (DF32) or double (FP64)
  bool use_df = false;
  bool fact_f32 = false;  // FP32 factorisation + FP64 polish (always for float chains; optional for FP64)
  int fast_factor = 0;    // tt_fit_options.fast_factor of the current precision (1, 3: FP64-class sketch basis)
  bool hp_sweep = false;  // the current sweep uses the FP64-class sketch basis (factorize_hp)
  int escale = 0;         // the fit runs on 2^-ea A, 2^-eb B; C, its spectra and norm get 2^escale back
  bool use_oz = true;     // DF32 chains: contractions on the tensor cores by the digit split
  bool oz_bf16 = false;   // ... with BF16 digit planes on kind::f16 (TT_PREC_BF16_SPLIT), else TF32 ones
  std::vector<void*> chain_bufs;  // buffers rebuilt when the chain precision changes
  // site-gauge segment-parallel fit: whether the sub-TTs have been merged since the last phase,
  // which phase ran last, and the orthogonality centre the merge left (-1: none)
  bool merged = true;
  int last_phase = 1;
  int oc_site = -1;
};

namespace {

// The lane the calling host thread works in: a segment thread sets it to its
// segment's lane; everywhere else it is the handle's own.
thread_local Work* tl_work = nullptr;
inline Work& W(tt_fit* h) { return tl_work ? *tl_work : h->w0; }
inline std::vector<Work*> lanes(tt_fit* h) {
  std::vector<Work*> v{&h->w0};
  for (auto& w : h->wseg) v.push_back(w.get());
  return v;
}

}  // namespace

namespace {

inline long long prodll(std::initializer_list<long long> v) {
  long long p = 1;
  for (auto x : v) p *= x;
  return p;
}

// ---------------------------------------------------------------------------
// small helpers on FP64 device matrices
// ---------------------------------------------------------------------------
// Contraction dispatch: the tensor-core kernel for TF32 chains whenever TMA can
// address both operands (16-byte aligned rows), the CUDA-core kernel otherwise
// (FP64 / FP32 chains, and the 1- or 2-wide bonds at the ends of the chain).
// Relative singular-value cut-off when the caller gives none: a little above
// the rounding level of the factorisation and of the contractions. An FP32
// factorisation resolves values down to ~1e-7 s_1 only; keeping smaller ones
// would feed its noise back into C.
inline double default_cutoff(int precision, bool fact_f32) {
  if (fact_f32) return 1e-6;
  return precision == TT_PREC_FP64 ? 1e-13 : precision == TT_PREC_DF32 ? 1e-12 : 1e-6;
}

// type of the exact factorisation for a chain type: FP64 for the FP64-class chains
template <typename T>
struct FactT {
  using type = T;
};
template <>
struct FactT<df32> {
  using type = double;
};

inline double round_up(long long x, long long m) { return (double)((x + m - 1) / m * m); }

template <typename T>
void gemm(tt_fit* h, const GemmArgs<T>& g, bool chain = false) {
  const size_t wse = W(h).gws_elems * sizeof(double) / sizeof(T);
  // MMA tiles are 128 x 128; K is issued in k-blocks, per 512-wide chunk for the digit split
  const double mn = round_up(g.M, 128) * round_up(g.N, 128);
  if constexpr (std::is_same<T, df32>::value) {
    Work& w = W(h);
    if (chain && h->use_oz && w.ozA && (long long)g.M * g.N * g.K >= (1ll << 21)) {
      cudaError_t e = gemm_oz(g, w.ozA, w.ozB, w.oz_slice, w.ozEA, w.ozEB, w.oz_exp, w.ozWs, w.oz_ws, h->sm_count,
                              w.errw, w.st, h->oz_bf16);
      if (e == cudaSuccess) {
        h->tc_launches += 1;
        const long long kc = OZ_CHUNK, kb = h->oz_bf16 ? 32 : 16;
        const double k_issued = (double)(g.K / kc * kc) + (g.K % kc ? round_up(g.K % kc, kb) : 0.0);
        const int pairs = OZ_DIGITS * (OZ_DIGITS + 1) / 2;  // digit pairs i + j < OZ_DIGITS
        w.tc_flops += 2.0 * mn * k_issued * pairs;
        return;
      }
      if (e != cudaErrorNotSupported) CK(e);
    }
  }
  if constexpr (sizeof(T) == 4) {
    const bool tc = h->precision == TT_PREC_TF32 || h->precision == TT_PREC_TF32_SPLIT;
    if (chain && tc && (long long)g.M * g.N * g.K >= (1ll << 18)) {
      cudaError_t e = gemm_tf32(g, (float*)W(h).gws, wse, h->sm_count, W(h).errw, W(h).st,
                                h->precision == TT_PREC_TF32_SPLIT);
      if (e == cudaSuccess) {
        h->tc_launches += 1;
        W(h).tc_flops += 2.0 * mn * round_up(g.K, 32) * (h->precision == TT_PREC_TF32_SPLIT ? 3 : 1);
        return;
      }
      if (e != cudaErrorNotSupported) CK(e);
    }
  }
  CK(gemm_simt<T>(g, (T*)W(h).gws, wse, h->sm_count, W(h).st));
  if (chain) W(h).cc_flops += 2.0 * g.M * g.N * g.K;
}

template <typename Tin, typename Tout>
void copymap(tt_fit* h, int rows, int cols, const Tin* in, IdxMap im, IdxMap in_, Tout* out, IdxMap om, IdxMap on,
             double scale = 1.0) {
  CK(copy_map<Tin, Tout>(rows, cols, in, im, in_, out, om, on, scale, W(h).st));
}

// QR on FP64 storage (input preparation and the guess): FP64 arithmetic; mixing
// FP32 arithmetic with FP64 storage is slower on this GPU (conversions run on
// the FP64 pipe).
void qr(tt_fit* h, int q, int p, double* X, double* Q, double* R) {
  CK(qr_householder<double, double>(q, p, X, Q, R, W(h).st));
}

// Row-major (rows x cols) -> column-major copy (ld rows).
void to_colmajor(tt_fit* h, int rows, int cols, const double* in, double* out) {
  copymap<double, double>(h, rows, cols, in, IdxMap::lin(cols), IdxMap::lin(1), out, IdxMap::lin(1), IdxMap::lin(rows));
}

// Input / guess preparation runs on its own stream with its own scratch, so
// that A and B are prepared concurrently; buffers that die during a sweep are
// released after the final synchronisation.
struct Prep {
  cudaStream_t st = nullptr;
  double *X = nullptr, *Q = nullptr, *R = nullptr, *ws = nullptr;
  size_t ws_elems = 0;
  std::vector<void*> dead;
};

// The FP64 path keeps FP64 arithmetic here; the others factorise in df32
// arithmetic (rounding ~1e-14, below what their sweeps resolve).
void prep_qr(tt_fit* h, Prep& P, int q, int p) {
  if (h->precision == TT_PREC_FP64) CK(qr_householder<double, double>(q, p, P.X, P.Q, P.R, P.st));
  else CK(qr_householder_df32(q, p, P.X, P.Q, P.R, P.st));
}

void prep_gemm(tt_fit* h, Prep& P, const GemmArgs<double>& g) {
  CK(gemm_simt<double>(g, P.ws, P.ws_elems, h->sm_count, P.st));
}

// Right-to-left RQ sweep: each core becomes the orthonormal-row factor of its
// transposed QR and the bond shrinks to min(rows, cols). With trim_only the
// sweep stops at the first step that trims nothing (bonds further left are
// then already within their bounds; the operator is the same either way).
void rq_sweep(tt_fit* h, Prep& P, std::vector<double*>& X, std::vector<int>& bond, const std::vector<int>& dA,
              const std::vector<int>& dB, int upto, bool trim_only) {
  const int L = (int)X.size();
  for (int j = L - 1; j >= upto; --j) {
    const int bl = bond[j], br = bond[j + 1], dd = dA[j] * dB[j];
    const int q = dd * br, p = bl, r = std::min(q, p);
    if (trim_only && r == bl) break;
    // core j row-major (bl x q) == column-major q x bl: QR of X_j^T
    CK(cudaMemcpyAsync(P.X, X[j], sizeof(double) * (size_t)q * p, cudaMemcpyDeviceToDevice, P.st));
    prep_qr(h, P, q, p);
    double* nc = h->pool.alloc<double>((size_t)r * q);
    CK(cudaMemcpyAsync(nc, P.Q, sizeof(double) * (size_t)q * r, cudaMemcpyDeviceToDevice, P.st));
    if (j > 0) {
      const int bl2 = bond[j - 1], dd2 = dA[j - 1] * dB[j - 1];
      double* np = h->pool.alloc<double>((size_t)bl2 * dd2 * r);
      GemmArgs<double> g;
      g.M = bl2 * dd2;
      g.N = r;
      g.K = bl;
      g.A = X[j - 1];
      g.am = IdxMap::lin(bl);
      g.ak = IdxMap::lin(1);
      g.B = P.R;
      g.bn = IdxMap::lin(1);
      g.bk = IdxMap::lin(r);
      g.b_kfast = false;
      g.C = np;
      g.cm = IdxMap::lin(r);
      g.cn = IdxMap::lin(1);
      prep_gemm(h, P, g);
      P.dead.push_back(X[j - 1]);
      X[j - 1] = np;
    }
    P.dead.push_back(X[j]);
    X[j] = nc;
    bond[j] = r;
  }
}

// Left-to-right QR sweep (Alg. 5 left_orthogonalize), bonds trimmed; QR steps at
// sites j0 .. j1 - 1 only when j1 >= 0.
void qr_sweep(tt_fit* h, Prep& P, std::vector<double*>& X, std::vector<int>& bond, const std::vector<int>& dA,
              const std::vector<int>& dB, int j0 = 0, int j1 = -1) {
  const int L = (int)X.size();
  for (int j = j0; j < (j1 >= 0 ? j1 : L - 1); ++j) {
    const int bl = bond[j], br = bond[j + 1], dd = dA[j] * dB[j];
    const int q = bl * dd, p = br, r = std::min(q, p);
    CK(copy_map<double, double>(q, p, X[j], IdxMap::lin(p), IdxMap::lin(1), P.X, IdxMap::lin(1), IdxMap::lin(q), 1.0,
                                P.st));
    prep_qr(h, P, q, p);
    double* nc = h->pool.alloc<double>((size_t)q * r);
    CK(copy_map<double, double>(q, r, P.Q, IdxMap::lin(1), IdxMap::lin(q), nc, IdxMap::lin(r), IdxMap::lin(1), 1.0,
                                P.st));
    const int dd2 = dA[j + 1] * dB[j + 1], br2 = bond[j + 2];
    const int N = dd2 * br2;
    double* nn = h->pool.alloc<double>((size_t)r * N);
    GemmArgs<double> g;
    g.M = r;
    g.N = N;
    g.K = br;
    g.A = P.R;
    g.am = IdxMap::lin(1);
    g.ak = IdxMap::lin(r);
    g.a_kfast = false;
    g.B = X[j + 1];
    g.bn = IdxMap::lin(1);
    g.bk = IdxMap::lin(N);
    g.b_kfast = false;
    g.C = nn;
    g.cm = IdxMap::lin(N);
    g.cn = IdxMap::lin(1);
    prep_gemm(h, P, g);
    P.dead.push_back(X[j]);
    P.dead.push_back(X[j + 1]);
    X[j] = nc;
    X[j + 1] = nn;
    bond[j + 1] = r;
  }
}

Prep make_prep(tt_fit* h, long long max_core) {
  Prep P;
  CK(cudaStreamCreateWithFlags(&P.st, cudaStreamNonBlocking));
  P.X = h->pool.alloc<double>(max_core);
  P.Q = h->pool.alloc<double>(max_core);
  P.R = h->pool.alloc<double>(max_core);
  P.ws_elems = (size_t)max_core * 16 + (1 << 20);
  P.ws = h->pool.alloc<double>(P.ws_elems);
  return P;
}

void finish_prep(tt_fit* h, Prep& P) {
  CK(cudaStreamSynchronize(P.st));
  for (void* d : P.dead) h->pool.release(d);
  h->pool.release(P.X);
  h->pool.release(P.Q);
  h->pool.release(P.R);
  h->pool.release(P.ws);
  P.dead.clear();
  cudaStreamDestroy(P.st);
  P.st = nullptr;
}

// Events, pinned mirrors and device flags of a lane.
void init_lane(tt_fit* h, Work& w, cudaStream_t st, bool own_stream) {
  w.st = st;
  w.own_stream = own_stream;
  w.dnorm = h->pool.alloc<double>(1);
  w.dk = h->pool.alloc<int>(4);
  w.ddinfo = h->pool.alloc<double>(4);
  w.errw = h->pool.alloc<uint32_t>(4);  // [0] error bits, [1] max Jacobi sweeps (diagnostic)
  CK(cudaMemsetAsync(w.errw, 0, 4 * sizeof(uint32_t), w.st));
  for (auto& e : w.ev) CK(cudaEventCreate(&e));
  CK(cudaMallocHost(&w.hk, sizeof(int) * 4));
  CK(cudaMallocHost(&w.hdinfo, sizeof(double) * 4));
  CK(cudaMallocHost(&w.herrw, sizeof(uint32_t) * 4));
  *w.herrw = 0;
}

void free_lane(Work& w) {
  if (w.st) cudaStreamSynchronize(w.st);
  for (auto& e : w.ev)
    if (e) cudaEventDestroy(e), e = nullptr;
  if (w.hk) cudaFreeHost(w.hk), w.hk = nullptr;
  if (w.hdinfo) cudaFreeHost(w.hdinfo), w.hdinfo = nullptr;
  if (w.herrw) cudaFreeHost(w.herrw), w.herrw = nullptr;
  if (w.own_stream && w.st) cudaStreamDestroy(w.st);
  w.st = nullptr;
}

void free_lanes(tt_fit* h) {
  for (auto& w : h->wseg) free_lane(*w);
  free_lane(h->w0);
}

void check_errw(tt_fit* h, const char* where) {
  if (*W(h).herrw & ERRW_NAN) throw TTError(TT_ERR_NUMERICAL, std::string("non-finite two-site tensor at ") + where);
  if (*W(h).herrw & ERRW_NOCONV) throw TTError(TT_ERR_NUMERICAL, std::string("Jacobi SVD did not converge at ") + where);
  if (*W(h).herrw & ERRW_TIMEOUT) throw TTError(TT_ERR_TIMEOUT, std::string("bounded device wait expired at ") + where);
  if (*W(h).herrw) throw TTError(TT_ERR_NUMERICAL, std::string("device error word set at ") + where);
}

// ---------------------------------------------------------------------------
// the contraction chain in working type T
// ---------------------------------------------------------------------------
template <typename T>
struct Chain {
  tt_fit* h;
  explicit Chain(tt_fit* hh) : h(hh) {}
  T* P(void* p) { return (T*)p; }

  // H1_j = L_{j-1} A_j B_j, stored [c0][s][t][a1][b1] (j is 0-based site index)
  void half_left(int j) {
    Dims& D = h->D;
    const int a0 = D.a[j], a1 = D.a[j + 1], b0 = D.b[j], b1 = D.b[j + 1], c0 = D.c[j];
    const int ds = D.ds[j], du = D.du[j], dt = D.dt[j];
    GemmArgs<T> g;
    g.M = c0 * b0;
    g.N = ds * du * a1;
    g.K = a0;
    g.A = P(h->Lenv[j]);
    g.am = IdxMap::lin(a0);
    g.ak = IdxMap::lin(1);
    g.B = P(h->Aop[j]);
    g.bn = IdxMap::lin(a0);
    g.bk = IdxMap::lin(1);
    g.C = P(W(h).X1);
    g.cm = IdxMap::two(b0, (long long)ds * a1 * b0 * du, du);
    g.cn = IdxMap::three(du, a1, (long long)a1 * b0 * du, 1, (long long)b0 * du);
    gemm<T>(h, g, true);
    GemmArgs<T> g2;
    g2.M = c0 * ds * a1;
    g2.N = dt * b1;
    g2.K = b0 * du;
    g2.A = P(W(h).X1);
    g2.am = IdxMap::lin((long long)b0 * du);
    g2.ak = IdxMap::lin(1);
    g2.B = P(h->Bl[j]);
    g2.bn = IdxMap::lin((long long)b0 * du);
    g2.bk = IdxMap::lin(1);
    g2.C = P(h->H1[j]);
    g2.cm = IdxMap::two(a1, (long long)dt * a1 * b1, b1);
    g2.cn = IdxMap::two(b1, (long long)a1 * b1, 1);
    // transposed copy H1t [a1][b1][c0][s][t] for the environment finish
    const long long K1 = (long long)c0 * ds * dt;
    g2.C2 = P(h->H1t[j]);
    g2.cm2 = IdxMap::two(a1, dt, (long long)b1 * K1);
    g2.cn2 = IdxMap::two(b1, 1, K1);
    gemm<T>(h, g2, true);
    W(h).flops += 2.0 * g.M * g.N * g.K + 2.0 * g2.M * g2.N * g2.K;
  }

  // H2_j = A_j B_j R_{j+1}, stored [s][t][c1][a0][b0] (bond indices of site j)
  void half_right(int j) {
    Dims& D = h->D;
    const int a1 = D.a[j], a2 = D.a[j + 1], b1 = D.b[j], b2 = D.b[j + 1], c2 = D.c[j + 1];
    const int ds = D.ds[j], du = D.du[j], dt = D.dt[j];
    GemmArgs<T> g;
    g.M = a1 * ds * du;
    g.N = c2 * b2;
    g.K = a2;
    g.A = P(h->Anat[j]);
    g.am = IdxMap::lin(a2);
    g.ak = IdxMap::lin(1);
    g.B = P(h->Renv[j + 1]);
    g.bn = IdxMap::lin(a2);
    g.bk = IdxMap::lin(1);
    g.C = P(W(h).Zs);
    g.cm = IdxMap::two(du, (long long)c2 * du * b2, b2);
    g.cn = IdxMap::two(b2, (long long)du * b2, 1);
    gemm<T>(h, g, true);
    GemmArgs<T> g2;
    g2.M = a1 * ds * c2;
    g2.N = b1 * dt;
    g2.K = du * b2;
    g2.A = P(W(h).Zs);
    g2.am = IdxMap::lin((long long)du * b2);
    g2.ak = IdxMap::lin(1);
    g2.B = P(h->Br[j]);
    g2.bn = IdxMap::lin((long long)du * b2);
    g2.bk = IdxMap::lin(1);
    g2.C = P(h->H2[j]);
    g2.cm = IdxMap::three(ds, c2, b1, (long long)dt * c2 * a1 * b1, (long long)a1 * b1);
    g2.cn = IdxMap::two(dt, 1, (long long)c2 * a1 * b1);
    // transposed copy H2t [a1][b1][s][t][c2] for the environment finish
    const long long K2 = (long long)ds * dt * c2;
    g2.C2 = P(h->H2t[j]);
    g2.cm2 = IdxMap::three(ds, c2, (long long)b1 * K2, (long long)dt * c2, 1);
    g2.cn2 = IdxMap::two(dt, K2, c2);
    gemm<T>(h, g2, true);
    W(h).flops += 2.0 * g.M * g.N * g.K + 2.0 * g2.M * g2.N * g2.K;
  }

  // Theta(window l, l+1) = H1_l . H2_{l+1}, row-major (c0 s1 t1) x (s2 t2 c2)
  void join(int l, int& m, int& n) {
    Dims& D = h->D;
    const int a1 = D.a[l + 1], b1 = D.b[l + 1], c0 = D.c[l], c2 = D.c[l + 2];
    m = c0 * D.ds[l] * D.dt[l];
    n = D.ds[l + 1] * D.dt[l + 1] * c2;
    GemmArgs<T> g;
    g.M = m;
    g.N = n;
    g.K = a1 * b1;
    g.A = P(h->H1[l]);
    g.am = IdxMap::lin((long long)a1 * b1);
    g.ak = IdxMap::lin(1);
    g.B = P(h->H2[l + 1]);
    g.bn = IdxMap::lin((long long)a1 * b1);
    g.bk = IdxMap::lin(1);
    g.C = P(W(h).Th);
    g.cm = IdxMap::lin(n);
    g.cn = IdxMap::lin(1);
    gemm<T>(h, g, true);
    W(h).flops += 2.0 * g.M * g.N * g.K;
  }

  // L_j (bond j+1) = Ut_j . H1_j ; stored [c][b][a]
  void finish_left(int j) {
    Dims& D = h->D;
    const int a1 = D.a[j + 1], b1 = D.b[j + 1], c0 = D.c[j], c1 = D.c[j + 1];
    const int K = c0 * D.ds[j] * D.dt[j];
    GemmArgs<T> g;
    g.M = c1;
    g.N = a1 * b1;
    g.K = K;
    g.A = P(h->Ut[j]);
    g.am = IdxMap::lin(K);
    g.ak = IdxMap::lin(1);
    g.B = P(h->H1t[j]);
    g.bn = IdxMap::lin(K);
    g.bk = IdxMap::lin(1);
    g.C = P(h->Lenv[j + 1]);
    g.cm = IdxMap::lin((long long)a1 * b1);
    g.cn = IdxMap::two(b1, 1, a1);
    gemm<T>(h, g, true);
    W(h).flops += 2.0 * g.M * g.N * g.K;
  }

  // R_j (bond j) = Vt_j . H2_j ; stored [c][b][a]
  void finish_right(int j) {
    Dims& D = h->D;
    const int a0 = D.a[j], b0 = D.b[j], c0 = D.c[j], c1 = D.c[j + 1];
    const int K = D.ds[j] * D.dt[j] * c1;
    GemmArgs<T> g;
    g.M = c0;
    g.N = a0 * b0;
    g.K = K;
    g.A = P(h->Vt[j]);
    g.am = IdxMap::lin(K);
    g.ak = IdxMap::lin(1);
    g.B = P(h->H2t[j]);
    g.bn = IdxMap::lin(K);
    g.bk = IdxMap::lin(1);
    g.C = P(h->Renv[j]);
    g.cm = IdxMap::lin((long long)a0 * b0);
    g.cn = IdxMap::two(b0, 1, a0);
    gemm<T>(h, g, true);
    W(h).flops += 2.0 * g.M * g.N * g.K;
  }
};

// ---------------------------------------------------------------------------
// factorisation of the m x n two-site matrix (Sec. 2.3.4 / Sec. 3.1) in type F
// (double on the FP64 path, float otherwise): U_M (m x p col-major, ld m),
// S (p, sorted), V_M (n x p, ld n). Returns p (computed singular triplets).
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Factorisation of a DF32 two-site matrix with an FP64-class basis and an FP32
// singular value decomposition: the randomized one (Sec. 3.1, exact = false),
// or the exact one of a window whose sketch would not be narrower than the
// matrix (exact = true: the basis of a tall Theta is that of Theta itself, the
// basis of a wide one the identity).
//
// The kept singular vectors sit at s_k ~ 1e-5 s_1 in this workload, so any step
// that rounds Theta, Y = Theta Omega or the basis Q to FP32 (absolute error
// ~6e-8 s_1) tilts them by ~1e-2 and moves C by ~1e-6 of its norm. Here every
// product with Theta and with the basis is double-FP32, and the two FP32 steps
// that remain are harmless:
//  * Q: the FP32 Householder R of the scaled Y (R only) is inverted in FP32 and
//    applied in double-FP32, Z = Y R^-1. Any non-singular right factor keeps
//    range(Y) exactly; it only conditions Z (cond(Z) ~ eps32 cond(Y)). The same
//    step once more on Z, then three double-FP32 Newton-Schulz steps, make it
//    orthonormal without moving its range. (An FP32 Cholesky factor of Z^T Z
//    would square cond(Z) and break down for the worst sketches of this fit.)
//  * B = Q^T Theta is formed in double-FP32. Its rows are graded (row i ~ s_i),
//    so rounding it entrywise to FP32 perturbs each row relative to itself, and
//    the one-sided Jacobi SVD (after an R-only QR of B^T) stays relatively
//    accurate (Demmel and Veselic, SIAM J. Matrix Anal. Appl. 13 (1992)).
//  * U = Q U_B and, when wanted, V = B^T U_B S^-1 in double-FP32.
// Writes U_M (m x r) and V_M (n x r, need != 1) as df32 into fUM / fVM, the
// FP32 singular values (of 2^-e B) into fS; returns r (the sketch width, or
// min(m, n) for an exact factorisation). A zero pivot of an R
// factor or a basis that is not orthonormal after the steps sets ERRW_HPFAIL:
// the caller then redoes the window with the all-FP32 factorisation.
// ---------------------------------------------------------------------------
int factorize_hp(tt_fit* h, int m, int n, int sweep, int site1, int need, bool exact) {
  Work& w = W(h);
  // basis width r: the sketch width, or for an exact factorisation the rank bound min(m, n)
  const int r = exact ? std::min(m, n) : h->chi_max + h->oversample;
  const bool ident = exact && m <= n;  // the basis of a wide exact window is the identity
  const df32* Th = (const df32*)w.Th;
  int* ex = w.dk + 1;  // exponent of max |Theta| (set by the caller)
  int* ey = w.dk + 2;  // exponent of max |Y|
  df32 *Om = (df32*)w.fOm, *Yd = (df32*)w.fY, *Zd = (df32*)w.fQ, *Gd = (df32*)w.pG, *Wd = (df32*)w.fVw;
  float *Y32 = (float*)w.fX, *R32 = (float*)w.fR, *Bt32 = (float*)w.fBt, *R2 = (float*)w.fR2;
  auto gram = [&](const df32* X, int rows) {  // Gd = X^T X (r x r), X rows x r column-major
    GemmArgs<df32> g;
    g.M = r; g.N = r; g.K = rows;
    g.A = X; g.am = IdxMap::lin(rows); g.ak = IdxMap::lin(1);
    g.B = X; g.bn = IdxMap::lin(rows); g.bk = IdxMap::lin(1);
    g.C = Gd; g.cm = IdxMap::lin(1); g.cn = IdxMap::lin(r);
    gemm<df32>(h, g);
  };
  auto apply = [&](const df32* X, int rows, const df32* Wm, df32* out, df32 alpha, df32 beta) {  // out = a X Wm + b out
    GemmArgs<df32> g;
    g.M = rows; g.N = r; g.K = r;
    g.A = X; g.am = IdxMap::lin(1); g.ak = IdxMap::lin(rows); g.a_kfast = false;
    g.B = Wm; g.bn = IdxMap::lin(r); g.bk = IdxMap::lin(1);
    g.C = out; g.cm = IdxMap::lin(1); g.cn = IdxMap::lin(rows);
    g.alpha = alpha;
    g.beta = beta;
    gemm<df32>(h, g);
  };
  auto rqr = [&](int q, float* X, float* R) {  // R (r x r) of the FP32 Householder QR of X (q x r)
    const bool cluster = q >= 128 && r >= 16;
    CK(qr_householder<float, float>(q, r, X, cluster ? nullptr : (float*)w.fUM, R, w.st));
  };
  const df32* Q = nullptr;  // m x r orthonormal basis (null: the identity, r = m)
  if (!ident) {
    if (exact) {  // Y = Theta, column-major
      copymap<df32, df32>(h, m, n, Th, IdxMap::lin(n), IdxMap::lin(1), Yd, IdxMap::lin(1), IdxMap::lin(m));
    } else {  // Y = Theta Omega (m x r, column-major); Omega is n x r row-major, as in the oracle
      CK(philox_fill<df32>(Om, (long long)n * r, h->seed, omega_stream(sweep, site1), 1.0, w.st));
      GemmArgs<df32> g;
      g.M = m; g.N = r; g.K = n;
      g.A = Th; g.am = IdxMap::lin(n); g.ak = IdxMap::lin(1);
      g.B = Om; g.bn = IdxMap::lin(1); g.bk = IdxMap::lin(r); g.b_kfast = false;
      g.C = Yd; g.cm = IdxMap::lin(1); g.cn = IdxMap::lin(m);
      gemm<df32>(h, g);
    }
    // FP32 preconditioner, twice: R of the scaled Y, inverted; Z1 = Y (2^-ey R^-1) has
    // cond ~ eps32 cond(Y) (up to ~1e4 for the sketches of this fit), and the same step on
    // Z1 leaves Z2 = Z1 R(Z1)^-1 within ~1e-3 of orthonormal
    CK(absmax_exponent<df32>(Yd, (long long)m * r, ey, w.st));
    CK(copy_pow2<df32, float>((long long)m * r, Yd, Y32, ey, w.st));
    rqr(m, Y32, R32);
    CK(tri_inv(r, R32, r, ey, Wd, w.errw, w.st));
    apply(Yd, m, Wd, Zd, df32(1.f, 0.f), df32(0.f, 0.f));
    copymap<df32, float>(h, m, r, Zd, IdxMap::lin(1), IdxMap::lin(m), Y32, IdxMap::lin(1), IdxMap::lin(m));
    rqr(m, Y32, R32);
    CK(tri_inv(r, R32, r, nullptr, Wd, w.errw, w.st));
    apply(Zd, m, Wd, Yd, df32(1.f, 0.f), df32(0.f, 0.f));
    df32 *X = Yd, *Xn = Zd;
    for (int it = 0; it < 3; ++it) {  // X <- X (3 I - X^T X) / 2; |X^T X - I| ~1e-3 -> 1e-6 -> 1e-12 -> rounding
      gram(X, m);
      if (it == 2) CK(ortho_check(r, Gd, 1e-6, w.errw, w.st));
      CK(cudaMemcpyAsync(Xn, X, sizeof(df32) * (size_t)m * r, cudaMemcpyDeviceToDevice, w.st));
      apply(X, m, Gd, Xn, df32(-0.5f, 0.f), df32(1.5f, 0.f));
      std::swap(X, Xn);
    }
    Q = X;
  }
  // B^T = Theta^T Q (n x r, column-major; Theta itself when the basis is the identity), its FP32
  // copy scaled by 2^-e (e of Theta), R-only QR
  const df32* Btd = Th;  // row-major m x n Theta is column-major n x m Theta^T
  if (!ident) {
    df32* bt = (df32*)w.fQ2;
    GemmArgs<df32> g;
    g.M = n; g.N = r; g.K = m;
    g.A = Th; g.am = IdxMap::lin(1); g.ak = IdxMap::lin(n); g.a_kfast = false;
    g.B = Q; g.bn = IdxMap::lin(m); g.bk = IdxMap::lin(1);
    g.C = bt; g.cm = IdxMap::lin(1); g.cn = IdxMap::lin(n);
    gemm<df32>(h, g);
    Btd = bt;
  }
  CK(copy_pow2<df32, float>((long long)n * r, Btd, Bt32, ex, w.st));
  rqr(n, Bt32, R2);
  // B = R2^T Q2^T: the left singular vectors U_B of B are the right ones of R2
  float *fX = (float*)w.fX, *fU = (float*)w.fU, *fV = (float*)w.fV, *fS = (float*)w.fS, *fVw = (float*)w.fVw;
  if (need == 1) {  // one-sided Jacobi on R2^T: U_B = its normalised columns
    copymap<float, float>(h, r, r, R2, IdxMap::lin(1), IdxMap::lin(r), fX, IdxMap::lin(r), IdxMap::lin(1));
    CK(jacobi_svd<float, float>(r, r, fX, fV, fS, nullptr, fVw, 60, w.errw, w.st));
  } else {          // on R2: U_B = the accumulated rotations
    CK(jacobi_svd<float, float>(r, r, R2, fU, fS, fV, fVw, 60, w.errw, w.st));
  }
  // U_M = Q U_B; V_M = B^T U_B S^-1 (S of 2^-e B, so the scale 2^-e comes back in)
  df32* UBd = (df32*)w.fR;
  copymap<float, df32>(h, r, r, fV, IdxMap::lin(r), IdxMap::lin(1), UBd, IdxMap::lin(r), IdxMap::lin(1));
  if (ident) {
    CK(cudaMemcpyAsync(w.fUM, UBd, sizeof(df32) * (size_t)r * r, cudaMemcpyDeviceToDevice, w.st));
  } else {
    GemmArgs<df32> g;
    g.M = m; g.N = r; g.K = r;
    g.A = Q; g.am = IdxMap::lin(1); g.ak = IdxMap::lin(m); g.a_kfast = false;
    g.B = UBd; g.bn = IdxMap::lin(r); g.bk = IdxMap::lin(1);
    g.C = (df32*)w.fUM; g.cm = IdxMap::lin(1); g.cn = IdxMap::lin(m);
    gemm<df32>(h, g);
  }
  if (need != 1) {
    df32* Dd = (df32*)w.fVw;
    CK(scale_cols_inv(r, r, fV, fS, ex, Dd, w.st));
    GemmArgs<df32> g;
    g.M = n; g.N = r; g.K = r;
    g.A = Btd; g.am = IdxMap::lin(1); g.ak = IdxMap::lin(n); g.a_kfast = false;
    g.B = Dd; g.bn = IdxMap::lin(r); g.bk = IdxMap::lin(1);
    g.C = (df32*)w.fVM; g.cm = IdxMap::lin(1); g.cn = IdxMap::lin(n);
    gemm<df32>(h, g);
  }
  CK(fix_signs<df32>(m, n, r, (df32*)w.fUM, m, need != 1 ? (df32*)w.fVM : nullptr, n, w.st));
  w.hp = true;
  return r;
}

template <typename T, typename F>
int factorize_body(tt_fit* h, int m, int n, int sweep, int site1, int need) {
  W(h).hp = false;
  F *fX = (F*)W(h).fX, *fQ = (F*)W(h).fQ, *fR = (F*)W(h).fR, *fU = (F*)W(h).fU, *fV = (F*)W(h).fV, *fVw = (F*)W(h).fVw;
  F *fS = (F*)W(h).fS, *fUM = (F*)W(h).fUM, *fVM = (F*)W(h).fVM, *fOm = (F*)W(h).fOm, *MF = (F*)W(h).fY;
  F *fBt = (F*)W(h).fBt, *fQ2 = (F*)W(h).fQ2, *fR2 = (F*)W(h).fR2;
  auto qrf = [&](int q, int p, F* X, F* Q, F* R) {
    CK(qr_householder<F, F>(q, p, X, Q, R, W(h).st));
  };
  auto jac = [&](int q, int p, F* Wm, F* U, F* S, F* V) {
    CK(jacobi_svd<F, F>(q, p, Wm, U, S, V, fVw, 60, W(h).errw, W(h).st));
  };
  // Theta (T, row-major) -> F copy scaled by 2^-e (e: exponent of max |Theta|, in dk[1]) so that its
  // squares stay inside the range of F; norm (flags NaN/Inf)
  int* ex = W(h).dk + 1;
  CK(absmax_exponent<T>((const T*)W(h).Th, (long long)m * n, ex, W(h).st));
  CK(copy_pow2<T, F>((long long)m * n, (const T*)W(h).Th, MF, ex, W(h).st));
  CK(frob_norm<F>(MF, (long long)m * n, W(h).dnorm, W(h).errw, W(h).st));
  const int ks = h->chi_max + h->oversample;
  if (h->update == TT_UPDATE_2SITE_RSVD && ks < std::min(m, n)) {
    if constexpr (std::is_same<T, df32>::value && std::is_same<F, float>::value) {
      if (h->hp_sweep && !W(h).hp_off && ks >= 16 && ks <= TRI_INV_MAX && std::min(m, n) >= 128 &&
          std::max(m, n) <= 1024)
        return factorize_hp(h, m, n, sweep, site1, need, false);
    }
    CK(philox_fill<F>(fOm, (long long)n * ks, h->seed, omega_stream(sweep, site1), 1.0, W(h).st));
    GemmArgs<F> g;  // Ysk = M Omega (m x ks, col-major)
    g.M = m; g.N = ks; g.K = n;
    g.A = MF; g.am = IdxMap::lin(n); g.ak = IdxMap::lin(1);
    g.B = fOm; g.bn = IdxMap::lin(1); g.bk = IdxMap::lin(ks); g.b_kfast = false;
    g.C = fX; g.cm = IdxMap::lin(1); g.cn = IdxMap::lin(m);
    gemm<F>(h, g);
    qrf(m, ks, fX, fQ, fR);                       // Q (m x ks)
    GemmArgs<F> g2;  // Bm^T = M^T Q (n x ks, col-major)
    g2.M = n; g2.N = ks; g2.K = m;
    g2.A = MF; g2.am = IdxMap::lin(1); g2.ak = IdxMap::lin(n); g2.a_kfast = false;
    g2.B = fQ; g2.bn = IdxMap::lin(m); g2.bk = IdxMap::lin(1);
    g2.C = fBt; g2.cm = IdxMap::lin(1); g2.cn = IdxMap::lin(n);
    gemm<F>(h, g2);
    qrf(n, ks, fBt, fQ2, fR2);                    // Bm^T = Q2 R2
    if (need == 1) {
      // only U_M = Q Vr is wanted: one-sided Jacobi on R2^T gives Vr as its
      // normalised columns, with no rotations to accumulate (and it converges
      // in fewer sweeps than on R2)
      copymap<F, F>(h, ks, ks, fR2, IdxMap::lin(1), IdxMap::lin(ks), fX, IdxMap::lin(ks), IdxMap::lin(1));
      CK(jacobi_svd<F, F>(ks, ks, fX, fV, fS, nullptr, fVw, 60, W(h).errw, W(h).st));
      GemmArgs<F> g3;  // U_M = Q Vr (m x ks)
      g3.M = m; g3.N = ks; g3.K = ks;
      g3.A = fQ; g3.am = IdxMap::lin(1); g3.ak = IdxMap::lin(m); g3.a_kfast = false;
      g3.B = fV; g3.bn = IdxMap::lin(ks); g3.bk = IdxMap::lin(1);
      g3.C = fUM; g3.cm = IdxMap::lin(1); g3.cn = IdxMap::lin(m);
      gemm<F>(h, g3);
      CK(fix_signs<F>(m, n, ks, fUM, m, (F*)nullptr, n, W(h).st));
      return ks;
    }
    jac(ks, ks, fR2, fU, fS, fV);                 // R2 = Ur S Vr^T
    GemmArgs<F> g3;  // U_M = Q Vr (m x ks)
    g3.M = m; g3.N = ks; g3.K = ks;
    g3.A = fQ; g3.am = IdxMap::lin(1); g3.ak = IdxMap::lin(m); g3.a_kfast = false;
    g3.B = fV; g3.bn = IdxMap::lin(ks); g3.bk = IdxMap::lin(1);
    g3.C = fUM; g3.cm = IdxMap::lin(1); g3.cn = IdxMap::lin(m);
    gemm<F>(h, g3);
    GemmArgs<F> g4;  // V_M = Q2 Ur (n x ks)
    g4.M = n; g4.N = ks; g4.K = ks;
    g4.A = fQ2; g4.am = IdxMap::lin(1); g4.ak = IdxMap::lin(n); g4.a_kfast = false;
    g4.B = fU; g4.bn = IdxMap::lin(ks); g4.bk = IdxMap::lin(1);
    g4.C = fVM; g4.cm = IdxMap::lin(1); g4.cn = IdxMap::lin(n);
    gemm<F>(h, g4);
    CK(fix_signs<F>(m, n, ks, fUM, m, fVM, n, W(h).st));
    return ks;
  }
  if constexpr (std::is_same<T, df32>::value && std::is_same<F, float>::value) {
    // an exact factorisation keeps the whole range of a tall Theta: its basis in FP64-class
    // arithmetic too (a wide one needs none)
    if (h->hp_sweep && !W(h).hp_off && std::min(m, n) <= TRI_INV_MAX && std::max(m, n) <= 1024)
      return factorize_hp(h, m, n, sweep, site1, need, true);
  }
  // exact: work on the tall orientation X (q x p col-major)
  const bool tr = m < n;
  const int q = tr ? n : m, p = tr ? m : n;
  if (tr) CK(cudaMemcpyAsync(fX, MF, sizeof(F) * (size_t)m * n, cudaMemcpyDeviceToDevice, W(h).st));
  else copymap<F, F>(h, m, n, MF, IdxMap::lin(n), IdxMap::lin(1), fX, IdxMap::lin(1), IdxMap::lin(m));
  F* Ufull;
  if (q > p) {
    qrf(q, p, fX, fQ, fR);                        // X = Qx Rx
    jac(p, p, fR, fU, fS, fV);                    // Rx = Ur S Vr^T
    GemmArgs<F> g;  // Ufull = Qx Ur (q x p)
    g.M = q; g.N = p; g.K = p;
    g.A = fQ; g.am = IdxMap::lin(1); g.ak = IdxMap::lin(q); g.a_kfast = false;
    g.B = fU; g.bn = IdxMap::lin(p); g.bk = IdxMap::lin(1);
    g.C = fBt; g.cm = IdxMap::lin(1); g.cn = IdxMap::lin(q);
    gemm<F>(h, g);
    Ufull = fBt;
  } else {
    jac(q, p, fX, fU, fS, fV);
    Ufull = fU;
  }
  // X = Ufull S Vr^T ; Theta = X (tr = false) or X^T (tr = true)
  const size_t qb = sizeof(F) * (size_t)q * p, pb = sizeof(F) * (size_t)p * p;
  if (!tr) {
    CK(cudaMemcpyAsync(fUM, Ufull, qb, cudaMemcpyDeviceToDevice, W(h).st));
    CK(cudaMemcpyAsync(fVM, fV, pb, cudaMemcpyDeviceToDevice, W(h).st));
  } else {
    CK(cudaMemcpyAsync(fUM, fV, pb, cudaMemcpyDeviceToDevice, W(h).st));
    CK(cudaMemcpyAsync(fVM, Ufull, qb, cudaMemcpyDeviceToDevice, W(h).st));
  }
  CK(fix_signs<F>(m, n, p, fUM, m, fVM, n, W(h).st));
  return p;
}

// The factorisation of Theta: that of 2^-e Theta, with the singular values and
// ||Theta|| scaled back (the singular vectors do not change).
template <typename T, typename F>
int factorize(tt_fit* h, int m, int n, int sweep, int site1, int need = 3) {
  const int p = factorize_body<T, F>(h, m, n, sweep, site1, need);
  CK(unscale_pow2<F>(p, (F*)W(h).fS, W(h).dnorm, W(h).dk + 1, W(h).st));
  return p;
}

// ---------------------------------------------------------------------------
// Gauge update of the non-FP64 paths. The FP32 factorisation gives singular
// vectors accurate to the FP32 level; Newton-Schulz steps in FP64,
// X <- X (3 I - X^T X) / 2, make the kept ones an isometry, and the other
// factor is the projection of the two-site tensor on it (the optimal factor for
// that isometry, Eq. fit_pde). One step maps a Gram deviation E to about
// (3/4) E^2: from the FP32 factor (|E| up to ~3e-5 at 512 rows) that is ~1e-9
// per core, and the deviations of the L-1 cores outside the orthogonality
// centre add up in ||C||^2, which the sweep reads off the last window alone.
// A second step takes each core to the FP64 rounding level. Because ||C||^2 is
// stationary under small rotations of the kept subspace, the FP32 rounding of
// the subspace enters ||C||^2 only at second order. Writes ||C_window|| to dn2[l].
// ---------------------------------------------------------------------------
constexpr int kNewtonSchulzSteps = 2;

// The steps run in double-FP32 (about 4x the FP64 rate of this GPU; rounding
// ~1e-14, far below what the sweeps resolve). X64 serves as the second buffer.
template <typename Fin>
void ns_orthonormalize(tt_fit* h, const Fin* Xin, int rows, int k, double* X64) {
  df32* G = (df32*)W(h).pG;
  df32 *X = (df32*)W(h).pT, *Xn = (df32*)X64;
  copymap<Fin, df32>(h, rows, k, Xin, IdxMap::lin(1), IdxMap::lin(rows), X, IdxMap::lin(1), IdxMap::lin(rows));
  for (int it = 0; it < kNewtonSchulzSteps; ++it) {
    GemmArgs<df32> g;  // G = X^T X (k x k)
    g.M = k; g.N = k; g.K = rows;
    g.A = X; g.am = IdxMap::lin(rows); g.ak = IdxMap::lin(1);
    g.B = X; g.bn = IdxMap::lin(rows); g.bk = IdxMap::lin(1);
    g.C = G; g.cm = IdxMap::lin(k); g.cn = IdxMap::lin(1);
    gemm<df32>(h, g);
    CK(cudaMemcpyAsync(Xn, X, sizeof(df32) * (size_t)rows * k, cudaMemcpyDeviceToDevice, W(h).st));
    GemmArgs<df32> g2;  // Xn = 1.5 X - 0.5 X G
    g2.M = rows; g2.N = k; g2.K = k;
    g2.A = X; g2.am = IdxMap::lin(1); g2.ak = IdxMap::lin(rows); g2.a_kfast = false;
    g2.B = G; g2.bn = IdxMap::lin(k); g2.bk = IdxMap::lin(1);
    g2.C = Xn; g2.cm = IdxMap::lin(1); g2.cn = IdxMap::lin(rows);
    g2.alpha = df32(-0.5f, 0.f);
    g2.beta = df32(1.5f, 0.f);
    gemm<df32>(h, g2);
    std::swap(X, Xn);
  }
  // the result is in X: convert in place if it is X64 already, else copy across
  copymap<df32, double>(h, rows, k, X, IdxMap::lin(1), IdxMap::lin(rows), X64, IdxMap::lin(1), IdxMap::lin(rows));
}

template <typename T, typename F>
void polish_update(tt_fit* h, int mode, int m, int n, int k, int l, bool both = false) {
  const T* Th = (const T*)W(h).Th;
  T* Ut = (T*)h->Ut[l];
  T* Vt = (T*)h->Vt[l + 1];
  T* P = (T*)W(h).pP;  // m x k (or k x n) projection, then the k x k block
  const int side = std::max(m, n);
  if (mode != 1) {  // left isometry U (m x k)
    ns_orthonormalize<F>(h, (const F*)W(h).fUM, m, k, W(h).pU);
    // Ut (k x m row-major) = U^T : same memory order as U column-major
    copymap<double, T>(h, 1, m * k, W(h).pU, IdxMap::lin(0), IdxMap::lin(1), Ut, IdxMap::lin(0), IdxMap::lin(1));
  }
  if (mode != 0 || both) {  // right isometry V (n x k)
    ns_orthonormalize<F>(h, (const F*)W(h).fVM, n, k, W(h).pV);
    copymap<double, T>(h, 1, n * k, W(h).pV, IdxMap::lin(0), IdxMap::lin(1), Vt, IdxMap::lin(0), IdxMap::lin(1));
  }
  if (mode == 0) {  // site, forward: C_l = U, C_{l+1} = U^T Theta
    copymap<double, double>(h, m, k, W(h).pU, IdxMap::lin(1), IdxMap::lin(m), h->C64[l], IdxMap::lin(k), IdxMap::lin(1));
    GemmArgs<T> g;
    g.M = k; g.N = n; g.K = m;
    g.A = Ut; g.am = IdxMap::lin(m); g.ak = IdxMap::lin(1);
    g.B = Th; g.bn = IdxMap::lin(1); g.bk = IdxMap::lin(n); g.b_kfast = false;
    g.C = P; g.cm = IdxMap::lin(n); g.cn = IdxMap::lin(1);
    gemm<T>(h, g);
    copymap<T, double>(h, 1, k * n, P, IdxMap::lin(0), IdxMap::lin(1), h->C64[l + 1], IdxMap::lin(0), IdxMap::lin(1));
    CK(frob_norm<T>(P, (long long)k * n, h->dn2 + l, nullptr, W(h).st));
  } else if (mode == 1) {  // site, backward: C_{l+1} = V^T, C_l = Theta V
    copymap<double, double>(h, 1, n * k, W(h).pV, IdxMap::lin(0), IdxMap::lin(1), h->C64[l + 1], IdxMap::lin(0),
                            IdxMap::lin(1));
    GemmArgs<T> g;
    g.M = m; g.N = k; g.K = n;
    g.A = Th; g.am = IdxMap::lin(n); g.ak = IdxMap::lin(1);
    g.B = Vt; g.bn = IdxMap::lin(n); g.bk = IdxMap::lin(1);
    g.C = P; g.cm = IdxMap::lin(k); g.cn = IdxMap::lin(1);
    gemm<T>(h, g);
    copymap<T, double>(h, 1, m * k, P, IdxMap::lin(0), IdxMap::lin(1), h->C64[l], IdxMap::lin(0), IdxMap::lin(1));
    CK(frob_norm<T>(P, (long long)m * k, h->dn2 + l, nullptr, W(h).st));
  } else {  // inverse: Psi_l = U s, Psi_{l+1} = s V^T, Y_l = 1/s with s = diag(U^T Theta V)
    GemmArgs<T> g;  // X = Theta V (m x k)
    g.M = m; g.N = k; g.K = n;
    g.A = Th; g.am = IdxMap::lin(n); g.ak = IdxMap::lin(1);
    g.B = Vt; g.bn = IdxMap::lin(n); g.bk = IdxMap::lin(1);
    g.C = P; g.cm = IdxMap::lin(k); g.cn = IdxMap::lin(1);
    gemm<T>(h, g);
    T* Pk = P + (size_t)side * k;
    GemmArgs<T> g2;  // Pk = U^T X (k x k)
    g2.M = k; g2.N = k; g2.K = m;
    g2.A = Ut; g2.am = IdxMap::lin(m); g2.ak = IdxMap::lin(1);
    g2.B = P; g2.bn = IdxMap::lin(1); g2.bk = IdxMap::lin(k); g2.b_kfast = false;
    g2.C = Pk; g2.cm = IdxMap::lin(k); g2.cn = IdxMap::lin(1);
    gemm<T>(h, g2);
    CK(inverse_gauge_update<T>(m, n, k, W(h).pU, W(h).pV, Pk, h->C64[l], h->C64[l + 1], h->Y[l + 1], W(h).st));
    CK(frob_norm<T>(Pk, (long long)k * k, h->dn2 + l, nullptr, W(h).st));
  }
}

// Whether the next sweep forms the randomized sketch basis in FP64-class
// arithmetic (fast_factor 3: always; 1: once the previous sweep changed ||C||^2
// by at most kHpDelta, i.e. near convergence, so that the sweeps that decide
// the converged C are FP64-class while the early ones keep the all-FP32
// update; the sweep map contracts what the early sweeps leave, and an accurate
// sweep from their state lands on the accurate fixed point).
constexpr double kHpDelta = 1e-3;
inline bool use_hp_basis(const tt_fit* h) {
  if (h->fast_factor == 3) return true;
  return h->fast_factor == 1 && h->delta <= kHpDelta;
}

template <typename T>
struct Sweeper {
  tt_fit* h;
  Chain<T> ch;
  explicit Sweeper(tt_fit* hh) : h(hh), ch(hh) {}

  void add(int stage, int e0, int e1) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, W(h).ev[e0], W(h).ev[e1]));
    W(h).stage_ms[stage] += ms;
  }
  // the previous window's gauge update has completed once the stream has been synchronised
  void resolve_gauge() {
    if (W(h).gauge_pending) add(4, 5, 6);
    W(h).gauge_pending = false;
    if (W(h).connect_pending) add(2, 8, 9);
    W(h).connect_pending = false;
  }

  // Environment handling of a window (0-based window l = sites l, l+1):
  //   ENV_SERIAL  Alg. 5: forward finishes L_l from the cached half of site l-1, backward R_{l+2};
  //   ENV_NONE    first window of a local sweep of Alg. 6: the stored boundary environment is used;
  //   ENV_CONNECT connection update of Alg. 6: both environments are finished first, both halves are
  //               fresh, and L_{l+1}, R_{l+1} across the new bond are finished afterwards.
  //   ENV_MERGE   merge update of the site-gauge scheme: both environments are already finished,
  //               both halves are fresh, and the environments across the new bond follow.
  enum { ENV_SERIAL = 0, ENV_NONE = 1, ENV_CONNECT = 2, ENV_MERGE = 3 };

  // one window update; returns kept sum of s^2 and the discarded fraction
  void window(int l, bool fwd, int sweep, double& n2, double& disc, int env = ENV_SERIAL) {
    Dims& D = h->D;
    const int L = D.L;
    CK(cudaEventRecord(W(h).ev[0], W(h).st));
    const bool boundary = env == ENV_CONNECT || env == ENV_MERGE;
    if (boundary) {
      if (env == ENV_CONNECT) {
        if (l >= 1) ch.finish_left(l - 1);
        if (l + 2 <= L - 1) ch.finish_right(l + 2);
      }
      CK(cudaEventRecord(W(h).ev[1], W(h).st));
      ch.half_left(l);
      ch.half_right(l + 1);
    } else if (fwd) {
      if (l >= 1 && env == ENV_SERIAL) ch.finish_left(l - 1);
      CK(cudaEventRecord(W(h).ev[1], W(h).st));
      ch.half_left(l);
    } else {
      if (l + 2 <= L - 1 && env == ENV_SERIAL) ch.finish_right(l + 2);
      CK(cudaEventRecord(W(h).ev[1], W(h).st));
      ch.half_right(l + 1);
    }
    CK(cudaEventRecord(W(h).ev[2], W(h).st));
    int m, n;
    ch.join(l, m, n);
    CK(cudaEventRecord(W(h).ev[3], W(h).st));
    int p;
    if (h->fact_f32) {
      // a forward step of the site gauge keeps only U (C_l = U, C_{l+1} = U^T Theta); a boundary
      // update also needs V, the basis of the right neighbour's environment
      const bool left_only = h->gauge != TT_GAUGE_INVERSE_CANONICAL && fwd && !boundary;
      p = factorize<T, float>(h, m, n, sweep, l + 1, left_only ? 1 : 3);
      CK(truncate_rule<float>((const float*)W(h).fS, p, W(h).dnorm, h->tol / L, h->chi_max, h->cutoff, W(h).dk, W(h).ddinfo,
                              W(h).st));
    } else {
      using FX = typename FactT<T>::type;
      p = factorize<T, FX>(h, m, n, sweep, l + 1);
      CK(truncate_rule<FX>((const FX*)W(h).fS, p, W(h).dnorm, h->tol / L, h->chi_max, h->cutoff, W(h).dk, W(h).ddinfo, W(h).st));
    }
    CK(cudaEventRecord(W(h).ev[4], W(h).st));
    CK(cudaMemcpyAsync(W(h).hk, W(h).dk, sizeof(int), cudaMemcpyDeviceToHost, W(h).st));
    CK(cudaMemcpyAsync(W(h).hdinfo, W(h).ddinfo, 2 * sizeof(double), cudaMemcpyDeviceToHost, W(h).st));
    CK(cudaMemcpyAsync(W(h).herrw, W(h).errw, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, W(h).st));
    CK(cudaStreamSynchronize(W(h).st));
    if (*W(h).herrw & ERRW_HPFAIL) {
      // the FP64-class sketch basis could not be formed (a rank-deficient sketch): clear the
      // flag and factorise this window again with the all-FP32 randomized update
      CK(cudaMemsetAsync(W(h).errw, 0, sizeof(uint32_t), W(h).st));
      W(h).hp_off = true;
      const bool left_only = h->gauge != TT_GAUGE_INVERSE_CANONICAL && fwd && !boundary;
      try {
        p = factorize<T, float>(h, m, n, sweep, l + 1, left_only ? 1 : 3);
      } catch (...) {
        W(h).hp_off = false;
        throw;
      }
      W(h).hp_off = false;
      CK(truncate_rule<float>((const float*)W(h).fS, p, W(h).dnorm, h->tol / L, h->chi_max, h->cutoff, W(h).dk,
                              W(h).ddinfo, W(h).st));
      CK(cudaEventRecord(W(h).ev[4], W(h).st));
      CK(cudaMemcpyAsync(W(h).hk, W(h).dk, sizeof(int), cudaMemcpyDeviceToHost, W(h).st));
      CK(cudaMemcpyAsync(W(h).hdinfo, W(h).ddinfo, 2 * sizeof(double), cudaMemcpyDeviceToHost, W(h).st));
      CK(cudaMemcpyAsync(W(h).herrw, W(h).errw, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, W(h).st));
      CK(cudaStreamSynchronize(W(h).st));
      ++W(h).hp_fallbacks;
    }
    add(2, 0, 1);
    add(0, 1, 2);
    add(1, 2, 3);
    add(3, 3, 4);
    resolve_gauge();
    if (h->fault_nan_pending) {
      h->fault_nan_pending = false;
      *W(h).herrw |= ERRW_NAN;
    }
    if (h->fault_noconv_pending) {
      h->fault_noconv_pending = false;
      *W(h).herrw |= ERRW_NOCONV;
    }
    char where[64];
    snprintf(where, sizeof where, "window %d", l + 1);
    check_errw(h, where);
    const int k = *W(h).hk;
    n2 = W(h).hdinfo[0];
    disc = W(h).hdinfo[1];
    if (k < 1 || k > D.cb[l + 1]) throw TTError(TT_ERR_NUMERICAL, "kept rank outside the bond capacity");
    D.c[l + 1] = k;
    // gauge update (Alg. 3 / Alg. 4)
    const int mode = (h->gauge == TT_GAUGE_INVERSE_CANONICAL) ? 2 : (fwd ? 0 : 1);
    CK(cudaEventRecord(W(h).ev[5], W(h).st));
    if (!h->fact_f32) {
      using FX = typename FactT<T>::type;
      CK(gauge_update<T, FX>(mode, m, n, (const FX*)W(h).fUM, m, (const FX*)W(h).fS, (const FX*)W(h).fVM, n, W(h).dk, h->C64[l],
                            h->C64[l + 1], h->Y[l + 1], (T*)h->Ut[l], (T*)h->Vt[l + 1], W(h).st));
    } else {
      // a forward boundary update of the site gauge also returns V, the basis of the right
      // neighbour's environment
      const bool both = boundary && mode == 0;
      if (W(h).hp) polish_update<T, df32>(h, mode, m, n, k, l, both);
      else polish_update<T, float>(h, mode, m, n, k, l, both);
    }
    CK(cudaEventRecord(W(h).ev[6], W(h).st));
    W(h).gauge_pending = true;
    if (boundary) {  // environments across the updated bond, for both neighbours
      CK(cudaEventRecord(W(h).ev[8], W(h).st));
      ch.finish_left(l);
      ch.finish_right(l + 1);
      CK(cudaEventRecord(W(h).ev[9], W(h).st));
      W(h).connect_pending = true;
    }
    // host copy of the kept spectrum for tt_fit_result
    if (h->fact_f32) {
      std::vector<float> sv(k);
      CK(cudaMemcpyAsync(sv.data(), W(h).fS, sizeof(float) * k, cudaMemcpyDeviceToHost, W(h).st));
      h->lam[l + 1].assign(sv.begin(), sv.end());
    } else {
      std::vector<double> sv(k);
      CK(cudaMemcpyAsync(sv.data(), W(h).fS, sizeof(double) * k, cudaMemcpyDeviceToHost, W(h).st));
      h->lam[l + 1].assign(sv.begin(), sv.end());
    }
  }

  void run(int n_sweeps) {
    const int L = h->D.L;
    for (int s = 0; s < n_sweeps; ++s) {
      if (h->converged) break;
      const int sweep = h->sweeps_done;
      h->hp_sweep = use_hp_basis(h);
      double n2 = 0, disc = 0, maxd = 0;
      if (h->forward) {
        for (int l = 0; l <= L - 2; ++l) {
          window(l, true, sweep, n2, disc);
          maxd = std::max(maxd, disc);
        }
      } else {
        for (int l = L - 2; l >= 0; --l) {
          window(l, false, sweep, n2, disc);
          maxd = std::max(maxd, disc);
        }
      }
      CK(cudaStreamSynchronize(W(h).st));
      resolve_gauge();
      if (h->fact_f32) {  // ||C||^2 from the FP64-orthonormal projection of the last window
        const int lw = h->forward ? L - 2 : 0;
        double nr = 0;
        CK(cudaMemcpy(&nr, h->dn2 + lw, sizeof(double), cudaMemcpyDeviceToHost));
        n2 = nr * nr;
      }
      h->delta = (h->last_n2 >= 0 && n2 > 0) ? std::fabs(n2 - h->last_n2) / n2 : INFINITY;
      h->last_n2 = n2;
      h->max_disc = maxd;
      h->sweeps_done++;
      h->forward = !h->forward;
      if (h->delta <= h->conv_tol) h->converged = true;
    }
  }

  // R_L .. R_3 and the halves H2_L .. H2_2 from the initial guess (Alg. 5)
  void precompute_right() {
    const int L = h->D.L;
    for (int j = L - 1; j >= 1; --j) {
      ch.half_right(j);
      if (j >= 2) ch.finish_right(j);
    }
    CK(cudaStreamSynchronize(W(h).st));
  }

  // The mirror, for a backward sweep from a left-canonical C: the left operands
  // from C, then L_1..L_{L-2} and the halves H1_0..H1_{L-2}.
  void precompute_left() {
    Dims& D = h->D;
    const int L = D.L;
    const bool inv = h->gauge == TT_GAUGE_INVERSE_CANONICAL;
    for (int j = 0; j + 2 < L; ++j)
      CK(scale_cols_t<T>(D.c[j] * D.ds[j] * D.dt[j], D.c[j + 1], h->C64[j], inv ? h->Y[j + 1] : nullptr,
                         (T*)h->Ut[j], W(h).st));
    for (int j = 0; j + 1 < L; ++j) {
      ch.half_left(j);
      if (j + 2 < L) ch.finish_left(j);
    }
    CK(cudaStreamSynchronize(W(h).st));
  }
};

// ---------------------------------------------------------------------------
void read_desc(const tt_mpo_desc* X, int& L, std::vector<int>& dout, std::vector<int>& din, std::vector<int>& bond) {
  if (!X || X->L < 1 || !X->d_out || !X->d_in || !X->bond || !X->cores)
    throw TTError(TT_ERR_INVALID_ARGUMENT, "MPO descriptor missing fields");
  if (X->dtype != TT_DTYPE_F64 && X->dtype != TT_DTYPE_F32) throw TTError(TT_ERR_INVALID_ARGUMENT, "unknown dtype");
  L = X->L;
  dout.assign(X->d_out, X->d_out + L);
  din.assign(X->d_in, X->d_in + L);
  bond.assign(X->bond, X->bond + L + 1);
  if (bond[0] != 1 || bond[L] != 1) throw TTError(TT_ERR_SHAPE_MISMATCH, "bond[0] and bond[L] must be 1");
  for (int l = 0; l < L; ++l) {
    if (dout[l] < 1 || din[l] < 1 || bond[l] < 1) throw TTError(TT_ERR_INVALID_ARGUMENT, "non-positive dimension");
    if (!X->cores[l]) throw TTError(TT_ERR_INVALID_ARGUMENT, "NULL core pointer");
  }
}

void upload(tt_fit* h, const tt_mpo_desc* X, const std::vector<int>& dout, const std::vector<int>& din,
            const std::vector<int>& bond, std::vector<double*>& out) {
  out.resize(X->L);
  for (int l = 0; l < X->L; ++l) {
    const long long n = prodll({bond[l], dout[l], din[l], bond[l + 1]});
    out[l] = h->pool.alloc<double>(n);
    if (X->dtype == TT_DTYPE_F64)
      copymap<double, double>(h, 1, (int)n, (const double*)X->cores[l], IdxMap::lin(0), IdxMap::lin(1), out[l],
                              IdxMap::lin(0), IdxMap::lin(1));
    else
      copymap<float, double>(h, 1, (int)n, (const float*)X->cores[l], IdxMap::lin(0), IdxMap::lin(1), out[l],
                             IdxMap::lin(0), IdxMap::lin(1));
  }
}

template <typename T>
T* calloc_chain(tt_fit* h, size_t n) {
  T* p = h->pool.alloc<T>(n);
  h->chain_bufs.push_back(p);
  return p;
}

template <typename T>
void build_operands(tt_fit* h) {
  Dims& D = h->D;
  const int L = D.L;
  h->Aop.assign(L, nullptr);
  h->Anat.assign(L, nullptr);
  h->Bl.assign(L, nullptr);
  h->Br.assign(L, nullptr);
  for (int j = 0; j < L; ++j) {
    const int a0 = D.a[j], a1 = D.a[j + 1], b0 = D.b[j], b1 = D.b[j + 1];
    const int ds = D.ds[j], du = D.du[j], dt = D.dt[j];
    T* aop = calloc_chain<T>(h, (size_t)a0 * ds * du * a1);
    T* anat = calloc_chain<T>(h, (size_t)a0 * ds * du * a1);
    T* bl = calloc_chain<T>(h, (size_t)b0 * du * dt * b1);
    T* br = calloc_chain<T>(h, (size_t)b0 * du * dt * b1);
    // A natural (a0, s, u, a1) -> row i = a0, col = (s u a1)
    copymap<double, T>(h, a0, ds * du * a1, h->A64[j], IdxMap::lin((long long)ds * du * a1), IdxMap::lin(1), anat,
                       IdxMap::lin((long long)ds * du * a1), IdxMap::lin(1));
    // Aop [s][u][a1][a0]: element (a0, n=(s u a1)) at n*a0n + a0
    copymap<double, T>(h, a0, ds * du * a1, h->A64[j], IdxMap::lin((long long)ds * du * a1), IdxMap::lin(1), aop,
                       IdxMap::lin(1), IdxMap::lin(a0));
    // B natural (b0, u, t, b1): row = b0, col = (u, t, b1) three-level
    // Bl [t][b1][b0][u]: offset ((t*b1n + b1)*b0n + b0)*du + u
    copymap<double, T>(h, b0, du * dt * b1, h->B64[j], IdxMap::lin((long long)du * dt * b1), IdxMap::lin(1), bl,
                       IdxMap::lin(du), IdxMap::three(dt, b1, 1, (long long)b1 * b0 * du, (long long)b0 * du));
    // Br [b0][t][u][b1]: offset ((b0*dt + t)*du + u)*b1n + b1
    copymap<double, T>(h, b0, du * dt * b1, h->B64[j], IdxMap::lin((long long)du * dt * b1), IdxMap::lin(1), br,
                       IdxMap::lin((long long)dt * du * b1), IdxMap::three(dt, b1, b1, (long long)du * b1, 1));
    h->Aop[j] = aop;
    h->Anat[j] = anat;
    h->Bl[j] = bl;
    h->Br[j] = br;
  }
}

template <typename T>
void allocate_chain(tt_fit* h) {
  Dims& D = h->D;
  const int L = D.L;
  h->Lenv.assign(L + 1, nullptr);
  h->Renv.assign(L + 1, nullptr);
  h->H1.assign(L, nullptr);
  h->H2.assign(L, nullptr);
  h->H1t.assign(L, nullptr);
  h->H2t.assign(L, nullptr);
  h->Ut.assign(L, nullptr);
  h->Vt.assign(L, nullptr);
  size_t x1 = 1, zs = 1;
  long long mmax = 1, nmax = 1;
  for (int j = 0; j <= L; ++j) {
    const long long e = prodll({D.a[j], D.b[j], D.cb[j]});
    h->Lenv[j] = calloc_chain<T>(h, e);
    h->Renv[j] = calloc_chain<T>(h, e);
  }
  for (int j = 0; j < L; ++j) {
    const int ds = D.ds[j], du = D.du[j], dt = D.dt[j];
    h->H1[j] = calloc_chain<T>(h, prodll({D.cb[j], ds, dt, D.a[j + 1], D.b[j + 1]}));
    h->H2[j] = calloc_chain<T>(h, prodll({D.a[j], D.b[j], ds, dt, D.cb[j + 1]}));
    h->H1t[j] = calloc_chain<T>(h, prodll({D.cb[j], ds, dt, D.a[j + 1], D.b[j + 1]}));
    h->H2t[j] = calloc_chain<T>(h, prodll({D.a[j], D.b[j], ds, dt, D.cb[j + 1]}));
    h->Ut[j] = calloc_chain<T>(h, prodll({D.cb[j + 1], D.cb[j], ds, dt}));
    h->Vt[j] = calloc_chain<T>(h, prodll({D.cb[j], ds, dt, D.cb[j + 1]}));
    x1 = std::max<size_t>(x1, prodll({D.cb[j], D.b[j], ds, du, D.a[j + 1]}));
    zs = std::max<size_t>(zs, prodll({D.a[j], ds, du, D.cb[j + 1], D.b[j + 1]}));
    mmax = std::max<long long>(mmax, (long long)D.cb[j] * ds * dt);
    nmax = std::max<long long>(nmax, (long long)ds * dt * D.cb[j + 1]);
  }
  const long long ks = h->chi_max + h->oversample;
  const long long side = std::max(std::max(mmax, nmax), ks);
  // the largest operand of any chain GEMM (environments, A/B operators, X1, Z, halves)
  size_t omax = std::max<size_t>(x1, zs);
  for (int j = 0; j <= L; ++j) omax = std::max<size_t>(omax, prodll({D.a[j], D.b[j], D.cb[j]}));
  for (int j = 0; j < L; ++j) {
    omax = std::max<size_t>(omax, prodll({D.cb[j], D.ds[j], D.dt[j], D.a[j + 1], D.b[j + 1]}));
    omax = std::max<size_t>(omax, prodll({D.a[j], D.b[j], D.ds[j], D.dt[j], D.cb[j + 1]}));
    omax = std::max<size_t>(omax, prodll({D.a[j], D.ds[j], D.du[j], D.a[j + 1]}));
    omax = std::max<size_t>(omax, prodll({D.b[j], D.du[j], D.dt[j], D.b[j + 1]}));
  }
  omax += 65536;
  auto scratch = [&](Work& w) {
    w.X1 = calloc_chain<T>(h, x1);
    w.Zs = calloc_chain<T>(h, zs);
    w.Th = calloc_chain<T>(h, (size_t)mmax * nmax);
    // split-K workspace: up to 16 partial M x N tiles of the largest GEMM output we split
    w.gws_elems = (size_t)std::max<long long>(mmax * nmax, 1) * 16 + (1 << 20);
    w.gws = calloc_chain<double>(h, w.gws_elems);
    w.fsz = (size_t)side * side;
    for (double** f : {&w.fX, &w.fQ, &w.fR, &w.fU, &w.fV, &w.fVw, &w.fUM, &w.fVM, &w.fOm, &w.fY, &w.fBt, &w.fQ2,
                       &w.fR2, &w.pU, &w.pV, &w.pG, &w.pT})
      *f = calloc_chain<double>(h, w.fsz);
    w.fS = calloc_chain<double>(h, side);
    w.pP = calloc_chain<double>(h, (size_t)side * ks + (size_t)ks * ks + 64);
    if (std::is_same<T, df32>::value) {  // the tensor-core GEMM of the DF32 chain
      w.oz_slice = (size_t)OZ_DIGITS * 2 * omax;
      w.oz_exp = omax;
      w.oz_ws = 2 * omax;
      w.ozA = calloc_chain<float>(h, w.oz_slice);
      w.ozB = calloc_chain<float>(h, w.oz_slice);
      w.ozEA = calloc_chain<int>(h, w.oz_exp);
      w.ozEB = calloc_chain<int>(h, w.oz_exp);
      w.ozWs = calloc_chain<df32>(h, w.oz_ws);
    }
  };
  scratch(h->w0);
  for (auto& w : h->wseg) scratch(*w);
  h->dn2 = calloc_chain<double>(h, L + 1);
}

// (Re)build the contraction chain in type T from the current C: operands,
// buffers, the right-environment operands Vt_j (site gauge C_j, inverse gauge
// Y_{j-1} Psi_j), trivial end environments, and the environments the next sweep
// reads: R_L..R_3 with their halves before a forward sweep (C right-canonical),
// L_1..L_{L-2} with theirs before a backward one (C left-canonical).
template <typename T>
void rebuild_chain(tt_fit* h) {
  Dims& D = h->D;
  const int L = D.L;
  CK(cudaStreamSynchronize(W(h).st));
  for (auto* w : lanes(h))
    if (w->st) CK(cudaStreamSynchronize(w->st));
  for (void* p : h->chain_bufs) h->pool.release(p);
  h->chain_bufs.clear();
  build_operands<T>(h);
  allocate_chain<T>(h);
  for (int j = 0; j < L; ++j) {
    const int rows = D.c[j], cols = D.ds[j] * D.dt[j] * D.c[j + 1];
    const bool inv = h->gauge == TT_GAUGE_INVERSE_CANONICAL && j > 0;
    CK(scale_rows<T>(rows, cols, h->C64[j], inv ? h->Y[j] : nullptr, (T*)h->Vt[j], W(h).st));
  }
  T one = T(1);
  CK(cudaMemcpyAsync(h->Lenv[0], &one, sizeof(T), cudaMemcpyHostToDevice, W(h).st));
  CK(cudaMemcpyAsync(h->Renv[L], &one, sizeof(T), cudaMemcpyHostToDevice, W(h).st));
  CK(cudaStreamSynchronize(W(h).st));
  Sweeper<T> sw(h);
  if (h->forward) sw.precompute_right();
  else sw.precompute_left();
}

// ---------------------------------------------------------------------------
// Segment-parallel fit (Sec. 4, Alg. 6), inverse canonical gauge.
// ---------------------------------------------------------------------------

// Contiguous segments of >= 2 sites, 0-based inclusive ranges. The sites are
// shared out as evenly as possible (the first L mod N_p segments get one
// more); edge_extra sites then move to each edge segment, taken one at a time
// from the inner segments in turn, as far as the inner segments keep 2 sites
// (Sec. 4.1: an edge segment has one neighbour, so it can do more local work).
std::vector<std::pair<int, int>> partition_sites(int L, int n_seg, int edge_extra) {
  std::vector<int> size(n_seg, L / n_seg);
  for (int i = 0; i < L % n_seg; ++i) size[i] += 1;
  if (n_seg >= 3 && edge_extra > 0) {
    int spare = 0;
    for (int i = 1; i < n_seg - 1; ++i) spare += size[i] - 2;
    const int take = std::max(0, std::min(edge_extra, spare / 2));
    size[0] += take;
    size[n_seg - 1] += take;
    for (int need = 2 * take, i = 0; need > 0; --need, ++i) size[1 + i % (n_seg - 2)] -= 1;
  }
  std::vector<std::pair<int, int>> out;
  for (int i = 0, s0 = 0; i < n_seg; ++i) {
    out.emplace_back(s0, s0 + size[i] - 1);
    s0 += size[i];
  }
  return out;
}

// Runs fn(0..n-1) on n host threads with the handle's device current; the
// first exception is rethrown here. Kernel launches of the threads are added
// to this thread's launch counter.
template <typename Fn>
void run_threads(tt_fit* h, int n, Fn fn) {
  std::vector<std::thread> th;
  std::vector<long long> launched(n, 0);
  std::mutex mu;
  std::exception_ptr first;
  for (int i = 0; i < n; ++i)
    th.emplace_back([&, i] {
      const long long l0 = tl_launches;
      try {
        CK(cudaSetDevice(h->device));
        fn(i);
      } catch (...) {
        std::lock_guard<std::mutex> g(mu);
        if (!first) first = std::current_exception();
      }
      launched[i] = tl_launches - l0;
      tl_work = nullptr;
    });
  for (auto& t : th) t.join();
  for (long long v : launched) tl_launches += v;
  if (first) std::rethrow_exception(first);
}

// ---------------------------------------------------------------------------
// Site-canonical segment-parallel fit (Sec. 4, the paper's scheme II) and its
// binary merge (Sec. 4.5).
// ---------------------------------------------------------------------------

// QR step of the site gauge at site j (0-based): C_j = Q (left-orthonormal),
// C_{j+1} <- R C_{j+1}, then L_j from the new C_j. FP64 arithmetic on the FP64
// cores, in the lane's factorisation scratch.
template <typename T>
void site_qr_step(tt_fit* h, int j) {
  Dims& D = h->D;
  Work& w = W(h);
  const int q = D.c[j] * D.ds[j] * D.dt[j], p = D.c[j + 1], r = std::min(q, p);
  const int rest = D.ds[j + 1] * D.dt[j + 1] * D.c[j + 2];
  to_colmajor(h, q, p, h->C64[j], w.fX);
  qr(h, q, p, w.fX, w.fQ, w.fR);
  copymap<double, double>(h, q, r, w.fQ, IdxMap::lin(1), IdxMap::lin(q), h->C64[j], IdxMap::lin(r), IdxMap::lin(1));
  copymap<double, T>(h, 1, q * r, w.fQ, IdxMap::lin(0), IdxMap::lin(1), (T*)h->Ut[j], IdxMap::lin(0), IdxMap::lin(1));
  GemmArgs<double> g;  // C_{j+1} <- R C_{j+1} (r x rest)
  g.M = r; g.N = rest; g.K = p;
  g.A = w.fR; g.am = IdxMap::lin(1); g.ak = IdxMap::lin(r); g.a_kfast = false;
  g.B = h->C64[j + 1]; g.bn = IdxMap::lin(1); g.bk = IdxMap::lin(rest); g.b_kfast = false;
  g.C = w.fY; g.cm = IdxMap::lin(rest); g.cn = IdxMap::lin(1);
  gemm<double>(h, g);
  CK(cudaMemcpyAsync(h->C64[j + 1], w.fY, sizeof(double) * (size_t)r * rest, cudaMemcpyDeviceToDevice, w.st));
  D.c[j + 1] = r;
  Chain<T> ch(h);
  ch.half_left(j);
  ch.finish_left(j);
}

// RQ step at site j: C_j = Q^T (right-orthonormal), C_{j-1} <- C_{j-1} R^T, then
// R_j from the new C_j.
template <typename T>
void site_rq_step(tt_fit* h, int j) {
  Dims& D = h->D;
  Work& w = W(h);
  const int q = D.ds[j] * D.dt[j] * D.c[j + 1], p = D.c[j], r = std::min(q, p);
  const int rows = D.c[j - 1] * D.ds[j - 1] * D.dt[j - 1];
  // C_j row-major (p x q) is C_j^T column-major (q x p)
  CK(cudaMemcpyAsync(w.fX, h->C64[j], sizeof(double) * (size_t)q * p, cudaMemcpyDeviceToDevice, w.st));
  qr(h, q, p, w.fX, w.fQ, w.fR);
  // C_j = Q^T (r x q row-major) = Q column-major; the right operand is the same
  CK(cudaMemcpyAsync(h->C64[j], w.fQ, sizeof(double) * (size_t)q * r, cudaMemcpyDeviceToDevice, w.st));
  copymap<double, T>(h, 1, q * r, w.fQ, IdxMap::lin(0), IdxMap::lin(1), (T*)h->Vt[j], IdxMap::lin(0), IdxMap::lin(1));
  GemmArgs<double> g;  // C_{j-1} <- C_{j-1} R^T (rows x r)
  g.M = rows; g.N = r; g.K = p;
  g.A = h->C64[j - 1]; g.am = IdxMap::lin(p); g.ak = IdxMap::lin(1);
  g.B = w.fR; g.bn = IdxMap::lin(1); g.bk = IdxMap::lin(r); g.b_kfast = false;
  g.C = w.fY; g.cm = IdxMap::lin(r); g.cn = IdxMap::lin(1);
  gemm<double>(h, g);
  CK(cudaMemcpyAsync(h->C64[j - 1], w.fY, sizeof(double) * (size_t)rows * r, cudaMemcpyDeviceToDevice, w.st));
  D.c[j] = r;
  Chain<T> ch(h);
  ch.half_right(j);
  ch.finish_right(j);
}

// The consistent sub-TTs after the last phase, as (first site, last site, centre):
// segments joined by that phase's connection updates form one unit each, with
// the centre on the right site of the connection; any other segment is a unit
// with its centre where its local sweep left it.
std::vector<std::array<int, 3>> site_units(const tt_fit* h) {
  const auto& segs = h->segs;
  const int ns = (int)segs.size();
  const int start = h->last_phase == 0 ? 0 : 1;  // first connected boundary (0-based segment)
  std::vector<std::array<int, 3>> units;
  for (int i = 0; i < ns;) {
    if (i >= start && (i - start) % 2 == 0 && i + 1 < ns) {
      units.push_back({segs[i].first, segs[i + 1].second, segs[i + 1].first});
      i += 2;
    } else {
      const bool forward = ((i % 2) == 0) == (h->last_phase == 0);
      units.push_back({segs[i].first, segs[i].second, forward ? segs[i].second : segs[i].first});
      i += 1;
    }
  }
  return units;
}

// Binary merge (Sec. 4.5): neighbouring units are joined pairwise, in rounds;
// the left unit's centre moves to its last site l by QR steps and the right
// unit's to its first site l + 1 by RQ steps, each step finishing the
// environment it passes; then window (l, l+1) is updated forward with both
// environments, drawing the sketches of phase index phases_done + r - 1 in
// round r. The joins of a round touch disjoint sites and run concurrently, each
// on the lane of its left unit's first segment. Returns ||C||^2 of the last
// update (kept sum of s^2, or the FP64-polished projection's).
template <typename T>
double site_merge(tt_fit* h) {
  auto units = site_units(h);
  double n2 = h->cur_n2;
  int lw = -1;
  auto lane_of = [&](int site) {
    for (size_t i = 0; i < h->segs.size(); ++i)
      if (site >= h->segs[i].first && site <= h->segs[i].second) return (int)i;
    return 0;
  };
  CK(cudaEventRecord(h->w0.ev[7], h->w0.st));
  for (auto& w : h->wseg) CK(cudaStreamWaitEvent(w->st, h->w0.ev[7], 0));
  for (int r = 1; units.size() > 1; ++r) {
    const int pairs = (int)units.size() / 2;
    std::vector<double> pn2(pairs, 0.0);
    run_threads(h, pairs, [&](int u) {
      const auto a = units[2 * u], b = units[2 * u + 1];
      tl_work = h->wseg[lane_of(a[0])].get();
      const int l = a[1];
      for (int j = a[2]; j < l; ++j) site_qr_step<T>(h, j);
      for (int j = b[2]; j > l + 1; --j) site_rq_step<T>(h, j);
      Sweeper<T> sw(h);
      double disc = 0;
      sw.window(l, true, h->phases_done + r - 1, pn2[u], disc, Sweeper<T>::ENV_MERGE);
      CK(cudaStreamSynchronize(W(h).st));
      sw.resolve_gauge();
    });
    std::vector<std::array<int, 3>> next;
    for (int u = 0; u < pairs; ++u) {
      next.push_back({units[2 * u][0], units[2 * u + 1][1], units[2 * u][1] + 1});
      n2 = pn2[u];
      lw = units[2 * u][1];
    }
    if (units.size() % 2) next.push_back(units.back());
    units = next;
  }
  for (auto& w : h->wseg) {
    CK(cudaEventRecord(w->ev[7], w->st));
    CK(cudaStreamWaitEvent(h->w0.st, w->ev[7], 0));
  }
  if (lw >= 0 && h->fact_f32) {
    double nr = 0;
    CK(cudaMemcpyAsync(&nr, h->dn2 + lw, sizeof(double), cudaMemcpyDeviceToHost, h->w0.st));
    CK(cudaStreamSynchronize(h->w0.st));
    n2 = nr * nr;
  }
  h->oc_site = units[0][2];
  h->merged = true;
  return n2;
}

// Initialisation of the site-gauge scheme (Sec. 4.2): C right-canonical with
// its centre at site 1 (RQ steps from the right end), which leaves every odd
// segment's centre on its first site; every even segment (1-based) then moves
// its centre to its last site by QR steps; every environment follows from
// these cores. A merged fit is re-partitioned the same way.
template <typename T>
void site_segment_init(tt_fit* h) {
  const int L = h->D.L;
  for (int j = L - 1; j >= 1; --j) site_rq_step<T>(h, j);
  for (size_t i = 1; i < h->segs.size(); i += 2)
    for (int j = h->segs[i].first; j < h->segs[i].second; ++j) site_qr_step<T>(h, j);
  CK(cudaStreamSynchronize(W(h).st));
  h->merged = true;
  h->last_phase = 1;
  h->oc_site = -1;
}

// Initial guess -> inverse canonical (Vidal) form by a left-to-right SVD sweep
// of the right-canonical guess (Sec. 4.2): core j = U S s.t. it is split as
// Psi_j = U S, Y_{j+1} = 1/S, and S V^T is carried into core j+1. Values
// <= cutoff * s_1 are dropped. The SVD is that of the fit's factorisation in
// the handle's factorisation precision.
template <typename T, typename F>
void vidal_init(tt_fit* h) {
  Dims& D = h->D;
  const int L = D.L;
  long long big = 1;
  for (int j = 0; j < L; ++j) big = std::max(big, prodll({D.cb[j], D.ds[j], D.dt[j], D.cb[j + 1]}));
  double* SV = h->pool.alloc<double>(big);  // S V^T, k x n
  double* Cn = h->pool.alloc<double>(big);  // new core j+1
  const int upd = h->update;
  h->update = TT_UPDATE_2SITE_SVD;
  try {
    for (int j = 0; j + 1 < L; ++j) {
      const int m = D.c[j] * D.ds[j] * D.dt[j], n = D.c[j + 1];
      copymap<double, T>(h, m, n, h->C64[j], IdxMap::lin(n), IdxMap::lin(1), (T*)W(h).Th, IdxMap::lin(n),
                         IdxMap::lin(1));
      const int p = factorize<T, F>(h, m, n, 0, j + 1);
      CK(truncate_rule<F>((const F*)W(h).fS, p, W(h).dnorm, 0.0, p, h->cutoff, W(h).dk, W(h).ddinfo, W(h).st));
      CK(cudaMemcpyAsync(W(h).hk, W(h).dk, sizeof(int), cudaMemcpyDeviceToHost, W(h).st));
      CK(cudaMemcpyAsync(W(h).herrw, W(h).errw, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, W(h).st));
      CK(cudaStreamSynchronize(W(h).st));
      check_errw(h, "the inverse-gauge initialisation");
      const int k = *W(h).hk;
      if (k < 1 || k > D.cb[j + 1]) throw TTError(TT_ERR_NUMERICAL, "initial rank outside the bond capacity");
      // Psi_j = U S (m x k), Y_{j+1} = 1/S, SV = S V^T (k x n); Ut_j = U^T is the left operand Psi_j Y_{j+1}
      CK(gauge_update<T, F>(2, m, n, (const F*)W(h).fUM, m, (const F*)W(h).fS, (const F*)W(h).fVM, n, W(h).dk,
                            h->C64[j], SV, h->Y[j + 1], (T*)h->Ut[j], (T*)h->Vt[j + 1], W(h).st));
      // core j+1 <- (S V^T) core j+1
      const int rest = D.ds[j + 1] * D.dt[j + 1] * D.c[j + 2];
      GemmArgs<double> g;
      g.M = k; g.N = rest; g.K = n;
      g.A = SV; g.am = IdxMap::lin(n); g.ak = IdxMap::lin(1);
      g.B = h->C64[j + 1]; g.bn = IdxMap::lin(1); g.bk = IdxMap::lin(rest); g.b_kfast = false;
      g.C = Cn; g.cm = IdxMap::lin(rest); g.cn = IdxMap::lin(1);
      gemm<double>(h, g);
      CK(cudaMemcpyAsync(h->C64[j + 1], Cn, sizeof(double) * (size_t)k * rest, cudaMemcpyDeviceToDevice, W(h).st));
      std::vector<F> sv(k);
      CK(cudaMemcpyAsync(sv.data(), W(h).fS, sizeof(F) * k, cudaMemcpyDeviceToHost, W(h).st));
      CK(cudaStreamSynchronize(W(h).st));
      h->lam[j + 1].assign(sv.begin(), sv.end());
      D.c[j + 1] = k;
    }
  } catch (...) {
    h->update = upd;
    throw;
  }
  h->update = upd;
  CK(cudaStreamSynchronize(W(h).st));
  h->pool.release(SV);
  h->pool.release(Cn);
}

// Every environment and every cached half from the current C (inverse gauge):
// right operands Y_{j} Psi_j, L_1..L_{L-1} with H1_0..H1_{L-2}, and
// R_{L-1}..R_1 with H2_{L-1}..H2_1.
template <typename T>
void all_envs(tt_fit* h) {
  Dims& D = h->D;
  const int L = D.L;
  for (int j = 0; j < L; ++j) {
    const int rows = D.c[j], cols = D.ds[j] * D.dt[j] * D.c[j + 1];
    CK(scale_rows<T>(rows, cols, h->C64[j], j > 0 ? h->Y[j] : nullptr, (T*)h->Vt[j], W(h).st));
    if (j + 1 < L)  // left operand (Psi_j Y_{j+1})^T
      CK(scale_cols_t<T>(D.c[j] * D.ds[j] * D.dt[j], D.c[j + 1], h->C64[j], h->Y[j + 1], (T*)h->Ut[j], W(h).st));
  }
  Chain<T> ch(h);
  for (int j = 0; j + 1 < L; ++j) {
    ch.half_left(j);
    ch.finish_left(j);
  }
  for (int j = L - 1; j >= 1; --j) {
    ch.half_right(j);
    ch.finish_right(j);
  }
  CK(cudaStreamSynchronize(W(h).st));
}

// One phase of Alg. 6 (see tt_fit_sweep in include/ttfit.h); returns ||C||^2
// of its last update in the algorithm's order, and the largest discarded
// fraction of its windows.
template <typename T>
double run_phase(tt_fit* h, int ph, int sweep_index, double& maxd) {
  const int ns = (int)h->segs.size();
  CK(cudaEventRecord(h->w0.ev[7], h->w0.st));  // the lanes start after the handle's queued work
  for (auto& w : h->wseg) CK(cudaStreamWaitEvent(w->st, h->w0.ev[7], 0));
  std::vector<double> n2s(ns, 0.0), dmax(ns, 0.0), cn2(ns, 0.0);
  std::vector<int> lastw(ns, -1);
  // (3)/(5): local half-sweeps, odd segments (1-based) forward in phase 0
  run_threads(h, ns, [&](int i) {
    tl_work = h->wseg[i].get();
    Sweeper<T> sw(h);
    const int s0 = h->segs[i].first, e0 = h->segs[i].second;
    const bool fwd = ((i % 2) == 0) == (ph == 0);
    double n2 = 0, disc = 0;
    if (fwd) {
      for (int l = s0; l <= e0 - 1; ++l) {
        sw.window(l, true, sweep_index, n2, disc, l == s0 ? Sweeper<T>::ENV_NONE : Sweeper<T>::ENV_SERIAL);
        dmax[i] = std::max(dmax[i], disc);
        lastw[i] = l;
      }
    } else {
      for (int l = e0 - 1; l >= s0; --l) {
        sw.window(l, false, sweep_index, n2, disc, l == e0 - 1 ? Sweeper<T>::ENV_NONE : Sweeper<T>::ENV_SERIAL);
        dmax[i] = std::max(dmax[i], disc);
        lastw[i] = l;
      }
    }
    CK(cudaStreamSynchronize(W(h).st));
    sw.resolve_gauge();
    n2s[i] = n2;
  });
  // (4)/(6): connection updates at the odd|even (phase 0) or even|odd (phase 1) boundaries,
  // done by the left segment
  std::vector<int> conns;
  for (int i = 0; i + 1 < ns; ++i)
    if (((i % 2) == 0) == (ph == 0)) conns.push_back(i);
  run_threads(h, (int)conns.size(), [&](int c) {
    const int i = conns[c];
    tl_work = h->wseg[i].get();
    Sweeper<T> sw(h);
    double disc = 0;
    sw.window(h->segs[i].second, true, sweep_index, cn2[i], disc, Sweeper<T>::ENV_CONNECT);
    CK(cudaStreamSynchronize(W(h).st));
    sw.resolve_gauge();
    dmax[i] = std::max(dmax[i], disc);
  });
  for (auto& w : h->wseg) {  // the handle's stream waits for every lane
    CK(cudaEventRecord(w->ev[7], w->st));
    CK(cudaStreamWaitEvent(h->w0.st, w->ev[7], 0));
  }
  maxd = *std::max_element(dmax.begin(), dmax.end());
  int lw;
  double n2;
  if (!conns.empty()) {
    lw = h->segs[conns.back()].second;
    n2 = cn2[conns.back()];
  } else {
    lw = lastw[ns - 1];
    n2 = n2s[ns - 1];
  }
  if (h->fact_f32) {  // ||C||^2 from the FP64-orthonormal projection of that window
    double nr = 0;
    CK(cudaMemcpyAsync(&nr, h->dn2 + lw, sizeof(double), cudaMemcpyDeviceToHost, h->w0.st));
    CK(cudaStreamSynchronize(h->w0.st));
    n2 = nr * nr;
  }
  return n2;
}

// ---------------------------------------------------------------------------
// Input preparation (Alg. 5 left_orthogonalize), shared by the fit and the
// zip-up entry points: an RQ sweep that trims every bond to its rank bound,
// then the QR sweep, for A and B concurrently. The fit is equivariant in the
// scale of A and B, so their last cores (which carry the norms) are then
// scaled by powers of two (exact) to norm ~1 and h->escale records what C
// gets back on export: long chains of normalised random cores (||A B|| ~
// 0.2^L) then stay inside the range of the FP32 / double-FP32 chains.
// mc: largest core of A and B (scratch of the sweeps).
// ---------------------------------------------------------------------------
void prepare_ab(tt_fit* h, long long mc) {
  Dims& D = h->D;
  const int L = D.L;
  Prep PA = make_prep(h, mc), PB = make_prep(h, mc);
  rq_sweep(h, PA, h->A64, D.a, D.ds, D.du, 1, true);
  rq_sweep(h, PB, h->B64, D.b, D.du, D.dt, 1, true);
  qr_sweep(h, PA, h->A64, D.a, D.ds, D.du);
  qr_sweep(h, PB, h->B64, D.b, D.du, D.dt);
  finish_prep(h, PA);
  finish_prep(h, PB);
  auto unit = [&](std::vector<double*>& X, const std::vector<int>& bd, const std::vector<int>& d1,
                  const std::vector<int>& d2) {
    const int j = L - 1;
    const long long n = prodll({bd[j], d1[j], d2[j], bd[j + 1]});
    CK(frob_norm<double>(X[j], n, W(h).dnorm, nullptr, W(h).st));
    double nrm = 0;
    CK(cudaMemcpyAsync(&nrm, W(h).dnorm, sizeof(double), cudaMemcpyDeviceToHost, W(h).st));
    CK(cudaStreamSynchronize(W(h).st));
    if (!(nrm > 0.0) || !std::isfinite(nrm)) return 0;
    const int e = (int)std::lround(std::log2(nrm));
    if (e == 0) return 0;
    double* y = h->pool.alloc<double>(n);
    CK(copy_map<double, double>(1, (int)n, X[j], IdxMap::lin(0), IdxMap::lin(1), y, IdxMap::lin(0), IdxMap::lin(1),
                                std::ldexp(1.0, -e), W(h).st));
    CK(cudaStreamSynchronize(W(h).st));
    h->pool.release(X[j]);
    X[j] = y;
    return e;
  };
  h->escale = unit(h->A64, D.a, D.ds, D.du) + unit(h->B64, D.b, D.du, D.dt);
}

// ---------------------------------------------------------------------------
// Zip-up contraction (Sec. 2.2, Alg. 2), run right to left on the prepared,
// left-canonical A and B: the mirror of the printed left-to-right pass, which
// the paper gives for left-canonical inputs. From site L down to 2, A_l, B_l
// and the remainder R_{l+1} (chi_A x chi x chi_B) contract into M_l, an
// (chi_A chi_B) x (d d' chi) matrix; its truncated factorisation (the fit's
// rule, Sec. 2.3.4) keeps the right singular vectors as C_l (orthonormal rows)
// and R_l = M_l V as the next remainder; site 1 takes the last remainder. C
// comes out right-canonical with the orthogonality centre at site 1, the form
// the fit starts from (Sec. 2.3.5).
// Factorisation of M (m x n):
// * randomized (Sec. 3.1) when k_s = chi_max + oversample < min(m, n): the
//   sketch Y = M^T Omega (Omega m x k_s row-major, Philox stream
//   (3 << 40) | l), its orthonormal basis Q (n x k_s) and Z = M Q (m x k_s);
//   otherwise exact, with Q = I and Z = M;
// * Z by one-sided Jacobi when m <= 1024; a taller Z through its Gram matrix
//   Z^T Z (Jacobi eigenvectors W, s_j = sqrt(eigenvalue)), whose squared
//   condition resolves s_j only down to ~sqrt(eps) s_1: enough for a guess
//   that the sweeps refine;
// * V = Q W, signs fixed as in the fit (largest-magnitude entry positive).
// T: arithmetic of the contractions and the factorisation (double, or float
// for the FP32-class precisions, with 3xTF32 tensor-core contractions for the
// TF32 ones). On return C[l] holds core l (FP64, row-major, bonds cb) and
// cb[1..L-1] the kept bonds.
// ---------------------------------------------------------------------------
inline uint64_t zipup_stream(int site1) { return (3ull << 40) | (uint64_t)site1; }

// Inputs of one zip-up: the two chains (FP64 device cores, row-major) with
// their bonds a, b and legs ds (X out), du (X in = Y out), dt (Y in), and the
// truncation and sketch parameters. The sketch of site l (1-based) draws the
// Philox stream stream_base | l.
struct ZipArgs {
  std::vector<double*> X, Y;
  std::vector<int> a, b, ds, du, dt;
  int chi_max = 1, oversample = 0;
  double tol = 0.0, cutoff = 0.0;
  bool rsvd = false;
  bool project = false;  // range finder only: keep the sketch's range (or M's whole row range), no SVD
  uint64_t stream_base = 3ull << 40;
};

// The zip-up of the fit's prepared A and B with its own parameters.
ZipArgs zip_of_fit(tt_fit* h) {
  ZipArgs z;
  z.X = h->A64;
  z.Y = h->B64;
  z.a = h->D.a;
  z.b = h->D.b;
  z.ds = h->D.ds;
  z.du = h->D.du;
  z.dt = h->D.dt;
  z.chi_max = h->chi_max;
  z.oversample = h->oversample;
  z.tol = h->tol;
  z.cutoff = h->cutoff;
  z.rsvd = h->update == TT_UPDATE_2SITE_RSVD;
  z.stream_base = 3ull << 40;
  return z;
}

// Identity MPO cores (1, d_l, d_l, 1) on the device.
std::vector<double*> identity_chain(tt_fit* h, const std::vector<int>& d) {
  std::vector<double*> I(d.size());
  for (size_t l = 0; l < d.size(); ++l) {
    std::vector<double> eye((size_t)d[l] * d[l], 0.0);
    for (int i = 0; i < d[l]; ++i) eye[(size_t)i * d[l] + i] = 1.0;
    I[l] = h->pool.alloc<double>(eye.size());
    CK(cudaMemcpyAsync(I[l], eye.data(), sizeof(double) * eye.size(), cudaMemcpyHostToDevice, W(h).st));
    CK(cudaStreamSynchronize(W(h).st));
  }
  return I;
}

template <typename T>
void zgemm(tt_fit* h, const GemmArgs<T>& g, T* ws, size_t wse, bool tc) {
  if constexpr (sizeof(T) == 4) {
    if (tc && (long long)g.M * g.N * g.K >= (1ll << 18)) {
      cudaError_t e = gemm_tf32(g, ws, wse, h->sm_count, W(h).errw, W(h).st, true);
      if (e == cudaSuccess) {
        h->tc_launches += 1;
        return;
      }
      if (e != cudaErrorNotSupported) CK(e);
    }
  }
  CK(gemm_simt<T>(g, ws, wse, h->sm_count, W(h).st));
}

template <typename T>
void zipup_rl(tt_fit* h, const ZipArgs& z, std::vector<double*>& C, std::vector<int>& cb) {
  const ZipArgs& D = z;
  const int L = (int)z.X.size();
  Work& w = W(h);
  cudaStream_t st = w.st;
  const bool tc = sizeof(T) == 4 && (h->precision == TT_PREC_TF32 || h->precision == TT_PREC_TF32_SPLIT);
  const int ks = z.chi_max + z.oversample;
  const bool rsvd_on = z.rsvd;
  C.assign(L, nullptr);
  cb.assign(L + 1, 1);
  // scratch for the largest site (chi of the remainder <= min(chi_max, chi_A chi_B of the next site))
  size_t sz_mn = 1, sz_t2 = 1, sz_om = 1, sz_nk = 1, sz_z = 1, sz_zc = 1, sz_u = 1, sz_pp = 1, sz_p = 1, sz_r = 1,
         sz_ab = 1;
  for (int l = 0; l < L; ++l) {
    const long long c = l == L - 1 ? 1 : std::min<long long>(z.chi_max, (long long)D.a[l + 1] * D.b[l + 1]);
    const long long m = (long long)D.a[l] * D.b[l], n = (long long)D.ds[l] * D.dt[l] * c;
    if (n > 1024) throw TTError(TT_ERR_INVALID_ARGUMENT, "zip-up: d d' chi above 1024 at a site");
    const bool rs = rsvd_on && ks < std::min(m, n);
    const long long p = rs ? ks : n;
    sz_mn = std::max<size_t>(sz_mn, m * n);
    sz_t2 = std::max<size_t>(sz_t2, (size_t)D.b[l] * D.dt[l] * c * D.du[l] * D.a[l + 1]);
    sz_ab = std::max<size_t>(sz_ab, std::max(prodll({D.a[l], D.ds[l], D.du[l], D.a[l + 1]}),
                                             prodll({D.b[l], D.du[l], D.dt[l], D.b[l + 1]})));
    if (rs) {
      sz_om = std::max<size_t>(sz_om, m * ks);
      sz_nk = std::max<size_t>(sz_nk, n * ks);
      sz_z = std::max<size_t>(sz_z, m * ks);
    }
    if (z.project && !rs) {  // QR of M^T: its copy and the R factor
      sz_zc = std::max<size_t>(sz_zc, m * n);
      sz_u = std::max<size_t>(sz_u, m * n);
    } else if (!rs && m < n) {
      sz_zc = std::max<size_t>(sz_zc, m * n);
      sz_u = std::max<size_t>(sz_u, m * n);
      sz_pp = std::max<size_t>(sz_pp, m * m);
    } else if (m <= 1024) {
      sz_zc = std::max<size_t>(sz_zc, m * p);
      sz_u = std::max<size_t>(sz_u, m * p);
    } else {
      sz_zc = std::max<size_t>(sz_zc, p * p);
      sz_u = std::max<size_t>(sz_u, p * p);
    }
    sz_pp = std::max<size_t>(sz_pp, p * p);
    sz_p = std::max<size_t>(sz_p, std::max(p, m));
    sz_r = std::max<size_t>(sz_r, m * std::min<long long>(z.chi_max, std::min(m, n)));
  }
  const size_t wse = (size_t)1 << 22;
  std::vector<void*> bufs;
  auto take = [&](size_t n) {
    T* p = h->pool.alloc<T>(n);
    bufs.push_back(p);
    return p;
  };
  T *Mr = take(sz_mn), *Mt = take(sz_mn), *T2 = take(sz_t2), *Om = take(sz_om), *Omt = take(sz_om);
  T *Y = take(sz_nk), *Q = take(sz_nk), *Rq = take((size_t)ks * ks), *Z = take(sz_z), *Zc = take(sz_zc);
  T *Ux = take(sz_u), *Sv = take(sz_p), *Vx = take(sz_pp), *Vw = take(sz_pp), *Vn = take(std::max(sz_nk, sz_mn));
  T *Rc = take(sz_r), *Rn = take(sz_r), *ws = take(wse);
  T *Al = nullptr, *Bl = nullptr;
  if (!std::is_same<T, double>::value) Al = take(sz_ab), Bl = take(sz_ab);
  {  // R_{L+1} = [[[1]]]
    const T one = T(1);
    CK(cudaMemcpyAsync(Rc, &one, sizeof(T), cudaMemcpyHostToDevice, st));
  }
  for (int l = L - 1; l >= 0; --l) {
    const int a0 = D.a[l], a1 = D.a[l + 1], b0 = D.b[l], b1 = D.b[l + 1];
    const int s = D.ds[l], u = D.du[l], t = D.dt[l], c = cb[l + 1];
    const long long m = (long long)a0 * b0, n = (long long)s * t * c;
    const T *Ap, *Bp;
    if constexpr (std::is_same<T, double>::value) {
      Ap = z.X[l];
      Bp = z.Y[l];
    } else {
      const long long na = prodll({a0, s, u, a1}), nb = prodll({b0, u, t, b1});
      copymap<double, T>(h, 1, (int)na, z.X[l], IdxMap::lin(0), IdxMap::lin(1), Al, IdxMap::lin(0), IdxMap::lin(1));
      copymap<double, T>(h, 1, (int)nb, z.Y[l], IdxMap::lin(0), IdxMap::lin(1), Bl, IdxMap::lin(0), IdxMap::lin(1));
      Ap = Al;
      Bp = Bl;
    }
    {  // T2[(b0 t c), (u a1)] = sum_{b1} B_l[(b0 u t), b1] R[(a1 c), b1]
      GemmArgs<T> g;
      g.M = b0 * u * t;
      g.N = a1 * c;
      g.K = b1;
      g.A = Bp;
      g.am = IdxMap::lin(b1);
      g.ak = IdxMap::lin(1);
      g.B = Rc;
      g.bn = IdxMap::lin(b1);
      g.bk = IdxMap::lin(1);
      g.C = T2;
      g.cm = IdxMap::three(u, t, (long long)t * c * u * a1, a1, (long long)c * u * a1);
      g.cn = IdxMap::two(c, 1, (long long)u * a1);
      zgemm<T>(h, g, ws, wse, tc);
    }
    {  // M[(a0 b0), (s t c)] = sum_{(u a1)} A_l[(a0 s), (u a1)] T2[(b0 t c), (u a1)], also as M^T
      GemmArgs<T> g;
      g.M = a0 * s;
      g.N = b0 * t * c;
      g.K = u * a1;
      g.A = Ap;
      g.am = IdxMap::lin((long long)u * a1);
      g.ak = IdxMap::lin(1);
      g.B = T2;
      g.bn = IdxMap::lin((long long)u * a1);
      g.bk = IdxMap::lin(1);
      g.C = Mr;
      g.cm = IdxMap::two(s, (long long)b0 * n, (long long)t * c);
      g.cn = IdxMap::three(t, c, n, c, 1);
      g.C2 = Mt;
      g.cm2 = IdxMap::two(s, b0, (long long)t * c * m);
      g.cn2 = IdxMap::three(t, c, 1, (long long)c * m, m);
      zgemm<T>(h, g, ws, wse, tc);
    }
    if (l == 0) {  // a0 = b0 = 1: the remainder is the first core
      C[0] = h->pool.alloc<double>(n);
      copymap<T, double>(h, 1, (int)n, Mr, IdxMap::lin(0), IdxMap::lin(1), C[0], IdxMap::lin(0), IdxMap::lin(1));
      break;
    }
    CK(frob_norm<T>(Mr, m * n, w.dnorm, w.errw, st));
    const bool rs = rsvd_on && ks < std::min(m, n);
    int p = (int)n;
    const T* Zp = Mt;  // Z column-major m x p
    if (rs) {
      p = ks;
      CK(philox_fill<T>(Om, m * ks, h->seed, z.stream_base | (uint64_t)(l + 1), 1.0, st));
      copymap<T, T>(h, (int)m, ks, Om, IdxMap::lin(ks), IdxMap::lin(1), Omt, IdxMap::lin(1), IdxMap::lin(m));
      GemmArgs<T> g;  // Y (n x k_s, column-major) = M^T Omega
      g.M = (int)n;
      g.N = ks;
      g.K = (int)m;
      g.A = Mt;
      g.am = IdxMap::lin(m);
      g.ak = IdxMap::lin(1);
      g.B = Omt;
      g.bn = IdxMap::lin(m);
      g.bk = IdxMap::lin(1);
      g.C = Y;
      g.cm = IdxMap::lin(1);
      g.cn = IdxMap::lin(n);
      zgemm<T>(h, g, ws, wse, tc);
      CK(qr_householder<T, T>((int)n, ks, Y, Q, Rq, st));
      GemmArgs<T> z;  // Z (m x k_s, column-major) = M Q
      z.M = (int)m;
      z.N = ks;
      z.K = (int)n;
      z.A = Mr;
      z.am = IdxMap::lin(n);
      z.ak = IdxMap::lin(1);
      z.B = Q;
      z.bn = IdxMap::lin(n);
      z.bk = IdxMap::lin(1);
      z.C = Z;
      z.cm = IdxMap::lin(1);
      z.cn = IdxMap::lin(m);
      zgemm<T>(h, z, ws, wse, tc);
      Zp = Z;
    }
    // C_l = V^T (k x (s t c)): V column-major is V^T row-major; R_l[a0, k, b0] = (M V)[(a0 b0), k]
    auto emit = [&](int k) {
      cb[l] = k;
      C[l] = h->pool.alloc<double>((size_t)k * n);
      copymap<T, double>(h, 1, (int)(k * n), Vn, IdxMap::lin(0), IdxMap::lin(1), C[l], IdxMap::lin(0),
                         IdxMap::lin(1));
      GemmArgs<T> g;
      g.M = (int)m;
      g.N = k;
      g.K = (int)n;
      g.A = Mr;
      g.am = IdxMap::lin(n);
      g.ak = IdxMap::lin(1);
      g.B = Vn;
      g.bn = IdxMap::lin(n);
      g.bk = IdxMap::lin(1);
      g.C = Rn;
      g.cm = IdxMap::two(b0, (long long)k * b0, 1);
      g.cn = IdxMap::lin(b0);
      zgemm<T>(h, g, ws, wse, tc);
      std::swap(Rc, Rn);
    };
    if (z.project) {  // range finder only (Sec. 3): V = Q, or M's whole row range where k_s >= min(m, n)
      if (rs) {
        CK(cudaMemcpyAsync(Vn, Q, sizeof(T) * n * ks, cudaMemcpyDeviceToDevice, st));
        emit(ks);
      } else {
        CK(cudaMemcpyAsync(Zc, Mr, sizeof(T) * m * n, cudaMemcpyDeviceToDevice, st));  // M^T, column-major
        CK(qr_householder<T, T>((int)n, (int)m, Zc, Vn, Ux, st));
        emit((int)std::min(m, n));
      }
      continue;
    }
    int pv = p;        // singular values in Sv, V = Vn (n x pv column-major)
    T* W_ = nullptr;   // V = Q W when randomized
    if (!rs && m < n) {  // M^T (n x m, column-major = M row-major) is the tall side: M^T = Ux S Vx^T
      CK(cudaMemcpyAsync(Zc, Mr, sizeof(T) * m * n, cudaMemcpyDeviceToDevice, st));
      CK(jacobi_svd<T, T>((int)n, (int)m, Zc, Vn, Sv, Vx, Vw, 60, w.errw, st));
      pv = (int)m;
    } else if (m <= 1024) {  // Z = Ux S W^T
      CK(cudaMemcpyAsync(Zc, Zp, sizeof(T) * m * p, cudaMemcpyDeviceToDevice, st));
      CK(jacobi_svd<T, T>((int)m, p, Zc, Ux, Sv, rs ? Vx : Vn, Vw, 60, w.errw, st));
      W_ = rs ? Vx : nullptr;
    } else {  // Gram matrix Z^T Z = W S^2 W^T
      GemmArgs<T> g;
      g.M = p;
      g.N = p;
      g.K = (int)m;
      g.A = Zp;
      g.am = IdxMap::lin(m);
      g.ak = IdxMap::lin(1);
      g.B = Zp;
      g.bn = IdxMap::lin(m);
      g.bk = IdxMap::lin(1);
      g.C = Zc;
      g.cm = IdxMap::lin(1);
      g.cn = IdxMap::lin(p);
      zgemm<T>(h, g, ws, wse, tc);
      CK(jacobi_svd<T, T>(p, p, Zc, Ux, Sv, rs ? Vx : Vn, Vw, 60, w.errw, st));
      CK(sqrt_clamp<T>(p, Sv, st));
      W_ = rs ? Vx : nullptr;
    }
    if (W_) {  // V = Q W (n x k_s)
      GemmArgs<T> g;
      g.M = (int)n;
      g.N = p;
      g.K = p;
      g.A = Q;
      g.am = IdxMap::lin(1);
      g.ak = IdxMap::lin(n);
      g.a_kfast = false;
      g.B = W_;
      g.bn = IdxMap::lin(p);
      g.bk = IdxMap::lin(1);
      g.C = Vn;
      g.cm = IdxMap::lin(1);
      g.cn = IdxMap::lin(n);
      zgemm<T>(h, g, ws, wse, false);
    }
    CK(fix_signs<T>((int)n, 0, pv, Vn, (int)n, nullptr, 0, st));
    CK(truncate_rule<T>(Sv, pv, w.dnorm, z.tol / L, z.chi_max, z.cutoff, w.dk, w.ddinfo, st));
    CK(cudaMemcpyAsync(w.hk, w.dk, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(w.herrw, w.errw, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    check_errw(h, ("zip-up site " + std::to_string(l + 1)).c_str());
    const int k = *w.hk;
    if (k < 1 || k > pv) throw TTError(TT_ERR_NUMERICAL, "zip-up: invalid kept rank");
    emit(k);
  }
  CK(cudaMemcpyAsync(w.herrw, w.errw, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  check_errw(h, "the zip-up");
  for (void* b : bufs) h->pool.release(b);
}

// Randomized bond projection of the A and B chains (Sec. 3.2): a rank-k
// projector on every bond, drawn once, since the fit never changes A or B.
// Each prepared (left-canonical) chain is swept right to left as its zip-up
// with the identity MPO, keeping the k-column Gaussian range of every bond
// (streams (4 << 40) | l for A, (5 << 40) | l for B; bonds narrower than k stay
// whole), in FP64 arithmetic. The fit does not depend on the gauge of A and B,
// so the projected chains stay right-canonical, unless the zip-up guess follows
// (left_canonical): it sketches the bonds of left-canonical chains, so they are
// brought back to that form by the QR sweep first.
// The contractions of the fit then run on bonds of at most k.
void project_ab(tt_fit* h, int k, long long mc, bool left_canonical) {
  Dims& D = h->D;
  for (int which = 0; which < 2; ++which) {
    std::vector<double*>& X = which ? h->B64 : h->A64;
    std::vector<int>& bx = which ? D.b : D.a;
    const std::vector<int>& dout = which ? D.du : D.ds;
    const std::vector<int>& din = which ? D.dt : D.du;
    ZipArgs z;
    z.X = X;
    z.Y = identity_chain(h, din);
    z.a = bx;
    z.b.assign(D.L + 1, 1);
    z.ds = dout;
    z.du = din;
    z.dt = din;
    z.chi_max = k;
    z.oversample = 0;
    z.tol = 0.0;
    z.cutoff = 0.0;
    z.rsvd = true;
    z.project = true;
    z.stream_base = (uint64_t)(4 + which) << 40;
    std::vector<double*> P;
    std::vector<int> pb;
    zipup_rl<double>(h, z, P, pb);  // FP64 in every precision: a one-off O(L chi^3) pass
    for (double* p : z.Y) h->pool.release(p);
    for (double* p : X) h->pool.release(p);
    X = P;
    bx = pb;
    if (left_canonical) {
      Prep PX = make_prep(h, mc);
      qr_sweep(h, PX, X, bx, dout, din);
      finish_prep(h, PX);
    }
  }
}

void setup(tt_fit* h, const std::vector<double*>& C0) {
  Dims& D = h->D;
  const int L = D.L;
  // C state: FP64 cores at capacity size, Y per bond = 1
  h->C64.assign(L, nullptr);
  h->Y.assign(L + 1, nullptr);
  h->lam.assign(L + 1, {});
  for (int j = 0; j < L; ++j) {
    const long long cap = prodll({D.cb[j], D.ds[j], D.dt[j], D.cb[j + 1]});
    h->C64[j] = h->pool.alloc<double>(cap);
    const long long n = prodll({D.c[j], D.ds[j], D.dt[j], D.c[j + 1]});
    CK(cudaMemcpyAsync(h->C64[j], C0[j], sizeof(double) * n, cudaMemcpyDeviceToDevice, W(h).st));
  }
  std::vector<double> ones(1024, 1.0);
  for (int j = 0; j <= L; ++j) {
    h->Y[j] = h->pool.alloc<double>(std::max(D.cb[j], 1));
    int n = D.c[j];
    for (int off = 0; off < n; off += 1024)
      CK(cudaMemcpyAsync(h->Y[j] + off, ones.data(), sizeof(double) * std::min(1024, n - off), cudaMemcpyHostToDevice,
                         W(h).st));
  }
  if (h->use_f32) rebuild_chain<float>(h);
  else if (h->use_df) rebuild_chain<df32>(h);
  else rebuild_chain<double>(h);
}

// Runs fn(i) for i < n on n host threads with device `dev` current; returns
// the first non-OK status (by index).
template <typename Fn>
tt_status run_handles(int n, int dev, Fn fn) {
  std::vector<tt_status> st(n, TT_OK);
  std::vector<std::thread> th;
  for (int i = 0; i < n; ++i)
    th.emplace_back([&, i] {
      if (cudaSetDevice(dev) != cudaSuccess) {
        st[i] = TT_ERR_CUDA;
        return;
      }
      st[i] = fn(i);
    });
  for (auto& t : th) t.join();
  for (tt_status x : st)
    if (x != TT_OK) return x;
  return TT_OK;
}

thread_local std::string g_create_error;

void poison(tt_fit* h, const TTError& e) {
  h->poisoned = true;
  h->last_error = e.what();
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* tt_status_string(tt_status s) {
  switch (s) {
    case TT_OK: return "ok";
    case TT_ERR_INVALID_ARGUMENT: return "invalid argument";
    case TT_ERR_SHAPE_MISMATCH: return "shape mismatch";
    case TT_ERR_OUT_OF_MEMORY: return "out of device memory";
    case TT_ERR_CUDA: return "CUDA error";
    case TT_ERR_NUMERICAL: return "numerical failure";
    case TT_ERR_TIMEOUT: return "device wait timed out";
    case TT_ERR_STATE: return "invalid handle state";
  }
  return "unknown status";
}

const char* tt_fit_last_error(const tt_fit* h) {
  if (h) return h->last_error.c_str();
  return g_create_error.empty() ? "NULL handle" : g_create_error.c_str();
}

// Adds the kernel launches issued on this thread while it lives to h->launches.
struct LaunchTally {
  tt_fit* h;
  long long l0;
  explicit LaunchTally(tt_fit* hh) : h(hh), l0(tl_launches) {}
  ~LaunchTally() {
    if (h) h->launches += tl_launches - l0;
  }
};

}  // extern "C"

namespace {

// Shared body of tt_mpo_zipup and tt_mpo_compress (B == nullptr: the identity
// MPO on X's input legs). A handle without a fit holds the prepared inputs,
// the lane (stream, flags) and the scratch; it is freed before returning.
tt_status zipup_entry(const char* what, const tt_mpo_desc* A, const tt_mpo_desc* B, int chi_max, double tol,
                      const tt_fit_options* opt, const tt_mpo_desc* Cd, int* bond_out) {
  g_create_error.clear();
  if (!Cd || !bond_out || chi_max < 1 || !(tol >= 0.0)) return TT_ERR_INVALID_ARGUMENT;
  tt_fit_options o{};
  o.struct_size = sizeof(o);
  o.update = TT_UPDATE_2SITE_SVD;
  o.oversample = 10;
  o.precision = TT_PREC_FP64;
  o.sv_cutoff = -1;
  o.prepare_inputs = 1;
  if (opt) {
    if (opt->struct_size != sizeof(tt_fit_options)) return TT_ERR_INVALID_ARGUMENT;
    o = *opt;
  }
  if (o.update != 0 && o.update != 1) return TT_ERR_INVALID_ARGUMENT;
  if (o.precision < 0 || o.precision > 5 || o.precision == TT_PREC_BF16_SPLIT || o.oversample < 0)
    return TT_ERR_INVALID_ARGUMENT;
  std::unique_ptr<tt_fit> hold(new tt_fit());
  tt_fit* h = hold.get();
  bool lane = false;
  try {
    int LA, LB, LC;
    std::vector<int> doA, diA, bA, doB, diB, bB, doC, diC, bC;
    read_desc(A, LA, doA, diA, bA);
    if (B) {
      read_desc(B, LB, doB, diB, bB);
    } else {  // identity: d_out = d_in = A.d_in, bond 1
      LB = LA;
      doB = diA;
      diB = diA;
      bB.assign(LA + 1, 1);
    }
    read_desc(Cd, LC, doC, diC, bC);
    if (LA != LB || LC != LA) return TT_ERR_SHAPE_MISMATCH;
    for (int l = 0; l < LA; ++l)
      if (diA[l] != doB[l] || doC[l] != doA[l] || diC[l] != diB[l]) return TT_ERR_SHAPE_MISMATCH;
    LaunchTally tally(h);
    h->L = LA;
    h->chi_max = chi_max;
    h->tol = tol;
    h->update = o.update;
    h->oversample = o.oversample;
    h->precision = o.precision;
    h->seed = o.seed;
    h->use_f32 = (o.precision != TT_PREC_FP64 && o.precision != TT_PREC_DF32);
    h->cutoff = o.sv_cutoff >= 0 ? o.sv_cutoff : default_cutoff(o.precision, h->use_f32);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev));
    h->device = dev;
    init_lane(h, h->w0, (cudaStream_t)o.stream, false);
    lane = true;
    Dims& D = h->D;
    D.L = LA;
    D.ds = doA;
    D.du = diA;
    D.dt = diB;
    D.a = bA;
    D.b = bB;
    upload(h, A, doA, diA, bA, h->A64);
    if (B) {
      upload(h, B, doB, diB, bB, h->B64);
    } else {
      h->B64 = identity_chain(h, diA);
    }
    CK(cudaStreamSynchronize(W(h).st));
    long long mc = 1;
    for (int l = 0; l < LA; ++l) {
      mc = std::max(mc, prodll({bA[l], doA[l], diA[l], bA[l + 1]}));
      mc = std::max(mc, prodll({bB[l], doB[l], diB[l], bB[l + 1]}));
    }
    if (o.prepare_inputs) prepare_ab(h, mc);
    std::vector<double*> Cc;
    std::vector<int> cb;
    const ZipArgs z = zip_of_fit(h);
    if (h->use_f32) zipup_rl<float>(h, z, Cc, cb);
    else zipup_rl<double>(h, z, Cc, cb);
    for (int l = 0; l <= LA; ++l)
      if (cb[l] > bC[l]) throw TTError(TT_ERR_SHAPE_MISMATCH, "a kept bond exceeds C.bond");
    for (int l = 0; l < LA; ++l) {
      const long long n = prodll({cb[l], doA[l], diB[l], cb[l + 1]});
      const double sc = l == 0 ? std::ldexp(1.0, h->escale) : 1.0;
      if (Cd->dtype == TT_DTYPE_F64)
        CK(copy_map<double, double>(1, (int)n, Cc[l], IdxMap::lin(0), IdxMap::lin(1), (double*)Cd->cores[l],
                                    IdxMap::lin(0), IdxMap::lin(1), sc, W(h).st));
      else
        CK(copy_map<double, float>(1, (int)n, Cc[l], IdxMap::lin(0), IdxMap::lin(1), (float*)Cd->cores[l],
                                   IdxMap::lin(0), IdxMap::lin(1), sc, W(h).st));
    }
    CK(cudaStreamSynchronize(W(h).st));
    for (int l = 0; l <= LA; ++l) bond_out[l] = cb[l];
    free_lanes(h);
    return TT_OK;
  } catch (const TTError& e) {
    g_create_error = std::string(what) + ": " + e.what();
    cudaGetLastError();
    cudaDeviceSynchronize();
    if (lane) free_lanes(h);
    return e.code;
  } catch (const std::bad_alloc&) {
    cudaDeviceSynchronize();
    if (lane) free_lanes(h);
    return TT_ERR_OUT_OF_MEMORY;
  } catch (...) {
    cudaDeviceSynchronize();
    if (lane) free_lanes(h);
    return TT_ERR_CUDA;
  }
}

}  // namespace

extern "C" {

tt_status tt_mpo_zipup(const tt_mpo_desc* A, const tt_mpo_desc* B, int chi_max, double tol,
                       const tt_fit_options* opt, const tt_mpo_desc* C, int* bond_out) {
  if (!B) return TT_ERR_INVALID_ARGUMENT;
  return zipup_entry("tt_mpo_zipup", A, B, chi_max, tol, opt, C, bond_out);
}

tt_status tt_mpo_compress(const tt_mpo_desc* X, int chi_max, double tol, const tt_fit_options* opt,
                          const tt_mpo_desc* C, int* bond_out) {
  return zipup_entry("tt_mpo_compress", X, nullptr, chi_max, tol, opt, C, bond_out);
}

tt_status tt_fit_create(const tt_mpo_desc* A, const tt_mpo_desc* B, int chi_max, double tol, int gauge,
                        const tt_fit_options* opt, tt_fit** out) {
  if (!out) return TT_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  g_create_error.clear();
  tt_fit* h = nullptr;
  try {
    if (chi_max < 1 || !(tol >= 0.0) || (gauge != 0 && gauge != 1)) return TT_ERR_INVALID_ARGUMENT;
    tt_fit_options o{};
    o.struct_size = sizeof(o);
    o.update = TT_UPDATE_2SITE_SVD;
    o.oversample = 10;
    o.precision = TT_PREC_FP64;
    o.init = TT_INIT_RANDOM;
    o.sv_cutoff = -1;
    o.conv_tol = -1;
    o.prepare_inputs = 1;
    if (opt) {
      if (opt->struct_size != sizeof(tt_fit_options)) return TT_ERR_INVALID_ARGUMENT;
      o = *opt;
    }
    if (o.update != 0 && o.update != 1) return TT_ERR_INVALID_ARGUMENT;
    if (o.precision < 0 || o.precision > 5 || o.oversample < 0) return TT_ERR_INVALID_ARGUMENT;
    if (o.init < 0 || o.init > 3 || (o.init == TT_INIT_GIVEN && !o.init_C)) return TT_ERR_INVALID_ARGUMENT;
    // BF16_SPLIT is the DF32 chain whose digit-split contractions run on BF16 digit planes
    const bool oz_bf16 = o.precision == TT_PREC_BF16_SPLIT;
    if (oz_bf16) o.precision = TT_PREC_DF32;
    if (o.edge_extra < 0) return TT_ERR_INVALID_ARGUMENT;
    if (o.fast_factor < 0 || o.fast_factor > 3) return TT_ERR_INVALID_ARGUMENT;
    if (o.ab_rank < 0 || (o.ab_rank > 0 && !o.prepare_inputs)) return TT_ERR_INVALID_ARGUMENT;
    int LA, LB;
    std::vector<int> doA, diA, bA, doB, diB, bB;
    read_desc(A, LA, doA, diA, bA);
    read_desc(B, LB, doB, diB, bB);
    if (LA != LB) return TT_ERR_SHAPE_MISMATCH;
    if (LA < 2) return TT_ERR_INVALID_ARGUMENT;
    if (o.n_segments > 1 && LA < 2 * o.n_segments) return TT_ERR_INVALID_ARGUMENT;  // >= 2 sites per segment
    for (int l = 0; l < LA; ++l)
      if (diA[l] != doB[l]) return TT_ERR_SHAPE_MISMATCH;
    h = new tt_fit();
    LaunchTally tally(h);
    h->fault = o.fault_inject;
    h->pool.fault = o.fault_inject & TT_FAULT_ALLOC_FAIL;
    h->fault_nan_pending = (o.fault_inject & TT_FAULT_NAN_INPUT) != 0;
    h->fault_noconv_pending = (o.fault_inject & TT_FAULT_SVD_NOCONV) != 0;
    h->L = LA;
    h->chi_max = chi_max;
    h->tol = tol;
    h->gauge = gauge;
    h->update = o.update;
    h->oversample = o.oversample;
    h->precision = o.precision;
    h->init = o.init;
    h->seed = o.seed;
    h->use_f32 = (o.precision != TT_PREC_FP64 && o.precision != TT_PREC_DF32);
    h->use_df = (o.precision == TT_PREC_DF32);
    h->oz_bf16 = oz_bf16;
    h->fact_f32 = h->use_f32 || o.fast_factor;
    h->fast_factor = o.fast_factor;
    h->cutoff_user = o.sv_cutoff >= 0;
    h->cutoff = h->cutoff_user ? o.sv_cutoff : default_cutoff(o.precision, h->fact_f32);
    h->conv_tol = o.conv_tol >= 0 ? o.conv_tol : tol;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev));
    h->device = dev;
    init_lane(h, h->w0, (cudaStream_t)o.stream, false);
    if (o.n_segments > 1) {  // Alg. 6: one lane (stream, scratch, host thread) per segment
      h->segs = partition_sites(LA, o.n_segments, o.edge_extra);
      for (int i = 0; i < o.n_segments; ++i) {
        h->wseg.emplace_back(new Work());
        cudaStream_t sti = nullptr;
        CK(cudaStreamCreateWithFlags(&sti, cudaStreamNonBlocking));
        init_lane(h, *h->wseg.back(), sti, true);
      }
    }
    Dims& D = h->D;
    D.L = LA;
    D.ds = doA;
    D.du = diA;
    D.dt = diB;
    D.a = bA;
    D.b = bB;
    upload(h, A, doA, diA, bA, h->A64);
    upload(h, B, doB, diB, bB, h->B64);
    CK(cudaStreamSynchronize(W(h).st));
    long long mc = 1;  // largest core of A, B (and a given guess): scratch of the preparation sweeps
    for (int l = 0; l < LA; ++l) {
      mc = std::max(mc, prodll({bA[l], doA[l], diA[l], bA[l + 1]}));
      mc = std::max(mc, prodll({bB[l], doB[l], diB[l], bB[l + 1]}));
    }
    if (o.init == TT_INIT_GIVEN) {
      const tt_mpo_desc* g = o.init_C;
      if (g->L == LA && g->bond && g->d_out && g->d_in)
        for (int l = 0; l < LA; ++l) mc = std::max(mc, prodll({g->bond[l], g->d_out[l], g->d_in[l], g->bond[l + 1]}));
    }
    // capacity of C bonds: min(chi_max, prod of local dims to the left / right)
    const int L = LA;
    D.cb.assign(L + 1, 1);
    for (int l = 1; l < L; ++l) {
      double left = 1, right = 1;
      for (int j = 0; j < l; ++j) left *= (double)D.ds[j] * D.dt[j];
      for (int j = l; j < L; ++j) right *= (double)D.ds[j] * D.dt[j];
      D.cb[l] = (int)std::min<double>(chi_max, std::min(left, right));
    }
    // initial guess (right-canonical, orthogonality centre at site 1). The random one does not
    // depend on A or B: it is drawn on its own pool of streams while A and B are prepared.
    std::vector<double*> C0(L);
    std::vector<int> cbond;
    struct StreamPool {  // destroyed on every exit, after its work has finished
      cudaStream_t s[8] = {};
      ~StreamPool() {
        for (auto& x : s)
          if (x) cudaStreamSynchronize(x), cudaStreamDestroy(x);
      }
    } guess_streams;
    const int NS = 8;
    cudaStream_t* pool = guess_streams.s;
    std::vector<void*> dead;
    if (o.init == TT_INIT_RANDOM) {
      cbond = D.cb;
      // core l >= 2: orthonormal-row factor of a Gaussian matrix; the cores are
      // independent, so their QRs run concurrently on the pool
      for (int i = 0; i < NS; ++i) CK(cudaStreamCreateWithFlags(&pool[i], cudaStreamNonBlocking));
      CK(cudaStreamSynchronize(W(h).st));
      for (int j = 0; j < L; ++j) {
        cudaStream_t sj = pool[j % NS];
        const long long n = prodll({cbond[j], D.ds[j], D.dt[j], cbond[j + 1]});
        C0[j] = h->pool.alloc<double>(n);
        CK(philox_fill<double>(C0[j], n, h->seed, init_stream(j + 1), 1.0, sj));
        if (j > 0) {  // q >= p by the bond rule
          const int q = D.ds[j] * D.dt[j] * cbond[j + 1], p = cbond[j];
          double* R = h->pool.alloc<double>((size_t)p * p);
          double* Q = h->pool.alloc<double>((size_t)q * p);
          if (h->precision == TT_PREC_FP64) CK(qr_householder<double, double>(q, p, C0[j], Q, R, sj));
          else CK(qr_householder_df32(q, p, C0[j], Q, R, sj));
          dead.push_back(C0[j]);
          dead.push_back(R);
          C0[j] = Q;
        }
      }
    }
    if (o.prepare_inputs) prepare_ab(h, mc);  // Alg. 5: left_orthogonalize(A), left_orthogonalize(B)
    if (o.ab_rank > 0) project_ab(h, o.ab_rank, mc, o.init == TT_INIT_ZIPUP);
    if (o.init == TT_INIT_RANDOM) {
      for (int i = 0; i < NS; ++i) {
        CK(cudaStreamSynchronize(pool[i]));
        cudaStreamDestroy(pool[i]);
        pool[i] = nullptr;
      }
      for (void* d : dead) h->pool.release(d);
    } else if (o.init == TT_INIT_ZIPUP) {  // Sec. 2.3.5: the zip-up contraction of A and B
      const ZipArgs z = zip_of_fit(h);
      if (h->use_f32) zipup_rl<float>(h, z, C0, cbond);
      else zipup_rl<double>(h, z, C0, cbond);
      for (int l = 1; l < L; ++l) D.cb[l] = std::max(D.cb[l], cbond[l]);
    } else {
      std::vector<int> dz, bz;
      const tt_mpo_desc* src = (o.init == TT_INIT_COPY_B) ? nullptr : o.init_C;
      std::vector<double*> G;
      if (src) {
        int LC;
        std::vector<int> doC, diC;
        read_desc(src, LC, doC, diC, bz);
        if (LC != L) throw TTError(TT_ERR_SHAPE_MISMATCH, "init_C length");
        for (int l = 0; l < L; ++l)
          if (doC[l] != D.ds[l] || diC[l] != D.dt[l]) throw TTError(TT_ERR_SHAPE_MISMATCH, "init_C local dims");
        upload(h, src, doC, diC, bz, G);
      } else {
        bz = D.b;
        G.resize(L);
        for (int l = 0; l < L; ++l) {
          const long long n = prodll({bz[l], D.du[l], D.dt[l], bz[l + 1]});
          G[l] = h->pool.alloc<double>(n);
          CK(cudaMemcpyAsync(G[l], h->B64[l], sizeof(double) * n, cudaMemcpyDeviceToDevice, W(h).st));
        }
        if (D.du != D.ds) throw TTError(TT_ERR_SHAPE_MISMATCH, "TT_INIT_COPY_B needs A.d_out == B.d_out");
      }
      CK(cudaStreamSynchronize(W(h).st));
      Prep PC = make_prep(h, mc);
      qr_sweep(h, PC, G, bz, D.ds, D.dt);
      rq_sweep(h, PC, G, bz, D.ds, D.dt, 1, false);
      finish_prep(h, PC);
      for (int l = 1; l < L; ++l) D.cb[l] = std::max(D.cb[l], bz[l]);
      C0 = G;
      cbond = bz;
    }
    D.c = cbond;
    setup(h, C0);
    if (h->segs.size() > 1 && gauge == TT_GAUGE_SITE_CANONICAL) {  // scheme II (Sec. 4.2)
      if (h->use_f32) {
        site_segment_init<float>(h);
        all_envs<float>(h);
      } else if (h->use_df) {
        site_segment_init<df32>(h);
        all_envs<df32>(h);
      } else {
        site_segment_init<double>(h);
        all_envs<double>(h);
      }
    } else if (h->segs.size() > 1) {  // inverse canonical form and every environment (Sec. 4.2)
      if (h->use_f32) {
        vidal_init<float, float>(h);
        all_envs<float>(h);
      } else if (h->use_df) {
        if (h->fact_f32) vidal_init<df32, float>(h);
        else vidal_init<df32, double>(h);
        all_envs<df32>(h);
      } else if (h->fact_f32) {
        vidal_init<double, float>(h);
        all_envs<double>(h);
      } else {
        vidal_init<double, double>(h);
        all_envs<double>(h);
      }
    }
    CK(cudaStreamSynchronize(W(h).st));
    for (auto* w : lanes(h))
    if (w->st) CK(cudaStreamSynchronize(w->st));
    for (int j = 0; j < L; ++j) h->pool.release(C0[j]);
    *out = h;
    return TT_OK;
  } catch (const TTError& e) {
    // preparation and guess streams may still run: let everything finish before
    // the handle's blocks go back to the process-wide cache
    g_create_error = std::string("tt_fit_create: ") + e.what();
    if (h) {
      cudaGetLastError();
      cudaDeviceSynchronize();
      free_lanes(h);
      delete h;
    }
    return e.code;
  } catch (const std::bad_alloc&) {
    if (h) {
      cudaDeviceSynchronize();
      free_lanes(h);
    }
    delete h;
    return TT_ERR_OUT_OF_MEMORY;
  } catch (...) {
    if (h) {
      cudaDeviceSynchronize();
      free_lanes(h);
    }
    delete h;
    return TT_ERR_CUDA;
  }
}

tt_status tt_fit_sweep(tt_fit* h, int n_sweeps, tt_sweep_report* rep) {
  if (!h || n_sweeps < 0) return TT_ERR_INVALID_ARGUMENT;
  if (h->poisoned) return TT_ERR_STATE;
  auto t0 = std::chrono::steady_clock::now();
  LaunchTally tally(h);
  try {
    for (Work* w : lanes(h)) {
      for (double& s : w->stage_ms) s = 0;
      w->flops = 0;
      w->tc_flops = 0;
      w->cc_flops = 0;
    }
    const long long launch0 = tl_launches;
    if (h->segs.size() > 1) {
      for (int s = 0; s < n_sweeps && !h->converged; ++s) {
        const int ph = h->phases_done % 2;
        double maxd = 0;
        h->hp_sweep = use_hp_basis(h);
        const double n2 = h->use_f32  ? run_phase<float>(h, ph, h->phases_done, maxd)
                          : h->use_df ? run_phase<df32>(h, ph, h->phases_done, maxd)
                                      : run_phase<double>(h, ph, h->phases_done, maxd);
        h->phases_done++;
        h->sweeps_done++;
        h->cur_n2 = n2;
        if (h->gauge == TT_GAUGE_SITE_CANONICAL) {  // the units carry their own centres until merged
          h->merged = false;
          h->last_phase = ph;
          h->oc_site = -1;
        }
        h->max_disc = maxd;
        if (ph == 1) {  // a full set of local sweeps is complete
          h->delta = (h->last_n2 >= 0 && n2 > 0) ? std::fabs(n2 - h->last_n2) / n2 : INFINITY;
          h->last_n2 = n2;
          if (h->delta <= h->conv_tol) h->converged = true;
        }
      }
    } else if (h->use_f32) {
      Sweeper<float> sw(h);
      sw.run(n_sweeps);
    } else if (h->use_df) {
      Sweeper<df32> sw(h);
      sw.run(n_sweeps);
    } else {
      Sweeper<double> sw(h);
      sw.run(n_sweeps);
    }
    CK(cudaStreamSynchronize(W(h).st));
    h->sweep_launches = tl_launches - launch0;
    h->have_times = true;
  } catch (const TTError& e) {
    poison(h, e);
    return e.code;
  } catch (...) {
    h->poisoned = true;
    h->last_error = "unexpected exception";
    return TT_ERR_CUDA;
  }
  if (rep) {
    rep->sweeps_done = h->sweeps_done;
    rep->converged = h->converged ? 1 : 0;
    rep->delta = h->delta;
    rep->norm2_C = std::ldexp(h->segs.size() > 1 ? h->cur_n2 : h->last_n2, 2 * h->escale);
    rep->max_discarded = h->max_disc;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return TT_OK;
}

tt_status tt_fit_merge(tt_fit* h, tt_sweep_report* rep) {
  if (!h) return TT_ERR_INVALID_ARGUMENT;
  if (h->poisoned) return TT_ERR_STATE;
  auto t0 = std::chrono::steady_clock::now();
  LaunchTally tally(h);
  try {
    if (!h->merged) {
      h->cur_n2 = h->use_f32  ? site_merge<float>(h)
                  : h->use_df ? site_merge<df32>(h)
                              : site_merge<double>(h);
      CK(cudaStreamSynchronize(h->w0.st));
    }
  } catch (const TTError& e) {
    poison(h, e);
    return e.code;
  }
  if (rep) {
    rep->sweeps_done = h->sweeps_done;
    rep->converged = h->converged ? 1 : 0;
    rep->delta = h->delta;
    rep->norm2_C = std::ldexp(h->segs.size() > 1 ? h->cur_n2 : h->last_n2, 2 * h->escale);
    rep->max_discarded = h->max_disc;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return TT_OK;
}

tt_status tt_fit_result(const tt_fit* hc, tt_mpo_desc* C, double* lambdas) {
  tt_fit* h = const_cast<tt_fit*>(hc);
  if (!h || !C) return TT_ERR_INVALID_ARGUMENT;
  LaunchTally tally(h);
  if (h->poisoned) return TT_ERR_STATE;
  if (!h->merged) {
    h->last_error = "tt_fit_result: the site-gauge segments are not merged (tt_fit_merge)";
    return TT_ERR_STATE;
  }
  const Dims& D = h->D;
  const int L = D.L;
  C->L = L;
  if (!C->d_out || !C->d_in || !C->bond) return TT_ERR_INVALID_ARGUMENT;
  int* dout = const_cast<int*>(C->d_out);
  int* din = const_cast<int*>(C->d_in);
  int* bond = const_cast<int*>(C->bond);
  for (int l = 0; l < L; ++l) {
    dout[l] = D.ds[l];
    din[l] = D.dt[l];
  }
  for (int l = 0; l <= L; ++l) bond[l] = D.c[l];
  try {
    const double sc = std::ldexp(1.0, h->escale);  // the scale taken off A and B at create time
    if (lambdas) {
      size_t off = 0;
      for (int l = 1; l < L; ++l) {
        const std::vector<double>& v = h->lam[l];
        for (int j = 0; j < D.c[l]; ++j) lambdas[off + j] = (j < (int)v.size()) ? sc * v[j] : 0.0;
        off += D.c[l];
      }
    }
    if (!C->cores) return TT_OK;
    if (C->dtype != TT_DTYPE_F64 && C->dtype != TT_DTYPE_F32) return TT_ERR_INVALID_ARGUMENT;
    for (int l = 0; l < L; ++l) {
      if (!C->cores[l]) return TT_ERR_INVALID_ARGUMENT;
      const int rows = D.c[l] * D.ds[l] * D.dt[l], cols = D.c[l + 1];
      // C_l = Psi_l Y_l for l < L (inverse gauge); Y = 1 in the site gauge
      const bool scale = (h->gauge == TT_GAUGE_INVERSE_CANONICAL) && (l < L - 1);
      // the input scale goes back into the orthogonality centre, so that the other cores keep
      // their canonical form: in the site gauge the last core after a forward sweep, else the first
      const int oc = h->oc_site >= 0 ? h->oc_site
                     : (h->gauge != TT_GAUGE_INVERSE_CANONICAL && !h->forward && h->segs.size() <= 1) ? L - 1 : 0;
      const double f = l == oc ? sc : 1.0;
      if (C->dtype == TT_DTYPE_F64 && f == 1.0) {
        CK(scale_cols(rows, cols, h->C64[l], scale ? h->Y[l + 1] : nullptr, (double*)C->cores[l], W(h).st));
      } else {
        double* tmp = h->pool.alloc<double>((size_t)rows * cols);
        CK(scale_cols(rows, cols, h->C64[l], scale ? h->Y[l + 1] : nullptr, tmp, W(h).st));
        if (C->dtype == TT_DTYPE_F64)
          CK(copy_map<double, double>(1, rows * cols, tmp, IdxMap::lin(0), IdxMap::lin(1), (double*)C->cores[l],
                                      IdxMap::lin(0), IdxMap::lin(1), f, W(h).st));
        else
          CK(copy_map<double, float>(1, rows * cols, tmp, IdxMap::lin(0), IdxMap::lin(1), (float*)C->cores[l],
                                     IdxMap::lin(0), IdxMap::lin(1), f, W(h).st));
        CK(cudaStreamSynchronize(W(h).st));
        h->pool.release(tmp);
      }
    }
    CK(cudaStreamSynchronize(W(h).st));
  } catch (const TTError& e) {
    poison(h, e);
    return e.code;
  }
  return TT_OK;
}

tt_status tt_fit_set_precision(tt_fit* h, int precision, int fast_factor) {
  if (!h || precision < 0 || precision > 5) return TT_ERR_INVALID_ARGUMENT;
  const bool oz_bf16 = precision == TT_PREC_BF16_SPLIT;  // the DF32 chain on BF16 digit planes
  if (oz_bf16) precision = TT_PREC_DF32;
  if (fast_factor < 0 || fast_factor > 3) return TT_ERR_INVALID_ARGUMENT;
  if (h->poisoned) return TT_ERR_STATE;
  if (h->segs.size() > 1 && h->phases_done % 2 != 0) {
    h->last_error = "tt_fit_set_precision: a segment-parallel fit switches between full sets of local sweeps";
    return TT_ERR_STATE;
  }
  if (h->segs.size() > 1 && h->gauge == TT_GAUGE_SITE_CANONICAL && !h->merged) {
    h->last_error = "tt_fit_set_precision: merge the site-gauge segments first (tt_fit_merge)";
    return TT_ERR_STATE;
  }
  LaunchTally tally(h);
  try {
    const bool f32 = precision != TT_PREC_FP64 && precision != TT_PREC_DF32;
    h->precision = precision;
    h->use_f32 = f32;
    h->use_df = precision == TT_PREC_DF32;
    h->oz_bf16 = oz_bf16;
    h->fact_f32 = f32 || fast_factor;
    h->fast_factor = fast_factor;
    if (!h->cutoff_user) h->cutoff = default_cutoff(precision, h->fact_f32);
    h->converged = false;
    if (f32) rebuild_chain<float>(h);
    else if (h->use_df) rebuild_chain<df32>(h);
    else rebuild_chain<double>(h);
    if (h->segs.size() > 1 && h->gauge == TT_GAUGE_SITE_CANONICAL) {
      // merged C, back to the scheme's initial gauge, every environment in the new type
      if (f32) site_segment_init<float>(h), all_envs<float>(h);
      else if (h->use_df) site_segment_init<df32>(h), all_envs<df32>(h);
      else site_segment_init<double>(h), all_envs<double>(h);
    } else if (h->segs.size() > 1) {  // the parallel fit needs every environment and half
      if (f32) all_envs<float>(h);
      else if (h->use_df) all_envs<df32>(h);
      else all_envs<double>(h);
    }
  } catch (const TTError& e) {
    poison(h, e);
    return e.code;
  }
  return TT_OK;
}

tt_status tt_fit_stage_times(const tt_fit* h, double out[7]) {
  if (!h || !out) return TT_ERR_INVALID_ARGUMENT;
  if (!h->have_times) return TT_ERR_STATE;
  for (int i = 0; i < 6; ++i) out[i] = 0;
  for (Work* w : lanes(const_cast<tt_fit*>(h))) {  // summed over the lanes (concurrent in a parallel fit)
    for (int i = 0; i < 5; ++i) out[i] += w->stage_ms[i];
    out[5] += w->flops;
  }
  out[6] = (double)h->sweep_launches;
  return TT_OK;
}

tt_status tt_fit_exec_flops(const tt_fit* h, double out[2]) {
  if (!h || !out) return TT_ERR_INVALID_ARGUMENT;
  if (!h->have_times) return TT_ERR_STATE;
  out[0] = out[1] = 0;
  for (Work* w : lanes(const_cast<tt_fit*>(h))) {
    out[0] += w->tc_flops;
    out[1] += w->cc_flops;
  }
  return TT_OK;
}

tt_status tt_partition(int L, int n_segments, int edge_extra, int* first, int* last) {
  if (L < 2 || n_segments < 1 || L < 2 * n_segments || edge_extra < 0 || !first || !last)
    return TT_ERR_INVALID_ARGUMENT;
  const auto segs = partition_sites(L, n_segments, edge_extra);
  for (int i = 0; i < n_segments; ++i) {
    first[i] = segs[i].first;
    last[i] = segs[i].second;
  }
  return TT_OK;
}

tt_status tt_fit_create_batched(int n, const tt_mpo_desc* A, const tt_mpo_desc* B, const int* chi_max, double tol,
                                int gauge, int n_segments, const tt_fit_options* opt, tt_fit** out) {
  if (n < 1 || !A || !B || !chi_max || !out) return TT_ERR_INVALID_ARGUMENT;
  for (int i = 0; i < n; ++i) out[i] = nullptr;
  tt_fit_options o{};
  o.struct_size = sizeof(o);
  o.update = TT_UPDATE_2SITE_SVD;
  o.oversample = 10;
  o.precision = TT_PREC_FP64;
  o.init = TT_INIT_RANDOM;
  o.sv_cutoff = -1;
  o.conv_tol = -1;
  o.prepare_inputs = 1;
  if (opt) {
    if (opt->struct_size != sizeof(tt_fit_options)) return TT_ERR_INVALID_ARGUMENT;
    o = *opt;
  }
  if (o.init == TT_INIT_GIVEN) return TT_ERR_INVALID_ARGUMENT;  // one guess cannot serve n pairs
  o.n_segments = n_segments;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TT_ERR_CUDA;
  // every handle gets a stream of its own, ordered after the caller's stream (where A, B were written)
  cudaStream_t caller = (cudaStream_t)o.stream;
  cudaEvent_t ready = nullptr;
  if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) return TT_ERR_CUDA;
  if (cudaEventRecord(ready, caller) != cudaSuccess) {
    cudaEventDestroy(ready);
    return TT_ERR_CUDA;
  }
  std::vector<cudaStream_t> sts(n, nullptr);
  tt_status r = TT_OK;
  for (int i = 0; i < n && r == TT_OK; ++i)
    if (cudaStreamCreateWithFlags(&sts[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamWaitEvent(sts[i], ready, 0) != cudaSuccess)
      r = TT_ERR_CUDA;
  if (r == TT_OK)
    r = run_handles(n, dev, [&](int i) {
      tt_fit_options oi = o;
      oi.stream = sts[i];
      tt_status si = tt_fit_create(&A[i], &B[i], chi_max[i], tol, gauge, &oi, &out[i]);
      if (si == TT_OK) {
        out[i]->w0.own_stream = true;  // destroyed with the handle
        sts[i] = nullptr;
      }
      return si;
    });
  cudaEventDestroy(ready);
  for (cudaStream_t x : sts)
    if (x) cudaStreamDestroy(x);
  if (r != TT_OK)
    for (int i = 0; i < n; ++i) {
      tt_fit_destroy(out[i]);
      out[i] = nullptr;
    }
  return r;
}

tt_status tt_fit_sweep_batched(int n, tt_fit* const* h, int n_sweeps, tt_sweep_report* rep) {
  if (n < 1 || !h || n_sweeps < 0) return TT_ERR_INVALID_ARGUMENT;
  for (int i = 0; i < n; ++i)
    if (!h[i]) return TT_ERR_INVALID_ARGUMENT;
  return run_handles(n, h[0]->device, [&](int i) { return tt_fit_sweep(h[i], n_sweeps, rep ? &rep[i] : nullptr); });
}

tt_status tt_fit_launch_count(const tt_fit* h, long long* n) {
  if (!h || !n) return TT_ERR_INVALID_ARGUMENT;
  *n = h->launches;
  return TT_OK;
}

size_t tt_device_cache_release(int device) { return block_cache().trim(device); }

tt_status tt_fit_jacobi_sweeps(const tt_fit* h, int* max_sweeps) {
  if (!h || !max_sweeps) return TT_ERR_INVALID_ARGUMENT;
  int m = 0;
  for (Work* w : lanes(const_cast<tt_fit*>(h)))
    if (w->herrw) m = std::max(m, (int)w->herrw[1]);
  *max_sweeps = m;
  return TT_OK;
}

void tt_fit_destroy(tt_fit* h) {
  if (!h) return;
  if (h->w0.st) cudaStreamSynchronize(h->w0.st);
  else cudaDeviceSynchronize();
  free_lanes(h);
  delete h;
}

}  // extern "C"
