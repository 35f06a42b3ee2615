// Adjoint of the fit's contraction chain: gradients of
//   f1(A, B) = ||X - A B||_F^2   (X = C, held fixed)   and
//   f2(A, B) = <X, A B> = tr(X^T A B)   (X = W, fixed)
// with respect to every core of A and B.
//
// <X, AB> is the three-layer network of the fit's environments (Sec. 2.3.3,
// Fig. envs); its derivative with respect to one core is the same network with
// that core cut out. ||AB||^2 = <AB, AB> is the four-layer network of two
// copies of A, B; each core occurs once per copy and the network is symmetric
// in the copies, so its derivative is twice the punched hole of one copy.
// Left environments are kept at every k-th site (checkpoints) and the ones in
// between are recomputed from the nearest checkpoint while the gradients are
// formed from right to left with running right environments.
//
// Every contraction is one GEMM on this library's kernels: the legs of each
// operand are grouped into M, N and K index maps (legs adjacent in memory in
// every tensor that carries them are fused), so no tensor is permuted in
// memory.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ttfit.h"
#include "common.cuh"
#include "kernels.h"

using namespace ttfit;

namespace {

struct GradError : std::runtime_error {
  tt_status code;
  GradError(tt_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define GK(...)                                                                                        \
  do {                                                                                                 \
    cudaError_t e_ = (__VA_ARGS__);                                                                    \
    if (e_ != cudaSuccess)                                                                             \
      throw GradError(e_ == cudaErrorMemoryAllocation ? TT_ERR_OUT_OF_MEMORY : TT_ERR_CUDA,             \
                      std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

// Device buffers owned by one call.
struct Arena {
  std::vector<void*> ptrs;
  template <typename T>
  T* alloc(size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      throw GradError(TT_ERR_OUT_OF_MEMORY, "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed");
    }
    ptrs.push_back(p);
    return (T*)p;
  }
  ~Arena() {
    for (void* p : ptrs) cudaFree(p);
  }
};

using Ext = std::map<char, long long>;

// A row-major tensor: its device data and the names of its legs, outermost first.
template <typename T>
struct Tn {
  T* p;
  std::string legs;
};

template <typename T>
struct Ctx {
  cudaStream_t st = nullptr;
  int sm_count = 1;
  T* ws = nullptr;  // split-K workspace
  size_t ws_elems = 0;
  bool tc = false;  // FP32: 3xTF32 products on the tensor cores
  Arena* ar = nullptr;
  T *sa = nullptr, *sb = nullptr;  // K-major copies of the operands of large tensor-core products
  size_t sa_n = 0, sb_n = 0;
};

long long stride_of(const std::string& legs, char c, const Ext& ext) {
  long long s = 1;
  for (int i = (int)legs.size() - 1; i >= 0; --i) {
    if (legs[i] == c) return s;
    s *= ext.at(legs[i]);
  }
  throw GradError(TT_ERR_INVALID_ARGUMENT, std::string("leg ") + c + " not in " + legs);
}

// One index group (M, N or K) of a GEMM: its legs in order, fused where the
// legs are adjacent in memory in all the tensors given, as an IdxMap of <= 3 levels.
IdxMap group_map(const std::vector<std::pair<long long, long long>>& dims) {  // (extent, stride), outer first
  if (dims.empty()) return IdxMap::lin(0);
  if (dims.size() == 1) return IdxMap::lin(dims[0].second);
  if (dims.size() == 2) return IdxMap::two((int)dims[1].first, dims[0].second, dims[1].second);
  return IdxMap::three((int)dims[1].first, (int)dims[2].first, dims[0].second, dims[1].second, dims[2].second);
}

struct Group {
  std::vector<std::vector<char>> dims;  // fused legs, outer first
  long long size = 1;
};

Group make_group(const std::string& order, const std::vector<const std::string*>& tensors, const Ext& ext) {
  Group g;
  for (char c : order) {
    g.size *= ext.at(c);
    if (!g.dims.empty()) {
      const char prev = g.dims.back().back();
      bool fuse = true;
      for (const std::string* t : tensors)
        if (stride_of(*t, prev, ext) != ext.at(c) * stride_of(*t, c, ext)) fuse = false;
      if (fuse) {
        g.dims.back().push_back(c);
        continue;
      }
    }
    g.dims.push_back({c});
  }
  if (g.dims.size() > 3) throw GradError(TT_ERR_INVALID_ARGUMENT, "contraction group with more than 3 strided legs");
  return g;
}

IdxMap map_in(const Group& g, const std::string& legs, const Ext& ext) {
  std::vector<std::pair<long long, long long>> d;
  for (const auto& f : g.dims) {
    long long e = 1;
    for (char c : f) e *= ext.at(c);
    d.emplace_back(e, stride_of(legs, f.back(), ext));
  }
  return group_map(d);
}

// C = alpha * contraction(A, B) + beta * C; the contracted legs are those of A
// and B that C does not carry.
template <typename T>
void einsum(Ctx<T>& cx, const Tn<const T>& A, const Tn<const T>& B, const Tn<T>& C, const Ext& ext, T alpha = T(1),
            T beta = T(0)) {
  std::string m, n, k;
  for (char c : A.legs) {
    const bool inB = B.legs.find(c) != std::string::npos, inC = C.legs.find(c) != std::string::npos;
    if (inC && !inB) m += c;
    else if (inB && !inC) k += c;
    else throw GradError(TT_ERR_INVALID_ARGUMENT, std::string("unsupported leg ") + c);
  }
  for (char c : B.legs) {
    const bool inA = A.legs.find(c) != std::string::npos, inC = C.legs.find(c) != std::string::npos;
    if (inC && !inA) n += c;
    else if (!(inA && !inC)) throw GradError(TT_ERR_INVALID_ARGUMENT, std::string("unsupported leg ") + c);
  }
  if (m.size() + n.size() != C.legs.size()) throw GradError(TT_ERR_INVALID_ARGUMENT, "output legs");
  const Group gm = make_group(m, {&A.legs, &C.legs}, ext);
  const Group gn = make_group(n, {&B.legs, &C.legs}, ext);
  const Group gk = make_group(k, {&A.legs, &B.legs}, ext);
  GemmArgs<T> g;
  g.M = (int)gm.size;
  g.N = (int)gn.size;
  g.K = (int)gk.size;
  g.A = A.p;
  g.am = map_in(gm, A.legs, ext);
  g.ak = map_in(gk, A.legs, ext);
  g.a_kfast = !k.empty() && A.legs.back() == k.back();
  g.B = B.p;
  g.bn = map_in(gn, B.legs, ext);
  g.bk = map_in(gk, B.legs, ext);
  g.b_kfast = !k.empty() && B.legs.back() == k.back();
  g.C = C.p;
  g.cm = map_in(gm, C.legs, ext);
  g.cn = map_in(gn, C.legs, ext);
  g.alpha = alpha;
  g.beta = beta;
  if constexpr (sizeof(T) == 4) {
    if (cx.tc && (long long)g.M * g.N * g.K >= (1ll << 18)) {
      cudaError_t e = gemm_tf32(g, cx.ws, cx.ws_elems, cx.sm_count, nullptr, cx.st, true);
      if (e == cudaSuccess) return;
      if (e != cudaErrorNotSupported) GK(e);
      // a large product whose operands TMA cannot load as they lie: copy them K-major first
      // (O(size) against the O(M N K) of the product)
      if ((long long)g.M * g.N * g.K >= (1ll << 24) && g.K % 4 == 0 && cx.ar) {
        const size_t na = (size_t)g.M * g.K, nb = (size_t)g.N * g.K;
        if (na > cx.sa_n) cx.sa = cx.ar->template alloc<T>(na), cx.sa_n = na;
        if (nb > cx.sb_n) cx.sb = cx.ar->template alloc<T>(nb), cx.sb_n = nb;
        GK(copy_map<T, T>(g.M, g.K, g.A, g.am, g.ak, cx.sa, IdxMap::lin(g.K), IdxMap::lin(1), 1.0, cx.st));
        GK(copy_map<T, T>(g.N, g.K, g.B, g.bn, g.bk, cx.sb, IdxMap::lin(g.K), IdxMap::lin(1), 1.0, cx.st));
        GemmArgs<T> h = g;
        h.A = cx.sa;
        h.am = IdxMap::lin(g.K);
        h.ak = IdxMap::lin(1);
        h.a_kfast = true;
        h.B = cx.sb;
        h.bn = IdxMap::lin(g.K);
        h.bk = IdxMap::lin(1);
        h.b_kfast = true;
        e = gemm_tf32(h, cx.ws, cx.ws_elems, cx.sm_count, nullptr, cx.st, true);
        if (e == cudaSuccess) return;
        if (e != cudaErrorNotSupported) GK(e);
      }
    }
  }
  GK(gemm_simt<T>(g, cx.ws, cx.ws_elems, cx.sm_count, cx.st));
}

// ---------------------------------------------------------------------------
// the adjoint sweep in working type T
// ---------------------------------------------------------------------------
template <typename T>
struct Grad {
  Ctx<T> cx;
  Arena& ar;
  int L = 0;
  std::vector<int> a, b, c, ds, du, dt;  // bonds (L+1) and local dims
  std::vector<T*> A, B, X;               // cores in T
  bool four = false;                     // f1 needs the four-layer terms
  int k_ckpt = 1;
  T *s1 = nullptr, *s2 = nullptr, *s3 = nullptr;  // contraction scratch
  Grad(Arena& arena) : ar(arena) {}

  Ext ext_site(int l) const {
    // legs: a,b,c left bonds (A, B, X); x,y,z right bonds; s = out, u = middle, t = in;
    // second copy (four layers): p, q left, z, w right, v middle
    return Ext{{'a', a[l]}, {'b', b[l]}, {'c', c[l]}, {'x', a[l + 1]}, {'y', b[l + 1]}, {'z', c[l + 1]},
               {'s', ds[l]}, {'u', du[l]}, {'t', dt[l]}};
  }
  Ext ext4(int l) const {
    return Ext{{'a', a[l]}, {'b', b[l]},     {'p', a[l]},     {'q', b[l]},     {'x', a[l + 1]}, {'y', b[l + 1]},
               {'z', a[l + 1]}, {'w', b[l + 1]}, {'s', ds[l]}, {'u', du[l]}, {'v', du[l]}, {'t', dt[l]}};
  }
  const T* cp(T* p) { return p; }

  // three layers: E[a b c] -> E'[x y z]
  void left3(int l, const T* E, T* out) {
    Ext e = ext_site(l);
    einsum<T>(cx, {E, "abc"}, {A[l], "asux"}, {s1, "bcsux"}, e);
    einsum<T>(cx, {s1, "bcsux"}, {B[l], "buty"}, {s2, "csxty"}, e);
    einsum<T>(cx, {s2, "csxty"}, {X[l], "cstz"}, {out, "xyz"}, e);
  }
  // three layers: R[x y z] -> R'[a b c]
  void right3(int l, const T* R, T* out) {
    Ext e = ext_site(l);
    einsum<T>(cx, {A[l], "asux"}, {R, "xyz"}, {s1, "asuyz"}, e);
    einsum<T>(cx, {s1, "asuyz"}, {B[l], "buty"}, {s2, "asbtz"}, e);
    einsum<T>(cx, {s2, "asbtz"}, {X[l], "cstz"}, {out, "abc"}, e);
  }
  // punched holes of <X, AB> at A_l and B_l: gA = alpha * hole + beta * gA
  void holes3(int l, const T* E, const T* R, T* gA, T* gB, T alpha, T beta) {
    Ext e = ext_site(l);
    einsum<T>(cx, {E, "abc"}, {X[l], "cstz"}, {s1, "abstz"}, e);
    einsum<T>(cx, {s1, "abstz"}, {B[l], "buty"}, {s2, "aszuy"}, e);
    einsum<T>(cx, {s2, "aszuy"}, {R, "xyz"}, {gA, "asux"}, e, alpha, beta);
    einsum<T>(cx, {E, "abc"}, {A[l], "asux"}, {s1, "bcsux"}, e);
    einsum<T>(cx, {s1, "bcsux"}, {X[l], "cstz"}, {s2, "buxtz"}, e);
    einsum<T>(cx, {s2, "buxtz"}, {R, "xyz"}, {gB, "buty"}, e, alpha, beta);
  }
  // four layers: F[a b p q] -> F'[x y z w]
  void left4(int l, const T* F, T* out) {
    Ext e = ext4(l);
    einsum<T>(cx, {F, "abpq"}, {A[l], "asux"}, {s1, "bpqsux"}, e);
    einsum<T>(cx, {s1, "bpqsux"}, {B[l], "buty"}, {s2, "pqsxty"}, e);
    einsum<T>(cx, {s2, "pqsxty"}, {A[l], "psvz"}, {s1, "qxtyvz"}, e);
    einsum<T>(cx, {s1, "qxtyvz"}, {B[l], "qvtw"}, {out, "xyzw"}, e);
  }
  // four layers: G[x y z w] -> G'[a b p q]
  void right4(int l, const T* G, T* out) {
    Ext e = ext4(l);
    einsum<T>(cx, {B[l], "qvtw"}, {G, "xyzw"}, {s1, "qvtxyz"}, e);
    einsum<T>(cx, {A[l], "psvz"}, {s1, "qvtxyz"}, {s2, "psqtxy"}, e);
    einsum<T>(cx, {B[l], "buty"}, {s2, "psqtxy"}, {s1, "bupsqx"}, e);
    einsum<T>(cx, {A[l], "asux"}, {s1, "bupsqx"}, {out, "abpq"}, e);
  }
  // punched holes of ||AB||^2 (one copy, times 2 by symmetry): g += 2 * hole
  void holes4(int l, const T* F, const T* G, T* gA, T* gB) {
    Ext e = ext4(l);
    einsum<T>(cx, {F, "abpq"}, {A[l], "psvz"}, {s1, "abqsvz"}, e);
    einsum<T>(cx, {s1, "abqsvz"}, {B[l], "qvtw"}, {s2, "abszwt"}, e);
    einsum<T>(cx, {s2, "abszwt"}, {B[l], "buty"}, {s1, "aszwuy"}, e);
    einsum<T>(cx, {s1, "aszwuy"}, {G, "xyzw"}, {gA, "asux"}, e, T(2), T(1));
    einsum<T>(cx, {F, "abpq"}, {A[l], "asux"}, {s1, "bpqsux"}, e);
    einsum<T>(cx, {s1, "bpqsux"}, {A[l], "psvz"}, {s2, "bquxvz"}, e);
    einsum<T>(cx, {s2, "bquxvz"}, {B[l], "qvtw"}, {s1, "buxztw"}, e);
    einsum<T>(cx, {s1, "buxztw"}, {G, "xyzw"}, {gB, "buty"}, e, T(2), T(1));
  }
  // ||X||^2 by two-layer transfer: N[c c'] -> N'[z z']
  void left2(int l, const T* N, T* out) {
    Ext e{{'c', c[l]}, {'d', c[l]}, {'z', c[l + 1]}, {'w', c[l + 1]}, {'s', ds[l]}, {'t', dt[l]}};
    einsum<T>(cx, {N, "cd"}, {X[l], "dstw"}, {s1, "cstw"}, e);
    einsum<T>(cx, {s1, "cstw"}, {X[l], "cstz"}, {out, "zw"}, e);
  }
};

template <typename T>
double read_scalar(const T* p, cudaStream_t st) {
  T v{};
  GK(cudaMemcpyAsync(&v, p, sizeof(T), cudaMemcpyDeviceToHost, st));
  GK(cudaStreamSynchronize(st));
  return (double)v;
}

void read_mpo(const tt_mpo_desc* d, int& L, std::vector<int>& dout, std::vector<int>& din, std::vector<int>& bond) {
  if (!d || d->L < 1 || !d->d_out || !d->d_in || !d->bond || !d->cores) throw GradError(TT_ERR_INVALID_ARGUMENT, "MPO");
  if (d->dtype != TT_DTYPE_F64 && d->dtype != TT_DTYPE_F32) throw GradError(TT_ERR_INVALID_ARGUMENT, "dtype");
  L = d->L;
  dout.assign(d->d_out, d->d_out + L);
  din.assign(d->d_in, d->d_in + L);
  bond.assign(d->bond, d->bond + L + 1);
  if (bond[0] != 1 || bond[L] != 1) throw GradError(TT_ERR_SHAPE_MISMATCH, "boundary bonds must be 1");
  for (int l = 0; l < L; ++l)
    if (dout[l] < 1 || din[l] < 1 || bond[l] < 1 || !d->cores[l]) throw GradError(TT_ERR_INVALID_ARGUMENT, "core");
}

template <typename T>
T* load_cores(Arena& ar, const tt_mpo_desc* d, int l, long long n, cudaStream_t st) {
  T* out = ar.alloc<T>(n);
  const IdxMap id = IdxMap::lin(1), z = IdxMap::lin(0);
  if (d->dtype == TT_DTYPE_F64) GK(copy_map<double, T>(1, (int)n, (const double*)d->cores[l], z, id, out, z, id, 1.0, st));
  else GK(copy_map<float, T>(1, (int)n, (const float*)d->cores[l], z, id, out, z, id, 1.0, st));
  return out;
}

template <typename T>
void store_cores(const T* in, const tt_mpo_desc* d, int l, long long n, cudaStream_t st) {
  const IdxMap id = IdxMap::lin(1), z = IdxMap::lin(0);
  if (d->dtype == TT_DTYPE_F64) GK(copy_map<T, double>(1, (int)n, in, z, id, (double*)d->cores[l], z, id, 1.0, st));
  else GK(copy_map<T, float>(1, (int)n, in, z, id, (float*)d->cores[l], z, id, 1.0, st));
}

template <typename T>
double run_grad(const tt_mpo_desc* Ad, const tt_mpo_desc* Bd, const tt_mpo_desc* Xd, int target, int ckpt,
                cudaStream_t st, const tt_mpo_desc* gAd, const tt_mpo_desc* gBd, bool tc = false) {
  Arena ar;
  Grad<T> G(ar);
  int LA, LB, LX, LgA, LgB;
  std::vector<int> doA, diA, bA, doB, diB, bB, doX, diX, bX, o1, i1, b1, o2, i2, b2;
  read_mpo(Ad, LA, doA, diA, bA);
  read_mpo(Bd, LB, doB, diB, bB);
  read_mpo(Xd, LX, doX, diX, bX);
  read_mpo(gAd, LgA, o1, i1, b1);
  read_mpo(gBd, LgB, o2, i2, b2);
  if (LA != LB || LA != LX || LgA != LA || LgB != LA) throw GradError(TT_ERR_SHAPE_MISMATCH, "lengths");
  const int L = LA;
  for (int l = 0; l < L; ++l) {
    if (diA[l] != doB[l] || doX[l] != doA[l] || diX[l] != diB[l]) throw GradError(TT_ERR_SHAPE_MISMATCH, "legs");
    if (o1[l] != doA[l] || i1[l] != diA[l] || o2[l] != doB[l] || i2[l] != diB[l])
      throw GradError(TT_ERR_SHAPE_MISMATCH, "gradient legs");
  }
  if (b1 != bA || b2 != bB) throw GradError(TT_ERR_SHAPE_MISMATCH, "gradient bonds");
  int dev = 0;
  GK(cudaGetDevice(&dev));
  GK(cudaDeviceGetAttribute(&G.cx.sm_count, cudaDevAttrMultiProcessorCount, dev));
  G.cx.st = st;
  G.cx.tc = tc;
  G.cx.ar = &ar;
  G.L = L;
  G.a = bA;
  G.b = bB;
  G.c = bX;
  G.ds = doA;
  G.du = diA;
  G.dt = diB;
  G.four = (target == TT_GRAD_RESIDUAL);
  G.k_ckpt = ckpt > 0 ? ckpt : std::max(1, (int)std::ceil(std::sqrt((double)L)));  // 0: about sqrt(L)
  // scratch: the largest intermediate of any contraction (leg strings as used by Grad)
  auto size_of = [](const char* legs, const Ext& e) {
    long long n = 1;
    for (const char* c = legs; *c; ++c) n *= e.at(*c);
    return n;
  };
  long long big = 1, e3 = 1, e4 = 1, core = 1;
  for (int l = 0; l < L; ++l) {
    const Ext x3 = G.ext_site(l);
    for (const char* legs : {"bcsux", "csxty", "asuyz", "asbtz", "abstz", "aszuy", "buxtz"})
      big = std::max(big, size_of(legs, x3));
    big = std::max(big, (long long)bX[l] * doX[l] * diX[l] * bX[l + 1]);  // two-layer step
    e3 = std::max({e3, (long long)bA[l] * bB[l] * bX[l], (long long)bA[l + 1] * bB[l + 1] * bX[l + 1]});
    core = std::max({core, (long long)bA[l] * doA[l] * diA[l] * bA[l + 1], (long long)bB[l] * doB[l] * diB[l] * bB[l + 1]});
    if (G.four) {
      const Ext x4 = G.ext4(l);
      for (const char* legs : {"bpqsux", "pqsxty", "qxtyvz", "qvtxyz", "psqtxy", "bupsqx", "abqsvz", "abszwt",
                               "aszwuy", "bquxvz", "buxztw"})
        big = std::max(big, size_of(legs, x4));
      e4 = std::max({e4, (long long)bA[l] * bB[l] * bA[l] * bB[l], (long long)bA[l + 1] * bB[l + 1] * bA[l + 1] * bB[l + 1]});
    }
  }
  long long maxc2 = 1;
  for (int l = 0; l <= L; ++l) maxc2 = std::max<long long>(maxc2, (long long)bX[l] * bX[l]);
  G.s1 = ar.alloc<T>(big);
  G.s2 = ar.alloc<T>(big);
  G.cx.ws_elems = (size_t)std::min<long long>(big, 1ll << 26) + (1 << 20);
  G.cx.ws = ar.alloc<T>(G.cx.ws_elems);
  for (int l = 0; l < L; ++l) {
    G.A.push_back(load_cores<T>(ar, Ad, l, (long long)bA[l] * doA[l] * diA[l] * bA[l + 1], st));
    G.B.push_back(load_cores<T>(ar, Bd, l, (long long)bB[l] * doB[l] * diB[l] * bB[l + 1], st));
    G.X.push_back(load_cores<T>(ar, Xd, l, (long long)bX[l] * doX[l] * diX[l] * bX[l + 1], st));
  }
  const T one = T(1);
  auto unit = [&](long long n) {
    T* p = ar.alloc<T>(n);
    GK(cudaMemcpyAsync(p, &one, sizeof(T), cudaMemcpyHostToDevice, st));
    return p;
  };
  // left pass: checkpoints of L^{(3)}_l (and L^{(4)}_l) at l = 0, k, 2k, ...; the values at the end
  const int k = G.k_ckpt;
  const int nck = (L + k - 1) / k;
  std::vector<T*> ck3(nck), ck4(nck);
  T* cur3 = ar.alloc<T>(e3);
  T* nxt3 = ar.alloc<T>(e3);
  T* cur4 = G.four ? ar.alloc<T>(e4) : nullptr;
  T* nxt4 = G.four ? ar.alloc<T>(e4) : nullptr;
  GK(cudaMemcpyAsync(cur3, &one, sizeof(T), cudaMemcpyHostToDevice, st));
  if (G.four) GK(cudaMemcpyAsync(cur4, &one, sizeof(T), cudaMemcpyHostToDevice, st));
  for (int l = 0; l < L; ++l) {
    if (l % k == 0) {
      const long long n3 = (long long)bA[l] * bB[l] * bX[l];
      ck3[l / k] = ar.alloc<T>(n3);
      GK(cudaMemcpyAsync(ck3[l / k], cur3, sizeof(T) * n3, cudaMemcpyDeviceToDevice, st));
      if (G.four) {
        const long long n4 = (long long)bA[l] * bB[l] * bA[l] * bB[l];
        ck4[l / k] = ar.alloc<T>(n4);
        GK(cudaMemcpyAsync(ck4[l / k], cur4, sizeof(T) * n4, cudaMemcpyDeviceToDevice, st));
      }
    }
    G.left3(l, cur3, nxt3);
    std::swap(cur3, nxt3);
    if (G.four) {
      G.left4(l, cur4, nxt4);
      std::swap(cur4, nxt4);
    }
  }
  const double xab = read_scalar(cur3, st);
  const double abab = G.four ? read_scalar(cur4, st) : 0.0;
  double xx = 0.0;
  if (G.four) {  // ||X||^2 by two-layer transfer
    T* m0 = unit(maxc2);
    T* m1 = ar.alloc<T>(maxc2);
    for (int l = 0; l < L; ++l) {
      G.left2(l, m0, m1);
      std::swap(m0, m1);
    }
    xx = read_scalar(m0, st);
  }
  // right-to-left: gradients with the running right environments and the recomputed left ones
  std::vector<T*> seg3(k), seg4(k);
  for (int i = 0; i < k; ++i) {
    seg3[i] = ar.alloc<T>(e3);
    if (G.four) seg4[i] = ar.alloc<T>(e4);
  }
  T* r3 = unit(e3);
  T* r3n = ar.alloc<T>(e3);
  T* r4 = G.four ? unit(e4) : nullptr;
  T* r4n = G.four ? ar.alloc<T>(e4) : nullptr;
  T* gA = ar.alloc<T>(core);
  T* gB = ar.alloc<T>(core);
  int loaded = -1;
  const T ia = G.four ? T(-2) : T(1);  // f1: -2 <X, AB> + ||AB||^2; f2: <X, AB>
  for (int l = L - 1; l >= 0; --l) {
    const int sg = l / k;
    if (sg != loaded) {  // recompute the left environments of this segment from its checkpoint
      const int l0 = sg * k;
      GK(cudaMemcpyAsync(seg3[0], ck3[sg], sizeof(T) * (size_t)bA[l0] * bB[l0] * bX[l0], cudaMemcpyDeviceToDevice, st));
      if (G.four)
        GK(cudaMemcpyAsync(seg4[0], ck4[sg], sizeof(T) * (size_t)bA[l0] * bB[l0] * bA[l0] * bB[l0],
                           cudaMemcpyDeviceToDevice, st));
      for (int j = l0; j < std::min(L, l0 + k) - 1; ++j) {
        G.left3(j, seg3[j - l0], seg3[j - l0 + 1]);
        if (G.four) G.left4(j, seg4[j - l0], seg4[j - l0 + 1]);
      }
      loaded = sg;
    }
    const long long nA = (long long)bA[l] * doA[l] * diA[l] * bA[l + 1];
    const long long nB = (long long)bB[l] * doB[l] * diB[l] * bB[l + 1];
    G.holes3(l, seg3[l - sg * k], r3, gA, gB, ia, T(0));
    if (G.four) G.holes4(l, seg4[l - sg * k], r4, gA, gB);
    store_cores<T>(gA, gAd, l, nA, st);
    store_cores<T>(gB, gBd, l, nB, st);
    if (l > 0) {
      G.right3(l, r3, r3n);
      std::swap(r3, r3n);
      if (G.four) {
        G.right4(l, r4, r4n);
        std::swap(r4, r4n);
      }
    }
  }
  GK(cudaStreamSynchronize(st));
  return G.four ? xx - 2.0 * xab + abab : xab;
}

}  // namespace

extern "C" tt_status tt_mpo_grad(const tt_mpo_desc* A, const tt_mpo_desc* B, const tt_mpo_desc* X, int target,
                                 int precision, int checkpoint_every, void* stream, const tt_mpo_desc* gA,
                                 const tt_mpo_desc* gB, double* value) {
  if (!A || !B || !X || !gA || !gB) return TT_ERR_INVALID_ARGUMENT;
  if (target != TT_GRAD_RESIDUAL && target != TT_GRAD_INNER) return TT_ERR_INVALID_ARGUMENT;
  if (precision != TT_PREC_FP64 && precision != TT_PREC_FP32 && precision != TT_PREC_TF32_SPLIT)
    return TT_ERR_INVALID_ARGUMENT;
  if (checkpoint_every < 0) return TT_ERR_INVALID_ARGUMENT;
  try {
    const double v = precision == TT_PREC_FP64
                         ? run_grad<double>(A, B, X, target, checkpoint_every, (cudaStream_t)stream, gA, gB)
                         : run_grad<float>(A, B, X, target, checkpoint_every, (cudaStream_t)stream, gA, gB,
                                           precision == TT_PREC_TF32_SPLIT);
    if (value) *value = v;
    return TT_OK;
  } catch (const GradError& e) {
    cudaGetLastError();
    return e.code;
  } catch (const std::bad_alloc&) {
    return TT_ERR_OUT_OF_MEMORY;
  } catch (...) {
    return TT_ERR_CUDA;
  }
}
