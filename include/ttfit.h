/*
 * ttfit.h -- C ABI of the GB300 variational MPO-MPO fit.
 *
 * The library approximates the product C ~ A B of two matrix product operators
 * by a bond-limited MPO C, minimising ||A B - C||_F^2 (Sec. 2.3, Eq. fit_min)
 * with the variational two-site fit (Alg. 5), whose local update is Alg. 3
 * (site-canonical gauge) or Alg. 4 (inverse-canonical gauge), optionally with
 * the randomized SVD of Sec. 3.1 in place of the exact SVD.
 *
 * Conventions shared by every entry point:
 *   - An MPO of length L has cores X_l of shape (chi_{l-1}, d_l, d'_l, chi_l),
 *     d the output leg and d' the input leg (Sec. 2, MPO definition), stored
 *     row-major in that index order; chi_0 = chi_L = 1.
 *   - C = A B contracts A's input leg with B's output leg (Sec. 2), so
 *     A.d_in[l] must equal B.d_out[l].
 *   - All core pointers are DEVICE pointers on the current CUDA device; all
 *     other pointers are host pointers.
 *   - No entry point throws; each returns a tt_status. A handle is bound to
 *     the stream in its options and is not thread-safe. Argument errors leave
 *     the handle usable; CUDA errors, device-side error words and numerical
 *     failures poison it (every later call returns TT_ERR_STATE).
 *   - There is no CPU fallback: every step of a sweep runs in this library's
 *     CUDA kernels on the device.
 */
#ifndef TTFIT_H
#define TTFIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TT_OK = 0,
  TT_ERR_INVALID_ARGUMENT = 1, /* NULL where a value is required, chi_max < 1, tol < 0, ... */
  TT_ERR_SHAPE_MISMATCH = 2,   /* L differ, A.d_in != B.d_out, bond[0] or bond[L] != 1      */
  TT_ERR_OUT_OF_MEMORY = 3,    /* a device allocation failed (nothing leaks)                */
  TT_ERR_CUDA = 4,             /* a CUDA runtime call or kernel launch failed               */
  TT_ERR_NUMERICAL = 5,        /* NaN/Inf in a local tensor, SVD did not converge           */
  TT_ERR_TIMEOUT = 6,          /* a bounded device-side wait gave up                        */
  TT_ERR_STATE = 7             /* handle poisoned by an earlier error, or wrong call order  */
} tt_status;

/* Gauge of C (Sec. 2.3.1). SITE: C_l cores with an orthogonality centre moved by
 * the sweep (Alg. 3). INVERSE: Psi_l cores and Y_l = Lambda_l^{-1} bond
 * vectors (Alg. 4); C_l = Psi_l Y_l (l < L), C_L = Psi_L. */
typedef enum { TT_GAUGE_SITE_CANONICAL = 0, TT_GAUGE_INVERSE_CANONICAL = 1 } tt_gauge;

/* Local update: exact truncated SVD of the two-site tensor (Sec. 2.3.4), or the
 * Gaussian-sketch randomized SVD (Sec. 3.1) with k = chi_max + oversample. */
typedef enum { TT_UPDATE_2SITE_SVD = 0, TT_UPDATE_2SITE_RSVD = 1 } tt_update;

/* Arithmetic of the contractions (environments, halves, two-site tensor).
 * FP64: FP64 CUDA-core kernels; FP64 factorisation (the 1e-10 parity path).
 * FP32: FP32 CUDA-core kernels. TF32: tensor-core kernels (tcgen05, TF32
 * operands, FP32 accumulation in tensor memory). TF32_SPLIT: the same with
 * each operand split into a TF32 high part and an FP32 remainder, three
 * products (hi*hi + hi*lo + lo*hi): about FP32 accuracy. DF32: every value
 * of the chain is a pair of floats hi + lo (about 48 significant bits);
 * small contractions run on the FP32 pipes (an exact FP32 product plus a
 * compensated sum per multiply-add), large ones on the tensor cores by a
 * fixed-point digit split: each 512-wide chunk of a row is cut into six 8-bit
 * digit planes, whose products accumulate exactly in FP32 at the leading
 * levels (FP64-class contractions at several times the FP64 rate of this
 * GPU); factorisation as for FP64. BF16_SPLIT: DF32 with the digit planes in
 * BF16 on kind::f16 MMAs (the digits are exact in BF16; twice the TF32 tensor
 * rate and half the bytes per plane); the same results as DF32 up to the
 * order of the FP32 sums in the non-exact digit levels. The zip-up entry
 * points reject it. The FP32, TF32 and TF32_SPLIT paths factorise in
 * FP32 and make the kept singular vectors an FP64 isometry (two
 * Newton-Schulz steps) before the gauge update; C is returned in FP64. */
typedef enum {
  TT_PREC_FP64 = 0,
  TT_PREC_FP32 = 1,
  TT_PREC_TF32 = 2,
  TT_PREC_BF16_SPLIT = 3,
  TT_PREC_TF32_SPLIT = 4,
  TT_PREC_DF32 = 5
} tt_precision;

/* Initial guess (Sec. 2.3.5). RANDOM: right-canonical MPO from a Philox4x32-10
 * Gaussian stream (core 1 Gaussian, core l>=2 the orthonormal-row factor of a
 * Gaussian matrix), bonds min(chi_max, prod d d' left, prod d d' right).
 * COPY_B: B itself. GIVEN: options.init_C. The guess is brought to
 * right-canonical form (orthogonality centre at site 1) before the sweeps.
 * ZIPUP: the zip-up contraction of the prepared A and B (tt_mpo_zipup, with
 * the fit's chi_max, tol, sv_cutoff, update, oversample and seed), which comes
 * out right-canonical; FP64 arithmetic for the FP64 and DF32 precisions, FP32
 * for the others (3xTF32 tensor-core contractions for the TF32 ones). */
typedef enum { TT_INIT_RANDOM = 0, TT_INIT_COPY_B = 1, TT_INIT_GIVEN = 2, TT_INIT_ZIPUP = 3 } tt_init;

typedef enum { TT_DTYPE_F64 = 0, TT_DTYPE_F32 = 1 } tt_dtype;

/* Describes an MPO held by the caller. Arrays d_out, d_in have L entries and
 * bond has L+1 (bond[0] = bond[L] = 1). cores[l] is a device pointer to
 * bond[l]*d_out[l]*d_in[l]*bond[l+1] values of type dtype, row-major
 * (chi_{l-1}, d, d', chi_l). The library never keeps these pointers. */
typedef struct {
  int L;
  const int* d_out;
  const int* d_in;
  const int* bond;
  void* const* cores;
  int dtype; /* tt_dtype */
} tt_mpo_desc;

/* Options; pass NULL for defaults. struct_size must be sizeof(tt_fit_options). */
typedef struct {
  size_t struct_size;
  int update;          /* tt_update, default TT_UPDATE_2SITE_SVD                          */
  int oversample;      /* sketch columns beyond chi_max (RSVD), default 10                 */
  uint64_t seed;       /* Philox key for the sketches and the random guess, default 0      */
  int precision;       /* tt_precision, default TT_PREC_FP64                              */
  int init;            /* tt_init, default TT_INIT_RANDOM                                 */
  const tt_mpo_desc* init_C; /* for TT_INIT_GIVEN                                          */
  double sv_cutoff;    /* drop s_j <= sv_cutoff * s_1; <0 = default: 1e-13 FP64, 1e-12 DF32 */
                       /* (FP64 factorisation), 1e-6 with an FP32 factorisation; follows  */
                       /* tt_fit_set_precision                                            */
  double conv_tol;     /* delta threshold; <0 = use tol                                    */
  void* stream;        /* cudaStream_t; NULL = legacy default stream                       */
  int prepare_inputs;  /* 1 (default): RQ + QR sweep of A and B (Alg. 5 left_orthogonalize) */
  uint32_t fault_inject; /* host-side fault injection for tests (TT_FAULT_*), default 0     */
  int fast_factor;     /* FP64 / DF32 only. 0 (default): FP64 SVD. 1-3: FP32 SVD, the kept     */
                       /* vectors made an FP64 isometry by Newton-Schulz steps. With DF32      */
                       /* contractions and the randomized update, 3 forms the sketch          */
                       /* Y = M Omega, its orthonormal basis Q and Q^T M in double-FP32 in     */
                       /* every sweep (kept subspace FP64-class, ~1e-10 of ||C||); 2 does the */
                       /* whole update in FP32 (~1e-6 of ||C||); 1 uses the FP32 update until */
                       /* a sweep changes ||C||^2 by <= 1e-3, then the double-FP32 basis, so  */
                       /* that the converged C is FP64-class.                                  */
  int n_segments;      /* segment-parallel fit (Sec. 4, Alg. 6): number of contiguous       */
                       /* segments N_p, each >= 2 sites; <= 1 (default) = serial Alg. 5.    */
                       /* Either gauge: the inverse one (scheme I) or the site one (scheme */
                       /* II, merged by tt_fit_merge); see tt_fit_sweep for what a sweep is. */
  int edge_extra;      /* sites moved from the inner segments to each edge segment (load   */
                       /* balance of Sec. 4.1: edge segments have one neighbour), default 0 */
  int ab_rank;         /* randomized bond projection of the A and B chains (Sec. 3.2): k > 0 */
                       /* puts a rank-k projector Q Q^T on every bond of A and of B, Q the    */
                       /* orthonormal range of a k-column Philox Gaussian sketch of the bond  */
                       /* (streams (4 << 40) | l for A, (5 << 40) | l for B, site l 1-based), */
                       /* drawn once at creation on the prepared chains (right to left; the  */
                       /* QR sweep again only before a zip-up guess); the fit then contracts */
                       /* bonds of at most k, in the environments and the update alike. The  */
                       /* fit approximates the product of the projected chains, so this needs */
                       /* A and B with decaying bond spectra. Needs prepare_inputs. 0 = off.  */
} tt_fit_options;

/* Host-side fault injection (tests only; nothing here touches the device). */
#define TT_FAULT_ALLOC_FAIL 0x1u  /* the create-time allocation reports out-of-memory       */
#define TT_FAULT_NAN_INPUT 0x2u   /* treat the first local tensor as containing a NaN       */
#define TT_FAULT_SVD_NOCONV 0x4u  /* report the first factorisation as not converged        */

/* Per-call summary of tt_fit_sweep. */
typedef struct {
  int sweeps_done;      /* directional sweeps completed since create                       */
  int converged;        /* 1 once delta <= conv_tol                                        */
  double delta;         /* |n2_s - n2_{s-1}| / n2_s of the last sweep (inf after the first) */
  double norm2_C;       /* ||C||^2 = sum of kept s^2 at the last window of the last sweep  */
  double max_discarded; /* max over the last sweep's windows of sqrt(sum_{j>k} s_j^2)/||M|| */
  double seconds;       /* wall time of this call (device work included)                   */
} tt_sweep_report;

typedef struct tt_fit tt_fit;

/* Create a fit of C ~ A B with at most chi_max bond dimension and truncation
 * tolerance tol (tau of Sec. 2.3.4: a window discards singular values while
 * sqrt(sum of discarded s^2) <= (tol / L) ||M||_F; tol = 0 caps by chi_max only).
 * A and B are copied (stream-ordered) and prepared: input canonicalisation
 * (Alg. 5), initial guess, right environments R_L..R_3 and their halves.
 * On success *out owns every device buffer; free it with tt_fit_destroy.
 * Errors: TT_ERR_INVALID_ARGUMENT, TT_ERR_SHAPE_MISMATCH, TT_ERR_OUT_OF_MEMORY,
 * TT_ERR_CUDA (then *out is NULL). */
tt_status tt_fit_create(const tt_mpo_desc* A, const tt_mpo_desc* B, int chi_max, double tol,
                        int gauge, const tt_fit_options* opt, tt_fit** out);

/* Run up to n_sweeps directional sweeps of Alg. 5 (forward l = 1..L-1, then
 * backward l = L-1..1, alternating; the direction continues across calls).
 * Stops early once converged. rep may be NULL. Synchronises the handle's
 * stream before returning.
 *
 * Segment-parallel handle (n_segments > 1, Sec. 4, Alg. 6): a sweep is one
 * phase, i.e. half of a full set of local sweeps. Phase 0: odd segments
 * (numbered from 1) sweep forward and even ones backward, all concurrently;
 * then the windows straddling the odd|even boundaries are updated by their
 * left segment. Phase 1: the directions swap and the even|odd boundaries
 * follow. Each segment runs on its own stream and host thread, with its own
 * scratch; the handle's stream waits for all of them. ||C||^2 of a set is
 * that of its last update (every Psi is an orthogonality centre in the
 * inverse gauge), and delta compares consecutive full sets, so convergence
 * is tested after every second phase. The sketch of a window in phase p of
 * set s uses sweep index 2 s + p.
 * Site gauge (scheme II): the same phases with the site-gauge update (Alg.
 * 3); segments are prepared (Sec. 4.2) with odd segments' orthogonality
 * centres on their first site and even segments' on their last. Every segment
 * then carries its own centre, so C is not exported until tt_fit_merge has
 * joined the segments. */
tt_status tt_fit_sweep(tt_fit* h, int n_sweeps, tt_sweep_report* rep);

/* Binary merge of a site-gauge segment-parallel fit (Sec. 4.5). After the last
 * phase the chain is a row of consistent units: the segments joined by that
 * phase's boundary updates, and the segments without one. Neighbouring units
 * are joined pairwise in rounds (O(log N_p) of them): the left unit's
 * orthogonality centre moves to its last site l by QR steps and the right
 * unit's to its first site l+1 by RQ steps, each step finishing the
 * environment it passes (O(L) in all), then window (l, l+1) is updated forward
 * with the sketches of phase index P + r - 1 in round r (P = phases run).
 * The joins of a round run concurrently on their segments' streams. Afterwards
 * C is one site-canonical MPO with its centre at the last window's right
 * site, and tt_fit_result may export it; further sweeps continue the local
 * phases from it. A no-op for any other handle or when already merged.
 * rep (nullable): norm2_C = ||C||^2 after the merge, other fields as after
 * the last sweep. Errors: TT_ERR_STATE (poisoned handle), and as tt_fit_sweep. */
tt_status tt_fit_merge(tt_fit* h, tt_sweep_report* rep);

/* Change the contraction precision for the following sweeps (the paper's
 * "cheap sweeps first, exact sweeps last", Sec. 5.3): the chain buffers are
 * rebuilt in the new arithmetic, and the environments the next sweep reads are
 * recomputed from the current C: R_L..R_3 before a forward sweep, L_1..L_{L-2}
 * before a backward one. A segment-parallel fit switches only between full sets
 * of local sweeps (else TT_ERR_STATE; the handle stays usable), in the site
 * gauge only once merged, after which the segments are prepared again. fast_factor as
 * in tt_fit_options; a default cut-off follows the new precision. Resets the
 * converged flag; delta keeps comparing consecutive sweeps. */
tt_status tt_fit_set_precision(tt_fit* h, int precision, int fast_factor);

/* Export C as a plain MPO. Two-step: with C->cores == NULL, fill
 * C->L, and the caller-provided arrays C->d_out, C->d_in (L ints) and C->bond
 * (L+1 ints); then call again with cores pointing to caller device buffers of
 * the reported sizes in C->dtype. lambdas (nullable, host) receives, for each
 * inner bond l = 1..L-1 in order, the bond[l] singular values of the last
 * update of that bond. In the inverse gauge C_l = Psi_l Y_l (l < L).
 * TT_ERR_STATE for a site-gauge segment-parallel fit that is not merged. */
tt_status tt_fit_result(const tt_fit* h, tt_mpo_desc* C, double* lambdas);

/* Free every buffer of the handle (NULL is a no-op). */
void tt_fit_destroy(tt_fit* h);

const char* tt_status_string(tt_status s);

/* Last error message of the handle ("" when none); valid until the next call.
 * With h == NULL: the message of the calling thread's last failed
 * tt_fit_create ("NULL handle" when there is none). */
const char* tt_fit_last_error(const tt_fit* h);

/* Per-stage device time of the last tt_fit_sweep call, in milliseconds, and
 * the algorithmic FP64/FP32 flops of the contraction stages it ran:
 * out[0] halves, out[1] two-site tensor, out[2] environment finish,
 * out[3] factorisation, out[4] gauge update, out[5] contraction flops
 * (minimal count), out[6] kernel launches issued. Returns TT_ERR_STATE if no
 * sweep ran. */
tt_status tt_fit_stage_times(const tt_fit* h, double out[7]);

/* The same contractions of the last tt_fit_sweep call as the hardware issued
 * them: out[0] tensor-core MMA flops, with the tiles padded to 128 x 128 and K
 * to the k-block, and every pass counted (3 for TF32_SPLIT, 21 digit pairs for
 * the DF32 and BF16_SPLIT digit split); out[1] flops of the contractions that
 * ran on the CUDA cores (2 M N K each, in the chain's own type). Against
 * out[5] of tt_fit_stage_times this separates the work the method needs from
 * the work its precision scheme adds (Sec. 2.3, Table 1 counts the former).
 * Returns TT_ERR_STATE if no sweep ran. */
tt_status tt_fit_exec_flops(const tt_fit* h, double out[2]);

/* Kernel launches issued by this handle since tt_fit_create, cumulative over
 * creation (input preparation, initial guess, right environments), sweeps,
 * precision switches and result export. Lets a caller check that the work it
 * timed ran in this library's kernels. */
tt_status tt_fit_launch_count(const tt_fit* h, long long* n);

/* Device memory of the handles comes from a process-wide cache of blocks:
 * tt_fit_destroy (and the release of buffers that a handle no longer needs)
 * returns blocks to it instead of freeing them, and later handles reuse them
 * without allocating (best fit: the smallest cached block of at least the size
 * asked for and at most twice it). At most a quarter of a device's memory (and
 * at most 64 GiB) stays cached; when an allocation fails the cache of that
 * device is emptied and the allocation retried. Cached memory stays with the
 * process until this call returns it. This call frees every cached block of `device`
 * (all devices if device < 0) and returns the number of bytes it held. Safe to
 * call at any time: cached blocks are not in use. Host-only otherwise (no
 * stream work). */
size_t tt_device_cache_release(int device);

/* The largest number of Jacobi sweeps that one singular value decomposition of
 * a two-site tensor (or of its randomized sketch) needed since tt_fit_create,
 * as of the last window that completed. A diagnostic of the factorisation
 * stage; the sweeps stop when no column pair is rotated. */
tt_status tt_fit_jacobi_sweeps(const tt_fit* h, int* max_sweeps);

/* The segments a fit with these options uses (Sec. 4.1): n_segments
 * contiguous ranges of >= 2 sites, first[i]..last[i] (0-based, inclusive,
 * arrays of n_segments). Sites are shared out evenly, the first L mod
 * n_segments segments taking one more; then up to edge_extra sites move to
 * each of the two edge segments, taken one at a time from the inner segments
 * in turn while each keeps >= 2 sites. Host-only; needs no GPU.
 * TT_ERR_INVALID_ARGUMENT if L < 2 n_segments or an argument is out of range. */
tt_status tt_partition(int L, int n_segments, int edge_extra, int* first, int* last);

/* Batched fits of independent pairs (A[i], B[i]) with their own chi_max[i]
 * (uneven sizes allowed), all with the same tol, gauge, n_segments and
 * options (opt->n_segments is overridden by n_segments; TT_INIT_GIVEN is
 * rejected). Each handle gets a stream of its own, ordered after opt->stream,
 * and is created on its own host thread; out[0..n-1] receive the handles,
 * each destroyed with tt_fit_destroy. On any error every handle created so far
 * is destroyed, out[] is set to NULL and the first failing status (by index)
 * is returned. */
tt_status tt_fit_create_batched(int n, const tt_mpo_desc* A, const tt_mpo_desc* B, const int* chi_max, double tol,
                                int gauge, int n_segments, const tt_fit_options* opt, tt_fit** out);

/* tt_fit_sweep on n handles concurrently (one host thread each, their own
 * streams). rep, if not NULL, has n entries. Returns the first non-OK status
 * by index; handles that failed are poisoned as by tt_fit_sweep, the others
 * completed their sweeps. */
tt_status tt_fit_sweep_batched(int n, tt_fit* const* h, int n_sweeps, tt_sweep_report* rep);

/* Objectives of the adjoint (tt_mpo_grad). */
typedef enum {
  TT_GRAD_RESIDUAL = 0, /* f1(A, B) = ||X - A B||_F^2, X (= C) held fixed   */
  TT_GRAD_INNER = 1     /* f2(A, B) = <X, A B> = tr(X^T A B), X (= W) fixed */
} tt_grad_target;

/* Adjoint of the fit's contraction chain (not in the paper, which does not
 * differentiate with respect to A or B): the value of the target and its
 * gradient with respect to every core of A and B, at fixed X (no
 * differentiation through the fit's factorisations).
 * <X, AB> is the three-layer network of the fit's environments (Sec. 2.3.3);
 * its gradient with respect to a core is the network with that core cut out.
 * ||AB||^2 uses four-layer environments (two copies of A, B); its gradient is
 * twice the punched hole of one copy, so d f1 = 2 (G^{ABAB} - G^{XAB}).
 * A, B, X: device MPOs (FP64 or FP32 cores, layouts as tt_mpo_desc),
 * A.d_in == B.d_out, X.d_out == A.d_out, X.d_in == B.d_in, equal L.
 * gA, gB: caller device buffers with the shapes (d_out, d_in, bond) of A and
 * B, FP64 or FP32; receive dtarget/dA_l and dtarget/dB_l. *value (host, may be
 * NULL) receives the target. precision: TT_PREC_FP64 or TT_PREC_FP32 (the
 * contractions and environments in that type), or TT_PREC_TF32_SPLIT (FP32
 * environments; the contractions whose operands TMA can load run as 3xTF32 on
 * the tensor cores, about FP32 accuracy, the others on the FP32 CUDA cores). checkpoint_every: left
 * environments are stored every k sites and recomputed in between during the
 * right-to-left gradient pass (1 = store all; 0 = about sqrt(L)), which bounds
 * memory at (L/k + k) environments; the four-layer ones hold (chi_A chi_B)^2
 * values. Runs on `stream` (cudaStream_t) and synchronises it. Errors:
 * TT_ERR_INVALID_ARGUMENT, TT_ERR_SHAPE_MISMATCH, TT_ERR_OUT_OF_MEMORY,
 * TT_ERR_CUDA. */
tt_status tt_mpo_grad(const tt_mpo_desc* A, const tt_mpo_desc* B, const tt_mpo_desc* X, int target, int precision,
                      int checkpoint_every, void* stream, const tt_mpo_desc* gA, const tt_mpo_desc* gB,
                      double* value);

/* Truncated SVD of one device matrix, the factorisation of the local update
 * (Sec. 2.3.4): M is m x n, row-major, FP64 (device). Computes the thin SVD
 * M = U diag(S) Vt in FP64 (one-sided Jacobi; singular values descending;
 * each pair signed so that the largest-magnitude entry of u_j is positive)
 * into caller device buffers U (m x r row-major), S (r), Vt (r x n
 * row-major), r = min(m, n) <= 1024, and returns in *k_out (host) the rank
 * the truncation rule keeps: k = min(chi_max, min{k : sqrt(sum_{j>k} s_j^2)
 * <= tau_rel ||M||_F}), values <= 1e-13 s_1 dropped, k >= 1. Allocates its
 * scratch with cudaMalloc, runs on `stream` (cudaStream_t, NULL = default)
 * and synchronises it. Errors: TT_ERR_INVALID_ARGUMENT (NULL pointer,
 * non-positive size, r > 1024), TT_ERR_OUT_OF_MEMORY, TT_ERR_CUDA,
 * TT_ERR_NUMERICAL (non-finite input, no convergence). */
tt_status tt_svd_truncated(const double* M, int m, int n, int chi_max, double tau_rel, double* U, double* S,
                           double* Vt, int* k_out, void* stream);

/* Same computation and arguments as tt_svd_truncated, for callers that must
 * not allocate device memory: for example code running while a caching
 * allocator owns the device's memory budget, or latency-critical loops where
 * a cudaMalloc / cudaFree would synchronise the device. This entry point calls
 * no cudaMalloc, cudaFree or other allocating routine. (The paper has no
 * counterpart; it is an interface convenience.)
 * Its scratch is a fixed 4 MiB device array inside the library (2^19
 * doubles), held on every GPU that loads the library until the process exits.
 * An m x n input needs 2 q r + 2 r^2 + r + 6 doubles of it (r = min(m, n),
 * q = max(m, n); e.g. up to 512 x 256); larger inputs return
 * TT_ERR_INVALID_ARGUMENT. The first call on a device looks up the array's
 * address on that device (cudaGetSymbolAddress); with lazy module loading (the
 * CUDA default) that is also when the array is committed. So make that first
 * call before any stream capture, and before a caching allocator claims the
 * device's memory (else it can fail with TT_ERR_CUDA). The address is cached per
 * device: after cudaDeviceReset on a device it is stale, and this entry point
 * must not be called on that device again in the same process. All calls on a device share the one array and
 * it keeps the last call's contents: calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Synchronises `stream` before returning. */
tt_status tt_svd_truncated_noalloc(const double* M, int m, int n, int chi_max, double tau_rel, double* U, double* S,
                                   double* Vt, int* k_out, void* stream);

/* Exact per-site product of two MPOs, the contraction step of the naive
 * algorithm (Sec. 2.1, Alg. 1, without its final compression):
 * C_l[(i_a i_b), s, t, (j_a j_b)] = sum_u A_l[i_a, s, u, j_a] B_l[i_b, u, t, j_b],
 * the combined bond index i_a * chi_B + i_b, so that C has bonds chi_A chi_B.
 * A, B: device MPOs of equal L with A.d_in == B.d_out, both FP64 or both FP32.
 * C: caller descriptor whose cores are device buffers of the same dtype with
 * bond[l] = A.bond[l] * B.bond[l], d_out = A.d_out, d_in = B.d_in; every
 * core is overwritten. One kernel launch per site on `stream` (cudaStream_t,
 * NULL = legacy default stream); returns without synchronising. Errors:
 * TT_ERR_INVALID_ARGUMENT (missing fields, mixed dtypes), TT_ERR_SHAPE_MISMATCH,
 * TT_ERR_CUDA. */
tt_status tt_mpo_naive_product(const tt_mpo_desc* A, const tt_mpo_desc* B, const tt_mpo_desc* C, void* stream);

/* Zip-up contraction C ~ A B (Sec. 2.2, Alg. 2) in one pass, right to left:
 * A and B are prepared as for the fit (RQ sweep, then the QR sweep: left-
 * canonical, the mirror of the right-canonical inputs the paper's
 * left-to-right pass takes); from site L down to 2 the remainder R_{l+1} is
 * contracted with A_l and B_l into the (chi_A chi_B) x (d d' chi) matrix M_l,
 * whose truncated factorisation (the fit's rule, Sec. 2.3.4, with tol as tau
 * and chi_max) keeps the right singular vectors as C_l and R_l = M_l V; site 1
 * takes the last remainder. The result is right-canonical (orthogonality
 * centre at site 1). opt (NULL = defaults) supplies update (randomized SVD of
 * Sec. 3.1 with k_s = chi_max + oversample columns and the Philox stream
 * (3 << 40) | l of seed, where k_s < min of M's sizes), oversample, seed,
 * precision (FP64 and DF32: FP64 arithmetic; FP32, TF32, TF32_SPLIT: FP32, with
 * 3xTF32 tensor-core contractions for the TF32 ones; BF16_SPLIT is rejected
 * with TT_ERR_INVALID_ARGUMENT), sv_cutoff, stream and
 * prepare_inputs; the other fields are ignored. M_l with more than 1024 rows is
 * factorised through its (sketch's) Gram matrix, which resolves singular
 * values only down to about sqrt(eps) s_1. Needs d d' chi_max <= 1024 and
 * input cores with d d' chi <= 1024 (the QR of the preparation).
 * C: caller descriptor (L, d_out = A.d_out, d_in = B.d_in, dtype FP64 or
 * FP32) whose cores are device buffers with room for bond[l] * d * d' *
 * bond[l+1] values; bond[l] >= min(chi_max, A.bond[l] B.bond[l],
 * prod_{j>=l} d_j d'_j) always suffices. Core l is written packed in the kept
 * bonds, (bond_out[l], d, d', bond_out[l+1]) row-major, and bond_out (host,
 * L+1 ints) receives the kept bonds. Synchronises the stream. Errors:
 * TT_ERR_INVALID_ARGUMENT, TT_ERR_SHAPE_MISMATCH (also when a kept bond
 * exceeds C.bond), TT_ERR_OUT_OF_MEMORY, TT_ERR_NUMERICAL, TT_ERR_CUDA. */
tt_status tt_mpo_zipup(const tt_mpo_desc* A, const tt_mpo_desc* B, int chi_max, double tol,
                       const tt_fit_options* opt, const tt_mpo_desc* C, int* bond_out);

/* compress(X, tol, chi_max) of Alg. 1 (Sec. 2.1): X is left-orthogonalised and
 * swept right to left; at each site the core absorbs the remainder and its
 * truncated factorisation keeps the right singular vectors. This is the
 * zip-up of X with the identity MPO (d_out = d_in = X.d_in, bond 1), so
 * options, output and errors are those of tt_mpo_zipup (C.d_in = X.d_in). */
tt_status tt_mpo_compress(const tt_mpo_desc* X, int chi_max, double tol, const tt_fit_options* opt,
                          const tt_mpo_desc* C, int* bond_out);

#ifdef __cplusplus
}
#endif
#endif /* TTFIT_H */
