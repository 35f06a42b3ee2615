"""Parity of the CUDA fit (through the C ABI) with the FP64 oracle on the same
seeded inputs. Results are compared as operators (the stable difference norm of
the oracle) plus per-bond dimensions and the convergence history; raw cores are
gauge-dependent (singular-vector signs) and are not compared."""
import math

import numpy as np
import pytest

from oracle.fit import FitOracle
from oracle.mpo import bonds, mpo_diff_norm, mpo_norm, to_dense
from paper_2606_23274_gb300.synth import gaussian_mpo, kron_sum_mpo, mpo_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_23274_gb300 import ttfit  # noqa: E402


def _gpu_fit(A, B, chi, tol, sweeps, **kw):
    f = ttfit.tt_fit_create(A, B, chi, tol, kw.pop("gauge", "site"), **kw)
    reps = [f.sweep(1) for _ in range(sweeps)]
    C = [c.cpu().numpy() for c in f.result()]
    lam = f.lambdas()
    b = f.bonds()
    f.destroy()
    return C, reps, b, lam


def _rel(X, Y):
    return mpo_diff_norm(X, Y) / mpo_norm(Y)


@pytest.mark.parametrize("gauge", ["site", "inverse"])
def test_exact_product_fp64(gauge):
    """chi_C = chi_A chi_B = 64 reproduces A B (dense 256 x 256 check)."""
    A, B = mpo_pair("gauss_L8_chi8", 0)
    C, reps, b, _ = _gpu_fit(A, B, 64, 0.0, 2, gauge=gauge, precision="fp64")
    D = to_dense(A) @ to_dense(B)
    assert np.linalg.norm(to_dense(C) - D) <= 1e-10 * np.linalg.norm(D)
    assert b == [1, 4, 16, 64, 64, 64, 16, 4, 1]


@pytest.mark.parametrize("gauge", ["site", "inverse"])
@pytest.mark.parametrize("update", ["svd", "rsvd"])
def test_truncated_fit_fp64_matches_oracle(gauge, update):
    A, B = mpo_pair("kron_L12_chi32", 1)
    chi, sweeps = 12, 4
    f = FitOracle(A, B, chi, 0.0, gauge=gauge, update=update, oversample=4, seed=3)
    f.sweep(sweeps, stop_on_converge=False)
    Co = f.result()
    C, reps, b, lam = _gpu_fit(A, B, chi, 0.0, sweeps, gauge=gauge, update=update, oversample=4, seed=3,
                               precision="fp64", conv_tol=0.0)
    assert b == f.bonds()
    assert _rel(C, Co) <= 1e-9
    for r, h in zip(reps, f.st.history):
        assert abs(r["norm2_C"] - h.norm2) <= 1e-11 * h.norm2
    # spectra where the cut is not degenerate (the oracle's gap report); the operator above is
    # compared everywhere
    pinned = f.pinned_bonds()
    print(gauge, update, "bonds with a degenerate cut (spectrum unpinned):",
          [l for l in range(1, len(lam) + 1) if l not in pinned])
    for l, (got, ref) in enumerate(zip(lam, f.lambdas()), 1):
        if l in pinned:
            assert np.allclose(got, ref, rtol=1e-9, atol=1e-12 * ref[0])


def test_fp32_contractions_match_oracle():
    A, B = mpo_pair("kron_L10_chi16", 2)
    f = FitOracle(A, B, 10, 0.0, seed=1, sv_cutoff=1e-6)
    f.sweep(4, stop_on_converge=False)
    C, reps, b, _ = _gpu_fit(A, B, 10, 0.0, 4, precision="fp32", seed=1, conv_tol=0.0)
    assert b == f.bonds()
    assert _rel(C, f.result()) <= 2e-5


def test_init_given_and_copy_b():
    A, B = mpo_pair("kron_L10_chi16", 4)
    C0 = gaussian_mpo(10, 2, 5, seed=77, which=3)
    for init, kw in (("given", dict(init_C=C0)), ("copy_b", {})):
        f = FitOracle(A, B, 8, 0.0, init=init, **kw)
        f.sweep(3, stop_on_converge=False)
        C, reps, b, _ = _gpu_fit(A, B, 8, 0.0, 3, init=init, precision="fp64", conv_tol=0.0, **kw)
        assert b == f.bonds()
        assert _rel(C, f.result()) <= 1e-9


def test_edge_cases_small_chains_and_ragged_dims():
    """L = 2 (a single window), chi_max = 1, local dims 3 x 2 and ragged bonds."""
    rng = np.random.default_rng(5)
    # L = 2
    A, B = mpo_pair("gauss_L8_chi8", 1, L=2)
    C, _, b, _ = _gpu_fit(A, B, 64, 0.0, 1, precision="fp64")
    D = to_dense(A) @ to_dense(B)
    assert np.linalg.norm(to_dense(C) - D) <= 1e-12 * np.linalg.norm(D)
    # chi_max = 1
    A, B = mpo_pair("kron_L10_chi16", 0)
    f = FitOracle(A, B, 1, 0.0)
    f.sweep(2, stop_on_converge=False)
    C, _, b, _ = _gpu_fit(A, B, 1, 0.0, 2, precision="fp64", conv_tol=0.0)
    assert b == [1] * 11
    assert _rel(C, f.result()) <= 1e-9
    # non-uniform local dims: A (chi, 3, 2, chi), B (chi, 2, 3, chi) -> C has 3 x 3 legs
    L = 5
    bA = [1, 3, 5, 4, 2, 1]
    bB = [1, 2, 4, 5, 3, 1]
    A = [rng.standard_normal((bA[l], 3, 2, bA[l + 1])) for l in range(L)]
    B = [rng.standard_normal((bB[l], 2, 3, bB[l + 1])) for l in range(L)]
    f = FitOracle(A, B, 6, 0.0)
    f.sweep(3, stop_on_converge=False)
    C, _, b, _ = _gpu_fit(A, B, 6, 0.0, 3, precision="fp64", conv_tol=0.0)
    assert b == f.bonds()
    assert _rel(C, f.result()) <= 1e-9


def test_tolerance_truncation_rule():
    """tau > 0 discards by the tau/L rule (Sec. 2.3.4) identically on both sides."""
    A, B = mpo_pair("kron_L12_chi32", 2)
    tau = 0.3
    f = FitOracle(A, B, 40, tau)
    f.sweep(3, stop_on_converge=False)
    C, _, b, _ = _gpu_fit(A, B, 40, tau, 3, precision="fp64", conv_tol=0.0)
    assert b == f.bonds()
    assert max(b) < 40
    assert _rel(C, f.result()) <= 1e-8


def test_convergence_stops_sweeps():
    A, B = mpo_pair("gauss_L8_chi8", 2)
    f = ttfit.tt_fit_create(A, B, 64, 1e-10, "site", precision="fp64")
    r = f.sweep(10)
    assert r["converged"] == 1 and r["sweeps_done"] < 10
    assert r["delta"] <= 1e-10
    f.destroy()


def test_error_paths_are_reported_and_poison():
    A, B = mpo_pair("gauss_L8_chi8", 0)
    # shape mismatch: A's input legs != B's output legs
    Bbad = [np.zeros((b.shape[0], 3, b.shape[2], b.shape[3])) for b in B]
    with pytest.raises(ttfit.TTError) as e:
        ttfit.tt_fit_create(A, Bbad, 8, 0.0)
    assert e.value.code == ttfit.TT_ERR_SHAPE_MISMATCH
    with pytest.raises(ttfit.TTError) as e:
        ttfit.tt_fit_create(A, B[:-1], 8, 0.0)
    assert e.value.code == ttfit.TT_ERR_SHAPE_MISMATCH
    with pytest.raises(ttfit.TTError) as e:
        ttfit.tt_fit_create(A, B, 0, 0.0)
    assert e.value.code == ttfit.TT_ERR_INVALID_ARGUMENT
    with pytest.raises(ttfit.TTError) as e:
        ttfit.tt_fit_create(A, B, 8, 0.0, fault_inject=ttfit.TT_FAULT_ALLOC_FAIL)
    assert e.value.code == ttfit.TT_ERR_OUT_OF_MEMORY
    for fault in (ttfit.TT_FAULT_NAN_INPUT, ttfit.TT_FAULT_SVD_NOCONV):
        f = ttfit.tt_fit_create(A, B, 8, 0.0, fault_inject=fault)
        with pytest.raises(ttfit.TTError) as e:
            f.sweep(1)
        assert e.value.code == ttfit.TT_ERR_NUMERICAL
        with pytest.raises(ttfit.TTError) as e:
            f.sweep(1)
        assert e.value.code == ttfit.TT_ERR_STATE
        f.destroy()
    # a healthy handle after the poisoned ones
    f = ttfit.tt_fit_create(A, B, 8, 0.0)
    f.sweep(1)
    f.destroy()


def test_float32_inputs_and_outputs():
    A, B = mpo_pair("gauss_L8_chi8", 3)
    A32 = [torch.from_numpy(a).float().cuda() for a in A]
    B32 = [torch.from_numpy(b).float().cuda() for b in B]
    f = ttfit.tt_fit_create(A32, B32, 64, 0.0, "site", precision="fp64")
    f.sweep(2)
    C = [c.cpu().double().numpy() for c in f.result(torch.float32)]
    f.destroy()
    D = to_dense([a.astype(np.float32).astype(np.float64) for a in A]) @ \
        to_dense([b.astype(np.float32).astype(np.float64) for b in B])
    assert np.linalg.norm(to_dense(C) - D) <= 1e-6 * np.linalg.norm(D)


@pytest.mark.parametrize("gauge", ["site", "inverse"])
def test_tf32_tensor_core_chain_exact_product(gauge):
    """TF32 tensor-core contractions (10-bit mantissa, FP32 accumulation) on the
    exact-product case: the unique optimum is A B itself, reproduced to the TF32
    rounding level (the join and halves run on tcgen05 here)."""
    A, B = mpo_pair("gauss_L8_chi8", 1)
    C, reps, b, _ = _gpu_fit(A, B, 64, 0.0, 2, gauge=gauge, precision="tf32", conv_tol=0.0)
    D = to_dense(A) @ to_dense(B)
    err = np.linalg.norm(to_dense(C) - D) / np.linalg.norm(D)
    print("tf32 exact-product rel err", err)
    assert err <= 1e-2
    assert b == [1, 4, 16, 64, 64, 64, 16, 4, 1]


def test_mixed_precision_fit_quality():
    """FP32, 3xTF32 and one-pass TF32 fits of a truncated product reach an optimum
    about as good as the FP64 oracle's (the fit has several local optima; the
    residual ||AB - C||^2 is compared, not the operator). One-pass TF32 (10-bit
    mantissa) stays within 15%; the split and FP32 paths within 0.1%."""
    A, B = mpo_pair("kron_L12_chi32", 5)
    from oracle.mpo import naive_product
    N = naive_product(A, B)
    nAB2 = mpo_norm(N) ** 2
    f = FitOracle(A, B, 16, 0.0)
    f.sweep(6, stop_on_converge=False)
    res_o = mpo_diff_norm(N, f.result()) ** 2
    for prec, slack in (("fp32", 1e-3), ("tf32x3", 1e-3), ("tf32", 1.5e-1)):
        C, reps, b, _ = _gpu_fit(A, B, 16, 0.0, 6, precision=prec, conv_tol=0.0)
        res = mpo_diff_norm(N, C) ** 2
        print(prec, "residual", res, "oracle", res_o)
        assert res <= res_o * (1 + slack) + 1e-12 * nAB2


@pytest.mark.parametrize("gauge", ["site", "inverse"])
def test_tf32x3_split_chain_matches_oracle(gauge):
    """3xTF32 tensor-core contractions (hi*hi + hi*lo + lo*hi) on the exact-product
    case: agreement with the dense product at the FP32 level."""
    A, B = mpo_pair("gauss_L8_chi8", 1)
    C, reps, b, _ = _gpu_fit(A, B, 64, 0.0, 2, gauge=gauge, precision="tf32x3", conv_tol=0.0)
    D = to_dense(A) @ to_dense(B)
    err = np.linalg.norm(to_dense(C) - D) / np.linalg.norm(D)
    print("tf32x3 exact-product rel err", err)
    assert err <= 2e-5


def _fast_pair(seed=2):
    """Kronecker-sum inputs with weights 0.5^k: the fit converges to 1e-12 in ~10 sweeps."""
    return kron_sum_mpo(10, 16, seed, 0, decay=0.5), kron_sum_mpo(10, 16, seed, 1, decay=0.5)


@pytest.mark.parametrize("n_lo", [1, 2])
def test_precision_switch_mid_fit(n_lo):
    """Cheap sweeps first, exact sweeps last (Sec. 5.3): FP32 sweeps, then the FP64
    chain with the FP64 SVD; the result matches the all-FP64 oracle fit. After
    one sweep the next one is backward (C left-canonical: the switch rebuilds the
    left environments), after two it is forward (the right ones)."""
    A, B = _fast_pair()
    f = FitOracle(A, B, 12, 0.0, seed=1)
    f.sweep(12, stop_on_converge=False)
    h = ttfit.tt_fit_create(A, B, 12, 0.0, "site", precision="fp32", seed=1, conv_tol=0.0)
    h.sweep(n_lo)
    h.set_precision("fp64")
    for _ in range(12 - n_lo):
        r = h.sweep(1)
    C = [c.cpu().numpy() for c in h.result()]
    h.destroy()
    assert f.st.history[-1].delta <= 1e-10                  # both runs have converged
    assert r["delta"] <= 1e-10
    assert _rel(C, f.result()) <= 1e-7


def test_fast_factor_fp64_converges():
    """FP64 contractions with the FP32 factorisation made an FP64 isometry: ||C||^2
    converges to the FP64 level and the residual matches the oracle's optimum."""
    A, B = _fast_pair(3)
    from oracle.mpo import naive_product
    N = naive_product(A, B)
    f = FitOracle(A, B, 12, 0.0)
    f.sweep(12, stop_on_converge=False)
    res_o = mpo_diff_norm(N, f.result()) ** 2
    h = ttfit.tt_fit_create(A, B, 12, 0.0, "site", precision="fp64", fast_factor=True, conv_tol=0.0)
    reps = [h.sweep(1) for _ in range(12)]
    C = [c.cpu().numpy() for c in h.result()]
    h.destroy()
    assert reps[-1]["delta"] <= 1e-10
    res = mpo_diff_norm(N, C) ** 2
    assert res <= res_o * (1 + 1e-6)


@pytest.mark.parametrize("precision", ["df32", "bf16_split"])
@pytest.mark.parametrize("gauge", ["site", "inverse"])
@pytest.mark.parametrize("update", ["svd", "rsvd"])
def test_df32_fit_matches_fp64_oracle(gauge, update, precision):
    """Double-FP32 contractions (FP64-class: the digit split on the TF32 or, for
    bf16_split, the BF16 tensor cores, the small ones on the FP32 pipes) with the
    FP64 factorisation: the same results as the FP64 oracle to 1e-9. The chain's
    K = 1024 contractions take the digit split with two chunks."""
    A, B = mpo_pair("kron_L12_chi32", 1)
    chi, sweeps = 12, 4
    f = FitOracle(A, B, chi, 0.0, gauge=gauge, update=update, oversample=4, seed=3, sv_cutoff=1e-12)
    f.sweep(sweeps, stop_on_converge=False)
    C, reps, b, lam = _gpu_fit(A, B, chi, 0.0, sweeps, gauge=gauge, update=update, oversample=4, seed=3,
                               precision=precision, sv_cutoff=1e-12, conv_tol=0.0)
    assert b == f.bonds()
    assert _rel(C, f.result()) <= 1e-9
    for r, h in zip(reps, f.st.history):
        assert abs(r["norm2_C"] - h.norm2) <= 1e-10 * h.norm2


def test_df32_exact_product():
    A, B = mpo_pair("gauss_L8_chi8", 0)
    C, _, b, _ = _gpu_fit(A, B, 64, 0.0, 2, precision="df32")
    D = to_dense(A) @ to_dense(B)
    assert np.linalg.norm(to_dense(C) - D) <= 1e-11 * np.linalg.norm(D)


def test_df32_fast_factor_converges():
    """The bench's second phase: DF32 contractions with the FP32 factorisation
    and FP64 polish reach delta <= 1e-10 and the FP64 oracle's operator."""
    A, B = _fast_pair(3)
    o = FitOracle(A, B, 12, 0.0)
    o.sweep(12, stop_on_converge=False)
    h = ttfit.tt_fit_create(A, B, 12, 0.0, "site", precision="df32", fast_factor=True, conv_tol=0.0)
    reps = [h.sweep(1) for _ in range(12)]
    assert reps[-1]["delta"] <= 1e-10
    # the FP32 subspace enters ||C||^2 only at second order: delta <= 1e-10
    # bounds the operator distance to about sqrt(delta)
    assert _rel([c.cpu().numpy() for c in h.result()], o.result()) <= 1e-5
    h.destroy()


def test_switch_tf32x3_to_df32_and_cutoff_follows_precision():
    """A 3xTF32 start (cut-off 1e-6) switched to DF32 keeps values down to the
    DF32 cut-off (1e-12), like an FP64 fit with that cut-off."""
    A, B = _fast_pair(2)
    o = FitOracle(A, B, 12, 0.0, sv_cutoff=1e-12)
    o.sweep(14, stop_on_converge=False)
    h = ttfit.tt_fit_create(A, B, 12, 0.0, "site", precision="tf32x3", conv_tol=0.0)
    h.sweep(2)
    h.set_precision("df32")
    for _ in range(12):
        rep = h.sweep(1)
    assert rep["delta"] <= 1e-10
    assert h.bonds() == o.bonds()
    assert _rel([c.cpu().numpy() for c in h.result()], o.result()) <= 1e-8
    h.destroy()


@pytest.mark.parametrize("precision,fast", [("fp64", True), ("df32", True), ("tf32x3", False), ("fp32", False)])
def test_fp32_factorisation_of_a_tiny_first_window(precision, fast):
    """From a random guess on a long chain the two-site tensors of the first
    sweep are tiny (the guess overlaps A B by ~1e-15): their squares underflow
    FP32 unless the factorisation works on 2^-e Theta. Every precision's first
    sweep must give the FP64 path's ||C||^2 (to its own accuracy), and C must be
    the fitted operator (its norm equals the reported one)."""
    A = kron_sum_mpo(30, 16, 0, 0)
    B = kron_sum_mpo(30, 16, 0, 1)
    ref = ttfit.tt_fit_create(A, B, 16, 0.0, "site", precision="fp64", conv_tol=0.0, sv_cutoff=1e-13)
    r0 = ref.sweep(1)
    ref.destroy()
    f = ttfit.tt_fit_create(A, B, 16, 0.0, "site", precision=precision, fast_factor=fast, conv_tol=0.0,
                            sv_cutoff=1e-13)
    r = f.sweep(1)
    C = [c.cpu().numpy() for c in f.result()]
    f.destroy()
    tol = 1e-3 if precision in ("tf32x3", "fp32") else 1e-6
    assert abs(r["norm2_C"] - r0["norm2_C"]) <= tol * r0["norm2_C"]
    assert abs(mpo_norm(C) ** 2 - r["norm2_C"]) <= 10 * tol * r["norm2_C"]


def test_block_cache_reuse_and_release():
    """Handles take their device blocks from a process-wide cache. A fit of
    (A, B) on fresh blocks, then a fit of other inputs with the same shapes
    (its blocks go back to the cache holding its data), then (A, B) again on
    those reused blocks: the two (A, B) results are bitwise equal, so nothing
    reads a block before writing it. Releasing the cache frees what it held."""
    A = kron_sum_mpo(10, 8, 2, 0)
    B = kron_sum_mpo(10, 8, 2, 1)
    A2 = kron_sum_mpo(10, 8, 2, 5)
    B2 = kron_sum_mpo(10, 8, 2, 6)
    kw = dict(precision="tf32x3", update="rsvd", seed=3)
    ttfit.tt_device_cache_release(-1)
    C0, r0, _, _ = _gpu_fit(A, B, 24, 0.0, 3, **kw)
    _gpu_fit(A2, B2, 24, 0.0, 3, **kw)
    C1, r1, _, _ = _gpu_fit(A, B, 24, 0.0, 3, **kw)
    for a, b in zip(C0, C1):
        assert np.array_equal(a, b)
    assert [r["norm2_C"] for r in r0] == [r["norm2_C"] for r in r1]
    assert ttfit.tt_device_cache_release(-1) > 0
    assert ttfit.tt_device_cache_release(-1) == 0


@pytest.mark.parametrize("precision,passes", [("fp64", None), ("df32", 21), ("bf16_split", 21), ("tf32x3", 3)])
def test_issued_flops_account_for_the_algorithmic_ones(precision, passes):
    """tt_fit_exec_flops against tt_fit_stage_times on the same sweeps: in FP64 every chain
    contraction runs on the CUDA cores, so the two counts agree exactly; on the tensor cores
    each algorithmic flop is issued once per pass (3xTF32: 3, digit split: 21 digit pairs) or
    more (tile and k-block padding)."""
    A, B = mpo_pair("kron_L12_chi32", 1)
    f = ttfit.tt_fit_create(A, B, 12, 0.0, "site", update="rsvd", oversample=4, seed=3, precision=precision,
                            conv_tol=0.0)
    try:
        for _ in range(2):
            f.sweep(1)
            alg = f.stage_times()["contraction_flops"]
            ex = f.exec_flops()
            assert alg > 0
            if passes is None:
                assert ex["tensor_core"] == 0.0 and ex["cuda_core"] == alg
            else:
                assert ex["tensor_core"] > 0.0
                assert ex["tensor_core"] / passes + ex["cuda_core"] >= alg * (1 - 1e-12)
                assert ex["cuda_core"] < alg
    finally:
        f.destroy()
