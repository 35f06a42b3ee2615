"""Segment-parallel fit (Sec. 4, Alg. 6, inverse gauge) and batched fits of
independent pairs on the GPU, through the C ABI, against the oracle's Alg. 6
simulation and its serial fit on the same seeded inputs."""
import numpy as np
import pytest

from oracle.fit import FitOracle
from oracle.mpo import mpo_diff_norm, mpo_norm, naive_product, to_dense
from oracle.parallel import ParallelFitOracle
from paper_2606_23274_gb300.synth import kron_sum_mpo, mpo_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_23274_gb300 import ttfit  # noqa: E402


def _rel(X, Y):
    return mpo_diff_norm(X, Y) / mpo_norm(Y)


def _cpu(C):
    return [c.cpu().numpy() for c in C]


@pytest.mark.parametrize("n_seg,edge", [(2, 0), (3, 0), (3, 1), (4, 1)])
@pytest.mark.parametrize("update", ["svd", "rsvd"])
def test_parallel_fp64_matches_oracle(n_seg, edge, update):
    """Two full sets of local sweeps: ||C||^2 after every phase, bonds, the
    operator and the spectra agree with the oracle's Alg. 6 simulation."""
    A, B = mpo_pair("kron_L12_chi32", 1)
    chi, sets = 12, 2
    p = ParallelFitOracle(A, B, chi, 0.0, n_seg, edge, update=update, oversample=4, seed=5)
    par = [p.full_sweep_set() for _ in range(sets)]
    f = ttfit.tt_fit_create(A, B, chi, 0.0, "inverse", update=update, oversample=4, seed=5, precision="fp64",
                            conv_tol=0.0, n_segments=n_seg, edge_extra=edge)
    reps = [f.sweep(1) for _ in range(2 * sets)]
    C = _cpu(f.result())
    assert f.bonds() == p.bonds()
    for s in range(sets):
        n2o = par[s][0]
        assert abs(reps[2 * s + 1]["norm2_C"] - n2o) <= 1e-11 * n2o
    assert reps[-1]["sweeps_done"] == 2 * sets
    assert _rel(C, p.result()) <= 1e-9
    for lg, lo in zip(f.lambdas(), p.lambdas()):
        assert np.allclose(lg[: len(lo)], lo, rtol=1e-9, atol=1e-12 * lo[0])
    f.destroy()


def test_parallel_exact_product_dense():
    """chi_C = chi_A chi_B: the parallel fit reproduces A B (dense 256 x 256)."""
    A, B = mpo_pair("gauss_L8_chi8", 0)
    f = ttfit.tt_fit_create(A, B, 64, 0.0, "inverse", precision="fp64", n_segments=3)
    f.sweep(4)
    D = to_dense(A) @ to_dense(B)
    assert np.linalg.norm(to_dense(_cpu(f.result())) - D) <= 1e-10 * np.linalg.norm(D)
    f.destroy()


def test_parallel_converges_like_the_oracle():
    """Weights 0.5^k: the GPU's Alg. 6 converges (delta <= 1e-13) to the
    oracle's Alg. 6 fixed point within 1e-8. That fixed point need not be the
    serial fit's (here it is a nearby stationary point, ~1 % higher residual),
    so against the serial fit only the residual is bounded."""
    A = kron_sum_mpo(16, 16, 4, 0, decay=0.5)
    B = kron_sum_mpo(16, 16, 4, 1, decay=0.5)
    f = ttfit.tt_fit_create(A, B, 12, 0.0, "inverse", precision="fp64", conv_tol=1e-13, n_segments=4,
                            edge_extra=1)
    rep = f.sweep(30)
    assert rep["converged"] == 1
    p = ParallelFitOracle(A, B, 12, 0.0, 4, 1)
    for _ in range(10):
        n2o, _ = p.full_sweep_set()
    C = _cpu(f.result())
    assert _rel(C, p.result()) <= 1e-8
    assert abs(rep["norm2_C"] - n2o) <= 1e-12 * n2o
    s = FitOracle(A, B, 12, 0.0, gauge="inverse")
    s.sweep(16, stop_on_converge=False)
    N = naive_product(A, B)
    assert mpo_diff_norm(N, C) <= 1.05 * mpo_diff_norm(N, s.result())
    f.destroy()


def test_parallel_fp32_quality():
    """FP32 contractions with the polished FP32 factorisation, 8 segments on
    L = 24 (two 12-site Kronecker sums side by side): the residual ||AB - C||
    is within 1e-3 (relative) of the FP64 oracle's parallel fit."""
    A = kron_sum_mpo(12, 16, 2, 0) + kron_sum_mpo(12, 16, 3, 0)
    B = kron_sum_mpo(12, 16, 2, 1) + kron_sum_mpo(12, 16, 3, 1)
    N = naive_product(A, B)
    p = ParallelFitOracle(A, B, 10, 0.0, 8, 1)
    for _ in range(4):
        p.full_sweep_set()
    res_o = mpo_diff_norm(N, p.result())
    f = ttfit.tt_fit_create(A, B, 10, 0.0, "inverse", precision="fp32", conv_tol=0.0, n_segments=8, edge_extra=1)
    f.sweep(8)
    res = mpo_diff_norm(N, _cpu(f.result()))
    assert res <= res_o * (1 + 1e-3) + 1e-5 * mpo_norm(N)
    f.destroy()


def test_parallel_precision_switch():
    """3xTF32 sets, then FP64 with the fast factorisation (FP32 subspace, FP64
    polish; its delta floor is ~1e-12): converges to the oracle's fixed point."""
    A = kron_sum_mpo(12, 16, 6, 0, decay=0.5)
    B = kron_sum_mpo(12, 16, 6, 1, decay=0.5)
    f = ttfit.tt_fit_create(A, B, 12, 0.0, "inverse", precision="tf32x3", conv_tol=1e-10, n_segments=3)
    f.sweep(1)
    with pytest.raises(ttfit.TTError) as e:
        f.set_precision("fp64", fast_factor=True)                # mid-set: refused
    assert e.value.code == ttfit.TT_ERR_STATE
    f.sweep(3)
    f.set_precision("fp64", fast_factor=True)
    rep = f.sweep(30)
    assert rep["converged"] == 1
    p = ParallelFitOracle(A, B, 12, 0.0, 3)
    for _ in range(12):
        p.full_sweep_set()
    # ||C||^2 is stationary at the fixed point, so delta <= 1e-10 bounds the
    # distance of the operators only to about sqrt(delta)
    assert _rel(_cpu(f.result()), p.result()) <= 1e-5
    f.destroy()


def test_parallel_rejects_bad_options():
    A, B = mpo_pair("kron_L10_chi16", 0)
    with pytest.raises(ttfit.TTError) as e:
        ttfit.tt_fit_create(A, B, 8, 0.0, "inverse", n_segments=6)  # 10 sites < 2 x 6
    assert e.value.code == ttfit.TT_ERR_INVALID_ARGUMENT


def test_batched_pairs_match_serial_oracle():
    """Independent pairs of different lengths and bond dimensions, one launch
    thread and stream each: every fit equals its own serial oracle fit."""
    specs = [(10, 16, 8), (14, 16, 12), (8, 8, 16), (12, 32, 10), (16, 16, 6), (9, 8, 8)]
    pairs = [(kron_sum_mpo(L, K, 20 + i, 0), kron_sum_mpo(L, K, 20 + i, 1)) for i, (L, K, _) in enumerate(specs)]
    chis = [c for _, _, c in specs]
    fits = ttfit.tt_fit_create_batched(pairs, chis, 0.0, "inverse", precision="fp64", conv_tol=0.0, seed=2)
    reps = [ttfit.tt_fit_sweep_batched(fits, 1) for _ in range(3)]
    for i, (A, B) in enumerate(pairs):
        o = FitOracle(A, B, chis[i], 0.0, gauge="inverse", seed=2)
        o.sweep(3, stop_on_converge=False)
        assert fits[i].bonds() == o.bonds()
        assert _rel(_cpu(fits[i].result()), o.result()) <= 1e-9
        for s in range(3):
            assert abs(reps[s][i]["norm2_C"] - o.st.history[s].norm2) <= 1e-11 * o.st.history[s].norm2
        fits[i].destroy()


def test_batched_segment_parallel_pairs():
    """Batched handles that are each segment-parallel (2 segments)."""
    pairs = [mpo_pair("kron_L12_chi32", s) for s in (7, 8)]
    fits = ttfit.tt_fit_create_batched(pairs, [10, 12], 0.0, "inverse", n_segments=2, precision="fp64",
                                       conv_tol=0.0)
    for _ in range(4):
        ttfit.tt_fit_sweep_batched(fits, 1)
    for f, (A, B), chi in zip(fits, pairs, [10, 12]):
        p = ParallelFitOracle(A, B, chi, 0.0, 2)
        p.full_sweep_set()
        p.full_sweep_set()
        assert _rel(_cpu(f.result()), p.result()) <= 1e-9
        f.destroy()


def test_parallel_df32_matches_oracle():
    A, B = mpo_pair("kron_L12_chi32", 1)
    p = ParallelFitOracle(A, B, 12, 0.0, 3, 1, update="rsvd", oversample=4, seed=5, sv_cutoff=1e-12)
    par = [p.full_sweep_set() for _ in range(2)]
    f = ttfit.tt_fit_create(A, B, 12, 0.0, "inverse", update="rsvd", oversample=4, seed=5, precision="df32",
                            sv_cutoff=1e-12, conv_tol=0.0, n_segments=3, edge_extra=1)
    reps = [f.sweep(1) for _ in range(4)]
    assert abs(reps[3]["norm2_C"] - par[1][0]) <= 1e-10 * par[1][0]
    assert _rel(_cpu(f.result()), p.result()) <= 1e-9
    f.destroy()


def test_batched_uneven_shapes_match_serial_fits():
    """Sixteen handles whose windows differ in shape (hence in the shared memory
    their factorisation kernels request) sweep concurrently, one host thread
    each, and give the same fits as one at a time. The kernels' shared-memory
    limits are process-wide, so a launch must never see a limit lowered by
    another thread (it then fails with an invalid argument)."""
    rng = np.random.default_rng(7)
    Ls = rng.integers(8, 15, size=16)
    chis = rng.choice([6, 8, 12, 16, 24], size=16)
    pairs = [(kron_sum_mpo(int(L), int(c), 300 + i, 0), kron_sum_mpo(int(L), int(c), 300 + i, 1))
             for i, (L, c) in enumerate(zip(Ls, chis))]
    kw = dict(update="rsvd", oversample=6, seed=2, precision="tf32x3", conv_tol=0.0)
    fits = ttfit.tt_fit_create_batched(pairs, [int(c) for c in chis], 0.0, "inverse", **kw)
    try:
        reps = ttfit.tt_fit_sweep_batched(fits, 3)
        got = [[c.cpu().numpy() for c in f.result()] for f in fits]
    finally:
        for f in fits:
            f.destroy()
    for (A, B), c, r, C in zip(pairs, chis, reps, got):
        f = ttfit.tt_fit_create(A, B, int(c), 0.0, "inverse", **kw)
        try:
            r1 = f.sweep(3)
            C1 = [x.cpu().numpy() for x in f.result()]
        finally:
            f.destroy()
        assert abs(r["norm2_C"] - r1["norm2_C"]) <= 1e-6 * r1["norm2_C"]
        assert mpo_diff_norm(C, C1) <= 1e-5 * mpo_norm(C1)
