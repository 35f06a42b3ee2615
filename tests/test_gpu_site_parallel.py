"""Parity of the site-canonical segment-parallel fit (Sec. 4, scheme II) and
its binary merge (Sec. 4.5) with the FP64 oracle, through the C ABI: ||C||^2
after every full set of local sweeps, after the merge, and the merged
operator, for several segment counts, both updates, and merges after a full
set or after an odd|even phase."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from mpo_props import diff_norm, norm2  # noqa: E402
from oracle.parallel import SiteParallelFitOracle  # noqa: E402
from paper_2606_23274_gb300 import ttfit  # noqa: E402
from paper_2606_23274_gb300.synth import kron_sum_mpo, mpo_pair  # noqa: E402


def _pair():
    return kron_sum_mpo(12, 5, 6, 0, decay=0.7), kron_sum_mpo(12, 5, 6, 1, decay=0.5)


@pytest.mark.parametrize("update", ["svd", "rsvd"])
@pytest.mark.parametrize("n_seg", [2, 3, 4])
@pytest.mark.parametrize("half", [False, True])
def test_site_parallel_fit_matches_oracle(n_seg, update, half):
    A, B = _pair()
    kw = dict(update=update, oversample=2, seed=4, conv_tol=0.0)
    ref = SiteParallelFitOracle(A, B, 10, 0.0, n_seg, **kw)
    f = ttfit.tt_fit_create(A, B, 10, 0.0, "site", precision="fp64", sv_cutoff=1e-13, n_segments=n_seg, **kw)
    try:
        for s in range(2):
            n2_ref, _ = ref.full_sweep_set()
            f.sweep(1)
            rep = f.sweep(1)
            assert abs(rep["norm2_C"] - n2_ref) <= 1e-10 * n2_ref, (s, rep["norm2_C"], n2_ref)
        if half:
            n2_ref = ref.half_set()
            rep = f.sweep(1)
            assert abs(rep["norm2_C"] - n2_ref) <= 1e-10 * n2_ref
        with pytest.raises(ttfit.TTError):
            f.result()  # not merged
        n2_ref = ref.merge()
        rep = f.merge()
        assert abs(rep["norm2_C"] - n2_ref) <= 1e-10 * n2_ref
        assert f.bonds() == ref.bonds()
        C = f.result()
        R = [torch.from_numpy(c).cuda() for c in ref.result()]
        e = diff_norm(C, R) / norm2(R) ** 0.5
        print(n_seg, update, half, "merged rel. Frobenius vs oracle", e)
        assert e <= 1e-10
        assert abs(norm2(C) - rep["norm2_C"]) <= 1e-10 * rep["norm2_C"]   # one orthogonality centre
    finally:
        f.destroy()


def test_site_parallel_continues_after_merge_and_switches_precision():
    """Sweeps continue from the merged C; a precision switch needs a merged fit and
    re-partitions it; the merged fit of the converged parallel run equals the serial
    optimum."""
    A, B = _pair()
    s = ttfit.tt_fit_create(A, B, 10, 0.0, "site", precision="fp64", conv_tol=0.0)
    s.sweep(12)
    C_ser = s.result()
    s.destroy()
    f = ttfit.tt_fit_create(A, B, 10, 0.0, "site", precision="tf32x3", n_segments=3, conv_tol=0.0)
    try:
        f.sweep(4)
        with pytest.raises(ttfit.TTError):
            f.set_precision("fp64")
        f.merge()
        f.set_precision("fp64")
        f.sweep(16)
        f.merge()
        C = f.result()
        e = diff_norm(C, C_ser) / norm2(C_ser) ** 0.5
        print("site parallel (3 segments) vs serial", e)
        assert e <= 1e-8
    finally:
        f.destroy()


def test_site_parallel_timed_workload():
    """L = 30, chi = 128 in 4 segments: 3xTF32 phases, then DF32 contractions with the
    FP64 factorisation, merged, against the FP64 serial fit. The Kronecker weights
    0.8^k make the kept spectrum degenerate at the cut, so fits of equal ||C||^2 differ
    by ~2e-4 in the operator (the FP64 serial and FP64 segment-parallel fits, in either
    gauge, do): ||C||^2, which is unique, is compared."""
    A, B = mpo_pair("kron_L30_chi128", seed=0)
    g = ttfit.tt_fit_create(A, B, 128, 1e-8, "site", update="rsvd", seed=0, precision="fp64", conv_tol=0.0)
    g.sweep(5)
    ref = g.result()
    g.destroy()
    f = ttfit.tt_fit_create(A, B, 128, 1e-8, "site", update="rsvd", seed=0, precision="tf32x3", n_segments=4,
                            edge_extra=2)
    try:
        f.sweep(2)
        f.merge()
        f.set_precision("df32", fast_factor=0)
        for _ in range(10):
            rep = f.sweep(2)
            if rep["converged"]:
                break
        rep = f.merge()
        C = f.result()
        e_n2 = rep["norm2_C"] / norm2(ref) - 1.0
        e = diff_norm(C, ref) / norm2(ref) ** 0.5
        print("site parallel L30 (4 segments, mixed): ||C||^2 rel", e_n2, "operator", e, "phases", rep["sweeps_done"])
        assert abs(e_n2) <= 1e-7
        assert abs(norm2(C) / rep["norm2_C"] - 1.0) <= 1e-10
    finally:
        f.destroy()
