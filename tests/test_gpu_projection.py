"""Parity of the fit on randomized bond projections of A and B (Sec. 3.2,
tt_fit_options.ab_rank) with the FP64 oracle, through the C ABI.

Both sides prepare A and B alike (reading of Alg. 5's preparation), draw the
same Philox sketch per bond and project right to left; the library keeps the
projected bond in a rotated basis (its zip-up factorisation), which the fit
does not see, so the fits agree to rounding."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from mpo_props import diff_norm, norm2  # noqa: E402
from oracle.fit import FitOracle  # noqa: E402
from paper_2606_23274_gb300 import ttfit  # noqa: E402
from paper_2606_23274_gb300.synth import mpo_pair  # noqa: E402


@pytest.mark.parametrize("gauge", ["site", "inverse"])
@pytest.mark.parametrize("update", ["svd", "rsvd"])
def test_projected_fit_matches_oracle(gauge, update):
    A, B = mpo_pair("kron_L10_chi16", seed=0)
    ref = FitOracle(A, B, 16, 1e-10, gauge=gauge, update=update, oversample=10, seed=3, conv_tol=0.0,
                    ab_rank=6)
    ref.sweep(4, stop_on_converge=False)
    f = ttfit.tt_fit_create(A, B, 16, 1e-10, gauge, update=update, oversample=10, seed=3, precision="fp64",
                            conv_tol=0.0, sv_cutoff=1e-13, ab_rank=6)
    try:
        for s in range(4):
            rep = f.sweep(1)
            want = ref.st.history[s].norm2
            print(gauge, update, s + 1, rep["norm2_C"], want)
            assert abs(rep["norm2_C"] - want) <= 1e-10 * want
            assert f.bonds() == ref.st.history[s].bonds
        C = f.result()
        R = [torch.from_numpy(c).cuda() for c in ref.result()]
        e = diff_norm(C, R) / norm2(R) ** 0.5
        print("rel. Frobenius vs oracle", e)
        assert e <= 1e-9
    finally:
        f.destroy()


def test_projection_wider_than_the_bonds_changes_nothing():
    A, B = mpo_pair("kron_L10_chi16", seed=1)
    out = []
    for k in (0, 16):
        f = ttfit.tt_fit_create(A, B, 16, 1e-10, "site", update="rsvd", seed=2, precision="fp64", conv_tol=0.0,
                                ab_rank=k)
        f.sweep(3)
        out.append(f.result())
        f.destroy()
    assert diff_norm(out[0], out[1]) <= 1e-11 * norm2(out[0]) ** 0.5


def test_projection_needs_prepared_inputs():
    A, B = mpo_pair("kron_L10_chi16", seed=0)
    with pytest.raises(ttfit.TTError):
        ttfit.tt_fit_create(A, B, 16, 1e-10, "site", prepare_inputs=False, ab_rank=4)
    with pytest.raises(ttfit.TTError):
        ttfit.tt_fit_create(A, B, 16, 1e-10, "site", ab_rank=-1)


def test_projected_timed_workload_mixed_precision():
    """L = 30, chi = 128 with rank-64 projections of A and B (the Kronecker weights
    0.8^k leave ~0.64^32 of the weight outside them): the bench's schedule against
    the FP64 fit of the same projected product, and the projected fit against the
    unprojected one."""
    A, B = mpo_pair("kron_L30_chi128", seed=0)
    res = {}
    for prec, k in (("fp64", 64), ("mixed", 64), ("fp64", 0)):
        lo = "tf32x3" if prec == "mixed" else "fp64"
        f = ttfit.tt_fit_create(A, B, 128, 1e-8, "site", update="rsvd", seed=0, precision=lo, ab_rank=k)
        n = 1
        f.sweep(1)
        if prec == "mixed":
            f.set_precision("df32", fast_factor=1)
        while n < 8:
            rep = f.sweep(1)
            n += 1
            if rep["converged"]:
                break
        res[(prec, k)] = f.result()
        f.destroy()
    ref = res[("fp64", 64)]
    e_mixed = diff_norm(res[("mixed", 64)], ref) / norm2(ref) ** 0.5
    e_proj = diff_norm(res[("fp64", 0)], ref) / norm2(res[("fp64", 0)]) ** 0.5
    print("mixed vs fp64 (projected)", e_mixed, "projected vs unprojected", e_proj)
    assert e_mixed <= 1e-6
    assert e_proj <= 1e-4
