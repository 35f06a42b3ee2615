"""The paper's second workload on the GPU (Sec. 5.1): random tensor trains with
entries uniform in [alpha, 1] and normalised cores. Their singular values decay
slowly, and ||A B|| falls like ~0.2^L, so a chain of the paper's length
(L = 102) sits far below the FP32 range unless the prepared inputs are
rescaled (the library takes exact powers of two off A and B and gives them
back to C on export)."""
import numpy as np
import pytest

from oracle.fit import FitOracle
from oracle.mpo import mpo_diff_norm, mpo_norm
from paper_2606_23274_gb300.synth import mpo_pair, uniform_mpo

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from mpo_props import diff_norm, norm2  # noqa: E402
from paper_2606_23274_gb300 import ttfit  # noqa: E402


def _fit(A, B, chi, sweeps, **kw):
    f = ttfit.tt_fit_create(A, B, chi, 0.0, kw.pop("gauge", "site"), conv_tol=0.0, **kw)
    try:
        reps = [f.sweep(1) for _ in range(sweeps)]
        return f.result(), reps, f.bonds(), f.lambdas()
    finally:
        f.destroy()


@pytest.mark.parametrize("gauge", ["site", "inverse"])
@pytest.mark.parametrize("update", ["svd", "rsvd"])
def test_uniform_fp64_matches_oracle(gauge, update):
    A, B = mpo_pair("uniform_L12_chi12", 0)
    chi, sweeps = 10, 4
    o = FitOracle(A, B, chi, 0.0, gauge=gauge, update=update, oversample=4, seed=2, conv_tol=0.0)
    o.sweep(sweeps, stop_on_converge=False)
    C, reps, b, lam = _fit(A, B, chi, sweeps, gauge=gauge, update=update, oversample=4, seed=2, precision="fp64")
    Cn = [c.cpu().numpy() for c in C]
    assert b == o.bonds()
    assert mpo_diff_norm(Cn, o.result()) <= 1e-9 * mpo_norm(o.result())
    for r, h in zip(reps, o.st.history):
        assert abs(r["norm2_C"] - h.norm2) <= 1e-10 * h.norm2
    for got, ref in zip(lam, o.lambdas()):
        assert np.allclose(got, ref, rtol=1e-8, atol=1e-12 * ref[0])


def test_uniform_long_chain_mixed_precision_stays_in_range():
    """L = 102 (the paper's length), chi = 8, alpha = -0.5: ||A B|| ~ 3e-62, far
    below FP32's range. After 6 sweeps of the exact update the FP64 GPU fit
    matches the FP64 oracle, and the 3xTF32 -> DF32 fit (whose chains have
    FP32's exponent range) matches it too."""
    L, chi, sweeps = 102, 8, 6
    A = uniform_mpo(L, 2, chi, 3, 0, -0.5)
    B = uniform_mpo(L, 2, chi, 3, 1, -0.5)
    o = FitOracle(A, B, chi, 0.0, update="svd", seed=1, conv_tol=0.0)
    o.sweep(sweeps, stop_on_converge=False)
    ref = o.result()
    n_ref = mpo_norm(ref)
    assert n_ref < 1e-50                                      # far below FP32's range
    C64, reps64, _, _ = _fit(A, B, chi, sweeps, update="svd", seed=1, precision="fp64")
    assert mpo_diff_norm([c.cpu().numpy() for c in C64], ref) <= 1e-9 * n_ref
    assert abs(reps64[-1]["norm2_C"] - o.st.history[-1].norm2) <= 1e-10 * n_ref ** 2
    f = ttfit.tt_fit_create(A, B, chi, 0.0, "site", update="svd", seed=1, precision="tf32x3", conv_tol=0.0)
    try:
        f.sweep(1)
        f.set_precision("df32", fast_factor=1)
        for _ in range(sweeps - 1):
            rep = f.sweep(1)
        C = f.result()
    finally:
        f.destroy()
    Cd = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in ref]
    err = diff_norm(C, Cd) / n_ref
    print("uniform L=102 chi=8: mixed vs oracle", err, "norm", n_ref)
    assert np.isfinite(err) and err <= 1e-6
    assert abs(rep["norm2_C"] - norm2(C)) <= 1e-9 * norm2(C)
