"""The timed configuration at full size: L = 30, chi_A = chi_B = chi_C = 128,
Kronecker-sum inputs (K = 128 terms), randomized update (k_s = 138), one 3xTF32
sweep, then DF32 sweeps with the FP64-polished FP32 factorisation: the launch
configuration bench.py times (its DF32 contractions with BF16 digit planes,
bf16_split; the TF32 digit planes, df32, are checked the same way). Where the oracle cannot follow, check what holds
at any size, with plain PyTorch FP64 on the device (tests/mpo_props.py):

* the fit converges to delta <= 1e-8;
* the reported ||C||^2 is the squared norm of the exported cores;
* at a converged fit the last update projected the two-site tensor on the
  environment basis (Alg. 3), so <C, A B> = ||C||^2 and the residual of
  Eq. fit_min is ||A B||^2 - ||C||^2;
* the exported cores are in one site-canonical gauge: every core left of the
  orthogonality centre left-orthonormal, or every core right of it
  right-orthonormal, depending on the direction of the last sweep;
* C agrees with the FP64 fit (FP64 contractions and factorisation, the path
  pinned to the oracle, same inputs, seed and sweep count) to a relative
  Frobenius error <= 1e-7 (measured 5e-9; the mixed-precision bound is 1e-6),
  by the stable difference norm.
(This file runs last among the GPU tests.)"""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from mpo_props import diff_norm, inner_ab, norm2  # noqa: E402
from paper_2606_23274_gb300 import ttfit  # noqa: E402
from paper_2606_23274_gb300.synth import mpo_pair  # noqa: E402


def _gram_dev(c, left: bool) -> float:
    """max |G - I| of a core's left (sum over c0, s, t) or right (sum over s, t, c1) Gram matrix."""
    m = c.reshape(-1, c.shape[-1]) if left else c.reshape(c.shape[0], -1).T
    G = m.T @ m
    return float((G - torch.eye(G.shape[0], dtype=G.dtype, device=G.device)).abs().max())


@pytest.mark.parametrize("hi", ["bf16_split", "df32"])
def test_timed_configuration_full_size(hi):
    A, B = mpo_pair("kron_L30_chi128", seed=0)
    f = ttfit.tt_fit_create(A, B, 128, 1e-8, "site", update="rsvd", oversample=10, seed=0, precision="tf32x3")
    try:
        rep = f.sweep(1)
        f.set_precision(hi, fast_factor=True)
        for _ in range(8):
            rep = f.sweep(1)
            if rep["converged"]:
                break
        assert rep["converged"] == 1 and rep["delta"] <= 1e-8
        C = f.result()
        n2 = norm2(C)
        assert abs(n2 - rep["norm2_C"]) <= 1e-9 * n2
        Ad = [torch.from_numpy(a).cuda() for a in A]
        Bd = [torch.from_numpy(b).cuda() for b in B]
        assert abs(inner_ab(C, Ad, Bd) - n2) <= 1e-7 * n2
        left = max(_gram_dev(c, True) for c in C[:-1])
        right = max(_gram_dev(c, False) for c in C[1:])
        assert min(left, right) <= 1e-9
        sweeps = rep["sweeps_done"]
    finally:
        f.destroy()
    g = ttfit.tt_fit_create(A, B, 128, 1e-8, "site", update="rsvd", oversample=10, seed=0, precision="fp64",
                            conv_tol=0.0)
    try:
        g.sweep(sweeps)
        Cref = g.result()
    finally:
        g.destroy()
    err = diff_norm(C, Cref) / norm2(Cref) ** 0.5
    print(f"timed configuration ({hi}): relative Frobenius error vs the FP64 fit after {sweeps} sweeps: {err:.3e}")
    assert err <= 1e-7
