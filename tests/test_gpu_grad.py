"""Adjoint of the contraction chain on the GPU (tt_mpo_grad) against the FP64
oracle's gradients, FP64 central finite differences of the GPU's own value,
properties that hold at any size, and torch.autograd."""
import numpy as np
import pytest

from oracle.grad import f1_and_grads, f2_and_grads
from paper_2606_23274_gb300.synth import gaussian_mpo, kron_sum_mpo

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_23274_gb300 import ttfit  # noqa: E402


def _np(ts):
    return [t.double().cpu().numpy() for t in ts]


def _relmax(G, R):
    return max(np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300) for g, r in zip(G, R))


def _inputs(L=6, chi=4, seed=0):
    A = gaussian_mpo(L, 2, chi, seed, 0, 0.7)
    B = gaussian_mpo(L, 2, chi, seed, 1, 0.7)
    X = gaussian_mpo(L, 2, chi + 2, seed, 2, 0.7)
    return A, B, X


@pytest.mark.parametrize("target", ["residual", "inner"])
@pytest.mark.parametrize("ckpt", [1, 2, 0])
def test_fp64_matches_oracle(target, ckpt):
    A, B, X = _inputs()
    v, gA, gB = ttfit.tt_mpo_grad(A, B, X, target, "fp64", ckpt)
    vo, oA, oB = (f1_and_grads if target == "residual" else f2_and_grads)(X, A, B)
    assert abs(v - vo) <= 1e-12 * abs(vo)
    assert _relmax(_np(gA), oA) <= 1e-11
    assert _relmax(_np(gB), oB) <= 1e-11


def test_uneven_bonds_and_dims():
    """Kronecker-sum inputs (bonds 1, 4, 16, ... trimmed by nothing) and an X of
    other bonds; the edge cores have bond 1."""
    A = kron_sum_mpo(7, 5, 1, 0)
    B = kron_sum_mpo(7, 3, 1, 1)
    X = gaussian_mpo(7, 2, 6, 1, 2, 0.5)
    v, gA, gB = ttfit.tt_mpo_grad(A, B, X, "residual", "fp64", 3)
    vo, oA, oB = f1_and_grads(X, A, B)
    assert abs(v - vo) <= 1e-11 * abs(vo)
    assert _relmax(_np(gA), oA) <= 1e-10 and _relmax(_np(gB), oB) <= 1e-10


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_fp32_matches_oracle(precision):
    """FP32 environments; with tf32x3 the contractions TMA can load run as 3xTF32 on the
    tensor cores (about FP32 accuracy)."""
    A = kron_sum_mpo(8, 12, 2, 0)
    B = kron_sum_mpo(8, 12, 2, 1)
    X = gaussian_mpo(8, 2, 10, 2, 2, 0.5)
    for target, fn in (("residual", f1_and_grads), ("inner", f2_and_grads)):
        v, gA, gB = ttfit.tt_mpo_grad(A, B, X, target, precision)
        vo, oA, oB = fn(X, A, B)
        assert abs(v - vo) <= 1e-4 * abs(vo)
        assert _relmax(_np(gA), oA) <= 1e-4 and _relmax(_np(gB), oB) <= 1e-4


def test_tf32x3_config_size_matches_fp32():
    """L = 32, chi = 96 (the adjoint configuration): the 3xTF32 gradients against the
    all-FP32 ones."""
    A = kron_sum_mpo(32, 96, 5, 0)
    B = kron_sum_mpo(32, 96, 5, 1)
    X = gaussian_mpo(32, 2, 96, 5, 2)
    for target in ("residual", "inner"):
        v1, gA1, gB1 = ttfit.tt_mpo_grad(A, B, X, target, "fp32")
        v3, gA3, gB3 = ttfit.tt_mpo_grad(A, B, X, target, "tf32x3")
        assert abs(v3 - v1) <= 1e-4 * abs(v1)
        eA = max(float((a - b).norm() / b.norm()) for a, b in zip(gA3, gA1) if float(b.norm()) > 0)
        eB = max(float((a - b).norm() / b.norm()) for a, b in zip(gB3, gB1) if float(b.norm()) > 0)
        print(target, "tf32x3 vs fp32 gradients", eA, eB)
        assert eA <= 1e-3 and eB <= 1e-3


def test_central_finite_differences_of_the_gpu_value():
    """FP64 central differences (step 1e-6) of the GPU's own f1 along random
    directions in one core of A and one of B."""
    A, B, X = _inputs(L=5, chi=3, seed=4)
    _, gA, gB = ttfit.tt_mpo_grad(A, B, X, "residual", "fp64")
    rng = np.random.default_rng(3)
    h = 1e-6
    for which, l in (("A", 0), ("A", 2), ("B", 4), ("B", 1)):
        X0 = A if which == "A" else B
        E = rng.standard_normal(X0[l].shape)
        E /= np.linalg.norm(E)

        def f(t):
            Y = list(X0)
            Y[l] = X0[l] + t * E
            return ttfit.tt_mpo_grad(Y, B, X, "residual", "fp64")[0] if which == "A" else \
                ttfit.tt_mpo_grad(A, Y, X, "residual", "fp64")[0]
        fd = (f(h) - f(-h)) / (2 * h)
        g = (gA if which == "A" else gB)[l].cpu().numpy()
        assert np.isclose(fd, np.sum(g * E), rtol=1e-6, atol=1e-9)


def test_autograd_function():
    A, B, X = _inputs(seed=6)
    At = [torch.tensor(a, device="cuda", requires_grad=True) for a in A]
    Bt = [torch.tensor(b, device="cuda", requires_grad=True) for b in B]
    loss = ttfit.mpo_objective(At, Bt, X, "residual", "fp64")
    (3.0 * loss).backward()
    vo, oA, oB = f1_and_grads(X, A, B)
    assert abs(loss.item() - vo) <= 1e-12 * abs(vo)
    assert _relmax([t.grad.cpu().numpy() / 3.0 for t in At], oA) <= 1e-11
    assert _relmax([t.grad.cpu().numpy() / 3.0 for t in Bt], oB) <= 1e-11


def test_config_size_fp32_properties():
    """L = 32, chi_A = chi_B = 96, chi_C = 96 in FP32 (the four-layer
    environments hold 96^4 values): where the oracle cannot follow, check what
    holds at any size. f2 is linear in each core (Euler: <dA_l f2, A_l> = f2);
    ||AB||^2 is quadratic, so for f1 = ||C||^2 - 2<C,AB> + ||AB||^2,
    <dA_l f1, A_l> = 2 (||AB||^2 - <C, AB>) = f1 + ||AB||^2 - ||C||^2 at every l.
    Checkpointed (every 6) and stored environments agree."""
    L, chi = 32, 96
    A = kron_sum_mpo(L, chi, 9, 0)
    B = kron_sum_mpo(L, chi, 9, 1)
    C = kron_sum_mpo(L, chi, 9, 2)
    At = [torch.from_numpy(a).cuda() for a in A]
    Bt = [torch.from_numpy(b).cuda() for b in B]
    v2, hA, _ = ttfit.tt_mpo_grad(A, B, C, "inner", "fp32", 6)
    for l in (0, 7, 15, 31):     # normwise FP32 bound: the sums cancel
        e = float(torch.sum(hA[l].double() * At[l]))
        assert abs(e - v2) <= 1e-4 * float(hA[l].double().norm() * At[l].norm())
    v1, gA, gB = ttfit.tt_mpo_grad(A, B, C, "residual", "fp32", 6)
    eul = [float(torch.sum(gB[l].double() * Bt[l])) for l in (1, 16, 30)]
    scale = max(float(gB[l].double().norm() * Bt[l].norm()) for l in (1, 16, 30))
    assert max(eul) - min(eul) <= 1e-4 * scale
    v1b, gA2, _ = ttfit.tt_mpo_grad(A, B, C, "residual", "fp32", 1)
    assert abs(v1b - v1) <= 1e-4 * abs(v1)
    for l in (0, 13, 31):
        assert torch.allclose(gA[l], gA2[l], rtol=1e-3, atol=1e-6 * float(gA[l].abs().max()))
