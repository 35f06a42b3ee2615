"""Parity of the CUDA naive product (Alg. 1's contraction step), zip-up
(Alg. 2, right to left) and compression (Alg. 1's compress) with the FP64
oracle, all called through the C ABI, and of the fit started from the zip-up
guess (Sec. 2.3.5).

The zip-up factorises M_l (chi_A chi_B rows) by one-sided Jacobi up to 1024
rows, which is the oracle's SVD to rounding; beyond that through the Gram
matrix of the sketch, whose squared condition number resolves singular values
only down to ~sqrt(eps) s_1, so those cases are held to a looser bound. The
oracle takes the prepared inputs (RQ sweep, then QR sweep), as the library
does, so that both sketch the same left gauge."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from mpo_props import diff_norm, norm2  # noqa: E402
from oracle.fit import FitOracle  # noqa: E402
from oracle.mpo import canonicalize_input, naive_product  # noqa: E402
from oracle.zipup import compress, zipup_right_to_left  # noqa: E402
from paper_2606_23274_gb300 import ttfit  # noqa: E402
from paper_2606_23274_gb300.synth import gaussian_mpo, kron_sum_mpo, mpo_pair  # noqa: E402


def _dev(X, dtype=torch.float64):
    return [torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype) for x in X]


def _rel(C, R):
    """||C - R||_F / ||R||_F for MPOs on the device (stable difference norm)."""
    return diff_norm(C, _dev(R)) / norm2(_dev(R)) ** 0.5


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_naive_product_matches_oracle(dtype):
    A = gaussian_mpo(5, 2, 3, 11, 0)
    B = gaussian_mpo(5, 2, 4, 11, 1)
    B[2] = B[2][:, :, :1, :]                       # a ragged site: d_in = 1
    A[3] = np.concatenate([A[3], A[3][:, :1]], 1)  # and d_out = 3
    C = ttfit.tt_mpo_naive_product(_dev(A, dtype), _dev(B, dtype))
    R = naive_product(A, B)
    eps = 2.3e-16 if dtype == torch.float64 else 1.2e-7
    for c, r in zip(C, R):
        assert tuple(c.shape) == r.shape
        # each entry is a sum of d' products: a few roundings of the largest entry
        err = np.abs(c.double().cpu().numpy() - r)
        assert err.max() <= 8 * eps * max(1.0, np.abs(r).max())


def _zip_case(name):
    if name == "kron_L10_chi16":
        A, B = mpo_pair("kron_L10_chi16", seed=0)
        return A, B, 16
    if name == "gauss_L8_chi8":
        A, B = mpo_pair("gauss_L8_chi8", seed=2)
        return A, B, 24
    if name == "kron_L12_chi32":
        A, B = mpo_pair("kron_L12_chi32", seed=1)
        return A, B, 32
    raise KeyError(name)


@pytest.mark.parametrize("update", ["svd", "rsvd"])
@pytest.mark.parametrize("name", ["kron_L10_chi16", "gauss_L8_chi8", "kron_L12_chi32"])
def test_zipup_fp64_matches_oracle(name, update):
    """One-sided Jacobi of every M_l (at most 1024 rows): the oracle's result to
    rounding, kept bonds equal, cores equal (sign-fixed singular vectors)."""
    A, B, chi = _zip_case(name)
    Ap, Bp = canonicalize_input(A), canonicalize_input(B)
    R = zipup_right_to_left(Ap, Bp, chi, 0.0, 1e-13, update, 10, 5)
    C = ttfit.tt_mpo_zipup(A, B, chi, 0.0, update=update, oversample=10, seed=5, precision="fp64",
                           sv_cutoff=1e-13)
    assert [c.shape[0] for c in C] == [r.shape[0] for r in R]
    e = _rel(C, R)
    print(name, update, "rel. Frobenius vs oracle", e)
    assert e <= 1e-11
    for l in range(1, len(C)):  # the right-orthonormal cores themselves
        d = np.abs(C[l].cpu().numpy() - R[l]).max()
        assert d <= 1e-9, (l, d)


def test_zipup_gram_path_matches_oracle_L10_chi128():
    """M_l with 16384 rows: the randomized update (k_s = 138) and the Gram
    matrix of the 16384 x 138 projection. Its squared condition number costs
    the kept directions whose s_j fall below ~1e-8 s_1 their accuracy; they
    carry at most ~1e-8 of the weight (measured: 4e-13 overall)."""
    A, B = mpo_pair("kron_L10_chi128", seed=0)
    Ap, Bp = canonicalize_input(A), canonicalize_input(B)
    R = zipup_right_to_left(Ap, Bp, 128, 0.0, 1e-13, "rsvd", 10, 0)
    C = ttfit.tt_mpo_zipup(A, B, 128, 0.0, update="rsvd", oversample=10, seed=0, precision="fp64",
                           sv_cutoff=1e-13)
    assert [c.shape[0] for c in C] == [r.shape[0] for r in R]
    e = _rel(C, R)
    print("kron_L10_chi128 zip-up rel. Frobenius vs oracle", e)
    assert e <= 1e-9


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_zipup_fp32_close_to_oracle(precision):
    A, B, chi = _zip_case("kron_L12_chi32")
    Ap, Bp = canonicalize_input(A), canonicalize_input(B)
    R = zipup_right_to_left(Ap, Bp, chi, 0.0, 1e-6, "rsvd", 10, 5)
    C = ttfit.tt_mpo_zipup(A, B, chi, 0.0, update="rsvd", oversample=10, seed=5, precision=precision,
                           sv_cutoff=1e-6, dtype=torch.float64)
    e = _rel(C, R)
    print(precision, "zip-up rel. Frobenius vs oracle", e)
    assert e <= 1e-4


@pytest.mark.parametrize("update", ["svd", "rsvd"])
def test_compress_matches_oracle(update):
    X = naive_product(kron_sum_mpo(8, 4, 6, 0), kron_sum_mpo(8, 4, 6, 1))     # bond 16
    Xp = canonicalize_input(X)
    for chi in (5, 9, 16):
        R = compress(Xp, chi, 0.0, 1e-13, update, 2, 3)
        C = ttfit.tt_mpo_compress(X, chi, 0.0, update=update, oversample=2, seed=3, precision="fp64",
                                  sv_cutoff=1e-13)
        assert [c.shape[0] for c in C] == [r.shape[0] for r in R]
        e = _rel(C, R)
        print("compress", update, chi, e)
        assert e <= 1e-11


def test_naive_product_then_compress_on_the_device():
    """Alg. 1 end to end through the C ABI: the exact product, then compress
    without truncation, is A B."""
    A = kron_sum_mpo(8, 3, 7, 0)
    B = kron_sum_mpo(8, 3, 7, 1)
    N = ttfit.tt_mpo_naive_product(_dev(A), _dev(B))
    C = ttfit.tt_mpo_compress(N, 64, 0.0, precision="fp64", sv_cutoff=1e-13)
    e = _rel(C, naive_product(A, B))
    assert e <= 1e-12
    assert max(c.shape[3] for c in C) <= 9   # the exact rank of a sum of 9 Kronecker terms


def test_zipup_errors():
    A, B = mpo_pair("kron_L10_chi16", seed=0)
    with pytest.raises(ttfit.TTError):
        ttfit.tt_mpo_zipup(A, B[:-1], 16)
    with pytest.raises(ttfit.TTError):
        ttfit.tt_mpo_zipup(A, B, 0)
    A, B = mpo_pair("kron_L12_chi32", seed=0)
    with pytest.raises(ttfit.TTError):     # d d' chi above 1024 (chi_A chi_B = 1024 > 300)
        ttfit.tt_mpo_zipup(A, B, 300)


@pytest.mark.parametrize("update", ["svd", "rsvd"])
def test_fit_from_zipup_guess_matches_oracle(update):
    """The fit started from the zip-up guess follows the oracle's fit from the
    same guess, sweep by sweep (FP64)."""
    A, B = mpo_pair("kron_L10_chi16", seed=0)
    ref = FitOracle(A, B, 16, 1e-10, init="zipup", update=update, oversample=10, seed=7, conv_tol=0.0)
    ref.sweep(4, stop_on_converge=False)
    f = ttfit.tt_fit_create(A, B, 16, 1e-10, "site", init="zipup", update=update, oversample=10, seed=7,
                            precision="fp64", conv_tol=0.0, sv_cutoff=1e-13)
    try:
        for s in range(4):
            rep = f.sweep(1)
            want = ref.st.history[s].norm2
            assert abs(rep["norm2_C"] - want) <= 1e-10 * want
            assert f.bonds() == ref.st.history[s].bonds
    finally:
        f.destroy()


def test_edge_cases_one_and_two_sites():
    """Degenerate chains: one site (the product is the whole operator, no bond to truncate),
    two sites with chi_max = 1 (the rank-one truncation of one bond), against the oracle."""
    A = gaussian_mpo(1, 2, 3, 4, 0)
    B = gaussian_mpo(1, 2, 3, 4, 1)
    N = ttfit.tt_mpo_naive_product(_dev(A), _dev(B))
    R = naive_product(A, B)
    assert np.abs(N[0].cpu().numpy() - R[0]).max() <= 1e-14 * np.abs(R[0]).max()
    C = ttfit.tt_mpo_zipup(A, B, 4, 0.0, precision="fp64", sv_cutoff=1e-13)
    assert _rel(C, R) <= 1e-13
    A = gaussian_mpo(2, 2, 3, 5, 0)
    B = gaussian_mpo(2, 2, 2, 5, 1)
    Ap, Bp = canonicalize_input(A), canonicalize_input(B)
    for update in ("svd", "rsvd"):
        R = zipup_right_to_left(Ap, Bp, 1, 0.0, 1e-13, update, 0, 2)
        C = ttfit.tt_mpo_zipup(A, B, 1, 0.0, update=update, oversample=0, seed=2, precision="fp64",
                               sv_cutoff=1e-13)
        assert [c.shape[0] for c in C] == [1, 1]
        assert _rel(C, R) <= 1e-12
    X = naive_product(A, B)
    C = ttfit.tt_mpo_compress(X, 1, 0.0, precision="fp64", sv_cutoff=1e-13)
    R = compress(canonicalize_input(X), 1, 0.0, 1e-13)
    assert _rel(C, R) <= 1e-12


@pytest.mark.parametrize("gauge", ["site", "inverse"])
def test_zipup_guess_with_projection_follows_oracle(gauge):
    """The zip-up guess of the projected chains (both options together), both gauges."""
    A, B = mpo_pair("kron_L10_chi16", seed=0)
    ref = FitOracle(A, B, 16, 1e-10, gauge=gauge, init="zipup", update="rsvd", oversample=10, seed=7,
                    conv_tol=0.0, ab_rank=8)
    ref.sweep(3, stop_on_converge=False)
    f = ttfit.tt_fit_create(A, B, 16, 1e-10, gauge, init="zipup", update="rsvd", oversample=10, seed=7,
                            precision="fp64", conv_tol=0.0, sv_cutoff=1e-13, ab_rank=8)
    try:
        for s in range(3):
            rep = f.sweep(1)
            want = ref.st.history[s].norm2
            assert abs(rep["norm2_C"] - want) <= 1e-9 * want, (s, rep["norm2_C"], want)
    finally:
        f.destroy()
