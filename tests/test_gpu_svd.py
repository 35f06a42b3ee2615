"""The standalone truncated SVD primitive (Sec. 2.3.4 factorisation) through the
C ABI, against LAPACK's SVD and the oracle's truncation rule."""
import numpy as np
import pytest

from oracle.fit import keep_rank

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_23274_gb300 import ttfit  # noqa: E402


@pytest.mark.parametrize("m,n", [(40, 40), (64, 24), (24, 64), (1, 7), (130, 200), (256, 33)])
def test_truncated_svd_matches_lapack(m, n):
    rng = np.random.default_rng(m * 1000 + n)
    M = rng.standard_normal((m, n)) * (0.9 ** np.arange(n))[None, :]
    U, S, Vt, k = ttfit.tt_svd_truncated(M, chi_max=10 ** 6, tau_rel=0.0)
    U, S, Vt = U.cpu().numpy(), S.cpu().numpy(), Vt.cpu().numpy()
    S_ref = np.linalg.svd(M, compute_uv=False)
    assert np.allclose(S, S_ref, rtol=1e-11, atol=1e-13 * S_ref[0])
    assert np.linalg.norm(U * S[None, :] @ Vt - M) <= 1e-12 * np.linalg.norm(M)
    r = min(m, n)
    assert np.allclose(U.T @ U, np.eye(r), atol=1e-12)
    assert np.allclose(Vt @ Vt.T, np.eye(r), atol=1e-12)
    i = np.argmax(np.abs(U), axis=0)
    assert np.all(U[i, np.arange(r)] > 0)                 # sign convention
    assert k == keep_rank(S_ref, float(np.linalg.norm(M)), 0.0, 1, 10 ** 6, 1e-13)


def test_truncation_rule_and_errors():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((50, 30)) * (0.6 ** np.arange(30))[None, :]
    S_ref = np.linalg.svd(M, compute_uv=False)
    nM = float(np.linalg.norm(M))
    for chi, tau in ((5, 0.0), (100, 1e-3), (100, 1e-1), (3, 1e-6)):
        _, _, _, k = ttfit.tt_svd_truncated(M, chi_max=chi, tau_rel=tau)
        assert k == keep_rank(S_ref, nM, tau, 1, chi, 1e-13)
    with pytest.raises(ttfit.TTError) as e:
        ttfit.tt_svd_truncated(M, chi_max=0)
    assert e.value.code == ttfit.TT_ERR_INVALID_ARGUMENT
    bad = M.copy()
    bad[3, 4] = np.nan
    with pytest.raises(ttfit.TTError) as e:
        ttfit.tt_svd_truncated(bad, chi_max=5)
    assert e.value.code == ttfit.TT_ERR_NUMERICAL
