"""The allocation-free truncated SVD entry point, for callers that cannot
allocate device memory (its scratch is a fixed device array inside the
library). Collected last so that a first failure here leaves every other test
already run; it must pass alone in a fresh process as well as after them."""
import ctypes as ct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_23274_gb300 import ttfit  # noqa: E402


def _noalloc(M, chi_max, tau_rel=0.0):
    lib = ttfit.load()
    fn = lib.tt_svd_truncated_noalloc
    fn.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_double, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                   ct.POINTER(ct.c_int), ct.c_void_p]
    fn.restype = ct.c_int
    M = torch.as_tensor(M, dtype=torch.float64).cuda().contiguous()
    m, n = M.shape
    r = min(m, n)
    U = torch.empty((m, r), dtype=torch.float64, device="cuda")
    S = torch.empty((r,), dtype=torch.float64, device="cuda")
    Vt = torch.empty((r, n), dtype=torch.float64, device="cuda")
    k = ct.c_int(-1)
    code = fn(M.data_ptr(), m, n, int(chi_max), float(tau_rel), U.data_ptr(), S.data_ptr(), Vt.data_ptr(),
              ct.byref(k), ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code, U.cpu().numpy(), S.cpu().numpy(), Vt.cpu().numpy(), k.value


def test_noalloc_matches_allocating_entry_point_twice():
    rng = np.random.default_rng(17)
    inputs = [rng.standard_normal((96, 40)) * (0.85 ** np.arange(40))[None, :],
              rng.standard_normal((30, 120)) * (0.7 ** np.arange(120))[None, :]]
    for M, chi, tau in zip(inputs, (12, 20), (0.0, 1e-4)):       # two calls in a row
        code, U, S, Vt, k = _noalloc(M, chi, tau)
        assert code == ttfit.TT_OK
        U0, S0, Vt0, k0 = ttfit.tt_svd_truncated(M, chi, tau)
        U0, S0, Vt0 = U0.cpu().numpy(), S0.cpu().numpy(), Vt0.cpu().numpy()
        assert k == k0
        assert np.allclose(S, S0, rtol=1e-12, atol=1e-14 * S0[0])
        assert np.allclose(U, U0, atol=1e-10) and np.allclose(Vt, Vt0, atol=1e-10)
        assert np.linalg.norm(U * S[None, :] @ Vt - M) <= 1e-12 * np.linalg.norm(M)


def test_noalloc_call_allocates_no_device_memory():
    """After a first call (which commits the library's fixed scratch on this
    device), a call leaves the device's free memory unchanged: nothing is
    allocated for it, by the library or by anything it calls."""
    lib = ttfit.load()
    fn = lib.tt_svd_truncated_noalloc
    fn.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_double, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                   ct.POINTER(ct.c_int), ct.c_void_p]
    fn.restype = ct.c_int
    rng = np.random.default_rng(5)
    m, n = 128, 64
    M = torch.as_tensor(rng.standard_normal((m, n)) * (0.8 ** np.arange(n))[None, :], device="cuda")
    U = torch.empty((m, n), dtype=torch.float64, device="cuda")
    S = torch.empty((n,), dtype=torch.float64, device="cuda")
    Vt = torch.empty((n, n), dtype=torch.float64, device="cuda")
    k = ct.c_int(-1)
    st = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (M.data_ptr(), m, n, 16, 0.0, U.data_ptr(), S.data_ptr(), Vt.data_ptr(), ct.byref(k), st)
    assert fn(*args) == ttfit.TT_OK                      # warm-up: commits the scratch
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert fn(*args) == ttfit.TT_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert k.value == 16


def test_noalloc_rejects_sizes_beyond_its_scratch():
    M = np.ones((600, 600))
    code, *_ = _noalloc(M, 10)
    assert code == ttfit.TT_ERR_INVALID_ARGUMENT
