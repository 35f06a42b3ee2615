"""CPU checks of the boundary: the C ABI library builds, loads and exports every
function include/ttfit.h declares, and the ctypes structs match the C layout.
No compute call is made here (there is no GPU)."""
import ctypes as ct
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _built_lib():
    from paper_2606_23274_gb300 import build, ttfit
    if shutil.which(os.environ.get("NVCC", "nvcc")) is None and not os.path.exists(ttfit.LIB_PATH):
        pytest.skip("nvcc not available")
    build.build()
    return ttfit


def test_library_exports_every_header_function():
    ttfit = _built_lib()
    names = ttfit.header_functions()
    assert set(names) >= {"tt_fit_create", "tt_fit_sweep", "tt_fit_result", "tt_fit_destroy",
                          "tt_status_string", "tt_fit_last_error", "tt_fit_stage_times"}
    lib = ct.CDLL(ttfit.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", ttfit.LIB_PATH], capture_output=True, text=True).stdout
    for n in names:
        assert f" T {n}" in out, n


def test_status_strings_without_gpu():
    ttfit = _built_lib()
    lib = ttfit.load()
    assert lib.tt_status_string(0) == b"ok"
    assert lib.tt_status_string(2) == b"shape mismatch"
    # argument checks that return before any device call
    h = ct.c_void_p()
    assert lib.tt_fit_create(None, None, 4, 0.0, 0, None, ct.byref(h)) == ttfit.TT_ERR_INVALID_ARGUMENT
    assert lib.tt_fit_sweep(None, 1, None) == ttfit.TT_ERR_INVALID_ARGUMENT
    n = ct.c_int(-1)
    assert lib.tt_fit_jacobi_sweeps(None, ct.byref(n)) == ttfit.TT_ERR_INVALID_ARGUMENT
    cnt = ct.c_longlong(-1)
    assert lib.tt_fit_launch_count(None, ct.byref(cnt)) == ttfit.TT_ERR_INVALID_ARGUMENT
    # the block cache is empty in a process that made no fit: nothing to free, no device call
    assert ttfit.tt_device_cache_release(-1) == 0


def test_ctypes_structs_match_c_layout():
    ttfit = _built_lib()
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "ttfit.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(tt_mpo_desc), sizeof(tt_fit_options), sizeof(tt_sweep_report));
  printf("%zu %zu %zu %zu %zu\n", offsetof(tt_fit_options, seed), offsetof(tt_fit_options, init_C),
         offsetof(tt_fit_options, stream), offsetof(tt_fit_options, fault_inject), offsetof(tt_mpo_desc, dtype));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe], text=True).split()
    sizes = [int(x) for x in out]
    assert sizes[0] == ct.sizeof(ttfit.tt_mpo_desc)
    assert sizes[1] == ct.sizeof(ttfit.tt_fit_options)
    assert sizes[2] == ct.sizeof(ttfit.tt_sweep_report)
    O = ttfit.tt_fit_options
    assert sizes[3:7] == [O.seed.offset, O.init_C.offset, O.stream.offset, O.fault_inject.offset]
    assert sizes[7] == ttfit.tt_mpo_desc.dtype.offset


def test_partition_matches_oracle_without_gpu():
    """tt_partition (host-only) lays out the same segments as the oracle's
    Alg. 6 simulation, for many lengths, segment counts and edge extras."""
    ttfit = _built_lib()
    from oracle.parallel import partition
    lib = ttfit.load()
    lib.tt_partition.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]
    lib.tt_partition.restype = ct.c_int
    for L in range(4, 70, 3):
        for n in range(1, L // 2 + 1, max(1, L // 12)):
            for e in (0, 1, 3, 7):
                first = (ct.c_int * n)()
                last = (ct.c_int * n)()
                assert lib.tt_partition(L, n, e, first, last) == ttfit.TT_OK
                assert [(a + 1, b + 1) for a, b in zip(first, last)] == partition(L, n, e), (L, n, e)
    one = (ct.c_int * 4)()
    assert lib.tt_partition(7, 4, 0, one, one) == ttfit.TT_ERR_INVALID_ARGUMENT   # 7 sites < 2 x 4
