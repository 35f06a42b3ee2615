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


def _host_desc(L, dout, din, bond, dtype=0, null_core=-1):
    """An MPO descriptor whose core pointers are never dereferenced by the checks below."""
    from paper_2606_23274_gb300 import ttfit
    keep = [(ct.c_int * L)(*dout), (ct.c_int * L)(*din), (ct.c_int * (L + 1))(*bond)]
    cores = (ct.c_void_p * L)(*[None if l == null_core else 0x1000 + 64 * l for l in range(L)])
    keep.append(cores)
    d = ttfit.tt_mpo_desc(L, keep[0], keep[1], keep[2], cores, dtype)
    return d, keep


def test_create_rejects_bad_arguments_before_any_device_call():
    """tt_fit_create's argument and shape checks (include/ttfit.h: argument errors return
    TT_ERR_INVALID_ARGUMENT, inconsistent legs or bonds TT_ERR_SHAPE_MISMATCH) run on the
    host before the first CUDA call, so they are exercised here without a GPU."""
    ttfit = _built_lib()
    lib = ttfit.load()
    INV, SHAPE = ttfit.TT_ERR_INVALID_ARGUMENT, ttfit.TT_ERR_SHAPE_MISMATCH
    L = 4
    A, ka = _host_desc(L, [2] * L, [2] * L, [1, 4, 4, 4, 1])
    B, kb = _host_desc(L, [2] * L, [3] * L, [1, 4, 4, 4, 1])

    def create(a=A, b=B, chi=8, tol=0.0, gauge=0, **opt):
        o = ttfit.tt_fit_options()
        o.struct_size = ct.sizeof(o)
        o.update, o.oversample, o.precision, o.sv_cutoff, o.conv_tol, o.prepare_inputs = 1, 10, 3, -1.0, -1.0, 1
        for k, v in opt.items():
            setattr(o, k, v)
        h = ct.c_void_p()
        st = lib.tt_fit_create(ct.byref(a), ct.byref(b), chi, ct.c_double(tol), gauge, ct.byref(o), ct.byref(h))
        assert not h.value  # nothing is handed out on failure
        return st

    lib.tt_fit_create.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_double, ct.c_int, ct.c_void_p,
                                  ct.c_void_p]
    # the problem: chi_max >= 1, tol >= 0 (not NaN), a known gauge
    assert create(chi=0) == INV
    assert create(tol=float("nan")) == INV
    assert create(gauge=2) == INV
    # options
    assert create(struct_size=8) == INV
    assert create(update=2) == INV
    assert create(precision=6) == INV and create(precision=-1) == INV
    assert create(oversample=-1) == INV
    assert create(init=4) == INV
    assert create(init=2) == INV                      # TT_INIT_GIVEN without init_C
    assert create(edge_extra=-1) == INV
    assert create(fast_factor=4) == INV
    assert create(ab_rank=-1) == INV
    assert create(ab_rank=2, prepare_inputs=0) == INV
    # shapes: C = A B contracts A's input legs with B's output legs (B's input legs only reach C)
    B3, kb3 = _host_desc(L, [3] * L, [2] * L, [1, 4, 4, 4, 1])
    assert create(b=B3) == SHAPE
    B5, kb5 = _host_desc(5, [2] * 5, [2] * 5, [1, 4, 4, 4, 4, 1])
    assert create(b=B5) == SHAPE                      # different lengths
    A1, ka1 = _host_desc(1, [2], [2], [1, 1])
    B1, kb1 = _host_desc(1, [2], [2], [1, 1])
    assert create(a=A1, b=B1) == INV                  # one site: no two-site window
    assert create(n_segments=3) == INV                # fewer than 2 sites per segment
    Abad, k1 = _host_desc(L, [2] * L, [2] * L, [2, 4, 4, 4, 1])
    assert create(a=Abad) == SHAPE                    # bond[0] != 1
    assert "bond[0]" in lib.tt_fit_last_error(None).decode()
    Adt, k2 = _host_desc(L, [2] * L, [2] * L, [1, 4, 4, 4, 1], dtype=7)
    assert create(a=Adt) == INV                       # unknown dtype
    Anull, k3 = _host_desc(L, [2] * L, [2] * L, [1, 4, 4, 4, 1], null_core=2)
    assert create(a=Anull) == INV
    assert "NULL core" in lib.tt_fit_last_error(None).decode()
    # every precision in the enum passes the option checks (BF16_SPLIT included); the shape check
    # that follows is what stops these
    for p in range(6):
        assert create(b=B3, precision=p) == SHAPE


def test_zipup_rejects_bad_options_before_any_device_call():
    """tt_mpo_zipup's option checks run on the host: BF16_SPLIT (not a zip-up precision), an unknown
    precision and a negative oversample are argument errors, as are chi_max < 1 and a missing C."""
    ttfit = _built_lib()
    lib = ttfit.load()
    INV = ttfit.TT_ERR_INVALID_ARGUMENT
    L = 4
    A, ka = _host_desc(L, [2] * L, [2] * L, [1, 4, 4, 4, 1])
    B, kb = _host_desc(L, [2] * L, [2] * L, [1, 4, 4, 4, 1])
    C, kc = _host_desc(L, [2] * L, [2] * L, [1, 4, 16, 4, 1])
    bonds = (ct.c_int * (L + 1))()
    lib.tt_mpo_zipup.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_double, ct.c_void_p, ct.c_void_p,
                                 ct.c_void_p]

    def zipup(chi=8, c=C, **opt):
        o = ttfit.tt_fit_options()
        o.struct_size = ct.sizeof(o)
        o.update, o.oversample, o.precision, o.sv_cutoff, o.prepare_inputs = 1, 10, 0, -1.0, 1
        for k, v in opt.items():
            setattr(o, k, v)
        return lib.tt_mpo_zipup(ct.byref(A), ct.byref(B), chi, ct.c_double(0.0), ct.byref(o),
                                ct.byref(c) if c is not None else None, bonds)

    assert zipup(precision=3) == INV
    assert zipup(precision=6) == INV
    assert zipup(oversample=-1) == INV
    assert zipup(chi=0) == INV
    assert zipup(c=None) == INV


def test_binding_builds_options_and_has_no_cpu_fallback():
    """The binding maps names to the header's enums (stream given, so no device is touched), and
    without a GPU a fit fails loudly instead of computing anywhere else."""
    ttfit = _built_lib()
    o, _ = ttfit._options(update="rsvd", precision="bf16_split", init="zipup", ab_rank=3, fast_factor=True,
                          n_segments=2, edge_extra=1, stream=0)
    assert (o.update, o.precision, o.init, o.ab_rank, o.fast_factor, o.n_segments, o.edge_extra) == \
        (1, 3, 3, 3, 1, 2, 1)
    assert ttfit.PRECISION == {"fp64": 0, "fp32": 1, "tf32": 2, "bf16_split": 3, "tf32x3": 4, "df32": 5}
    with pytest.raises(KeyError):
        ttfit._options(precision="fp16", stream=0)
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2606_23274_gb300.synth import gaussian_mpo
    A = gaussian_mpo(4, 2, 2, 0, 0)
    with pytest.raises(RuntimeError):    # torch finds no device for the inputs; nothing falls back
        ttfit.tt_fit_create(A, A, 4, 0.0)
