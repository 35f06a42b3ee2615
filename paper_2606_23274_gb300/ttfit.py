"""Python binding of the C ABI in include/ttfit.h (argument marshalling only).

Every step of a sweep runs in libttfit.so's CUDA kernels; this module only
builds the descriptor structs from torch tensors, passes device pointers and
the current CUDA stream, and checks return codes. Importing it on a machine
without the built library raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libttfit.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "ttfit.h")

TT_OK, TT_ERR_INVALID_ARGUMENT, TT_ERR_SHAPE_MISMATCH, TT_ERR_OUT_OF_MEMORY = 0, 1, 2, 3
TT_ERR_CUDA, TT_ERR_NUMERICAL, TT_ERR_TIMEOUT, TT_ERR_STATE = 4, 5, 6, 7
GAUGE = {"site": 0, "inverse": 1}
UPDATE = {"svd": 0, "rsvd": 1}
PRECISION = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16_split": 3, "tf32x3": 4, "df32": 5}
INIT = {"random": 0, "copy_b": 1, "given": 2, "zipup": 3}
TT_FAULT_ALLOC_FAIL, TT_FAULT_NAN_INPUT, TT_FAULT_SVD_NOCONV = 0x1, 0x2, 0x4
DTYPE_F64, DTYPE_F32 = 0, 1


class tt_mpo_desc(ct.Structure):
    _fields_ = [("L", ct.c_int), ("d_out", ct.POINTER(ct.c_int)), ("d_in", ct.POINTER(ct.c_int)),
                ("bond", ct.POINTER(ct.c_int)), ("cores", ct.POINTER(ct.c_void_p)), ("dtype", ct.c_int)]


class tt_fit_options(ct.Structure):
    _fields_ = [("struct_size", ct.c_size_t), ("update", ct.c_int), ("oversample", ct.c_int),
                ("seed", ct.c_uint64), ("precision", ct.c_int), ("init", ct.c_int),
                ("init_C", ct.POINTER(tt_mpo_desc)), ("sv_cutoff", ct.c_double), ("conv_tol", ct.c_double),
                ("stream", ct.c_void_p), ("prepare_inputs", ct.c_int), ("fault_inject", ct.c_uint32),
                ("fast_factor", ct.c_int), ("n_segments", ct.c_int), ("edge_extra", ct.c_int),
                ("ab_rank", ct.c_int)]


class tt_sweep_report(ct.Structure):
    _fields_ = [("sweeps_done", ct.c_int), ("converged", ct.c_int), ("delta", ct.c_double),
                ("norm2_C", ct.c_double), ("max_discarded", ct.c_double), ("seconds", ct.c_double)]


class TTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


_lib = None


def load():
    """Load libttfit.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first (no CPU fallback)")
        lib = ct.CDLL(LIB_PATH)
        lib.tt_fit_create.argtypes = [ct.POINTER(tt_mpo_desc), ct.POINTER(tt_mpo_desc), ct.c_int, ct.c_double,
                                      ct.c_int, ct.POINTER(tt_fit_options), ct.POINTER(ct.c_void_p)]
        lib.tt_fit_create.restype = ct.c_int
        lib.tt_fit_sweep.argtypes = [ct.c_void_p, ct.c_int, ct.POINTER(tt_sweep_report)]
        lib.tt_fit_merge.argtypes = [ct.c_void_p, ct.POINTER(tt_sweep_report)]
        lib.tt_fit_merge.restype = ct.c_int
        lib.tt_fit_sweep.restype = ct.c_int
        lib.tt_fit_result.argtypes = [ct.c_void_p, ct.POINTER(tt_mpo_desc), ct.POINTER(ct.c_double)]
        lib.tt_fit_result.restype = ct.c_int
        lib.tt_fit_destroy.argtypes = [ct.c_void_p]
        lib.tt_fit_destroy.restype = None
        lib.tt_status_string.argtypes = [ct.c_int]
        lib.tt_status_string.restype = ct.c_char_p
        lib.tt_fit_last_error.argtypes = [ct.c_void_p]
        lib.tt_fit_last_error.restype = ct.c_char_p
        lib.tt_svd_truncated.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_double, ct.c_void_p,
                                         ct.c_void_p, ct.c_void_p, ct.POINTER(ct.c_int), ct.c_void_p]
        lib.tt_svd_truncated.restype = ct.c_int
        lib.tt_fit_exec_flops.argtypes = [ct.c_void_p, ct.POINTER(ct.c_double)]
        lib.tt_fit_exec_flops.restype = ct.c_int
        lib.tt_fit_set_precision.argtypes = [ct.c_void_p, ct.c_int, ct.c_int]
        lib.tt_fit_set_precision.restype = ct.c_int
        lib.tt_fit_stage_times.argtypes = [ct.c_void_p, ct.POINTER(ct.c_double)]
        lib.tt_fit_stage_times.restype = ct.c_int
        lib.tt_fit_launch_count.argtypes = [ct.c_void_p, ct.POINTER(ct.c_longlong)]
        lib.tt_fit_launch_count.restype = ct.c_int
        lib.tt_fit_create_batched.argtypes = [ct.c_int, ct.POINTER(tt_mpo_desc), ct.POINTER(tt_mpo_desc),
                                              ct.POINTER(ct.c_int), ct.c_double, ct.c_int, ct.c_int,
                                              ct.POINTER(tt_fit_options), ct.POINTER(ct.c_void_p)]
        lib.tt_fit_create_batched.restype = ct.c_int
        lib.tt_fit_sweep_batched.argtypes = [ct.c_int, ct.POINTER(ct.c_void_p), ct.c_int,
                                             ct.POINTER(tt_sweep_report)]
        lib.tt_fit_sweep_batched.restype = ct.c_int
        lib.tt_mpo_grad.argtypes = [ct.POINTER(tt_mpo_desc), ct.POINTER(tt_mpo_desc), ct.POINTER(tt_mpo_desc),
                                    ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.POINTER(tt_mpo_desc),
                                    ct.POINTER(tt_mpo_desc), ct.POINTER(ct.c_double)]
        lib.tt_mpo_grad.restype = ct.c_int
        lib.tt_fit_jacobi_sweeps.argtypes = [ct.c_void_p, ct.POINTER(ct.c_int)]
        lib.tt_fit_jacobi_sweeps.restype = ct.c_int
        lib.tt_mpo_naive_product.argtypes = [ct.POINTER(tt_mpo_desc), ct.POINTER(tt_mpo_desc),
                                             ct.POINTER(tt_mpo_desc), ct.c_void_p]
        lib.tt_mpo_naive_product.restype = ct.c_int
        for name in ("tt_mpo_zipup",):
            getattr(lib, name).argtypes = [ct.POINTER(tt_mpo_desc), ct.POINTER(tt_mpo_desc), ct.c_int, ct.c_double,
                                           ct.POINTER(tt_fit_options), ct.POINTER(tt_mpo_desc),
                                           ct.POINTER(ct.c_int)]
            getattr(lib, name).restype = ct.c_int
        lib.tt_mpo_compress.argtypes = [ct.POINTER(tt_mpo_desc), ct.c_int, ct.c_double, ct.POINTER(tt_fit_options),
                                        ct.POINTER(tt_mpo_desc), ct.POINTER(ct.c_int)]
        lib.tt_mpo_compress.restype = ct.c_int
        lib.tt_device_cache_release.argtypes = [ct.c_int]
        lib.tt_device_cache_release.restype = ct.c_size_t
        _lib = lib
    return _lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/ttfit.h."""
    import re
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:tt_status|void|const char\*)\s+(tt_\w+)\s*\(", txt, re.M)))


class _Desc:
    """Keeps the ctypes arrays of one tt_mpo_desc alive."""

    def __init__(self, cores, dtype_code=None):
        import torch
        L = len(cores)
        shapes = [tuple(c.shape) for c in cores]
        self.d_out = (ct.c_int * L)(*[s[1] for s in shapes])
        self.d_in = (ct.c_int * L)(*[s[2] for s in shapes])
        self.bond = (ct.c_int * (L + 1))(*([s[0] for s in shapes] + [shapes[-1][3]]))
        self.tensors = [c.contiguous() for c in cores]
        if dtype_code is None:
            dtype_code = DTYPE_F64 if self.tensors[0].dtype == torch.float64 else DTYPE_F32
        self.ptrs = (ct.c_void_p * L)(*[t.data_ptr() for t in self.tensors])
        self.desc = tt_mpo_desc(L, self.d_out, self.d_in, self.bond, self.ptrs, dtype_code)


def _as_device(cores, device):
    import torch
    out = []
    for c in cores:
        if isinstance(c, np.ndarray):
            c = torch.from_numpy(np.ascontiguousarray(c))
        out.append(c.to(device=device))
    return out


def _check(code, h=None, what=""):
    if code != TT_OK:
        lib = load()
        msg = lib.tt_status_string(code).decode()
        detail = lib.tt_fit_last_error(h if (h is not None and h.value) else None).decode()
        if detail and detail != "NULL handle":
            msg += ": " + detail
        raise TTError(code, f"{what}: {msg}")


def _options(update="svd", oversample=10, seed=0, precision="fp64", init="random", init_C=None, sv_cutoff=-1.0,
             conv_tol=-1.0, stream=None, prepare_inputs=True, fault_inject=0, fast_factor=False, n_segments=1,
             edge_extra=0, ab_rank=0, device="cuda"):
    """tt_fit_options from keyword arguments; returns (options, keep-alive objects)."""
    import torch
    o = tt_fit_options()
    o.struct_size = ct.sizeof(tt_fit_options)
    o.update = UPDATE[update] if isinstance(update, str) else int(update)
    o.oversample = int(oversample)
    o.seed = int(seed)
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.init = INIT[init] if isinstance(init, str) else int(init)
    dC = None
    if init_C is not None:
        dC = _Desc(_as_device(init_C, device))
        o.init_C = ct.pointer(dC.desc)
    o.sv_cutoff = float(sv_cutoff)
    o.conv_tol = float(conv_tol)
    if stream is None:
        stream = torch.cuda.current_stream()
    o.stream = ct.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    o.prepare_inputs = 1 if prepare_inputs else 0
    o.fault_inject = int(fault_inject)
    o.fast_factor = int(fast_factor)
    o.n_segments = int(n_segments)
    o.edge_extra = int(edge_extra)
    o.ab_rank = int(ab_rank)
    return o, dC


def tt_fit_create(A: Sequence, B: Sequence, chi_max: int, tol: float, gauge="site", *, device="cuda", **kw):
    """Create a fit handle (see tt_fit_create in include/ttfit.h). A, B: lists of
    (chi_l, d, d', chi_r) tensors (torch CUDA tensors, or host arrays that are copied).
    Keywords: update, oversample, seed, precision, init, init_C, sv_cutoff, conv_tol,
    stream, prepare_inputs, fault_inject, fast_factor, n_segments, edge_extra, ab_rank."""
    lib = load()
    dA = _Desc(_as_device(A, device))
    dB = _Desc(_as_device(B, device))
    o, _keep = _options(device=device, **kw)
    h = ct.c_void_p()
    g = GAUGE[gauge] if isinstance(gauge, str) else int(gauge)
    code = lib.tt_fit_create(ct.byref(dA.desc), ct.byref(dB.desc), int(chi_max), float(tol), g, ct.byref(o),
                             ct.byref(h))
    _check(code, None, "tt_fit_create")
    return Fit(h, device, len(A))


def tt_fit_create_batched(pairs: Sequence, chi_max: Sequence[int], tol: float, gauge="inverse", *, n_segments=1,
                          device="cuda", **kw):
    """tt_fit_create_batched: one handle per (A, B) pair, each with its own stream."""
    lib = load()
    n = len(pairs)
    dAs = [_Desc(_as_device(A, device)) for A, _ in pairs]
    dBs = [_Desc(_as_device(B, device)) for _, B in pairs]
    arrA = (tt_mpo_desc * n)(*[d.desc for d in dAs])
    arrB = (tt_mpo_desc * n)(*[d.desc for d in dBs])
    chis = (ct.c_int * n)(*[int(c) for c in chi_max])
    o, _keep = _options(device=device, **kw)
    outs = (ct.c_void_p * n)()
    g = GAUGE[gauge] if isinstance(gauge, str) else int(gauge)
    code = lib.tt_fit_create_batched(n, arrA, arrB, chis, float(tol), g, int(n_segments), ct.byref(o), outs)
    _check(code, None, "tt_fit_create_batched")
    return [Fit(ct.c_void_p(outs[i]), device, len(pairs[i][0])) for i in range(n)]


def tt_fit_sweep_batched(fits: Sequence["Fit"], n_sweeps: int) -> list[dict]:
    """tt_fit_sweep_batched over the handles; returns one report per handle."""
    n = len(fits)
    reps = (tt_sweep_report * n)()
    hs = (ct.c_void_p * n)(*[f.h.value for f in fits])
    code = load().tt_fit_sweep_batched(n, hs, int(n_sweeps), reps)
    if code != TT_OK:  # name the first failing handle and its own message
        for i, f in enumerate(fits):
            msg = load().tt_fit_last_error(f.h).decode()
            if msg:
                raise TTError(code, f"tt_fit_sweep_batched: handle {i}: {msg}")
    _check(code, None, "tt_fit_sweep_batched")
    return [{k: getattr(r, k) for k, _ in tt_sweep_report._fields_} for r in reps]


GRAD_TARGET = {"residual": 0, "inner": 1}


def tt_mpo_grad(A, B, X, target="residual", precision="fp32", checkpoint_every=0, stream=None, device="cuda"):
    """Value and gradients of f1 = ||X - AB||^2 (target "residual") or f2 = <X, AB>
    ("inner") with respect to every core of A and B, X fixed (tt_mpo_grad in
    include/ttfit.h). Returns (value, [dA_l], [dB_l]) with the gradients as device
    tensors of the cores' dtype."""
    import torch
    lib = load()
    Ad, Bd, Xd = (_as_device(M, device) for M in (A, B, X))
    dA, dB, dX = _Desc(Ad), _Desc(Bd), _Desc(Xd)
    gA = [torch.empty_like(c) for c in dA.tensors]
    gB = [torch.empty_like(c) for c in dB.tensors]
    dgA, dgB = _Desc(gA), _Desc(gB)
    if stream is None:
        stream = torch.cuda.current_stream()
    v = ct.c_double(0.0)
    code = lib.tt_mpo_grad(ct.byref(dA.desc), ct.byref(dB.desc), ct.byref(dX.desc), GRAD_TARGET[target],
                           PRECISION[precision], int(checkpoint_every),
                           ct.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)),
                           ct.byref(dgA.desc), ct.byref(dgB.desc), ct.byref(v))
    _check(code, None, "tt_mpo_grad")
    return v.value, gA, gB


def _objective_function():
    import torch

    class MPOObjective(torch.autograd.Function):
        """f1 or f2 as a differentiable function of the cores of A and B (X fixed).
        The library returns the value and every gradient from one call; backward
        scales the saved gradients by the incoming one."""

        @staticmethod
        def forward(ctx, target, X, precision, checkpoint_every, nA, *cores):
            A, B = list(cores[:nA]), list(cores[nA:])
            v, gA, gB = tt_mpo_grad(A, B, X, target, precision, checkpoint_every, device=cores[0].device)
            ctx.save_for_backward(*gA, *gB)
            return torch.tensor(v, dtype=cores[0].dtype, device=cores[0].device)

        @staticmethod
        def backward(ctx, gout):
            return (None, None, None, None, None) + tuple(gout * g for g in ctx.saved_tensors)

    return MPOObjective


_MPOObjective = None


def mpo_objective(A, B, X, target="residual", precision="fp32", checkpoint_every=0):
    """Differentiable f1 = ||X - AB||^2 or f2 = <X, AB> of the torch CUDA tensors
    A (cores), B (cores); X is a constant MPO."""
    global _MPOObjective
    if _MPOObjective is None:
        _MPOObjective = _objective_function()
    return _MPOObjective.apply(target, X, precision, checkpoint_every, len(A), *A, *B)


def tt_svd_truncated(M, chi_max: int, tau_rel: float = 0.0, stream=None):
    """Truncated SVD of a device (or host) FP64 matrix through the C ABI:
    returns (U, S, Vt, k) with the thin factors as device tensors."""
    import torch
    lib = load()
    M = torch.as_tensor(M, dtype=torch.float64).cuda().contiguous()
    m, n = M.shape
    r = min(m, n)
    U = torch.empty((m, r), dtype=torch.float64, device=M.device)
    S = torch.empty((r,), dtype=torch.float64, device=M.device)
    Vt = torch.empty((r, n), dtype=torch.float64, device=M.device)
    k = ct.c_int(0)
    if stream is None:
        stream = torch.cuda.current_stream()
    code = lib.tt_svd_truncated(M.data_ptr(), m, n, int(chi_max), float(tau_rel), U.data_ptr(), S.data_ptr(),
                                Vt.data_ptr(), ct.byref(k), ct.c_void_p(stream.cuda_stream))
    _check(code, None, "tt_svd_truncated")
    return U, S, Vt, k.value


def tt_mpo_naive_product(A, B, stream=None, device="cuda"):
    """Exact per-site product C_l = A_l x B_l (Alg. 1's contraction step,
    tt_mpo_naive_product); returns the cores of C (bond chi_A chi_B) as device
    tensors of the inputs' dtype."""
    import torch
    lib = load()
    Ad, Bd = _as_device(A, device), _as_device(B, device)
    dA, dB = _Desc(Ad), _Desc(Bd)
    C = [torch.empty((a.shape[0] * b.shape[0], a.shape[1], b.shape[2], a.shape[3] * b.shape[3]), dtype=a.dtype,
                     device=a.device) for a, b in zip(dA.tensors, dB.tensors)]
    dC = _Desc(C)
    if stream is None:
        stream = torch.cuda.current_stream()
    code = lib.tt_mpo_naive_product(ct.byref(dA.desc), ct.byref(dB.desc), ct.byref(dC.desc),
                                    ct.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)))
    _check(code, None, "tt_mpo_naive_product")
    return C


def _zipup_call(name, X, Y, chi_max, tol, dtype, device, kw):
    import torch
    lib = load()
    Xd = _as_device(X, device)
    dX = _Desc(Xd)
    dY = _Desc(_as_device(Y, device)) if Y is not None else None
    L = len(Xd)
    dout = [x.shape[1] for x in Xd]
    din = [y.shape[2] for y in (dY.tensors if dY else Xd)]
    if len(din) != L:  # the library reports the mismatch
        din = dout
    cap = [1] * (L + 1)
    right = 1
    for l in range(L - 1, 0, -1):
        right *= dout[l] * din[l]
        ab = Xd[l].shape[0] * (dY.tensors[l].shape[0] if dY and l < len(dY.tensors) else 1)
        cap[l] = int(min(chi_max, ab, right))
    dt = dtype or Xd[0].dtype
    C = [torch.empty((cap[l], dout[l], din[l], cap[l + 1]), dtype=dt, device=Xd[0].device) for l in range(L)]
    dC = _Desc(C)
    o, _keep = _options(device=device, **kw)
    bonds = (ct.c_int * (L + 1))()
    if dY is not None:
        code = lib.tt_mpo_zipup(ct.byref(dX.desc), ct.byref(dY.desc), int(chi_max), float(tol), ct.byref(o),
                                ct.byref(dC.desc), bonds)
    else:
        code = lib.tt_mpo_compress(ct.byref(dX.desc), int(chi_max), float(tol), ct.byref(o), ct.byref(dC.desc), bonds)
    _check(code, None, name)
    b = list(bonds)
    return [C[l].reshape(-1)[: b[l] * dout[l] * din[l] * b[l + 1]].reshape(b[l], dout[l], din[l], b[l + 1])
            for l in range(L)]


def tt_mpo_zipup(A, B, chi_max: int, tol: float = 0.0, *, dtype=None, device="cuda", **kw):
    """Zip-up contraction C ~ A B (Alg. 2, tt_mpo_zipup). Keywords as for
    tt_fit_create (update, oversample, seed, precision, sv_cutoff, stream,
    prepare_inputs); returns the cores of C as device tensors (dtype: that of A
    unless given)."""
    return _zipup_call("tt_mpo_zipup", A, B, chi_max, tol, dtype, device, kw)


def tt_mpo_compress(X, chi_max: int, tol: float = 0.0, *, dtype=None, device="cuda", **kw):
    """compress() of Alg. 1 (tt_mpo_compress): truncated SVD sweep of X."""
    return _zipup_call("tt_mpo_compress", X, None, chi_max, tol, dtype, device, kw)


def tt_device_cache_release(device: int = -1) -> int:
    """Frees the device blocks cached for reuse by later fits (all devices if
    device < 0); returns the bytes freed (tt_device_cache_release)."""
    return int(load().tt_device_cache_release(int(device)))


def tt_fit_sweep(fit: "Fit", n_sweeps: int):
    return fit.sweep(n_sweeps)


def tt_fit_result(fit: "Fit", dtype=None):
    return fit.result(dtype)


def tt_fit_destroy(fit: "Fit"):
    fit.destroy()


class Fit:
    """Owner of a tt_fit handle."""

    def __init__(self, handle: ct.c_void_p, device, L: int):
        self.h = handle
        self.device = device
        self.L = L

    def sweep(self, n_sweeps: int = 1) -> dict:
        rep = tt_sweep_report()
        _check(load().tt_fit_sweep(self.h, int(n_sweeps), ct.byref(rep)), self.h, "tt_fit_sweep")
        return {k: getattr(rep, k) for k, _ in tt_sweep_report._fields_}

    def merge(self) -> dict:
        """tt_fit_merge: joins the segments of a site-gauge segment-parallel fit."""
        rep = tt_sweep_report()
        _check(load().tt_fit_merge(self.h, ct.byref(rep)), self.h, "tt_fit_merge")
        return {k: getattr(rep, k) for k, _ in tt_sweep_report._fields_}

    def bonds(self) -> list[int]:
        L = self.L
        d_out = (ct.c_int * L)()
        d_in = (ct.c_int * L)()
        bond = (ct.c_int * (L + 1))()
        desc = tt_mpo_desc(L, d_out, d_in, bond, None, DTYPE_F64)
        _check(load().tt_fit_result(self.h, ct.byref(desc), None), self.h, "tt_fit_result")
        self._dims = (list(d_out), list(d_in), list(bond))
        return list(bond)

    def result(self, dtype=None):
        """C as a list of device tensors (chi_l, d, d', chi_r)."""
        import torch
        dtype = dtype or torch.float64
        bond = self.bonds()
        d_out, d_in, _ = self._dims
        L = len(d_out)
        cores = [torch.empty((bond[l], d_out[l], d_in[l], bond[l + 1]), dtype=dtype, device=self.device)
                 for l in range(L)]
        ptrs = (ct.c_void_p * L)(*[c.data_ptr() for c in cores])
        desc = tt_mpo_desc(L, (ct.c_int * L)(*d_out), (ct.c_int * L)(*d_in), (ct.c_int * (L + 1))(*bond), ptrs,
                           DTYPE_F64 if dtype == torch.float64 else DTYPE_F32)
        _check(load().tt_fit_result(self.h, ct.byref(desc), None), self.h, "tt_fit_result")
        torch.cuda.current_stream().synchronize()
        return cores

    def lambdas(self) -> list[np.ndarray]:
        bond = self.bonds()
        n = sum(bond[1:-1])
        buf = (ct.c_double * max(n, 1))()
        d_out, d_in, _ = self._dims
        L = len(d_out)
        desc = tt_mpo_desc(L, (ct.c_int * L)(*d_out), (ct.c_int * L)(*d_in), (ct.c_int * (L + 1))(*bond), None,
                           DTYPE_F64)
        _check(load().tt_fit_result(self.h, ct.byref(desc), buf), self.h, "tt_fit_result")
        out, off = [], 0
        for b in bond[1:-1]:
            out.append(np.array(buf[off:off + b]))
            off += b
        return out

    def set_precision(self, precision, fast_factor=False):
        """Switch the contraction precision for the following sweeps (see include/ttfit.h)."""
        prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
        _check(load().tt_fit_set_precision(self.h, prec, int(fast_factor)), self.h, "tt_fit_set_precision")

    def stage_times(self) -> dict:
        v = (ct.c_double * 7)()
        _check(load().tt_fit_stage_times(self.h, v), self.h, "tt_fit_stage_times")
        keys = ["halves_ms", "join_ms", "env_finish_ms", "factorize_ms", "gauge_ms", "contraction_flops",
                "launches"]
        return dict(zip(keys, list(v)))

    def exec_flops(self) -> dict:
        """The last sweep's contractions as issued: tensor-core MMA flops (padding and split
        passes included) and CUDA-core flops."""
        v = (ct.c_double * 2)()
        _check(load().tt_fit_exec_flops(self.h, v), self.h, "tt_fit_exec_flops")
        return {"tensor_core": v[0], "cuda_core": v[1]}

    def launch_count(self) -> int:
        """Kernel launches this fit has issued since creation (tt_fit_launch_count)."""
        n = ct.c_longlong(0)
        _check(load().tt_fit_launch_count(self.h, ct.byref(n)), self.h, "tt_fit_launch_count")
        return int(n.value)

    def jacobi_sweeps(self) -> int:
        """Most Jacobi sweeps one factorisation has needed (tt_fit_jacobi_sweeps)."""
        n = ct.c_int(0)
        _check(load().tt_fit_jacobi_sweeps(self.h, ct.byref(n)), self.h, "tt_fit_jacobi_sweeps")
        return n.value
    def destroy(self):
        if self.h is not None and self.h.value:
            load().tt_fit_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
