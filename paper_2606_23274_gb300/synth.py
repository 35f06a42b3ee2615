"""Seeded synthetic MPO workloads.

This module only draws random numbers and lays them out as MPO cores; it holds
none of the fit's arithmetic, so both the CUDA path and the FP64 oracle take
their inputs from here.

An MPO of length L is a list of cores ``X[l]`` of shape
``(chi[l], d_out[l], d_in[l], chi[l+1])`` with ``chi[0] = chi[L] = 1``
(Sec. 2, the MPO definition). All arrays are float64, C-contiguous.

Workloads (the synthetic stand-ins for the paper's random tensor trains):

* ``gaussian_mpo``: every core entry i.i.d. N(0,1) * scale with uniform inner
  bond chi.
* ``kron_sum_mpo``: ``A = sum_k w_k (x)_l a_{k,l}`` with ``w_k = decay**k`` and
  ``a_{k,l}`` i.i.d. 2x2 N(0,1) factors scaled by ``factor_scale``; written as a
  diagonal-bond MPO of bond K (exact: the bond trimming to the true rank
  ``min(K, d^2l, d^2(L-l))`` happens in each implementation's canonicalisation).
* ``uniform_mpo``: entries uniform in [alpha, 1], then each core divided by its
  Frobenius norm (Sec. 5.1's random tensor trains).
"""
from __future__ import annotations

import numpy as np

__all__ = ["gaussian_mpo", "kron_sum_mpo", "uniform_mpo", "mpo_pair", "WORKLOADS"]


def _rng(seed: int, which: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(which)])


def gaussian_mpo(L: int, d: int, chi: int, seed: int, which: int = 0, scale: float | None = None):
    """Cores i.i.d. N(0,1)*scale, bonds [1, chi, ..., chi, 1]; default scale 1/sqrt(d*chi)."""
    if scale is None:
        scale = 1.0 / np.sqrt(d * chi)
    rng = _rng(seed, which)
    bonds = [1] + [chi] * (L - 1) + [1]
    return [rng.standard_normal((bonds[l], d, d, bonds[l + 1])) * scale for l in range(L)]


def kron_sum_mpo(L: int, K: int, seed: int, which: int = 0, decay: float = 0.8,
                 factor_scale: float = 0.5, d: int = 2):
    """Diagonal-bond MPO of ``sum_{k<K} decay**k * kron_l a_{k,l}``.

    ``factor_scale`` multiplies every d x d factor (0.5 makes E||a||_F^2 = 1 for
    d = 2, so the operator norm does not grow like 2^L; it is a global scale the
    fit is equivariant to).
    """
    rng = _rng(seed, which)
    a = rng.standard_normal((L, K, d, d)) * factor_scale
    w = decay ** np.arange(K, dtype=np.float64)
    cores = []
    for l in range(L):
        chl = 1 if l == 0 else K
        chr_ = 1 if l == L - 1 else K
        X = np.zeros((chl, d, d, chr_))
        for k in range(K):
            il = 0 if l == 0 else k
            ir = 0 if l == L - 1 else k
            f = a[l, k] * (w[k] if l == 0 else 1.0)
            X[il, :, :, ir] += f
        cores.append(X)
    return cores


def uniform_mpo(L: int, d: int, chi: int, seed: int, which: int = 0, alpha: float = -0.5):
    """Entries uniform in [alpha, 1]; each core then divided by its Frobenius norm."""
    rng = _rng(seed, which)
    bonds = [1] + [chi] * (L - 1) + [1]
    cores = []
    for l in range(L):
        X = rng.uniform(alpha, 1.0, size=(bonds[l], d, d, bonds[l + 1]))
        cores.append(X / np.linalg.norm(X))
    return cores


def mpo_pair(workload: str, seed: int = 0, **kw):
    """(A, B) for a named workload; A from stream 0, B from stream 1 of ``seed``."""
    spec = dict(WORKLOADS[workload])
    spec.update(kw)
    kind = spec.pop("kind")
    spec.pop("chi_C", None)
    spec.pop("note", None)
    if kind == "gaussian":
        return (gaussian_mpo(spec["L"], spec.get("d", 2), spec["chi"], seed, 0, spec.get("scale")),
                gaussian_mpo(spec["L"], spec.get("d", 2), spec["chi"], seed, 1, spec.get("scale")))
    if kind == "kron":
        return (kron_sum_mpo(spec["L"], spec["K"], seed, 0, spec.get("decay", 0.8)),
                kron_sum_mpo(spec["L"], spec["K"], seed, 1, spec.get("decay", 0.8)))
    if kind == "uniform":
        return (uniform_mpo(spec["L"], spec.get("d", 2), spec["chi"], seed, 0, spec.get("alpha", -0.5)),
                uniform_mpo(spec["L"], spec.get("d", 2), spec["chi"], seed, 1, spec.get("alpha", -0.5)))
    raise KeyError(kind)


# Named workloads: L sites, local dims 2x2.
WORKLOADS = {
    # exact product fits in chi_C = chi_A * chi_B = 64
    "gauss_L8_chi8": dict(kind="gaussian", L=8, chi=8, scale=1.0 / np.sqrt(16.0), chi_C=64),
    # sum of 64 Kronecker terms, fit to chi_C = 64
    "kron_L20_chi64": dict(kind="kron", L=20, K=64, chi_C=64),
    # sum of 128 Kronecker terms, fit to chi_C = 128 (the timed workload)
    "kron_L30_chi128": dict(kind="kron", L=30, K=128, chi_C=128),
    # small cases for parity tests
    "kron_L10_chi16": dict(kind="kron", L=10, K=16, chi_C=16),
    "kron_L12_chi32": dict(kind="kron", L=12, K=32, chi_C=32),
    "uniform_L12_chi12": dict(kind="uniform", L=12, chi=12, alpha=-0.5, chi_C=12),
    # the paper's random tensor trains (Sec. 5.1): entries uniform in [alpha, 1], cores normalised;
    # ||A B|| falls like ~0.2^L, far below the FP32 range at these lengths
    "uniform_L102_chi30": dict(kind="uniform", L=102, chi=30, alpha=-0.33, chi_C=30),
    "uniform_L102_chi100": dict(kind="uniform", L=102, chi=100, alpha=-0.5, chi_C=100),
    "uniform_L50_chi128": dict(kind="uniform", L=50, chi=128, alpha=-0.5, chi_C=128),
    # the timed workload's window shapes (chi = 128 at the middle sites) on a short chain, for profiling
    "kron_L10_chi128": dict(kind="kron", L=10, K=128, chi_C=128),
}
