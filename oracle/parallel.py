"""Plain FP64 simulation of the segment-parallel fit in the inverse canonical
gauge (Sec. 4, Alg. 6).

ORACLE: test infrastructure only (tests/, smoke(), bench.py's CPU legs).

The chain is cut into N_p contiguous segments (sub-TTs). Segments run local
half-sweeps "in parallel"; here they run one after the other inside each phase,
which is equivalent because within a phase they touch disjoint sites and
disjoint environments. A full set of local sweeps is:

  (3) odd segments sweep forward, even segments backward;
  (4) connection updates at the odd|even boundaries: the left segment finishes
      L_{l-1}, the right one R_{l+2}; the window (l, l+1) is updated;
  (5) odd segments sweep backward, even segments forward;
  (6) connection updates at the even|odd boundaries.

Readings taken here, where the paper is silent or ambiguous:
* Segments are numbered from 1, so the first segment is odd.
* Initialisation (Sec. 4.2): the initial guess is brought to inverse canonical
  form by a left-to-right SVD sweep of the right-canonical guess (Psi_l = U S,
  Y_l = S^-1; this is the exact Vidal form). Every environment, including the
  boundary ones that the paper initialises as "identities (or random orthogonal
  matrices)", is computed exactly from that guess.
* A connection update is performed by the left segment (any one of the two
  may do it, Sec. 4.4).
* ||C||^2 after a set of local sweeps is the sum of the kept s^2 of the last
  connection update (every Psi is an orthogonality centre in this gauge).
"""
from __future__ import annotations

import math

import numpy as np

from .fit import FitOracle, fix_signs, keep_rank, left_env, local_tensor, right_env, exact_svd, randomized_svd
from . import philox


def partition(L: int, n_seg: int, edge_extra: int = 0):
    """Contiguous segments (first site, last site), 1-based, edge segments get
    ``edge_extra`` more sites (Sec. 4.1 load balance). Every segment has >= 2 sites."""
    base = [L // n_seg] * n_seg
    for i in range(L % n_seg):
        base[i] += 1
    if n_seg >= 3 and edge_extra:
        spare = sum(b - 2 for b in base[1:-1])          # sites the inner segments can give
        take = max(0, min(edge_extra, spare // 2))
        for e in (0, n_seg - 1):
            base[e] += take
        inner = list(range(1, n_seg - 1))
        need = 2 * take
        i = 0
        while need > 0:
            base[inner[i % len(inner)]] -= 1
            need -= 1
            i += 1
    out, s = [], 1
    for n in base:
        out.append((s, s + n - 1))
        s += n
    assert out[-1][1] == L and all(b - a + 1 >= 2 for a, b in out)
    return out


class ParallelFitOracle(FitOracle):
    """Alg. 6 in the inverse gauge on top of the serial oracle's state."""

    def __init__(self, A, B, chi_max, tol, n_seg, edge_extra=0, **kw):
        kw["gauge"] = "inverse"
        super().__init__(A, B, chi_max, tol, **kw)
        self.segs = partition(self.L, n_seg, edge_extra)
        self._to_inverse_form()
        self._all_envs()
        self.set_count = 0
        self.par_history = []

    # initial guess -> inverse canonical form (left-to-right SVD sweep)
    def _to_inverse_form(self):
        st, L = self.st, self.L
        P = [p.copy() for p in st.Psi]
        for l in range(1, L):
            a0, d, dp, a1 = P[l - 1].shape
            U, S, Vt = np.linalg.svd(P[l - 1].reshape(a0 * d * dp, a1), full_matrices=False)
            k = max(1, int(np.count_nonzero(S > self.sv_cutoff * S[0])))
            U, Vt = fix_signs(U[:, :k], Vt[:k, :])
            S = S[:k]
            P[l - 1] = (U * S[None, :]).reshape(a0, d, dp, k)          # Psi_l = U S
            st.Y[l] = 1.0 / S                                           # Y_l = S^-1
            st.S[l] = S.copy()
            P[l] = np.einsum("k,ka,axyb->kxyb", S, Vt, P[l])          # S V^T carried right
        # the last core keeps the carried S V^T: Psi_L = Lambda_{L-1} Gamma_L
        st.Psi = P

    def _all_envs(self):
        st, L = self.st, self.L
        st.Lenv = [None] * (L + 2)
        st.Renv = [None] * (L + 2)
        st.Lenv[0] = np.ones((1, 1, 1))
        st.Renv[L + 1] = np.ones((1, 1, 1))
        for l in range(1, L + 1):
            st.Lenv[l] = left_env(st.Lenv[l - 1], st.A[l - 1], st.B[l - 1], self._c_left(l))
        for l in range(L, 0, -1):
            st.Renv[l] = right_env(st.Renv[l + 1], st.A[l - 1], st.B[l - 1], self._c_right(l))

    def _local(self, seg, forward, sweep_index):
        ls, le = seg
        st = self.st
        n2 = None
        if forward:
            for l in range(ls, le):
                if l > ls:
                    st.Lenv[l - 1] = left_env(st.Lenv[l - 2], st.A[l - 2], st.B[l - 2], self._c_left(l - 1))
                n2, _ = self._update(l, True, sweep_index)
        else:
            for l in range(le - 1, ls - 1, -1):
                if l < le - 1:
                    st.Renv[l + 2] = right_env(st.Renv[l + 3], st.A[l + 1], st.B[l + 1], self._c_right(l + 2))
                n2, _ = self._update(l, False, sweep_index)
        return n2

    def _connect(self, left_seg, right_seg, sweep_index):
        st = self.st
        l = left_seg[1]                     # window (l, l+1) straddles the boundary
        st.Lenv[l - 1] = left_env(st.Lenv[l - 2], st.A[l - 2], st.B[l - 2], self._c_left(l - 1))
        st.Renv[l + 2] = right_env(st.Renv[l + 3], st.A[l + 1], st.B[l + 1], self._c_right(l + 2))
        n2, _ = self._update(l, True, sweep_index)
        # both neighbours then rebuild the environment across the new boundary bond
        st.Lenv[l] = left_env(st.Lenv[l - 1], st.A[l - 1], st.B[l - 1], self._c_left(l))
        st.Renv[l + 1] = right_env(st.Renv[l + 2], st.A[l], st.B[l], self._c_right(l + 1))
        return n2

    def full_sweep_set(self):
        """Steps (3)-(6) of Alg. 6 once; returns ||C||^2 after the last connection."""
        segs = self.segs
        s = self.set_count
        n2 = None
        for phase in (0, 1):
            for i, seg in enumerate(segs):
                odd = (i % 2 == 0)                          # segment i+1 is odd
                forward = odd if phase == 0 else not odd
                v = self._local(seg, forward, 2 * s + phase)
                n2 = v if v is not None else n2
            for i in range(len(segs) - 1):
                # phase 0: odd|even boundaries (i even), phase 1: even|odd (i odd)
                if (i % 2 == 0) == (phase == 0):
                    n2 = self._connect(segs[i], segs[i + 1], 2 * s + phase)
        prev = self.par_history[-1] if self.par_history else None
        delta = abs(n2 - prev) / n2 if prev is not None and n2 > 0 else math.inf
        self.par_history.append(n2)
        self.set_count += 1
        return n2, delta

    def result(self):
        return super().result()
