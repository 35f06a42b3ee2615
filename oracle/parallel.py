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
from .mpo import qr_pos


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


class SiteParallelFitOracle(ParallelFitOracle):
    """Alg. 6 in the site-canonical gauge (the paper's scheme II, Sec. 4) and the
    binary merge (Sec. 4.5). Readings taken here:

    * Initialisation (Sec. 4.2): the right-canonical guess already has every odd
      segment's orthogonality centre (OC) on its left-most site; every even segment
      moves its OC to its right-most site by QR steps inside the segment (the
      operator is unchanged). Every environment is then computed from these cores.
    * Local sweeps and connection updates are those of the inverse-gauge scheme with
      the site-gauge update (Alg. 3): a forward update leaves C_l = U, C_{l+1} = S V^T.
      Environments are built from orthonormal cores only, so after a connection
      update R_{l+1} is built from V^T (the bond basis), not from S V^T.
    * Until merged, the chain is a row of consistent units, each a sub-TT with one
      OC: after a phase with connection updates at the boundaries (l, l+1) each pair
      of segments joined there is one unit with its OC at l + 1; a segment without a
      connection is a unit with its OC where its sweep left it. The product of the
      cores counts every unit's weight, so it is not the fitted operator. merge()
      joins neighbouring units pairwise, in rounds: the left unit's OC moves to its
      last site l by QR steps, the right unit's to its first site l + 1 by RQ steps,
      each step finishing the environment it passes, then the window (l, l+1) is
      updated forward (the sketches of phase index P + r - 1 in round r, P = phases
      run so far). After the rounds C is one site-canonical MPO. When the last phase
      connected the odd|even boundaries, its connections are the first round of the
      paper's merge (boundaries after segments 1, 3, 5, ...), the next round joins
      across the boundaries after segments 2, 6, ..., and so on.
    """

    def __init__(self, A, B, chi_max, tol, n_seg, edge_extra=0, **kw):
        kw["gauge"] = "site"
        FitOracle.__init__(self, A, B, chi_max, tol, **kw)
        self.segs = partition(self.L, n_seg, edge_extra)
        for i, (ls, le) in enumerate(self.segs):
            if i % 2 == 1:                                  # even segment (1-based)
                for l in range(ls, le):
                    self._qr_step(l)
        self._all_envs()
        self.set_count = 0
        self.par_history = []
        self.merged = True
        self.last_phase = 1

    def _qr_step(self, l):
        """Site l (1-based) left-orthonormal: C_l = Q, C_{l+1} <- R C_{l+1}."""
        st = self.st
        a0, d, dp, a1 = st.Psi[l - 1].shape
        Q, R = qr_pos(st.Psi[l - 1].reshape(a0 * d * dp, a1))
        k = Q.shape[1]
        st.Psi[l - 1] = Q.reshape(a0, d, dp, k)
        st.Psi[l] = np.einsum("ka,axyb->kxyb", R, st.Psi[l])
        st.Y[l] = np.ones(k)

    def _rq_step(self, l):
        """Site l (1-based) right-orthonormal: C_l = Q^T, C_{l-1} <- C_{l-1} R^T."""
        st = self.st
        a0, d, dp, a1 = st.Psi[l - 1].shape
        Q, R = qr_pos(st.Psi[l - 1].reshape(a0, d * dp * a1).T)
        k = Q.shape[1]
        st.Psi[l - 1] = Q.T.reshape(k, d, dp, a1)
        st.Psi[l - 2] = np.einsum("axyb,kb->axyk", st.Psi[l - 2], R)
        st.Y[l - 1] = np.ones(k)

    def _boundary_update(self, l, sweep_index):
        """Forward update of window (l, l+1) from the stored L_{l-1}, R_{l+2}; then the
        environments across the new bond, from U and from the bond basis V^T."""
        st = self.st
        n2, _ = self._update(l, True, sweep_index)
        self.final_boundary, self.last_boundary_n2 = l, n2
        U, S, Vt = self.last_factors
        st.Lenv[l] = left_env(st.Lenv[l - 1], st.A[l - 1], st.B[l - 1], st.Psi[l - 1])
        st.Renv[l + 1] = right_env(st.Renv[l + 2], st.A[l], st.B[l], Vt.reshape(st.Psi[l].shape))
        return n2

    def _connect(self, left_seg, right_seg, sweep_index):
        st = self.st
        l = left_seg[1]
        st.Lenv[l - 1] = left_env(st.Lenv[l - 2], st.A[l - 2], st.B[l - 2], self._c_left(l - 1))
        st.Renv[l + 2] = right_env(st.Renv[l + 3], st.A[l + 1], st.B[l + 1], self._c_right(l + 2))
        return self._boundary_update(l, sweep_index)

    def full_sweep_set(self):
        n2, delta = super().full_sweep_set()
        self.merged = False
        self.last_phase = 1
        return n2, delta

    def half_set(self):
        """Steps (3)-(4) only: odd segments forward, even backward, then the odd|even
        connections (the phase that ends in the paper's first merge round)."""
        segs = self.segs
        s = self.set_count
        n2 = None
        for i, seg in enumerate(segs):
            v = self._local(seg, i % 2 == 0, 2 * s)
            n2 = v if v is not None else n2
        for i in range(0, len(segs) - 1, 2):
            n2 = self._connect(segs[i], segs[i + 1], 2 * s)
        self.merged = False
        self.last_phase = 0
        self.half_done = True
        return n2

    def _units(self):
        """Consistent sub-TTs after the last phase: (first site, last site, OC site)."""
        segs, ns = self.segs, len(self.segs)
        start = 0 if self.last_phase == 0 else 1            # first connected boundary (0-based segment)
        units, i = [], 0
        while i < ns:
            if (i - start) % 2 == 0 and i + 1 < ns and i >= start:
                units.append((segs[i][0], segs[i + 1][1], segs[i + 1][0]))
                i += 2
            else:
                forward = (i % 2 == 0) == (self.last_phase == 0)
                units.append((segs[i][0], segs[i][1], segs[i][1] if forward else segs[i][0]))
                i += 1
        return units

    def merge(self):
        """Sec. 4.5's binary merge; returns ||C||^2 of its last update."""
        st = self.st
        if self.merged:
            return None
        units = self._units()
        phases = 2 * self.set_count + (1 if getattr(self, "half_done", False) else 0)
        n2 = self.last_boundary_n2 if len(units) == 1 else None     # one unit: already consistent
        r = 1
        while len(units) > 1:
            nxt = []
            for u in range(0, len(units) - 1, 2):
                (fa, la, oa), (fb, lb, ob) = units[u], units[u + 1]
                for j in range(oa, la):                     # the left unit's OC to its last site
                    self._qr_step(j)
                    st.Lenv[j] = left_env(st.Lenv[j - 1], st.A[j - 1], st.B[j - 1], st.Psi[j - 1])
                for j in range(ob, fb, -1):                 # the right unit's OC to its first site
                    self._rq_step(j)
                    st.Renv[j] = right_env(st.Renv[j + 1], st.A[j - 1], st.B[j - 1], st.Psi[j - 1])
                n2 = self._boundary_update(la, phases + r - 1)
                nxt.append((fa, lb, la + 1))
            if len(units) % 2:
                nxt.append(units[-1])
            units = nxt
            r += 1
        self.merged = True
        return n2
