"""Plain FP64 variational fit of C ~ A B (Sec. 2.3, Algs. 3-5) with the
randomized-SVD update (Sec. 3.1).

ORACLE: test infrastructure only. Imported by tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline / reference leg; never by the product path. It
shares no code with the CUDA path; only the seeded inputs of
paper_2606_23274_gb300.synth are common.

Readings of the paper taken here, where it is silent or ambiguous:

* Env/sweep indices (Alg. 5): L_0 = R_{L+1} = [1] (Sec. 2.3.3); R_L..R_3 are
  precomputed; a forward step at site l first builds L_{l-1} (l >= 2), a
  backward step first builds R_{l+2} (l <= L-2).
* A and B are prepared by Alg. 5's left_orthogonalize, preceded by an RQ sweep
  that only trims bonds to their exact rank bound; their gauge never changes
  the product AB, so the same prepared A, B serve both gauges.
* Initial guess: random right-canonical MPO (OC at site 1), bonds
  min(chi_max, prod of local dims to the left, to the right); core 1 Gaussian,
  core l >= 2 the orthonormal-row factor of a Gaussian matrix. A given guess
  (or a copy of B) is trimmed by a QR sweep and then right-orthogonalized by
  an RQ sweep; neither changes the operator.
  The zip-up guess (Sec. 2.3.5) is the right-to-left zip-up of the prepared
  A, B (oracle/zipup.py) with the fit's chi_max, tau, cut-off, update and
  seed: right-canonical with the orthogonality centre at site 1 as it comes.
  In the inverse gauge Psi_l = C0_l and Y_l = 1.
* Randomized bond projection (Sec. 3.2, option ab_rank = k): the projectors
  depend only on A and B, which the fit never changes, so they are drawn once:
  A and B are replaced by their projected chains (oracle/zipup.py
  project_bonds, streams (4 << 40) | l for A and (5 << 40) | l for B; they
  come out right-canonical, and the fit does not depend on their gauge), and
  the fit runs on them in either gauge. The zip-up guess left-orthogonalizes
  its inputs itself.
* Truncation (Sec. 2.3.4): keep k = min(chi_max, min{k : sqrt(sum_{j>k} s_j^2)
  <= (tau/L) ||M||_F}), then drop s_j <= sv_cutoff * s_1 (Sec. 2.3.1 allows
  dropping very small values before inversion; applied in both gauges), k >= 1.
* Randomized update (Sec. 3.1): sketch width k_s = chi_max + oversample; when
  k_s >= min(m, n) the exact SVD is used. Omega is a fresh Philox Gaussian
  matrix per (sweep, window), n x k_s row-major.
* Singular pairs carry a fixed sign: the largest-magnitude entry of u_j is
  positive (the paper leaves the sign open; the sketch of Sec. 3.1 is not
  invariant under sign changes of the bond basis, so both sides fix it).
* Non-unique results: at a cut with s_k / s_{k+1} <= 1 + 1e-6 the kept subspace is not
  unique; gaps() reports the ratio per bond and pinned_bonds() the bonds whose spectrum
  parity is meaningful.
* Convergence: ||C||^2 = sum of kept s^2 at the last window of a sweep (the
  orthogonality centre); delta_s = | ||C||^2_s - ||C||^2_{s-1} | / ||C||^2_s.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import philox
from .mpo import canonicalize_input, left_orthogonalize, qr_pos, right_orthogonalize


# --------------------------------------------------------------------------
# environments (Sec. 2.3.3, Fig. envs): three pairwise contractions each
# --------------------------------------------------------------------------
def left_env(Lp, Al, Bl, Cl):
    """L_l[a1,b1,c1] = sum L_{l-1}[a0,b0,c0] A_l[a0,s,u,a1] B_l[b0,u,t,b1] C_l[c0,s,t,c1]."""
    T = np.einsum("abc,asux->bcsux", Lp, Al)          # first diagram
    T = np.einsum("bcsux,buty->csxty", T, Bl)         # second diagram
    return np.einsum("csxty,cstz->xyz", T, Cl)        # third diagram


def right_env(Rn, Al, Bl, Cl):
    """R_l[a0,b0,c0] = sum A_l[a0,s,u,a1] B_l[b0,u,t,b1] C_l[c0,s,t,c1] R_{l+1}[a1,b1,c1]."""
    T = np.einsum("asux,xyz->asuyz", Al, Rn)
    T = np.einsum("asuyz,buty->asbtz", T, Bl)
    return np.einsum("asbtz,cstz->abc", T, Cl)


def local_tensor(Lp, A1, B1, A2, B2, Rn):
    """The 6-leg right-hand side of Eq. (fit_pde), Fig. derivatives (d):
    Theta[c0,s1,t1,s2,t2,c2] = sum L A_l B_l A_{l+1} B_{l+1} R."""
    H1 = np.einsum("abc,asux,buty->cstxy", Lp, A1, B1, optimize=True)
    H2 = np.einsum("xpvg,yvqh,ghz->xypqz", A2, B2, Rn, optimize=True)
    return np.einsum("cstxy,xypqz->cstpqz", H1, H2)


# --------------------------------------------------------------------------
# factorizations (Sec. 2.3.4 truncated SVD, Sec. 3.1 randomized SVD)
# --------------------------------------------------------------------------
def keep_rank(S, norm_M, tau, L, chi_max, sv_cutoff):
    """Number of singular values kept by the truncation rule (Sec. 2.3.4)."""
    n = len(S)
    k = min(chi_max, n)
    if tau > 0.0:
        tail2 = np.concatenate([np.cumsum((S ** 2)[::-1])[::-1], [0.0]])  # tail2[j] = sum_{i>=j} s_i^2
        thr = (tau / L) * norm_M
        kmin = next(j for j in range(1, n + 1) if math.sqrt(max(tail2[j], 0.0)) <= thr or j == n)
        k = min(k, kmin)
    if n:
        k = min(k, int(np.count_nonzero(S > sv_cutoff * S[0])))   # an all-zero M keeps k = 1
    return max(k, 1)


def fix_signs(U, Vt):
    """Sign convention of each singular pair: the entry of largest magnitude of
    u_j is positive (first such index on ties). The pair (u_j, v_j) is defined
    only up to a common sign; fixing it makes the bond bases, and with them the
    Gaussian sketch of the randomized update, reproducible."""
    if U.shape[1] == 0:
        return U, Vt
    i = np.argmax(np.abs(U), axis=0)
    sgn = np.where(U[i, np.arange(U.shape[1])] < 0, -1.0, 1.0)
    return U * sgn[None, :], Vt * sgn[:, None]


def exact_svd(M):
    U, S, Vt = np.linalg.svd(M, full_matrices=False)
    return U, S, Vt


def randomized_svd(M, ks, seed, stream):
    """Sec. 3.1: M Omega = Q R; Q^T M = U S V^T; U~ = Q U."""
    m, n = M.shape
    Omega = philox.normals(seed, stream, n * ks).reshape(n, ks)
    Y = M @ Omega
    Q, _ = qr_pos(Y)
    Bm = Q.T @ M
    Ub, S, Vt = np.linalg.svd(Bm, full_matrices=False)
    return Q @ Ub, S, Vt


# --------------------------------------------------------------------------
# initial guess (Sec. 2.3.5)
# --------------------------------------------------------------------------
def init_bonds(dout, din, chi_max):
    L = len(dout)
    loc = [dout[l] * din[l] for l in range(L)]
    out = [1]
    for l in range(1, L):
        left = math.prod(loc[:l])
        right = math.prod(loc[l:])
        out.append(min(chi_max, left, right))
    out.append(1)
    return out


def random_right_canonical(dout, din, chi_max, seed):
    b = init_bonds(dout, din, chi_max)
    C = []
    for l in range(len(dout)):
        shape = (b[l], dout[l], din[l], b[l + 1])
        G = philox.normals(seed, philox.init_stream(l + 1), int(np.prod(shape))).reshape(shape)
        if l > 0:
            Q, _ = qr_pos(G.reshape(b[l], -1).T)          # rows of G^T -> orthonormal rows
            G = Q.T.reshape(shape)
        C.append(G)
    return C


# --------------------------------------------------------------------------
# the fit (Alg. 5 with Alg. 3 or Alg. 4 as the update)
# --------------------------------------------------------------------------
@dataclass
class SweepRecord:
    norm2: float
    delta: float
    max_discarded: float
    bonds: list


@dataclass
class FitState:
    A: list
    B: list
    Psi: list                      # C cores (site gauge: C_l; inverse gauge: Psi_l)
    Y: list                        # Y_l per bond l = 0..L (site gauge: all ones)
    S: list = field(default_factory=list)   # kept singular values of the last update per bond
    Lenv: list = field(default_factory=list)
    Renv: list = field(default_factory=list)
    history: list = field(default_factory=list)
    sweeps_done: int = 0
    forward: bool = True
    converged: bool = False


class FitOracle:
    def __init__(self, A, B, chi_max, tol, gauge="site", update="svd", oversample=10,
                 seed=0, sv_cutoff=1e-13, conv_tol=None, init="random", init_C=None,
                 prepare_inputs=True, ab_rank=0):
        assert gauge in ("site", "inverse") and update in ("svd", "rsvd")
        L = len(A)
        assert len(B) == L and L >= 2
        for l in range(L):
            assert A[l].shape[2] == B[l].shape[1], "A's input leg must match B's output leg"
        self.L, self.chi_max, self.tau = L, int(chi_max), float(tol)
        self.gauge, self.update_kind = gauge, update
        self.oversample, self.seed, self.sv_cutoff = int(oversample), int(seed), float(sv_cutoff)
        self.conv_tol = float(tol if conv_tol is None else conv_tol)
        A = [np.asarray(x, np.float64) for x in A]
        B = [np.asarray(x, np.float64) for x in B]
        if prepare_inputs:                       # Alg. 5: left_orthogonalize(A), (B)
            A, B = canonicalize_input(A), canonicalize_input(B)
        if ab_rank > 0:                          # Sec. 3.2: rank-k projectors on the A and B bonds
            from .zipup import project_bonds
            A = project_bonds(A, ab_rank, seed, 0)
            B = project_bonds(B, ab_rank, seed, 1)
        dout = [a.shape[1] for a in A]
        din = [b.shape[2] for b in B]
        if init == "random":
            C0 = random_right_canonical(dout, din, self.chi_max, self.seed)
        elif init == "copy_b":                   # QR sweep (trims bonds), then RQ sweep
            C0 = right_orthogonalize(left_orthogonalize(B))
        elif init == "zipup":                    # Sec. 2.3.5: the zip-up contraction as the guess
            from .zipup import zipup_right_to_left   # right to left on the left-canonical A, B
            C0 = zipup_right_to_left(A, B, self.chi_max, self.tau, self.sv_cutoff, update, self.oversample,
                                     self.seed)
        elif init == "given":
            C0 = right_orthogonalize(left_orthogonalize([np.asarray(x, np.float64) for x in init_C]))
        else:
            raise ValueError(init)
        self.gap = [math.inf] * (L + 1)  # per bond: s_k / s_{k+1} of its latest update
        Y = [np.ones(1)] + [np.ones(C0[l].shape[3]) for l in range(L - 1)] + [np.ones(1)]
        self.st = FitState(A=A, B=B, Psi=C0, Y=Y, S=[None] * (L + 1))
        self._precompute_right_envs()

    # cores seen by the environments: Psi_l Y_l (left) and Y_{l-1} Psi_l (right)
    def _c_left(self, l):
        st = self.st
        return st.Psi[l - 1] * st.Y[l][None, None, None, :]

    def _c_right(self, l):
        st = self.st
        return st.Y[l - 1][:, None, None, None] * st.Psi[l - 1]

    def _precompute_right_envs(self):
        st, L = self.st, self.L
        st.Lenv = [None] * (L + 2)
        st.Renv = [None] * (L + 2)
        st.Lenv[0] = np.ones((1, 1, 1))
        st.Renv[L + 1] = np.ones((1, 1, 1))
        for l in range(L, 2, -1):                # Alg. 5: for l in L..3
            st.Renv[l] = right_env(st.Renv[l + 1], st.A[l - 1], st.B[l - 1], self._c_right(l))

    def _update(self, l, forward, sweep_index):
        """Alg. 3 (site gauge) or Alg. 4 (inverse gauge) at window (l, l+1)."""
        st, L = self.st, self.L
        Theta = local_tensor(st.Lenv[l - 1], st.A[l - 1], st.B[l - 1], st.A[l], st.B[l], st.Renv[l + 2])
        c0, d1, e1, d2, e2, c2 = Theta.shape
        M = Theta.reshape(c0 * d1 * e1, d2 * e2 * c2)
        m, n = M.shape
        norm_M = float(np.linalg.norm(M))
        ks = self.chi_max + self.oversample
        if self.update_kind == "rsvd" and ks < min(m, n):
            U, S, Vt = randomized_svd(M, ks, self.seed, philox.omega_stream(sweep_index, l))
        else:
            U, S, Vt = exact_svd(M)
        k = keep_rank(S, norm_M, self.tau, L, self.chi_max, self.sv_cutoff)
        disc = math.sqrt(float(np.sum(S[k:] ** 2))) / norm_M if norm_M > 0 else 0.0
        # gap at the cut, s_k / s_{k+1} (inf when nothing is cut): where it is ~1 the kept subspace
        # is not unique, and neither are the bond's spectrum and cores in another arithmetic
        self.gap[l] = float(S[k - 1] / S[k]) if k < len(S) and S[k] > 0 else math.inf
        U, Vt = fix_signs(U[:, :k], Vt[:k, :])
        S = S[:k]
        st.S[l] = S.copy()
        self.last_factors = (U, S, Vt)
        if self.gauge == "site":
            if forward:                           # C_l, C_{l+1} <- U, S V^T
                left, right = U, S[:, None] * Vt
            else:                                 # C_l, C_{l+1} <- U S, V^T
                left, right = U * S[None, :], Vt
            st.Y[l] = np.ones(k)
        else:                                     # Psi_l <- U S, Psi_{l+1} <- S V^T, Y_l <- S^-1
            left, right = U * S[None, :], S[:, None] * Vt
            st.Y[l] = np.where(S > 0, 1.0 / np.where(S > 0, S, 1.0), 0.0)
        st.Psi[l - 1] = left.reshape(c0, d1, e1, k)
        st.Psi[l] = right.reshape(k, d2, e2, c2)
        return float(np.sum(S ** 2)), disc

    def sweep(self, n_sweeps=1, stop_on_converge=True):
        """Alg. 5's sweep loop; each call of the loop body is one directional sweep."""
        st, L = self.st, self.L
        for _ in range(n_sweeps):
            if st.converged and stop_on_converge:
                break
            s = st.sweeps_done
            max_disc = 0.0
            if st.forward:
                for l in range(1, L):
                    if l >= 2:
                        st.Lenv[l - 1] = left_env(st.Lenv[l - 2], st.A[l - 2], st.B[l - 2], self._c_left(l - 1))
                    n2, disc = self._update(l, True, s)
                    max_disc = max(max_disc, disc)
            else:
                for l in range(L - 1, 0, -1):
                    if l <= L - 2:
                        st.Renv[l + 2] = right_env(st.Renv[l + 3], st.A[l + 1], st.B[l + 1], self._c_right(l + 2))
                    n2, disc = self._update(l, False, s)
                    max_disc = max(max_disc, disc)
            prev = st.history[-1].norm2 if st.history else None
            delta = abs(n2 - prev) / n2 if (prev is not None and n2 > 0) else math.inf
            st.history.append(SweepRecord(n2, delta, max_disc, self.bonds()))
            st.sweeps_done += 1
            st.forward = not st.forward
            if delta <= self.conv_tol:
                st.converged = True
        return st.history

    def bonds(self):
        return [1] + [p.shape[3] for p in self.st.Psi]

    def result(self):
        """C as a plain MPO: C_l = Psi_l Y_l (l < L), C_L = Psi_L."""
        L = self.L
        return [self._c_left(l) if l < L else self.st.Psi[L - 1].copy() for l in range(1, L + 1)]

    def lambdas(self):
        """Kept singular values of the last update of each inner bond 1..L-1."""
        return [s.copy() for s in self.st.S[1:self.L]]

    def gaps(self):
        """s_k / s_{k+1} at the cut of the last update of each inner bond 1..L-1 (inf: no cut)."""
        return list(self.gap[1:self.L])

    def pinned_bonds(self, rel=1e-6):
        """Inner bonds (1-based) whose cut is not degenerate, gap > 1 + rel: their kept spectrum and
        subspace are unique; at the others parity of the spectrum is declared unpinned."""
        return [l for l, g in enumerate(self.gaps(), 1) if g > 1.0 + rel]


def fit(A, B, chi_max, tol, n_sweeps, **kw):
    """Convenience wrapper: run ``n_sweeps`` directional sweeps, return (C, oracle)."""
    stop = kw.pop("stop_on_converge", True)
    f = FitOracle(A, B, chi_max, tol, **kw)
    f.sweep(n_sweeps, stop_on_converge=stop)
    return f.result(), f
