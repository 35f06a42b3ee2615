"""Plain FP64 zip-up contraction of two MPOs (Sec. 2.2, Alg. 2), used as the
fit's initial guess (Sec. 2.3.5).

ORACLE: test infrastructure only. Imported by tests/ (and through them nothing
else); never by the product path. It shares no code with the CUDA path; only
the seeded inputs of paper_2606_23274_gb300.synth are common.

Alg. 2 runs left to right on right-canonical inputs. Its mirror runs right to
left on left-canonical inputs (the paper notes that it applies to TTs brought
into left-canonical form) and leaves C right-canonical with the orthogonality
centre on site 1, which is the form the fit starts from; the GPU builds that
one. Readings taken here:

* Each step factorises the reshaped remainder with the truncation rule of the
  fit (Sec. 2.3.4: keep min(chi_max, smallest k with sqrt(sum_{j>k} s_j^2) <=
  (tau / L) ||M||_F) values, then drop s_j <= sv_cutoff s_1, k >= 1).
* With update="rsvd" the factorisation is the randomized SVD of Sec. 3.1 (the
  paper: "can be reduced ... using randomized SVDs"), applied to the side whose
  singular vectors become the new core, with k_s = chi_max + oversample and the
  Philox Gaussian of stream zipup_stream(site); when k_s is not narrower than
  the matrix the exact SVD is used.
* The sign convention of the fit (largest-magnitude entry of each kept vector
  positive) is applied to the kept singular vectors.
"""
from __future__ import annotations

import numpy as np

from . import philox
from .fit import fix_signs, keep_rank
from .mpo import left_orthogonalize, qr_pos, right_orthogonalize


def zipup_stream(site: int) -> int:
    """Philox stream of the zip-up sketch at a site (1-based): distinct from the
    fit's sweep sketches and initial guess."""
    return (3 << 40) | int(site)


def _factor(M, chi_max, tau, L, sv_cutoff, update, oversample, seed, site):
    """Truncated factorisation M ~ U S V^T by the fit's rule; returns U (signed), S, Vt."""
    U, S, Vt, _ = _factor_full(M, chi_max, tau, L, sv_cutoff, update, oversample, seed, site)
    return U, S, Vt


def zipup_left_to_right(A, B, chi_max, tau=0.0, sv_cutoff=1e-13, update="svd", oversample=10, seed=0):
    """Alg. 2 as printed: inputs right-canonicalised; R_0 = [[[1]]]; at site l,
    R'' = R_{l-1} A_l B_l reshaped (chi d d') x (chi_A chi_B); C_l = U, R_l = S V^T;
    the last remainder is absorbed into C_L."""
    A = right_orthogonalize([np.asarray(x, np.float64) for x in A])
    B = right_orthogonalize([np.asarray(x, np.float64) for x in B])
    L = len(A)
    R = np.ones((1, 1, 1))                                     # [c, a, b]
    C = []
    for l in range(L):
        T = np.einsum("cab,asux->cbsux", R, A[l])
        T = np.einsum("cbsux,buty->cstxy", T, B[l])            # [c, s, t, a', b']
        c, s, t, x, y = T.shape
        if l == L - 1:                                         # x = y = 1: the remainder is the last core
            C.append(T.reshape(c, s, t, 1))
            break
        U, S, Vt = _factor(T.reshape(c * s * t, x * y), chi_max, tau, L, sv_cutoff, update, oversample, seed,
                           l + 1)
        k = S.shape[0]
        C.append(U.reshape(c, s, t, k))
        R = (S[:, None] * Vt).reshape(k, x, y)
    return C


def zipup_right_to_left(A, B, chi_max, tau=0.0, sv_cutoff=1e-13, update="svd", oversample=10, seed=0):
    """The mirror of Alg. 2: inputs left-canonicalised; R_{L+1} = [[[1]]]; at site l,
    M = A_l B_l R_{l+1} reshaped (chi_A chi_B) x (d d' chi); C_l = V^T (right-orthonormal),
    R_l = U S; the last remainder is C_1."""
    A = left_orthogonalize([np.asarray(x, np.float64) for x in A])
    B = left_orthogonalize([np.asarray(x, np.float64) for x in B])
    L = len(A)
    R = np.ones((1, 1, 1))                                     # [a, b, c]
    C = [None] * L
    for l in range(L - 1, -1, -1):
        T = np.einsum("asux,xyc->asuyc", A[l], R)
        T = np.einsum("asuyc,buty->abstc", T, B[l])            # [a0, b0, s, t, c]
        a, b, s, t, c = T.shape
        if l == 0:                                             # a = b = 1: the remainder is the first core
            C[0] = T.reshape(1, s, t, c)
            break
        # the new core spans the right singular vectors: factorise M^T = V S U^T
        V, S, Ut = _factor(T.reshape(a * b, s * t * c).T, chi_max, tau, L, sv_cutoff, update, oversample, seed,
                           l + 1)
        k = S.shape[0]
        C[l] = V.T.reshape(k, s, t, c)
        R = (Ut.T * S[None, :]).reshape(a, b, k)
    return C


def compress(X, chi_max, tau=0.0, sv_cutoff=1e-13, update="svd", oversample=10, seed=0, return_discarded=False):
    """compress() of Alg. 1 (Sec. 2.1): the standard SVD compression, which the
    paper names without spelling out. Reading: X is left-orthogonalized, then swept
    right to left; at site l the core absorbs the remainder, M = X_l R_{l+1}
    reshaped chi_{l-1} x (d d' chi), and the truncated factorisation of M^T (the
    rule and sketch streams of the zip-up) gives C_l = V^T (right-orthonormal) and
    R_l = U S. With return_discarded, also the discarded weight
    sqrt(sum_{j>k} s_j^2) of every factorisation (of the kept spectrum of the
    sketch under update="rsvd")."""
    X = left_orthogonalize([np.asarray(x, np.float64) for x in X])
    L = len(X)
    R = np.ones((1, 1))                                        # [a, c]
    C = [None] * L
    disc = []
    for l in range(L - 1, -1, -1):
        T = np.einsum("astx,xc->astc", X[l], R)
        a, s, t, c = T.shape
        if l == 0:
            C[0] = T
            break
        M = T.reshape(a, s * t * c)
        V, S, Ut, full = _factor_full(M.T, chi_max, tau, L, sv_cutoff, update, oversample, seed, l + 1)
        k = S.shape[0]
        disc.append(float(np.sqrt(np.sum(full[k:] ** 2))))
        C[l] = V.T.reshape(k, s, t, c)
        R = Ut.T * S[None, :]
    return (C, disc[::-1]) if return_discarded else C


def _factor_full(M, chi_max, tau, L, sv_cutoff, update, oversample, seed, site):
    """_factor, also returning every singular value it computed."""
    m, n = M.shape
    norm_M = float(np.linalg.norm(M))
    ks = chi_max + oversample
    if update == "rsvd" and ks < min(m, n):
        Om = philox.normals(seed, zipup_stream(site), n * ks).reshape(n, ks)
        Q, _ = np.linalg.qr(M @ Om)
        Ub, S, Vt = np.linalg.svd(Q.T @ M, full_matrices=False)
        U = Q @ Ub
    else:
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
    k = keep_rank(S, norm_M, tau, L, chi_max, sv_cutoff)
    Uk, Vtk = fix_signs(U[:, :k], Vt[:k, :])
    return Uk, S[:k], Vtk, S


def project_stream(which: int, site: int) -> int:
    """Philox stream of the bond projector of A (which = 0) or B (which = 1) at a site (1-based)."""
    return ((4 + int(which)) << 40) | int(site)


def project_bonds(X, k, seed=0, which=0):
    """Randomized bond projection of one MPO chain (Sec. 3.2): a projector Q Q^T of
    rank k on every bond. Reading: X (left-orthogonalized, so that everything left of
    a bond is an isometry) is swept right to left; at site l the core with the
    remainder absorbed, M = X_l R_{l+1} reshaped chi_{l-1} x (d d' k), gets the
    range finder of Sec. 3: Y = M^T Omega (Omega chi_{l-1} x k Gaussian, stream
    project_stream(which, l)), Q = the orthonormal factor of Y (d d' k x k, the QR
    with a non-negative diagonal of R, which fixes the bond basis the zip-up sketches);
    X_l <- Q^T and R_l = M Q. Where k >= min of M's sizes the bond is kept whole
    (Q = the orthonormal factor of M^T). The result is right-canonical."""
    X = left_orthogonalize([np.asarray(x, np.float64) for x in X])
    L = len(X)
    R = np.ones((1, 1))
    out = [None] * L
    for l in range(L - 1, -1, -1):
        T = np.einsum("astx,xc->astc", X[l], R)
        a, s, t, c = T.shape
        if l == 0:
            out[0] = T
            break
        M = T.reshape(a, s * t * c)
        if k < min(M.shape):
            Om = philox.normals(seed, project_stream(which, l + 1), a * k).reshape(a, k)
            Q, _ = qr_pos(M.T @ Om)
        else:
            Q, _ = qr_pos(M.T)
        out[l] = Q.T.reshape(Q.shape[1], s, t, c)
        R = M @ Q
    return out
