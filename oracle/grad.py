"""Gradients of the fit's objectives with respect to the cores of A and B: the
adjoint of the environment and local contraction chain, at fixed C.

ORACLE: test infrastructure only (tests/, smoke(), bench.py's CPU legs). Plain
FP64 numpy; nothing here is used by the CUDA path.

The paper states the fit's objective (Eq. fit_min, ||A B - C||_F^2 minimised
over C) and builds it from environments (Fig. envs); it does not differentiate
with respect to A or B. Readings taken here, where the paper is silent:

* "At fixed gauge": C (or W) is a constant MPO; nothing is differentiated
  through the fit's SVDs or iterations.
* f1(A, B) = ||C - A B||_F^2 = ||C||^2 - 2 <C, AB> + ||AB||^2.
* f2(A, B) = tr(W^T A B) = <W, AB> for a fixed MPO W.
* <X, AB> is the three-layer network of the fit's environments (Sec. 2.3.3):
  L_l[a1, b1, c1] = sum L_{l-1}[a0, b0, c0] A_l[a0, s, u, a1] B_l[b0, u, t, b1]
  X_l[c0, s, t, c1], and the mirror R_l. Its derivative with respect to A_l is
  the network with A_l cut out (a punched hole):
  G^X_A,l[a0, s, u, a1] = sum L_{l-1}[a0,b0,c0] X_l[c0,s,t,c1] B_l[b0,u,t,b1] R_{l+1}[a1,b1,c1],
  and for B_l the mirror.
* ||AB||^2 = <AB, AB> uses four-layer environments F_l[a, b, p, q] (two copies
  of A, B). A_l occurs once in each copy and the network is symmetric in the
  copies, so d||AB||^2/dA_l is twice the punched hole of one copy.

Index convention: cores X_l[left, out, in, right]; C = AB contracts A's input
leg with B's output leg.
"""
from __future__ import annotations

import numpy as np

_ONE3 = np.ones((1, 1, 1))
_ONE4 = np.ones((1, 1, 1, 1))


# ---------------------------------------------------------------- three layers
def _left3(Lp, X, A, B):
    """L_l from L_{l-1}: the fit's left environment with X in the place of C."""
    T = np.einsum("abc,asux->bcsux", Lp, A)
    T = np.einsum("bcsux,buty->csxty", T, B)
    return np.einsum("csxty,cstz->xyz", T, X)


def _right3(Rn, X, A, B):
    T = np.einsum("asux,xyz->asuyz", A, Rn)
    T = np.einsum("asuyz,buty->asbtz", T, B)
    return np.einsum("asbtz,cstz->abc", T, X)


def inner(X, A, B) -> float:
    """<X, A B> = sum over all indices of X (A B) (elementwise), by transfer."""
    E = _ONE3
    for l in range(len(A)):
        E = _left3(E, X[l], A[l], B[l])
    return float(E.reshape(-1)[0])


def inner_grads(X, A, B):
    """(dA, dB): d<X, AB>/dA_l and d<X, AB>/dB_l for every site (punched holes)."""
    L = len(A)
    Le = [_ONE3]
    for l in range(L - 1):
        Le.append(_left3(Le[-1], X[l], A[l], B[l]))
    Re = [None] * (L + 1)
    Re[L] = _ONE3
    for l in range(L - 1, 0, -1):
        Re[l] = _right3(Re[l + 1], X[l], A[l], B[l])
    gA, gB = [], []
    for l in range(L):
        Lp, Rn = Le[l], Re[l + 1]
        # A_l hole: L[a0,b0,c0] X[c0,s,t,c1] B[b0,u,t,b1] R[a1,b1,c1]
        T = np.einsum("abc,cstz->abstz", Lp, X[l])
        T = np.einsum("abstz,buty->asuyz", T, B[l])
        gA.append(np.einsum("asuyz,xyz->asux", T, Rn))
        # B_l hole: L[a0,b0,c0] A[a0,s,u,a1] X[c0,s,t,c1] R[a1,b1,c1]
        T = np.einsum("abc,asux->bcsux", Lp, A[l])
        T = np.einsum("bcsux,cstz->buxtz", T, X[l])
        gB.append(np.einsum("buxtz,xyz->buty", T, Rn))
    return gA, gB


# ----------------------------------------------------------------- four layers
def _left4(F, A, B):
    """F_l[x, y, z, w] = sum F_{l-1}[a, b, p, q] A[a,s,u,x] B[b,u,t,y] A[p,s,v,z] B[q,v,t,w]."""
    T = np.einsum("abpq,asux->bpqsux", F, A)
    T = np.einsum("bpqsux,buty->pqsxty", T, B)
    T = np.einsum("pqsxty,psvz->qxytvz", T, A)
    return np.einsum("qxytvz,qvtw->xyzw", T, B)


def _right4(G, A, B):
    """Mirror of _left4: G_l[a, b, p, q] from G_{l+1}[x, y, z, w]."""
    T = np.einsum("qvtw,xyzw->qvtxyz", B, G)
    T = np.einsum("psvz,qvtxyz->pqstxy", A, T)
    T = np.einsum("buty,pqstxy->bpqsux", B, T)
    return np.einsum("asux,bpqsux->abpq", A, T)


def norm2_ab(A, B) -> float:
    """||A B||_F^2 = <AB, AB> by four-layer transfer."""
    F = _ONE4
    for l in range(len(A)):
        F = _left4(F, A[l], B[l])
    return float(F.reshape(-1)[0])


def norm2_ab_grads(A, B):
    """(dA, dB): d||AB||^2/dA_l and /dB_l (twice the punched hole of one copy)."""
    L = len(A)
    Fl = [_ONE4]
    for l in range(L - 1):
        Fl.append(_left4(Fl[-1], A[l], B[l]))
    Fr = [None] * (L + 1)
    Fr[L] = _ONE4
    for l in range(L - 1, 0, -1):
        Fr[l] = _right4(Fr[l + 1], A[l], B[l])
    gA, gB = [], []
    for l in range(L):
        F, G, Al, Bl = Fl[l], Fr[l + 1], A[l], B[l]
        # the second copy with its right environment: K[p, q, s, t, x, y]
        K = np.einsum("psvz,qvtw->pqstzw", Al, Bl)
        K = np.einsum("pqstzw,xyzw->pqstxy", K, G)
        # hole at A of the first copy: F[a,b,p,q] B[b,u,t,y] K[p,q,s,t,x,y]
        T = np.einsum("abpq,pqstxy->abstxy", F, K)
        gA.append(2.0 * np.einsum("abstxy,buty->asux", T, Bl))
        # hole at B of the first copy: F[a,b,p,q] A[a,s,u,x] K[p,q,s,t,x,y]
        gB.append(2.0 * np.einsum("abstxy,asux->buty", T, Al))
    return gA, gB


# ------------------------------------------------------------------- objectives
def f1_and_grads(C, A, B):
    """f1 = ||C - AB||_F^2 and its gradients with respect to every A_l, B_l."""
    cc = _norm2(C)
    ci = inner(C, A, B)
    nn = norm2_ab(A, B)
    gI = inner_grads(C, A, B)
    gN = norm2_ab_grads(A, B)
    gA = [n - 2.0 * i for n, i in zip(gN[0], gI[0])]
    gB = [n - 2.0 * i for n, i in zip(gN[1], gI[1])]
    return cc - 2.0 * ci + nn, gA, gB


def f2_and_grads(W, A, B):
    """f2 = tr(W^T A B) = <W, AB> and its gradients."""
    gA, gB = inner_grads(W, A, B)
    return inner(W, A, B), gA, gB


def _norm2(X) -> float:
    """||X||_F^2 of one MPO by two-layer transfer."""
    E = np.ones((1, 1))
    for c in X:
        T = np.einsum("ab,astx->bstx", E, c)
        E = np.einsum("bstx,bsty->xy", T, c)
    return float(E.reshape(-1)[0])

