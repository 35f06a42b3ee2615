"""Plain PyTorch FP64 contractions of MPOs used as checkers at sizes the
oracle cannot follow (they run on whatever device the cores are on). Cores are
(chi_l, d_out, d_in, chi_r); C = A B contracts A's input leg with B's output
leg (Sec. 2.2). Pinned to the oracle and to dense products in
tests/test_mpo_props.py."""
import torch


def norm2(C) -> float:
    """||C||_F^2 by two-layer transfer: E'[c1, e1] = sum E[c0, e0] C[c0,s,t,c1] C[e0,s,t,e1]."""
    E = torch.ones((1, 1), dtype=torch.float64, device=C[0].device)
    for c in C:
        c = c.double()
        T = torch.tensordot(E, c, dims=([0], [0]))             # [e0, s, t, c1]
        E = torch.tensordot(T, c, dims=([0, 1, 2], [0, 1, 2]))  # [c1, e1]
    return float(E.reshape(-1)[0])


def inner_ab(C, A, B) -> float:
    """<C, A B> by three-layer transfer (the fit's environments, Sec. 2.3.3):
    E'[a1, b1, c1] = sum E[a0, b0, c0] A[a0, s, u, a1] B[b0, u, t, b1] C[c0, s, t, c1]."""
    dev = C[0].device
    E = torch.ones((1, 1, 1), dtype=torch.float64, device=dev)
    for a, b, c in zip(A, B, C):
        a, b, c = a.double().to(dev), b.double().to(dev), c.double()
        T1 = torch.tensordot(E, a, dims=([0], [0]))                     # [b0, c0, s, u, a1]
        T2 = torch.tensordot(T1, b, dims=([0, 3], [0, 1]))              # [c0, s, a1, t, b1]
        E = torch.tensordot(T2, c, dims=([0, 1, 3], [0, 1, 2]))         # [a1, b1, c1]
    return float(E.reshape(-1)[0])


def diff_norm(X, Y) -> float:
    """||X - Y||_F, computed stably: the direct-sum MPO X (+) (-Y) (block bonds)
    is left-orthogonalised by Householder QR in FP64 and the norm read off its
    last core, so the result does not suffer the cancellation of
    ||X||^2 + ||Y||^2 - 2 <X, Y> (the error metric of Sec. 5)."""
    L = len(X)
    dev = X[0].device
    if L == 1:
        return float(torch.linalg.norm(X[0].double() - Y[0].double().to(dev)))
    R = None
    for l in range(L):
        x, y = X[l].double(), Y[l].double().to(dev)
        if l == 0:
            D = torch.cat([x, -y], dim=3)
        elif l == L - 1:
            D = torch.cat([x, y], dim=0)
        else:
            a0, d, dp, a1 = x.shape
            b0, _, _, b1 = y.shape
            D = torch.zeros((a0 + b0, d, dp, a1 + b1), dtype=torch.float64, device=dev)
            D[:a0, :, :, :a1] = x
            D[a0:, :, :, a1:] = y
        if R is not None:
            D = torch.tensordot(R, D, dims=([1], [0]))
        if l == L - 1:
            return float(torch.linalg.norm(D))
        a0, d, dp, a1 = D.shape
        _, R = torch.linalg.qr(D.reshape(a0 * d * dp, a1))
