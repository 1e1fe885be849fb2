"""Algorithm 2 (ChFSI filter) and Algorithm 3 (R-ChFSI filter), step by step in FP64.

Operators are passed as callables so that a test can inject an inexact product (a
perturbed matrix, an approximate inverse, rounded inputs):
    H(Y)      the filter operator of Algorithm 2 (H = B^-1 A, or D^-1 A when inexact)
    AD(R)     the product A D^-1 R of Algorithm 3's loop
    Dinv(R)   D^-1 R used by the final reconstruction of Algorithm 3
"""
import numpy as np

from .chebyshev import affine


def chfsi_filter(H, X, lmin, lT, lmax, p):
    """Algorithm 2: Y_p = C_p(H) X by the sigma-scaled three-term recurrence."""
    e, c, sigma1 = affine(lmin, lT, lmax)
    gamma = 2.0 / sigma1
    sigma = sigma1
    Xk = np.array(X, copy=True)
    Yk = (sigma1 / e) * (H(X) - c * X)
    for _ in range(2, p + 1):
        sigma2 = 1.0 / (gamma - sigma)
        Xk = (2.0 * sigma2 / e) * H(Yk) - (2.0 * sigma2 / e) * c * Yk - sigma * sigma2 * Xk
        Xk, Yk = Yk, Xk
        sigma = sigma2
    return Yk


def rchfsi_filter(AD, Dinv, X, lam, W, lmin, lT, lmax, p, return_state=False):
    """Algorithm 3 (R-ChFSI filter).

    X     (m, n) current Ritz vectors X^(i)
    lam   (n,)   current Ritz values (the diagonal of Lambda^(i))
    W     (m, n) the residual A X - B X Lambda (the algorithm's input "Y")
    Returns Y_p = D^-1 R_Y + X Lambda_Y.  With return_state the final (R_Y, Lambda_Y)
    are returned too.
    """
    e, c, sigma1 = affine(lmin, lT, lmax)
    gamma = 2.0 / sigma1
    sigma = sigma1
    lam = np.asarray(lam, dtype=np.float64)
    RX = np.zeros_like(W)
    RY = (sigma1 / e) * W
    LX = np.ones_like(lam)
    LY = (sigma1 / e) * (lam - c)
    for _ in range(2, p + 1):
        sigma2 = 1.0 / (gamma - sigma)
        a = 2.0 * sigma2 / e
        RX = a * AD(RY) - a * c * RY - sigma * sigma2 * RX + a * W * LY[None, :]
        LX = a * LY * lam - a * c * LY - sigma * sigma2 * LX
        RX, RY = RY, RX
        LX, LY = LY, LX
        sigma = sigma2
    Yp = Dinv(RY) + X * LY[None, :]
    if return_state:
        return Yp, RY, LY
    return Yp


def lambda_p(lam, lmin, lT, lmax, p):
    """Lambda_p = C_p(Lambda) by the eigenvalue recurrence of Proposition 3.3
    (Lambda_0 = I, Lambda_1 = (sigma_1/e)(Lambda - cI))."""
    e, c, sigma1 = affine(lmin, lT, lmax)
    gamma = 2.0 / sigma1
    sigma = sigma1
    lam = np.asarray(lam, dtype=np.float64)
    LX = np.ones_like(lam)
    LY = (sigma1 / e) * (lam - c)
    for _ in range(2, p + 1):
        sigma2 = 1.0 / (gamma - sigma)
        a = 2.0 * sigma2 / e
        LX = a * LY * lam - a * c * LY - sigma * sigma2 * LX
        LX, LY = LY, LX
        sigma = sigma2
    return LY
