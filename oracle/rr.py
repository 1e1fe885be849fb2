"""Rayleigh-Ritz projection for a non-orthogonal basis and the eigen-residual.

Section 2.1 / Algorithm 1 steps 2-3: solve Y^H A Y E = Y^H B Y E Lambda for the Ritz
values (ascending) and set X = Y E, which is B-orthonormal.  The columns of Y are first
scaled to unit 2-norm (the span, hence the Ritz pairs, is unchanged) to keep the Gram
matrices well scaled.  The small dense pencil is solved by LAPACK (scipy.linalg.eigh),
which normalises E so that E^H (Y^H B Y) E = I.
"""
import numpy as np
import scipy.linalg as sla


def column_norms(Y):
    return np.sqrt(np.sum(np.abs(Y) ** 2, axis=0))


def rayleigh_ritz(Y, A, B):
    """Returns (X, eps, AX, BX).  A and B are callables applying the exact operators."""
    Ys = Y / column_norms(Y)[None, :]
    AY = A(Ys)
    BY = B(Ys)
    GA = Ys.conj().T @ AY
    GB = Ys.conj().T @ BY
    GA = 0.5 * (GA + GA.conj().T)
    GB = 0.5 * (GB + GB.conj().T)
    eps, E = sla.eigh(GA, GB)
    return Ys @ E, eps, AY @ E, BY @ E


def residual(AX, BX, eps):
    """W = A X - B X diag(eps) and its column 2-norms r_j."""
    W = AX - BX * eps[None, :]
    return W, column_norms(W)
