"""Algorithm 1 (subspace iteration accelerated by a Chebyshev filter) in FP64.

The filter is either Algorithm 2 (ChFSI, operator D^-1 A) or Algorithm 3 (R-ChFSI,
operator A D^-1 and residual input).  Readings where the paper is silent:
  * initial guess: the caller's X0, followed by one Rayleigh-Ritz step so that X is
    B-orthonormal with Ritz values before the first filter;
  * bounds: lmax from the Lanczos estimate (or prescribed); lmin = eps_1 and
    lT = eps_N, the smallest and largest current Ritz values (or prescribed);
  * convergence: max over the first nev columns of ||A x_j - eps_j B x_j|| /
    (||A|| ||x_j||) <= tol, tested before each filter; the absolute residuals of the
    paper are returned too.
"""
import numpy as np

from .filters import chfsi_filter, rchfsi_filter
from .rr import rayleigh_ritz, residual, column_norms


def solve(A, B, X0, nev, p, tol, max_iter, lmax, normA, method="rchfsi",
          A_filter=None, Dinv=None, bounds=None, min_iter=0):
    """A, B, A_filter, Dinv: callables (A_filter defaults to A, Dinv to identity).

    Returns dict(X, eps, rel, abs, iters, history_rel, history_abs).
    bounds: optional fixed (lmin, lT, lmax); otherwise Ritz-value bounds and `lmax`.
    """
    Af = A if A_filter is None else A_filter
    Di = (lambda R: R) if Dinv is None else Dinv
    AD = lambda R: Af(Di(R))   # noqa: E731  A D^-1 (Algorithm 3)
    H = lambda Y: Di(Af(Y))    # noqa: E731  D^-1 A (Algorithm 2)
    X, eps, AX, BX = rayleigh_ritz(X0, A, B)
    hist_rel, hist_abs = [], []
    it = 0
    while True:
        W, r = residual(AX, BX, eps)
        rel = r / (normA * column_norms(X))
        hist_rel.append(rel[:nev].max())
        hist_abs.append(r[:nev].max())
        if (hist_rel[-1] <= tol and it >= min_iter) or it >= max_iter:
            break
        if bounds is None:
            lmin, lT, lmx = eps[0], eps[-1], lmax
        else:
            lmin, lT, lmx = bounds
        if method == "rchfsi":
            Y = rchfsi_filter(AD, Di, X, eps, W, lmin, lT, lmx, p)
        elif method == "chfsi":
            Y = chfsi_filter(H, X, lmin, lT, lmx, p)
        else:
            raise ValueError(method)
        X, eps, AX, BX = rayleigh_ritz(Y, A, B)
        it += 1
    return {"X": X, "eps": eps, "rel": rel, "abs": r, "iters": it,
            "history_rel": np.array(hist_rel), "history_abs": np.array(hist_abs)}
