"""Chebyshev polynomials, the affine map and the sigma-scaled recurrence coefficients.

Section 2.1: L(x) = (x - c)/e with c = (lmax + lT)/2, e = (lmax - lT)/2;
C_k(x) = T_k(L(x)) / T_k(L(a_low)) with a_low = lmin.  The scaled recurrence uses
sigma_1 = e / (lmin - c), sigma_{k+1} = 1 / (2/sigma_1 - sigma_k) and, for k >= 1,
    a_k = 2 sigma_{k+1} / e,   b_k = -2 sigma_{k+1} c / e,   c_k = -sigma_k sigma_{k+1}
(definitions following the inexact ChFSI recurrence in Section 3.2.1).
"""
import numpy as np


def affine(lmin, lT, lmax):
    """(e, c, sigma_1) of the first line of Algorithms 2 and 3."""
    e = 0.5 * (lmax - lT)
    c = 0.5 * (lmax + lT)
    sigma1 = e / (lmin - c)
    return e, c, sigma1


def recurrence_coefficients(lmin, lT, lmax, p):
    """[(a_k, b_k, c_k) for k = 1..p-1]: the step that produces degree k+1 from k and k-1.

    Algorithms 2/3 run their loop for k = 2..p with sigma_2 <- 1/(gamma - sigma); entry
    j of this list (j = 0..p-2) is that loop's iteration producing degree j + 2.
    """
    e, c, sigma1 = affine(lmin, lT, lmax)
    gamma = 2.0 / sigma1
    sigma = sigma1
    out = []
    for _ in range(2, p + 1):
        sigma2 = 1.0 / (gamma - sigma)
        out.append((2.0 * sigma2 / e, -2.0 * sigma2 * c / e, -sigma * sigma2))
        sigma = sigma2
    return out


def cheb_T(k, x):
    """T_k(x) in closed form: cos(k acos x) on [-1,1], cosh(k acosh x) for x > 1,
    (-1)^k cosh(k acosh(-x)) for x < -1."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(k * np.arccos(x[inside]))
    hi = x > 1.0
    out[hi] = np.cosh(k * np.arccosh(x[hi]))
    lo = x < -1.0
    out[lo] = (-1.0) ** k * np.cosh(k * np.arccosh(-x[lo]))
    return out


def scaled_cheb(k, x, lmin, lT, lmax):
    """C_k(x) = T_k(L(x)) / T_k(L(lmin))."""
    e, c, _ = affine(lmin, lT, lmax)
    return cheb_T(k, (np.asarray(x) - c) / e) / cheb_T(k, np.array([(lmin - c) / e]))[0]
