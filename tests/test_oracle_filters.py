"""Pins of Algorithm 2 and Algorithm 3 (oracle) against closed forms and identities."""
import numpy as np
import pytest

import workloads as wl
from oracle import filters
from oracle.chebyshev import scaled_cheb, affine, recurrence_coefficients


def _problem(m=60, seed=3):
    lam = np.sort(np.random.default_rng(seed).uniform(-1.0, 8.0, m))
    q = wl.orthogonal(m, seed + 1)
    return wl.dense_from_spectrum(q, lam), lam, q


def test_chfsi_filter_prescribed_spectrum():
    """C_p(A) X = Q diag(C_p(lambda)) Q^T X exactly (B = I)."""
    a, lam, q = _problem()
    X = np.random.default_rng(5).standard_normal((a.shape[0], 7))
    lmin, lT, lmax = lam[0] - 0.1, lam[10], lam[-1] + 0.2
    for p in (2, 5, 16):
        Y = filters.chfsi_filter(lambda v: a @ v, X, lmin, lT, lmax, p)
        ref = (q * scaled_cheb(p, lam, lmin, lT, lmax)[None, :]) @ (q.T @ X)
        np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("p", [2, 3, 9, 20])
def test_rchfsi_equals_chfsi_standard(p):
    """With D = B = I, Algorithm 3 reproduces Algorithm 2 for any X and diagonal Lambda
    (algebraic equivalence stated after Algorithm 3)."""
    a, lam, _ = _problem()
    rng = np.random.default_rng(11)
    X = rng.standard_normal((a.shape[0], 6))
    L = rng.uniform(-1, 3, 6)
    W = a @ X - X * L[None, :]
    lmin, lT, lmax = lam[0] - 0.1, lam[12], lam[-1] + 0.2
    Y3 = filters.rchfsi_filter(lambda r: a @ r, lambda r: r, X, L, W, lmin, lT, lmax, p)
    Y2 = filters.chfsi_filter(lambda v: a @ v, X, lmin, lT, lmax, p)
    np.testing.assert_allclose(Y3, Y2, rtol=0, atol=1e-11 * np.abs(Y2).max())


def test_rchfsi_equals_chfsi_generalized_exact_inverse():
    """B diagonal SPD and D = B: Algorithm 3 with A D^-1 equals Algorithm 2 with H = B^-1 A."""
    a, lam, _ = _problem(m=50, seed=7)
    rng = np.random.default_rng(13)
    bd = rng.uniform(0.5, 3.0, 50)
    X = rng.standard_normal((50, 5))
    L = rng.uniform(-0.5, 1.0, 5)
    W = a @ X - (bd[:, None] * X) * L[None, :]
    ev = np.linalg.eigvalsh(a / np.sqrt(bd)[:, None] / np.sqrt(bd)[None, :])
    lmin, lT, lmax = ev[0] - 0.1, ev[8], ev[-1] + 0.1
    Y3 = filters.rchfsi_filter(lambda r: a @ (r / bd[:, None]), lambda r: r / bd[:, None], X, L, W,
                               lmin, lT, lmax, 11)
    Y2 = filters.chfsi_filter(lambda v: (a @ v) / bd[:, None], X, lmin, lT, lmax, 11)
    np.testing.assert_allclose(Y3, Y2, rtol=0, atol=1e-11 * np.abs(Y2).max())


def test_rchfsi_fixed_point_any_D():
    """Exact eigenpairs give W = 0 and Y_p = X C_p(Lambda) whatever D^-1 is."""
    a, lam, q = _problem()
    X = q[:, :5]
    L = lam[:5]
    W = a @ X - X * L[None, :]
    dinv = np.random.default_rng(3).uniform(0.3, 2.0, a.shape[0])
    lmin, lT, lmax = lam[0] - 0.1, lam[9], lam[-1] + 0.2
    Y = filters.rchfsi_filter(lambda r: a @ (dinv[:, None] * r), lambda r: dinv[:, None] * r, X, L,
                              W, lmin, lT, lmax, 14)
    ref = X * scaled_cheb(14, L, lmin, lT, lmax)[None, :]
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def _shifted_chfsi(a, b, dinv, X, L, lmin, lT, lmax, p):
    """Independent derivation for D != B: Y'_k = D^-1 Z_k + X Lambda_k obeys
    Y'_{k+1} = a_k D^-1 A Y'_k + b_k Y'_k + c_k Y'_{k-1} + a_k (I - D^-1 B) X Lambda Lambda_k
    with Y'_0 = X, Y'_1 = (s1/e)(D^-1 A - c) X + (s1/e)(I - D^-1 B) X Lambda."""
    e, c, s1 = affine(lmin, lT, lmax)
    corr = X * L[None, :] - dinv @ (b @ X) * L[None, :]
    Yprev = X.copy()
    Ycur = (s1 / e) * (dinv @ (a @ X) - c * X) + (s1 / e) * corr
    Lprev = np.ones_like(L)
    Lcur = (s1 / e) * (L - c)
    for (ak, bk, ck) in recurrence_coefficients(lmin, lT, lmax, p):
        Ynew = ak * dinv @ (a @ Ycur) + bk * Ycur + ck * Yprev + ak * corr * Lcur[None, :]
        Lnew = ak * Lcur * L + bk * Lcur + ck * Lprev
        Yprev, Ycur, Lprev, Lcur = Ycur, Ynew, Lcur, Lnew
    return Ycur


@pytest.mark.parametrize("p", [2, 6, 15])
def test_rchfsi_inexact_inverse_matches_shifted_recurrence(p):
    """D^-1 != B^-1 (dense, non-symmetric perturbation allowed): Algorithm 3's output equals
    the shifted ChFSI recurrence with the correction term, derived from the inexact
    residual recurrence of Section 3.2.2."""
    rng = np.random.default_rng(21)
    m = 40
    a = wl.dense_from_spectrum(wl.orthogonal(m, 2), np.linspace(-1, 5, m))
    bq = wl.orthogonal(m, 4)
    b = wl.dense_from_spectrum(bq, np.linspace(1, 3, m))
    dinv = np.linalg.inv(b) + 0.05 * rng.standard_normal((m, m))
    X = rng.standard_normal((m, 4))
    L = rng.uniform(-1, 0.5, 4)
    W = a @ X - (b @ X) * L[None, :]
    lmin, lT, lmax = -1.5, 0.8, 9.0
    Y3 = filters.rchfsi_filter(lambda r: a @ (dinv @ r), lambda r: dinv @ r, X, L, W, lmin, lT, lmax, p)
    Ys = _shifted_chfsi(a, b, dinv, X, L, lmin, lT, lmax, p)
    np.testing.assert_allclose(Y3, Ys, rtol=0, atol=1e-10 * np.abs(Ys).max())


def test_complex_hermitian_equivalence():
    """Complex Hermitian A, B = I: Algorithm 3 equals Algorithm 2."""
    rng = np.random.default_rng(8)
    m = 30
    g = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    q, _ = np.linalg.qr(g)
    lam = np.linspace(-2, 4, m)
    a = (q * lam) @ q.conj().T
    a = 0.5 * (a + a.conj().T)
    X = rng.standard_normal((m, 4)) + 1j * rng.standard_normal((m, 4))
    L = rng.uniform(-2, 0, 4)
    W = a @ X - X * L[None, :]
    Y3 = filters.rchfsi_filter(lambda r: a @ r, lambda r: r, X, L, W, -2.1, 0.0, 4.2, 9)
    Y2 = filters.chfsi_filter(lambda v: a @ v, X, -2.1, 0.0, 4.2, 9)
    np.testing.assert_allclose(Y3, Y2, rtol=0, atol=1e-11 * np.abs(Y2).max())


def test_pins_catch_planted_mistakes(monkeypatch):
    """A plausible mistake planted in the oracle's Algorithm 3 (dropped W Lambda_Y term,
    sign error on c_k, Lambda update left out) is caught by the equivalence pin."""
    a, lam, _ = _problem()
    rng = np.random.default_rng(11)
    X = rng.standard_normal((a.shape[0], 6))
    L = rng.uniform(-1, 3, 6)
    W = a @ X - X * L[None, :]
    lmin, lT, lmax = lam[0] - 0.1, lam[12], lam[-1] + 0.2
    Y2 = filters.chfsi_filter(lambda v: a @ v, X, lmin, lT, lmax, 9)

    def mutant(kind):
        e, c, s1 = affine(lmin, lT, lmax)
        g, s = 2.0 / s1, s1
        RX, RY = np.zeros_like(W), (s1 / e) * W
        LX, LY = np.ones_like(L), (s1 / e) * (L - c)
        for _ in range(2, 10):
            s2 = 1.0 / (g - s)
            ak = 2 * s2 / e
            term = 0 if kind == "drop" else ak * W * LY[None, :]
            sgn = -1.0 if kind == "sign" else 1.0
            RX = ak * a @ RY - ak * c * RY - sgn * s * s2 * RX + term
            if kind != "lam":
                LX = ak * LY * L - ak * c * LY - s * s2 * LX
                LX, LY = LY, LX
            RX, RY = RY, RX
            s = s2
        return RY + X * LY[None, :]

    for kind in ("drop", "sign", "lam"):
        assert np.abs(mutant(kind) - Y2).max() > 1e-6 * np.abs(Y2).max(), kind
