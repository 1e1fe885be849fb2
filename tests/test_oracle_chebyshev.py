"""Pins of the Chebyshev scalars (Section 2.1; a_k, b_k, c_k of Section 3.2.1) against
closed forms that do not use the recurrence."""
import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

from oracle import chebyshev as ch
from oracle.filters import lambda_p

pytestmark = pytest.mark.filterwarnings("ignore")


def test_cheb_T_matches_library_series():
    x = np.concatenate([np.linspace(-3.0, -1.0001, 7), np.linspace(-1, 1, 11), np.linspace(1.0001, 3, 7)])
    for k in range(0, 13):
        coef = np.zeros(k + 1)
        coef[k] = 1.0
        ref = npc.chebval(x, coef)
        np.testing.assert_allclose(ch.cheb_T(k, x), ref, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("bounds", [(-1.2, 0.5, 10.3), (0.95, 4.5, 202.9), (-5.0, -4.0, 1.0)])
@pytest.mark.parametrize("p", [1, 2, 3, 8, 20, 31])
def test_lambda_recurrence_equals_closed_form(bounds, p):
    """Lambda_p from the recurrence of Proposition 3.3 equals T_p(L(lam))/T_p(L(lmin))."""
    lmin, lT, lmax = bounds
    lam = np.concatenate([np.linspace(lmin, lT, 9), np.linspace(lT, lmax, 9)])
    got = lambda_p(lam, lmin, lT, lmax, p)
    ref = ch.scaled_cheb(p, lam, lmin, lT, lmax)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


def test_normalisation_at_lmin_and_bounded_on_unwanted():
    lmin, lT, lmax = -1.0, 2.0, 9.0
    for p in (4, 10, 25):
        assert abs(lambda_p(np.array([lmin]), lmin, lT, lmax, p)[0] - 1.0) < 1e-13
        cu = lambda_p(np.linspace(lT, lmax, 50), lmin, lT, lmax, p)
        ref_bound = 1.0 / abs(ch.cheb_T(p, np.array([(lmin - 0.5 * (lmax + lT)) / (0.5 * (lmax - lT))]))[0])
        assert np.abs(cu).max() <= ref_bound * (1 + 1e-12)


def test_coefficients_reproduce_scalar_polynomials():
    """C_{k+1}(x) = a_k x C_k(x) + b_k C_k(x) + c_k C_{k-1}(x) with the returned triples."""
    lmin, lT, lmax, p = -0.7, 1.3, 6.1, 12
    x = np.linspace(-2.0, 7.0, 41)
    e, c, s1 = ch.affine(lmin, lT, lmax)
    Cprev = np.ones_like(x)
    Ccur = (s1 / e) * (x - c)
    for k, (a, b, cc) in enumerate(ch.recurrence_coefficients(lmin, lT, lmax, p), start=1):
        Cprev, Ccur = Ccur, a * x * Ccur + b * Ccur + cc * Cprev
        np.testing.assert_allclose(Ccur, ch.scaled_cheb(k + 1, x, lmin, lT, lmax), rtol=1e-11,
                                   atol=1e-13)
