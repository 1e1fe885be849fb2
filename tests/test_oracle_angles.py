"""Pins of the oracle's maximum principal angle (Definition 2.1) against closed forms.

The definition: tan angle(X, Y) = || X_perp^H Y (X^H Y)^+ ||_2 with orthonormal bases, and the
angle is pi/2 when X^H Y is rank deficient.  Each case below has a known answer, so a wrong
complement basis, a missing pseudo-inverse or a dropped conjugate fails one of them.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.angles import max_angle


def _e(n, i):
    v = np.zeros((n, 1))
    v[i] = 1.0
    return v


@pytest.mark.parametrize("t", [1e-6, 0.3, np.pi / 4, 1.2, np.pi / 2 - 1e-3])
def test_single_vector_rotated_by_t(t):
    """span{e1} against span{cos t e1 + sin t e2}: the angle is t (tan t above and below 1)."""
    n = 6
    x = _e(n, 0)
    y = np.cos(t) * _e(n, 0) + np.sin(t) * _e(n, 1)
    assert max_angle(x, y) == pytest.approx(t, rel=1e-10, abs=1e-12)
    assert max_angle(y, x) == pytest.approx(t, rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("t", [0.1, 0.7, 1.4])
def test_two_dimensional_subspaces_one_rotated_direction(t):
    """X = span{e1, e2}, Y = span{e1, cos t e2 + sin t e3}: principal angles 0 and t, maximum t."""
    n = 7
    X = np.hstack([_e(n, 0), _e(n, 1)])
    Y = np.hstack([_e(n, 0), np.cos(t) * _e(n, 1) + np.sin(t) * _e(n, 2)])
    assert max_angle(X, Y) == pytest.approx(t, rel=1e-10)


def test_basis_choice_does_not_matter():
    """Non-orthonormal, mixed bases of the same two subspaces give the same angle."""
    n, t = 8, 0.55
    X = np.hstack([_e(n, 0), _e(n, 1)])
    Y = np.hstack([_e(n, 0), np.cos(t) * _e(n, 1) + np.sin(t) * _e(n, 2)])
    rng = np.random.default_rng(3)
    M1 = rng.standard_normal((2, 2)) + 3 * np.eye(2)
    M2 = rng.standard_normal((2, 2)) + 3 * np.eye(2)
    assert max_angle(X @ M1, Y @ M2) == pytest.approx(t, rel=1e-10)


def test_orthogonal_directions_give_right_angle():
    """X^H Y rank deficient: span{e1} vs span{e2}, and a 2-D pair sharing only one direction."""
    n = 5
    assert max_angle(_e(n, 0), _e(n, 1)) == pytest.approx(np.pi / 2)
    X = np.hstack([_e(n, 0), _e(n, 1)])
    Y = np.hstack([_e(n, 0), _e(n, 2)])
    assert max_angle(X, Y) == pytest.approx(np.pi / 2)


def test_identical_subspaces_give_zero():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((30, 4))
    Y = X @ (rng.standard_normal((4, 4)) + 4 * np.eye(4))
    assert max_angle(X, Y) <= 1e-12


@pytest.mark.parametrize("t", [0.2, 1.0])
def test_complex_rotation_uses_the_conjugate(t):
    """span{e1} against span{cos t e1 + i sin t e2} in C^n: the angle is t (a missing conjugate
    in X^H Y would still give t here, so the second case puts the phase on the shared direction:
    span{e1} vs span{i cos t e1 + sin t e2} is also t)."""
    n = 4
    x = _e(n, 0).astype(complex)
    y1 = np.cos(t) * _e(n, 0) + 1j * np.sin(t) * _e(n, 1)
    y2 = 1j * np.cos(t) * _e(n, 0) + np.sin(t) * _e(n, 1)
    assert max_angle(x, y1) == pytest.approx(t, rel=1e-10)
    assert max_angle(x, y2) == pytest.approx(t, rel=1e-10)
    # a complex 2-D pair: X = span{e1, e2}, Y = span{e1, (cos t) e2 + (i sin t) e3}
    X = np.hstack([_e(n, 0), _e(n, 1)]).astype(complex)
    Y = np.hstack([_e(n, 0), np.cos(t) * _e(n, 1) + 1j * np.sin(t) * _e(n, 2)])
    assert max_angle(X, Y) == pytest.approx(t, rel=1e-10)


def test_random_subspaces_match_svd_principal_angles():
    """Against the SVD definition of principal angles (LAPACK through scipy), on random subspaces of
    equal dimension where X^H Y has full rank."""
    rng = np.random.default_rng(11)
    for n, q in ((20, 3), (50, 7), (12, 6)):
        X = rng.standard_normal((n, q))
        Y = X + 0.4 * rng.standard_normal((n, q))
        ref = float(np.max(sla.subspace_angles(X, Y)))
        assert max_angle(X, Y) == pytest.approx(ref, rel=1e-9)
