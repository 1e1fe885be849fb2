"""Pins of the oracle's Rayleigh-Ritz, residual and Lanczos bound."""
import numpy as np
import scipy.linalg as sla

import workloads as wl
from oracle import rr, lanczos


def _pencil(m=40, seed=2):
    q = wl.orthogonal(m, seed)
    lam = np.linspace(-1.0, 6.0, m)
    b = wl.dense_from_spectrum(q, np.linspace(1.0, 5.0, m))
    a = wl.dense_from_spectrum(q, lam * np.linspace(1.0, 5.0, m))
    return a, b, lam, q      # shared eigenbasis: generalized eigenvalues are exactly lam


def test_rr_b_orthonormal_and_rayleigh_quotients():
    a, b, lam, _ = _pencil()
    Y = np.random.default_rng(1).standard_normal((40, 9))
    X, eps, AX, BX = rr.rayleigh_ritz(Y, lambda v: a @ v, lambda v: b @ v)
    np.testing.assert_allclose(X.T @ b @ X, np.eye(9), atol=1e-12)
    np.testing.assert_allclose(np.diag(X.T @ a @ X), eps, atol=1e-12)
    np.testing.assert_allclose(AX, a @ X, atol=1e-11)
    np.testing.assert_allclose(BX, b @ X, atol=1e-11)
    assert np.all(np.diff(eps) >= 0)
    # Courant-Fischer: the j-th Ritz value is >= the j-th eigenvalue
    assert np.all(eps >= lam[:9] - 1e-12)


def test_rr_invariant_subspace_gives_exact_eigenvalues():
    """Y spanning an invariant subspace (mixed by a random nonsingular G) gives the exact
    generalized eigenvalues and zero residual."""
    a, b, lam, q = _pencil()
    idx = np.array([0, 3, 4, 7, 11])
    Y = q[:, idx] @ np.random.default_rng(2).standard_normal((5, 5))
    X, eps, AX, BX = rr.rayleigh_ritz(Y, lambda v: a @ v, lambda v: b @ v)
    np.testing.assert_allclose(eps, lam[idx], atol=1e-12)
    W, r = rr.residual(AX, BX, eps)
    assert r.max() < 1e-11


def test_rr_full_space_is_dense_generalized_eig():
    """Subspace = whole space: Ritz values are all generalized eigenvalues (closed form)."""
    a, b, lam, _ = _pencil(m=30)
    Y = np.random.default_rng(4).standard_normal((30, 30))
    _, eps, _, _ = rr.rayleigh_ritz(Y, lambda v: a @ v, lambda v: b @ v)
    np.testing.assert_allclose(eps, lam, atol=1e-10)


def test_rr_complex_hermitian():
    rng = np.random.default_rng(3)
    m = 24
    g = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    q, _ = np.linalg.qr(g)
    lam = np.linspace(-3, 3, m)
    a = (q * lam) @ q.conj().T
    Y = q[:, :4] @ (rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
    X, eps, _, _ = rr.rayleigh_ritz(Y, lambda v: a @ v, lambda v: v)
    np.testing.assert_allclose(eps, lam[:4], atol=1e-12)
    np.testing.assert_allclose(X.conj().T @ X, np.eye(4), atol=1e-12)


def test_lanczos_upper_bound_and_full_run():
    m = 20
    q = wl.orthogonal(m, 9)
    lam = np.linspace(-2.0, 7.5, m)
    a = wl.dense_from_spectrum(q, lam)
    v0 = np.random.default_rng(1).standard_normal(m)
    for k in (3, 6, 10):
        assert lanczos.upper_bound(lambda v: a @ v, None, v0, k) >= lam[-1] - 1e-12
        assert lanczos.norm_estimate(lambda v: a @ v, v0, k) <= 7.5 + 1e-12
    al, be = lanczos.lanczos_tridiag(lambda v: a @ v, v0, m)
    th = lanczos.ritz_values(al, be)
    np.testing.assert_allclose(th[[0, -1]], lam[[0, -1]], atol=1e-9)


def test_lanczos_scaled_operator_matches_similar_matrix():
    """With diagonal D the bound is for the spectrum of D^-1 A (similar to D^-1/2 A D^-1/2)."""
    m = 25
    a = wl.dense_from_spectrum(wl.orthogonal(m, 3), np.linspace(0.5, 4.0, m))
    d = np.random.default_rng(2).uniform(0.5, 2.0, m)
    ev = np.sort(np.real(np.linalg.eigvals(d[:, None] * a)))
    v0 = np.ones(m)
    assert lanczos.upper_bound(lambda v: a @ v, d, v0, 8) >= ev[-1] - 1e-12
    al, be = lanczos.lanczos_tridiag(lambda v: np.sqrt(d) * (a @ (np.sqrt(d) * v)), v0, m)
    np.testing.assert_allclose(lanczos.ritz_values(al, be)[-1], ev[-1], rtol=1e-9)
    np.testing.assert_allclose(sla.eigvalsh(a, np.diag(1 / d))[-1], ev[-1], rtol=1e-9)
