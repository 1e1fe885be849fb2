"""k-step Lanczos estimates of spectral bounds.

The paper only asks for estimates of lmax (Section 2.1).  Reading used here: run k
steps of the three-term Lanczos process (no re-orthogonalisation) on the symmetric
operator S = D^-1/2 A D^-1/2, which is similar to the filter operators D^-1 A and
A D^-1, from the unit start vector v0; the upper bound is theta_max(T_k) + beta_k.
"""
import numpy as np


def lanczos_tridiag(S, v0, k):
    """Returns (alpha[0:k], beta[0:k]) of the Lanczos process for the callable S."""
    v = v0 / np.linalg.norm(v0)
    v_prev = np.zeros_like(v)
    alpha = np.zeros(k)
    beta = np.zeros(k)
    b_prev = 0.0
    for j in range(k):
        w = S(v)
        alpha[j] = np.real(np.vdot(v, w))
        w = w - alpha[j] * v - b_prev * v_prev
        beta[j] = np.linalg.norm(w)
        v_prev, v = v, w / beta[j]
        b_prev = beta[j]
    return alpha, beta


def ritz_values(alpha, beta):
    k = len(alpha)
    T = np.diag(alpha) + np.diag(beta[: k - 1], 1) + np.diag(beta[: k - 1], -1)
    return np.linalg.eigvalsh(T)


def upper_bound(A, dinv_diag, v0, k=10):
    """theta_max + beta_k for S = D^-1/2 A D^-1/2 (dinv_diag = None means D = I)."""
    if dinv_diag is None:
        S = A
    else:
        s = np.sqrt(dinv_diag)
        S = lambda v: s * A(s * v)  # noqa: E731
    alpha, beta = lanczos_tridiag(S, v0, k)
    return ritz_values(alpha, beta)[-1] + beta[-1]


def norm_estimate(A, v0, k=10):
    """||A||_2 estimate max(|theta_min|, |theta_max|) from k Lanczos steps on A."""
    alpha, beta = lanczos_tridiag(A, v0, k)
    th = ritz_values(alpha, beta)
    return max(abs(th[0]), abs(th[-1]))
