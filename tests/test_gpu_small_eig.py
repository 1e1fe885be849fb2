"""This library's small dense FP64 kernels of the Rayleigh-Ritz step (Section 2.1, Algorithm 1):
Cholesky with L^-1, Householder tridiagonalisation, bisection and inverse iteration
(eig_mode="tridiag").  Ritz pairs are compared with the oracle's (LAPACK) on the same inputs."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import rr
from gpu_helpers import ensure_built, dense_case, make_solver, relfro

from paper_2503_22652_gb300 import Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    ensure_built()


def _check_rr(A, Bm, Y, X, ev, rtol=1e-11, vec_tol=1e-9):
    Xr, evr, _, _ = rr.rayleigh_ritz(Y, lambda v: A @ v, lambda v: Bm @ v)
    np.testing.assert_allclose(ev, evr, rtol=rtol, atol=rtol * np.abs(evr).max())
    assert np.all(np.diff(ev) >= 0)
    N = Y.shape[1]
    np.testing.assert_allclose(X.T @ Bm @ X, np.eye(N), atol=1e-11)
    # projected A is diagonal in the returned basis (Ritz vectors, any rotation inside clusters)
    np.testing.assert_allclose(X.T @ A @ X, np.diag(ev), atol=1e-10 * np.abs(ev).max())
    return Xr, evr


# (m, N): N = 1, 2, 3 edge cases; 36 and 240 on the thread-block-cluster path; 480 and 1100 on the
# cooperative-grid path
@pytest.mark.parametrize("m,N,gen", [(50, 1, False), (60, 2, True), (70, 3, False), (280, 36, True),
                                     (900, 240, True), (700, 480, True), (1300, 1100, False)])
def test_rayleigh_ritz_tridiag_parity(m, N, gen):
    case = dense_case(m=m, N=N, generalized=gen)
    Bm = case["B"] if gen else np.eye(m)
    s = make_solver(case, N, eig_mode="tridiag")
    X, ev = s.rayleigh_ritz(case["X"])
    Xr, evr = _check_rr(case["A"], Bm, case["X"], X, ev)
    sg = np.sign(np.sum(X * (Bm @ Xr), axis=0))
    assert relfro(X * sg[None, :], Xr) <= 1e-8


def test_rayleigh_ritz_tridiag_degenerate():
    """Ritz values with exact multiplicities (subspace spanned by eigenvectors of a matrix with a
    multiplicity-8 and a multiplicity-3 eigenvalue): inverse iteration with Gram-Schmidt inside
    the clusters still returns an orthonormal basis of Ritz vectors."""
    m, N = 300, 40
    rng = np.random.default_rng(41)
    lam = np.sort(rng.uniform(-1.0, 9.0, m))
    lam[5:13] = lam[5]
    lam[20:23] = lam[20]
    Q = wl.orthogonal(m, 42)
    A = wl.dense_from_spectrum(Q, lam)
    Y = Q[:, :N] @ rng.standard_normal((N, N))
    s = Solver(m, nev=N // 2, block=N, eig_mode="tridiag")
    s.set_dense(A)
    X, ev = s.rayleigh_ritz(Y)
    np.testing.assert_allclose(ev, lam[:N], rtol=1e-11, atol=1e-11 * np.abs(lam[:N]).max())
    np.testing.assert_allclose(X.T @ X, np.eye(N), atol=1e-11)
    R = A @ X - X * ev[None, :]
    assert np.linalg.norm(R, axis=0).max() <= 1e-10 * np.abs(lam).max()


def test_rayleigh_ritz_tridiag_complex():
    """Complex Hermitian problem: the embedded projected matrix has every eigenvalue twice."""
    m, N = 200, 24
    rng = np.random.default_rng(43)
    Z = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    A = 0.5 * (Z + Z.conj().T)
    Y = rng.standard_normal((m, N)) + 1j * rng.standard_normal((m, N))
    s = Solver(m, nev=N // 2, block=N, field="complex", eig_mode="tridiag")
    s.set_dense(A)
    X, ev = s.rayleigh_ritz(Y)
    _, evr, _, _ = rr.rayleigh_ritz(Y, lambda v: A @ v, lambda v: v)
    np.testing.assert_allclose(ev, evr, rtol=1e-10, atol=1e-10 * np.abs(evr).max())
    np.testing.assert_allclose(X.conj().T @ X, np.eye(N), atol=1e-10)
    np.testing.assert_allclose(X.conj().T @ A @ X, np.diag(ev), atol=1e-9 * np.abs(ev).max())


@pytest.mark.parametrize("precision", ["tf32", "fp64"])
def test_solve_tridiag_dense_generalized(precision):
    m = 600
    c = wl.dense_config2(m=m)
    ref = sla.eigh(c["A"], c["B"], eigvals_only=True)[:30]
    s = Solver(m, nev=30, block=40, degree=30, precision=precision, max_iter=200, eig_mode="tridiag")
    s.set_dense(c["A"], B=c["B"], Dinv=c["Dinv"])
    X, ev, res, st = s.solve(wl.gaussian_block(m, 40, seed=2))
    assert st["max_rel_residual"] <= 1e-8
    np.testing.assert_allclose(ev[:30], ref, atol=1e-9 * np.abs(ref).max())


def test_solve_tridiag_fe():
    p = wl.fe_problem(3)
    from oracle import fe as ofe
    A = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"]).toarray()
    B = ofe.assemble(p["cell_dofs"], p["B_cell"], p["m"]).toarray()
    ref = sla.eigh(A, B, eigvals_only=True)[:7]
    s = Solver(p["m"], nev=7, block=12, degree=20, precision="tf32", max_iter=150, eig_mode="tridiag")
    s.set_fe(p["cell_dofs"], p["A_cells"], p["B_cell"], p["Dinv"])
    X, ev, res, st = s.solve(wl.gaussian_block(p["m"], 12, seed=2))
    assert st["max_rel_residual"] <= 1e-8
    np.testing.assert_allclose(ev[:7], ref, atol=1e-9 * np.abs(ref).max())


def test_rayleigh_ritz_syevd_parity():
    """The library eigensolver (cuSOLVER dsyevd) stays available as eig_mode="syevd"."""
    case = dense_case(m=280, N=36, generalized=True)
    s = make_solver(case, 36, eig_mode="syevd")
    X, ev = s.rayleigh_ritz(case["X"])
    _check_rr(case["A"], case["B"], case["X"], X, ev)


@pytest.mark.parametrize("N", [7, 40, 240])
def test_rayleigh_ritz_tridiag_exact_diagonal(N):
    """An exactly diagonal projected matrix (integer spectrum, Y = unit vectors): every Householder
    step has nothing to annihilate (tau = 0), and Sturm minors of trial points that hit an integer
    are exactly zero, the case the check-free Sturm count hands to the substituting recount.  The
    Ritz values are the integers to a few ulps."""
    m = N + 13
    lam = np.arange(m, dtype=np.float64)[::-1] - 3.0          # ..., -2, -3, descending on the diagonal
    A = np.diag(lam)
    Y = np.eye(m)[:, :N]
    s = Solver(m, nev=max(1, N // 2), block=N, eig_mode="tridiag")
    s.set_dense(A)
    X, ev = s.rayleigh_ritz(Y)
    want = np.sort(lam[:N])
    # the multisection interval closes to a few ulps around each integer
    np.testing.assert_allclose(ev, want, rtol=0, atol=8 * np.finfo(float).eps * np.abs(lam).max())
    np.testing.assert_allclose(np.abs(X.T @ X), np.eye(N), atol=1e-14)
    np.testing.assert_allclose(X.T @ A @ X, np.diag(ev), atol=1e-13 * np.abs(lam).max())
