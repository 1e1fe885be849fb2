"""Parity of the FP64 building blocks (residual, Rayleigh-Ritz, Lanczos) and of full solves with
the oracle, through the C ABI."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import rr, lanczos, solver as osolver
from gpu_helpers import ensure_built, dense_case, make_solver, relfro

from paper_2503_22652_gb300 import Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    ensure_built()


def test_residual_parity():
    case = dense_case(m=300, N=30, generalized=True)
    s = make_solver(case, 30)
    W, r = s.residual(case["X"], case["L"])
    Wref, rref = rr.residual(case["A"] @ case["X"], case["B"] @ case["X"], case["L"])
    assert relfro(W, Wref) <= 1e-13
    np.testing.assert_allclose(r, rref, rtol=1e-12)


@pytest.mark.parametrize("gen", [False, True])
def test_rayleigh_ritz_parity(gen):
    case = dense_case(m=280, N=36, generalized=gen)
    Bm = case["B"] if gen else np.eye(280)
    Y = case["X"]
    s = make_solver(case, 36)
    X, ev = s.rayleigh_ritz(Y)
    Xr, evr, _, _ = rr.rayleigh_ritz(Y, lambda v: case["A"] @ v, lambda v: Bm @ v)
    np.testing.assert_allclose(ev, evr, rtol=1e-11, atol=1e-11 * np.abs(evr).max())
    # B-orthonormal, and each Ritz vector equals the oracle's up to sign
    np.testing.assert_allclose(X.T @ Bm @ X, np.eye(36), atol=1e-11)
    sg = np.sign(np.sum(X * (Bm @ Xr), axis=0))
    assert relfro(X * sg[None, :], Xr) <= 1e-9


def test_lanczos_parity():
    case = dense_case(m=400, N=8, generalized=True)
    s = make_solver(case, 8)
    v0 = np.random.default_rng(1).standard_normal(400)
    lmax, nA = s.lanczos_bounds(v0, 10)
    A = lambda v: case["A"] @ v  # noqa: E731
    assert abs(lmax - lanczos.upper_bound(A, case["Dinv"], v0, 10)) <= 1e-10 * abs(lmax)
    assert abs(nA - lanczos.norm_estimate(A, v0, 10)) <= 1e-10 * abs(nA)


def _cfg1_solver(precision, m=1000):
    c = wl.dense_config1(m=m)
    s = Solver(m, nev=50, block=60, degree=20, precision=precision, max_iter=60)
    s.set_dense(c["A"])
    return c, s


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32", "bf16"])
def test_solve_config1_all_precisions(precision):
    """Standard problem, m = 1000, nev = 50, block 60, degree 20: every precision reaches the
    1e-8 relative residual with eigenvalues within 1e-9 of the prescribed spectrum."""
    c, s = _cfg1_solver(precision)
    X0 = wl.gaussian_block(1000, 60, seed=2)
    X, ev, res, st = s.solve(X0)
    assert st["max_rel_residual"] <= 1e-8
    lam = c["lam"][:50]
    scale = np.maximum(np.abs(lam), 1e-2 * (c["lam"][-1] - c["lam"][0]))
    assert np.all(np.abs(ev[:50] - lam) <= 1e-9 * scale)
    # independent residual check on the host
    R = c["A"] @ X[:, :50] - X[:, :50] * ev[:50][None, :]
    rel = np.linalg.norm(R, axis=0) / (st["normA"] * np.linalg.norm(X[:, :50], axis=0))
    assert rel.max() <= 1.5e-8


def test_solve_matches_oracle_iterates():
    """FP64 R-ChFSI on the GPU follows the oracle's iteration (same bounds, same history)."""
    m, N = 400, 24
    c = wl.dense_config2(m=m)
    X0 = wl.gaussian_block(m, N, seed=2)
    s = Solver(m, nev=20, block=N, degree=12, precision="fp64", max_iter=12, min_iter=12, tol=0.0)
    s.set_dense(c["A"], B=c["B"], Dinv=c["Dinv"])
    X, ev, res, st = s.solve(X0, allow_not_converged=True)
    A = lambda v: c["A"] @ v  # noqa: E731
    Bf = lambda v: c["B"] @ v  # noqa: E731
    D = lambda v: c["Dinv"][:, None] * v  # noqa: E731
    lmax = lanczos.upper_bound(A, c["Dinv"], X0[:, 0], 10)
    nA = lanczos.norm_estimate(A, X0[:, 0], 10)
    ref = osolver.solve(A, Bf, X0, 20, 12, 0.0, 12, lmax, nA, Dinv=D)
    np.testing.assert_allclose(st["lmax"], lmax, rtol=1e-10)
    np.testing.assert_allclose(ev, ref["eps"], rtol=1e-9, atol=1e-12)
    h = st["history"]
    np.testing.assert_allclose(h[:6], ref["history_rel"][:6], rtol=1e-4)


def test_solve_generalized_dense_bruteforce():
    """Dense generalized problem (m = 600, nev = 30) with D^-1 = diag(B)^-1: TF32 R-ChFSI reaches
    the tolerance with eigenvalues equal to the dense generalized eigensolver's."""
    m = 600
    c = wl.dense_config2(m=m)
    ref = sla.eigh(c["A"], c["B"], eigvals_only=True)[:30]
    X0 = wl.gaussian_block(m, 40, seed=2)
    for prec in ("fp64", "tf32"):
        s = Solver(m, nev=30, block=40, degree=30, precision=prec, max_iter=200)
        s.set_dense(c["A"], B=c["B"], Dinv=c["Dinv"])
        X, ev, res, st = s.solve(X0)
        assert st["max_rel_residual"] <= 1e-8
        np.testing.assert_allclose(ev[:30], ref, atol=1e-9 * np.abs(ref).max())


def test_chfsi_stagnates_where_rchfsi_converges():
    """Section 4.1.3 behaviour on the GPU: with D^-1 = B^-1 + zeta E (zeta = 1e-3) ChFSI stalls
    at O(zeta) while R-ChFSI converges."""
    t = wl.toy_generalized(1e-3, m=600, n=10)
    X0 = wl.gaussian_block(600, 10, seed=2)
    out = {}
    for meth in ("chfsi", "rchfsi"):
        s = Solver(600, nev=10, block=10, degree=8, method=meth, max_iter=40, min_iter=40, tol=0.0,
                   bounds=(t["lmin"], t["lT"], t["lmax"]))
        s.set_dense(t["A"], B=t["B"], Dinv_dense=t["Dinv_dense"])
        _, _, _, st = s.solve(X0, allow_not_converged=True)
        out[meth] = st["max_abs_residual"]
    assert out["chfsi"] > 1e-5
    assert out["rchfsi"] < 1e-11


def test_solve_inplace_block_matches_copy():
    """solve(..., inplace=True) uses the caller's host array as the rchfsi_solve in/out block: the
    same Ritz pairs as the copying call, written into that array."""
    case = dense_case(m=300, N=24, generalized=True)
    s = make_solver(case, 24, precision="tf32", tol=1e-8, max_iter=200)
    X_ref, ev_ref, _, st_ref = s.solve(case["X"])
    Xw = np.ascontiguousarray(case["X"].copy())
    X, ev, _, st = s.solve(Xw, inplace=True)
    assert X is Xw
    assert st["iterations"] == st_ref["iterations"]
    np.testing.assert_allclose(ev, ev_ref, rtol=1e-12, atol=1e-12 * np.abs(ev_ref).max())
    assert relfro(Xw, X_ref) <= 1e-10
