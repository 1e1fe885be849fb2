"""The FP64-accurate products from BF16 tensor-core slices (rr_mode="emulated") in the residual /
Rayleigh-Ritz steps: parity with the oracle and with the FP64 (DFMA) mode, and full solves."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import rr, fe as ofe
from gpu_helpers import ensure_built, dense_case, make_solver, relfro

from paper_2503_22652_gb300 import Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    ensure_built()


@pytest.mark.parametrize("m,N,gen", [(280, 36, True), (333, 9, False), (1000, 120, True), (64, 17, False)])
def test_rayleigh_ritz_emulated_parity(m, N, gen):
    case = dense_case(m=m, N=N, generalized=gen)
    Bm = case["B"] if gen else np.eye(m)
    Y = case["X"]
    s = make_solver(case, N, rr_mode="emulated")
    X, ev = s.rayleigh_ritz(Y)
    Xr, evr, _, _ = rr.rayleigh_ritz(Y, lambda v: case["A"] @ v, lambda v: Bm @ v)
    np.testing.assert_allclose(ev, evr, rtol=1e-11, atol=1e-11 * np.abs(evr).max())
    np.testing.assert_allclose(X.T @ Bm @ X, np.eye(N), atol=1e-11)
    sg = np.sign(np.sum(X * (Bm @ Xr), axis=0))
    assert relfro(X * sg[None, :], Xr) <= 1e-9
    # same library, DFMA products
    s64 = make_solver(case, N, rr_mode="fp64")
    X64, ev64 = s64.rayleigh_ritz(Y)
    np.testing.assert_allclose(ev, ev64, rtol=1e-12, atol=1e-12 * np.abs(ev64).max())


def test_emulated_products_resolve_tiny_columns():
    """Columns of very different magnitudes (per-row / per-column exponent scaling)."""
    case = dense_case(m=256, N=24, generalized=True)
    Y = case["X"] * np.logspace(-12, 3, 24)[None, :]
    s = make_solver(case, 24, rr_mode="emulated")
    _, ev = s.rayleigh_ritz(Y)
    _, evr, _, _ = rr.rayleigh_ritz(Y, lambda v: case["A"] @ v, lambda v: case["B"] @ v)
    np.testing.assert_allclose(ev, evr, rtol=1e-10, atol=1e-10 * np.abs(evr).max())


@pytest.mark.parametrize("precision", ["fp64", "tf32", "bf16"])
def test_solve_emulated_rr_dense_generalized(precision):
    m = 600
    c = wl.dense_config2(m=m)
    ref = sla.eigh(c["A"], c["B"], eigvals_only=True)[:30]
    s = Solver(m, nev=30, block=40, degree=30, precision=precision, max_iter=200, rr_mode="emulated")
    s.set_dense(c["A"], B=c["B"], Dinv=c["Dinv"])
    X, ev, res, st = s.solve(wl.gaussian_block(m, 40, seed=2))
    assert st["max_rel_residual"] <= 1e-8
    np.testing.assert_allclose(ev[:30], ref, atol=1e-9 * np.abs(ref).max())
    R = c["A"] @ X[:, :30] - (c["B"] @ X[:, :30]) * ev[:30][None, :]
    rel = np.linalg.norm(R, axis=0) / (st["normA"] * np.linalg.norm(X[:, :30], axis=0))
    assert rel.max() <= 1.5e-8


def test_solve_emulated_rr_fe():
    p = wl.fe_problem(2)
    A = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"]).toarray()
    B = ofe.assemble(p["cell_dofs"], p["B_cell"], p["m"]).toarray()
    ref = sla.eigh(A, B, eigvals_only=True)[:7]
    s = Solver(p["m"], nev=7, block=12, degree=10, precision="tf32", max_iter=150, rr_mode="emulated")
    s.set_fe(p["cell_dofs"], p["A_cells"], p["B_cell"], p["Dinv"])
    X, ev, res, st = s.solve(wl.gaussian_block(p["m"], 12, seed=2))
    assert st["max_rel_residual"] <= 1e-8
    np.testing.assert_allclose(ev[:7], ref, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("m,N,gen", [(280, 36, True), (333, 9, False), (120, 1, False), (64, 17, False)])
def test_rayleigh_ritz_jacobi_eigensolver(m, N, gen):
    """This library's Jacobi eigensolver for the projected matrix gives the oracle's Ritz pairs."""
    case = dense_case(m=m, N=N, generalized=gen)
    Bm = case["B"] if gen else np.eye(m)
    s = make_solver(case, N, eig_mode="jacobi")
    X, ev = s.rayleigh_ritz(case["X"])
    Xr, evr, _, _ = rr.rayleigh_ritz(case["X"], lambda v: case["A"] @ v, lambda v: Bm @ v)
    np.testing.assert_allclose(ev, evr, rtol=1e-11, atol=1e-11 * np.abs(evr).max())
    assert np.all(np.diff(ev) >= 0)
    np.testing.assert_allclose(X.T @ Bm @ X, np.eye(N), atol=1e-11)
    sg = np.sign(np.sum(X * (Bm @ Xr), axis=0))
    assert relfro(X * sg[None, :], Xr) <= 1e-9


def test_solve_jacobi_eigensolver():
    m = 600
    c = wl.dense_config2(m=m)
    ref = sla.eigh(c["A"], c["B"], eigvals_only=True)[:30]
    s = Solver(m, nev=30, block=40, degree=30, precision="tf32", max_iter=200, eig_mode="jacobi")
    s.set_dense(c["A"], B=c["B"], Dinv=c["Dinv"])
    X, ev, res, st = s.solve(wl.gaussian_block(m, 40, seed=2))
    assert st["max_rel_residual"] <= 1e-8
    np.testing.assert_allclose(ev[:30], ref, atol=1e-9 * np.abs(ref).max())
