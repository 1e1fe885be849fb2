"""Parity of the finite-element (cell-matrix) operator path with the oracle, through the C ABI."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import fe as ofe, filters, rr
from gpu_helpers import ensure_built, relfro, round_mantissa

from paper_2503_22652_gb300 import Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    ensure_built()


@pytest.fixture(scope="module")
def fe3():
    p = wl.fe_problem(3)          # 27 cells, 1728 dofs
    A = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"])
    B = ofe.assemble(p["cell_dofs"], p["B_cell"], p["m"])
    return p, A, B


def _inputs(p, A, B, N, seed=4):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((p["m"], N))
    L = np.sort(rng.uniform(-20.0, 30.0, N))
    W = A @ X - (B @ X) * L[None, :]
    return X, L, W


def _solver(p, N, precision="fp64", **kw):
    s = Solver(p["m"], nev=max(1, N // 2), block=N, precision=precision, **kw)
    s.set_fe(p["cell_dofs"], p["A_cells"], p["B_cell"], p["Dinv"])
    return s


@pytest.mark.parametrize("N", [1, 40, 70])
def test_fe_residual_and_rr_parity(fe3, N):
    p, A, B = fe3
    X, L, W = _inputs(p, A, B, N)
    s = _solver(p, N)
    Wg, r = s.residual(X, L)
    assert relfro(Wg, W) <= 1e-13
    if N > 1:
        Xg, ev = s.rayleigh_ritz(X)
        _, evr, _, _ = rr.rayleigh_ritz(X, lambda v: A @ v, lambda v: B @ v)
        np.testing.assert_allclose(ev, evr, rtol=1e-10, atol=1e-10 * np.abs(evr).max())


@pytest.mark.parametrize("p_deg", [1, 2, 9])
@pytest.mark.parametrize("method", ["rchfsi", "chfsi"])
def test_fe_filter_fp64_parity(fe3, p_deg, method):
    p, A, B = fe3
    N = 40
    X, L, W = _inputs(p, A, B, N)
    d = p["Dinv"]
    lmin, lT, lmax = -25.0, 40.0, 2500.0
    s = _solver(p, N)
    if method == "rchfsi":
        ref = filters.rchfsi_filter(lambda R: A @ (d[:, None] * R), lambda R: d[:, None] * R, X, L, W,
                                    lmin, lT, lmax, p_deg)
        got = s.filter(X, L, W, lmin, lT, lmax, p_deg)
    else:
        ref = filters.chfsi_filter(lambda Y: d[:, None] * (A @ Y), X, lmin, lT, lmax, p_deg)
        got = s.chfsi_filter(X, lmin, lT, lmax, p_deg)
    assert relfro(got, ref) <= 1e-12


@pytest.mark.parametrize("prec,tol", [("fp32", 5e-5), ("tf32", 5e-3), ("bf16", 5e-2)])
def test_fe_filter_lowp(fe3, prec, tol):
    """Reduced-precision FE filter against the FP64 oracle filter, error measured relative to the
    part of Y_p produced by the low-precision recurrence, ||Y_p - X Lambda_p||."""
    p, A, B = fe3
    N = 48
    X, L, W = _inputs(p, A, B, N)
    d = p["Dinv"]
    lmin, lT, lmax, deg = -25.0, 40.0, 2500.0, 8
    ref = filters.rchfsi_filter(lambda R: A @ (d[:, None] * R), lambda R: d[:, None] * R, X, L, W,
                                lmin, lT, lmax, deg)
    base = X * filters.lambda_p(L, lmin, lT, lmax, deg)[None, :]
    got = _solver(p, N, precision=prec).filter(X, L, W, lmin, lT, lmax, deg)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref - base)
    assert err <= tol, err


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32", "bf16"])
def test_fe_solve_small_mesh(precision):
    """Periodic 2^3 mesh with wells (512 dofs): R-ChFSI with the lumped-mass D^-1 converges to the
    dense generalized eigenvalues in every precision."""
    p = wl.fe_problem(2)
    A = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"]).toarray()
    B = ofe.assemble(p["cell_dofs"], p["B_cell"], p["m"]).toarray()
    ref = sla.eigh(A, B, eigvals_only=True)[:7]
    s = _solver(p, 12, precision=precision, degree=10, max_iter=150)
    s.set_params(nev=7)
    X0 = wl.gaussian_block(p["m"], 12, seed=2)
    X, ev, res, st = s.solve(X0)
    assert st["max_rel_residual"] <= 1e-8
    np.testing.assert_allclose(ev[:7], ref, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("N", [1, 7, 64, 100, 131])
def test_fe_fp64_products_tensor_core_parity(fe3, N):
    """The FP64-accurate FE products from BF16 slices (rr_mode "emulated", several 64-wide column
    tiles, widths that are not a multiple of 8) equal the assembled-matrix products to FP64
    accuracy, like the DFMA path."""
    p, A, B = fe3
    X, L, W = _inputs(p, A, B, N, seed=N)
    for mode in ("emulated", "fp64"):
        s = _solver(p, N, rr_mode=mode)
        Wg, _ = s.residual(X, L)
        assert relfro(Wg, W) <= 1e-13, mode


def test_fe_fp64_products_tensor_core_complex():
    q = wl.fe_kpoint_problem(3, (0.3, -0.2, 0.1))
    A = ofe.assemble(q["cell_dofs"], q["A_cells"], q["m"])
    B = ofe.assemble(q["cell_dofs"], q["B_cell"], q["m"])
    rng = np.random.default_rng(8)
    N = 70
    X = rng.standard_normal((q["m"], N)) + 1j * rng.standard_normal((q["m"], N))
    L = np.sort(rng.uniform(-20.0, 30.0, N))
    W = A @ X - (B @ X) * L[None, :]
    s = Solver(q["m"], nev=10, block=N, field="complex", rr_mode="emulated")
    s.set_fe(q["cell_dofs"], q["A_cells"], q["B_cell"], q["Dinv"])
    Wg, _ = s.residual(X, L)
    assert relfro(Wg, W) <= 1e-13


def test_fe_fp64_products_mark_nonfinite_columns(fe3):
    """The FP64-accurate products sum in fixed point on per-column scales: a NaN in one column of X
    makes that column of the residual NaN and leaves the other columns exact."""
    p, A, B = fe3
    N = 70
    X, L, W = _inputs(p, A, B, N, seed=3)
    Xb = X.copy()
    Xb[17, 5] = np.nan
    s = _solver(p, N, rr_mode="emulated")
    Wg, _ = s.residual(Xb, L)
    assert np.all(np.isnan(Wg[:, 5]))
    keep = np.arange(N) != 5
    assert np.all(np.isfinite(Wg[:, keep]))
    assert relfro(Wg[:, keep], W[:, keep]) <= 1e-13


def test_fe_operator_replaced_on_the_same_handle(fe3):
    """rchfsi_set_operator on a handle that already holds an FE operator reuses its allocations but
    repacks every cell image: the products and the filter follow the new cell matrices."""
    p, A, B = fe3
    N = 40
    X, L, _ = _inputs(p, A, B, N, seed=6)
    s = Solver(p["m"], nev=N // 2, block=N, precision="tf32", rr_mode="emulated")
    s.set_fe(p["cell_dofs"], p["A_cells"], p["B_cell"], p["Dinv"])
    s.residual(X, L)
    d = p["Dinv"]
    s.filter(X, L, A @ X - (B @ X) * L[None, :], -25.0, 40.0, 2500.0, 6)
    # a second operator: the cell matrices scaled and shifted by the cell mass
    A2_cells = 1.7 * p["A_cells"] + 0.3 * p["B_cell"][None, :, :]
    A2 = ofe.assemble(p["cell_dofs"], A2_cells, p["m"])
    s.set_fe(p["cell_dofs"], A2_cells, p["B_cell"], p["Dinv"])
    W2 = A2 @ X - (B @ X) * L[None, :]
    Wg, _ = s.residual(X, L)
    assert relfro(Wg, W2) <= 1e-13
    ref = filters.rchfsi_filter(lambda R: A2 @ (d[:, None] * R), lambda R: d[:, None] * R, X, L, W2,
                                -25.0, 40.0, 2500.0, 6)
    base = X * filters.lambda_p(L, -25.0, 40.0, 2500.0, 6)[None, :]
    got = s.filter(X, L, W2, -25.0, 40.0, 2500.0, 6)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref - base) <= 5e-3
