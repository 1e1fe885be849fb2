"""Filter parity at the tile widths and launch shapes the kernels use on the benchmark problems.

The other parity tests run small problems, where every kernel takes its narrow-tile, single-wave
paths.  Here the same comparisons with the oracle run at the shapes of the benchmark workloads:

* dense generalized problem of order 4000 with a 240-column block (Algorithm 3 in TF32 and BF16):
  one 128 x 240 accumulator tile per CTA (256 TMEM columns) and the product split over K;
* finite-element operator on a periodic 6^3 mesh (216 cells, 13,824 dofs, more cells than SMs)
  with a 600-column block and a width that is not a multiple of the column tile;
* complex Hermitian (Bloch k-point) finite-element filter with 128 and more columns.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import fe as ofe, filters
from gpu_helpers import ensure_built, lowp_reference, relfro

from paper_2503_22652_gb300 import Solver

pytestmark = pytest.mark.gpu

# tolerances as in the smaller dense and FE tests (error relative to ||Y_p - X Lambda_p||)
DENSE_LOWP = {"tf32": (10, 10, "truncate", 2e-3), "bf16": (7, 7, "nearest", 2e-2)}
FE_LOWP = {"tf32": 5e-3, "bf16": 5e-2}


@pytest.fixture(scope="module", autouse=True)
def _build():
    ensure_built()


@pytest.fixture(scope="module")
def dense4000():
    m, N = 4000, 240
    c = wl.dense_config2(m=m)
    d = c["Dinv"]
    # the spectrum of the filter operator D^-1 A is that of the symmetric D^-1/2 A D^-1/2
    r = np.sqrt(d)
    ev = sla.eigvalsh(r[:, None] * c["A"] * r[None, :])
    span = ev[-1] - ev[0]
    bounds = (ev[0] - 0.05 * span, ev[0] + 0.3 * span, ev[-1] + 0.02 * span)
    rng = np.random.default_rng(41)
    X = rng.standard_normal((m, N))
    L = np.sort(rng.uniform(ev[0], ev[0] + 0.3 * span, N))
    W = c["A"] @ X - (c["B"] @ X) * L[None, :]
    return dict(A=c["A"], B=c["B"], Dinv=d, Dinv_dense=None, A_filter=None, X=X, L=L, W=W, bounds=bounds)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_dense_filter_m4000_block240(dense4000, prec):
    case = dense4000
    m, N = case["X"].shape
    bits_op, bits_r, mode, tol = DENSE_LOWP[prec]
    lmin, lT, lmax = case["bounds"]
    p = 4
    ref = lowp_reference(case, p, bits_op, bits_r, mode, lmin, lT, lmax)
    s = Solver(m, nev=200, block=N, precision=prec)
    s.set_dense(case["A"], B=case["B"], Dinv=case["Dinv"])
    got = s.filter(case["X"], case["L"], case["W"], lmin, lT, lmax, p)
    base = case["X"] * filters.lambda_p(case["L"], lmin, lT, lmax, p)[None, :]
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref - base)
    assert err <= tol, err
    # FP64 on the same handle: the full-width FP64 path against the exact oracle filter
    s.set_params(precision="fp64")
    d = case["Dinv"]
    ref64 = filters.rchfsi_filter(lambda R: case["A"] @ (d[:, None] * R), lambda R: d[:, None] * R, case["X"],
                                  case["L"], case["W"], lmin, lT, lmax, p)
    assert relfro(s.filter(case["X"], case["L"], case["W"], lmin, lT, lmax, p), ref64) <= 1e-12


@pytest.fixture(scope="module")
def fe6():
    p = wl.fe_problem(6)     # 216 cells, 13,824 dofs
    A = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"])
    B = ofe.assemble(p["cell_dofs"], p["B_cell"], p["m"])
    return p, A, B


@pytest.mark.parametrize("prec", ["tf32", "bf16", "fp64"])
@pytest.mark.parametrize("N", [600, 601])
def test_fe_filter_6cubed_block600(fe6, prec, N):
    p, A, B = fe6
    rng = np.random.default_rng(N)
    X = rng.standard_normal((p["m"], N))
    L = np.sort(rng.uniform(-20.0, 30.0, N))
    W = A @ X - (B @ X) * L[None, :]
    d = p["Dinv"]
    lmin, lT, lmax, deg = -25.0, 40.0, 2500.0, 8
    ref = filters.rchfsi_filter(lambda R: A @ (d[:, None] * R), lambda R: d[:, None] * R, X, L, W,
                                lmin, lT, lmax, deg)
    s = Solver(p["m"], nev=N // 2, block=N, precision=prec)
    s.set_fe(p["cell_dofs"], p["A_cells"], p["B_cell"], p["Dinv"])
    got = s.filter(X, L, W, lmin, lT, lmax, deg)
    if prec == "fp64":
        assert relfro(got, ref) <= 1e-12
    else:
        base = X * filters.lambda_p(L, lmin, lT, lmax, deg)[None, :]
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref - base)
        assert err <= FE_LOWP[prec], err


@pytest.mark.parametrize("N", [600, 130])
def test_fe_fp64_products_6cubed(fe6, N):
    """FP64-accurate FE products (rr_mode "emulated") with more cells than CTAs (several items per
    CTA, both barrier phases), every 64-column tile of a 600-wide block and a ragged last tile,
    against the assembled sparse products."""
    p, A, B = fe6
    rng = np.random.default_rng(N + 1)
    X = rng.standard_normal((p["m"], N))
    L = np.sort(rng.uniform(-20.0, 30.0, N))
    W = A @ X - (B @ X) * L[None, :]
    s = Solver(p["m"], nev=N // 2, block=N, rr_mode="emulated")
    s.set_fe(p["cell_dofs"], p["A_cells"], p["B_cell"], p["Dinv"])
    Wg, _ = s.residual(X, L)
    assert relfro(Wg, W) <= 1e-13
    # the cell contributions are summed in integers: a repeat is bitwise identical
    assert np.array_equal(s.residual(X, L)[0], Wg)


@pytest.fixture(scope="module")
def kp4():
    p = wl.fe_kpoint_problem(4, (0.15, -0.35, 0.25))     # 64 cells, 4,096 complex dofs
    A = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"])
    B = ofe.assemble(p["cell_dofs"], p["B_cell"], p["m"])
    return p, A, B


@pytest.mark.parametrize("prec", ["fp64", "tf32", "bf16"])
@pytest.mark.parametrize("N", [128, 200])
def test_fe_kpoint_filter_wide_block(kp4, prec, N):
    p, A, B = kp4
    rng = np.random.default_rng(7 * N)
    X = rng.standard_normal((p["m"], N)) + 1j * rng.standard_normal((p["m"], N))
    L = np.sort(rng.uniform(-20.0, 30.0, N))
    W = A @ X - (B @ X) * L[None, :]
    d = p["Dinv"]
    lmin, lT, lmax, deg = -25.0, 40.0, 2500.0, 8
    ref = filters.rchfsi_filter(lambda R: A @ (d[:, None] * R), lambda R: d[:, None] * R, X, L, W,
                                lmin, lT, lmax, deg)
    s = Solver(p["m"], field="complex", nev=N // 2, block=N, precision=prec)
    s.set_fe(p["cell_dofs"], p["A_cells"], p["B_cell"], p["Dinv"])
    got = s.filter(X, L, W, lmin, lT, lmax, deg)
    if prec == "fp64":
        assert relfro(got, ref) <= 1e-12
    else:
        base = X * filters.lambda_p(L, lmin, lT, lmax, deg)[None, :]
        assert np.linalg.norm(got - ref) <= FE_LOWP[prec] * np.linalg.norm(ref - base)
