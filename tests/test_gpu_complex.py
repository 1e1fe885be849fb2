"""Complex Hermitian problems (Bloch k-point operators, Section 4.2 workloads) through the C ABI:
FP64 parity of the filters, residual, Rayleigh-Ritz and Lanczos with the oracle run in complex
arithmetic, and full solves against LAPACK's complex generalized eigensolver."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import fe as ofe, filters, lanczos, rr
from gpu_helpers import ensure_built, relfro

from paper_2503_22652_gb300 import Server, Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    ensure_built()


def herm_case(m, seed=11, degenerate=False):
    """Seeded Hermitian A with a spread spectrum and a real SPD B (diagonally dominant)."""
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    Q, _ = np.linalg.qr(Z)
    lam = np.sort(rng.uniform(-1.0, 9.0, m))
    if degenerate:
        lam[2:5] = lam[2]     # a triple complex eigenvalue
        lam[7:9] = lam[7]     # a double one
    A = (Q * lam[None, :]) @ Q.conj().T
    A = 0.5 * (A + A.conj().T)
    G = rng.standard_normal((m, m))
    B = np.eye(m) + 0.1 * (G @ G.T) / m
    return A, B, 1.0 / np.diag(B)


def cblock(m, N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, N)) + 1j * rng.standard_normal((m, N))


def filter_bounds(A, d):
    ev = np.sort(np.real(np.linalg.eigvals(d[:, None] * A)))
    span = ev[-1] - ev[0]
    return ev[0] - 0.05 * span, ev[0] + 0.3 * span, ev[-1] + 0.02 * span


def dense_solver(A, B, d, N, **kw):
    s = Solver(A.shape[0], field="complex", nev=kw.pop("nev", max(1, N // 2)), block=N, **kw)
    s.set_dense(A, B=B, Dinv=d)
    return s


def test_dense_residual_rr_lanczos_parity():
    m, N = 240, 24
    A, B, d = herm_case(m)
    X = cblock(m, N, 1)
    L = np.sort(np.random.default_rng(2).uniform(-1.0, 2.0, N))
    s = dense_solver(A, B, d, N)
    W, r = s.residual(X, L)
    Wref, rref = rr.residual(A @ X, B @ X, L)
    assert relfro(W, Wref) <= 1e-13
    np.testing.assert_allclose(r, rref, rtol=1e-12)
    Xg, ev = s.rayleigh_ritz(X)
    _, evr, _, _ = rr.rayleigh_ritz(X, lambda v: A @ v, lambda v: B @ v)
    np.testing.assert_allclose(ev, evr, rtol=1e-10, atol=1e-10 * np.abs(evr).max())
    # returned Ritz vectors: complex B-orthonormal and diagonalise the projected A
    np.testing.assert_allclose(Xg.conj().T @ B @ Xg, np.eye(N), atol=1e-10)
    np.testing.assert_allclose(Xg.conj().T @ A @ Xg, np.diag(ev), atol=1e-9 * np.abs(ev).max())
    v0 = cblock(m, 1, 3)[:, 0]
    lmax, nA = s.lanczos_bounds(v0, 10)
    Aop = lambda v: A @ v  # noqa: E731
    assert abs(lmax - lanczos.upper_bound(Aop, d, v0, 10)) <= 1e-10 * abs(lmax)
    assert abs(nA - lanczos.norm_estimate(Aop, v0, 10)) <= 1e-10 * abs(nA)


@pytest.mark.parametrize("method", ["rchfsi", "chfsi"])
@pytest.mark.parametrize("p_deg", [1, 2, 11])
def test_dense_filter_fp64_parity(method, p_deg):
    m, N = 200, 20
    A, B, d = herm_case(m, seed=5)
    X = cblock(m, N, 6)
    lmin, lT, lmax = filter_bounds(A, d)
    L = np.sort(np.random.default_rng(7).uniform(lmin, lT, N))
    W = A @ X - (B @ X) * L[None, :]
    s = dense_solver(A, B, d, N)
    if method == "rchfsi":
        ref = filters.rchfsi_filter(lambda R: A @ (d[:, None] * R), lambda R: d[:, None] * R, X, L, W,
                                    lmin, lT, lmax, p_deg)
        got = s.filter(X, L, W, lmin, lT, lmax, p_deg)
    else:
        ref = filters.chfsi_filter(lambda Y: d[:, None] * (A @ Y), X, lmin, lT, lmax, p_deg)
        got = s.chfsi_filter(X, lmin, lT, lmax, p_deg)
    assert got.dtype == np.complex128
    assert relfro(got, ref) <= 1e-12


def _check_solution(A, B, X, ev, nev, normA, scale_floor):
    lam = sla.eigh(A, B, eigvals_only=True)[:nev]
    scale = np.maximum(np.abs(lam), scale_floor)
    assert np.all(np.abs(ev[:nev] - lam) <= 1e-9 * scale)
    R = A @ X[:, :nev] - (B @ X[:, :nev]) * ev[:nev][None, :]
    rel = np.linalg.norm(R, axis=0) / (normA * np.linalg.norm(X[:, :nev], axis=0))
    assert rel.max() <= 1.5e-8


@pytest.mark.parametrize("precision", ["fp64", "tf32", "bf16"])
def test_dense_solve(precision):
    m, nev, N = 400, 20, 28
    A, B, d = herm_case(m, seed=8)
    s = dense_solver(A, B, d, N, nev=nev, degree=16, precision=precision, max_iter=80)
    X, ev, res, st = s.solve(cblock(m, N, 9))
    assert st["max_rel_residual"] <= 1e-8
    _check_solution(A, B, X, ev, nev, st["normA"], 0.1)


def test_dense_solve_degenerate():
    """Repeated complex eigenvalues: clusters of more than two equal embedded Ritz values are
    orthonormalised in the complex B inner product before one vector per complex pair is kept."""
    m, nev, N = 300, 12, 18
    A, B, d = herm_case(m, seed=12, degenerate=True)
    s = dense_solver(A, B, d, N, nev=nev, degree=16, precision="tf32", max_iter=80)
    X, ev, res, st = s.solve(cblock(m, N, 13))
    assert st["max_rel_residual"] <= 1e-8
    _check_solution(A, B, X, ev, nev, st["normA"], 0.1)
    G = X[:, :nev].conj().T @ B @ X[:, :nev]
    np.testing.assert_allclose(G, np.eye(nev), atol=1e-8)


@pytest.fixture(scope="module")
def kp3():
    p = wl.fe_kpoint_problem(3, (0.1, 0.2, -0.3))     # 27 cells, 1728 complex dofs
    A = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"])
    B = ofe.assemble(p["cell_dofs"], p["B_cell"], p["m"])
    return p, A, B


def _fe_solver(p, N, **kw):
    s = Solver(p["m"], field="complex", nev=kw.pop("nev", max(1, N // 2)), block=N, **kw)
    s.set_fe(p["cell_dofs"], p["A_cells"], p["B_cell"], p["Dinv"])
    return s


def test_fe_kpoint_residual_and_filter_parity(kp3):
    p, A, B = kp3
    N = 24
    X = cblock(p["m"], N, 21)
    L = np.sort(np.random.default_rng(22).uniform(-20.0, 30.0, N))
    W = A @ X - (B @ X) * L[None, :]
    s = _fe_solver(p, N)
    Wg, r = s.residual(X, L)
    assert relfro(Wg, W) <= 1e-13
    d = p["Dinv"]
    lmin, lT, lmax = -25.0, 40.0, 2500.0
    for deg in (1, 9):
        ref = filters.rchfsi_filter(lambda R: A @ (d[:, None] * R), lambda R: d[:, None] * R, X, L, W,
                                    lmin, lT, lmax, deg)
        assert relfro(s.filter(X, L, W, lmin, lT, lmax, deg), ref) <= 1e-12
        ref = filters.chfsi_filter(lambda Y: d[:, None] * (A @ Y), X, lmin, lT, lmax, deg)
        assert relfro(s.chfsi_filter(X, lmin, lT, lmax, deg), ref) <= 1e-12


@pytest.mark.parametrize("prec,tol", [("fp32", 5e-5), ("tf32", 5e-3), ("bf16", 5e-2)])
def test_fe_kpoint_filter_lowp(kp3, prec, tol):
    """Reduced-precision complex FE filter against the FP64 oracle filter, error measured relative
    to the part of Y_p produced by the low-precision recurrence, ||Y_p - X Lambda_p||."""
    p, A, B = kp3
    N = 32
    X = cblock(p["m"], N, 23)
    L = np.sort(np.random.default_rng(24).uniform(-20.0, 30.0, N))
    W = A @ X - (B @ X) * L[None, :]
    d = p["Dinv"]
    lmin, lT, lmax, deg = -25.0, 40.0, 2500.0, 8
    ref = filters.rchfsi_filter(lambda R: A @ (d[:, None] * R), lambda R: d[:, None] * R, X, L, W,
                                lmin, lT, lmax, deg)
    got = _fe_solver(p, N, precision=prec).filter(X, L, W, lmin, lT, lmax, deg)
    lp = filters.lambda_p(L, lmin, lT, lmax, deg)
    base = X * lp[None, :]
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref - base)


@pytest.mark.parametrize("precision", ["fp64", "tf32"])
def test_fe_kpoint_solve(kp3, precision):
    p, A, B = kp3
    nev, N = 7, 12
    s = _fe_solver(p, N, nev=nev, degree=20, precision=precision, max_iter=150)
    X, ev, res, st = s.solve(cblock(p["m"], N, 25))
    assert st["max_rel_residual"] <= 1e-8
    Ad, Bd = A.toarray(), B.toarray()
    _check_solution(Ad, Bd, X, ev, nev, st["normA"], 1.0)


def test_server_complex_requests():
    m, nev, N = 160, 8, 12
    A, B, d = herm_case(m, seed=31)
    srv = Server(slots=2)
    try:
        X0 = cblock(m, N, 32)
        t = srv.submit(m, nev, N, X0=X0, dense=dict(A=A, B=B, Dinv=d), field="complex", precision=2,
                       degree=16, max_iter=80)
        out = None
        import time
        t0 = time.time()
        while out is None and time.time() - t0 < 120:
            out = srv.poll(t, want_vectors=True)
            time.sleep(0.01)
        assert out is not None and out["status"] == 0
        lam = sla.eigh(A, B, eigvals_only=True)[:nev]
        np.testing.assert_allclose(out["evals"][:nev], lam, rtol=1e-9, atol=1e-9)
        assert out["X"].dtype == np.complex128
    finally:
        srv.close()
