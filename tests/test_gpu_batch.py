"""rchfsi_solve_batch: several problems (k-points of a Bloch problem, real FE problems, a dense one)
solved together, with the batched tensor-core filter.  Each result must equal the result of the
same problem solved alone (both to the 1e-8 relative residual; eigenvalues within 1e-9 of LAPACK)."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import fe as ofe
from gpu_helpers import ensure_built

from paper_2503_22652_gb300 import Solver, solve_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    ensure_built()


def _kp(n, kappa):
    p = wl.fe_kpoint_problem(n, kappa)
    A = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"]).toarray()
    B = ofe.assemble(p["cell_dofs"], p["B_cell"], p["m"]).toarray()
    return p, A, B


def _solver(p, nev, N, precision="tf32", field="complex", **kw):
    s = Solver(p["m"], nev=nev, block=N, degree=kw.pop("degree", 20), precision=precision, field=field,
               max_iter=kw.pop("max_iter", 150), **kw)
    s.set_fe(p["cell_dofs"], p["A_cells"], p["B_cell"], p["Dinv"])
    return s


def _x0(m, N, seed, cplx=True):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, N))
    return X + 1j * rng.standard_normal((m, N)) if cplx else X


def _check(A, B, X, ev, nev, normA):
    lam = sla.eigh(A, B, eigvals_only=True)[:nev]
    np.testing.assert_allclose(ev[:nev], lam, atol=1e-9 * np.abs(lam).max())
    R = A @ X[:, :nev] - (B @ X[:, :nev]) * ev[:nev][None, :]
    rel = np.linalg.norm(R, axis=0) / (normA * np.linalg.norm(X[:, :nev], axis=0))
    assert rel.max() <= 1.5e-8


@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_batch_kpoints_equals_alone(precision):
    specs = [(2, (0.1, 0.2, -0.3)), (3, (-0.4, 0.05, 0.25)), (2, (0.45, -0.45, 0.0)), (3, (0.0, 0.3, 0.1))]
    probs = [_kp(n, k) for n, k in specs]
    nev, N = 6, 10
    X0 = [_x0(p["m"], N, 50 + i) for i, (p, _, _) in enumerate(probs)]
    batch = solve_batch([_solver(p, nev, N, precision) for p, _, _ in probs], X0)
    for (p, A, B), x0, (X, ev, res, st) in zip(probs, X0, batch):
        assert st["status"] == 0 and st["max_rel_residual"] <= 1e-8
        _check(A, B, X, ev, nev, st["normA"])
        Xa, eva, resa, sta = _solver(p, nev, N, precision).solve(x0)
        np.testing.assert_allclose(ev[:nev], eva[:nev], atol=1e-9 * np.abs(eva[:nev]).max())


def test_batch_mixed_problems():
    """Real FE problems (batched filter), a complex k-point problem in another precision and a
    dense problem (filtered one by one) in the same call."""
    fe2 = wl.fe_problem(2)
    fe3 = wl.fe_problem(3)
    kp, Ak, Bk = _kp(2, (0.2, -0.1, 0.3))
    d = wl.dense_config2(m=300)
    sol = [_solver(fe2, 6, 10, field="real"), _solver(fe3, 6, 10, field="real"),
           _solver(kp, 5, 8, precision="bf16")]
    sd = Solver(300, nev=20, block=28, degree=20, precision="tf32", max_iter=150)
    sd.set_dense(d["A"], B=d["B"], Dinv=d["Dinv"])
    sol.append(sd)
    X0 = [_x0(fe2["m"], 10, 1, False), _x0(fe3["m"], 10, 2, False), _x0(kp["m"], 8, 3), _x0(300, 28, 4, False)]
    out = solve_batch(sol, X0)
    for p, (X, ev, res, st) in zip([fe2, fe3], out[:2]):
        A = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"]).toarray()
        B = ofe.assemble(p["cell_dofs"], p["B_cell"], p["m"]).toarray()
        _check(A, B, X, ev, 6, st["normA"])
    X, ev, res, st = out[2]
    _check(Ak, Bk, X, ev, 5, st["normA"])
    X, ev, res, st = out[3]
    _check(d["A"], d["B"], X, ev, 20, st["normA"])


def test_batch_one_problem_not_converged():
    """A problem that runs out of iterations leaves the batch with NOT_CONVERGED; the others finish."""
    probs = [_kp(2, (0.1, 0.2, 0.3)), _kp(2, (0.3, 0.1, -0.2))]
    sol = [_solver(probs[0][0], 6, 10), _solver(probs[1][0], 6, 10, max_iter=2)]
    X0 = [_x0(p["m"], 10, 7 + i) for i, (p, _, _) in enumerate(probs)]
    out = solve_batch(sol, X0, allow_not_converged=True)
    assert out[0][3]["status"] == 0
    assert out[1][3]["status"] != 0 and out[1][3]["iterations"] == 2
    p, A, B = probs[0]
    _check(A, B, out[0][0], out[0][1], 6, out[0][3]["normA"])
