"""The method-level failure statuses of rchfsi_solve / rchfsi_rayleigh_ritz, provoked by inputs made
on the host (no device fault is involved):

* ILL_CONDITIONED: an indefinite B, so the Gram matrix Y^T B Y of the Rayleigh-Ritz step of
  Section 2.1 has no Cholesky factor;
* NUMERIC: a NaN in the initial block;
* STAGNATED: classical ChFSI (Algorithm 2) with an approximate inverse D^-1 = B^-1 + zeta E,
  zeta = 1e-2 (the generalized toy problem of Section 4.1), whose residual stops improving at
  O(zeta) -- the behaviour the residual-based filter is built to avoid.
"""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import ensure_built

from paper_2503_22652_gb300 import RChFSIError, Solver, _lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    ensure_built()


def _indefinite_pencil(m=200, seed=5):
    q = wl.orthogonal(m, seed)
    A = wl.dense_from_spectrum(q, np.linspace(-1.0, 10.0, m))
    mu = np.linspace(1.0, 3.0, m)
    mu[: m // 2] = -3.0                # half the spectrum of B negative: tr(B) < 0, so the Gram
                                       # matrix of any block is indefinite with high probability
    B = wl.dense_from_spectrum(wl.orthogonal(m, seed + 1), mu)
    return A, B


def test_indefinite_B_is_ill_conditioned():
    m, N = 200, 24
    A, B = _indefinite_pencil(m)
    s = Solver(m, nev=10, block=N, degree=8)
    s.set_dense(A, B=B, Dinv=1.0 / np.abs(np.diag(B)))
    Y = wl.gaussian_block(m, N, seed=9)
    with pytest.raises(RChFSIError) as e:
        s.rayleigh_ritz(Y)
    assert e.value.code == _lib.ERR_ILL_CONDITIONED
    with pytest.raises(RChFSIError) as e:
        s.solve(Y)
    assert e.value.code == _lib.ERR_ILL_CONDITIONED


@pytest.mark.parametrize("col", [0, 5])
def test_nan_in_initial_block_is_numeric(col):
    """A NaN in the first column reaches the Lanczos start vector, elsewhere the first
    Rayleigh-Ritz step; both end in NUMERIC before any filter runs."""
    m, N = 300, 20
    c = wl.dense_config1(m=m)
    s = Solver(m, nev=8, block=N, degree=10)
    s.set_dense(c["A"])
    X0 = wl.gaussian_block(m, N, seed=3)
    X0[17, col] = np.nan
    with pytest.raises(RChFSIError) as e:
        s.solve(X0)
    assert e.value.code == _lib.ERR_NUMERIC


def test_chfsi_with_inexact_inverse_stagnates():
    t = wl.toy_generalized(1e-2)
    m, N = t["A"].shape[0], 10
    s = Solver(m, nev=10, block=N, degree=8, method="chfsi", max_iter=100, stall_iters=5,
               bounds=(t["lmin"], t["lT"], t["lmax"]))
    s.set_dense(t["A"], B=t["B"], Dinv_dense=t["Dinv_dense"])
    X, ev, res, st = s.solve(wl.gaussian_block(m, N, seed=2), allow_not_converged=True)
    assert st["status"] == _lib.ERR_STAGNATED
    assert st["iterations"] < 100
    # it stopped at the O(zeta) floor, far above the tolerance
    assert st["max_rel_residual"] > 1e-6
    # the residual-based filter on the same problem and handle keeps converging well below it
    s.set_params(method="rchfsi", stall_iters=0)
    _, _, _, st3 = s.solve(wl.gaussian_block(m, N, seed=2), allow_not_converged=True)
    assert st3["status"] in (_lib.OK, _lib.ERR_NOT_CONVERGED)
    assert st3["max_rel_residual"] < 1e-2 * st["max_rel_residual"]


def test_nearly_dependent_block_goes_through_shifted_cholesky_qr():
    """A Gaussian initial block with eight pairs of columns that agree to 1e-10: the Gram matrix of
    the first Rayleigh-Ritz step has no Cholesky factor in FP64, so the basis is preconditioned by
    one shifted Cholesky QR step (B inner product) and the solve proceeds to the prescribed
    eigenvalues.  The rounding that decides whether a pivot of a near-singular Gram matrix comes out
    positive varies with the data, so several seeded blocks are tried and at least one must take
    the retry."""
    m, N, nev = 300, 24, 10
    c = wl.dense_config1(m=m)
    retried = 0
    for seed in (3, 4, 5):
        X0 = wl.gaussian_block(m, N, seed=seed)
        rng = np.random.default_rng(seed)
        for j in range(0, 16, 2):
            X0[:, j + 1] = X0[:, j] + 1e-10 * rng.standard_normal(m)
        s = Solver(m, nev=nev, block=N, degree=12, max_iter=100)
        s.set_dense(c["A"])
        X, ev, res, st = s.solve(X0)
        assert st["status"] == _lib.OK and st["max_rel_residual"] <= 1e-8
        np.testing.assert_allclose(ev[:nev], c["lam"][:nev], atol=1e-9 * 11.0)
        retried += st["cholqr_retries"] > 0
    assert retried >= 1
