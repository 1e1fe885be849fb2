"""The controlled-error studies of Section 4.1 run through the GPU path (C ABI):
  * standard toy problem, filter matrix A~ = A + eps E (Section 4.1.2): ChFSI stagnates at O(eps),
    R-ChFSI keeps converging at the unperturbed rate;
  * generalized toy problem, D^-1 = B^-1 + zeta E (Section 4.1.3): same contrast in zeta;
  * the convergence-condition diagnostic (Section 4.1.4, Eq. 5 of Section 3) at zeta = 1e-3: the
    filtering error saturates at O(zeta) for ChFSI and decays with the residual for R-ChFSI;
  * reduced-precision filters (FP32 / TF32 / BF16) on the unperturbed toys: R-ChFSI follows the
    FP64 convergence history, the inexact products being absorbed by the residual form."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import chebyshev
from gpu_helpers import ensure_built

from paper_2503_22652_gb300 import Solver

pytestmark = pytest.mark.gpu

ITERS = 100
P = 8


@pytest.fixture(scope="module", autouse=True)
def _build():
    ensure_built()


def _run(t, method, precision="fp64", iters=ITERS):
    m = t["A"].shape[0]
    s = Solver(m, nev=10, block=10, degree=P, precision=precision, method=method, max_iter=iters,
               min_iter=iters, tol=0.0, bounds=(t["lmin"], t["lT"], t["lmax"]))
    s.set_dense(t["A"], B=t["B"], A_filter=t.get("A_filter"), Dinv_dense=t.get("Dinv_dense"))
    X0 = wl.gaussian_block(m, 10, seed=2)
    X, ev, res, st = s.solve(X0, allow_not_converged=True)
    return X, ev, st


@pytest.mark.parametrize("eps", [0.0, 1e-4, 1e-3, 1e-2])
def test_standard_toy_perturbed_filter_matrix(eps):
    """This seeded realisation converges more slowly than the paper's (the oracle gives the same
    absolute residual, 3.7e-10, after 100 iterations), so R-ChFSI is required to keep converging
    (three more orders from iteration 40 to 100) rather than to reach round-off."""
    t = wl.toy_standard(eps)
    _, ev3, st3 = _run(t, "rchfsi")
    _, ev2, st2 = _run(t, "chfsi")
    h3, h2 = st3["history"], st2["history"]
    assert h3[-1] <= 1e-11 and h3[-1] < 1e-3 * h3[40]
    np.testing.assert_allclose(ev3[:10], t["lam"][:10], rtol=1e-11)
    if eps == 0.0:
        # algebraic equivalence of the two recurrences with the same operator (Section 3)
        assert abs(h2[-1] - h3[-1]) <= 0.1 * h3[-1]
    else:
        # ChFSI stagnates at a residual of the order of the perturbation
        assert h2[-1] >= 0.01 * eps / np.abs(t["lam"]).max()
        assert h2[-1] > 1e3 * h3[-1]


@pytest.mark.parametrize("zeta", [0.0, 1e-4, 1e-3, 1e-2])
def test_generalized_toy_approximate_inverse(zeta):
    t = wl.toy_generalized(zeta)
    X3, ev3, st3 = _run(t, "rchfsi")
    _, ev2, st2 = _run(t, "chfsi")
    h3, h2 = st3["history"], st2["history"]
    if zeta <= 1e-3:
        assert h3[-1] <= 1e-12
        np.testing.assert_allclose(ev3[:10], t["lam"][:10], rtol=1e-11)
    else:
        # zeta = 1e-2: R-ChFSI still converges monotonically (the paper reports a subspace angle
        # of ~6e-8 after 100 iterations); ChFSI does not
        assert h3[-1] <= 1e-7 and h3[-1] < h3[20]
    if zeta == 0.0:
        assert h2[-1] <= 1e-12
    else:
        assert h2[-1] > 1e2 * h3[-1]


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_toy_reduced_precision_filters(precision):
    """Unperturbed toy problems with the products of the filter in reduced precision: R-ChFSI
    follows the FP64 filter's convergence history (the inexact products are absorbed by the
    residual form) down to the round-off floor of the FP64 residual / Rayleigh-Ritz steps."""
    for t, floor in ((wl.toy_standard(0.0), 1e-11), (wl.toy_generalized(0.0), 1e-12)):
        _, ev, st = _run(t, "rchfsi", precision=precision)
        _, _, st64 = _run(t, "rchfsi")
        h, h64 = st["history"], st64["history"]
        assert h[-1] <= floor
        assert h[70] <= 10 * h64[70] + 1e-14
        np.testing.assert_allclose(ev[:10], t["lam"][:10], rtol=1e-11)


def _angle(X, Q, B):
    """Largest principal angle between span(X) and span(Q) (B inner product)."""
    L = np.linalg.cholesky(B)
    Qx = np.linalg.qr(L.T @ X)[0]
    Qq = np.linalg.qr(L.T @ Q)[0]
    s = np.linalg.svd(Qq.T @ Qx, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))


def test_convergence_condition_diagnostic():
    """Eq. 5 at zeta = 1e-3 (Section 4.1.4): the filtering error ||B^1/2 Delta_p|| of each filter
    (approximate-inverse filter minus the exact-inverse filter on the same block) saturates at
    O(zeta) for ChFSI and decays with the residual for R-ChFSI, and the condition
    |C_p(l_n)| - |C_p(l_n+1)| > ||Delta^_p|| (sec theta + csc theta) holds throughout for R-ChFSI
    but fails for ChFSI once its subspace stops improving."""
    zeta, n, iters = 1e-3, 10, 40
    t = wl.toy_generalized(zeta)
    ex = wl.toy_generalized(0.0)
    m = t["A"].shape[0]
    A, B = t["A"], t["B"]
    bounds = (t["lmin"], t["lT"], t["lmax"])
    lam_all = np.sort(sla.eigh(A, B, eigvals_only=True))
    Qn = sla.eigh(A, B)[1][:, :n]
    Bh = sla.sqrtm(B).real
    cp = np.abs(chebyshev.scaled_cheb(P, np.array([lam_all[n - 1], lam_all[n]]), *bounds))
    lhs = cp[0] - cp[1]

    def handle(dinv):
        s = Solver(m, nev=n, block=n, degree=P, bounds=bounds)
        s.set_dense(A, B=B, Dinv_dense=dinv)
        return s

    sa, se = handle(t["Dinv_dense"]), handle(ex["Dinv_dense"])
    out = {}
    for method in ("rchfsi", "chfsi"):
        X, lam = sa.rayleigh_ritz(wl.gaussian_block(m, n, seed=2))
        errs, rhs = [], []
        for it in range(iters):
            W, _ = sa.residual(X, lam)
            if method == "rchfsi":
                Ya = sa.filter(X, lam, W, *bounds, P)
                Ye = se.filter(X, lam, W, *bounds, P)
            else:
                Ya = sa.chfsi_filter(X, *bounds, P)
                Ye = se.chfsi_filter(X, *bounds, P)
            # filtering error relative to the filtered block's scale
            d = np.linalg.norm(Bh @ (Ya - Ye), 2) / np.linalg.norm(Bh @ Ye, 2)
            th = _angle(X, Qn, B)
            errs.append(d)
            rhs.append(d * (1.0 / np.cos(th) + 1.0 / max(np.sin(th), 1e-300)))
            X, lam = sa.rayleigh_ritz(Ya)
        out[method] = (np.array(errs), np.array(rhs))
    e3, r3 = out["rchfsi"]
    e2, r2 = out["chfsi"]
    assert e3[-1] < 1e-3 * e3[0] and e3[-1] < 1e-10   # decays with the residual
    assert e2[-1] > 0.1 * e2[0] or e2[-1] > 1e-6        # saturates
    assert e2[-5:].min() > 1e3 * e3[-5:].max()
    assert np.all(r3[5:] < lhs)                         # condition holds for R-ChFSI
    assert r2[-1] > lhs                                 # and is eventually violated for ChFSI
