"""Full-solve pins of the oracle (Algorithm 1 with Algorithms 2/3): prescribed spectra,
brute-force dense eigensolves and the behaviour the paper reports for its toy problems."""
import json
import os

import numpy as np
import scipy.linalg as sla
import pytest

import workloads as wl
from oracle import solver, lanczos, angles

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_toy.json")))


def test_toy_construction_matches_printed_values():
    t = wl.toy_standard(0.0)
    lam = t["lam"]
    assert abs(lam[-1] - GOLD["lambda_m_approx"]) < 0.05
    assert abs((lam[GOLD["n"]] - lam[GOLD["n"] - 1]) - GOLD["spectral_gap"]) < 1e-12
    assert abs(lam[-1] / lam[0] - GOLD["kappa_A_approx"]) < 0.5
    assert abs(t["lmin"] - GOLD["bounds"]["lmin"]) < 1e-12
    assert abs(t["lT"] - GOLD["bounds"]["lT"]) < 1e-12
    assert abs(t["lmax"] - lam[-1] - GOLD["bounds"]["lmax_minus_lambda_m"]) < 1e-12
    g = wl.toy_generalized(1e-3)
    eb = np.linalg.eigvalsh(g["B"])
    assert abs(eb[-1] / eb[0] - GOLD["kappa_B"]) < 1e-9
    # ||D^-1 - B^-1||_2 = zeta exactly by construction
    assert abs(np.abs(np.linalg.eigvalsh(g["Dinv_dense"] - g["Binv"])).max() - 1e-3) < 1e-12
    # shared eigenbasis: generalized eigenvalues are a_j / b_j
    np.testing.assert_allclose(sla.eigh(g["A"], g["B"], eigvals_only=True)[:10], g["lam"][:10],
                               atol=1e-11)


def _run_toy_gen(zeta, method, iters):
    t = wl.toy_generalized(zeta)
    X0 = wl.gaussian_block(1000, 10, seed=2)
    r = solver.solve(lambda v: t["A"] @ v, lambda v: t["B"] @ v, X0, 10, GOLD["p"], 0.0, iters,
                     None, 1.0, method=method, Dinv=lambda v: t["Dinv_dense"] @ v,
                     bounds=(t["lmin"], t["lT"], t["lmax"]))
    return t, r


def test_toy_generalized_exact_inverse_both_methods():
    """zeta = 0: both methods converge identically to ~1e-13 residual (Section 4.1.3)."""
    _, r2 = _run_toy_gen(0.0, "chfsi", 60)
    t, r3 = _run_toy_gen(0.0, "rchfsi", 60)
    tol = 10 * GOLD["exact_inverse_residual_order"]
    assert r2["history_abs"][-1] < tol and r3["history_abs"][-1] < tol
    np.testing.assert_allclose(r2["eps"], r3["eps"], atol=1e-12)
    np.testing.assert_allclose(r3["eps"], t["lam"][:10], atol=1e-12)


def test_toy_generalized_rchfsi_robust_chfsi_stagnates():
    """zeta = 1e-3: ChFSI stagnates at O(zeta), R-ChFSI reaches ~1e-14 (Section 4.1.3)."""
    _, r2 = _run_toy_gen(1e-3, "chfsi", 60)
    _, r3 = _run_toy_gen(1e-3, "rchfsi", 60)
    assert r2["history_abs"][-1] > 1e-1 * 1e-3
    assert r3["history_abs"][-1] < 100 * GOLD["rchfsi_residual_order_small_zeta"]


@pytest.mark.slow
def test_toy_generalized_large_zeta_angle():
    """zeta = 1e-2, 100 iterations: R-ChFSI reaches at least the printed subspace angle
    (~6e-8), ChFSI stays at an O(zeta) angle."""
    t, r3 = _run_toy_gen(1e-2, "rchfsi", GOLD["iterations"])
    _, r2 = _run_toy_gen(1e-2, "chfsi", GOLD["iterations"])
    bj = 1.0 + 4.0 * np.arange(1000) / 999
    bh = (t["Q"] * np.sqrt(bj)) @ t["Q"].T
    target = bh @ t["Q"][:, :10]
    a3 = angles.max_angle(target, bh @ r3["X"])
    a2 = angles.max_angle(target, bh @ r2["X"])
    assert a3 < 10 * GOLD["rchfsi_angle_zeta_1e-2_iter100"]
    assert a2 > 1e-2 * 1e-2


def test_toy_standard_perturbed_filter_matrix():
    """B = I, filter uses A + eps E, RR uses A: ChFSI stalls at O(eps), R-ChFSI keeps
    converging (Section 4.1.2)."""
    t = wl.toy_standard(1e-3)
    X0 = wl.gaussian_block(1000, 10, seed=2)
    kw = dict(A_filter=lambda v: t["A_filter"] @ v, bounds=(t["lmin"], t["lT"], t["lmax"]))
    r2 = solver.solve(lambda v: t["A"] @ v, lambda v: v, X0, 10, 8, 0.0, 90, None, 1.0,
                      method="chfsi", **kw)
    r3 = solver.solve(lambda v: t["A"] @ v, lambda v: v, X0, 10, 8, 0.0, 90, None, 1.0,
                      method="rchfsi", **kw)
    assert r2["history_abs"][-1] > 1e-1 * 1e-3
    assert r3["history_abs"][-1] < 1e-7 and r3["history_abs"][-1] < r3["history_abs"][-20] / 10


def test_dense_standard_config1_prescribed_spectrum():
    """Dense standard problem (m = 1000, nev = 50, block 60, degree 20, Lanczos bounds):
    converged eigenvalues equal the prescribed ones."""
    c = wl.dense_config1()
    A = lambda v: c["A"] @ v  # noqa: E731
    X0 = wl.gaussian_block(1000, 60, seed=2)
    lmax = lanczos.upper_bound(A, None, X0[:, 0], 10)
    nA = lanczos.norm_estimate(A, X0[:, 0], 10)
    r = solver.solve(A, lambda v: v, X0, 50, 20, 1e-8, 40, lmax, nA)
    assert r["history_rel"][-1] <= 1e-8
    err = np.abs(r["eps"][:50] - c["lam"][:50])
    assert np.all(err <= 1e-9 * np.maximum(np.abs(c["lam"][:50]), 1e-2 * 11.05))


def test_dense_generalized_small_bruteforce():
    """Generalized problem with dense SPD B and D^-1 = diag(B)^-1 (m = 200, nev = 12):
    R-ChFSI converges to the brute-force dense eigenvalues; ChFSI stalls."""
    c = wl.dense_config2(m=200)
    A = lambda v: c["A"] @ v  # noqa: E731
    B = lambda v: c["B"] @ v  # noqa: E731
    D = lambda v: c["Dinv"][:, None] * v  # noqa: E731
    ref = sla.eigh(c["A"], c["B"], eigvals_only=True)
    X0 = wl.gaussian_block(200, 16, seed=2)
    lmax = lanczos.upper_bound(A, c["Dinv"], X0[:, 0], 10)
    nA = lanczos.norm_estimate(A, X0[:, 0], 10)
    r3 = solver.solve(A, B, X0, 12, 12, 1e-10, 150, lmax, nA, Dinv=D)
    assert r3["history_rel"][-1] <= 1e-10
    np.testing.assert_allclose(r3["eps"][:12], ref[:12], atol=1e-9 * np.abs(ref).max())
    r2 = solver.solve(A, B, X0, 12, 12, 1e-10, 40, lmax, nA, Dinv=D, method="chfsi")
    assert r2["history_rel"][-1] > 1e-8


def test_convergence_condition_diagnostic_oracle():
    """Section 4.1.4 (Eq. 5) on the oracle, zeta = 1e-3: the filtering error of ChFSI saturates at
    O(zeta) and the condition |C_p(l_n)| - |C_p(l_n+1)| > ||Delta^_p|| (sec + csc) fails, while for
    R-ChFSI the filtering error decays to round-off and the condition holds."""
    import scipy.linalg as sla
    from oracle import chebyshev, filters, rr
    zeta, n, iters, p = 1e-3, 10, 30, 8
    t = wl.toy_generalized(zeta)
    ex = wl.toy_generalized(0.0)
    A, B = t["A"], t["B"]
    m = A.shape[0]
    bounds = (t["lmin"], t["lT"], t["lmax"])
    lam_all, V = sla.eigh(A, B)
    L = np.linalg.cholesky(B)
    Qq = np.linalg.qr(L.T @ V[:, :n])[0]
    Bh = sla.sqrtm(B).real
    cp = np.abs(chebyshev.scaled_cheb(p, np.array([lam_all[n - 1], lam_all[n]]), *bounds))
    lhs = cp[0] - cp[1]
    Da, De = t["Dinv_dense"], ex["Dinv_dense"]
    res = {}
    for method in ("rchfsi", "chfsi"):
        X, lam, AX, BX = rr.rayleigh_ritz(wl.gaussian_block(m, n, seed=2), lambda v: A @ v, lambda v: B @ v)
        errs, rhs = [], []
        for _ in range(iters):
            W = AX - BX * lam[None, :]
            if method == "rchfsi":
                Ya = filters.rchfsi_filter(lambda R: A @ (Da @ R), lambda R: Da @ R, X, lam, W, *bounds, p)
                Ye = filters.rchfsi_filter(lambda R: A @ (De @ R), lambda R: De @ R, X, lam, W, *bounds, p)
            else:
                Ya = filters.chfsi_filter(lambda Y: Da @ (A @ Y), X, *bounds, p)
                Ye = filters.chfsi_filter(lambda Y: De @ (A @ Y), X, *bounds, p)
            d = np.linalg.norm(Bh @ (Ya - Ye), 2) / np.linalg.norm(Bh @ Ye, 2)
            s = np.linalg.svd(Qq.T @ np.linalg.qr(L.T @ X)[0], compute_uv=False).min()
            th = float(np.arccos(np.clip(s, -1.0, 1.0)))
            errs.append(d)
            rhs.append(d * (1.0 / np.cos(th) + 1.0 / max(np.sin(th), 1e-300)))
            X, lam, AX, BX = rr.rayleigh_ritz(Ya, lambda v: A @ v, lambda v: B @ v)
        res[method] = (np.array(errs), np.array(rhs))
    e3, r3 = res["rchfsi"]
    e2, r2 = res["chfsi"]
    assert e3[-1] < 1e-12 and e2[-1] > 1e-6
    assert np.all(r3[5:] < lhs) and r2[-1] > lhs
