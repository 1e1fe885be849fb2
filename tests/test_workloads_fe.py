"""Pins of the finite-element generator and of the oracle's cell assembly, and of the
dense generalized construction."""
import numpy as np
import scipy.linalg as sla

import workloads as wl
from oracle import fe as ofe, solver, lanczos


def _periodic_1d(n, mat):
    g = 4 * n
    out = np.zeros((g, g), dtype=mat.dtype)
    for c in range(n):
        idx = (4 * c + np.arange(5)) % g
        out[np.ix_(idx, idx)] += mat
    return out


def test_1d_element_matrices():
    m1, k1, g1 = wl.fe_1d_matrices(0.5)
    assert abs(m1.sum() - 0.5) < 1e-14                 # integral of 1 over the element
    np.testing.assert_allclose(k1 @ np.ones(5), 0, atol=1e-12)   # constants in the kernel
    np.testing.assert_allclose(g1 @ np.ones(5), 0, atol=1e-12)   # derivative of a constant
    x, _ = wl.gll_1d()
    xs = (x + 1) * 0.25                                 # node coordinates on [0, h]
    assert abs(xs @ g1 @ np.ones(5)) < 1e-13
    assert abs(np.ones(5) @ g1 @ xs - 0.5) < 1e-13      # int 1 * d/dx(x) = h
    assert abs(xs @ k1 @ xs - 0.5) < 1e-12              # int (x')^2 = h


def test_separable_spectrum_at_zero_potential():
    """V = 0: A = 0.5(K x M x M + M x K x M + M x M x K), B = M x M x M, so the pencil's
    eigenvalues are 0.5 (k_a + k_b + k_c) with k from the 1D periodic pencil."""
    n = 2
    p = wl.fe_problem(n, v_scale=0.0)
    A = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"]).toarray()
    B = ofe.assemble(p["cell_dofs"], p["B_cell"], p["m"]).toarray()
    m1, k1, _ = wl.fe_1d_matrices(0.5)
    kap = sla.eigh(_periodic_1d(n, k1), _periodic_1d(n, m1), eigvals_only=True)
    ref = np.sort((0.5 * (kap[:, None, None] + kap[None, :, None] + kap[None, None, :])).ravel())
    got = sla.eigh(A, B, eigvals_only=True)
    np.testing.assert_allclose(got, ref, atol=1e-9 * ref.max())
    # lumped mass sums to the box volume
    assert abs((1.0 / p["Dinv"]).sum() - p["box"] ** 3) < 1e-10


def test_1d_pencil_continuum_limit():
    n = 8
    m1, k1, _ = wl.fe_1d_matrices(0.5)
    kap = sla.eigh(_periodic_1d(n, k1), _periodic_1d(n, m1), eigvals_only=True)
    L = 0.5 * n
    cont = np.sort(np.array([(2 * np.pi * j / L) ** 2 for j in range(-3, 4)]))
    np.testing.assert_allclose(kap[:7], cont, rtol=1e-4, atol=1e-9)   # Q4 discretisation error


def test_kpoint_operator_hermitian_and_free_electron_limit():
    n = 2
    kappa = np.array([0.2, -0.3, 0.1])
    p = wl.fe_kpoint_problem(n, kappa, v_scale=0.0)
    A = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"]).toarray()
    B = ofe.assemble(p["cell_dofs"], p["B_cell"], p["m"]).toarray()
    np.testing.assert_allclose(A, A.conj().T, atol=1e-12)
    got = sla.eigh(A, B, eigvals_only=True)[:3]
    k = np.array(p["kpoint"])
    L = p["box"]
    G = [2 * np.pi / L * np.array(v) for v in np.ndindex(3, 3, 3)]
    G = [g - 2 * np.pi / L for g in G]
    free = np.sort([0.5 * np.sum((g + k) ** 2) for g in G])[:3]
    np.testing.assert_allclose(got, free, rtol=1e-3)


def test_oracle_solve_small_fe_matches_dense():
    """Periodic 2^3 mesh (512 dofs, 7 bound states below a gap) with the seeded wells: R-ChFSI with the
    lumped-mass approximate inverse converges to the dense eigenvalues."""
    p = wl.fe_problem(2)
    A = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"])
    B = ofe.assemble(p["cell_dofs"], p["B_cell"], p["m"])
    ref = sla.eigh(A.toarray(), B.toarray(), eigvals_only=True)
    Ap = lambda v: A @ v  # noqa: E731
    X0 = wl.gaussian_block(p["m"], 12, seed=2)
    lmax = lanczos.upper_bound(Ap, p["Dinv"], X0[:, 0], 10)
    nA = lanczos.norm_estimate(Ap, X0[:, 0], 10)
    r = solver.solve(Ap, lambda v: B @ v, X0, 7, 10, 1e-10, 100, lmax, nA,
                     Dinv=lambda v: p["Dinv"][:, None] * v)
    assert r["history_rel"][-1] <= 1e-10
    np.testing.assert_allclose(r["eps"][:7], ref[:7], atol=1e-12 * np.abs(ref).max())


def test_dense_generalized_construction():
    c = wl.dense_config2(m=300)
    s = np.exp(np.random.default_rng(4).uniform(np.log(0.5), np.log(50.0), 300))
    np.testing.assert_allclose(np.diag(c["B"]), s, rtol=1e-15)
    np.testing.assert_allclose(c["B"], c["B"].T, atol=0)
    assert np.linalg.eigvalsh(c["B"]).min() > 0
    np.testing.assert_allclose(c["Dinv"], 1 / s, rtol=1e-15)
